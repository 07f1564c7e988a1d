"""The 2D hot path at the benchmark's full size (1024 x 1024 cells, 64 particles per cell per
species, 134,217,728 particles) in the benchmark's launch configuration (CUDA graph of 8 steps,
re-sort check every 8 steps, diagnostics every 10), with particle ids on:

  * sampled parity: 4096 particles, chosen by id, against the oracle's single-particle step
    (gather, Boris, Krook drag, move) in the same seeded fields -- the whole oracle cannot run
    at this size, one particle at a time can;
  * charge continuity over the whole grid for the first step: (rho^1 - rho^0)/dt + div J = 0,
    rho from the oracle's CIC charge deposit of the particles before and after the step, J the
    step's current read back from the device;
  * after 8 steps every particle id is present exactly once.

Tolerances: per-particle momentum 1e-5 relative and position 1e-5 cell (as the small-size
tests).  Continuity: every current term is rounded to the fixed-point grid 2^-S (error uniform
in +-2^-S/2, standard deviation 2^-S/sqrt(12)); div J at a node combines the four currents
around it, each fed by the particles of about two cells (2 x 128 terms), so the rounding residual
has a standard deviation of sqrt(8 x 128 / 12) 2^-S / dx ~ 9.2 x 2^-S / dx, and its maximum
over the 2^20 nodes stays below 6 of those; plus 1e-6 of the largest |div J| for the FP32 shape
factors.
"""
import os

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

N, PPC = 1024, 64


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


@pytest.fixture(scope="module")
def load():
    L = pi.weibel_load_parallel(ndim=2, nx=N, ny=N, ppc=PPC, T_perp_beam=0.1, T_bg=0.001, nu=0.1,
                                seed=2, workers=max(1, min(16, os.cpu_count() or 1)))
    wl = L.workload
    # private copies: the shared-memory segments are released at once
    sp = [pi.SpeciesLoad(s.name, s.q, s.m, s.w, s.nu, s.cell.copy(), s.offset.copy(), s.u.copy())
          for s in wl.species]
    L.close()
    return pi.Workload("warm_beam_krook_2d_1024x1024_ppc64", 2, N, N, 1, wl.dx, wl.dy, wl.dz, wl.dt, 0, sp)


def _fields(wl, seed=3, amp=0.05):
    rng = np.random.default_rng(seed)
    E = (amp * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    B = (amp * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    return E, B


def _rho(wl, parts):
    """CIC charge density of both species (oracle), parts = [(cell, offset)] per species."""
    import oracle
    sim = oracle.Simulation(2, wl.nx, wl.ny, dx=wl.dx, dt=wl.dt)
    for s, (cell, off) in zip(wl.species, parts):
        X = (cell % wl.nx) + off[0].astype(np.float64)
        Y = (cell // wl.nx) + off[1].astype(np.float64)
        z = np.zeros(1)
        sim.add_species(s.q, s.m, s.w, 0.0, X, Y, None, z, z, z)
    return sim.rho()


def test_fullsize_one_step(pic, load):
    import oracle
    wl = load
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=8, diag_interval=10,
                                   diag_capacity=64, flags=pic.PIC_FLAG_KEEP_J)
    E0, B0 = _fields(wl)
    eng.set_fields(E0, B0)
    eng.step(1)
    _, _, J = eng.fields(with_J=True)
    S = eng.fixed_point_shift()
    after = []
    for s in range(2):
        cell, off, u, ids = eng.particles(s)
        o = np.argsort(ids)
        assert np.array_equal(ids[o], np.arange(wl.species[s].n))
        after.append((cell[o], off[:, o], u[:, o]))
    eng.close()

    # -- sampled parity against the oracle's single-particle step
    sim = oracle.Simulation(2, wl.nx, wl.ny, dx=wl.dx, dt=wl.dt)
    for a in range(3):
        sim.E[a][...] = E0[a].reshape(wl.ny, wl.nx)
        sim.B[a][...] = B0[a].reshape(wl.ny, wl.nx)
    rng = np.random.default_rng(11)
    for s, sp in enumerate(wl.species):
        ubar = None
        if sp.nu > 0:
            cnt = np.bincount(sp.cell, minlength=wl.ncell)
            ubar = np.stack([np.bincount(sp.cell, sp.u[a].astype(np.float64), minlength=wl.ncell)
                             for a in range(3)]) / np.maximum(cnt, 1)
        cell1, off1, u1 = after[s]
        for p in rng.choice(sp.n, 2048, replace=False):
            c = int(sp.cell[p])
            X = c % wl.nx + float(sp.offset[0, p])
            Y = c // wl.nx + float(sp.offset[1, p])
            ub = None if ubar is None else ubar[:, c]
            Xo, Yo, _, uo = sim.push_particle(sp.q / sp.m, sp.nu, X, Y, 0.0,
                                              sp.u[:, p].astype(np.float64), ub)
            ug = u1[:, p].astype(np.float64)
            assert np.linalg.norm(ug - uo) <= 1e-5 * max(np.linalg.norm(uo), 1e-12), (s, p)
            Xg = cell1[p] % wl.nx + float(off1[0, p])
            Yg = cell1[p] // wl.nx + float(off1[1, p])
            dX = (Xg - Xo + wl.nx / 2) % wl.nx - wl.nx / 2
            dY = (Yg - Yo + wl.ny / 2) % wl.ny - wl.ny / 2
            assert abs(dX) < 1e-5 and abs(dY) < 1e-5, (s, p, dX, dY)

    # -- charge continuity over the whole grid
    rho0 = _rho(wl, [(sp.cell, sp.offset) for sp in wl.species])
    rho1 = _rho(wl, [(c, o) for c, o, _ in after])
    jx = J[0].astype(np.float64).reshape(wl.ny, wl.nx) * 2.0 ** -S
    jy = J[1].astype(np.float64).reshape(wl.ny, wl.nx) * 2.0 ** -S
    div = (jx - np.roll(jx, 1, axis=1)) / wl.dx + (jy - np.roll(jy, 1, axis=0)) / wl.dy
    res = (rho1 - rho0) / wl.dt + div
    sigma = np.sqrt(8 * 2 * PPC / 12.0) * 2.0 ** -S / wl.dx
    tol = 1e-6 * np.abs(div).max() + 6 * sigma
    assert np.abs(res).max() <= tol, (np.abs(res).max(), tol)


def test_fullsize_ids_conserved_over_steps(pic, load):
    wl = load
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=8, diag_interval=10,
                                   diag_capacity=64)
    eng.step(8)
    for s in range(2):
        _, off, u, ids = eng.particles(s)
        assert ids.shape[0] == wl.species[s].n
        assert np.array_equal(np.sort(ids), np.arange(wl.species[s].n))
        assert np.isfinite(u).all() and (off >= 0).all() and (off < 1).all()
    assert eng.stats()["flags"] == 0
    eng.close()
