"""3D3V CUDA path (through the C ABI) against the FP64 oracle on identical seeded inputs.

The workloads are small boxes of the hot-beam 3D configuration (beam along z, gamma = 3,
T_perp = 0.2, 8 particles per cell per species, dx = dy = dz = 0.1, dt = 0.05) that span several
8 x 8 x 4 tiles.  Tolerances follow the 2D tests:
  * current after one step: |J_gpu - J_oracle| <= 1e-5 max|J| + 60 * 2^-S (at most ~60 terms per
    node per component rounded to 2^-S, FP32 shape factors);
  * per-particle momentum: relative error <= 1e-5 over the first 20 steps;
  * field-energy history within 1% of the oracle's once it is above the start-up noise.
"""
import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _box(nx=16, ny=16, nz=24, ppc=8, T=0.2, nu=0.0, T_bg=0.0, seed=31):
    return pi.weibel_load(ndim=3, nx=nx, ny=ny, nz=nz, ppc=ppc, T_perp_beam=T, T_bg=T_bg, nu=nu,
                          seed=seed, name=f"hot_beam_3d_box_{nx}x{ny}x{nz}")


def _periodic_diff(a, b, n):
    d = a - b
    return (d + n / 2) % n - n / 2


def _check_particles(eng, sim, wl, tol=1e-5):
    for s in range(len(wl.species)):
        cell, off, u, ids = eng.particles(s)
        order = np.argsort(ids)
        assert np.array_equal(ids[order], np.arange(len(ids)))
        ug = u[:, order].astype(np.float64)
        so = sim.species[s]
        uo = so.u
        err = np.linalg.norm(ug - uo, axis=0) / np.maximum(np.linalg.norm(uo, axis=0), 1e-12)
        assert err.max() < tol, (s, err.max())
        c = cell[order]
        X = (c % wl.nx) + off[0, order].astype(np.float64)
        Y = (c // wl.nx) % wl.ny + off[1, order].astype(np.float64)
        Z = c // (wl.nx * wl.ny) + off[2, order].astype(np.float64)
        assert np.abs(_periodic_diff(X, so.X, wl.nx)).max() < 1e-4
        assert np.abs(_periodic_diff(Y, so.Y, wl.ny)).max() < 1e-4
        assert np.abs(_periodic_diff(Z, so.Z, wl.nz)).max() < 1e-4


def _seed_fields(eng, sim, wl, amp=0.05, seed=3):
    rng = np.random.default_rng(seed)
    E0 = (amp * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    B0 = (amp * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    eng.set_fields(E0, B0)
    for a in range(3):
        sim.E[a][...] = E0[a].reshape(wl.nz, wl.ny, wl.nx)
        sim.B[a][...] = B0[a].reshape(wl.nz, wl.ny, wl.nx)


@pytest.mark.parametrize("nu", [0.0, 0.1])
def test_one_step_current_and_fields_3d(pic, nu):
    import oracle
    wl = _box(nu=nu, T_bg=0.001 if nu else 0.0, seed=41)
    eng = pic.Engine.from_workload(wl, track_ids=True, flags=pic.PIC_FLAG_KEEP_J)
    sim = oracle.Simulation.from_workload(wl)
    _seed_fields(eng, sim, wl)
    eng.step(1)
    sim.step(1)
    E, B, J = eng.fields(with_J=True)
    S = eng.fixed_point_shift()
    for a in range(3):
        jo = sim.J[a].reshape(-1)
        jg = J[a].astype(np.float64) * 2.0 ** -S
        scale = np.abs(jo).max()
        assert np.abs(jg - jo).max() <= 1e-5 * scale + 60 * 2.0 ** -S, a
        eo = sim.E[a].reshape(-1)
        bo = sim.B[a].reshape(-1)
        assert np.abs(E[a] - eo).max() <= 1e-5 * (np.abs(eo).max() + 1e-3), a
        assert np.abs(B[a] - bo).max() <= 1e-5 * (np.abs(bo).max() + 1e-3), a
    _check_particles(eng, sim, wl)
    eng.close()


@pytest.mark.parametrize("nu", [0.0, 0.1])
def test_particles_first_20_steps_3d(pic, nu):
    import oracle
    wl = _box(nx=16, ny=16, nz=32, nu=nu, T_bg=0.001 if nu else 0.0, seed=43)
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=8)
    sim = oracle.Simulation.from_workload(wl)
    for chunk in (1, 4, 15):
        eng.step(chunk)
        sim.step(chunk, record=False)
        _check_particles(eng, sim, wl)
    eng.close()


def test_energy_history_3d(pic):
    import oracle
    wl = _box(nx=16, ny=16, nz=16, seed=45)
    n = 120
    eng = pic.Engine.from_workload(wl, sort_interval=8, diag_interval=1, diag_capacity=n)
    eng.step(n)
    recs = eng.diag()
    eng.close()
    sim = oracle.Simulation.from_workload(wl)
    sim.step(n)
    assert len(recs) == n
    for key in ("WE", "WB"):
        g = np.array([r[key] for r in recs]).sum(1)
        o = sim.history_array(key).sum(1)
        assert np.all(np.abs(g[1:] - o[1:]) <= 0.01 * o[1:]), key
    ekg = np.array([r["Ekin"] for r in recs])
    eko = sim.history_array("Ekin")
    assert np.abs(ekg - eko).max() <= 1e-5 * np.abs(eko).max()


def test_sort_interval_invariance_3d(pic):
    """Deposits are integers and every code path evaluates the same formulas, so the particle
    order (sort every step, every 7 steps, never) cannot change any bit of the fields."""
    wl = _box(nx=16, ny=16, nz=16, seed=47)
    out = []
    for k in (1, 7, 0):
        eng = pic.Engine.from_workload(wl, sort_interval=k, flags=pic.PIC_FLAG_KEEP_J)
        eng.step(15)
        out.append(eng.fields(with_J=True))
        eng.close()
    for E, B, J in out[1:]:
        assert np.array_equal(E, out[0][0]) and np.array_equal(B, out[0][1])
        assert np.array_equal(J, out[0][2])


def _lower_half(wl):
    """Keep the particles of the lower half of the box (z < nz/2): 2x the mean density there."""
    import dataclasses
    half = wl.nx * wl.ny * (wl.nz // 2)
    sp = []
    for s in wl.species:
        k = s.cell < half
        sp.append(dataclasses.replace(s, cell=s.cell[k], offset=s.offset[:, k], u=s.u[:, k]))
    return dataclasses.replace(wl, species=sp)


def test_tight_capacity_spills_3d(pic):
    """16 particles per cell per species in the lower half of the box and 16 slots per cell:
    every step cells overflow their stay and immigrant areas, the spill list and its kernel carry
    the excess, and fields and particles still match a roomy run bit for bit."""
    wl = _lower_half(_box(nx=16, ny=16, nz=16, ppc=16, seed=49))
    res = []
    for cc in ((16, 16), (0, 0)):
        eng = pic.Engine.from_workload(wl, track_ids=True, cell_capacity=cc, sort_interval=4)
        spilled = 0
        for _ in range(3):
            eng.step(3)
            spilled = max(spilled, max(eng.stats()["spilled"]))
        eng.step(3)
        E, B, _ = eng.fields()
        parts = []
        for s in range(2):
            cell, off, u, ids = eng.particles(s)
            o = np.argsort(ids)
            parts.append((cell[o], off[:, o], u[:, o]))
        res.append((E, B, parts, spilled))
        eng.close()
    (E0, B0, P0, sp0), (E1, B1, P1, _) = res
    assert sp0 > 0                      # the tight run did spill
    assert np.array_equal(E0, E1) and np.array_equal(B0, B1)
    for (c0, o0, u0), (c1, o1, u1) in zip(P0, P1):
        assert np.array_equal(c0, c1) and np.array_equal(o0, o1) and np.array_equal(u0, u1)
