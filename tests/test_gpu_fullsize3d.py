"""The 3D hot path and the moment recorder at the 3D workload's full size (256 x 256 x 512 cells,
8 particles per cell per species, 536,870,912 particles), benchmark launch configuration, ids on:

  * sampled parity: 2048 particles per species against the oracle's single-particle step in the
    same seeded fields (1e-5 relative in u, 1e-5 cell in position);
  * after 2 steps every id is present exactly once;
  * the recorder at load: every coarse cell (4 x 4 x 512 cells) holds exactly 8 particles per
    cell and species, so n_b and n_p equal the loaded densities (0.1, 0.9) to FP32 rounding, and
    the variances are non-negative.
"""
import os

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

NX, NY, NZ, PPC = 256, 256, 512, 8


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


@pytest.fixture(scope="module")
def load():
    L = pi.weibel_load_parallel(ndim=3, nx=NX, ny=NY, nz=NZ, ppc=PPC, T_perp_beam=0.2, seed=3,
                                workers=max(1, min(16, os.cpu_count() or 1)))
    wl = L.workload
    sp = [pi.SpeciesLoad(s.name, s.q, s.m, s.w, s.nu, s.cell.copy(), s.offset.copy(), s.u.copy())
          for s in wl.species]
    L.close()
    return pi.Workload("hot_beam_3d_256x256x512_ppc8", 3, NX, NY, NZ, wl.dx, wl.dy, wl.dz, wl.dt, 0, sp)


def test_fullsize3d(pic, load):
    import oracle
    wl = load
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=8, diag_interval=10, diag_capacity=64)
    # recorder at load
    rows = eng.record_moments(4, 4).cpu().numpy()
    assert np.allclose(rows[0], 0.1, rtol=1e-6) and np.allclose(rows[1], 0.9, rtol=1e-6)
    assert (rows[4:8] >= 0).all()
    rng = np.random.default_rng(5)
    E0 = (0.05 * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    B0 = (0.05 * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    eng.set_fields(E0, B0)
    eng.step(1)
    after = []
    for s in range(2):
        cell, off, u, ids = eng.particles(s)
        n = wl.species[s].n
        inv = np.full(n, -1, np.int64)
        inv[ids] = np.arange(ids.shape[0])
        assert (inv >= 0).all() and ids.shape[0] == n
        after.append((cell, off, u, inv))
    eng.step(1)
    for s in range(2):
        ids = eng.particles(s)[3]
        assert ids.shape[0] == wl.species[s].n and np.array_equal(np.bincount(ids, minlength=ids.shape[0]), np.ones(ids.shape[0], np.int64))
    assert eng.stats()["flags"] == 0
    eng.close()

    sim = oracle.Simulation(3, NX, NY, NZ, dx=wl.dx, dt=wl.dt)
    for a in range(3):
        sim.E[a][...] = E0[a].reshape(NZ, NY, NX)
        sim.B[a][...] = B0[a].reshape(NZ, NY, NX)
    for s, sp in enumerate(wl.species):
        cell1, off1, u1, inv = after[s]
        for p in rng.choice(sp.n, 2048, replace=False):
            c = int(sp.cell[p])
            X = c % NX + float(sp.offset[0, p])
            Y = (c // NX) % NY + float(sp.offset[1, p])
            Z = c // (NX * NY) + float(sp.offset[2, p])
            Xo, Yo, Zo, uo = sim.push_particle(sp.q / sp.m, sp.nu, X, Y, Z, sp.u[:, p].astype(np.float64))
            q = inv[p]
            ug = u1[:, q].astype(np.float64)
            assert np.linalg.norm(ug - uo) <= 1e-5 * max(np.linalg.norm(uo), 1e-12), (s, p)
            c1 = int(cell1[q])
            got = (c1 % NX + float(off1[0, q]), (c1 // NX) % NY + float(off1[1, q]), c1 // (NX * NY) + float(off1[2, q]))
            for g, o, L in zip(got, (Xo, Yo, Zo), (NX, NY, NZ)):
                assert abs((g - o + L / 2) % L - L / 2) < 1e-5, (s, p)
