"""The batched scan at full size in the benchmark's launch configuration: 256 independent 2D
runs (grids from {128, 192, 256, 384, 512}^2, 32 particles per cell per species,
1,470,103,552 particles), beam T_perp ~ U[0, 1], background Krook nu from {0, 0.01, 0.1, 1}, two
slots per mean particle, one launch set for all runs; particle ids on.

  * sampled parity of step 2: 512 particles per species of each of four runs (the largest, the
    smallest, one with nu = 1 and the hottest) against the oracle's single-particle step in the
    run's own fields after step 1 (1e-5 relative momentum, 1e-5 cell);
  * per-run equivalence: one run stepped alone, with the same settings, is bitwise equal to the
    same run inside the batch after 3 steps (the per-run plain launch the scan is compared with);
  * every id of every run is present exactly once after 3 steps.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

PPC = 32


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _engine_kw(pic):
    cc = 2 * PPC
    return dict(dx=0.1, dt=0.05, sort_interval=8, diag_interval=10, diag_capacity=64,
                cell_capacity=(cc, cc), track_ids=True)


def test_fullsize_scan(pic):
    import oracle
    table = pi.scan_table(256)
    runs = [(nx, ny, 1, (nx * ny * PPC,) * 2) for nx, ny, _, _ in table]
    eng = pic.Engine(2, nspecies=2, runs=runs, **_engine_kw(pic))
    picks = sorted({int(np.argmax([nx * ny for nx, ny, _, _ in table])),
                    int(np.argmin([nx * ny for nx, ny, _, _ in table])),
                    next(r for r, t in enumerate(table) if t[3] == 1.0),
                    int(np.argmax([t[2] for t in table]))})
    kept = {}
    workers = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        for r, wl in pool.imap_unordered(pi.scan_run, [(r, table[r], PPC) for r in range(len(table))]):
            for i, s in enumerate(wl.species):
                eng.load_species(i, s.q, s.m, s.w, s.nu, s.cell, s.offset, s.u, run=r)
            if r in picks:
                kept[r] = wl
    rng = np.random.default_rng(21)
    eng.step(1)

    def state(r):
        out = []
        for s in range(2):
            cell, off, u, ids = eng.particles(s, run=r)
            inv = np.full(ids.shape[0], -1, np.int64)
            inv[ids] = np.arange(ids.shape[0])
            out.append((cell, off, u, inv))
        return out

    before = {r: state(r) for r in picks}
    fields = {r: eng.fields(run=r)[:2] for r in picks}
    eng.step(1)
    after = {r: state(r) for r in picks}

    # step 2 of each picked run against the oracle's single-particle step in the GPU's fields
    # after step 1, with the drag means of the background's momenta after step 1
    for r in picks:
        wl = kept[r]
        sim = oracle.Simulation(2, wl.nx, wl.ny, dx=wl.dx, dt=wl.dt)
        E1, B1 = fields[r]
        for a_ in range(3):
            sim.E[a_][...] = E1[a_].reshape(wl.ny, wl.nx)
            sim.B[a_][...] = B1[a_].reshape(wl.ny, wl.nx)
        for s, sp in enumerate(wl.species):
            cell0, off0, u0, inv0 = before[r][s]
            cell1, off1, u1, inv1 = after[r][s]
            ubar = None
            if sp.nu > 0:
                cnt = np.bincount(cell0, minlength=wl.ncell)
                ubar = np.stack([np.bincount(cell0, u0[a_].astype(np.float64), minlength=wl.ncell)
                                 for a_ in range(3)]) / np.maximum(cnt, 1)
            for p in rng.choice(sp.n, 512, replace=False):
                q0, q1 = inv0[p], inv1[p]
                c = int(cell0[q0])
                X = c % wl.nx + float(off0[0, q0])
                Y = c // wl.nx + float(off0[1, q0])
                ub = None if ubar is None else ubar[:, c]
                Xo, Yo, _, uo = sim.push_particle(sp.q / sp.m, sp.nu, X, Y, 0.0,
                                                  u0[:, q0].astype(np.float64), ub)
                ug = u1[:, q1].astype(np.float64)
                assert np.linalg.norm(ug - uo) <= 1e-5 * max(np.linalg.norm(uo), 1e-12), (r, s, p)
                Xg = cell1[q1] % wl.nx + float(off1[0, q1])
                Yg = cell1[q1] // wl.nx + float(off1[1, q1])
                assert abs((Xg - Xo + wl.nx / 2) % wl.nx - wl.nx / 2) < 1e-5
                assert abs((Yg - Yo + wl.ny / 2) % wl.ny - wl.ny / 2) < 1e-5

    # per-run equivalence and id permutation after 3 steps
    eng.step(1)
    ref = picks[-1]
    batch_state = [eng.particles(s, run=ref) for s in range(2)]
    for r in range(len(table)):
        for s in range(2):
            ids = eng.particles(s, run=r)[3]
            n = table[r][0] * table[r][1] * PPC
            assert ids.shape[0] == n and (np.bincount(ids, minlength=n) == 1).all(), (r, s)
    assert eng.stats()["flags"] == 0
    eng.close()
    one = pic.Engine.from_workload(kept[ref], **{k: v for k, v in _engine_kw(pic).items() if k not in ("dx", "dt")})
    one.step(3)
    for s in range(2):
        cb, ob, ub, ib = batch_state[s]
        co, oo, uo, io = one.particles(s)
        a, b = np.argsort(ib), np.argsort(io)
        assert np.array_equal(ib[a], io[b])
        assert np.array_equal(cb[a], co[b]) and np.array_equal(ob[:, a], oo[:, b])
        assert np.array_equal(ub[:, a], uo[:, b])
    one.close()
