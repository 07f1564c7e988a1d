"""Batched scan: independent 2D runs of different sizes, beam temperatures and collision rates
stepped together (one set of launches / one CUDA graph) give bitwise the same histories,
fields, particles and growth rates as the same runs stepped one at a time; the same for a batch
of 3D runs."""
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


def _scan_runs():
    # grids, beam temperature and Krook rate vary per run, as in the parameter scan
    spec = [((32, 48), 0.3, 0.0), ((64, 32), 0.0, 0.1), ((16, 16), 1.0, 1.0), ((48, 48), 0.05, 0.01),
            ((32, 32), 0.5, 0.1)]
    return [pi.weibel_load(ndim=2, nx=n[0], ny=n[1], ppc=8, T_perp_beam=T, T_bg=0.001, nu=nu,
                           seed=1000 + r)
            for r, (n, T, nu) in enumerate(spec)]


def _state(eng, run, nsp=2):
    E, B, _ = eng.fields(run=run)
    parts = []
    for s in range(nsp):
        cell, off, u, ids = eng.particles(s, run=run)
        o = np.argsort(ids)
        parts.append((cell[o], off[:, o], u[:, o]))
    return E, B, parts


def test_batch_equals_single_runs(pic):
    wls = _scan_runs()
    nsteps = 48
    batch = pic.Engine.from_workloads(wls, track_ids=True, diag_interval=1, diag_capacity=64,
                                      sort_interval=8)
    batch.step(nsteps)
    for r, wl in enumerate(wls):
        single = pic.Engine.from_workload(wl, track_ids=True, diag_interval=1, diag_capacity=64,
                                          sort_interval=8)
        single.step(nsteps)
        assert batch.diag(run=r) == single.diag(), r
        Eb, Bb, Pb = _state(batch, r)
        Es, Bs, Ps = _state(single, 0)
        assert np.array_equal(Eb, Es) and np.array_equal(Bb, Bs), r
        for (c, o, u), (c0, o0, u0) in zip(Pb, Ps):
            assert np.array_equal(c, c0) and np.array_equal(o, o0) and np.array_equal(u, u0), r
        gb = batch.fit_growth(width=8, t_noise=0.5, start_factor=1.5, end_factor=None, run=r)
        gs = single.fit_growth(width=8, t_noise=0.5, start_factor=1.5, end_factor=None)
        assert (np.isnan(gb[0]) and np.isnan(gs[0])) or gb == gs, (r, gb, gs)
        single.close()
    batch.close()


def test_batch_run_matches_oracle(pic):
    """One run of a batch, particle by particle against the FP64 oracle for 12 steps."""
    import oracle
    wls = _scan_runs()
    batch = pic.Engine.from_workloads(wls, track_ids=True, diag_interval=0)
    batch.step(12)
    r = 3
    wl = wls[r]
    sim = oracle.Simulation.from_workload(wl)
    sim.step(12, record=False)
    for s in range(2):
        cell, off, u, ids = batch.particles(s, run=r)
        o = np.argsort(ids)
        ug = u[:, o].astype(np.float64)
        uo = sim.species[s].u
        err = np.linalg.norm(ug - uo, axis=0) / np.maximum(np.linalg.norm(uo, axis=0), 1e-12)
        assert err.max() < 1e-5, (s, err.max())
    batch.close()


def test_batch_rejects_bad_run_index(pic):
    wls = _scan_runs()[:2]
    batch = pic.Engine.from_workloads(wls)
    with pytest.raises(pic.PicError):
        batch.diag(run=2)
    with pytest.raises(pic.PicError):
        batch.fields(run=-1)
    batch.close()


def test_batch_3d_equals_single_runs(pic):
    """3D runs of different sizes in one context (particles binned by tile, the tiles of all runs
    numbered together): bitwise the same histories, fields and particles as each run alone,
    including a run with Krook drag."""
    spec = [((16, 16, 16), 0.2, 0.0), ((8, 16, 8), 0.05, 0.1), ((16, 8, 24), 0.3, 0.0)]
    wls = [pi.weibel_load(ndim=3, nx=n[0], ny=n[1], nz=n[2], ppc=4, T_perp_beam=T, T_bg=0.01, nu=nu,
                          seed=2000 + r)
           for r, (n, T, nu) in enumerate(spec)]
    nsteps = 12
    batch = pic.Engine.from_workloads(wls, track_ids=True, diag_interval=1, diag_capacity=32, sort_interval=4)
    batch.step(nsteps)
    for r, wl in enumerate(wls):
        single = pic.Engine.from_workload(wl, track_ids=True, diag_interval=1, diag_capacity=32, sort_interval=4)
        single.step(nsteps)
        assert batch.diag(run=r) == single.diag(), r
        Eb, Bb, Pb = _state(batch, r)
        Es, Bs, Ps = _state(single, 0)
        assert np.array_equal(Eb, Es) and np.array_equal(Bb, Bs), r
        for (c, o, u), (c0, o0, u0) in zip(Pb, Ps):
            assert np.array_equal(c, c0) and np.array_equal(o, o0) and np.array_equal(u, u0), r
        single.close()
    assert batch.stats()["flags"] == 0
    batch.close()
