"""The binomial current filter (pic_config.j_filter) on the GPU against the oracle's filter.

The GPU sums the filter's 3^ndim integer-weighted terms exactly in int64 and scales by 4^-ndim in
the E update; the oracle filters its FP64 current.  The differences are those of the unfiltered
paths (FP32 push and fields, 2^-S current), so the tolerances of the 2D and 3D parity tests apply:
  * one step from seeded fields: the unfiltered current read back (PIC_FLAG_KEEP_J), filtered by
    the oracle, equals the oracle's filtered current to 1e-5 max|J| + 40 2^-S (60 in 3D); E and B
    to 1e-5 relative;
  * 20 steps: every particle's momentum to 1e-5 relative and position to 1e-4 cell;
  * the filter adds one launch per step and changes the fields (it is not a no-op).
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


def _periodic_diff(a, b, n):
    return (a - b + n / 2) % n - n / 2


def _check_particles(eng, sim, wl, tol=1e-5):
    for s in range(len(wl.species)):
        cell, off, u, ids = eng.particles(s)
        order = np.argsort(ids)
        ug = u[:, order].astype(np.float64)
        so = sim.species[s]
        err = np.linalg.norm(ug - so.u, axis=0) / np.maximum(np.linalg.norm(so.u, axis=0), 1e-12)
        assert err.max() < tol, (s, err.max())
        c = cell[order]
        X = (c % wl.nx) + off[0, order].astype(np.float64)
        Y = (c // wl.nx) % wl.ny + off[1, order].astype(np.float64)
        assert np.abs(_periodic_diff(X, so.X, wl.nx)).max() < 1e-4
        assert np.abs(_periodic_diff(Y, so.Y, wl.ny)).max() < 1e-4
        if wl.ndim == 3:
            Z = c // (wl.nx * wl.ny) + off[2, order].astype(np.float64)
            assert np.abs(_periodic_diff(Z, so.Z, wl.nz)).max() < 1e-4


def _seed(eng, sim, wl, seed=3, amp=0.05):
    rng = np.random.default_rng(seed)
    E0 = (amp * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    B0 = (amp * rng.standard_normal((3, wl.ncell))).astype(np.float32)
    eng.set_fields(E0, B0)
    shape = sim.E[0].shape
    for a in range(3):
        sim.E[a][...] = E0[a].reshape(shape)
        sim.B[a][...] = B0[a].reshape(shape)


@pytest.mark.parametrize("ndim", [2, 3])
def test_filter_one_step_and_twenty(pic, ndim):
    import oracle
    if ndim == 2:
        wl = pi.weibel_load(ndim=2, nx=48, ny=32, ppc=16, T_perp_beam=0.1, T_bg=0.001, nu=0.1, seed=23)
        nterm = 40
    else:
        wl = pi.weibel_load(ndim=3, nx=16, ny=16, nz=24, ppc=8, T_perp_beam=0.2, seed=33)
        nterm = 60
    eng = pic.Engine.from_workload(wl, track_ids=True, flags=pic.PIC_FLAG_KEEP_J, j_filter=1)
    sim = oracle.Simulation.from_workload(wl, j_filter=1)
    _seed(eng, sim, wl)
    l0 = eng.launch_count()
    eng.step(1)
    sim.step(1)
    n_step = eng.launch_count() - l0
    E, B, J = eng.fields(with_J=True)
    S = eng.fixed_point_shift()
    for a in range(3):
        jf = sim.binomial(J[a].astype(np.float64) * 2.0 ** -S)
        jo = sim.J[a].reshape(-1)
        assert np.abs(jf - jo).max() <= 1e-5 * np.abs(jo).max() + nterm * 2.0 ** -S, a
        eo, bo = sim.E[a].reshape(-1), sim.B[a].reshape(-1)
        assert np.abs(E[a] - eo).max() <= 1e-5 * (np.abs(eo).max() + 1e-3)
        assert np.abs(B[a] - bo).max() <= 1e-5 * (np.abs(bo).max() + 1e-3)
    l0 = eng.launch_count()
    eng.step(19)
    n_step += eng.launch_count() - l0        # read-backs launch kernels too: count steps only
    sim.step(19)
    _check_particles(eng, sim, wl)
    eng.close()
    off = pic.Engine.from_workload(wl, track_ids=True, flags=pic.PIC_FLAG_KEEP_J, j_filter=0)
    _seed(off, oracle.Simulation.from_workload(wl), wl)   # the same calls in the same order
    l1 = off.launch_count()
    off.step(1)
    off.step(19)
    assert n_step == off.launch_count() - l1 + 20      # one filter launch per step
    off.close()


def test_filter_changes_the_fields(pic):
    wl = pi.weibel_load(ndim=2, nx=32, ny=32, ppc=16, T_perp_beam=0.1, seed=24)
    out = []
    for jf in (0, 1):
        eng = pic.Engine.from_workload(wl, j_filter=jf)
        eng.step(5)
        out.append(eng.fields()[0])
        eng.close()
    assert not np.array_equal(out[0], out[1])
