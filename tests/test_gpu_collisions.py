"""Binary electron-ion collisions (pic_set_collisions) against the oracle's collisions: the two
sides draw the same Philox4x32-10 numbers (each implements the generator from its published
definition), so particles can be compared one by one.  Tolerance: each collision turns u by an
angle of order 0.1-1 rad through ~12 FP32 operations on quantities of size |u| (relative rounding
2^-24 each), i.e. up to ~7e-7 |u| per step on top of the collisionless push; over 20 steps that
accumulates to ~1.4e-5 |u| in the worst (linear) case, so the per-particle bar is 3e-5 here
instead of the collisionless 1e-5.  The draws themselves agree exactly (a mismatch would show as
errors of order tan(theta/2) ~ 0.1 of |u|)."""
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


def _check(eng, sim, tol=3e-5):
    for s in range(2):
        cell, off, u, ids = eng.particles(s)
        k = np.argsort(ids)
        ug = u[:, k].astype(np.float64)
        uo = sim.species[s].u
        err = np.linalg.norm(ug - uo, axis=0) / np.maximum(np.linalg.norm(uo, axis=0), 1e-12)
        assert err.max() < tol, (s, err.max())


@pytest.mark.parametrize("ndim", [2, 3])
def test_collisions_match_oracle(pic, ndim):
    import oracle
    if ndim == 2:
        wl = pi.weibel_load(ndim=2, nx=32, ny=32, ppc=16, T_perp_beam=0.1, T_bg=0.01, seed=91)
    else:
        wl = pi.weibel_load(ndim=3, nx=16, ny=16, nz=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, seed=92)
    nu, seed = 0.5, 0x1234_5678_9ABC_DEF0
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=8)
    eng.set_collisions(1, nu, seed)
    sim = oracle.Simulation.from_workload(wl)
    sim.set_collisions(1, nu, seed)
    for chunk in (1, 4, 15):
        eng.step(chunk)
        sim.step(chunk, record=False)
        _check(eng, sim)
    eng.close()


def test_collisions_independent_of_particle_order(pic):
    wl = pi.weibel_load(ndim=2, nx=32, ny=32, ppc=16, T_perp_beam=0.1, T_bg=0.01, seed=93)
    out = []
    for k in (1, 7, 0):
        eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=k, flags=pic.PIC_FLAG_KEEP_J)
        eng.set_collisions(1, 1.0, 77)
        eng.step(15)
        out.append(eng.fields(with_J=True))
        eng.close()
    for E, B, J in out[1:]:
        assert np.array_equal(E, out[0][0]) and np.array_equal(B, out[0][1]) and np.array_equal(J, out[0][2])


def test_zero_rate_and_missing_ids(pic):
    wl = pi.weibel_load(ndim=2, nx=32, ny=32, ppc=8, T_perp_beam=0.1, T_bg=0.01, seed=94)
    a = pic.Engine.from_workload(wl, track_ids=True)
    b = pic.Engine.from_workload(wl, track_ids=True)
    b.set_collisions(1, 0.0, 5)
    a.step(6)
    b.step(6)
    for s in range(2):
        pa, pb = a.particles(s), b.particles(s)          # slot order varies: compare by id
        ka, kb = np.argsort(pa[3]), np.argsort(pb[3])
        assert np.array_equal(pa[2][:, ka], pb[2][:, kb])
    a.close()
    b.close()
    c = pic.Engine.from_workload(wl)
    with pytest.raises(pic.PicError):
        c.set_collisions(1, 1.0, 5)
    c.close()
