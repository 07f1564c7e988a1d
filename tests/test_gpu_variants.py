"""Every compiled variant of the 2D particle kernel (tile shape 16 x 16, 32 x 8, 8 x 32; 2, 3 or
4 CTAs per SM) computes the same step: after 25 steps of a warm-beam Krook run with particles
crossing tile edges, the particles (by id), E, B and the last step's J are bitwise equal to the
default variant's, and the first of them matches the FP64 oracle."""
import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

VARIANTS = [((16, 16), 3), ((16, 16), 2), ((16, 16), 4), ((32, 8), 2), ((32, 8), 3), ((32, 8), 4),
            ((8, 32), 2), ((8, 32), 3), ((8, 32), 4)]


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _run(pic, wl, tile, ctas, steps):
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, flags=pic.PIC_FLAG_KEEP_J,
                                   tile=tile, ctas_per_sm=ctas)
    eng.step(steps)
    E, B, J = eng.fields()
    parts = []
    for s in range(2):
        cell, off, u, ids = eng.particles(s)
        o = np.argsort(ids)
        parts.append((cell[o], off[:, o], u[:, o]))
    st = eng.stats()
    eng.close()
    return E, B, J, parts, st


def test_variants_bitwise_equal(pic):
    import oracle
    wl = pi.weibel_load(ndim=2, nx=64, ny=32, ppc=16, T_perp_beam=0.3, T_bg=0.01, nu=0.1, seed=31)
    ref = _run(pic, wl, *VARIANTS[0], 25)
    assert ref[4]["flags"] == 0
    for tile, ctas in VARIANTS[1:]:
        got = _run(pic, wl, tile, ctas, 25)
        assert got[4]["flags"] == 0
        for a, b in zip(got[:3], ref[:3]):
            assert np.array_equal(a, b), (tile, ctas)
        for (c, o, u), (c0, o0, u0) in zip(got[3], ref[3]):
            assert np.array_equal(c, c0) and np.array_equal(o, o0) and np.array_equal(u, u0), (tile, ctas)
    sim = oracle.Simulation.from_workload(wl)
    sim.step(25)
    for s in range(2):
        _, _, u = ref[3][s]
        uo = sim.species[s].u
        err = np.abs(u.astype(np.float64) - uo).max() / np.abs(uo).max()
        assert err < 1e-4, (s, err)
