"""The autotuner of the 2D particle kernel (pic_autotune): it times every compiled variant whose
tile divides the grid on the next steps of the run, keeps the fastest and records it in the
tuning cache; the run itself is bitwise what it would have been with one fixed variant, and a new
context of the same workload with default tile settings starts with the cached pick."""
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


def _state(eng):
    E, B, _ = eng.fields()
    parts = []
    for s in range(2):
        cell, off, u, ids = eng.particles(s)
        o = np.argsort(ids)
        parts.append((cell[o], off[:, o], u[:, o]))
    return E, B, parts


def test_autotune_picks_fastest_keeps_run_and_caches(pic, tmp_path):
    wl = pi.weibel_load(ndim=2, nx=64, ny=64, ppc=8, T_perp_beam=0.1, T_bg=0.001, nu=0.1, seed=17)
    cache = tmp_path / "tune.jsonl"
    pic.set_tune_cache(str(cache))
    try:
        a = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, diag_interval=0)
        assert a.tile_config() == (16, 16, 3)                      # nothing cached yet
        a.step(3)
        tune = a.autotune(6)                                       # 9 variants x (4 + 8) steps
        assert len(tune) == 9
        assert {(t[0], t[1], t[2]) for t in tune} == {(x, y, c) for x, y in ((16, 16), (32, 8), (8, 32))
                                                      for c in (2, 3, 4)}
        best = min(tune, key=lambda t: t[3])
        assert a.tile_config() == best[:3]
        a.step(5)
        total = 3 + 9 * 12 + 5
        b = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, diag_interval=0, tile=(16, 16),
                                     ctas_per_sm=3)
        b.step(total)
        sa, sb = _state(a), _state(b)
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        for (c, o, u), (c0, o0, u0) in zip(sa[2], sb[2]):
            assert np.array_equal(c, c0) and np.array_equal(o, o0) and np.array_equal(u, u0)
        lines = cache.read_text().strip().splitlines()
        assert len(lines) == 1 and '"tile_x": %d' % best[0] in lines[0]
        c2 = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, diag_interval=0)
        assert c2.tile_config() == best[:3]                       # the cached pick
        d = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, diag_interval=0, tile=(8, 32),
                                     ctas_per_sm=2)
        assert d.tile_config() == (8, 32, 2)                      # explicit settings win
        pic.set_tune_cache(str(cache))                            # reload from the file
        e = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, diag_interval=0)
        assert e.tile_config() == best[:3]
        for eng in (a, b, c2, d, e):
            eng.close()
    finally:
        pic.set_tune_cache(None)


def test_autotune_skips_shapes_that_do_not_divide_the_grid(pic):
    wl = pi.weibel_load(ndim=2, nx=48, ny=48, ppc=4, T_perp_beam=0.1, T_bg=0.001, nu=0.0, seed=18)
    pic.set_tune_cache(None)
    eng = pic.Engine.from_workload(wl, sort_interval=4, diag_interval=0)
    tune = eng.autotune(4)
    assert {(t[0], t[1]) for t in tune} == {(16, 16)}
    eng.close()
    pic.set_tune_cache(None)
