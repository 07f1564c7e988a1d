"""Checkpoint and resume (pic_checkpoint / pic_restore).

A run interrupted at step 17 (inside a CUDA-graph period of 8 steps), written to a file, restored
into a fresh engine of the same configuration and continued to step 40 is bit for bit the
uninterrupted run: particles (compared by id, since the slot order of a cell's particles is not
unique), E, B, J, the diagnostic history and the step count.  The state covers Krook drag on the
background, binary collisions (counter-based draws keyed by id and step), a per-cell drag map,
a batch of two runs of different grids, and a 3D run.  A checkpoint of another configuration, a
truncated file and a file that is not a checkpoint are refused with PIC_EINVAL and leave the
engine as it was.
"""
import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

STOP, END = 17, 40


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _workloads(ndim):
    if ndim == 2:
        return [pi.weibel_load(ndim=2, nx=32, ny=32, ppc=16, T_perp_beam=0.1, T_bg=0.01, nu=0.2, seed=95),
                pi.weibel_load(ndim=2, nx=48, ny=32, ppc=16, T_perp_beam=0.3, T_bg=0.01, nu=0.1, seed=96)]
    return [pi.weibel_load(ndim=3, nx=16, ny=16, nz=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, nu=0.2, seed=97)]


def _kw(pic, sort_interval=8):
    return dict(track_ids=True, sort_interval=sort_interval, diag_interval=1, diag_capacity=64,
                flags=pic.PIC_FLAG_KEEP_J)


def _loaded(pic, wls, **kw):
    import torch
    eng = pic.Engine.from_workloads(wls, **kw)
    eng.set_collisions(1, 0.5, 0x5EED_0001, run=0)
    if len(wls) > 1:
        eng.set_collisions(0, 0.2, 0x5EED_0002, run=1)
        g = torch.Generator().manual_seed(3)
        nu = (0.3 * torch.rand((32 // 4) * (48 // 4), generator=g)).to(torch.float32).cuda()
        eng.set_drag_map(1, nu, bx=4, by=4, run=1)
    return eng


def _blank(pic, wls, **kw):
    """An engine of the same configuration with nothing loaded."""
    w0 = wls[0]
    runs = [(wl.nx, wl.ny, wl.nz, tuple(s.n for s in wl.species)) for wl in wls]
    return pic.Engine(w0.ndim, dx=w0.dx, dy=w0.dy, dz=w0.dz, dt=w0.dt, nspecies=len(w0.species),
                      runs=runs, **kw)


def _state(eng, nruns):
    out = []
    for r in range(nruns):
        parts = []
        for s in range(2):
            cell, off, u, ids = eng.particles(s, run=r)
            k = np.argsort(ids)
            parts.append((ids[k], cell[k], off[:, k], u[:, k]))
        out.append((parts, eng.fields(with_J=True, run=r), eng.diag(run=r)))
    return out


def _assert_same(a, b):
    for (pa, fa, da), (pb, fb, db) in zip(a, b):
        for x, y in zip(pa, pb):
            for u, v in zip(x, y):
                assert np.array_equal(u, v)
        for u, v in zip(fa, fb):
            assert np.array_equal(u, v)
        assert da == db


@pytest.mark.parametrize("ndim", [2, 3])
def test_resume_is_bitwise_the_uninterrupted_run(pic, ndim, tmp_path):
    wls = _workloads(ndim)
    path = str(tmp_path / "run.ckpt")
    ref = _loaded(pic, wls, **_kw(pic))
    ref.step(END)
    want = _state(ref, len(wls))
    ref.close()

    eng = _loaded(pic, wls, **_kw(pic))
    eng.step(STOP)
    eng.checkpoint(path)
    before = _state(eng, len(wls))
    eng.close()

    res = _blank(pic, wls, **_kw(pic))
    res.restore(path)
    assert res.step_count() == STOP
    assert res.loaded == [[s.n for s in wl.species] for wl in wls]
    _assert_same(_state(res, len(wls)), before)
    res.step(END - STOP)
    assert res.step_count() == END
    _assert_same(_state(res, len(wls)), want)
    res.close()


def test_restore_refuses_bad_files(pic, tmp_path):
    wls = _workloads(2)
    path = str(tmp_path / "run.ckpt")
    eng = _loaded(pic, wls, **_kw(pic))
    eng.step(5)
    eng.checkpoint(path)
    eng.close()
    data = open(path, "rb").read()

    other = _blank(pic, wls, **_kw(pic, sort_interval=4))       # another schedule
    with pytest.raises(pic.PicError) as e:
        other.restore(path)
    assert e.value.code == -1
    other.close()
    single = _blank(pic, wls[:1], **_kw(pic))                   # another batch
    with pytest.raises(pic.PicError) as e:
        single.restore(path)
    assert e.value.code == -1
    single.close()

    res = _blank(pic, wls, **_kw(pic))
    for name, blob in (("short", data[:-4096]), ("junk", b"not a checkpoint" * 16),
                       ("long", data + b"\0")):
        bad = str(tmp_path / name)
        open(bad, "wb").write(blob)
        with pytest.raises(pic.PicError) as e:
            res.restore(bad)
        assert e.value.code == -1
        assert res.step_count() == 0 and res.loaded == [[0, 0], [0, 0]]
    res.restore(path)                                           # still usable
    assert res.step_count() == 5
    res.step(3)
    res.sync()
    res.close()
