"""Device-side failure paths, exercised without faulting or hanging the GPU.

* A non-finite field value (set through pic_set_fields) makes the particles that gather it
  non-finite: the step keeps those particles unmoved, leaves them out of the current, sets the
  sticky PIC_EBADPART flag, and computes every other particle exactly as a run without the bad
  value does (2D and 3D).
* The closure network's bounded completion wait: a test kernel waits on a barrier that nothing
  arrives on (no tensor-core work in flight) with a limit of a few hundred polls; the give-up
  is reported by pic_mlp_status as PIC_ETIMEOUT, clears on read, and the next forward call runs
  and returns the same outputs as before.
"""
import ctypes

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

PIC_EBADPART, PIC_ETIMEOUT, PIC_EINVAL = -5, -6, -1
FLAG_BADPART = 1


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _particles(eng, ns):
    out = []
    for s in range(ns):
        cell, off, u, ids = eng.particles(s)
        o = np.argsort(ids)
        out.append((cell[o], off[:, o], u[:, o]))
    return out


def _cell_coords(cell, dims):
    c = cell.astype(np.int64)
    coords = []
    for n in dims:
        coords.append(c % n)
        c //= n
    return coords


def _periodic_dist(a, b, n):
    d = np.abs(a - b) % n
    return np.minimum(d, n - d)


@pytest.mark.parametrize("ndim", [2, 3])
def test_nonfinite_field_flags_badpart_and_spares_the_rest(pic, ndim):
    if ndim == 2:
        wl = pi.weibel_load(ndim=2, nx=32, ny=32, ppc=8, T_perp_beam=0.1, T_bg=0.001, nu=0.1, seed=41)
        dims = (32, 32)
    else:
        wl = pi.weibel_load(ndim=3, nx=16, ny=16, nz=16, ppc=4, T_perp_beam=0.2, T_bg=0.0, nu=0.0,
                            seed=42)
        dims = (16, 16, 16)
    ncell = int(np.prod(dims))
    rng = np.random.default_rng(3)
    E = (1e-3 * rng.standard_normal((3, ncell))).astype(np.float32)
    B = (1e-3 * rng.standard_normal((3, ncell))).astype(np.float32)
    node = tuple(d // 2 for d in dims)
    flat = 0
    for k in reversed(range(ndim)):
        flat = flat * dims[k] + node[k]
    Ebad = E.copy()
    Ebad[0, flat] = np.nan
    res = []
    for EE in (E, Ebad):
        eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4)
        eng.set_fields(EE, B)
        eng.step(1)
        if EE is E:
            eng.sync()
            flags = eng.clear_flags()
        else:
            with pytest.raises(pic.PicError) as e:
                eng.sync()
            assert e.value.code == PIC_EBADPART
            flags = eng.clear_flags()
            eng.sync()                          # cleared: reads back normally
        res.append((flags, _particles(eng, len(wl.species))))
        eng.close()
    (f0, good), (f1, bad) = res
    assert f0 == 0 and f1 & FLAG_BADPART
    nbad = 0
    for s, sp in enumerate(wl.species):
        (c0, o0, u0), (c1, o1, u1) = good[s], bad[s]
        same = (c0 == c1) & np.all(o0 == o1, axis=0) & np.all(u0 == u1, axis=0)
        kept = (c1 == sp.cell) & np.all(o1 == sp.offset, axis=0) & np.all(u1 == sp.u, axis=0)
        assert np.all(same | kept), s
        changed = ~same
        nbad += int(changed.sum())
        # the particles kept unmoved sit next to the bad node
        xyz = _cell_coords(sp.cell[changed], dims)
        for k in range(ndim):
            assert np.all(_periodic_dist(xyz[k], node[k], dims[k]) <= 2), (s, k)
    assert nbad > 0


def test_network_wait_timeout_is_reported_and_recovers(pic):
    import torch
    from oracle import mlp
    L = pic.lib()
    assert L.pic_mlp_status(1) in (0, PIC_ETIMEOUT)        # start clean
    rng = np.random.default_rng(5)
    p = mlp.init_params(seed=5)
    x = rng.normal(0, 1, (1000, 9)).astype(np.float32)
    net = pic.ClosureNet(p, np.zeros(9), np.ones(9))
    xd = torch.as_tensor(np.ascontiguousarray(x.T), device="cuda")
    y0 = net.forward(xd).cpu().numpy()
    stream = torch.cuda.Stream()
    assert L.pic_mlp_wait_test(0, ctypes.c_void_p(stream.cuda_stream)) == PIC_EINVAL
    assert L.pic_mlp_wait_test(1 << 21, ctypes.c_void_p(stream.cuda_stream)) == PIC_EINVAL
    assert L.pic_mlp_wait_test(200, ctypes.c_void_p(stream.cuda_stream)) == 0
    stream.synchronize()
    assert L.pic_mlp_status(0) == PIC_ETIMEOUT              # sticky
    assert L.pic_mlp_status(1) == PIC_ETIMEOUT              # reported, then cleared
    assert L.pic_mlp_status(0) == 0
    y1 = net.forward(xd).cpu().numpy()                      # the network runs again
    assert L.pic_mlp_status(0) == 0
    assert np.array_equal(y0, y1)
