"""pic_load_species reads arrays the device can address (pinned host memory here) directly in
the binning kernel, and copies other host arrays to the device first: both paths load the same
particles, and a run started from either is bitwise the same (2D and 3D, a drag species)."""
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


def _run(pic, wl, pinned):
    import torch
    eng = pic.Engine(wl.ndim, wl.nx, wl.ny, wl.nz, dx=wl.dx, dt=wl.dt, capacity=[s.n for s in wl.species],
                     sort_interval=4, diag_interval=1, diag_capacity=64, track_ids=True)
    keep = []
    for i, s in enumerate(wl.species):
        c, o, u = s.cell, s.offset, s.u
        if pinned:
            t = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (c, o, u)]
            keep.append(t)
            c, o, u = (x.numpy() for x in t)
        eng.load_species(i, s.q, s.m, s.w, s.nu, c, o, u)
    loaded = [eng.particles(s) for s in range(len(wl.species))]
    eng.step(6)
    E, B, _ = eng.fields()
    parts = []
    for s in range(len(wl.species)):
        cell, off, u, ids = eng.particles(s)
        o = np.argsort(ids)
        parts.append((cell[o], off[:, o], u[:, o]))
    recs = eng.diag()
    eng.close()
    return loaded, E, B, parts, [r["WB"] for r in recs]


@pytest.mark.parametrize("ndim", [2, 3])
def test_pinned_and_pageable_loads_agree(pic, ndim):
    if ndim == 2:
        wl = pi.weibel_load(ndim=2, nx=64, ny=32, ppc=16, T_perp_beam=0.3, T_bg=0.01, nu=0.1, seed=61)
    else:
        wl = pi.weibel_load(ndim=3, nx=16, ny=16, nz=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, nu=0.1, seed=62)
    a = _run(pic, wl, pinned=False)
    b = _run(pic, wl, pinned=True)
    for (c0, o0, u0, i0), (c1, o1, u1, i1) in zip(a[0], b[0]):
        k0, k1 = np.argsort(i0), np.argsort(i1)
        assert np.array_equal(i0[k0], i1[k1]) and np.array_equal(c0[k0], c1[k1])
        assert np.array_equal(o0[:, k0], o1[:, k1]) and np.array_equal(u0[:, k0], u1[:, k1])
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    for (c0, o0, u0), (c1, o1, u1) in zip(a[3], b[3]):
        assert np.array_equal(c0, c1) and np.array_equal(o0, o1) and np.array_equal(u0, u1)
    assert a[4] == b[4]
