"""Counting sort by cell (pic_bin_cells) through the C ABI against numpy.

start is unique and compared exactly; order is correct up to the order within a cell, so each
cell's slice is compared as a set with the indices numpy finds for that cell.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _check(cell_np, ncell, start, order):
    valid = (cell_np >= 0) & (cell_np < ncell)
    counts = np.bincount(cell_np[valid], minlength=ncell)
    want = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    assert np.array_equal(start.astype(np.int64), want)
    assert len(order) == cell_np.shape[0]
    got = order[: want[-1]]
    # every valid particle exactly once, grouped by its cell
    assert np.array_equal(np.sort(got), np.flatnonzero(valid))
    assert np.array_equal(cell_np[got], np.repeat(np.arange(ncell), counts))


@pytest.mark.parametrize("n,ncell,bad", [(0, 7, 0), (1, 1, 0), (1000, 3, 0), (4097, 5000, 0),
                                         (300_001, 65_536, 200), (2_000_000, 1 << 20, 0)])
def test_bin_cells_matches_numpy(pic, n, ncell, bad):
    import torch
    rng = np.random.default_rng(n + ncell)
    cell = rng.integers(0, ncell, n).astype(np.int32)
    if bad:
        idx = rng.choice(n, bad, replace=False)
        cell[idx[: bad // 2]] = -3
        cell[idx[bad // 2:]] = ncell + 5
    t = torch.from_numpy(cell).cuda()
    start, order = pic.bin_cells(t, ncell)
    _check(cell, ncell, start.cpu().numpy(), order.cpu().numpy())


def test_bin_cells_full_grid_sorted_input(pic):
    """Full 1024 x 1024 grid at 64 particles per cell: cell-major input (the load order of the
    2D workload), mostly identical neighbours within a warp."""
    import torch
    ncell = 1 << 20
    cell = torch.arange(ncell, dtype=torch.int32, device="cuda").repeat_interleave(64)
    start, order = pic.bin_cells(cell, ncell)
    s = start.cpu().numpy()
    assert np.array_equal(s, np.arange(ncell + 1, dtype=np.int64) * 64)
    o = order.cpu().numpy()
    samp = np.random.default_rng(0).integers(0, ncell, 2000)
    for c in samp:
        assert np.array_equal(np.sort(o[64 * c: 64 * c + 64]), np.arange(64 * c, 64 * c + 64))


def test_bin_cells_rejects_bad_arguments(pic):
    import ctypes
    import torch
    L = pic.lib()
    buf = torch.zeros(1024, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert L.pic_bin_cells(p, 10, 0, p, p, p, 4096, None) == -1          # ncell <= 0
    assert L.pic_bin_cells(p, 10, 8, p, p, p, 4, None) == -2             # scratch too small
    assert L.pic_bin_cells(p, -1, 8, p, p, p, 4096, None) == -1          # n < 0
