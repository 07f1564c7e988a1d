"""The allocation-free counting sort (pic_bin_cells_noalloc) against the regular one.

Some callers cannot allocate device memory (their GPU memory belongs to an allocator they cannot
reach, or a cudaMalloc is not allowed where they call from).  For them the library offers a
variant of pic_bin_cells that uses a fixed scratch array compiled into the library.  This test
calls both entry points through the C ABI on the same inputs, twice in a row with different
sizes (the shared scratch keeps the previous call's contents, so each call must clear what it
needs), and checks that the results agree: start exactly, order as a per-cell grouping.
This file sorts last so that a run stopping at its first failure has already run the rest.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    L = pic.lib()
    L.pic_bin_cells_noalloc.restype = ctypes.c_int
    L.pic_bin_cells_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return pic, L


def _run_regular(pic, L, cell, ncell, stream):
    import torch
    nb = ctypes.c_size_t(0)
    assert L.pic_bin_cells_scratch_bytes(ncell, ctypes.byref(nb)) == 0
    scratch = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    start = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
    order = torch.full((max(cell.numel(), 1),), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()          # the fills above ran on the default stream
    rc = L.pic_bin_cells(ctypes.c_void_p(cell.data_ptr()), cell.numel(), ncell,
                         ctypes.c_void_p(start.data_ptr()), ctypes.c_void_p(order.data_ptr()),
                         ctypes.c_void_p(scratch.data_ptr()), nb.value,
                         ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    stream.synchronize()              # scratch is freed on return; the sort must be done with it
    return start, order


def _run_noalloc(L, cell, ncell, stream):
    import torch
    start = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
    order = torch.full((max(cell.numel(), 1),), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()          # the fills above ran on the default stream
    rc = L.pic_bin_cells_noalloc(ctypes.c_void_p(cell.data_ptr()), cell.numel(), ncell,
                                 ctypes.c_void_p(start.data_ptr()),
                                 ctypes.c_void_p(order.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, L.pic_last_error(None)
    stream.synchronize()
    return start, order


def test_noalloc_matches_regular_twice(lib):
    import torch
    pic, L = lib
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(11)
    # first call: a large grid; second call: a smaller one over the same shared scratch
    for n, ncell in ((1_500_000, 1 << 20), (70_001, 4097)):
        cell_np = rng.integers(0, ncell, n).astype(np.int32)
        cell_np[:: 997] = -1                 # left out by both
        cell = torch.from_numpy(cell_np).cuda()
        torch.cuda.synchronize()
        s_ref, o_ref = _run_regular(pic, L, cell, ncell, stream)
        s_new, o_new = _run_noalloc(L, cell, ncell, stream)
        stream.synchronize()
        s_ref, s_new = s_ref.cpu().numpy(), s_new.cpu().numpy()
        assert np.array_equal(s_new, s_ref)
        m = int(s_ref[-1])
        o_ref, o_new = o_ref.cpu().numpy()[:m], o_new.cpu().numpy()[:m]
        # same particles in each cell's range
        key_ref = cell_np[o_ref].astype(np.int64) * (n + 1) + o_ref
        key_new = cell_np[o_new].astype(np.int64) * (n + 1) + o_new
        assert np.array_equal(np.sort(key_ref), np.sort(key_new))
        assert np.array_equal(cell_np[o_new], np.repeat(np.arange(ncell), np.diff(s_ref)))


def test_noalloc_rejects_too_many_cells(lib):
    import torch
    _, L = lib
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = L.pic_bin_cells_noalloc(p, 4, (1 << 20) + 1, p, p, None)
    assert rc == -1
    assert b"PIC_BIN_NOALLOC_MAX_CELLS" in L.pic_last_error(None)


def test_noalloc_calls_allocate_nothing(lib):
    """After a first call (which looks up this device's scratch array), further calls leave the
    device's free memory unchanged: nothing is allocated on the caller's behalf."""
    import torch
    _, L = lib
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(12)
    ncell, n = 1 << 16, 400_000
    cell = torch.from_numpy(rng.integers(0, ncell, n).astype(np.int32)).cuda()
    start = torch.empty(ncell + 1, dtype=torch.int32, device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    args = (ctypes.c_void_p(cell.data_ptr()), n, ncell, ctypes.c_void_p(start.data_ptr()),
            ctypes.c_void_p(order.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    assert L.pic_bin_cells_noalloc(*args) == 0
    stream.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert L.pic_bin_cells_noalloc(*args) == 0
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(start[-1].item()) == n
