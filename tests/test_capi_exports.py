"""The C-ABI library builds, loads without a GPU and exports every function of include/pic.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpic():
    from paper_0808_4078_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared("pic.h")
    for must in ("pic_init", "pic_load_species", "pic_step", "pic_diag", "pic_required_bytes",
                 "pic_free", "pic_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(libpic):
    missing = [n for n in _declared("pic.h") if not hasattr(libpic, n)]
    assert not missing, missing


def test_required_bytes_and_config_errors_without_gpu(libpic):
    import paper_0808_4078_gb300 as pic
    cap = lambda a, b: (ctypes.c_int64 * 2)(a, b)
    ccap = lambda a=0, b=0: (ctypes.c_int32 * 2)(a, b)
    cfg = pic.Config(2, 64, 64, 1, 0.1, 0.1, 0.1, 0.05, 2, cap(65536, 65536), ccap(), 8, 1, 100,
                     0, 0, 0, 0, 0)
    n = pic.required_bytes(cfg)
    # automatic cell capacity 8 x 16 = 128 slots; 2 buffers x 2 species x 4096 cells x 128 x 20 B
    assert n >= 2 * 2 * 4096 * 128 * 20 + 64 * 64 * (24 + 24)
    bad = pic.Config(2, 60, 64, 1, 0.1, 0.1, 0.1, 0.05, 2, cap(1, 1), ccap(), 8, 1, 100,
                     0, 0, 0, 0, 0)
    with pytest.raises(pic.PicError) as e:
        pic.required_bytes(bad)
    assert e.value.code == -1
    courant = pic.Config(2, 64, 64, 1, 0.1, 0.1, 0.1, 0.08, 2, cap(1, 1), ccap(), 8, 1, 100,
                         0, 0, 0, 0, 0)
    with pytest.raises(pic.PicError):
        pic.required_bytes(courant)
    filt = pic.Config(2, 64, 64, 1, 0.1, 0.1, 0.1, 0.05, 2, cap(65536, 65536), ccap(), 8, 1, 100,
                      0, 0, 0, 0, 0, 1)
    assert pic.required_bytes(filt) >= n + 64 * 64 * 24      # the filtered current, int64 x 3
    filt.j_filter = 2
    with pytest.raises(pic.PicError):
        pic.required_bytes(filt)
    tight = pic.Config(2, 64, 64, 1, 0.1, 0.1, 0.1, 0.05, 2, cap(65536, 65536), ccap(16, 16), 8, 1,
                       100, 0, 0, 0, 0, 0)
    with pytest.raises(pic.PicError):     # slots must hold 2 x the mean per cell
        pic.required_bytes(tight)


def _batch_bytes(cfg, dims, caps):
    import numpy as np
    import paper_0808_4078_gb300 as pic
    d = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1)
    c = np.ascontiguousarray(caps, dtype=np.int64).reshape(-1)
    n = ctypes.c_size_t(0)
    rc = pic.lib().pic_required_bytes_batch(ctypes.byref(cfg), len(d) // 3, d.ctypes.data_as(ctypes.c_void_p),
                                            c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n))
    return rc, n.value


def test_batch_geometry_without_gpu(libpic):
    """Host-side geometry of batches and 3D grids: sizes add up, bad entries are refused."""
    import paper_0808_4078_gb300 as pic
    z2 = lambda: (ctypes.c_int64 * 2)(0, 0)
    cfg = pic.Config(2, 0, 0, 1, 0.1, 0.1, 0.1, 0.05, 2, z2(), (ctypes.c_int32 * 2)(32, 32), 8, 1,
                     16, 0, 0, 0, 0, 0, 0)
    rc1, a = _batch_bytes(cfg, [64, 64, 1], [64 * 64 * 4] * 2)
    rc2, b = _batch_bytes(cfg, [32, 48, 1], [32 * 48 * 4] * 2)
    rc3, ab = _batch_bytes(cfg, [64, 64, 1, 32, 48, 1], [64 * 64 * 4] * 2 + [32 * 48 * 4] * 2)
    assert rc1 == rc2 == rc3 == 0
    assert max(a, b) < ab <= a + b + (1 << 20)                   # one arena holds both runs
    assert _batch_bytes(cfg, [64, 64, 1, 30, 48, 1], [1] * 4)[0] == -1       # not a tile multiple
    assert _batch_bytes(cfg, [64, 64, 1, 0, 48, 1], [1] * 4)[0] == -1        # empty grid
    assert _batch_bytes(cfg, [64, 64, 1], [1, -1])[0] == -1                  # negative capacity
    assert _batch_bytes(cfg, [64, 64, 1], [1 << 31, 0])[0] == -1             # >= 2^31 particles
    cfg.cell_capacity[0] = cfg.cell_capacity[1] = 65535
    assert _batch_bytes(cfg, [4096, 4096, 1], [1, 1])[0] == -1               # slots >= 2^31
    cfg.cell_capacity[0] = cfg.cell_capacity[1] = 0
    cfg.tile_x = 8
    assert _batch_bytes(cfg, [64, 64, 1], [1, 1])[0] == -1                   # 8 x 16 is not a 2D tile
    for tx, ty in ((32, 8), (8, 32), (16, 16)):
        cfg.tile_x, cfg.tile_y = tx, ty
        for ctas in (0, 2, 3, 4):
            cfg.ctas_per_sm = ctas
            assert _batch_bytes(cfg, [64, 64, 1], [1, 1])[0] == 0, (tx, ty, ctas)
        for ctas in (1, 5):
            cfg.ctas_per_sm = ctas
            assert _batch_bytes(cfg, [64, 64, 1], [1, 1])[0] == -1           # no such variant
    cfg.ctas_per_sm = 0
    cfg.tile_x, cfg.tile_y = 32, 8
    assert _batch_bytes(cfg, [48, 64, 1], [1, 1])[0] == -1                   # 48 not a multiple of 32
    cfg.tile_x = cfg.tile_y = 0
    c3 = pic.Config(3, 16, 16, 8, 0.1, 0.1, 0.1, 0.05, 2, z2(), (ctypes.c_int32 * 2)(0, 0), 8, 1,
                    16, 0, 0, 0, 0, 0, 0)
    rc, n3 = _batch_bytes(c3, [16, 16, 8], [16 * 16 * 8 * 8] * 2)
    assert rc == 0 and n3 > 2 * 2 * 2048 * 24 * 24       # species x buffers x cells x 3*8 slots x 24 B
    assert _batch_bytes(c3, [16, 16, 6], [1, 1])[0] == -1                     # z not a multiple of 4
    c3.dt = 0.06                                                              # Courant: 0.06 sqrt(300) > 1
    assert _batch_bytes(c3, [16, 16, 8], [1, 1])[0] == -1


def test_checkpoint_argument_errors_without_gpu(libpic):
    import paper_0808_4078_gb300 as pic
    lib = pic.lib()
    assert lib.pic_checkpoint(None, b"/nonexistent/x.ckpt") == -1
    assert lib.pic_restore(None, b"/nonexistent/x.ckpt") == -1
    assert lib.pic_loaded_count(None, 0, 0) == -1


def test_hybrid_required_bytes_and_config_errors_without_gpu(libpic):
    import paper_0808_4078_gb300 as pic
    lib = pic.lib()
    nb = ctypes.c_size_t(0)
    ok = pic.HybridConfig(256, 128, 0.1, 0.1, 0.05, 1.0, 0.0, 0.01, 1000, 0.0, 0, 0)
    assert lib.pic_hybrid_required_bytes(ctypes.byref(ok), ctypes.byref(nb)) == 0
    # particles 24 B + id + sort buffer and index (60 B), grid 5 x 8 B + 7 x 4 B + one 8 B complex
    assert nb.value >= 1000 * 60 + 256 * 128 * (40 + 28 + 8)
    for bad in (pic.HybridConfig(96, 128, 0.1, 0.1, 0.05, 1.0, 0.0, 0.01, 10, 0.0, 0, 0),     # not 2^k
                pic.HybridConfig(4096, 8, 0.1, 0.1, 0.05, 1.0, 0.0, 0.01, 10, 0.0, 0, 0),     # > 2048
                pic.HybridConfig(64, 64, 0.1, 0.1, 0.1, 1.0, 0.0, 0.01, 10, 0.0, 0, 0),       # dt = dx
                pic.HybridConfig(64, 64, 0.1, 0.1, 0.05, 0.0, 0.0, 0.01, 10, 0.0, 0, 0),      # n0 = 0
                pic.HybridConfig(64, 64, 0.1, 0.1, 0.05, 1.0, -1.0, 0.01, 10, 0.0, 0, 0),     # nu < 0
                pic.HybridConfig(64, 64, 0.1, 0.1, 0.05, 1.0, 0.0, 0.01, -1, 0.0, 0, 0),      # capacity
                pic.HybridConfig(64, 64, 0.1, 0.1, 0.05, 1.0, 0.0, 0.01, 10, 0.0, 5000)):  # max_iter
        assert lib.pic_hybrid_required_bytes(ctypes.byref(bad), ctypes.byref(nb)) == -1


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_0808_4078_gb300 as pic
    monkeypatch.setattr(pic, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pic, "_lib", None)
    with pytest.raises(RuntimeError):
        pic.lib()
