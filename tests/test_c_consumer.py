"""The boundary from plain C: tests/c/abi_consumer.c compiles as C99 against include/pic.h with
every warning an error, links against libpic.so, and runs without a GPU.  Every public struct
has the layout the Python binding's ctypes mirrors assume (size and the offset of each field),
and the host-only calls give the binding's results."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MIRRORS = {"pic_config": "Config", "pic_species": "Species", "pic_diag_rec": "DiagRec",
           "pic_stats": "Stats", "pic_kernel_time": "KernelTime",
           "pic_hybrid_config": "HybridConfig", "pic_mlp_norm": "MlpNorm", "pic_tune_entry": "TuneEntry"}


@pytest.fixture(scope="module")
def consumer(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_0808_4078_gb300 import build
    lib = build.build()
    d = tmp_path_factory.mktemp("cabi")
    exe = str(d / "abi_consumer")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_consumer.c"), "-o", exe, "-L", libdir, "-lpic",
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    return dict(line.rsplit(" ", 1) for line in r.stdout.splitlines())


def test_struct_layouts_match_the_binding(consumer):
    import paper_0808_4078_gb300 as pic
    for cname, pyname in MIRRORS.items():
        cls = getattr(pic, pyname)
        assert int(consumer[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(consumer[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)
    c_fields = {k.split(".")[1] for k in consumer if k.startswith("pic_config.")}
    assert c_fields == {f for f, _ in pic.Config._fields_}


def test_host_calls_from_c(consumer):
    import paper_0808_4078_gb300 as pic
    cap = (ctypes.c_int64 * 2)(65536, 65536)
    cfg = pic.Config(2, 64, 64, 1, 0.1, 0.1, 0.1, 0.05, 2, cap, (ctypes.c_int32 * 2)(0, 0), 8, 1, 100,
                     0, 0, 0, 0, 0, 0, 0)
    assert consumer["required_rc"] == "0"
    assert int(consumer["required_bytes"]) == pic.required_bytes(cfg)
    assert consumer["bad_rc"] == "-1" and consumer["bad_has_text"] == "1"
    assert consumer["hybrid_rc"] == "0" and int(consumer["hybrid_bytes"]) > 64 * 32 * 16 * 44
    assert consumer["checkpoint_null"] == "-1" and consumer["loaded_null"] == "-1"
    assert consumer["step_count_null"] == "-1"
