"""The bounds-checked build and the NVTX ranges.

libpic_debug.so (build.build(debug=True), compiled with -DPIC_DEBUG_BOUNDS) checks every index
into the particle kernels' shared tiles and their one-cell halo before the access; a failed check
skips the access and sets the sticky flag that fails the next synchronising call with
PIC_EBOUNDS.  A small 2D Krook run (particles crossing tile edges, drag moments) and a small 3D
run with drag go through the debug library in a child process (PIC_DEBUG_BOUNDS=1 selects it):
no flag is raised, the child really loaded libpic_debug.so, and its particles and fields are
bitwise equal to the normal library's.

PIC_FLAG_NVTX (ranges per pic_step call and per phase, steps launched directly) changes no
result: bitwise equal to the same run without it.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import pic_inputs as pi
import paper_0808_4078_gb300 as pic
out = sys.argv[1]
res = {}
cases = {
    "2d": pi.weibel_load(ndim=2, nx=64, ny=32, ppc=16, T_perp_beam=0.3, T_bg=0.01, nu=0.1, seed=41),
    "3d": pi.weibel_load(ndim=3, nx=16, ny=16, nz=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, nu=0.1, seed=42),
}
arrays = {}
for name, wl in cases.items():
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, flags=pic.PIC_FLAG_KEEP_J)
    eng.step(12)
    E, B, J = eng.fields(with_J=True)
    arrays[name + "_E"], arrays[name + "_B"], arrays[name + "_J"] = E, B, J
    for s in range(2):
        cell, off, u, ids = eng.particles(s)
        o = np.argsort(ids)
        arrays[f"{name}_cell{s}"], arrays[f"{name}_off{s}"], arrays[f"{name}_u{s}"] = cell[o], off[:, o], u[:, o]
    res[name] = eng.stats()["flags"]
    eng.close()
res["lib"] = [l.split()[-1] for l in open("/proc/self/maps") if "libpic" in l][:1]
np.savez(out + ".npz", **arrays)
json.dump(res, open(out + ".json", "w"))
"""


@pytest.fixture(scope="module")
def libs():
    import __graft_entry__ as ge
    ge.build()
    from paper_0808_4078_gb300 import build
    return build.build(), build.build(debug=True)


def _child(tmp_path, name, debug):
    env = dict(os.environ)
    env["PIC_DEBUG_BOUNDS"] = "1" if debug else "0"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    out = str(tmp_path / name)
    r = subprocess.run([sys.executable, "-c", CHILD, out], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.load(open(out + ".json")), dict(np.load(out + ".npz"))


def test_debug_bounds_build_clean_and_equal(libs, tmp_path):
    lib, lib_debug = libs
    meta_d, arr_d = _child(tmp_path, "debug", True)
    meta_n, arr_n = _child(tmp_path, "normal", False)
    assert meta_d["lib"] and os.path.basename(meta_d["lib"][0]) == "libpic_debug.so", meta_d
    assert meta_n["lib"] and os.path.basename(meta_n["lib"][0]) == "libpic.so", meta_n
    assert meta_d["2d"] == 0 and meta_d["3d"] == 0, meta_d
    assert meta_n["2d"] == 0 and meta_n["3d"] == 0, meta_n
    assert arr_d.keys() == arr_n.keys()
    for k in arr_n:
        assert np.array_equal(arr_d[k], arr_n[k]), k


def test_nvtx_flag_changes_nothing(libs):
    import paper_0808_4078_gb300 as pic
    wl = pi.weibel_load(ndim=2, nx=64, ny=32, ppc=16, T_perp_beam=0.3, T_bg=0.01, nu=0.1, seed=43)

    def run(flags):
        eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=4, flags=flags)
        eng.step(9)
        E, B, J = eng.fields(with_J=True)
        parts = []
        for s in range(2):
            cell, off, u, ids = eng.particles(s)
            o = np.argsort(ids)
            parts += [cell[o], off[:, o], u[:, o]]
        st = eng.stats()
        eng.close()
        return [E, B, J] + parts, st

    ref, st0 = run(pic.PIC_FLAG_KEEP_J)
    got, st1 = run(pic.PIC_FLAG_KEEP_J | pic.PIC_FLAG_NVTX)
    assert st0["flags"] == 0 and st1["flags"] == 0
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
