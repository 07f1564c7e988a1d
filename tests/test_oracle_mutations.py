"""Planted mistakes in the oracle must fail a pin.

Each case compiles a copy of oracle/pic_oracle.c with one plausible error (a dropped factor,
a flipped sign, a wrong stagger or index) in a temporary directory, runs the pin suite against
that copy on the CPU, and requires it to fail.  The repository's oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "drag_sign": ("u[a] -= dragf * ubar_c[a];", "u[a] += dragf * ubar_c[a];"),
    "gather_Ex_stagger": ("EB[0] = interp2(g, g->Ex, X, Y, 0.5, 0.0);",
                          "EB[0] = interp2(g, g->Ex, X, Y, 0.0, 0.0);"),
    "gather_Bz_stagger": ("EB[5] = interp2(g, g->Bz, X, Y, 0.5, 0.5);",
                          "EB[5] = interp2(g, g->Bz, X, Y, 0.5, 0.0);"),
    "jz_weight_order": ("double wz = S0x[k] * S0y[l] / 3.0 + S0x[k] * S1y[l] / 6.0",
                        "double wz = S0x[k] * S0y[l] / 6.0 + S0x[k] * S1y[l] / 3.0"),
    "esirkepov_half": ("acc += DSx[k] * (S0y[l] + 0.5 * DSy[l]);",
                       "acc += DSx[k] * (S0y[l] + 1.0 * DSy[l]);"),
    "yee_current_sign": ("g->Ez[c] += dt * (dBy_dx - dBx_dy - g->Jz[c]);",
                         "g->Ez[c] += dt * (dBy_dx - dBx_dy + g->Jz[c]);"),
    "yee_faraday_sign": ("g->By[c] += h * dEz_dx;", "g->By[c] -= h * dEz_dx;"),
    "boris_rotation_sign": ("double upl[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),",
                            "double upl[3] = {um[0] - (up[1] * s[2] - up[2] * s[1]),"),
    "move_without_gamma": ("P1[0] = P0[0] + g->dt * u[0] / gam / g->dx;",
                           "P1[0] = P0[0] + g->dt * u[0] / g->dx;"),
    "boris_t_without_gamma": ("double t[3] = {h * EB[3] / gm, h * EB[4] / gm, h * EB[5] / gm};",
                              "double t[3] = {h * EB[3], h * EB[4] / gm, h * EB[5] / gm};"),
    "kinetic_diag_volume": ("d->Ekin[si] += s->w * (gmid - 1.0) * dV;",
                            "d->Ekin[si] += s->w * (gmid - 1.0);"),
    "yee3d_curl_sign": ("g->Bx[c] -= h * (dEz_dy - dEy_dz);", "g->Bx[c] -= h * (dEz_dy + dEy_dz);"),
    "esirkepov3d_third": ("+ 0.5 * S0[1][l] * DS[2][m] + DS[1][l] * DS[2][m] / 3.0);",
                          "+ 0.5 * S0[1][l] * DS[2][m] + DS[1][l] * DS[2][m] / 2.0);"),
    "gather3d_Ez_stagger": ("EB[2] = interp3(g, g->Ez, X, Y, Z, 0.0, 0.0, 0.5);",
                            "EB[2] = interp3(g, g->Ez, X, Y, Z, 0.0, 0.0, 0.0);"),
    "moments_component": ("s->ubar[3 * c + 2] += s->uz[p];", "s->ubar[3 * c + 2] += s->ux[p];"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "pic_oracle.c")).read()
    assert old in src, f"mutation anchor for {name} no longer in the oracle"
    d = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "pic_inputs"), d / "pic_inputs",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (d / "tests").mkdir()
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), d / "tests" / f)
    (d / "oracle" / "pic_oracle.c").write_text(src.replace(old, new, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=d, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 1, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"
