"""Planted mistakes in the oracle must fail a pin.

Each case compiles a copy of oracle/pic_oracle.c with one plausible error (a dropped factor,
a flipped sign, a wrong stagger or index) in a temporary directory, runs the pin suite against
that copy on the CPU, and requires it to fail.  The hybrid model's oracle (oracle/hybrid.py)
gets the same treatment against its own pins.  The repository's oracle is never modified.
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


HYBRID_MUTATIONS = {
    "uniform_plasma_density": ("return np.maximum(self.n0 - nb, 0.0)",
                               "return np.maximum(self.n0 - nb.mean() + 0.0 * nb, 0.0)"),
    "force_plasma_sign": ("f = uz / g - bpp", "f = uz / g + bpp"),
    "ohmic_term_dropped": ("rhs = jb + n_p * (bp - a - self.nu * dt * bp)", "rhs = jb + n_p * (bp - a)"),
    "plasma_update_without_friction": ("self.beta_p = bp + a_new - a - self.nu * dt * bp",
                                       "self.beta_p = bp + a_new - a"),
    "canonical_momentum_without_a": ("uz = P + ua", "uz = P"),
    "move_without_gamma": ("X = (X + dt * ux / (g2 * self.dx)) % self.nx", "X = (X + dt * ux / self.dx) % self.nx"),
    "current_without_gamma": ("jb = self._deposit(self.X, self.Y, self.w * uzs / gs)",
                              "jb = self._deposit(self.X, self.Y, self.w * uzs)"),
    "gradient_x_weights": ("gx = ((1 - fy) * (F[j0, i1] - F[j0, i0]) + fy * (F[j1, i1] - F[j1, i0])) / self.dx",
                           "gx = ((1 - fx) * (F[j0, i1] - F[j0, i0]) + fx * (F[j1, i1] - F[j1, i0])) / self.dx"),
    "laplacian_wrong_spacing": ("return (sp.kron(sp.identity(ny), ring(nx, dx)) + sp.kron(ring(ny, dy), sp.identity(nx))).tocsc()",
                                "return (sp.kron(sp.identity(ny), ring(nx, dx)) + sp.kron(ring(ny, dx), sp.identity(nx))).tocsc()"),
    "energy_uniform_density": ("0.5 * np.sum(self.plasma_density() * self.beta_p ** 2) * dA",
                               "0.5 * self.n0 * np.sum(self.beta_p ** 2) * dA"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(HYBRID_MUTATIONS))
def test_planted_hybrid_mistake_is_caught(name, tmp_path):
    old, new = HYBRID_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "hybrid.py")).read()
    assert old in src, f"mutation anchor for {name} no longer in the hybrid oracle"
    d = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    (d / "tests").mkdir()
    for f in ("conftest.py", "test_oracle_hybrid.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), d / "tests" / f)
    (d / "oracle" / "hybrid.py").write_text(src.replace(old, new, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_hybrid.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=d, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 1, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"


# Mistakes in the closed forms (oracle/theory.py: the cold two-fluid relation, Eqs. 11, 12
# and 14) and in the growth fit (oracle/fit.py), caught by the pins that use them.
THEORY_MUTATIONS = {
    "theory.py": {
        "eq12_collision_term_dropped": ("coeffs = [k2 + 1.0, 1j * k2 * nu,", "coeffs = [k2 + 1.0, 0.0 * nu,"),
        "eq12_constant_term_sign": ("1j * nu * (b - a * k2)]", "1j * nu * (b + a * k2)]"),
        "eq11_threshold_sign": ("return cs2 - beta0 * beta0 * nb / n0", "return cs2 + beta0 * beta0 * nb / n0"),
        "cold_coupling_sign": ("A * k2 * C - k2 * D * D]", "A * k2 * C + k2 * D * D]"),
        "cold_B_gamma_power": ("B += n / g ** 3", "B += n / g"),
    },
    "fit.py": {
        "fit_energy_not_amplitude": ("best = (0.5 * slope,", "best = (slope,"),
        "fit_noise_level_ignored": ("ok = (W > lo) & (W < hi)", "ok = (W > 0) & (W < hi)"),
    },
}
_THEORY_CASES = [(f, n) for f in sorted(THEORY_MUTATIONS) for n in sorted(THEORY_MUTATIONS[f])]


@pytest.mark.slow
@pytest.mark.parametrize("fname,name", _THEORY_CASES)
def test_planted_theory_mistake_is_caught(fname, name, tmp_path):
    old, new = THEORY_MUTATIONS[fname][name]
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert old in src, f"mutation anchor for {name} no longer in oracle/{fname}"
    d = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "pic_inputs"), d / "pic_inputs",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (d / "tests").mkdir()
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), d / "tests" / f)
    (d / "oracle" / fname).write_text(src.replace(old, new, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-k", "dispersion or fit or cold_weibel or below_cold",
                        "-p", "no:cacheprovider"], cwd=d, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 1, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"
