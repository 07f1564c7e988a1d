"""Planted mistakes in the oracle must fail a pin.

Each case copies the oracle to a temporary directory with one plausible error (a dropped
factor, a flipped sign, a wrong stagger, index or operand) in one of its files, runs the pins of
that part against the copy on the CPU (the C library is rebuilt there), and requires a pin to
fail.  Covered: the PIC step (oracle/pic_oracle.c against the main pins), the hybrid model, the
closed forms and the growth fit, the collision operator and its generator, the current filter,
the per-cell drag, the closure moments and the network.  The repository's oracle is never
modified.
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


def _pins_fail_on_copy(fname, old, new, pin_file, tmp_path, select=None):
    """Copy the oracle (and the seeded-input module) to tmp_path with one replacement in
    oracle/<fname>, run the pin file against the copy, and report whether a pin failed."""
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert old in src, f"mutation anchor no longer in oracle/{fname}: {old!r}"
    d = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "pic_inputs"), d / "pic_inputs",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (d / "tests").mkdir()
    for f in ("conftest.py", pin_file):
        shutil.copy(os.path.join(ROOT, "tests", f), d / "tests" / f)
    (d / "oracle" / fname).write_text(src.replace(old, new, 1))
    cmd = [sys.executable, "-m", "pytest", "tests/" + pin_file, "-q", "-x", "-p", "no:cacheprovider"]
    if select:
        cmd += ["-k", select]
    r = subprocess.run(cmd, cwd=d, capture_output=True, text=True, timeout=600)
    return r.returncode == 1, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    failed, out = _pins_fail_on_copy("pic_oracle.c", old, new, "test_oracle_pins.py", tmp_path)
    assert failed, f"planted mistake {name} passed every pin:\n{out}"


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
    failed, out = _pins_fail_on_copy("hybrid.py", old, new, "test_oracle_hybrid.py", tmp_path)
    assert failed, f"planted mistake {name} passed every pin:\n{out}"


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
    failed, out = _pins_fail_on_copy(fname, old, new, "test_oracle_pins.py", tmp_path,
                                     select="dispersion or fit or cold_weibel or below_cold")
    assert failed, f"planted mistake {name} passed every pin:\n{out}"


# Mistakes in the collision operator, the current filter and the per-cell drag (oracle C
# library), in the closure moments (oracle/closure.py) and in the network (oracle/mlp.py),
# each against its own pin file.
COMPONENT_MUTATIONS = {
    "collision_variance": ("pic_oracle.c", "test_oracle_collisions.py",
                           "orc_collide_ion(u, sqrt(0.5 * coll->nu_coll * g->dt), r);",
                           "orc_collide_ion(u, sqrt(coll->nu_coll * g->dt), r);"),
    "collision_cos_term": ("pic_oracle.c", "test_oracle_collisions.py",
                           "omc = 2.0 * delta * delta / (1.0 + delta * delta);",
                           "omc = delta * delta / (1.0 + delta * delta);"),
    "collision_azimuth_sign": ("pic_oracle.c", "test_oracle_collisions.py",
                               "d[1] = (u[1] * u[2] / uperp) * sn * cp + (u[0] * umag / uperp) * sn * sp",
                               "d[1] = (u[1] * u[2] / uperp) * sn * cp - (u[0] * umag / uperp) * sn * sp"),
    "philox_multiplier": ("pic_oracle.c", "test_oracle_collisions.py",
                          "p0 = (uint64_t)0xD2511F53u * c0", "p0 = (uint64_t)0xD2511F55u * c0"),
    "filter_neighbour": ("pic_oracle.c", "test_oracle_filter.py",
                         "F[c] = 0.25 * (t[m] + 2.0 * t[c] + t[p]);", "F[c] = 0.25 * (t[m] + 2.0 * t[c] + t[c]);"),
    "filter_one_axis": ("pic_oracle.c", "test_oracle_filter.py",
                        "for (int axis = 0; axis < g->ndim; axis++) {", "for (int axis = 0; axis < 1; axis++) {"),
    "drag_map_negative_rate": ("pic_oracle.c", "test_oracle_closure_drag.py",
                               "df = r > 0.0 ? 1.0 - exp(-r * g->dt) : 0.0;", "df = 1.0 - exp(-r * g->dt);"),
    "closure_tperp_half": ("closure.py", "test_oracle_closure.py",
                           'out[4 + 2 * si] = 0.5 * (var["x"] + var["y"])', 'out[4 + 2 * si] = (var["x"] + var["y"])'),
    "closure_vxb_sign": ("closure.py", "test_oracle_closure.py",
                         "fz = s.q * (EB[:, 2] + vx * EB[:, 4] - vy * EB[:, 3])",
                         "fz = s.q * (EB[:, 2] + vx * EB[:, 4] + vy * EB[:, 3])"),
    "closure_label_sign": ("closure.py", "test_oracle_closure.py",
                           "nu + (np.asarray(fz_mean) - np.asarray(fz_p)) / uz_p",
                           "nu + (np.asarray(fz_p) - np.asarray(fz_mean)) / uz_p"),
    "closure_w_es_no_zmean": ("closure.py", "test_oracle_closure.py",
                              "zmean = Ec.mean(axis=0, keepdims=True) if sim.ndim == 3 else Ec",
                              "zmean = 0.0 * Ec"),
    "closure_samples_mean_of_ratios": ("closure.py", "test_oracle_closure.py",
                                       "lab = nu_p + (m[10] - m[9]) / m[3]",
                                       "lab = nu_p + ((rows[w * window:(w + 1) * window, 10] - "
                                       "rows[w * window:(w + 1) * window, 9]) / rows[w * window:(w + 1) * window, 3]).mean(0)"),
    "closure_samples_uz_mask": ("closure.py", "test_oracle_closure.py",
                                "keep = (np.abs(m[3]) >= uz_min) & np.isfinite(lab)", "keep = np.isfinite(lab)"),
    "mlp_dsilu": ("mlp.py", "test_oracle_mlp.py",
                  "return s * (1.0 + z * (1.0 - s))", "return s * (1.0 + z * s)"),
    "mlp_w2_gradient_operand": ("mlp.py", "test_oracle_mlp.py",
                                'g["W2"] = d2.T @ c["h1"]', 'g["W2"] = d2.T @ c["h2"]'),
    "mlp_adam_bias_correction": ("mlp.py", "test_oracle_mlp.py",
                                 "vh = v / (1 - beta2 ** t)", "vh = v"),
    "mlp_bf16_ties_up": ("mlp.py", "test_oracle_mlp.py",
                         "r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16", "r = ((b + 0x8000) >> 16) << 16"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(COMPONENT_MUTATIONS))
def test_planted_component_mistake_is_caught(name, tmp_path):
    fname, pin_file, old, new = COMPONENT_MUTATIONS[name]
    failed, out = _pins_fail_on_copy(fname, old, new, pin_file, tmp_path)
    assert failed, f"planted mistake {name} passed every pin:\n{out}"
