"""Pins of the closure moments (oracle.closure) against values fixed by hand or by the
mathematics, independent of the code under test:

  * means and variances of a few hand-placed particles (closed forms);
  * densities of a uniform load: n = sum w / cells reproduces the loaded densities exactly;
  * a Maxwellian sample recovers its temperature within sampling error;
  * W_ES of E_z = A sin(2 pi m k / nz): A^2 / 2 (mean of sin^2 over whole periods); z-uniform
    fields give 0;
  * uniform fields: the mean particle force equals the force of the mean fields (the force is
    linear in v), so the label is exactly the Krook rate;
  * a z-alternating B_y with velocities correlated to it: the label's fluctuation part by hand.
"""
import numpy as np
import pytest

import oracle
from oracle import closure


def _sim3(nx=8, ny=8, nz=4):
    return oracle.Simulation(3, nx, ny, nz, dx=0.1, dt=0.05)


def _add(sim, X, Y, Z, u, w=0.25, q=-1.0, nu=0.0):
    u = np.asarray(u, dtype=np.float64)
    sim.add_species(q, 1.0, w, nu, np.asarray(X, float), np.asarray(Y, float),
                    None if Z is None else np.asarray(Z, float), u[0], u[1], u[2])


def test_hand_placed_means_and_variances():
    sim = _sim3()
    # beam: two particles in coarse cell 0 (cells 0..3 x 0..3), u = (1,0,2) and (3,0,4)
    _add(sim, [0.5, 2.5], [0.5, 3.5], [0.5, 3.5], [[1, 3], [0, 0], [2, 4]], w=0.5)
    # background: one particle in coarse cell 3 (x 4..7, y 4..7) with u = (0, 1, -1)
    _add(sim, [6.2], [5.1], [1.0], [[0], [1], [-1]], w=0.2, nu=0.3)
    m = closure.coarse_moments(sim, 4, 4)
    cells = 4 * 4 * 4
    assert m.shape == (12, 4)
    assert m[0, 0] == pytest.approx(1.0 / cells)            # n_b = 2 * 0.5 / 64
    assert m[0, 1:].tolist() == [0.0, 0.0, 0.0]
    assert m[1, 3] == pytest.approx(0.2 / cells)
    assert m[2, 0] == pytest.approx(3.0)                     # <u_z> = (2 + 4) / 2
    assert m[4, 0] == pytest.approx(0.5)                     # (Var ux = 1, Var uy = 0) / 2
    assert m[5, 0] == pytest.approx(1.0)                     # Var uz
    assert m[3, 3] == pytest.approx(-1.0)
    assert m[6, 3] == pytest.approx(0.0, abs=1e-15) and m[7, 3] == pytest.approx(0.0, abs=1e-15)
    # no fields: no force, label = nu
    assert m[9, 3] == 0.0 and m[10, 3] == 0.0
    assert m[11, 3] == pytest.approx(0.3)
    assert m[11, 0] == 0.0                                   # no background there: uz_p = 0


def test_uniform_load_densities():
    import pic_inputs as pi
    wl = pi.weibel_load(ndim=3, nx=8, ny=8, nz=4, ppc=4, T_perp_beam=0.2, seed=5)
    sim = oracle.Simulation.from_workload(wl)
    m = closure.coarse_moments(sim, 4, 2)
    assert np.allclose(m[0], 0.1, rtol=1e-12) and np.allclose(m[1], 0.9, rtol=1e-12)


def test_maxwellian_temperature():
    rng = np.random.default_rng(7)
    n = 200_000
    T = 0.04
    sim = oracle.Simulation(2, 4, 4, dx=0.1, dt=0.05)
    X, Y = rng.random(n) * 4, rng.random(n) * 4
    u = rng.normal(0.0, np.sqrt(T), (3, n))
    u[2] += 0.5
    _add(sim, X, Y, None, u, w=1.0 / n)
    m = closure.coarse_moments(sim, 4, 4)
    se = T * np.sqrt(2.0 / n)                                 # standard error of a variance
    assert abs(m[5, 0] - T) < 5 * se
    assert abs(m[4, 0] - T) < 5 * se
    assert abs(m[2, 0] - 0.5) < 5 * np.sqrt(T / n)


def test_w_es_sinusoid_and_z_uniform():
    sim = _sim3(8, 8, 16)
    A, mode = 0.3, 3
    k = np.arange(16)
    sim.E[2][...] = (A * np.sin(2 * np.pi * mode * k / 16))[:, None, None]
    sim.E[0][...] = np.linspace(0, 1, 8)[None, None, :]       # depends on x only: no z fluctuation
    _add(sim, [1.0], [1.0], [1.0], [[0], [0], [1]])
    _add(sim, [1.0], [1.0], [1.0], [[0], [0], [-1]])
    m = closure.coarse_moments(sim, 2, 4)
    assert np.allclose(m[8], A * A / 2, rtol=1e-12)


def test_uniform_fields_label_is_krook_rate():
    rng = np.random.default_rng(3)
    sim = _sim3(8, 8, 4)
    for a, v in enumerate((0.01, -0.02, 0.03)):
        sim.E[a][...] = v
    for a, v in enumerate((0.2, -0.1, 0.05)):
        sim.B[a][...] = v
    n = 500
    _add(sim, rng.random(n) * 8, rng.random(n) * 8, rng.random(n) * 4, rng.normal(0, 0.3, (3, n)))
    u = rng.normal(0, 0.1, (3, n))
    u[2] -= 0.1
    _add(sim, rng.random(n) * 8, rng.random(n) * 8, rng.random(n) * 4, u, nu=0.7)
    m = closure.coarse_moments(sim, 4, 4)
    assert np.allclose(m[9], m[10], rtol=1e-12, atol=1e-15)
    assert np.allclose(m[11][m[3] != 0], 0.7, rtol=1e-10)


def test_fluctuating_by_friction_by_hand():
    """B_y = B1 (-1)^k; two background particles at By lattice points of layers k = 0 and 1 with
    u_x = +a and -a, u_z = b: each feels q v_x B_y = q a B1 / gamma (same sign), the mean field
    Bbar_y is 0, so nu_eff = nu + (0 - q a B1 / gamma) / b."""
    sim = _sim3(4, 4, 2)
    B1, a, b, nu = 0.4, 0.3, -0.2, 0.05
    sim.B[1][...] = (B1 * np.array([1.0, -1.0]))[:, None, None]
    # By sits at (i + 1/2, j, k + 1/2): put the particles exactly there
    _add(sim, [1.0], [1.0], [1.0], [[0], [0], [0]])             # a beam particle (not used)
    _add(sim, [1.5, 1.5], [1.0, 1.0], [0.5, 1.5], [[a, -a], [0, 0], [b, b]], nu=nu)
    m = closure.coarse_moments(sim, 4, 4)
    g = np.sqrt(1 + a * a + b * b)
    q = -1.0
    assert m[9, 0] == pytest.approx(q * a * B1 / g, rel=1e-12)
    assert m[10, 0] == pytest.approx(0.0, abs=1e-15)
    assert m[11, 0] == pytest.approx(nu + (0.0 - q * a * B1 / g) / b, rel=1e-12)


def test_label_from_time_means():
    uz = np.array([0.1, 0.1, 0.0])
    lab = closure.label_from_rows(uz, np.array([0.02, 0.0, 1.0]), np.array([0.0, 0.01, 2.0]), 0.5)
    assert np.allclose(lab, [0.5 - 0.2, 0.5 + 0.1, 0.0])


def test_samples_average_windows_then_form_the_ratio():
    """Windows of 2 snapshots; the label is the ratio of the window means (here 0.1 + (2 - 1) / 0.5
    = 2.1 for window 0, not the mean of the per-snapshot ratios, 2.6); the cell whose mean drift
    is below uz_min is dropped; order is (window, cell)."""
    nc = 3
    rows = np.zeros((5, 12, nc))        # 5 snapshots: 2 windows, the last snapshot unused
    rows[:, 0] = np.arange(5)[:, None] + np.array([0.0, 10.0, 20.0])   # n_b: window means 0.5, 2.5
    rows[0, 3], rows[1, 3] = 0.25, 0.75                                 # uz_p: mean 0.5 in window 0
    rows[2, 3], rows[3, 3] = 1.0, 1.0
    rows[:, 3, 2] = 1e-4                                                # cell 2: drift stopped
    rows[:, 9] = 1.0                                                    # Fz_p
    rows[:, 10] = 2.0                                                   # Fz_mean
    rows[4] = 99.0                                                      # ignored remainder
    f, lab = closure.samples(rows, 2, 0.1, 1e-3)
    assert f.shape == (9, 4) and lab.shape == (4,)
    assert np.allclose(f[0], [0.5, 10.5, 2.5, 12.5])
    assert np.allclose(lab[:2], 0.1 + 1.0 / 0.5)
    assert np.allclose(lab[2:], 0.1 + 1.0 / 1.0)
    per_snapshot = np.mean([0.1 + 1.0 / 0.25, 0.1 + 1.0 / 0.75])
    assert abs(per_snapshot - lab[0]) > 0.4


def test_samples_of_uniform_krook_rows_recover_the_rate():
    """Without field fluctuations (Fz_p = Fz_mean) every kept label is the Krook rate itself."""
    rng = np.random.default_rng(2)
    rows = rng.normal(size=(8, 12, 16))
    rows[:, 3] = -0.1 + 0.01 * rng.normal(size=(8, 16))
    rows[:, 10] = rows[:, 9]
    f, lab = closure.samples(rows, 4, 0.37, 0.05)
    assert lab.shape == (32,) and np.allclose(lab, 0.37)
    assert np.allclose(f[8], rows[:4, 8].mean(0).tolist() + rows[4:, 8].mean(0).tolist())
