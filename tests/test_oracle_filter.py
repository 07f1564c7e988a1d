"""Pins of the oracle's binomial current filter (one 1-2-1 pass per axis, periodic), fixed by
its definition rather than by its code:

  * a Fourier mode is an eigenvector with eigenvalue prod_a cos^2(k_a dx_a / 2) (2D and 3D);
  * the grid-scale (Nyquist) mode is removed, the mean is kept (the total current is conserved);
  * in a step the filter acts on the current the E update uses and nowhere else: after one step
    from the same state, E(filter) - E(no filter) = -dt (F J - J) exactly, J the step's current.
"""
import numpy as np

import oracle
import pic_inputs as pi


def test_fourier_mode_2d():
    nx, ny = 24, 16
    sim = oracle.Simulation(2, nx, ny)
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    for mx, my in ((1, 0), (3, 2), (5, 7), (12, 8)):
        F = np.cos(2 * np.pi * mx * i / nx + 0.3) * np.sin(2 * np.pi * my * j / ny + 0.7)
        want = np.cos(np.pi * mx / nx) ** 2 * np.cos(np.pi * my / ny) ** 2 * F
        assert np.abs(sim.binomial(F).reshape(ny, nx) - want).max() < 1e-14


def test_fourier_mode_3d():
    nx, ny, nz = 8, 6, 10
    sim = oracle.Simulation(3, nx, ny, nz)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    F = np.cos(2 * np.pi * (2 * i / nx + 1 * j / ny + 3 * k / nz))
    want = (np.cos(np.pi * 2 / nx) * np.cos(np.pi * 1 / ny) * np.cos(np.pi * 3 / nz)) ** 2 * F
    assert np.abs(sim.binomial(F).reshape(F.shape) - want).max() < 1e-14


def test_nyquist_removed_and_mean_kept():
    nx, ny = 16, 8
    sim = oracle.Simulation(2, nx, ny)
    alt = ((-1.0) ** np.arange(nx))[None, :] * np.ones((ny, 1))
    assert np.abs(sim.binomial(alt)).max() < 1e-15
    rng = np.random.default_rng(0)
    F = rng.standard_normal((ny, nx))
    assert abs(sim.binomial(F).sum() - F.sum()) < 1e-12


def test_filter_acts_on_the_e_update_current():
    wl = pi.weibel_load(ndim=2, nx=16, ny=16, ppc=4, T_perp_beam=0.1, seed=9)
    on = oracle.Simulation.from_workload(wl, j_filter=1)
    off = oracle.Simulation.from_workload(wl)
    rng = np.random.default_rng(2)
    for a in range(3):
        f = 0.05 * rng.standard_normal((wl.ny, wl.nx))
        b = 0.05 * rng.standard_normal((wl.ny, wl.nx))
        on.E[a][...] = f
        off.E[a][...] = f
        on.B[a][...] = b
        off.B[a][...] = b
    on.step(1)
    off.step(1)
    for a in range(3):
        J = off.J[a]
        FJ = off.binomial(J).reshape(J.shape)
        assert np.abs(on.J[a] - FJ).max() < 1e-15 * max(np.abs(J).max(), 1.0)
        assert np.abs((on.E[a] - off.E[a]) + wl.dt * (FJ - J)).max() < 1e-13
