"""Pins of the closure-driven drag in the oracle (per-cell Krook rates replacing the scalar):

  * a constant map reproduces the scalar-rate run bit for bit;
  * one step in zero fields is the closed form u1 = u0 - (1 - exp(-nu_c dt)) <u0>_c per cell
    (Boris does nothing without fields; the first step's deposit only changes the fields after
    the push);
  * negative rates act as 0.
"""
import numpy as np

import oracle
import pic_inputs as pi


def _wl(seed=3):
    return pi.weibel_load(ndim=2, nx=16, ny=16, ppc=8, T_perp_beam=0.1, T_bg=0.01, nu=0.2, seed=seed)


def test_constant_map_equals_scalar_rate():
    wl = _wl()
    a = oracle.Simulation.from_workload(wl)
    b = oracle.Simulation.from_workload(wl)
    b.set_nu_cell(1, np.full(wl.ncell, 0.2))
    a.step(10)
    b.step(10)
    for sa, sb in zip(a.species, b.species):
        assert np.array_equal(sa.u, sb.u) and np.array_equal(sa.X, sb.X)
    for k in range(3):
        assert np.array_equal(a.E[k], b.E[k])


def test_one_step_closed_form_per_cell():
    wl = _wl(5)
    sim = oracle.Simulation.from_workload(wl)
    rng = np.random.default_rng(1)
    rates = rng.uniform(0, 2.0, wl.ncell)
    rates[::7] = -0.5                                    # acts as 0
    sim.set_nu_cell(1, rates)
    bg = sim.species[1]
    u0 = bg.u.copy()
    cell = (np.floor(bg.Y).astype(int) % wl.ny) * wl.nx + (np.floor(bg.X).astype(int) % wl.nx)
    cnt = np.bincount(cell, minlength=wl.ncell)
    mean = np.stack([np.bincount(cell, u0[a], minlength=wl.ncell) / np.maximum(cnt, 1) for a in range(3)])
    f = np.where(rates > 0, 1 - np.exp(-rates * wl.dt), 0.0)
    sim.step(1, record=False)
    want = u0 - f[cell] * mean[:, cell]
    assert np.allclose(bg.u, want, rtol=0, atol=1e-15)
    # the beam (no drag) is untouched in zero fields
    assert np.array_equal(sim.species[0].u, pi_u(wl, 0))


def pi_u(wl, s):
    return wl.species[s].u.astype(np.float64)
