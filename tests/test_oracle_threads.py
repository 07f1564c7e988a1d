"""The all-core build of the oracle (OpenMP particle loop, per-thread current and moment arrays)
against the single-threaded build the other tests pin: the same per-particle arithmetic with
sums in another order, so the two agree to FP64 round-off after many steps.  The all-core build
only times the oracle on every host core (the benchmark's CPU baseline)."""
import numpy as np

import oracle
import pic_inputs as pi


def _compare(wl, steps):
    a = oracle.Simulation.from_workload(wl)
    b = oracle.Simulation.from_workload(wl, threads=True)
    a.step(steps)
    b.step(steps)
    for sa, sb in zip(a.species, b.species):
        assert np.abs(sa.u - sb.u).max() <= 1e-12 * max(1.0, np.abs(sa.u).max())
        assert np.abs(sa.X - sb.X).max() <= 1e-10
    for c in range(3):
        scale = max(np.abs(a.E[c]).max(), 1e-30)
        assert np.abs(a.E[c] - b.E[c]).max() <= 1e-11 * scale
    for ha, hb in zip(a.history, b.history):
        assert np.allclose(ha["Ekin"], hb["Ekin"], rtol=1e-12, atol=0)
        assert np.allclose(ha["WB"], hb["WB"], rtol=1e-10, atol=1e-300)


def test_threads_match_serial_2d_krook():
    wl = pi.weibel_load(ndim=2, nx=32, ny=32, ppc=8, T_perp_beam=0.1, T_bg=0.001, nu=0.1, seed=3)
    _compare(wl, 30)


def test_threads_match_serial_3d():
    wl = pi.weibel_load(ndim=3, nx=8, ny=8, nz=16, ppc=4, T_perp_beam=0.2, T_bg=0.0, nu=0.0, seed=4)
    _compare(wl, 10)
