"""The paper's four simulation cases on the oracle.  Cases (a) and (b): a cold beam filaments
with and without collisions of the background (W_B grows by more than 30x in a 24^2 box within
t = 25; measured ~200x, ~200x with the Krook reading, ~700x with binary collisions).

Cases (c) and (d): a hot beam (T_perp ~ 70 keV = 0.137 m c^2,
v_b = 0.9 c, n_p / n_b = 9) in a collisionless background shows no filamentation growth, and the
same beam in a collisional background grows again (the simulation section: collisions of the
return-current electrons revive the instability).  Collision rate nu = 0.15 w_p as in the paper.

The collisional (resistive) growth lives at long wavelengths, k below about k_pe = w_p / c
(Eq. 12 puts its maximum, 0.073 w_p for these parameters, at k ~ 0.31 c / w_p; Eq. 12 is
non-relativistic, so only the qualitative statement is pinned).  The box is therefore 20 skin
depths long along x, as in the paper, and thin along y to keep the CPU cost low.

Checked, with W_B the transverse magnetic energy relative to its level at t ~ 2:
  * PIC oracle without collisions: max W_B over t <= 75 stays below 10 (measured ~3);
  * PIC oracle with the Krook reading of Eq. 3 on the background: above 30 (measured ~68);
  * PIC oracle with binary electron-ion collisions of the background: above 30 (measured ~160);
  * hybrid model (Eqs. 1-6) without / with nu: below 20 / above 60 (measured ~13 / ~240).
"""
import math

import numpy as np
import pytest

import pic_inputs as pi

GB = 1 / math.sqrt(1 - 0.81)
NX, NY, PPC, T_END, NU = 200, 8, 8, 75.0, 0.15


def _growth(t, W):
    w0 = W[(t > 1.5) & (t <= 2.5)].mean()
    return W[t <= T_END].max() / w0


def _pic(oracle_lib, kind):
    wl = pi.weibel_load(ndim=2, nx=NX, ny=NY, ppc=PPC, gamma_b=GB, T_perp_beam=0.137, seed=9,
                        nu=NU if kind == "krook" else 0.0)
    sim = oracle_lib.Simulation.from_workload(wl)
    if kind == "binary":
        sim.set_collisions(1, NU, 12345)
    sim.step(int(round(T_END / wl.dt)))
    WB = sim.history_array("WB")
    return _growth(sim.history_array("t"), WB[:, 0] + WB[:, 1])


def _hybrid(nu):
    from oracle import hybrid
    L = pi.hybrid_beam_load(nx=NX, ny=NY, ppc=PPC, gamma_b=GB, T_perp_beam=0.137, nu=nu, seed=6)
    sim = hybrid.HybridSim(NX, NY, L.dx, L.dx, L.dt, n0=1.0, nu=nu, w=L.w)
    sim.load(L.X, L.Y, L.ux, L.uy, L.uz, L.beta_p0)
    W, t = [], []
    for n in range(int(round(T_END / L.dt)) // 10):
        sim.step(10)
        W.append(sim.energies()[0])
        t.append((n + 1) * 10 * L.dt)
    return _growth(np.array(t), np.array(W))


@pytest.mark.slow
def test_collisions_revive_the_hot_beam_instability(oracle_lib):
    g = {k: _pic(oracle_lib, k) for k in ("none", "krook", "binary")}
    assert g["none"] < 10.0, g
    assert g["krook"] > 30.0, g
    assert g["binary"] > 30.0, g


@pytest.mark.slow
def test_hybrid_model_collisions_revive_the_instability():
    g0, g1 = _hybrid(0.0), _hybrid(NU)
    assert g0 < 20.0, (g0, g1)
    assert g1 > 60.0, (g0, g1)


@pytest.mark.parametrize("kind", ["none", "krook", "binary"])
def test_cold_beam_filaments_with_and_without_collisions(oracle_lib, kind):
    wl = pi.weibel_load(ndim=2, nx=24, ny=24, ppc=16, gamma_b=GB, T_perp_beam=0.0, seed=9,
                        nu=NU if kind == "krook" else 0.0)
    sim = oracle_lib.Simulation.from_workload(wl)
    if kind == "binary":
        sim.set_collisions(1, NU, 12345)
    sim.step(500)
    WB = sim.history_array("WB")
    W, t = WB[:, 0] + WB[:, 1], sim.history_array("t")
    assert W[-50:].mean() / W[(t > 0.5) & (t <= 2.5)].mean() > 30.0
