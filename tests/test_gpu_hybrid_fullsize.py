"""The hybrid model at the benchmark's full size (1024 x 1024 nodes, 16 beam particles per cell,
16,777,216 particles, collisional plasma flow nu = 0.1), graph-replayed steps as in the
benchmark.  The oracle cannot step this size, but it can check each part of a GPU step:

  * sampled parity: 4096 particles pushed by the oracle in the GPU's fields of step 1 land where
    the GPU's step 2 put them (1e-5 cell, momenta 1e-5 of the largest transverse momentum);
  * the field solve: with the oracle's FP64 deposit of the GPU's step-2 particles, the GPU's
    a^2 satisfies (lap - n_p) a^2 = rhs to 1e-4 of the initial residual (the FP32 correction
    solve stops at 1e-5; FP32 positions and currents add a few 1e-6);
  * the plasma-flow update beta_p^2 = beta_p^1 + a^2 - a^1 - nu dt beta_p^1 holds to rounding;
  * the three energies equal the oracle's formulas on the GPU's state.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, PPC = 1024, 16


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def test_hybrid_fullsize_two_steps(pic):
    import pic_inputs as pi
    from oracle import hybrid
    L = pi.hybrid_beam_load(nx=N, ny=N, ppc=PPC, seed=6)
    eng = pic.HybridEngine(N, N, L.dx, L.dx, L.dt, 1.0, L.nu, L.w, L.n)
    eng.load(L.X, L.Y, L.ux, L.uy, L.uz, L.beta_p0)
    eng.step(1)
    s1 = eng.state()
    eng.step(1)
    s2 = eng.state()
    e_gpu = eng.energies()
    st = eng.stats()
    eng.close()
    assert st["unconverged_steps"] == 0

    sim = hybrid.HybridSim(N, N, L.dx, L.dx, L.dt, n0=1.0, nu=L.nu, w=L.w)
    sim.load(L.X[:1], L.Y[:1], L.ux[:1], L.uy[:1], L.uz[:1], L.beta_p0)
    sim.a = s1["a"].copy()
    sim.beta_p = s1["beta_p"].copy()

    # -- sampled particle parity
    rng = np.random.default_rng(7)
    idx = rng.choice(L.n, 4096, replace=False)
    P = L.uz[idx]                                   # a = 0 at load
    Xo, Yo, uxo, uyo = sim.push(s1["X"][idx], s1["Y"][idx], s1["ux"][idx], s1["uy"][idx], P)
    dX = (s2["X"][idx] - Xo + N / 2) % N - N / 2
    dY = (s2["Y"][idx] - Yo + N / 2) % N - N / 2
    assert np.abs(dX).max() < 1e-5 and np.abs(dY).max() < 1e-5
    umax = max(np.abs(uxo).max(), np.abs(uyo).max())
    assert np.abs(s2["ux"][idx] - uxo).max() < 1e-5 * umax
    assert np.abs(s2["uy"][idx] - uyo).max() < 1e-5 * umax

    # -- the field solve of step 2 with the oracle's deposit of the GPU's particles
    X2, Y2 = s2["X"], s2["Y"]
    uzs = L.uz + sim._interp(s1["a"], X2, Y2)
    gs = np.sqrt(1.0 + s2["ux"] ** 2 + s2["uy"] ** 2 + uzs ** 2)
    jb = sim._deposit(X2, Y2, L.w * uzs / gs)
    sim.X, sim.Y = X2, Y2
    n_p = sim.plasma_density()
    a1, b1 = s1["a"], s1["beta_p"]
    rhs = jb + n_p * (b1 - a1 - L.nu * L.dt * b1)
    A = hybrid.laplacian_matrix(N, N, L.dx, L.dx)
    op = lambda a: (A @ a.reshape(-1)).reshape(N, N) - n_p * a
    r_init = np.linalg.norm(rhs - op(a1))
    r_fin = np.linalg.norm(rhs - op(s2["a"]))
    assert r_init > 0 and r_fin <= 1e-4 * r_init, (r_fin, r_init)

    # -- plasma-flow update
    want = b1 + (s2["a"] - a1) - L.nu * L.dt * b1
    assert np.allclose(s2["beta_p"], want, rtol=1e-12, atol=1e-15)

    # -- energies of the GPU state by the oracle's formulas
    sim.a, sim.beta_p = s2["a"], s2["beta_p"]
    sim.P = L.uz
    sim.ux, sim.uy = s2["ux"], s2["uy"]
    e_orc = sim.energies()
    assert abs(e_gpu[1] / e_orc[1] - 1) < 1e-6 and abs(e_gpu[2] / e_orc[2] - 1) < 1e-6
    assert abs(e_gpu[0] / e_orc[0] - 1) < 1e-9
