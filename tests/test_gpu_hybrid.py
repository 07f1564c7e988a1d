"""The hybrid model on the GPU (pic_hybrid_*) against the FP64 oracle (oracle.hybrid).

The GPU keeps particles in FP32 and solves the field correction in FP32, so parity is at FP32
level.  Tolerances: one push is about ten FP32 operations per quantity (relative rounding
~1e-6 after a step); the correction solve stops at a relative residual of 1e-5 of the
step's initial residual; ten steps of a warm beam in fields of a few 1e-3 compound these to a
few 1e-5 -- the tests allow 2e-4 (relative to the largest value of each array) and 1e-4 cell.
  * a quiet, current-neutral cold beam is a steady state (no transverse momentum at all, a and
    beta_p spatially uniform);
  * one collisional step from that state: a = nu dt beta_p0 (Ohm's law closed form);
  * ten steps of a warm beam on a non-square grid with a ragged particle count: a, beta_p,
    positions, momenta and the three energies against the oracle;
  * a seeded single mode grows at the model's linear rate within 2%;
  * Eq. 7: the collisionless total energy drift stays below 1% of the peak magnetic energy and
    falls with dt, as in the oracle;
  * bitwise reproducibility, independence of the periodic sort, graph = direct launches,
    solver convergence, and argument errors;
  * edge cases: no beam at all (the plasma current switches off in one step, closed form) and
    the largest grid sides (2048 x 16 and 16 x 2048 nodes) against the oracle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _lattice(nx, ny, m):
    sub = (np.arange(m) + 0.5) / m
    gx, gy = np.meshgrid(sub, sub, indexing="xy")
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    X = (cx[..., None, None] + gx[None, None]).reshape(-1)
    Y = (cy[..., None, None] + gy[None, None]).reshape(-1)
    return X, Y


G0 = 3.0
U0 = np.sqrt(G0 ** 2 - 1)
B0 = U0 / G0
BP0 = -0.1 * B0 / 0.9


def _pair(pic, nx, ny, dx, dt, nu, w, X, Y, ux, uy, uz, bp, **kw):
    from oracle import hybrid
    eng = pic.HybridEngine(nx, ny, dx, dx, dt, 1.0, nu, w, X.shape[0], **kw)
    eng.load(X, Y, ux, uy, uz, bp)
    sim = hybrid.HybridSim(nx, ny, dx, dx, dt, n0=1.0, nu=nu, w=w)
    sim.load(X, Y, ux, uy, uz, bp)
    return eng, sim


def test_steady_state(pic):
    X, Y = _lattice(16, 16, 4)
    n = X.shape[0]
    eng = pic.HybridEngine(16, 16, 0.1, 0.1, 0.05, 1.0, 0.0, 0.1 / 16, n)
    eng.load(X, Y, np.zeros(n), np.zeros(n), np.full(n, U0), BP0)
    eng.step(20)
    st = eng.state()
    assert np.all(st["ux"] == 0) and np.all(st["uy"] == 0)
    assert np.ptp(st["a"]) < 1e-12 and abs(st["a"]).max() < 1e-6
    assert np.ptp(st["beta_p"]) < 1e-12
    assert eng.stats()["unconverged_steps"] == 0
    eng.close()


def test_resistive_step(pic):
    nu, dt = 0.3, 0.05
    X, Y = _lattice(16, 16, 4)
    n = X.shape[0]
    eng = pic.HybridEngine(16, 16, 0.1, 0.1, dt, 1.0, nu, 0.1 / 16, n)
    eng.load(X, Y, np.zeros(n), np.zeros(n), np.full(n, U0), BP0)
    eng.step(1)
    st = eng.state()
    assert np.allclose(st["a"], nu * dt * BP0, rtol=1e-4, atol=0)
    assert np.allclose(st["beta_p"], BP0, rtol=1e-5, atol=0)
    eng.close()


def _warm(nx, ny, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, nx, n)
    Y = rng.uniform(0, ny, n)
    ux = 0.05 * rng.standard_normal(n)
    uy = 0.05 * rng.standard_normal(n)
    uz = U0 + 0.05 * rng.standard_normal(n)
    return X, Y, ux, uy, uz


def _rel(g, o):
    return np.abs(g - o).max() / max(np.abs(o).max(), 1e-30)


def test_parity_warm_beam(pic):
    nx, ny, n = 32, 16, 32 * 16 * 8 + 37
    X, Y, ux, uy, uz = _warm(nx, ny, n, 4)
    w = 0.1 * nx * ny / n
    eng, sim = _pair(pic, nx, ny, 0.2, 0.05, 0.05, w, X, Y, ux, uy, uz, BP0)
    assert np.allclose(eng.energies(), sim.energies(), rtol=1e-6)
    eng.step(10)
    sim.step(10)
    st = eng.state()
    assert abs(sim.a).max() > 1e-4                 # the fields are not trivial
    assert _rel(st["a"], sim.a) < 2e-4
    assert _rel(st["beta_p"], sim.beta_p) < 2e-4
    dX = (st["X"] - sim.X + nx / 2) % nx - nx / 2
    dY = (st["Y"] - sim.Y + ny / 2) % ny - ny / 2
    assert np.abs(dX).max() < 1e-4 and np.abs(dY).max() < 1e-4
    assert _rel(st["ux"], sim.ux) < 2e-4 and _rel(st["uy"], sim.uy) < 2e-4
    e_g, e_o = eng.energies(), sim.energies()
    assert abs(e_g[0] / e_o[0] - 1) < 1e-3        # magnetic energy is quadratic in a
    assert abs(e_g[1] / e_o[1] - 1) < 1e-5 and abs(e_g[2] / e_o[2] - 1) < 1e-4
    s = eng.stats()
    assert s["steps"] == 10 and s["unconverged_steps"] == 0 and 0 < s["cg_iterations"] <= 10 * 16
    eng.close()


def test_bitwise_reproducible(pic):
    nx, ny, n = 32, 32, 32 * 32 * 4
    X, Y, ux, uy, uz = _warm(nx, ny, n, 8)
    out = []
    for _ in range(2):
        eng = pic.HybridEngine(nx, ny, 0.2, 0.2, 0.05, 1.0, 0.02, 0.1 / 4, n)
        eng.load(X, Y, ux, uy, uz, BP0)
        eng.step(5)
        out.append(eng.state())
        eng.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


def test_sort_does_not_change_results(pic):
    """Deposits are exact integer sums, so sorting the beam by cell every step and never
    sorting (after the load) give bitwise the same state, in the load order."""
    nx, ny, n = 32, 16, 32 * 16 * 8 + 11
    X, Y, ux, uy, uz = _warm(nx, ny, n, 12)
    out = []
    for si in (1, 1000000):
        eng = pic.HybridEngine(nx, ny, 0.2, 0.2, 0.05, 1.0, 0.05, 0.1 / 8, n, sort_interval=si)
        eng.load(X, Y, ux, uy, uz, BP0)
        eng.step(12)
        out.append((eng.state(), eng.energies()))
        eng.close()
    for k in out[0][0]:
        assert np.array_equal(out[0][0][k], out[1][0][k]), k
    assert np.array_equal(out[0][1], out[1][1])


def test_graph_matches_direct_launches(pic):
    """The graph's while node runs only the iterations the solve needs; direct launches run
    max_iter iterations whose kernels return at once after convergence: same arithmetic."""
    nx, ny, n = 64, 32, 64 * 32 * 4 + 5
    X, Y, ux, uy, uz = _warm(nx, ny, n, 9)
    out, launches = [], []
    for flags in (0, pic.PIC_FLAG_NO_GRAPH):
        eng = pic.HybridEngine(nx, ny, 0.2, 0.2, 0.05, 1.0, 0.1, 0.1 / 4, n, flags=flags)
        eng.load(X, Y, ux, uy, uz, BP0)
        eng.step(6)
        out.append(eng.state())
        s = eng.stats()
        launches.append(eng.launch_count())
        iters = s["cg_iterations"]
        eng.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
    assert launches[1] == 6 * (3 + 4 * 16)
    assert launches[0] == 6 * 3 + 5 * iters and launches[0] < launches[1]


def test_growth_rate(pic):
    from oracle import hybrid
    nx, ny, m, dx, dt = 64, 8, 4, 0.1, 0.05
    X, Y = _lattice(nx, ny, m)
    n = X.shape[0]
    X = X + 1e-4 * np.sin(2 * np.pi * X / nx)
    eng = pic.HybridEngine(nx, ny, dx, dx, dt, 1.0, 0.0, 0.1 / (m * m), n)
    eng.load(X, Y, np.zeros(n), np.zeros(n), np.full(n, U0), BP0)
    amp, t = [], []
    for k in range(1000):
        eng.step(1)
        if k % 10 == 9:
            a = eng.state()["a"]
            amp.append(abs(np.fft.rfft(a.mean(axis=0))[1]))
            t.append((k + 1) * dt)
    amp, t = np.array(amp), np.array(t)
    sel = t >= 20.0
    assert amp[-1] < 1e-2
    g = np.polyfit(t[sel], np.log(amp[sel]), 1)[0]
    k = 2 * np.pi / (nx * dx)
    want = hybrid.linear_growth_rate((2 / dx) * np.sin(k * dx / 2), B0, G0, 0.1)
    assert abs(g / want - 1) < 0.02, (g, want)
    eng.close()


def _drift(pic, dt, nx=16, dx=0.25, T=40.0, m=2):
    X, Y = _lattice(nx, nx, m)
    n = X.shape[0]
    rng = np.random.default_rng(1)
    eng = pic.HybridEngine(nx, nx, dx, dx, dt, 1.0, 0.0, 0.1 / (m * m), n)
    eng.load((X + 0.05 * rng.standard_normal(n)) % nx, (Y + 0.05 * rng.standard_normal(n)) % nx,
             np.zeros(n), np.zeros(n), np.full(n, U0), BP0)
    E0 = eng.energies().sum()
    drift, emag = 0.0, 0.0
    for _ in range(int(round(T / dt))):
        eng.step(1)
        e = eng.energies()
        drift = max(drift, abs(e.sum() - E0))
        emag = max(emag, e[0])
    eng.close()
    return drift, emag


def test_eq7_energy_conservation(pic):
    d1, m1 = _drift(pic, 0.1)
    d2, m2 = _drift(pic, 0.05)
    assert m2 > 1e-2
    assert d2 < 0.01 * m2, (d2, m2)
    assert d1 / d2 > 1.5, (d1, d2)


def test_empty_beam(pic):
    nu, dt, bp0 = 0.3, 0.05, -0.04
    eng = pic.HybridEngine(16, 8, 0.1, 0.1, dt, 1.0, nu, 0.0, 0)
    eng.load(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), bp0)
    eng.step(3)
    st = eng.state()
    assert np.allclose(st["a"], -bp0 * (1 - nu * dt), rtol=1e-6, atol=0)
    assert np.abs(st["beta_p"]).max() < 1e-9
    assert eng.stats()["unconverged_steps"] == 0
    eng.close()


@pytest.mark.parametrize("nx,ny", [(2048, 16), (16, 2048)])
def test_largest_grid_sides(pic, nx, ny):
    from oracle import hybrid
    n = nx * ny * 2 + 3
    X, Y, ux, uy, uz = _warm(nx, ny, n, 13)
    w = 0.1 * nx * ny / n
    eng, sim = _pair(pic, nx, ny, 0.2, 0.05, 0.05, w, X, Y, ux, uy, uz, BP0)
    eng.step(3)
    sim.step(3)
    st = eng.state()
    assert _rel(st["a"], sim.a) < 2e-4 and _rel(st["beta_p"], sim.beta_p) < 2e-4
    assert np.abs((st["X"] - sim.X + nx / 2) % nx - nx / 2).max() < 1e-4
    assert np.abs((st["Y"] - sim.Y + ny / 2) % ny - ny / 2).max() < 1e-4
    eng.close()


def test_argument_errors(pic):
    with pytest.raises(Exception):
        pic.HybridEngine(24, 16, 0.1, 0.1, 0.05, 1.0, 0.0, 0.01, 10)     # not a power of two
    with pytest.raises(Exception):
        pic.HybridEngine(16, 16, 0.1, 0.1, 0.2, 1.0, 0.0, 0.01, 10)      # dt >= dx
    eng = pic.HybridEngine(16, 16, 0.1, 0.1, 0.05, 1.0, 0.0, 0.01, 4)
    with pytest.raises(Exception):
        eng.load(np.array([1.0, 2.0, 16.5, 3.0]), np.ones(4), np.zeros(4), np.zeros(4), np.ones(4), 0.0)
    with pytest.raises(Exception):
        eng.load(np.ones(5), np.ones(5), np.zeros(5), np.zeros(5), np.ones(5), 0.0)   # above capacity
    eng.close()
