"""The seeded load recipe (pic_inputs), shared by the CUDA path and the oracle: exactly ppc
particles per cell and species, in-cell offsets in [0, 1), FP32 values, the beam drift
u_z = sqrt(gamma_b^2 - 1), temperatures within sampling error, zero sampled net current along z
(the paper's current-neutral start), the same arrays for the same seed, and the scan table's
grid sizes and collision rates."""
import math

import numpy as np
import pytest

import pic_inputs as pi


@pytest.mark.parametrize("ndim", [2, 3])
def test_weibel_load_recipe(ndim):
    kw = dict(nx=16, ny=16, nz=8) if ndim == 3 else dict(nx=32, ny=32)
    wl = pi.weibel_load(ndim=ndim, ppc=16, gamma_b=3.0, nb=0.1, T_perp_beam=0.1, T_bg=0.001,
                        nu=0.1, seed=11, **kw)
    beam, bg = wl.species
    assert (beam.q, bg.q) == (-1.0, -1.0) and bg.nu == 0.1 and beam.nu == 0.0
    assert beam.w == pytest.approx(0.1 / 16) and bg.w == pytest.approx(0.9 / 16)
    for s in (beam, bg):
        assert s.cell.dtype == np.int32 and s.offset.dtype == np.float32 and s.u.dtype == np.float32
        assert np.array_equal(np.bincount(s.cell, minlength=wl.ncell), np.full(wl.ncell, 16))
        assert s.offset.shape == (ndim, s.n) and s.offset.min() >= 0.0 and s.offset.max() < 1.0
    n = beam.n
    assert np.all(beam.u[2] == np.float32(math.sqrt(8.0)))                  # cold along z
    ub = beam.u.astype(np.float64)
    for a in (0, 1):                                                       # T_perp = 0.1
        assert abs(ub[a].mean()) < 1e-6
        assert ub[a].var() == pytest.approx(0.1, rel=4 * math.sqrt(2 / n))
    up = bg.u.astype(np.float64)
    for a in (0, 1):
        assert up[a].var() == pytest.approx(0.001, rel=4 * math.sqrt(2 / n))
    # zero net current: sum_p w v_z over both species, against the beam's own current
    vz = lambda s: (s.u[2].astype(np.float64) / np.sqrt(1 + (s.u.astype(np.float64) ** 2).sum(0)))
    jb = beam.w * vz(beam).sum()
    jp = bg.w * vz(bg).sum()
    assert abs(jb + jp) < 1e-6 * abs(jb)


def test_cold_return_current_drift():
    """Cold beam and background: every background particle drifts at the return-current velocity
    beta_p = -(nb / np) beta_b = -0.104757 (gamma_p = 1.005533), beta_b = sqrt(8) / 3."""
    wl = pi.weibel_load(ndim=2, nx=16, ny=16, ppc=4, gamma_b=3.0, nb=0.1, seed=2)
    bg = wl.species[1]
    assert np.all(bg.u[2] == bg.u[2][0]) and np.all(bg.u[:2] == 0)
    uz = float(bg.u[2][0])
    beta_p = uz / math.sqrt(1 + uz * uz)
    assert beta_p == pytest.approx(-(0.1 / 0.9) * math.sqrt(8.0) / 3.0, rel=1e-6)
    assert math.sqrt(1 + uz * uz) == pytest.approx(1.005533, abs=1e-6)


def test_loads_are_seeded():
    a = pi.weibel_load(ndim=2, nx=16, ny=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, seed=5)
    b = pi.weibel_load(ndim=2, nx=16, ny=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, seed=5)
    c = pi.weibel_load(ndim=2, nx=16, ny=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, seed=6)
    for sa, sb, sc in zip(a.species, b.species, c.species):
        assert np.array_equal(sa.offset, sb.offset) and np.array_equal(sa.u, sb.u)
        assert not np.array_equal(sa.offset, sc.offset)


def test_lattice_load_is_quiet():
    wl = pi.weibel_load(ndim=2, nx=8, ny=8, ppc=4, lattice=True, seed=1)
    for s in wl.species:
        pat = s.offset[:, :4]
        assert np.array_equal(np.sort(pat[0]), np.float32([0.25, 0.25, 0.75, 0.75]))
        assert np.array_equal(s.offset, np.tile(pat, (1, 64)))


def test_hybrid_load_is_current_neutral():
    L = pi.hybrid_beam_load(nx=32, ny=16, ppc=8, gamma_b=3.0, nb=0.1, T_perp_beam=0.1, seed=6)
    assert L.n == 32 * 16 * 8 and L.w == pytest.approx(0.1 / 8)
    assert L.X.min() >= 0 and L.X.max() < 32 and L.Y.min() >= 0 and L.Y.max() < 16
    bz = L.uz / np.sqrt(1 + L.ux ** 2 + L.uy ** 2 + L.uz ** 2)
    assert 0.1 * bz.mean() + 0.9 * L.beta_p0 == pytest.approx(0.0, abs=1e-12)


def test_scan_table():
    t = pi.scan_table(256)
    assert len(t) == 256 and t == pi.scan_table(256)
    nx, ny, T, nu = map(np.array, zip(*t))
    assert set(nx) <= set(pi.SCAN_SIZES) and set(ny) <= set(pi.SCAN_SIZES)
    assert set(nu) <= set(pi.SCAN_NU) and len(set(nu)) == len(pi.SCAN_NU)
    assert T.min() >= 0 and T.max() < 1
    assert 2 * 32 * np.sum(nx * ny) == 1470103552          # particles of the 256-run benchmark
