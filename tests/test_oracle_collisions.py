"""Pins of the oracle's binary electron-ion collisions (Takizuka & Abe 1977 with an immobile
partner) and of its counter-based generator, each independent of the code under test:

  * Philox4x32-10 reproduces the known-answer vectors published with the generator
    (Random123: zero counter and key, all-ones, and the pi-digits vector);
  * one collision keeps |u| exactly, along the axis too (u_perp = 0);
  * tan(theta/2) recovered from u . u' is half-normal with variance sigma^2 = nu dt / 2 and the
    azimuth of the kick is uniform;
  * a charge-free drifting ensemble (no fields, no currents) relaxes as <u_z>_n = U E[cos theta]^n,
    with E[cos theta] = E[(1 - delta^2) / (1 + delta^2)] for delta ~ N(0, sigma^2) computed by
    numerical quadrature; for small nu dt that is exp(-nu t) (the Takizuka-Abe small-angle
    variance sigma^2 = nu dt / 2 gives the rate nu to first order in nu dt);
  * nu = 0 leaves a run bit for bit unchanged.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle
import pic_inputs as pi


def test_philox_known_answers():
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert oracle.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert oracle.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_collision_keeps_magnitude():
    rng = np.random.default_rng(3)
    for k in range(200):
        u = rng.normal(0, 2, 3) if k % 10 else np.array([0.0, 0.0, rng.normal(0, 2)])
        r = rng.integers(0, 2 ** 32, 4)
        u1 = oracle.collide_ion(u, 0.3, r)
        assert np.linalg.norm(u1) == pytest.approx(np.linalg.norm(u), rel=1e-14)


def _angles(n, sigma, seed=5):
    rng = np.random.default_rng(seed)
    u = np.array([0.3, -0.4, 1.2])
    t, az = [], []
    e1 = np.cross(u, [0, 0, 1.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u / np.linalg.norm(u), e1)
    for _ in range(n):
        u1 = oracle.collide_ion(u, sigma, rng.integers(0, 2 ** 32, 4))
        c = np.clip(u @ u1 / (u @ u), -1, 1)
        t.append(np.sqrt((1 - c) / (1 + c)))
        d = u1 - u
        az.append(np.arctan2(d @ e2, d @ e1))
    return np.array(t), np.array(az)


def test_scattering_angle_and_azimuth_distribution():
    sigma = 0.2
    t, az = _angles(20000, sigma)
    n = t.size
    # E[delta^2] = sigma^2 with standard error sigma^2 sqrt(2 / n)
    assert abs((t ** 2).mean() - sigma ** 2) < 5 * sigma ** 2 * np.sqrt(2.0 / n)
    # uniform azimuth: mean of cos and sin vanish (standard error 1/sqrt(2n))
    assert abs(np.cos(az).mean()) < 5 / np.sqrt(2 * n)
    assert abs(np.sin(az).mean()) < 5 / np.sqrt(2 * n)


@pytest.mark.parametrize("nu,nsteps,exp_tol", [(2.0, 20, 0.2), (0.4, 50, 0.03)])
def test_drift_relaxes_at_the_collision_rate(nu, nsteps, exp_tol):
    dt, n = 0.05, 40000
    sim = oracle.Simulation(2, 8, 8, dx=0.1, dt=dt)
    rng = np.random.default_rng(9)
    U = 0.5
    sim.add_species(0.0, 1.0, 0.01, 0.0, rng.random(n) * 8, rng.random(n) * 8, None,
                    np.zeros(n), np.zeros(n), np.full(n, U))
    sim.set_collisions(0, nu, seed=12345)
    sim.step(nsteps, record=False)
    sigma = np.sqrt(0.5 * nu * dt)
    f = lambda d: (1 - d * d) / (1 + d * d) * np.exp(-0.5 * (d / sigma) ** 2) / (sigma * np.sqrt(2 * np.pi))
    ecos, _ = integrate.quad(f, -np.inf, np.inf, epsabs=1e-14)
    want = U * ecos ** nsteps
    got = sim.species[0].uz.mean()
    se = U / np.sqrt(n)                                   # |u_z| <= U: a generous standard error
    assert abs(got - want) < 5 * se, (got, want)
    assert want == pytest.approx(U * np.exp(-nu * dt * nsteps), rel=exp_tol)
    assert np.allclose(np.linalg.norm(sim.species[0].u, axis=0), U, rtol=1e-13)


def test_zero_rate_is_identity():
    wl = pi.weibel_load(ndim=2, nx=16, ny=16, ppc=4, T_perp_beam=0.1, T_bg=0.01, seed=3)
    a = oracle.Simulation.from_workload(wl)
    b = oracle.Simulation.from_workload(wl)
    b.set_collisions(1, 0.0, seed=1)
    a.step(5)
    b.step(5)
    for sa, sb in zip(a.species, b.species):
        assert np.array_equal(sa.u, sb.u)
