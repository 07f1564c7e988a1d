"""Closed forms used to pin the oracle -- TEST INFRASTRUCTURE ONLY.

cold_growth_rate   cold relativistic two-fluid filamentation (Weibel) growth rate for k
                   transverse to the drift.  The paper's Eq. (12) is non-relativistic and
                   quasi-neutral; an EM PIC run of a gamma = 3 beam is pinned instead by the
                   cold-fluid relation derived here (our reading): linearise the cold momentum,
                   continuity, Faraday and Ampere equations for species s of density n_s and
                   drift v_s along z, perturbation exp(i k x - i w t), fields (E_x, E_z, B_y).
                   With x = w^2, A = sum n/g, B = sum n/g^3, C = sum n v^2/g, D = sum n v/g:
                       (x - A)(x^2 - (k^2 + B) x - k^2 C) - k^2 D^2 = 0,
                   and the growth rate is sqrt(-x) for the negative real root.
warm_threshold     Eq. (11): modified sound speed cbar_s^2 = c_s^2 - beta0^2 nb/n0.
resistive_roots    Eq. (12): w^2 = c_s^2 k^2 - w_b^2 beta0^2 k^2 / (k^2 + k_pe^2/(1 + i nu/w)),
                   written as a cubic in w (k_pe = 1 in units of w_p/c, w_b^2 = nb).
resistive_growth_small_nu  Eq. (14): w ~ i nu beta0^2 nb / (cbar_s^2 n0).
"""
from __future__ import annotations

import numpy as np


def fluid_moments(species):
    """species: iterable of (n, v) with v the drift speed along z (units c)."""
    A = B = C = D = 0.0
    for n, v in species:
        g = 1.0 / np.sqrt(1.0 - v * v)
        A += n / g
        B += n / g ** 3
        C += n * v * v / g
        D += n * v / g
    return A, B, C, D


def cold_dispersion_coeffs(k, species):
    """Coefficients (highest power first) of the cubic in x = w^2."""
    A, B, C, D = fluid_moments(species)
    k2 = k * k
    # (x - A)(x^2 - (k2 + B) x - k2 C) - k2 D^2
    return np.array([1.0, -(k2 + B) - A, -k2 * C + A * (k2 + B), A * k2 * C - k2 * D * D])


def cold_growth_rate(k, species):
    """Largest growth rate sqrt(-x) over the negative real roots x = w^2 (0 if none)."""
    r = np.roots(cold_dispersion_coeffs(k, species))
    neg = [z.real for z in r if abs(z.imag) < 1e-12 * max(1.0, abs(z)) and z.real < 0]
    return float(np.sqrt(-min(neg))) if neg else 0.0


def cold_growth_rate_kinf(species):
    """k -> infinity limit: (x - A)(x + C) + D^2 = 0, negative root."""
    A, B, C, D = fluid_moments(species)
    disc = (A - C) ** 2 + 4.0 * (A * C - D * D)
    x = 0.5 * ((A - C) - np.sqrt(disc))
    return float(np.sqrt(-x))


def weibel_species(gamma_b=3.0, nb=0.1):
    """Beam (nb, +v_b) and background (1 - nb, v_p) with nb v_b + np v_p = 0."""
    vb = np.sqrt(1.0 - 1.0 / gamma_b ** 2)
    npl = 1.0 - nb
    return [(nb, vb), (npl, -nb * vb / npl)]


def warm_threshold(cs2, beta0, nb, n0=1.0):
    """Eq. (11): cbar_s^2; the beam is Weibel-unstable (collisionless) iff it is < 0."""
    return cs2 - beta0 * beta0 * nb / n0


def resistive_roots(k, cs2, beta0, nb, nu):
    """Roots w of Eq. (12) with k_pe = 1 and w_b^2 = nb, as the cubic
    (k^2+1) w^3 + i k^2 nu w^2 + (b - a (k^2+1)) w + i nu (b - a k^2) = 0,
    a = cs2 k^2, b = nb beta0^2 k^2."""
    k2 = k * k
    a = cs2 * k2
    b = nb * beta0 * beta0 * k2
    coeffs = [k2 + 1.0, 1j * k2 * nu, b - a * (k2 + 1.0), 1j * nu * (b - a * k2)]
    return np.roots(coeffs)


def resistive_growth_small_nu(cs2, beta0, nb, nu, n0=1.0):
    """Eq. (14): the purely growing root i nu beta0^2 nb / (cbar_s^2 n0)."""
    return nu * beta0 * beta0 * nb / (warm_threshold(cs2, beta0, nb, n0) * n0)
