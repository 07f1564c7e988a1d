"""Growth rates of Eq. (12) on the GPU (pic_dispersion_growth) against the oracle's roots
(oracle.theory.resistive_roots, numpy's companion-matrix eigenvalues) on the same k grid.

The GPU solves each cubic in FP64 by Durand-Kerner iteration and Newton polishing; both sides
then agree to ~1e-12 in the growth rate.  The k of the maximum is compared where the oracle's
maximum is separated from the next grid point's value (otherwise either k is a valid answer).
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


def _oracle_scan(p, ks):
    from oracle import theory
    g = np.array([max(r.imag for r in theory.resistive_roots(k, *p)) for k in ks])
    return g


def test_matches_oracle_roots(pic):
    rng = np.random.default_rng(17)
    n, nk, kmin, kmax = 24, 257, 0.01, 4.0
    params = np.stack([rng.uniform(0.0, 0.3, n), rng.uniform(0.5, 0.99, n),
                       rng.uniform(0.02, 0.3, n), rng.choice([0.0, 0.01, 0.1, 1.0], n)], axis=1)
    g, kst = pic.dispersion_growth(params, kmin, kmax, nk)
    ks = kmin + (kmax - kmin) * np.arange(nk) / (nk - 1)
    for i in range(n):
        go = _oracle_scan(params[i], ks)
        j = int(np.argmax(go))
        assert abs(g[i] - go[j]) <= 1e-10 * max(1.0, abs(go[j])), (i, g[i], go[j])
        others = np.delete(go, j)
        if go[j] - others.max() > 1e-9:
            assert kst[i] == pytest.approx(ks[j], abs=1e-12), i


def test_known_values(pic):
    # the paper's parameters (beta0 = 0.9, nb = 0.1) with c_s^2 = 0.18, nu = 0.15: ~0.0591 at
    # k ~ 0.272; a collisionless warm beam above the Eq. (11) threshold is stable (real roots)
    p = [[0.18, 0.9, 0.1, 0.15], [0.18, 0.9, 0.1, 0.0]]
    g, k = pic.dispersion_growth(p, 0.01, 2.0, 1991)
    assert g[0] == pytest.approx(0.059079, rel=1e-4) and k[0] == pytest.approx(0.2718, abs=2e-3)
    assert abs(g[1]) < 1e-12
