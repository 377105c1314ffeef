"""Pins of the grid selection term (VT on a regular grid, Sec. "Population
acceleration"): the oracle's grid sum against numpy's trapezoid of scipy's
densities on the same nodes, and against the Monte Carlo selection term of
the synthetic campaign (whose detection probability is sigmoid((m1 - 20)/5))."""
import numpy as np
import pytest
from scipy import integrate, special, stats

from paper_1904_02863_gb300 import synth


def campaign_pdet(m1, q):
    return np.broadcast_to(special.expit((m1[:, None] - 20.0) / 5.0), (m1.size, q.size)).copy()


def ref_density_grid(m1, q, L):
    alpha, beta, mmin, mmax, lam, mu, sig = L[:7]
    pl = stats.truncpareto(alpha - 1.0, mmax / mmin, scale=mmin).pdf(m1)
    tn = stats.truncnorm((mmin - mu) / sig, (mmax - mu) / sig, loc=mu, scale=sig).pdf(m1)
    pm = np.where((m1 > mmin) & (m1 <= mmax), (1 - lam) * pl + lam * tn, 0.0)
    out = np.zeros((m1.size, q.size))
    for a, m in enumerate(m1):
        if pm[a] == 0.0:
            continue
        norm, _ = integrate.quad(lambda x: x ** beta, mmin / m, 1.0, epsabs=0, epsrel=1e-13)
        inside = (q * m >= mmin) & (q <= 1.0)
        out[a] = pm[a] * np.where(inside, q ** beta / norm, 0.0)
    return out


def test_grid_sum_matches_numpy_trapezoid_of_scipy_densities(oracle):
    m1 = np.linspace(3.0, 100.0, 181)
    q = np.linspace(0.02, 1.0, 47)
    pdet = campaign_pdet(m1, q)
    lams = synth.make_lambdas(4, 11, seed=61)
    got, flags = oracle.xi_grid(m1, q, pdet, lams)
    for k, L in enumerate(lams):
        f = ref_density_grid(m1, q, L) * pdet
        ref = np.trapezoid(np.trapezoid(f, q, axis=1), m1)
        assert got[k] == pytest.approx(np.log(ref), abs=1e-11)
    assert (flags == 0).all()


def test_grid_matches_the_monte_carlo_selection_term(oracle):
    """Both estimate int p(m1, q | Lambda) P_det: dense grid vs 2e6 injection draws."""
    m1 = np.linspace(3.0, 100.0, 3001)
    q = np.linspace(0.03, 1.0, 801)
    pdet = campaign_pdet(m1, q)
    lams = synth.make_lambdas(3, 11, seed=62)
    grid, _ = oracle.xi_grid(m1, q, pdet, lams)
    inj = synth.make_injections(2 * 10**6, 6, seed=63)
    cat = synth.make_catalog(1, 10, 6, seed=64)
    _, mc, neff, _ = oracle.loglik(cat, inj, lams)
    for k in range(len(lams)):
        tol = 4.0 / np.sqrt(neff[k]) + 5e-3   # Monte Carlo scatter + grid (edge) error
        assert abs(grid[k] - mc[k]) < tol, (grid[k], mc[k], tol)


def test_grid_invalid_lambda(oracle):
    m1 = np.linspace(3.0, 100.0, 20)
    q = np.linspace(0.02, 1.0, 10)
    L = synth.make_lambdas(1, 11, seed=65)
    L[0, 6] = -1.0
    lx, fl = oracle.xi_grid(m1, q, campaign_pdet(m1, q), L)
    assert lx[0] == 0.0 and fl[0] & oracle.FLAG_INVALID_LAMBDA
