"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

The paper prints no worked ln L value, so the oracle is pinned by:
* quadrature: every density integrates to 1 over its support;
* library densities (scipy.stats truncpareto, loguniform, truncnorm, beta) and
  textbook special cases (alpha = 0 uniform, Beta(1, 1) = 1, xi_t = 0 -> 1/4,
  kappa = 1 -> 3 z^2 / 8);
* the mean reweighting factor is 1 when samples come from a normalised
  distribution and are divided by its pdf (Eq. (poplike) recycling identity);
* xi = 1 when every injection is found and Lambda is the draw distribution;
* the -N ln xi term equals the 1/R-prior rate marginal of the first likelihood
  equation of Sec. "Population acceleration", by numerical quadrature over R;
* a brute-force ln L on a hand-chosen tiny catalog built from scipy densities.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from paper_1904_02863_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_catalog.json")
L0 = synth.LAMBDA0[:11]
BOX_LAMBDAS = synth.make_lambdas(4, 12, seed=7)


def _lam(**kw):
    L = synth.LAMBDA0.copy()
    for k, v in kw.items():
        L[synth.PARAMS.index(k)] = v
    return L


MASS_CASES = [_lam(), _lam(alpha=1.0), _lam(alpha=0.0), _lam(alpha=-1.5, lam=0.0),
              _lam(lam=1.0, mpp=20.0, sigpp=8.0), _lam(lam=0.0)] + list(BOX_LAMBDAS)


# --------------------------------------------------------------------------- densities
@pytest.mark.parametrize("L", MASS_CASES)
def test_mass_density_integrates_to_one(oracle, L):
    mmin, mmax, mu = L[2], L[3], L[5]
    val, err = integrate.quad(lambda m: oracle.p_m1(m, L), mmin, mmax,
                              points=[min(max(mu, mmin + 1e-9), mmax - 1e-9)], epsabs=1e-13, epsrel=1e-12, limit=400)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("alpha", [1.0, 1.7, 2.3, 3.5])
def test_mass_power_law_matches_scipy(oracle, alpha):
    L = _lam(alpha=alpha, lam=0.0)
    mmin, mmax = L[2], L[3]
    ref = (stats.loguniform(mmin, mmax) if alpha == 1.0
           else stats.truncpareto(alpha - 1.0, mmax / mmin, scale=mmin))
    for m in np.linspace(mmin + 0.01, mmax, 23):
        assert oracle.p_m1(m, L) == pytest.approx(ref.pdf(m), rel=1e-13)


def test_mass_uniform_special_case(oracle):
    L = _lam(alpha=0.0, lam=0.0)
    assert oracle.p_m1(17.0, L) == pytest.approx(1.0 / (L[3] - L[2]), rel=1e-14)


@pytest.mark.parametrize("mu,sigma", [(35.0, 4.0), (20.0, 8.0), (78.0, 3.0)])
def test_mass_gaussian_matches_scipy_truncnorm(oracle, mu, sigma):
    L = _lam(lam=1.0, mpp=mu, sigpp=sigma)
    mmin, mmax = L[2], L[3]
    ref = stats.truncnorm((mmin - mu) / sigma, (mmax - mu) / sigma, loc=mu, scale=sigma)
    for m in np.linspace(mmin + 0.01, mmax, 19):
        assert oracle.p_m1(m, L) == pytest.approx(ref.pdf(m), rel=1e-12)


def test_mass_mixture_is_linear_in_lambda(oracle):
    m = 33.3
    p0, p1, pm = (oracle.p_m1(m, _lam(lam=v)) for v in (0.0, 1.0, 0.37))
    assert pm == pytest.approx(0.63 * p0 + 0.37 * p1, rel=1e-14)


def test_mass_support_edges(oracle):
    L = _lam()
    assert oracle.p_m1(L[2], L) == 0.0            # m1 = mmin excluded
    assert oracle.p_m1(L[3], L) > 0.0             # m1 = mmax included
    assert oracle.p_m1(np.nextafter(L[3], 1e9), L) == 0.0


@pytest.mark.parametrize("beta", [-2.5, -1.0, 0.0, 1.0, 2.0])
@pytest.mark.parametrize("m1", [5.2, 20.0, 79.0])
def test_mass_ratio_integrates_to_one(oracle, beta, m1):
    L = _lam(beta=beta)
    lo = L[2] / m1
    val, _ = integrate.quad(lambda q: oracle.p_q(q, m1, L), lo, 1.0, epsabs=1e-13, epsrel=1e-12, limit=200)
    assert abs(val - 1.0) < 1e-10
    assert oracle.p_q(0.9 * lo, m1, L) == 0.0 and oracle.p_q(1.0 + 1e-12, m1, L) == 0.0
    # shape: ratio to q = 1 is q^beta
    q = 0.5 * (1.0 + lo)
    assert oracle.p_q(q, m1, L) / oracle.p_q(1.0, m1, L) == pytest.approx(q ** beta, rel=1e-13)


@pytest.mark.parametrize("beta", [-1.0, 0.0, 1.3, 2.0])
@pytest.mark.parametrize("eps", [1e-13, 1e-9, 1e-6, 1e-3, 0.1])
def test_mass_ratio_near_degenerate_support(oracle, beta, eps):
    """m1 a hair above mmin: the q support shrinks to [mmin/m1, 1] and the density
    at q = 1 grows like 1/(1 - mmin/m1).  Pinned against the closed form in
    50-digit arithmetic (catches 1 - x^(1+beta) and ln(mmin/m1) cancellation)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    L = _lam(beta=beta)
    m1 = float(np.nextafter(L[2] * (1.0 + eps), np.inf))
    r = mp.mpf(L[2]) / mp.mpf(m1)
    exact = 1 / (-mp.log(r)) if beta == -1.0 else (1 + mp.mpf(beta)) / (1 - r ** (1 + mp.mpf(beta)))
    assert oracle.p_q(1.0, m1, L) == pytest.approx(float(exact), rel=1e-14)


@pytest.mark.parametrize("ac,bc", [(2.0, 5.0), (1.0, 1.0), (1.0, 3.0), (3.7, 2.2), (0.6, 1.4)])
def test_spin_magnitude_matches_scipy_beta(oracle, ac, bc):
    L = _lam(alpha_chi=ac, beta_chi=bc)
    for a in np.linspace(0.013, 0.987, 17):
        assert oracle.p_chi(a, L) == pytest.approx(stats.beta.pdf(a, ac, bc), rel=1e-12)
    val, _ = integrate.quad(lambda a: oracle.p_chi(a, L), 0.0, 1.0, epsabs=1e-12, epsrel=1e-11, limit=200)
    assert abs(val - 1.0) < 1e-8
    assert oracle.p_chi(-1e-12, L) == 0.0 and oracle.p_chi(1.0 + 1e-12, L) == 0.0


def test_spin_magnitude_edges(oracle):
    assert oracle.p_chi(0.3, _lam(alpha_chi=1.0, beta_chi=1.0)) == 1.0
    assert oracle.p_chi(0.0, _lam(alpha_chi=1.0, beta_chi=3.0)) == pytest.approx(3.0, rel=1e-14)  # 0^0 = 1
    assert oracle.p_chi(1.0, _lam(alpha_chi=2.0, beta_chi=5.0)) == 0.0


@pytest.mark.parametrize("xi,sig", [(0.5, 0.5), (1.0, 0.1), (0.2, 1.5), (0.0, 0.5)])
def test_tilt_matches_scipy_truncnorm(oracle, xi, sig):
    L = _lam(xi_t=xi, sigma_t=sig)
    g = stats.truncnorm(-2.0 / sig, 0.0, loc=1.0, scale=sig)
    rng = np.random.default_rng(3)
    for c1, c2 in rng.uniform(-1, 1, (15, 2)):
        ref = (1 - xi) / 4 + xi * g.pdf(c1) * g.pdf(c2)
        assert oracle.p_tilt(c1, c2, L) == pytest.approx(ref, rel=1e-12)
    val, _ = integrate.dblquad(lambda y, x: oracle.p_tilt(x, y, L), -1, 1, -1, 1, epsabs=1e-11, epsrel=1e-10)
    assert abs(val - 1.0) < 1e-8
    if xi == 0.0:
        assert oracle.p_tilt(0.1, -0.7, L) == 0.25


def test_redshift_density(oracle):
    nodes = np.linspace(0.0, 2.0, 1024)
    for kappa in (0.0, 1.0, 2.7, 4.0):
        L = _lam(kappa=kappa)
        vals = np.array([oracle.p_z(z, L) for z in nodes])
        # normalised exactly against its own 1024-node trapezoid rule
        assert abs(np.trapezoid(vals, nodes) - 1.0) < 1e-13
        exact, _ = integrate.quad(lambda z: (1 + z) ** (kappa - 1) * z * z, 0, 2, epsabs=1e-14, epsrel=1e-13)
        # trapezoid error bound (b - a) h^2 / 12 max|f''|
        h = 2.0 / 1023
        f2 = max(abs(np.gradient(np.gradient((1 + nodes) ** (kappa - 1) * nodes ** 2, nodes), nodes)))
        assert abs(oracle.z_norm(kappa) - exact) <= 2.0 * h * h / 12.0 * f2 * 1.05
    # kappa = 1 is 3 z^2 / 8 up to the trapezoid error
    L = _lam(kappa=1.0)
    assert oracle.p_z(1.3, L) == pytest.approx(3 * 1.3 ** 2 / 8, rel=2e-6)
    assert oracle.p_z(2.0 + 1e-12, L) == 0.0


# --------------------------------------------------------------------------- whole-sample identities
@pytest.mark.parametrize("n_dims", [6, 7])
def test_mean_weight_is_one_under_a_normalised_proposal(oracle, n_dims):
    """Recycling identity behind Eq. (poplike): E_q[p(theta|Lambda)/q(theta)] = 1."""
    rng = np.random.Generator(np.random.PCG64(11 + n_dims))
    th = synth.draw_injections(rng, 60000, n_dims)
    q = synth.draw_pdf(th)
    for L in synth.make_lambdas(3, 12, seed=5 + n_dims):
        w = np.array([oracle.p_theta(t, L) for t in th]) / q
        se = w.std() / math.sqrt(len(w))
        assert abs(w.mean() - 1.0) < 5 * se + 1e-3, (w.mean(), se)


# Lambda* for the self-prior pin: every clipped sample is inside its support (mmin below the
# clip at 5, uniform spins so that a = 0 or 1 keeps density 1).
LAMBDA_STAR = np.array([2.3, 1.0, 4.9, 80.0, 0.1, 35.0, 4.0, 1.0, 1.0, 0.5, 0.5, 2.7])


@pytest.mark.parametrize("n_dims", [6, 7])
def test_weights_are_one_when_the_prior_is_the_population(oracle, n_dims):
    """With pi(theta_ij) := p(theta_ij | Lambda*), every weight p/pi is 1, so each event mean is 1
    and ln L(Lambda*) = -N ln xi(Lambda*) up to rounding (sum of N logs of means of ones)."""
    cat = synth.make_catalog(7, [1, 30, 200, 5, 64, 13, 99], n_dims, seed=31 + n_dims)
    L = LAMBDA_STAR[:11 + (n_dims == 7)]
    prior = np.array([oracle.p_theta(t, L) for t in cat.theta])
    assert (prior > 0).all()
    cat = synth.Catalog(cat.offsets, cat.theta, prior)
    inj = synth.make_injections(20000, n_dims, seed=33 + n_dims)
    lnL, lnxi, _, flags = oracle.loglik(cat, inj, L[None, :])
    assert flags[0] & ~np.uint32(oracle.FLAG_LOW_NEFF) == 0
    assert abs(lnL[0] + cat.n_events * lnxi[0]) <= 1e-13 * cat.n_events * (1 + abs(lnxi[0]))
    # and away from Lambda* the event term is no longer zero
    L2 = L.copy()
    L2[0] = 3.0
    lnL2, lnxi2, _, _ = oracle.loglik(cat, inj, L2[None, :])
    assert abs(lnL2[0] + cat.n_events * lnxi2[0]) > 1e-3


@pytest.mark.parametrize("n_dims", [6, 7])
def test_xi_is_one_at_the_draw_distribution(oracle, n_dims):
    inj = synth.make_injections(20000, n_dims, seed=3, detect=False)
    assert inj.n_found == inj.n_draw
    cat = synth.make_catalog(2, 10, n_dims, seed=1)
    lnL, lnxi, neff, flags = oracle.loglik(cat, inj, synth.LAMBDA_DRAW[None, :11 + (n_dims == 7)])
    expect = 1.0
    if n_dims == 7:  # the model normalises z^2 by its trapezoid, the draw pdf by 8/3
        nodes = np.linspace(0.0, 2.0, 1024)
        expect = (8.0 / 3.0) / np.trapezoid(nodes ** 2, nodes)
    assert math.exp(lnxi[0]) == pytest.approx(expect, rel=1e-13)
    # every weight equal -> N_eff = n_draw * xi^2 / (xi^2 (1 - 1/n)) is huge (variance ~ rounding)
    assert neff[0] > 1e6


def test_minus_N_ln_xi_is_the_rate_marginal(oracle):
    """-N ln xi = ln int_0^inf R^(N-1) e^(-R xi) dR - ln Gamma(N)."""
    cat = synth.make_catalog(3, 40, 6, seed=21)
    inj = synth.make_injections(5000, 6, seed=22)
    L = synth.make_lambdas(1, 11, seed=23)
    lnL, lnxi, _, _ = oracle.loglik(cat, inj, L)
    # per-event ln means from single-event runs (N = 1)
    sum_ln_mean = 0.0
    for i in range(3):
        sub = synth.Catalog(cat.offsets[i:i + 2] - cat.offsets[i], cat.theta[cat.offsets[i]:cat.offsets[i + 1]],
                            cat.prior[cat.offsets[i]:cat.offsets[i + 1]])
        l1, x1, _, _ = oracle.loglik(sub, inj, L)
        sum_ln_mean += l1[0] + x1[0]
    xi = math.exp(lnxi[0])
    N = 3
    rate_int, _ = integrate.quad(lambda R: R ** (N - 1) * math.exp(-R * xi), 0, np.inf, epsabs=0, epsrel=1e-12)
    assert lnL[0] + math.lgamma(N) == pytest.approx(sum_ln_mean + math.log(rate_int), rel=1e-10)


# --------------------------------------------------------------------------- brute force on the hand example
def _ref_density(th, L):
    alpha, beta, mmin, mmax, lam, mu, sig, ac, bc, xit, sigt = L
    m1, q, a1, a2, c1, c2 = th
    if not (mmin < m1 <= mmax) or not (q * m1 >= mmin and q <= 1.0):
        return 0.0
    pl = (stats.loguniform(mmin, mmax).pdf(m1) if alpha == 1.0
          else stats.truncpareto(alpha - 1.0, mmax / mmin, scale=mmin).pdf(m1))
    pp = stats.truncnorm((mmin - mu) / sig, (mmax - mu) / sig, loc=mu, scale=sig).pdf(m1)
    pm = (1 - lam) * pl + lam * pp
    qn, _ = integrate.quad(lambda x: x ** beta, mmin / m1, 1.0, epsabs=0, epsrel=1e-13)
    pq = q ** beta / qn
    pa = stats.beta.pdf(a1, ac, bc) * stats.beta.pdf(a2, ac, bc)
    g = stats.truncnorm(-2.0 / sigt, 0.0, loc=1.0, scale=sigt)
    pt = (1 - xit) / 4 + xit * g.pdf(c1) * g.pdf(c2)
    return pm * pq * pa * pt


def test_brute_force_tiny_catalog(oracle):
    g = json.load(open(GOLDEN))
    cat = synth.Catalog(np.array(g["offsets"], np.int64), np.array(g["theta"]), np.array(g["prior"]))
    inj = synth.Injections(np.array(g["injections"]), np.array(g["p_draw"]), g["n_draw"])
    lams = np.array(g["lambdas"])
    lnL, lnxi, neff, flags = oracle.loglik(cat, inj, lams)
    for k, L in enumerate(lams):
        wi = [_ref_density(t, L) / p for t, p in zip(inj.theta, inj.p_draw)]
        xi = math.fsum(wi) / inj.n_draw
        means = []
        for i in range(cat.n_events):
            a, b = cat.offsets[i], cat.offsets[i + 1]
            means.append(math.fsum(_ref_density(cat.theta[j], L) / cat.prior[j] for j in range(a, b)) / (b - a))
        assert lnxi[k] == pytest.approx(math.log(xi), rel=1e-11, abs=1e-12)
        if min(means) == 0.0:
            assert lnL[k] == -np.inf and flags[k] & oracle.FLAG_ZERO_EVENT
        else:
            ref = math.fsum(math.log(m) for m in means) - cat.n_events * math.log(xi)
            assert lnL[k] == pytest.approx(ref, rel=1e-11)
    # row 2 (mmin = 6) leaves event 2 without support
    assert lnL[2] == -np.inf and flags[2] & oracle.FLAG_ZERO_EVENT
    assert np.isfinite(lnL[:2]).all()


@pytest.mark.parametrize("bad", [dict(sigpp=0.0), dict(sigma_t=-0.1), dict(mmin=80.0), dict(mmin=0.0),
                                 dict(xi_t=1.5), dict(lam=-0.1), dict(alpha_chi=0.0), dict(beta_chi=np.nan)])
def test_invalid_lambda_is_minus_inf_and_flagged(oracle, bad):
    g = json.load(open(GOLDEN))
    cat = synth.Catalog(np.array(g["offsets"], np.int64), np.array(g["theta"]), np.array(g["prior"]))
    inj = synth.Injections(np.array(g["injections"]), np.array(g["p_draw"]), g["n_draw"])
    L = _lam(**bad)[None, :11]
    lnL, lnxi, neff, flags = oracle.loglik(cat, inj, L)
    assert lnL[0] == -np.inf and flags[0] & oracle.FLAG_INVALID_LAMBDA
    assert not np.isnan(lnL[0])


# --------------------------------------------------------------------------- effective sample count of xi
# N_eff of the Monte Carlo selection term (Sec. "Population acceleration": xi is a sample mean over the
# N_draw injections, the missed ones contributing 0) is xi^2 divided by the variance of that sample mean.
# Three pins that do not restate the oracle's formula: a two-class worked example with exact weights, the
# variance of the explicit zero-padded draw vector (numpy), and the scatter of xi over independent
# injection sets. The LOW_NEFF flag (N_eff < 4 N) is pinned on both sides of its threshold.
def _exact_weight_injections(oracle, L, weights, n_draw):
    """Found injections inside the support whose weights p/p_draw are the given numbers."""
    th = np.array([[20.0 + 3.0 * k, 0.7, 0.3, 0.4, 0.2, 0.6] for k in range(len(weights))])
    p = np.array([oracle.p_theta(t, L) for t in th])
    assert (p > 0).all()
    return synth.Injections(th, p / np.asarray(weights, float), n_draw)


def _small_catalog(n_events):
    g = json.load(open(GOLDEN))
    th = np.array(g["theta"][:1] * n_events)
    return synth.Catalog(np.arange(n_events + 1, dtype=np.int64), th, np.full(n_events, 7.5))


def test_neff_two_class_worked_example(oracle):
    """Draws x = (1, 1, 2, 2, 2, 0, 0, 0, 0, 0): mean 0.8, E[x^2] = 1.4, so the variance of the mean is
    (1.4 - 0.64) / 10 = 0.076 and N_eff = 0.64 / 0.076 = 160 / 19."""
    L = L0
    inj = _exact_weight_injections(oracle, L, [1.0, 1.0, 2.0, 2.0, 2.0], 10)
    for n_events, low in ((2, False), (3, True)):  # 4N = 8 < 8.42 < 12 = 4N
        lnL, lnxi, neff, flags = oracle.loglik(_small_catalog(n_events), inj, L[None, :])
        assert math.exp(lnxi[0]) == pytest.approx(0.8, rel=1e-14)
        assert neff[0] == pytest.approx(160.0 / 19.0, rel=1e-12)
        assert bool(flags[0] & oracle.FLAG_LOW_NEFF) == low, (n_events, neff[0])


def test_neff_is_the_variance_of_the_padded_draw_vector(oracle):
    g = json.load(open(GOLDEN))
    cat = synth.Catalog(np.array(g["offsets"], np.int64), np.array(g["theta"]), np.array(g["prior"]))
    inj = synth.Injections(np.array(g["injections"]), np.array(g["p_draw"]), g["n_draw"])
    lams = np.array(g["lambdas"])
    _, lnxi, neff, flags = oracle.loglik(cat, inj, lams)
    for k, L in enumerate(lams):
        x = np.zeros(inj.n_draw)
        x[:inj.n_found] = [_ref_density(t, L) / p for t, p in zip(inj.theta, inj.p_draw)]
        var_of_mean = np.var(x) / inj.n_draw
        assert neff[k] == pytest.approx(np.mean(x) ** 2 / var_of_mean, rel=1e-10)
        assert bool(flags[k] & oracle.FLAG_LOW_NEFF) == (neff[k] < 4 * cat.n_events)


def test_neff_predicts_the_scatter_of_xi(oracle):
    """Over independent injection sets, Var(xi_hat) = xi^2 / N_eff (to sampling error)."""
    L = L0[None, :]
    cat = _small_catalog(1)
    xis, pred = [], []
    for r in range(300):
        inj = synth.make_injections(3000, 6, seed=1000 + r)
        _, lnxi, neff, _ = oracle.loglik(cat, inj, L)
        xis.append(math.exp(lnxi[0]))
        pred.append(math.exp(2 * lnxi[0]) / neff[0])
    ratio = np.var(xis, ddof=1) / np.mean(pred)
    assert 0.75 < ratio < 1.33, ratio
