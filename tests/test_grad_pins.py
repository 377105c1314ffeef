"""Pins of the oracle's gradient of ln L with respect to Lambda (derived from Eq. poplike:
d ln L = sum_i (sum_j w g)/S_i - N (sum_k w g)/(sum_k w), g the score of p(theta|Lambda)).

* digamma against scipy;
* every component against Richardson-extrapolated central differences of the oracle's own
  ln L (pinned in test_oracle_pins.py), away from the support edges where ln L jumps,
  including the alpha = 1 and beta = -1 limits and kappa with redshift;
* the score identity E[d ln p / d Lambda] = 0 under p itself, at the injection draw
  distribution (a point of the model family), from 10^6 draws."""
import numpy as np
import pytest
from scipy import special

from paper_1904_02863_gb300 import synth

NAMES = synth.PARAMS


def test_digamma_against_scipy(oracle):
    x = np.concatenate([np.geomspace(1e-3, 1e3, 400), [0.5, 1.0, 2.0, 9.99, 10.0, 10.01]])
    got = np.array([oracle.digamma(v) for v in x])
    np.testing.assert_allclose(got, special.digamma(x), rtol=2e-15, atol=2e-15)


EDGE_STEP = 1e-7


def clear_of_samples(L, cat, inj):
    """Move mmin and mmax off every sample's m1 and q m1 by more than the difference stencil
    (ln L jumps where a sample crosses the support edge; the gradient has no such term)."""
    m1 = np.concatenate([cat.theta[:, 0], inj.theta[:, 0]])
    m2 = np.concatenate([cat.theta[:, 0] * cat.theta[:, 1], inj.theta[:, 0] * inj.theta[:, 1]])
    for p, pts in ((2, np.concatenate([m1, m2])), (3, m1)):
        h = EDGE_STEP * abs(L[p])
        while np.min(np.abs(pts - L[p])) < 10 * h:
            L[p] += 7.3 * h
    return L


def fd_grad(oracle, cat, inj, L, h_rel=1e-4):
    """Central differences with one Richardson step (error O(h^4)); a smaller step on the
    support edges mmin, mmax (kept clear of every sample by clear_of_samples)."""
    P = len(L)
    g = np.zeros(P)
    for p in range(P):
        h = (EDGE_STEP if p in (2, 3) else h_rel) * max(abs(L[p]), 1.0)
        rows = []
        for s in (2.0, 1.0, -1.0, -2.0):
            x = L.copy()
            x[p] += s * h
            rows.append(x)
        f = oracle.loglik(cat, inj, np.array(rows), nthreads=1)[0]
        d1 = (f[1] - f[2]) / (2 * h)
        d2 = (f[0] - f[3]) / (4 * h)
        g[p] = (4 * d1 - d2) / 3
    return g


def small_case(n_dims, seed):
    cat = synth.make_catalog(4, 300, n_dims, seed=seed)
    inj = synth.make_injections(20000, n_dims, seed=seed + 1)
    return cat, inj


# Lambda away from the sample pile-ups at m1 = 5 (clip), q m1 = 5 (nudge) and m1 = 80 (clip).
BASE = np.array([2.6, 1.3, 4.4, 86.0, 0.2, 33.0, 5.0, 2.5, 4.5, 0.6, 0.7, 2.2])


@pytest.mark.parametrize("label,override,n_dims", [
    ("generic", {}, 6),
    ("alpha = 1", {0: 1.0}, 6),
    ("beta = -1", {1: -1.0}, 6),
    ("redshift", {}, 7),
])
def test_gradient_matches_finite_differences(oracle, label, override, n_dims):
    cat, inj = small_case(n_dims, seed=71 if n_dims == 6 else 73)
    L = BASE[: 11 + (n_dims == 7)].copy()
    for k, v in override.items():
        L[k] = v
    L = clear_of_samples(L, cat, inj)
    lnL, grad, fl = oracle.loglik_grad(cat, inj, L[None, :], nthreads=1)
    assert np.isfinite(lnL[0]) and (int(fl[0]) & ~4) == 0
    ref = fd_grad(oracle, cat, inj, L)
    scale = np.maximum(np.abs(ref), 1.0)
    bad = np.abs(grad[0] - ref) > 2e-6 * scale
    assert not bad.any(), {NAMES[p]: (grad[0][p], ref[p]) for p in np.where(bad)[0]}


def test_mean_score_under_the_population_itself(oracle):
    """theta ~ p(theta | Lambda) (the generator's inverse-CDF samplers): the score has mean 0 for
    every parameter that leaves the support alone, and differentiating the normalisation
    over the moving upper edge gives E[g_mmax] = -p_m1(mmax).  5 sigma of the Monte Carlo
    mean.  mmin is left to the finite differences: the q density at its lower edge grows like
    1/(m1 - mmin), so the flux through q = mmin/m1, and E[g_mmin], are infinite."""
    L = BASE.copy()
    rng = np.random.Generator(np.random.PCG64(91))
    th = synth.draw_truths(rng, 200000, 7, lam=L)
    G = np.array([oracle.score(t, L)[1] for t in th])
    assert np.isfinite(G).all()
    mean, sem = G.mean(0), G.std(0) / np.sqrt(len(G))
    expect = np.zeros(len(L))
    expect[3] = -oracle.p_m1(L[3], L)
    z = np.abs(mean - expect) / sem
    z[2] = 0.0
    assert (z < 5).all(), {NAMES[p]: (mean[p], expect[p], z[p]) for p in range(len(L)) if z[p] >= 5}
    assert abs(expect[3]) > 20 * sem[3]   # the edge term is resolved, not lost in the noise
