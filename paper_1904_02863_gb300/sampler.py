"""Batched ensemble sampler over Lambda (the step above the likelihood).

The paper runs its population likelihood inside stochastic samplers (MCMC,
nested sampling) and notes that the sampler itself is hard to parallelise
(Introduction).  What parallelises is the likelihood of many proposals at
once: here the affine-invariant ensemble sampler of Goodman & Weare (2010,
"stretch move") keeps W walkers in two halves; each half-step proposes a
move for every walker of one half from the other half, and evaluates all W/2
proposals in ONE batched call (one graph replay of the GPU pipeline).

``log_prob`` is any callable mapping a [M, P] array of Lambda to M log
densities (e.g. :func:`population_log_posterior`); -inf rejects.
"""
from __future__ import annotations

import numpy as np


def stretch_sample(log_prob, p0, n_steps, a=2.0, seed=0, thin=1):
    """Run the stretch-move ensemble sampler.

    p0: initial walkers [W, P] (W even, W >= 2 P recommended).
    Returns (chain [n_steps // thin, W, P], log_prob [n_steps // thin, W], acceptance fraction [W]).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.array(p0, dtype=np.float64, copy=True)
    W, P = x.shape
    if W % 2 or W < 4:
        raise ValueError("need an even number of walkers, at least 4")
    lp = np.asarray(log_prob(x), dtype=np.float64)
    half = W // 2
    halves = (np.arange(half), np.arange(half, W))
    accepted = np.zeros(W)
    chain, lps = [], []
    for step in range(n_steps):
        for s in (0, 1):
            mine, other = halves[s], halves[1 - s]
            # z ~ g(z) proportional to 1/sqrt(z) on [1/a, a]
            z = ((a - 1.0) * rng.random(half) + 1.0) ** 2 / a
            partners = x[other[rng.integers(0, half, half)]]
            prop = partners + z[:, None] * (x[mine] - partners)
            lp_prop = np.asarray(log_prob(prop), dtype=np.float64)
            log_ratio = (P - 1) * np.log(z) + lp_prop - lp[mine]
            ok = np.log(rng.random(half)) < np.where(np.isnan(log_ratio), -np.inf, log_ratio)
            x[mine[ok]] = prop[ok]
            lp[mine[ok]] = lp_prop[ok]
            accepted[mine[ok]] += 1
        if (step + 1) % thin == 0:
            chain.append(x.copy())
            lps.append(lp.copy())
    return np.array(chain), np.array(lps), accepted / n_steps


def population_log_posterior(likelihood, lo, hi, mode=None):
    """log p(Lambda | data) up to a constant: ln L from the GPU library, uniform prior on [lo, hi].

    ``likelihood`` is a :class:`paper_1904_02863_gb300.binding.Likelihood` with catalog and
    injections loaded; one call evaluates the whole batch of proposals.
    """
    from . import binding as B
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    m = B.POP_MODE_F32 if mode is None else mode

    def log_prob(lam):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        inside = np.all((lam >= lo) & (lam <= hi), axis=1)
        out = np.full(len(lam), -np.inf)
        if inside.any():
            out[inside] = likelihood(lam[inside], m)[0]
        return out

    return log_prob
