"""The batched ensemble sampler: correct on an analytic target (CPU), and driving
the GPU likelihood with one batched call per half-ensemble (GPU)."""
import numpy as np
import pytest

from paper_1904_02863_gb300 import sampler


def test_stretch_move_samples_a_correlated_gaussian():
    """Pinned against the target's known moments: mean and covariance of a 3-d normal."""
    mean = np.array([1.0, -2.0, 0.5])
    A = np.array([[1.0, 0.6, 0.0], [0.6, 2.0, -0.3], [0.0, -0.3, 0.5]])
    inv = np.linalg.inv(A)
    calls = []

    def log_prob(x):
        calls.append(len(x))
        d = x - mean
        return -0.5 * np.einsum("ij,jk,ik->i", d, inv, d)

    rng = np.random.default_rng(0)
    p0 = mean + 0.1 * rng.normal(size=(64, 3))
    chain, lp, acc = sampler.stretch_sample(log_prob, p0, 3000, seed=1)
    s = chain[500:].reshape(-1, 3)
    assert np.allclose(s.mean(0), mean, atol=0.08)
    assert np.allclose(np.cov(s.T), A, atol=0.12)
    assert 0.2 < acc.mean() < 0.9
    assert set(calls[1:]) == {32}  # every call is one half-ensemble batch


def test_rejects_outside_the_support():
    def log_prob(x):
        return np.where(np.all(np.abs(x) < 1, axis=1), 0.0, -np.inf)

    p0 = np.random.default_rng(2).uniform(-0.5, 0.5, (16, 2))
    chain, lp, acc = sampler.stretch_sample(log_prob, p0, 400, seed=3)
    assert np.all(np.abs(chain) < 1)
    assert np.allclose(chain[100:].reshape(-1, 2).std(0), 1 / np.sqrt(3), atol=0.06)


@pytest.mark.gpu
def test_population_sampler_on_the_gpu_likelihood():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_02863_gb300 import binding as B
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(60, 500, 6, seed=501)
    inj = synth.make_injections(200000, 6, seed=502)
    like = B.Likelihood(0).load(cat, inj)
    box = synth.LAMBDA_BOX[:11]
    logp = sampler.population_log_posterior(like, box[:, 0], box[:, 1])
    p0 = synth.make_lambdas(64, 11, seed=503)
    chain, lp, acc = sampler.stretch_sample(logp, p0, 60, seed=4)
    assert np.isfinite(lp[-1]).all()
    assert lp[-1].mean() > lp[0].mean()   # walkers climb from the prior box towards the posterior
    assert acc.mean() > 0.05
    like.close()
