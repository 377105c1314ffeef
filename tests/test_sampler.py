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


@pytest.mark.gpu
def test_gpu_driven_chain_equals_the_oracle_driven_chain():
    """The same seeded stretch-move run, once on the GPU FP64 ln L and once on the CPU oracle:
    with ln L equal to FP64 tolerance, every accept/reject decision is the same, so the chains are
    identical and their log-probabilities agree to 1e-12 relative."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1904_02863_gb300 import binding as B
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(12, [300, 17, 410, 64, 999, 5, 250, 128, 700, 33, 81, 160], 6, seed=511)
    inj = synth.make_injections(30000, 6, seed=512)
    box = synth.LAMBDA_BOX[:11]
    lo, hi = box[:, 0], box[:, 1]
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F64)
    gpu_logp = sampler.population_log_posterior(like, lo, hi, mode=B.POP_MODE_F64)

    def oracle_logp(lam):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        inside = np.all((lam >= lo) & (lam <= hi), axis=1)
        out = np.full(len(lam), -np.inf)
        if inside.any():
            out[inside] = oracle.loglik(cat, inj, lam[inside])[0]
        return out

    p0 = synth.make_lambdas(32, 11, seed=513)
    c_gpu, lp_gpu, acc_gpu = sampler.stretch_sample(gpu_logp, p0, 25, seed=5)
    c_cpu, lp_cpu, acc_cpu = sampler.stretch_sample(oracle_logp, p0, 25, seed=5)
    like.close()
    np.testing.assert_array_equal(c_gpu, c_cpu)
    np.testing.assert_array_equal(acc_gpu, acc_cpu)
    fin = np.isfinite(lp_cpu)
    np.testing.assert_array_equal(np.isfinite(lp_gpu), fin)
    np.testing.assert_allclose(lp_gpu[fin], lp_cpu[fin], rtol=1e-12, atol=1e-9)
    assert acc_cpu.mean() > 0.05   # the run moved, so the comparison is not vacuous
