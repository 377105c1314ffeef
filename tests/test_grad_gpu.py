"""GPU parity of the gradient d ln L / d Lambda (pop_loglik_grad, FP64) against the oracle's
analytic gradient, and against finite differences of the GPU's own ln L.

Tolerance.  Per pair, both sides evaluate the weight within ~100 u and its score terms
(differences of O(10) quantities: ln m1 against the power-law constant, (m1 - mpp)/sigpp^2
against the edge densities, ...) within ~1e3 u of their size; the sums over a catalog's
samples and events add at most n u of the summed magnitudes.  With scores of O(10) for
the Lambda here: |dG_p| <= 1e-10 (|G_p| + 10 N)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1904_02863_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


BASE = np.array([2.6, 1.3, 4.4, 86.0, 0.2, 33.0, 5.0, 2.5, 4.5, 0.6, 0.7, 2.2])


def special_rows(P, n=12, seed=1001):
    from paper_1904_02863_gb300 import synth
    L = synth.make_lambdas(n, P, seed=seed)
    L[0] = BASE[:P]
    L[1, 0] = 1.0      # alpha = 1
    L[2, 1] = -1.0     # beta = -1
    L[3, 4] = 0.0      # lam = 0
    L[4, 4] = 1.0      # lam = 1
    L[5, 9] = 0.0      # xi_t = 0
    L[6, 10] = -0.5    # invalid: sigma_t < 0
    return L


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


def check(got, ref, n_events):
    lnL, G, fl = got
    rl, rG, rfl = ref
    np.testing.assert_array_equal(fl, rfl)
    fin = np.isfinite(rl)
    np.testing.assert_array_equal(np.isfinite(lnL), fin)
    scale = np.abs(rl[fin]) + 1.0
    assert (np.abs(lnL[fin] - rl[fin]) <= 1e-12 * scale + 1e-12 * n_events * 10).all()
    tol = 1e-10 * (np.abs(rG) + 10 * n_events)
    bad = np.abs(G - rG) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], G[bad][:5], rG[bad][:5])
    assert (G[~fin] == 0).all()


@pytest.mark.parametrize("n_dims", [6, 7])
def test_gradient_matches_oracle(B, oracle, n_dims):
    from paper_1904_02863_gb300 import synth
    sizes = np.array([1, 700, 4097, 300, 5000, 64, 8193, 20])
    cat = synth.make_catalog(len(sizes), sizes, n_dims, seed=1002 + n_dims)
    inj = synth.make_injections(60000, n_dims, seed=1010 + n_dims)
    P = 11 + (n_dims == 7)
    lam = special_rows(P)
    like = B.Likelihood(0).load(cat, inj)
    got = B.pop_loglik_grad(like.ctx, lam)
    ref = oracle.loglik_grad(cat, inj, lam)
    check(got, ref, cat.n_events)
    # the same ln L as pop_loglik (another kernel, another rounding order)
    lnL = like(lam, B.POP_MODE_F64)[0]
    fin = np.isfinite(lnL)
    np.testing.assert_allclose(got[0][fin], lnL[fin], rtol=1e-12, atol=1e-9)
    like.close()


def test_gradient_matches_finite_differences_of_the_gpu_ln_l(B):
    """Richardson-extrapolated central differences of pop_loglik (FP64), away from the sample
    pile-ups at the support edges: an oracle-free check of the gradient kernel."""
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(6, 2000, 6, seed=1020)
    inj = synth.make_injections(100000, 6, seed=1021)
    like = B.Likelihood(0).load(cat, inj)
    L = clear_of_samples(BASE[:11].copy(), cat, inj)
    G = B.pop_loglik_grad(like.ctx, L[None, :])[1][0]
    rows = []
    hs = []
    for p in range(11):
        h = (EDGE_STEP if p in (2, 3) else 1e-4) * max(abs(L[p]), 1.0)
        hs.append(h)
        for s in (2.0, 1.0, -1.0, -2.0):
            x = L.copy()
            x[p] += s * h
            rows.append(x)
    f = like(np.array(rows), B.POP_MODE_F64)[0].reshape(11, 4)
    fd = np.array([(4 * (f[p, 1] - f[p, 2]) / (2 * hs[p]) - (f[p, 0] - f[p, 3]) / (4 * hs[p])) / 3 for p in range(11)])
    np.testing.assert_allclose(G, fd, rtol=2e-6, atol=2e-6 * np.maximum(np.abs(fd), 1.0).max())
    like.close()


def test_gradient_catalog_scale_sampled(B, oracle):
    """300 events x 4096 samples and 3e5 injection draws, K = 256 rows on the GPU, 2 rows
    through the oracle."""
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(300, 4096, 6, seed=1030)
    inj = synth.make_injections(300000, 6, seed=1031)
    lam = synth.make_lambdas(256, 11, seed=1032)
    like = B.Likelihood(0).load(cat, inj)
    got = B.pop_loglik_grad(like.ctx, lam)
    pick = np.array([0, 255])
    ref = oracle.loglik_grad(cat, inj, lam[pick])
    check((got[0][pick], got[1][pick], got[2][pick]), ref, cat.n_events)
    like.close()


def test_gradient_errors(B):
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(3, 100, 6, seed=1040)
    inj = synth.make_injections(5000, 6, seed=1041)
    like = B.Likelihood(0)
    lam = synth.make_lambdas(3, 11, seed=1042)
    B.pop_load_events(like.ctx, cat.offsets, cat.theta, cat.prior)
    with pytest.raises(B.PopError) as e:
        B.pop_loglik_grad(like.ctx, lam)          # no injections
    assert e.value.status == B.POP_ESTATE
    B.pop_load_injections(like.ctx, inj.n_draw, inj.theta, inj.p_draw)
    with pytest.raises(B.PopError) as e:
        B.pop_loglik_grad(like.ctx, np.zeros((3, 12)))
    assert e.value.status == B.POP_EINVAL
    assert B.pop_loglik_grad(like.ctx, np.zeros((0, 11)))[0].shape == (0,)
    like.close()
