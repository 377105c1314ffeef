"""The ln xi surrogate on the GPU: the tcgen05 GEMM against numpy, the network's
forward and gradients against the FP64 oracle given identical BF16-rounded
weights and inputs, one Adam step against the oracle's update, training on the
injection reweighting itself, the trust gate, and checkpoints."""
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


@pytest.fixture(scope="module")
def ctx(B):
    c = B.pop_create(0)
    yield c
    B.pop_destroy(c)


def bf16(a):
    from oracle import mlp_oracle as M
    return M.round_bf16(a)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 256, 64), (256, 64, 256), (384, 256, 4096), (128, 112, 192)])
def test_tcgen05_gemm_matches_numpy(B, ctx, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(0, 1, (M, K))
    Bm = rng.normal(0, 1, (N, K))
    C = B.pop_mlp_gemm_check(ctx, A, Bm)
    ref = bf16(A) @ bf16(Bm).T
    np.testing.assert_allclose(C, ref, rtol=1e-5, atol=1e-4 * np.sqrt(K))


def random_params(seed=0):
    from oracle import mlp_oracle as M
    rng = np.random.default_rng(seed)
    L = M.LAYERS
    return [(rng.uniform(-1, 1, (b, a)) * np.sqrt(3.0 / a), rng.normal(0, 0.1, b)) for a, b in zip(L, L[1:])]


def to_gpu_params(B, ctx, params):
    from oracle import mlp_oracle as M
    flat = M.flatten(params).astype(np.float32)
    B.pop_mlp_set_params(ctx, flat)
    # the network computes with BF16 copies of the weights (biases stay FP32)
    return [(bf16(W.astype(np.float32)), b.astype(np.float32).astype(np.float64)) for W, b in params]


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def cosine(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def test_forward_matches_oracle(B, ctx):
    from oracle import mlp_oracle as M
    params = random_params(1)
    pb = to_gpu_params(B, ctx, params)
    x = np.random.default_rng(2).uniform(-1, 1, (300, 12))
    y = B.pop_mlp_forward(ctx, x)
    ref, _ = M.forward(pb, bf16(x), round_fn=bf16)
    assert rel_err(y, ref) < 1e-2 and cosine(y, ref) > 0.9999


def test_gradients_match_oracle(B, ctx):
    from oracle import mlp_oracle as M
    params = random_params(3)
    pb = to_gpu_params(B, ctx, params)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (1000, 12))
    t = rng.normal(0, 1, (1000, 2))
    g, loss = B.pop_mlp_gradients(ctx, x, t)
    ref_loss, ref = M.loss_and_grads(pb, bf16(x), t, round_fn=bf16)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    gp = M.unflatten(g.astype(np.float64))
    for (dW, db), (rW, rb) in zip(gp, ref):
        assert rel_err(dW, rW) < 1e-2 and cosine(dW, rW) > 0.999
        assert rel_err(db, rb) < 1e-2 and cosine(db, rb) > 0.999


def test_adam_step_matches_oracle(B, ctx):
    from oracle import mlp_oracle as M
    params = random_params(5)
    to_gpu_params(B, ctx, params)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (256, 12))
    t = rng.normal(0, 1, (256, 2))
    g, _ = B.pop_mlp_gradients(ctx, x, t)
    p0 = B.pop_mlp_get_params(ctx).astype(np.float64)
    B.pop_mlp_train_step(ctx, x, t, 1e-3)
    p1 = B.pop_mlp_get_params(ctx).astype(np.float64)
    gp = M.unflatten(g.astype(np.float64))
    z = M.zeros_like(gp)
    exp, _, _ = M.adam_step(M.unflatten(p0), gp, z, M.zeros_like(gp), 1, lr=1e-3)
    np.testing.assert_allclose(p1, M.flatten(exp), rtol=1e-5, atol=1e-7)


@pytest.fixture(scope="module")
def trained(B):
    """Surrogate problem: 10 events x 1000 samples with redshift, 1e5 injection draws."""
    from paper_1904_02863_gb300 import synth
    cat, inj, lam = synth.make_workload("f32_z_10x1000_inj1e5_surrogate")
    like = B.Likelihood(0).load(cat, inj)
    box = synth.LAMBDA_BOX[:12]
    rmse = B.pop_xi_surrogate_train(like.ctx, 40000, box[:, 0], box[:, 1], epochs=30, seed=7)
    yield like, cat, inj, lam, rmse
    like.close()


def test_surrogate_trains_and_tracks_the_monte_carlo_xi(B, trained):
    like, cat, inj, lam, rmse = trained
    info = B.pop_xi_surrogate_info(like.ctx)
    assert info["heldout_rmse"] == pytest.approx(rmse)
    assert rmse < 0.1, info
    lx, ln, fb = B.pop_xi_surrogate_infer(like.ctx, lam[:256])
    mc = like(lam[:256], B.POP_MODE_F64)
    ok = np.isfinite(mc[1])
    assert np.sqrt(np.mean((lx[ok] - mc[1][ok]) ** 2)) < 0.1
    # ln N_eff of the Monte Carlo estimate is itself noisy (a variance estimate): RMS only
    assert np.sqrt(np.mean((ln[ok] - np.log(mc[2][ok])) ** 2)) < 0.5


def test_surrogate_fallback_outside_the_box(B, trained):
    from paper_1904_02863_gb300 import synth
    like, cat, inj, lam, rmse = trained
    out = lam[:4].copy()
    out[:, 0] = synth.LAMBDA_BOX[0, 1] + 0.5  # alpha above the training box
    _, _, fb = B.pop_xi_surrogate_infer(like.ctx, out)
    assert fb.all()


def test_surrogate_checkpoint_round_trip(B, trained, tmp_path):
    like, cat, inj, lam, rmse = trained
    path = tmp_path / "xi.ckpt"
    B.pop_xi_surrogate_save(like.ctx, path)
    a = B.pop_xi_surrogate_infer(like.ctx, lam[:64])
    ctx2 = B.pop_create(0)
    B.pop_xi_surrogate_load(ctx2, path)
    b = B.pop_xi_surrogate_infer(ctx2, lam[:64])
    np.testing.assert_array_equal(a[0], b[0])
    assert B.pop_xi_surrogate_info(ctx2) == B.pop_xi_surrogate_info(like.ctx)
    np.testing.assert_array_equal(B.pop_xi_surrogate_error(ctx2, lam[:64]), B.pop_xi_surrogate_error(like.ctx, lam[:64]))
    B.pop_destroy(ctx2)


def test_per_lambda_gate_holds_the_budget(B, trained):
    """The network is used for a Lambda only where N x its error bound fits the budget, in
    pop_xi_surrogate_infer and in pop_loglik alike; there ln L differs from the Monte Carlo form
    by N |d ln xi| <= the budget.  The error bounds themselves cover the network's actual
    deviation from the Monte Carlo ln xi on all but a few of 1024 fresh Lambda."""
    like, cat, inj, lam, rmse = trained
    N = cat.n_events
    L = lam[:1024]
    err = B.pop_xi_surrogate_error(like.ctx, L)
    assert np.isfinite(err).all() and (err > 0).all()
    mc = like(L, B.POP_MODE_F32)
    fin = np.isfinite(mc[0])
    try:
        B.pop_xi_surrogate_set_budget(like.ctx, 1e9)   # only the other conditions remain
        _, _, fb_free = B.pop_xi_surrogate_infer(like.ctx, L)
        su = like(L, B.POP_MODE_F32_SURROGATE)
        used = (su[3] & B.POP_FLAG_SURROGATE_USED) != 0
        assert used.mean() > 0.9, used.mean()
        d = np.abs(su[0] - mc[0])
        ok = used & fin
        coverage = np.mean(d[ok] <= N * err[ok] + 1e-6)
        print(f"error bound covers {coverage:.4f} of rows; N x bound quantiles "
              f"{np.quantile(N * err, [0.1, 0.5, 0.9])}")
        assert coverage >= 0.99, coverage
        for budget in (1.0, 0.25, 0.05, 1e-4):
            B.pop_xi_surrogate_set_budget(like.ctx, budget)
            _, _, fb = B.pop_xi_surrogate_infer(like.ctx, L)
            np.testing.assert_array_equal(fb, (fb_free | (N * err > budget)).astype(np.uint8))
            su = like(L, B.POP_MODE_F32_SURROGATE)
            used = (su[3] & B.POP_FLAG_SURROGATE_USED) != 0
            np.testing.assert_array_equal(used, fb == 0)
            np.testing.assert_array_equal(((su[3] & B.POP_FLAG_MC_FALLBACK) != 0), fb == 1)
            d = np.abs(su[0] - mc[0])[used & fin]
            print(f"budget {budget}: used {used.mean():.3f}, max |dlnL| {d.max() if d.size else 0:.3g}")
            assert d.size == 0 or d.max() <= budget + 1e-6, (budget, d.max())
        assert not used.any()   # 1e-4 nats is below every bound
    finally:
        B.pop_xi_surrogate_set_budget(like.ctx, 0.25)


def test_loglik_with_surrogate_xi(B, trained):
    """POP_MODE_F32_SURROGATE: same per-event part as the FP32 Monte Carlo form, ln xi from
    the network where the gate accepts it, Monte Carlo xi (flagged) where it does not."""
    from paper_1904_02863_gb300 import synth
    like, cat, inj, lam, rmse = trained
    L = lam[:300].copy()
    L[:5, 0] = synth.LAMBDA_BOX[0, 1] + 0.3   # outside the training box -> Monte Carlo
    B.pop_xi_surrogate_set_budget(like.ctx, 1e9)   # the box and the trust gate decide here
    mc = like(L, B.POP_MODE_F32)
    su = like(L, B.POP_MODE_F32_SURROGATE)
    lx, _, fb = B.pop_xi_surrogate_infer(like.ctx, L)
    used = (su[3] & B.POP_FLAG_SURROGATE_USED) != 0
    fell = (su[3] & B.POP_FLAG_MC_FALLBACK) != 0
    np.testing.assert_array_equal(used, fb == 0)
    np.testing.assert_array_equal(fell, fb == 1)
    assert fell[:5].all()
    info = B.pop_xi_surrogate_info(like.ctx)
    assert info["trusted"], info   # the seeded training must pass the gate, else this test is vacuous
    assert used[5:].mean() > 0.9, used[5:].mean()
    fin = np.isfinite(mc[0])
    # Monte Carlo rows reproduce the FP32 form exactly; surrogate rows differ only by -N (ln xi_s - ln xi_mc)
    np.testing.assert_array_equal(su[0][fell & fin], mc[0][fell & fin])
    N = cat.n_events
    np.testing.assert_allclose(su[1][used], lx[used], rtol=1e-12)
    np.testing.assert_allclose(su[0][used & fin], mc[0][used & fin] - N * (lx[used & fin] - mc[1][used & fin]),
                               rtol=1e-9, atol=1e-6)
    B.pop_xi_surrogate_set_budget(like.ctx, 0.25)


def test_surrogate_skips_the_injection_work(B):
    """With many injections (1e7 draws, 1.1e6 found) the selection term dominates the cost
    of a small catalog; where the network is used (here every Lambda the trust gate, the box and
    N_eff >= 4 N admit, with no error budget) it replaces that work."""
    import time
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(10, 1000, 6, seed=401)
    inj = synth.make_injections(10**7, 6, seed=402)
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F32)
    box = synth.LAMBDA_BOX[:11]
    B.pop_xi_surrogate_train(like.ctx, 40000, box[:, 0], box[:, 1], epochs=30, seed=3)
    L = synth.make_lambdas(2048, 11, seed=403)
    err = B.pop_xi_surrogate_error(like.ctx, L)
    print(f"N x error bound quantiles (10/50/90%): {np.quantile(10 * err, [0.1, 0.5, 0.9])}")
    B.pop_xi_surrogate_set_budget(like.ctx, 1e9)   # the cost of the skipped work, not the gate
    times = {}
    for mode in (B.POP_MODE_F32, B.POP_MODE_F32_SURROGATE):
        like(L, mode)
        t0 = time.perf_counter()
        for _ in range(5):
            out = like(L, mode)
        times[mode] = time.perf_counter() - t0
    used = (out[3] & B.POP_FLAG_SURROGATE_USED) != 0
    info = B.pop_xi_surrogate_info(like.ctx)
    assert info["trusted"], info
    assert used.mean() > 0.9, used.mean()
    assert times[B.POP_MODE_F32_SURROGATE] < 0.5 * times[B.POP_MODE_F32], times
    like.close()


def test_surrogate_more_accurate_than_its_training_estimate(B, trained):
    """What the network gains: its ln xi is closer to a 10x larger injection set's than
    the Monte Carlo estimate it was trained on (it averages the Monte Carlo scatter).  The
    10x-injection truth and the Monte Carlo ln xi both come from the FP64 CPU oracle."""
    import oracle
    from paper_1904_02863_gb300 import synth
    like, cat, inj, lam, rmse = trained
    big = synth.make_injections(inj.n_draw * 10, 7, seed=synth.seed_for(5, 1) + 99)
    L = lam[:384]
    ref = oracle.loglik(cat, big, L)[1]
    mc = oracle.loglik(cat, inj, L)[1]
    lx, _, fb = B.pop_xi_surrogate_infer(like.ctx, L)
    ok = np.isfinite(ref) & np.isfinite(mc)
    assert ok.mean() > 0.9
    err_mc = np.sqrt(np.mean((mc[ok] - ref[ok]) ** 2))
    err_sur = np.sqrt(np.mean((lx[ok] - ref[ok]) ** 2))
    assert err_sur < err_mc, (err_sur, err_mc)
