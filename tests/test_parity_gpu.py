"""GPU parity: the CUDA path (through the C-ABI) against the FP64 CPU oracle.

FP64 mode: |d ln L| <= 1e-12 * (|sum_i ln(S_i/n_i)| + N |ln xi|), ln xi to 1e-12
relative, flags identical.  FP32 mode: |d ln L| <= 0.05 nats against the oracle
on the same (FP64) inputs: the FP32 features are formed from the unrounded
inputs and the support decisions are taken in FP64, so the difference is the
rounding of the features and the FP32 arithmetic.
Sizes span several 4096-sample chunks, ragged tails and K not a multiple of
any Lambda tile; the full catalog-scale workload is checked on sampled Lambda.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_catalog.json")


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


def f64_tol(ref_lnL, ref_lnxi, n_events):
    a = np.abs(np.where(np.isfinite(ref_lnL), ref_lnL, 0.0) + n_events * ref_lnxi)
    return 1e-12 * (a + n_events * np.abs(ref_lnxi)) + 1e-13


def assert_f64_parity(got, ref, n_events):
    lnL, lnxi, neff, flags = got
    r_lnL, r_lnxi, r_neff, r_flags = ref
    assert not np.isnan(lnL).any()
    np.testing.assert_array_equal(flags, r_flags)
    fin = np.isfinite(r_lnL)
    np.testing.assert_array_equal(np.isfinite(lnL), fin)
    np.testing.assert_array_equal(lnL[~fin], r_lnL[~fin])
    tol = f64_tol(r_lnL, r_lnxi, n_events)
    bad = np.abs(lnL[fin] - r_lnL[fin]) > tol[fin]
    assert not bad.any(), (np.abs(lnL - r_lnL)[fin][bad][:5], tol[fin][bad][:5])
    xf = np.isfinite(r_lnxi)
    np.testing.assert_allclose(lnxi[xf], r_lnxi[xf], rtol=1e-12, atol=1e-13)
    nf = np.isfinite(r_neff) & (r_neff > 0)
    np.testing.assert_allclose(neff[nf], r_neff[nf], rtol=1e-8)


def tiny():
    from paper_1904_02863_gb300 import synth
    g = json.load(open(GOLDEN))
    cat = synth.Catalog(np.array(g["offsets"], np.int64), np.array(g["theta"]), np.array(g["prior"]))
    inj = synth.Injections(np.array(g["injections"]), np.array(g["p_draw"]), g["n_draw"])
    return cat, inj, np.array(g["lambdas"])


@pytest.fixture(scope="module")
def small(B):
    from paper_1904_02863_gb300 import synth
    cat, inj, lam = synth.make_workload("f64_10x1000_inj1e5")
    like = B.Likelihood(0).load(cat, inj)
    yield like, cat, inj, lam
    like.close()


@pytest.fixture(scope="module")
def ragged(B):
    """Events spanning 1..4 chunks with ragged tails, redshift on, injections ragged too."""
    from paper_1904_02863_gb300 import synth
    sizes = np.array([1, 4095, 4096, 4097, 9000, 12289, 37, 700])
    cat = synth.make_catalog(len(sizes), sizes, 7, seed=101)
    inj = synth.make_injections(150000, 7, seed=102)
    lam = synth.make_lambdas(37, 12, seed=103)
    like = B.Likelihood(0).load(cat, inj)
    yield like, cat, inj, lam
    like.close()


def test_f64_small_catalog(B, small, oracle):
    like, cat, inj, lam = small
    got = like(lam, B.POP_MODE_F64)
    ref = oracle.loglik(cat, inj, lam)
    assert_f64_parity(got, ref, cat.n_events)


def test_f64_tiny_golden_with_support_edges(B, oracle):
    cat, inj, lam = tiny()
    # add a row where no injection and no event has support (xi = 0) and an invalid row
    extra = np.array([[2.3, 1.0, 60.0, 70.0, 0.1, 65.0, 4.0, 2.0, 5.0, 0.5, 0.5],
                      [2.3, 1.0, 5.0, 80.0, 0.1, 35.0, -4.0, 2.0, 5.0, 0.5, 0.5]])
    lam = np.concatenate([lam, extra])
    like = B.Likelihood(0).load(cat, inj)
    got = like(lam, B.POP_MODE_F64)
    ref = oracle.loglik(cat, inj, lam)
    assert_f64_parity(got, ref, cat.n_events)
    assert got[3][3] & B.POP_FLAG_ZERO_XI and got[3][4] & B.POP_FLAG_INVALID_LAMBDA
    assert got[0][2] == -np.inf and got[3][2] & B.POP_FLAG_ZERO_EVENT
    like.close()


def test_f64_ragged_multichunk_redshift(B, ragged, oracle):
    like, cat, inj, lam = ragged
    assert_f64_parity(like(lam, B.POP_MODE_F64), oracle.loglik(cat, inj, lam), cat.n_events)


def test_f64_model_limits(B, small, oracle):
    """alpha = 1, beta = -1, lam in {0, 1}, xi_t in {0, 1}, alpha_chi = 1: the limit branches."""
    like, cat, inj, lam = small
    base = lam[:1].copy()
    rows = []
    for idx, v in [(0, 1.0), (1, -1.0), (4, 0.0), (4, 1.0), (9, 0.0), (9, 1.0), (7, 1.0), (8, 1.0), (0, 0.0),
                   (1, -2.5)]:
        r = base.copy()
        r[0, idx] = v
        rows.append(r)
    L = np.concatenate(rows)
    assert_f64_parity(like(L, B.POP_MODE_F64), oracle.loglik(cat, inj, L), cat.n_events)


@pytest.mark.parametrize("beta", [-1.0, 0.0, 1.7])
def test_lower_mass_edge(B, small, oracle, beta):
    """mmin next to the 5 Msun clip, where 16% of the samples sit and the q
    normalisation 1 - (mmin/m1)^(1+beta) nearly vanishes: the weights of those
    samples are huge and carry the per-event sums."""
    like, cat, inj, lam = small
    rows = []
    for mmin in (5 - 1e-3, 5 - 1e-6, 5 - 1e-10, 5 + 1e-12, 4.97, 5.04):
        r = synth_lambda0()
        r[1], r[2] = beta, mmin
        rows.append(r)
    L = np.array(rows)
    assert_f64_parity(like(L, B.POP_MODE_F64), oracle.loglik(cat, inj, L), cat.n_events)
    ref = oracle.loglik(cat, inj, L)
    got32 = like(L, B.POP_MODE_F32)
    np.testing.assert_array_equal(got32[3], ref[3])
    d = np.abs(got32[0] - ref[0])
    assert np.max(d) < 5e-3, d


def synth_lambda0():
    from paper_1904_02863_gb300 import synth
    return synth.LAMBDA0[:11].copy()


def test_invalid_lambda_rows(B, small, oracle):
    like, cat, inj, lam = small
    L = np.repeat(lam[:1], 6, axis=0)
    L[0, 6] = 0.0        # sigpp
    L[1, 2] = L[1, 3]    # mmin = mmax
    L[2, 9] = 1.2        # xi_t
    L[3, 7] = -1.0       # alpha_chi
    L[4, 0] = np.inf
    L[5, 10] = np.nan
    lnL, lnxi, neff, flags = like(L, B.POP_MODE_F64)
    assert (lnL == -np.inf).all() and (flags & B.POP_FLAG_INVALID_LAMBDA).all()
    assert not np.isnan(lnL).any() and not np.isnan(lnxi).any()


def test_graphs_tilings_and_memory_paths_agree(B, small):
    import torch
    like, cat, inj, lam = small
    ref = like(lam, B.POP_MODE_F64)[0]
    B.pop_set_graphs(like.ctx, False)
    direct = like(lam, B.POP_MODE_F64)[0]
    B.pop_set_graphs(like.ctx, True)
    np.testing.assert_array_equal(direct, ref)
    dev = like(torch.from_numpy(lam).cuda(), B.POP_MODE_F64)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dev[0].cpu().numpy(), ref)
    saved = B.pop_get_tiling(like.ctx, B.POP_MODE_F64)
    for T in (1, 2, 4, 8, 16):
        for nt in (128, 256, 512):
            B.pop_set_tiling(like.ctx, B.POP_MODE_F64, T, nt)
            out = like(lam, B.POP_MODE_F64)[0]
            if nt == saved[1]:
                np.testing.assert_array_equal(out, ref)   # same summation order
            else:
                np.testing.assert_allclose(out, ref, rtol=1e-13)
    B.pop_set_tiling(like.ctx, B.POP_MODE_F64, *saved)
    f32 = like(lam, B.POP_MODE_F32)[0]
    saved32 = B.pop_get_tiling(like.ctx, B.POP_MODE_F32)
    for nt in (32, 64, 128, 256):
        # One Lambda per thread, each summing whole chunks in a fixed order: the tiling does
        # not change a bit of the result.
        B.pop_set_tiling(like.ctx, B.POP_MODE_F32, nt, nt)
        np.testing.assert_array_equal(like(lam, B.POP_MODE_F32)[0], f32)
    with pytest.raises(B.PopError):
        B.pop_set_tiling(like.ctx, B.POP_MODE_F32, 8, 256)
    B.pop_set_tiling(like.ctx, B.POP_MODE_F32, *saved32)
    # Nor does the lane a Lambda lands on (the lanes are ordered by mmin within each batch).
    perm = np.random.default_rng(5).permutation(len(lam))
    np.testing.assert_array_equal(like(lam[perm], B.POP_MODE_F32)[0], f32[perm])


def test_device_resident_inputs(B, oracle):
    import torch
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(5, 900, 6, seed=55)
    inj = synth.make_injections(30000, 6, seed=56)
    lam = synth.make_lambdas(19, 11, seed=57)
    ctx = B.pop_create(0, torch.cuda.current_stream())
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    B.pop_load_events(ctx, cat.offsets, t(cat.theta), t(cat.prior))
    B.pop_load_injections(ctx, inj.n_draw, t(inj.theta), t(inj.p_draw))
    out = B.pop_loglik(ctx, t(lam), B.POP_MODE_F64)
    torch.cuda.synchronize()
    got = [o.cpu().numpy() for o in out]
    got[3] = got[3].view(np.uint32)
    assert_f64_parity(got, oracle.loglik(cat, inj, lam), cat.n_events)
    B.pop_destroy(ctx)


def test_uneven_batches_reuse_scratch(B, ragged, oracle):
    like, cat, inj, lam = ragged
    from paper_1904_02863_gb300 import synth
    big = synth.make_lambdas(300, 12, seed=104)
    for K in (1, 64, 300, 7, 200):
        L = big[:K]
        got = like(L, B.POP_MODE_F64)
        pick = np.unique(np.linspace(0, K - 1, min(K, 5)).astype(int))
        ref = oracle.loglik(cat, inj, L[pick])
        assert_f64_parity([g[pick] for g in got], ref, cat.n_events)
    lnL = like(big[:0], B.POP_MODE_F64)[0]
    assert lnL.shape == (0,)


def test_f32_small_catalog(B, oracle):
    """FP32 storage and weights, 10 events x 1000 samples, all K = 1024 Lambda: |d ln L| and the
    relative d xi against the oracle.

    xi bound: an FP32 weight is 2^x with x a sum of at most 8 base-2 terms; with every term and
    partial sum below 64 in magnitude, each rounding moves x by at most 64 u (u = 2^-24), so
    |dx| <= 8 * 64 u = 3.1e-5 and the weight's relative error is at most ln2 |dx| + the few ulp
    of ex2.approx / rcp.approx, under 5e-5.  xi is a mean of positive weights (Kahan-summed), so
    its relative error has the same bound; larger terms belong to weights too small to matter.
    """
    from paper_1904_02863_gb300 import synth
    cat, inj, lam = synth.make_workload("f32_10x1000_inj1e5")
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F32)
    lnL, lnxi, _, flags = like(lam, B.POP_MODE_F32)
    ref, ref_xi, _, ref_flags = oracle.loglik(cat, inj, lam)
    np.testing.assert_array_equal(flags, ref_flags)
    d = np.abs(lnL - ref)
    assert np.max(d) <= 0.05, np.max(d)
    xf = np.isfinite(ref_xi)
    np.testing.assert_array_equal(np.isfinite(lnxi), xf)
    rel = np.abs(np.expm1(lnxi[xf] - ref_xi[xf]))
    assert rel.max() <= 5e-5, rel.max()
    like.close()


def test_f32_gate_at_1000_events(B, oracle):
    """The 0.05-nat FP32 budget at N = 1000 events."""
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(1000, 256, 6, seed=201)
    inj = synth.make_injections(10**6, 6, seed=202)
    lam = synth.make_lambdas(24, 11, seed=203)
    lam[0] = synth.LAMBDA0[:11]
    like = B.Likelihood(0).load(cat, inj)
    lnL32 = like(lam, B.POP_MODE_F32)[0]
    ref = oracle.loglik(cat, inj, lam)[0]
    assert np.max(np.abs(lnL32 - ref)) <= 0.05, np.abs(lnL32 - ref)
    like.close()


def test_load_errors_leave_context_usable(B, small, oracle):
    like, cat, inj, lam = small
    before = like(lam[:5], B.POP_MODE_F64)[0]
    bad = cat.theta.copy()
    bad[3, 0] = np.nan
    with pytest.raises(B.PopError) as e:
        B.pop_load_events(like.ctx, cat.offsets, bad, cat.prior)
    assert e.value.status == B.POP_EINVAL
    pr = cat.prior.copy()
    pr[7] = 0.0
    with pytest.raises(B.PopError) as e:
        B.pop_load_events(like.ctx, cat.offsets, cat.theta, pr)
    assert e.value.status == B.POP_EINVAL
    with pytest.raises(B.PopError) as e:
        B.pop_load_events(like.ctx, np.array([0, 5, 5]), cat.theta[:5], cat.prior[:5])
    assert e.value.status == B.POP_EINVAL
    with pytest.raises(B.PopError) as e:
        B.pop_loglik(like.ctx, lam[:, :10], B.POP_MODE_F64)
    assert e.value.status == B.POP_EINVAL
    np.testing.assert_array_equal(like(lam[:5], B.POP_MODE_F64)[0], before)


def test_state_errors(B):
    from paper_1904_02863_gb300 import synth
    ctx = B.pop_create(0)
    lam = synth.make_lambdas(3, 11, seed=1)
    with pytest.raises(B.PopError) as e:
        B.pop_loglik(ctx, lam)
    assert e.value.status == B.POP_ESTATE
    cat = synth.make_catalog(2, 50, 6, seed=2)
    inj = synth.make_injections(5000, 6, seed=3)
    B.pop_load_events(ctx, cat.offsets, cat.theta, cat.prior, storage=B.POP_STORE_F64)
    B.pop_load_injections(ctx, inj.n_draw, inj.theta, inj.p_draw, storage=B.POP_STORE_F64)
    with pytest.raises(B.PopError) as e:
        B.pop_loglik(ctx, lam, B.POP_MODE_F32)
    assert e.value.status == B.POP_ESTATE
    B.pop_destroy(ctx)


def test_autotune_and_cache(B, small, oracle, tmp_path):
    like, cat, inj, lam = small
    like(lam, B.POP_MODE_F64)
    path = str(tmp_path / "tune.txt")
    t1 = B.pop_autotune(like.ctx, B.POP_MODE_F64, len(lam), path)
    assert os.path.getsize(path) > 0
    B.pop_set_tiling(like.ctx, B.POP_MODE_F64, 1, 128)
    t2 = B.pop_autotune(like.ctx, B.POP_MODE_F64, len(lam), path)  # read back from the cache
    assert t1 == t2
    assert_f64_parity(like(lam, B.POP_MODE_F64), oracle.loglik(cat, inj, lam), cat.n_events)
    like(lam, B.POP_MODE_F32)
    B.pop_autotune(like.ctx, B.POP_MODE_F32, len(lam), None)
    B.pop_set_tiling(like.ctx, B.POP_MODE_F64, 8, 256)


def test_ragged_redshift_scale_sampled(B, oracle):
    """The batching form at full size: 2000 ragged events (S_i ~ U{500..16000}, 1.67e7 samples),
    redshift on, 1.97e6 injections, FP32; uneven batches replay one graph (K read on the device).
    The oracle checks sampled rows of every batch."""
    from paper_1904_02863_gb300 import synth
    cat, inj, lam = synth.make_workload("f32_ragged2000_s500to16000_z")
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F32)
    picks = []
    for k in (64, 200, 1000, 4096):
        got = like(lam[:k], B.POP_MODE_F32)[0]
        picks.append((lam[k - 1], got[k - 1]))
    L = np.array([p[0] for p in picks])
    ref = oracle.loglik(cat, inj, L)[0]
    got = np.array([p[1] for p in picks])
    assert np.max(np.abs(got - ref)) <= 0.05, np.abs(got - ref)
    like.close()


def test_catalog_scale_sampled(B, oracle):
    """The benchmark's workload (1000 events x 4096 samples, 1e7 draws, K = 1024) in
    its launch configuration; the oracle checks a sample of the Lambda rows.  The FP32 sample
    adds the rows whose mmin lies closest above an m1 with q = 1: there the mass-ratio
    normalisation 1/(1 - (mmin/m1)^(1+beta)) is largest and most sensitive to m1."""
    from paper_1904_02863_gb300 import synth
    cat, inj, lam = synth.make_workload("f64_catalog_1000x4096_inj1e7")
    like = B.Likelihood(0).load(cat, inj)
    got = like(lam, B.POP_MODE_F64)
    got32 = like(lam, B.POP_MODE_F32)
    pick = np.array([0, 1, 511, 1023])
    ref = oracle.loglik(cat, inj, lam[pick])
    assert_f64_parity([g[pick] for g in got], ref, cat.n_events)
    edge = np.unique(np.concatenate([pick, near_edge_rows(cat, lam, 6)]))
    ref32 = oracle.loglik(cat, inj, lam[edge])
    np.testing.assert_array_equal(got32[3][edge], ref32[3])
    d = np.abs(got32[0][edge] - ref32[0])
    assert np.max(d) <= 0.05, d
    like.close()


def near_edge_rows(cat, lam, n):
    """The n Lambda rows with the smallest (m1 - mmin) / mmin > 0 over the samples with q = 1."""
    m1 = np.sort(cat.theta[cat.theta[:, 1] == 1.0, 0])
    mmin = lam[:, 2]
    i = np.searchsorted(m1, mmin, side="right")
    gap = np.where(i < m1.size, (m1[np.minimum(i, m1.size - 1)] - mmin) / mmin, np.inf)
    return np.argsort(gap)[:n]
