"""GPU parity of POP_MODE_FF (sample weights in float-float arithmetic) against the FP64
oracle, held to the FP64 mode's tolerance: |d ln L| <= 1e-12 (|sum_i ln(S_i/n_i)| + N |ln xi|),
ln xi to 1e-12 relative, flags identical.

Why the FP64 bar holds: each weight is within a few 1e-14 relative (float-float operations
carry ~2^-48; the exponentials' arguments are good to ~2^-47 times the sum of their terms'
magnitudes, below 100 here), so ln(S_i/n_i) moves by at most a few 1e-14 per event and ln L
by N times that, two orders below the bar; near the lower mass edge the q normalisation
takes the exact FP64 gap, where float-float alone would lose its relative accuracy."""
import numpy as np
import pytest

from test_parity_gpu import assert_f64_parity, f64_tol, tiny

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
def small(B):
    from paper_1904_02863_gb300 import synth
    cat, inj, lam = synth.make_workload("f64_10x1000_inj1e5")
    like = B.Likelihood(0).load(cat, inj)
    yield like, cat, inj, lam
    like.close()


def test_ff_small_catalog(B, small, oracle):
    like, cat, inj, lam = small
    assert_f64_parity(like(lam, B.POP_MODE_FF), oracle.loglik(cat, inj, lam), cat.n_events)


def test_ff_tiny_golden_with_support_edges(B, oracle):
    cat, inj, lam = tiny()
    extra = np.array([[2.3, 1.0, 60.0, 70.0, 0.1, 65.0, 4.0, 2.0, 5.0, 0.5, 0.5],
                      [2.3, 1.0, 5.0, 80.0, 0.1, 35.0, -4.0, 2.0, 5.0, 0.5, 0.5]])
    lam = np.concatenate([lam, extra])
    like = B.Likelihood(0).load(cat, inj)
    got = like(lam, B.POP_MODE_FF)
    assert_f64_parity(got, oracle.loglik(cat, inj, lam), cat.n_events)
    assert got[3][3] & B.POP_FLAG_ZERO_XI and got[3][4] & B.POP_FLAG_INVALID_LAMBDA
    like.close()


def test_ff_ragged_multichunk_redshift(B, oracle):
    from paper_1904_02863_gb300 import synth
    sizes = np.array([1, 4095, 4096, 4097, 9000, 12289, 37, 700])
    cat = synth.make_catalog(len(sizes), sizes, 7, seed=101)
    inj = synth.make_injections(150000, 7, seed=102)
    lam = synth.make_lambdas(37, 12, seed=103)
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F64)
    assert_f64_parity(like(lam, B.POP_MODE_FF), oracle.loglik(cat, inj, lam), cat.n_events)
    like.close()


def test_ff_model_limits(B, small, oracle):
    """alpha = 1, beta = -1, lam in {0, 1}, xi_t in {0, 1}, alpha_chi = beta_chi = 1, alpha = 0 and
    beta < -1 (1 + beta < 0: the q normalisation changes sign)."""
    like, cat, inj, lam = small
    base = lam[:1].copy()
    rows = []
    for idx, v in [(0, 1.0), (1, -1.0), (4, 0.0), (4, 1.0), (9, 0.0), (9, 1.0), (7, 1.0), (8, 1.0), (0, 0.0),
                   (1, -2.5)]:
        r = base.copy()
        r[0, idx] = v
        rows.append(r)
    L = np.concatenate(rows)
    assert_f64_parity(like(L, B.POP_MODE_FF), oracle.loglik(cat, inj, L), cat.n_events)


@pytest.mark.parametrize("beta", [-1.0, 0.0, 1.7])
def test_ff_lower_mass_edge(B, small, oracle, beta):
    """mmin next to the 5 Msun clip where 16% of the samples sit: the q normalisation of those
    samples nearly vanishes, their weights carry the event sums, and ln(mmin/m1) comes from the
    exact FP64 gap (down to 1e-10 relative) and the expm1 series."""
    from paper_1904_02863_gb300 import synth
    like, cat, inj, lam = small
    rows = []
    for mmin in (5 - 1e-3, 5 - 1e-6, 5 - 1e-10, 5 + 1e-12, 4.97, 5.04, 4.9, 4.7):
        r = synth.LAMBDA0[:11].copy()
        r[1], r[2] = beta, mmin
        rows.append(r)
    L = np.array(rows)
    assert_f64_parity(like(L, B.POP_MODE_FF), oracle.loglik(cat, inj, L), cat.n_events)


def test_ff_invalid_rows_and_order_independence(B, small):
    like, cat, inj, lam = small
    L = np.repeat(lam[:1], 6, axis=0)
    L[0, 6] = 0.0
    L[1, 2] = L[1, 3]
    L[2, 9] = 1.2
    L[3, 7] = -1.0
    L[4, 0] = np.inf
    L[5, 10] = np.nan
    lnL, lnxi, neff, flags = like(L, B.POP_MODE_FF)
    assert (lnL == -np.inf).all() and (flags & B.POP_FLAG_INVALID_LAMBDA).all()
    assert not np.isnan(lnL).any() and not np.isnan(lnxi).any()
    # one Lambda per thread over whole chunks: the lane a Lambda lands on changes no bit
    ref = like(lam, B.POP_MODE_FF)[0]
    perm = np.random.default_rng(7).permutation(len(lam))
    np.testing.assert_array_equal(like(lam[perm], B.POP_MODE_FF)[0], ref[perm])
    B.pop_set_graphs(like.ctx, False)
    np.testing.assert_array_equal(like(lam, B.POP_MODE_FF)[0], ref)
    B.pop_set_graphs(like.ctx, True)


def test_ff_needs_f64_storage(B):
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(3, 200, 6, seed=71)
    inj = synth.make_injections(20000, 6, seed=72)
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F32)
    with pytest.raises(B.PopError) as e:
        like(synth.make_lambdas(4, 11, seed=73), B.POP_MODE_FF)
    assert e.value.status == B.POP_ESTATE
    like.close()


def test_ff_parts_match_the_whole(B, oracle):
    """The event-partition parts (sum_i ln(S_i/n_i), sum w, sum w^2) in float-float."""
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(5, 3000, 6, seed=81)
    inj = synth.make_injections(200000, 6, seed=82)
    lam = synth.make_lambdas(20, 11, seed=83)
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F64)
    ev, sw, sw2, fl = B.pop_loglik_parts(like.ctx, lam, B.POP_MODE_FF)
    rev, rsw, rsw2, rfl = oracle.loglik_parts(cat, inj, lam)
    np.testing.assert_array_equal(fl, rfl)
    fin = np.isfinite(rev)
    np.testing.assert_allclose(ev[fin], rev[fin], rtol=1e-12, atol=1e-12 * cat.n_events)
    np.testing.assert_allclose(sw, rsw, rtol=1e-12)
    np.testing.assert_allclose(sw2, rsw2, rtol=1e-12)
    like.close()


def test_ff_catalog_scale(B, oracle):
    """The benchmark's workload (1000 events x 4096 samples, 1e7 draws, K = 1024): every row
    against the FP64 kernel's within the FP64 bar, sampled rows against the oracle."""
    from paper_1904_02863_gb300 import synth
    cat, inj, lam = synth.make_workload("f64_catalog_1000x4096_inj1e7")
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F64)
    ff = like(lam, B.POP_MODE_FF)
    f64 = like(lam, B.POP_MODE_F64)
    np.testing.assert_array_equal(ff[3], f64[3])
    fin = np.isfinite(f64[0])
    tol = f64_tol(f64[0], f64[1], cat.n_events)
    assert (np.abs(ff[0][fin] - f64[0][fin]) <= tol[fin]).all(), np.max(np.abs(ff[0][fin] - f64[0][fin]) / tol[fin])
    pick = np.array([0, 1, 511, 1023])
    assert_f64_parity([g[pick] for g in ff], oracle.loglik(cat, inj, lam[pick]), cat.n_events)
    like.close()


def ff_value(x):
    """x rounded to a float-float value (FP32 hi, then the FP32 rounding of the rest), as staged."""
    hi = x.astype(np.float32).astype(np.float64)
    return hi + (x - hi).astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def ctx(B):
    c = B.pop_create(0)
    yield c
    B.pop_destroy(c)


def rel_err(y, ref):
    return np.abs(y - ref) / np.maximum(np.abs(ref), 1e-300)


def test_ff_packed_fma_is_fused(B, ctx):
    """The error-free product rests on fma.rn.f32x2 rounding once: hi^2 - fl(hi^2) is exact."""
    x = np.random.default_rng(1).uniform(-100.0, 100.0, 4001)
    hi = x.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(B.pop_math_check(ctx, 7, x), hi * hi)


def test_ff_square_and_reciprocal(B, ctx):
    x = np.random.default_rng(2).uniform(-100.0, 100.0, 4001)
    v = ff_value(x)
    assert rel_err(B.pop_math_check(ctx, 6, x), v * v).max() < 1e-13
    assert rel_err(B.pop_math_check(ctx, 5, x), 1.0 / v).max() < 1e-13


def test_ff_exp_and_expm1(B, ctx):
    """exp on [-60, 87] within (2 + |x|) 1e-14 relative (the argument's own float-float
    rounding scales with |x|; below about e^-70 the lo part leaves the FP32 normal range and
    the result keeps FP32 precision, which matters nowhere for a weight sum); expm1 within 1e-13
    relative below 1/16 (the series, down to |x| = 1e-12) and 2e-13 above it (the table form's
    absolute error, a few 2^-48, against a result of 1/16 at the switch)."""
    rng = np.random.default_rng(3)
    x = rng.uniform(-60.0, 87.0, 20001)
    v = ff_value(x)
    e = rel_err(B.pop_math_check(ctx, 3, x), np.exp(v))
    assert (e <= (2.0 + np.abs(v)) * 1e-14).all(), e.max()
    assert (B.pop_math_check(ctx, 3, np.array([-88.0, -1e3])) == 0.0).all()
    x = np.concatenate([rng.uniform(-30.0, 30.0, 8000), rng.uniform(-0.07, 0.07, 8000),
                        np.sign(rng.uniform(-1, 1, 2000)) * 10.0 ** rng.uniform(-12, -1, 2000)])
    v = ff_value(x)
    e = rel_err(B.pop_math_check(ctx, 4, x), np.expm1(v))
    bar = np.where(np.abs(v) < 0.0625, 1e-13, 2e-13)
    assert (e < bar).all(), (e.max(), v[np.argmax(e / bar)])
