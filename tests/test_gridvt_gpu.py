"""GPU parity of the grid selection term (through the C-ABI) against the oracle's grid sum.

Tolerances follow from the arithmetic.  Every term of the sum is positive, so
the oracle's running sum over n nodes is within (n - 1) u of the exact sum of
its terms (u = 2^-53), the GPU's node sums (nb terms), row combine (64 + row
tiles) likewise.  Each term's own evaluation differs between the two sides by
at most ~1024 u: the GPU takes ln(mmin/m1) as ln mmin - ln m1 outside ~2^-6 of
the lower mass edge, whose two rounded logs (|ln| < 8, half-ulp 2^-51 each)
give a relative error up to 2 x 2^-51 / ln(1 + 2^-6) ~ 520 u in the q
normalisation; the exponents (|arg| < 30, one rounding each) add ~60 u.
FP64:  |d ln xi| <= (n + nb + 128 + 1024) u.
FP32 mode adds, in units of u32 = 2^-24: pdet rounded to FP32 (1); U =
wq 2^(beta log2 q) with an FP32 exponent |arg| < 20 (~14) and exp2f (2 ulp)
and two roundings (24 in all); the FP32 row factor W (exponents |arg| < 30
rounded three times, ~62, exp2f, log1pf, expm1f, the reciprocal and four
products, 81 in all); the FP32 sum of a 32-node chunk (31) and the FP32
running sum over the chunks (n_chunks; the kernel runs one per quarter of the q
range, which only shortens it).  Its row combine (exact products, float-float
sums) is as accurate as the FP64 one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


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


@pytest.fixture
def ctx(B):
    c = B.pop_create(0)
    yield c
    B.pop_destroy(c)


def exact_grid():
    """181 x 45 nodes that are exact binary fractions: m1 = 2 + a/2, q = k/40 (k = 2..46, so
    nb = 39 of them are <= 1).  fl64(q m1) hits mmin = 5 exactly at several nodes.  pdet is
    not separable (a transposed index would show)."""
    m1 = 2.0 + 0.5 * np.arange(181)
    q = np.arange(2, 47) / 40.0
    pdet = (1.0 / (1.0 + np.exp(-(m1[:, None] - 20.0) / 5.0))) * (0.2 + 0.8 * q[None, :] ** 0.7)
    pdet[::17, ::5] = 0.0
    return m1, q, np.ascontiguousarray(pdet)


def special_lambdas(n=100, seed=701):
    from paper_1904_02863_gb300 import synth
    L = synth.make_lambdas(n, 11, seed=seed)
    L[0, 2] = 5.0                       # mmin on a node; q m1 = mmin exactly at (10, 0.5), (20, 0.25), ...
    L[1, 1] = -1.0                      # beta = -1: 1 / (q ln(m1/mmin))
    L[2, 0] = 1.0                       # alpha = 1: 1 / (m1 ln(mmax/mmin))
    L[3, 4] = 0.0                       # no Gaussian peak
    L[4, 4] = 1.0                       # only the Gaussian peak
    L[5, 2], L[5, 3] = 95.0, 99.0       # mass range above every node: xi = 0
    L[6, 6] = -1.0                      # invalid: sigpp < 0
    L[7, 2] = np.nan                    # invalid: non-finite
    L[8, 1] = -2.5                      # steep q law
    L[9, 2], L[9, 3] = 2.0, 92.0        # support covering the whole grid
    return L


def f64_tol(n_nodes, nb):
    return (n_nodes + nb + 128 + 1024) * U64


def f32_tol(n_nodes, nb):
    n_chunks = (nb + 31) // 32
    return f64_tol(n_nodes, nb) + (1 + 24 + 81 + 31 + n_chunks + 2) * U32


def check(got, ref, tol):
    lx, fl = got
    rx, rfl = ref
    np.testing.assert_array_equal(fl, rfl)
    fin = np.isfinite(rx)
    np.testing.assert_array_equal(np.isfinite(lx), fin)
    np.testing.assert_array_equal(lx[~fin], rx[~fin])
    d = np.abs(lx[fin] - rx[fin])
    assert d.max(initial=0.0) <= tol, (d.max(), tol)


def test_grid_f64_matches_oracle(B, ctx, oracle):
    m1, q, pdet = exact_grid()
    lam = special_lambdas()
    B.pop_load_vt_grid(ctx, m1, q, pdet)
    got = B.pop_xi_grid(ctx, lam, B.POP_MODE_F64)
    ref = oracle.xi_grid(m1, q, pdet, lam)
    check(got, ref, f64_tol(m1.size * q.size, 39))
    assert got[1][5] == B.POP_FLAG_ZERO_XI and got[1][6] == B.POP_FLAG_INVALID_LAMBDA
    assert got[1][7] == B.POP_FLAG_INVALID_LAMBDA and got[0][6] == 0.0


def test_grid_f32_matches_oracle(B, ctx, oracle):
    m1, q, pdet = exact_grid()
    lam = special_lambdas()
    B.pop_load_vt_grid(ctx, m1, q, pdet)
    got = B.pop_xi_grid(ctx, lam, B.POP_MODE_F32)
    ref = oracle.xi_grid(m1, q, pdet, lam)
    check(got, ref, f32_tol(m1.size * q.size, 39))


def test_grid_column_order_does_not_change_results(B, ctx):
    """Results are bit-identical whatever column the mmin sort gives a Lambda."""
    m1, q, pdet = exact_grid()
    lam = special_lambdas(300, seed=702)
    B.pop_load_vt_grid(ctx, m1, q, pdet)
    p = np.random.default_rng(3).permutation(len(lam))
    for mode in (B.POP_MODE_F64, B.POP_MODE_F32):
        a = B.pop_xi_grid(ctx, lam, mode)[0]
        b = B.pop_xi_grid(ctx, lam[p], mode)[0]
        np.testing.assert_array_equal(a[p], b)
        np.testing.assert_array_equal(a, B.pop_xi_grid(ctx, lam, mode)[0])


def test_grid_two_slices_and_uneven_batches(B, ctx, oracle):
    """K above one 8192-column slice, then smaller batches reusing the scratch (FP32: partial
    128-column tiles, several q parts of a 33-node axis, the per-slice work queues)."""
    from paper_1904_02863_gb300 import synth
    m1 = np.linspace(3.0, 100.0, 70)
    q = np.linspace(0.05, 1.0, 33)
    pdet = np.ascontiguousarray(synth.campaign_pdet(m1)[:, None] * np.ones((1, q.size)))
    B.pop_load_vt_grid(ctx, m1, q, pdet)
    lam = synth.make_lambdas(8192 + 77, 12, seed=703)
    ref = oracle.xi_grid(m1, q, pdet, lam)
    check(B.pop_xi_grid(ctx, lam, B.POP_MODE_F64), ref, f64_tol(m1.size * q.size, 33))
    check(B.pop_xi_grid(ctx, lam, B.POP_MODE_F32), ref, f32_tol(m1.size * q.size, 33))
    for K in (1, 63, 65, 127, 129, 1000):
        sub = (ref[0][:K], ref[1][:K])
        check(B.pop_xi_grid(ctx, lam[:K], B.POP_MODE_F64), sub, f64_tol(m1.size * q.size, 33))
        check(B.pop_xi_grid(ctx, lam[:K], B.POP_MODE_F32), sub, f32_tol(m1.size * q.size, 33))


def test_grid_from_device_tensors(B, ctx, oracle):
    import torch
    m1, q, pdet = exact_grid()
    B.pop_load_vt_grid(ctx, torch.from_numpy(m1).cuda(), torch.from_numpy(q).cuda(), torch.from_numpy(pdet).cuda())
    lam = special_lambdas(20, seed=704)
    check(B.pop_xi_grid(ctx, lam, B.POP_MODE_F64), oracle.xi_grid(m1, q, pdet, lam),
          f64_tol(m1.size * q.size, 39))


def test_grid_minimal_and_all_q_inside(B, ctx, oracle):
    m1 = np.array([4.0, 60.0])
    q = np.array([0.2, 1.0])
    pdet = np.array([[0.3, 0.9], [1.0, 0.5]])
    B.pop_load_vt_grid(ctx, m1, q, pdet)
    lam = special_lambdas(12, seed=705)
    check(B.pop_xi_grid(ctx, lam, B.POP_MODE_F64), oracle.xi_grid(m1, q, pdet, lam), f64_tol(4, 2))


def test_grid_load_errors(B, ctx):
    m1, q, pdet = exact_grid()
    bad_cases = [
        (m1[::-1].copy(), q, pdet),                       # not increasing
        (m1, np.r_[q[:3], q[2], q[4:]], pdet),            # repeated node
        (m1[:1], q, pdet[:1]),                            # one node
        (m1, q + 1.0, pdet),                              # no q <= 1
    ]
    for a, b, p in bad_cases:
        with pytest.raises(B.PopError) as e:
            B.pop_load_vt_grid(ctx, a, b, p)
        assert e.value.status == B.POP_EINVAL
    for v in (-0.1, np.nan, np.inf):
        p = pdet.copy()
        p[50, 10] = v
        with pytest.raises(B.PopError) as e:
            B.pop_load_vt_grid(ctx, m1, q, p)
        assert e.value.status == B.POP_EINVAL
    p = pdet.copy()
    p[50, 44] = np.nan  # at a node with q > 1: not used
    B.pop_load_vt_grid(ctx, m1, q, p)
    with pytest.raises(B.PopError) as e:
        B.pop_xi_grid(ctx, special_lambdas()[:3], B.POP_MODE_F32_SURROGATE)
    assert e.value.status == B.POP_EINVAL
    assert B.pop_xi_grid(ctx, np.zeros((0, 11)))[0].shape == (0,)


def test_loglik_with_grid_selection(B, oracle):
    """ln L = sum_i ln(S_i / n_i) - N ln xi_grid: the event part from the oracle's
    ln L + N ln xi (Monte Carlo), the selection part from its grid sum."""
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(12, np.array([1, 700, 4096, 4097, 300, 5000, 20, 900, 1000, 64, 4095, 8193]), 6,
                             seed=706)
    inj = synth.make_injections(20000, 6, seed=707)
    m1, q, pdet = synth.campaign_vt_grid(301, 97)
    lam = synth.make_lambdas(70, 11, seed=708)
    lam[5, 6] = -1.0
    r_lnL, r_lnxi, _, r_fl = oracle.loglik(cat, inj, lam)
    g_lnxi, g_fl = oracle.xi_grid(m1, q, pdet, lam)
    N = cat.n_events
    events = r_lnL + N * r_lnxi
    like = B.Likelihood(0)
    B.pop_load_events(like.ctx, cat.offsets, cat.theta, cat.prior)   # no injections needed
    B.pop_load_vt_grid(like.ctx, m1, q, pdet)
    with pytest.raises(B.PopError):
        B.pop_loglik(like.ctx, lam)          # the default source still wants injections
    B.pop_set_xi_source(like.ctx, B.POP_XI_GRID)
    lnL, lnxi, neff, fl = B.pop_loglik(like.ctx, lam, B.POP_MODE_F64)
    valid = (r_fl & B.POP_FLAG_INVALID_LAMBDA) == 0
    np.testing.assert_array_equal(fl[~valid], B.POP_FLAG_INVALID_LAMBDA)
    assert (fl[valid] & ~np.uint32(B.POP_FLAG_ZERO_EVENT) == 0).all()
    assert np.isinf(neff[valid]).all()
    fin = valid & np.isfinite(events)
    tolx = f64_tol(m1.size * q.size, q.size)
    np.testing.assert_allclose(lnxi[valid], g_lnxi[valid], rtol=0, atol=tolx)
    exp = events - N * g_lnxi
    tol = 1e-12 * (np.abs(events) + N * np.abs(g_lnxi)) + N * tolx + 1e-12
    assert (np.abs(lnL[fin] - exp[fin]) <= tol[fin]).all(), np.abs(lnL[fin] - exp[fin]).max()
    # FP32 mode through the same graph path: FP32 event weights (0.05 nats) and the FP32 grid sum.
    lnL32 = B.pop_loglik(like.ctx, lam, B.POP_MODE_F32)[0]
    assert np.max(np.abs(lnL32[fin] - exp[fin])) < 0.05
    # back to the injections
    B.pop_load_injections(like.ctx, inj.n_draw, inj.theta, inj.p_draw)
    B.pop_set_xi_source(like.ctx, B.POP_XI_INJECTIONS)
    lnL_mc = B.pop_loglik(like.ctx, lam, B.POP_MODE_F64)[0]
    np.testing.assert_allclose(lnL_mc[fin], r_lnL[fin], rtol=1e-11)
    like.close()


def test_dense_campaign_grid_sampled(B, ctx, oracle):
    """The dense 3001 x 801 campaign grid with K = 1024 Lambda in one call (the
    measured configuration), checked against the oracle on 6 sampled Lambda."""
    from paper_1904_02863_gb300 import synth
    m1, q, pdet = synth.campaign_vt_grid()
    lam = synth.make_lambdas(1024, 11, seed=709)
    B.pop_load_vt_grid(ctx, m1, q, pdet)
    pick = np.array([0, 1, 255, 512, 800, 1023])
    ref = oracle.xi_grid(m1, q, pdet, lam[pick])
    got64 = B.pop_xi_grid(ctx, lam, B.POP_MODE_F64)
    check((got64[0][pick], got64[1][pick]), ref, f64_tol(m1.size * q.size, q.size))
    got32 = B.pop_xi_grid(ctx, lam, B.POP_MODE_F32)
    check((got32[0][pick], got32[1][pick]), ref, f32_tol(m1.size * q.size, q.size))
    assert np.isfinite(got64[0]).all()
