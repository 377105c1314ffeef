"""GPU parity on the degenerate shapes of the recycled likelihood (Eq. poplike, with the
Monte Carlo selection term of Sec. "Population acceleration"), in every mode.

* an empty Lambda batch (K = 0), then a one-row batch, in each mode;
* a catalog of one-sample events beside one event of many chunks;
* a single found injection, and a campaign where every draw was found (n_found = n_draw).

FP64 and float-float: the FP64 parity bar (1e-12 of |sum_i ln(S_i/n_i)| + N |ln xi|,
flags identical); FP32: 0.05 nats against the oracle, flags identical.
"""
import numpy as np
import pytest

from test_parity_gpu import assert_f64_parity

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


def check_all_modes(B, like, cat, inj, lam, oracle):
    ref = oracle.loglik(cat, inj, lam)
    assert_f64_parity(like(lam, B.POP_MODE_F64), ref, cat.n_events)
    assert_f64_parity(like(lam, B.POP_MODE_FF), ref, cat.n_events)
    ref32 = ref
    got32 = like(lam, B.POP_MODE_F32)
    np.testing.assert_array_equal(got32[3], ref32[3])
    fin = np.isfinite(ref32[0])
    np.testing.assert_array_equal(np.isfinite(got32[0]), fin)
    d = np.abs(got32[0][fin] - ref32[0][fin])
    assert d.size == 0 or d.max() <= 0.05, d.max()


def test_empty_then_one_row_batch_every_mode(B, oracle):
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(4, 1500, 6, seed=611)
    inj = synth.make_injections(20000, 6, seed=612)
    lam = synth.make_lambdas(1, 11, seed=613)
    like = B.Likelihood(0).load(cat, inj)
    for mode in (B.POP_MODE_F64, B.POP_MODE_F32, B.POP_MODE_FF):
        out = like(lam[:0], mode)
        assert all(o.shape == (0,) for o in out), mode
    check_all_modes(B, like, cat, inj, lam, oracle)
    like.close()


def test_one_sample_events_beside_a_long_event(B, oracle):
    """300 events of one sample each and one event of 3 chunks + a tail: per-event sums of a
    single weight, and a segmented sum that crosses many work items."""
    from paper_1904_02863_gb300 import synth
    sizes = np.ones(301, np.int64)
    sizes[150] = 3 * 4096 + 77
    cat = synth.make_catalog(len(sizes), sizes, 6, seed=621)
    # Spin magnitudes clipped to exactly 0 or 1 have zero Beta density when alpha_chi or
    # beta_chi > 1; keep them inside so that one-sample events do not vanish (pi has no spin term).
    cat.theta[:, 2:4] = np.clip(cat.theta[:, 2:4], 0.02, 0.98)
    inj = synth.make_injections(30000, 6, seed=622)
    lam = synth.make_lambdas(41, 11, seed=623)
    # Most rows keep every one-sample event inside the mass support (mmin < 5 <= m2,
    # m1 <= 80 <= mmax), so ln L stays finite; the last rows keep the box's own edges.
    rng = np.random.Generator(np.random.PCG64(624))
    lam[:33, 2] = rng.uniform(4.0, 4.99, 33)
    lam[:33, 3] = rng.uniform(80.0, 90.0, 33)
    like = B.Likelihood(0).load(cat, inj)
    check_all_modes(B, like, cat, inj, lam, oracle)
    assert np.isfinite(like(lam[:33], B.POP_MODE_F64)[0]).all()
    like.close()


def test_single_found_injection(B, oracle):
    """xi from one injection in the bulk of every support of the Lambda box: xi = w / n_draw."""
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(5, 900, 6, seed=631)
    inj = synth.Injections(np.array([[30.0, 0.8, 0.3, 0.6, 0.2, -0.4]]), np.array([2.5e-3]), 1000)
    lam = synth.make_lambdas(23, 11, seed=633)
    like = B.Likelihood(0).load(cat, inj)
    check_all_modes(B, like, cat, inj, lam, oracle)
    like.close()


def test_every_draw_found(B, oracle):
    """n_found = n_draw: the campaign's estimator without missed draws."""
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(6, 1200, 6, seed=641)
    inj = synth.make_injections(40000, 6, seed=642)
    inj = synth.Injections(inj.theta, inj.p_draw, inj.n_found)
    lam = synth.make_lambdas(19, 11, seed=643)
    like = B.Likelihood(0).load(cat, inj)
    check_all_modes(B, like, cat, inj, lam, oracle)
    like.close()


@pytest.mark.parametrize("n_dims", [6, 7])
def test_unit_weights_when_the_prior_is_the_population(B, oracle, n_dims):
    """pi(theta) := p(theta | Lambda*) from the oracle makes every GPU weight p_GPU / p_oracle; at
    Lambda* each is 1 up to rounding, so ln L(Lambda*) = -N ln xi(Lambda*): FP64 and float-float to
    N * 1e-13 (per-sample agreement of the two densities), FP32 to N * 2e-5 (its per-weight
    budget).  Lambda* has mmin below the samples' clip at 5 and uniform spins, so every sample
    is inside the support."""
    from paper_1904_02863_gb300 import synth
    L = np.array([2.3, 1.0, 4.9, 80.0, 0.1, 35.0, 4.0, 1.0, 1.0, 0.5, 0.5, 2.7])[:11 + (n_dims == 7)]
    cat = synth.make_catalog(40, np.arange(40) * 97 % 5000 + 1, n_dims, seed=661 + n_dims)
    inj = synth.make_injections(50000, n_dims, seed=663 + n_dims)
    N = cat.n_events
    for mode, theta, tol in ((B.POP_MODE_F64, cat.theta, 1e-13), (B.POP_MODE_FF, cat.theta, 1e-13),
                             (B.POP_MODE_F32, cat.theta, 2e-5)):
        prior = np.array([oracle.p_theta(t, L) for t in theta])
        assert (prior > 0).all()
        c = synth.Catalog(cat.offsets, theta, prior)
        like = B.Likelihood(0).load(c, inj)
        lnL, lnxi, _, flags = like(L[None, :], mode)
        like.close()
        assert flags[0] & ~np.uint32(B.POP_FLAG_LOW_NEFF) == 0, (mode, flags)
        assert abs(lnL[0] + N * lnxi[0]) <= tol * N * (1 + abs(lnxi[0])), (mode, lnL[0] + N * lnxi[0])


def test_f32_upper_mass_edge_is_decided_in_fp64(B, oracle):
    """FP32 mode keeps m1 <= mmax exactly as the oracle does, also where m1 and mmax round to the
    same float or to neighbouring ones: one-sample events at m1 = mmax, its FP64 neighbours, the
    floats below and above mmax and the midpoint between them, against mmax that is not a float,
    is a float, and is that midpoint.  Each such event is in or out of the support (ZERO_EVENT)
    exactly as the oracle says, and ln L stays within the FP32 budget."""
    from paper_1904_02863_gb300 import synth
    def up(x):
        return float(np.nextafter(x, np.inf))

    def dn(x):
        return float(np.nextafter(x, -np.inf))

    base = 70.3                                   # not a float
    hi32 = float(np.float32(base))                # rounds up: the float above 70.3
    assert hi32 > base
    lo32 = float(np.nextafter(np.float32(hi32), np.float32(0)))   # the float below 70.3
    mid = 0.5 * (lo32 + hi32)                     # where rounding to float changes
    m1s = [base, up(base), dn(base), up(up(base)), lo32, up(lo32), dn(lo32), hi32, dn(hi32), up(hi32), mid, up(mid),
           dn(mid), 30.0]
    theta = np.array([[m, 0.9, 0.3, 0.4, 0.2, 0.5] for m in m1s])
    # one event per value, then one event holding all of them
    theta = np.concatenate([theta, theta])
    n = len(m1s)
    offsets = np.concatenate([np.arange(n + 1), [2 * n]]).astype(np.int64)
    cat = synth.Catalog(offsets, theta, theta[:, 0] / 4.0)
    inj = synth.make_injections(30000, 6, seed=671)
    rows = []
    for mmax in (base, lo32, hi32, mid, up(mid), dn(base)):
        L = synth.LAMBDA0[:11].copy()
        L[3] = mmax
        rows.append(L)
    lam = np.array(rows)
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F32)
    got = like(lam, B.POP_MODE_F32)
    ref = oracle.loglik(cat, inj, lam)
    like.close()
    np.testing.assert_array_equal(got[3], ref[3])
    assert (ref[3] & B.POP_FLAG_ZERO_EVENT).all()   # the one-sample events above mmax are empty
    # per-event agreement: the same rows evaluated on each event alone
    for i in range(n):
        sub = synth.Catalog(np.array([0, 1], np.int64), theta[i:i + 1], cat.prior[i:i + 1])
        like = B.Likelihood(0).load(sub, inj, storage=B.POP_STORE_F32)
        g = like(lam, B.POP_MODE_F32)
        like.close()
        r = oracle.loglik(sub, inj, lam)
        np.testing.assert_array_equal(g[3], r[3])
        fin = np.isfinite(r[0])
        np.testing.assert_array_equal(np.isfinite(g[0]), fin)
        assert np.all(np.abs(g[0][fin] - r[0][fin]) <= 1e-3), (m1s[i], g[0] - r[0])
