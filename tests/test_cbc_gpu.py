"""GPU parity of the single-event CBC likelihood (through the C-ABI) against the oracle's
direct evaluation of Eq. (cbclike).

Tolerances follow from the arithmetic.  The oracle adds n = n_det M terms in order,
so its sum is within n u sum|t| of the exact sum of its terms (u = 2^-53,
t_ij = -ln(2 pi S) - w |d - h|^2, w = (2/T)/S); the GPU adds the same quantities
regrouped (data constants, template norms, the time-shifted sums), each within
the same kind of bound, and its exponentials (an exact phase every 32 bins, then
the recurrence e <- e w: 31 products of ~3 u each) are within ~100 u.
FP64: |d ln L| <= (n + 300) u sum|t|.

FP32 mode: the time-shifted sums SP = sum_j P_j e_j, SQ = sum_j Q_j e_j run in FP32
(P = w conj(d) hp, Q = w conj(d) hc rounded to FP32; e_j from the hardware sine and
cosine of the exact phase on [-pi, pi), within 2^-21.19 absolute plus the rounding of
the phase to FP32, ~8 u32, then up to 15 FP32 complex products (an anchor every 16
bins), ~3 u32 each; an FP32 running sum per thread of at most CB / 256 bins, then 5
shuffle levels).  Every term P_j e_j carries at most eps = (8 + 45 + 8 + n_acc + 5 + 4) u32
of |P_j| (n_acc = the bins a thread adds), and ln L takes 2 Re(alpha SP + beta SQ), so
|d ln L| <= FP64 bound + 2 sum_i (|alpha_i| E_P,i + |beta_i| E_Q,i) eps,
E_P,i = sum_j |P_ij| (E_Q likewise).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24
RUN32 = 16   # bins per exact phase in FP32 (the library's FP32 run length)


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


def response(c, th):
    f = c.f0 + c.df * np.arange(c.M)
    out = []
    for i in range(c.n_det):
        Fp, Fc, dt = th[2 + 3 * i: 5 + 3 * i]
        out.append(th[0] * np.exp(1j * th[1]) * (Fp * c.hp + Fc * c.hc) * np.exp(-2j * np.pi * f * dt))
    return np.stack(out)


def bounds(c, th, n_acc):
    """(FP64 bound, FP32 bound) on |d ln L| for each row of th."""
    w = 2 * c.df / c.psd
    n = c.n_det * c.M
    EP = np.sum(w * np.abs(c.data) * np.abs(c.hp)[None, :], axis=1)
    EQ = np.sum(w * np.abs(c.data) * np.abs(c.hc)[None, :], axis=1)
    eps = (8 + 3 * (RUN32 - 1) + 8 + n_acc + 5 + 4) * U32
    b64, b32 = [], []
    for t in th:
        h = response(c, t)
        s = np.sum(np.abs(np.log(2 * np.pi * c.psd)) + w * (np.abs(c.data) + np.abs(h)) ** 2)
        b64.append((n + 300) * U64 * s)
        amp = abs(t[0])
        al = amp * np.abs(t[2::3][: c.n_det])
        be = amp * np.abs(t[3::3][: c.n_det])
        b32.append(b64[-1] + 2 * np.sum(al * EP + be * EQ) * eps)
    return np.array(b64), np.array(b32)


def run_both(B, ctx, oracle, c, th):
    B.pop_cbc_load(ctx, c.f0, c.df, c.data, c.psd, c.hp, c.hc)
    ref = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th)
    g64, f64 = B.pop_cbc_loglik(ctx, th, B.POP_MODE_F64)
    g32, f32 = B.pop_cbc_loglik(ctx, th, B.POP_MODE_F32)
    assert (f64 == 0).all() and (f32 == 0).all()
    return ref, g64, g32


def test_cbc_parity_ragged(B, ctx, oracle):
    """M = 5003 (not a multiple of the runs), 3 detectors, K = 37 (not a multiple of any tile)."""
    from paper_1904_02863_gb300 import synth
    c = synth.make_cbc(5003, seed=901)
    th = synth.make_cbc_thetas(c, 37, seed=902)
    ref, g64, g32 = run_both(B, ctx, oracle, c, th)
    b64, b32 = bounds(c, th, n_acc=8 * 4)
    assert (np.abs(g64 - ref) <= b64).all(), (np.abs(g64 - ref).max(), b64.min())
    assert (np.abs(g32 - ref) <= b32).all(), (np.abs(g32 - ref).max(), b32.min())


def test_cbc_single_bin_single_detector(B, ctx, oracle):
    from paper_1904_02863_gb300 import synth
    c = synth.make_cbc(1, n_det=1, seed=903)
    th = synth.make_cbc_thetas(c, 5, seed=904)
    ref, g64, g32 = run_both(B, ctx, oracle, c, th)
    b64, b32 = bounds(c, th, n_acc=1)
    assert (np.abs(g64 - ref) <= b64).all(), (np.abs(g64 - ref), b64)
    assert (np.abs(g32 - ref) <= b32).all(), (np.abs(g32 - ref), b32)


def test_cbc_time_shift_period_and_large_shifts(B, ctx, oracle):
    """dt + T (f0 / df an integer) leaves ln L unchanged; large dt keep full phase accuracy."""
    from paper_1904_02863_gb300 import synth
    c = synth.make_cbc(4096, seed=905)
    th = synth.make_cbc_thetas(c, 8, seed=906)
    T = 1.0 / c.df
    far = th.copy()
    far[:, 4::3] += 37 * T
    B.pop_cbc_load(ctx, c.f0, c.df, c.data, c.psd, c.hp, c.hc)
    a = B.pop_cbc_loglik(ctx, th, B.POP_MODE_F64)[0]
    b = B.pop_cbc_loglik(ctx, far, B.POP_MODE_F64)[0]
    ref = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th)
    b64, _ = bounds(c, th, n_acc=8)
    assert (np.abs(b - a) <= 2 * b64).all()
    assert (np.abs(a - ref) <= b64).all()


def test_cbc_bns_length_sampled(B, ctx, oracle):
    """M = 2^18 bins (128 s from 20 Hz to 2068 Hz), 3 detectors, K = 256 rows in one call (the
    measured configuration), checked against the oracle on 4 sampled rows."""
    from paper_1904_02863_gb300 import synth
    c = synth.make_cbc(2 ** 18, T=128.0, seed=907)
    th = synth.make_cbc_thetas(c, 256, seed=908)
    B.pop_cbc_load(ctx, c.f0, c.df, c.data, c.psd, c.hp, c.hc)
    g64 = B.pop_cbc_loglik(ctx, th, B.POP_MODE_F64)[0]
    g32 = B.pop_cbc_loglik(ctx, th, B.POP_MODE_F32)[0]
    pick = np.array([0, 1, 128, 255])
    ref = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th[pick])
    b64, b32 = bounds(c, th[pick], n_acc=8 * 16)
    assert (np.abs(g64[pick] - ref) <= b64).all(), (np.abs(g64[pick] - ref), b64)
    assert (np.abs(g32[pick] - ref) <= b32).all(), (np.abs(g32[pick] - ref), b32)
    assert np.argmax(g64) == 0 and np.argmax(g32) == 0   # the truth row is the best of the batch


def test_cbc_invalid_rows_and_errors(B, ctx):
    from paper_1904_02863_gb300 import synth
    c = synth.make_cbc(300, seed=909)
    th = synth.make_cbc_thetas(c, 6, seed=910)
    th[2, 4] = np.nan
    th[4, 0] = np.inf
    with pytest.raises(B.PopError) as e:
        B.pop_cbc_loglik(ctx, th)
    assert e.value.status == B.POP_ESTATE
    B.pop_cbc_load(ctx, c.f0, c.df, c.data, c.psd, c.hp, c.hc)
    lnL, fl = B.pop_cbc_loglik(ctx, th)
    assert fl[2] == B.POP_FLAG_INVALID_LAMBDA and fl[4] == B.POP_FLAG_INVALID_LAMBDA
    assert np.isneginf(lnL[[2, 4]]).all() and np.isfinite(np.delete(lnL, [2, 4])).all()
    with pytest.raises(B.PopError) as e:
        B.pop_cbc_loglik(ctx, th[:, :-1])
    assert e.value.status == B.POP_EINVAL
    bad = c.psd.copy()
    bad[1, 7] = 0.0
    with pytest.raises(B.PopError) as e:
        B.pop_cbc_load(ctx, c.f0, c.df, c.data, bad, c.hp, c.hc)
    assert e.value.status == B.POP_EINVAL
    d = c.data.copy()
    d[0, 3] = np.nan
    with pytest.raises(B.PopError) as e:
        B.pop_cbc_load(ctx, c.f0, c.df, d, c.psd, c.hp, c.hc)
    # the earlier data stay loaded after a failed load
    np.testing.assert_array_equal(B.pop_cbc_loglik(ctx, th)[0], lnL)
