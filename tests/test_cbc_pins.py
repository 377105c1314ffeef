"""Pins of the single-event CBC likelihood oracle (Eq. cbclike, Sec. "Single-event
Likelihood acceleration"):  ln L = sum_i sum_j [-ln(2 pi S_ij) - (2/T)|d_ij - h_ij|^2/S_ij],
h_ij = A e^{i phi} (Fp_i hp_j + Fc_i hc_j) e^{-2 pi i f_j dt_i}, T = 1/df.

Each pin rests on something other than the formula itself: a template equal to the
data, the statistics of Gaussian noise at the PSD (the 2/T normalisation), the sign
and period of the time shift, symmetries of the response, a hand-computed single
bin, the exact quadratic dependence on A, and the optimal-SNR identity."""
import numpy as np
import pytest

from paper_1904_02863_gb300 import synth


def response(c, th):
    f = c.f0 + c.df * np.arange(c.M)
    A, phi = th[0], th[1]
    out = []
    for i in range(c.n_det):
        Fp, Fc, dt = th[2 + 3 * i: 5 + 3 * i]
        out.append(A * np.exp(1j * phi) * (Fp * c.hp + Fc * c.hc) * np.exp(-2j * np.pi * f * dt))
    return np.stack(out)


def psd_term(c):
    return -np.sum(np.log(2 * np.pi * c.psd))


def test_template_equal_to_the_data_leaves_only_the_psd_term(oracle):
    c = synth.make_cbc(2048, seed=11)
    th = c.truth.copy()
    th[0], th[1] = 0.83, 0.4
    c.data = response(c, th)
    got = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th)[0]
    assert got == pytest.approx(psd_term(c), rel=1e-13)


def test_pure_noise_has_unit_mean_per_bin(oracle):
    """d = Gaussian noise with E|n|^2 = T S / 2 and h = 0: (2/T)|n|^2/S is exponential with
    mean 1, so ln L = sum ln(1/2 pi S) - (n_det M +- 5 sqrt(n_det M))."""
    c = synth.make_cbc(8192, seed=12, snr=0.0)
    th = c.truth.copy()
    th[0] = 0.0
    got = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th)[0]
    n = c.n_det * c.M
    assert abs((psd_term(c) - got) - n) < 5 * np.sqrt(n)


def test_time_shift_sign_and_period(oracle):
    """Data = the template moved by exp(-2 pi i f dt0): dt = dt0 reproduces it exactly, dt0 + T
    too (f0/df is an integer), and -dt0 does not."""
    c = synth.make_cbc(1024, n_det=2, seed=13)
    th = c.truth.copy()
    th[4], th[7] = 0.0123, -0.0071
    c.data = response(c, th)
    T = 1.0 / c.df
    assert (c.f0 / c.df).is_integer()
    at = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th)[0]
    shifted = th.copy()
    shifted[4] += T
    shifted[7] -= 2 * T
    flipped = th.copy()
    flipped[4], flipped[7] = -th[4], -th[7]
    per = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, np.stack([shifted, flipped]))
    assert at == pytest.approx(psd_term(c), rel=1e-13)
    assert per[0] == pytest.approx(at, rel=1e-10)
    assert per[1] < at - 1.0


def test_response_symmetries(oracle):
    c = synth.make_cbc(512, seed=14)
    th = synth.make_cbc_thetas(c, 3, seed=15)
    base = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th)
    neg = th.copy()
    neg[:, 0] *= -1
    neg[:, 1] += np.pi                       # -A e^{i(phi + pi)} = A e^{i phi}
    turn = th.copy()
    turn[:, 1] += 2 * np.pi
    swap = th.copy()
    for i in range(c.n_det):                 # (Fp, hp) <-> (Fc, hc)
        swap[:, 2 + 3 * i], swap[:, 3 + 3 * i] = th[:, 3 + 3 * i], th[:, 2 + 3 * i]
    np.testing.assert_allclose(oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, neg), base, rtol=1e-12)
    np.testing.assert_allclose(oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, turn), base, rtol=1e-12)
    np.testing.assert_allclose(oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hc, c.hp, swap), base, rtol=1e-12)


def test_single_bin_by_hand(oracle):
    """One detector, one bin: d = 0, S = 2, hp = 3 + 4i, Fp = 1, A = 0.5: |h|^2 = 6.25 whatever
    phi and dt, so ln L = -ln(4 pi) - (2 df) 6.25 / 2."""
    df = 0.25
    got = oracle.cbc_loglik(30.0, df, np.zeros((1, 1), complex), np.array([[2.0]]), np.array([3 + 4j]),
                            np.array([0j]), np.array([[0.5, 1.1, 1.0, 0.7, 0.013]]))[0]
    assert got == pytest.approx(-np.log(4 * np.pi) - 2 * df * 6.25 / 2, rel=1e-15)


def test_exactly_quadratic_in_the_amplitude(oracle):
    """ln L(A) = c0 + c1 A - c2 A^2: third differences vanish, and c2 = (2/T) sum |u|^2/S
    (steps of 300 in A, around the signal's amplitude, so the quadratic term dominates)."""
    c = synth.make_cbc(1024, seed=16)
    th = np.repeat(c.truth[None, :], 4, axis=0)
    step = 300.0
    th[:, 0] = step * np.arange(4)
    L = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th)
    d3 = L[3] - 3 * L[2] + 3 * L[1] - L[0]
    assert abs(d3) < 1e-12 * np.abs(L).sum()
    u = response(c, np.concatenate([[1.0], th[0, 1:]]))
    c2 = 2 * c.df * np.sum(np.abs(u) ** 2 / c.psd)
    assert -(L[2] - 2 * L[1] + L[0]) / (2 * step ** 2) == pytest.approx(c2, rel=1e-11)


def test_noise_averaged_log_likelihood_ratio_is_half_the_snr_squared(oracle):
    """d = h + n: ln L(h) - ln L(0) = sum (2/T)(2 Re(n* h) + |h|^2)/S has mean rho^2/2 and
    standard deviation rho, with rho^2 = sum 4 df |h|^2 / S (the optimal SNR)."""
    c = synth.make_cbc(4096, seed=17, snr=12.0)
    h = response(c, c.truth)
    rho2 = np.sum(4 * c.df * np.abs(h) ** 2 / c.psd)
    assert rho2 == pytest.approx(144.0, rel=1e-10)
    zero = c.truth.copy()
    zero[0] = 0.0
    L = oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, np.stack([c.truth, zero]))
    assert abs((L[0] - L[1]) - rho2 / 2) < 5 * np.sqrt(rho2)
