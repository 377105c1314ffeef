"""Seeded synthetic inputs for the population likelihood (Sec. "Population acceleration").

This module is shared by the tests, the benchmark and the checker.  It draws
numbers and knows the pdf of its OWN injection draw distribution (a property of
the synthetic injection campaign, as a real campaign ships ``p_draw`` with its
injections); it evaluates none of the population-model densities, none of the
per-Lambda normalisations and no part of the likelihood.

Stand-in for the paper's GWTC-1 posteriors (Sec. "Population acceleration"):
those samples are not available offline, so catalogs are synthesised with the
shapes of the paper's workload.

* Truths theta_i are drawn from the population at LAMBDA0.
* Posterior samples are theta_ij = clip(theta_i + eps), eps ~ N(0, diag(3, .1, .1, .1, .1, .1[, .1])),
  clipped to m1 in [5, 80], q in [5/m1, 1] (then nudged up by ulps until
  fl64(q*m1) >= 5), a in [0, 1], cos(tilt) in [-1, 1], z in [1e-3, 2].
* The single-event prior is pi = m1/4 (uniform in component masses, isotropic
  tilts), times 3 z^2 / 8 when redshift is present.
* Found injections are drawn from a broad draw distribution (power law 2.5 in m1
  on [3, 100], q uniform on [3/m1, 1], uniform spins and tilts, z ~ 3 z^2/8) and
  kept when sigmoid((m1 - 20)/5) > U(0, 1).

Single-event CBC workload (Sec. "Single-event Likelihood acceleration"): a
leading-order stationary-phase chirp as the template (no waveform library is
used), a smooth synthetic PSD in whitened units, per-detector antenna factors
and arrival-time offsets, Gaussian noise at the PSD, scaled to a target SNR.
Also the regular (m1, q) grid of the injection campaign for the grid VT.

Everything is a numpy ``Generator(PCG64(seed))`` stream.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Lambda layout at the C-ABI, in this order (11 parameters, 12 with kappa).
PARAMS = ("alpha", "beta", "mmin", "mmax", "lam", "mpp", "sigpp",
          "alpha_chi", "beta_chi", "xi_t", "sigma_t", "kappa")

# Truth population for the synthetic catalogs; kappa0 = 2.7 is a choice of this
# generator (the workload names none).
LAMBDA0 = np.array([2.3, 1.0, 5.0, 80.0, 0.1, 35.0, 4.0, 2.0, 5.0, 0.5, 0.5, 2.7])

# The injection draw distribution expressed as a point of the model family
# (lam = 0 and xi_t = 0 make mpp, sigpp, sigma_t irrelevant).
LAMBDA_DRAW = np.array([2.5, 0.0, 3.0, 100.0, 0.0, 35.0, 4.0, 1.0, 1.0, 0.0, 0.5, 1.0])

# Uniform prior box around LAMBDA0 for the Lambda batches.
LAMBDA_BOX = np.array([
    [1.5, 3.5], [0.0, 2.0], [4.0, 6.0], [70.0, 90.0], [0.0, 0.3], [28.0, 42.0],
    [2.0, 8.0], [1.0, 4.0], [2.0, 8.0], [0.0, 1.0], [0.1, 1.5], [0.0, 4.0]])

SEED_BASE = 1904_02863 * 10

# Draw-distribution constants (this generator's own campaign).
_DRAW_ALPHA, _DRAW_MLO, _DRAW_MHI = 2.5, 3.0, 100.0
_CLIP_MLO, _CLIP_MHI = 5.0, 80.0
_Z_LO = 1e-3


def seed_for(workload: int, stream: int = 0) -> int:
    """Seed of a numbered workload and sub-stream.

    Workloads: 1 FP64 10 x 1000, 2 FP64 catalog 1000 x 4096, 3 FP32 10 x 1000,
    4 ragged 2000 events with redshift, 5 surrogate with redshift, 6 single-event CBC.
    Sub-streams: 0 events or data, 1 injections, 2 Lambdas or parameter rows,
    3 ragged sample counts."""
    return SEED_BASE + workload + 1000 * stream


@dataclass
class Catalog:
    offsets: np.ndarray   # int64 [N+1], offsets[0] = 0
    theta: np.ndarray     # float64 [offsets[-1], n_dims]  (m1, q, a1, a2, c1, c2[, z])
    prior: np.ndarray     # float64 [offsets[-1]]  pi(theta) > 0

    @property
    def n_events(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_dims(self) -> int:
        return self.theta.shape[1]


@dataclass
class Injections:
    theta: np.ndarray     # float64 [n_found, n_dims]
    p_draw: np.ndarray    # float64 [n_found]
    n_draw: int           # found + missed

    @property
    def n_found(self) -> int:
        return self.theta.shape[0]


# --------------------------------------------------------------------------- sampling helpers
def _powerlaw_icdf(u, slope, lo, hi):
    """Inverse CDF of x^slope on [lo, hi] (lo, hi arrays or scalars)."""
    if slope == -1.0:
        return lo * np.exp(u * np.log(hi / lo))
    e = slope + 1.0
    a, b = lo ** e, hi ** e
    return (a + u * (b - a)) ** (1.0 / e)


def _truncnorm_draw(rng, n, mu, sigma, lo, hi):
    from scipy.special import ndtr, ndtri
    a, b = ndtr((lo - mu) / sigma), ndtr((hi - mu) / sigma)
    u = rng.random(n)
    return np.clip(mu + sigma * ndtri(a + u * (b - a)), lo, hi)


def _redshift_draw(rng, n, kappa):
    grid = np.linspace(0.0, 2.0, 20001)
    f = (1.0 + grid) ** (kappa - 1.0) * grid ** 2
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    return np.interp(rng.random(n), cdf, grid)


def draw_truths(rng, n, n_dims, lam=LAMBDA0):
    """n truths from the population at ``lam`` (inverse-CDF and library samplers)."""
    alpha, beta, mmin, mmax, mix, mpp, sigpp, ach, bch, xit, sigt = lam[:11]
    gauss = rng.random(n) < mix
    m1 = _powerlaw_icdf(rng.random(n), -alpha, mmin, mmax)
    m1[gauss] = _truncnorm_draw(rng, int(gauss.sum()), mpp, sigpp, mmin, mmax)
    q = _powerlaw_icdf(rng.random(n), beta, mmin / m1, 1.0)
    a1, a2 = rng.beta(ach, bch, n), rng.beta(ach, bch, n)
    aligned = rng.random(n) < xit
    c1, c2 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    na = int(aligned.sum())
    c1[aligned] = _truncnorm_draw(rng, na, 1.0, sigt, -1.0, 1.0)
    c2[aligned] = _truncnorm_draw(rng, na, 1.0, sigt, -1.0, 1.0)
    cols = [m1, q, a1, a2, c1, c2]
    if n_dims == 7:
        cols.append(_redshift_draw(rng, n, lam[11]))
    return np.stack(cols, axis=1)


def _nudge_q(q, m1, mlo):
    """Raise q by ulps until the fp64 product q*m1 is >= mlo (q stays <= 1)."""
    bad = q * m1 < mlo
    while bad.any():
        q[bad] = np.nextafter(q[bad], 2.0)
        bad = q * m1 < mlo
    return q


# --------------------------------------------------------------------------- public generators
def make_catalog(n_events, sizes, n_dims=6, seed=0, scatter=(3.0, 0.1)):
    """Synthetic posterior samples for ``n_events`` events.

    ``sizes`` is an int (dense: S samples per event) or an array of per-event counts.
    Returns a CSR ``Catalog``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.full(n_events, int(sizes), np.int64) if np.isscalar(sizes) else np.asarray(sizes, np.int64)
    offsets = np.zeros(n_events + 1, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    truths = draw_truths(rng, n_events, n_dims)
    total = int(offsets[-1])
    theta = np.repeat(truths, sizes, axis=0)
    sd = np.full(n_dims, scatter[1])
    sd[0] = scatter[0]
    theta += rng.standard_normal((total, n_dims)) * sd
    m1 = np.clip(theta[:, 0], _CLIP_MLO, _CLIP_MHI)
    q = np.clip(theta[:, 1], _CLIP_MLO / m1, 1.0)
    theta[:, 0], theta[:, 1] = m1, _nudge_q(q, m1, _CLIP_MLO)
    theta[:, 2:4] = np.clip(theta[:, 2:4], 0.0, 1.0)
    theta[:, 4:6] = np.clip(theta[:, 4:6], -1.0, 1.0)
    prior = theta[:, 0] / 4.0
    if n_dims == 7:
        theta[:, 6] = np.clip(theta[:, 6], _Z_LO, 2.0)
        prior = prior * (3.0 * theta[:, 6] ** 2 / 8.0)
    return Catalog(offsets, np.ascontiguousarray(theta), prior)


def draw_pdf(theta):
    """pdf of this generator's injection draw distribution at ``theta`` [n, d]."""
    m1 = theta[:, 0]
    a = _DRAW_ALPHA
    norm = (a - 1.0) / (_DRAW_MLO ** (1.0 - a) - _DRAW_MHI ** (1.0 - a))
    p = norm * m1 ** (-a)                       # m1 ~ m1^-2.5 on [3, 100]
    p = p / (1.0 - _DRAW_MLO / m1)              # q uniform on [3/m1, 1]
    p = p * 0.25                                # a1, a2 uniform; c1, c2 uniform on [-1, 1]
    if theta.shape[1] == 7:
        p = p * (3.0 * theta[:, 6] ** 2 / 8.0)  # z ~ 3 z^2 / 8 on [0, 2]
    return p


def draw_injections(rng, n, n_dims=6):
    """n draws from the injection draw distribution (before detection)."""
    m1 = _powerlaw_icdf(rng.random(n), -_DRAW_ALPHA, _DRAW_MLO, _DRAW_MHI)
    q = _DRAW_MLO / m1 + rng.random(n) * (1.0 - _DRAW_MLO / m1)
    q = _nudge_q(np.minimum(q, 1.0), m1, _DRAW_MLO)
    cols = [m1, q, rng.random(n), rng.random(n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)]
    if n_dims == 7:
        cols.append(2.0 * rng.random(n) ** (1.0 / 3.0))
    return np.stack(cols, axis=1)


def make_injections(n_draw, n_dims=6, seed=0, detect=True, block=1 << 20):
    """Found injections of ``n_draw`` draws; ``detect=False`` keeps every draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kept = []
    for start in range(0, n_draw, block):
        n = min(block, n_draw - start)
        th = draw_injections(rng, n, n_dims)
        if detect:
            u = rng.random(n)
            th = th[1.0 / (1.0 + np.exp(-(th[:, 0] - 20.0) / 5.0)) > u]
        kept.append(th)
    theta = np.ascontiguousarray(np.concatenate(kept))
    return Injections(theta, draw_pdf(theta), int(n_draw))


def make_lambdas(K, n_params=11, seed=0, box=LAMBDA_BOX):
    """K Lambda points drawn uniformly from ``box`` (row-major [K, n_params])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = box[:n_params, 0], box[:n_params, 1]
    return np.ascontiguousarray(lo + rng.random((K, n_params)) * (hi - lo))


def campaign_pdet(m1):
    """Detection probability of this generator's campaign: sigmoid((m1 - 20)/5), as in make_injections."""
    return 1.0 / (1.0 + np.exp(-(np.asarray(m1, np.float64) - 20.0) / 5.0))


def campaign_vt_grid(n_m1=3001, n_q=801, m1_range=(3.0, 100.0), q_range=(0.03, 1.0)):
    """Regular (m1, q) grid over the injection campaign's mass range: nodes and pdet [n_m1, n_q]."""
    m1 = np.linspace(m1_range[0], m1_range[1], n_m1)
    q = np.linspace(q_range[0], q_range[1], n_q)
    pdet = np.ascontiguousarray(np.broadcast_to(campaign_pdet(m1)[:, None], (n_m1, n_q)))
    return m1, q, pdet


# --------------------------------------------------------------------------- single-event CBC workload
@dataclass
class CbcData:
    f0: float             # first bin frequency (Hz)
    df: float             # bin spacing (Hz); the segment length is T = 1/df
    data: np.ndarray      # complex128 [n_det, M] strain data (whitened units)
    psd: np.ndarray       # float64 [n_det, M] one-sided noise power spectral density
    hp: np.ndarray        # complex128 [M] plus polarisation of the template
    hc: np.ndarray        # complex128 [M] cross polarisation
    truth: np.ndarray     # float64 [2 + 3 n_det] the signal's (A, phi, Fp_i, Fc_i, dt_i)

    @property
    def n_det(self) -> int:
        return self.psd.shape[0]

    @property
    def M(self) -> int:
        return self.psd.shape[1]


def cbc_psd(f, scale=1.0, f_knee=150.0):
    """A smooth synthetic noise curve: steep low-frequency wall, flat bucket, rising high end."""
    x = np.asarray(f, np.float64) / f_knee
    return scale * (x ** -4.0 + 2.0 + 2.0 * x * x)


def cbc_chirp(f, chirp_mass_s=5.9e-6, t_c=0.0, phi_c=0.0, cos_iota=0.6):
    """Leading-order stationary-phase chirp (unit amplitude scale): hp = f^(-7/6) (1 + cos^2 iota)/2 e^{i Psi},
    hc = -i cos(iota) f^(-7/6) e^{i Psi}, Psi = 2 pi f t_c - phi_c - pi/4 + (3/128) (pi Mc f)^(-5/3)."""
    f = np.asarray(f, np.float64)
    psi = 2.0 * np.pi * f * t_c - phi_c - np.pi / 4 + 3.0 / 128.0 * (np.pi * chirp_mass_s * f) ** (-5.0 / 3.0)
    base = f ** (-7.0 / 6.0) * np.exp(1j * psi)
    return base * (1.0 + cos_iota ** 2) / 2.0, -1j * cos_iota * base


def make_cbc(M=4096, n_det=3, T=4.0, f0=20.0, snr=20.0, seed=0):
    """Synthetic single-event data: the chirp seen by n_det detectors (own antenna factors
    and arrival-time offsets) plus Gaussian noise at the synthetic PSD, M bins from f0 in
    steps of 1/T, signal scaled to the given network SNR."""
    rng = np.random.Generator(np.random.PCG64(seed))
    df = 1.0 / T
    f = f0 + df * np.arange(M)
    hp, hc = cbc_chirp(f)
    psd = np.stack([cbc_psd(f, scale=1.0 + 0.3 * i) for i in range(n_det)])
    Fp = rng.uniform(-0.8, 0.8, n_det)
    Fc = rng.uniform(-0.8, 0.8, n_det)
    dt = rng.uniform(-0.02, 0.02, n_det)
    resp = (Fp[:, None] * hp[None, :] + Fc[:, None] * hc[None, :]) * np.exp(-2j * np.pi * f[None, :] * dt[:, None])
    rho2 = float(np.sum(4.0 * df * np.abs(resp) ** 2 / psd))
    A = snr / np.sqrt(rho2)
    sig = np.sqrt(T * psd / 4.0)   # each of Re, Im: E|n|^2 = T S / 2
    noise = sig * (rng.standard_normal((n_det, M)) + 1j * rng.standard_normal((n_det, M)))
    data = A * resp + noise
    truth = np.concatenate([[A, 0.0], np.stack([Fp, Fc, dt], axis=1).ravel()])
    return CbcData(f0, df, np.ascontiguousarray(data), np.ascontiguousarray(psd), hp, hc, truth)


def make_cbc_thetas(cbc, K, seed=0):
    """K parameter rows scattered around the truth (amplitude +-30%, phase +-0.5, antenna +-0.2, time +-1 ms)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = cbc.n_det
    th = np.repeat(cbc.truth[None, :], K, axis=0)
    th[:, 0] *= rng.uniform(0.7, 1.3, K)
    th[:, 1] += rng.uniform(-0.5, 0.5, K)
    for i in range(n):
        th[:, 2 + 3 * i] += rng.uniform(-0.2, 0.2, K)
        th[:, 3 + 3 * i] += rng.uniform(-0.2, 0.2, K)
        th[:, 4 + 3 * i] += rng.uniform(-1e-3, 1e-3, K)
    if K:
        th[0] = cbc.truth
    return np.ascontiguousarray(th)


def round_to_f32(x):
    """Storage quantisation of the FP32 layout: values rounded to float32, promoted back."""
    return np.asarray(x, np.float32).astype(np.float64)


# --------------------------------------------------------------------------- workload presets
WORKLOADS = {
    # name: seed_id (the seed_for workload number), n_events, sizes, n_dims, n_draw, K, storage
    "f64_10x1000_inj1e5": dict(seed_id=1, n_events=10, sizes=1000, n_dims=6, n_draw=10**5, K=100, storage="f64"),
    "f64_catalog_1000x4096_inj1e7": dict(seed_id=2, n_events=1000, sizes=4096, n_dims=6, n_draw=10**7, K=1024, storage="f64"),
    "f32_10x1000_inj1e5": dict(seed_id=3, n_events=10, sizes=1000, n_dims=6, n_draw=10**5, K=1024, storage="f32"),
    "f32_ragged2000_s500to16000_z": dict(seed_id=4, n_events=2000, sizes=(500, 16000), n_dims=7, n_draw=18 * 10**6,
                        K=(64, 200, 1000, 4096), storage="f32"),
    "f32_z_10x1000_inj1e5_surrogate": dict(seed_id=5, n_events=10, sizes=1000, n_dims=7, n_draw=10**5, K=1024, storage="f32"),
}


def make_workload(name, scale=1.0):
    """Catalog, injections and a Lambda batch of a named workload.

    ``scale`` < 1 shrinks the event count and the draw count (parity cases).
    """
    w = WORKLOADS[name]
    cfg = w["seed_id"]
    n_events = max(1, int(round(w["n_events"] * scale)))
    sizes = w["sizes"]
    if isinstance(sizes, tuple):
        rng = np.random.Generator(np.random.PCG64(seed_for(cfg, 3)))
        sizes = rng.integers(sizes[0], sizes[1] + 1, n_events)
    cat = make_catalog(n_events, sizes, w["n_dims"], seed=seed_for(cfg, 0))
    inj = make_injections(max(1000, int(w["n_draw"] * scale)), w["n_dims"], seed=seed_for(cfg, 1))
    K = w["K"] if np.isscalar(w["K"]) else max(w["K"])
    lam = make_lambdas(K, 11 + (w["n_dims"] == 7), seed=seed_for(cfg, 2))
    return cat, inj, lam
