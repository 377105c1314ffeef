/*
 * Plain, slow FP64 CPU oracle of the population likelihood.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load this library.  The GPU
 * library shares no code, header, table or constant with this file.
 *
 * What it computes (paper, Sec. "Population acceleration"):
 *
 *   ln L(Lambda) = sum_i ln[ (1/n_i) sum_j p(theta_ij | Lambda) / pi(theta_ij) ]
 *                  - N ln xi(Lambda)
 *
 * The product over events of sums of reweighted posterior samples is the
 * "recycling" estimate of Eq. (poplike).  The -N ln xi term is what the rate
 * factor R^N exp(-R VT) of the first equation of that section leaves after R is
 * marginalised under a 1/R prior: int R^(N-1) exp(-R VT) dR = Gamma(N) VT^-N,
 * with VT proportional to xi.  The 1/n_i factor (a mean instead of the paper's
 * plain sum) only shifts ln L by a Lambda-independent constant.
 *
 * The selection term is the Monte Carlo integral over found injections that
 * the same section mentions (its cost grows with the number of events):
 *   xi(Lambda) = (1/N_draw) sum_{k found} p(theta_k | Lambda) / p_draw(theta_k).
 *
 * The population density p(theta|Lambda) (the section cites the mass, spin
 * magnitude and spin orientation models without writing them out) is the
 * product of
 *   p(m1)      = (1-lam) PL(m1; -alpha, mmin, mmax) + lam N_T(m1; mpp, sigpp, [mmin, mmax])
 *   p(q | m1)  = (1+beta) q^beta / (1 - (mmin/m1)^(1+beta))   on q in [mmin/m1, 1]
 *   p(a)       = Beta(a; alpha_chi, beta_chi) for a1 and a2
 *   p(c1, c2)  = (1-xi_t)/4 + xi_t G(c1) G(c2), G = normal(1, sigma_t) truncated to [-1, 1]
 *   p(z)       = (1+z)^(kappa-1) z^2 / I(kappa) on [0, 2], I by a 1024-node trapezoid
 * Support is closed except mmin < m1 (m1 = mmin would leave q a single point);
 * the q test is fl64(q*m1) >= mmin.
 *
 * Every density is evaluated directly per sample with libm (pow, exp, log,
 * erf, lgamma, expm1).  There is no blocking, fusion or reordering.
 *
 * Also here: the gradient of ln L with respect to Lambda (from the analytic
 * score of each density), the selection term on a regular (m1, q) grid, the
 * additive parts of ln L for split catalogs, and the single-event CBC
 * likelihood of the paper's Sec. "Single-event Likelihood acceleration" (each
 * at its function).
 * It is built with -ffp-contract=off so that q*m1 rounds once, as stated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Result flags (bit values are the library's public interface). */
#define OR_FLAG_INVALID_LAMBDA 1u
#define OR_FLAG_ZERO_EVENT 2u
#define OR_FLAG_LOW_NEFF 4u
#define OR_FLAG_ZERO_XI 32u

/* Lambda indices, in the order of the C-ABI. */
enum { P_ALPHA, P_BETA, P_MMIN, P_MMAX, P_LAM, P_MPP, P_SIGPP, P_ACHI, P_BCHI, P_XIT, P_SIGT, P_KAPPA };

static const double SQRT2 = 1.4142135623730950488;
static const double SQRT2PI = 2.5066282746310005024;

/* Validity of a Lambda point (outside it ln L = -inf, flagged). */
int pop_oracle_lambda_valid(const double* L, int n_params)
{
    for (int p = 0; p < n_params; ++p)
        if (!isfinite(L[p])) return 0;
    if (!(L[P_MMIN] > 0.0) || !(L[P_MMIN] < L[P_MMAX])) return 0;
    if (!(L[P_LAM] >= 0.0 && L[P_LAM] <= 1.0)) return 0;
    if (!(L[P_SIGPP] > 0.0) || !(L[P_SIGT] > 0.0)) return 0;
    if (!(L[P_ACHI] > 0.0) || !(L[P_BCHI] > 0.0)) return 0;
    if (!(L[P_XIT] >= 0.0 && L[P_XIT] <= 1.0)) return 0;
    return 1;
}

/* Power law x^-alpha normalised on [a, b]; the alpha = 1 limit is 1/(x ln(b/a)). */
static double powerlaw_pdf(double x, double alpha, double a, double b)
{
    if (alpha == 1.0) return 1.0 / (x * log(b / a));
    return pow(x, -alpha) * (1.0 - alpha) / (pow(b, 1.0 - alpha) - pow(a, 1.0 - alpha));
}

/* Normal(mu, sigma) truncated to [a, b]; normalisation by erf. */
static double truncnorm_pdf(double x, double mu, double sigma, double a, double b)
{
    double z = 0.5 * (erf((b - mu) / (SQRT2 * sigma)) - erf((a - mu) / (SQRT2 * sigma)));
    double g = exp(-0.5 * (x - mu) * (x - mu) / (sigma * sigma)) / (SQRT2PI * sigma);
    return g / z;
}

/* Primary mass density on mmin < m1 <= mmax. */
double pop_oracle_p_m1(double m1, const double* L)
{
    double mmin = L[P_MMIN], mmax = L[P_MMAX], lam = L[P_LAM];
    if (!(m1 > mmin && m1 <= mmax)) return 0.0;
    double pl = powerlaw_pdf(m1, L[P_ALPHA], mmin, mmax);
    double pp = lam > 0.0 ? truncnorm_pdf(m1, L[P_MPP], L[P_SIGPP], mmin, mmax) : 0.0;
    return (1.0 - lam) * pl + lam * pp;
}

/* Mass-ratio density q^beta on [mmin/m1, 1].  The normalisation
 * 1 - (mmin/m1)^(1+beta) is evaluated as -expm1((1+beta) ln(mmin/m1)) with
 * ln(mmin/m1) = log1p((mmin - m1)/m1): the same numbers without cancellation
 * (mmin - m1 is exact when m1 is near mmin, where the density is largest);
 * beta = -1 is the 1/(q ln(m1/mmin)) limit. */
double pop_oracle_p_q(double q, double m1, const double* L)
{
    double beta = L[P_BETA], mmin = L[P_MMIN];
    if (!(q * m1 >= mmin && q <= 1.0)) return 0.0;
    double ln_ratio = log1p((mmin - m1) / m1);
    if (beta == -1.0) return 1.0 / (q * -ln_ratio);
    double norm = -expm1((1.0 + beta) * ln_ratio);
    return (1.0 + beta) * pow(q, beta) / norm;
}

/* Beta(alpha_chi, beta_chi) density of one spin magnitude (pow: 0^0 = 1). */
double pop_oracle_p_chi(double a, const double* L)
{
    double ac = L[P_ACHI], bc = L[P_BCHI];
    if (!(a >= 0.0 && a <= 1.0)) return 0.0;
    double lnB = lgamma(ac) + lgamma(bc) - lgamma(ac + bc);
    return pow(a, ac - 1.0) * pow(1.0 - a, bc - 1.0) / exp(lnB);
}

/* Aligned/isotropic tilt mixture of the two cosines. */
double pop_oracle_p_tilt(double c1, double c2, const double* L)
{
    double xit = L[P_XIT], sig = L[P_SIGT];
    if (!(c1 >= -1.0 && c1 <= 1.0 && c2 >= -1.0 && c2 <= 1.0)) return 0.0;
    double g1 = truncnorm_pdf(c1, 1.0, sig, -1.0, 1.0);
    double g2 = truncnorm_pdf(c2, 1.0, sig, -1.0, 1.0);
    return (1.0 - xit) / 4.0 + xit * g1 * g2;
}

/* Trapezoid rule for (1+z)^(kappa-1) z^2 on 1024 equispaced nodes of [0, 2]. */
double pop_oracle_z_norm(double kappa)
{
    const int n = 1024;
    double h = 2.0 / (n - 1), s = 0.0;
    for (int k = 0; k < n; ++k) {
        double z = 2.0 * k / (n - 1);
        double f = pow(1.0 + z, kappa - 1.0) * z * z;
        s += (k == 0 || k == n - 1) ? 0.5 * f : f;
    }
    return s * h;
}

double pop_oracle_p_z(double z, const double* L)
{
    if (!(z >= 0.0 && z <= 2.0)) return 0.0;
    return pow(1.0 + z, L[P_KAPPA] - 1.0) * z * z / pop_oracle_z_norm(L[P_KAPPA]);
}

/* p(theta | Lambda) for one sample (n_dims 6: m1,q,a1,a2,c1,c2; 7 adds z). */
double pop_oracle_p_theta(const double* th, int n_dims, const double* L)
{
    double p = pop_oracle_p_m1(th[0], L);
    if (p == 0.0) return 0.0;
    p *= pop_oracle_p_q(th[1], th[0], L);
    p *= pop_oracle_p_chi(th[2], L) * pop_oracle_p_chi(th[3], L);
    p *= pop_oracle_p_tilt(th[4], th[5], L);
    if (n_dims == 7) p *= pop_oracle_p_z(th[6], L);
    return p;
}

/* The same with a precomputed redshift normalisation (one trapezoid per Lambda). */
static double p_theta_znorm(const double* th, int n_dims, const double* L, double znorm)
{
    double p = pop_oracle_p_m1(th[0], L);
    if (p == 0.0) return 0.0;
    p *= pop_oracle_p_q(th[1], th[0], L);
    p *= pop_oracle_p_chi(th[2], L) * pop_oracle_p_chi(th[3], L);
    p *= pop_oracle_p_tilt(th[4], th[5], L);
    if (n_dims == 7) {
        double z = th[6];
        if (!(z >= 0.0 && z <= 2.0)) return 0.0;
        p *= pow(1.0 + z, L[P_KAPPA] - 1.0) * z * z / znorm;
    }
    return p;
}

/*
 * ln L for K Lambda points.
 *   offsets[n_events+1] (CSR), theta[offsets[n] * n_dims], prior[offsets[n]]
 *   inj_theta[n_found * n_dims], p_draw[n_found], n_draw >= n_found
 *   lambda[K * n_params], n_params = 11 + (n_dims == 7)
 * Outputs (any but out_lnL may be NULL): ln L, ln xi, N_eff, flags.
 * Returns 0, or -1 on inconsistent sizes.
 */
int pop_oracle_loglik(int64_t n_events, const int64_t* offsets, int n_dims,
                      const double* theta, const double* prior,
                      int64_t n_found, int64_t n_draw, const double* inj_theta, const double* p_draw,
                      int64_t K, int n_params, const double* lambda, int nthreads,
                      double* out_lnL, double* out_lnxi, double* out_neff, uint32_t* out_flags)
{
    if (n_events < 1 || (n_dims != 6 && n_dims != 7) || n_params != 11 + (n_dims == 7) ||
        n_draw < n_found || n_draw < 1 || K < 0 || !out_lnL)
        return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < K; ++k) {
        const double* L = lambda + k * n_params;
        uint32_t flags = 0;
        double lnL, lnxi = 0.0, neff = 0.0;
        if (!pop_oracle_lambda_valid(L, n_params)) {
            flags |= OR_FLAG_INVALID_LAMBDA;
            lnL = -INFINITY;
        } else {
            double znorm = n_dims == 7 ? pop_oracle_z_norm(L[P_KAPPA]) : 1.0;
            /* Selection term and its effective sample count. */
            double sw = 0.0, sw2 = 0.0;
            for (int64_t j = 0; j < n_found; ++j) {
                double w = p_theta_znorm(inj_theta + j * n_dims, n_dims, L, znorm) / p_draw[j];
                sw += w;
                sw2 += w * w;
            }
            double xi = sw / (double)n_draw;
            double var = sw2 / ((double)n_draw * (double)n_draw) - xi * xi / (double)n_draw;
            neff = var > 0.0 ? xi * xi / var : INFINITY;
            /* Recycled per-event Monte Carlo integrals. */
            double sum_ln = 0.0;
            for (int64_t i = 0; i < n_events; ++i) {
                double s = 0.0;
                int64_t n_i = offsets[i + 1] - offsets[i];
                for (int64_t j = offsets[i]; j < offsets[i + 1]; ++j)
                    s += p_theta_znorm(theta + j * n_dims, n_dims, L, znorm) / prior[j];
                if (s == 0.0) flags |= OR_FLAG_ZERO_EVENT;
                sum_ln += log(s / (double)n_i);
            }
            if (xi == 0.0) {
                flags |= OR_FLAG_ZERO_XI;
                lnL = -INFINITY;
                lnxi = -INFINITY;
                neff = 0.0;
            } else {
                lnxi = log(xi);
                lnL = (flags & OR_FLAG_ZERO_EVENT) ? -INFINITY : sum_ln - (double)n_events * lnxi;
            }
            if (neff < 4.0 * (double)n_events) flags |= OR_FLAG_LOW_NEFF;
        }
        out_lnL[k] = lnL;
        if (out_lnxi) out_lnxi[k] = lnxi;
        if (out_neff) out_neff[k] = neff;
        if (out_flags) out_flags[k] = flags;
    }
    return 0;
}

/*
 * The additive parts of ln L for K Lambda points, over the given events and
 * found injections: sum_i ln(S_i / n_i) (-inf when some S_i = 0), and
 * sum_k w_k and sum_k w_k^2 over the injections (not divided by n_draw).
 * Events and injections split into disjoint sets give parts that add up to
 * those of the whole set; ln L then follows as in pop_oracle_loglik.
 * Flags: invalid Lambda (parts -inf, 0, 0) and zero event only.
 */
int pop_oracle_loglik_parts(int64_t n_events, const int64_t* offsets, int n_dims,
                            const double* theta, const double* prior,
                            int64_t n_found, const double* inj_theta, const double* p_draw,
                            int64_t K, int n_params, const double* lambda, int nthreads,
                            double* out_events, double* out_sum_w, double* out_sum_w2, uint32_t* out_flags)
{
    if (n_events < 0 || (n_dims != 6 && n_dims != 7) || n_params != 11 + (n_dims == 7) || n_found < 0 || K < 0 ||
        !out_events || !out_sum_w || !out_sum_w2 || !out_flags)
        return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < K; ++k) {
        const double* L = lambda + k * n_params;
        uint32_t flags = 0;
        double sum_ln = 0.0, sw = 0.0, sw2 = 0.0;
        if (!pop_oracle_lambda_valid(L, n_params)) {
            flags |= OR_FLAG_INVALID_LAMBDA;
            sum_ln = -INFINITY;
        } else {
            double znorm = n_dims == 7 ? pop_oracle_z_norm(L[P_KAPPA]) : 1.0;
            for (int64_t j = 0; j < n_found; ++j) {
                double w = p_theta_znorm(inj_theta + j * n_dims, n_dims, L, znorm) / p_draw[j];
                sw += w;
                sw2 += w * w;
            }
            for (int64_t i = 0; i < n_events; ++i) {
                double s = 0.0;
                int64_t n_i = offsets[i + 1] - offsets[i];
                for (int64_t j = offsets[i]; j < offsets[i + 1]; ++j)
                    s += p_theta_znorm(theta + j * n_dims, n_dims, L, znorm) / prior[j];
                if (s == 0.0) flags |= OR_FLAG_ZERO_EVENT;
                sum_ln += log(s / (double)n_i);
            }
            if (flags & OR_FLAG_ZERO_EVENT) sum_ln = -INFINITY;
        }
        out_events[k] = sum_ln;
        out_sum_w[k] = sw;
        out_sum_w2[k] = sw2;
        out_flags[k] = flags;
    }
    return 0;
}

/*
 * Selection term on a regular grid (Sec. "Population acceleration": VT on a
 * regular grid, limited to low dimension, no spin effects).  With a detection
 * probability pdet[a * n_q + b] given at the grid nodes (m1_a, q_b), the grid
 * estimate of xi(Lambda) = int p(m1, q | Lambda) P_det(m1, q) dm1 dq is the
 * two-dimensional trapezoid rule over the nodes:
 *   xi_grid = sum_a sum_b wa_a wq_b p(m1_a | Lambda) p(q_b | m1_a, Lambda) pdet[a, b]
 * with wa, wq the trapezoid weights of the (not necessarily uniform) node sets.
 * The spin and tilt densities integrate to one and are left out.  Output: ln xi_grid
 * (-inf when it is 0; invalid Lambda -> 0 and the returned flag bit 1).
 */
int pop_oracle_xi_grid(int n_m1, const double* m1, int n_q, const double* q, const double* pdet,
                       int64_t K, int n_params, const double* lambda, double* out_lnxi, uint32_t* out_flags)
{
    if (n_m1 < 2 || n_q < 2 || K < 0 || !out_lnxi) return -1;
    for (int64_t k = 0; k < K; ++k) {
        const double* L = lambda + k * n_params;
        if (!pop_oracle_lambda_valid(L, n_params)) {
            out_lnxi[k] = 0.0;
            if (out_flags) out_flags[k] = OR_FLAG_INVALID_LAMBDA;
            continue;
        }
        double s = 0.0;
        for (int a = 0; a < n_m1; ++a) {
            double wa = 0.5 * ((a + 1 < n_m1 ? m1[a + 1] : m1[a]) - (a > 0 ? m1[a - 1] : m1[a]));
            double pm = pop_oracle_p_m1(m1[a], L);
            if (pm == 0.0) continue;
            for (int b = 0; b < n_q; ++b) {
                double wq = 0.5 * ((b + 1 < n_q ? q[b + 1] : q[b]) - (b > 0 ? q[b - 1] : q[b]));
                s += wa * wq * pm * pop_oracle_p_q(q[b], m1[a], L) * pdet[(int64_t)a * n_q + b];
            }
        }
        out_lnxi[k] = s > 0.0 ? log(s) : -INFINITY;
        if (out_flags) out_flags[k] = s > 0.0 ? 0u : OR_FLAG_ZERO_XI;
    }
    return 0;
}

/* Digamma psi(x), x > 0: the recurrence psi(x) = psi(x + 1) - 1/x up to x >= 10,
 * then the asymptotic series ln x - 1/(2x) - sum B_2k / (2k x^2k) (Abramowitz &
 * Stegun 6.3.18) to x^-12. */
double pop_oracle_digamma(double x)
{
    double r = 0.0;
    while (x < 10.0) {
        r -= 1.0 / x;
        x += 1.0;
    }
    const double x2 = 1.0 / (x * x);
    const double series = x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132 - x2 * (691.0 / 32760))))));
    return r + log(x) - 0.5 / x - series;
}

static double std_normal_pdf(double t) { return exp(-0.5 * t * t) / SQRT2PI; }

/*
 * p(theta | Lambda) and its score g[p] = d ln p(theta | Lambda) / d Lambda_p for the
 * n_params parameters, inside the support (the support's own edges, where the
 * density jumps, have no derivative and are left out).  Term by term:
 *   power law  PL = x^-alpha C, C = (1-alpha) / (b^(1-alpha) - a^(1-alpha)):
 *     d ln PL/d alpha = -ln x + d ln C/d alpha,  d ln C/d alpha = -1/(1-alpha) + (b^s ln b - a^s ln a)/(b^s - a^s)
 *     (s = 1 - alpha; at alpha = 1, (ln a + ln b)/2); d ln C/d a = PL(a), d ln C/d b = -PL(b)
 *     (a normalised density f = g / int_a^b g has d ln(1/int)/d a = f(a)).
 *   truncated normal N_T = phi((x-mu)/sigma) / (sigma Z) on [a, b]:
 *     d/d mu: (x-mu)/sigma^2 + N_T(b) - N_T(a);  d/d sigma: -1/sigma + (x-mu)^2/sigma^3 + b' N_T(b) - a' N_T(a)
 *     (a' = (a-mu)/sigma, b' = (b-mu)/sigma); d/d a: N_T(a); d/d b: -N_T(b).
 *   p(m1) = (1-lam) PL + lam N_T: d/d lam = (N_T - PL)/p(m1); the rest weighted by each part.
 *   p(q|m1) = (1+beta) q^beta / (1 - rho), rho = (mmin/m1)^(1+beta):
 *     d/d beta = 1/(1+beta) + ln q + rho ln(mmin/m1)/(1 - rho)   (beta = -1: ln q - ln(mmin/m1)/2)
 *     d/d mmin = (1+beta) rho / (mmin (1 - rho))                 (beta = -1: 1/(mmin ln(m1/mmin)))
 *   Beta(a; ac, bc): d/d ac = ln a - psi(ac) + psi(ac+bc), d/d bc = ln(1-a) - psi(bc) + psi(ac+bc), per spin.
 *   tilts T = (1-xi)/4 + xi G1 G2, G = phi((c-1)/sigma_t)/(sigma_t Z_t), Z_t = erf(sqrt2/sigma_t)/2:
 *     d/d xi = (G1 G2 - 1/4)/T;  d/d sigma_t = xi G1 G2 (-2/sigma_t + dc/sigma_t^3 + 4 phi(2/sigma_t)/(sigma_t^2 Z_t)) / T,
 *     dc = (c1-1)^2 + (c2-1)^2.
 *   redshift Z(z) = (1+z)^(kappa-1) z^2 / I(kappa): d/d kappa = ln(1+z) - I'(kappa)/I(kappa), I' the
 *     same trapezoid of (1+z)^(kappa-1) ln(1+z) z^2.
 * Returns p (0 outside the support; g is then left at 0).
 */
static double score_theta(const double* th, int n_dims, const double* L, double znorm, double dznorm, double* g)
{
    for (int p = 0; p < 12; ++p) g[p] = 0.0;
    const double m1 = th[0], q = th[1], a1 = th[2], a2 = th[3], c1 = th[4], c2 = th[5];
    const double alpha = L[P_ALPHA], beta = L[P_BETA], mmin = L[P_MMIN], mmax = L[P_MMAX], lam = L[P_LAM];
    const double mu = L[P_MPP], sig = L[P_SIGPP], ac = L[P_ACHI], bc = L[P_BCHI], xit = L[P_XIT], sigt = L[P_SIGT];
    const double p = p_theta_znorm(th, n_dims, L, znorm);
    if (p == 0.0) return 0.0;
    /* primary mass */
    const double pl = powerlaw_pdf(m1, alpha, mmin, mmax);
    const double pla = powerlaw_pdf(mmin, alpha, mmin, mmax), plb = powerlaw_pdf(mmax, alpha, mmin, mmax);
    double dlnC_alpha;
    if (alpha == 1.0) {
        dlnC_alpha = 0.5 * (log(mmin) + log(mmax));
    } else {
        const double s = 1.0 - alpha, bs = pow(mmax, s), as = pow(mmin, s);
        dlnC_alpha = -1.0 / s + (bs * log(mmax) - as * log(mmin)) / (bs - as);
    }
    const double nt = truncnorm_pdf(m1, mu, sig, mmin, mmax);
    const double nta = truncnorm_pdf(mmin, mu, sig, mmin, mmax), ntb = truncnorm_pdf(mmax, mu, sig, mmin, mmax);
    const double ap = (mmin - mu) / sig, bp = (mmax - mu) / sig;
    const double pm = (1.0 - lam) * pl + lam * nt;
    const double fpl = (1.0 - lam) * pl / pm, fnt = lam * nt / pm; /* shares of the two parts */
    g[P_ALPHA] += fpl * (-log(m1) + dlnC_alpha);
    g[P_LAM] += (nt - pl) / pm;
    g[P_MPP] += fnt * ((m1 - mu) / (sig * sig) + ntb - nta);
    g[P_SIGPP] += fnt * (-1.0 / sig + (m1 - mu) * (m1 - mu) / (sig * sig * sig) + bp * ntb - ap * nta);
    g[P_MMIN] += fpl * pla + fnt * nta;
    g[P_MMAX] += -fpl * plb - fnt * ntb;
    /* mass ratio */
    const double lr = log1p((mmin - m1) / m1); /* ln(mmin/m1) */
    if (beta == -1.0) {
        g[P_BETA] += log(q) - 0.5 * lr;
        g[P_MMIN] += 1.0 / (mmin * -lr);
    } else {
        const double rho = exp((1.0 + beta) * lr);
        const double one_minus = -expm1((1.0 + beta) * lr);
        g[P_BETA] += 1.0 / (1.0 + beta) + log(q) + rho * lr / one_minus;
        g[P_MMIN] += (1.0 + beta) * rho / (mmin * one_minus);
    }
    /* spin magnitudes */
    const double psab = pop_oracle_digamma(ac + bc);
    g[P_ACHI] += log(a1) + log(a2) - 2.0 * pop_oracle_digamma(ac) + 2.0 * psab;
    g[P_BCHI] += log(1.0 - a1) + log(1.0 - a2) - 2.0 * pop_oracle_digamma(bc) + 2.0 * psab;
    /* tilts */
    const double zt = 0.5 * erf(SQRT2 / sigt);
    const double G1 = std_normal_pdf((c1 - 1.0) / sigt) / (sigt * zt), G2 = std_normal_pdf((c2 - 1.0) / sigt) / (sigt * zt);
    const double T = (1.0 - xit) / 4.0 + xit * G1 * G2;
    const double dc = (c1 - 1.0) * (c1 - 1.0) + (c2 - 1.0) * (c2 - 1.0);
    g[P_XIT] += (G1 * G2 - 0.25) / T;
    g[P_SIGT] += xit * G1 * G2 *
                 (-2.0 / sigt + dc / (sigt * sigt * sigt) + 4.0 * std_normal_pdf(2.0 / sigt) / (sigt * sigt * zt)) / T;
    /* redshift */
    if (n_dims == 7) g[P_KAPPA] += log1p(th[6]) - dznorm / znorm;
    return p;
}

static double z_norm_dkappa(double kappa);

/* p(theta | Lambda) and its score g[n_params] (0 outside the support). */
double pop_oracle_score(const double* th, int n_dims, const double* L, int n_params, double* g)
{
    double gg[12];
    const double zn = n_dims == 7 ? pop_oracle_z_norm(L[P_KAPPA]) : 1.0;
    const double dz = n_dims == 7 ? z_norm_dkappa(L[P_KAPPA]) : 0.0;
    const double p = score_theta(th, n_dims, L, zn, dz, gg);
    for (int k = 0; k < n_params; ++k) g[k] = gg[k];
    return p;
}

/* d I / d kappa for the 1024-node trapezoid I of pop_oracle_z_norm. */
static double z_norm_dkappa(double kappa)
{
    const int n = 1024;
    double h = 2.0 / (n - 1), s = 0.0;
    for (int k = 0; k < n; ++k) {
        double z = 2.0 * k / (n - 1);
        double f = pow(1.0 + z, kappa - 1.0) * log1p(z) * z * z;
        s += (k == 0 || k == n - 1) ? 0.5 * f : f;
    }
    return s * h;
}

/*
 * ln L and its gradient d ln L / d Lambda (n_params components, the C-ABI
 * order) for K Lambda points; derived from Eq. (poplike) with the -N ln xi
 * term (the paper does not differentiate it):
 *   d ln L = sum_i (sum_j w_ij g_ij) / S_i - N (sum_k w_k g_k) / (sum_k w_k),
 * g the score of p(theta|Lambda) at each sample.  Where ln L = -inf (invalid
 * Lambda, an empty event, xi = 0) the gradient is 0.  Outputs as
 * pop_oracle_loglik plus out_grad[K * n_params].
 */
int pop_oracle_loglik_grad(int64_t n_events, const int64_t* offsets, int n_dims, const double* theta,
                           const double* prior, int64_t n_found, int64_t n_draw, const double* inj_theta,
                           const double* p_draw, int64_t K, int n_params, const double* lambda, int nthreads,
                           double* out_lnL, double* out_grad, uint32_t* out_flags)
{
    if (!out_grad) return -1;
    int rc = pop_oracle_loglik(n_events, offsets, n_dims, theta, prior, n_found, n_draw, inj_theta, p_draw, K,
                               n_params, lambda, nthreads, out_lnL, NULL, NULL, out_flags);
    if (rc != 0) return rc;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < K; ++k) {
        const double* L = lambda + k * n_params;
        double* G = out_grad + k * n_params;
        for (int p = 0; p < n_params; ++p) G[p] = 0.0;
        if (!isfinite(out_lnL[k])) continue;
        const double znorm = n_dims == 7 ? pop_oracle_z_norm(L[P_KAPPA]) : 1.0;
        const double dznorm = n_dims == 7 ? z_norm_dkappa(L[P_KAPPA]) : 0.0;
        double g[12], sw = 0.0, swg[12] = {0};
        for (int64_t j = 0; j < n_found; ++j) {
            const double w = score_theta(inj_theta + j * n_dims, n_dims, L, znorm, dznorm, g) / p_draw[j];
            sw += w;
            for (int p = 0; p < n_params; ++p) swg[p] += w * g[p];
        }
        for (int p = 0; p < n_params; ++p) G[p] = -(double)n_events * swg[p] / sw;
        for (int64_t i = 0; i < n_events; ++i) {
            double s = 0.0, sg[12] = {0};
            for (int64_t j = offsets[i]; j < offsets[i + 1]; ++j) {
                const double w = score_theta(theta + j * n_dims, n_dims, L, znorm, dznorm, g) / prior[j];
                s += w;
                for (int p = 0; p < n_params; ++p) sg[p] += w * g[p];
            }
            for (int p = 0; p < n_params; ++p) G[p] += sg[p] / s;
        }
    }
    return 0;
}

/*
 * Single-event CBC likelihood (paper, Sec. "Single-event Likelihood
 * acceleration", Eq. (cbclike)), for K parameter rows:
 *
 *   ln L = sum_i sum_j [ -ln(2 pi S_ij) - (2/T) |d_ij - h_ij|^2 / S_ij ]
 *
 * over n_det detectors i and M frequency bins j, f_j = f0 + j df, T = 1/df.
 * The template seen by detector i is the response to the two polarisations,
 * moved in time by the per-detector factor exp(-2 pi i f dt_i) the same section
 * describes, with an overall amplitude and phase:
 *
 *   h_ij = A e^{i phi} (Fp_i hp_j + Fc_i hc_j) e^{-2 pi i f_j dt_i}
 *
 * theta row k = (A, phi, Fp_1, Fc_1, dt_1, ..., Fp_n, Fc_n, dt_n).
 * data[(i M + j) * 2 + {0,1}] = Re, Im d_ij; psd[i M + j] = S_ij > 0;
 * hp[2 j + {0,1}], hc[2 j + {0,1}] = the polarisations.  Every term is
 * evaluated directly (libm cos, sin, log) and summed in order.
 */
int pop_oracle_cbc_loglik(int n_det, int64_t M, double f0, double df, const double* data, const double* psd,
                          const double* hp, const double* hc, int64_t K, const double* theta, int nthreads,
                          double* out_lnL)
{
    if (n_det < 1 || M < 1 || !(df > 0.0) || K < 0 || !out_lnL) return -1;
    const double two_over_T = 2.0 * df;
    const double two_pi = 6.283185307179586476925;
    const int P = 2 + 3 * n_det;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < K; ++k) {
        const double* th = theta + k * P;
        const double A = th[0], phi = th[1];
        const double cre = A * cos(phi), cim = A * sin(phi);
        double lnL = 0.0;
        for (int i = 0; i < n_det; ++i) {
            const double Fp = th[2 + 3 * i], Fc = th[3 + 3 * i], dt = th[4 + 3 * i];
            for (int64_t j = 0; j < M; ++j) {
                const double f = f0 + (double)j * df;
                /* response to the polarisations, times A e^{i phi} */
                const double ure = Fp * hp[2 * j] + Fc * hc[2 * j];
                const double uim = Fp * hp[2 * j + 1] + Fc * hc[2 * j + 1];
                const double vre = cre * ure - cim * uim;
                const double vim = cre * uim + cim * ure;
                /* time shift exp(-2 pi i f dt) */
                const double ang = two_pi * f * dt;
                const double ere = cos(ang), eim = -sin(ang);
                const double hre = vre * ere - vim * eim;
                const double him = vre * eim + vim * ere;
                const double S = psd[(int64_t)i * M + j];
                const double rre = data[((int64_t)i * M + j) * 2] - hre;
                const double rim = data[((int64_t)i * M + j) * 2 + 1] - him;
                lnL += -log(two_pi * S) - two_over_T * (rre * rre + rim * rim) / S;
            }
        }
        out_lnL[k] = lnL;
    }
    return 0;
}

/* Threads the OpenMP runtime would use (1 without OpenMP). */
int pop_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
