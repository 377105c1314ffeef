// Gradient of ln L with respect to Lambda, in the same pass as ln L (FP64).
//
// Derived from Eq. (poplike) with the -N ln xi term (the paper does not
// differentiate it):
//
//   d ln L / d Lambda_p = sum_i (sum_j w_ij g_ij,p) / S_i - N (sum_k w_k g_k,p) / (sum_k w_k),
//
// g = d ln p(theta|Lambda) / d Lambda, the score of the population density.  The
// kernel keeps, per (chunk, Lambda), the sums of w and of w g_p for the 11 or 12
// parameters (forward-mode: every pair carries its weight and its weight's
// derivatives), with the same persistent (chunk x Lambda-tile) items, warp vote
// on the support and table-driven exponentials as the FP64 weight kernel.  The
// mixture is split into its power-law and peak parts so that d/d lam holds at
// lam = 0 and 1, and the tilt mixture likewise for xi_t.
//
// Score terms (the support's own edges, where the density jumps, have none):
//   alpha: W1 (dlnC_alpha - ln m1)                 lam: A2 - A1
//   mpp:   W2 ((m1 - mpp)/sigpp^2 + N_T(mmax) - N_T(mmin))
//   sigpp: W2 (-1/sigpp + (m1 - mpp)^2/sigpp^3 + b' N_T(mmax) - a' N_T(mmin))
//   mmin:  W1 PL(mmin) + W2 N_T(mmin) + w (1+beta) rho / (mmin (1 - rho)),  rho = (mmin/m1)^(1+beta)
//   mmax:  -W1 PL(mmax) - W2 N_T(mmax)
//   beta:  w (1/(1+beta) + ln q + rho ln(mmin/m1) / (1 - rho))
//   alpha_chi, beta_chi: w (ln a1 + ln a2 - 2 psi(ac) + 2 psi(ac+bc)), likewise with ln(1-a)
//   xi_t:  (w / T) (G1 G2 - 1/4);   sigma_t: (w / T) xi_t G1 G2 (-2/sigma_t + dc/sigma_t^3 + 4 phi(2/sigma_t)/(sigma_t^2 Z_t))
//   kappa: w (ln(1+z) - I'(kappa)/I(kappa))
// with W1 = (1-lam) A1, W2 = lam A2 the two parts of w = W1 + W2, T the tilt factor.
#include <math.h>

#include "pop_internal.h"

namespace pop {

namespace {

constexpr double G_SQRT2 = 1.4142135623730950488;
constexpr double G_SQRT2PI = 2.5066282746310005024;
constexpr int G_Z_NODES = 1024;

struct alignas(16) LamG {
    long long mmin_bits, mmax_bits;
    double beta, ac1, bc1, km1;      // exponents of ln q, ln a, ln(1-a), ln(1+z)
    double nalpha, c1, c2;           // power-law and peak log-constants (without 1-lam, lam)
    double mu, nh;                   // mpp, -1/(2 sigpp^2)
    double b1, inv_b1, mmin, lmmin, inv_mmin;
    double nht, ctp, t0, xi, lam;    // tilts: G1 G2 = exp(nht dc + ctp), T = t0 + xi G1 G2
    double dlnC_alpha, PLa, PLb, NTa, NTb, ap, bp, inv_s, inv_s2, inv_s3;
    double c_ac2, c_bc2, st_c, inv_st3, dlnI;
    int beta_m1, valid;
};

// psi(x), x > 0: recurrence up to x >= 10, then the asymptotic series
// (Abramowitz & Stegun 6.3.18) through x^-12.
__device__ double digamma_d(double x)
{
    double acc = 0.0;
    for (int i = 0; i < 64 && x < 10.0; ++i) {
        acc -= 1.0 / x;
        x += 1.0;
    }
    // psi ~ ln x - 1/(2x) - t S(t), t = 1/x^2,
    // S = 1/12 - t/120 + t^2/252 - t^3/240 + t^4/132 - 691 t^5/32760 (Horner from the inside).
    const double t = 1.0 / (x * x);
    double s = -691.0 / 32760.0;
    s = fma(s, t, 1.0 / 132.0);
    s = fma(s, t, -1.0 / 240.0);
    s = fma(s, t, 1.0 / 252.0);
    s = fma(s, t, -1.0 / 120.0);
    s = fma(s, t, 1.0 / 12.0);
    return acc + log(x) - 0.5 / x - t * s;
}

__device__ double std_phi(double t) { return exp(-0.5 * t * t) / G_SQRT2PI; }

// One warp per Lambda: the redshift trapezoid and its kappa-derivative on the lanes,
// the rest on lane 0.
__global__ void grad_prologue_kernel(const double* __restrict__ lambda, const int64_t* __restrict__ dK, int n_params,
                                     LamG* __restrict__ out, const double2* __restrict__ ztab,
                                     const double2* __restrict__ exptab, ExpConsts kc)
{
    const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= *dK) return;
    const double* L = lambda + k * n_params;
    const bool has_z = n_params == 12;
    double I = 0.0, dI = 0.0;
    if (has_z) {
        const double km1 = L[P_KAPPA] - 1.0;
        // node i: (ln(1 + z_i), w_i z_i^2); one table-driven exponential per node
        for (int i = lane; i < G_Z_NODES; i += 32) {
            const double2 t = ztab[i];
            const double f = t.y * exp_tab(km1 * t.x, exptab, kc);
            I += f;
            dI = fma(f, t.x, dI);
        }
        for (int o = 16; o > 0; o >>= 1) {
            I += __shfl_xor_sync(0xffffffffu, I, o);
            dI += __shfl_xor_sync(0xffffffffu, dI, o);
        }
        I *= 2.0 / (G_Z_NODES - 1);
        dI *= 2.0 / (G_Z_NODES - 1);
    }
    if (lane != 0) return;
    LamG c;
    bool ok = true;
    for (int p = 0; p < n_params; ++p) ok = ok && isfinite(L[p]);
    const double alpha = L[P_ALPHA], beta = L[P_BETA], mmin = L[P_MMIN], mmax = L[P_MMAX], lam = L[P_LAM];
    const double mu = L[P_MPP], sig = L[P_SIGPP], ac = L[P_ACHI], bc = L[P_BCHI], xit = L[P_XIT], sigt = L[P_SIGT];
    ok = ok && mmin > 0.0 && mmin < mmax && lam >= 0.0 && lam <= 1.0 && sig > 0.0 && sigt > 0.0 && ac > 0.0 &&
         bc > 0.0 && xit >= 0.0 && xit <= 1.0;
    c.valid = ok;
    if (!ok) {
        c.mmin_bits = 0x7ff0000000000000LL;  // +inf: no sample is ever in the support
        c.mmax_bits = 0;
        out[k] = c;
        return;
    }
    c.mmin_bits = __double_as_longlong(mmin);
    c.mmax_bits = __double_as_longlong(mmax);
    c.beta = beta;
    c.ac1 = ac - 1.0;
    c.bc1 = bc - 1.0;
    c.km1 = has_z ? L[P_KAPPA] - 1.0 : 0.0;
    c.beta_m1 = beta == -1.0;
    c.b1 = 1.0 + beta;
    c.inv_b1 = c.beta_m1 ? 0.0 : 1.0 / c.b1;
    c.mmin = mmin;
    c.lmmin = log(mmin);
    c.inv_mmin = 1.0 / mmin;
    // power law: C = (1-alpha)/(b^s - a^s), s = 1 - alpha (alpha = 1: 1/ln(b/a))
    double lC, dlnC;
    if (alpha == 1.0) {
        lC = -log(log(mmax / mmin));
        dlnC = 0.5 * (log(mmin) + log(mmax));
    } else {
        const double s = 1.0 - alpha, bs = pow(mmax, s), as = pow(mmin, s);
        lC = log(s / (bs - as));
        dlnC = -1.0 / s + (bs * log(mmax) - as * log(mmin)) / (bs - as);
    }
    c.nalpha = -alpha;
    c.dlnC_alpha = dlnC;
    c.PLa = exp(-alpha * log(mmin) + lC);
    c.PLb = exp(-alpha * log(mmax) + lC);
    // truncated normal on [mmin, mmax]
    const double ap = (mmin - mu) / sig, bp = (mmax - mu) / sig;
    const double Z = 0.5 * (erf(bp / G_SQRT2) - erf(ap / G_SQRT2));
    const double Cg = 1.0 / (G_SQRT2PI * sig * Z);
    c.mu = mu;
    c.nh = -0.5 / (sig * sig);
    c.ap = ap;
    c.bp = bp;
    c.NTa = exp(-0.5 * ap * ap) * Cg;
    c.NTb = exp(-0.5 * bp * bp) * Cg;
    c.inv_s = 1.0 / sig;
    c.inv_s2 = c.inv_s * c.inv_s;
    c.inv_s3 = c.inv_s2 * c.inv_s;
    // spins
    const double lnB = lgamma(ac) + lgamma(bc) - lgamma(ac + bc);
    const double psab = digamma_d(ac + bc);
    c.c_ac2 = 2.0 * (psab - digamma_d(ac));
    c.c_bc2 = 2.0 * (psab - digamma_d(bc));
    // tilts: G = phi((c-1)/sigma_t) / (sigma_t Z_t), Z_t = erf(sqrt2/sigma_t)/2
    const double Zt = 0.5 * erf(G_SQRT2 / sigt);
    const double Ct = 1.0 / (G_SQRT2PI * sigt * Zt);
    c.nht = -0.5 / (sigt * sigt);
    c.ctp = 2.0 * log(Ct);
    c.t0 = 0.25 * (1.0 - xit);
    c.xi = xit;
    c.lam = lam;
    c.st_c = -2.0 / sigt + 4.0 * std_phi(2.0 / sigt) / (sigt * sigt * Zt);
    c.inv_st3 = 1.0 / (sigt * sigt * sigt);
    // shared log-constants of both mass parts
    const double lb1 = c.beta_m1 ? 0.0 : log(fabs(c.b1));
    const double lI = has_z ? log(I) : 0.0;
    const double common = lb1 - 2.0 * lnB - lI;
    c.c1 = common + lC;
    c.c2 = common + log(Cg);
    c.dlnI = has_z ? dI / I : 0.0;
    out[k] = c;
}

struct GSample {
    double lm1, m1, lq, sa, sb, dc, nlpi, lz1, invm1;
    long long m1b, m2b;
};

template <bool HAS_Z>
__device__ __forceinline__ void load_g(const FeatF64& F, int64_t s, GSample& x)
{
    const double* b = F.base;
    const int64_t st = F.stride;
    x.lm1 = __ldg(b + F_LM1 * st + s);
    x.m1 = __ldg(b + F_M1 * st + s);
    x.lq = __ldg(b + F_LQ * st + s);
    x.sa = __ldg(b + F_SA * st + s);
    x.sb = __ldg(b + F_SB * st + s);
    x.dc = __ldg(b + F_DC * st + s);
    x.nlpi = __ldg(b + F_NLPI * st + s);
    x.lz1 = HAS_Z ? __ldg(b + F_LZ1 * st + s) : 0.0;
    x.invm1 = __ldg(b + F_INVM1 * st + s);
    x.m1b = __double_as_longlong(x.m1);
    x.m2b = __double_as_longlong(__ldg(b + F_M2 * st + s));
}

constexpr int NG = 13;  // w and w g_p for up to 12 parameters

// The weight of one pair and its derivatives, added to acc (acc[0] += w, acc[1 + p] += w g_p,
// acc[NG] += w^2) when `in` (the pair is inside the support).
template <bool HAS_Z>
__device__ __forceinline__ void weight_grad(const GSample& x, const LamG& c, const double2* __restrict__ tab,
                                            const ExpConsts& kc, bool in, double (&acc)[NG + 1])
{
    auto add = [&](int p, double v) { acc[p] = in ? acc[p] + v : acc[p]; };
    double aE = fma(c.beta, x.lq, x.nlpi);
    aE = fma(c.ac1, x.sa, aE);
    aE = fma(c.bc1, x.sb, aE);
    if (HAS_Z) aE = fma(c.km1, x.lz1, aE);
    const double E1 = exp_tab(fma(c.nalpha, x.lm1, aE + c.c1), tab, kc);
    const double d = x.m1 - c.mu;
    const double E2 = exp_tab(fma(c.nh * d, d, aE + c.c2), tab, kc);
    double lr = c.lmmin - x.lm1;
    if (llabs(x.m1b - c.mmin_bits) < NEAR_EDGE_BITS) lr = log1p_near0(x.invm1 * (c.mmin - x.m1));
    double em = 0.0, r;
    if (c.beta_m1) {
        r = rcp_pos(-lr);
    } else {
        em = expm1_tab(c.b1 * lr, tab, kc);  // rho - 1, rho = (mmin/m1)^(1+beta)
        r = rcp_pos(fabs(em));
    }
    const double GG = exp_tab(fma(c.nht, x.dc, c.ctp), tab, kc);  // G1 G2
    const double tt = fma(c.xi, GG, c.t0);
    const double A1r = E1 * r, A2r = E2 * r;                     // parts before the tilt factor
    const double A1 = A1r * tt, A2 = A2r * tt;
    const double W1 = (1.0 - c.lam) * A1, W2 = c.lam * A2;
    const double w = W1 + W2;
    const double wt = (1.0 - c.lam) * A1r + c.lam * A2r;          // w / tt
    add(0, w);
    acc[NG] = in ? fma(w, w, acc[NG]) : acc[NG];
    add(1 + P_ALPHA, W1 * (c.dlnC_alpha - x.lm1));
    add(1 + P_LAM, A2 - A1);
    add(1 + P_MPP, W2 * fma(d, c.inv_s2, c.NTb - c.NTa));
    add(1 + P_SIGPP, W2 * (fma(d * d, c.inv_s3, -c.inv_s) + (c.bp * c.NTb - c.ap * c.NTa)));
    double qn, gb;
    if (c.beta_m1) {
        qn = c.inv_mmin * r;                  // 1 / (mmin ln(m1/mmin))
        gb = x.lq - 0.5 * lr;
    } else {
        const double inv_em = c.b1 > 0.0 ? -r : r;   // 1/em: em < 0 when 1 + beta > 0
        const double rho = em + 1.0;
        qn = -c.b1 * rho * c.inv_mmin * inv_em;      // (1+beta) rho / (mmin (1 - rho))
        gb = c.inv_b1 + x.lq - rho * lr * inv_em;    // 1/(1+beta) + ln q + rho lr / (1 - rho)
    }
    add(1 + P_MMIN, fma(W1, c.PLa, fma(W2, c.NTa, w * qn)));
    add(1 + P_MMAX, -fma(W1, c.PLb, W2 * c.NTb));
    add(1 + P_BETA, w * gb);
    add(1 + P_ACHI, w * (x.sa + c.c_ac2));
    add(1 + P_BCHI, w * (x.sb + c.c_bc2));
    add(1 + P_XIT, wt * (GG - 0.25));
    add(1 + P_SIGT, wt * c.xi * GG * fma(x.dc, c.inv_st3, c.st_c));
    if (HAS_Z) add(1 + P_KAPPA, w * (x.lz1 - c.dlnI));
}

__device__ __forceinline__ bool in_support_g(const GSample& x, const LamG& c)
{
    return (x.m1b > c.mmin_bits) & (x.m1b <= c.mmax_bits) & (x.m2b >= c.mmin_bits);
}

constexpr int GRAD_THREADS = 256;

// part[(k * n_chunks + c) * NG + 0..12]: sums of w and w g over chunk c for Lambda k;
// part2[k * n_inj + c']: sum of w^2 over injection chunk c'.
template <bool HAS_Z>
__global__ void __launch_bounds__(GRAD_THREADS)
grad_weight_kernel(FeatF64 ev, FeatF64 inj, WorkDesc wd, const LamG* __restrict__ lam,
                   const int64_t* __restrict__ dK, int n_params, double* __restrict__ part,
                   double* __restrict__ part2, const double2* __restrict__ exptab, ExpConsts kc,
                   unsigned long long* __restrict__ queue)
{
    extern __shared__ double2 stab[];
    __shared__ double red[GRAD_THREADS / 32][NG + 1];
    __shared__ LamG scl;
    for (int i = threadIdx.x; i < EXP_TABLE_SIZE; i += GRAD_THREADS) stab[i] = exptab[i];
    const int64_t K = *dK;
    const int64_t n_items = (int64_t)wd.n_chunks * K;
    const int n_inj = wd.n_chunks - wd.n_ev_chunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Items come from a queue (zeroed before the launch), chunk-major, so a chunk's Lambda run
    // together; blocks that finish early take more.
    __shared__ unsigned long long s_item;
    for (;;) {
        __syncthreads();  // the previous item is done with scl, red and s_item
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t item = (int64_t)s_item;
        if (item >= n_items) break;
        const int c = (int)(item / K);
        const int64_t k = item - (int64_t)c * K;
        {
            constexpr int W = (int)(sizeof(LamG) / 8);
            for (int i = threadIdx.x; i < W; i += GRAD_THREADS)
                reinterpret_cast<double*>(&scl)[i] = reinterpret_cast<const double*>(lam + k)[i];
        }
        __syncthreads();
        const LamG& cl = scl;
        const Chunk ch = wd.chunks[c];
        const FeatF64 F = ch.inj ? inj : ev;
        double acc[NG + 1];
#pragma unroll
        for (int p = 0; p <= NG; ++p) acc[p] = 0.0;
        // Same trip count on every thread (slots past the end are dead samples), so the
        // whole warp takes part in the support vote; warps wholly outside the support skip.
        for (int base = 0; base < ch.len; base += GRAD_THREADS) {
            const int j = base + threadIdx.x;
            GSample x{0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0, 0};  // dead slot: finite, out of support
            if (j < ch.len) load_g<HAS_Z>(F, ch.start + j, x);
            const bool in = j < ch.len && in_support_g(x, cl);
            if (__any_sync(0xffffffffu, in)) weight_grad<HAS_Z>(x, cl, stab, kc, in, acc);
        }
#pragma unroll
        for (int p = 0; p <= NG; ++p) {
            double v = acc[p];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][p] = v;
        }
        __syncthreads();
        if (threadIdx.x <= NG) {
            double s = 0.0;
            for (int w = 0; w < GRAD_THREADS / 32; ++w) s += red[w][threadIdx.x];
            if (threadIdx.x < NG) part[(k * wd.n_chunks + c) * NG + threadIdx.x] = s;
            else if (ch.inj) part2[k * n_inj + (c - wd.n_ev_chunks)] = s;
        }
    }
}

constexpr int GFIN_THREADS = 128;

template <int NT>
__device__ double block_sum_g(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < NT / 32; ++i) s += sh[i];
    return s;
}

// ln L, ln xi, N_eff, flags (as the finalise kernel) and the gradient [K][n_params].
__global__ void __launch_bounds__(GFIN_THREADS)
grad_finalise_kernel(const double* __restrict__ part, const double* __restrict__ part2,
                     const int32_t* __restrict__ ecb, const int64_t* __restrict__ off, int64_t n_events,
                     int32_t n_chunks, int32_t n_ev_chunks, int64_t n_draw, const LamG* __restrict__ lam,
                     const int64_t* __restrict__ dK, int n_params, double* lnL, double* lnxi, double* neff,
                     uint32_t* flags, double* grad)
{
    __shared__ double sh[GFIN_THREADS / 32];
    const int64_t k = blockIdx.x;
    if (k >= *dK) return;
    double* G = grad + k * n_params;
    if (!lam[k].valid) {
        if (threadIdx.x == 0) {
            lnL[k] = -INFINITY;
            lnxi[k] = 0.0;
            neff[k] = 0.0;
            flags[k] = POP_FLAG_INVALID_LAMBDA;
        }
        if (threadIdx.x < n_params) G[threadIdx.x] = 0.0;
        return;
    }
    const double* pk = part + k * (int64_t)n_chunks * NG;
    double s_ln = 0.0, zero = 0.0, gs[12];
    for (int p = 0; p < 12; ++p) gs[p] = 0.0;
    for (int64_t i = threadIdx.x; i < n_events; i += GFIN_THREADS) {
        double S = 0.0, Sg[12];
        for (int p = 0; p < 12; ++p) Sg[p] = 0.0;
        for (int32_t c = ecb[i]; c < ecb[i + 1]; ++c) {
            S += pk[c * NG];
            for (int p = 0; p < n_params; ++p) Sg[p] += pk[c * NG + 1 + p];
        }
        if (S == 0.0) {
            zero = 1.0;
        } else {
            s_ln += log(S / (double)(off[i + 1] - off[i]));
            for (int p = 0; p < n_params; ++p) gs[p] += Sg[p] / S;
        }
    }
    const int32_t n_inj = n_chunks - n_ev_chunks;
    double sw = 0.0, sw2 = 0.0, swg[12];
    for (int p = 0; p < 12; ++p) swg[p] = 0.0;
    for (int32_t c = threadIdx.x; c < n_inj; c += GFIN_THREADS) {
        const double* q = pk + (int64_t)(n_ev_chunks + c) * NG;
        sw += q[0];
        sw2 += part2[k * n_inj + c];
        for (int p = 0; p < n_params; ++p) swg[p] += q[1 + p];
    }
    s_ln = block_sum_g<GFIN_THREADS>(s_ln, sh);
    zero = block_sum_g<GFIN_THREADS>(zero, sh);
    sw = block_sum_g<GFIN_THREADS>(sw, sh);
    sw2 = block_sum_g<GFIN_THREADS>(sw2, sh);
    for (int p = 0; p < n_params; ++p) {
        gs[p] = block_sum_g<GFIN_THREADS>(gs[p], sh);
        swg[p] = block_sum_g<GFIN_THREADS>(swg[p], sh);
    }
    if (threadIdx.x != 0) return;
    uint32_t fl = 0;
    const double nd = (double)n_draw;
    const double xi = sw / nd;
    const double var = sw2 / (nd * nd) - xi * xi / nd;
    double ne = var > 0.0 ? xi * xi / var : INFINITY;
    double out, lx;
    if (zero > 0.0) fl |= POP_FLAG_ZERO_EVENT;
    if (xi == 0.0) {
        fl |= POP_FLAG_ZERO_XI;
        out = -INFINITY;
        lx = -INFINITY;
        ne = 0.0;
    } else {
        lx = log(xi);
        out = (fl & POP_FLAG_ZERO_EVENT) ? -INFINITY : s_ln - (double)n_events * lx;
    }
    if (ne < 4.0 * (double)n_events) fl |= POP_FLAG_LOW_NEFF;
    lnL[k] = out;
    lnxi[k] = lx;
    neff[k] = ne;
    flags[k] = fl;
    const bool fin = isfinite(out);
    for (int p = 0; p < n_params; ++p) G[p] = fin ? gs[p] - (double)n_events * swg[p] / sw : 0.0;
}

}  // namespace

size_t lam_grad_bytes() { return sizeof(LamG); }

cudaError_t launch_grad_prologue(const double* lambda, const int64_t* dK, int64_t K_cap, int n_params, void* lam_g,
                                 cudaStream_t s, const double2* ztab, const double2* exptab, ExpConsts kc)
{
    if (K_cap <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((K_cap * 32 + threads - 1) / threads);
    grad_prologue_kernel<<<blocks, threads, 0, s>>>(lambda, dK, n_params, static_cast<LamG*>(lam_g), ztab, exptab,
                                                    kc);
    return cudaGetLastError();
}

cudaError_t launch_grad_weight(int grid, FeatF64 ev, FeatF64 inj, WorkDesc wd, const void* lam_g, const int64_t* dK,
                               int n_params, double* part, double* part2, const double2* exptab, ExpConsts kc,
                               unsigned long long* queue, cudaStream_t s)
{
    const LamG* lg = static_cast<const LamG*>(lam_g);
    const cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (wd.has_z)
        grad_weight_kernel<true><<<grid, GRAD_THREADS, WEIGHT_F64_DYN_SMEM, s>>>(ev, inj, wd, lg, dK, n_params, part,
                                                                               part2, exptab, kc, queue);
    else
        grad_weight_kernel<false><<<grid, GRAD_THREADS, WEIGHT_F64_DYN_SMEM, s>>>(ev, inj, wd, lg, dK, n_params, part,
                                                                                part2, exptab, kc, queue);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalise(const double* part, const double* part2, const int32_t* ecb, const int64_t* off,
                                 int64_t n_events, int32_t n_chunks, int32_t n_ev_chunks, int64_t n_draw,
                                 const void* lam_g, const int64_t* dK, int64_t K_cap, int n_params, double* lnL,
                                 double* lnxi, double* neff, uint32_t* flags, double* grad, cudaStream_t s)
{
    if (K_cap <= 0) return cudaSuccess;
    grad_finalise_kernel<<<(unsigned)K_cap, GFIN_THREADS, 0, s>>>(part, part2, ecb, off, n_events, n_chunks,
                                                                  n_ev_chunks, n_draw,
                                                                  static_cast<const LamG*>(lam_g), dK, n_params, lnL,
                                                                  lnxi, neff, flags, grad);
    return cudaGetLastError();
}

int grad_grid_size(int sm_count)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, grad_weight_kernel<false>, GRAD_THREADS,
                                                      WEIGHT_F64_DYN_SMEM) != cudaSuccess ||
        occ < 1)
        occ = 1;
    return occ * sm_count;
}

}  // namespace pop
