// One-time pack kernels, the per-Lambda prologue and the finalise kernel.
//
// Paper, Sec. "Population acceleration": the N x n_i sample arrays go to the
// GPU once (pack), the population model is evaluated for every sample and
// Lambda (weight kernels, separate files), then the per-event sums, their
// logarithms and the cross-event sum are formed on the device and only the
// log-likelihood comes back (finalise).
#include <math.h>

#include "pop_internal.h"

namespace pop {

namespace {

constexpr double SQRT2 = 1.4142135623730950488;
constexpr double SQRT2PI = 2.5066282746310005024;
constexpr double LN2 = 0.69314718055994530942;
constexpr double LOG2E = 1.4426950408889634074;
constexpr int Z_NODES = 1024;  // redshift normalisation: trapezoid on 1024 nodes of [0, 2]

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// Reads one sample; returns false when the inputs are not usable at all
// (non-finite, or pi <= 0), true otherwise.  `live` is false when the sample
// lies outside the Lambda-independent part of the support.
struct RawSample {
    double m1, q, a1, a2, c1, c2, z, pi;
};

__device__ __forceinline__ bool read_sample(const double* theta, const double* prior, int64_t j, int nd,
                                            RawSample& s, bool& live)
{
    const double* th = theta + j * nd;
    s.m1 = th[0]; s.q = th[1]; s.a1 = th[2]; s.a2 = th[3]; s.c1 = th[4]; s.c2 = th[5];
    s.z = nd == 7 ? th[6] : 1.0;
    s.pi = prior[j];
    bool ok = finite_d(s.m1) && finite_d(s.q) && finite_d(s.a1) && finite_d(s.a2) && finite_d(s.c1) &&
              finite_d(s.c2) && finite_d(s.z) && finite_d(s.pi) && s.pi > 0.0;
    live = ok && s.m1 > 0.0 && s.q > 0.0 && s.q <= 1.0 && s.a1 >= 0.0 && s.a1 <= 1.0 && s.a2 >= 0.0 &&
           s.a2 <= 1.0 && s.c1 >= -1.0 && s.c1 <= 1.0 && s.c2 >= -1.0 && s.c2 <= 1.0 && s.z >= 0.0 && s.z <= 2.0;
    return ok;
}

__device__ __forceinline__ double log_or_zero(double x) { return x > 0.0 ? log(x) : LOG_ZERO; }

// Output slot j takes input sample perm[j] (the load-time order, see pack_samples).
__global__ void pack_f64_kernel(const double* __restrict__ theta, const double* __restrict__ prior,
                                const int64_t* __restrict__ perm, int64_t n, int nd, double* __restrict__ feat,
                                int64_t stride, unsigned long long* bad)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        RawSample s;
        bool live;
        if (!read_sample(theta, prior, perm ? perm[j] : j, nd, s, live)) atomicAdd(bad, 1ull);
        double f[F_COUNT64] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (live) {
            f[F_LM1] = log(s.m1);
            f[F_M1] = s.m1;
            f[F_INVM1] = 1.0 / s.m1;
            f[F_LQ] = log(s.q);
            f[F_SA] = (s.a1 > 0.0 && s.a2 > 0.0) ? log(s.a1) + log(s.a2) : LOG_ZERO;
            f[F_SB] = (s.a1 < 1.0 && s.a2 < 1.0) ? log(1.0 - s.a1) + log(1.0 - s.a2) : LOG_ZERO;
            f[F_DC] = (s.c1 - 1.0) * (s.c1 - 1.0) + (s.c2 - 1.0) * (s.c2 - 1.0);
            f[F_NLPI] = -log(s.pi);
            if (nd == 7) {
                f[F_NLPI] = s.z > 0.0 ? f[F_NLPI] + 2.0 * log(s.z) : LOG_ZERO;
                f[F_LZ1] = log1p(s.z);
            }
            f[F_M2] = __dmul_rn(s.q, s.m1);  // one rounding, as the support test is defined
        }
#pragma unroll
        for (int r = 0; r < F_COUNT64; ++r) feat[r * stride + j] = f[r];
    }
}

// The FP32 features are formed in FP64 from the unrounded inputs and rounded once
// each; m1 and fl64(q m1) are also kept in FP64 for the exact support decisions.
__global__ void pack_f32_kernel(const double* __restrict__ theta, const double* __restrict__ prior,
                                const int64_t* __restrict__ perm, int64_t n, int nd, float* __restrict__ feat,
                                double* __restrict__ m2, double* __restrict__ m1d, int64_t stride,
                                unsigned long long* bad)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        RawSample s;
        bool live;
        if (!read_sample(theta, prior, perm ? perm[j] : j, nd, s, live)) atomicAdd(bad, 1ull);
        float f[F_COUNT32] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        double mm = 0.0, m1 = 0.0;
        if (live) {
            const double l2m1 = log2(s.m1);
            f[F_LM1] = (float)l2m1;
            f[F32_LM1LO] = (float)(l2m1 - (double)f[F_LM1]);
            f[F_M1] = __double2float_rd(s.m1);  // toward -inf: the FP32 upper-edge test never drops a sample
            m1 = s.m1;
            f[F_LQ] = (float)log2(s.q);
            f[F_SA] = (s.a1 > 0.0 && s.a2 > 0.0) ? (float)(log2(s.a1) + log2(s.a2)) : (float)LOG_ZERO;
            f[F_SB] = (s.a1 < 1.0 && s.a2 < 1.0) ? (float)(log2(1.0 - s.a1) + log2(1.0 - s.a2)) : (float)LOG_ZERO;
            f[F_DC] = (float)((s.c1 - 1.0) * (s.c1 - 1.0) + (s.c2 - 1.0) * (s.c2 - 1.0));
            double nl = -log2(s.pi);
            if (nd == 7) {
                nl = s.z > 0.0 ? nl + 2.0 * log2(s.z) : LOG_ZERO;
                f[F_LZ1] = (float)(log1p(s.z) * LOG2E);
            }
            f[F_NLPI] = (float)nl;
            mm = __dmul_rn(s.q, s.m1);  // one rounding, as the support test is defined
        }
#pragma unroll
        for (int r = 0; r < F_COUNT32; ++r) feat[r * stride + j] = f[r];
        m2[j] = mm;
        m1d[j] = m1;
    }
}

__device__ __forceinline__ int64_t dbits(double x) { return __double_as_longlong(x); }

// Redshift normalisation per Lambda, I(kappa) = trapezoid of (1+z)^(kappa-1) z^2 on
// z_k = 2k/1023: one block of 4 warps per Lambda, the threads share the 1024 nodes (a warp per
// Lambda left each scheduler under two warps to hide the exponentials' latency).  With ztab (node i:
// ln(1 + z_i) and its trapezoid weight times z_i^2) each node costs one table-driven
// exponential; without it (callers that hold no tables) the logarithm and exponential are
// evaluated directly.
constexpr int ZINT_THREADS = 128;
static_assert(ZINT_THREADS == 128, "the block's four warp partials are added in order below");

__global__ void __launch_bounds__(ZINT_THREADS)
zint_kernel(const double* __restrict__ lambda, const int64_t* __restrict__ dK, int n_params,
            const double2* __restrict__ ztab, const double2* __restrict__ exptab, ExpConsts kc,
            double* __restrict__ zint)
{
    __shared__ double s_part[ZINT_THREADS / 32];
    const int64_t k = blockIdx.x;
    if (k >= *dK) return;  // the same for the whole block
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double km1 = lambda[k * n_params + P_KAPPA] - 1.0;
    double zs = 0.0;
    if (ztab) {
        for (int i = threadIdx.x; i < Z_NODES; i += ZINT_THREADS) {
            const double2 t = ztab[i];
            zs = fma(t.y, exp_tab(km1 * t.x, exptab, kc), zs);
        }
    } else {
        for (int i = threadIdx.x; i < Z_NODES; i += ZINT_THREADS) {
            double z = 2.0 * i / (Z_NODES - 1);
            double f = exp(km1 * log1p(z)) * z * z;
            zs += (i == 0 || i == Z_NODES - 1) ? 0.5 * f : f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) zs += __shfl_xor_sync(0xffffffffu, zs, o);
    if (lane == 0) s_part[w] = zs;
    __syncthreads();
    if (threadIdx.x == 0)
        zint[k] = (((s_part[0] + s_part[1]) + s_part[2]) + s_part[3]) * (2.0 / (Z_NODES - 1));
}

// Per-Lambda constants, 32 Lambda per block of 4 warps, lane = Lambda: the special functions
// of a warp's 32 Lambda share each FP64 instruction (an FP64 warp instruction costs the same for
// one lane or 32), and the block's 4 warps, on the SM's 4 schedulers, split them: warps 1-3 take
// the lgamma and erf terms, warp 0 the logs meanwhile, then combines.  zint from zint_kernel when
// the model has redshift.
constexpr int PRO_THREADS = 128;

__global__ void __launch_bounds__(PRO_THREADS)
prologue_kernel(const double* __restrict__ lambda, const int64_t* __restrict__ dK, int n_params,
                LamF64* __restrict__ c64, LamF32* __restrict__ c32, const double* __restrict__ zint)
{
    __shared__ double s_lb[32], s_lab[32], s_cg[32], s_ct[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * 32LL + lane;
    const bool live = k < *dK;
    const double* L = lambda + (live ? k : 0) * n_params;
    const bool has_z = n_params == 12;

    bool valid = live;
    for (int p = 0; p < n_params && live; ++p) valid = valid && finite_d(L[p]);
    // Lanes past K or with bad rows evaluate the special functions at 1 (their results unused).
    const double one = 1.0;
    const double alpha = valid ? L[P_ALPHA] : one, beta = valid ? L[P_BETA] : one;
    const double mmin = valid ? L[P_MMIN] : one, mmax = valid ? L[P_MMAX] : 2.0;
    const double lam = valid ? L[P_LAM] : 0.5, mu = valid ? L[P_MPP] : one, sig = valid ? L[P_SIGPP] : one;
    const double ach = valid ? L[P_ACHI] : one, bch = valid ? L[P_BCHI] : one;
    const double xit = valid ? L[P_XIT] : 0.5, sigt = valid ? L[P_SIGT] : one;
    valid = valid && mmin > 0.0 && mmin < mmax && lam >= 0.0 && lam <= 1.0 && sig > 0.0 && sigt > 0.0 &&
            ach > 0.0 && bch > 0.0 && xit >= 0.0 && xit <= 1.0;
    double lmmin = 0.0, ln_cpl = 0.0, ln_qn = 0.0, ln_iz = 0.0, l1lam = 0.0, l2mmin = 0.0;
    const double b1 = 1.0 + beta;
    const int beta_m1 = b1 == 0.0;
    if (w == 1) {
        s_lb[lane] = lgamma(ach) + lgamma(bch);
    } else if (w == 2) {
        s_lab[lane] = lgamma(ach + bch);
        // Tilt: C_t = 1 / (sigma_t sqrt(2 pi) * erf(sqrt2 / sigma_t) / 2); ct = ln(xi_t C_t^2).
        s_ct[lane] = log(xit) - 2.0 * log(sigt * SQRT2PI * 0.5 * erf(SQRT2 / sigt));
    } else if (w == 3) {
        // Truncated Gaussian on [mmin, mmax]: C_g = 1 / (sigma sqrt(2 pi) Z_m).
        const double zm = 0.5 * (erf((mmax - mu) / (SQRT2 * sig)) - erf((mmin - mu) / (SQRT2 * sig)));
        s_cg[lane] = log(lam) - log(sig * SQRT2PI * zm);
    } else {
        lmmin = log(mmin);
        const double lmmax = log(mmax);
        // Power law: C_pl = (1-alpha) / (mmax^(1-alpha) - mmin^(1-alpha)), in logs.
        if (alpha == 1.0) {
            ln_cpl = -log(lmmax - lmmin);
        } else {
            const double oma = 1.0 - alpha;
            ln_cpl = log(fabs(oma)) - oma * lmmin - log(fabs(expm1(oma * (lmmax - lmmin))));
        }
        ln_qn = beta_m1 ? 0.0 : log(fabs(b1));
        ln_iz = has_z && live ? log(zint[k]) : 0.0;
        l1lam = log1p(-lam);
        l2mmin = log2(mmin);
    }
    __syncthreads();  // the one barrier: warps 1-3 have written their terms
    if (w != 0 || !live) return;

    LamF64 c;
    LamF32 f;
    if (!valid) {
        c = LamF64{};
        c.mmin_bits = dbits(INFINITY);
        c.mmax_bits = dbits(INFINITY);
        c.valid = 0;
        f = LamF32{};
        f.mmin_bits = c.mmin_bits;
        f.mmax_bits = c.mmax_bits;
        f.thr_hi = INFINITY;
        f.valid = 0;
        c64[k] = c;
        c32[k] = f;
        return;
    }
    const double ln_beta = s_lb[lane] - s_lab[lane];
    const double common = ln_qn - 2.0 * ln_beta - ln_iz;
    const double ln_cg = s_cg[lane];

    c.mmin_bits = dbits(mmin);
    c.mmax_bits = dbits(mmax);
    c.nalpha = -alpha;
    c.cpl = common + l1lam + ln_cpl;
    c.mu = mu;
    c.nh = -0.5 / (sig * sig);
    c.cg = common + ln_cg;
    c.beta = beta;
    c.ac = ach - 1.0;
    c.bc = bch - 1.0;
    c.km1 = has_z ? L[P_KAPPA] - 1.0 : 0.0;
    c.b1 = b1;
    c.mmin = mmin;
    c.lmmin = lmmin;
    c.kq = beta_m1 ? 1.0 : b1;
    c.kqlmmin = c.kq * lmmin;
    c.nht = -0.5 / (sigt * sigt);
    c.ct = s_ct[lane];
    c.t0 = 0.25 * (1.0 - xit);
    c.gs = 1.0 / (SQRT2 * sig);
    c.gc = -mu * c.gs;
    const double cmax = fmax(c.cpl, c.cg);
    c.mix_swap = c.cg > c.cpl;
    c.rmix = exp(fmin(c.cpl, c.cg) - cmax);
    c.t0m = exp(cmax) * c.t0;
    c.ctm = c.ct + cmax;
    c.beta_m1 = beta_m1;
    c.valid = 1;
    c64[k] = c;

    // FP32 copy in base-2 units.  With beta = -1 the q normalisation ln(m1/mmin)
    // is formed from base-2 logs, so 1/ln 2 joins the constant.
    const double fix = beta_m1 ? -log(LN2) : 0.0;
    f.mmin_bits = c.mmin_bits;
    f.mmax_bits = c.mmax_bits;
    f.thr_hi = __double2float_rd(mmax);
    f.nalpha = (float)c.nalpha;
    f.cpl = (float)((c.cpl + fix) * LOG2E);
    f.mu = (float)mu;
    f.nh = (float)(c.nh * LOG2E);
    f.cg = (float)((c.cg + fix) * LOG2E);
    f.beta = (float)beta;
    f.ac = (float)c.ac;
    f.bc = (float)c.bc;
    f.km1 = (float)c.km1;
    const double b1f = beta_m1 ? 1.0 : b1;
    f.lmmin = (float)l2mmin;
    f.b1 = (float)b1f;
    f.nb1 = (float)-b1f;
    f.b1lmmin_lo = (float)(b1f * (l2mmin - (double)f.lmmin));
    f.nht = (float)(c.nht * LOG2E);
    f.ct = (float)(c.ct * LOG2E);
    f.t0 = (float)c.t0;
    f.beta_m1 = beta_m1;
    f.valid = 1;
    c32[k] = f;
}

constexpr int FIN_THREADS = 256;

// ln L = sum_i ln(S_i / n_i) - N ln xi, plus ln xi, N_eff and flags.
__global__ void __launch_bounds__(FIN_THREADS)
finalise_kernel(const double* __restrict__ part, const double* __restrict__ part2,
                const int32_t* __restrict__ ecb, const int64_t* __restrict__ off, int64_t n_events,
                int32_t n_chunks, int32_t n_ev_chunks, int64_t n_draw, const LamF64* __restrict__ lam,
                const int64_t* __restrict__ dK, double* lnL, double* lnxi, double* neff, uint32_t* flags,
                SurrogateXi sx, const double* __restrict__ grid_xi, double* __restrict__ parts,
                const LogEntry* __restrict__ logtab, LogConsts logc, const double* __restrict__ inv_n)
{
    __shared__ double sh[FIN_THREADS / 32][3];
    const int64_t k = blockIdx.x;
    if (k >= *dK) return;
    if (!lam[k].valid) {
        if (threadIdx.x == 0) {
            lnL[k] = -INFINITY;
            lnxi[k] = 0.0;
            neff[k] = 0.0;
            flags[k] = POP_FLAG_INVALID_LAMBDA;
            if (parts) {
                parts[3 * k] = -INFINITY;
                parts[3 * k + 1] = 0.0;
                parts[3 * k + 2] = 0.0;
            }
        }
        return;
    }
    const double* pk = part + k * (int64_t)n_chunks;
    double s_ln = 0.0;
    int zero = 0;
    for (int64_t i = threadIdx.x; i < n_events; i += FIN_THREADS) {
        double S = 0.0;
        for (int32_t c = ecb[i]; c < ecb[i + 1]; ++c) S += pk[c];
        if (S == 0.0) {
            zero = 1;
        } else if (logtab) {
            // ln(S/n) as log_pos(S (1/n)) (within 1 ulp of S/n; 8 FP64 operations against the
            // division's and the library log's dozens), 1/n from the table or a Newton step.
            s_ln += log_pos(S * (inv_n ? inv_n[i] : rcp_pos((double)(off[i + 1] - off[i]))), logtab, logc);
        } else {
            s_ln += log(S / (double)(off[i + 1] - off[i]));
        }
    }
    const int32_t n_inj = n_chunks - n_ev_chunks;
    const double* p2 = part2 + k * (int64_t)n_inj;
    double sw = 0.0, sw2 = 0.0;
    for (int32_t c = threadIdx.x; c < n_inj; c += FIN_THREADS) {
        sw += pk[n_ev_chunks + c];
        sw2 += p2[c];
    }
    // One fixed-order reduction of the three sums: the shuffle tree in the warps that hold any
    // item (an FP64 warp instruction costs the same with idle lanes), the warps' partials added
    // in order by three lanes of warp 0; the zero-event flag by the barrier's OR.
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v[3] = {s_ln, sw, sw2};
    if ((int64_t)w * 32 < max(n_events, (int64_t)n_inj)) {  // warp-uniform; later warps hold zeros
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q) sh[w][q] = v[q];
    const int any_zero = __syncthreads_or(zero);
    if (w != 0) return;
    double tot = 0.0;
    if (lane < 3)
        for (int u = 0; u < FIN_THREADS / 32; ++u) tot += sh[u][lane];
    s_ln = __shfl_sync(0xffffffffu, tot, 0);
    sw = __shfl_sync(0xffffffffu, tot, 1);
    sw2 = __shfl_sync(0xffffffffu, tot, 2);
    const double zero_any = any_zero ? 1.0 : 0.0;
    if (threadIdx.x != 0) return;
    if (parts) {  // the additive parts: event log-sum, injection sum w and sum w^2
        parts[3 * k] = zero_any > 0.0 ? -INFINITY : s_ln;
        parts[3 * k + 1] = sw;
        parts[3 * k + 2] = sw2;
    }
    uint32_t fl = 0;
    const double nd = (double)n_draw;
    double xi = sw / nd;
    const double var = sw2 / (nd * nd) - xi * xi / nd;
    double ne = var > 0.0 ? xi * xi / var : INFINITY;
    double out, lx;
    if (zero_any > 0.0) fl |= POP_FLAG_ZERO_EVENT;
    if (grid_xi) {  // selection term from the grid: no Monte Carlo variance
        xi = grid_xi[k];
        ne = INFINITY;
    }
    if (sx.need_mc) {
        if (sx.need_mc[k]) {
            fl |= POP_FLAG_MC_FALLBACK;
        } else {  // selection term from the surrogate network
            fl |= POP_FLAG_SURROGATE_USED;
            xi = exp(sx.lnxi[k]);
            ne = exp(sx.neff[k]);
        }
    }
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
}

// One warp per block of M1MAX_BLOCK samples.  The values are clamped at 0 from below (an upper
// bound is all the caller needs), so their float bits order like the values.
__global__ void m1_blockmax_kernel(const float* __restrict__ m1, int64_t n, float* __restrict__ m1max)
{
    static_assert(M1MAX_BLOCK == 64, "two samples per lane");
    const int64_t nb = (n + M1MAX_BLOCK - 1) / M1MAX_BLOCK;
    const int lane = threadIdx.x & 31;
    for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; b < nb;
         b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t j = b * M1MAX_BLOCK + lane;
        float v = j < n ? fmaxf(m1[j], 0.0f) : 0.0f;
        if (j + 32 < n) v = fmaxf(v, m1[j + 32]);
        const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
        if (lane == 0) m1max[b] = __uint_as_float(mx);
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 65535LL * 32) b = 65535LL * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_pack_f64(const double* theta, const double* prior, const int64_t* perm, int64_t n, int n_dims,
                            double* feat, int64_t stride, unsigned long long* bad, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    pack_f64_kernel<<<grid_for(n, 256), 256, 0, s>>>(theta, prior, perm, n, n_dims, feat, stride, bad);
    return cudaGetLastError();
}

cudaError_t launch_m1_blockmax(const float* feat, int64_t stride, int64_t n, float* m1max, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + M1MAX_BLOCK - 1) / M1MAX_BLOCK;
    m1_blockmax_kernel<<<grid_for(nb * 32, 256), 256, 0, s>>>(feat + F_M1 * stride, n, m1max);
    return cudaGetLastError();
}

cudaError_t launch_pack_f32(const double* theta, const double* prior, const int64_t* perm, int64_t n, int n_dims,
                            float* feat, double* m2, double* m1d, int64_t stride, unsigned long long* bad,
                            cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    pack_f32_kernel<<<grid_for(n, 256), 256, 0, s>>>(theta, prior, perm, n, n_dims, feat, m2, m1d, stride, bad);
    return cudaGetLastError();
}

cudaError_t launch_prologue(const double* lambda, const int64_t* dK, int64_t K_cap, int n_params, LamF64* c64,
                            LamF32* c32, double* zint, cudaStream_t s, const double2* ztab, const double2* exptab,
                            ExpConsts kc)
{
    if (K_cap <= 0) return cudaSuccess;
    if (n_params == 12) {
        if (!zint) return cudaErrorInvalidValue;
        zint_kernel<<<(unsigned)K_cap, ZINT_THREADS, 0, s>>>(lambda, dK, n_params, ztab, exptab, kc, zint);
    }
    // 32 Lambda per block (4 warps), so that a small batch still spreads over many SMs.
    prologue_kernel<<<(unsigned)((K_cap + 31) / 32), PRO_THREADS, 0, s>>>(lambda, dK, n_params, c64, c32, zint);
    return cudaGetLastError();
}

void build_z_table(double2* tab)
{
    for (int i = 0; i < Z_NODES; ++i) {
        const double z = 2.0 * i / (Z_NODES - 1);
        tab[i] = make_double2(log1p(z), ((i == 0 || i == Z_NODES - 1) ? 0.5 : 1.0) * z * z);
    }
}

cudaError_t launch_finalise(const double* part, const double* part2, const int32_t* ecb, const int64_t* off,
                            int64_t n_events, int32_t n_chunks, int32_t n_ev_chunks, int64_t n_draw,
                            const LamF64* lam, const int64_t* dK, int64_t K_cap, double* lnL, double* lnxi,
                            double* neff, uint32_t* flags, cudaStream_t s, SurrogateXi sx, const double* grid_xi,
                            double* parts, const LogEntry* logtab, LogConsts logc, const double* inv_n)
{
    if (K_cap <= 0) return cudaSuccess;
    finalise_kernel<<<(unsigned)K_cap, FIN_THREADS, 0, s>>>(part, part2, ecb, off, n_events, n_chunks, n_ev_chunks,
                                                            n_draw, lam, dK, lnL, lnxi, neff, flags, sx, grid_xi, parts,
                                                            logtab, logc, inv_n);
    return cudaGetLastError();
}

}  // namespace pop
