// Selection term on a regular (m1, q) grid: pdet packing, the per-Lambda
// q-node factors U_b, the masked node contraction and its fixed-order
// reduction (paper, Sec. "Population acceleration": VT on a regular grid with
// GPU acceleration, low-dimensional, no spin effects).
//
// Work layout.  The contraction sum_a W_a sum_{b >= b0} pdet[a, b] U_b runs over
// tiles of m1 rows x Lambda columns whose chunks of 32 q nodes (packed pdet and U)
// are staged in shared memory by cp.async.bulk copies that complete on mbarriers.
// In both forms a setup kernel first computes W_a and b0 of every (row, column) pair
// at full occupancy: FP64 with the table-driven exp/expm1 of the FP64 weight kernel,
// FP32 with CUDA's exp2f/log1pf/expm1f; the support decisions are FP64 in both.
// FP64: tiles of 32 rows x 64 columns in 4 parts of the q range, one CTA each, 2 x 4
// (row, column) accumulators per thread.  FP32: persistent CTAs contract tiles of 128
// rows x 128 columns in 4 parts of the q range with 8 x 8 accumulators per thread (see
// the FP32 section).
// Lambda columns are placed in ascending mmin order (a counting sort per slice)
// so that the columns of a thread or warp have nearly the same lower q edges:
// chunks at or past every edge run unmasked, chunks below all of them are
// skipped, and only the chunks between use a per-pair mask.  The result of a
// column does not depend on where the sort puts it: the sum over b of a pair runs
// in node order, and the sum over rows in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "pop.h"
#include "pop_f32x2.cuh"
#include "pop_gridvt.h"
#include "pop_internal.h"

namespace pop {

namespace {

constexpr int GV_THREADS = 256;

// mbarrier polls before a wait gives up.  A poll of a phase that is not complete suspends the
// thread about 3.8 us on GB300 (measured through pop_wait_check), so this is about 1 s; a
// tile's bulk copies complete within microseconds.
constexpr int GV_WAIT_LIMIT = 1 << 18;
constexpr int GV_BUCKETS = 1024;        // mmin buckets of the column sort
constexpr double GV_SQRT2 = 1.4142135623730950488;
constexpr double GV_SQRT2PI = 2.5066282746310005024;
constexpr double GV_LOG2E = 1.4426950408889634074;

struct GvNodes {
    const double* m1;     // [na]
    const double* lnm1;   // [na]
    const double* invm1;  // [na]
    const double* wa;     // [na]
    const float* m1f;     // [na] m1 rounded to FP32 ...
    const float* m1lf;    // [na] ... and the rest, m1 - m1f, rounded to FP32
    const float* invm1f;  // [na]
    const float* l2m1f;   // [na] log2 m1
    const float* waf;     // [na]
    const double* q;      // [nbp]
    const double* lnq;    // [nbp]
    const float* qf;      // [nbp]
    const float* l2q_h;   // [nbp] log2 q as an FP32 (hi, lo) pair
    const float* l2q_l;
    const float* wqf;     // [nbp]
    const int* qbk;       // [nqb + 1] first node of each of nqb equal-width bins over [qf[0], qf[nb - 1]]
    float qb0, qbinv;     // qf[0] and 1 / bin width (0 with one bin)
    int nqb;
    int na, nb, nbp;
};

// Per-column constants of the primary-mass and mass-ratio densities.  The
// log-normalisations lcpl and lcg include ln|1 + beta| (0 when beta = -1).
struct GvLam {
    double nalpha;  // exponent of m1 in the power law (-alpha)
    double lcpl;    // ln((1 - lam) C_pl |1 + beta|)   (-inf when lam = 1)
    double mu, nh;  // Gaussian peak: mpp and -1 / (2 sigpp^2)
    double lcg;     // ln(lam C_g |1 + beta|), C_g = 1 / (sqrt(2 pi) sigpp Z)   (-inf when lam = 0)
    double b1;      // 1 + beta
    double beta;
    float beta_h, beta_l;  // beta as an FP32 (hi, lo) pair
    double mmin, lmmin;
    long long mmin_bits, mmax_bits;  // non-negative doubles order like their bit patterns
    float nalpha_f, l2cpl_f, nh2_f, l2cg_f, b1_f;  // FP32 form, base-2 logs
    float mu_h, mu_l, mmin_f, mmin_l;              // mpp and mmin as FP32 (hi, lo) pairs
    int beta_m1;    // beta == -1: the q normalisation is ln(m1 / mmin)
    int live;       // a valid Lambda occupies the column
};

// Domain of the population model (the same rules as the likelihood's).
__device__ bool gv_valid(const double* L, int P)
{
    for (int p = 0; p < P; ++p)
        if (!isfinite(L[p])) return false;
    return L[P_MMIN] > 0.0 && L[P_MMIN] < L[P_MMAX] && L[P_LAM] >= 0.0 && L[P_LAM] <= 1.0 && L[P_SIGPP] > 0.0 &&
           L[P_SIGT] > 0.0 && L[P_ACHI] > 0.0 && L[P_BCHI] > 0.0 && L[P_XIT] >= 0.0 && L[P_XIT] <= 1.0;
}

__device__ void gv_consts(const double* L, int P, GvLam& c)
{
    c.live = gv_valid(L, P);
    if (!c.live) return;
    const double alpha = L[P_ALPHA], beta = L[P_BETA], mmin = L[P_MMIN], mmax = L[P_MMAX], lam = L[P_LAM];
    c.beta_m1 = beta == -1.0;
    const double lb1 = c.beta_m1 ? 0.0 : log(fabs(1.0 + beta));
    // Power law x^-alpha on [mmin, mmax]: ln of its normalisation (alpha = 1: 1 / ln(mmax / mmin)).
    const double lpl = alpha == 1.0 ? -log(log(mmax / mmin))
                                    : log((1.0 - alpha) / (pow(mmax, 1.0 - alpha) - pow(mmin, 1.0 - alpha)));
    c.nalpha = -alpha;
    c.lcpl = log1p(-lam) + lpl + lb1;
    const double mu = L[P_MPP], sig = L[P_SIGPP];
    c.mu = mu;
    c.nh = -0.5 / (sig * sig);
    if (lam > 0.0) {
        const double z = 0.5 * (erf((mmax - mu) / (GV_SQRT2 * sig)) - erf((mmin - mu) / (GV_SQRT2 * sig)));
        c.lcg = log(lam / (GV_SQRT2PI * sig * z)) + lb1;
    } else {
        c.lcg = -INFINITY;
    }
    c.b1 = 1.0 + beta;
    c.beta = beta;
    c.beta_h = (float)beta;
    c.beta_l = (float)(beta - (double)c.beta_h);
    c.mmin = mmin;
    c.lmmin = log(mmin);
    c.mmin_bits = __double_as_longlong(mmin);
    c.mmax_bits = __double_as_longlong(mmax);
    c.nalpha_f = (float)c.nalpha;
    c.l2cpl_f = (float)(c.lcpl * GV_LOG2E);
    c.nh2_f = (float)(c.nh * GV_LOG2E);
    c.l2cg_f = (float)(c.lcg * GV_LOG2E);
    c.b1_f = (float)c.b1;
    c.mu_h = (float)mu;
    c.mu_l = (float)(mu - (double)c.mu_h);
    c.mmin_f = (float)mmin;
    c.mmin_l = (float)(mmin - (double)c.mmin_f);
}

// First q node with fl64(q_b m1) >= mmin.  The product rounds once and is
// monotone in q, so the support in b is the suffix [b0, nb).
// An FP32 search for thr = mmin_f / m1_f gives j.  thr is within 2^-21 of
// x = mmin/m1 and every FP32 node within 2^-24 of its FP64 node, so a node
// whose FP32 value is above thr (1 + 2^-18) is above x (1 + 2^-19) and passes
// the FP64 test (which rounds once, 2^-53), and one below thr (1 - 2^-18)
// fails it.  When both neighbours of j are that clear, j is exact; otherwise
// (a node within ~2^-18 of the edge) the FP64 test itself moves j.
// The FP32 search starts from the bin of thr: a binary search over the bin's nodes, then a
// walk to the first node >= thr (the bin index is a rounded float, so the bin can miss by a node).
__device__ __forceinline__ int gv_edge(const GvNodes& g, double m1, double mmin, float thr)
{
    const float x = (thr - g.qb0) * g.qbinv;
    const int k = !(x > 0.0f) ? 0 : (x >= (float)g.nqb ? g.nqb - 1 : (int)x);
    int lo = __ldg(g.qbk + k), hi = __ldg(g.qbk + k + 1);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (g.qf[mid] >= thr) hi = mid;
        else lo = mid + 1;
    }
    int j = lo;
    while (j > 0 && g.qf[j - 1] >= thr) --j;
    while (j < g.nb && g.qf[j] < thr) ++j;
    const bool clear_above = j == g.nb || g.qf[j] >= thr * (1.0f + 0x1p-18f);
    const bool clear_below = j == 0 || g.qf[j - 1] < thr * (1.0f - 0x1p-18f);
    if (clear_above && clear_below) return j;
    while (j > 0 && __dmul_rn(g.q[j - 1], m1) >= mmin) --j;
    while (j < g.nb && __dmul_rn(g.q[j], m1) < mmin) ++j;
    return j;
}

// Mass support mmin < m1 <= mmax on bit patterns (every padding row has m1 = 0).
__device__ __forceinline__ bool gv_in_mass(long long mb, const GvLam& c)
{
    return c.live && mb > c.mmin_bits && mb <= c.mmax_bits;
}

// W_a and b0 of one (row, column) pair, FP64: wa p(m1) (1+beta) / |expm1((1+beta) ln(mmin/m1))|
// with the table-driven exponentials (tab in shared memory).  A pair outside the mass support
// (or with an empty q range) gets b0 = nb and contributes nothing.
__device__ __forceinline__ void gv_pair64(const GvNodes& g, const GvLam& c, int a, const double2* tab,
                                          const ExpConsts& kc, double& W, int& b0)
{
    W = 0.0;
    b0 = g.nb;
    const double m1 = g.m1[a];
    const long long mb = __double_as_longlong(m1);
    if (!gv_in_mass(mb, c)) return;
    const double lm = g.lnm1[a];
    const double e1 = exp_tab(fma(c.nalpha, lm, c.lcpl), tab, kc);
    const double d = m1 - c.mu;
    const double e2 = exp_tab(fma(c.nh * d, d, c.lcg), tab, kc);
    // ln(mmin/m1): the log difference, or near the edge log1p((mmin - m1)/m1) by its series
    // (mmin - m1 is exact there).
    double lr = c.lmmin - lm;
    if (llabs(mb - c.mmin_bits) < NEAR_EDGE_BITS) lr = log1p_near0(g.invm1[a] * (c.mmin - m1));
    const double den = c.beta_m1 ? -lr : fabs(expm1_tab(c.b1 * lr, tab, kc));
    W = g.wa[a] * (e1 + e2) * rcp_pos(den);
    b0 = gv_edge(g, m1, c.mmin, __fdividef(c.mmin_f, g.m1f[a]));
}

// Per-row and per-column constants of the FP32 form, packed for 16-byte loads.
struct alignas(16) GvRow32 {
    double m1;
    float m1f, m1lf, l2m1f, invm1f, waf, pad;  // m1 as an FP32 (hi, lo) pair, log2 m1, 1/m1, trapezoid weight
};
struct alignas(16) GvCol32 {
    long long mmin_bits, mmax_bits;  // -1 in both for a column without a valid Lambda
    float nalpha_f, l2cpl_f, mu_h, mu_l, nh2_f, l2cg_f, mmin_f, mmin_l, b1_f;
    int beta_m1, pad[2];
};
static_assert(sizeof(GvRow32) == 32 && sizeof(GvCol32) == 64, "two and four 16-byte words");

template <class T>
__device__ __forceinline__ T gv_ld16(const T* p)
{
    T v;
    const int4* s = reinterpret_cast<const int4*>(p);
    int4* d = reinterpret_cast<int4*>(&v);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(T) / 16); ++w) d[w] = __ldg(s + w);
    return v;
}

// The same pair in the FP32 form: base-2 exponentials and log1p/expm1 in FP32
// (CUDA exp2f, log1pf, expm1f).  m1 - mpp and mmin - m1 come from (hi, lo) FP32
// pairs; within ~2^-6 of the lower mass edge mmin - m1 is taken in FP64, where
// it is exact.
__device__ __forceinline__ void gv_pair32(const GvNodes& g, const GvCol32& c, const GvRow32& r, int a, float& W,
                                          int& b0)
{
    W = 0.0f;
    b0 = g.nb;
    const long long mb = __double_as_longlong(r.m1);
    if (!(mb > c.mmin_bits && mb <= c.mmax_bits)) return;
    const float e1 = exp2f(fmaf(c.nalpha_f, r.l2m1f, c.l2cpl_f));
    const float d = (r.m1f - c.mu_h) + (r.m1lf - c.mu_l);
    const float e2 = exp2f(fmaf(c.nh2_f * d, d, c.l2cg_f));
    const double mmin = __longlong_as_double(c.mmin_bits);
    float t;
    if (llabs(mb - c.mmin_bits) < NEAR_EDGE_BITS) t = (float)(g.invm1[a] * (mmin - r.m1));
    else t = ((c.mmin_f - r.m1f) + (c.mmin_l - r.m1lf)) * r.invm1f;
    const float lr = log1pf(t);
    const float den = c.beta_m1 ? -lr : fabsf(expm1f(c.b1_f * lr));
    W = r.waf * (e1 + e2) * __frcp_rn(den);
    b0 = gv_edge(g, r.m1, mmin, __fdividef(c.mmin_f, r.m1f));
}

__device__ __forceinline__ int slice_count(const int64_t* dK, int64_t slice0, int S)
{
    const int64_t n = *dK - slice0;
    return (int)(n < 0 ? 0 : (n > S ? S : n));
}

// ---------------------------------------------------------------- column sort
// perm[r] = Lambda index of column r of the slice (-1 in the padding).  The
// columns go in ascending mmin by buckets, and inside every 64-column tile in
// ascending mmax: a warp's 16 columns then share nearly the same support in
// both m1 (dead rows are dead for the whole warp) and q.  Order inside an
// mmin bucket is arbitrary: every column's result is independent of its position.
__global__ void __launch_bounds__(1024)
gv_sort_kernel(const double* __restrict__ lambda, int P, const int64_t* __restrict__ dK, int64_t slice0, int S,
               int32_t* __restrict__ perm)
{
    // Dynamic shared memory: histogram [GV_BUCKETS + 1], columns [S], mmax keys [S].
    extern __shared__ int gv_sort_smem[];
    int* hist = gv_sort_smem;
    int32_t* sperm = gv_sort_smem + (GV_BUCKETS + 4);
    float* skey = reinterpret_cast<float*>(sperm + S);
    __shared__ double s_lo[32], s_hi[32];
    const int n = slice_count(dK, slice0, S);
    double lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double m = lambda[(slice0 + i) * P + P_MMIN];
        if (isfinite(m)) {
            lo = fmin(lo, m);
            hi = fmax(hi, m);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    for (int i = threadIdx.x; i <= GV_BUCKETS; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    lo = INFINITY;
    hi = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        lo = fmin(lo, s_lo[w]);
        hi = fmax(hi, s_hi[w]);
    }
    const double scale = hi > lo ? GV_BUCKETS / (hi - lo) : 0.0;
    auto bucket = [&](double m) -> int {
        if (!isfinite(m)) return GV_BUCKETS;
        const int b = (int)((m - lo) * scale);
        return b < 0 ? 0 : (b >= GV_BUCKETS ? GV_BUCKETS - 1 : b);
    };
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&hist[bucket(lambda[(slice0 + i) * P + P_MMIN])], 1);
    __syncthreads();
    // Exclusive prefix sum of the buckets by one warp: each lane scans 32 buckets,
    // a shuffle scan gives the lane offsets; the non-finite bucket goes last.
    static_assert(GV_BUCKETS == 32 * 32, "one warp scans the buckets");
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        int tot = 0;
        for (int b = 32 * l; b < 32 * l + 32; ++b) tot += hist[b];
        int incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (l >= o) incl += v;
        }
        int run = incl - tot;
        for (int b = 32 * l; b < 32 * l + 32; ++b) {
            const int h = hist[b];
            hist[b] = run;
            run += h;
        }
        if (l == 31) hist[GV_BUCKETS] = run;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int pos = atomicAdd(&hist[bucket(lambda[(slice0 + i) * P + P_MMIN])], 1);
        sperm[pos] = (int32_t)(slice0 + i);
    }
    const int npad = (n + GV_TL - 1) / GV_TL * GV_TL;
    for (int r = n + threadIdx.x; r < npad; r += blockDim.x) sperm[r] = -1;
    __syncthreads();
    // Rank by mmax inside each 64-column tile (padding and non-finite keys last, ties by
    // position); the keys go to shared memory first, as floats (ordering only).
    for (int r = threadIdx.x; r < npad; r += blockDim.x) {
        const int32_t k = sperm[r];
        const double m = k >= 0 ? lambda[(int64_t)k * P + P_MMAX] : INFINITY;
        skey[r] = isfinite(m) ? (float)m : INFINITY;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < npad; r += blockDim.x) {
        const int t0 = r / GV_TL * GV_TL;
        const float kr = skey[r];
        int rank = 0;
        for (int u = t0; u < t0 + GV_TL; ++u) {
            const float ku = skey[u];
            rank += (ku < kr) || (ku == kr && u < r);
        }
        perm[t0 + rank] = sperm[r];
    }
}

// Per-column constants of the slice (live = 0 for padding columns).
__global__ void gv_lamc_kernel(const double* __restrict__ lambda, int P, const int32_t* __restrict__ perm,
                               const int64_t* __restrict__ dK, int64_t slice0, int S, GvLam* __restrict__ lamc,
                               GvCol32* __restrict__ lamc32)
{
    const int n = slice_count(dK, slice0, S);
    const int npad = (n + 127) / 128 * 128;  // whole tiles of both contractions (64 and 128 columns)
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= npad) return;
    const int k = r < n ? perm[r] : -1;
    GvLam c;
    c.live = 0;
    c.beta = 0.0;
    if (k >= 0) gv_consts(lambda + (int64_t)k * P, P, c);
    lamc[r] = c;
    GvCol32 c32{};
    c32.mmin_bits = c.live ? c.mmin_bits : -1;
    c32.mmax_bits = c.live ? c.mmax_bits : -1;
    if (c.live) {
        c32.nalpha_f = c.nalpha_f;
        c32.l2cpl_f = c.l2cpl_f;
        c32.mu_h = c.mu_h;
        c32.mu_l = c.mu_l;
        c32.nh2_f = c.nh2_f;
        c32.l2cg_f = c.l2cg_f;
        c32.mmin_f = c.mmin_f;
        c32.mmin_l = c.mmin_l;
        c32.b1_f = c.b1_f;
        c32.beta_m1 = c.beta_m1;
    }
    lamc32[r] = c32;
}

// ---------------------------------------------------------------- tile order
// Launch order of the row tiles, heaviest first, so that the light tiles (near
// the lower mass edge, above mmax, outside every support) fill the end of the
// launch.  The work of a row tile is estimated from 16 columns spread over the
// slice and every 4th row: the number of q nodes in the support of each (row,
// column) pair.  Up to GV_ORDER_MAX row tiles; beyond that the order is the identity.
constexpr int GV_ORDER_MAX = 4096;

__global__ void __launch_bounds__(1024)
gv_order_kernel(GvNodes g, const GvLam* __restrict__ lamc, const int64_t* __restrict__ dK, int64_t slice0, int S,
                int TA, int32_t* __restrict__ rt_order)
{
    __shared__ float est[GV_ORDER_MAX];
    __shared__ long long s_mmin[16], s_mmax[16];
    __shared__ float s_thr[16];
    const int n_rt = g.na / TA;
    const int n = slice_count(dK, slice0, S);
    if (n_rt > GV_ORDER_MAX || n == 0) {
        for (int r = threadIdx.x; r < n_rt; r += blockDim.x) rt_order[r] = r;
        return;
    }
    const int ns = n < 16 ? n : 16;
    if (threadIdx.x < ns) {
        const GvLam& c = lamc[(int)((int64_t)threadIdx.x * n / ns)];
        s_mmin[threadIdx.x] = c.live ? c.mmin_bits : LLONG_MAX;
        s_mmax[threadIdx.x] = c.mmax_bits;
        s_thr[threadIdx.x] = c.mmin_f;
    }
    __syncthreads();
    // Thread (rt, s): over every 4th row of row tile rt, the q nodes at or above
    // mmin/m1 for sampled column s, from the q range (an estimate that assumes
    // evenly spread q nodes); then a sum over the 16 columns of a half warp.
    const float q0 = g.qf[0], qspan = g.qf[g.nb - 1] - g.qf[0];
    for (int t0 = 0; t0 < n_rt * 16; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const int rt = t >> 4, sc = t & 15;
        float w = 0.0f;
        if (rt < n_rt && sc < ns) {
#pragma unroll 4
            for (int i = 0; i < TA; i += 4) {
                const int a = rt * TA + i;
                const long long mb = __double_as_longlong(__ldg(g.m1 + a));
                if (!(mb > s_mmin[sc] && mb <= s_mmax[sc])) continue;
                const float thr = __fdividef(s_thr[sc], __ldg(g.m1f + a));
                const float frac = qspan > 0.0f ? fminf(fmaxf((thr - q0) / qspan, 0.0f), 1.0f) : 0.0f;
                w += (1.0f - frac) * (float)g.nb;
            }
        }
        for (int o = 8; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (sc == 0 && rt < n_rt) est[rt] = w;
    }
    __syncthreads();
    for (int rt = threadIdx.x; rt < n_rt; rt += blockDim.x) {
        const float e = est[rt];
        int rank = 0;
        for (int u = 0; u < n_rt; ++u) rank += (est[u] > e) || (est[u] == e && u < rt);
        rt_order[rank] = rt;
    }
}

// ---------------------------------------------------------------- U_b per column
// U[lt][b][c] = wq_b q_b^beta for column r = lt * 64 + c (0 for padding
// columns, invalid Lambda and nodes past nb), FP64.
__global__ void gv_u_kernel(GvNodes g, const double* __restrict__ wq, const GvLam* __restrict__ lamc,
                            const int64_t* __restrict__ dK, int64_t slice0, int S, const double2* __restrict__ tab,
                            ExpConsts kc, double* __restrict__ U)
{
    const int n = slice_count(dK, slice0, S);
    const int64_t total = (int64_t)((n + GV_TL - 1) / GV_TL) * g.nbp * GV_TL;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % GV_TL);
        const int64_t rest = t / GV_TL;
        const int b = (int)(rest % g.nbp);
        const int lt = (int)(rest / g.nbp);
        const GvLam& L = lamc[lt * GV_TL + c];
        double u = 0.0;
        if (L.live && b < g.nb && g.q[b] > 0.0) u = wq[b] * exp_tab(L.beta * g.lnq[b], tab, kc);
        U[t] = u;
    }
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t gv_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void gv_bar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void gv_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk copy global -> shared that completes `bytes` of transaction on `bar`
// (both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void gv_bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

// Waits for the phase of the given parity; false after `limit` polls (GV_WAIT_LIMIT in the
// contraction).
__device__ __forceinline__ bool gv_wait(uint32_t bar, uint32_t parity, int limit = GV_WAIT_LIMIT)
{
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// N consecutive elements of a staged row as 16-byte vectors (N * sizeof(T) a multiple of 16).
template <class T, int N>
__device__ __forceinline__ void gv_load(const T* src, T (&v)[N])
{
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int h = 0; h < N / 2; ++h) {
            const double2 x = *reinterpret_cast<const double2*>(src + 2 * h);
            v[2 * h] = x.x;
            v[2 * h + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int h = 0; h < N / 4; ++h) {
            const float4 x = *reinterpret_cast<const float4*>(src + 4 * h);
            v[4 * h] = x.x;
            v[4 * h + 1] = x.y;
            v[4 * h + 2] = x.z;
            v[4 * h + 3] = x.w;
        }
    }
}

// ---------------------------------------------------------------- FP64 contraction
// Tile shapes.  2 m1 rows x 4 Lambda columns per thread; a warp is 8 x 4 threads
// (16 rows x 16 consecutive columns); a CTA is 2 x 4 warps (32 rows x 64 columns).
// The FP64 pipe (two lanes per SM and clock) binds, so small thread tiles cost nothing.
// A setup kernel computes W_a and b0 of every pair once; the contraction's items are a
// tile and one of 4 fixed parts of the q range (the top parts, the heaviest, first), which
// makes the last wave of CTAs short.
constexpr int G64_RA = 2, G64_TA = 16 * G64_RA, G64_STAGES = 2, G64_QP = 4;
constexpr int G64_PAIRS = G64_TA * GV_TL;  // pairs of a tile, 8 per thread
__host__ __device__ constexpr size_t g64_smem() { return (size_t)G64_STAGES * GV_BC * (G64_TA + GV_TL) * sizeof(double); }

// Thread t of an FP64 contraction CTA: rows 2 ty .. 2 ty + 1, columns 4 tx .. 4 tx + 3.
__host__ __device__ inline int g64_ty(int t) { return 8 * ((t >> 5) >> 2) + ((t & 31) >> 2); }
__host__ __device__ inline int g64_tx(int t) { return 4 * ((t >> 5) & 3) + (t & 3); }

// W (w64) and b0 (b0g) of pair k = 4 i + j of thread t of tile (rt, lt) at
// ((rt * n_lt + lt) * 8 + k) * 256 + t: row 2 ty(t) + i, column 4 tx(t) + j; W = 0 for a pair
// without support.  The exponential table is staged in shared memory once per block.
__global__ void __launch_bounds__(GV_THREADS)
gv_setup64_kernel(GvNodes g, const GvLam* __restrict__ lamc, const int64_t* __restrict__ dK, int64_t slice0, int S,
                  const double2* __restrict__ tab_g, ExpConsts kc, double* __restrict__ w64, int* __restrict__ b0g)
{
    __shared__ double2 tab[EXP_TABLE_SIZE];
    for (int i = threadIdx.x; i < EXP_TABLE_SIZE; i += GV_THREADS) tab[i] = tab_g[i];
    __syncthreads();
    const int n = slice_count(dK, slice0, S);
    const int n_lt = (n + GV_TL - 1) / GV_TL;
    const int total = (g.na / G64_TA) * n_lt * G64_PAIRS;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int t = e & (GV_THREADS - 1), k = (e >> 8) & 7, item = e >> 11;
        const int rt = item / n_lt, lt = item - rt * n_lt;
        double W;
        int b0;
        gv_pair64(g, lamc[lt * GV_TL + g64_tx(t) * 4 + (k & 3)], rt * G64_TA + g64_ty(t) * G64_RA + (k >> 2), tab, kc,
                  W, b0);
        w64[e] = b0 < g.nb ? W : 0.0;
        b0g[e] = b0;
    }
}
static_assert(G64_PAIRS == 8 * GV_THREADS, "setup index layout");

// part[rt * 4 + qp][r] = sum over the 32 rows of row tile rt of W_a sum_{b >= b0} pdet[a, b] U_b
// over the nodes b of q part qp, for every column r of the CTA's Lambda tile, FP64 throughout.
__global__ void __launch_bounds__(GV_THREADS, 3)
gv_main_kernel(GvNodes g, const double* __restrict__ pd, const double* __restrict__ U, const double* __restrict__ w64,
               const int* __restrict__ b0g, const int32_t* __restrict__ rt_order, const int64_t* __restrict__ dK,
               int64_t slice0, int S, double* __restrict__ part, int* __restrict__ err)
{
    using T = double;
    constexpr int RA = G64_RA, STAGES = G64_STAGES, TA = G64_TA;
    constexpr int PD_ELEMS = GV_BC * TA, U_ELEMS = GV_BC * GV_TL;  // one chunk of each operand
    constexpr uint32_t PD_BYTES = PD_ELEMS * sizeof(T), U_BYTES = U_ELEMS * sizeof(T);
    extern __shared__ __align__(128) unsigned char gv_dyn[];
    T* sp = reinterpret_cast<T*>(gv_dyn);  // [STAGES][BC][TA] pdet
    T* su = sp + STAGES * PD_ELEMS;        // [STAGES][BC][64] U
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ int s_tmin;
    __shared__ double red[16][GV_TL];

    const int n = slice_count(dK, slice0, S);
    const int n_lt = (n + GV_TL - 1) / GV_TL;
    const unsigned per_part = (unsigned)(g.na / TA) * (unsigned)n_lt;
    // Linear block index -> (q part, heaviest parts first; row tile in launch order; Lambda tile).
    if (blockIdx.x >= per_part * G64_QP) return;
    const int qp = G64_QP - 1 - (int)(blockIdx.x / per_part);
    const unsigned rem = blockIdx.x % per_part;
    const int rt = rt_order[rem / n_lt], lt = (int)(rem % n_lt);
    const int tid = threadIdx.x, ty = g64_ty(tid), tx = g64_tx(tid);
    if (tid == 0) {
        s_tmin = INT_MAX;
        for (int st = 0; st < STAGES; ++st) gv_bar_init(gv_saddr(&bar[st]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int64_t pbase = (int64_t)(rt * n_lt + lt) * G64_PAIRS + tid;
    T W[RA][4];
    int b0[RA][4];
    int tmin = INT_MAX, tmax = -1;
#pragma unroll
    for (int i = 0; i < RA; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            W[i][j] = w64[pbase + (4 * i + j) * GV_THREADS];
            b0[i][j] = b0g[pbase + (4 * i + j) * GV_THREADS];
            if (b0[i][j] < g.nb) {
                tmin = min(tmin, b0[i][j]);
                tmax = max(tmax, b0[i][j]);
            }
        }
    if (tmin != INT_MAX) atomicMin(&s_tmin, tmin);
    __syncthreads();
    double* out = part + ((int64_t)rt * G64_QP + qp) * S + lt * GV_TL;
    const int nch = g.nbp / GV_BC;
    const int cq0 = qp * nch / G64_QP, cq1 = (qp + 1) * nch / G64_QP;
    const int c0 = max(cq0, s_tmin / GV_BC);  // s_tmin = INT_MAX: no pair of the tile has support
    if (c0 >= cq1) {
        if (tid < GV_TL) out[tid] = 0.0;
        return;
    }
    const T* pd_tile = pd + (int64_t)rt * g.nbp * TA;
    const T* u_tile = U + (int64_t)lt * g.nbp * GV_TL;
    auto issue = [&](int c) {
        const int st = (c - c0) % STAGES;
        const uint32_t b = gv_saddr(&bar[st]);
        gv_expect_tx(b, PD_BYTES + U_BYTES);
        gv_bulk_load(gv_saddr(sp + st * PD_ELEMS), pd_tile + (int64_t)c * PD_ELEMS, PD_BYTES, b);
        gv_bulk_load(gv_saddr(su + st * U_ELEMS), u_tile + (int64_t)c * U_ELEMS, U_BYTES, b);
    };
    if (tid == 0)
        for (int c = c0; c < cq1 && c < c0 + STAGES; ++c) issue(c);

    T acc[RA][4];
#pragma unroll
    for (int i = 0; i < RA; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int s = c0; s < cq1; ++s) {
        const bool ok = gv_wait(gv_saddr(&bar[(s - c0) % STAGES]), (uint32_t)(((s - c0) / STAGES) & 1));
        if (__syncthreads_or(!ok)) {
            // Give up: flag it, let the copies already issued land (bounded), leave NaN.
            if (tid == 0) {
                atomicExch(err, 1);
                for (int d = s; d < cq1 && d < s + STAGES; ++d)
                    gv_wait(gv_saddr(&bar[(d - c0) % STAGES]), (uint32_t)(((d - c0) / STAGES) & 1));
            }
            __syncthreads();
            if (tid < GV_TL) out[tid] = NAN;
            return;
        }
        const int cb = s * GV_BC;
        if (cb + GV_BC > tmin) {  // else below every support edge of this thread
            const int st = (s - c0) % STAGES;
            const T* ps = sp + st * PD_ELEMS + ty * RA;
            const T* us = su + st * U_ELEMS + tx * 4;
            const int bend = min(GV_BC, g.nb - cb);  // the last chunk stops at the last q node
            if (cb >= tmax) {  // every pair of the thread has support on the whole chunk
#pragma unroll 4
                for (int bb = 0; bb < bend; ++bb) {
                    T p[RA], u[4];
                    gv_load(ps + bb * TA, p);
                    gv_load(us + bb * GV_TL, u);
#pragma unroll
                    for (int i = 0; i < RA; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(p[i], u[j], acc[i][j]);
                }
            } else {  // a support edge inside the chunk: per-pair mask
#pragma unroll 2
                for (int bb = 0; bb < bend; ++bb) {
                    const int b = cb + bb;
                    T p[RA], u[4];
                    gv_load(ps + bb * TA, p);
                    gv_load(us + bb * GV_TL, u);
#pragma unroll
                    for (int i = 0; i < RA; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(p[i], b >= b0[i][j] ? u[j] : T(0), acc[i][j]);
                }
            }
        }
        __syncthreads();  // the stage is free again
        if (tid == 0 && s + STAGES < cq1) issue(s + STAGES);
    }

    // Fixed-order combine (W = 0 without support): rows of the thread, then the 16 row groups.
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < RA; ++i) t += W[i][j] * acc[i][j];
        red[ty][tx * 4 + j] = t;
    }
    __syncthreads();
    if (tid < GV_TL) {
        double sum = 0.0;
        for (int y = 0; y < 16; ++y) sum += red[y][tid];
        out[tid] = sum;
    }
}

// ---------------------------------------------------------------- FP32 contraction
// A setup kernel computes W_a and b0 of every (row, column) pair at full occupancy (FP32 W
// as gv_pair32 defines it), in the order the contraction reads them.  The contraction's
// persistent CTAs (one per SM) take items from a queue: a tile of 128 m1 rows x 128 Lambda
// columns and one of 4 fixed parts of the q range, the top parts (the heaviest) first.
// A thread holds 8 rows x 8 columns as 32 packed (row, row + 1) accumulator pairs: per q
// node, two 16-byte shared loads of its 8 pdet values, two of its 8 U values and 32
// f32x2 FMAs, so that the SM's one shared-memory path (a warp's 16-byte load takes 2.5 to
// 4 SM cycles) stays below the FMA pipe's rate (4 x 4 tiles would cap the FMA pipe at
// two thirds of it).  The rows and columns of a staged chunk are stored
// in the order the threads read them (g32_perm).  A warp covers 32 rows x 64 columns and
// decides per 8-node sub-block, from the lowest and highest support edge of its pairs,
// whether the sub-block is below every edge (skipped), past every edge (no mask) or in
// between (per-pair masks built from the edges kept in shared memory).  Every pair's sum
// still runs over its own in-support nodes in node order, 32-node chunk sums added into a
// running sum per q part, so the result does not depend on the tiling.
constexpr int G32_T = 128;      // m1 rows and Lambda columns of a tile
constexpr int G32_STAGES = 4;   // staged chunks in flight
constexpr int G32_CPB = 2;      // chunks per barrier step
constexpr int G32_SUB = 8;      // q nodes per masking decision
constexpr int G32_QP = 4;       // parts of the q range (items per tile)
constexpr int G32_CHUNK = GV_BC * G32_T;  // floats of one pdet or U chunk
constexpr int G32_PAIRS = G32_T * G32_T;  // pairs of a tile, 64 per thread
__host__ __device__ constexpr size_t g32_stage_bytes() { return (size_t)G32_STAGES * 2 * G32_CHUNK * sizeof(float); }
__host__ __device__ constexpr size_t g32_smem() { return g32_stage_bytes() + (size_t)G32_PAIRS * sizeof(int); }
static_assert(g32_stage_bytes() >= 16 * G32_T * sizeof(double), "the row combine fits the stages");

// Thread t of a contraction CTA: rows 8 ty .. 8 ty + 7, columns 8 tx .. 8 tx + 7 of its tile.
__host__ __device__ inline int g32_ty(int t) { return 4 * ((t >> 5) >> 1) + ((t & 31) >> 3); }
__host__ __device__ inline int g32_tx(int t) { return 8 * ((t >> 5) & 1) + (t & 7); }
// Row (or column) of a tile stored at position pos of a staged node: pos = 64 h + 4 t + e holds
// row 8 t + 4 h + e, so thread t's 8 rows are two 16-byte words and a warp's words are contiguous.
__host__ __device__ inline int g32_perm(int pos) { return ((pos >> 2) & 15) * 8 + (pos >> 6) * 4 + (pos & 3); }

// One 8-node sub-block.  ps / us: this thread's words in the stage's pdet / U chunk at the
// sub-block's first node; mk (MASK): bit n of byte k is set when node n is in the support of
// pair k = 8 i + j (row i, column j of the thread).
template <bool MASK>
__device__ __forceinline__ void g32_block(const float* ps, const float* us, const uint32_t (&mk)[16], f2 (&acc)[4][8])
{
#pragma unroll
    for (int bb = 0; bb < G32_SUB; ++bb) {
        const ulonglong2 pa = *reinterpret_cast<const ulonglong2*>(ps + bb * G32_T);
        const ulonglong2 pb = *reinterpret_cast<const ulonglong2*>(ps + bb * G32_T + 64);
        const float4 ua = *reinterpret_cast<const float4*>(us + bb * G32_T);
        const float4 ub = *reinterpret_cast<const float4*>(us + bb * G32_T + 64);
        const f2 p[4] = {pa.x, pa.y, pb.x, pb.y};
        const float u[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if constexpr (!MASK) {
                const f2 uj = bc(u[j]);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][j] = fma2(p[i], uj, acc[i][j]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k0 = 16 * i + j, k1 = k0 + 8;
                    const bool in0 = (mk[k0 >> 2] >> (8 * (k0 & 3) + bb)) & 1u;
                    const bool in1 = (mk[k1 >> 2] >> (8 * (k1 & 3) + bb)) & 1u;
                    acc[i][j] = fma2(p[i], pk(in0 ? u[j] : 0.0f, in1 ? u[j] : 0.0f), acc[i][j]);
                }
            }
        }
    }
}

// W (wg) and b0 (b0g) of pair k = 8 i + j of thread t of tile (rt, lt) at
// ((rt * n_lt + lt) * 64 + k) * 256 + t: row 8 ty(t) + i, column 8 tx(t) + j; W = 0 for a pair
// without support (b0 = nb).  wmm[(rt * n_lt + lt) * 8 + w] = (lowest, highest) support edge
// over the pairs of warp w of the contraction (unsigned 0xffffffff and -1 when it has none; the
// array is 0xff bytes at the launch).  A warp-wide read of the contraction is one contiguous line.
__global__ void gv_setup32_kernel(GvNodes g, const GvRow32* __restrict__ rows, const GvCol32* __restrict__ cols,
                                  const int64_t* __restrict__ dK, int64_t slice0, int S, float* __restrict__ wg,
                                  int* __restrict__ b0g, int2* __restrict__ wmm)
{
    const int n = slice_count(dK, slice0, S);
    const int n_lt = (n + G32_T - 1) / G32_T;
    const int total = (g.na / G32_T) * n_lt * G32_PAIRS;  // a multiple of 32: warps stay whole
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int t = e & (GV_THREADS - 1), k = (e >> 8) & 63, item = e >> 14;
        const int rt = item / n_lt, lt = item - rt * n_lt;
        float W;
        int b0;
        const int a = rt * G32_T + g32_ty(t) * 8 + (k >> 3);
        gv_pair32(g, gv_ld16(cols + lt * G32_T + g32_tx(t) * 8 + (k & 7)), gv_ld16(rows + a), a, W, b0);
        const bool in = b0 < g.nb;
        wg[e] = in ? W : 0.0f;
        b0g[e] = b0;
        const unsigned lo = __reduce_min_sync(0xffffffffu, in ? (unsigned)b0 : 0xffffffffu);
        const int hi = __reduce_max_sync(0xffffffffu, in ? b0 : -1);
        if ((t & 31) == 0 && lo != 0xffffffffu) {
            int2* m = wmm + item * 8 + (t >> 5);
            atomicMin(reinterpret_cast<unsigned*>(&m->x), lo);
            atomicMax(&m->y, hi);
        }
    }
}
static_assert(GV_THREADS == 256 && G32_PAIRS == 64 * GV_THREADS, "setup index layout");

// Exact product and float-float accumulation (Knuth's TwoSum, an FMA for the product's error).
__device__ __forceinline__ void g32_ff_add(float& sh, float& sl, float w, float r)
{
    const float p = w * r;
    const float pe = fmaf(w, r, -p);
    const float s = sh + p;
    const float bp = s - sh;
    sl += ((sh - (s - bp)) + (p - bp)) + pe;
    sh = s;
}

// part[rt * 4 + qp][r] = sum over the 128 rows of row tile rt of W_a times the FP32 sum of
// pdet[a, b] U_b over the nodes b >= b0 of q part qp (32-node chunk sums added into an FP32
// running sum), FP32 row factor, the products and their sum over rows in float-float (exact
// products, FP32 pairs carrying the rounding errors), rounded to FP64.  *queue is zero at the
// launch.
__global__ void __launch_bounds__(GV_THREADS, 1)
gv_main32_kernel(GvNodes g, const float* __restrict__ pd, const float* __restrict__ U, const float* __restrict__ wg,
                 const int* __restrict__ b0g, const int2* __restrict__ wmm, const int32_t* __restrict__ rt_order,
                 const int64_t* __restrict__ dK, int64_t slice0, int S, unsigned* __restrict__ queue,
                 double* __restrict__ part, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char gv_dyn[];
    float* sp = reinterpret_cast<float*>(gv_dyn);   // [STAGES][pdet chunk, U chunk]
    int* b0s = reinterpret_cast<int*>(gv_dyn + g32_stage_bytes());  // [64][256] support edges of the item
    float2* red = reinterpret_cast<float2*>(gv_dyn);  // [16][128], over the stages once an item's chunks are done
    __shared__ __align__(8) uint64_t bar[G32_STAGES];
    __shared__ __align__(8) uint64_t ebar;  // the item's support edges
    __shared__ int s_tmin;
    __shared__ unsigned s_item;

    const int n = slice_count(dK, slice0, S);
    const int n_lt = (n + G32_T - 1) / G32_T;
    const unsigned per_part = (unsigned)(g.na / G32_T) * (unsigned)n_lt;
    const unsigned n_items = per_part * G32_QP;
    const int nch = g.nbp / GV_BC;
    const int tid = threadIdx.x, ty = g32_ty(tid), tx = g32_tx(tid);
    if (tid == 0) {
        for (int st = 0; st < G32_STAGES; ++st) gv_bar_init(gv_saddr(&bar[st]));
        gv_bar_init(gv_saddr(&ebar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    unsigned seq = 0;    // chunks this CTA has staged so far: chunk number seq goes to stage seq % STAGES
    unsigned n_ecp = 0;  // support-edge copies this CTA has issued
    bool dead = false;   // a wait gave up: the CTA only marks its remaining items
    for (;;) {
        // This thread's reads of the stages, the edges and the row combine (generic proxy) are
        // ordered before the next bulk copies (async proxy) into the same bytes.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();  // the previous item is done with the stages, b0s, red and s_item
        if (tid == 0) {
            s_item = atomicAdd(queue, 1u);
            s_tmin = INT_MAX;
        }
        __syncthreads();
        const unsigned item = s_item;
        if (item >= n_items) break;
        const int qp = G32_QP - 1 - (int)(item / per_part);
        const unsigned rem = item % per_part;
        const int rt = rt_order[rem / n_lt], lt = (int)(rem % n_lt);
        double* out = part + ((int64_t)rt * G32_QP + qp) * S + lt * G32_T;
        if (dead) {
            if (tid < G32_T) out[tid] = NAN;
            continue;
        }
        const int tile = rt * n_lt + lt;
        const int2 mm = wmm[tile * 8 + (tid >> 5)];
        const int wmin = mm.x < 0 ? INT_MAX : mm.x, wmax = mm.y;  // 0xffffffff: no support in the warp
        if ((tid & 31) == 0) atomicMin(&s_tmin, wmin);
        __syncthreads();
        const int cq0 = qp * nch / G32_QP, cq1 = (qp + 1) * nch / G32_QP;
        const int c_lo = max(cq0, s_tmin / GV_BC);  // s_tmin = INT_MAX: no pair of the tile has support
        if (c_lo >= cq1) {
            if (tid < G32_T) out[tid] = 0.0;
            continue;
        }
        const float* pd_tile = pd + (int64_t)rt * g.nbp * G32_T;
        const float* u_tile = U + (int64_t)lt * g.nbp * G32_T;
        auto issue = [&](int c) {
            const int st = (int)((seq + (unsigned)(c - c_lo)) % G32_STAGES);
            const uint32_t b = gv_saddr(&bar[st]);
            gv_expect_tx(b, 2 * G32_CHUNK * sizeof(float));
            gv_bulk_load(gv_saddr(sp + st * 2 * G32_CHUNK), pd_tile + (int64_t)c * G32_CHUNK, G32_CHUNK * sizeof(float), b);
            gv_bulk_load(gv_saddr(sp + st * 2 * G32_CHUNK + G32_CHUNK), u_tile + (int64_t)c * G32_CHUNK,
                         G32_CHUNK * sizeof(float), b);
        };
        auto wait = [&](int c) {
            const unsigned q = seq + (unsigned)(c - c_lo);
            return gv_wait(gv_saddr(&bar[q % G32_STAGES]), (q / G32_STAGES) & 1u);
        };
        if (tid == 0) {
            gv_expect_tx(gv_saddr(&ebar), G32_PAIRS * sizeof(int));
            gv_bulk_load(gv_saddr(b0s), b0g + (int64_t)tile * G32_PAIRS, G32_PAIRS * sizeof(int), gv_saddr(&ebar));
            for (int c = c_lo; c < cq1 && c < c_lo + G32_STAGES; ++c) issue(c);
        }
        const uint32_t eparity = n_ecp & 1u;
        ++n_ecp;

        f2 acc[4][8], run[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = run[i][j] = 0ull;
        bool ok = gv_wait(gv_saddr(&ebar), eparity);
        for (int s = c_lo; s < cq1; s += G32_CPB) {
            const int e = min(s + G32_CPB, cq1);
            for (int c = s; c < e; ++c) ok &= wait(c);
            if (__syncthreads_or(!ok)) {
                // Give up: flag it and let the copies already issued land (bounded).
                if (tid == 0) {
                    atomicExch(err, 1);
                    gv_wait(gv_saddr(&ebar), eparity);
                    for (int d = s; d < cq1 && d < s + G32_STAGES; ++d) wait(d);
                }
                ok = false;
                break;
            }
            for (int c = s; c < e; ++c) {
                const int cb = c * GV_BC;
                if (cb + GV_BC <= wmin) continue;  // below every support edge of the warp
                const int st = (int)((seq + (unsigned)(c - c_lo)) % G32_STAGES);
                const float* ps = sp + st * 2 * G32_CHUNK + ty * 4;
                const float* us = sp + st * 2 * G32_CHUNK + G32_CHUNK + tx * 4;
#pragma unroll 1
                for (int sb = 0; sb < GV_BC; sb += G32_SUB) {
                    const int b = cb + sb;
                    if (b + G32_SUB <= wmin || b >= g.nb) continue;
                    uint32_t mk[16];
                    if (b >= wmax) {
                        g32_block<false>(ps + sb * G32_T, us + sb * G32_T, mk, acc);
                    } else {
#pragma unroll
                        for (int r = 0; r < 16; ++r) {
                            uint32_t m = 0;
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const int d = b0s[(4 * r + h) * GV_THREADS + tid] - b;  // first in-support node
                                const uint32_t byte = d <= 0 ? 0xffu : (d >= G32_SUB ? 0u : (0xffu << d) & 0xffu);
                                m |= byte << (8 * h);
                            }
                            mk[r] = m;
                        }
                        g32_block<true>(ps + sb * G32_T, us + sb * G32_T, mk, acc);
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        run[i][j] = add2(run[i][j], acc[i][j]);
                        acc[i][j] = 0ull;
                    }
            }
            __syncthreads();  // the step's stages are free again
            if (tid == 0)
                for (int c = s + G32_STAGES; c < cq1 && c < s + G32_STAGES + G32_CPB; ++c) issue(c);
        }
        seq += (unsigned)(cq1 - c_lo);
        if (!ok) {
            dead = true;
            if (tid < G32_T) out[tid] = NAN;
            continue;
        }
        // Fixed-order combine (W = 0 without support): rows of the thread (i = 0..7), then the
        // 16 row groups, in float-float.
        const float* wt = wg + (int64_t)tile * G32_PAIRS + tid;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float sh = 0.0f, sl = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float r0, r1;
                upk(run[i][j], r0, r1);
                g32_ff_add(sh, sl, wt[(16 * i + j) * GV_THREADS], r0);
                g32_ff_add(sh, sl, wt[(16 * i + 8 + j) * GV_THREADS], r1);
            }
            red[ty * G32_T + tx * 8 + j] = make_float2(sh, sl);
        }
        __syncthreads();
        if (tid < G32_T) {
            float sh = 0.0f, sl = 0.0f;
            for (int y = 0; y < 16; ++y) {
                const float2 v = red[y * G32_T + tid];
                const float s = sh + v.x;
                const float bp = s - sh;
                sl += ((sh - (s - bp)) + (v.x - bp)) + v.y;
                sh = s;
            }
            out[tid] = (double)sh + (double)sl;
        }
    }
}

// U of the FP32 contraction: U[lt][b][pos] = wq_b q_b^beta for column lt * 128 + g32_perm(pos)
// (0 for padding columns, invalid Lambda and nodes past nb).
__global__ void gv_u32_kernel(GvNodes g, const GvLam* __restrict__ lamc, const int64_t* __restrict__ dK,
                              int64_t slice0, int S, float* __restrict__ U)
{
    const int n = slice_count(dK, slice0, S);
    const int64_t total = (int64_t)((n + G32_T - 1) / G32_T) * g.nbp * G32_T;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int pos = (int)(t % G32_T);
        const int64_t rest = t / G32_T;
        const int b = (int)(rest % g.nbp);
        const int lt = (int)(rest / g.nbp);
        const GvLam& L = lamc[lt * G32_T + g32_perm(pos)];
        float u = 0.0f;
        if (L.live && b < g.nb && g.q[b] > 0.0)
            u = g.wqf[b] * exp2f(fmaf(L.beta_h, g.l2q_h[b], fmaf(L.beta_h, g.l2q_l[b], L.beta_l * g.l2q_h[b])));
        U[t] = u;
    }
}

// xi[k] = sum over the row tiles of part[rt][r], k = perm[r]: one warp per column,
// lane l sums row tiles l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void gv_reduce_kernel(const double* __restrict__ part, int n_rt, const int32_t* __restrict__ perm,
                                 const int64_t* __restrict__ dK, int64_t slice0, int S, double* __restrict__ xi)
{
    const int n = slice_count(dK, slice0, S);
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;  // whole warps leave together
    double sum = 0.0;
    for (int rt = lane; rt < n_rt; rt += 32) sum += part[(int64_t)rt * S + r];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) xi[perm[r]] = sum;
}

__global__ void gv_out_kernel(const double* __restrict__ xi, const double* __restrict__ lambda, int P,
                              const int64_t* __restrict__ dK, double* __restrict__ lnxi, uint32_t* __restrict__ flags)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= *dK) return;
    if (!gv_valid(lambda + k * P, P)) {
        lnxi[k] = 0.0;
        flags[k] = POP_FLAG_INVALID_LAMBDA;
        return;
    }
    const double x = xi[k];
    lnxi[k] = x > 0.0 ? log(x) : -INFINITY;
    flags[k] = x > 0.0 ? 0u : (uint32_t)POP_FLAG_ZERO_XI;
}

// pdet [n_m1][n_q] -> [na / TA][nbp][TA] in T (zeros in the padding), position c of a node
// holding row c (FP64 tiles of 32) or row g32_perm(c) (FP32 tiles of 128); *bad = 1 when a
// used entry is not finite or negative.
template <class T>
__global__ void gv_pack_kernel(const double* __restrict__ pdet, int n_m1, int n_q, int na, int nb, int nbp, int TA,
                               T* __restrict__ out, int* __restrict__ bad)
{
    const int64_t total = (int64_t)na * nbp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % TA);
        const int64_t rest = t / TA;
        const int b = (int)(rest % nbp);
        const int a = (int)(rest / nbp) * TA + (sizeof(T) == 4 ? g32_perm(c) : c);
        double v = 0.0;
        if (a < n_m1 && b < nb) {
            v = pdet[(int64_t)a * n_q + b];
            if (!(isfinite(v) && v >= 0.0)) {
                atomicExch(bad, 1);
                v = 0.0;
            }
        }
        out[t] = (T)v;
    }
}

int blocks_for(int64_t n, int threads, int cap)
{
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}


size_t sort_smem(int S) { return sizeof(int) * (GV_BUCKETS + 4) + (sizeof(int32_t) + sizeof(float)) * (size_t)S; }

}  // namespace

GridVT::~GridVT()
{
    for (cudaEvent_t e : {ev0, ev1, ev2, ev3})
        if (e) cudaEventDestroy(e);
}

int GridVT::load(int n1, const double* m1_nodes, int nq, const double* q_nodes, const double* pdet, bool on_device,
                 cudaStream_t s)
{
    auto bad = [&](int st, const char* m) {
        err_msg = m;
        return st;
    };
    if (n1 < 2 || nq < 2) return bad(POP_EINVAL, "pop_load_vt_grid: need at least 2 nodes on each axis");
    if ((int64_t)n1 * nq > (1LL << 28)) return bad(POP_EINVAL, "pop_load_vt_grid: more than 2^28 grid nodes");
    if (!m1_nodes || !q_nodes || !pdet) return bad(POP_EINVAL, "pop_load_vt_grid: NULL pointer");
    std::vector<double> hm(n1), hq(nq);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    if (cudaMemcpy(hm.data(), m1_nodes, sizeof(double) * n1, kind) != cudaSuccess ||
        cudaMemcpy(hq.data(), q_nodes, sizeof(double) * nq, kind) != cudaSuccess)
        return bad(POP_ECUDA, "pop_load_vt_grid: copying the nodes failed");
    for (int a = 0; a < n1; ++a)
        if (!std::isfinite(hm[a]) || (a > 0 && !(hm[a] > hm[a - 1])))
            return bad(POP_EINVAL, "pop_load_vt_grid: m1 nodes must be finite and strictly increasing");
    for (int b = 0; b < nq; ++b)
        if (!std::isfinite(hq[b]) || (b > 0 && !(hq[b] > hq[b - 1])))
            return bad(POP_EINVAL, "pop_load_vt_grid: q nodes must be finite and strictly increasing");
    int nb_ = 0;
    while (nb_ < nq && hq[nb_] <= 1.0) ++nb_;
    if (nb_ == 0) return bad(POP_EINVAL, "pop_load_vt_grid: no q node <= 1");
    const int na_ = (n1 + GV_ROW_PAD - 1) / GV_ROW_PAD * GV_ROW_PAD;
    const int nbp_ = (nb_ + GV_BC - 1) / GV_BC * GV_BC;
    // Trapezoid weights over all nodes (a node's weight is half the span to its neighbours),
    // and the per-node logs and reciprocals of the setup.  Padding rows keep m1 = 0 (no support).
    std::vector<double> wm(na_, 0.0), lm(na_, 0.0), im(na_, 0.0), m(na_, 0.0);
    std::vector<float> mf(na_, 0.0f), mlf(na_, 0.0f), imf(na_, 0.0f), l2mf(na_, 0.0f), wmf(na_, 0.0f);
    std::vector<double> wqv(nbp_, 0.0), qv(nbp_, 0.0), lqv(nbp_, 0.0);
    std::vector<float> qfv(nbp_, 0.0f), l2qhv(nbp_, 0.0f), l2qlv(nbp_, 0.0f), wqfv(nbp_, 0.0f);
    for (int a = 0; a < n1; ++a) {
        const double hi = a + 1 < n1 ? hm[a + 1] : hm[a], lo = a > 0 ? hm[a - 1] : hm[a];
        wm[a] = 0.5 * (hi - lo);
        m[a] = hm[a];
        lm[a] = hm[a] > 0.0 ? std::log(hm[a]) : 0.0;
        im[a] = hm[a] > 0.0 ? 1.0 / hm[a] : 0.0;
        mf[a] = (float)hm[a];
        mlf[a] = (float)(hm[a] - (double)mf[a]);
        imf[a] = (float)im[a];
        l2mf[a] = hm[a] > 0.0 ? (float)std::log2(hm[a]) : 0.0f;
        wmf[a] = (float)wm[a];
    }
    for (int b = 0; b < nb_; ++b) {
        const double hi = b + 1 < nq ? hq[b + 1] : hq[b], lo = b > 0 ? hq[b - 1] : hq[b];
        wqv[b] = 0.5 * (hi - lo);
        qv[b] = hq[b];
        lqv[b] = hq[b] > 0.0 ? std::log(hq[b]) : 0.0;
        qfv[b] = (float)hq[b];
        const double l2 = hq[b] > 0.0 ? std::log2(hq[b]) : 0.0;
        l2qhv[b] = (float)l2;
        l2qlv[b] = (float)(l2 - (double)l2qhv[b]);
        wqfv[b] = (float)wqv[b];
    }
    std::vector<GvRow32> r32(na_);
    for (int a = 0; a < na_; ++a) r32[a] = GvRow32{m[a], mf[a], mlf[a], l2mf[a], imf[a], wmf[a], 0.0f};
    // Bins of the support-edge search: up to 1024 of equal width over the FP32 nodes.
    int nqb_ = 1;
    float qb0_ = qfv[0], qbinv_ = 0.0f;
    if (nb_ >= 2 && qfv[nb_ - 1] > qfv[0]) {
        nqb_ = std::min(1024, nb_);
        qbinv_ = (float)(nqb_ / ((double)qfv[nb_ - 1] - (double)qfv[0]));
    }
    std::vector<int> qbkv(nqb_ + 1, nb_);
    for (int k = 0, j = 0; k < nqb_; ++k) {
        const double edge = (double)qfv[0] + (double)k / (double)qbinv_;
        while (j < nb_ && (double)qfv[j] < edge) ++j;
        qbkv[k] = k == 0 ? 0 : j;
    }
    DevBuf dm, dlm, dim, dwa, dmf, dmlf, dimf, dl2m, dwaf, dq, dlq, dwq, dqf, dl2qh, dl2ql, dwqf, dqbk, dr32, p64, p32,
        tmp, dbad;
    auto ck = [&](cudaError_t e) { return e == cudaSuccess; };
    const size_t packed = (size_t)na_ * nbp_;
    const size_t d_na = sizeof(double) * na_, f_na = sizeof(float) * na_;
    const size_t d_nb = sizeof(double) * nbp_, f_nb = sizeof(float) * nbp_;
    if (!ck(dm.alloc(d_na)) || !ck(dlm.alloc(d_na)) || !ck(dim.alloc(d_na)) || !ck(dwa.alloc(d_na)) ||
        !ck(dmf.alloc(f_na)) || !ck(dmlf.alloc(f_na)) || !ck(dimf.alloc(f_na)) || !ck(dl2m.alloc(f_na)) || !ck(dwaf.alloc(f_na)) || !ck(dq.alloc(d_nb)) ||
        !ck(dlq.alloc(d_nb)) || !ck(dwq.alloc(d_nb)) || !ck(dqf.alloc(f_nb)) || !ck(dl2qh.alloc(f_nb)) ||
        !ck(dl2ql.alloc(f_nb)) || !ck(dwqf.alloc(f_nb)) || !ck(dqbk.alloc(sizeof(int) * (nqb_ + 1))) ||
        !ck(dr32.alloc(sizeof(GvRow32) * na_)) ||
        !ck(p64.alloc(sizeof(double) * packed)) || !ck(p32.alloc(sizeof(float) * packed)) ||
        !ck(dbad.alloc(sizeof(int))))
        return bad(POP_ENOMEM, "pop_load_vt_grid: device allocation failed");
    if (!tab.p) {
        std::vector<double2> ht(EXP_TABLE_SIZE);
        build_exp_table(ht.data(), &kc);
        if (!ck(tab.alloc(sizeof(double2) * EXP_TABLE_SIZE)) ||
            !ck(cudaMemcpy(tab.p, ht.data(), sizeof(double2) * EXP_TABLE_SIZE, cudaMemcpyHostToDevice)))
            return bad(POP_ENOMEM, "pop_load_vt_grid: exponential table");
    }
    const double* src = pdet;
    if (!on_device) {
        if (!ck(tmp.alloc(sizeof(double) * (size_t)n1 * nq))) return bad(POP_ENOMEM, "pop_load_vt_grid: allocation");
        if (!ck(cudaMemcpyAsync(tmp.p, pdet, sizeof(double) * (size_t)n1 * nq, cudaMemcpyHostToDevice, s)))
            return bad(POP_ECUDA, "pop_load_vt_grid: copying pdet failed");
        src = tmp.as<double>();
    }
    auto up = [&](DevBuf& d, const void* h, size_t n) {
        return ck(cudaMemcpyAsync(d.p, h, n, cudaMemcpyHostToDevice, s));
    };
    bool okc = up(dm, m.data(), d_na) && up(dlm, lm.data(), d_na) && up(dim, im.data(), d_na) &&
               up(dwa, wm.data(), d_na) && up(dmf, mf.data(), f_na) &&
               up(dmlf, mlf.data(), f_na) && up(dimf, imf.data(), f_na) && up(dl2m, l2mf.data(), f_na) &&
               up(dwaf, wmf.data(), f_na) && up(dq, qv.data(), d_nb) && up(dlq, lqv.data(), d_nb) &&
               up(dwq, wqv.data(), d_nb) && up(dqf, qfv.data(), f_nb) && up(dl2qh, l2qhv.data(), f_nb) &&
               up(dl2ql, l2qlv.data(), f_nb) && up(dwqf, wqfv.data(), f_nb) &&
               up(dqbk, qbkv.data(), sizeof(int) * (nqb_ + 1)) && up(dr32, r32.data(), sizeof(GvRow32) * na_) &&
               ck(cudaMemsetAsync(dbad.p, 0, sizeof(int), s));
    if (!okc) return bad(POP_ECUDA, "pop_load_vt_grid: copying the nodes failed");
    const int pb = blocks_for((int64_t)packed, 256, 152 * 32);
    gv_pack_kernel<double><<<pb, 256, 0, s>>>(src, n1, nq, na_, nb_, nbp_, G64_TA, p64.as<double>(),
                                              dbad.as<int>());
    gv_pack_kernel<float><<<pb, 256, 0, s>>>(src, n1, nq, na_, nb_, nbp_, G32_T, p32.as<float>(),
                                             dbad.as<int>());
    if (!ck(cudaGetLastError())) return bad(POP_ECUDA, "pop_load_vt_grid: pack kernel launch failed");
    int hbad = 0;
    if (!ck(cudaMemcpyAsync(&hbad, dbad.p, sizeof(int), cudaMemcpyDeviceToHost, s)) || !ck(cudaStreamSynchronize(s)))
        return bad(POP_ECUDA, "pop_load_vt_grid: pack kernel failed");
    if (hbad) return bad(POP_EINVAL, "pop_load_vt_grid: pdet must be finite and >= 0 at every node with q <= 1");
    if (!ev0) {
        if (!ck(cudaEventCreate(&ev0)) || !ck(cudaEventCreate(&ev1)) || !ck(cudaEventCreate(&ev2)) ||
            !ck(cudaEventCreate(&ev3)))
            return bad(POP_ECUDA, "pop_load_vt_grid: cudaEventCreate failed");
    }
    if (!err.p) {
        if (!ck(err.alloc(sizeof(int))) || !ck(cudaMemsetAsync(err.p, 0, sizeof(int), s)) ||
            !ck(cudaStreamSynchronize(s)))
            return bad(POP_ENOMEM, "pop_load_vt_grid: allocation failed");
    }
    m1.swap(dm);
    lnm1.swap(dlm);
    invm1.swap(dim);
    wa.swap(dwa);
    m1f.swap(dmf);
    m1lf.swap(dmlf);
    invm1f.swap(dimf);
    l2m1f.swap(dl2m);
    waf.swap(dwaf);
    q.swap(dq);
    lnq.swap(dlq);
    wq.swap(dwq);
    qf.swap(dqf);
    l2qh.swap(dl2qh);
    l2ql.swap(dl2ql);
    wqf.swap(dwqf);
    qbk.swap(dqbk);
    rows32.swap(dr32);
    nqb = nqb_;
    qb0 = qb0_;
    qbinv = qbinv_;
    pd64.swap(p64);
    pd32.swap(p32);
    n_m1 = n1;
    n_q = nq;
    na = na_;
    nb = nb_;
    nbp = nbp_;
    k_cap = 0;  // the scratch depends on the grid shape
    slice = 0;
    return POP_OK;
}

cudaError_t GridVT::ensure(int64_t K)
{
    if (K <= k_cap && slice > 0) return cudaSuccess;
    const int64_t cap = std::max<int64_t>(std::max<int64_t>(K, k_cap), 64);
    // Columns per slice, a multiple of 128: up to GV_SLICE, fewer on tall grids (the pair buffers,
    // 12 na S bytes, up to 1.5 GiB).
    const int64_t s_mem = std::max<int64_t>(G32_T, ((int64_t)3 << 29) / (12 * (int64_t)na) / G32_T * G32_T);
    const int S = (int)std::min<int64_t>(std::min<int64_t>((cap + G32_T - 1) / G32_T * G32_T, GV_SLICE), s_mem);
    DevBuf p, u, pt, x, lcb, lcb32, od, qu, w, b, mm;
    cudaError_t e;
    const int n_sl = (int)((cap + S - 1) / S);
    if ((e = p.alloc(sizeof(int32_t) * S)) != cudaSuccess) return e;
    if ((e = od.alloc(sizeof(int32_t) * (size_t)(na / G64_TA))) != cudaSuccess) return e;
    if ((e = lcb.alloc(sizeof(GvLam) * S)) != cudaSuccess) return e;
    if ((e = lcb32.alloc(sizeof(GvCol32) * S)) != cudaSuccess) return e;
    if ((e = u.alloc(sizeof(double) * (size_t)S * nbp)) != cudaSuccess) return e;
    // Partial sums: na / 32 row tiles x 4 q parts in the FP64 form, na / 128 row tiles x 4 q parts
    // in the FP32 form.
    static_assert(G32_QP * G64_TA <= G32_T * G64_QP, "the FP32 partial sums fit the FP64 rows");
    if ((e = pt.alloc(sizeof(double) * (size_t)(na / G64_TA) * G64_QP * S)) != cudaSuccess) return e;
    if ((e = x.alloc(sizeof(double) * cap)) != cudaSuccess) return e;
    if ((e = qu.alloc(sizeof(unsigned) * n_sl)) != cudaSuccess) return e;
    // Row factors (FP64, or FP32 in the same bytes) and support edges of every pair of a slice.
    if ((e = w.alloc(sizeof(double) * (size_t)na * S)) != cudaSuccess) return e;
    if ((e = b.alloc(sizeof(int) * (size_t)na * S)) != cudaSuccess) return e;
    if ((e = mm.alloc(sizeof(int2) * 8 * (size_t)(na / G32_T) * (S / G32_T))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(gv_main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g64_smem())) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(gv_main32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g32_smem())) !=
        cudaSuccess)
        return e;
    int dev = 0, n_sm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gv_main32_kernel, GV_THREADS, g32_smem())) !=
            cudaSuccess)
        return e;
    g32_ctas = std::max(1, n_sm * per_sm);
    if ((e = cudaFuncSetAttribute(gv_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem(S))) !=
        cudaSuccess)
        return e;
    perm.swap(p);
    order.swap(od);
    queue.swap(qu);
    wg.swap(w);
    b0g.swap(b);
    wmm.swap(mm);
    lamc.swap(lcb);
    lamc32.swap(lcb32);
    U.swap(u);
    part.swap(pt);
    xi.swap(x);
    k_cap = cap;
    slice = S;
    return cudaSuccess;
}

cudaError_t GridVT::enqueue(int mode, const double* lambda, int n_params, const int64_t* dK, int64_t K_cap, bool timed,
                            unsigned rec, cudaStream_t s)
{
    if (K_cap <= 0) return cudaSuccess;
    if (K_cap > k_cap || slice <= 0) return cudaErrorInvalidValue;
    const GvNodes g{m1.as<double>(), lnm1.as<double>(), invm1.as<double>(), wa.as<double>(), m1f.as<float>(),
                    m1lf.as<float>(), invm1f.as<float>(), l2m1f.as<float>(), waf.as<float>(), q.as<double>(),
                    lnq.as<double>(), qf.as<float>(), l2qh.as<float>(), l2ql.as<float>(), wqf.as<float>(),
                    qbk.as<int>(), qb0, qbinv, nqb, na, nb, nbp};
    const double2* tb = tab.as<double2>();
    GvLam* lcp = lamc.as<GvLam>();
    const int n_sl = (int)((K_cap + slice - 1) / slice);
    cudaError_t e;
    if (timed && (e = cudaEventRecordWithFlags(ev0, s, rec)) != cudaSuccess) return e;
    if (mode != 0 && (e = cudaMemsetAsync(queue.p, 0, sizeof(unsigned) * n_sl, s)) != cudaSuccess) return e;
    for (int sl = 0; sl < n_sl; ++sl) {
        const int64_t s0 = (int64_t)sl * slice;
        gv_sort_kernel<<<1, 1024, sort_smem(slice), s>>>(lambda, n_params, dK, s0, slice, perm.as<int32_t>());
        gv_lamc_kernel<<<(slice + 31) / 32, 32, 0, s>>>(lambda, n_params, perm.as<int32_t>(), dK, s0, slice, lcp,
                                                        lamc32.as<GvCol32>());
        const int ub = blocks_for((int64_t)slice * nbp, 256, 152 * 16);
        if (mode == 0)
            gv_u_kernel<<<ub, 256, 0, s>>>(g, wq.as<double>(), lcp, dK, s0, slice, tb, kc, U.as<double>());
        else
            gv_u32_kernel<<<ub, 256, 0, s>>>(g, lcp, dK, s0, slice, U.as<float>());
        const int ta = mode == 0 ? G64_TA : G32_T;
        const int n_rt = na / ta;
        gv_order_kernel<<<1, 1024, 0, s>>>(g, lcp, dK, s0, slice, ta, order.as<int32_t>());
        if (timed && sl == 0 && (e = cudaEventRecordWithFlags(ev1, s, rec)) != cudaSuccess) return e;
        if (mode == 0) {
            gv_setup64_kernel<<<blocks_for((int64_t)na * slice, GV_THREADS, 152 * 8), GV_THREADS, 0, s>>>(
                g, lcp, dK, s0, slice, tb, kc, wg.as<double>(), b0g.as<int>());
            const unsigned grid = (unsigned)n_rt * (unsigned)(slice / GV_TL) * G64_QP;
            gv_main_kernel<<<grid, GV_THREADS, g64_smem(), s>>>(g, pd64.as<double>(), U.as<double>(), wg.as<double>(),
                                                               b0g.as<int>(), order.as<int32_t>(), dK, s0, slice,
                                                               part.as<double>(), err.as<int>());
        } else {
            if ((e = cudaMemsetAsync(wmm.p, 0xff, sizeof(int2) * 8 * (size_t)n_rt * (slice / G32_T), s)) !=
                cudaSuccess)
                return e;
            gv_setup32_kernel<<<blocks_for((int64_t)na * slice, 256, 152 * 32), 256, 0, s>>>(
                g, rows32.as<GvRow32>(), lamc32.as<GvCol32>(), dK, s0, slice, wg.as<float>(), b0g.as<int>(),
                wmm.as<int2>());
            const unsigned items = (unsigned)n_rt * (unsigned)(slice / G32_T) * G32_QP;
            gv_main32_kernel<<<std::min<unsigned>(items, (unsigned)g32_ctas), GV_THREADS, g32_smem(), s>>>(
                g, pd32.as<float>(), U.as<float>(), wg.as<float>(), b0g.as<int>(), wmm.as<int2>(), order.as<int32_t>(),
                dK, s0, slice,
                queue.as<unsigned>() + sl, part.as<double>(), err.as<int>());
        }
        if (timed && sl == 0 && (e = cudaEventRecordWithFlags(ev2, s, rec)) != cudaSuccess) return e;
        gv_reduce_kernel<<<(slice + 7) / 8, 256, 0, s>>>(part.as<double>(), mode == 0 ? n_rt * G64_QP : n_rt * G32_QP,
                                                         perm.as<int32_t>(), dK, s0, slice, xi.as<double>());
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (timed && (e = cudaEventRecordWithFlags(ev3, s, rec)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t GridVT::out_lnxi(const double* lambda, int n_params, const int64_t* dK, int64_t K_cap, double* lnxi,
                             uint32_t* flags, cudaStream_t s)
{
    if (K_cap <= 0) return cudaSuccess;
    gv_out_kernel<<<(unsigned)((K_cap + 255) / 256), 256, 0, s>>>(xi.as<double>(), lambda, n_params, dK, lnxi, flags);
    return cudaGetLastError();
}

namespace {

// One thread: an mbarrier expecting one arrival; with `arrive` the thread gives it, otherwise
// nothing ever completes the phase and the bounded wait of the contraction runs out of polls,
// which sets the error word exactly as a contraction tile that gives up does.
__global__ void gv_wait_check_kernel(int arrive, int polls, int* __restrict__ err)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = gv_saddr(&bar);
    gv_bar_init(b);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
    if (!gv_wait(b, 0u, polls)) atomicExch(err, 1);
}

}  // namespace

cudaError_t launch_wait_check(int arrive, int polls, int* err, cudaStream_t s)
{
    gv_wait_check_kernel<<<1, 1, 0, s>>>(arrive, polls, err);
    return cudaGetLastError();
}

cudaError_t GridVT::take_error(int* h, cudaStream_t s)
{
    *h = 0;
    cudaError_t e = cudaMemcpyAsync(h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && *h) e = cudaMemsetAsync(err.p, 0, sizeof(int), s);
    return e;
}

}  // namespace pop
