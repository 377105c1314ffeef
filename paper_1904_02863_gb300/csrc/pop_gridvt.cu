// Selection term on a regular (m1, q) grid: pdet packing, the per-Lambda
// q-node factors U_b, the masked node contraction and its fixed-order
// reduction (paper, Sec. "Population acceleration": VT on a regular grid with
// GPU acceleration, low-dimensional, no spin effects).
//
// Work layout.  The contraction sum_a W_a sum_{b >= b0} pdet[a, b] U_b runs as
// tiles of 64 m1 rows x 64 Lambda columns, one CTA each, every thread holding
// a 4 x 4 block of (row, column) accumulators.  Chunks of 32 q nodes of the
// packed pdet tile and of U are staged in shared memory by cp.async.bulk
// copies that complete on an mbarrier (two stages).  Each thread computes W_a
// and b0 of its own 16 pairs, so nothing per (row, Lambda) pair is stored.
// Lambda columns are placed in ascending mmin order (a counting sort per slice)
// so that the 4 columns of a thread have nearly the same lower q edges: chunks
// at or past every edge of the thread run unmasked, chunks below all of them
// are skipped, and only the chunks between use a per-pair mask.  The result of
// a column does not depend on where the sort puts it: the sum over b of a pair
// runs in node order, and the sum over rows in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "pop.h"
#include "pop_gridvt.h"
#include "pop_internal.h"

namespace pop {

namespace {

constexpr int GV_THREADS = 256;
constexpr int GV_STAGES = 2;
constexpr int GV_WAIT_LIMIT = 1 << 22;  // mbarrier polls before a wait gives up
constexpr int GV_BUCKETS = 1024;        // mmin buckets of the column sort
constexpr double GV_SQRT2 = 1.4142135623730950488;
constexpr double GV_SQRT2PI = 2.5066282746310005024;

struct GvNodes {
    const double* m1;    // [na]
    const double* lnm1;  // [na]
    const double* wa;    // [na]
    const double* q;     // [nbp]
    int na, nb, nbp, n_rt;
};

// Per-column constants of the primary-mass and mass-ratio densities.
struct GvLam {
    double nalpha;  // exponent of m1 in the power law (-alpha)
    double cpl;     // (1 - lam) x power-law normalisation
    double mu, nh;  // Gaussian peak: mpp and -1 / (2 sigpp^2)
    double cg;      // lam / (sqrt(2 pi) sigpp Z), 0 when lam = 0
    double b1;      // 1 + beta
    double mmin, mmax;
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
    const double alpha = L[P_ALPHA], mmin = L[P_MMIN], mmax = L[P_MMAX], lam = L[P_LAM];
    if (alpha == 1.0) {  // x^-1 / ln(mmax / mmin)
        c.nalpha = -1.0;
        c.cpl = (1.0 - lam) / log(mmax / mmin);
    } else {
        c.nalpha = -alpha;
        c.cpl = (1.0 - lam) * (1.0 - alpha) / (pow(mmax, 1.0 - alpha) - pow(mmin, 1.0 - alpha));
    }
    const double mu = L[P_MPP], sig = L[P_SIGPP];
    c.mu = mu;
    c.nh = -0.5 / (sig * sig);
    if (lam > 0.0) {
        const double z = 0.5 * (erf((mmax - mu) / (GV_SQRT2 * sig)) - erf((mmin - mu) / (GV_SQRT2 * sig)));
        c.cg = lam / (GV_SQRT2PI * sig * z);
    } else {
        c.cg = 0.0;
    }
    c.b1 = 1.0 + L[P_BETA];
    c.beta_m1 = L[P_BETA] == -1.0;
    c.mmin = mmin;
    c.mmax = mmax;
}

// W_a and b0 of one (row, column) pair.  A pair outside the mass support (or
// with an empty q range) gets b0 = nb and contributes nothing.
__device__ __forceinline__ void gv_pair(const GvNodes& g, const GvLam& c, int a, double& W, int& b0)
{
    W = 0.0;
    b0 = g.nb;
    if (!c.live) return;
    const double m1 = g.m1[a];
    if (!(m1 > c.mmin && m1 <= c.mmax)) return;  // also every padding row (m1 = 0)
    double pm = c.cpl * exp(c.nalpha * g.lnm1[a]);
    if (c.cg != 0.0) {
        const double d = m1 - c.mu;
        pm += c.cg * exp(c.nh * d * d);
    }
    // ln(mmin / m1) without cancellation: mmin - m1 is exact near the edge.
    const double lr = log1p((c.mmin - m1) / m1);
    const double cq = c.beta_m1 ? 1.0 / -lr : c.b1 / -expm1(c.b1 * lr);
    W = g.wa[a] * pm * cq;
    // First q node with fl64(q m1) >= mmin; the product rounds once, and it is
    // monotone in q, so the support in b is the suffix [b0, nb).
    int lo = 0, hi = g.nb;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__dmul_rn(g.q[mid], m1) >= c.mmin) hi = mid;
        else lo = mid + 1;
    }
    b0 = lo;
}

__device__ __forceinline__ int slice_count(const int64_t* dK, int64_t slice0, int S)
{
    const int64_t n = *dK - slice0;
    return (int)(n < 0 ? 0 : (n > S ? S : n));
}

// ---------------------------------------------------------------- column sort
// perm[r] = Lambda index of column r of the slice, ascending in mmin by
// buckets (order inside a bucket is arbitrary); -1 in the padding columns.
__global__ void __launch_bounds__(1024)
gv_sort_kernel(const double* __restrict__ lambda, int P, const int64_t* __restrict__ dK, int64_t slice0, int S,
               int32_t* __restrict__ perm)
{
    __shared__ int hist[GV_BUCKETS + 1];
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
    if (threadIdx.x == 0) {
        int s = 0;
        for (int b = 0; b <= GV_BUCKETS; ++b) {
            const int h = hist[b];
            hist[b] = s;
            s += h;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int pos = atomicAdd(&hist[bucket(lambda[(slice0 + i) * P + P_MMIN])], 1);
        perm[pos] = (int32_t)(slice0 + i);
    }
    const int npad = (n + GV_TL - 1) / GV_TL * GV_TL;
    for (int r = n + threadIdx.x; r < npad; r += blockDim.x) perm[r] = -1;
}

// ---------------------------------------------------------------- U_b per column
// U[lt][b][c] = wq_b q_b^beta for column r = lt * 64 + c (0 for padding
// columns, invalid Lambda and nodes past nb).
template <class T>
__global__ void gv_u_kernel(GvNodes g, const double* __restrict__ wq, const double* __restrict__ lambda, int P,
                            const int32_t* __restrict__ perm, const int64_t* __restrict__ dK, int64_t slice0, int S,
                            T* __restrict__ U)
{
    const int n = slice_count(dK, slice0, S);
    const int64_t total = (int64_t)((n + GV_TL - 1) / GV_TL) * g.nbp * GV_TL;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % GV_TL);
        const int64_t rest = t / GV_TL;
        const int b = (int)(rest % g.nbp);
        const int lt = (int)(rest / g.nbp);
        const int r = lt * GV_TL + c;
        double u = 0.0;
        const int k = r < n ? perm[r] : -1;
        if (k >= 0 && b < g.nb) {
            const double* L = lambda + (int64_t)k * P;
            const double qb = g.q[b];
            if (qb > 0.0 && gv_valid(L, P)) u = wq[b] * pow(qb, L[P_BETA]);
        }
        U[t] = (T)u;
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

// Waits for the phase of the given parity; false after GV_WAIT_LIMIT polls.
__device__ __forceinline__ bool gv_wait(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < GV_WAIT_LIMIT; ++i) {
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

// Four consecutive-by-vector elements of a staged row: idx as produced by gv_lanes.
template <class T>
__device__ __forceinline__ void gv_load4(const T* row, int i0, T (&v)[4])
{
    if constexpr (sizeof(T) == 8) {  // two 16-byte vectors, 32 elements apart
        const double2 x = *reinterpret_cast<const double2*>(row + i0);
        const double2 y = *reinterpret_cast<const double2*>(row + i0 + 32);
        v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
    } else {
        const float4 x = *reinterpret_cast<const float4*>(row + i0);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
}

// ---------------------------------------------------------------- contraction
// part[rt][r] = sum over the 64 rows of row tile rt of W_a sum_{b >= b0} pdet[a, b] U_b
// for every column r of Lambda tile blockIdx.y.  T = double: FP64 throughout.
// T = float: FP32 pdet and U, FP32 sums per 32-node chunk added into an FP32
// running sum, FP64 W and row combine.
template <class T>
__global__ void __launch_bounds__(GV_THREADS, 2)
gv_main_kernel(GvNodes g, const T* __restrict__ pd, const T* __restrict__ U, const double* __restrict__ lambda,
               int P, const int32_t* __restrict__ perm, const int64_t* __restrict__ dK, int64_t slice0, int S,
               double* __restrict__ part, int* __restrict__ err)
{
    constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte vector
    constexpr int STAGE = GV_BC * GV_TA;   // elements of one operand chunk (GV_TA == GV_TL)
    constexpr uint32_t CHUNK_BYTES = STAGE * sizeof(T);
    static_assert(GV_TA == GV_TL, "square CTA tile");
    extern __shared__ __align__(128) unsigned char gv_dyn[];
    T* sp = reinterpret_cast<T*>(gv_dyn);  // [STAGES][BC][64] pdet
    T* su = sp + GV_STAGES * STAGE;        // [STAGES][BC][64] U
    __shared__ __align__(8) uint64_t bar[GV_STAGES];
    __shared__ GvLam lc[GV_TL];
    __shared__ int s_tmin;
    __shared__ double red[GV_THREADS / 16][GV_TL];

    const int n = slice_count(dK, slice0, S);
    const int rt = blockIdx.x, lt = blockIdx.y;
    if (lt * GV_TL >= n) return;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < GV_TL) {
        const int r = lt * GV_TL + tid;
        const int k = r < n ? perm[r] : -1;
        GvLam c;
        c.live = 0;
        if (k >= 0) gv_consts(lambda + (int64_t)k * P, P, c);
        lc[tid] = c;
    }
    if (tid == 0) {
        s_tmin = INT_MAX;
        for (int st = 0; st < GV_STAGES; ++st) gv_bar_init(gv_saddr(&bar[st]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // This thread's rows and columns: index j -> (j / V) * 16V + t V + j % V, so
    // that the 16-byte shared-memory reads of a quarter warp are contiguous.
    int row[4], col[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        col[j] = (j / V) * (16 * V) + tx * V + (j % V);
        row[j] = (j / V) * (16 * V) + ty * V + (j % V);
    }
    double W[4][4];
    int b0[4][4];
    int tmin = INT_MAX, tmax = -1;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            gv_pair(g, lc[col[j]], rt * GV_TA + row[i], W[i][j], b0[i][j]);
            if (b0[i][j] < g.nb) {
                tmin = min(tmin, b0[i][j]);
                tmax = max(tmax, b0[i][j]);
            }
        }
    if (tmin != INT_MAX) atomicMin(&s_tmin, tmin);
    __syncthreads();
    double* out = part + (int64_t)rt * S + lt * GV_TL;
    if (s_tmin >= g.nb) {  // no pair of the tile has support
        if (tid < GV_TL) out[tid] = 0.0;
        return;
    }
    const int nch = g.nbp / GV_BC;
    const int c0 = s_tmin / GV_BC;
    const T* pd_tile = pd + (int64_t)rt * g.nbp * GV_TA;
    const T* u_tile = U + (int64_t)lt * g.nbp * GV_TL;
    auto issue = [&](int c) {
        const int st = (c - c0) % GV_STAGES;
        const uint32_t b = gv_saddr(&bar[st]);
        gv_expect_tx(b, 2 * CHUNK_BYTES);
        gv_bulk_load(gv_saddr(sp + st * STAGE), pd_tile + (int64_t)c * STAGE, CHUNK_BYTES, b);
        gv_bulk_load(gv_saddr(su + st * STAGE), u_tile + (int64_t)c * STAGE, CHUNK_BYTES, b);
    };
    if (tid == 0)
        for (int c = c0; c < nch && c < c0 + GV_STAGES; ++c) issue(c);

    T acc[4][4];
    float run[4][4];  // FP32 form: running sum of the chunk sums
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = T(0);
            run[i][j] = 0.0f;
        }
    for (int c = c0; c < nch; ++c) {
        const int st = (c - c0) % GV_STAGES;
        const bool ok = gv_wait(gv_saddr(&bar[st]), (uint32_t)(((c - c0) / GV_STAGES) & 1));
        if (__syncthreads_or(!ok)) {
            // Give up: flag it, let the copies already issued land (bounded), leave NaN.
            if (tid == 0) {
                atomicExch(err, 1);
                for (int d = c; d < nch && d < c + GV_STAGES; ++d)
                    gv_wait(gv_saddr(&bar[(d - c0) % GV_STAGES]), (uint32_t)(((d - c0) / GV_STAGES) & 1));
            }
            __syncthreads();
            if (tid < GV_TL) out[tid] = NAN;
            return;
        }
        const int cb = c * GV_BC;
        if (cb + GV_BC > tmin) {
            const T* ps = sp + st * STAGE;
            const T* us = su + st * STAGE;
            if (cb >= tmax) {  // every pair of the thread has support on the whole chunk
#pragma unroll 4
                for (int bb = 0; bb < GV_BC; ++bb) {
                    T p[4], u[4];
                    gv_load4(ps + bb * GV_TA, row[0], p);
                    gv_load4(us + bb * GV_TL, col[0], u);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(p[i], u[j], acc[i][j]);
                }
            } else {  // a support edge inside the chunk: per-pair mask
#pragma unroll 2
                for (int bb = 0; bb < GV_BC; ++bb) {
                    const int b = cb + bb;
                    T p[4], u[4];
                    gv_load4(ps + bb * GV_TA, row[0], p);
                    gv_load4(us + bb * GV_TL, col[0], u);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(p[i], b >= b0[i][j] ? u[j] : T(0), acc[i][j]);
                }
            }
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        run[i][j] += acc[i][j];
                        acc[i][j] = 0.0f;
                    }
            }
        }
        __syncthreads();  // the stage is free again
        if (tid == 0 && c + GV_STAGES < nch) issue(c + GV_STAGES);
    }

    // Fixed-order combine: rows of the thread (i = 0..3), then the 16 row groups.
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double a = sizeof(T) == 4 ? (double)run[i][j] : (double)acc[i][j];
            t += b0[i][j] < g.nb ? W[i][j] * a : 0.0;
        }
        red[ty][col[j]] = t;
    }
    __syncthreads();
    if (tid < GV_TL) {
        double s = 0.0;
        for (int y = 0; y < GV_THREADS / 16; ++y) s += red[y][tid];
        out[tid] = s;
    }
}

// xi[k] = sum over row tiles (in order) of part[rt][r], k = perm[r].
__global__ void gv_reduce_kernel(const double* __restrict__ part, int n_rt, const int32_t* __restrict__ perm,
                                 const int64_t* __restrict__ dK, int64_t slice0, int S, double* __restrict__ xi)
{
    const int n = slice_count(dK, slice0, S);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double s = 0.0;
    for (int rt = 0; rt < n_rt; ++rt) s += part[(int64_t)rt * S + r];
    xi[perm[r]] = s;
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

// pdet [n_m1][n_q] -> [n_rt][nbp][64] in FP64 and FP32 (zeros in the padding);
// *bad = 1 when a used entry is not finite or negative.
__global__ void gv_pack_kernel(const double* __restrict__ pdet, int n_m1, int n_q, int nb, int nbp, int n_rt,
                               double* __restrict__ pd64, float* __restrict__ pd32, int* __restrict__ bad)
{
    const int64_t total = (int64_t)n_rt * nbp * GV_TA;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % GV_TA);
        const int64_t rest = t / GV_TA;
        const int b = (int)(rest % nbp);
        const int a = (int)(rest / nbp) * GV_TA + c;
        double v = 0.0;
        if (a < n_m1 && b < nb) {
            v = pdet[(int64_t)a * n_q + b];
            if (!(isfinite(v) && v >= 0.0)) {
                atomicExch(bad, 1);
                v = 0.0;
            }
        }
        pd64[t] = v;
        pd32[t] = (float)v;
    }
}

int blocks_for(int64_t n, int threads, int cap)
{
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

size_t main_smem(int mode) { return (size_t)2 * GV_STAGES * GV_BC * GV_TA * (mode == 0 ? 8 : 4); }

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
    const int na_ = (n1 + GV_TA - 1) / GV_TA * GV_TA;
    const int nbp_ = (nb_ + GV_BC - 1) / GV_BC * GV_BC;
    // Trapezoid weights over all nodes (a node's weight is half the span to its neighbours).
    std::vector<double> wm(na_, 0.0), lm(na_, 0.0), m(na_, 0.0), wqv(nbp_, 0.0), qv(nbp_, 0.0);
    for (int a = 0; a < n1; ++a) {
        const double hi = a + 1 < n1 ? hm[a + 1] : hm[a], lo = a > 0 ? hm[a - 1] : hm[a];
        wm[a] = 0.5 * (hi - lo);
        m[a] = hm[a];
        lm[a] = hm[a] > 0.0 ? std::log(hm[a]) : 0.0;
    }
    for (int b = 0; b < nb_; ++b) {
        const double hi = b + 1 < nq ? hq[b + 1] : hq[b], lo = b > 0 ? hq[b - 1] : hq[b];
        wqv[b] = 0.5 * (hi - lo);
        qv[b] = hq[b];
    }
    const int n_rt_ = na_ / GV_TA;
    DevBuf dm, dlm, dwa, dq, dwq, p64, p32, tmp, dbad;
    auto ck = [&](cudaError_t e) { return e == cudaSuccess; };
    const size_t packed = (size_t)n_rt_ * nbp_ * GV_TA;
    if (!ck(dm.alloc(sizeof(double) * na_)) || !ck(dlm.alloc(sizeof(double) * na_)) ||
        !ck(dwa.alloc(sizeof(double) * na_)) || !ck(dq.alloc(sizeof(double) * nbp_)) ||
        !ck(dwq.alloc(sizeof(double) * nbp_)) || !ck(p64.alloc(sizeof(double) * packed)) ||
        !ck(p32.alloc(sizeof(float) * packed)) || !ck(dbad.alloc(sizeof(int))))
        return bad(POP_ENOMEM, "pop_load_vt_grid: device allocation failed");
    const double* src = pdet;
    if (!on_device) {
        if (!ck(tmp.alloc(sizeof(double) * (size_t)n1 * nq))) return bad(POP_ENOMEM, "pop_load_vt_grid: allocation");
        if (!ck(cudaMemcpyAsync(tmp.p, pdet, sizeof(double) * (size_t)n1 * nq, cudaMemcpyHostToDevice, s)))
            return bad(POP_ECUDA, "pop_load_vt_grid: copying pdet failed");
        src = tmp.as<double>();
    }
    bool okc = ck(cudaMemcpyAsync(dm.p, m.data(), sizeof(double) * na_, cudaMemcpyHostToDevice, s)) &&
               ck(cudaMemcpyAsync(dlm.p, lm.data(), sizeof(double) * na_, cudaMemcpyHostToDevice, s)) &&
               ck(cudaMemcpyAsync(dwa.p, wm.data(), sizeof(double) * na_, cudaMemcpyHostToDevice, s)) &&
               ck(cudaMemcpyAsync(dq.p, qv.data(), sizeof(double) * nbp_, cudaMemcpyHostToDevice, s)) &&
               ck(cudaMemcpyAsync(dwq.p, wqv.data(), sizeof(double) * nbp_, cudaMemcpyHostToDevice, s)) &&
               ck(cudaMemsetAsync(dbad.p, 0, sizeof(int), s));
    if (!okc) return bad(POP_ECUDA, "pop_load_vt_grid: copying the nodes failed");
    gv_pack_kernel<<<blocks_for((int64_t)packed, 256, 152 * 32), 256, 0, s>>>(src, n1, nq, nb_, nbp_, n_rt_,
                                                                              p64.as<double>(), p32.as<float>(),
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
    wa.swap(dwa);
    q.swap(dq);
    wq.swap(dwq);
    pd64.swap(p64);
    pd32.swap(p32);
    n_m1 = n1;
    n_q = nq;
    na = na_;
    nb = nb_;
    nbp = nbp_;
    n_rt = n_rt_;
    k_cap = 0;  // the scratch depends on the grid shape
    slice = 0;
    return POP_OK;
}

cudaError_t GridVT::ensure(int64_t K)
{
    if (K <= k_cap && slice > 0) return cudaSuccess;
    const int64_t cap = std::max<int64_t>(std::max<int64_t>(K, k_cap), 64);
    const int S = (int)std::min<int64_t>((cap + GV_TL - 1) / GV_TL * GV_TL, GV_SLICE);
    DevBuf p, u, pt, x;
    cudaError_t e;
    if ((e = p.alloc(sizeof(int32_t) * S)) != cudaSuccess) return e;
    if ((e = u.alloc(sizeof(double) * (size_t)S * nbp)) != cudaSuccess) return e;
    if ((e = pt.alloc(sizeof(double) * (size_t)n_rt * S)) != cudaSuccess) return e;
    if ((e = x.alloc(sizeof(double) * cap)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(gv_main_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)main_smem(0))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(gv_main_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)main_smem(1))) != cudaSuccess)
        return e;
    perm.swap(p);
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
    const GvNodes g{m1.as<double>(), lnm1.as<double>(), wa.as<double>(), q.as<double>(), na, nb, nbp, n_rt};
    const int n_sl = (int)((K_cap + slice - 1) / slice);
    cudaError_t e;
    if (timed && (e = cudaEventRecordWithFlags(ev0, s, rec)) != cudaSuccess) return e;
    for (int sl = 0; sl < n_sl; ++sl) {
        const int64_t s0 = (int64_t)sl * slice;
        gv_sort_kernel<<<1, 1024, 0, s>>>(lambda, n_params, dK, s0, slice, perm.as<int32_t>());
        const int64_t u_elems = (int64_t)slice * nbp;
        const int ub = blocks_for(u_elems, 256, 152 * 16);
        if (mode == 0)
            gv_u_kernel<double><<<ub, 256, 0, s>>>(g, wq.as<double>(), lambda, n_params, perm.as<int32_t>(), dK, s0,
                                                  slice, U.as<double>());
        else
            gv_u_kernel<float><<<ub, 256, 0, s>>>(g, wq.as<double>(), lambda, n_params, perm.as<int32_t>(), dK, s0,
                                                 slice, U.as<float>());
        if (timed && sl == 0 && (e = cudaEventRecordWithFlags(ev1, s, rec)) != cudaSuccess) return e;
        const dim3 grid((unsigned)n_rt, (unsigned)(slice / GV_TL));
        if (mode == 0)
            gv_main_kernel<double><<<grid, GV_THREADS, main_smem(0), s>>>(
                g, pd64.as<double>(), U.as<double>(), lambda, n_params, perm.as<int32_t>(), dK, s0, slice,
                part.as<double>(), err.as<int>());
        else
            gv_main_kernel<float><<<grid, GV_THREADS, main_smem(1), s>>>(
                g, pd32.as<float>(), U.as<float>(), lambda, n_params, perm.as<int32_t>(), dK, s0, slice,
                part.as<double>(), err.as<int>());
        if (timed && sl == 0 && (e = cudaEventRecordWithFlags(ev2, s, rec)) != cudaSuccess) return e;
        gv_reduce_kernel<<<(slice + 255) / 256, 256, 0, s>>>(part.as<double>(), n_rt, perm.as<int32_t>(), dK, s0,
                                                             slice, xi.as<double>());
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

cudaError_t GridVT::take_error(int* h, cudaStream_t s)
{
    *h = 0;
    cudaError_t e = cudaMemcpyAsync(h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && *h) e = cudaMemsetAsync(err.p, 0, sizeof(int), s);
    return e;
}

}  // namespace pop
