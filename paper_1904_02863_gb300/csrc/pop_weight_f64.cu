// FP64 sample-weight kernel with per-(event chunk, Lambda) segmented sums.
//
// Paper, Sec. "Population acceleration": evaluating the population model for
// every posterior sample is the embarrassingly parallel hot loop of the
// recycled likelihood, Eq. (poplike).  Here one persistent grid walks work
// items (chunk of one event's samples or of the injections) x (tile of T
// Lambda points).  Every thread keeps one sample's features in registers and
// evaluates its weight for the T Lambda points of the tile, whose constants
// sit in shared memory; the block then reduces the T partial sums in a fixed
// order (shuffle tree, then warps in order) and writes one FP64 partial per
// (Lambda, chunk) — no atomics, bit-reproducible.
//
// w(theta) = [exp(aE + cpl - alpha ln m1) + exp(aE + cg - (m1-mu)^2/(2 sig^2))]
//            * [(1-xi_t)/4 + exp(ct - dc/(2 sig_t^2))] / |expm1((1+beta) ln(mmin/m1))|,
// evaluated with max(cpl, cg) moved into the tilt factor (LamF64::rmix, t0m, ctm)
// with aE = -ln pi + beta ln q + (alpha_chi-1)(ln a1 + ln a2) + (beta_chi-1)(ln(1-a1) + ln(1-a2))
//          [+ (kappa-1) ln(1+z)], and every Lambda-only factor folded into cpl, cg, ct.
#include <math.h>

#include <algorithm>

#include "pop_internal.h"

namespace pop {

namespace {

struct F64Sample {
    double lm1, m1, lq, sa, sb, dc, nlpi, lz1, invm1;
    int64_t m1b, m2b;  // bit patterns of m1, m2 (non-negative doubles compare as integers)
};


template <bool HAS_Z>
__device__ __forceinline__ void load_f64(const FeatF64& F, int64_t s, F64Sample& x)
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

template <bool HAS_Z>
__device__ __forceinline__ double weight_f64(const F64Sample& x, const LamF64& c, const double2* __restrict__ tab,
                                             const ExpConsts& kc)
{
    // Weight inside the support (the caller applies in_support).
    double aE = fma(c.beta, x.lq, x.nlpi);
    aE = fma(c.ac, x.sa, aE);
    aE = fma(c.bc, x.sb, aE);
    if (HAS_Z) aE = fma(c.km1, x.lz1, aE);
    // The mass mixture (1-lam) C_pl m1^-alpha + lam C_g N(m1) with the larger of its two
    // constants (cpl, cg in logs) moved into the tilt factor: e1 + rmix e2 (or e2 + rmix e1),
    // rmix <= 1, so neither exponential needs its constant added (2 FP64 ops fewer).
    const double e1 = exp_tab(fma(c.nalpha, x.lm1, aE), tab, kc);
    // Gaussian exponent -(m1 - mu)^2 / (2 sig^2) = -y^2 with y = (m1 - mu) / (sqrt2 sig) formed
    // by one fma from per-Lambda constants (3 FP64 ops instead of 4).  The rounding of
    // gc = -mu gs shifts y by at most |mu gs| 1.1e-16, so the exponent by 2|y| |mu gs| 1.1e-16
    // absolute: of the order of the roundings of the subtract-and-square form at the same y.
    const double y = fma(x.m1, c.gs, c.gc);
    const double e2 = exp_tab(fma(-y, y, aE), tab, kc);
    const double mix = fma(c.rmix, c.mix_swap ? e1 : e2, c.mix_swap ? e2 : e1);
    // u = kq ln(mmin/m1) for the q normalisation, one fma with kq ln mmin folded into a
    // per-Lambda constant (kq = 1 + beta, or 1 for beta = -1, whose normalisation is
    // ln(m1/mmin) = -u).  Within ~3% of the lower edge the log difference would cancel,
    // so ln(mmin/m1) is log1p((mmin - m1)/m1) by its series (mmin - m1 is exact there);
    // the test runs on bit patterns (integer pipe).
    double u = fma(-c.kq, x.lm1, c.kqlmmin);
    if (llabs(x.m1b - c.mmin_bits) < NEAR_EDGE_BITS) u = c.kq * log1p_near0(x.invm1 * (c.mmin - x.m1));
    const double den = c.beta_m1 ? -u : fabs(expm1_tab(u, tab, kc));
    const double tt = c.t0m + exp_tab(fma(c.nht, x.dc, c.ctm), tab, kc);
    return mix * tt * rcp_pos(den);
}

// Support: mmin < m1 <= mmax and fl64(q m1) >= mmin, compared on bit patterns
// (integer pipe; non-negative doubles order like their bits).
__device__ __forceinline__ bool in_support(const F64Sample& x, const LamF64& c)
{
    return (x.m1b > c.mmin_bits) & (x.m1b <= c.mmax_bits) & (x.m2b >= c.mmin_bits);
}

// A sample outside every support (m1 = 0): weight 0 for any Lambda.
__device__ __forceinline__ void dead_f64(F64Sample& x)
{
    x.lm1 = x.m1 = x.lq = x.sa = x.sb = x.dc = x.nlpi = x.lz1 = x.invm1 = 0.0;
    x.m1b = x.m2b = 0;
}

// Copies the 2^(j/2048) table into shared memory (once per block of the persistent grid).
template <int NT>
__device__ __forceinline__ void load_table(double2* dst, const double2* __restrict__ src)
{
    for (int i = threadIdx.x; i < EXP_TABLE_SIZE; i += NT) dst[i] = src[i];
}

template <int T, int NT, bool HAS_Z>
__global__ void __launch_bounds__(NT)
weight_f64_kernel(FeatF64 ev, FeatF64 inj, WorkDesc wd, const LamF64* __restrict__ lam,
                  const int64_t* __restrict__ dK, double* __restrict__ part, double* __restrict__ part2,
                  const double2* __restrict__ exptab, ExpConsts kc, unsigned long long* __restrict__ queue)
{
    extern __shared__ double2 stab[];  // EXP_TABLE_SIZE entries (dynamic shared memory)
    __shared__ LamF64 sl[T];
    __shared__ double red[NT / 32][T];
    __shared__ double red2[NT / 32][T];
    load_table<NT>(stab, exptab);
    const int64_t K = *dK;
    const int64_t n_tiles = (K + T - 1) / T;
    const int64_t n_items = (int64_t)wd.n_chunks * n_tiles;
    const int n_inj_chunks = wd.n_chunks - wd.n_ev_chunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // Items come from a queue (zeroed before the launch), in chunk-major order, so a chunk's
    // Lambda tiles still run together; blocks that finish early take more.
    __shared__ unsigned long long s_item;
    for (;;) {
        __syncthreads();  // the previous item is done with sl / red / s_item
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t item = (int64_t)s_item;
        if (item >= n_items) break;
        const int c = (int)(item / n_tiles);
        const int64_t k0 = (item - (int64_t)c * n_tiles) * T;
        const int tn = (int)(K - k0 < T ? K - k0 : T);
        {
            constexpr int W = (int)(sizeof(LamF64) / 8);
            double* dst = reinterpret_cast<double*>(sl);
            for (int i = threadIdx.x; i < T * W; i += NT) {
                const int l = i / W;
                const int64_t src = k0 + (l < tn ? l : tn - 1);
                dst[i] = reinterpret_cast<const double*>(lam + src)[i - l * W];
            }
        }
        __syncthreads();
        const Chunk ch = wd.chunks[c];
        const FeatF64 F = ch.inj ? inj : ev;
        double acc[T], acc2[T];
#pragma unroll
        for (int l = 0; l < T; ++l) acc[l] = acc2[l] = 0.0;
        // Same trip count on every thread (slots past the end are dead samples), so
        // the whole warp takes part in the support vote.  Samples are stored in
        // increasing q m1 within an event, so the ones below a Lambda's lower mass
        // edge are contiguous and their warps skip the FP64 arithmetic.
        for (int base = 0; base < ch.len; base += NT) {
            const int j = base + threadIdx.x;
            F64Sample x;
            if (j < ch.len) load_f64<HAS_Z>(F, ch.start + j, x);
            else dead_f64(x);
#pragma unroll
            for (int l = 0; l < T; ++l) {
                const LamF64& cl = sl[l];
                const bool in = in_support(x, cl);
                // Warps with no lane in the support add nothing (and spend no FP64 operation).
                if (__any_sync(0xffffffffu, in)) {
                    double w = weight_f64<HAS_Z>(x, cl, stab, kc);
                    w = in ? w : 0.0;
                    acc[l] += w;
                    if (ch.inj) acc2[l] = fma(w, w, acc2[l]);
                }
            }
        }
#pragma unroll
        for (int l = 0; l < T; ++l) {
            double v = acc[l], v2 = acc2[l];
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                if (ch.inj) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
            }
            if (lane == 0) {
                red[warp][l] = v;
                red2[warp][l] = v2;
            }
        }
        __syncthreads();
        if (threadIdx.x < tn) {
            const int l = threadIdx.x;
            double s = 0.0, s2 = 0.0;
            for (int w = 0; w < NT / 32; ++w) {
                s += red[w][l];
                s2 += red2[w][l];
            }
            part[(k0 + l) * wd.n_chunks + c] = s;
            if (ch.inj) part2[(k0 + l) * n_inj_chunks + (c - wd.n_ev_chunks)] = s2;
        }
    }
}

template <int T, int NT>
const void* pick_f64(bool has_z)
{
    return has_z ? (const void*)weight_f64_kernel<T, NT, true> : (const void*)weight_f64_kernel<T, NT, false>;
}

template <int NT>
const void* pick_f64_t(int T, bool has_z)
{
    switch (T) {
        case 1: return pick_f64<1, NT>(has_z);
        case 2: return pick_f64<2, NT>(has_z);
        case 4: return pick_f64<4, NT>(has_z);
        case 8: return pick_f64<8, NT>(has_z);
        case 16: return pick_f64<16, NT>(has_z);
        default: return nullptr;
    }
}

}  // namespace

const void* weight_f64_fn(const Tiling& t, bool has_z)
{
    switch (t.block_threads) {
        case 128: return pick_f64_t<128>(t.lambda_tile, has_z);
        case 256: return pick_f64_t<256>(t.lambda_tile, has_z);
        case 512: return pick_f64_t<512>(t.lambda_tile, has_z);
        default: return nullptr;
    }
}

cudaError_t launch_weight_f64(const Tiling& t, int grid, FeatF64 ev, FeatF64 inj, WorkDesc wd, const LamF64* lam,
                              const int64_t* dK, double* part, double* part2, const double2* exptab,
                              ExpConsts kc, unsigned long long* queue, cudaStream_t s)
{
    const void* fn = weight_f64_fn(t, wd.has_z != 0);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&ev, &inj, &wd, &lam, &dK, &part, &part2, &exptab, &kc, &queue};
    return cudaLaunchKernel(fn, dim3(grid), dim3(t.block_threads), args, WEIGHT_F64_DYN_SMEM, s);
}

namespace {

__global__ void math_check_kernel(int fn, int64_t n, const double* __restrict__ x, double* __restrict__ y,
                                  const double2* __restrict__ exptab, ExpConsts kc,
                                  const LogEntry* __restrict__ logtab, LogConsts logc)
{
    extern __shared__ double2 stab[];
    load_table<256>(stab, exptab);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fn == 0 ? exp_tab(x[i], stab, kc)
                       : (fn == 1 ? expm1_tab(x[i], stab, kc) : (fn == 2 ? rcp_pos(x[i]) : log_pos(x[i], logtab, logc)));
}

}  // namespace

cudaError_t launch_math_check(int fn, int64_t n, const double* x, double* y, const double2* exptab, ExpConsts kc,
                              const LogEntry* logtab, LogConsts logc, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    math_check_kernel<<<(unsigned)blocks, 256, WEIGHT_F64_DYN_SMEM, s>>>(fn, n, x, y, exptab, kc, logtab, logc);
    return cudaGetLastError();
}

}  // namespace pop
