// FP32 sample-weight kernel with compensated per-thread sums.
//
// Same work decomposition as the FP64 kernel (persistent grid over
// chunk x Lambda-tile items, features in registers, Lambda constants in shared
// memory).  Each thread takes two samples per step, so one read of a Lambda's
// constants serves two weights and the two dependency chains overlap.  The
// features and constants are in base-2 log units so every exponential is one
// ex2.approx (MUFU) and the q normalisation's reciprocal one rcp.approx.  Per
// (thread, Lambda) the weights are summed with Kahan compensation; warps and
// then the block combine the (sum, compensation) pairs with an error-free
// two-sum, and one thread per Lambda widens the block result to FP64 for the
// partial.  The per-Lambda constants come from the FP64 prologue; the
// per-event log and the cross-event sum are FP64 in the finalise kernel.
#include <math.h>

#include "pop_internal.h"

namespace pop {

namespace {

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcpf(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2^u - 1.  ex2(u) - 1 loses relative accuracy as u -> 0, so |u| < 1/8 uses
// the Taylor series of e^x - 1 in x = u ln 2 to fifth order (truncation below
// 1e-8 relative there).  The series is evaluated only in warps where some lane
// needs it (samples within a few percent of mmin).
__device__ __forceinline__ float exp2m1f(float u)
{
    constexpr float c1 = 0.693147180559945f;    // ln2
    constexpr float c2 = 0.240226506959101f;    // ln2^2 / 2
    constexpr float c3 = 0.0555041086648216f;   // ln2^3 / 6
    constexpr float c4 = 0.00961812910762848f;  // ln2^4 / 24
    constexpr float c5 = 0.00133335581464284f;  // ln2^5 / 120
    float e = ex2f(u) - 1.0f;
    const bool small = fabsf(u) < 0.125f;
    if (__any_sync(0xffffffffu, small)) {
        float p = fmaf(c5, u, c4);
        p = fmaf(p, u, c3);
        p = fmaf(p, u, c2);
        p = fmaf(p, u, c1);
        p *= u;
        e = small ? p : e;
    }
    return e;
}

struct F32Sample {
    float lm1, m1, lq, sa, sb, dc, nlpi, lz1, lm1lo;
    int64_t m2b;
};

template <bool HAS_Z>
__device__ __forceinline__ void load_f32(const FeatF32& F, int64_t s, F32Sample& x)
{
    const float* b = F.base;
    const int64_t st = F.stride;
    x.lm1 = __ldg(b + F_LM1 * st + s);
    x.m1 = __ldg(b + F_M1 * st + s);
    x.lq = __ldg(b + F_LQ * st + s);
    x.sa = __ldg(b + F_SA * st + s);
    x.sb = __ldg(b + F_SB * st + s);
    x.dc = __ldg(b + F_DC * st + s);
    x.nlpi = __ldg(b + F_NLPI * st + s);
    x.lz1 = HAS_Z ? __ldg(b + F_LZ1 * st + s) : 0.0f;
    x.lm1lo = __ldg(b + F32_LM1LO * st + s);
    x.m2b = __double_as_longlong(__ldg(F.m2 + s));
}

// A sample outside every support (m1 = 0): weight 0 for any Lambda.
__device__ __forceinline__ void dead_f32(F32Sample& x)
{
    x.lm1 = x.m1 = x.lq = x.sa = x.sb = x.dc = x.nlpi = x.lz1 = x.lm1lo = 0.0f;
    x.m2b = 0;
}

// Support: mmin < m1 <= mmax (exact against the rounded-down float thresholds) and
// fl64(q m1) >= mmin on the FP64 bit pattern.
__device__ __forceinline__ bool in_support(const F32Sample& x, const LamF32& c)
{
    return (x.m1 > c.thr_lo) & (x.m1 <= c.thr_hi) & (x.m2b >= c.mmin_bits);
}

// Weight inside the support (the caller applies in_support).
template <bool HAS_Z>
__device__ __forceinline__ float weight_f32(const F32Sample& x, const LamF32& c)
{
    float aE = fmaf(c.beta, x.lq, x.nlpi);
    aE = fmaf(c.ac, x.sa, aE);
    aE = fmaf(c.bc, x.sb, aE);
    if (HAS_Z) aE = fmaf(c.km1, x.lz1, aE);
    const float e1 = ex2f(fmaf(c.nalpha, x.lm1, aE + c.cpl));
    const float d = x.m1 - c.mu;
    const float e2 = ex2f(fmaf(c.nh * d, d, aE + c.cg));
    // u = (1+beta) log2(mmin/m1): the hi parts cancel exactly near m1 = mmin and
    // the lo parts carry the difference.
    const float u = fmaf(c.b1, c.lmmin - x.lm1, fmaf(c.nb1, x.lm1lo, c.b1lmmin_lo));
    const float den = c.beta_m1 ? -u : fabsf(exp2m1f(u));
    const float tt = c.t0 + ex2f(fmaf(c.nht, x.dc, c.ct));
    return (e1 + e2) * tt * rcpf(den);
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float w)
{
    const float y = w - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// (s, c) += (s2, c2) for compensated pairs of value s - c (error-free two-sum of the sums).
__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2)
{
    const float S = s + s2;
    const float bp = S - s;
    const float e = (s - (S - bp)) + (s2 - bp);
    c = (c + c2) - e;
    s = S;
}

__device__ __forceinline__ void warp_combine(float& s, float& c)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        pair_add(s, c, s2, c2);
    }
}

template <int T, int NT, bool HAS_Z>
__global__ void __launch_bounds__(NT)
weight_f32_kernel(FeatF32 ev, FeatF32 inj, WorkDesc wd, const LamF32* __restrict__ lam,
                  const int64_t* __restrict__ dK, double* __restrict__ part, double* __restrict__ part2,
                  const uint8_t* __restrict__ need_mc)
{
    constexpr int NW = NT / 32;
    __shared__ LamF32 sl[T];
    __shared__ float rs[NW][T], rc[NW][T], rs2[NW][T], rc2[NW][T];
    const int64_t K = *dK;
    const int64_t n_tiles = (K + T - 1) / T;
    const int64_t n_items = (int64_t)wd.n_chunks * n_tiles;
    const int n_inj_chunks = wd.n_chunks - wd.n_ev_chunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int c = (int)(item / n_tiles);
        const int64_t k0 = (item - (int64_t)c * n_tiles) * T;
        const int tn = (int)(K - k0 < T ? K - k0 : T);
        if (need_mc && c >= wd.n_ev_chunks) {  // injection item: needed only for Monte Carlo xi
            bool any = false;
            for (int l = 0; l < tn; ++l) any |= need_mc[k0 + l] != 0;
            if (!any) continue;  // same decision on every thread of the block
        }
        __syncthreads();
        {
            constexpr int W = (int)(sizeof(LamF32) / 4);
            float* dst = reinterpret_cast<float*>(sl);
            for (int i = threadIdx.x; i < T * W; i += NT) {
                const int l = i / W;
                const int64_t src = k0 + (l < tn ? l : tn - 1);
                dst[i] = reinterpret_cast<const float*>(lam + src)[i - l * W];
            }
        }
        __syncthreads();
        const Chunk ch = wd.chunks[c];
        const FeatF32 F = ch.inj ? inj : ev;
        float s[T], cp[T], s2[T], cp2[T];
#pragma unroll
        for (int l = 0; l < T; ++l) s[l] = cp[l] = s2[l] = cp2[l] = 0.0f;
        // Every thread runs the same number of steps (slots past the end are dead
        // samples), so all 32 lanes reach the warp vote inside exp2m1f together.
        for (int base = 0; base < ch.len; base += 2 * NT) {
            const int j = base + threadIdx.x;
            F32Sample x0, x1;
            if (j < ch.len) load_f32<HAS_Z>(F, ch.start + j, x0);
            else dead_f32(x0);
            if (j + NT < ch.len) load_f32<HAS_Z>(F, ch.start + j + NT, x1);
            else dead_f32(x1);
#pragma unroll
            for (int l = 0; l < T; ++l) {
                const LamF32 cl = sl[l];
                const bool in0 = in_support(x0, cl), in1 = in_support(x1, cl);
                // Samples are stored in increasing q m1 per event: warps wholly below the
                // lower mass edge skip the arithmetic.
                if (__any_sync(0xffffffffu, in0 | in1)) {
                    // Evaluated on every lane (exp2m1f votes across the warp), then selected.
                    float w0 = weight_f32<HAS_Z>(x0, cl);
                    float w1 = weight_f32<HAS_Z>(x1, cl);
                    w0 = in0 ? w0 : 0.0f;
                    w1 = in1 ? w1 : 0.0f;
                    kahan_add(s[l], cp[l], w0 + w1);
                    if (ch.inj) kahan_add(s2[l], cp2[l], fmaf(w0, w0, w1 * w1));
                }
            }
        }
#pragma unroll
        for (int l = 0; l < T; ++l) {
            warp_combine(s[l], cp[l]);
            if (ch.inj) warp_combine(s2[l], cp2[l]);
            if (lane == 0) {
                rs[warp][l] = s[l];
                rc[warp][l] = cp[l];
                rs2[warp][l] = s2[l];
                rc2[warp][l] = cp2[l];
            }
        }
        __syncthreads();
        if (threadIdx.x < tn) {  // one thread per Lambda, all in warp 0
            const int l = threadIdx.x;
            float a = rs[0][l], ac = rc[0][l], b = rs2[0][l], bc = rc2[0][l];
            for (int w = 1; w < NW; ++w) {
                pair_add(a, ac, rs[w][l], rc[w][l]);
                pair_add(b, bc, rs2[w][l], rc2[w][l]);
            }
            part[(k0 + l) * wd.n_chunks + c] = (double)a - (double)ac;
            if (ch.inj) part2[(k0 + l) * n_inj_chunks + (c - wd.n_ev_chunks)] = (double)b - (double)bc;
        }
    }
}

template <int T, int NT>
const void* pick_f32(bool has_z)
{
    return has_z ? (const void*)weight_f32_kernel<T, NT, true> : (const void*)weight_f32_kernel<T, NT, false>;
}

template <int NT>
const void* pick_f32_t(int T, bool has_z)
{
    switch (T) {
        case 2: return pick_f32<2, NT>(has_z);
        case 4: return pick_f32<4, NT>(has_z);
        case 8: return pick_f32<8, NT>(has_z);
        case 16: return pick_f32<16, NT>(has_z);
        case 32: return pick_f32<32, NT>(has_z);
        default: return nullptr;
    }
}

}  // namespace

const void* weight_f32_fn(const Tiling& t, bool has_z)
{
    switch (t.block_threads) {
        case 128: return pick_f32_t<128>(t.lambda_tile, has_z);
        case 256: return pick_f32_t<256>(t.lambda_tile, has_z);
        case 512: return pick_f32_t<512>(t.lambda_tile, has_z);
        default: return nullptr;
    }
}

cudaError_t launch_weight_f32(const Tiling& t, int grid, FeatF32 ev, FeatF32 inj, WorkDesc wd, const LamF32* lam,
                              const int64_t* dK, double* part, double* part2, SurrogateXi sx, cudaStream_t s)
{
    const void* fn = weight_f32_fn(t, wd.has_z != 0);
    if (!fn) return cudaErrorInvalidValue;
    const uint8_t* need = sx.need_mc;
    void* args[] = {&ev, &inj, &wd, &lam, &dK, &part, &part2, &need};
    return cudaLaunchKernel(fn, dim3(grid), dim3(t.block_threads), args, 0, s);
}

}  // namespace pop
