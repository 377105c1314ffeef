// Surrogate network kernels: the tcgen05 BF16 GEMM of training with TMEM
// accumulators and fused epilogues, plus the small CUDA-core kernels of the
// input/output layers, the reductions, transposes and Adam.  (The inference
// forward is one fused kernel, pop_mlp_fused.cu.)
//
// GEMM: C[M x N] = A[M x K] . B[N x K]^T with A and B K-major BF16 in global
// memory, M a multiple of 128 (one CTA per 128 rows = 128 TMEM lanes), N a
// multiple of 16 up to 256 (FP32 accumulator columns), K a multiple of 64.  A CTA
// takes 64 of the N columns when N is a multiple of 64 (all of them otherwise), so
// the network's small batches still spread over many SMs.  Its 64-wide K tiles
// of A (128 rows) and B come by 2-D TMA loads (128-byte swizzle) into a ring of up
// to four stages, all issued ahead, so that the copies of later tiles run under
// the MMAs of earlier ones; one thread issues the four K = 16 tcgen05.mma of a
// tile and commits them to the stage's mbarrier, and refills the stage of the
// tile before once its MMAs are done.  Every wait has a time limit: on time-out
// the CTA sets the error flag, waits once more for what it issued and frees its
// TMEM.  The epilogue reads the accumulator with tcgen05.ld (warp w owns lanes
// 32w..32w+31 = its 32 rows).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <random>
#include <tuple>
#include <map>

#include "pop_internal.h"
#include "pop_mlp.h"
#include "pop_tc.cuh"

namespace pop {

namespace {

using bf16 = __nv_bfloat16;
using namespace tc;

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;
constexpr int TC_THREADS = 128;
constexpr int TC_STAGES = 4;                      // ring depth (K tiles in flight)
constexpr uint32_t TC_A_TILE = TC_BM * TC_BK * 2;  // 16 KB
// Dynamic shared memory: 1 KB to align the base, 1 KB of barriers, then the ring.
constexpr int TC_SMEM_MAX = 2048 + TC_STAGES * (TC_A_TILE + 256 * TC_BK * 2);

enum { EPI_FWD = 0, EPI_BWD = 1, EPI_F32 = 2 };

// Columns per CTA of a GEMM with N columns (both the kernel and its launcher use this).
__host__ __device__ __forceinline__ int gemm_bn(int N) { return N % 64 == 0 ? 64 : N; }

// TMEM columns of a CTA with bn accumulator columns (a power of two, at least 32).
__host__ __device__ __forceinline__ uint32_t gemm_tmem_cols(int bn)
{
    uint32_t c = 32;
    while ((int)c < bn) c <<= 1;
    return c;
}

// Bytes of one ring stage: an A tile and a B tile of bn rows (a multiple of 1024).
__host__ __device__ __forceinline__ uint32_t gemm_stage_bytes(int bn) { return TC_A_TILE + (uint32_t)bn * TC_BK * 2; }

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ __forceinline__ float siluf_(float z) { return z * sigmoidf_(z); }
__device__ __forceinline__ float dsiluf_(float z)
{
    const float s = sigmoidf_(z);
    return s * (1.0f + z * (1.0f - s));
}

struct GemmArgs {
    const bf16* A;
    int lda;
    const bf16* B;
    int ldb;
    int M, N, K, k_split;  // blockIdx.y covers K range [y * k_split, (y + 1) * k_split)
    int epi;
    const float* bias;     // EPI_FWD
    float* Z;              // EPI_FWD: pre-activation out; EPI_BWD: pre-activation of the layer below (in)
    int ldz;
    bf16* H;               // EPI_FWD: SiLU(Z) out; EPI_BWD: dZ out
    int ldh;
    float* C;              // EPI_F32: C + blockIdx.y * c_split_stride
    int ldc;
    int64_t c_split_stride;
    int* err;
};

__global__ void __launch_bounds__(TC_THREADS)
gemm_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
               const __grid_constant__ GemmArgs g)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gb = smem_raw + (base - raw);
    const uint32_t bar_full = base;                 // TC_STAGES barriers: tile landed
    const uint32_t bar_done = base + 8 * TC_STAGES; // TC_STAGES barriers: its MMAs finished
    const uint32_t bar_fin = base + 16 * TC_STAGES; // every MMA issued so far finished
    uint32_t* tslot = reinterpret_cast<uint32_t*>(gb + 16 * TC_STAGES + 8);
    const uint32_t ring = base + 1024;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_BM;
    const int bn = gemm_bn(g.N);
    const int n0 = blockIdx.z * bn;
    const int kbeg = blockIdx.y * g.k_split;
    const int kend = min(g.K, kbeg + g.k_split);
    const int nk = (kend - kbeg) / TC_BK;
    const int S = min(TC_STAGES, nk);
    const uint32_t sbytes = gemm_stage_bytes(bn);
    const uint32_t ncols = gemm_tmem_cols(bn);

    if (warp == 0) tmem_alloc(smem_u32(tslot), ncols);
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_done + 8 * s, 1);
        }
        mbar_init(bar_fin, 1);
        for (int t = 0; t < S; ++t) {  // one arrival per stage, expecting both tiles' bytes
            const uint32_t st = ring + t * sbytes;
            mbar_expect_tx(bar_full + 8 * t, sbytes);
            tma_copy_2d(st, &map_a, kbeg + t * TC_BK, m0, bar_full + 8 * t);
            tma_copy_2d(st + TC_A_TILE, &map_b, kbeg + t * TC_BK, n0, bar_full + 8 * t);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_bf16(TC_BM, bn);
    int bad = 0, t = 0, issued = S;
    uint32_t full_ph = 0, done_ph = 0;
    if (tid == 0) {
        for (; t < nk; ++t) {
            const int s = t % S;
            if (!mbar_wait(bar_full + 8 * s, (full_ph >> s) & 1u)) {
                bad = 1;
                break;
            }
            full_ph ^= 1u << s;
            tc_fence_after();
            const uint32_t st = ring + s * sbytes;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
                mma_bf16(tmem, sdesc_sw128(st + kk * 32), sdesc_sw128(st + TC_A_TILE + kk * 32), idesc,
                         (t > 0 || kk > 0) ? 1u : 0u);
            mma_commit(bar_done + 8 * s);
            // The stage of the tile before takes the tile S after it once its MMAs are done.
            if (t >= 1 && t - 1 + S < nk) {
                const int sp = (t - 1) % S;
                if (!mbar_wait(bar_done + 8 * sp, (done_ph >> sp) & 1u)) {
                    ++t;
                    bad = 1;
                    break;
                }
                done_ph ^= 1u << sp;
                const uint32_t sq = ring + sp * sbytes;
                const int k0 = kbeg + (t - 1 + S) * TC_BK;
                mbar_expect_tx(bar_full + 8 * sp, sbytes);
                tma_copy_2d(sq, &map_a, k0, m0, bar_full + 8 * sp);
                tma_copy_2d(sq + TC_A_TILE, &map_b, k0, n0, bar_full + 8 * sp);
                ++issued;
            }
        }
        mma_commit(bar_fin);
    }
    int failed = __syncthreads_or(bad);
    if (!failed) failed = __syncthreads_or(!mbar_wait(bar_fin, 0));
    tc_fence_after();
    if (!failed) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        // Each thread owns one row: 16 consecutive columns per step, stored as 16-byte vectors
        // (the leading dimensions are multiples of 16 elements).
        for (int c0 = 0; c0 < bn; c0 += 16) {
            const int col = n0 + c0;
            float v[16];
            tmem_ld16(trow + (uint32_t)c0, v);
            if (g.epi == EPI_FWD) {
                float z[16];
                __align__(16) bf16 hb[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    z[j] = v[j] + g.bias[col + j];
                    hb[j] = __float2bfloat16(siluf_(z[j]));
                }
                float4* zd = reinterpret_cast<float4*>(g.Z + (size_t)row * g.ldz + col);
#pragma unroll
                for (int q = 0; q < 4; ++q) zd[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
                uint4* hd = reinterpret_cast<uint4*>(g.H + (size_t)row * g.ldh + col);
                hd[0] = reinterpret_cast<const uint4*>(hb)[0];
                hd[1] = reinterpret_cast<const uint4*>(hb)[1];
            } else if (g.epi == EPI_BWD) {
                const float4* zs = reinterpret_cast<const float4*>(g.Z + (size_t)row * g.ldz + col);
                __align__(16) bf16 hb[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 z = zs[q];
                    hb[4 * q] = __float2bfloat16(v[4 * q] * dsiluf_(z.x));
                    hb[4 * q + 1] = __float2bfloat16(v[4 * q + 1] * dsiluf_(z.y));
                    hb[4 * q + 2] = __float2bfloat16(v[4 * q + 2] * dsiluf_(z.z));
                    hb[4 * q + 3] = __float2bfloat16(v[4 * q + 3] * dsiluf_(z.w));
                }
                uint4* hd = reinterpret_cast<uint4*>(g.H + (size_t)row * g.ldh + col);
                hd[0] = reinterpret_cast<const uint4*>(hb)[0];
                hd[1] = reinterpret_cast<const uint4*>(hb)[1];
            } else {
                float4* cd = reinterpret_cast<float4*>(g.C + blockIdx.y * g.c_split_stride + (size_t)row * g.ldc + col);
#pragma unroll
                for (int q = 0; q < 4; ++q) cd[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    } else if (tid == 0) {
        atomicExch(g.err, 1);
        // Let the MMAs and copies in flight finish before the TMEM and the shared memory go.
        mma_commit(bar_fin);
        mbar_wait(bar_fin, 0);
        for (int u = t; u < issued; ++u) {
            const int s = u % S;
            mbar_wait(bar_full + 8 * s, (full_ph >> s) & 1u);
            full_ph ^= 1u << s;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

cudaError_t set_gemm_attributes()
{
    return cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX);
}

// The TMA maps of the GEMM operands, made once per (buffer, rows, width, box rows): a map is a
// function of those alone, so a cached one stays valid when a buffer is freed and another takes
// its address.
const CUtensorMap* operand_map(const void* ptr, int rows, int cols, int box_rows)
{
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, int>, CUtensorMap> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(ptr, rows, cols, box_rows);
    auto it = cache.find(key);
    if (it != cache.end()) return &it->second;
    if (cache.size() > 512) cache.clear();
    CUtensorMap m;
    if (!make_tile_map(&m, ptr, rows, cols, box_rows)) return nullptr;
    return &cache.emplace(key, m).first->second;
}

cudaError_t launch_gemm(const GemmArgs& g, int k_splits, cudaStream_t s)
{
    if (g.M % TC_BM || g.N % 16 || g.N > 256 || g.N < 16 || g.K % TC_BK || g.k_split % TC_BK || g.k_split <= 0 ||
        (int64_t)g.k_split * k_splits < g.K || (int64_t)g.k_split * (k_splits - 1) >= g.K)
        return cudaErrorInvalidValue;
    if (g.lda % 8 || g.ldb % 8 || (g.epi == EPI_F32 ? g.ldc : g.ldz) % 16 || (g.epi != EPI_F32 && g.ldh % 16))
        return cudaErrorInvalidValue;  // TMA row strides and the epilogue's 16-byte stores need these
    const int bn = gemm_bn(g.N);
    // A: M rows x lda (the K tiles' x coordinates stay below K <= lda); B: N rows x ldb.
    const CUtensorMap* ma = operand_map(g.A, g.M, g.lda, TC_BM);
    const CUtensorMap* mb = operand_map(g.B, g.N, g.ldb, bn);
    if (!ma || !mb) return cudaErrorInvalidValue;
    const int nk = std::min(g.k_split, g.K) / TC_BK;
    const int smem = 2048 + std::min(TC_STAGES, std::max(nk, 1)) * (int)gemm_stage_bytes(bn);
    gemm_tc_kernel<<<dim3(g.M / TC_BM, k_splits, g.N / bn), TC_THREADS, smem, s>>>(*ma, *mb, g);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ CUDA-core kernels
struct Box {
    double lo[MLP_IN], hi[MLP_IN];
};

// x0[r][c] = 2 (Lambda[r][c] - lo) / (hi - lo) - 1 for c < P (else 0); rows >= K are zero.
__global__ void normalise_kernel(const double* __restrict__ lam, int64_t K, int P, Box box, bf16* __restrict__ x0,
                                 int64_t rows_pad, uint8_t* __restrict__ outside)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows_pad * MLP_IN_PAD) return;
    const int64_t r = i / MLP_IN_PAD;
    const int c = (int)(i % MLP_IN_PAD);
    float v = 0.0f;
    if (r < K && c < P) v = (float)(2.0 * (lam[r * P + c] - box.lo[c]) / (box.hi[c] - box.lo[c]) - 1.0);
    x0[i] = __float2bfloat16(v);
    if (c == 0 && r < K && outside) {
        uint8_t o = 0;
        for (int p = 0; p < P; ++p) {
            const double x = lam[r * P + p];
            o |= !(x >= box.lo[p] && x <= box.hi[p]);
        }
        outside[r] = o;
    }
}

// Output layer (2 units) on CUDA cores: one warp per row, fixed-order shuffle sum.
__global__ void out_fwd_kernel(const bf16* __restrict__ h4, const float* __restrict__ w4, const float* __restrict__ b4,
                               float* __restrict__ y, int64_t rows)
{
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    float a0 = 0.f, a1 = 0.f;
    for (int i = lane; i < MLP_HID; i += 32) {
        const float h = __bfloat162float(h4[row * MLP_HID + i]);
        a0 = fmaf(h, w4[i], a0);
        a1 = fmaf(h, w4[MLP_HID + i], a1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (lane == 0) {
        y[row * 2] = a0 + b4[0];
        y[row * 2 + 1] = a1 + b4[1];
    }
}

// dY = 2 (Y - T) / B on the first B rows, 0 on the padding; row_loss = sum_o (Y - T)^2.
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t B, int64_t rows_pad,
                                 float* __restrict__ dy, float* __restrict__ row_loss)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows_pad) return;
    float l = 0.f, g0 = 0.f, g1 = 0.f;
    if (r < B) {
        const float r0 = y[r * 2] - t[r * 2], r1 = y[r * 2 + 1] - t[r * 2 + 1];
        l = r0 * r0 + r1 * r1;
        g0 = 2.f * r0 / (float)B;
        g1 = 2.f * r1 / (float)B;
    }
    dy[r * 2] = g0;
    dy[r * 2 + 1] = g1;
    row_loss[r] = l;
}

// dZ4 = (dY W4) * SiLU'(Z4), BF16.
__global__ void out_bwd_kernel(const float* __restrict__ dy, const float* __restrict__ w4, const float* __restrict__ z4,
                               bf16* __restrict__ dz4, int64_t rows_pad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows_pad * MLP_HID) return;
    const int64_t r = i / MLP_HID;
    const int c = (int)(i % MLP_HID);
    const float dh = dy[r * 2] * w4[c] + dy[r * 2 + 1] * w4[MLP_HID + c];
    dz4[i] = __float2bfloat16(dh * dsiluf_(z4[i]));
}

// Column reductions over the batch, in two passes with a fixed order: RED_SLICES row slices
// each give a partial (8 warps over the slice's rows, then the warps in order), and a second
// pass adds the slices in order.  512 blocks instead of 8 keep the SMs busy.
constexpr int RED_SLICES = 64;
constexpr int RED_COLS = 2 * MLP_HID + 2;  // widest partial row: dW4 (2 x 256) and db4 (2)

// part[slice][c] = sum over the slice's rows of X[r][c].
template <class T>
__global__ void colsum_part_kernel(const T* __restrict__ x, int64_t rows, int cols, float* __restrict__ part)
{
    __shared__ float sp[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const int64_t per = (rows + RED_SLICES - 1) / RED_SLICES;
    const int64_t r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
    float s = 0.f;
    if (c < cols)
        for (int64_t r = r0 + w; r < r1; r += 8) s += (float)x[r * cols + c];
    sp[w][lane] = s;
    __syncthreads();
    if (w == 0 && c < cols) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += sp[i][lane];
        part[(int64_t)blockIdx.y * RED_COLS + c] = t;
    }
}

// part[slice][o * 256 + c] = sum over the slice of dY[r][o] H4[r][c]; part[slice][512 + o] = sum dY[r][o].
__global__ void out_wgrad_part_kernel(const float* __restrict__ dy, const bf16* __restrict__ h4, int64_t rows,
                                      float* __restrict__ part)
{
    __shared__ float sp[4][8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const int64_t per = (rows + RED_SLICES - 1) / RED_SLICES;
    const int64_t r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
    float s0 = 0.f, s1 = 0.f, b0 = 0.f, b1 = 0.f;
    for (int64_t r = r0 + w; r < r1; r += 8) {
        const float h = __bfloat162float(h4[r * MLP_HID + c]);
        s0 = fmaf(dy[r * 2], h, s0);
        s1 = fmaf(dy[r * 2 + 1], h, s1);
        b0 += dy[r * 2];
        b1 += dy[r * 2 + 1];
    }
    sp[0][w][lane] = s0;
    sp[1][w][lane] = s1;
    sp[2][w][lane] = b0;
    sp[3][w][lane] = b1;
    __syncthreads();
    if (w == 0) {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        for (int i = 0; i < 8; ++i)
            for (int q = 0; q < 4; ++q) t[q] += sp[q][i][lane];
        float* pr = part + (int64_t)blockIdx.y * RED_COLS;
        pr[c] = t[0];
        pr[MLP_HID + c] = t[1];
        if (blockIdx.x == 0 && lane == 0) {
            pr[2 * MLP_HID] = t[2];
            pr[2 * MLP_HID + 1] = t[3];
        }
    }
}

// out[c] = sum over the slices, in order, of part[slice][c], for c < cols.
__global__ void slices_sum_kernel(const float* __restrict__ part, int cols, float* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float t = 0.f;
    for (int s = 0; s < RED_SLICES; ++s) t += part[(int64_t)s * RED_COLS + c];
    out[c] = t;
}

// out[C x R] = in[R x C]^T (BF16), 32 x 32 tiles.
__global__ void transpose_kernel(const bf16* __restrict__ in, int64_t R, int C, bf16* __restrict__ out)
{
    __shared__ bf16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[i][threadIdx.x] = in[r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[c * R + r] = tile[threadIdx.x][i];
    }
}

// out[i] = sum_s parts[s][i] in order; the first `cols` of every row of width `ld` are kept
// (out has row width `cols`).
__global__ void splitk_reduce_kernel(const float* __restrict__ parts, int S, int64_t stride, int rows, int ld,
                                     int cols, float* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const int64_t r = i / cols, c = i % cols;
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += parts[k * stride + r * ld + c];
    out[i] = s;
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                            float bc1, float bc2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// BF16 GEMM copies of the FP32 master weights: w0p [256 x 64] (zero-padded), w[l] [256 x 256],
// wt[l] = w[l]^T, w4f = BF16-rounded W4 as FP32.
__global__ void refresh_kernel(const float* __restrict__ p, bf16* __restrict__ w0p, bf16* __restrict__ w1,
                               bf16* __restrict__ w2, bf16* __restrict__ w3, bf16* __restrict__ wt1,
                               bf16* __restrict__ wt2, bf16* __restrict__ wt3, float* __restrict__ w4f)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nh = (int64_t)MLP_HID * MLP_HID;
    if (i < (int64_t)MLP_HID * MLP_IN_PAD) {
        const int64_t r = i / MLP_IN_PAD, c = i % MLP_IN_PAD;
        w0p[i] = __float2bfloat16(c < MLP_IN ? p[off_w(0) + r * MLP_IN + c] : 0.0f);
    }
    if (i < nh) {
        const int64_t r = i / MLP_HID, c = i % MLP_HID;
        bf16* ws[3] = {w1, w2, w3};
        bf16* wts[3] = {wt1, wt2, wt3};
        for (int l = 0; l < 3; ++l) {
            const bf16 v = __float2bfloat16(p[off_w(l + 1) + i]);
            ws[l][i] = v;
            wts[l][c * MLP_HID + r] = v;
        }
    }
    if (i < (int64_t)MLP_OUT * MLP_HID) w4f[i] = __bfloat162float(__float2bfloat16(p[off_w(4) + i]));
}

__global__ void gather_rows_kernel(const bf16* __restrict__ xall, const float* __restrict__ tall,
                                   const int64_t* __restrict__ idx, int64_t B, int64_t rows_pad, bf16* __restrict__ x0,
                                   float* __restrict__ t)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows_pad * MLP_IN_PAD) return;
    const int64_t r = i / MLP_IN_PAD, c = i % MLP_IN_PAD;
    const bool live = r < B;
    const int64_t src = live ? idx[r] : 0;
    x0[i] = live ? xall[src * MLP_IN_PAD + c] : __float2bfloat16(0.0f);
    if (c < 2) t[r * 2 + c] = live ? tall[src * 2 + c] : 0.0f;
}

unsigned grid1(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int Surrogate::enqueue_gate(const double* d_lambda, int64_t k_cap, int P, const int64_t* dK, double n_events,
                            uint8_t* need, double* lnxi, double* lnneff)
{
    const int64_t rp = (k_cap + TC_BM - 1) / TC_BM * TC_BM;
    if (rp > cap || (int64_t)outside.bytes < k_cap) {
        err = "surrogate buffers not sized for the batch";
        return POP_ESTATE;
    }
    // normalise -> network -> gate in one launch (pop_mlp_fused.cu)
    return fused_forward(d_lambda, P, nullptr, k_cap, dK, nullptr, outside.as<uint8_t>(), n_events, need, lnxi,
                         lnneff);
}

int Surrogate::ensure_gate(int64_t k_cap)
{
    int rc = ensure_rows(k_cap);
    if (rc != POP_OK) return rc;
    if ((int64_t)outside.bytes < k_cap) {
        const cudaError_t e = outside.alloc((size_t)k_cap);
        if (e != cudaSuccess) {
            err = cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? POP_ENOMEM : POP_ECUDA;
        }
    }
    return POP_OK;
}

// ================================================================== Surrogate
#define SK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                             \
            return e_ == cudaErrorMemoryAllocation ? POP_ENOMEM : POP_ECUDA;                      \
        }                                                                                         \
    } while (0)

int Surrogate::init(int dev, cudaStream_t s)
{
    device = dev;
    stream = s;
    SK(set_gemm_attributes());
    SK(params.alloc(sizeof(float) * MLP_N_PARAMS));
    SK(adam_m.alloc(sizeof(float) * MLP_N_PARAMS));
    SK(adam_v.alloc(sizeof(float) * MLP_N_PARAMS));
    SK(grads.alloc(sizeof(float) * MLP_N_PARAMS));
    SK(w0p.alloc(sizeof(bf16) * MLP_HID * MLP_IN_PAD));
    for (int l = 0; l < 3; ++l) {
        SK(w[l].alloc(sizeof(bf16) * MLP_HID * MLP_HID));
        SK(wt[l].alloc(sizeof(bf16) * MLP_HID * MLP_HID));
    }
    SK(w4f.alloc(sizeof(float) * MLP_OUT * MLP_HID));
    SK(err_flag.alloc(sizeof(int)));
    SK(cudaMemsetAsync(err_flag.p, 0, sizeof(int), stream));
    SK(dw0.alloc(sizeof(float) * MLP_HID * MLP_IN_PAD));
    SK(red.alloc(sizeof(float) * RED_SLICES * RED_COLS));
    return prepare_fused();
}

int Surrogate::ensure_rows(int64_t rows)
{
    rows = (rows + TC_BM - 1) / TC_BM * TC_BM;
    if (rows <= cap) return POP_OK;
    SK(x0.alloc(sizeof(bf16) * rows * MLP_IN_PAD));
    for (int l = 0; l < 4; ++l) {
        SK(z[l].alloc(sizeof(float) * rows * MLP_HID));
        SK(h[l].alloc(sizeof(bf16) * rows * MLP_HID));
    }
    SK(y.alloc(sizeof(float) * rows * 2));
    SK(dy.alloc(sizeof(float) * rows * 2 + sizeof(float) * rows));  // dY, then per-row loss
    SK(dz[0].alloc(sizeof(bf16) * rows * MLP_HID));
    SK(dz[1].alloc(sizeof(bf16) * rows * MLP_HID));
    SK(dzt.alloc(sizeof(bf16) * rows * MLP_HID));
    SK(ht.alloc(sizeof(bf16) * rows * MLP_HID));
    const int64_t splits = std::max<int64_t>(1, rows / 512);
    SK(parts.alloc(sizeof(float) * splits * MLP_HID * MLP_HID));
    cap = rows;
    return POP_OK;
}

int Surrogate::refresh_bf16()
{
    refresh_kernel<<<grid1((int64_t)MLP_HID * MLP_HID, 256), 256, 0, stream>>>(
        params.as<float>(), w0p.as<bf16>(), w[0].as<bf16>(), w[1].as<bf16>(), w[2].as<bf16>(), wt[0].as<bf16>(),
        wt[1].as<bf16>(), wt[2].as<bf16>(), w4f.as<float>());
    SK(cudaGetLastError());
    return POP_OK;
}

int Surrogate::set_params_host(const float* flat)
{
    SK(cudaMemcpyAsync(params.p, flat, sizeof(float) * MLP_N_PARAMS, cudaMemcpyHostToDevice, stream));
    SK(cudaMemsetAsync(adam_m.p, 0, sizeof(float) * MLP_N_PARAMS, stream));
    SK(cudaMemsetAsync(adam_v.p, 0, sizeof(float) * MLP_N_PARAMS, stream));
    adam_step = 0;
    has_params = true;
    return refresh_bf16();
}

int Surrogate::get_params_host(float* flat)
{
    SK(cudaMemcpyAsync(flat, params.p, sizeof(float) * MLP_N_PARAMS, cudaMemcpyDeviceToHost, stream));
    SK(cudaStreamSynchronize(stream));
    return POP_OK;
}

int Surrogate::init_params(uint64_t seed)
{
    // Uniform(-sqrt(3/fan_in), sqrt(3/fan_in)) weights (unit-variance pre-activations), zero biases.
    std::vector<float> p(MLP_N_PARAMS, 0.0f);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    const int fan_in[MLP_LAYERS] = {MLP_IN, MLP_HID, MLP_HID, MLP_HID, MLP_HID};
    const int fan_out[MLP_LAYERS] = {MLP_HID, MLP_HID, MLP_HID, MLP_HID, MLP_OUT};
    for (int l = 0; l < MLP_LAYERS; ++l) {
        const double a = std::sqrt(3.0 / fan_in[l]);
        for (int64_t i = 0; i < (int64_t)fan_in[l] * fan_out[l]; ++i) p[off_w(l) + i] = (float)(a * u(rng));
    }
    return set_params_host(p.data());
}

int Surrogate::forward(int64_t rows_pad)
{
    GemmArgs g{};
    g.err = err_flag.as<int>();
    const bf16* in = x0.as<bf16>();
    int ld_in = MLP_IN_PAD;
    const bf16* ws[4] = {w0p.as<bf16>(), w[0].as<bf16>(), w[1].as<bf16>(), w[2].as<bf16>()};
    for (int l = 0; l < 4; ++l) {
        g.A = in;
        g.lda = ld_in;
        g.B = ws[l];
        g.ldb = l == 0 ? MLP_IN_PAD : MLP_HID;
        g.M = (int)rows_pad;
        g.N = MLP_HID;
        g.K = l == 0 ? MLP_IN_PAD : MLP_HID;
        g.k_split = g.K;
        g.epi = EPI_FWD;
        g.bias = params.as<float>() + off_b(l);
        g.Z = z[l].as<float>();
        g.ldz = MLP_HID;
        g.H = h[l].as<bf16>();
        g.ldh = MLP_HID;
        SK(launch_gemm(g, 1, stream));
        in = h[l].as<bf16>();
        ld_in = MLP_HID;
    }
    out_fwd_kernel<<<grid1(rows_pad * 32, 256), 256, 0, stream>>>(h[3].as<bf16>(), w4f.as<float>(),
                                                                  params.as<float>() + off_b(4), y.as<float>(),
                                                                  rows_pad);
    SK(cudaGetLastError());
    return POP_OK;
}

int Surrogate::backward(int64_t rows, int64_t rows_pad, const float* t)
{
    float* gr = grads.as<float>();
    float* dyp = dy.as<float>();
    float* row_loss = dyp + rows_pad * 2;
    loss_grad_kernel<<<grid1(rows_pad, 256), 256, 0, stream>>>(y.as<float>(), t, rows, rows_pad, dyp, row_loss);
    out_wgrad_part_kernel<<<dim3(MLP_HID / 32, RED_SLICES), 256, 0, stream>>>(dyp, h[3].as<bf16>(), rows_pad,
                                                                             red.as<float>());
    // off_w(4) .. off_b(4) + 2 is one contiguous run: dW4 (2 x 256) then db4 (2)
    slices_sum_kernel<<<grid1(RED_COLS, 256), 256, 0, stream>>>(red.as<float>(), RED_COLS, gr + off_w(4));
    out_bwd_kernel<<<grid1(rows_pad * MLP_HID, 256), 256, 0, stream>>>(dyp, w4f.as<float>(), z[3].as<float>(),
                                                                        dz[0].as<bf16>(), rows_pad);
    SK(cudaGetLastError());
    // Split-K over the batch for the weight gradients: stages of 64 rows, about 512 rows per CTA.
    const int64_t want = std::max<int64_t>(1, rows_pad / 512);
    const int k_split = (int)(((rows_pad + want - 1) / want + TC_BK - 1) / TC_BK * TC_BK);
    const int splits = (int)((rows_pad + k_split - 1) / k_split);
    int cur = 0;
    for (int l = 3; l >= 0; --l) {
        const bf16* dzc = dz[cur].as<bf16>();
        const int in_w = l == 0 ? MLP_IN_PAD : MLP_HID;
        const bf16* hin = l == 0 ? x0.as<bf16>() : h[l - 1].as<bf16>();
        transpose_kernel<<<dim3(MLP_HID / 32, (unsigned)(rows_pad / 32)), dim3(32, 8), 0, stream>>>(
            dzc, rows_pad, MLP_HID, dzt.as<bf16>());
        transpose_kernel<<<dim3(in_w / 32, (unsigned)(rows_pad / 32)), dim3(32, 8), 0, stream>>>(
            hin, rows_pad, in_w, ht.as<bf16>());
        SK(cudaGetLastError());
        // dW_l = dZ^T H: M = 256 outputs, N = layer inputs, K = batch rows (split-K partials).
        GemmArgs g{};
        g.err = err_flag.as<int>();
        g.A = dzt.as<bf16>();
        g.lda = (int)rows_pad;
        g.B = ht.as<bf16>();
        g.ldb = (int)rows_pad;
        g.M = MLP_HID;
        g.N = in_w;
        g.K = (int)rows_pad;
        g.k_split = k_split;
        g.epi = EPI_F32;
        g.C = parts.as<float>();
        g.ldc = in_w;
        g.c_split_stride = (int64_t)MLP_HID * in_w;
        SK(launch_gemm(g, splits, stream));
        float* dwl = l == 0 ? dw0.as<float>() : gr + off_w(l);
        splitk_reduce_kernel<<<grid1((int64_t)MLP_HID * in_w, 256), 256, 0, stream>>>(
            parts.as<float>(), splits, (int64_t)MLP_HID * in_w, MLP_HID, in_w, in_w, dwl);
        if (l == 0)  // keep the 12 real input columns of the padded input layer
            splitk_reduce_kernel<<<grid1((int64_t)MLP_HID * MLP_IN, 256), 256, 0, stream>>>(
                dw0.as<float>(), 1, 0, MLP_HID, MLP_IN_PAD, MLP_IN, gr + off_w(0));
        colsum_part_kernel<bf16><<<dim3(MLP_HID / 32, RED_SLICES), 256, 0, stream>>>(dzc, rows_pad, MLP_HID,
                                                                                   red.as<float>());
        slices_sum_kernel<<<grid1(MLP_HID, 256), 256, 0, stream>>>(red.as<float>(), MLP_HID, gr + off_b(l));
        SK(cudaGetLastError());
        if (l > 0) {  // dZ_l = (dZ_{l+1} W_l) * SiLU'(Z_l)
            GemmArgs b{};
            b.err = err_flag.as<int>();
            b.A = dzc;
            b.lda = MLP_HID;
            b.B = wt[l - 1].as<bf16>();
            b.ldb = MLP_HID;
            b.M = (int)rows_pad;
            b.N = MLP_HID;
            b.K = MLP_HID;
            b.k_split = MLP_HID;
            b.epi = EPI_BWD;
            b.Z = z[l - 1].as<float>();
            b.ldz = MLP_HID;
            b.H = dz[cur ^ 1].as<bf16>();
            b.ldh = MLP_HID;
            SK(launch_gemm(b, 1, stream));
            cur ^= 1;
        }
    }
    return POP_OK;
}

int Surrogate::adam(float lr)
{
    ++adam_step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)adam_step));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)adam_step));
    adam_kernel<<<grid1(MLP_N_PARAMS, 256), 256, 0, stream>>>(params.as<float>(), adam_m.as<float>(),
                                                             adam_v.as<float>(), grads.as<float>(), MLP_N_PARAMS, lr,
                                                             b1, b2, 1e-8f, bc1, bc2);
    SK(cudaGetLastError());
    return refresh_bf16();
}

int Surrogate::check_error()
{
    int h = 0;
    SK(cudaMemcpyAsync(&h, err_flag.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
    SK(cudaStreamSynchronize(stream));
    if (h) {
        err = "a tensor-core wait timed out";
        cudaMemsetAsync(err_flag.p, 0, sizeof(int), stream);
        return POP_ETIMEOUT;
    }
    return POP_OK;
}

int Surrogate::normalise(const double* lambda, int64_t K, int P, uint8_t* outside, __nv_bfloat16* dst)
{
    const int64_t rows_pad = (K + TC_BM - 1) / TC_BM * TC_BM;
    Box box;
    for (int i = 0; i < MLP_IN; ++i) {
        box.lo[i] = lo[i];
        box.hi[i] = hi[i];
    }
    normalise_kernel<<<grid1(rows_pad * MLP_IN_PAD, 256), 256, 0, stream>>>(lambda, K, P, box,
                                                                           dst ? dst : x0.as<bf16>(), rows_pad,
                                                                           outside);
    SK(cudaGetLastError());
    return POP_OK;
}

cudaError_t mlp_gemm_check(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K, int* err,
                           cudaStream_t s)
{
    cudaError_t e = set_gemm_attributes();
    if (e != cudaSuccess) return e;
    GemmArgs g{};
    g.A = A;
    g.lda = K;
    g.B = B;
    g.ldb = K;
    g.M = M;
    g.N = N;
    g.K = K;
    g.k_split = K;
    g.epi = EPI_F32;
    g.C = C;
    g.ldc = N;
    g.err = err;
    return launch_gemm(g, 1, s);
}

// Training-data gather (used by the training loop in pop_api.cu).
cudaError_t mlp_gather(const __nv_bfloat16* xall, const float* tall, const int64_t* idx, int64_t B, int64_t rows_pad,
                       __nv_bfloat16* x0, float* t, cudaStream_t s)
{
    gather_rows_kernel<<<grid1(rows_pad * MLP_IN_PAD, 256), 256, 0, s>>>(xall, tall, idx, B, rows_pad, x0, t);
    return cudaGetLastError();
}

}  // namespace pop
