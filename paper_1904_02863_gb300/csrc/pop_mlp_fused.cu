// The surrogate network's inference forward in one launch.
//
// One CTA of 512 threads takes 128 rows (TMEM lanes) through normalise -> 4 x (256-wide
// tcgen05 GEMM + bias + SiLU) -> the 2-unit output layer -> the per-Lambda gate, without
// leaving the SM:
//   * the activations stay in shared memory as the A operand of the next layer: 4 chunks
//     of 128 rows x 64 K (BF16), each in the 128-byte swizzle layout (rows 128 bytes
//     apart, the 16-byte units of row r XOR-permuted by r mod 8);
//   * the weights come in 13 tiles of 256 rows x 64 K (one for the input layer, four for
//     each hidden layer) by 2-D TMA loads (cp.async.bulk.tensor, the same swizzle) into a
//     3-slot ring of mbarriers, so the copies of the next tiles run under the MMAs;
//   * one thread issues the four K = 16 MMAs of a tile into the 128 x 256 FP32
//     accumulator in TMEM and commits them to the tile slot's barrier; the slot of the
//     previous tile is refilled as soon as its MMAs are done;
//   * after a layer's last MMA, warp w reads rows 32 (w mod 4) .. +31 (the lanes its
//     position in the warpgroup may access) and columns 64 (w / 4) .. +63 of the
//     accumulator (tcgen05.ld), adds the bias, applies SiLU, rounds to BF16 and writes its
//     part of the next layer's operand; after the last hidden layer the 16 warps form the
//     two outputs from partial sums that are added in a fixed order.  Sixteen warps, not
//     four, hide the latencies of this epilogue, which is most of the kernel's work.
// Every wait has an iteration limit; a CTA that gives up sets the error flag, marks its
// rows as needing the Monte Carlo selection term, waits (again with a limit) for the copies
// and MMAs it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include "pop_internal.h"
#include "pop_mlp.h"
#include "pop_tc.cuh"

namespace pop {

namespace {

using bf16 = __nv_bfloat16;
using namespace tc;

constexpr int FR = 128;                             // rows per CTA = TMEM lanes
constexpr int FT = 512;                             // threads: 4 lane quarters x 4 column groups
constexpr int KC = 64;                              // K per tile: one 128-byte swizzle row of BF16
constexpr uint32_t ACT_CHUNK = FR * KC * 2;         // 16 KB
constexpr uint32_t W_TILE = MLP_HID * KC * 2;       // 32 KB
constexpr int NSTAGE = 3;                           // weight ring slots
constexpr int N_TILES = 1 + 3 * (MLP_HID / KC);     // 13
constexpr uint32_t OFF_ACT = 0;
constexpr uint32_t OFF_W = 4 * ACT_CHUNK;           // 64 KB
constexpr uint32_t OFF_BAR = OFF_W + NSTAGE * W_TILE;
constexpr uint32_t OFF_BIAS = OFF_BAR + 128;                 // 4 x 256 biases, then W4 (2 x 256), FP32
constexpr uint32_t OFF_RED = OFF_BIAS + (4 + 2) * MLP_HID * 4;  // output partials [4 groups][128 rows][2]
constexpr uint32_t SMEM_USED = OFF_RED + 4 * FR * 2 * 4;
constexpr uint32_t SMEM_LAUNCH = SMEM_USED + 1024;  // room to align the base to 1024 bytes

struct FusedArgs {
    const double* lambda;    // [rows x P] (NULL when x0 is given)
    int P;
    const bf16* x0;          // [rows x 64] normalised inputs, or NULL
    int64_t K_cap;
    const int64_t* dK;       // rows to compute (device), or NULL for K_cap
    double lo[MLP_IN], hi[MLP_IN];
    const float* bias[4];    // hidden-layer biases
    const float* w4f;        // [2 x 256] output weights (BF16-rounded, as FP32)
    const float* b4;         // [2]
    float* y;                // [rows x 2] standardised outputs, or NULL
    uint8_t* outside;        // [rows] Lambda outside the training box, or NULL
    uint8_t* need;           // gate outputs, or NULL
    double* lnxi;
    double* lnneff;
    double mu0, sd0, mu1, sd1, n_events, budget;
    int trusted;
    ErrTable table;
    int* err;                // set when a wait gives up; read at the start for earlier failures
};

// Tile t of the weight sequence: its layer and its 64-wide K chunk.
__device__ __forceinline__ void tile_of(int t, int& layer, int& kc)
{
    layer = t == 0 ? 0 : 1 + (t - 1) / (MLP_HID / KC);
    kc = t == 0 ? 0 : (t - 1) % (MLP_HID / KC);
}

// SiLU with the hardware exponential and reciprocal (its result is rounded to BF16 next).
__device__ __forceinline__ float silu_(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// Byte offset of 16-byte unit u (columns 8u..8u+7 of a 64-wide chunk) of row r in a
// 128-byte-swizzle chunk.
__device__ __forceinline__ uint32_t sw128(int r, int u) { return (uint32_t)(r * 128 + ((u ^ (r & 7)) << 4)); }

__global__ void __launch_bounds__(FT, 1)
mlp_fused_fwd_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                     const __grid_constant__ CUtensorMap map2, const __grid_constant__ CUtensorMap map3,
                     const __grid_constant__ FusedArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    const int64_t K = a.dK ? *a.dK : a.K_cap;
    const int64_t r0 = (int64_t)blockIdx.x * FR;
    if (r0 >= K) return;  // a CTA wholly past the batch (graph replay with fewer rows)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* g = smem_raw + (base - raw);
    const uint32_t bar_full = base + OFF_BAR;           // NSTAGE barriers: tile landed
    const uint32_t bar_done = bar_full + 8 * NSTAGE;    // NSTAGE barriers: its MMAs finished
    const uint32_t bar_layer = bar_done + 8 * NSTAGE;   // every MMA issued so far finished
    uint32_t* tslot = reinterpret_cast<uint32_t*>(g + OFF_BAR + 64);
    float* sbias = reinterpret_cast<float*>(g + OFF_BIAS);  // [4][256] then W4 [2][256]
    float* sred = reinterpret_cast<float*>(g + OFF_RED);    // [4][128][2]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cgrp = warp >> 2;     // TMEM lanes 32 quarter.., columns 64 cgrp..
    const int r = quarter * 32 + lane;                  // this thread's row in the tile (epilogue)
    const int64_t row = r0 + r;
    const bool live = row < K;
    auto map_of = [&](int layer) { return layer == 0 ? &map0 : layer == 1 ? &map1 : layer == 2 ? &map2 : &map3; };
    const bool earlier_failure = *a.err != 0;

    if (warp == 0) tmem_alloc(smem_u32(tslot), MLP_HID);
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_done + 8 * s, 1);
        }
        mbar_init(bar_layer, 1);
        for (int t = 0; t < NSTAGE; ++t) {
            int layer, kc;
            tile_of(t, layer, kc);
            tma_load_2d(base + OFF_W + t * W_TILE, map_of(layer), kc * KC, 0, bar_full + 8 * t, W_TILE);
        }
    }
    for (int i = tid; i < 4 * MLP_HID; i += FT) sbias[i] = __ldg(a.bias[i / MLP_HID] + i % MLP_HID);
    for (int i = tid; i < 2 * MLP_HID; i += FT) sbias[4 * MLP_HID + i] = __ldg(a.w4f + i);

    // The inputs, normalised to [-1, 1] (or given), into activation chunk 0: thread t writes
    // units 2 (t / 128) and 2 (t / 128) + 1 of row t mod 128.
    {
        const int ir = tid & (FR - 1), part = tid >> 7;
        const int64_t irow = r0 + ir;
        for (int u = 2 * part; u < 2 * part + 2; ++u) {
            __align__(16) bf16 e[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = 8 * u + i;
                float x = 0.0f;
                if (irow < K) {
                    if (a.x0) x = __bfloat162float(a.x0[irow * MLP_IN_PAD + c]);
                    else if (c < a.P)
                        x = (float)(2.0 * (a.lambda[irow * a.P + c] - a.lo[c]) / (a.hi[c] - a.lo[c]) - 1.0);
                }
                e[i] = __float2bfloat16(x);
            }
            *reinterpret_cast<uint4*>(g + OFF_ACT + sw128(ir, u)) = *reinterpret_cast<const uint4*>(e);
        }
    }
    // Outside the training box (threads 0..127, one row each; the same rows as the gate's).
    uint8_t outside = 0;
    if (tid < FR && r0 + tid < K && !a.x0) {
        for (int p = 0; p < a.P; ++p) {
            const double v = a.lambda[(r0 + tid) * a.P + p];
            outside |= !(v >= a.lo[p] && v <= a.hi[p]);
        }
        if (a.outside) a.outside[r0 + tid] = outside;
    }
    fence_proxy_async();  // the generic-proxy stores, visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_bf16(FR, MLP_HID);
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);

    uint32_t full_ph = 0, done_ph = 0, layer_ph = 0;  // phase bits (thread 0 uses the first two)
    int t = 0, issued = NSTAGE;                        // tiles consumed, tiles whose copy was issued
    bool failed = false;
    float y0 = 0.0f, y1 = 0.0f;
    for (int l = 0; l < 4; ++l) {
        const int nk = l == 0 ? 1 : MLP_HID / KC;
        int bad = 0;
        if (tid == 0) {
            for (int j = 0; j < nk; ++j, ++t) {
                const int s = t % NSTAGE;
                if (!mbar_wait(bar_full + 8 * s, (full_ph >> s) & 1u)) {
                    bad = 1;
                    break;
                }
                full_ph ^= 1u << s;
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < KC / 16; ++kk)
                    mma_bf16(tmem, sdesc_sw128(base + OFF_ACT + j * ACT_CHUNK + kk * 32),
                             sdesc_sw128(base + OFF_W + s * W_TILE + kk * 32), idesc, (j > 0 || kk > 0) ? 1u : 0u);
                mma_commit(bar_done + 8 * s);
                // The previous tile's slot takes the tile NSTAGE after it once its MMAs are done.
                if (t >= 1 && t - 1 + NSTAGE < N_TILES) {
                    const int sp = (t - 1) % NSTAGE;
                    if (!mbar_wait(bar_done + 8 * sp, (done_ph >> sp) & 1u)) {
                        ++t;  // tile t was consumed
                        bad = 1;
                        break;
                    }
                    done_ph ^= 1u << sp;
                    int layer, kc;
                    tile_of(t - 1 + NSTAGE, layer, kc);
                    tma_load_2d(base + OFF_W + sp * W_TILE, map_of(layer), kc * KC, 0, bar_full + 8 * sp, W_TILE);
                    ++issued;
                }
            }
            mma_commit(bar_layer);
        }
        if (__syncthreads_or(bad)) {
            failed = true;
            break;
        }
        if (__syncthreads_or(!mbar_wait(bar_layer, layer_ph))) {
            failed = true;
            break;
        }
        layer_ph ^= 1u;
        tc_fence_after();
        const float* bias = sbias + l * MLP_HID;
        unsigned char* chunk = g + OFF_ACT + cgrp * ACT_CHUNK;  // columns 64 cgrp .. of the next operand
#pragma unroll 1
        for (int b = 0; b < KC / 16; ++b) {
            const int c0 = cgrp * KC + 16 * b;
            float v[16];
            tmem_ld16(trow + (uint32_t)c0, v);
            __align__(16) bf16 hb[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) hb[j] = __float2bfloat16(silu_(v[j] + bias[c0 + j]));
            if (l < 3) {
                *reinterpret_cast<uint4*>(chunk + sw128(r, 2 * b)) = reinterpret_cast<const uint4*>(hb)[0];
                *reinterpret_cast<uint4*>(chunk + sw128(r, 2 * b + 1)) = reinterpret_cast<const uint4*>(hb)[1];
            } else {
                const float* w4 = sbias + 4 * MLP_HID;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float h = __bfloat162float(hb[j]);
                    y0 = fmaf(h, w4[c0 + j], y0);
                    y1 = fmaf(h, w4[MLP_HID + c0 + j], y1);
                }
            }
        }
        if (l == 3) {
            sred[(cgrp * FR + r) * 2] = y0;
            sred[(cgrp * FR + r) * 2 + 1] = y1;
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    // Threads 0..127 (column group 0: row = tid) finish their row.
    if (failed) {
        if (tid == 0) {
            atomicExch(a.err, 1);
            // Let the MMAs and copies in flight finish before the TMEM and the shared memory go.
            mma_commit(bar_layer);
            mbar_wait(bar_layer, layer_ph);
            for (int u = t; u < issued; ++u) {
                const int s = u % NSTAGE;
                mbar_wait(bar_full + 8 * s, (full_ph >> s) & 1u);
                full_ph ^= 1u << s;
            }
        }
    } else if (tid < FR && live) {
        // the four column groups' partials, in order
        y0 = __ldg(a.b4);
        y1 = __ldg(a.b4 + 1);
        float p0 = 0.0f, p1 = 0.0f;
        for (int q = 0; q < 4; ++q) {
            p0 += sred[(q * FR + r) * 2];
            p1 += sred[(q * FR + r) * 2 + 1];
        }
        y0 += p0;
        y1 += p1;
        if (a.y) {
            a.y[row * 2] = y0;
            a.y[row * 2 + 1] = y1;
        }
    }
    if (tid < FR && live && a.need) {
        const double lx = (double)y0 * a.sd0 + a.mu0;
        const double ln = (double)y1 * a.sd1 + a.mu1;
        a.lnxi[row] = lx;
        a.lnneff[row] = ln;
        a.need[row] = (uint8_t)need_monte_carlo(a.trusted != 0, outside != 0, failed || earlier_failure, lx, ln,
                                                a.n_events, a.budget, a.table);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, MLP_HID);
}

// cuTensorMapEncodeTiled from the driver (the runtime links statically; the driver has it).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* m, const void* ptr, int rows, int cols) { return make_tile_map(m, ptr, rows, cols, MLP_HID); }

}  // namespace

bool make_tile_map(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc || box_rows < 1 || box_rows > 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int Surrogate::prepare_fused()
{
    // The GEMM copies of the weights never move: the maps are made once, after they are allocated.
    bool ok = make_map(&wmap[0], w0p.p, MLP_HID, MLP_IN_PAD);
    for (int l = 0; l < 3; ++l) ok = ok && make_map(&wmap[l + 1], w[l].p, MLP_HID, MLP_HID);
    if (!ok) {
        err = "cuTensorMapEncodeTiled failed for the network's weights";
        return POP_ECUDA;
    }
    const cudaError_t e =
        cudaFuncSetAttribute(mlp_fused_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LAUNCH);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return POP_ECUDA;
    }
    wmaps_ok = true;
    return POP_OK;
}

int Surrogate::fused_forward(const double* d_lambda, int P, const __nv_bfloat16* x0_in, int64_t K_cap,
                             const int64_t* dK, float* y_out, uint8_t* outside_out, double n_events, uint8_t* need,
                             double* lnxi, double* lnneff)
{
    if (K_cap <= 0) return POP_OK;
    if (!wmaps_ok) {
        err = "the fused forward was not prepared";
        return POP_ESTATE;
    }
    FusedArgs a{};
    a.lambda = d_lambda;
    a.P = P;
    a.x0 = x0_in;
    a.K_cap = K_cap;
    a.dK = dK;
    for (int i = 0; i < MLP_IN; ++i) {
        a.lo[i] = lo[i];
        a.hi[i] = hi[i];
    }
    for (int l = 0; l < 4; ++l) a.bias[l] = params.as<float>() + off_b(l);
    a.w4f = w4f.as<float>();
    a.b4 = params.as<float>() + off_b(4);
    a.y = y_out;
    a.outside = outside_out;
    a.need = need;
    a.lnxi = lnxi;
    a.lnneff = lnneff;
    a.mu0 = mu[0];
    a.sd0 = sd[0];
    a.mu1 = mu[1];
    a.sd1 = sd[1];
    a.n_events = n_events;
    a.budget = budget;
    a.trusted = trusted ? 1 : 0;
    a.table = table;
    a.err = err_flag.as<int>();
    const unsigned grid = (unsigned)((K_cap + FR - 1) / FR);
    mlp_fused_fwd_kernel<<<grid, FT, SMEM_LAUNCH, stream>>>(wmap[0], wmap[1], wmap[2], wmap[3], a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return POP_ECUDA;
    }
    return POP_OK;
}

}  // namespace pop
