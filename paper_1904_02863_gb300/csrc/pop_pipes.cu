// Per-SM pipe throughput of the operations the kernels are bound by: FP64 FMA (the FP64
// weight, gradient and grid kernels), FP32 FMA scalar and packed (the float-float kernel, the
// FP32 grid and CBC sums), the MUFU ex2 and rcp of the FP32 weight, and 16-byte shared-memory
// loads (the FP32 grid contraction's operand path).  Their rooflines need these rates, and the
// GPU's data sheet gives none of the MUFU or shared-load ones.
//
// One CTA of 1024 threads per SM (the dynamic shared memory request leaves room for one), each
// thread running 8 independent dependency chains of the operation, so that 32 warps x 8 chains
// cover the pipe's latency.  The chains depend on a clock read at the start and end in a shared
// store before a block barrier, after which thread 0 reads the clock again; the rate is thread
// operations per SM clock, 1024 x 8 x iters / cycles, one value per CTA (thread 0's start read
// is within one warp scheduling step of the others').
#include <algorithm>
#include <vector>

#include "pop.h"
#include "pop_internal.h"

namespace pop {

namespace {

constexpr int PIPE_THREADS = 1024;
constexpr int PIPE_CHAINS = 8;
constexpr int PIPE_SMEM = 120 * 1024;  // more than half an SM's shared memory: one CTA per SM

__device__ __forceinline__ float mufu_ex2(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_rcp(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// OP: 0 DFMA, 1 FFMA, 2 MUFU ex2, 3 MUFU rcp, 4 fma.rn.f32x2, 5 and 6 16-byte shared loads with
// 32 and 4 distinct addresses per warp.  Values stay finite and away from denormals:
// x <- 0.999 x + 1e-3 converges to 1; x <- 2^-x stays in (0, 1]; x <- 1/(x + 1) converges to 0.618.
template <int OP>
__global__ void __launch_bounds__(PIPE_THREADS) pipe_rate_kernel(int iters, float* __restrict__ sink,
                                                                 long long* __restrict__ cycles)
{
    extern __shared__ float pad[];  // one CTA per SM; also receives each thread's results
    double d[PIPE_CHAINS];
    float f[PIPE_CHAINS];
    unsigned long long p2[PIPE_CHAINS];  // packed FP32 pairs
    if (OP >= 5)
        for (int i = threadIdx.x; i < PIPE_SMEM / 4; i += PIPE_THREADS) pad[i] = 1e-3f * (float)(i & 63);
    __syncthreads();
    // The chains start from the clock value (its top bits are 0, which the compiler cannot know),
    // so no operation of them can be scheduled before this read.
    const long long t0 = clock64();
    const int z = (int)(t0 >> 62);
#pragma unroll
    for (int j = 0; j < PIPE_CHAINS; ++j) {
        d[j] = 0.5 + 1e-3 * (threadIdx.x + j + z);
        f[j] = 0.5f + 1e-3f * (float)((threadIdx.x + j + z) & 255);
        asm("mov.b64 %0, {%1, %2};" : "=l"(p2[j]) : "f"(f[j]), "f"(0.25f));
    }
    // Shared loads: word offsets of a warp's lanes (a multiple of 4: 16-byte aligned), 32 distinct
    // 16-byte words or 4 (lanes 8m .. 8m + 7 share one).
    const int lane = threadIdx.x & 31;
    const int off = (OP == 6 ? (lane >> 3) : lane) * 4 + (z << 2);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PIPE_CHAINS; ++j) {
            if (OP == 0) d[j] = fma(d[j], 0.999, 1e-3);
            if (OP == 1) f[j] = fmaf(f[j], 0.999f, 1e-3f);
            if (OP == 2) f[j] = mufu_ex2(-f[j]);
            if (OP == 3) f[j] = mufu_rcp(f[j] + 1.0f);  // not x <- 1/x, whose pairs the compiler folds
            if (OP == 4)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;"
                             : "+l"(p2[j])
                             : "l"(0x3f7fbe773f7fbe77ull), "l"(0x3a83126f3a83126full));  // (0.999, 0.999), (1e-3, 1e-3)
            if (OP >= 5) {
                const float4 v = *reinterpret_cast<const float4*>(pad + ((off + 128 * j + 16 * (i & 7)) & 4095));
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
        }
    }
    // The chains end in a shared-memory store before the barrier, and the closing clock read
    // follows the barrier, so every operation lies between the two reads.
    float s = acc.x + acc.y + acc.z + acc.w;
#pragma unroll
    for (int j = 0; j < PIPE_CHAINS; ++j) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p2[j]));
        s += f[j] + (float)d[j] + lo + hi;
    }
    __syncthreads();  // every shared load of the chains is done
    pad[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        cycles[blockIdx.x] = clock64() - t0;
        sink[blockIdx.x] = pad[(t0 & 1) ? 1 : 0];  // keeps the stores live
    }
}

}  // namespace

}  // namespace pop

using namespace pop;

namespace {

constexpr int N_RATES = 7;

int pipe_rates_on_current_device(double* rates, int n_rates)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POP_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return POP_ECUDA;
    const void* fns[N_RATES] = {(const void*)pipe_rate_kernel<0>, (const void*)pipe_rate_kernel<1>,
                                (const void*)pipe_rate_kernel<2>, (const void*)pipe_rate_kernel<3>,
                                (const void*)pipe_rate_kernel<4>, (const void*)pipe_rate_kernel<5>,
                                (const void*)pipe_rate_kernel<6>};
    // Iterations for about half a million cycles at the expected rates (2, 128, 32, 16, 128 per SM
    // clock; about 1/4 and 1/2 of a warp instruction per SM clock for the shared loads).
    const int iters[N_RATES] = {128, 8192, 2048, 1024, 4096, 2048, 2048};
    // Each chain step is one thread operation, except the packed FMA (two lanes) and the shared
    // loads (counted per warp instruction).
    const double per_step[N_RATES] = {1.0, 1.0, 1.0, 1.0, 2.0, 1.0 / 32.0, 1.0 / 32.0};
    n_rates = std::min(n_rates, N_RATES);
    for (int k = 0; k < n_rates; ++k)
        if (cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, PIPE_SMEM) != cudaSuccess)
            return POP_ECUDA;
    float* sink = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * sms) != cudaSuccess) return POP_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess) {
        cudaFree(sink);
        return POP_ENOMEM;
    }
    int rc = POP_OK;
    std::vector<long long> h(sms);
    for (int k = 0; k < n_rates && rc == POP_OK; ++k) {
        for (int rep = 0; rep < 2 && rc == POP_OK; ++rep) {  // the first launch warms up; the second is kept
            void* args[] = {(void*)&iters[k], (void*)&sink, (void*)&cyc};
            if (cudaLaunchKernel(fns[k], dim3(sms), dim3(PIPE_THREADS), args, PIPE_SMEM, 0) != cudaSuccess ||
                cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = POP_ECUDA;
        }
        if (rc != POP_OK) break;
        std::sort(h.begin(), h.end());
        const double med = (double)h[sms / 2];
        rates[k] = med > 0 ? (double)PIPE_THREADS * PIPE_CHAINS * iters[k] * per_step[k] / med : 0.0;
    }
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}

}  // namespace

extern "C" int pop_pipe_rates_n(int device, double* rates, int n_rates)
{
    if (!rates || device < 0 || n_rates < 1) return POP_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return POP_ECUDA;
    const int rc = pipe_rates_on_current_device(rates, n_rates);
    cudaSetDevice(prev);
    return rc;
}

extern "C" int pop_pipe_rates(int device, double* rates) { return pop_pipe_rates_n(device, rates, 4); }
