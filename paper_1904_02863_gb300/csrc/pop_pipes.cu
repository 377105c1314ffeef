// Per-SM pipe throughput of the operations the weight kernels are bound by: FP64 FMA (the FP64
// weight, gradient and grid kernels), FP32 FMA (the float-float kernel), and the MUFU ex2 and rcp
// of the FP32 weight.  Their rooflines need these rates, and the GPU's data sheet gives none of
// the MUFU ones.
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

// OP: 0 DFMA, 1 FFMA, 2 MUFU ex2, 3 MUFU rcp.  Values stay finite and away from denormals:
// x <- 0.999 x + 1e-3 converges to 1; x <- 2^-x stays in (0, 1]; x <- 1/(x + 1) converges to 0.618.
template <int OP>
__global__ void __launch_bounds__(PIPE_THREADS) pipe_rate_kernel(int iters, float* __restrict__ sink,
                                                                 long long* __restrict__ cycles)
{
    extern __shared__ float pad[];  // one CTA per SM; also receives each thread's results
    double d[PIPE_CHAINS];
    float f[PIPE_CHAINS];
    __syncthreads();
    // The chains start from the clock value (its top bits are 0, which the compiler cannot know),
    // so no operation of them can be scheduled before this read.
    const long long t0 = clock64();
    const int z = (int)(t0 >> 62);
#pragma unroll
    for (int j = 0; j < PIPE_CHAINS; ++j) {
        d[j] = 0.5 + 1e-3 * (threadIdx.x + j + z);
        f[j] = 0.5f + 1e-3f * (float)((threadIdx.x + j + z) & 255);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PIPE_CHAINS; ++j) {
            if (OP == 0) d[j] = fma(d[j], 0.999, 1e-3);
            if (OP == 1) f[j] = fmaf(f[j], 0.999f, 1e-3f);
            if (OP == 2) f[j] = mufu_ex2(-f[j]);
            if (OP == 3) f[j] = mufu_rcp(f[j] + 1.0f);  // not x <- 1/x, whose pairs the compiler folds
        }
    }
    // The chains end in a shared-memory store before the barrier, and the closing clock read
    // follows the barrier, so every operation lies between the two reads.
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < PIPE_CHAINS; ++j) s += f[j] + (float)d[j];
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

int pipe_rates_on_current_device(double* rates)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POP_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return POP_ECUDA;
    const void* fns[4] = {(const void*)pipe_rate_kernel<0>, (const void*)pipe_rate_kernel<1>,
                          (const void*)pipe_rate_kernel<2>, (const void*)pipe_rate_kernel<3>};
    // Iterations for about half a million cycles at the expected rates (2, 128, 32, 16 per SM clock).
    const int iters[4] = {128, 8192, 2048, 1024};
    for (int k = 0; k < 4; ++k)
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
    for (int k = 0; k < 4 && rc == POP_OK; ++k) {
        for (int rep = 0; rep < 2 && rc == POP_OK; ++rep) {  // the first launch warms up; the second is kept
            void* args[] = {(void*)&iters[k], (void*)&sink, (void*)&cyc};
            if (cudaLaunchKernel(fns[k], dim3(sms), dim3(PIPE_THREADS), args, PIPE_SMEM, 0) != cudaSuccess ||
                cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = POP_ECUDA;
        }
        if (rc != POP_OK) break;
        std::sort(h.begin(), h.end());
        const double med = (double)h[sms / 2];
        rates[k] = med > 0 ? (double)PIPE_THREADS * PIPE_CHAINS * iters[k] / med : 0.0;
    }
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}

}  // namespace

extern "C" int pop_pipe_rates(int device, double* rates)
{
    if (!rates || device < 0) return POP_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return POP_ECUDA;
    const int rc = pipe_rates_on_current_device(rates);
    cudaSetDevice(prev);
    return rc;
}
