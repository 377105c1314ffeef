// pop_loglik_f64_noalloc: ln L without any device allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is entirely
// owned by an outer pool or framework (allocations outside it fail or are
// forbidden), and latency-critical sampler loops that must not allocate or
// free while they run.  They own their inputs and outputs as device buffers
// and call this entry point, which takes no context.  Its scratch (per-Lambda
// constants, per-(Lambda, event) partial sums, the injection sums) lives in
// the file-scope array below, which every GPU that loads libpop.so holds until
// the process exits.  The arithmetic is the FP64 path of pop_loglik; the
// weight kernel here is a variant that reads the raw samples (no packed
// feature arrays, so nothing to allocate) and sums each event in one work item.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include "pop.h"
#include "pop_internal.h"

using namespace pop;

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)POP_NOALLOC_SCRATCH_BYTES;
constexpr int MAX_DEVICES = 64;
constexpr int INJ_CHUNK = 4096;   // injections per work item
constexpr int TILE = 8;           // Lambda points per work item
constexpr int THREADS = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Error text goes to the caller's buffer (msg may be NULL).
struct Msg {
    char* buf;
    int len;
    int operator()(int status, const std::string& m) const
    {
        if (buf && len > 0) snprintf(buf, (size_t)len, "pop_loglik_f64_noalloc: %s", m.c_str());
        return status;
    }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the scratch sections for a problem size.
struct Layout {
    size_t k, bad, c64, c32, zint, ecb, part, part2, total;
};

Layout layout(int64_t n_events, int64_t n_inj_chunks, int64_t K)
{
    Layout L;
    L.k = 0;
    L.bad = 8;
    L.c64 = 256;
    L.c32 = align256(L.c64 + sizeof(LamF64) * (size_t)K);
    L.zint = align256(L.c32 + sizeof(LamF32) * (size_t)K);
    L.ecb = align256(L.zint + sizeof(double) * (size_t)K);
    L.part = align256(L.ecb + sizeof(int32_t) * (size_t)(n_events + 1));
    L.part2 = align256(L.part + sizeof(double) * (size_t)K * (size_t)(n_events + n_inj_chunks));
    L.total = L.part2 + sizeof(double) * (size_t)K * (size_t)n_inj_chunks;
    return L;
}

// Writes K, clears the bad-input count (or sets it to 1 when the CSR offsets do
// not start at 0 or end at n_samples) and lays out one work chunk per event.
__global__ void setup_kernel(int64_t* dK, int64_t K, unsigned long long* bad, int32_t* ecb, int64_t n_events,
                             const int64_t* offsets, int64_t n_samples)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) {
        *dK = K;
        *bad = (offsets[0] != 0 || offsets[n_events] != n_samples) ? 1ull : 0ull;
    }
    if (i <= n_events) ecb[i] = (int32_t)i;  // one work chunk per event
}

// Restores the calling thread's current device on every return path.
struct DeviceGuard {
    int prev = -1;
    DeviceGuard() { (void)cudaGetDevice(&prev); }
    ~DeviceGuard()
    {
        if (prev >= 0) (void)cudaSetDevice(prev);
    }
};

// True when p is device or managed memory of `device` (host, pinned and
// unregistered pointers are refused before any kernel could read them).
bool on_device(const void* p, int device)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}

struct RawSet {
    const double* theta;
    const double* prior;
};

struct Sample {
    double lm1, m1, lq, sa, sb, dc, nlpi, lz1, invm1;
    int64_t m1b, m2b;
};

// Features of one raw sample; returns false for unusable input (non-finite or pi <= 0).
__device__ __forceinline__ bool make_sample(const RawSet& r, int64_t j, int nd, Sample& x)
{
    const double* th = r.theta + j * nd;
    const double m1 = th[0], q = th[1], a1 = th[2], a2 = th[3], c1 = th[4], c2 = th[5];
    const double z = nd == 7 ? th[6] : 1.0;
    const double pi = r.prior[j];
    const bool ok = isfinite(m1) && isfinite(q) && isfinite(a1) && isfinite(a2) && isfinite(c1) && isfinite(c2) &&
                    isfinite(z) && isfinite(pi) && pi > 0.0;
    const bool live = ok && m1 > 0.0 && q > 0.0 && q <= 1.0 && a1 >= 0.0 && a1 <= 1.0 && a2 >= 0.0 && a2 <= 1.0 &&
                      c1 >= -1.0 && c1 <= 1.0 && c2 >= -1.0 && c2 <= 1.0 && z >= 0.0 && z <= 2.0;
    x = Sample{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (live) {
        x.lm1 = log(m1);
        x.m1 = m1;
        x.invm1 = 1.0 / m1;
        x.lq = log(q);
        x.sa = (a1 > 0.0 && a2 > 0.0) ? log(a1) + log(a2) : LOG_ZERO;
        x.sb = (a1 < 1.0 && a2 < 1.0) ? log(1.0 - a1) + log(1.0 - a2) : LOG_ZERO;
        x.dc = (c1 - 1.0) * (c1 - 1.0) + (c2 - 1.0) * (c2 - 1.0);
        x.nlpi = -log(pi);
        if (nd == 7) {
            x.nlpi = z > 0.0 ? x.nlpi + 2.0 * log(z) : LOG_ZERO;
            x.lz1 = log1p(z);
        }
        x.m2b = __double_as_longlong(__dmul_rn(q, m1));
    }
    x.m1b = __double_as_longlong(x.m1);
    return ok;
}

template <bool HAS_Z>
__device__ __forceinline__ double weight(const Sample& x, const LamF64& c)
{
    const bool in = (x.m1b > c.mmin_bits) & (x.m1b <= c.mmax_bits) & (x.m2b >= c.mmin_bits);
    double aE = fma(c.beta, x.lq, x.nlpi);
    aE = fma(c.ac, x.sa, aE);
    aE = fma(c.bc, x.sb, aE);
    if (HAS_Z) aE = fma(c.km1, x.lz1, aE);
    const double e1 = exp(fma(c.nalpha, x.lm1, aE + c.cpl));
    const double d = x.m1 - c.mu;
    const double e2 = exp(fma(c.nh * d, d, aE + c.cg));
    double lr = c.lmmin - x.lm1;
    if (llabs(x.m1b - c.mmin_bits) < NEAR_EDGE_BITS) lr = log1p_near0(x.invm1 * (c.mmin - x.m1));
    const double den = c.beta_m1 ? -lr : fabs(expm1(c.b1 * lr));
    const double tt = c.t0 + exp(fma(c.nht, x.dc, c.ct));
    const double w = (e1 + e2) * tt / den;
    return in ? w : 0.0;
}

struct RawDesc {
    RawSet ev, inj;
    const int64_t* offsets;
    int64_t n_events, n_samples, n_found;
    int32_t n_inj_chunks;
    int32_t nd;
};

template <bool HAS_Z>
__global__ void __launch_bounds__(THREADS)
weight_raw_kernel(RawDesc a, const LamF64* __restrict__ lam, const int64_t* __restrict__ dK,
                  double* __restrict__ part, double* __restrict__ part2, unsigned long long* bad)
{
    __shared__ LamF64 sl[TILE];
    __shared__ double red[THREADS / 32][TILE];
    __shared__ double red2[THREADS / 32][TILE];
    const int64_t K = *dK;
    const int64_t n_tiles = (K + TILE - 1) / TILE;
    const int64_t n_chunks = a.n_events + a.n_inj_chunks;
    const int64_t n_items = n_chunks * n_tiles;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t c = item / n_tiles;
        const int64_t tile = item - c * n_tiles;
        const int64_t k0 = tile * TILE;
        const int tn = (int)(K - k0 < TILE ? K - k0 : TILE);
        __syncthreads();
        {
            constexpr int W = (int)(sizeof(LamF64) / 8);
            double* dst = reinterpret_cast<double*>(sl);
            for (int i = threadIdx.x; i < TILE * W; i += THREADS) {
                const int l = i / W;
                dst[i] = reinterpret_cast<const double*>(lam + k0 + (l < tn ? l : tn - 1))[i - l * W];
            }
        }
        __syncthreads();
        const bool inj = c >= a.n_events;
        int64_t start, len;
        if (!inj) {
            start = a.offsets[c];
            const int64_t end = a.offsets[c + 1];
            // Malformed offsets are counted and their event skipped (never read out of range).
            if (start < 0 || end <= start || end > a.n_samples) {
                if (tile == 0 && threadIdx.x == 0) atomicAdd(bad, 1ull);
                start = 0;
                len = 0;
            } else {
                len = end - start;
            }
        } else {
            start = (c - a.n_events) * INJ_CHUNK;
            len = a.n_found - start < INJ_CHUNK ? a.n_found - start : INJ_CHUNK;
        }
        const RawSet& R = inj ? a.inj : a.ev;
        double acc[TILE], acc2[TILE];
#pragma unroll
        for (int l = 0; l < TILE; ++l) acc[l] = acc2[l] = 0.0;
        for (int64_t j = threadIdx.x; j < len; j += THREADS) {
            Sample x;
            if (!make_sample(R, start + j, a.nd, x) && tile == 0) atomicAdd(bad, 1ull);
#pragma unroll
            for (int l = 0; l < TILE; ++l) {
                const double w = weight<HAS_Z>(x, sl[l]);
                acc[l] += w;
                if (inj) acc2[l] = fma(w, w, acc2[l]);
            }
        }
#pragma unroll
        for (int l = 0; l < TILE; ++l) {
            double v = acc[l], v2 = acc2[l];
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
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
            for (int w = 0; w < THREADS / 32; ++w) {
                s += red[w][l];
                s2 += red2[w][l];
            }
            part[(k0 + l) * n_chunks + c] = s;
            if (inj) part2[(k0 + l) * a.n_inj_chunks + (c - a.n_events)] = s2;
        }
    }
}

}  // namespace

extern "C" int pop_loglik_f64_noalloc(int device, void* stream, int64_t n_events, const int64_t* offsets,
                                      int64_t n_samples, int n_dims, const double* theta, const double* prior,
                                      int64_t n_found, int64_t n_draw, const double* inj_theta,
                                      const double* p_draw, int64_t K, int n_params, const double* lambda,
                                      double* out_lnL, double* out_lnxi, double* out_neff, uint32_t* out_flags,
                                      char* msg, int msg_len)
{
    const Msg fail{msg, msg_len};
    if (msg && msg_len > 0) msg[0] = 0;
    if (n_events < 1 || n_samples < n_events) return fail(POP_EINVAL, "need n_samples >= n_events >= 1");
    if (n_dims != 6 && n_dims != 7) return fail(POP_EINVAL, "n_dims must be 6 or 7");
    if (n_params != 11 + (n_dims == 7)) return fail(POP_EINVAL, "n_params must be 11 (12 with redshift)");
    if (n_found < 1 || n_draw < n_found) return fail(POP_EINVAL, "need n_draw >= n_found >= 1");
    if (K < 0) return fail(POP_EINVAL, "K < 0");
    if (!offsets || !theta || !prior || !inj_theta || !p_draw || (K > 0 && (!lambda || !out_lnL || !out_lnxi ||
                                                                             !out_neff || !out_flags)))
        return fail(POP_EINVAL, "a device pointer is NULL");
    if (device < 0 || device >= MAX_DEVICES) return fail(POP_EINVAL, "device index out of range");
    if (K == 0) return POP_OK;
    const int64_t n_inj_chunks = (n_found + INJ_CHUNK - 1) / INJ_CHUNK;
    if (K > (1LL << 24) || n_events > (1LL << 30) || n_inj_chunks > (1LL << 30))
        return fail(POP_EINVAL, "sizes beyond the scratch limit");
    const Layout Lo = layout(n_events, n_inj_chunks, K);
    if (Lo.total > SCRATCH_BYTES) {
        char m[256];
        snprintf(m, sizeof m, "needs %zu scratch bytes for K=%lld, %lld events, %lld injection chunks; the limit is %zu "
                 "(POP_NOALLOC_SCRATCH_BYTES): split the Lambda batch", Lo.total, (long long)K,
                 (long long)n_events, (long long)n_inj_chunks, SCRATCH_BYTES);
        return fail(POP_EINVAL, m);
    }
    const DeviceGuard guard;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(POP_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    {
        const void* ptrs[] = {offsets, theta, prior, inj_theta, p_draw, lambda, out_lnL, out_lnxi, out_neff, out_flags};
        const char* names[] = {"offsets", "theta", "prior", "inj_theta", "p_draw", "lambda", "out_lnL", "out_lnxi",
                               "out_neff", "out_flags"};
        for (int i = 0; i < 10; ++i)
            if (!on_device(ptrs[i], device))
                return fail(POP_EINVAL, std::string(names[i]) + " is not device memory of device " +
                                            std::to_string(device));
    }
    unsigned char* base = nullptr;
    {
        // One-time set-up per device: the symbol's device address (host code
        // only sees a host-side stand-in for the array).
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[device]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(POP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_addr[device] = p;
        }
        base = static_cast<unsigned char*>(g_scratch_addr[device]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t* dK = reinterpret_cast<int64_t*>(base + Lo.k);
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(base + Lo.bad);
    LamF64* c64 = reinterpret_cast<LamF64*>(base + Lo.c64);
    LamF32* c32 = reinterpret_cast<LamF32*>(base + Lo.c32);
    double* zint = reinterpret_cast<double*>(base + Lo.zint);
    int32_t* ecb = reinterpret_cast<int32_t*>(base + Lo.ecb);
    double* part = reinterpret_cast<double*>(base + Lo.part);
    double* part2 = reinterpret_cast<double*>(base + Lo.part2);

    setup_kernel<<<(unsigned)((n_events + 1 + 255) / 256), 256, 0, s>>>(dK, K, bad, ecb, n_events, offsets,
                                                                         n_samples);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(POP_ECUDA, cudaGetErrorString(e));
    if ((e = launch_prologue(lambda, dK, K, n_params, c64, c32, zint, s)) != cudaSuccess)
        return fail(POP_ECUDA, cudaGetErrorString(e));
    RawDesc a{{theta, prior}, {inj_theta, p_draw}, offsets, n_events, n_samples, n_found, (int32_t)n_inj_chunks,
              n_dims};
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const void* fn = n_dims == 7 ? (const void*)weight_raw_kernel<true> : (const void*)weight_raw_kernel<false>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, THREADS, 0) != cudaSuccess || occ < 1) occ = 1;
    void* args[] = {&a, &c64, &dK, &part, &part2, &bad};
    if ((e = cudaLaunchKernel(fn, dim3(sms * occ), dim3(THREADS), args, 0, s)) != cudaSuccess)
        return fail(POP_ECUDA, cudaGetErrorString(e));
    if ((e = launch_finalise(part, part2, ecb, offsets, n_events, (int32_t)(n_events + n_inj_chunks),
                             (int32_t)n_events, n_draw, c64, dK, K, out_lnL, out_lnxi, out_neff, out_flags, s)) !=
        cudaSuccess)
        return fail(POP_ECUDA, cudaGetErrorString(e));
    unsigned long long h_bad = 0;
    if ((e = cudaMemcpyAsync(&h_bad, bad, sizeof h_bad, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(POP_ECUDA, cudaGetErrorString(e));
    if (h_bad)
        return fail(POP_EINVAL, "malformed offsets (offsets[0] != 0, offsets[N] != n_samples, an empty or "
                                "out-of-range event), non-finite samples or prior/p_draw <= 0");
    return POP_OK;
}
