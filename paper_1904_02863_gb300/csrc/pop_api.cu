// Host runtime behind the C-ABI of include/pop.h: the context, device buffers,
// input validation, the one-time pack, CUDA-graph replay of
// prologue -> weight -> finalise, and the tiling autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "pop.h"
#include "pop_cbc.h"
#include "pop_devbuf.h"
#include "pop_gridvt.h"
#include "pop_internal.h"
#include "pop_trace.h"
#include "pop_mlp.h"

#include <memory>

using namespace pop;

namespace {

thread_local std::string g_create_error;

// Samples per work chunk (events are split at this length): 4096, halved down to 256 while a
// set would have fewer than about one chunk per SM, so that small sets still fill the GPU.
constexpr int CHUNK_LEN_MAX = 4096, CHUNK_LEN_MIN = 256, CHUNK_TARGET = 152;

int chunk_len_for(int64_t n)
{
    int len = CHUNK_LEN_MAX;
    while (len > CHUNK_LEN_MIN && n / len < CHUNK_TARGET) len >>= 1;
    return len;
}
constexpr int64_t ALIGN_ELEMS = 64;

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// One packed sample set (events or injections) in either or both precisions.
struct SampleSet {
    int64_t n = 0;
    int64_t stride = 0;
    int n_dims = 0;
    int storage = 0;
    int chunk_len = CHUNK_LEN_MAX;  // samples per work chunk of this set
    DevBuf f64, f32, m2, m1d, m1sort, m1pos, m1max;
    void swap(SampleSet& o)
    {
        std::swap(n, o.n);
        std::swap(chunk_len, o.chunk_len);
        std::swap(stride, o.stride);
        std::swap(n_dims, o.n_dims);
        std::swap(storage, o.storage);
        f64.swap(o.f64);
        f32.swap(o.f32);
        m2.swap(o.m2);
        m1d.swap(o.m1d);
        m1sort.swap(o.m1sort);
        m1pos.swap(o.m1pos);
        m1max.swap(o.m1max);
    }
    FeatF32 feat32() const
    {
        return FeatF32{f32.as<float>(), m2.as<double>(), m1d.as<double>(), m1sort.as<double>(), m1pos.as<uint2>(),
                       m1max.as<float>(), n, stride};
    }
};

struct Graph {
    cudaGraphExec_t exec = nullptr;
    int64_t k_cap = -1;
    uint64_t version = 0;
    uint64_t sur_version = 0;
    Tiling tiling{};
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        k_cap = -1;
    }
};

}  // namespace

struct pop_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;  // created here when the caller passed the legacy default stream
    std::string err;
    int sm_count = 0;
    std::string device_name;

    SampleSet ev, inj;
    std::vector<int64_t> h_offsets;
    DevBuf d_offsets;        // int64 [N+1]
    DevBuf d_inv_n;          // double [N]: 1/n_i
    int64_t n_draw = 0;

    // Work chunks: event chunks first, then injection chunks.
    DevBuf d_chunks, d_ecb;  // Chunk [n_chunks], int32 [N+1]
    int32_t n_chunks = 0, n_ev_chunks = 0;
    bool chunks_dirty = true;
    uint64_t version = 1;    // bumped whenever buffers the graphs point at change

    // Per-call scratch, sized for K_cap Lambda points.
    int64_t k_cap = 0;
    int n_params_cap = 12;
    DevBuf d_lambda, d_c64, d_c32, d_part, d_part2, d_lnL, d_lnxi, d_neff, d_flags, d_K;
    DevBuf d_parts;          // [K][3]: sum_i ln(S_i/n_i), sum w, sum w^2 (pop_loglik_parts)
    DevBuf d_zint;           // [K]: the redshift normalisation of each Lambda (prologue)
    DevBuf d_lamg, d_gpart, d_grad;  // gradient: per-Lambda constants, [K][n_chunks][13] sums, [K][12]
    int64_t grad_cap = 0;
    int32_t grad_chunks = -1;
    int32_t part_chunks = -1, part_inj = -1;

    Tiling tiling[2] = {{8, 256, 0}, {128, 128, 0}};
    bool use_graphs = true;
    Graph graph[4];  // per mode: F64, F32, F32 + surrogate, float-float
    DevBuf d_need, d_slnxi, d_slnneff;  // surrogate mode: Monte Carlo mask, ln xi, ln N_eff per Lambda
    DevBuf d_order, d_nmc;   // FP32 / float-float kernels: lane order [2][K_cap]; Lambda needing the injections
    DevBuf d_queue;          // the weight kernels' work-item counter
    cudaEvent_t ev_t0 = nullptr, ev_w0 = nullptr, ev_w1 = nullptr, ev_t1 = nullptr;
    DevBuf d_exptab;         // 2^(j/2048) as (hi, lo) for the FP64 exponentials
    DevBuf d_logtab;         // log_tab's table (the finalise's per-event logs)
    LogConsts logc{};
    DevBuf d_ztab;           // redshift trapezoid nodes (ln(1 + z_i), w_i z_i^2)
    ExpConsts expc{};
    DevBuf d_fftab;          // 2^(j/2048) as FP32 (hi, lo) for the float-float exponentials
    FFConsts ffk{};
    std::unique_ptr<Surrogate> sur;  // ln xi network, created on first use
    std::unique_ptr<GridVT> grid;    // grid selection term, created by pop_load_vt_grid
    std::unique_ptr<CbcState> cbc;   // single-event CBC likelihood, created by pop_cbc_load
    int xi_source = POP_XI_INJECTIONS;
    bool timed = false;
    int64_t last_K = 0;
    int last_params = 0;
};

namespace {

int fail(pop_ctx* c, int status, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return status;
}

int cuda_fail(pop_ctx* c, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? POP_ENOMEM : POP_ECUDA, m);
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

bool valid_mem(int mem) { return mem == POP_MEM_HOST || mem == POP_MEM_DEVICE; }

cudaMemcpyKind in_kind(int mem) { return mem == POP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind out_kind(int mem) { return mem == POP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

__global__ void set_k_kernel(int64_t* dK, int64_t K) { *dK = K; }

// Whether a sample lies inside the Lambda-independent part of the support (the
// pack kernels' test; non-finite rows are rejected there).
bool live_sample(const double* v, int n_dims)
{
    const double z = n_dims == 7 ? v[6] : 1.0;
    return v[0] > 0.0 && v[1] > 0.0 && v[1] <= 1.0 && v[2] >= 0.0 && v[2] <= 1.0 && v[3] >= 0.0 && v[3] <= 1.0 &&
           v[4] >= -1.0 && v[4] <= 1.0 && v[5] >= -1.0 && v[5] <= 1.0 && z >= 0.0 && z <= 2.0 && std::isfinite(v[0]);
}

// Load-time order of the samples: within every segment [seg[s], seg[s+1]) the
// samples are sorted by (m2, m1) with m2 = fl64(q m1), compared lexicographically
// (m2 = m1 = 0 for a sample outside the Lambda-independent support).  The lower
// support edge, m1 > mmin and m2 >= mmin, is then a suffix of every segment (m2 <= m1
// for q <= 1): the FP64 kernel's warps below it skip the arithmetic and the FP32
// kernel finds its first index by binary search.  Sums over a segment do not depend
// on the order (beyond rounding).
std::vector<int64_t> support_order(const double* theta, int64_t n, int n_dims, const std::vector<int64_t>& seg)
{
    std::vector<std::pair<double, double>> key(n);
    for (int64_t j = 0; j < n; ++j) {
        const double* v = theta + j * n_dims;
        // Rows with a non-finite coordinate are rejected by the pack kernel; any key will do for them.
        key[j] = live_sample(v, n_dims) ? std::make_pair(v[1] * v[0], v[0]) : std::make_pair(0.0, 0.0);
    }
    std::vector<int64_t> perm(n);
    for (int64_t j = 0; j < n; ++j) perm[j] = j;
    for (size_t s = 0; s + 1 < seg.size(); ++s)
        std::stable_sort(perm.begin() + seg[s], perm.begin() + seg[s + 1],
                         [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    return perm;
}

// Pack theta/prior (host or device) into a new SampleSet, in support_order.
int pack_samples(pop_ctx* c, int64_t n, int n_dims, const double* theta, const double* prior, int storage,
                 int mem, SampleSet& out, const char* what, const std::vector<int64_t>& seg)
{
    out.n = n;
    out.n_dims = n_dims;
    out.storage = storage;
    out.chunk_len = chunk_len_for(n);
    const int64_t cl = out.chunk_len;
    out.stride = round_up(std::max<int64_t>(n, 1), ALIGN_ELEMS);
    const double* th = theta;
    const double* pr = prior;
    DevBuf tmp_th, tmp_pr, bad, dperm;
    std::vector<double> m1sort;  // FP32 storage: the set's m1 in increasing order, and for each
    std::vector<uint2> m1pos;    // its (position, chunk index within the set)
    {
        std::vector<double> host_th;
        const double* hth = theta;
        if (mem == POP_MEM_DEVICE) {
            host_th.resize((size_t)n * n_dims);
            CK(cudaMemcpyAsync(host_th.data(), theta, sizeof(double) * n * n_dims, cudaMemcpyDeviceToHost,
                               c->stream), "copy theta to host");
            CK(cudaStreamSynchronize(c->stream), "sync");
            hth = host_th.data();
        }
        const std::vector<int64_t> perm = support_order(hth, n, n_dims, seg);
        CK(dperm.alloc(sizeof(int64_t) * std::max<int64_t>(n, 1)), "cudaMalloc(order)");
        CK(cudaMemcpyAsync(dperm.p, perm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream),
           "copy order");
        if (storage & POP_STORE_F32) {
            // Chunks are the chunk_len pieces of every segment (build_chunks makes the same cut).
            std::vector<std::pair<double, uint2>> e((size_t)n);
            uint32_t chunk = 0;
            for (size_t sg = 0; sg + 1 < seg.size(); ++sg)
                for (int64_t c0 = seg[sg]; c0 < seg[sg + 1]; c0 += cl, ++chunk) {
                    const int64_t len = std::min<int64_t>(cl, seg[sg + 1] - c0);
                    for (int64_t i = c0; i < c0 + len; ++i) {
                        const double* v = hth + perm[i] * n_dims;
                        e[i] = {live_sample(v, n_dims) ? v[0] : 0.0, make_uint2((uint32_t)i, chunk)};
                    }
                }
            std::sort(e.begin(), e.end(), [](const std::pair<double, uint2>& a, const std::pair<double, uint2>& b) {
                return a.first < b.first || (a.first == b.first && a.second.x < b.second.x);
            });
            m1sort.resize((size_t)std::max<int64_t>(n, 1));
            m1pos.resize((size_t)std::max<int64_t>(n, 1));
            for (int64_t i = 0; i < n; ++i) {
                m1sort[i] = e[i].first;
                m1pos[i] = e[i].second;
            }
        }
        CK(cudaStreamSynchronize(c->stream), "sync");
    }
    if (mem == POP_MEM_HOST) {
        CK(tmp_th.alloc(sizeof(double) * n * n_dims), "cudaMalloc(theta staging)");
        CK(tmp_pr.alloc(sizeof(double) * n), "cudaMalloc(prior staging)");
        CK(cudaMemcpyAsync(tmp_th.p, theta, sizeof(double) * n * n_dims, cudaMemcpyHostToDevice, c->stream),
           "copy theta");
        CK(cudaMemcpyAsync(tmp_pr.p, prior, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "copy prior");
        th = tmp_th.as<double>();
        pr = tmp_pr.as<double>();
    }
    CK(bad.alloc(sizeof(unsigned long long)), "cudaMalloc(flag)");
    CK(cudaMemsetAsync(bad.p, 0, sizeof(unsigned long long), c->stream), "memset");
    if (storage & POP_STORE_F64) {
        CK(out.f64.alloc(sizeof(double) * F_COUNT64 * out.stride), "cudaMalloc(f64 features)");
        CK(launch_pack_f64(th, pr, dperm.as<int64_t>(), n, n_dims, out.f64.as<double>(), out.stride,
                           bad.as<unsigned long long>(),
                           c->stream), "pack_f64");
    }
    if (storage & POP_STORE_F32) {
        CK(out.f32.alloc(sizeof(float) * F_COUNT32 * out.stride), "cudaMalloc(f32 features)");
        CK(out.m2.alloc(sizeof(double) * out.stride), "cudaMalloc(m2)");
        CK(out.m1d.alloc(sizeof(double) * out.stride), "cudaMalloc(m1)");
        CK(out.m1sort.alloc(sizeof(double) * m1sort.size()), "cudaMalloc(m1 order)");
        CK(out.m1pos.alloc(sizeof(uint2) * m1pos.size()), "cudaMalloc(m1 order)");
        CK(cudaMemcpyAsync(out.m1sort.p, m1sort.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream),
           "copy m1 order");
        CK(cudaMemcpyAsync(out.m1pos.p, m1pos.data(), sizeof(uint2) * n, cudaMemcpyHostToDevice, c->stream),
           "copy m1 order");
        CK(launch_pack_f32(th, pr, dperm.as<int64_t>(), n, n_dims, out.f32.as<float>(), out.m2.as<double>(),
                           out.m1d.as<double>(), out.stride, bad.as<unsigned long long>(), c->stream), "pack_f32");
        CK(out.m1max.alloc(sizeof(float) * (size_t)((n + M1MAX_BLOCK - 1) / M1MAX_BLOCK + 1)), "cudaMalloc(m1 maxima)");
        CK(launch_m1_blockmax(out.f32.as<float>(), out.stride, n, out.m1max.as<float>(), c->stream), "m1 maxima");
    }
    unsigned long long h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, bad.p, sizeof(h_bad), cudaMemcpyDeviceToHost, c->stream), "copy flag");
    CK(cudaStreamSynchronize(c->stream), "pack sync");
    if (h_bad) {
        char m[160];
        snprintf(m, sizeof m, "%s: %llu samples with non-finite coordinates or a prior/p_draw <= 0", what, h_bad);
        return fail(c, POP_EINVAL, m);
    }
    return POP_OK;
}

// (Re)build the chunk table from the loaded events and injections.
int build_chunks(pop_ctx* c)
{
    if (!c->chunks_dirty) return POP_OK;
    std::vector<Chunk> ch;
    std::vector<int32_t> ecb(c->h_offsets.size());
    const int64_t N = (int64_t)c->h_offsets.size() - 1;
    for (int64_t i = 0; i < N; ++i) {
        ecb[i] = (int32_t)ch.size();
        for (int64_t s = c->h_offsets[i]; s < c->h_offsets[i + 1]; s += c->ev.chunk_len)
            ch.push_back(Chunk{s, (int32_t)std::min<int64_t>(c->ev.chunk_len, c->h_offsets[i + 1] - s), 0});
    }
    ecb[N] = (int32_t)ch.size();
    const int32_t n_ev = (int32_t)ch.size();
    for (int64_t s = 0; s < c->inj.n; s += c->inj.chunk_len)
        ch.push_back(Chunk{s, (int32_t)std::min<int64_t>(c->inj.chunk_len, c->inj.n - s), 1});
    if (ch.size() > (size_t)INT32_MAX / 2) return fail(c, POP_EINVAL, "too many work chunks");
    DevBuf dch, decb;
    CK(dch.alloc(sizeof(Chunk) * ch.size()), "cudaMalloc(chunks)");
    CK(decb.alloc(sizeof(int32_t) * ecb.size()), "cudaMalloc(ecb)");
    CK(cudaMemcpyAsync(dch.p, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice, c->stream), "copy chunks");
    CK(cudaMemcpyAsync(decb.p, ecb.data(), sizeof(int32_t) * ecb.size(), cudaMemcpyHostToDevice, c->stream),
       "copy ecb");
    CK(cudaStreamSynchronize(c->stream), "chunk sync");
    c->d_chunks.swap(dch);
    c->d_ecb.swap(decb);
    c->n_chunks = (int32_t)ch.size();
    c->n_ev_chunks = n_ev;
    c->chunks_dirty = false;
    c->version++;
    return POP_OK;
}

// Scratch for K Lambda points (grows only).
int ensure_scratch(pop_ctx* c, int64_t K)
{
    const int32_t n_inj = c->n_chunks - c->n_ev_chunks;
    if (K <= c->k_cap && c->part_chunks == c->n_chunks && c->part_inj == n_inj) return POP_OK;
    const int64_t cap = std::max<int64_t>(std::max<int64_t>(K, c->k_cap), 64);
    DevBuf lam, c64, c32, part, part2, lnL, lnxi, neff, flags, dK, parts3;
    CK(lam.alloc(sizeof(double) * cap * 12), "cudaMalloc(lambda)");
    CK(parts3.alloc(sizeof(double) * cap * 3), "cudaMalloc(parts)");
    CK(c64.alloc(sizeof(LamF64) * cap), "cudaMalloc(consts64)");
    CK(c32.alloc(sizeof(LamF32) * cap), "cudaMalloc(consts32)");
    CK(part.alloc(sizeof(double) * cap * c->n_chunks), "cudaMalloc(partials)");
    CK(part2.alloc(sizeof(double) * cap * std::max<int32_t>(n_inj, 1)), "cudaMalloc(partials2)");
    CK(lnL.alloc(sizeof(double) * cap), "cudaMalloc(lnL)");
    CK(lnxi.alloc(sizeof(double) * cap), "cudaMalloc(lnxi)");
    CK(neff.alloc(sizeof(double) * cap), "cudaMalloc(neff)");
    CK(flags.alloc(sizeof(uint32_t) * cap), "cudaMalloc(flags)");
    CK(dK.alloc(sizeof(int64_t)), "cudaMalloc(K)");
    DevBuf need, slnxi, slnneff, order, nmc, queue;
    CK(need.alloc(cap), "cudaMalloc(need)");
    CK(order.alloc(sizeof(int32_t) * 2 * cap), "cudaMalloc(order)");
    CK(nmc.alloc(sizeof(int32_t)), "cudaMalloc(n_mc)");
    CK(queue.alloc(sizeof(unsigned long long)), "cudaMalloc(queue)");
    CK(slnxi.alloc(sizeof(double) * cap), "cudaMalloc(surrogate lnxi)");
    CK(slnneff.alloc(sizeof(double) * cap), "cudaMalloc(surrogate lnneff)");
    DevBuf zint;
    CK(zint.alloc(sizeof(double) * cap), "cudaMalloc(redshift normalisation)");
    c->d_zint.swap(zint);
    c->d_need.swap(need);
    c->d_order.swap(order);
    c->d_nmc.swap(nmc);
    c->d_queue.swap(queue);
    c->d_slnxi.swap(slnxi);
    c->d_slnneff.swap(slnneff);
    if (c->d_lambda.p)  // keep the last Lambda batch (the autotuner reuses it)
        CK(cudaMemcpyAsync(lam.p, c->d_lambda.p, std::min(lam.bytes, c->d_lambda.bytes), cudaMemcpyDeviceToDevice,
                           c->stream), "copy lambda");
    c->d_lambda.swap(lam);
    c->d_c64.swap(c64);
    c->d_c32.swap(c32);
    c->d_part.swap(part);
    c->d_part2.swap(part2);
    c->d_lnL.swap(lnL);
    c->d_lnxi.swap(lnxi);
    c->d_neff.swap(neff);
    c->d_flags.swap(flags);
    c->d_K.swap(dK);
    c->d_parts.swap(parts3);
    c->k_cap = cap;
    c->part_chunks = c->n_chunks;
    c->part_inj = n_inj;
    c->version++;
    return POP_OK;
}

int grid_size(pop_ctx* c, int mode)
{
    if (mode == POP_MODE_FF) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, weight_ff_fn(c->ev.n_dims == 7), weight_ff_threads(), 0) !=
            cudaSuccess)
            occ = 1;
        return std::max(1, occ) * c->sm_count;
    }
    const Tiling& t = c->tiling[mode];
    const void* fn = mode == POP_MODE_F64 ? weight_f64_fn(t, c->ev.n_dims == 7) : weight_f32_fn(t, c->ev.n_dims == 7);
    int occ = 0;
    const int dyn = mode == POP_MODE_F64 ? WEIGHT_F64_DYN_SMEM : 0;
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t.block_threads, dyn) != cudaSuccess) occ = 1;
    if (t.blocks_per_sm > 0) occ = std::min(occ, t.blocks_per_sm);
    return std::max(1, occ) * c->sm_count;
}

// Enqueue prologue -> weight -> finalise for the K stored in d_K.
int enqueue_pipeline(pop_ctx* c, int mode, int n_params, int grid, bool capturing)
{
    // Inside a capture the timing events must become external event-record
    // nodes, or the replayed graph would never record them.
    const unsigned rec = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    const int m = (mode == POP_MODE_F64 || mode == POP_MODE_FF) ? 0 : 1;  // FP64 or FP32 grid term and partials
    // With the grid selection term the injections are not part of the work list.
    const bool use_grid = c->xi_source == POP_XI_GRID;
    const int32_t n_items = use_grid ? c->n_ev_chunks : c->n_chunks;
    WorkDesc wd{c->d_chunks.as<Chunk>(), n_items, c->n_ev_chunks, c->ev.n_dims == 7};
    CK(cudaEventRecordWithFlags(c->ev_t0, c->stream, rec), "event");
    CK(launch_prologue(c->d_lambda.as<double>(), c->d_K.as<int64_t>(), c->k_cap, n_params, c->d_c64.as<LamF64>(),
                       c->d_c32.as<LamF32>(), c->d_zint.as<double>(), c->stream, c->d_ztab.as<double2>(),
                       c->d_exptab.as<double2>(), c->expc), "prologue");
    SurrogateXi sx{nullptr, nullptr, nullptr};
    if (mode == POP_MODE_F32_SURROGATE) {
        // ln xi from the network for every Lambda, and which Lambda still need the Monte Carlo xi.
        const int64_t n_events = (int64_t)c->h_offsets.size() - 1;
        const int rc = c->sur->enqueue_gate(c->d_lambda.as<double>(), c->k_cap, n_params, c->d_K.as<int64_t>(),
                                            (double)n_events, c->d_need.as<uint8_t>(), c->d_slnxi.as<double>(),
                                            c->d_slnneff.as<double>());
        if (rc != POP_OK) return fail(c, rc, "surrogate: " + c->sur->err);
        sx = SurrogateXi{c->d_need.as<uint8_t>(), c->d_slnxi.as<double>(), c->d_slnneff.as<double>()};
    }
    CK(cudaEventRecordWithFlags(c->ev_w0, c->stream, rec), "event");
    if (mode == POP_MODE_FF) {
        FeatF64 e{c->ev.f64.as<double>(), c->ev.stride}, j{c->inj.f64.as<double>(), c->inj.stride};
        CK(launch_lam_order(c->d_c32.as<LamF32>(), c->d_K.as<int64_t>(), nullptr, c->k_cap, c->d_order.as<int32_t>(),
                            c->d_nmc.as<int32_t>(), c->stream), "lambda order");
        CK(launch_weight_ff(grid, e, j, wd, c->d_c64.as<LamF64>(), c->d_order.as<int32_t>(), c->d_nmc.as<int32_t>(),
                            c->d_queue.as<unsigned long long>(), c->k_cap, c->d_K.as<int64_t>(), c->d_part.as<double>(), c->d_part2.as<double>(),
                            c->d_fftab.as<float2>(), c->ffk, c->stream), "weight_ff");
    } else if (m == 0) {
        FeatF64 e{c->ev.f64.as<double>(), c->ev.stride}, j{c->inj.f64.as<double>(), c->inj.stride};
        CK(launch_weight_f64(c->tiling[0], grid, e, j, wd, c->d_c64.as<LamF64>(), c->d_K.as<int64_t>(),
                             c->d_part.as<double>(), c->d_part2.as<double>(), c->d_exptab.as<double2>(), c->expc,
                             c->d_queue.as<unsigned long long>(), c->stream), "weight_f64");
    } else {
        FeatF32 e = c->ev.feat32();
        FeatF32 j = c->inj.feat32();
        CK(launch_lam_order(c->d_c32.as<LamF32>(), c->d_K.as<int64_t>(), sx.need_mc, c->k_cap,
                            c->d_order.as<int32_t>(), c->d_nmc.as<int32_t>(), c->stream), "lambda order");
        CK(launch_weight_f32(c->tiling[1], grid, e, j, wd, c->d_c32.as<LamF32>(), c->d_order.as<int32_t>(),
                             c->d_nmc.as<int32_t>(), c->d_queue.as<unsigned long long>(), c->k_cap, c->d_K.as<int64_t>(), c->d_part.as<double>(),
                             c->d_part2.as<double>(), c->stream), "weight_f32");
        CK(launch_upper_edge_fixup(e, j, wd, c->d_c32.as<LamF32>(), sx.need_mc, c->k_cap, c->d_K.as<int64_t>(),
                                   c->d_part.as<double>(), c->d_part2.as<double>(), c->stream), "upper-edge fix-up");
    }
    CK(cudaEventRecordWithFlags(c->ev_w1, c->stream, rec), "event");
    if (use_grid)
        CK(c->grid->enqueue(m, c->d_lambda.as<double>(), n_params, c->d_K.as<int64_t>(), c->k_cap, true, rec,
                            c->stream), "grid selection term");
    CK(launch_finalise(c->d_part.as<double>(), c->d_part2.as<double>(), c->d_ecb.as<int32_t>(),
                       c->d_offsets.as<int64_t>(), c->ev.n == 0 ? 0 : (int64_t)c->h_offsets.size() - 1,
                       n_items, c->n_ev_chunks, c->n_draw, c->d_c64.as<LamF64>(), c->d_K.as<int64_t>(),
                       c->k_cap, c->d_lnL.as<double>(), c->d_lnxi.as<double>(), c->d_neff.as<double>(),
                       c->d_flags.as<uint32_t>(), c->stream, sx, use_grid ? c->grid->xi.as<double>() : nullptr,
                       c->d_parts.as<double>(), c->d_logtab.as<LogEntry>(), c->logc, c->d_inv_n.as<double>()),
       "finalise");
    CK(cudaEventRecordWithFlags(c->ev_t1, c->stream, rec), "event");
    return POP_OK;
}

int run_pipeline(pop_ctx* c, int mode, int n_params)
{
    const int m = mode == POP_MODE_F64 ? 0 : 1;  // tiling slot (the float-float kernel has one fixed tiling)
    const int grid = grid_size(c, mode == POP_MODE_FF ? POP_MODE_FF : m);
    uint64_t sur_version = 0;
    if (mode == POP_MODE_F32_SURROGATE) {  // buffers first: nothing may be allocated during a capture
        const int rc = c->sur->ensure_gate(c->k_cap);
        if (rc != POP_OK) return fail(c, rc, "surrogate: " + c->sur->err);
        sur_version = c->sur->version;
    }
    if (!c->use_graphs) return enqueue_pipeline(c, mode, n_params, grid, false);
    Graph& g = c->graph[mode];
    const Tiling& t = c->tiling[m];
    const bool stale = !g.exec || g.k_cap != c->k_cap || g.version != c->version || g.tiling.lambda_tile != t.lambda_tile ||
                       g.tiling.block_threads != t.block_threads || g.tiling.blocks_per_sm != t.blocks_per_sm ||
                       c->last_params != n_params || g.sur_version != sur_version;
    if (stale) {
        g.reset();
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int rc = enqueue_pipeline(c, mode, n_params, grid, true);
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (rc != POP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        CK(e, "end capture");
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e, "graph instantiate");
        g.k_cap = c->k_cap;
        g.version = c->version;
        g.tiling = t;
        g.sur_version = sur_version;
    }
    CK(cudaGraphLaunch(g.exec, c->stream), "graph launch");
    return POP_OK;
}

bool tiling_ok(int mode, const Tiling& t)
{
    return (mode == POP_MODE_F64 ? weight_f64_fn(t, false) : weight_f32_fn(t, false)) != nullptr &&
           t.blocks_per_sm >= 0 && t.blocks_per_sm <= 32;
}

}  // namespace

namespace pop {

// Tang's table: T_j = 2^(j/2048) = hi + lo, and the reduction constants 2048/ln2
// and ln2/2048, all from long double (extended or quad) arithmetic.
void build_exp_table(double2* tab, ExpConsts* kc)
{
    for (int j = 0; j < EXP_TABLE_SIZE; ++j) {
        const long double v = exp2l((long double)j / EXP_TABLE_SIZE);
        const double hi = (double)v;
        tab[j] = make_double2(hi, (double)(v - (long double)hi));
    }
    const long double ln2 = logl(2.0L);
    kc->inv_l = (float)(EXP_TABLE_SIZE / ln2);
    kc->l = (double)(ln2 / EXP_TABLE_SIZE);
}

// log_tab's table: F_j = 1 + j/128, 1/F_j rounded, ln F_j = hi + lo with hi rounded to the grid
// of 2^-43, and ln 2 split the same way, all from long double arithmetic.
void build_log_table(LogEntry* tab, LogConsts* k)
{
    auto grid43 = [](long double v) { return (double)(ldexpl(nearbyintl(ldexpl(v, 43)), -43)); };
    for (int j = 0; j < LOG_TABLE_SIZE; ++j) {
        const long double F = 1.0L + (long double)j / 128.0L;
        const long double lnF = logl(F);
        const double h = grid43(lnF);
        tab[j] = LogEntry{(double)(1.0L / F), h, (double)(lnF - (long double)h)};
    }
    const long double ln2 = logl(2.0L);
    k->l_hi = grid43(ln2);
    k->l_lo = (double)(ln2 - (long double)k->l_hi);
}

}  // namespace pop

// Context accessors for the surrogate entry points (pop_surrogate.cu).
namespace pop {

int ctx_fail(pop_ctx* c, int status, const std::string& msg) { return fail(c, status, msg); }
cudaStream_t ctx_stream(pop_ctx* c) { return c->stream; }
int ctx_device(pop_ctx* c) { return c->device; }
int64_t ctx_n_events(pop_ctx* c) { return c->ev.n ? (int64_t)c->h_offsets.size() - 1 : 0; }
int ctx_n_dims(pop_ctx* c) { return c->ev.n_dims; }
int ctx_has_storage(pop_ctx* c, int storage)
{
    return c->ev.n && c->inj.n && (c->ev.storage & storage) && (c->inj.storage & storage);
}
Surrogate* ctx_surrogate(pop_ctx* c, int* status)
{
    *status = POP_OK;
    if (!c->sur) {
        std::unique_ptr<Surrogate> s(new Surrogate());
        const int rc = s->init(c->device, c->stream);
        if (rc != POP_OK) {
            *status = fail(c, rc, "surrogate: " + s->err);
            return nullptr;
        }
        c->sur = std::move(s);
    }
    return c->sur.get();
}

}  // namespace pop

// ============================================================== C-ABI
extern "C" {

int pop_math_check(pop_ctx* c, int fn, int64_t n, const double* x, double* y, int mem)
{
    if (!c) return POP_EINVAL;
    if (fn < 0 || fn > 8 || n < 0 || (n > 0 && (!x || !y)) || !valid_mem(mem))
        return fail(c, POP_EINVAL, "pop_math_check: bad arguments");
    if (n == 0) return POP_OK;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const double* dx = x;
    double* dy = y;
    DevBuf bx, by;
    if (mem == POP_MEM_HOST) {
        CK(bx.alloc(sizeof(double) * n), "cudaMalloc");
        CK(by.alloc(sizeof(double) * n), "cudaMalloc");
        CK(cudaMemcpyAsync(bx.p, x, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "copy x");
        dx = bx.as<double>();
        dy = by.as<double>();
    }
    if (fn <= 2 || fn == 8)
        CK(launch_math_check(fn, n, dx, dy, c->d_exptab.as<double2>(), c->expc, c->d_logtab.as<LogEntry>(), c->logc,
                             c->stream),
           "math_check");
    else
        CK(launch_ff_math_check(fn, n, dx, dy, c->d_fftab.as<float2>(), c->ffk, c->stream), "ff_math_check");
    if (mem == POP_MEM_HOST) {
        CK(cudaMemcpyAsync(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "copy y");
        CK(cudaStreamSynchronize(c->stream), "sync");
    }
    return POP_OK;
}

int pop_wait_check(pop_ctx* c, int arrive, int polls)
{
    if (!c) return POP_EINVAL;
    if (polls < 1 || polls > POP_WAIT_CHECK_MAX_POLLS) return fail(c, POP_EINVAL, "pop_wait_check: polls out of range");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    DevBuf err;
    CK(err.alloc(sizeof(int)), "cudaMalloc");
    CK(cudaMemsetAsync(err.p, 0, sizeof(int), c->stream), "memset");
    CK(launch_wait_check(arrive != 0, polls, err.as<int>(), c->stream), "wait_check");
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy error word");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (bad) return fail(c, POP_ETIMEOUT, "pop_wait_check: the bounded wait gave up after " + std::to_string(polls) + " polls");
    return POP_OK;
}

int pop_version(void) { return 10000; }

const char* pop_status_string(int s)
{
    switch (s) {
        case POP_OK: return "POP_OK";
        case POP_EINVAL: return "POP_EINVAL";
        case POP_ENOMEM: return "POP_ENOMEM";
        case POP_ECUDA: return "POP_ECUDA";
        case POP_ESTATE: return "POP_ESTATE";
        case POP_ETIMEOUT: return "POP_ETIMEOUT";
        case POP_ENUMERIC: return "POP_ENUMERIC";
        default: return "POP_UNKNOWN";
    }
}

const char* pop_last_error(const pop_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int pop_create(pop_ctx** out, int device, void* stream)
{
    pop_ctx* c = nullptr;
    if (!out) return fail(nullptr, POP_EINVAL, "pop_create: out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        return fail(nullptr, POP_ECUDA, std::string("pop_create: no CUDA device (") + cudaGetErrorString(e) + ")");
    if (device < 0 || device >= n) return fail(nullptr, POP_EINVAL, "pop_create: device index out of range");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, POP_ECUDA, std::string("pop_create: ") + cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return fail(nullptr, POP_ECUDA, std::string("pop_create: ") + cudaGetErrorString(e));
    if (prop.major < 10) return fail(nullptr, POP_ECUDA, "pop_create: the library is built for sm_103a (GB300)");
    c = new pop_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (!c->stream) {
        // The legacy default stream cannot be captured into a graph; a blocking
        // stream keeps the same ordering with respect to it.
        e = cudaStreamCreate(&c->stream);
        if (e != cudaSuccess) {
            delete c;
            return fail(nullptr, POP_ECUDA, std::string("pop_create: ") + cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    c->sm_count = prop.multiProcessorCount;
    c->device_name = prop.name;
    {
        std::vector<double2> tab(EXP_TABLE_SIZE);
        build_exp_table(tab.data(), &c->expc);
        e = c->d_exptab.alloc(sizeof(double2) * EXP_TABLE_SIZE);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_exptab.p, tab.data(), sizeof(double2) * EXP_TABLE_SIZE, cudaMemcpyHostToDevice);
        std::vector<LogEntry> ltab(LOG_TABLE_SIZE);
        build_log_table(ltab.data(), &c->logc);
        if (e == cudaSuccess) e = c->d_logtab.alloc(sizeof(LogEntry) * LOG_TABLE_SIZE);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_logtab.p, ltab.data(), sizeof(LogEntry) * LOG_TABLE_SIZE, cudaMemcpyHostToDevice);
        std::vector<double2> ztab(REDSHIFT_NODES);
        build_z_table(ztab.data());
        if (e == cudaSuccess) e = c->d_ztab.alloc(sizeof(double2) * REDSHIFT_NODES);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_ztab.p, ztab.data(), sizeof(double2) * REDSHIFT_NODES, cudaMemcpyHostToDevice);
        std::vector<float2> ftab(FF_TABLE_SIZE);
        build_ff_table(ftab.data(), &c->ffk);
        if (e == cudaSuccess) e = c->d_fftab.alloc(sizeof(float2) * FF_TABLE_SIZE);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_fftab.p, ftab.data(), sizeof(float2) * FF_TABLE_SIZE, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            pop_destroy(c);
            return fail(nullptr, e == cudaErrorMemoryAllocation ? POP_ENOMEM : POP_ECUDA,
                        std::string("pop_create: ") + cudaGetErrorString(e));
        }
    }
    cudaEvent_t* evs[] = {&c->ev_t0, &c->ev_w0, &c->ev_w1, &c->ev_t1};
    for (cudaEvent_t* ev : evs) {
        e = cudaEventCreate(ev);
        if (e != cudaSuccess) {
            pop_destroy(c);
            return fail(nullptr, POP_ECUDA, std::string("pop_create: ") + cudaGetErrorString(e));
        }
    }
    *out = c;
    return POP_OK;
}

int pop_destroy(pop_ctx* c)
{
    if (!c) return POP_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (Graph& g : c->graph) g.reset();
    cudaEvent_t evs[] = {c->ev_t0, c->ev_w0, c->ev_w1, c->ev_t1};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return POP_OK;
}

int pop_validate_events(int64_t n_events, const int64_t* offsets, int n_dims, char* msg, int msg_len)
{
    auto say = [&](const char* m) {
        if (msg && msg_len > 0) snprintf(msg, (size_t)msg_len, "%s", m);
        return POP_EINVAL;
    };
    if (n_events < 1) return say("n_events must be >= 1");
    if (!offsets) return say("offsets is NULL");
    if (n_dims != 6 && n_dims != 7) return say("n_dims must be 6 or 7");
    if (offsets[0] != 0) return say("offsets[0] must be 0");
    for (int64_t i = 0; i < n_events; ++i)
        if (offsets[i + 1] <= offsets[i]) return say("every event needs >= 1 sample (offsets strictly increasing)");
    if (offsets[n_events] > ((int64_t)1 << 40)) return say("too many samples");
    if (msg && msg_len > 0) msg[0] = 0;
    return POP_OK;
}

int pop_load_events(pop_ctx* c, int64_t n_events, const int64_t* offsets, int n_dims, const double* theta,
                    const double* prior, int storage, int mem)
{
    pop::TraceRange trace_("pop_load_events");
    if (!c) return POP_EINVAL;
    char m[200];
    if (pop_validate_events(n_events, offsets, n_dims, m, sizeof m) != POP_OK)
        return fail(c, POP_EINVAL, std::string("pop_load_events: ") + m);
    if (!theta || !prior) return fail(c, POP_EINVAL, "pop_load_events: theta/prior is NULL");
    if (storage < 1 || storage > 3) return fail(c, POP_EINVAL, "pop_load_events: storage must be F64, F32 or both");
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, "pop_load_events: bad mem");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const int64_t n = offsets[n_events];
    SampleSet s;
    int rc = pack_samples(c, n, n_dims, theta, prior, storage, mem, s, "pop_load_events",
                          std::vector<int64_t>(offsets, offsets + n_events + 1));
    if (rc != POP_OK) return rc;
    DevBuf doff, dinv;
    std::vector<double> inv(n_events);  // 1/n_i, correctly rounded, for the finalise
    for (int64_t i = 0; i < n_events; ++i) inv[i] = 1.0 / (double)(offsets[i + 1] - offsets[i]);
    CK(doff.alloc(sizeof(int64_t) * (n_events + 1)), "cudaMalloc(offsets)");
    CK(dinv.alloc(sizeof(double) * std::max<int64_t>(n_events, 1)), "cudaMalloc(1/n)");
    CK(cudaMemcpyAsync(doff.p, offsets, sizeof(int64_t) * (n_events + 1), cudaMemcpyHostToDevice, c->stream),
       "copy offsets");
    CK(cudaMemcpyAsync(dinv.p, inv.data(), sizeof(double) * n_events, cudaMemcpyHostToDevice, c->stream), "copy 1/n");
    CK(cudaStreamSynchronize(c->stream), "sync");
    c->ev.swap(s);
    c->d_offsets.swap(doff);
    c->d_inv_n.swap(dinv);
    c->h_offsets.assign(offsets, offsets + n_events + 1);
    if (c->inj.n && c->inj.n_dims != n_dims) {  // stale injections of another layout
        SampleSet none;
        c->inj.swap(none);
        c->n_draw = 0;
    }
    c->chunks_dirty = true;
    c->version++;
    return POP_OK;
}

int pop_load_injections(pop_ctx* c, int64_t n_found, int64_t n_draw, int n_dims, const double* theta,
                        const double* p_draw, int storage, int mem)
{
    pop::TraceRange trace_("pop_load_injections");
    if (!c) return POP_EINVAL;
    if (c->ev.n == 0) return fail(c, POP_ESTATE, "pop_load_injections: load events first");
    if (n_found < 1 || n_draw < n_found) return fail(c, POP_EINVAL, "pop_load_injections: need n_draw >= n_found >= 1");
    if (n_dims != c->ev.n_dims) return fail(c, POP_EINVAL, "pop_load_injections: n_dims differs from the events");
    if (!theta || !p_draw) return fail(c, POP_EINVAL, "pop_load_injections: theta/p_draw is NULL");
    if (storage < 1 || storage > 3) return fail(c, POP_EINVAL, "pop_load_injections: bad storage");
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, "pop_load_injections: bad mem");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    SampleSet s;
    int rc = pack_samples(c, n_found, n_dims, theta, p_draw, storage, mem, s, "pop_load_injections",
                          std::vector<int64_t>{0, n_found});
    if (rc != POP_OK) return rc;
    c->inj.swap(s);
    c->n_draw = n_draw;
    c->chunks_dirty = true;
    c->version++;
    return POP_OK;
}

}  // extern "C"

namespace {

// Validation and one evaluation of the pipeline for K Lambda rows (results stay on the device).
int loglik_run(pop_ctx* c, int64_t K, int n_params, const double* lambda, int mode, int mem, const char* who)
{
    const std::string w(who);
    const bool use_grid = c->xi_source == POP_XI_GRID;
    if (c->ev.n == 0) return fail(c, POP_ESTATE, w + ": load events first");
    if (!use_grid && c->inj.n == 0) return fail(c, POP_ESTATE, w + ": load injections first");
    if (use_grid && mode == POP_MODE_F32_SURROGATE)
        return fail(c, POP_EINVAL, w + ": the surrogate mode replaces the injection selection term, not the grid");
    if (K < 0) return fail(c, POP_EINVAL, w + ": K < 0");
    if (n_params != 11 + (c->ev.n_dims == 7))
        return fail(c, POP_EINVAL, w + ": n_params must be 11 (12 with redshift samples)");
    if (mode != POP_MODE_F64 && mode != POP_MODE_F32 && mode != POP_MODE_F32_SURROGATE && mode != POP_MODE_FF)
        return fail(c, POP_EINVAL, w + ": bad mode");
    if (mode == POP_MODE_F32_SURROGATE && (!c->sur || !c->sur->trained))
        return fail(c, POP_ESTATE, w + ": surrogate not trained (pop_xi_surrogate_train or _load)");
    if (mode == POP_MODE_F32_SURROGATE && c->sur->n_params != n_params)
        return fail(c, POP_EINVAL, w + ": the surrogate was trained for another n_params");
    const int need = (mode == POP_MODE_F64 || mode == POP_MODE_FF) ? POP_STORE_F64 : POP_STORE_F32;
    if (!(c->ev.storage & need) || (!use_grid && !(c->inj.storage & need)))
        return fail(c, POP_ESTATE, w + ": the loaded storage does not include this mode's precision");
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, w + ": bad mem");
    if (K == 0) return POP_OK;
    if (!lambda) return fail(c, POP_EINVAL, w + ": lambda is NULL");
    if (K > (1LL << 24)) return fail(c, POP_EINVAL, w + ": K too large");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    int rc = build_chunks(c);
    if (rc != POP_OK) return rc;
    rc = ensure_scratch(c, K);
    if (rc != POP_OK) return rc;
    if (use_grid && (c->grid->k_cap < c->k_cap || c->grid->slice <= 0)) {
        CK(c->grid->ensure(c->k_cap), "grid scratch");
        c->version++;  // the graphs point at the grid scratch
    }
    CK(cudaMemcpyAsync(c->d_lambda.p, lambda, sizeof(double) * K * n_params, in_kind(mem), c->stream), "copy lambda");
    set_k_kernel<<<1, 1, 0, c->stream>>>(c->d_K.as<int64_t>(), K);
    CK(cudaGetLastError(), "set K");
    rc = run_pipeline(c, mode, n_params);
    if (rc != POP_OK) return rc;
    c->last_params = n_params;
    c->last_K = K;
    c->timed = true;
    return POP_OK;
}

// The parts stay in [K][3] on the device; they are split into the three caller arrays here.
__global__ void split_parts_kernel(const double* parts, const uint32_t* flags, const int64_t* dK, double* ev,
                                   double* sw, double* sw2, uint32_t* fl)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= *dK) return;
    ev[k] = parts[3 * k];
    sw[k] = parts[3 * k + 1];
    sw2[k] = parts[3 * k + 2];
    if (fl) fl[k] = flags[k] & (POP_FLAG_INVALID_LAMBDA | POP_FLAG_ZERO_EVENT);
}

// After a synchronous (host-memory) call: the grid contraction's error word.
int check_grid_error(pop_ctx* c, const char* who)
{
    if (c->xi_source != POP_XI_GRID) return POP_OK;
    int bad = 0;
    CK(c->grid->take_error(&bad, c->stream), "grid error word");
    if (bad) return fail(c, POP_ETIMEOUT, std::string(who) + ": a bounded wait of the grid contraction gave up");
    return POP_OK;
}

}  // namespace

extern "C" {

int pop_loglik(pop_ctx* c, int64_t K, int n_params, const double* lambda, int mode, double* out_lnL,
               double* out_lnxi, double* out_neff, uint32_t* out_flags, int mem)
{
    pop::TraceRange trace_("pop_loglik");
    if (!c) return POP_EINVAL;
    if (K > 0 && !out_lnL) return fail(c, POP_EINVAL, "pop_loglik: out_lnL is NULL");
    int rc = loglik_run(c, K, n_params, lambda, mode, mem, "pop_loglik");
    if (rc != POP_OK || K == 0) return rc;
    CK(cudaMemcpyAsync(out_lnL, c->d_lnL.p, sizeof(double) * K, out_kind(mem), c->stream), "copy lnL");
    if (out_lnxi) CK(cudaMemcpyAsync(out_lnxi, c->d_lnxi.p, sizeof(double) * K, out_kind(mem), c->stream), "copy lnxi");
    if (out_neff) CK(cudaMemcpyAsync(out_neff, c->d_neff.p, sizeof(double) * K, out_kind(mem), c->stream), "copy neff");
    if (out_flags)
        CK(cudaMemcpyAsync(out_flags, c->d_flags.p, sizeof(uint32_t) * K, out_kind(mem), c->stream), "copy flags");
    if (mem == POP_MEM_HOST) {
        CK(cudaStreamSynchronize(c->stream), "sync");
        return check_grid_error(c, "pop_loglik");
    }
    return POP_OK;
}

int pop_loglik_parts(pop_ctx* c, int64_t K, int n_params, const double* lambda, int mode, double* out_events,
                     double* out_sum_w, double* out_sum_w2, uint32_t* out_flags, int mem)
{
    pop::TraceRange trace_("pop_loglik_parts");
    if (!c) return POP_EINVAL;
    if (c->xi_source != POP_XI_INJECTIONS)
        return fail(c, POP_EINVAL, "pop_loglik_parts: needs the injection selection term");
    if (mode != POP_MODE_F64 && mode != POP_MODE_F32 && mode != POP_MODE_FF)
        return fail(c, POP_EINVAL, "pop_loglik_parts: mode must be POP_MODE_F64, POP_MODE_F32 or POP_MODE_FF");
    if (K > 0 && (!out_events || !out_sum_w || !out_sum_w2))
        return fail(c, POP_EINVAL, "pop_loglik_parts: an output is NULL");
    int rc = loglik_run(c, K, n_params, lambda, mode, mem, "pop_loglik_parts");
    if (rc != POP_OK || K == 0) return rc;
    double *ev = out_events, *sw = out_sum_w, *sw2 = out_sum_w2;
    uint32_t* fl = out_flags;
    DevBuf tmp;
    if (mem == POP_MEM_HOST) {  // split into device scratch, then copy out
        CK(tmp.alloc((sizeof(double) * 3 + sizeof(uint32_t)) * K), "cudaMalloc(parts)");
        ev = tmp.as<double>();
        sw = ev + K;
        sw2 = sw + K;
        fl = reinterpret_cast<uint32_t*>(sw2 + K);
    }
    split_parts_kernel<<<(unsigned)((K + 255) / 256), 256, 0, c->stream>>>(
        c->d_parts.as<double>(), c->d_flags.as<uint32_t>(), c->d_K.as<int64_t>(), ev, sw, sw2,
        (out_flags || mem == POP_MEM_HOST) ? fl : nullptr);
    CK(cudaGetLastError(), "split parts");
    if (mem == POP_MEM_HOST) {
        CK(cudaMemcpyAsync(out_events, ev, sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream), "copy events");
        CK(cudaMemcpyAsync(out_sum_w, sw, sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream), "copy sum_w");
        CK(cudaMemcpyAsync(out_sum_w2, sw2, sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream), "copy sum_w2");
        if (out_flags)
            CK(cudaMemcpyAsync(out_flags, fl, sizeof(uint32_t) * K, cudaMemcpyDeviceToHost, c->stream), "copy flags");
        CK(cudaStreamSynchronize(c->stream), "sync");
    }
    return POP_OK;
}

int pop_loglik_grad(pop_ctx* c, int64_t K, int n_params, const double* lambda, double* out_lnL, double* out_grad,
                    uint32_t* out_flags, int mem)
{
    pop::TraceRange trace_("pop_loglik_grad");
    if (!c) return POP_EINVAL;
    if (c->xi_source != POP_XI_INJECTIONS)
        return fail(c, POP_EINVAL, "pop_loglik_grad: needs the injection selection term");
    if (c->ev.n == 0 || c->inj.n == 0) return fail(c, POP_ESTATE, "pop_loglik_grad: load events and injections first");
    if (!(c->ev.storage & POP_STORE_F64) || !(c->inj.storage & POP_STORE_F64))
        return fail(c, POP_ESTATE, "pop_loglik_grad: needs FP64 storage");
    if (n_params != 11 + (c->ev.n_dims == 7))
        return fail(c, POP_EINVAL, "pop_loglik_grad: n_params must be 11 (12 with redshift samples)");
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, "pop_loglik_grad: bad mem");
    if (K < 0 || K > (1LL << 24)) return fail(c, POP_EINVAL, "pop_loglik_grad: K out of range");
    if (K == 0) return POP_OK;
    if (!lambda || !out_lnL || !out_grad) return fail(c, POP_EINVAL, "pop_loglik_grad: NULL pointer");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    int rc = build_chunks(c);
    if (rc != POP_OK) return rc;
    rc = ensure_scratch(c, K);
    if (rc != POP_OK) return rc;
    if (K > c->grad_cap || c->grad_chunks != c->n_chunks) {
        const int64_t cap = std::max<int64_t>(K, c->grad_cap);
        DevBuf lg, gp, gr;
        CK(lg.alloc(lam_grad_bytes() * cap), "cudaMalloc(grad constants)");
        CK(gp.alloc(sizeof(double) * 13 * cap * c->n_chunks), "cudaMalloc(grad partials)");
        CK(gr.alloc(sizeof(double) * 12 * cap), "cudaMalloc(grad)");
        c->d_lamg.swap(lg);
        c->d_gpart.swap(gp);
        c->d_grad.swap(gr);
        c->grad_cap = cap;
        c->grad_chunks = c->n_chunks;
    }
    CK(cudaMemcpyAsync(c->d_lambda.p, lambda, sizeof(double) * K * n_params, in_kind(mem), c->stream), "copy lambda");
    set_k_kernel<<<1, 1, 0, c->stream>>>(c->d_K.as<int64_t>(), K);
    CK(cudaGetLastError(), "set K");
    CK(cudaEventRecord(c->ev_t0, c->stream), "event");
    CK(launch_grad_prologue(c->d_lambda.as<double>(), c->d_K.as<int64_t>(), K, n_params, c->d_lamg.p, c->stream,
                            c->d_ztab.as<double2>(), c->d_exptab.as<double2>(), c->expc),
       "grad prologue");
    WorkDesc wd{c->d_chunks.as<Chunk>(), c->n_chunks, c->n_ev_chunks, c->ev.n_dims == 7};
    FeatF64 e{c->ev.f64.as<double>(), c->ev.stride}, j{c->inj.f64.as<double>(), c->inj.stride};
    CK(cudaEventRecord(c->ev_w0, c->stream), "event");
    CK(launch_grad_weight(grad_grid_size(c->sm_count), e, j, wd, c->d_lamg.p, c->d_K.as<int64_t>(), n_params,
                          c->d_gpart.as<double>(), c->d_part2.as<double>(), c->d_exptab.as<double2>(), c->expc,
                          c->d_queue.as<unsigned long long>(), c->stream),
       "grad weight");
    CK(cudaEventRecord(c->ev_w1, c->stream), "event");
    CK(launch_grad_finalise(c->d_gpart.as<double>(), c->d_part2.as<double>(), c->d_ecb.as<int32_t>(),
                            c->d_offsets.as<int64_t>(), (int64_t)c->h_offsets.size() - 1, c->n_chunks, c->n_ev_chunks,
                            c->n_draw, c->d_lamg.p, c->d_K.as<int64_t>(), K, n_params, c->d_lnL.as<double>(),
                            c->d_lnxi.as<double>(), c->d_neff.as<double>(), c->d_flags.as<uint32_t>(),
                            c->d_grad.as<double>(), c->stream),
       "grad finalise");
    CK(cudaEventRecord(c->ev_t1, c->stream), "event");
    c->timed = true;
    CK(cudaMemcpyAsync(out_lnL, c->d_lnL.p, sizeof(double) * K, out_kind(mem), c->stream), "copy lnL");
    CK(cudaMemcpyAsync(out_grad, c->d_grad.p, sizeof(double) * K * n_params, out_kind(mem), c->stream), "copy grad");
    if (out_flags)
        CK(cudaMemcpyAsync(out_flags, c->d_flags.p, sizeof(uint32_t) * K, out_kind(mem), c->stream), "copy flags");
    if (mem == POP_MEM_HOST) CK(cudaStreamSynchronize(c->stream), "sync");
    return POP_OK;
}

int pop_cbc_load(pop_ctx* c, int n_det, int64_t M, double f0, double df, const double* data, const double* psd,
                 const double* hp, const double* hc, int mem)
{
    pop::TraceRange trace_("pop_cbc_load");
    if (!c) return POP_EINVAL;
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, "pop_cbc_load: bad mem");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    std::unique_ptr<CbcState> fresh;
    CbcState* st = c->cbc.get();
    if (!st) {
        fresh.reset(new CbcState());
        st = fresh.get();
    }
    const int rc = st->load(n_det, M, f0, df, data, psd, hp, hc, mem == POP_MEM_DEVICE, c->stream);
    if (rc != POP_OK) return fail(c, rc, st->err);
    if (fresh) c->cbc = std::move(fresh);
    return POP_OK;
}

int pop_cbc_loglik(pop_ctx* c, int64_t K, int n_params, const double* theta, int mode, double* out_lnL,
                   uint32_t* out_flags, int mem)
{
    pop::TraceRange trace_("pop_cbc_loglik");
    if (!c) return POP_EINVAL;
    if (!c->cbc) return fail(c, POP_ESTATE, "pop_cbc_loglik: load data first (pop_cbc_load)");
    CbcState& st = *c->cbc;
    if (n_params != 2 + 3 * st.n_det) return fail(c, POP_EINVAL, "pop_cbc_loglik: n_params must be 2 + 3 n_det");
    if (mode != POP_MODE_F64 && mode != POP_MODE_F32) return fail(c, POP_EINVAL, "pop_cbc_loglik: bad mode");
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, "pop_cbc_loglik: bad mem");
    if (K < 0 || K > (1LL << 24)) return fail(c, POP_EINVAL, "pop_cbc_loglik: K out of range");
    if (K == 0) return POP_OK;
    if (!theta || !out_lnL) return fail(c, POP_EINVAL, "pop_cbc_loglik: theta/out_lnL is NULL");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const int rc = st.run(K, theta, mem == POP_MEM_DEVICE, mode == POP_MODE_F64 ? 0 : 1, c->stream);
    if (rc != POP_OK) return fail(c, rc, st.err);
    CK(cudaMemcpyAsync(out_lnL, st.lnL.p, sizeof(double) * K, out_kind(mem), c->stream), "copy lnL");
    if (out_flags)
        CK(cudaMemcpyAsync(out_flags, st.flags.p, sizeof(uint32_t) * K, out_kind(mem), c->stream), "copy flags");
    if (mem == POP_MEM_HOST) CK(cudaStreamSynchronize(c->stream), "sync");
    return POP_OK;
}

int pop_cbc_last_ms(pop_ctx* c, double* sum_ms, double* total_ms)
{
    if (!c) return POP_EINVAL;
    if (!c->cbc || !c->cbc->timed) return fail(c, POP_ESTATE, "pop_cbc_last_ms: no pop_cbc_loglik yet");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaEventSynchronize(c->cbc->ev3), "event sync");
    float w = 0.f, t = 0.f;
    CK(cudaEventElapsedTime(&w, c->cbc->ev1, c->cbc->ev2), "elapsed");
    CK(cudaEventElapsedTime(&t, c->cbc->ev0, c->cbc->ev3), "elapsed");
    if (sum_ms) *sum_ms = w;
    if (total_ms) *total_ms = t;
    return POP_OK;
}

int pop_load_vt_grid(pop_ctx* c, int n_m1, const double* m1, int n_q, const double* q, const double* pdet, int mem)
{
    pop::TraceRange trace_("pop_load_vt_grid");
    if (!c) return POP_EINVAL;
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, "pop_load_vt_grid: bad mem");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    std::unique_ptr<GridVT> fresh;
    GridVT* g = c->grid.get();
    if (!g) {
        fresh.reset(new GridVT());
        g = fresh.get();
    }
    const int rc = g->load(n_m1, m1, n_q, q, pdet, mem == POP_MEM_DEVICE, c->stream);
    if (rc != POP_OK) return fail(c, rc, g->err_msg);
    if (fresh) c->grid = std::move(fresh);
    c->version++;
    return POP_OK;
}

int pop_set_xi_source(pop_ctx* c, int source)
{
    if (!c) return POP_EINVAL;
    if (source != POP_XI_INJECTIONS && source != POP_XI_GRID)
        return fail(c, POP_EINVAL, "pop_set_xi_source: source must be POP_XI_INJECTIONS or POP_XI_GRID");
    if (source == POP_XI_GRID && !c->grid) return fail(c, POP_ESTATE, "pop_set_xi_source: load a grid first");
    if (source != c->xi_source) {
        c->xi_source = source;
        c->version++;
    }
    return POP_OK;
}

int pop_xi_grid(pop_ctx* c, int64_t K, int n_params, const double* lambda, int mode, double* out_lnxi,
                uint32_t* out_flags, int mem)
{
    pop::TraceRange trace_("pop_xi_grid");
    if (!c) return POP_EINVAL;
    if (!c->grid) return fail(c, POP_ESTATE, "pop_xi_grid: load a grid first (pop_load_vt_grid)");
    if (K < 0 || K > (1LL << 24)) return fail(c, POP_EINVAL, "pop_xi_grid: K out of range");
    if (n_params != 11 && n_params != 12) return fail(c, POP_EINVAL, "pop_xi_grid: n_params must be 11 or 12");
    if (mode != POP_MODE_F64 && mode != POP_MODE_F32) return fail(c, POP_EINVAL, "pop_xi_grid: bad mode");
    if (!valid_mem(mem)) return fail(c, POP_EINVAL, "pop_xi_grid: bad mem");
    if (K == 0) return POP_OK;
    if (!lambda || !out_lnxi) return fail(c, POP_EINVAL, "pop_xi_grid: lambda/out_lnxi is NULL");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    GridVT& g = *c->grid;
    if (K > g.k_cap || g.slice <= 0) {
        CK(g.ensure(K), "grid scratch");
        c->version++;
    }
    if (K > g.k_cap_own) {
        DevBuf l, k, x, f;
        CK(l.alloc(sizeof(double) * K * 12), "cudaMalloc(lambda)");
        CK(k.alloc(sizeof(int64_t)), "cudaMalloc(K)");
        CK(x.alloc(sizeof(double) * K), "cudaMalloc(lnxi)");
        CK(f.alloc(sizeof(uint32_t) * K), "cudaMalloc(flags)");
        g.own_lambda.swap(l);
        g.own_K.swap(k);
        g.own_lnxi.swap(x);
        g.own_flags.swap(f);
        g.k_cap_own = K;
    }
    CK(cudaMemcpyAsync(g.own_lambda.p, lambda, sizeof(double) * K * n_params, in_kind(mem), c->stream), "copy lambda");
    set_k_kernel<<<1, 1, 0, c->stream>>>(g.own_K.as<int64_t>(), K);
    CK(cudaGetLastError(), "set K");
    const int m = mode == POP_MODE_F64 ? 0 : 1;
    CK(g.enqueue(m, g.own_lambda.as<double>(), n_params, g.own_K.as<int64_t>(), K, true, cudaEventRecordDefault,
                 c->stream), "grid selection term");
    CK(g.out_lnxi(g.own_lambda.as<double>(), n_params, g.own_K.as<int64_t>(), K, g.own_lnxi.as<double>(),
                  g.own_flags.as<uint32_t>(), c->stream), "grid output");
    CK(cudaMemcpyAsync(out_lnxi, g.own_lnxi.p, sizeof(double) * K, out_kind(mem), c->stream), "copy lnxi");
    if (out_flags)
        CK(cudaMemcpyAsync(out_flags, g.own_flags.p, sizeof(uint32_t) * K, out_kind(mem), c->stream), "copy flags");
    int bad = 0;
    CK(g.take_error(&bad, c->stream), "grid error word");  // synchronises the stream
    if (bad) return fail(c, POP_ETIMEOUT, "pop_xi_grid: a bounded wait of the grid contraction gave up");
    return POP_OK;
}

int pop_xi_grid_last_ms(pop_ctx* c, double* contraction_ms, double* total_ms)
{
    if (!c) return POP_EINVAL;
    if (!c->grid || c->grid->k_cap == 0) return fail(c, POP_ESTATE, "pop_xi_grid_last_ms: no grid evaluation yet");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaEventSynchronize(c->grid->ev3), "event sync");
    float w = 0.f, t = 0.f;
    CK(cudaEventElapsedTime(&w, c->grid->ev1, c->grid->ev2), "elapsed");
    CK(cudaEventElapsedTime(&t, c->grid->ev0, c->grid->ev3), "elapsed");
    if (contraction_ms) *contraction_ms = w;
    if (total_ms) *total_ms = t;
    return POP_OK;
}

int pop_set_tiling(pop_ctx* c, int mode, int lambda_tile, int block_threads, int blocks_per_sm)
{
    if (!c) return POP_EINVAL;
    if (mode != POP_MODE_F64 && mode != POP_MODE_F32) return fail(c, POP_EINVAL, "pop_set_tiling: bad mode");
    Tiling t{lambda_tile, block_threads, blocks_per_sm};
    if (!tiling_ok(mode, t)) return fail(c, POP_EINVAL, "pop_set_tiling: unsupported tiling");
    c->tiling[mode] = t;
    return POP_OK;
}

int pop_get_tiling(pop_ctx* c, int mode, int* lambda_tile, int* block_threads, int* blocks_per_sm)
{
    if (!c) return POP_EINVAL;
    if (mode != POP_MODE_F64 && mode != POP_MODE_F32) return fail(c, POP_EINVAL, "pop_get_tiling: bad mode");
    const Tiling& t = c->tiling[mode];
    if (lambda_tile) *lambda_tile = t.lambda_tile;
    if (block_threads) *block_threads = t.block_threads;
    if (blocks_per_sm) *blocks_per_sm = t.blocks_per_sm;
    return POP_OK;
}

int pop_set_graphs(pop_ctx* c, int enable)
{
    if (!c) return POP_EINVAL;
    c->use_graphs = enable != 0;
    return POP_OK;
}

int pop_last_kernel_ms(pop_ctx* c, double* weight_ms, double* total_ms)
{
    if (!c) return POP_EINVAL;
    if (!c->timed) return fail(c, POP_ESTATE, "pop_last_kernel_ms: no pop_loglik yet");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaEventSynchronize(c->ev_t1), "event sync");
    float w = 0.f, t = 0.f;
    CK(cudaEventElapsedTime(&w, c->ev_w0, c->ev_w1), "elapsed");
    CK(cudaEventElapsedTime(&t, c->ev_t0, c->ev_t1), "elapsed");
    if (weight_ms) *weight_ms = w;
    if (total_ms) *total_ms = t;
    return POP_OK;
}

int pop_autotune(pop_ctx* c, int mode, int64_t K, const char* cache_path)
{
    pop::TraceRange trace_("pop_autotune");
    if (!c) return POP_EINVAL;
    if (mode != POP_MODE_F64 && mode != POP_MODE_F32) return fail(c, POP_EINVAL, "pop_autotune: bad mode");
    if (c->ev.n == 0 || c->inj.n == 0) return fail(c, POP_ESTATE, "pop_autotune: load events and injections first");
    if (c->last_K < 1 || K < 1 || K > c->last_K)
        return fail(c, POP_ESTATE, "pop_autotune: needs a previous pop_loglik with at least K Lambda points");
    const int need = mode == POP_MODE_F64 ? POP_STORE_F64 : POP_STORE_F32;
    if (!(c->ev.storage & need) || !(c->inj.storage & need))
        return fail(c, POP_ESTATE, "pop_autotune: the loaded storage does not include this mode's precision");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    char key[512];
    snprintf(key, sizeof key, "%s|mode=%d|chunks=%d|ev_chunks=%d|K=%lld|dims=%d", c->device_name.c_str(), mode,
             c->n_chunks, c->n_ev_chunks, (long long)K, c->ev.n_dims);
    for (char* p = key; *p; ++p)
        if (*p == ' ') *p = '_';
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        Tiling best{};
        bool found = false;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k;
            Tiling t{};
            if (ls >> k >> t.lambda_tile >> t.block_threads >> t.blocks_per_sm && k == key && tiling_ok(mode, t)) {
                best = t;
                found = true;
            }
        }
        if (found) {
            c->tiling[mode] = best;
            return POP_OK;
        }
    }
    // FP64: Lambda per item x threads per block.  FP32: one Lambda per thread, 32 to 256 per block.
    const int tiles64[] = {1, 2, 4, 8, 16};
    const int threads64[] = {128, 256, 512};
    const int threads32[] = {32, 64, 128, 256};
    const Tiling saved = c->tiling[mode];
    const int n_params = c->last_params;
    int rc = build_chunks(c);
    if (rc != POP_OK) return rc;
    rc = ensure_scratch(c, K);
    if (rc != POP_OK) return rc;
    set_k_kernel<<<1, 1, 0, c->stream>>>(c->d_K.as<int64_t>(), K);
    CK(cudaGetLastError(), "set K");
    CK(launch_prologue(c->d_lambda.as<double>(), c->d_K.as<int64_t>(), c->k_cap, n_params, c->d_c64.as<LamF64>(),
                       c->d_c32.as<LamF32>(), c->d_zint.as<double>(), c->stream, c->d_ztab.as<double2>(),
                       c->d_exptab.as<double2>(), c->expc), "prologue");
    if (mode == POP_MODE_F32)
        CK(launch_lam_order(c->d_c32.as<LamF32>(), c->d_K.as<int64_t>(), nullptr, c->k_cap, c->d_order.as<int32_t>(),
                            c->d_nmc.as<int32_t>(), c->stream), "lambda order");
    float best_ms = 1e30f;
    Tiling best = saved;
    WorkDesc wd{c->d_chunks.as<Chunk>(), c->n_chunks, c->n_ev_chunks, c->ev.n_dims == 7};
    const int n_cand = mode == POP_MODE_F64 ? 15 : 4;
    for (int ci = 0; ci < n_cand; ++ci) {
        {
            const Tiling t = mode == POP_MODE_F64 ? Tiling{tiles64[ci / 3], threads64[ci % 3], 0}
                                                  : Tiling{threads32[ci], threads32[ci], 0};
            c->tiling[mode] = t;
            const int grid = grid_size(c, mode);
            float ms[3];
            for (int r = -1; r < 3; ++r) {
                CK(cudaEventRecord(c->ev_w0, c->stream), "event");
                cudaError_t e;
                if (mode == POP_MODE_F64) {
                    FeatF64 ev{c->ev.f64.as<double>(), c->ev.stride}, ij{c->inj.f64.as<double>(), c->inj.stride};
                    e = launch_weight_f64(t, grid, ev, ij, wd, c->d_c64.as<LamF64>(), c->d_K.as<int64_t>(),
                                          c->d_part.as<double>(), c->d_part2.as<double>(),
                                          c->d_exptab.as<double2>(), c->expc, c->d_queue.as<unsigned long long>(),
                                          c->stream);
                } else {
                    FeatF32 ev = c->ev.feat32();
                    FeatF32 ij = c->inj.feat32();
                    e = launch_weight_f32(t, grid, ev, ij, wd, c->d_c32.as<LamF32>(), c->d_order.as<int32_t>(),
                                          c->d_nmc.as<int32_t>(), c->d_queue.as<unsigned long long>(), c->k_cap, c->d_K.as<int64_t>(),
                                          c->d_part.as<double>(), c->d_part2.as<double>(), c->stream);
                }
                if (e != cudaSuccess) {
                    c->tiling[mode] = saved;
                    return cuda_fail(c, e, "autotune launch");
                }
                CK(cudaEventRecord(c->ev_w1, c->stream), "event");
                CK(cudaEventSynchronize(c->ev_w1), "event sync");
                if (r >= 0) CK(cudaEventElapsedTime(&ms[r], c->ev_w0, c->ev_w1), "elapsed");
            }
            std::sort(ms, ms + 3);
            if (ms[1] < best_ms) {
                best_ms = ms[1];
                best = t;
            }
        }
    }
    c->tiling[mode] = best;
    c->timed = false;
    if (cache_path) {
        std::ofstream out(cache_path, std::ios::app);
        out << key << " " << best.lambda_tile << " " << best.block_threads << " " << best.blocks_per_sm << "\n";
    }
    return POP_OK;
}

}  // extern "C"
