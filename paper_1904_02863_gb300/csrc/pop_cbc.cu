// Single-event CBC likelihood on the GPU (paper, Sec. "Single-event Likelihood
// acceleration", Eq. (cbclike)): the one-time data preparation, the per-row
// prologue, the time-shifted sums over frequency bins, and the finalise.
//
// Time shifts.  The factor e^{-2 pi i f_j dt} is e^{-2 pi i t_j} with t_j =
// f0 dt + j (df dt) turns.  Both terms are held modulo 1 as 64-bit fixed-point
// fractions of a turn, so t_j mod 1 is exact at any bin (integer multiply-add,
// no loss of phase at large f dt).  Each thread walks runs of RUN consecutive
// bins: the first exponential of a run comes from sincospi of the exact phase,
// the next ones from the recurrence e_{j+1} = e_j w, w = e^{-2 pi i df dt}.
//
// Work items are (detector, tile of TK rows, chunk of bins); every item writes
// its own partial sums (FP64), and the finalise adds them in a fixed order, so
// results repeat bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pop.h"
#include "pop_cbc.h"
#include "pop_f32x2.cuh"

namespace pop {

namespace {

constexpr int CBC_THREADS = 256;
constexpr int PREP_THREADS = 256;
constexpr int PREP_BLOCKS_MAX = 152 * 8;
constexpr double TWO_PI = 6.283185307179586476925;

template <class T>
struct CbcCfg;
// TK rows per work item; RUN bins per exact-phase anchor (the recurrence e <- e w between
// anchors adds about 3 roundings per product: RUN - 1 products).
// SUB bins' loads a thread issues together (their registers: SUB x 4 values).
// MIN_BLOCKS: resident blocks per SM that the register budget allows.  FP64: 3 (80 registers;
// a few values spill to L1 outside the bins' loop, and the extra warps keep the FP64 pipe busier:
// 0.85 of its peak against 0.83 with 2).  FP32: 2.
template <>
struct CbcCfg<double> {
    static constexpr int TK = 4;
    static constexpr int RUN = 32;
    static constexpr int SUB = 4;
    static constexpr int MIN_BLOCKS = 3;
};
template <>
struct CbcCfg<float> {
    static constexpr int TK = 8;
    static constexpr int RUN = 16;
    static constexpr int SUB = 8;
    static constexpr int MIN_BLOCKS = 2;
};

// Per (row, detector) constants.
struct alignas(16) CbcRow {
    double2 alpha, beta;   // A e^{i phi} Fp, A e^{i phi} Fc
    double2 w64;           // e^{-2 pi i df dt}
    float2 w32;
    unsigned long long a, b;  // f0 dt and df dt modulo 1, as 64-bit fractions of a turn
    int valid;
};

// x - floor(x) as a 64-bit fraction of a turn (exact: x's 53 bits fit in 64).
__device__ __forceinline__ unsigned long long turns_fixed(double x)
{
    const double fr = x - floor(x);        // [0, 1)
    const double hi = floor(fr * 4294967296.0);
    const double lo = (fr * 4294967296.0 - hi) * 4294967296.0;
    return ((unsigned long long)hi << 32) | (unsigned long long)lo;
}

__global__ void cbc_prologue_kernel(const double* __restrict__ theta, int n_det, double f0, double df,
                                    const int64_t* __restrict__ dK, CbcRow* __restrict__ rows,
                                    uint32_t* __restrict__ flags)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= *dK) return;
    const int P = 2 + 3 * n_det;
    const double* th = theta + k * P;
    bool ok = true;
    for (int p = 0; p < P; ++p) ok = ok && isfinite(th[p]);
    flags[k] = ok ? 0u : (uint32_t)POP_FLAG_INVALID_LAMBDA;
    double s, c;
    sincos(ok ? th[1] : 0.0, &s, &c);
    const double cre = ok ? th[0] * c : 0.0, cim = ok ? th[0] * s : 0.0;
    for (int i = 0; i < n_det; ++i) {
        CbcRow r;
        const double Fp = ok ? th[2 + 3 * i] : 0.0, Fc = ok ? th[3 + 3 * i] : 0.0, dt = ok ? th[4 + 3 * i] : 0.0;
        r.alpha = make_double2(cre * Fp, cim * Fp);
        r.beta = make_double2(cre * Fc, cim * Fc);
        const double bt = df * dt;
        double ws, wc;
        sincospi(2.0 * (bt - floor(bt)), &ws, &wc);
        r.w64 = make_double2(wc, -ws);
        r.w32 = make_float2((float)wc, (float)-ws);
        r.a = turns_fixed(f0 * dt);
        r.b = turns_fixed(bt);
        r.valid = ok;
        rows[k * n_det + i] = r;
    }
}

// e^{-2 pi i t} for t = the fixed-point turn fraction (signed, in [-1/2, 1/2)).  FP32:
// the angle 2 pi t lies in [-pi, pi), where the hardware sine and cosine (__sinf,
// __cosf) are within 2^-21.19 absolute; with the rounding of t to FP32 the anchor is
// within ~8 ulp of 1.
__device__ __forceinline__ void anchor(unsigned long long t, float& er, float& ei)
{
    const float x = (float)(int)(t >> 32) * (0x1p-31f * 3.14159265358979f);  // 2 pi t in [-pi, pi)
    er = __cosf(x);
    ei = -__sinf(x);
}

__device__ __forceinline__ void anchor(unsigned long long t, double& er, double& ei)
{
    const double x = (double)(long long)t * 0x1p-63;
    double s, c;
    sincospi(x, &s, &c);
    er = c;
    ei = -s;
}

}  // namespace

// (Re P, Im P, Re Q, Im Q) of one bin in FP64.
struct alignas(16) PQ64 {
    double pr, pi, qr, qi;
};

namespace {

template <class T>
struct Vec4T;
template <>
struct Vec4T<float> {
    using type = float4;
};
template <>
struct Vec4T<double> {
    using type = PQ64;
};

__device__ __forceinline__ void load_pq(const PQ64* p, double (&v)[4])
{
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 x = __ldg(q), y = __ldg(q + 1);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

__device__ __forceinline__ void load_pq(const float4* p, float (&v)[4])
{
    const float4 x = __ldg(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}

// Partial sums SP, SQ (as Re, Im, Re, Im) of one work item for TK rows.
template <class T>
__global__ void __launch_bounds__(CBC_THREADS, CbcCfg<T>::MIN_BLOCKS)
cbc_sum_kernel(const typename Vec4T<T>::type* __restrict__ pq, const CbcRow* __restrict__ rows, int n_det, int64_t M,
               int n_tiles, int n_chunks, int64_t CB, const int64_t* __restrict__ dK, double* __restrict__ part)
{
    constexpr int TK = CbcCfg<T>::TK;
    const int item = blockIdx.x;
    const int chunk = item % n_chunks;
    const int tile = (item / n_chunks) % n_tiles;
    const int det = item / (n_chunks * n_tiles);
    const int64_t K = *dK;
    const int64_t k0 = (int64_t)tile * TK;
    if (k0 >= K) return;
    __shared__ unsigned long long sa[TK], sb[TK];  // phases at f0 and per bin (read at the anchors)
    T wr[TK], wi[TK];
#pragma unroll
    for (int t = 0; t < TK; ++t) {
        const int64_t k = k0 + t < K ? k0 + t : k0;  // rows past K repeat row k0 (results unused)
        const CbcRow& r = rows[k * n_det + det];
        if (threadIdx.x == 0) {
            sa[t] = r.a;
            sb[t] = r.b;
        }
        if constexpr (sizeof(T) == 4) {
            wr[t] = r.w32.x;
            wi[t] = r.w32.y;
        } else {
            wr[t] = r.w64.x;
            wi[t] = r.w64.y;
        }
    }
    __syncthreads();
    T acc[TK][4];
#pragma unroll
    for (int t = 0; t < TK; ++t)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[t][c] = T(0);
    const int64_t j_begin = (int64_t)chunk * CB;
    const int64_t j_end = min(M, j_begin + CB);
    const typename Vec4T<T>::type* base = pq + (int64_t)det * M;
    constexpr int RUN_T = CbcCfg<T>::RUN;
    constexpr int SUB = CbcCfg<T>::SUB;
    // (P e, Q e) accumulated for every row; then e <- e w.
    auto step = [&](const T (&v)[4], T (&er)[TK], T (&ei)[TK]) {
#pragma unroll
        for (int t = 0; t < TK; ++t) {
            acc[t][0] = fma(v[0], er[t], fma(-v[1], ei[t], acc[t][0]));
            acc[t][1] = fma(v[0], ei[t], fma(v[1], er[t], acc[t][1]));
            acc[t][2] = fma(v[2], er[t], fma(-v[3], ei[t], acc[t][2]));
            acc[t][3] = fma(v[2], ei[t], fma(v[3], er[t], acc[t][3]));
            const T nr = fma(er[t], wr[t], -ei[t] * wi[t]);
            const T ni = fma(er[t], wi[t], ei[t] * wr[t]);
            er[t] = nr;
            ei[t] = ni;
        }
    };
    // A thread takes runs of RUN_T consecutive bins: one exact anchor per run, then the
    // recurrence, the bins in batches of SUB whose loads go out together.
    if constexpr (sizeof(T) == 4) {
        // FP32: rows (2p, 2p+1) in the halves of packed f32x2 registers, the bin's P and Q
        // broadcast to both halves; the same fmas as the scalar path, one instruction per pair.
        constexpr int TP = TK / 2;
        f2 a2[TP][4], w2r[TP], w2i[TP], w2n[TP];
#pragma unroll
        for (int q = 0; q < TP; ++q) {
#pragma unroll
            for (int c = 0; c < 4; ++c) a2[q][c] = 0ull;
            w2r[q] = pk(wr[2 * q], wr[2 * q + 1]);
            w2i[q] = pk(wi[2 * q], wi[2 * q + 1]);
            w2n[q] = pk(-wi[2 * q], -wi[2 * q + 1]);
        }
        auto step2 = [&](const float (&v)[4], f2 (&e2r)[TP], f2 (&e2i)[TP]) {
            const f2 b0 = bc(v[0]), b1 = bc(v[1]), n1 = bc(-v[1]), b2 = bc(v[2]), b3 = bc(v[3]), n3 = bc(-v[3]);
#pragma unroll
            for (int q = 0; q < TP; ++q) {
                a2[q][0] = fma2(b0, e2r[q], fma2(n1, e2i[q], a2[q][0]));
                a2[q][1] = fma2(b0, e2i[q], fma2(b1, e2r[q], a2[q][1]));
                a2[q][2] = fma2(b2, e2r[q], fma2(n3, e2i[q], a2[q][2]));
                a2[q][3] = fma2(b2, e2i[q], fma2(b3, e2r[q], a2[q][3]));
                const f2 nr = fma2(e2r[q], w2r[q], mul2(e2i[q], w2n[q]));
                const f2 ni = fma2(e2r[q], w2i[q], mul2(e2i[q], w2r[q]));
                e2r[q] = nr;
                e2i[q] = ni;
            }
        };
        for (int64_t j0 = j_begin + (int64_t)threadIdx.x * RUN_T; j0 < j_end; j0 += (int64_t)CBC_THREADS * RUN_T) {
            const int64_t jr = min(j_end, j0 + RUN_T);
            f2 e2r[TP], e2i[TP];
            {
                float er[TK], ei[TK];
#pragma unroll
                for (int t = 0; t < TK; ++t) anchor(sa[t] + (unsigned long long)j0 * sb[t], er[t], ei[t]);
#pragma unroll
                for (int q = 0; q < TP; ++q) {
                    e2r[q] = pk(er[2 * q], er[2 * q + 1]);
                    e2i[q] = pk(ei[2 * q], ei[2 * q + 1]);
                }
            }
            for (int64_t js = j0; js < jr; js += SUB) {
                if (jr - js >= SUB) {
                    float v[SUB][4];
#pragma unroll
                    for (int r = 0; r < SUB; ++r) load_pq(base + js + r, v[r]);
#pragma unroll
                    for (int r = 0; r < SUB; ++r) step2(v[r], e2r, e2i);
                } else {
                    for (int r = 0; r < (int)(jr - js); ++r) {
                        float v[4];
                        load_pq(base + js + r, v);
                        step2(v, e2r, e2i);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < TP; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) upk(a2[q][c], acc[2 * q][c], acc[2 * q + 1][c]);
    } else
    for (int64_t j0 = j_begin + (int64_t)threadIdx.x * RUN_T; j0 < j_end; j0 += (int64_t)CBC_THREADS * RUN_T) {
        const int64_t jr = min(j_end, j0 + RUN_T);
        T er[TK], ei[TK];
#pragma unroll
        for (int t = 0; t < TK; ++t) anchor(sa[t] + (unsigned long long)j0 * sb[t], er[t], ei[t]);
        for (int64_t js = j0; js < jr; js += SUB) {
            if (jr - js >= SUB) {
                T v[SUB][4];
#pragma unroll
                for (int r = 0; r < SUB; ++r) load_pq(base + js + r, v[r]);
#pragma unroll
                for (int r = 0; r < SUB; ++r) step(v[r], er, ei);
            } else {
                for (int r = 0; r < (int)(jr - js); ++r) {
                    T v[4];
                    load_pq(base + js + r, v);
                    step(v, er, ei);
                }
            }
        }
    }
    // Fixed-order block sum: warp shuffle tree in T, then the 8 warps in FP64.
    __shared__ double sh[CBC_THREADS / 32][TK * 4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < TK; ++t)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            T v = acc[t][c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sh[w][t * 4 + c] = (double)v;
        }
    __syncthreads();
    if (threadIdx.x < TK * 4) {
        double s = 0.0;
        for (int u = 0; u < CBC_THREADS / 32; ++u) s += sh[u][threadIdx.x];
        part[(int64_t)item * TK * 4 + threadIdx.x] = s;
    }
}

// ln L per row: C + sum_i [2 Re(alpha SP + beta SQ) - |alpha hp + beta hc|^2 terms].
template <int TK>
__global__ void cbc_finalise_kernel(const double* __restrict__ part, const CbcRow* __restrict__ rows,
                                    const double* __restrict__ norms, double C, int n_det, int n_tiles, int n_chunks,
                                    const int64_t* __restrict__ dK, double* __restrict__ lnL,
                                    const uint32_t* __restrict__ flags)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= *dK) return;
    if (flags[k]) {
        lnL[k] = -INFINITY;
        return;
    }
    const int tile = (int)(k / TK), t = (int)(k % TK);
    double sum = C;
    for (int i = 0; i < n_det; ++i) {
        double sp_r = 0.0, sp_i = 0.0, sq_r = 0.0, sq_i = 0.0;
        for (int c = 0; c < n_chunks; ++c) {
            const double* p = part + ((((int64_t)i * n_tiles + tile) * n_chunks + c) * TK + t) * 4;
            sp_r += p[0];
            sp_i += p[1];
            sq_r += p[2];
            sq_i += p[3];
        }
        const CbcRow& r = rows[k * n_det + i];
        const double2 al = r.alpha, be = r.beta;
        const double* nm = norms + 4 * i;
        const double cross = 2.0 * (al.x * sp_r - al.y * sp_i + be.x * sq_r - be.y * sq_i);
        const double a2 = al.x * al.x + al.y * al.y, b2 = be.x * be.x + be.y * be.y;
        // Re(alpha conj(beta) Hpc)
        const double abr = al.x * be.x + al.y * be.y, abi = al.y * be.x - al.x * be.y;
        const double hh = a2 * nm[0] + b2 * nm[1] + 2.0 * (abr * nm[2] - abi * nm[3]);
        sum += cross - hh;
    }
    lnL[k] = sum;
}

// Data preparation: P, Q per bin and the per-block partial sums of the constants
// (c = -ln(2 pi S) - w |d|^2, w |hp|^2, w |hc|^2, w hp conj(hc)) in FP64.
__global__ void __launch_bounds__(PREP_THREADS)
cbc_prep_kernel(const double* __restrict__ data, const double* __restrict__ psd, const double* __restrict__ hp,
                const double* __restrict__ hc, int n_det, int64_t M, double df, PQ64* __restrict__ pq64,
                float4* __restrict__ pq32, double* __restrict__ bpart, int* __restrict__ bad)
{
    const int det = blockIdx.y;
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t j = blockIdx.x * (int64_t)PREP_THREADS + threadIdx.x; j < M; j += (int64_t)gridDim.x * PREP_THREADS) {
        const int64_t ij = (int64_t)det * M + j;
        const double S = psd[ij];
        const double dr = data[2 * ij], di = data[2 * ij + 1];
        const double pr = hp[2 * j], pi = hp[2 * j + 1], cr = hc[2 * j], ci = hc[2 * j + 1];
        if (!(isfinite(S) && S > 0.0 && isfinite(dr) && isfinite(di) && isfinite(pr) && isfinite(pi) &&
              isfinite(cr) && isfinite(ci))) {
            atomicExch(bad, 1);
            pq64[ij] = PQ64{0.0, 0.0, 0.0, 0.0};
            pq32[ij] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const double w = 2.0 * df / S;
        // P = w conj(d) hp, Q = w conj(d) hc
        const double Pr = w * (dr * pr + di * pi), Pi = w * (dr * pi - di * pr);
        const double Qr = w * (dr * cr + di * ci), Qi = w * (dr * ci - di * cr);
        pq64[ij] = PQ64{Pr, Pi, Qr, Qi};
        pq32[ij] = make_float4((float)Pr, (float)Pi, (float)Qr, (float)Qi);
        s[0] += -log(TWO_PI * S) - w * (dr * dr + di * di);
        s[1] += w * (pr * pr + pi * pi);
        s[2] += w * (cr * cr + ci * ci);
        s[3] += w * (pr * cr + pi * ci);  // Re(hp conj(hc))
        s[4] += w * (pi * cr - pr * ci);  // Im(hp conj(hc))
    }
    __shared__ double sh[PREP_THREADS / 32][5];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int c = 0; c < 5; ++c) {
        double v = s[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int u = 0; u < PREP_THREADS / 32; ++u) v += sh[u][threadIdx.x];
        bpart[((int64_t)det * gridDim.x + blockIdx.x) * 5 + threadIdx.x] = v;
    }
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

CbcState::~CbcState()
{
    for (cudaEvent_t e : {ev0, ev1, ev2, ev3})
        if (e) cudaEventDestroy(e);
}

int CbcState::load(int nd, int64_t m, double f0_, double df_, const double* data, const double* psd,
                   const double* hp, const double* hc, bool on_device, cudaStream_t s)
{
    auto fail = [&](int st, const char* msg) {
        err = msg;
        return st;
    };
    if (nd < 1 || nd > 64 || m < 1 || m > (int64_t(1) << 30)) return fail(POP_EINVAL, "pop_cbc_load: bad n_det or M");
    if (!std::isfinite(f0_) || !(df_ > 0.0) || !std::isfinite(df_)) return fail(POP_EINVAL, "pop_cbc_load: bad f0/df");
    if (!data || !psd || !hp || !hc) return fail(POP_EINVAL, "pop_cbc_load: NULL pointer");
    DevBuf d64, d32, nrm, tmp, bp, dbad;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    const int64_t nm = (int64_t)nd * m;
    if (!ok(d64.alloc(sizeof(PQ64) * nm)) || !ok(d32.alloc(sizeof(float4) * nm)) ||
        !ok(nrm.alloc(sizeof(double) * 4 * nd)) || !ok(dbad.alloc(sizeof(int))))
        return fail(POP_ENOMEM, "pop_cbc_load: device allocation failed");
    const double *ddata = data, *dpsd = psd, *dhp = hp, *dhc = hc;
    if (!on_device) {
        const size_t bytes = sizeof(double) * (size_t)(2 * nm + nm + 4 * m);
        if (!ok(tmp.alloc(bytes))) return fail(POP_ENOMEM, "pop_cbc_load: device allocation failed");
        double* t = tmp.as<double>();
        bool c = ok(cudaMemcpyAsync(t, data, sizeof(double) * 2 * nm, cudaMemcpyHostToDevice, s)) &&
                 ok(cudaMemcpyAsync(t + 2 * nm, psd, sizeof(double) * nm, cudaMemcpyHostToDevice, s)) &&
                 ok(cudaMemcpyAsync(t + 3 * nm, hp, sizeof(double) * 2 * m, cudaMemcpyHostToDevice, s)) &&
                 ok(cudaMemcpyAsync(t + 3 * nm + 2 * m, hc, sizeof(double) * 2 * m, cudaMemcpyHostToDevice, s));
        if (!c) return fail(POP_ECUDA, "pop_cbc_load: copy to the device failed");
        ddata = t;
        dpsd = t + 2 * nm;
        dhp = t + 3 * nm;
        dhc = t + 3 * nm + 2 * m;
    }
    const int blocks = (int)std::min<int64_t>(PREP_BLOCKS_MAX / nd + 1, (m + PREP_THREADS - 1) / PREP_THREADS);
    if (!ok(bp.alloc(sizeof(double) * 5 * nd * blocks)) || !ok(cudaMemsetAsync(dbad.p, 0, sizeof(int), s)))
        return fail(POP_ENOMEM, "pop_cbc_load: device allocation failed");
    cbc_prep_kernel<<<dim3(blocks, nd), PREP_THREADS, 0, s>>>(ddata, dpsd, dhp, dhc, nd, m, df_, d64.as<PQ64>(),
                                                              d32.as<float4>(), bp.as<double>(), dbad.as<int>());
    if (!ok(cudaGetLastError())) return fail(POP_ECUDA, "pop_cbc_load: prep kernel launch failed");
    std::vector<double> hb((size_t)5 * nd * blocks);
    int hbad = 0;
    if (!ok(cudaMemcpyAsync(hb.data(), bp.p, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaMemcpyAsync(&hbad, dbad.p, sizeof(int), cudaMemcpyDeviceToHost, s)) || !ok(cudaStreamSynchronize(s)))
        return fail(POP_ECUDA, "pop_cbc_load: prep kernel failed");
    if (hbad) return fail(POP_EINVAL, "pop_cbc_load: psd must be finite and > 0, data and templates finite");
    // Fixed-order combine of the block partials (FP64, host).
    double c_sum = 0.0;
    std::vector<double> hn((size_t)4 * nd, 0.0);
    for (int i = 0; i < nd; ++i) {
        double v[5] = {0, 0, 0, 0, 0};
        for (int bl = 0; bl < blocks; ++bl)
            for (int c = 0; c < 5; ++c) v[c] += hb[((size_t)i * blocks + bl) * 5 + c];
        c_sum += v[0];
        for (int c = 0; c < 4; ++c) hn[4 * i + c] = v[1 + c];
    }
    if (!ok(cudaMemcpy(nrm.p, hn.data(), sizeof(double) * hn.size(), cudaMemcpyHostToDevice)))
        return fail(POP_ECUDA, "pop_cbc_load: copy failed");
    if (!ev0 && (!ok(cudaEventCreate(&ev0)) || !ok(cudaEventCreate(&ev1)) || !ok(cudaEventCreate(&ev2)) ||
                 !ok(cudaEventCreate(&ev3))))
        return fail(POP_ECUDA, "pop_cbc_load: cudaEventCreate failed");
    pq64.swap(d64);
    pq32.swap(d32);
    norms.swap(nrm);
    n_det = nd;
    M = m;
    f0 = f0_;
    df = df_;
    C = c_sum;
    k_cap = 0;  // per-call scratch depends on n_det
    timed = false;
    return POP_OK;
}

int CbcState::run(int64_t K, const double* theta_in, bool theta_on_device, int mode, cudaStream_t s)
{
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    const int TK = mode == 0 ? CbcCfg<double>::TK : CbcCfg<float>::TK;
    const int RUN = mode == 0 ? CbcCfg<double>::RUN : CbcCfg<float>::RUN;
    const int n_tiles = (int)((K + TK - 1) / TK);
    // Chunks of the bins (multiples of the run).  The items are alike, so a launch lasts
    // ceil(items / resident blocks) item times: the chunk count is the one whose waves times a
    // thread's bins (plus a per-item cost for the block sum, as bins) is least.
    int occ = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, mode == 0 ? (const void*)cbc_sum_kernel<double> : (const void*)cbc_sum_kernel<float>, CBC_THREADS, 0);
    const int64_t slots = (int64_t)std::max(occ, 1) * std::max(sms, 1);
    const int64_t per_chunk = (int64_t)n_det * n_tiles;
    constexpr int64_t ITEM_COST_BINS = 8;
    int64_t CB = round_up(M, (int64_t)RUN), best = INT64_MAX;
    for (int64_t n = 1; n <= 4 * slots / std::max<int64_t>(per_chunk, 1) + 16; ++n) {
        const int64_t cb = round_up((M + n - 1) / n, (int64_t)RUN);
        const int64_t nc = (M + cb - 1) / cb;
        const int64_t waves = (per_chunk * nc + slots - 1) / slots;
        const int64_t cost = waves * (round_up(cb, (int64_t)RUN * CBC_THREADS) / CBC_THREADS + ITEM_COST_BINS);
        if (cost < best) {
            best = cost;
            CB = cb;
        }
    }
    const int n_chunks = (int)((M + CB - 1) / CB);
    const int64_t n_items = (int64_t)n_det * n_tiles * n_chunks;
    const int P = 2 + 3 * n_det;
    if (K > k_cap || part.bytes < sizeof(double) * 4 * 8 * (size_t)n_items) {
        const int64_t cap = std::max<int64_t>(K, k_cap);
        const int64_t max_items = (int64_t)n_det * ((cap + 3) / 4) * n_chunks * 2;  // covers both modes
        DevBuf th, kd, rw, pt, ln, fl;
        if (!ok(th.alloc(sizeof(double) * P * cap)) || !ok(kd.alloc(sizeof(int64_t))) ||
            !ok(rw.alloc(sizeof(CbcRow) * n_det * cap)) || !ok(pt.alloc(sizeof(double) * 4 * 8 * max_items)) ||
            !ok(ln.alloc(sizeof(double) * cap)) || !ok(fl.alloc(sizeof(uint32_t) * cap))) {
            err = "pop_cbc_loglik: device allocation failed";
            return POP_ENOMEM;
        }
        theta.swap(th);
        K_dev.swap(kd);
        rows.swap(rw);
        part.swap(pt);
        lnL.swap(ln);
        flags.swap(fl);
        k_cap = cap;
    }
    if (n_items > (int64_t)INT32_MAX) {
        err = "pop_cbc_loglik: too many work items";
        return POP_EINVAL;
    }
    const bool good =
        ok(cudaEventRecord(ev0, s)) &&
        ok(cudaMemcpyAsync(theta.p, theta_in, sizeof(double) * P * K,
                           theta_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s)) &&
        ok(cudaMemcpyAsync(K_dev.p, &K, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (!good) {
        err = "pop_cbc_loglik: copy failed";
        return POP_ECUDA;
    }
    cbc_prologue_kernel<<<(unsigned)((K + 127) / 128), 128, 0, s>>>(theta.as<double>(), n_det, f0, df,
                                                                     K_dev.as<int64_t>(), rows.as<CbcRow>(),
                                                                     flags.as<uint32_t>());
    cudaEventRecord(ev1, s);
    if (mode == 0)
        cbc_sum_kernel<double><<<(unsigned)n_items, CBC_THREADS, 0, s>>>(
            pq64.as<PQ64>(), rows.as<CbcRow>(), n_det, M, n_tiles, n_chunks, CB, K_dev.as<int64_t>(),
            part.as<double>());
    else
        cbc_sum_kernel<float><<<(unsigned)n_items, CBC_THREADS, 0, s>>>(
            pq32.as<float4>(), rows.as<CbcRow>(), n_det, M, n_tiles, n_chunks, CB, K_dev.as<int64_t>(),
            part.as<double>());
    cudaEventRecord(ev2, s);
    const unsigned fb = (unsigned)((K + 127) / 128);
    if (mode == 0)
        cbc_finalise_kernel<CbcCfg<double>::TK><<<fb, 128, 0, s>>>(part.as<double>(), rows.as<CbcRow>(),
                                                                   norms.as<double>(), C, n_det, n_tiles, n_chunks,
                                                                   K_dev.as<int64_t>(), lnL.as<double>(),
                                                                   flags.as<uint32_t>());
    else
        cbc_finalise_kernel<CbcCfg<float>::TK><<<fb, 128, 0, s>>>(part.as<double>(), rows.as<CbcRow>(),
                                                                  norms.as<double>(), C, n_det, n_tiles, n_chunks,
                                                                  K_dev.as<int64_t>(), lnL.as<double>(),
                                                                  flags.as<uint32_t>());
    cudaEventRecord(ev3, s);
    if (!ok(cudaGetLastError())) {
        err = "pop_cbc_loglik: kernel launch failed";
        return POP_ECUDA;
    }
    timed = true;
    return POP_OK;
}

}  // namespace pop
