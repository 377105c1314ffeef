// Internal types shared by the host runtime (pop_api.cu) and the kernels
// (pop_kernels.cu).  Nothing here is part of the public C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pop.h"
#include "pop_ff.cuh"
#include "pop_math.cuh"

namespace pop {

// Lambda parameter indices in the C-ABI row order.
enum { P_ALPHA, P_BETA, P_MMIN, P_MMAX, P_LAM, P_MPP, P_SIGPP, P_ACHI, P_BCHI, P_XIT, P_SIGT, P_KAPPA };

// Packed per-sample feature rows (structure of arrays, row r at base + r*stride).
// FP64 layout rows: natural logs.  FP32 layout rows: base-2 logs (so every
// exponential is one ex2), and m2 kept in a separate FP64 row for the exact
// q-support test.
enum { F_LM1, F_M1, F_LQ, F_SA, F_SB, F_DC, F_NLPI, F_LZ1, F_M2, F_INVM1, F_COUNT64 = 10 };
// FP32 layout: the same first eight rows, then the low part of log2 m1
// (log2 m1 = row F_LM1 + row F32_LM1LO to ~1e-15), so that the q
// normalisation (1+beta) log2(mmin/m1) keeps its relative accuracy as m1 -> mmin.
enum { F32_LM1LO = 8, F_COUNT32 = 9 };

// Sentinel for ln 0 in the spin-magnitude and z logs: finite, so that a zero
// exponent gives 0 * sentinel = 0 (0^0 = 1) and a positive one underflows.
constexpr double LOG_ZERO = -1e30;

// Per-Lambda constants of the FP64 weight (natural-log units).
struct alignas(16) LamF64 {
    int64_t mmin_bits;   // bit pattern of mmin (+inf when Lambda is invalid)
    int64_t mmax_bits;   // bit pattern of mmax
    double nalpha;       // -alpha
    double cpl;          // ln|1+beta| - 2 ln B - ln I + ln((1-lam) C_pl)
    double mu;           // mpp
    double nh;           // -1 / (2 sigpp^2)
    double cg;           // ln|1+beta| - 2 ln B - ln I + ln(lam C_g)
    double beta;         // q exponent
    double ac, bc;       // alpha_chi - 1, beta_chi - 1
    double km1;          // kappa - 1 (0 without redshift)
    double b1;           // 1 + beta
    double mmin;         // mmin (for (mmin - m1)/m1 near the lower mass edge)
    double lmmin;        // ln mmin
    double kq;           // 1 + beta, or 1 when beta == -1
    double kqlmmin;      // kq ln mmin: u = kq ln(mmin/m1) = fma(-kq, ln m1, kqlmmin)
    double nht;          // -1 / (2 sigma_t^2)
    double ct;           // ln(xi_t C_t^2)
    double t0;           // (1 - xi_t) / 4
    double gs;           // 1 / (sqrt2 sigpp): the Gaussian exponent is -y^2, y = fma(m1, gs, gc)
    double gc;           // -mpp gs
    // The mass mixture with the larger of its two constants factored out into the tilt term:
    // w = [e^(aE - alpha ln m1) + rmix e^(aE - y^2)] (t0m + e^(ctm - dc/(2 sigma_t^2))) / den when
    // cpl >= cg (mix_swap 0), the two exponentials' roles exchanged otherwise; cmax = max(cpl, cg).
    double rmix;         // e^(min(cpl, cg) - cmax), in [0, 1]
    double t0m;          // e^cmax t0
    double ctm;          // ct + cmax
    int32_t beta_m1;     // beta == -1: q normalisation is ln(m1/mmin)
    int32_t valid;
    int32_t mix_swap;    // cg > cpl: rmix scales the power-law exponential
};

// Per-Lambda constants of the FP32 weight (base-2 units).
struct alignas(16) LamF32 {
    int64_t mmin_bits;   // FP64 bit pattern of mmin, for the exact m2 >= mmin test
    int64_t mmax_bits;   // FP64 bit pattern of mmax, for the exact m1 <= mmax test of the fix-up
    float thr_hi;        // rd32(mmax): m1 <= mmax implies rd32(m1) <= thr_hi; the converse fails
                         // only for m1 in (mmax, next float above thr_hi), which the fix-up removes
    float nalpha, cpl, mu, nh, cg, beta, ac, bc, km1;
    // q normalisation exponent u = b1 ((lmmin - lm1) + (lmmin_lo - lm1_lo)) in base 2,
    // evaluated as fma(b1, lmmin - lm1, fma(nb1, lm1_lo, b1lmmin_lo)); with
    // beta = -1, b1 = 1 and the normalisation is -u.
    float b1, nb1, lmmin, b1lmmin_lo;
    float nht, ct, t0;
    int32_t beta_m1;
    int32_t valid;
};

// One work chunk: a contiguous run of samples of one event, or of injections.
struct Chunk {
    int64_t start;       // first sample in its feature block
    int32_t len;         // samples in the chunk (>= 1)
    int32_t inj;         // 0 = event chunk, 1 = injection chunk
};

struct FeatF64 {
    const double* base;  // [F_COUNT64][stride]
    int64_t stride;
};

constexpr int M1MAX_BLOCK = 64;  // samples per block of FeatF32::m1max

struct FeatF32 {
    const float* base;     // [F_COUNT32][stride]; row F_M1 holds rd32(m1) (rounded toward -inf)
    const double* m2;      // [stride]: fl64(q m1)
    const double* m1d;     // [stride]: m1 in FP64 (0 outside the Lambda-independent support)
    const double* m1sort;  // [n]: m1d of the whole set in increasing order
    const uint2* m1pos;    // [n]: (position, chunk index within the set) of each m1sort entry
    const float* m1max;    // [ceil(n / M1MAX_BLOCK)]: the largest rd32(m1) of each block of samples
    int64_t n;
    int64_t stride;
};

// Everything the weight kernel needs about the loaded data.
struct WorkDesc {
    const Chunk* chunks;     // [n_chunks]: event chunks first, then injection chunks
    int32_t n_chunks;
    int32_t n_ev_chunks;
    int32_t has_z;
};

// Launch-time options of the weight kernels.
struct Tiling {
    int lambda_tile;     // Lambda points per work item
    int block_threads;   // threads per block
    int blocks_per_sm;   // 0 = occupancy maximum
};

// ---------------------------------------------------------------- kernel launchers
// All launch on `s` and return the launch error (cudaSuccess when queued).
cudaError_t launch_pack_f64(const double* theta, const double* prior, const int64_t* perm, int64_t n, int n_dims,
                            double* feat, int64_t stride, unsigned long long* bad, cudaStream_t s);
cudaError_t launch_pack_f32(const double* theta, const double* prior, const int64_t* perm, int64_t n, int n_dims,
                            float* feat, double* m2, double* m1d, int64_t stride, unsigned long long* bad,
                            cudaStream_t s);
// m1max[b] = the largest rd32(m1) (feature row F_M1 of the packed FP32 features) over samples
// [M1MAX_BLOCK b, M1MAX_BLOCK (b + 1)) of the n.
cudaError_t launch_m1_blockmax(const float* feat, int64_t stride, int64_t n, float* m1max, cudaStream_t s);
// ztab (REDSHIFT_NODES entries, build_z_table) and exptab make the redshift trapezoid one
// table-driven exponential per node; with ztab NULL it is evaluated directly.
constexpr int REDSHIFT_NODES = 1024;
// zint: device scratch of K_cap doubles for the redshift normalisation (used, and required,
// when n_params == 12).
cudaError_t launch_prologue(const double* lambda, const int64_t* dK, int64_t K_cap, int n_params,
                            LamF64* c64, LamF32* c32, double* zint, cudaStream_t s, const double2* ztab = nullptr,
                            const double2* exptab = nullptr, ExpConsts kc = ExpConsts{});
// Host: node i of the redshift trapezoid on [0, 2]: (ln(1 + z_i), w_i z_i^2), w = 1/2 at the ends.
void build_z_table(double2* tab);
// The FP64 weight kernel keeps the 2^(j/2048) table of its exponentials in dynamic shared memory.
constexpr int WEIGHT_F64_DYN_SMEM = EXP_TABLE_SIZE * (int)sizeof(double2);
// The weight kernels take their work items from *queue, which each launcher zeroes (a memset
// on the stream) before the launch.
cudaError_t launch_weight_f64(const Tiling& t, int grid, FeatF64 ev, FeatF64 inj, WorkDesc wd,
                              const LamF64* lam, const int64_t* dK, double* part, double* part2,
                              const double2* exptab, ExpConsts kc, unsigned long long* queue, cudaStream_t s);
// Evaluates the FP64 weight kernel's exp (fn 0), expm1 (fn 1) or reciprocal (fn 2) on x[n].
cudaError_t launch_math_check(int fn, int64_t n, const double* x, double* y, const double2* exptab, ExpConsts kc,
                              const LogEntry* logtab, LogConsts logc, cudaStream_t s);
// Host: the 2^(j/2048) table (hi, lo) and the reduction constants, in extended precision.
void build_exp_table(double2* tab, ExpConsts* kc);
// log_tab's table and constants, from long double arithmetic.
void build_log_table(LogEntry* tab, LogConsts* k);
// Selection term from the surrogate (all NULL when the Monte Carlo xi is used for every Lambda):
// need_mc[k] = 1 keeps the Monte Carlo xi for Lambda k, else ln xi = lnxi[k], N_eff = neff[k].
struct SurrogateXi {
    const uint8_t* need_mc;
    const double* lnxi;
    const double* neff;
};
// FP32 weight kernel: one Lambda per thread, lambda_tile == block_threads Lambda per work item.
// order[0, K) and order[K_cap, K_cap + *n_mc) are the Lambda of the event and injection items in
// lane order (launch_lam_order); only the first *n_mc of the injection order get injection items.
cudaError_t launch_weight_f32(const Tiling& t, int grid, FeatF32 ev, FeatF32 inj, WorkDesc wd,
                              const LamF32* lam, const int32_t* order, const int32_t* n_mc,
                              unsigned long long* queue, int64_t K_cap, const int64_t* dK, double* part,
                              double* part2, cudaStream_t s);
// After launch_weight_f32: removes from the partials the samples that the FP32 upper-edge test
// kept although m1 > mmax (one thread per Lambda; need_mc as for the weight kernel, or NULL).
cudaError_t launch_upper_edge_fixup(FeatF32 ev, FeatF32 inj, WorkDesc wd, const LamF32* lam,
                                    const uint8_t* need_mc, int64_t K_cap, const int64_t* dK, double* part,
                                    double* part2, cudaStream_t s);
// Float-float weight kernel (POP_MODE_FF): weight_ff_threads() Lambda per block, one per thread, with the
// lane order of launch_lam_order (need_mc NULL); fftab = 2^(j/2048) as FP32 (hi, lo) pairs.
const void* weight_ff_fn(bool has_z);
int weight_ff_threads();
cudaError_t launch_weight_ff(int grid, FeatF64 ev, FeatF64 inj, WorkDesc wd, const LamF64* lam, const int32_t* order,
                             const int32_t* n_mc, unsigned long long* queue, int64_t K_cap, const int64_t* dK,
                             double* part, double* part2, const float2* fftab, FFConsts kc, cudaStream_t s);
// Evaluates the float-float functions on x[n] (pairs of x packed as the kernel packs samples), each
// result widened to hi + lo in FP64: fn 3 exp, 4 expm1 (series below |x| = 1/16), 5 reciprocal,
// 6 square, 7 the exact square of the FP32 hi part (packed fma error term).
cudaError_t launch_ff_math_check(int fn, int64_t n, const double* x, double* y, const float2* fftab, FFConsts kc,
                                 cudaStream_t s);
// Host: the FP32 (hi, lo) table of 2^(j/2048) and the reduction constants, in extended precision.
void build_ff_table(float2* tab, FFConsts* kc);
// Lane order of the FP32 weight kernel: Lambda by mmin; for the injection items the Lambda with
// need_mc[k] != 0 first (all K when need_mc is NULL), their number in *n_mc.  order[2 K_cap].
cudaError_t launch_lam_order(const LamF32* lam, const int64_t* dK, const uint8_t* need_mc, int64_t K_cap,
                             int32_t* order, int32_t* n_mc, cudaStream_t s);
cudaError_t launch_finalise(const double* part, const double* part2, const int32_t* ev_chunk_begin,
                            const int64_t* offsets, int64_t n_events, int32_t n_chunks, int32_t n_ev_chunks,
                            int64_t n_draw, const LamF64* lam, const int64_t* dK, int64_t K_cap,
                            double* lnL, double* lnxi, double* neff, uint32_t* flags, cudaStream_t s,
                            SurrogateXi sx = SurrogateXi{nullptr, nullptr, nullptr},
                            const double* grid_xi = nullptr,  // xi per Lambda from the grid (N_eff = +inf)
                            double* parts = nullptr,          // [K][3]: sum_i ln(S_i/n_i), sum w, sum w^2
                            const LogEntry* logtab = nullptr,  // table of log_tab (NULL: the library's log)
                            LogConsts logc = LogConsts{0.0, 0.0},
                            const double* inv_n = nullptr);   // 1/n_i [N] (NULL: formed in the kernel)

// Gradient of ln L (pop_grad.cu): per-Lambda constants (lam_grad_bytes() each), the
// weight-and-derivative sums per (chunk, Lambda) ([K][n_chunks][13] doubles, plus the
// injection sum w^2 in part2 as for ln L), and the finalise with grad[K][n_params].
size_t lam_grad_bytes();
cudaError_t launch_grad_prologue(const double* lambda, const int64_t* dK, int64_t K_cap, int n_params, void* lam_g,
                                 cudaStream_t s, const double2* ztab, const double2* exptab, ExpConsts kc);
cudaError_t launch_grad_weight(int grid, FeatF64 ev, FeatF64 inj, WorkDesc wd, const void* lam_g, const int64_t* dK,
                               int n_params, double* part, double* part2, const double2* exptab, ExpConsts kc,
                               unsigned long long* queue, cudaStream_t s);
cudaError_t launch_grad_finalise(const double* part, const double* part2, const int32_t* ecb, const int64_t* off,
                                 int64_t n_events, int32_t n_chunks, int32_t n_ev_chunks, int64_t n_draw,
                                 const void* lam_g, const int64_t* dK, int64_t K_cap, int n_params, double* lnL,
                                 double* lnxi, double* neff, uint32_t* flags, double* grad, cudaStream_t s);
int grad_grid_size(int sm_count);

// Kernel function of a tiling (nullptr when that instantiation does not exist).
const void* weight_f64_fn(const Tiling& t, bool has_z);
const void* weight_f32_fn(const Tiling& t, bool has_z);

}  // namespace pop
