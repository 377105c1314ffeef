// Surrogate network for ln xi (internal; the C-ABI wrappers live in pop_api.cu).
//
// The paper announces a learned selection term that keeps spin effects in VT
// at no extra run-time cost (Sec. "Population acceleration", next to the Monte
// Carlo VT).  Here: normalised Lambda (12 inputs) -> 4 x 256 SiLU -> 2 outputs
// (standardised ln xi and ln N_eff), BF16 weights and activations on 5th-gen
// tensor cores (tcgen05.mma, FP32 accumulators in TMEM), FP32 master weights
// and Adam.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pop_devbuf.h"

namespace pop {

constexpr int MLP_IN = 12;
constexpr int MLP_HID = 256;
constexpr int MLP_OUT = 2;
constexpr int MLP_IN_PAD = 64;  // K of the input layer's GEMM (zero padded)
constexpr int MLP_LAYERS = 5;
// Flat FP32 parameter vector: W0 [256x12], b0, W1 [256x256], b1, W2, b2, W3, b3, W4 [2x256], b4.
constexpr int64_t MLP_N_PARAMS = (int64_t)MLP_HID * MLP_IN + MLP_HID + 3 * ((int64_t)MLP_HID * MLP_HID + MLP_HID) +
                                 (int64_t)MLP_OUT * MLP_HID + MLP_OUT;

// Layer offsets in the flat parameter vector.
__host__ __device__ constexpr int64_t off_w(int l)
{
    return l == 0 ? 0
                  : (int64_t)MLP_HID * MLP_IN + MLP_HID + (int64_t)(l - 1) * ((int64_t)MLP_HID * MLP_HID + MLP_HID);
}
__host__ __device__ constexpr int64_t off_b(int l)
{
    return off_w(l) +
           (l == 0 ? (int64_t)MLP_HID * MLP_IN : (l == 4 ? (int64_t)MLP_OUT * MLP_HID : (int64_t)MLP_HID * MLP_HID));
}

// Per-Lambda error model of the network's ln xi, from the held-out pairs: the pairs are split
// into ERR_BINS bins of equal count by the network's own ln N_eff prediction (the Monte Carlo
// scatter of the targets, ~1/sqrt(N_eff), is what the network cannot learn), and each bin keeps
// ERR_MARGIN times the largest |ln xi_net - ln xi-hat| of its pairs.  A Lambda uses the network
// only when N times its bin's error is within the budget (nats of ln L).
constexpr int ERR_BINS = 16;
constexpr double ERR_MARGIN = 1.25;
constexpr double DEFAULT_BUDGET_NATS = 0.25;

struct ErrTable {
    double edge[ERR_BINS - 1];  // increasing ln N_eff bin edges
    double err[ERR_BINS];       // error bound of ln xi per bin
};

__host__ __device__ inline double err_bound(const ErrTable& t, double ln_neff)
{
    int b = 0;
    for (int i = 0; i < ERR_BINS - 1; ++i) b += ln_neff >= t.edge[i] ? 1 : 0;
    return t.err[b];
}

// Whether the Monte Carlo xi is needed for one Lambda: untrusted network, Lambda outside the
// training box, a timed-out wait, a non-finite prediction, predicted N_eff < 4 N, or N times the
// error bound above the budget.  The same decision on the host (pop_xi_surrogate_infer) and on
// the device (inside pop_loglik).
__host__ __device__ inline bool need_monte_carlo(bool trusted, bool outside, bool timed_out, double lnxi,
                                                 double ln_neff, double n_events, double budget, const ErrTable& t)
{
    const bool ok = trusted && !outside && !timed_out && isfinite(lnxi) && exp(ln_neff) >= 4.0 * n_events &&
                    n_events * err_bound(t, ln_neff) <= budget;
    return !ok;
}

struct Surrogate {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // Normalisation: x = 2 (Lambda - lo) / (hi - lo) - 1; targets standardised with mu, sd.
    int n_params = 0;
    double lo[MLP_IN] = {}, hi[MLP_IN] = {};
    double mu[MLP_OUT] = {0, 0}, sd[MLP_OUT] = {1, 1};
    bool has_params = false;
    bool trained = false;
    bool trusted = false;
    double heldout_rmse = 0, heldout_mc_noise = 0, heldout_excess = 0;
    double target_seconds = 0, fit_seconds = 0;  // last training: target generation, fitting
    int64_t fit_rows = 0;                      // rows through forward + backward in the last fit
    ErrTable table{};                          // per-Lambda error model (held-out pairs)
    double budget = DEFAULT_BUDGET_NATS;       // largest N x error bound the gate accepts
    int64_t adam_step = 0;

    DevBuf params, adam_m, adam_v, grads;  // FP32 [MLP_N_PARAMS]
    DevBuf w0p, w[3], wt[3], w4f;          // BF16 GEMM copies (w0p [256x64]); w4f FP32 of the BF16-rounded W4
    DevBuf err_flag;                       // int: a bounded tcgen05 wait gave up
    int64_t cap = 0;                       // rows of the activation buffers
    DevBuf x0, z[4], h[4], y, dy, dz[2], dzt, ht, parts, dw0, red;
    CUtensorMap wmap[4];                   // TMA maps of w0p, w[0..2]: 256 x 64 BF16 tiles, 128-byte swizzle
    bool wmaps_ok = false;

    int init(int dev, cudaStream_t s);
    int ensure_rows(int64_t rows);
    int set_params_host(const float* flat);
    int get_params_host(float* flat);
    int init_params(uint64_t seed);
    int refresh_bf16();
    // Forward on rows of x0 (already normalised, [rows_pad x 64] BF16); outputs y [rows_pad x 2].
    int forward(int64_t rows_pad);
    // Loss gradients on the batch in x0 with targets t (device [rows x 2]); fills `grads`.
    int backward(int64_t rows, int64_t rows_pad, const float* t);
    int adam(float lr);
    int check_error();
    // Normalise K Lambda rows (device, row-major [K x P]) into dst (default x0, [pad128(K) x 64]);
    // outside[k] = 1 outside the box (may be NULL).
    int normalise(const double* lambda, int64_t K, int P, uint8_t* outside, __nv_bfloat16* dst = nullptr);

    // Inside pop_loglik (no host synchronisation, graph-capturable): for the k_cap rows of
    // d_lambda, need[k] = Monte Carlo xi required, lnxi[k], lnneff[k] from the network; rows
    // k >= *dK are left untouched.  ensure_gate(k_cap) must have run before.
    DevBuf outside;
    uint64_t version = 0;  // bumped when the parameters or the normalisation change
    int ensure_gate(int64_t k_cap);
    int enqueue_gate(const double* d_lambda, int64_t k_cap, int P, const int64_t* dK, double n_events, uint8_t* need,
                     double* lnxi, double* lnneff);

    // The inference forward in one launch (pop_mlp_fused.cu): rows [0, K) (K = *dK when dK is not
    // NULL, else K_cap) from Lambda rows (normalised in the kernel, outside[] set) or, when x0 is not
    // NULL, from normalised BF16 inputs [rows x 64]; y[rows x 2] when y is not NULL; with need
    // not NULL, also the gate's need / lnxi / lnneff.  No host synchronisation.
    int fused_forward(const double* d_lambda, int P, const __nv_bfloat16* x0, int64_t K_cap, const int64_t* dK,
                      float* y, uint8_t* outside, double n_events, uint8_t* need, double* lnxi, double* lnneff);
    int prepare_fused();  // tensor maps of the weight copies and the kernel's shared-memory size (init)
};

// TMA map of a row-major [rows x cols] BF16 matrix read in box_rows x 64-column tiles with the
// 128-byte swizzle (false when the driver refuses it).  cols x 2 bytes must be a multiple of 16.
bool make_tile_map(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows);

// Diagnostic: C[M x N] = A[M x K] B[N x K]^T on the tensor cores (FP32 out).
cudaError_t mlp_gemm_check(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K,
                           int* err, cudaStream_t s);
// x0/t rows = xall/tall rows idx[0..B) (zero padding up to rows_pad).
cudaError_t mlp_gather(const __nv_bfloat16* xall, const float* tall, const int64_t* idx, int64_t B, int64_t rows_pad,
                       __nv_bfloat16* x0, float* t, cudaStream_t s);

}  // namespace pop
