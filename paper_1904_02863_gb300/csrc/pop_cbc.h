// Single-event CBC likelihood (paper, Sec. "Single-event Likelihood
// acceleration", Eq. (cbclike)).  Internal to libpop.so.
//
//   ln L = sum_i sum_j [ -ln(2 pi S_ij) - (2/T) |d_ij - h_ij|^2 / S_ij ],
//   h_ij = A e^{i phi} (Fp_i hp_j + Fc_i hc_j) e^{-2 pi i f_j dt_i},  f_j = f0 + j df,  T = 1/df.
//
// With w = (2/T)/S, alpha_i = A e^{i phi} Fp_i, beta_i = A e^{i phi} Fc_i and
// e_ij = e^{-2 pi i f_j dt_i}, expanding |d - h|^2 gives
//
//   ln L = C + sum_i [ 2 Re(alpha_i SP_i + beta_i SQ_i)
//                      - |alpha_i|^2 Hpp_i - |beta_i|^2 Hcc_i - 2 Re(alpha_i conj(beta_i) Hpc_i) ]
//
// with the data constants C = sum_ij [-ln(2 pi S) - w |d|^2], Hpp_i = sum_j w |hp|^2,
// Hcc_i = sum_j w |hc|^2, Hpc_i = sum_j w hp conj(hc) (once, at load), and per
// parameter row the time-shifted sums SP_i = sum_j P_ij e_ij, SQ_i = sum_j Q_ij e_ij,
// P = w conj(d) hp, Q = w conj(d) hc: the only per-row work, one complex
// exponential and two complex multiply-adds per bin and detector.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pop_devbuf.h"

namespace pop {

struct CbcState {
    int n_det = 0;
    int64_t M = 0;
    double f0 = 0.0, df = 0.0;
    DevBuf pq64, pq32;  // [n_det][M] (P, Q) as double4 / float4: (Re P, Im P, Re Q, Im Q)
    double C = 0.0;     // sum_ij [-ln(2 pi S) - w |d|^2]
    DevBuf norms;       // [n_det][4] double: Hpp, Hcc, Re Hpc, Im Hpc
    // Per-call scratch.
    int64_t k_cap = 0;
    DevBuf theta, K_dev, rows, part, lnL, flags;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    bool timed = false;
    std::string err;

    CbcState() = default;
    CbcState(const CbcState&) = delete;
    CbcState& operator=(const CbcState&) = delete;
    ~CbcState();

    // Validate, copy and precompute (synchronous).  Pointers in host or device memory.
    int load(int n_det_, int64_t M_, double f0_, double df_, const double* data, const double* psd, const double* hp,
             const double* hc, bool on_device, cudaStream_t s);
    // ln L for K rows theta[K][2 + 3 n_det] (device), FP64 (mode 0) or FP32 (mode 1) sums.
    int run(int64_t K, const double* theta_in, bool theta_on_device, int mode, cudaStream_t s);
};

}  // namespace pop
