// Selection term on a regular (m1, q) grid (paper, Sec. "Population
// acceleration": VT evaluated on a regular grid with GPU acceleration, limited
// to a low-dimensional space, no spin effects).  Internal to libpop.so.
//
// With trapezoid weights wa (m1 nodes) and wq (q nodes) and the detection
// probability pdet at the nodes,
//   xi_grid(Lambda) = sum_a sum_b wa_a wq_b p(m1_a | Lambda) p(q_b | m1_a, Lambda) pdet[a, b]
//                   = sum_a W_a(Lambda) sum_{b = b0(a, Lambda)}^{nb - 1} pdet[a, b] U_b(Lambda)
// where U_b = wq_b q_b^beta, W_a = wa_a p(m1_a) (1+beta) / (1 - (mmin/m1_a)^(1+beta))
// (1 / ln(m1_a/mmin) when beta = -1), nb = number of q nodes <= 1 and b0 the
// first q node with fl64(q_b m1_a) >= mmin.  The inner sum is a masked
// contraction over the nodes; it is all of the work.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pop_devbuf.h"
#include "pop_math.cuh"

namespace pop {

constexpr int GV_ROW_PAD = 128; // m1 rows are padded to a multiple of this (every row tile height divides it)
constexpr int GV_TL = 64;      // Lambda columns per CTA tile
constexpr int GV_BC = 32;      // q nodes per staged chunk
constexpr int GV_SLICE = 8192; // Lambda columns per slice (bounds the U scratch)

struct GridVT {
    int n_m1 = 0, n_q = 0;  // nodes as loaded
    int na = 0;             // m1 rows padded to GV_ROW_PAD
    int nb = 0;             // q nodes with q <= 1 (the q support never reaches past 1)
    int nbp = 0;            // nb padded to GV_BC
    DevBuf m1, lnm1, invm1, wa;  // FP64 [na]: nodes, ln m1, 1/m1, trapezoid weights (0 in the padding)
    DevBuf m1f, m1lf, invm1f;    // FP32 [na]: m1 as a (hi, lo) pair, 1/m1
    DevBuf l2m1f, waf;           // FP32 [na]: log2 m1, trapezoid weights
    DevBuf q, lnq, wq;           // FP64 [nbp]: nodes, ln q, trapezoid weights
    DevBuf qf;                   // FP32 [nbp]: nodes (first guess of the support edge)
    DevBuf l2qh, l2ql, wqf;      // FP32 [nbp]: log2 q as a (hi, lo) pair, trapezoid weights
    DevBuf qbk;                  // [nqb + 1] first q node of each bin of the support-edge search
    DevBuf rows32;               // [na] FP32 form's per-row constants, packed
    float qb0 = 0.0f, qbinv = 0.0f;
    int nqb = 1;
    DevBuf pd64, pd32;           // pdet packed in row tiles [na / TA][nbp][TA], TA = 32 (FP64) or 128 (FP32)
    DevBuf tab;                  // 2^(j/2048) as (hi, lo) for the FP64 exponentials
    ExpConsts kc{};

    // Scratch, sized by ensure() for batches of up to k_cap Lambda.
    int64_t k_cap = 0;
    int slice = 0;          // columns per slice, a multiple of 128
    DevBuf perm, lamc, order, U, part, xi, err;  // lamc: per-column constants; order: row tiles, heaviest first
    DevBuf lamc32;                               // per-column constants of the FP32 form, packed
    DevBuf queue;                                // FP32 contraction: one item counter per slice
    DevBuf wg, b0g;                              // W (FP64, or FP32 in the same bytes) and b0 of every pair of a slice
    DevBuf wmm;                                  // FP32 contraction: each warp's lowest and highest support edge
    int g32_ctas = 0;                            // resident CTAs of the FP32 contraction (persistent grid)
    // Standalone evaluation (pop_xi_grid): own Lambda, K and outputs.
    int64_t k_cap_own = 0;
    DevBuf own_lambda, own_K, own_lnxi, own_flags;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    std::string err_msg;

    GridVT() = default;
    GridVT(const GridVT&) = delete;
    GridVT& operator=(const GridVT&) = delete;
    ~GridVT();

    // Copy the nodes and pdet (pointers in host or device memory), validate,
    // pack.  Returns a pop_status; err_msg has the text.  Synchronous.
    int load(int n_m1_, const double* m1_nodes, int n_q_, const double* q_nodes, const double* pdet, bool on_device,
             cudaStream_t s);
    // Scratch for batches of up to K Lambda (no allocation afterwards, so the
    // enqueue below may run inside a stream capture).
    cudaError_t ensure(int64_t K);
    // xi_grid for the K (read from dK) Lambda rows of lambda[K_cap][n_params]
    // into xi[k] (FP64): sort by mmin, U, the pairs' W and b0, masked
    // contraction, fixed-order reduction, per slice.  mode: 0 = FP64
    // throughout, 1 = FP32 W, pdet, U and node sums (FP64 support edges, an
    // exact-product float-float row combine, FP64 reduction).  Events ev0..ev3
    // bracket the whole and the contraction (setup included) of the first slice
    // when `timed`.
    cudaError_t enqueue(int mode, const double* lambda, int n_params, const int64_t* dK, int64_t K_cap, bool timed,
                        unsigned record_flags, cudaStream_t s);
    // pop_xi_grid: ln xi and flags (1 = invalid Lambda, 32 = xi = 0).
    cudaError_t out_lnxi(const double* lambda, int n_params, const int64_t* dK, int64_t K_cap, double* lnxi,
                         uint32_t* flags, cudaStream_t s);
    // Device error word (nonzero after a bounded wait gave up); reads and clears it.
    cudaError_t take_error(int* h, cudaStream_t s);
};

// One bounded mbarrier wait of the contraction's kind (gv_wait) with the given poll limit, on a
// barrier that the waiting thread completes first (arrive != 0) or that nothing completes;
// sets *err to 1 when the wait gives up.
cudaError_t launch_wait_check(int arrive, int polls, int* err, cudaStream_t s);

}  // namespace pop
