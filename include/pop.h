/*
 * pop.h — C-ABI of libpop.so, the GB300 (sm_103a) population-likelihood library.
 *
 * Method (paper "Parallelized Inference for Gravitational-Wave Astronomy",
 * Sec. "Population acceleration"): for a batch of population hyper-parameters
 * Lambda the library returns
 *
 *     ln L(Lambda) = sum_i ln[ (1/n_i) sum_j p(theta_ij | Lambda) / pi(theta_ij) ] - N ln xi(Lambda)
 *
 * The inner sum is the "recycling" Monte Carlo integral of Eq. (poplike) over
 * the n_i posterior samples theta_ij of event i, each divided by the prior pi
 * of the single-event analysis.  The -N ln xi term is the rate factor
 * R^N exp(-R VT(Lambda)) of the first equation of that section with R
 * marginalised under a 1/R prior (VT proportional to xi).  xi(Lambda) is the
 * Monte Carlo selection integral over found injections that the same section
 * describes:  xi = (1/N_draw) sum_{k found} p(theta_k | Lambda) / p_draw(theta_k).
 *
 * The population density p(theta | Lambda) is the product of
 *   primary mass   (1-lam) PL(m1; -alpha, [mmin, mmax]) + lam N(m1; mpp, sigpp) truncated to [mmin, mmax]
 *   mass ratio     (1+beta) q^beta / (1 - (mmin/m1)^(1+beta)) on [mmin/m1, 1]   (beta = -1: 1/(q ln(m1/mmin)))
 *   spin sizes     Beta(a1; alpha_chi, beta_chi) Beta(a2; alpha_chi, beta_chi)
 *   spin tilts     (1-xi_t)/4 + xi_t G(cos t1) G(cos t2), G = N(1, sigma_t) truncated to [-1, 1]
 *   redshift       (1+z)^(kappa-1) z^2 / I(kappa) on [0, 2], I = 1024-node trapezoid   (optional)
 * with support mmin < m1 <= mmax, fl64(q*m1) >= mmin, q <= 1, a in [0,1],
 * cos in [-1,1], z in [0,2]; the weight is 0 outside it.
 *
 * Conventions for every entry point:
 *   - returns a pop_status (0 = POP_OK); errors never abort the process and a
 *     failing call leaves the context as it was (pop_last_error has the text);
 *   - sample coordinates theta are row-major [n, n_dims], n_dims = 6
 *     (m1, q, a1, a2, cos t1, cos t2) or 7 (+ z);
 *   - Lambda rows are row-major [K, n_params], n_params = 11
 *     (alpha, beta, mmin, mmax, lam, mpp, sigpp, alpha_chi, beta_chi, xi_t, sigma_t)
 *     or 12 (+ kappa), and n_params must equal 11 + (n_dims == 7);
 *   - `mem` says where caller pointers live (POP_MEM_HOST or POP_MEM_DEVICE);
 *     all data is copied, the caller keeps ownership of its buffers;
 *   - one context drives one GPU on one stream; calls on a context are not
 *     thread-safe.  There is no CPU fallback: without a usable GPU,
 *     pop_create fails with POP_ECUDA.
 */
#ifndef POP_H
#define POP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pop_ctx pop_ctx;

typedef enum {
    POP_OK = 0,
    POP_EINVAL = -1,    /* bad argument or malformed input */
    POP_ENOMEM = -2,    /* device or pinned-host allocation failed */
    POP_ECUDA = -3,     /* CUDA runtime error (text in pop_last_error) */
    POP_ESTATE = -4,    /* events/injections not loaded, or surrogate not trained */
    POP_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
    POP_ENUMERIC = -6   /* surrogate gate failed; Monte Carlo xi was used */
} pop_status;

/* Storage of the packed per-sample features (bit mask, both may be kept). */
enum { POP_STORE_F64 = 1, POP_STORE_F32 = 2 };

/* Arithmetic of pop_loglik.
 *   POP_MODE_F64: FP64 everywhere (needs POP_STORE_F64 features).
 *   POP_MODE_F32: FP32 sample weights with compensated per-thread sums; FP64
 *                 per-Lambda constants, partial combines, per-event log,
 *                 cross-event sum and xi (needs POP_STORE_F32 features).
 *   POP_MODE_F32_SURROGATE: as POP_MODE_F32, with ln xi from the trained MLP
 *                 and Monte Carlo xi only for the Lambda the gate rejects.
 *   POP_MODE_FF:  the FP64 result to within the FP64 mode's tolerance, with the
 *                 sample weights in float-float arithmetic (each value an
 *                 unevaluated sum of two FP32 numbers, ~48 significant bits,
 *                 on the FP32 pipe) and FP64 for the exact gap m1 - mmin near
 *                 the lower mass edge; weights below e^-87 count as 0.  Uses
 *                 the POP_STORE_F64 features; per-Lambda constants, partials,
 *                 logs and sums in FP64 as in POP_MODE_F64. */
enum { POP_MODE_F64 = 0, POP_MODE_F32 = 1, POP_MODE_F32_SURROGATE = 2, POP_MODE_FF = 3 };

enum { POP_MEM_HOST = 0, POP_MEM_DEVICE = 1 };

/* Per-Lambda result flags (out_flags).  ln L = -inf is a legitimate value,
 * not an error.  NaN is never returned for a Lambda whose densities are
 * representable in FP64; beyond that range (|1+beta| or |1-alpha| times
 * ln(mmax/mmin) above ~700, or sigma below ~1e-154) ln L may be NaN. */
enum {
    POP_FLAG_INVALID_LAMBDA = 1u,  /* Lambda outside the model's domain: ln L = -inf */
    POP_FLAG_ZERO_EVENT = 2u,      /* some event has sum_j w_ij = 0: ln L = -inf */
    POP_FLAG_LOW_NEFF = 4u,        /* injection effective sample count < 4 N */
    POP_FLAG_SURROGATE_USED = 8u,  /* ln xi came from the surrogate */
    POP_FLAG_MC_FALLBACK = 16u,    /* surrogate rejected, Monte Carlo xi used */
    POP_FLAG_ZERO_XI = 32u         /* xi = 0 (no found injection has weight): ln L = -inf */
};

/* Create a context on CUDA device `device` that issues all work on `stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = the
 * legacy default stream).  *out receives the context; destroy it with
 * pop_destroy.  Fails with POP_ECUDA when no usable GPU is present. */
int pop_create(pop_ctx** out, int device, void* stream);

/* Free every device and host buffer of the context.  NULL is accepted. */
int pop_destroy(pop_ctx* ctx);

/* Text of the last error on `ctx` (or of the last pop_create failure when ctx
 * is NULL).  Valid until the next call on the same context. */
const char* pop_last_error(const pop_ctx* ctx);

/* Static name of a pop_status value. */
const char* pop_status_string(int status);

/* ABI version (major * 10000 + minor * 100 + patch). */
int pop_version(void);

/* Host-only validation of a CSR event layout, without a context or a GPU:
 * n_events >= 1, offsets[0] = 0, offsets non-decreasing with every n_i >= 1,
 * n_dims in {6, 7}.  Writes a message into msg[msg_len] (may be NULL). */
int pop_validate_events(int64_t n_events, const int64_t* offsets, int n_dims, char* msg, int msg_len);

/* Load the per-event posterior samples (paper: the N x n_i sample arrays are
 * moved to the GPU once; Sec. "Population acceleration").
 *   offsets[n_events+1]  int64, host memory always, CSR row starts (dense
 *                        [N, S] data is offsets[i] = i*S)
 *   theta[offsets[N] * n_dims], prior[offsets[N]] (pi > 0, finite) in `mem`
 *   storage              POP_STORE_F64 and/or POP_STORE_F32
 * A one-time pack kernel turns the samples into per-sample features
 * (log-masses, summed spin logs, tilt distance, -ln pi) in FP64 and stores
 * them in the requested precision(s).  Replaces previously loaded events.
 * POP_EINVAL on malformed offsets, non-finite theta or pi <= 0. */
int pop_load_events(pop_ctx* ctx, int64_t n_events, const int64_t* offsets, int n_dims,
                    const double* theta, const double* prior, int storage, int mem);

/* Load the found injections of the selection term (same section: Monte Carlo
 * integral over found injections).
 *   theta[n_found * n_dims], p_draw[n_found] (> 0, finite) in `mem`
 *   n_draw = number of draws, found and missed (n_draw >= n_found >= 1).
 * n_dims must equal that of the loaded events (load events first). */
int pop_load_injections(pop_ctx* ctx, int64_t n_found, int64_t n_draw, int n_dims,
                        const double* theta, const double* p_draw, int storage, int mem);

/* Evaluate ln L for K Lambda points.
 *   lambda[K * n_params] in `mem`; out_lnL[K] required; out_lnxi[K] (ln xi),
 *   out_neff[K] (injection effective sample count xi^2 / Var[xi]) and
 *   out_flags[K] may be NULL; all outputs in `mem`.
 * With POP_MEM_DEVICE the call is asynchronous on the context stream; with
 * POP_MEM_HOST it returns after the results are in the host buffers.
 * K may be 0.  Scratch grows to the largest K seen and is reused. */
int pop_loglik(pop_ctx* ctx, int64_t K, int n_params, const double* lambda, int mode,
               double* out_lnL, double* out_lnxi, double* out_neff, uint32_t* out_flags, int mem);

/* The additive parts of ln L for K Lambda rows, for splitting a catalog over
 * several GPUs (each loads a disjoint range of events and a disjoint share of the
 * found injections, all with the same total n_draw):
 *   out_events[k] = sum_i ln(S_i/n_i) over the loaded events (-inf when some S_i = 0)
 *   out_sum_w[k]  = sum over the loaded injections of w = p(theta|Lambda)/p_draw
 *   out_sum_w2[k] = sum of w^2
 *   out_flags[k]  = POP_FLAG_INVALID_LAMBDA (parts -inf, 0, 0) | POP_FLAG_ZERO_EVENT  (may be NULL)
 * Parts of disjoint sets add up to those of their union, and then, with N the
 * total number of events, xi = sum_w / n_draw, ln L = events - N ln xi and
 * N_eff = xi^2 / (sum_w2 / n_draw^2 - xi^2 / n_draw), as pop_loglik computes them.
 * Modes POP_MODE_F64 and POP_MODE_F32, with the injection selection term;
 * outputs in `mem` (asynchronous with POP_MEM_DEVICE, as pop_loglik). */
int pop_loglik_parts(pop_ctx* ctx, int64_t K, int n_params, const double* lambda, int mode, double* out_events,
                     double* out_sum_w, double* out_sum_w2, uint32_t* out_flags, int mem);

/* ln L and its gradient with respect to Lambda, for gradient-based samplers (not
 * in the paper; derived from the likelihood above):
 *   d ln L / d Lambda_p = sum_i (sum_j w_ij g_ij,p) / S_i - N (sum_k w_k g_k,p) / (sum_k w_k),
 * g the score d ln p(theta|Lambda) / d Lambda of the population density (its
 * support's edges, where the density jumps, contribute nothing).  FP64, with the
 * injection selection term; lambda[K * n_params] and the outputs out_lnL[K],
 * out_grad[K * n_params] (row-major, the Lambda order) and out_flags[K] (may be
 * NULL) in `mem`.  Where ln L = -inf the gradient is 0.  Synchronous for host
 * outputs. */
int pop_loglik_grad(pop_ctx* ctx, int64_t K, int n_params, const double* lambda, double* out_lnL, double* out_grad,
                    uint32_t* out_flags, int mem);

/* ------------------------------------------------------------------ grid selection term
 * The paper evaluates VT on a regular grid with GPU acceleration, limited to a
 * low-dimensional space without spin effects (Sec. "Population acceleration").
 * Here the grid spans (m1, q) and the selection term is the two-dimensional
 * trapezoid rule over its nodes:
 *
 *   xi_grid(Lambda) = sum_a sum_b wa_a wq_b p(m1_a | Lambda) p(q_b | m1_a, Lambda) pdet[a, b]
 *
 * with wa_a = (m1_{a+1} - m1_{a-1}) / 2 (one-sided at the ends, same for wq)
 * and the mass and mass-ratio densities and supports of the population model
 * above (the spin and redshift densities integrate to one and drop out).
 * The spin-free grid cannot include the spin dependence of detectability; the
 * injection term can. */

/* Selection-term source of pop_loglik. */
enum { POP_XI_INJECTIONS = 0, POP_XI_GRID = 1 };

/* Load the grid: nodes m1[n_m1] and q[n_q] (finite, strictly increasing,
 * n_m1, n_q >= 2, n_m1 * n_q <= 2^28, at least one q <= 1) and the detection
 * probability pdet[n_m1 * n_q], row-major [a][b], finite and >= 0 at every node
 * with q <= 1 (nodes with q > 1 only shape the weights).  All three arrays in
 * `mem`; copied (FP64 and an FP32 copy, packed in 64-row tiles).  Replaces a
 * previously loaded grid; synchronous.  POP_EINVAL on malformed input. */
int pop_load_vt_grid(pop_ctx* ctx, int n_m1, const double* m1, int n_q, const double* q, const double* pdet,
                     int mem);

/* Choose the selection term of pop_loglik: POP_XI_INJECTIONS (default, needs
 * pop_load_injections) or POP_XI_GRID (needs pop_load_vt_grid).  With the grid,
 * pop_loglik needs no injections, returns out_neff = +inf (no Monte Carlo
 * variance, so POP_FLAG_LOW_NEFF is never set) and rejects
 * POP_MODE_F32_SURROGATE (which replaces the injection term). */
int pop_set_xi_source(pop_ctx* ctx, int source);

/* ln xi_grid for K Lambda rows (lambda[K * n_params], n_params 11 or 12, kappa
 * unused), without events: out_lnxi[K] (0 for an invalid Lambda, -inf when
 * xi_grid = 0) and out_flags[K] (may be NULL: POP_FLAG_INVALID_LAMBDA,
 * POP_FLAG_ZERO_XI), all in `mem`; synchronous.
 *   POP_MODE_F64: FP64 throughout.
 *   POP_MODE_F32: FP32 pdet, q-node factors and node sums (an FP32 sum per
 *                 32 nodes, added into an FP32 running sum); FP64 per-row
 *                 factors, support edges and row combine.
 * POP_ETIMEOUT when a bounded device-side wait of the contraction gave up
 * (outputs then undefined). */
int pop_xi_grid(pop_ctx* ctx, int64_t K, int n_params, const double* lambda, int mode, double* out_lnxi,
                uint32_t* out_flags, int mem);

/* Duration in milliseconds of the last grid evaluation (pop_xi_grid, or the
 * grid part of pop_loglik): the node contraction kernel of the first 8192
 * Lambda, and the whole grid term (CUDA events on the context stream). */
int pop_xi_grid_last_ms(pop_ctx* ctx, double* contraction_ms, double* total_ms);

/* ------------------------------------------------------------------ single-event CBC likelihood
 * Paper, Sec. "Single-event Likelihood acceleration", Eq. (cbclike): for
 * n_det detectors and M frequency bins f_j = f0 + j df (T = 1/df),
 *
 *   ln L(theta) = sum_i sum_j [ -ln(2 pi S_ij) - (2/T) |d_ij - h_ij(theta)|^2 / S_ij ]
 *   h_ij = A e^{i phi} (Fp_i hp_j + Fc_i hc_j) e^{-2 pi i f_j dt_i}
 *
 * with the frequency-domain template given by its two polarisations hp, hc
 * (from any waveform model), and per parameter row theta the amplitude A,
 * phase phi and, per detector, the antenna factors Fp_i, Fc_i and the
 * arrival-time shift dt_i (the per-detector time-shift exponential the
 * section names as the likelihood's second largest cost). */

/* Load data d[n_det][M] and templates (complex, interleaved Re, Im doubles:
 * data[(i M + j) 2 + {0, 1}], hp[2 j + {0, 1}], hc[2 j + {0, 1}]) and the PSD
 * psd[n_det][M] (> 0), all in `mem`, finite.  The data-only terms, the
 * template norms and w conj(d) hp, w conj(d) hc (w = (2/T)/S) are formed once
 * here in FP64.  Replaces earlier CBC data; synchronous. */
int pop_cbc_load(pop_ctx* ctx, int n_det, int64_t M, double f0, double df, const double* data, const double* psd,
                 const double* hp, const double* hc, int mem);

/* ln L for K rows theta[K][n_params], n_params = 2 + 3 n_det, in the order
 * (A, phi, Fp_1, Fc_1, dt_1, ..., Fp_n, Fc_n, dt_n).  out_lnL[K] required,
 * out_flags[K] may be NULL (POP_FLAG_INVALID_LAMBDA for a non-finite row, whose
 * ln L is -inf).  mode POP_MODE_F64 (FP64 throughout) or POP_MODE_F32 (FP32
 * time shifts and bin sums, FP64 phases modulo one turn, per-block combines
 * and the final assembly).  Outputs in `mem`; asynchronous with POP_MEM_DEVICE. */
int pop_cbc_loglik(pop_ctx* ctx, int64_t K, int n_params, const double* theta, int mode, double* out_lnL,
                   uint32_t* out_flags, int mem);

/* Duration in milliseconds of the last pop_cbc_loglik: the time-shifted bin
 * sums kernel, and the whole call on the device. */
int pop_cbc_last_ms(pop_ctx* ctx, double* sum_ms, double* total_ms);

/* Tiling of the persistent weight kernel for `mode`, with resident blocks per
 * SM (0 = occupancy maximum).  POP_MODE_F64: Lambda points per work item (1, 2,
 * 4, 8 or 16) and threads per block (128, 256 or 512).  POP_MODE_F32: one Lambda
 * per thread, so lambda_tile == block_threads, 32, 64, 128 or 256; its results
 * do not depend on the tiling.  POP_EINVAL for any other combination.  Takes
 * effect at the next pop_loglik. */
int pop_set_tiling(pop_ctx* ctx, int mode, int lambda_tile, int block_threads, int blocks_per_sm);

/* Read back the tiling in use for `mode` (any pointer may be NULL). */
int pop_get_tiling(pop_ctx* ctx, int mode, int* lambda_tile, int* block_threads, int* blocks_per_sm);

/* Autotune the tiling of `mode` on the loaded data for batches of K Lambda
 * (times every candidate with CUDA events on the context stream and keeps the
 * fastest).  When cache_path is non-NULL the choice is read from / appended to
 * that text file, keyed by device name, mode, and data shape. */
int pop_autotune(pop_ctx* ctx, int mode, int64_t K, const char* cache_path);

/* Use CUDA-graph replay for pop_loglik (1, default) or direct launches (0). */
int pop_set_graphs(pop_ctx* ctx, int enable);

/* Duration in milliseconds of the weight kernel of the last pop_loglik or
 * pop_loglik_grad, and of the whole call on the device (CUDA events around
 * them on the context stream; waits for that call). */
int pop_last_kernel_ms(pop_ctx* ctx, double* weight_ms, double* total_ms);

/* Diagnostic: evaluate the FP64 weight kernel's own device functions on x[n]
 * and write y[n] (both in `mem`): fn 0 = exp (Tang's table-driven method,
 * 2048-entry table; 0 below x = -707, +inf above 709.7), fn 1 = expm1, fn 2 =
 * reciprocal of a positive normal x (hardware seed + one cubic Newton step).
 * fn 3..7 evaluate the float-float functions of POP_MODE_FF on x rounded to a
 * float-float value, returning hi + lo: 3 = exp (0 below x = -87), 4 = expm1
 * (Taylor series below |x| = 1/16, Tang's table above), 5 = reciprocal, 6 =
 * square, 7 = the exact square of the FP32 high part (packed FMA error term).
 * fn 8 = ln x (the finalise's per-event log: Tang's table-driven logarithm with
 * a 129-entry table for positive normal x, the library's log elsewhere).
 * The test suite checks them against libm and CUDA's functions. */
int pop_math_check(pop_ctx* ctx, int fn, int64_t n, const double* x, double* y, int mem);

/* Largest poll limit pop_wait_check accepts: the grid contraction's and the
 * tensor-core GEMM's own limit, about 1 s of polls (a poll of a phase that is
 * not complete suspends the thread about 3.8 us on GB300). */
#define POP_WAIT_CHECK_MAX_POLLS (1 << 18)

/* Diagnostic of failure detection (the paper has no counterpart).  The grid
 * contraction's shared-memory copies complete on mbarriers, and every wait on
 * one is bounded: after a fixed number of polls it gives up, raises an error
 * word on the device and lets the kernel return, and the host call reports
 * POP_ETIMEOUT instead of hanging.  This runs one such wait, with the same
 * device function and the given poll limit (1..POP_WAIT_CHECK_MAX_POLLS), on a
 * barrier that the waiting thread first completes itself (arrive != 0: returns
 * POP_OK) or that nothing completes (arrive == 0: returns POP_ETIMEOUT after
 * `polls` polls).  No GPU fault or hang is involved, and the context stays
 * usable.  Synchronous on the context stream.  POP_EINVAL for a poll limit out
 * of range. */
int pop_wait_check(pop_ctx* ctx, int arrive, int polls);

/* Diagnostic: the per-SM throughput of the pipes the weight kernels are bound
 * by, measured on `device` (the paper has no counterpart; the rooflines of
 * the weight kernels need these rates, and the data sheet gives no MUFU
 * figure).  One CTA of 1024 threads per SM runs 8 independent chains of one
 * operation per thread; clock64 around the chains gives thread operations per
 * SM clock (median over the SMs):
 *   rates[0] FP64 fma, rates[1] FP32 fma, rates[2] MUFU ex2.approx.f32,
 *   rates[3] MUFU rcp.approx.f32.
 * rates: a host array of 4 doubles, owned by the caller.  Synchronous, a few
 * milliseconds; allocates two small device buffers and frees them.  Restores
 * the calling thread's current device.  POP_EINVAL for a NULL rates or a negative
 * device, POP_ECUDA when a CUDA call fails. */
int pop_pipe_rates(int device, double* rates);

/* pop_pipe_rates with more rates: rates[0..n_rates) of, in order, the four above,
 *   rates[4] FP32 lanes of packed fma.rn.f32x2 per SM clock,
 *   rates[5] warp-wide 16-byte shared loads (ld.shared.v4, 32 distinct addresses) per SM clock,
 *   rates[6] the same with 4 distinct addresses (8 lanes on each word).
 * n_rates is clamped to 7; rates: a host array of n_rates doubles, owned by the caller.
 * Synchronous; POP_EINVAL for a NULL rates, a negative device or n_rates < 1, POP_ECUDA when
 * a CUDA call fails; restores the calling thread's current device. */
int pop_pipe_rates_n(int device, double* rates, int n_rates);

/* ------------------------------------------------------------------ ln xi surrogate
 * The paper announces a learned selection term that includes spin effects in
 * VT at no extra run-time cost (Sec. "Population acceleration", right after the
 * Monte Carlo VT).  Here it is a network on the normalised Lambda
 * (x = 2 (Lambda - lo)/(hi - lo) - 1, 12 inputs, kappa = 0 when absent) ->
 * 4 x 256 SiLU -> (ln xi, ln N_eff) standardised; BF16 weights and
 * activations on the tcgen05 tensor cores with FP32 accumulators, FP32 master
 * weights and Adam.  Flat FP32 parameter layout (201218 floats): W0 [256 x 12],
 * b0 [256], W1 [256 x 256], b1, W2, b2, W3, b3, W4 [2 x 256], b4 [2]; W row-major
 * [out][in]. */

/* Train on n_pairs Lambda drawn uniformly (seeded) from the box
 * [lambda_lo, lambda_hi] (n_params values each), with targets ln xi-hat and
 * ln N_eff from the loaded injections (the Monte Carlo selection term itself,
 * FP32 arithmetic when FP32 storage is loaded, else FP64); heldout_frac of the
 * pairs are held out.
 * Mean-squared loss on the standardised targets, mini-batches of 4096, Adam
 * with cosine learning-rate decay over `epochs`.  The surrogate is trusted when
 * its held-out ln xi error beyond the targets' own Monte Carlo scatter
 * (sqrt(max(0, rmse^2 - mean(1/N_eff)))) is at most 0.01.
 * *out_heldout_rmse (may be NULL) = held-out RMS error of ln xi vs the targets. */
int pop_xi_surrogate_train(pop_ctx* ctx, int64_t n_pairs, double heldout_frac, uint64_t seed,
                           const double* lambda_lo, const double* lambda_hi, int n_params, int epochs,
                           double* out_heldout_rmse);

/* Held-out statistics of the trained surrogate (any pointer may be NULL). */
int pop_xi_surrogate_info(pop_ctx* ctx, double* heldout_rmse, double* mc_noise, double* excess, int* trusted);

/* ln xi (and ln N_eff, may be NULL) predicted for K Lambda rows; out_fallback[k]
 * (may be NULL) = 1 when the Monte Carlo xi must be used instead: surrogate
 * not trusted, Lambda outside the training box, predicted N_eff < 4 N, or
 * N * (the Lambda's error bound, pop_xi_surrogate_error) above the budget
 * (pop_xi_surrogate_set_budget).  pop_loglik in POP_MODE_F32_SURROGATE takes
 * the same decision for every Lambda.  All arrays in `mem`; synchronous. */
int pop_xi_surrogate_infer(pop_ctx* ctx, int64_t K, int n_params, const double* lambda, double* out_lnxi,
                           double* out_lnneff, uint8_t* out_fallback, int mem);

/* The surrogate's error bound on ln xi for each of K Lambda rows (out_err[K],
 * in `mem`; synchronous).  From the held-out pairs of the training: they are
 * split into 16 bins of equal count by the network's predicted ln N_eff (the
 * Monte Carlo scatter of the targets, which the network cannot learn, grows
 * like 1/sqrt(N_eff)), and a bin's bound is 1.25 x its largest held-out
 * |ln xi_net - ln xi-hat|.  A Lambda's ln L from the surrogate then differs
 * from the Monte Carlo one by N x that bound at most, for all but about one in
 * (pairs per bin) Lambda.  This is a per-Lambda reading of the paper's learned
 * VT (Sec. "Population acceleration"), which gives no error model. */
int pop_xi_surrogate_error(pop_ctx* ctx, int64_t K, int n_params, const double* lambda, double* out_err, int mem);

/* Wall time of the last pop_xi_surrogate_train in this context: generating the
 * targets (the Monte Carlo selection term over the pairs) and fitting (forward,
 * backward and Adam over every mini-batch, synchronised at the end), and the
 * rows that went through forward and backward (epochs x steps x batch).  Any
 * pointer may be NULL; POP_ESTATE when nothing was trained here (a loaded
 * checkpoint has no timings). */
int pop_xi_surrogate_train_stats(pop_ctx* ctx, double* target_seconds, double* fit_seconds, int64_t* fit_rows);

/* Largest N x error bound (nats of ln L) for which a Lambda uses the network;
 * default 0.25.  Takes effect on the next call; POP_EINVAL for a negative or
 * NaN budget.  Saved in checkpoints. */
int pop_xi_surrogate_set_budget(pop_ctx* ctx, double nats);

/* Checkpoint of the trained surrogate (weights, normalisation, held-out
 * statistics) as a versioned binary file; load restores it. */
int pop_xi_surrogate_save(pop_ctx* ctx, const char* path);
int pop_xi_surrogate_load(pop_ctx* ctx, const char* path);

/* Network-level access (host memory), for checks and custom training:
 * set/get the flat FP32 parameters (n = 201218; setting resets Adam), forward
 * on B normalised inputs x[B x 12] -> y[B x 2], the loss
 * (1/B) sum (y - t)^2 and its gradients (flat layout), and one Adam step
 * (beta 0.9/0.999, eps 1e-8) on a batch. */
int pop_mlp_set_params(pop_ctx* ctx, const float* params, int64_t n);
int pop_mlp_get_params(pop_ctx* ctx, float* params, int64_t n);
int pop_mlp_forward(pop_ctx* ctx, int64_t B, const float* x, float* y);
int pop_mlp_gradients(pop_ctx* ctx, int64_t B, const float* x, const float* t, float* grads, double* loss);
int pop_mlp_train_step(pop_ctx* ctx, int64_t B, const float* x, const float* t, float lr);

/* Diagnostic: C[M x N] = A[M x K] B[N x K]^T with A and B rounded to BF16, on
 * the tcgen05 tensor cores with an FP32 accumulator (host arrays, row-major;
 * M a multiple of 128, N a multiple of 16 up to 256, K a multiple of 64). */
int pop_mlp_gemm_check(pop_ctx* ctx, int M, int N, int K, const float* A, const float* B, float* C);

/* Bytes of the scratch array that pop_loglik_f64_noalloc uses (16 MiB). */
#define POP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* ln L in FP64 (as pop_loglik with POP_MODE_F64) without allocating anything.
 *
 * The paper has no counterpart: this is an interface for callers that cannot
 * call cudaMalloc — code whose device memory all belongs to an outer pool or
 * framework, or a sampler loop that must not allocate or free while it runs.
 * There is no context: the caller passes every input and output as a device
 * pointer it owns, and the library calls no cudaMalloc, cudaFree or other
 * allocating routine.  Scratch (per-Lambda constants and per-(Lambda, event)
 * partial sums) lives in one static device array of POP_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads libpop.so holds until the process exits.
 *
 *   device, stream   CUDA device index and cudaStream_t (NULL = legacy stream)
 *   offsets[n_events+1]  int64 CSR row starts (device); n_samples = offsets[N]
 *   theta[n_samples * n_dims], prior[n_samples]              (device, as pop_load_events)
 *   inj_theta[n_found * n_dims], p_draw[n_found], n_draw     (device, as pop_load_injections)
 *   lambda[K * n_params]                                     (device, as pop_loglik)
 *   out_lnL, out_lnxi, out_neff (double[K]), out_flags (uint32[K])  (device, all required)
 *   msg[msg_len]     host buffer for the error text (may be NULL)
 *
 * Every pointer but msg must be device (or managed) memory of `device`;
 * anything else (host, pinned host, another GPU's memory) fails with
 * POP_EINVAL before any GPU work.  The calling thread's current device is
 * restored before the call returns.
 *
 * The scratch needed is about K * 8 * (n_events + 2 * ceil(n_found / 4096))
 * + K * 256 bytes; a call above POP_NOALLOC_SCRATCH_BYTES fails with
 * POP_EINVAL before any GPU work (split the Lambda batch).  Malformed offsets
 * (offsets[0] != 0, offsets[N] != n_samples, an event with no samples or one
 * that ends beyond n_samples), non-finite samples and prior/p_draw <= 0 give
 * POP_EINVAL after the kernels ran (outputs then undefined; the kernels never
 * read outside the buffers).  The call is synchronous: it copies a count of
 * malformed inputs to the host and waits for the stream before it returns.
 * The first call on a device looks up the array's device address (module load
 * and symbol lookup), so make that first call before any stream capture.  All
 * calls share the one array and each call rewrites every scratch word it
 * reads, so nothing carries over from the previous call; calls that overlap on
 * the GPU (other threads or streams) race on it. */
int pop_loglik_f64_noalloc(int device, void* stream, int64_t n_events, const int64_t* offsets,
                           int64_t n_samples, int n_dims, const double* theta, const double* prior,
                           int64_t n_found, int64_t n_draw, const double* inj_theta, const double* p_draw,
                           int64_t K, int n_params, const double* lambda, double* out_lnL, double* out_lnxi,
                           double* out_neff, uint32_t* out_flags, char* msg, int msg_len);

#ifdef __cplusplus
}
#endif

#endif /* POP_H */
