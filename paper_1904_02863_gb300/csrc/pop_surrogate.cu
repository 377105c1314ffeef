// C-ABI of the ln xi surrogate: training on (Lambda, ln xi-hat) pairs that the
// injection reweighting itself produces, inference with its trust gate,
// checkpoints, and network-level entry points for checks.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <random>
#include <string>
#include <vector>

#include "pop.h"
#include "pop_devbuf.h"
#include "pop_internal.h"
#include "pop_trace.h"
#include "pop_mlp.h"

namespace pop {
int ctx_fail(pop_ctx* c, int status, const std::string& msg);
cudaStream_t ctx_stream(pop_ctx* c);
int ctx_device(pop_ctx* c);
int64_t ctx_n_events(pop_ctx* c);
int ctx_n_dims(pop_ctx* c);
int ctx_has_storage(pop_ctx* c, int storage);
Surrogate* ctx_surrogate(pop_ctx* c, int* status);
}  // namespace pop

using namespace pop;

namespace {

constexpr int64_t TRAIN_BATCH = 4096;
constexpr int64_t GEN_BATCH = 8192;
constexpr double GATE_EXCESS = 0.01;  // surrogate error beyond the targets' own Monte Carlo scatter
constexpr char CKPT_MAGIC[8] = {'P', 'O', 'P', 'X', 'I', 'M', 'L', '1'};

#define CKC(call, what)                                                                                     \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return ctx_fail(c, e_ == cudaErrorMemoryAllocation ? POP_ENOMEM : POP_ECUDA,                    \
                            std::string(what) + ": " + cudaGetErrorString(e_));                             \
    } while (0)

#define SUR(call)                                                                                           \
    do {                                                                                                    \
        const int rc_ = (call);                                                                             \
        if (rc_ != POP_OK) return ctx_fail(c, rc_, "surrogate: " + s->err);                                 \
    } while (0)

uint16_t to_bf16_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest, ties to even
    return (uint16_t)(u >> 16);
}

int64_t pad128(int64_t n) { return (n + 127) / 128 * 128; }

// Host rows x[B x 12] (already normalised) -> s->x0 (BF16, zero-padded to [pad128(B) x 64]).
int upload_inputs(pop_ctx* c, Surrogate* s, int64_t B, const float* x)
{
    const int64_t rp = pad128(B);
    SUR(s->ensure_rows(rp));
    std::vector<uint16_t> hx((size_t)rp * MLP_IN_PAD, 0);
    for (int64_t r = 0; r < B; ++r)
        for (int k = 0; k < MLP_IN; ++k) hx[r * MLP_IN_PAD + k] = to_bf16_bits(x[r * MLP_IN + k]);
    CKC(cudaMemcpyAsync(s->x0.p, hx.data(), hx.size() * 2, cudaMemcpyHostToDevice, s->stream), "copy inputs");
    return POP_OK;
}

// ln xi, ln N_eff and the fallback mask for K Lambda rows (device Lambda, host outputs; any
// output but lnxi may be NULL).
int infer_device(pop_ctx* c, Surrogate* s, int64_t K, int P, const double* d_lambda, double* lnxi, double* lnneff,
                 uint8_t* fallback)
{
    const int64_t rp = pad128(K);
    SUR(s->ensure_rows(rp));
    DevBuf outside;
    CKC(outside.alloc(std::max<int64_t>(K, 1)), "cudaMalloc");
    SUR(s->fused_forward(d_lambda, P, nullptr, K, nullptr, s->y.as<float>(), outside.as<uint8_t>(), 0.0, nullptr,
                         nullptr, nullptr));
    SUR(s->check_error());
    std::vector<float> y((size_t)rp * 2);
    std::vector<uint8_t> out(K);
    CKC(cudaMemcpyAsync(y.data(), s->y.p, y.size() * 4, cudaMemcpyDeviceToHost, s->stream), "copy y");
    CKC(cudaMemcpyAsync(out.data(), outside.p, K, cudaMemcpyDeviceToHost, s->stream), "copy mask");
    CKC(cudaStreamSynchronize(s->stream), "sync");
    const double n_events = (double)ctx_n_events(c);
    for (int64_t k = 0; k < K; ++k) {
        // the gate kernel's arithmetic: FP32 outputs widened, then scaled in FP64
        const double lx = (double)y[k * 2] * s->sd[0] + s->mu[0];
        const double ln = (double)y[k * 2 + 1] * s->sd[1] + s->mu[1];
        lnxi[k] = lx;
        if (lnneff) lnneff[k] = ln;
        if (fallback)
            fallback[k] = (uint8_t)need_monte_carlo(s->trusted, out[k] != 0, false, lx, ln, n_events, s->budget,
                                                    s->table);
    }
    return POP_OK;
}

// The per-Lambda error table from the held-out pairs: bins of equal count by predicted ln N_eff,
// each bin's bound ERR_MARGIN x its largest |ln xi_net - ln xi-hat|.
void build_err_table(Surrogate* s, const std::vector<double>& pred_lnneff, const std::vector<double>& abs_err)
{
    const size_t n = abs_err.size();
    std::vector<size_t> idx(n);
    for (size_t i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return pred_lnneff[a] < pred_lnneff[b]; });
    for (int b = 0; b < ERR_BINS; ++b) {
        const size_t i0 = n * (size_t)b / ERR_BINS, i1 = n * (size_t)(b + 1) / ERR_BINS;
        double m = 0.0;
        for (size_t i = i0; i < i1; ++i) m = std::max(m, abs_err[idx[i]]);
        // an empty bin (fewer pairs than bins) keeps no claim: never within a budget
        s->table.err[b] = i1 > i0 ? ERR_MARGIN * m : INFINITY;
        if (b > 0) s->table.edge[b - 1] = i0 < n ? pred_lnneff[idx[i0]] : INFINITY;
    }
}

}  // namespace

extern "C" {

int pop_mlp_gemm_check(pop_ctx* c, int M, int N, int K, const float* A, const float* B, float* C)
{
    if (!c) return POP_EINVAL;
    if (M <= 0 || M % 128 || N < 16 || N > 256 || N % 16 || K <= 0 || K % 64 || !A || !B || !C)
        return ctx_fail(c, POP_EINVAL, "pop_mlp_gemm_check: need M % 128 == 0, N in 16..256 step 16, K % 64 == 0");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    std::vector<uint16_t> ha((size_t)M * K), hb((size_t)N * K);
    for (size_t i = 0; i < ha.size(); ++i) ha[i] = to_bf16_bits(A[i]);
    for (size_t i = 0; i < hb.size(); ++i) hb[i] = to_bf16_bits(B[i]);
    DevBuf da, db, dc;
    CKC(da.alloc(ha.size() * 2), "cudaMalloc");
    CKC(db.alloc(hb.size() * 2), "cudaMalloc");
    CKC(dc.alloc((size_t)M * N * 4), "cudaMalloc");
    CKC(cudaMemcpyAsync(da.p, ha.data(), ha.size() * 2, cudaMemcpyHostToDevice, s->stream), "copy");
    CKC(cudaMemcpyAsync(db.p, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice, s->stream), "copy");
    CKC(mlp_gemm_check(da.as<__nv_bfloat16>(), db.as<__nv_bfloat16>(), dc.as<float>(), M, N, K,
                       s->err_flag.as<int>(), s->stream), "gemm");
    SUR(s->check_error());
    CKC(cudaMemcpyAsync(C, dc.p, (size_t)M * N * 4, cudaMemcpyDeviceToHost, s->stream), "copy");
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

int pop_mlp_set_params(pop_ctx* c, const float* params, int64_t n)
{
    if (!c) return POP_EINVAL;
    if (!params || n != MLP_N_PARAMS) return ctx_fail(c, POP_EINVAL, "pop_mlp_set_params: need 201218 floats");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    SUR(s->set_params_host(params));
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

int pop_mlp_get_params(pop_ctx* c, float* params, int64_t n)
{
    if (!c) return POP_EINVAL;
    if (!params || n != MLP_N_PARAMS) return ctx_fail(c, POP_EINVAL, "pop_mlp_get_params: need 201218 floats");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->has_params) return ctx_fail(c, POP_ESTATE, "pop_mlp_get_params: no parameters yet");
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    SUR(s->get_params_host(params));
    return POP_OK;
}

int pop_mlp_forward(pop_ctx* c, int64_t B, const float* x, float* y)
{
    if (!c) return POP_EINVAL;
    if (B < 1 || !x || !y) return ctx_fail(c, POP_EINVAL, "pop_mlp_forward: bad arguments");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->has_params) return ctx_fail(c, POP_ESTATE, "pop_mlp_forward: no parameters yet");
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    int rc = upload_inputs(c, s, B, x);
    if (rc != POP_OK) return rc;
    SUR(s->fused_forward(nullptr, 0, s->x0.as<__nv_bfloat16>(), B, nullptr, s->y.as<float>(), nullptr, 0.0, nullptr,
                         nullptr, nullptr));
    SUR(s->check_error());
    CKC(cudaMemcpyAsync(y, s->y.p, (size_t)B * 2 * 4, cudaMemcpyDeviceToHost, s->stream), "copy y");
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

int pop_mlp_gradients(pop_ctx* c, int64_t B, const float* x, const float* t, float* grads, double* loss)
{
    if (!c) return POP_EINVAL;
    if (B < 1 || !x || !t || !grads) return ctx_fail(c, POP_EINVAL, "pop_mlp_gradients: bad arguments");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->has_params) return ctx_fail(c, POP_ESTATE, "pop_mlp_gradients: no parameters yet");
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    int rc = upload_inputs(c, s, B, x);
    if (rc != POP_OK) return rc;
    const int64_t rp = pad128(B);
    DevBuf dt;
    CKC(dt.alloc((size_t)rp * 2 * 4), "cudaMalloc");
    CKC(cudaMemsetAsync(dt.p, 0, (size_t)rp * 2 * 4, s->stream), "memset");
    CKC(cudaMemcpyAsync(dt.p, t, (size_t)B * 2 * 4, cudaMemcpyHostToDevice, s->stream), "copy t");
    SUR(s->forward(rp));
    SUR(s->backward(B, rp, dt.as<float>()));
    SUR(s->check_error());
    CKC(cudaMemcpyAsync(grads, s->grads.p, MLP_N_PARAMS * 4, cudaMemcpyDeviceToHost, s->stream), "copy grads");
    if (loss) {
        std::vector<float> rl(rp);
        CKC(cudaMemcpyAsync(rl.data(), s->dy.as<float>() + rp * 2, rp * 4, cudaMemcpyDeviceToHost, s->stream),
            "copy loss");
        CKC(cudaStreamSynchronize(s->stream), "sync");
        double sum = 0;
        for (int64_t i = 0; i < B; ++i) sum += rl[i];
        *loss = sum / (double)B;
    }
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

int pop_mlp_train_step(pop_ctx* c, int64_t B, const float* x, const float* t, float lr)
{
    if (!c) return POP_EINVAL;
    std::vector<float> g(MLP_N_PARAMS);
    int rc = pop_mlp_gradients(c, B, x, t, g.data(), nullptr);
    if (rc != POP_OK) return rc;
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    SUR(s->adam(lr));
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

int pop_xi_surrogate_train(pop_ctx* c, int64_t n_pairs, double heldout_frac, uint64_t seed, const double* lambda_lo,
                           const double* lambda_hi, int n_params, int epochs, double* out_heldout_rmse)
{
    pop::TraceRange trace_("pop_xi_surrogate_train");
    if (!c) return POP_EINVAL;
    if (!ctx_has_storage(c, POP_STORE_F64) && !ctx_has_storage(c, POP_STORE_F32))
        return ctx_fail(c, POP_ESTATE, "pop_xi_surrogate_train: load events and injections first");
    if (n_params != 11 + (ctx_n_dims(c) == 7))
        return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_train: n_params must match the loaded samples");
    if (n_pairs < 256 || !(heldout_frac > 0.0 && heldout_frac < 0.5) || epochs < 1 || !lambda_lo || !lambda_hi)
        return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_train: need n_pairs >= 256, 0 < heldout_frac < 0.5, "
                                       "epochs >= 1 and a prior box");
    for (int p = 0; p < n_params; ++p)
        if (!(lambda_hi[p] > lambda_lo[p]) || !std::isfinite(lambda_lo[p]) || !std::isfinite(lambda_hi[p]))
            return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_train: empty or non-finite prior box");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");

    // 1. Lambda drawn uniformly from the box; targets from the Monte Carlo selection term.
    const auto t_gen = std::chrono::steady_clock::now();
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    std::vector<double> lam((size_t)n_pairs * n_params);
    for (int64_t k = 0; k < n_pairs; ++k)
        for (int p = 0; p < n_params; ++p)
            lam[k * n_params + p] = lambda_lo[p] + u01(rng) * (lambda_hi[p] - lambda_lo[p]);
    // FP32 arithmetic (error ~1e-6 in ln xi) is far below the targets' Monte Carlo scatter.
    const int mode = ctx_has_storage(c, POP_STORE_F32) ? POP_MODE_F32 : POP_MODE_F64;
    std::vector<double> lnL(n_pairs), lnxi(n_pairs), neff(n_pairs);
    std::vector<uint32_t> flags(n_pairs);
    for (int64_t k0 = 0; k0 < n_pairs; k0 += GEN_BATCH) {
        const int64_t nb = std::min(GEN_BATCH, n_pairs - k0);
        const int rc = pop_loglik(c, nb, n_params, lam.data() + k0 * n_params, mode, lnL.data() + k0,
                                  lnxi.data() + k0, neff.data() + k0, flags.data() + k0, POP_MEM_HOST);
        if (rc != POP_OK) return rc;
    }
    const double target_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_gen).count();
    std::vector<int64_t> keep;
    for (int64_t k = 0; k < n_pairs; ++k)
        if (std::isfinite(lnxi[k]) && neff[k] > 0.0 && std::isfinite(neff[k]) && !(flags[k] & POP_FLAG_INVALID_LAMBDA))
            keep.push_back(k);
    if ((int64_t)keep.size() < 256) return ctx_fail(c, POP_ENUMERIC, "pop_xi_surrogate_train: too few usable pairs");
    std::shuffle(keep.begin(), keep.end(), rng);
    const int64_t n_hold = std::max<int64_t>(1, (int64_t)std::llround(heldout_frac * (double)keep.size()));
    const int64_t n_train = (int64_t)keep.size() - n_hold;

    // 2. Standardised targets (ln xi, ln N_eff) on the training split.
    for (int i = 0; i < MLP_IN; ++i) {
        s->lo[i] = i < n_params ? lambda_lo[i] : 0.0;
        s->hi[i] = i < n_params ? lambda_hi[i] : 1.0;
    }
    s->n_params = n_params;
    for (int o = 0; o < 2; ++o) {
        double m = 0, v = 0;
        for (int64_t i = 0; i < n_train; ++i) {
            const int64_t k = keep[i];
            m += o == 0 ? lnxi[k] : std::log(neff[k]);
        }
        m /= (double)n_train;
        for (int64_t i = 0; i < n_train; ++i) {
            const int64_t k = keep[i];
            const double d = (o == 0 ? lnxi[k] : std::log(neff[k])) - m;
            v += d * d;
        }
        s->mu[o] = m;
        s->sd[o] = std::sqrt(v / (double)n_train) + 1e-12;
    }
    const int64_t nk = (int64_t)keep.size();
    std::vector<double> lam_k((size_t)nk * n_params);
    std::vector<float> tk((size_t)nk * 2);
    for (int64_t i = 0; i < nk; ++i) {
        const int64_t k = keep[i];
        std::copy(lam.begin() + k * n_params, lam.begin() + (k + 1) * n_params, lam_k.begin() + i * n_params);
        tk[i * 2] = (float)((lnxi[k] - s->mu[0]) / s->sd[0]);
        tk[i * 2 + 1] = (float)((std::log(neff[k]) - s->mu[1]) / s->sd[1]);
    }
    DevBuf d_lam, xall, tall, idx, tb;
    CKC(d_lam.alloc(lam_k.size() * 8), "cudaMalloc");
    CKC(cudaMemcpyAsync(d_lam.p, lam_k.data(), lam_k.size() * 8, cudaMemcpyHostToDevice, s->stream), "copy");
    SUR(s->ensure_rows(TRAIN_BATCH));
    CKC(xall.alloc((size_t)pad128(nk) * MLP_IN_PAD * 2), "cudaMalloc");
    SUR(s->normalise(d_lam.as<double>(), nk, n_params, nullptr, xall.as<__nv_bfloat16>()));
    CKC(tall.alloc(tk.size() * 4), "cudaMalloc");
    CKC(cudaMemcpyAsync(tall.p, tk.data(), tk.size() * 4, cudaMemcpyHostToDevice, s->stream), "copy");
    CKC(idx.alloc(std::max<int64_t>(n_train, 1) * 8), "cudaMalloc");
    CKC(tb.alloc((size_t)TRAIN_BATCH * 2 * 4), "cudaMalloc");

    // 3. Adam on shuffled mini-batches, cosine learning-rate decay.
    CKC(cudaStreamSynchronize(s->stream), "sync");
    const auto t_fit = std::chrono::steady_clock::now();
    SUR(s->init_params(seed ^ 0x9E3779B97F4A7C15ull));
    const int64_t B = std::min<int64_t>(TRAIN_BATCH, n_train);
    const int64_t steps_per_epoch = std::max<int64_t>(1, n_train / B);
    const int64_t total = steps_per_epoch * epochs;
    const double lr0 = 2e-3, lr1 = 2e-5;
    std::vector<int64_t> order(n_train);
    for (int64_t i = 0; i < n_train; ++i) order[i] = i;
    int64_t step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        CKC(cudaMemcpyAsync(idx.p, order.data(), n_train * 8, cudaMemcpyHostToDevice, s->stream), "copy order");
        for (int64_t b = 0; b < steps_per_epoch; ++b, ++step) {
            const double lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + std::cos(M_PI * (double)step / (double)total));
            CKC(mlp_gather(xall.as<__nv_bfloat16>(), tall.as<float>(), idx.as<int64_t>() + b * B, B, pad128(B),
                           s->x0.as<__nv_bfloat16>(), tb.as<float>(), s->stream), "gather");
            SUR(s->forward(pad128(B)));
            SUR(s->backward(B, pad128(B), tb.as<float>()));
            SUR(s->adam((float)lr));
        }
        // keep the host copy of the order alive until the queued copies are done
        CKC(cudaStreamSynchronize(s->stream), "sync");
    }
    SUR(s->check_error());
    s->has_params = true;
    s->fit_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_fit).count();
    s->fit_rows = total * B;
    s->target_seconds = target_seconds;

    // 4. Held-out error in ln xi, and the targets' own Monte Carlo scatter (Var ln xi-hat ~ 1/N_eff).
    std::vector<int64_t> hold(keep.begin() + n_train, keep.end());
    std::vector<double> hl((size_t)n_hold * n_params);
    for (int64_t i = 0; i < n_hold; ++i)
        std::copy(lam.begin() + hold[i] * n_params, lam.begin() + (hold[i] + 1) * n_params, hl.begin() + i * n_params);
    DevBuf d_hl;
    CKC(d_hl.alloc(hl.size() * 8), "cudaMalloc");
    CKC(cudaMemcpyAsync(d_hl.p, hl.data(), hl.size() * 8, cudaMemcpyHostToDevice, s->stream), "copy");
    std::vector<double> pred(n_hold), pred_ln(n_hold), abs_err(n_hold);
    const int rc = infer_device(c, s, n_hold, n_params, d_hl.as<double>(), pred.data(), pred_ln.data(), nullptr);
    if (rc != POP_OK) return rc;
    double se = 0, noise = 0;
    for (int64_t i = 0; i < n_hold; ++i) {
        const double d = pred[i] - lnxi[hold[i]];
        se += d * d;
        noise += 1.0 / neff[hold[i]];
        abs_err[i] = std::fabs(d);
    }
    build_err_table(s, pred_ln, abs_err);
    s->heldout_rmse = std::sqrt(se / (double)n_hold);
    s->heldout_mc_noise = std::sqrt(noise / (double)n_hold);
    s->heldout_excess = std::sqrt(std::max(0.0, s->heldout_rmse * s->heldout_rmse -
                                                  s->heldout_mc_noise * s->heldout_mc_noise));
    s->trusted = s->heldout_excess <= GATE_EXCESS;
    s->trained = true;
    s->version++;
    if (out_heldout_rmse) *out_heldout_rmse = s->heldout_rmse;
    return POP_OK;
}

int pop_xi_surrogate_info(pop_ctx* c, double* heldout_rmse, double* mc_noise, double* excess, int* trusted)
{
    if (!c) return POP_EINVAL;
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->trained) return ctx_fail(c, POP_ESTATE, "pop_xi_surrogate_info: not trained");
    if (heldout_rmse) *heldout_rmse = s->heldout_rmse;
    if (mc_noise) *mc_noise = s->heldout_mc_noise;
    if (excess) *excess = s->heldout_excess;
    if (trusted) *trusted = s->trusted ? 1 : 0;
    return POP_OK;
}

int pop_xi_surrogate_infer(pop_ctx* c, int64_t K, int n_params, const double* lambda, double* out_lnxi,
                           double* out_lnneff, uint8_t* out_fallback, int mem)
{
    pop::TraceRange trace_("pop_xi_surrogate_infer");
    if (!c) return POP_EINVAL;
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->trained) return ctx_fail(c, POP_ESTATE, "pop_xi_surrogate_infer: surrogate not trained");
    if (n_params != s->n_params) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_infer: n_params differs");
    if (K < 0 || (K > 0 && (!lambda || !out_lnxi)) || (mem != POP_MEM_HOST && mem != POP_MEM_DEVICE))
        return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_infer: bad arguments");
    if (K == 0) return POP_OK;
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    DevBuf dl;
    const double* d_lambda = lambda;
    if (mem == POP_MEM_HOST) {
        CKC(dl.alloc((size_t)K * n_params * 8), "cudaMalloc");
        CKC(cudaMemcpyAsync(dl.p, lambda, (size_t)K * n_params * 8, cudaMemcpyHostToDevice, s->stream), "copy");
        d_lambda = dl.as<double>();
    }
    std::vector<double> lx(K), ln(K);
    std::vector<uint8_t> fb(K);
    const int rc = infer_device(c, s, K, n_params, d_lambda, lx.data(), ln.data(), fb.data());
    if (rc != POP_OK) return rc;
    const cudaMemcpyKind kind = mem == POP_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
    CKC(cudaMemcpyAsync(out_lnxi, lx.data(), K * 8, kind, s->stream), "copy");
    if (out_lnneff) CKC(cudaMemcpyAsync(out_lnneff, ln.data(), K * 8, kind, s->stream), "copy");
    if (out_fallback) CKC(cudaMemcpyAsync(out_fallback, fb.data(), K, kind, s->stream), "copy");
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

int pop_xi_surrogate_save(pop_ctx* c, const char* path)
{
    if (!c) return POP_EINVAL;
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->trained || !path) return ctx_fail(c, POP_ESTATE, "pop_xi_surrogate_save: not trained or no path");
    std::vector<float> p(MLP_N_PARAMS);
    SUR(s->get_params_host(p.data()));
    std::ofstream f(path, std::ios::binary);
    if (!f) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_save: cannot open file");
    const int32_t version = 2, np = s->n_params, trusted = s->trusted;
    const int64_t n = MLP_N_PARAMS;
    f.write(CKPT_MAGIC, 8);
    f.write((const char*)&version, 4);
    f.write((const char*)&np, 4);
    f.write((const char*)s->lo, sizeof s->lo);
    f.write((const char*)s->hi, sizeof s->hi);
    f.write((const char*)s->mu, sizeof s->mu);
    f.write((const char*)s->sd, sizeof s->sd);
    f.write((const char*)&s->heldout_rmse, 8);
    f.write((const char*)&s->heldout_mc_noise, 8);
    f.write((const char*)&s->heldout_excess, 8);
    f.write((const char*)&trusted, 4);
    f.write((const char*)&s->table, sizeof s->table);
    f.write((const char*)&s->budget, 8);
    f.write((const char*)&n, 8);
    f.write((const char*)p.data(), n * 4);
    if (!f) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_save: write failed");
    return POP_OK;
}

int pop_xi_surrogate_load(pop_ctx* c, const char* path)
{
    if (!c) return POP_EINVAL;
    if (!path) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_load: no path");
    std::ifstream f(path, std::ios::binary);
    if (!f) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_load: cannot open file");
    char magic[8];
    int32_t version = 0, np = 0, trusted = 0;
    int64_t n = 0;
    double lo[MLP_IN], hi[MLP_IN], mu[2], sd[2], rmse, noise, excess, budget = DEFAULT_BUDGET_NATS;
    ErrTable table{};
    f.read(magic, 8);
    f.read((char*)&version, 4);
    f.read((char*)&np, 4);
    f.read((char*)lo, sizeof lo);
    f.read((char*)hi, sizeof hi);
    f.read((char*)mu, sizeof mu);
    f.read((char*)sd, sizeof sd);
    f.read((char*)&rmse, 8);
    f.read((char*)&noise, 8);
    f.read((char*)&excess, 8);
    f.read((char*)&trusted, 4);
    if (version == 2) {
        f.read((char*)&table, sizeof table);
        f.read((char*)&budget, 8);
    } else {  // version 1 has no per-Lambda table: every Lambda gets no error claim
        for (int b = 0; b < ERR_BINS; ++b) table.err[b] = INFINITY;
        for (int b = 0; b < ERR_BINS - 1; ++b) table.edge[b] = INFINITY;
    }
    f.read((char*)&n, 8);
    if (!f || memcmp(magic, CKPT_MAGIC, 8) != 0 || (version != 1 && version != 2) || n != MLP_N_PARAMS ||
        (np != 11 && np != 12))
        return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_load: not a surrogate checkpoint of a known version");
    std::vector<float> p(n);
    f.read((char*)p.data(), n * 4);
    if (!f) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_load: truncated file");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    SUR(s->set_params_host(p.data()));
    memcpy(s->lo, lo, sizeof lo);
    memcpy(s->hi, hi, sizeof hi);
    memcpy(s->mu, mu, sizeof mu);
    memcpy(s->sd, sd, sizeof sd);
    s->n_params = np;
    s->heldout_rmse = rmse;
    s->heldout_mc_noise = noise;
    s->heldout_excess = excess;
    s->trusted = trusted != 0;
    s->table = table;
    s->budget = budget;
    s->trained = true;
    s->version++;
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

int pop_xi_surrogate_train_stats(pop_ctx* c, double* target_seconds, double* fit_seconds, int64_t* fit_rows)
{
    if (!c) return POP_EINVAL;
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->trained || s->fit_rows == 0)
        return ctx_fail(c, POP_ESTATE, "pop_xi_surrogate_train_stats: no training in this context");
    if (target_seconds) *target_seconds = s->target_seconds;
    if (fit_seconds) *fit_seconds = s->fit_seconds;
    if (fit_rows) *fit_rows = s->fit_rows;
    return POP_OK;
}

int pop_xi_surrogate_set_budget(pop_ctx* c, double nats)
{
    if (!c) return POP_EINVAL;
    if (!(nats >= 0.0)) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_set_budget: need a budget >= 0 nats");
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    s->budget = nats;
    s->version++;  // the captured gate holds the budget
    return POP_OK;
}

int pop_xi_surrogate_error(pop_ctx* c, int64_t K, int n_params, const double* lambda, double* out_err, int mem)
{
    pop::TraceRange trace_("pop_xi_surrogate_error");
    if (!c) return POP_EINVAL;
    int st;
    Surrogate* s = ctx_surrogate(c, &st);
    if (!s) return st;
    if (!s->trained) return ctx_fail(c, POP_ESTATE, "pop_xi_surrogate_error: surrogate not trained");
    if (n_params != s->n_params) return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_error: n_params differs");
    if (K < 0 || (K > 0 && (!lambda || !out_err)) || (mem != POP_MEM_HOST && mem != POP_MEM_DEVICE))
        return ctx_fail(c, POP_EINVAL, "pop_xi_surrogate_error: bad arguments");
    if (K == 0) return POP_OK;
    CKC(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    DevBuf dl;
    const double* d_lambda = lambda;
    if (mem == POP_MEM_HOST) {
        CKC(dl.alloc((size_t)K * n_params * 8), "cudaMalloc");
        CKC(cudaMemcpyAsync(dl.p, lambda, (size_t)K * n_params * 8, cudaMemcpyHostToDevice, s->stream), "copy");
        d_lambda = dl.as<double>();
    }
    std::vector<double> lx(K), ln(K), e(K);
    const int rc = infer_device(c, s, K, n_params, d_lambda, lx.data(), ln.data(), nullptr);
    if (rc != POP_OK) return rc;
    for (int64_t k = 0; k < K; ++k) e[k] = err_bound(s->table, ln[k]);
    CKC(cudaMemcpyAsync(out_err, e.data(), K * 8, mem == POP_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice,
                        s->stream), "copy");
    CKC(cudaStreamSynchronize(s->stream), "sync");
    return POP_OK;
}

}  // extern "C"
