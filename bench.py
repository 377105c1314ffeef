"""Throughput of the population likelihood on GB300.

Workload: 1000 events x 4096 posterior samples each (dense), 10^7 injection
draws (about 1.1e6 found), batches of K = 1024 Lambda points, the mass + spin
model; synthetic, seeded data shaped like a catalog (no real posteriors
offline).  One step = one pop_loglik over the K-batch: per-Lambda prologue,
sample weights for every (sample, Lambda) and (injection, Lambda) pair,
per-event segmented sums, selection term, finalise.  The headline form is
plain FP64; the FP32 form is timed in the same run and reported under
"forms".  The feature arrays (375 MB FP64, 208 MB FP32) exceed the 129 MB L2,
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank evaluates its own K-batch (replicas, weak scaling);
rank 0 prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1904_02863_gb300 import replicas, synth  # noqa: E402

METRIC = "ln L(Lambda) evals/s at 1000 events x 4096 samples + 1e6 inj"
WORKLOAD = "f64_catalog_1000x4096_inj1e7"

# Algorithmic FP64-pipe operations per (sample, Lambda) pair of the weight
# kernel: 13 add/mul/fma + 3 exp (2 each) + 1 expm1 (6) + 1 reciprocal (3);
# +1 fma for the squared weight on injection pairs.  (The exponentials' table
# index, exp's table value times 1 + (e^r - 1 - r) and expm1's series coefficient
# are formed in FP32 and integer operations, off the FP64 pipe; the mass mixture's
# larger constant sits in the tilt factor, so neither mass exponent adds its own.)
FP64_OPS_PER_PAIR = 28
FP64_OPS_PER_INJ_PAIR = 29
# GB300: 2 FP64 FMA lanes per SM per clock (1.25 TFLOP/s nominal at 2070 MHz
# over 152 SMs); peak op rate = 2 * SMs * clock.
FP64_LANES_PER_SM = 2
FP32_LANES_PER_SM = 128
# MUFU issue slots per SM per clock in ex2.approx units (rcp.approx takes two), and per
# in-support pair of the FP32 weight (4 ex2 + 1 rcp).
MUFU_SLOTS_PER_SM = 32
MUFU_SLOTS_PER_PAIR = 6
# FP32 lane operations (FMA pipe) per in-support pair of the float-float weight kernel, from its
# ncu capture (profiles/weight_ff_catalog400x4096_K1024_full.md): FMA pipe 70.35% of 45.39 M active
# cycles x 128 lanes x 152 SMs over 1.718e9 in-support pairs.
FF_OPS_PER_PAIR = 362
SMS = 152
SM_MAX_MHZ = 2070.0
def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# The network's training is a seconds-long loop of GEMMs: its denominator is the sustained cuBLAS
# BF16 rate the GB300s measured (the profiling recipe's 1.7 PFLOP/s when the file is absent).
_PEAKS = _measured_peaks()
BF16_PEAK_TFLOPS = float(_PEAKS.get("bf16_tflops_sustained") or 1700.0)
BF16_PEAK_BASIS = "of measured (sustained)" if _PEAKS.get("bf16_tflops_sustained") else "of fallback (sustained)"
# DRAM bytes per (sample or injection) unit of one weight_f64 launch, from the ncu capture in
# profiles/weight_f64_catalog400x4096_K64_full.md (153.90 MB / 2,077,126 units); a launch
# reads every chunk from DRAM once, so traffic scales with the units.
F64_DRAM_BYTES_PER_UNIT = 153.90e6 / 2077126


def in_support_pairs(theta, lam):
    """(sample, Lambda) pairs inside the support (mmin < m1 <= mmax, fl64(q m1) >= mmin).

    Only those carry algorithmic work: outside the support the weight is 0 by
    definition and no density is evaluated.  Exact count, per Lambda.
    """
    m1 = theta[:, 0]
    m2 = theta[:, 1] * theta[:, 0]
    m2s = np.sort(m2)
    mmin, mmax = lam[:, 2], lam[:, 3]
    total = int((len(m2s) - np.searchsorted(m2s, mmin, side="left")).sum())
    # remove m1 > mmax (the few high-mass samples) and m1 <= mmin with m2 >= mmin (q = 1 ties)
    hi = m1 > mmax.min()
    tie = m2 >= m1
    for k0 in range(0, len(lam), 64):  # bounded temporaries on large catalogs
        a, b = mmin[None, k0:k0 + 64], mmax[None, k0:k0 + 64]
        total -= int(((m2[hi, None] >= a) & (m1[hi, None] > b)).sum())
        total -= int(((m2[tie, None] >= a) & (m1[tie, None] <= a)).sum())
    return total


def ff_roofline(pairs, weight_ms):
    """The float-float weight kernel against the FP32 FMA pipe (128 lanes per SM per clock): FF_OPS_PER_PAIR
    FP32 lane operations per in-support pair, counted from the kernel's executed FMA-pipe instructions."""
    peak = FP32_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6
    achieved = FF_OPS_PER_PAIR * pairs / (weight_ms * 1e-3)
    return {"bound": "alu", "kernel": "weight_ff_kernel", "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "Top/s (FP32 FMA pipe)", "frac": achieved / peak, "traffic": None, "weight_ms": weight_ms,
            "in_support_pairs": pairs, "ops_per_in_support_pair": FF_OPS_PER_PAIR,
            "peak_basis": "128 FP32 lanes/SM/clk x 152 SMs x 2070 MHz"}


def f32_roofline(pairs, weight_ms):
    """The FP32 weight kernel against its binding unit, MUFU: per in-support pair 4 ex2.approx
    (32 per SM per clock on GB300) and 1 rcp.approx (16 per clock, two ex2 slots), against 22
    FP32 lane operations on the FMA pipe (128 per SM per clock): 6/32 > 22/128 clocks."""
    peak = MUFU_SLOTS_PER_SM * SMS * SM_MAX_MHZ * 1e6
    achieved = MUFU_SLOTS_PER_PAIR * pairs / (weight_ms * 1e-3)
    return {"bound": "alu", "kernel": "weight_f32_kernel", "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "T MUFU slots/s", "frac": achieved / peak, "traffic": None, "weight_ms": weight_ms,
            "in_support_pairs": pairs, "slots_per_in_support_pair": MUFU_SLOTS_PER_PAIR,
            "peak_basis": "MUFU ex2 32/SM/clk (rcp 16: 2 slots) x 152 SMs x 2070 MHz, rates measured by pop_pipe_rates"}


def grid_support_triples(m1, q, lam):
    """(m1 node, q node, Lambda) triples inside the support of the grid selection term:
    mmin < m1 <= mmax, q <= 1 and fl64(q m1) >= mmin.  One FMA each is the algorithmic
    work of the node contraction.  Exact count."""
    nb = int(np.searchsorted(q, 1.0, side="right"))
    qq = q[:nb]
    total = 0
    for L in lam:
        mmin, mmax = L[2], L[3]
        rows = m1[(m1 > mmin) & (m1 <= mmax)]
        b0 = np.searchsorted(qq, mmin / rows, side="left")
        for _ in range(2):  # the exact edge: fl64(q m1) >= mmin
            dn = (b0 > 0) & (qq[np.maximum(b0 - 1, 0)] * rows >= mmin)
            b0 = np.where(dn, b0 - 1, b0)
            up = (b0 < nb) & (qq[np.minimum(b0, nb - 1)] * rows < mmin)
            b0 = np.where(up, b0 + 1, b0)
        total += int((nb - b0).sum())
    return total


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--oracle-lambdas", type=int, default=32, help="Lambda rows in the CPU sample")
    p.add_argument("--events", type=int, default=1000, help="events (a smaller catalog for profiling captures)")
    p.add_argument("--K", type=int, default=1024, help="Lambda points per step")
    p.add_argument("--mode", default="both", choices=["both", "f64", "f32", "ff"],
                   help="both: the FP64 headline and every form; f64 / f32 / ff: that mode alone")
    p.add_argument("--workload", default="catalog",
                   choices=["catalog", "ragged", "grid", "cbc", "grad", "sampler", "learned", "scan"],
                   help="catalog: 1000 events x 4096 samples + 1e7 injection draws (default; every form); "
                        "ragged: 2000 ragged CSR events + redshift, uneven batches; "
                        "sampler: the stretch-move ensemble sampler driving FP32 ln L on the catalog; "
                        "learned: 10 x 1000 + redshift with the trained ln xi network; "
                        "scan: evals/s and roofline over 1e4 .. 2e7 posterior samples")
    return p.parse_args()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    return replicas.init_from_env()


barrier = replicas.barrier
max_over_ranks = replicas.max_over_ranks


def cpu_baseline(cat, inj, lam, n_rows, gpu_f64=None):
    """The oracle timed on the first ``n_rows`` Lambda of the batch.  Given the FP64 kernel's
    outputs for the batch, also reports their distance to the oracle on those rows, in units of
    the FP64 tolerance 1e-12 (|sum_i ln(S_i/n_i)| + N |ln xi|)."""
    import oracle
    cores = host_cores()
    sub = lam[:n_rows]
    t0 = time.perf_counter()
    ref = oracle.loglik(cat, inj, sub, nthreads=cores)
    dt = time.perf_counter() - t0
    out = {"value": n_rows / dt, "unit": "evals/s", "cores": min(cores, n_rows), "kind": "oracle",
           "sample": f"{n_rows} Lambda rows of the same workload (full 1000x4096 catalog and "
                     f"{inj.n_found} found injections per row), FP64, OpenMP over Lambda",
           "seconds": dt}
    # The paper compares against single-threaded CPU code: the same oracle on one thread.
    n1 = min(2, n_rows)
    t0 = time.perf_counter()
    oracle.loglik(cat, inj, lam[:n1], nthreads=1)
    dt1 = time.perf_counter() - t0
    out["single_thread"] = {"value": n1 / dt1, "unit": "evals/s", "cores": 1, "rows": n1, "seconds": dt1}
    if gpu_f64 is not None:
        n = cat.n_events
        g = [np.asarray(x)[:n_rows] for x in gpu_f64]
        fin = np.isfinite(ref[0]) & np.isfinite(g[0])
        tol = 1e-12 * (np.abs(np.where(fin, ref[0], 0.0) + n * ref[1]) + n * np.abs(ref[1])) + 1e-13
        ratio = float(np.max(np.abs(g[0][fin] - ref[0][fin]) / tol[fin])) if fin.any() else 0.0
        out["parity_f64_kernel"] = {
            "rows": int(n_rows), "max_abs_dlnL": float(np.max(np.abs(g[0][fin] - ref[0][fin]))) if fin.any() else 0.0,
            "max_over_f64_tol": ratio,
            "flags_equal": bool((g[3].view(np.uint32) == ref[3].view(np.uint32)).all()),
            "finite_rows_agree": bool((np.isfinite(ref[0]) == np.isfinite(g[0])).all())}
    return out


def dlnl_stats(d):
    """mean, 99th percentile and max of |Delta ln L| (0 for no rows)."""
    if d.size == 0:
        return {"rows": 0, "mean": 0.0, "p99": 0.0, "max": 0.0}
    return {"rows": int(d.size), "mean": float(d.mean()), "p99": float(np.quantile(d, 0.99)), "max": float(d.max())}


def precision_vs(res, ref, rows=None):
    """|Delta ln L| and the relative Delta xi of the outputs ``res`` against ``ref`` over every
    Lambda of the batch (rows where both ln L are finite), or over the boolean mask ``rows``."""
    a, b = res[0], ref[0]
    both = np.isfinite(a) & np.isfinite(b)
    if rows is not None:
        both &= rows
    d = np.abs(a[both] - b[both])
    dxi = np.abs(np.expm1(res[1][both] - ref[1][both]))
    return {"finite_rows_agree": bool((np.isfinite(a) == np.isfinite(b)).all()), "abs_dlnL": dlnl_stats(d),
            "rel_dxi_max": float(dxi.max()) if dxi.size else 0.0}


def time_mode(B, like, dev_lam, outs, mode, steps, warmup, world, stream):
    """(ms over ``steps`` pop_loglik calls on device buffers, mean weight-kernel ms): CUDA events on
    the context's stream, a barrier and a synchronize on both sides, max over ranks."""
    import torch
    for _ in range(warmup):
        B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wms = []
    start.record(stream)
    for _ in range(steps):
        B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
        wms.append(B.pop_last_kernel_ms(like.ctx)[0])
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    return max_over_ranks(start.elapsed_time(stop), world), statistics.mean(wms)


def host_outputs(outs):
    r = [o.cpu().numpy().copy() for o in outs]
    r[3] = r[3].view(np.uint32)
    return r


def ff_form(B, like, lam, dev_lam, outs, args, world, stream, n_pairs, n_events, f64):
    """FP64-grade ln L with the sample weights in float-float arithmetic (POP_MODE_FF): its
    evals/s, and its distance to the FP64 kernel's ln L (``f64``, host outputs) in units of the
    FP64 parity tolerance 1e-12 (|sum_i ln(S_i/n_i)| + N |ln xi|) for every Lambda of the batch."""
    ms, w = time_mode(B, like, dev_lam, outs, B.POP_MODE_FF, args.steps, args.warmup, world, stream)
    ffh = host_outputs(outs)
    n = n_events
    fin = np.isfinite(f64[0])
    a = np.abs(np.where(fin, f64[0], 0.0) + n * f64[1])
    tol = 1e-12 * (a + n * np.abs(f64[1])) + 1e-13
    ratio = float(np.max(np.abs(ffh[0][fin] - f64[0][fin]) / tol[fin])) if fin.any() else 0.0
    K = len(lam)
    return {"value": world * K * args.steps / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms / args.steps,
            "weight_ms": w, "dtype": "float-float (2 x f32)", "roofline": ff_roofline(n_pairs, w),
            "max_dlnL_over_f64_tol": ratio, "flags_equal": bool((ffh[3] == f64[3]).all()),
            "in_support_pairs": n_pairs}


# Tensor-core work of one training row (forward + backward, the 12-input layer unpadded):
# forward 2 (12*256 + 3*256^2 + 256*2), weight gradients the same, input gradients
# 2 (3*256^2 + 256*2); Adam and the SiLU epilogues are not counted.
MLP_FLOP_PER_ROW = 2 * (12 * 256 + 3 * 256 ** 2 + 256 * 2) * 2 + 2 * (3 * 256 ** 2 + 256 * 2)


def train_surrogate(B, like, n_params, n_pairs, epochs, seed):
    """Trains the ln xi network on the context's own injections; returns the training report."""
    box = synth.LAMBDA_BOX[:n_params]
    t0 = time.perf_counter()
    B.pop_xi_surrogate_train(like.ctx, n_pairs, box[:, 0], box[:, 1], epochs=epochs, seed=seed)
    train_s = time.perf_counter() - t0
    info = B.pop_xi_surrogate_info(like.ctx)
    st = B.pop_xi_surrogate_train_stats(like.ctx)
    fit_tflops = st["fit_rows"] * MLP_FLOP_PER_ROW / st["fit_seconds"] / 1e12
    return {"pairs": n_pairs, "heldout_frac": 0.1, "epochs": epochs, "seconds": train_s,
            "target_seconds": st["target_seconds"], "fit_seconds": st["fit_seconds"],
            "fit_tflops": fit_tflops, "fit_frac_of_bf16_peak": fit_tflops / BF16_PEAK_TFLOPS,
            "bf16_peak_tflops": BF16_PEAK_TFLOPS, "bf16_peak_basis": BF16_PEAK_BASIS,
            "heldout_rmse_lnxi": info["heldout_rmse"], "heldout_mc_noise": info["mc_noise"],
            "trusted": info["trusted"]}


def gated_form(B, like, lam, dev_lam, outs, args, world, stream, ref64, mc32, steps, budget):
    """POP_MODE_F32_SURROGATE at one error budget: evals/s, the share of Lambda on the network,
    and |Delta ln L| against the FP64 kernel on all rows and on the network's rows (where it is
    at most the budget when the error bounds hold)."""
    B.pop_xi_surrogate_set_budget(like.ctx, budget)
    ms, w = time_mode(B, like, dev_lam, outs, B.POP_MODE_F32_SURROGATE, steps, args.warmup, world, stream)
    sur = host_outputs(outs)
    used = (sur[3] & B.POP_FLAG_SURROGATE_USED) != 0
    K = len(lam)
    return {"budget_nats": budget, "value": world * K * steps / (ms * 1e-3), "ms_per_step": ms / steps,
            "weight_ms": w, "surrogate_used_frac": float(used.mean()),
            "vs_f64": precision_vs(sur, ref64), "vs_f64_network_rows": precision_vs(sur, ref64, used)["abs_dlnL"],
            "vs_f32_mc_network_rows": dlnl_stats(np.abs(sur[0] - mc32[0])[used & np.isfinite(mc32[0])])}


def surrogate_form(B, like, lam, dev_lam, outs, args, world, stream, ref64, mc32, n_params=11, steps=None,
                   seed=None, budgets=(0.25,)):
    """FP32 weights + the trained ln xi network, which replaces the Monte Carlo xi for the Lambda
    whose error bound times N fits the budget (pop_xi_surrogate_error); Monte Carlo elsewhere.

    Training (2e5 Lambda from the prior box, 10% held out, targets from this workload's own
    injections, 60 epochs) is setup, reported separately with its tensor-core rate.  The
    ungated entry (budget 1e9) shows what the gate keeps out.
    """
    steps = steps or args.steps
    train = train_surrogate(B, like, n_params, 200000, 60, seed if seed is not None else synth.seed_for(2, 5))
    err = B.pop_xi_surrogate_error(like.ctx, lam)
    n_events = like.n_events
    out = {"dtype": "f32+bf16 network", "training": train,
           "n_x_err_bound_nats": {"p10": float(np.quantile(n_events * err, 0.1)),
                                  "p50": float(np.quantile(n_events * err, 0.5)),
                                  "p90": float(np.quantile(n_events * err, 0.9))}}
    for b in budgets:
        out[f"budget_{b:g}"] = gated_form(B, like, lam, dev_lam, outs, args, world, stream, ref64, mc32, steps, b)
    out["ungated"] = gated_form(B, like, lam, dev_lam, outs, args, world, stream, ref64, mc32, steps, 1e9)
    B.pop_xi_surrogate_set_budget(like.ctx, 0.25)
    first = out[f"budget_{budgets[0]:g}"]
    out["value"] = first["value"]
    out["unit"] = "evals/s"
    return out


def grid_form(B, like, lam, dev_lam, outs, args, world, stream):
    """ln L with the selection term on the dense (m1, q) campaign grid (3001 x 801
    nodes, the paper's grid VT) instead of the injections, FP64 and FP32; the
    grid's node contraction gets its own roofline (FP64 pipe, resp. FP32 FMA)."""
    m1, q, pdet = synth.campaign_vt_grid()
    B.pop_load_vt_grid(like.ctx, m1, q, pdet)
    B.pop_set_xi_source(like.ctx, B.POP_XI_GRID)
    triples = grid_support_triples(m1, q, lam)
    K = len(lam)
    out = {"grid": {"m1_nodes": int(m1.size), "q_nodes": int(q.size), "pdet": "sigmoid((m1 - 20)/5)",
                    "in_support_triples": triples}}
    peaks = {"f64": (FP64_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6, "2 FP64 lanes/SM/clk x 152 SMs x 2070 MHz",
                     "Top/s (FP64 pipe)", "gv_setup64_kernel + gv_main_kernel"),
             "f32": (FP32_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6, "128 FP32 FMA lanes/SM/clk x 152 SMs x 2070 MHz",
                     "Top/s (FP32 FMA)", "gv_setup32_kernel + gv_main32_kernel")}
    for name, mode in (("f64", B.POP_MODE_F64), ("f32", B.POP_MODE_F32)):
        ms, w = time_mode(B, like, dev_lam, outs, mode, args.steps, args.warmup, world, stream)
        cms, tms = B.pop_xi_grid_last_ms(like.ctx)
        peak, basis, unit, kern = peaks[name]
        ach = triples / (cms * 1e-3)
        out[name] = {"value": world * K * args.steps / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms / args.steps,
                     "weight_ms": w, "grid_ms": tms, "dtype": name,
                     "roofline": {"bound": "alu", "kernel": kern, "achieved": ach / 1e12, "peak": peak / 1e12,
                                  "unit": unit, "frac": ach / peak, "contraction_ms": cms,
                                  "ops_per_launch": triples, "peak_basis": basis, "traffic": None}}
    B.pop_set_xi_source(like.ctx, B.POP_XI_INJECTIONS)
    return out


# FP64-pipe operations per in-support (sample, Lambda) pair of the gradient kernel: the weight
# split into its power-law and peak parts (3 exp, 1 expm1, 1 reciprocal and their FMAs), the
# 11-12 score terms and the 14 sums, with the loop-invariant terms hoisted: the DFMA + DADD + DMUL
# count per in-support pair of the ncu capture in profiles/grad_weight_catalog100x4096_K16_full.md
# (105), less the FP64 operations that the 3 exp (5 each) and the expm1 (4) no longer spend on
# the FP64 pipe: 86.
FP64_OPS_PER_GRAD_PAIR = 86


def grad_form(B, like, lam, args, world, n_pairs):
    """ln L and its gradient with respect to Lambda (pop_loglik_grad, FP64) on the same workload
    and K; the gradient kernel gets its own roofline (FP64 pipe)."""
    K = len(lam)
    for _ in range(args.warmup):
        B.pop_loglik_grad(like.ctx, lam)
    barrier(world)
    ws, ts = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        B.pop_loglik_grad(like.ctx, lam)
        w, t = B.pop_last_kernel_ms(like.ctx)
        ws.append(w)
        ts.append(t)
    wall = max_over_ranks(time.perf_counter() - t0, world)
    w, t = max_over_ranks(statistics.median(ws), world), max_over_ranks(statistics.median(ts), world)
    peak = FP64_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6
    ach = n_pairs * FP64_OPS_PER_GRAD_PAIR / (w * 1e-3)
    return {"value": world * K / (t * 1e-3), "unit": "evals/s (ln L + gradient)", "ms_per_call": t,
            "weight_ms": w, "dtype": "f64",
            "e2e": {"value": world * K * args.steps / wall, "unit": "evals/s", "h2d_bytes_per_step": int(lam.nbytes),
                    "d2h_bytes_per_step": int(K * 8 * (lam.shape[1] + 1) + 4 * K)},
            "roofline": {"bound": "alu", "kernel": "grad_weight_kernel", "achieved": ach / 1e12, "peak": peak / 1e12,
                         "unit": "Top/s (FP64 pipe)", "frac": ach / peak, "ops_per_in_support_pair":
                             FP64_OPS_PER_GRAD_PAIR, "traffic": None}}


# FMA-pipe operations per (bin, parameter row, detector) unit of the CBC sums kernel:
# two complex multiply-adds (P e, Q e: 8) and the time-shift recurrence e <- e w (4).
CBC_FMA_PER_UNIT = 12


def cbc_form(B, like, args, world, rank):
    """Second workload: the single-event CBC likelihood (Eq. cbclike) with per-detector
    time shifts, M = 2^18 bins (128 s from 20 Hz), 3 detectors, K = 256 parameter rows per
    call, FP64 and FP32; the time-shifted sums kernel gets its own roofline, and the
    oracle (direct evaluation) is timed on 16 rows beside it."""
    M, K, T = 2 ** 18, 256, 128.0
    c = synth.make_cbc(M, T=T, seed=synth.seed_for(6, 0))
    th = synth.make_cbc_thetas(c, K, seed=synth.seed_for(6, 2) + 7919 * rank)
    B.pop_cbc_load(like.ctx, c.f0, c.df, c.data, c.psd, c.hp, c.hc)
    units = K * c.n_det * M
    out = {"config": {"bins": M, "detectors": c.n_det, "K": K, "segment_s": T, "f_min_hz": c.f0,
                      "template": "leading-order stationary-phase chirp", "l2": "P, Q arrays 25 MB FP32 (L2-resident)"}}
    peaks = {"f64": (FP64_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6, "Top/s (FP64 pipe)", "cbc_sum_kernel<double>"),
             "f32": (FP32_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6, "Top/s (FP32 FMA)", "cbc_sum_kernel<float>")}
    for name, mode in (("f64", B.POP_MODE_F64), ("f32", B.POP_MODE_F32)):
        for _ in range(args.warmup):
            B.pop_cbc_loglik(like.ctx, th, mode)
        sums, tots = [], []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            B.pop_cbc_loglik(like.ctx, th, mode)
            a, b = B.pop_cbc_last_ms(like.ctx)
            sums.append(a)
            tots.append(b)
        wall = time.perf_counter() - t0
        sm, tm = statistics.median(sums), statistics.median(tots)
        peak, unit, kern = peaks[name]
        ach = units * CBC_FMA_PER_UNIT / (sm * 1e-3)
        out[name] = {"value": world * K / (tm * 1e-3), "unit": "evals/s", "ms_per_call": tm, "sum_kernel_ms": sm,
                     "e2e": {"value": world * K * args.steps / wall, "unit": "evals/s",
                             "h2d_bytes_per_step": int(th.nbytes), "d2h_bytes_per_step": int(K * 12)},
                     "roofline": {"bound": "alu", "kernel": kern, "achieved": ach / 1e12, "peak": peak / 1e12,
                                  "unit": unit, "frac": ach / peak, "ops_per_launch": units * CBC_FMA_PER_UNIT,
                                  "peak_basis": "lanes/SM/clk x 152 SMs x 2070 MHz", "traffic": None}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        n = 16
        t0 = time.perf_counter()
        oracle.cbc_loglik(c.f0, c.df, c.data, c.psd, c.hp, c.hc, th[:n], nthreads=host_cores())
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n / dt, "unit": "evals/s", "cores": min(host_cores(), n), "kind": "oracle",
                               "sample": f"{n} parameter rows of the same data, FP64, OpenMP over rows"}
    return out


def run_grid(args, B, rank, local, world):
    """Standalone grid selection term: ln xi_grid (pop_xi_grid) for K = 1024 Lambda on the
    3001 x 801 campaign grid, FP64 headline and FP32 form; value = Lambda evaluated / s."""
    import torch
    m1, q, pdet = synth.campaign_vt_grid()
    K = 1024
    lam = synth.make_lambdas(K, 11, seed=synth.seed_for(2, 2) + 7919 * rank)
    ctx = B.pop_create(local, torch.cuda.current_stream(local))
    B.pop_load_vt_grid(ctx, m1, q, pdet)
    triples = grid_support_triples(m1, q, lam)
    res = {}
    with Clocks(local) as clk:
        for name, mode in (("f64", B.POP_MODE_F64), ("f32", B.POP_MODE_F32)):
            for _ in range(args.warmup):
                B.pop_xi_grid(ctx, lam, mode)
            barrier(world)
            c_ms, t_ms = [], []
            t0 = time.perf_counter()
            for _ in range(args.steps):
                B.pop_xi_grid(ctx, lam, mode)
                c, t = B.pop_xi_grid_last_ms(ctx)
                c_ms.append(c)
                t_ms.append(t)
            wall = max_over_ranks(time.perf_counter() - t0, world)
            res[name] = (max_over_ranks(statistics.median(c_ms), world), max_over_ranks(statistics.median(t_ms), world),
                         wall)
    B.pop_destroy(ctx)
    c64, t64, w64 = res["f64"]
    c32, t32, w32 = res["f32"]
    peak64 = FP64_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6
    line = {"metric": "ln xi_grid(Lambda) evals/s, 3001 x 801 (m1, q) grid", "value": world * K / (t64 * 1e-3),
            "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t64,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "grid_vt_3001x801", "K": K, "in_support_triples": triples,
                       "parallelism": f"replicas{world}", "l2": "grid and scratch L2-resident (29 MB)"},
            "roofline": {"bound": "alu", "kernel": "gv_setup64_kernel + gv_main_kernel", "achieved": triples / (c64 * 1e-3) / 1e12,
                         "peak": peak64 / 1e12, "unit": "Top/s (FP64 pipe)",
                         "frac": triples / (c64 * 1e-3) / peak64, "traffic": None},
            "e2e": {"value": world * K * args.steps / w64, "unit": "evals/s", "h2d_bytes_per_step": int(lam.nbytes),
                    "d2h_bytes_per_step": int(K * 12)},
            "forms": {"f32": {"value": world * K / (t32 * 1e-3), "unit": "evals/s", "contraction_ms": c32,
                              "frac_of_ffma_peak": triples / (c32 * 1e-3) / (FP32_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6)}},
            "gpu_launches": 7 * args.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)


def run_cbc(args, B, rank, local, world):
    """Second workload alone: the single-event CBC likelihood form (see cbc_form)."""
    import torch
    like = B.Likelihood(local, torch.cuda.current_stream(local))
    with Clocks(local) as clk:
        f = cbc_form(B, like, args, world, rank)
    like.close()
    f64 = f["f64"]
    line = {"metric": "single-event CBC ln L evals/s, 3 detectors x 2^18 bins", "value": f64["value"],
            "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": f64["ms_per_call"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": dict(f["config"], workload="cbc_bns_2e18",
                                                                 parallelism=f"replicas{world}"),
            "roofline": f64["roofline"], "e2e": f64["e2e"], "forms": {"f32": f["f32"]},
            "gpu_launches": 3 * args.steps, "clocks": clk.summary()}
    if "cpu_baseline" in f:
        line["cpu_baseline"] = f["cpu_baseline"]
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)


def run_sampler(args, B, rank, local, world):
    """The ensemble sampler over Lambda on the catalog workload: 2048 walkers, each half-step one
    batch of 1024 proposals through pop_loglik (FP32 weights), from Python with host arrays.
    One step = one sweep of both halves; value = proposals evaluated per second, host time
    around the whole loop (proposal arithmetic, copies and the GPU pipeline)."""
    import torch
    from paper_1904_02863_gb300 import sampler
    cat, inj, _ = synth.make_workload(WORKLOAD, scale=args.events / 1000.0)
    like = B.Likelihood(local, torch.cuda.current_stream(local)).load(cat, inj, storage=B.POP_STORE_F32)
    box = synth.LAMBDA_BOX[:11]
    log_prob = sampler.population_log_posterior(like, box[:, 0], box[:, 1], mode=B.POP_MODE_F32)
    W = 2048
    p0 = synth.make_lambdas(W, 11, seed=synth.seed_for(2, 2) + 7919 * rank)
    chain, _, _ = sampler.stretch_sample(log_prob, p0, max(args.warmup, 1), seed=11 + rank)
    p0 = chain[-1]
    torch.cuda.synchronize()
    barrier(world)
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        chain, lps, acc = sampler.stretch_sample(log_prob, p0, args.steps, seed=12 + rank)
        torch.cuda.synchronize()
        wall = max_over_ranks(time.perf_counter() - t0, world)
    evals = world * args.steps * W
    line = {"metric": "ensemble-sampler proposals evaluated/s (stretch move, 2048 walkers, FP32 ln L, 1000 x 4096 catalog)",
            "value": evals / wall, "unit": "proposals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sampler_catalog_1000x4096", "walkers": W, "batch_per_half_step": W // 2,
                       "events": cat.n_events, "n_found": int(inj.n_found), "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (FP32 features 44 B/sample)"},
            "acceptance": float(acc.mean()),
            "e2e": {"value": evals / wall, "unit": "proposals/s", "h2d_bytes_per_step": 2 * (W // 2) * 11 * 8,
                    "d2h_bytes_per_step": 2 * (W // 2) * 28},
            "gpu_launches": 2 * 5 * args.steps, "clocks": clk.summary()}
    like.close()
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)


def run_grad(args, B, rank, local, world):
    """ln L and its gradient alone, on the catalog workload (--events, --K as for the headline)."""
    import torch
    cat, inj, _ = synth.make_workload(WORKLOAD, scale=args.events / 1000.0)
    lam = synth.make_lambdas(args.K, 11, seed=synth.seed_for(2, 2) + 7919 * rank)
    like = B.Likelihood(local, torch.cuda.current_stream(local)).load(cat, inj, storage=B.POP_STORE_F64)
    n_pairs = in_support_pairs(cat.theta, lam) + in_support_pairs(inj.theta, lam)
    with Clocks(local) as clk:
        f = grad_form(B, like, lam, args, world, n_pairs)
    like.close()
    line = {"metric": "ln L(Lambda) + gradient evals/s", "value": f["value"], "unit": f["unit"], "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms_per_call"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.events == 1000 else f"{WORKLOAD}_events{args.events}",
                       "events": cat.n_events, "n_found": int(inj.n_found), "K": args.K,
                       "parallelism": f"replicas{world}"},
            "roofline": f["roofline"], "e2e": f["e2e"], "gpu_launches": 4 * args.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)


RAGGED = "f32_ragged2000_s500to16000_z"


def ragged_measure(B, args, rank, local, world):
    """Batching form: 2000 events with S_i ~ U{500..16000} in CSR (about 1.65e7 samples), redshift
    on (12 parameters), 1.8e7 injection draws, FP32 weights.  Uneven Lambda batches
    (64, 200, 1000, 4096 in turn) replay one graph captured at 4096 with K read on the device;
    the tiling comes from the autotuner.  One step = one batch; value = Lambda evaluated / s.
    The oracle checks the last row of each batch size (|d ln L|, flags)."""
    import torch
    cat, inj, _ = synth.make_workload(RAGGED)
    sizes = (64, 200, 1000, 4096)
    lam = synth.make_lambdas(max(sizes), 12, seed=synth.seed_for(4, 2) + 7919 * rank)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        like = B.Likelihood(local, stream).load(cat, inj, storage=B.POP_STORE_F32)
        dev = torch.from_numpy(lam).cuda()
        outs = [torch.empty(max(sizes), dtype=torch.float64, device="cuda") for _ in range(3)] + \
               [torch.empty(max(sizes), dtype=torch.int32, device="cuda")]
        B.pop_loglik(like.ctx, dev, B.POP_MODE_F32, out=outs)
        B.pop_autotune(like.ctx, B.POP_MODE_F32, max(sizes))
        seq = [sizes[s % len(sizes)] for s in range(max(args.steps, len(sizes)))]
        view = lambda k: [o[:k] for o in outs]
        last = {}
        for k in sizes:
            B.pop_loglik(like.ctx, dev[:k], B.POP_MODE_F32, out=view(k))
            torch.cuda.synchronize()
            last[k] = (float(outs[0][k - 1].item()), int(outs[3][k - 1].item()) & 0xFFFFFFFF)
        for s in range(args.warmup):
            k = sizes[s % len(sizes)]
            B.pop_loglik(like.ctx, dev[:k], B.POP_MODE_F32, out=view(k))
        torch.cuda.synchronize()
        barrier(world)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wms = []
        start.record(stream)
        for k in seq:
            B.pop_loglik(like.ctx, dev[:k], B.POP_MODE_F32, out=view(k))
            wms.append(B.pop_last_kernel_ms(like.ctx)[0])
        stop.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(start.elapsed_time(stop), world)
        support = {k: in_support_pairs(cat.theta, lam[:k]) + in_support_pairs(inj.theta, lam[:k]) for k in sizes}
        t0 = time.perf_counter()
        for k in seq:
            B.pop_loglik(like.ctx, lam[:k], B.POP_MODE_F32)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        tiling = B.pop_get_tiling(like.ctx, B.POP_MODE_F32)
        like.close()
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        rows = np.array([k - 1 for k in sizes])
        ref = oracle.loglik(cat, inj, lam[rows], nthreads=host_cores())
        got = np.array([last[k][0] for k in sizes])
        fl = np.array([last[k][1] for k in sizes], dtype=np.uint32)
        fin = np.isfinite(ref[0])
        parity = {"rows": len(rows), "max_abs_dlnL_vs_oracle": float(np.max(np.abs(got[fin] - ref[0][fin])))
                  if fin.any() else 0.0, "flags_equal": bool((fl == ref[3]).all())}
    evals = world * sum(seq)
    return {"value": evals / (ms * 1e-3), "unit": "evals/s", "steps": len(seq), "ms_per_step": ms / len(seq),
            "dtype": "f32", "config": {"workload": RAGGED, "events": cat.n_events, "samples": int(cat.offsets[-1]),
                                       "n_draw": int(inj.n_draw), "n_found": int(inj.n_found),
                                       "K_sequence": list(sizes), "tiling_f32": tiling,
                                       "l2": "inputs larger than L2 (FP32 features 32 B/sample streamed)"},
            "roofline": f32_roofline(sum(support[k] for k in seq), sum(wms)),
            "e2e": {"value": evals / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": int(8 * 12 * np.mean(seq)),
                    "d2h_bytes_per_step": int(28 * np.mean(seq))},
            "parity_vs_oracle": parity, "gpu_launches": 6 * len(seq)}


def run_ragged(args, B, rank, local, world):
    """The batching form alone (see ragged_measure), as its own JSON line."""
    with Clocks(local) as clk:
        r = ragged_measure(B, args, rank, local, world)
    line = {"metric": "ln L(Lambda) evals/s, ragged 2000-event catalog + redshift (batching form)",
            "value": r["value"], "unit": "evals/s", "n_gpus": world, "steps": r["steps"], "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": dict(r["config"], parallelism=f"replicas{world}"),
            "roofline": r["roofline"], "e2e": r["e2e"], "gpu_launches": r["gpu_launches"], "clocks": clk.summary(),
            "parity_vs_oracle": r["parity_vs_oracle"]}
    if rank == 0:
        print(json.dumps(_rounded(line), default=_jsonable), flush=True)


LEARNED = "f32_z_10x1000_inj1e5_surrogate"


def learned_measure(B, args, rank, local, world):
    """The learned form at its own size: 10 events x 1000 samples with redshift (12-dimensional
    Lambda), 1e5 injection draws, K = 1024.  The ln xi network is trained on 2e5 pairs from this
    injection set's reweighting (10% held out, 60 epochs); ln L evals/s of the FP32 + network form
    against the plain FP64 and FP32 Monte Carlo forms, with |Delta ln L| against FP64 on every row."""
    import torch
    cat, inj, lam = synth.make_workload(LEARNED)
    lam = synth.make_lambdas(len(lam), 12, seed=synth.seed_for(5, 2) + 7919 * rank)
    steps = max(args.steps, 200)   # a step is tens of microseconds
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        like = B.Likelihood(local, stream).load(cat, inj)
        dev_lam = torch.from_numpy(lam).cuda()
        outs = [torch.empty(len(lam), dtype=torch.float64, device="cuda") for _ in range(3)] + \
               [torch.empty(len(lam), dtype=torch.int32, device="cuda")]
        K = len(lam)
        res = {}
        for name, mode in (("f64", B.POP_MODE_F64), ("f32", B.POP_MODE_F32)):
            B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
            ms, w = time_mode(B, like, dev_lam, outs, mode, steps, args.warmup, world, stream)
            res[name] = {"value": world * K * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                         "out": host_outputs(outs)}
        sur = surrogate_form(B, like, lam, dev_lam, outs, args, world, stream, res["f64"]["out"], res["f32"]["out"],
                             n_params=12, steps=steps, seed=synth.seed_for(5, 5), budgets=(0.25, 1.0))
        like.close()
    return {"config": {"workload": LEARNED, "events": cat.n_events, "samples_per_event": 1000, "n_dims": 7,
                       "n_draw": int(inj.n_draw), "n_found": int(inj.n_found), "K": K, "steps": steps},
            "f64": {"value": res["f64"]["value"], "ms_per_step": res["f64"]["ms_per_step"]},
            "f32": {"value": res["f32"]["value"], "ms_per_step": res["f32"]["ms_per_step"],
                    "vs_f64": precision_vs(res["f32"]["out"], res["f64"]["out"])},
            "f32_surrogate": sur}


def run_learned(args, B, rank, local, world):
    """The learned form alone (see learned_measure), as its own JSON line."""
    with Clocks(local) as clk:
        r = learned_measure(B, args, rank, local, world)
    sur = r["f32_surrogate"]
    line = {"metric": "ln L(Lambda) evals/s, learned selection term (FP32 + network), 10 x 1000 + redshift",
            "value": sur["value"], "unit": "evals/s", "n_gpus": world, "steps": r["config"]["steps"],
            "warmup": args.warmup, "ms_per_step": sur["budget_0.25"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": dict(r["config"], parallelism=f"replicas{world}", l2="inputs L2-resident (small workload)"),
            "forms": {"f64": r["f64"], "f32": r["f32"], "f32_surrogate": sur}, "clocks": clk.summary(),
            "gpu_launches": 12 * r["config"]["steps"]}
    if rank == 0:
        print(json.dumps(_rounded(line), default=_jsonable), flush=True)


def run_reference(args, rank, world):
    """CPU oracle arm: rank 0 only."""
    if rank != 0:
        return
    cat, inj, lam = synth.make_workload(WORKLOAD)
    import oracle
    oracle.build()
    cores = host_cores()
    rows = max(1, min(args.oracle_lambdas, 64))
    for _ in range(min(args.warmup, 1)):
        oracle.loglik(cat, inj, lam[:min(rows, cores)], nthreads=cores)
    times = []
    for s in range(args.steps):
        sub = lam[(s * rows) % 1024:][:rows]
        t0 = time.perf_counter()
        oracle.loglik(cat, inj, sub, nthreads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = rows * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "events": 1000, "samples_per_event": 4096,
                                            "n_draw": 10**7, "n_found": inj.n_found, "K": 1024,
                                            "step_sample_rows": rows},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": min(cores, rows), "kind": "oracle",
                             "sample": f"{rows} Lambda rows per step of the full workload"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line, default=_jsonable), flush=True)


def _jsonable(o):
    if isinstance(o, np.integer):
        return int(o)
    if isinstance(o, np.floating):
        return float(o)
    raise TypeError(type(o).__name__)


def run_scan(args, B, rank, local, world):
    """Analogue of the paper's speed-up-versus-samples figure (Sec. "Population acceleration",
    Fig. 4): FP64 and FP32 ln L evals/s at K = 1024 over N*S = 1e4 .. 2e7 posterior samples
    (S = min(4096, N*S) samples per event), with injections in the catalog workload's proportion
    (2 N S draws, about 0.22 N S found), the roofline fraction of each point, and the oracle timed
    beside it on 16 rows (up to 3e6 samples).  The saturation point is the smallest N*S whose FP64
    fraction is within 10% of the largest."""
    import torch
    points = [10 ** 4, 3 * 10 ** 4, 10 ** 5, 3 * 10 ** 5, 10 ** 6, 3 * 10 ** 6, 10 ** 7, 2 * 10 ** 7]
    K = 1024
    lam = synth.make_lambdas(K, 11, seed=synth.seed_for(7, 2) + 7919 * rank)
    dev_lam = torch.from_numpy(lam).cuda()
    rows = []
    with Clocks(local) as clk:
        for ns in points:
            S = min(4096, ns)
            N = ns // S
            cat = synth.make_catalog(N, S, 6, seed=synth.seed_for(7, 0) + ns)
            inj = synth.make_injections(2 * ns, 6, seed=synth.seed_for(7, 1) + ns)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                like = B.Likelihood(local, stream).load(cat, inj)
                outs = [torch.empty(K, dtype=torch.float64, device="cuda") for _ in range(3)] + \
                       [torch.empty(K, dtype=torch.int32, device="cuda")]
                pairs = in_support_pairs(cat.theta, lam) + in_support_pairs(inj.theta, lam)
                steps = int(min(200, max(args.steps, 2e9 / max(pairs, 1))))
                pt = {"samples": ns, "events": N, "samples_per_event": S, "n_found": int(inj.n_found),
                      "in_support_pairs": pairs, "steps": steps}
                for name, mode in (("f64", B.POP_MODE_F64), ("f32", B.POP_MODE_F32)):
                    B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
                    B.pop_autotune(like.ctx, mode, 64 if mode == B.POP_MODE_F64 else K)
                    ms, w = time_mode(B, like, dev_lam, outs, mode, steps, args.warmup, world, stream)
                    if mode == B.POP_MODE_F64:
                        ops = in_support_pairs(cat.theta, lam) * FP64_OPS_PER_PAIR + \
                            in_support_pairs(inj.theta, lam) * FP64_OPS_PER_INJ_PAIR
                        frac = ops / (w * 1e-3) / (FP64_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6)
                    else:
                        frac = f32_roofline(pairs, w)["frac"]
                    pt[name] = {"value": world * K * steps / (ms * 1e-3), "ms_per_step": ms / steps, "weight_ms": w,
                                "roofline_frac": frac}
                like.close()
            if rank == 0 and not args.no_cpu_baseline and ns <= 3 * 10 ** 6:
                import oracle
                n = 16
                t0 = time.perf_counter()
                oracle.loglik(cat, inj, lam[:n], nthreads=host_cores())
                pt["oracle"] = {"value": n / (time.perf_counter() - t0), "rows": n, "cores": min(n, host_cores())}
            rows.append(pt)
    best = max(r["f64"]["roofline_frac"] for r in rows)
    sat = next(r["samples"] for r in rows if r["f64"]["roofline_frac"] >= 0.9 * best)
    best32 = max(r["f32"]["roofline_frac"] for r in rows)
    sat32 = next(r["samples"] for r in rows if r["f32"]["roofline_frac"] >= 0.9 * best32)
    top = rows[-1]
    line = {"metric": "ln L(Lambda) evals/s versus posterior samples N*S (K = 1024), FP64 and FP32",
            "value": top["f64"]["value"], "unit": "evals/s", "n_gpus": world, "steps": top["steps"],
            "warmup": args.warmup, "ms_per_step": top["f64"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "scan_samples_1e4_to_2e7_K1024", "K": K, "parallelism": f"replicas{world}",
                       "injections": "2 N S draws, sigmoid((m1 - 20)/5) detection"},
            "saturation_samples_f64": sat, "saturation_samples_f32": sat32, "points": rows,
            "clocks": clk.summary(), "gpu_launches": sum(r["steps"] * 10 for r in rows)}
    if rank == 0:
        print(json.dumps(_rounded(line), default=_jsonable), flush=True)


def _rounded(o, sig=6):
    """Floats rounded to `sig` significant digits (a shorter JSON line; the values are measurements)."""
    if isinstance(o, dict):
        return {k: _rounded(v, sig) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_rounded(v, sig) for v in o]
    if isinstance(o, (float, np.floating)):
        x = float(o)
        return float(f"{x:.{sig}g}") if np.isfinite(x) else x
    return o


def summarise(line):
    """The figures of every form in a few hundred characters, for the end of the JSON line."""
    f = line.get("forms", {})
    r4 = lambda x: None if x is None else float(f"{x:.4g}")
    out = {"f64": {"evals_s": r4(line["value"]), "frac": r4(line["roofline"]["frac"]),
                   "parity_over_tol": r4(line.get("cpu_baseline", {}).get("parity_f64_kernel", {})
                                         .get("max_over_f64_tol"))}}
    if "f64_ff" in f:
        out["f64_ff"] = {"evals_s": r4(f["f64_ff"]["value"]), "frac": r4(f["f64_ff"]["roofline"]["frac"]),
                         "max_over_tol": r4(f["f64_ff"]["max_dlnL_over_f64_tol"])}
    if "grad_f64" in f:
        out["grad_f64"] = {"evals_s": r4(f["grad_f64"]["value"]), "frac": r4(f["grad_f64"]["roofline"]["frac"])}
    if "grid_selection" in f:
        g = f["grid_selection"]
        out["grid"] = {"f64_frac": r4(g["f64"]["roofline"]["frac"]), "f32_frac": r4(g["f32"]["roofline"]["frac"])}
    if "cbc_likelihood" in f:
        c = f["cbc_likelihood"]
        out["cbc"] = {"f64_evals_s": r4(c["f64"]["value"]), "f64_frac": r4(c["f64"]["roofline"]["frac"]),
                      "f32_evals_s": r4(c["f32"]["value"]), "f32_frac": r4(c["f32"]["roofline"]["frac"])}
    if "ragged" in f:
        g = f["ragged"]
        out["ragged"] = {"evals_s": r4(g["value"]), "frac": r4(g["roofline"]["frac"]),
                         "dlnL_vs_oracle": r4((g.get("parity_vs_oracle") or {}).get("max_abs_dlnL_vs_oracle"))}
    if "learned" in f:
        g = f["learned"]
        sur = g["f32_surrogate"]
        out["learned_c5"] = {"f64_evals_s": r4(g["f64"]["value"]), "f32_evals_s": r4(g["f32"]["value"]),
                             "fit_tflops": r4(sur["training"]["fit_tflops"]),
                             **{b: {"evals_s": r4(sur[b]["value"]), "used": r4(sur[b]["surrogate_used_frac"]),
                                    "dlnL_max": r4(sur[b]["vs_f64"]["abs_dlnL"]["max"]),
                                    "dlnL_max_net": r4(sur[b]["vs_f64_network_rows"]["max"])}
                                for b in ("budget_0.25", "budget_1", "ungated") if b in sur}}
    if "f32_surrogate" in f:
        sur = f["f32_surrogate"]
        out["f32_surrogate"] = {b: {"evals_s": r4(sur[b]["value"]), "used": r4(sur[b]["surrogate_used_frac"]),
                                    "dlnL_max": r4(sur[b]["vs_f64"]["abs_dlnL"]["max"]),
                                    "dlnL_max_net": r4(sur[b]["vs_f64_network_rows"]["max"])}
                                for b in ("budget_0.25", "ungated") if b in sur}
        out["f32_surrogate"]["fit_tflops"] = r4(sur["training"]["fit_tflops"])
    if "f32" in f:
        out["f32"] = {"evals_s": r4(f["f32"]["value"]), "frac": r4(f["f32"]["roofline"]["frac"]),
                      "dlnL_max_vs_f64": r4(f["f32"]["vs_f64"]["abs_dlnL"]["max"]),
                      "dlnL_p99_vs_f64": r4(f["f32"]["vs_f64"]["abs_dlnL"]["p99"])}
    return out


def main():
    args = parse()
    rank, local, world = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    torch.cuda.set_device(local)
    from paper_1904_02863_gb300 import binding as B
    from paper_1904_02863_gb300 import build
    build.build()
    standalone = {"ragged": run_ragged, "grid": run_grid, "cbc": run_cbc, "grad": run_grad, "sampler": run_sampler,
                  "learned": run_learned, "scan": run_scan}
    if args.workload in standalone:
        standalone[args.workload](args, B, rank, local, world)
        return

    scale = args.events / 1000.0
    cat, inj, _ = synth.make_workload(WORKLOAD, scale=scale)
    workload = WORKLOAD if args.events == 1000 else f"{WORKLOAD}_events{args.events}"
    K = args.K
    lam = synth.make_lambdas(K, 11, seed=synth.seed_for(2, 2) + 7919 * rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    like = B.Likelihood(local, stream).load(cat, inj)
    dev_lam = torch.from_numpy(lam).cuda()
    outs = [torch.empty(K, dtype=torch.float64, device="cuda") for _ in range(3)] + \
           [torch.empty(K, dtype=torch.int32, device="cuda")]

    head = {"f32": B.POP_MODE_F32, "ff": B.POP_MODE_FF}.get(args.mode, B.POP_MODE_F64)
    # Tiling from the autotuner (FP64 on the first 64 Lambda rows: its launches are long); the
    # float-float kernel has one fixed tiling.
    for mode in ([head] if args.mode != "both" else [B.POP_MODE_F64, B.POP_MODE_F32]):
        B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
        if mode != B.POP_MODE_FF:
            B.pop_autotune(like.ctx, mode, min(K, 64) if mode == B.POP_MODE_F64 else K)
    with Clocks(local) as clk:
        ms_h, w_h = time_mode(B, like, dev_lam, outs, head, args.steps, args.warmup, world, stream)
        if args.mode == "both":
            ms32, w32 = time_mode(B, like, dev_lam, outs, B.POP_MODE_F32, args.steps, args.warmup, world, stream)
            out32 = host_outputs(outs)

    # End to end through the public API with pinned host buffers.
    h_lam = torch.from_numpy(lam).pin_memory()
    h_out = [torch.empty(K, dtype=torch.float64).pin_memory() for _ in range(3)] + \
            [torch.empty(K, dtype=torch.int32).pin_memory()]
    B.pop_loglik(like.ctx, h_lam, head, out=h_out)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        B.pop_loglik(like.ctx, h_lam, head, out=h_out)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)

    # Untimed FP64 outputs for the precision reports.
    ref64 = None
    if head == B.POP_MODE_F64 or args.mode == "both":
        B.pop_loglik(like.ctx, dev_lam, B.POP_MODE_F64, out=outs)
        ref64 = host_outputs(outs)

    n_ev_pairs = in_support_pairs(cat.theta, lam)
    n_inj_pairs = in_support_pairs(inj.theta, lam)
    all_pairs = (int(cat.offsets[-1]) + int(inj.n_found)) * K
    clocks = clk.summary()
    value = world * K * args.steps / (ms_h * 1e-3)
    if head == B.POP_MODE_F64:
        ops = n_ev_pairs * FP64_OPS_PER_PAIR + n_inj_pairs * FP64_OPS_PER_INJ_PAIR
        peak_tops = FP64_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12  # FP64 pipe ops/s (FMA = 1 op)
        achieved_tops = ops / (w_h * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Top/s (FP64 pipe)",
                    "frac": achieved_tops / peak_tops,
                    "traffic": F64_DRAM_BYTES_PER_UNIT * (int(cat.offsets[-1]) + int(inj.n_found)),
                    "traffic_basis": "ncu dram bytes of a 400-event capture scaled by units",
                    "kernel": "weight_f64_kernel",
                    "weight_ms": w_h, "ops_per_launch": ops,
                    "in_support_pairs": n_ev_pairs + n_inj_pairs, "all_pairs": all_pairs,
                    "ops_per_in_support_pair": FP64_OPS_PER_PAIR,
                    "peak_basis": "2 FP64 lanes/SM/clk x 152 SMs x 2070 MHz"}
    elif head == B.POP_MODE_F32:
        roofline = f32_roofline(n_ev_pairs + n_inj_pairs, w_h)
    else:
        roofline = ff_roofline(n_ev_pairs + n_inj_pairs, w_h)
    # Measured pipe rates (thread operations per SM clock) beside the constants the rooflines use.
    pipe = dict(B.pop_pipe_rates(local), unit="thread ops per SM clock", source="pop_pipe_rates, this run")
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_h / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {B.POP_MODE_F64: "f64", B.POP_MODE_F32: "f32"}.get(head, "float-float"),
        "data": "synthetic",
        "config": {"workload": workload, "events": cat.n_events, "samples_per_event": 4096,
                   "n_draw": int(inj.n_draw), "n_found": int(inj.n_found), "K": K,
                   "mode": {B.POP_MODE_F64: "POP_MODE_F64", B.POP_MODE_F32: "POP_MODE_F32"}.get(head, "POP_MODE_FF"),
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (FP64 features 80 B/sample)",
                   "tiling_f64": B.pop_get_tiling(like.ctx, B.POP_MODE_F64),
                   "tiling_f32": B.pop_get_tiling(like.ctx, B.POP_MODE_F32)},
        "roofline": roofline,
        "e2e": {"value": world * K * args.steps / e2e_s, "unit": "evals/s",
                "h2d_bytes_per_step": int(lam.nbytes), "d2h_bytes_per_step": int(K * (8 * 3 + 4))},
        # set K, prologue, weight, finalise (+ the FP32 kernel's Lambda order and upper-edge fix-up)
        "gpu_launches": (4 if head == B.POP_MODE_F64 else 6) * args.steps,
        "clocks": clocks,
        "pipe_rates": pipe,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cat, inj, lam, args.oracle_lambdas,
                                             ref64 if head == B.POP_MODE_F64 else None)
    if args.mode == "both":
        # Largest first, so that the driver's record (the end of the line) keeps the compact ones.
        forms = {}
        forms["grid_selection"] = grid_form(B, like, lam, dev_lam, outs, args, world, stream)
        forms["cbc_likelihood"] = cbc_form(B, like, args, world, rank)
        forms["grad_f64"] = grad_form(B, like, lam, args, world, n_ev_pairs + n_inj_pairs)
        forms["f64_ff"] = ff_form(B, like, lam, dev_lam, outs, args, world, stream, n_ev_pairs + n_inj_pairs,
                                  cat.n_events, ref64)
        forms["f32_surrogate"] = surrogate_form(B, like, lam, dev_lam, outs, args, world, stream, ref64, out32)
        forms["f32"] = {"value": world * K * args.steps / (ms32 * 1e-3), "unit": "evals/s",
                        "ms_per_step": ms32 / args.steps, "weight_ms": w32, "dtype": "f32",
                        "roofline": f32_roofline(n_ev_pairs + n_inj_pairs, w32), "vs_f64": precision_vs(out32, ref64)}
        like.close()
        like = None
        forms["ragged"] = ragged_measure(B, args, rank, local, world)
        forms["learned"] = learned_measure(B, args, rank, local, world)
        line["forms"] = forms
        line["summary"] = summarise(line)
    if like is not None:
        like.close()
    if rank == 0:
        print(json.dumps(_rounded(line), default=_jsonable), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
