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
# kernel: 15 add/mul/fma + 3 exp (7 each) + 1 expm1 (10) + 1 reciprocal (3);
# +1 fma for the squared weight on injection pairs.
FP64_OPS_PER_PAIR = 49
FP64_OPS_PER_INJ_PAIR = 50
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
# DRAM bytes per (sample or injection) unit of one weight_f64 launch, from the ncu capture in
# profiles/weight_f64_catalog400x4096_K64_full.md (154.18 MB / 2,077,126 units); a launch
# reads every chunk from DRAM once, so traffic scales with the units.
F64_DRAM_BYTES_PER_UNIT = 154.18e6 / 2077126


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
    p.add_argument("--workload", default="catalog", choices=["catalog", "ragged", "grid", "cbc", "grad", "sampler"],
                   help="catalog: 1000 events x 4096 samples + 1e7 injection draws (default); "
                        "ragged: 2000 ragged CSR events + redshift, uneven batches; "
                        "sampler: the stretch-move ensemble sampler driving FP32 ln L on the catalog")
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


def precision_vs(res, ref):
    """|Delta ln L| and the relative Delta xi of the outputs ``res`` against ``ref`` over every
    Lambda of the batch (rows where both ln L are finite)."""
    a, b = res[0], ref[0]
    both = np.isfinite(a) & np.isfinite(b)
    d = np.abs(a[both] - b[both])
    dxi = np.abs(np.expm1(res[1][both] - ref[1][both]))
    return {"rows": int(a.size), "finite_rows_agree": bool((np.isfinite(a) == np.isfinite(b)).all()),
            "abs_dlnL": {"mean": float(d.mean()) if d.size else 0.0, "max": float(d.max()) if d.size else 0.0},
            "rel_dxi_max": float(dxi.max()) if dxi.size else 0.0}


def f64_on_rounded_inputs(B, cat, inj, dev_lam, device, stream):
    """The FP64 kernel's outputs on the catalog and injections rounded to float32 (what the FP32
    layout stores): against these, an FP32 form's difference is its arithmetic error alone."""
    import torch
    cat32 = synth.Catalog(cat.offsets, synth.round_to_f32(cat.theta), synth.round_to_f32(cat.prior))
    inj32 = synth.Injections(synth.round_to_f32(inj.theta), synth.round_to_f32(inj.p_draw), inj.n_draw)
    like = B.Likelihood(device, stream).load(cat32, inj32)
    K = dev_lam.shape[0]
    outs = [torch.empty(K, dtype=torch.float64, device="cuda") for _ in range(3)] + \
           [torch.empty(K, dtype=torch.int32, device="cuda")]
    B.pop_loglik(like.ctx, dev_lam, B.POP_MODE_F64, out=outs)
    torch.cuda.synchronize()
    res = [o.cpu().numpy().copy() for o in outs]
    like.close()
    return res


def ff_form(B, like, lam, dev_lam, outs, timed, args, world, n_pairs, n_events):
    """FP64-grade ln L with the sample weights in float-float arithmetic (POP_MODE_FF): its
    evals/s, and its distance to the FP64 kernel's ln L in units of the FP64 parity tolerance
    1e-12 (|sum_i ln(S_i/n_i)| + N |ln xi|) for every Lambda of the batch."""
    import torch
    ms, w = timed(B.POP_MODE_FF)
    ff = [o.clone() for o in outs]
    B.pop_loglik(like.ctx, dev_lam, B.POP_MODE_F64, out=outs)
    torch.cuda.synchronize()
    f64 = [o.cpu().numpy() for o in outs]
    ffh = [o.cpu().numpy() for o in ff]
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


def surrogate_form(B, like, lam, dev_lam, outs, timed, args, world, ref64=None, ref64_rounded=None):
    """FP32 weights + the trained ln xi network (Monte Carlo xi only where its gate says so).

    Training (2e5 Lambda from the prior box, 10% held out, targets from this
    workload's own injections, 60 epochs) is setup, timed separately.
    """
    import torch
    box = synth.LAMBDA_BOX[:11]
    t0 = time.perf_counter()
    B.pop_xi_surrogate_train(like.ctx, 200000, box[:, 0], box[:, 1], epochs=60, seed=synth.seed_for(2, 5))
    train_s = time.perf_counter() - t0
    info = B.pop_xi_surrogate_info(like.ctx)
    ms, w = timed(B.POP_MODE_F32_SURROGATE)
    sur = [o.clone() for o in outs]
    B.pop_loglik(like.ctx, dev_lam, B.POP_MODE_F32, out=outs)
    torch.cuda.synchronize()
    used = (sur[3].cpu().numpy().view(np.uint32) & B.POP_FLAG_SURROGATE_USED) != 0
    d = (sur[0] - outs[0]).abs().cpu().numpy()
    fin = np.isfinite(d)
    K = len(lam)
    return {"value": world * K * args.steps / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms / args.steps,
            "weight_ms": w, "dtype": "f32+bf16 network", "train_seconds": train_s,
            "heldout_rmse_lnxi": info["heldout_rmse"], "heldout_mc_noise": info["mc_noise"],
            "trusted": info["trusted"], "surrogate_used_frac": float(used.mean()),
            "abs_dlnL_vs_f32_mc": {"mean": float(d[fin].mean()), "max": float(d[fin].max())},
            **precision_fields([o.cpu().numpy() for o in sur], ref64, ref64_rounded)}


def precision_fields(res, ref64, ref64_rounded):
    """The form's distance to the FP64 kernel (which matches the oracle to 1e-12): on the original
    inputs (arithmetic and float32 storage) and on the float32-rounded inputs (arithmetic alone,
    the quantity the 0.05-nat FP32 bar applies to)."""
    out = {}
    if ref64 is not None:
        out["vs_f64"] = precision_vs(res, ref64)
    if ref64_rounded is not None:
        out["vs_f64_rounded_inputs"] = precision_vs(res, ref64_rounded)
    return out


def grid_form(B, like, lam, timed, args, world):
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
                     "Top/s (FP64 pipe)", "gv_main_kernel<double>"),
             "f32": (FP32_LANES_PER_SM * SMS * SM_MAX_MHZ * 1e6, "128 FP32 FMA lanes/SM/clk x 152 SMs x 2070 MHz",
                     "Top/s (FP32 FMA)", "gv_main_kernel<float>")}
    for name, mode in (("f64", B.POP_MODE_F64), ("f32", B.POP_MODE_F32)):
        ms, w = timed(mode)
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
# split into its power-law and peak parts (4 exp, 1 expm1, 1 reciprocal and their FMAs), the
# 11-12 score terms and the 14 sums, with the loop-invariant terms hoisted: 105, the DFMA + DADD
# + DMUL count per in-support pair of the ncu capture in profiles/grad_weight_catalog100x4096_K16_full.md.
FP64_OPS_PER_GRAD_PAIR = 105


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
            "roofline": {"bound": "alu", "kernel": "gv_main_kernel<double>", "achieved": triples / (c64 * 1e-3) / 1e12,
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


def run_ragged(args, B, rank, local, world):
    """Batching form: 2000 events with S_i ~ U{500..16000} in CSR (about 1.65e7 samples), redshift
    on (12 parameters), 1.8e7 injection draws, FP32 weights.  Uneven Lambda batches
    (64, 200, 1000, 4096 in turn) replay one graph captured at 4096 with K read on the device;
    the tiling comes from the autotuner.  One step = one batch; value = Lambda evaluated / s."""
    import torch
    cat, inj, _ = synth.make_workload("f32_ragged2000_s500to16000_z")
    sizes = (64, 200, 1000, 4096)
    lam = synth.make_lambdas(max(sizes), 12, seed=synth.seed_for(4, 2) + 7919 * rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    like = B.Likelihood(local, stream).load(cat, inj, storage=B.POP_STORE_F32)
    dev = torch.from_numpy(lam).cuda()
    outs = [torch.empty(max(sizes), dtype=torch.float64, device="cuda") for _ in range(3)] + \
           [torch.empty(max(sizes), dtype=torch.int32, device="cuda")]
    B.pop_loglik(like.ctx, dev, B.POP_MODE_F32, out=outs)
    B.pop_autotune(like.ctx, B.POP_MODE_F32, max(sizes))
    seq = [sizes[s % len(sizes)] for s in range(args.steps)]
    view = lambda k: [o[:k] for o in outs]
    for s in range(args.warmup):
        k = sizes[s % len(sizes)]
        B.pop_loglik(like.ctx, dev[:k], B.POP_MODE_F32, out=view(k))
    torch.cuda.synchronize()
    barrier(world)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wms = []
    with Clocks(local) as clk:
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
    evals = world * sum(seq)
    line = {"metric": "ln L(Lambda) evals/s, ragged 2000-event catalog + redshift (batching form)",
            "value": evals / (ms * 1e-3), "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "f32_ragged2000_s500to16000_z", "events": cat.n_events, "samples": int(cat.offsets[-1]),
                       "n_draw": int(inj.n_draw), "n_found": int(inj.n_found), "K_sequence": list(sizes),
                       "tiling_f32": B.pop_get_tiling(like.ctx, B.POP_MODE_F32), "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (FP32 features 44 B/sample)"},
            "roofline": f32_roofline(sum(support[k] for k in seq), sum(wms)),
            "e2e": {"value": evals / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": int(8 * 12 * np.mean(seq)),
                    "d2h_bytes_per_step": int(28 * np.mean(seq))},
            "gpu_launches": 5 * args.steps, "clocks": clk.summary()}
    like.close()
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)


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
    if args.workload == "ragged":
        run_ragged(args, B, rank, local, world)
        return
    if args.workload == "grid":
        run_grid(args, B, rank, local, world)
        return
    if args.workload == "cbc":
        run_cbc(args, B, rank, local, world)
        return
    if args.workload == "grad":
        run_grad(args, B, rank, local, world)
        return
    if args.workload == "sampler":
        run_sampler(args, B, rank, local, world)
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

    def timed(mode):
        for _ in range(args.warmup):
            B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wms = []
        start.record(stream)
        for _ in range(args.steps):
            B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
            wms.append(B.pop_last_kernel_ms(like.ctx)[0])
        stop.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ms = max_over_ranks(start.elapsed_time(stop), world)
        return ms, statistics.mean(wms)

    head = {"f32": B.POP_MODE_F32, "ff": B.POP_MODE_FF}.get(args.mode, B.POP_MODE_F64)
    # Tiling from the autotuner (FP64 on the first 64 Lambda rows: its launches are long); the
    # float-float kernel has one fixed tiling.
    for mode in ([head] if args.mode != "both" else [B.POP_MODE_F64, B.POP_MODE_F32]):
        B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
        if mode != B.POP_MODE_FF:
            B.pop_autotune(like.ctx, mode, min(K, 64) if mode == B.POP_MODE_F64 else K)
    with Clocks(local) as clk:
        ms_h, w_h = timed(head)
        if args.mode == "both":
            ms32, w32 = timed(B.POP_MODE_F32)

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

    def run_once(mode):
        B.pop_loglik(like.ctx, dev_lam, mode, out=outs)
        torch.cuda.synchronize()
        return [o.cpu().numpy().copy() for o in outs]

    # Untimed reference outputs for the precision report.
    ref64 = run_once(B.POP_MODE_F64) if (head == B.POP_MODE_F64 or args.mode == "both") else None

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
        # set K, prologue, weight, finalise (+ the FP32 kernel's Lambda order)
        "gpu_launches": (4 if head == B.POP_MODE_F64 else 5) * args.steps,
        "clocks": clocks,
        "pipe_rates": pipe,
    }
    if args.mode == "both":
        ref64_r = f64_on_rounded_inputs(B, cat, inj, dev_lam, local, stream)
        line["forms"] = {"f32": {"value": world * K * args.steps / (ms32 * 1e-3), "unit": "evals/s",
                                 "ms_per_step": ms32 / args.steps, "weight_ms": w32, "dtype": "f32",
                                 "roofline": f32_roofline(n_ev_pairs + n_inj_pairs, w32),
                                 **precision_fields(run_once(B.POP_MODE_F32), ref64, ref64_r)}}
        line["forms"]["f64_ff"] = ff_form(B, like, lam, dev_lam, outs, timed, args, world, n_ev_pairs + n_inj_pairs,
                                          cat.n_events)
        line["forms"]["f32_surrogate"] = surrogate_form(B, like, lam, dev_lam, outs, timed, args, world,
                                                             ref64, ref64_r)
        line["forms"]["grid_selection"] = grid_form(B, like, lam, timed, args, world)
        line["forms"]["cbc_likelihood"] = cbc_form(B, like, args, world, rank)
        line["forms"]["grad_f64"] = grad_form(B, like, lam, args, world, n_ev_pairs + n_inj_pairs)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cat, inj, lam, args.oracle_lambdas,
                                             ref64 if head == B.POP_MODE_F64 else None)
    like.close()
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
