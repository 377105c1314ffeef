"""Thin ctypes binding of libpop.so (include/pop.h), same names as the C-ABI.

Argument marshalling only: every step of the likelihood runs in the library's
CUDA kernels.  Host inputs are numpy arrays (passed with POP_MEM_HOST); device
inputs are torch CUDA tensors (passed by pointer with POP_MEM_DEVICE).  torch
supplies device memory and the stream, nothing else.  There is no fallback:
if libpop.so is missing or no GPU is usable, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpop.so")

POP_OK, POP_EINVAL, POP_ENOMEM, POP_ECUDA, POP_ESTATE, POP_ETIMEOUT, POP_ENUMERIC = 0, -1, -2, -3, -4, -5, -6
POP_STORE_F64, POP_STORE_F32 = 1, 2
POP_MODE_F64, POP_MODE_F32, POP_MODE_F32_SURROGATE, POP_MODE_FF = 0, 1, 2, 3
POP_MEM_HOST, POP_MEM_DEVICE = 0, 1
POP_FLAG_INVALID_LAMBDA, POP_FLAG_ZERO_EVENT, POP_FLAG_LOW_NEFF = 1, 2, 4
POP_FLAG_SURROGATE_USED, POP_FLAG_MC_FALLBACK, POP_FLAG_ZERO_XI = 8, 16, 32
POP_XI_INJECTIONS, POP_XI_GRID = 0, 1

# Every symbol include/pop.h declares (checked by the CPU test suite).
EXPORTS = (
    "pop_create", "pop_destroy", "pop_last_error", "pop_status_string", "pop_version",
    "pop_validate_events", "pop_load_events", "pop_load_injections", "pop_loglik",
    "pop_set_tiling", "pop_get_tiling", "pop_autotune", "pop_set_graphs", "pop_last_kernel_ms",
    "pop_loglik_f64_noalloc", "pop_math_check", "pop_wait_check", "pop_pipe_rates", "pop_pipe_rates_n",
    "pop_xi_surrogate_train", "pop_xi_surrogate_info", "pop_xi_surrogate_infer", "pop_xi_surrogate_save",
    "pop_xi_surrogate_load", "pop_mlp_set_params", "pop_mlp_get_params", "pop_mlp_forward", "pop_mlp_gradients",
    "pop_mlp_train_step", "pop_mlp_gemm_check",
    "pop_load_vt_grid", "pop_set_xi_source", "pop_xi_grid", "pop_xi_grid_last_ms", "pop_loglik_parts",
    "pop_cbc_load", "pop_cbc_loglik", "pop_cbc_last_ms", "pop_loglik_grad",
    "pop_xi_surrogate_error", "pop_xi_surrogate_set_budget", "pop_xi_surrogate_train_stats",
)
MLP_N_PARAMS = 201218
POP_NOALLOC_SCRATCH_BYTES = 16 << 20


class PopError(RuntimeError):
    """A pop_status other than POP_OK, with the library's error text; .status holds the code."""
    def __init__(self, status, message):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpop.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "pop_create": (i32, [ctypes.POINTER(vp), i32, vp]),
        "pop_destroy": (i32, [vp]),
        "pop_last_error": (ctypes.c_char_p, [vp]),
        "pop_status_string": (ctypes.c_char_p, [i32]),
        "pop_version": (i32, []),
        "pop_validate_events": (i32, [i64, vp, i32, ctypes.c_char_p, i32]),
        "pop_load_events": (i32, [vp, i64, vp, i32, vp, vp, i32, i32]),
        "pop_load_injections": (i32, [vp, i64, i64, i32, vp, vp, i32, i32]),
        "pop_loglik": (i32, [vp, i64, i32, vp, i32, vp, vp, vp, vp, i32]),
        "pop_set_tiling": (i32, [vp, i32, i32, i32, i32]),
        "pop_get_tiling": (i32, [vp, i32, vp, vp, vp]),
        "pop_autotune": (i32, [vp, i32, i64, ctypes.c_char_p]),
        "pop_set_graphs": (i32, [vp, i32]),
        "pop_last_kernel_ms": (i32, [vp, ctypes.POINTER(d), ctypes.POINTER(d)]),
        "pop_loglik_f64_noalloc": (i32, [i32, vp, i64, vp, i64, i32, vp, vp, i64, i64, vp, vp, i64, i32, vp,
                                         vp, vp, vp, vp, ctypes.c_char_p, i32]),
        "pop_math_check": (i32, [vp, i32, i64, vp, vp, i32]),
        "pop_wait_check": (i32, [vp, i32, i32]),
        "pop_pipe_rates": (i32, [i32, vp]),
        "pop_pipe_rates_n": (i32, [i32, vp, i32]),
        "pop_xi_surrogate_train": (i32, [vp, i64, d, ctypes.c_uint64, vp, vp, i32, i32, ctypes.POINTER(d)]),
        "pop_xi_surrogate_info": (i32, [vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d),
                                        ctypes.POINTER(i32)]),
        "pop_xi_surrogate_infer": (i32, [vp, i64, i32, vp, vp, vp, vp, i32]),
        "pop_xi_surrogate_error": (i32, [vp, i64, i32, vp, vp, i32]),
        "pop_xi_surrogate_set_budget": (i32, [vp, d]),
        "pop_xi_surrogate_train_stats": (i32, [vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(i64)]),
        "pop_xi_surrogate_save": (i32, [vp, ctypes.c_char_p]),
        "pop_xi_surrogate_load": (i32, [vp, ctypes.c_char_p]),
        "pop_mlp_set_params": (i32, [vp, vp, i64]),
        "pop_mlp_get_params": (i32, [vp, vp, i64]),
        "pop_mlp_forward": (i32, [vp, i64, vp, vp]),
        "pop_mlp_gradients": (i32, [vp, i64, vp, vp, vp, ctypes.POINTER(d)]),
        "pop_mlp_train_step": (i32, [vp, i64, vp, vp, ctypes.c_float]),
        "pop_mlp_gemm_check": (i32, [vp, i32, i32, i32, vp, vp, vp]),
        "pop_load_vt_grid": (i32, [vp, i32, vp, i32, vp, vp, i32]),
        "pop_loglik_parts": (i32, [vp, i64, i32, vp, i32, vp, vp, vp, vp, i32]),
        "pop_cbc_load": (i32, [vp, i32, i64, d, d, vp, vp, vp, vp, i32]),
        "pop_loglik_grad": (i32, [vp, i64, i32, vp, vp, vp, vp, i32]),
        "pop_cbc_loglik": (i32, [vp, i64, i32, vp, i32, vp, vp, i32]),
        "pop_cbc_last_ms": (i32, [vp, ctypes.POINTER(d), ctypes.POINTER(d)]),
        "pop_set_xi_source": (i32, [vp, i32]),
        "pop_xi_grid": (i32, [vp, i64, i32, vp, i32, vp, vp, i32]),
        "pop_xi_grid_last_ms": (i32, [vp, ctypes.POINTER(d), ctypes.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    """Name of a pop_status value (the number itself if the library cannot be loaded)."""
    try:
        return load_library().pop_status_string(status).decode()
    except Exception:
        return str(status)


def _check(ctx, rc):
    if rc != POP_OK:
        msg = load_library().pop_last_error(ctx)
        raise PopError(rc, msg.decode() if msg else "")


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _arg(x, dtype):
    """(pointer, mem, keepalive) of a numpy array or a torch CUDA tensor."""
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.uint32: torch.int32, np.int64: torch.int64}[dtype]
        if not x.is_contiguous() or x.dtype != want:
            raise TypeError(f"tensor arguments must be contiguous tensors of {want}")
        return ctypes.c_void_p(x.data_ptr()), POP_MEM_DEVICE if x.is_cuda else POP_MEM_HOST, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), POP_MEM_HOST, a


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------------ C-ABI mirrors
def pop_version() -> int:
    """ABI version of the loaded library (major * 10000 + minor * 100 + patch)."""
    return load_library().pop_version()


def pop_validate_events(n_events, offsets, n_dims):
    """Host-only CSR check; returns (status, message)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    buf = ctypes.create_string_buffer(256)
    rc = load_library().pop_validate_events(int(n_events), off.ctypes.data_as(ctypes.c_void_p), int(n_dims), buf, 256)
    return rc, buf.value.decode()


def pop_create(device: int = 0, stream=None):
    """A context on `device` whose work runs on `stream` (a torch.cuda.Stream; None = the
    legacy default stream).  It owns all device memory of the calls made on it."""
    ctx = ctypes.c_void_p()
    rc = load_library().pop_create(ctypes.byref(ctx), int(device), _stream_ptr(stream))
    _check(None, rc)
    return ctx


def pop_destroy(ctx):
    """Frees every buffer of the context."""
    _check(ctx, load_library().pop_destroy(ctx))


def pop_last_error(ctx) -> str:
    """Text of the last error on the context (or of the last failed pop_create for None)."""
    return load_library().pop_last_error(ctx).decode()


def pop_load_events(ctx, offsets, theta, prior, storage=POP_STORE_F64 | POP_STORE_F32):
    """Copies a ragged catalog: CSR offsets [N+1] (host), theta [offsets[-1], 6 or 7] and the
    single-event prior [offsets[-1]] (both numpy, or both CUDA tensors), and packs the features
    in the requested storage(s).  Replaces earlier events; the caller keeps its arrays."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    tp, mem, k1 = _arg(theta, np.float64)
    pp, mem2, k2 = _arg(prior, np.float64)
    if mem != mem2:
        raise TypeError("theta and prior must both be host arrays or both device tensors")
    n_dims = int(theta.shape[1])
    _check(ctx, load_library().pop_load_events(ctx, len(off) - 1, off.ctypes.data_as(ctypes.c_void_p), n_dims,
                                               tp, pp, int(storage), mem))


def pop_load_injections(ctx, n_draw, theta, p_draw, storage=POP_STORE_F64 | POP_STORE_F32):
    """Copies the found injections theta [n_found, n_dims] with their draw pdf p_draw [n_found];
    n_draw counts found and missed draws.  Load the events first (same n_dims)."""
    tp, mem, k1 = _arg(theta, np.float64)
    pp, mem2, k2 = _arg(p_draw, np.float64)
    if mem != mem2:
        raise TypeError("theta and p_draw must both be host arrays or both device tensors")
    _check(ctx, load_library().pop_load_injections(ctx, int(theta.shape[0]), int(n_draw), int(theta.shape[1]),
                                                   tp, pp, int(storage), mem))


def pop_loglik(ctx, lambdas, mode=POP_MODE_F64, out=None):
    """ln L, ln xi, N_eff, flags for each row of ``lambdas``.

    numpy input -> numpy outputs (synchronous).  torch CUDA input -> torch CUDA
    outputs (asynchronous on the context stream); ``out`` may supply them.
    """
    lp, mem, keep = _arg(lambdas, np.float64)
    K, P = int(lambdas.shape[0]), int(lambdas.shape[1])
    if out is not None:
        ptrs = [_arg(r, dt)[0] for r, dt in zip(out, (np.float64, np.float64, np.float64, np.uint32))]
        _check(ctx, load_library().pop_loglik(ctx, K, P, lp, int(mode), *ptrs, mem))
        return out
    if mem == POP_MEM_HOST:
        res = (np.empty(K), np.empty(K), np.empty(K), np.empty(K, np.uint32))
        ptrs = [r.ctypes.data_as(ctypes.c_void_p) for r in res]
    else:
        import torch
        dev = lambdas.device
        res = (torch.empty(K, dtype=torch.float64, device=dev), torch.empty(K, dtype=torch.float64, device=dev),
                      torch.empty(K, dtype=torch.float64, device=dev), torch.empty(K, dtype=torch.int32, device=dev))
        ptrs = [ctypes.c_void_p(r.data_ptr()) for r in res]
    _check(ctx, load_library().pop_loglik(ctx, K, P, lp, int(mode), *ptrs, mem))
    return res


def pop_loglik_grad(ctx, lambdas):
    """(ln L, d ln L / d Lambda [K, n_params], flags) in FP64 (host arrays; synchronous)."""
    lam = np.ascontiguousarray(np.atleast_2d(lambdas), dtype=np.float64)
    K, P = lam.shape
    lnL, grad, fl = np.empty(K), np.empty((K, P)), np.empty(K, np.uint32)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(ctx, load_library().pop_loglik_grad(ctx, K, P, vp(lam), vp(lnL), vp(grad), vp(fl), POP_MEM_HOST))
    return lnL, grad, fl


def pop_loglik_parts(ctx, lambdas, mode=POP_MODE_F64):
    """(sum_i ln(S_i/n_i), sum w, sum w^2, flags) over the loaded events and injections (host arrays)."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    K, P = lam.shape
    res = (np.empty(K), np.empty(K), np.empty(K), np.empty(K, np.uint32))
    ptrs = [r.ctypes.data_as(ctypes.c_void_p) for r in res]
    _check(ctx, load_library().pop_loglik_parts(ctx, K, P, lam.ctypes.data_as(ctypes.c_void_p), int(mode), *ptrs,
                                                POP_MEM_HOST))
    return res


def pop_cbc_load(ctx, f0, df, data, psd, hp, hc):
    """Single-event CBC data: data [n_det, M] complex, psd [n_det, M], hp and hc [M] complex (host arrays)."""
    d = np.ascontiguousarray(np.asarray(data, np.complex128))
    S = np.ascontiguousarray(psd, dtype=np.float64)
    a = np.ascontiguousarray(np.asarray(hp, np.complex128))
    b = np.ascontiguousarray(np.asarray(hc, np.complex128))
    n_det, M = S.shape
    if d.shape != S.shape or a.shape != (M,) or b.shape != (M,):
        raise ValueError("pop_cbc_load: inconsistent shapes")
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(ctx, load_library().pop_cbc_load(ctx, n_det, M, float(f0), float(df), vp(d), vp(S), vp(a), vp(b),
                                            POP_MEM_HOST))


def pop_cbc_loglik(ctx, thetas, mode=POP_MODE_F64):
    """ln L and flags for each row of thetas [K, 2 + 3 n_det] (host arrays; synchronous)."""
    th = np.ascontiguousarray(np.atleast_2d(thetas), dtype=np.float64)
    K, P = th.shape
    out, fl = np.empty(K), np.empty(K, np.uint32)
    _check(ctx, load_library().pop_cbc_loglik(ctx, K, P, th.ctypes.data_as(ctypes.c_void_p), int(mode),
                                              out.ctypes.data_as(ctypes.c_void_p),
                                              fl.ctypes.data_as(ctypes.c_void_p), POP_MEM_HOST))
    return out, fl


def pop_cbc_last_ms(ctx):
    """(sums-kernel ms, whole-call ms) of the last pop_cbc_loglik, from CUDA events."""
    w, t = ctypes.c_double(), ctypes.c_double()
    _check(ctx, load_library().pop_cbc_last_ms(ctx, ctypes.byref(w), ctypes.byref(t)))
    return w.value, t.value


def pop_set_tiling(ctx, mode, lambda_tile, block_threads, blocks_per_sm=0):
    """Fixes the weight kernel's tiling for `mode` (Lambda per work item, threads per block,
    blocks per SM; 0 = as many as fit)."""
    _check(ctx, load_library().pop_set_tiling(ctx, int(mode), int(lambda_tile), int(block_threads), int(blocks_per_sm)))


def pop_get_tiling(ctx, mode):
    """(lambda_tile, block_threads, blocks_per_sm) that `mode` currently uses."""
    t, b, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(ctx, load_library().pop_get_tiling(ctx, int(mode), ctypes.byref(t), ctypes.byref(b), ctypes.byref(s)))
    return t.value, b.value, s.value


def pop_autotune(ctx, mode, K, cache_path=None):
    """Times the candidate tilings of `mode` on a batch of K Lambda, keeps the fastest (cached in
    `cache_path` per device and workload when given) and returns it."""
    cp = cache_path.encode() if cache_path else None
    _check(ctx, load_library().pop_autotune(ctx, int(mode), int(K), cp))
    return pop_get_tiling(ctx, mode)


def pop_set_graphs(ctx, enable: bool):
    """Turns CUDA-graph replay of the evaluation pipeline on (default) or off."""
    _check(ctx, load_library().pop_set_graphs(ctx, 1 if enable else 0))


def pop_last_kernel_ms(ctx):
    """(weight-kernel ms, whole-pipeline ms) of the last pop_loglik, from CUDA events."""
    w, t = ctypes.c_double(), ctypes.c_double()
    _check(ctx, load_library().pop_last_kernel_ms(ctx, ctypes.byref(w), ctypes.byref(t)))
    return w.value, t.value


POP_WAIT_CHECK_MAX_POLLS = 1 << 18


def pop_wait_check(ctx, arrive, polls):
    """One bounded mbarrier wait of the grid contraction's kind on the GPU: returns None when the
    barrier completes (arrive=True) and raises PopError(POP_ETIMEOUT) when it gives up after
    ``polls`` polls (arrive=False)."""
    _check(ctx, load_library().pop_wait_check(ctx, int(bool(arrive)), int(polls)))


PIPE_RATE_NAMES = ("dfma", "ffma", "ex2", "rcp", "ffma2_lanes", "lds128_32addr", "lds128_4addr")


def pop_pipe_rates(device=0):
    """Measured rates per SM clock: thread operations for "dfma", "ffma", "ex2", "rcp"; FP32 lanes
    of packed fma.rn.f32x2 ("ffma2_lanes"); warp-wide 16-byte shared loads with 32 and 4 distinct
    addresses ("lds128_32addr", "lds128_4addr")."""
    r = np.zeros(len(PIPE_RATE_NAMES))
    _check(None, load_library().pop_pipe_rates_n(int(device), r.ctypes.data_as(ctypes.c_void_p), r.size))
    return dict(zip(PIPE_RATE_NAMES, (float(v) for v in r)))


def pop_math_check(ctx, fn, x):
    """The FP64 kernel's exp (0), expm1 (1) or reciprocal (2), the float-float kernel's exp (3),
    expm1 (4), reciprocal (5), square (6) and exact FP32 hi-part square (7), or the finalise's
    ln (8), evaluated on the GPU."""
    xa = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(xa)
    _check(ctx, load_library().pop_math_check(ctx, int(fn), xa.size, xa.ctypes.data_as(ctypes.c_void_p),
                                              y.ctypes.data_as(ctypes.c_void_p), POP_MEM_HOST))
    return y


def pop_load_vt_grid(ctx, m1_nodes, q_nodes, pdet):
    """Grid selection term: nodes and pdet [len(m1), len(q)] (numpy arrays or CUDA tensors)."""
    mp, mem, k1 = _arg(m1_nodes, np.float64)
    qp, mem2, k2 = _arg(q_nodes, np.float64)
    pp, mem3, k3 = _arg(pdet, np.float64)
    if not (mem == mem2 == mem3):
        raise TypeError("m1, q and pdet must all be host arrays or all device tensors")
    n1, nq = int(m1_nodes.shape[0]), int(q_nodes.shape[0])
    if tuple(pdet.shape) != (n1, nq):
        raise ValueError(f"pdet must have shape ({n1}, {nq})")
    _check(ctx, load_library().pop_load_vt_grid(ctx, n1, mp, nq, qp, pp, mem))


def pop_set_xi_source(ctx, source):
    """Selection term of pop_loglik: POP_XI_INJECTIONS (default) or POP_XI_GRID."""
    _check(ctx, load_library().pop_set_xi_source(ctx, int(source)))


def pop_xi_grid(ctx, lambdas, mode=POP_MODE_F64):
    """ln xi_grid and flags for each row of ``lambdas`` (host arrays; synchronous)."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    K, P = lam.shape
    lx, fl = np.empty(K), np.empty(K, np.uint32)
    _check(ctx, load_library().pop_xi_grid(ctx, K, P, lam.ctypes.data_as(ctypes.c_void_p), int(mode),
                                           lx.ctypes.data_as(ctypes.c_void_p), fl.ctypes.data_as(ctypes.c_void_p),
                                           POP_MEM_HOST))
    return lx, fl


def pop_xi_grid_last_ms(ctx):
    """(contraction-kernel ms, whole grid-term ms) of the last grid evaluation."""
    w, t = ctypes.c_double(), ctypes.c_double()
    _check(ctx, load_library().pop_xi_grid_last_ms(ctx, ctypes.byref(w), ctypes.byref(t)))
    return w.value, t.value


def _f32(a, shape=None):
    x = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and x.shape != shape:
        raise ValueError(f"expected shape {shape}, got {x.shape}")
    return x, x.ctypes.data_as(ctypes.c_void_p)


def pop_mlp_gemm_check(ctx, A, B):
    """C = A B^T on the tensor cores (A [M x K], B [N x K] rounded to BF16)."""
    a, pa = _f32(A)
    b, pb = _f32(B)
    M, K = a.shape
    N = b.shape[0]
    c = np.empty((M, N), np.float32)
    _check(ctx, load_library().pop_mlp_gemm_check(ctx, M, N, K, pa, pb, c.ctypes.data_as(ctypes.c_void_p)))
    return c


def pop_mlp_set_params(ctx, flat):
    """Sets the network's FP32 master parameters from a flat array of MLP_N_PARAMS floats."""
    p, pp = _f32(flat, (MLP_N_PARAMS,))
    _check(ctx, load_library().pop_mlp_set_params(ctx, pp, MLP_N_PARAMS))


def pop_mlp_get_params(ctx):
    """The network's FP32 master parameters as a flat array of MLP_N_PARAMS floats."""
    out = np.empty(MLP_N_PARAMS, np.float32)
    _check(ctx, load_library().pop_mlp_get_params(ctx, out.ctypes.data_as(ctypes.c_void_p), MLP_N_PARAMS))
    return out


def pop_mlp_forward(ctx, x):
    """Network outputs [B, 2] for normalised inputs x [B, 12] (BF16 tensor cores, FP32 accumulate)."""
    xa, px = _f32(x)
    y = np.empty((xa.shape[0], 2), np.float32)
    _check(ctx, load_library().pop_mlp_forward(ctx, xa.shape[0], px, y.ctypes.data_as(ctypes.c_void_p)))
    return y


def pop_mlp_gradients(ctx, x, t):
    """(flat parameter gradients, loss) of the mean squared error against targets t [B, 2]."""
    xa, px = _f32(x)
    ta, pt = _f32(t)
    g = np.empty(MLP_N_PARAMS, np.float32)
    loss = ctypes.c_double()
    _check(ctx, load_library().pop_mlp_gradients(ctx, xa.shape[0], px, pt, g.ctypes.data_as(ctypes.c_void_p),
                                                 ctypes.byref(loss)))
    return g, loss.value


def pop_mlp_train_step(ctx, x, t, lr):
    """One Adam step (beta 0.9 / 0.999, eps 1e-8) of the network on the batch (x, t)."""
    xa, px = _f32(x)
    ta, pt = _f32(t)
    _check(ctx, load_library().pop_mlp_train_step(ctx, xa.shape[0], px, pt, float(lr)))


def pop_xi_surrogate_train(ctx, n_pairs, lo, hi, epochs=100, heldout_frac=0.1, seed=0):
    """Trains the ln xi network on n_pairs Lambda drawn uniformly from the box [lo, hi], with
    targets from the loaded injections; returns the held-out error in ln xi."""
    lo_a = np.ascontiguousarray(lo, dtype=np.float64)
    hi_a = np.ascontiguousarray(hi, dtype=np.float64)
    rmse = ctypes.c_double()
    _check(ctx, load_library().pop_xi_surrogate_train(ctx, int(n_pairs), float(heldout_frac), int(seed),
                                                      lo_a.ctypes.data_as(ctypes.c_void_p),
                                                      hi_a.ctypes.data_as(ctypes.c_void_p), lo_a.size, int(epochs),
                                                      ctypes.byref(rmse)))
    return rmse.value


def pop_xi_surrogate_info(ctx):
    """Held-out error, the targets' Monte Carlo scatter, their difference and the trust gate."""
    r, n, e, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(ctx, load_library().pop_xi_surrogate_info(ctx, ctypes.byref(r), ctypes.byref(n), ctypes.byref(e),
                                                     ctypes.byref(t)))
    return {"heldout_rmse": r.value, "mc_noise": n.value, "excess": e.value, "trusted": bool(t.value)}


def pop_xi_surrogate_infer(ctx, lambdas):
    """(ln xi, ln N_eff, fallback mask) from the trained network for each Lambda row."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    K, P = lam.shape
    lx, ln, fb = np.empty(K), np.empty(K), np.empty(K, np.uint8)
    _check(ctx, load_library().pop_xi_surrogate_infer(ctx, K, P, lam.ctypes.data_as(ctypes.c_void_p),
                                                      lx.ctypes.data_as(ctypes.c_void_p),
                                                      ln.ctypes.data_as(ctypes.c_void_p),
                                                      fb.ctypes.data_as(ctypes.c_void_p), POP_MEM_HOST))
    return lx, ln, fb


def pop_xi_surrogate_error(ctx, lambdas):
    """The surrogate's error bound on ln xi for each Lambda row (from its held-out pairs)."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    K, P = lam.shape
    err = np.empty(K)
    _check(ctx, load_library().pop_xi_surrogate_error(ctx, K, P, lam.ctypes.data_as(ctypes.c_void_p),
                                                      err.ctypes.data_as(ctypes.c_void_p), POP_MEM_HOST))
    return err


def pop_xi_surrogate_train_stats(ctx):
    """Seconds spent on the targets and on the fit of the last training, and the rows fitted."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(ctx, load_library().pop_xi_surrogate_train_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
    return {"target_seconds": a.value, "fit_seconds": b.value, "fit_rows": n.value}


def pop_xi_surrogate_set_budget(ctx, nats):
    """Largest N x error bound (nats of ln L) for which a Lambda uses the network (default 0.25)."""
    _check(ctx, load_library().pop_xi_surrogate_set_budget(ctx, float(nats)))


def pop_xi_surrogate_save(ctx, path):
    """Writes the trained network, its normalisation and held-out statistics to `path`."""
    _check(ctx, load_library().pop_xi_surrogate_save(ctx, str(path).encode()))


def pop_xi_surrogate_load(ctx, path):
    """Reads a network written by pop_xi_surrogate_save."""
    _check(ctx, load_library().pop_xi_surrogate_load(ctx, str(path).encode()))


def pop_loglik_f64_noalloc(offsets, theta, prior, n_draw, inj_theta, p_draw, lambdas, out, stream=None):
    """FP64 ln L with no device allocation by the library (see include/pop.h).

    Every argument but ``n_draw`` is a contiguous CUDA tensor the caller owns,
    all on one GPU (offsets int64, the rest float64; ``out`` = (lnL, lnxi,
    neff, flags int32), each of length K).  The call runs on that GPU, on
    ``stream`` (default: torch's current stream there, so that it is ordered
    after the work that wrote the inputs).  Synchronous; raises PopError on
    failure, ValueError when a tensor is not on the GPU of ``offsets``.
    """
    tensors = (offsets, theta, prior, inj_theta, p_draw, lambdas) + tuple(out)
    if not all(_is_torch(t) and t.is_cuda for t in tensors):
        raise ValueError("pop_loglik_f64_noalloc takes CUDA tensors only")
    device = offsets.device.index
    if any(t.device.index != device for t in tensors):
        raise ValueError(f"every tensor must be on cuda:{device}, the device of offsets")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device)
    ptr = lambda t, dt: _arg(t, dt)[0]
    msg = ctypes.create_string_buffer(512)
    rc = load_library().pop_loglik_f64_noalloc(
        int(device), _stream_ptr(stream), int(offsets.shape[0]) - 1, ptr(offsets, np.int64), int(theta.shape[0]),
        int(theta.shape[1]), ptr(theta, np.float64), ptr(prior, np.float64), int(inj_theta.shape[0]), int(n_draw),
        ptr(inj_theta, np.float64), ptr(p_draw, np.float64), int(lambdas.shape[0]), int(lambdas.shape[1]),
        ptr(lambdas, np.float64), ptr(out[0], np.float64), ptr(out[1], np.float64), ptr(out[2], np.float64),
        ptr(out[3], np.uint32), msg, 512)
    if rc != POP_OK:
        raise PopError(rc, msg.value.decode())
    return out


# ------------------------------------------------------------------ convenience
class Likelihood:
    """One context: load a catalog and injections once, evaluate many Lambda batches."""

    def __init__(self, device=0, stream=None):
        if stream is None:
            import torch
            torch.cuda.set_device(device)
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.ctx = pop_create(device, stream)

    def load(self, catalog, injections, storage=POP_STORE_F64 | POP_STORE_F32):
        self.n_events = catalog.n_events
        pop_load_events(self.ctx, catalog.offsets, catalog.theta, catalog.prior, storage)
        pop_load_injections(self.ctx, injections.n_draw, injections.theta, injections.p_draw, storage)
        return self

    def __call__(self, lambdas, mode=POP_MODE_F64):
        return pop_loglik(self.ctx, lambdas, mode)

    def close(self):
        if self.ctx:
            pop_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
