"""ctypes wrapper of the plain FP64 CPU oracle (``pop_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are its only users.  The product
library never imports, links or runs it, and the two share no code.

``build()`` compiles ``liboracle.so`` next to this file with gcc (OpenMP when
the compiler has it).  Functions mirror the C entry points one to one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pop_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FLAG_INVALID_LAMBDA = 1
FLAG_ZERO_EVENT = 2
FLAG_LOW_NEFF = 4
FLAG_ZERO_XI = 32


def build(force: bool = False) -> str:
    """Compile the oracle with gcc; returns the path of the shared library."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        # POP_ORACLE_LIB points the pins at another build of this file (the mutation tests
        # plant mistakes in a copy and check that the pins catch them).
        lib = ctypes.CDLL(os.environ.get("POP_ORACLE_LIB") or build())
        d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        for name in ("pop_oracle_p_m1", "pop_oracle_p_chi", "pop_oracle_p_z"):
            getattr(lib, name).argtypes = [d, p]
            getattr(lib, name).restype = d
        lib.pop_oracle_p_q.argtypes = [d, d, p]
        lib.pop_oracle_p_q.restype = d
        lib.pop_oracle_p_tilt.argtypes = [d, d, p]
        lib.pop_oracle_p_tilt.restype = d
        lib.pop_oracle_z_norm.argtypes = [d]
        lib.pop_oracle_z_norm.restype = d
        lib.pop_oracle_p_theta.argtypes = [p, i32, p]
        lib.pop_oracle_p_theta.restype = d
        lib.pop_oracle_lambda_valid.argtypes = [p, i32]
        lib.pop_oracle_lambda_valid.restype = i32
        lib.pop_oracle_loglik.argtypes = [i64, p, i32, p, p, i64, i64, p, p, i64, i32, p, i32, p, p, p, p]
        lib.pop_oracle_loglik.restype = i32
        lib.pop_oracle_max_threads.restype = i32
        lib.pop_oracle_loglik_parts.argtypes = [i64, p, i32, p, p, i64, p, p, i64, i32, p, i32, p, p, p, p]
        lib.pop_oracle_loglik_parts.restype = i32
        lib.pop_oracle_loglik_grad.argtypes = [i64, p, i32, p, p, i64, i64, p, p, i64, i32, p, i32, p, p, p]
        lib.pop_oracle_loglik_grad.restype = i32
        lib.pop_oracle_score.argtypes = [p, i32, p, i32, p]
        lib.pop_oracle_score.restype = d
        lib.pop_oracle_digamma.argtypes = [d]
        lib.pop_oracle_digamma.restype = d
        lib.pop_oracle_cbc_loglik.argtypes = [i32, i64, d, d, p, p, p, p, i64, p, i32, p]
        lib.pop_oracle_cbc_loglik.restype = i32
        lib.pop_oracle_xi_grid.argtypes = [i32, p, i32, p, p, i64, i32, p, p, p]
        lib.pop_oracle_xi_grid.restype = i32
        _lib = lib
    return _lib


def _lam(L):
    a = np.ascontiguousarray(L, dtype=np.float64)
    if a.shape[-1] < 12:
        a = np.concatenate([a, np.ones(12 - a.shape[-1])])
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def p_m1(m1, L):
    a = _lam(L)
    return _load().pop_oracle_p_m1(float(m1), _ptr(a))


def p_q(q, m1, L):
    a = _lam(L)
    return _load().pop_oracle_p_q(float(q), float(m1), _ptr(a))


def p_chi(x, L):
    a = _lam(L)
    return _load().pop_oracle_p_chi(float(x), _ptr(a))


def p_tilt(c1, c2, L):
    a = _lam(L)
    return _load().pop_oracle_p_tilt(float(c1), float(c2), _ptr(a))


def p_z(z, L):
    a = _lam(L)
    return _load().pop_oracle_p_z(float(z), _ptr(a))


def z_norm(kappa):
    return _load().pop_oracle_z_norm(float(kappa))


def p_theta(theta, L):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    a = _lam(L)
    return _load().pop_oracle_p_theta(_ptr(th), th.shape[-1], _ptr(a))


def lambda_valid(L):
    a = np.ascontiguousarray(L, dtype=np.float64)
    return bool(_load().pop_oracle_lambda_valid(_ptr(a), a.shape[-1]))


def max_threads():
    return _load().pop_oracle_max_threads()


def xi_grid(m1_nodes, q_nodes, pdet, lambdas):
    """ln xi on a regular (m1, q) grid with detection probability pdet [n_m1, n_q]; (lnxi, flags)."""
    m1 = np.ascontiguousarray(m1_nodes, dtype=np.float64)
    q = np.ascontiguousarray(q_nodes, dtype=np.float64)
    pd = np.ascontiguousarray(pdet, dtype=np.float64)
    lam = np.ascontiguousarray(np.atleast_2d(lambdas), dtype=np.float64)
    K, P = lam.shape
    out, fl = np.empty(K), np.empty(K, np.uint32)
    rc = _load().pop_oracle_xi_grid(m1.size, _ptr(m1), q.size, _ptr(q), _ptr(pd), K, P, _ptr(lam), _ptr(out),
                                    _ptr(fl))
    if rc != 0:
        raise ValueError("oracle rejected the grid")
    return out, fl


def loglik_parts(catalog, injections, lambdas, nthreads=0):
    """(sum_i ln(S_i/n_i), sum_k w_k, sum_k w_k^2, flags) for each row of ``lambdas`` over the given
    events and found injections; parts of disjoint sets add up to those of their union."""
    lam = np.ascontiguousarray(np.atleast_2d(lambdas), dtype=np.float64)
    K, P = lam.shape
    off = np.ascontiguousarray(catalog.offsets, dtype=np.int64)
    th = np.ascontiguousarray(catalog.theta, dtype=np.float64)
    pr = np.ascontiguousarray(catalog.prior, dtype=np.float64)
    ith = np.ascontiguousarray(injections.theta, dtype=np.float64)
    pd = np.ascontiguousarray(injections.p_draw, dtype=np.float64)
    out = np.empty(K), np.empty(K), np.empty(K), np.empty(K, np.uint32)
    rc = _load().pop_oracle_loglik_parts(len(off) - 1, _ptr(off), th.shape[1], _ptr(th), _ptr(pr), ith.shape[0],
                                         _ptr(ith), _ptr(pd), K, P, _ptr(lam), int(nthreads),
                                         _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(out[3]))
    if rc != 0:
        raise ValueError("oracle rejected the input sizes")
    return out


def score(theta, L):
    """(p(theta | Lambda), d ln p / d Lambda) for one sample."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    a = np.ascontiguousarray(L, dtype=np.float64)
    g = np.empty(a.size)
    pv = _load().pop_oracle_score(_ptr(th), th.size, _ptr(a), a.size, _ptr(g))
    return pv, g


def digamma(x):
    return _load().pop_oracle_digamma(float(x))


def loglik_grad(catalog, injections, lambdas, nthreads=0):
    """(ln L, d ln L / d Lambda [K, n_params], flags) for each row of ``lambdas``."""
    lam = np.ascontiguousarray(np.atleast_2d(lambdas), dtype=np.float64)
    K, P = lam.shape
    off = np.ascontiguousarray(catalog.offsets, dtype=np.int64)
    th = np.ascontiguousarray(catalog.theta, dtype=np.float64)
    pr = np.ascontiguousarray(catalog.prior, dtype=np.float64)
    ith = np.ascontiguousarray(injections.theta, dtype=np.float64)
    pd = np.ascontiguousarray(injections.p_draw, dtype=np.float64)
    lnL, grad, fl = np.empty(K), np.empty((K, P)), np.empty(K, np.uint32)
    rc = _load().pop_oracle_loglik_grad(len(off) - 1, _ptr(off), th.shape[1], _ptr(th), _ptr(pr), ith.shape[0],
                                        int(injections.n_draw), _ptr(ith), _ptr(pd), K, P, _ptr(lam), int(nthreads),
                                        _ptr(lnL), _ptr(grad), _ptr(fl))
    if rc != 0:
        raise ValueError("oracle rejected the input sizes")
    return lnL, grad, fl


def cbc_loglik(f0, df, data, psd, hp, hc, thetas, nthreads=0):
    """Single-event CBC ln L (Eq. cbclike) for each row of ``thetas`` [K, 2 + 3 n_det];
    data [n_det, M] complex, psd [n_det, M], hp and hc [M] complex."""
    d = np.ascontiguousarray(np.asarray(data, np.complex128)).view(np.float64)
    S = np.ascontiguousarray(psd, dtype=np.float64)
    a = np.ascontiguousarray(np.asarray(hp, np.complex128)).view(np.float64)
    b = np.ascontiguousarray(np.asarray(hc, np.complex128)).view(np.float64)
    th = np.ascontiguousarray(np.atleast_2d(thetas), dtype=np.float64)
    n_det, M = S.shape
    if th.shape[1] != 2 + 3 * n_det or data.shape != S.shape or len(hp) != M or len(hc) != M:
        raise ValueError("inconsistent CBC shapes")
    out = np.empty(th.shape[0])
    rc = _load().pop_oracle_cbc_loglik(n_det, M, float(f0), float(df), _ptr(d), _ptr(S), _ptr(a), _ptr(b),
                                       th.shape[0], _ptr(th), int(nthreads), _ptr(out))
    if rc != 0:
        raise ValueError("oracle rejected the CBC inputs")
    return out


def loglik(catalog, injections, lambdas, nthreads=0):
    """ln L, ln xi, N_eff and flags for each row of ``lambdas`` [K, P]."""
    lam = np.ascontiguousarray(np.atleast_2d(lambdas), dtype=np.float64)
    K, P = lam.shape
    off = np.ascontiguousarray(catalog.offsets, dtype=np.int64)
    th = np.ascontiguousarray(catalog.theta, dtype=np.float64)
    pr = np.ascontiguousarray(catalog.prior, dtype=np.float64)
    ith = np.ascontiguousarray(injections.theta, dtype=np.float64)
    pd = np.ascontiguousarray(injections.p_draw, dtype=np.float64)
    out = np.empty(K), np.empty(K), np.empty(K), np.empty(K, np.uint32)
    rc = _load().pop_oracle_loglik(len(off) - 1, _ptr(off), th.shape[1], _ptr(th), _ptr(pr),
                                   ith.shape[0], int(injections.n_draw), _ptr(ith), _ptr(pd),
                                   K, P, _ptr(lam), int(nthreads),
                                   _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(out[3]))
    if rc != 0:
        raise ValueError("oracle rejected the input sizes")
    return out
