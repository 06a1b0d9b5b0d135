"""CPU oracle for non-binary LDPC decoding (test infrastructure): min-max
(Alg. 2) and FFT-based sum-product (Alg. 1).

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
may import this package.  The decoder library and its Python binding never do.
The arithmetic lives in ``nbldpc_oracle.c`` (min-max) and ``fftspa_oracle.c``
(FFT-SPA, in double precision), plain C built with gcc; this module only
compiles them and marshals numpy arrays through ctypes.

Every function follows Alg. 2 or Alg. 1 of the paper (see the C sources for
the step-by-step citations and the readings taken where the paper is silent).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("nbldpc_oracle.c", "fftspa_oracle.c")]
_DEPS = _SRCS + [os.path.join(_HERE, "oracle_common.h")]
_LIB = os.path.join(_HERE, "liboracle_nbldpc.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, plain C, no SIMD intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(map(os.path.getmtime, _DEPS)):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Werror",
                               *_SRCS, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            L.orc_gf_tables.argtypes = [ctypes.c_int, ctypes.c_uint, i32p, i32p]
            L.orc_gf_mul_all.argtypes = [ctypes.c_int, ctypes.c_uint, i32p, i32p]
            L.orc_check_update.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, i32p, u8p, u8p]
            L.orc_check_update_counted.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, i32p, u8p, u8p,
                                                   ctypes.POINTER(ctypes.c_longlong)]
            L.orc_decode.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                                     i32p, i32p, i32p, u8p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, u8p, i32p, u8p]
            L.orc_decode_cap.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                                         i32p, i32p, i32p, u8p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, u8p, i32p, u8p]
            L.orc_decode_trace.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                                           i32p, i32p, i32p, u8p, ctypes.c_int, ctypes.c_int,
                                           i32p, i32p, i32p, u8p]
            L.orc_syndrome_ok.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                                          i32p, i32p, i32p, u8p, ctypes.c_int, u8p]
            f32p = ctypes.POINTER(ctypes.c_float)
            f64p = ctypes.POINTER(ctypes.c_double)
            L.orc_wht.argtypes = [ctypes.c_int, f64p]
            L.orc_fft_check_update.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, i32p, f64p, f64p]
            L.orc_fftspa_decode.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                                            i32p, i32p, i32p, f32p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, u8p, i32p, u8p, f64p]
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def gf_tables(q: int, poly: int):
    """(exp[q-1], log[q]) or None when the polynomial is not primitive."""
    e = np.zeros(max(q - 1, 1), np.int32)
    lg = np.zeros(q, np.int32)
    if lib().orc_gf_tables(q, poly, _p(e, ctypes.c_int32), _p(lg, ctypes.c_int32)):
        return None
    return e, lg


def gf_mul_all(q: int, poly: int):
    """(mul[q, q], inv[q]) through the oracle's own exp/log tables."""
    m = np.zeros(q * q, np.int32)
    inv = np.zeros(q, np.int32)
    if lib().orc_gf_mul_all(q, poly, _p(m, ctypes.c_int32), _p(inv, ctypes.c_int32)):
        return None
    return m.reshape(q, q), inv


def check_update(q: int, poly: int, h, alpha: np.ndarray) -> np.ndarray:
    """beta [d, q] for one check node with coefficients h[d] and messages alpha [d, q]."""
    h = np.ascontiguousarray(h, np.int32)
    a = np.ascontiguousarray(alpha, np.uint8)
    d = h.size
    b = np.zeros((d, q), np.uint8)
    rc = lib().orc_check_update(q, poly, d, _p(h, ctypes.c_int32), _p(a, ctypes.c_uint8),
                                _p(b, ctypes.c_uint8))
    if rc:
        raise ValueError("invalid check")
    return b


def check_update_pairs(q: int, poly: int, h, alpha: np.ndarray):
    """(beta [d, q], pairs [3]): the check update and the (x', x'') pairs its forward, backward
    and beta remaining-edge blocks visited."""
    h = np.ascontiguousarray(h, np.int32)
    a = np.ascontiguousarray(alpha, np.uint8)
    d = h.size
    b = np.zeros((d, q), np.uint8)
    pairs = np.zeros(3, np.int64)
    rc = lib().orc_check_update_counted(q, poly, d, _p(h, ctypes.c_int32), _p(a, ctypes.c_uint8),
                                        _p(b, ctypes.c_uint8), _p(pairs, ctypes.c_longlong))
    if rc:
        raise ValueError("invalid check")
    return b, pairs


def _code_arrays(code):
    return (np.ascontiguousarray(code.row_ptr, np.int32), np.ascontiguousarray(code.col_idx, np.int32),
            np.ascontiguousarray(code.coef, np.int32))


def decode(code, gamma: np.ndarray, max_iters: int, early_stop: int, threads: int = 1, cap: int = 255):
    """(symbols [F, N] uint8, iterations [F] int32, ok [F] uint8) for gamma [F, N, q] uint8.

    cap: saturation of the variable-node messages (255: 8-bit messages; 65535: 16-bit)."""
    g = np.ascontiguousarray(gamma, np.uint8)
    f = g.shape[0]
    assert g.shape[1:] == (code.n, code.q)
    rp, ci, cf = _code_arrays(code)
    sym = np.zeros((f, code.n), np.uint8)
    its = np.zeros(f, np.int32)
    ok = np.zeros(f, np.uint8)
    L = lib()

    def run(lo, hi):
        if hi <= lo:
            return 0
        return L.orc_decode_cap(code.q, code.poly, code.n, code.m, _p(rp, ctypes.c_int32),
                                _p(ci, ctypes.c_int32), _p(cf, ctypes.c_int32),
                                _p(g[lo:hi], ctypes.c_uint8), hi - lo, max_iters, early_stop, cap,
                                _p(sym[lo:hi], ctypes.c_uint8), _p(its[lo:hi], ctypes.c_int32),
                                _p(ok[lo:hi], ctypes.c_uint8))

    if threads <= 1 or f <= 1:
        rc = run(0, f)
    else:
        # one frame per task: ctypes releases the GIL during the C call
        with ThreadPoolExecutor(max_workers=threads) as ex:
            rc = max([abs(r) for r in ex.map(lambda i: run(i, i + 1), range(f))] + [0])
    if rc:
        raise ValueError("oracle rejected the code or arguments")
    return sym, its, ok


def decode_trace(code, gamma: np.ndarray, iters: int, cap: int = 255):
    """One frame (gamma [N, q]) decoded for exactly `iters` iterations without early stop:
    (beta [E, q], S [N, q], alpha [E, q], symbols [N]) of the last iteration, edges in CSR order."""
    g = np.ascontiguousarray(gamma, np.uint8)
    assert g.shape == (code.n, code.q)
    rp, ci, cf = _code_arrays(code)
    e = int(rp[-1])
    beta = np.zeros((e, code.q), np.int32)
    s = np.zeros((code.n, code.q), np.int32)
    alpha = np.zeros((e, code.q), np.int32)
    sym = np.zeros(code.n, np.uint8)
    rc = lib().orc_decode_trace(code.q, code.poly, code.n, code.m, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32),
                                _p(cf, ctypes.c_int32), _p(g, ctypes.c_uint8), int(iters), int(cap),
                                _p(beta, ctypes.c_int32), _p(s, ctypes.c_int32), _p(alpha, ctypes.c_int32),
                                _p(sym, ctypes.c_uint8))
    if rc:
        raise ValueError("oracle rejected the code or arguments")
    return beta, s, alpha, sym


def syndrome_ok(code, words: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(words, np.uint8)
    rp, ci, cf = _code_arrays(code)
    out = np.zeros(w.shape[0], np.uint8)
    rc = lib().orc_syndrome_ok(code.q, code.poly, code.n, code.m, _p(rp, ctypes.c_int32),
                               _p(ci, ctypes.c_int32), _p(cf, ctypes.c_int32),
                               _p(w, ctypes.c_uint8), w.shape[0], _p(out, ctypes.c_uint8))
    if rc:
        raise ValueError("bad field")
    return out


# ------------------------------------------------------------------ FFT-SPA
def wht(v: np.ndarray) -> np.ndarray:
    """Radix-2 Walsh-Hadamard transform of a length-q vector (float64 copy)."""
    a = np.array(v, np.float64).copy()
    lib().orc_wht(a.size, _p(a, ctypes.c_double))
    return a


def fft_check_update(q: int, poly: int, h, u: np.ndarray) -> np.ndarray:
    """v' [d, q] (float64) of one check with coefficients h[d] and messages u [d, q]."""
    h = np.ascontiguousarray(h, np.int32)
    a = np.ascontiguousarray(u, np.float64)
    d = h.size
    out = np.zeros((d, q), np.float64)
    if lib().orc_fft_check_update(q, poly, d, _p(h, ctypes.c_int32), _p(a, ctypes.c_double),
                                  _p(out, ctypes.c_double)):
        raise ValueError("invalid check")
    return out


def fftspa_decode(code, prob: np.ndarray, max_iters: int, early_stop: int, threads: int = 1,
                  want_app: bool = False):
    """FFT-SPA (Alg. 1) in float64 for prob [F, N, q] float32 channel probabilities.

    Returns (symbols [F, N] uint8, iterations [F] int32, ok [F] uint8) and, with
    want_app, the normalized a-posteriori vectors [F, N, q] float64."""
    pr = np.ascontiguousarray(prob, np.float32)
    f = pr.shape[0]
    assert pr.shape[1:] == (code.n, code.q)
    rp, ci, cf = _code_arrays(code)
    sym = np.zeros((f, code.n), np.uint8)
    its = np.zeros(f, np.int32)
    ok = np.zeros(f, np.uint8)
    app = np.zeros((f, code.n, code.q), np.float64) if want_app else None
    L = lib()

    def run(lo, hi):
        if hi <= lo:
            return 0
        ap = _p(app[lo:hi], ctypes.c_double) if want_app else None
        return L.orc_fftspa_decode(code.q, code.poly, code.n, code.m, _p(rp, ctypes.c_int32),
                                   _p(ci, ctypes.c_int32), _p(cf, ctypes.c_int32),
                                   _p(pr[lo:hi], ctypes.c_float), hi - lo, max_iters, early_stop,
                                   _p(sym[lo:hi], ctypes.c_uint8), _p(its[lo:hi], ctypes.c_int32),
                                   _p(ok[lo:hi], ctypes.c_uint8), ap)

    if threads <= 1 or f <= 1:
        rc = run(0, f)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            rc = max([abs(r) for r in ex.map(lambda i: run(i, i + 1), range(f))] + [0])
    if rc:
        raise ValueError("oracle rejected the code or arguments")
    return (sym, its, ok, app) if want_app else (sym, its, ok)
