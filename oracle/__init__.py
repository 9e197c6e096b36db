"""Plain FP64 CPU oracle for the approximate overlap-save convolution of
Anam & Andreopoulos (arXiv 1201.3018).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the CUDA
library and its binding) never imports this package, and this package never
imports the product.

The arithmetic lives in ``apx_oracle.c`` (plain loops, FP64, no fused
multiply-add); this module compiles it with gcc on first use and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apx_oracle.c")
_HDR = os.path.join(_HERE, "apx_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# mode word (op | core | pack), same bit layout as the public ABI
OP_CONV, OP_XCORR = 0x0, 0x1
CORE_DIRECT, CORE_FFT, CORE_TC = 0x00, 0x10, 0x30
PACK_AUTO, PACK_NONE, PACK_SYM, PACK_ASYM2, PACK_ASYM3 = 0x000, 0x100, 0x200, 0x300, 0x400
LITERAL = 0x2000  # the paper-literal symmetric form (Eq. 6 eps, FP64 Eqs. 11-15 with u_sys)
BLK_FULL, BLK_SYM, BLK_ASYM2, BLK_ASYM3, BLK_ZERO, BLK_NONFINITE, BLK_TC = 0, 1, 2, 3, 4, 5, 6
OK, ERR_ARG, ERR_WBLOCK, ERR_RANGE, ERR_INEXACT = 0, -1, -2, -3, -4


class BlockStats(C.Structure):
    _fields_ = [("mode", C.c_int32), ("Sq", C.c_int32), ("Kq", C.c_int32), ("b", C.c_int32),
                ("cs", C.c_float), ("maxabs", C.c_float), ("sigma2", C.c_double),
                ("snr_pred_db", C.c_double), ("fft_err", C.c_double)]


class Plan(C.Structure):
    _fields_ = [("L", C.c_int64), ("N", C.c_int32), ("Nodd", C.c_int32), ("Wblock", C.c_int32),
                ("W", C.c_int32), ("fft", C.c_int32), ("head", C.c_int32), ("P", C.c_int64), ("out_len", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and \
            os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=gnu11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(L):
    d, f, i32, i64, u32, vp = C.c_double, C.c_float, C.c_int32, C.c_int64, C.c_uint32, C.c_void_p
    sig = {
        "or_conv_ref": (None, [vp, i64, vp, i32, vp]),
        "or_xcorr_ref": (None, [vp, i64, vp, i32, vp]),
        "or_conv_int": (None, [vp, i64, vp, i32, vp]),
        "or_conv_ref_at": (None, [vp, i64, vp, i32, vp, i64, vp]),
        "or_plan": (C.c_int, [i64, i32, i32, C.c_int, C.POINTER(Plan)]),
        "or_block_start": (i64, [C.POINTER(Plan), i64]),
        "or_block_out_range": (None, [C.POINTER(Plan), i64, C.POINTER(i32), C.POINTER(i32)]),
        "or_maxabs": (f, [vp, i64]),
        "or_second_moment": (d, [vp, i64, f]),
        "or_bits": (i32, [i64]),
        "or_exact_ok": (C.c_int, [C.c_int, i32, i32, i32]),
        "or_qmax_direct": (i32, [C.c_int, i32]),
        "or_qmax_fft": (i32, [C.c_int, i32, i32]),
        "or_snr_model_lin": (d, [d, f, d, f, i32, i32]),
        "or_snr_model_db": (d, [d, f, d, f, i32, i32]),
        "or_snr_feasible": (C.c_int, [d, f, d, f, i32, i32, d]),
        "or_snr_margin_db": (d, [i32]),
        "or_fft_err_digits": (d, [C.c_int, i32, d, d, i32]),
        "or_compand_factor": (f, [i32, f]),
        "or_compand": (None, [vp, i64, f, vp]),
        "or_pack_sym_signal": (None, [vp, i32, i32, vp]),
        "or_pack_sym_kernel": (None, [vp, i32, i32, vp]),
        "or_pack_sym_kernel_printed": (None, [vp, i32, i32, vp]),
        "or_pack_asym_signal": (None, [vp, i32, i32, i32, vp]),
        "or_conv_f64": (None, [vp, i64, vp, i64, vp, i64]),
        "or_conv_f64_fft": (C.c_int, [vp, i64, vp, i64, vp, i64, i64]),
        "or_unpack_sym": (C.c_int, [vp, i32, i32, i64, i32, vp]),
        "or_unpack_sym_digits": (C.c_int, [vp, i32, i32, i32, vp]),
        "or_unpack_sym_fp64": (None, [vp, i32, i32, d, d, d, vp]),
        "or_unpack_asym": (C.c_int, [vp, i32, i32, i32, i64, i32, i32, vp]),
        "or_apx_conv": (C.c_int, [vp, i64, vp, i32, i32, u32, d, i32, i32, vp, vp, vp, C.c_int, vp]),
        "or_filterbank": (C.c_int, [vp, i64, vp, i32, i32, i32, i32, i32, i64, i64, vp, i64, vp, vp, C.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _i64(x):
    return np.ascontiguousarray(x, dtype=np.int64)


# ---------------------------------------------------------------- definitions
def conv_ref(s, k):
    """Eq. (1) in FP64, brute force: length L + N - 1."""
    s, k = _f64(s), _f64(k)
    r = np.empty(len(s) + len(k) - 1, np.float64)
    lib().or_conv_ref(_p(s), len(s), _p(k), len(k), _p(r))
    return r


def xcorr_ref(s, t):
    """Cross-correlation by its definition, sum_n s[n + l] t[n], stored at index l + N - 1."""
    s, t = _f64(s), _f64(t)
    r = np.empty(len(s) + len(t) - 1, np.float64)
    lib().or_xcorr_ref(_p(s), len(s), _p(t), len(t), _p(r))
    return r


def conv_ref_at(s, k, idx):
    """Eq. (1) at the given output indices."""
    s, k, idx = _f64(s), _f64(k), _i64(idx)
    r = np.empty(len(idx), np.float64)
    lib().or_conv_ref_at(_p(s), len(s), _p(k), len(k), _p(idx), len(idx), _p(r))
    return r


def conv_int(s, k):
    s, k = _i64(s), _i64(k)
    r = np.empty(len(s) + len(k) - 1, np.int64)
    lib().or_conv_int(_p(s), len(s), _p(k), len(k), _p(r))
    return r


# ---------------------------------------------------------------- steps
def plan(L, N, Wblock, fft=False):
    p = Plan()
    rc = lib().or_plan(L, N, Wblock, 1 if fft else 0, C.byref(p))
    if rc:
        raise ValueError("or_plan rc=%d" % rc)
    return p


def block_start(p, i):
    return lib().or_block_start(C.byref(p), i)


def block_out_range(p, i):
    lo, hi = C.c_int32(), C.c_int32()
    lib().or_block_out_range(C.byref(p), i, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def maxabs(x):
    x = _f32(x)
    return lib().or_maxabs(_p(x), len(x))


def second_moment(x, m=None):
    x = _f32(x)
    if m is None:
        m = maxabs(x)
    return lib().or_second_moment(_p(x), len(x), m)


def bits(rmax):
    return lib().or_bits(int(rmax))


def exact_ok(blk, nodd, S, K):
    return bool(lib().or_exact_ok(blk, nodd, S, K))


def qmax_direct(blk, nodd):
    return lib().or_qmax_direct(blk, nodd)


def qmax_fft(blk, nodd, wblock):
    return lib().or_qmax_fft(blk, nodd, wblock)


def snr_model_db(sig2_s, Ms, sig2_k, Mk, S, K):
    return lib().or_snr_model_db(sig2_s, Ms, sig2_k, Mk, S, K)


def snr_model_lin(sig2_s, Ms, sig2_k, Mk, S, K):
    return lib().or_snr_model_lin(sig2_s, Ms, sig2_k, Mk, S, K)


def snr_feasible(sig2_s, Ms, sig2_k, Mk, S, K, thr_lin):
    return bool(lib().or_snr_feasible(sig2_s, Ms, sig2_k, Mk, S, K, thr_lin))


def snr_margin_db(W):
    """dB by which the Section IV.D model must clear the target (W outputs per block)."""
    return lib().or_snr_margin_db(W)


def fft_err_digits(blk, log2n, l1_kbar, l2_sbar, b):
    return lib().or_fft_err_digits(blk, log2n, l1_kbar, l2_sbar, b)


def compand_factor(Q, m):
    return lib().or_compand_factor(Q, m)


def compand(x, c):
    x = _f32(x)
    q = np.empty(len(x), np.int32)
    lib().or_compand(_p(x), len(x), c, _p(q))
    return q


def pack_sym_signal(sq, b):
    sq = _i32(sq)
    out = np.empty(len(sq) // 2, np.float64)
    lib().or_pack_sym_signal(_p(sq), len(sq), b, _p(out))
    return out


def pack_sym_kernel(kq, b, printed=False):
    """kq holds N' taps (odd count)."""
    kq = _i32(np.concatenate([kq, [0]]))  # room for k~[N'] = 0
    nodd = len(kq) - 1
    out = np.empty((nodd + 1) // 2, np.float64)
    fn = lib().or_pack_sym_kernel_printed if printed else lib().or_pack_sym_kernel
    fn(_p(kq), nodd, b, _p(out))
    return out


def pack_asym_signal(sq, M, b):
    sq = _i32(sq)
    Ls = (len(sq) + M - 1) // M
    out = np.empty(Ls, np.float64)
    lib().or_pack_asym_signal(_p(sq), len(sq), M, b, _p(out))
    return out


def conv_f64(a, k, nr):
    a, k = _f64(a), _f64(k)
    r = np.empty(nr, np.float64)
    lib().or_conv_f64(_p(a), len(a), _p(k), len(k), _p(r), nr)
    return r


def conv_f64_fft(a, k, nr, n):
    a, k = _f64(a), _f64(k)
    r = np.empty(nr, np.float64)
    rc = lib().or_conv_f64_fft(_p(a), len(a), _p(k), len(k), _p(r), nr, n)
    if rc:
        raise ValueError("or_conv_f64_fft rc=%d" % rc)
    return r


def unpack_sym(rbar, wstart, rmax, b):
    rbar = _f64(rbar)
    rq = np.zeros(2 * len(rbar), np.int64)
    rc = lib().or_unpack_sym(_p(rbar), len(rbar), wstart, int(rmax), b, _p(rq))
    if rc:
        raise ArithmeticError("or_unpack_sym rc=%d" % rc)
    return rq


def unpack_sym_digits(rbar, wstart, b):
    rbar = _f64(rbar)
    rq = np.zeros(2 * len(rbar), np.int64)
    rc = lib().or_unpack_sym_digits(_p(rbar), len(rbar), wstart, b, _p(rq))
    if rc:
        raise ArithmeticError("or_unpack_sym_digits rc=%d" % rc)
    return rq


def unpack_sym_fp64(rbar, wstart, rmax, eps, u_sys):
    rbar = _f64(rbar)
    rq = np.zeros(2 * len(rbar), np.float64)
    lib().or_unpack_sym_fp64(_p(rbar), len(rbar), wstart, float(rmax), eps, u_sys, _p(rq))
    return rq


def unpack_asym(rbar, Ls, M, rmax, b, nout):
    rbar = _f64(rbar)
    rq = np.zeros(nout, np.int64)
    rc = lib().or_unpack_asym(_p(rbar), len(rbar), Ls, M, int(rmax), b, nout, _p(rq))
    if rc:
        raise ArithmeticError("or_unpack_asym rc=%d" % rc)
    return rq


# ---------------------------------------------------------------- pipeline
def apx_conv(s, k, Wblock, mode, snr_db=0.0, Sq=0, Kq=0, nthreads=1, want_int=True, want=None):
    """The whole method (a1..a9).  Returns (r_out float32, rq int64 or None,
    stats list of BlockStats, rc).  `want` (bool mask over the L+N-1 outputs)
    limits the full-precision outputs computed; packed blocks and statistics
    are always computed in full."""
    s, k = _f32(s), _f32(k)
    L, N = len(s), len(k)
    fft = (mode & 0xF0) == CORE_FFT
    try:
        p = plan(L, N, Wblock, fft)
        P = p.P
    except ValueError:
        P = 1
    r = np.zeros(L + N - 1, np.float32)
    rq = np.zeros(L + N - 1, np.int64) if want_int else None
    st = (BlockStats * max(P, 1))()
    wm = None if want is None else np.ascontiguousarray(want, dtype=np.uint8)
    rc = lib().or_apx_conv(_p(s), L, _p(k), N, Wblock, mode, float(snr_db), Sq, Kq, _p(r),
                           _p(rq) if want_int else None, st, nthreads, None if wm is None else _p(wm))
    return r, rq, list(st), rc


def filterbank(s, kbank, T, Sq, Kq, blocks=None, nthreads=0):
    """Exact-integer filterbank (Eqs. (1), (2), (16) per block of T outputs).
    kbank: (F, N).  Returns (y float32 (F, L+N-1), yq int64 (F, L+N-1),
    block_cs float32 (nb,)); only `blocks` = (b0, b1) are computed when given
    (the other entries stay zero)."""
    s, kb = _f32(s), _f32(np.atleast_2d(kbank))
    L = len(s)
    F, N = kb.shape
    out_len = L + N - 1
    nb = (out_len + T - 1) // T
    b0, b1 = (0, nb) if blocks is None else blocks
    y = np.zeros((F, out_len), np.float32)
    yq = np.zeros((F, out_len), np.int64)
    cs = np.zeros(nb, np.float32)
    rc = lib().or_filterbank(_p(s), L, _p(kb), F, N, T, Sq, Kq, b0, b1, _p(y), out_len, _p(yq), _p(cs),
                             nthreads)
    if rc:
        raise ArithmeticError("or_filterbank rc=%d" % rc)
    return y, yq, cs


def stats_arrays(stats):
    """BlockStats list -> dict of numpy arrays."""
    out = {}
    for name, _ in BlockStats._fields_:
        out[name] = np.array([getattr(s, name) for s in stats])
    return out
