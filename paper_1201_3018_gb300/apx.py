"""Python binding of libapx.so (argument marshalling only).

Every step of the method runs in the library's CUDA kernels; this module turns
torch tensors into device pointers and sizes, calls the C ABI declared in
``include/apx.h`` and raises on a non-zero status.  PyTorch supplies device
memory and streams.  There is no fallback: if the library is missing or no GPU
is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapx.so")
_lock = threading.Lock()
_lib = None

APX_OK, APX_ERR_ARG, APX_ERR_WBLOCK, APX_ERR_RANGE, APX_ERR_NONFINITE = 0, -1, -2, -3, -4
APX_ERR_OOM, APX_ERR_BUDGET, APX_ERR_CUDA, APX_ERR_TIMEOUT, APX_ERR_CHECK = -5, -6, -7, -8, -9
OP_CONV, OP_XCORR = 0x000, 0x001
CORE_DIRECT, CORE_FFT, CORE_AUTO, CORE_TC = 0x000, 0x010, 0x020, 0x030
PACK_AUTO, PACK_NONE, PACK_SYM, PACK_ASYM2, PACK_ASYM3 = 0x000, 0x100, 0x200, 0x300, 0x400
FULL_FP64 = 0x1000
LITERAL = 0x2000
BLK_FULL, BLK_SYM, BLK_ASYM2, BLK_ASYM3, BLK_ZERO, BLK_NONFINITE, BLK_TC = 0, 1, 2, 3, 4, 5, 6

# apx_request as a numpy record (80 bytes, natural C alignment)
REQUEST_DTYPE = np.dtype({"names": ["s_in", "L", "k", "N", "r_out", "W_block", "mode", "snr_target_db", "S_q", "K_q",
                                    "rq_out", "stats"],
                          "formats": ["<u8", "<i8", "<u8", "<i4", "<u8", "<i4", "<u4", "<f8", "<i4", "<i4", "<u8",
                                      "<u8"],
                          "offsets": [0, 8, 16, 24, 32, 40, 44, 48, 56, 60, 64, 72], "itemsize": 80})
STATS_DTYPE = np.dtype([("mode", "<i4"), ("Sq", "<i4"), ("Kq", "<i4"), ("b", "<i4"), ("cs", "<f4"),
                        ("maxabs", "<f4"), ("sigma2", "<f8"), ("snr_pred_db", "<f8"), ("fft_err", "<f8")])
assert STATS_DTYPE.itemsize == 48

class Request(C.Structure):
    """apx_request of include/apx.h."""
    _fields_ = [("s_in", C.c_void_p), ("L", C.c_int64), ("k", C.c_void_p), ("N", C.c_int32),
                ("r_out", C.c_void_p), ("W_block", C.c_int32), ("mode", C.c_uint32), ("snr_target_db", C.c_double),
                ("S_q", C.c_int32), ("K_q", C.c_int32), ("rq_out", C.c_void_p), ("stats", C.c_void_p)]


assert C.sizeof(Request) == 80

# (restype, argtypes) of every entry point in include/apx.h
_vp, _i32, _i64, _u32, _d, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double, C.c_size_t
SIGNATURES = {
    "apx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _sz]),
    "apx_destroy": (None, [_vp]),
    "apx_plan_blocks": (C.c_int, [_i64, _i32, _i32, _u32, C.POINTER(_i64), C.POINTER(_i32)]),
    "apx_plan_candidates": (C.c_int, [_i64, _i32, _i32, _u32, _d, C.POINTER(_i32), C.POINTER(_i32),
                                      C.POINTER(_i32)]),
    "apx_conv": (C.c_int, [_vp, _vp, _i64, _vp, _i32, _i32, _u32, _d, _vp, _vp, _vp, _vp]),
    "apx_conv_fixed": (C.c_int, [_vp, _vp, _i64, _vp, _i32, _i32, _u32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "apx_conv_full": (C.c_int, [_vp, _vp, _i64, _vp, _i32, _i32, _u32, _vp, _vp]),
    "apx_conv_host": (C.c_int, [_vp, _vp, _i64, _vp, _i32, _i32, _u32, _d, _i32, _i32, _vp, _vp]),
    "apx_sync": (C.c_int, [_vp, _vp]),
    "apx_launch_count": (_i64, [_vp]),
    "apx_strerror": (C.c_char_p, [C.c_int]),
    "apx_profile": (C.c_int, [_vp, C.c_int]),
    "apx_conv_fft_static": (C.c_int, [_vp, _i64, _vp, _i32, _i32, _u32, _d, _vp, _vp]),
    "apx_conv_batch": (C.c_int, [_vp, _vp, _i32, _vp]),
    "apx_graph_create": (C.c_int, [_vp, _vp, _i32, _vp, C.POINTER(C.c_void_p)]),
    "apx_graph_launch": (C.c_int, [_vp, _vp]),
    "apx_graph_launch_count": (_i64, [_vp]),
    "apx_graph_destroy": (None, [_vp]),
    "apx_kernel_create": (C.c_int, [_vp, _vp, _i32, _i32, _u32, _vp, C.POINTER(C.c_void_p)]),
    "apx_conv_prepared": (C.c_int, [_vp, _vp, _vp, _i64, C.c_double, _vp, _vp, _vp, _vp]),
    "apx_kernel_destroy": (None, [_vp]),
    "apx_profile_read": (C.c_int, [_vp, _vp, _vp]),
    "apx_conv_batch_host": (C.c_int, [_vp, _vp, _i32, _vp]),
    "apx_test_stall_next": (C.c_int, [_vp]),
    "apx_test_skew_tickets": (C.c_int, [_vp, _i64]),
    "apx_filterbank": (C.c_int, [_vp, _vp, _i64, _vp, _i32, _i32, _i32, _i32, _vp, _i64, _vp, _vp, _vp]),
    "apx_filterbank_blocks": (C.c_int, [_i64, _i32, _i32, _i32, _i32, C.POINTER(_i32), C.POINTER(_i64)]),
    "apx_server_create": (C.c_int, [_vp, _i32, _i32, _i32, _d, C.POINTER(C.c_void_p)]),
    "apx_server_submit": (C.c_int, [_vp, _vp, C.POINTER(_i64)]),
    "apx_server_poll": (C.c_int, [_vp, _i64, C.POINTER(_i32)]),
    "apx_server_destroy": (None, [_vp]),
    "apx_server_test_stall_next": (C.c_int, [_vp]),
    "apx_server_launch_count": (_i64, [_vp]),
}
PHASES = ("direct", "spectra", "fft", "tc_prep", "tc_mma")


def filterbank_blocks(L, F, N, Sq=127, Kq=127):
    """(outputs per block T, number of blocks) of apx_filterbank, as the library
    chooses them (apx_filterbank_blocks)."""
    T, nb = _i32(), _i64()
    _check("apx_filterbank_blocks", lib().apx_filterbank_blocks(L, F, N, Sq, Kq, C.byref(T), C.byref(nb)))
    return T.value, nb.value


class ApxError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (fn, strerror(status), status))


def lib():
    """Load libapx.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            # APX_LIB selects another build of the same library (the bounds-checked
            # libapx_checked.so in the tests)
            path = os.environ.get("APX_LIB") or LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError("libapx.so is not built (%s); run __graft_entry__.build()" % path)
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().apx_strerror(int(status)).decode()


def _check(fn, rc):
    if rc != APX_OK:
        raise ApxError(fn, rc)
    return rc


def plan_blocks(L: int, N: int, W_block: int, mode: int = 0):
    P, W = _i64(), _i32()
    _check("apx_plan_blocks", lib().apx_plan_blocks(L, N, W_block, mode, C.byref(P), C.byref(W)))
    return P.value, W.value


def plan_candidates(L: int, N: int, W_block: int, mode: int, snr_db: float = 0.0):
    """The packing candidates a call with this mode and target gives its blocks,
    in the order they are tried: a list of (APX_BLK_*, S_q = K_q, b)."""
    blk, q, b = (_i32 * 3)(), (_i32 * 3)(), (_i32 * 3)()
    n = lib().apx_plan_candidates(L, N, W_block, mode, float(snr_db), blk, q, b)
    if n < 0:
        raise ApxError("apx_plan_candidates", n)
    return [(blk[j], q[j], b[j]) for j in range(n)]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev_f32(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)
    return t


def _check_call(s, k, r, device, rq=None, stats=None, W_block=None, mode=0):
    """Sizes and devices of a call's tensors: r (and rq) hold L+N-1 outputs,
    stats one record per block, and every tensor is on `device` (the device the
    library launches on), so that a wrong tensor is a Python error rather than
    an out-of-bounds or cross-device access on the GPU."""
    import torch
    out = s.numel() + k.numel() - 1
    if r.numel() < out:
        raise ValueError("r_out holds %d floats, the call writes L+N-1 = %d" % (r.numel(), out))
    if rq is not None and not (rq.is_cuda and rq.dtype == torch.int32 and rq.is_contiguous() and rq.numel() >= out):
        raise ValueError("rq_out must be a contiguous int32 CUDA tensor of at least L+N-1 = %d entries" % out)
    if stats is not None:
        P, _ = plan_blocks(s.numel(), k.numel(), W_block, mode)
        if not (stats.is_cuda and stats.is_contiguous() and stats.numel() * stats.element_size() >= P * STATS_DTYPE.itemsize):
            raise ValueError("stats must be a contiguous CUDA tensor of at least %d bytes" % (P * STATS_DTYPE.itemsize))
    for name, t in (("s_in", s), ("k", k), ("r_out", r), ("rq_out", rq), ("stats", stats)):
        if t is not None and t.device.index != device:
            raise ValueError("%s is on cuda:%s, the call runs on cuda:%d" % (name, t.device.index, device))


class Graph:
    """A captured batch (apx_graph)."""

    def __init__(self, h):
        self._h = h

    def launch(self, stream=None):
        return _check("apx_graph_launch", lib().apx_graph_launch(self._h, _stream(stream)))

    def launch_count(self):
        return lib().apx_graph_launch_count(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().apx_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PreparedKernel:
    """A kernel prepared once and kept resident (apx_kernel)."""

    def __init__(self, h, N, W_block, mode):
        self._h, self.N, self.W_block, self.mode = h, N, W_block, mode

    def close(self):
        if getattr(self, "_h", None):
            lib().apx_kernel_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apx_conv_fft_static(s, k, W_block, mode, snr_db, r, stream=None):
    """Allocation-free FFT-core call (no context): s, k, r are CUDA float32
    tensors on the current device."""
    import torch
    _dev_f32(s, "s_in"); _dev_f32(k, "k"); _dev_f32(r, "r_out")
    _check_call(s, k, r, torch.cuda.current_device())  # the entry point's scratch belongs to the current device
    return _check("apx_conv_fft_static", lib().apx_conv_fft_static(_ptr(s), s.numel(), _ptr(k), k.numel(), W_block,
                                                                   mode, float(snr_db), _ptr(r), _stream(stream)))


class Server:
    """apx_server: the persistent serving kernel on a context's device.
    submit() enqueues one request and returns its sequence number (None when
    every slot or template entry is in use); poll(seq) returns None while the
    request is in flight, else its status code (APX_OK, ...)."""

    def __init__(self, ctx, slots: int = 256, templates: int = 64, ctas: int = 0, idle_ms: float = 20.0):
        h = C.c_void_p()
        _check("apx_server_create", lib().apx_server_create(ctx._h, slots, templates, ctas, float(idle_ms),
                                                             C.byref(h)))
        self._h = h
        self._ctx = ctx  # the context must outlive the server
        self._req = Request()
        self._seq = _i64()
        self._st = _i32()

    def submit(self, s_ptr, L, k_ptr, N, r_ptr, W_block, mode, snr_db):
        """Pointers are device addresses or page-locked host addresses (ints)."""
        q = self._req
        q.s_in, q.L, q.k, q.N, q.r_out = s_ptr, L, k_ptr, N, r_ptr
        q.W_block, q.mode, q.snr_target_db = W_block, mode, float(snr_db)
        q.S_q = q.K_q = 0
        q.rq_out = q.stats = None
        rc = lib().apx_server_submit(self._h, C.byref(q), C.byref(self._seq))
        if rc == APX_ERR_BUDGET:
            return None
        _check("apx_server_submit", rc)
        return self._seq.value

    def poll(self, seq):
        rc = lib().apx_server_poll(self._h, seq, C.byref(self._st))
        if rc < 0:
            raise ApxError("apx_server_poll", rc)
        return self._st.value if rc == 1 else None

    def test_stall_next(self):
        """Failure-path test hook (apx_server_test_stall_next)."""
        return _check("apx_server_test_stall_next", lib().apx_server_test_stall_next(self._h))

    def launch_count(self):
        return lib().apx_server_launch_count(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().apx_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """An apx_ctx on one device: owns the prepared-kernel workspace."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self.device = device
        h = C.c_void_p()
        _check("apx_create", lib().apx_create(C.byref(h), device, budget_bytes))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().apx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def launch_count(self) -> int:
        return lib().apx_launch_count(self._h)

    def profile(self, enable: bool = True):
        _check("apx_profile", lib().apx_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{phase: (total_ms, launches)} since the previous read."""
        ms = (C.c_double * len(PHASES))()
        n = (C.c_int64 * len(PHASES))()
        _check("apx_profile_read", lib().apx_profile_read(self._h, ms, n))
        return {ph: (ms[i], n[i]) for i, ph in enumerate(PHASES)}

    # ---------------------------------------------------------------- raw entry points
    def apx_conv(self, s, k, W_block, mode, snr_db, r, rq=None, stats=None, stream=None):
        _dev_f32(s, "s_in"); _dev_f32(k, "k"); _dev_f32(r, "r_out")
        _check_call(s, k, r, self.device, rq, stats, W_block, mode)
        return _check("apx_conv", lib().apx_conv(self._h, _ptr(s), s.numel(), _ptr(k), k.numel(), W_block, mode,
                                                 float(snr_db), _ptr(r), _ptr(rq), _ptr(stats), _stream(stream)))

    def apx_conv_fixed(self, s, k, W_block, mode, Sq, Kq, r, rq=None, stats=None, stream=None):
        _dev_f32(s, "s_in"); _dev_f32(k, "k"); _dev_f32(r, "r_out")
        _check_call(s, k, r, self.device, rq, stats, W_block, mode)
        return _check("apx_conv_fixed", lib().apx_conv_fixed(self._h, _ptr(s), s.numel(), _ptr(k), k.numel(),
                                                             W_block, mode, Sq, Kq, _ptr(r), _ptr(rq),
                                                             _ptr(stats), _stream(stream)))

    def apx_conv_full(self, s, k, W_block, mode, r, stream=None):
        _dev_f32(s, "s_in"); _dev_f32(k, "k"); _dev_f32(r, "r_out")
        _check_call(s, k, r, self.device)
        return _check("apx_conv_full", lib().apx_conv_full(self._h, _ptr(s), s.numel(), _ptr(k), k.numel(),
                                                           W_block, mode, _ptr(r), _stream(stream)))

    def apx_filterbank(self, s, k_bank, Sq, Kq, y, yq=None, block_cs=None, stream=None):
        """s: (L,) float32; k_bank: (F, N) float32; y: (F, ldy) float32 with
        ldy >= L+N-1 (rows may be padded); yq: None or int32 like y; block_cs:
        None or float32 (blocks,).  All CUDA tensors."""
        import torch
        _dev_f32(s, "s_in"); _dev_f32(k_bank, "k_bank")
        F, N = k_bank.shape
        if not (y.is_cuda and y.dtype == torch.float32 and y.dim() == 2 and y.shape[0] == F and y.stride(1) == 1):
            raise TypeError("y must be a (F, ldy) float32 CUDA tensor with unit inner stride")
        if yq is not None and not (yq.is_cuda and yq.dtype == torch.int32 and yq.shape == y.shape
                                   and yq.stride() == y.stride()):
            raise TypeError("yq must be an int32 CUDA tensor shaped and strided like y")
        if block_cs is not None:
            _dev_f32(block_cs, "block_cs")
        return _check("apx_filterbank", lib().apx_filterbank(self._h, _ptr(s), s.numel(), _ptr(k_bank), F, N, Sq, Kq,
                                                             _ptr(y), y.stride(0), _ptr(yq), _ptr(block_cs),
                                                             _stream(stream)))

    def apx_conv_host(self, s_host, k_host, W_block, mode, snr_db=0.0, Sq=0, Kq=0, r_host=None, stream=None):
        """s_host, k_host, r_host: contiguous float32 CPU tensors (pinned for speed)."""
        L, N = s_host.numel(), k_host.numel()
        return _check("apx_conv_host", lib().apx_conv_host(self._h, _ptr(s_host), L, _ptr(k_host), N, W_block,
                                                           mode, float(snr_db), Sq, Kq, _ptr(r_host),
                                                           _stream(stream)))

    def apx_sync(self, stream=None):
        return _check("apx_sync", lib().apx_sync(self._h, _stream(stream)))

    # ---------------------------------------------------------------- batches
    @staticmethod
    def make_requests(items):
        """items: dicts with s, k, r (CUDA float32 tensors), mode, and optional
        W_block, snr_db, Sq, Kq, rq (int32 CUDA tensor, L+N-1) and stats (CUDA
        tensor of one apx_block_stats record per block).  Returns a ctypes
        array of Request."""
        arr = (Request * len(items))()
        for q, it in zip(arr, items):
            s, k, r = it["s"], it["k"], it["r"]
            _dev_f32(s, "s_in"); _dev_f32(k, "k"); _dev_f32(r, "r_out")
            q.s_in, q.L, q.k, q.N, q.r_out = s.data_ptr(), s.numel(), k.data_ptr(), k.numel(), r.data_ptr()
            q.W_block = int(it.get("W_block", 0))
            q.mode = int(it.get("mode", 0))
            q.snr_target_db = float(it.get("snr_db", 0.0))
            q.S_q, q.K_q = int(it.get("Sq", 0)), int(it.get("Kq", 0))
            rq, st = it.get("rq"), it.get("stats")
            if rq is not None and not (rq.is_cuda and rq.dtype == __import__("torch").int32 and rq.is_contiguous()
                                       and rq.numel() >= s.numel() + k.numel() - 1):
                raise ValueError("rq must be a contiguous int32 CUDA tensor of L+N-1 entries")
            q.rq_out = None if rq is None else rq.data_ptr()
            q.stats = None if st is None else st.data_ptr()
        return arr

    def apx_conv_batch(self, reqs, stream=None):
        return _check("apx_conv_batch", lib().apx_conv_batch(self._h, reqs, len(reqs), _stream(stream)))

    def test_stall_next(self):
        """Failure-path test hook (apx_test_stall_next)."""
        return _check("apx_test_stall_next", lib().apx_test_stall_next(self._h))

    def test_skew_tickets(self, n):
        """Failure-path test hook (apx_test_skew_tickets)."""
        return _check("apx_test_skew_tickets", lib().apx_test_skew_tickets(self._h, int(n)))

    def apx_conv_batch_host(self, reqs, stream=None):
        """reqs: a numpy array of REQUEST_DTYPE (or a ctypes array of Request)
        whose pointers are host addresses."""
        ptr = reqs.ctypes.data if isinstance(reqs, np.ndarray) else C.cast(reqs, C.c_void_p).value
        return _check("apx_conv_batch_host", lib().apx_conv_batch_host(self._h, ptr, len(reqs), _stream(stream)))

    def prepare_kernel(self, k, W_block, mode, stream=None):
        """apx_kernel_create: returns a PreparedKernel (FFT core, PACK_AUTO or
        PACK_NONE)."""
        _dev_f32(k, "k")
        h = C.c_void_p()
        _check("apx_kernel_create", lib().apx_kernel_create(self._h, _ptr(k), k.numel(), W_block, mode,
                                                             _stream(stream), C.byref(h)))
        return PreparedKernel(h, k.numel(), W_block, mode)

    def apx_conv_prepared(self, kp, s, snr_db, r, rq=None, stats=None, stream=None):
        _dev_f32(s, "s_in"); _dev_f32(r, "r_out")
        return _check("apx_conv_prepared", lib().apx_conv_prepared(self._h, kp._h, _ptr(s), s.numel(), float(snr_db),
                                                                   _ptr(r), _ptr(rq), _ptr(stats), _stream(stream)))

    def graph(self, reqs, stream=None):
        """Capture the batch once; returns a Graph (launch() replays it)."""
        h = C.c_void_p()
        _check("apx_graph_create", lib().apx_graph_create(self._h, reqs, len(reqs), _stream(stream), C.byref(h)))
        return Graph(h)

    # ---------------------------------------------------------------- convenience
    def conv(self, s, k, W_block, mode=0, snr_db=None, Sq=None, Kq=None, want_int=False, want_stats=False,
             stream=None):
        """Allocate outputs and run apx_conv / apx_conv_fixed / apx_conv_full.
        Returns (r, rq or None, stats ndarray or None)."""
        import torch
        L, N = s.numel(), k.numel()
        r = torch.empty(L + N - 1, dtype=torch.float32, device=s.device)
        rq = torch.empty(L + N - 1, dtype=torch.int32, device=s.device) if want_int else None
        st = None
        if want_stats:
            P, _ = plan_blocks(L, N, W_block, mode)
            st = torch.empty(P * STATS_DTYPE.itemsize, dtype=torch.uint8, device=s.device)
        pack = mode & 0xF00
        if pack == PACK_NONE and rq is None and st is None:
            self.apx_conv_full(s, k, W_block, mode, r, stream=stream)
        elif Sq is not None and pack != PACK_NONE:
            self.apx_conv_fixed(s, k, W_block, mode, Sq, Kq, r, rq, st, stream=stream)
        else:
            self.apx_conv(s, k, W_block, mode, 0.0 if snr_db is None else snr_db, r, rq, st, stream=stream)
        stats = None
        if st is not None:
            stats = np.frombuffer(st.cpu().numpy().tobytes(), dtype=STATS_DTYPE)
        return r, rq, stats
