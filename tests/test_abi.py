"""CPU-side checks of the C ABI: the library builds and loads, exports every
function include/apx.h declares, and its host-only planner agrees with the
oracle's block geometry.  No compute call runs here (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libapx():
    from paper_1201_3018_gb300 import build as b
    b.build()
    from paper_1201_3018_gb300 import apx
    return apx


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(apx_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(libapx):
    L = C.CDLL(libapx.LIB_PATH)
    declared = _declared()
    assert "apx_conv" in declared and "apx_conv_full" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(libapx.SIGNATURES), "binding and header disagree"


def test_strerror(libapx):
    for code in range(0, -9, -1):
        msg = libapx.strerror(code)
        assert msg and msg != "unknown status"
    assert libapx.strerror(-99) == "unknown status"


@pytest.mark.parametrize("fft", [False, True])
@pytest.mark.parametrize("L,N,Wb", [(1, 1, 4), (100, 7, 32), (1000, 64, 256), (513, 8, 64), (10, 29, 32),
                                    (65536, 64, 1024), (1 << 20, 4096, 8192), (999, 1, 8)])
def test_plan_matches_oracle(libapx, fft, L, N, Wb):
    mode = libapx.CORE_FFT if fft else libapx.CORE_DIRECT
    P, W = libapx.plan_blocks(L, N, Wb, mode)
    p = O.plan(L, N, Wb, fft)
    assert (P, W) == (p.P, p.W)


@pytest.mark.parametrize("fft", [False, True])
@pytest.mark.parametrize("N,Wb", [(7, 64), (64, 1024), (257, 2048), (1024, 4096), (4096, 8192), (300, 16384),
                                  (8191, 16384), (4096, 16384), (16380, 16384), (1, 16384), (2047, 4096)])
@pytest.mark.parametrize("snr", [0.0, 12.0, 20.0, 30.0, 45.0, 60.0, 90.0])
def test_candidates_match_oracle(libapx, fft, N, Wb, snr):
    """The host half of the Section IV.D selection against the oracle's own
    arithmetic: the largest S_q = K_q per packing (exact FP64 packed sums, and the FFT
    bound's guide for the FFT core), eps = 2^-b, the Table 1 order, and the
    candidates left out because their model misses the target even at ratios 1."""
    mode = (libapx.CORE_FFT if fft else libapx.CORE_DIRECT) | libapx.PACK_AUTO
    got = libapx.plan_candidates(100000, N, Wb, mode, snr)
    nodd = N if N % 2 else N + 1
    thr = 10.0 ** ((snr + O.snr_margin_db(Wb - nodd - 1)) / 10.0)  # Section IV.D minimum and margin
    want = []
    for blk in (O.BLK_SYM, O.BLK_ASYM3, O.BLK_ASYM2):
        Q = O.qmax_fft(blk, nodd, Wb) if fft else O.qmax_direct(blk, nodd)
        if Q >= 1 and O.snr_model_lin(1.0, 1.0, 1.0, 1.0, Q, Q) >= 0.99 * thr:
            want.append((blk, Q, O.bits(nodd * Q * Q)))
    assert got == want


def test_candidates_forced_and_none(libapx):
    for pack, blk in ((libapx.PACK_SYM, O.BLK_SYM), (libapx.PACK_ASYM2, O.BLK_ASYM2),
                      (libapx.PACK_ASYM3, O.BLK_ASYM3)):
        got = libapx.plan_candidates(5000, 65, 1024, libapx.CORE_DIRECT | pack, 200.0)  # never left out
        Q = O.qmax_direct(blk, 65)
        assert got == ([(blk, Q, O.bits(65 * Q * Q))] if Q >= 1 else got)
    assert libapx.plan_candidates(5000, 65, 1024, libapx.CORE_DIRECT | libapx.PACK_NONE, 0.0) == []
    with pytest.raises(libapx.ApxError):
        libapx.plan_candidates(5000, 65, 65, libapx.CORE_DIRECT | libapx.PACK_AUTO, 0.0)  # W_block too small


@pytest.mark.parametrize("N,Wb,snr", [(64, 1024, 45.0), (1, 512, 30.0), (449, 2048, 40.0), (200, 8192, 55.0),
                                      (64, 1024, 70.0)])
def test_tc_candidates_match_oracle(libapx, N, Wb, snr):
    """The tensor-core core's one candidate: the largest S_q = K_q with
    N' S_q K_q <= 2^24 and S_q <= 2048, no packing digits (b = 0), left out
    when its model misses the target even at ratios 1."""
    got = libapx.plan_candidates(100000, N, Wb, libapx.CORE_TC | libapx.PACK_AUTO, snr)
    nodd = N if N % 2 else N + 1
    thr = 10.0 ** ((snr + O.snr_margin_db(Wb - nodd - 1)) / 10.0)
    Q = O.qmax_direct(O.BLK_TC, nodd)
    want = [(O.BLK_TC, Q, 0)] if O.snr_model_lin(1.0, 1.0, 1.0, 1.0, Q, Q) >= 0.99 * thr else []
    assert got == want
    assert libapx.plan_candidates(100000, N, Wb, libapx.CORE_TC | libapx.PACK_NONE, snr) == []


def test_tc_geometry_errors(libapx):
    """W_block a multiple of 64 up to 8192 (the block's rows fill at most one
    128-row tile), N' <= 449 (at most eight K slices), automatic or no packing."""
    for N, Wb, status in ((64, 1000, libapx.APX_ERR_WBLOCK), (64, 16384, libapx.APX_ERR_WBLOCK),
                          (450, 2048, libapx.APX_ERR_ARG)):
        with pytest.raises(libapx.ApxError) as e:
            libapx.plan_candidates(100000, N, Wb, libapx.CORE_TC | libapx.PACK_AUTO, 45.0)
        assert e.value.status == status
    with pytest.raises(libapx.ApxError) as e:
        libapx.plan_candidates(100000, 64, 1024, libapx.CORE_TC | libapx.PACK_ASYM2, 45.0)
    assert e.value.status == libapx.APX_ERR_ARG
    assert libapx.plan_candidates(100000, 449, 2048, libapx.CORE_TC | libapx.PACK_AUTO, 30.0)[0][0] == O.BLK_TC
    P, W = libapx.plan_blocks(100000, 64, 1024, libapx.CORE_TC)  # the direct core's blocks
    assert (P, W) == libapx.plan_blocks(100000, 64, 1024, libapx.CORE_DIRECT)


def test_plan_errors(libapx):
    with pytest.raises(libapx.ApxError) as e:
        libapx.plan_blocks(100, 3, 31, 0)
    assert e.value.status == libapx.APX_ERR_WBLOCK
    with pytest.raises(libapx.ApxError) as e:
        libapx.plan_blocks(100, 3, 24, libapx.CORE_FFT)
    assert e.value.status == libapx.APX_ERR_WBLOCK
    with pytest.raises(libapx.ApxError) as e:
        libapx.plan_blocks(0, 3, 16, 0)
    assert e.value.status == libapx.APX_ERR_ARG
    with pytest.raises(libapx.ApxError) as e:
        libapx.plan_blocks(100, 3, 16, 0x7000)
    assert e.value.status == libapx.APX_ERR_ARG
    with pytest.raises(libapx.ApxError) as e:
        libapx.plan_blocks(100, 3, 32768, 0)
    assert e.value.status == libapx.APX_ERR_WBLOCK


def test_null_arguments_rejected_without_gpu(libapx):
    L = libapx.lib()
    assert L.apx_conv(None, None, 10, None, 3, 16, 0, 30.0, None, None, None, None) == libapx.APX_ERR_ARG
    assert L.apx_sync(None, None) == libapx.APX_ERR_ARG
    assert L.apx_create(None, 0, 0) == libapx.APX_ERR_ARG


def test_header_constants_match_binding():
    """Every mode, status, block-kind and phase constant of include/apx.h has
    the same value in the Python binding."""
    from paper_1201_3018_gb300 import apx
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "apx.h")).read()
    defs = dict(re.findall(r"#define\s+APX_(\w+)\s+\(?(-?(?:0x)?[0-9A-Fa-f]+)u?\)?", hdr))
    checked = 0
    for name, val in defs.items():
        v = int(val, 0)
        py = name if name.startswith(("OK", "ERR_")) else name
        if hasattr(apx, "APX_" + name):
            assert getattr(apx, "APX_" + name) == v, name
            checked += 1
        elif hasattr(apx, py):
            assert getattr(apx, py) == v, name
            checked += 1
    assert checked >= 25, checked
    assert int(defs["NPHASES"]) == len(apx.PHASES)


def test_request_record_matches_struct():
    from paper_1201_3018_gb300 import apx
    for name, _ in apx.Request._fields_:
        assert apx.REQUEST_DTYPE.fields[name][1] == getattr(apx.Request, name).offset, name
    assert apx.REQUEST_DTYPE.itemsize == C.sizeof(apx.Request) == 80


@pytest.mark.parametrize("F,Q", [(1, 127), (2, 127), (3, 127), (32, 127), (1, 16), (2, 16), (32, 16)])
def test_filterbank_blocks(libapx, F, Q):
    """The filterbank's block geometry as the header states it: T = 128 P with
    P = 256 (one kernel), 128 (two kernels, or FP8 operands when S_q, K_q <= 16)
    or 64 phases per row, and ceil((L+N-1) / T) blocks."""
    L, N = 100000, 1024
    T, nb = libapx.filterbank_blocks(L, F, N, Q, Q)
    P = 256 if F == 1 else (128 if (F == 2 or Q <= 16) else 64)
    assert T == 128 * P and nb == -(-(L + N - 1) // T)
    with pytest.raises(libapx.ApxError) as e:
        libapx.filterbank_blocks(L, 0, N, Q, Q)
    assert e.value.status == libapx.APX_ERR_ARG
    with pytest.raises(libapx.ApxError) as e:
        libapx.filterbank_blocks(L, F, N, 4096, Q)
    assert e.value.status == libapx.APX_ERR_RANGE
