"""Pins of the oracle's tensor-core core (CORE_TC): the direct core's blocks,
each companded (Eq. 2) at S_q = K_q = Q, the largest Q with N' Q^2 <= 2^24 and
Q <= 2048, its integers convolved exactly (Eq. 1 on s~ and k~) and scaled back
(Eq. 16); blocks whose Section IV.D model misses the target plus its margin run
full precision.  The bound is pinned by what FP16 and FP32 arithmetic do, the
integers by a brute-force integer convolution, the selection by measurement."""
import numpy as np
import pytest

import oracle as O
from paper_1201_3018_gb300 import workloads as wl


def test_tc_bound_values():
    # Q^2 N' <= 2^24 and Q <= 2048: 508 at N' = 65 (2^24 / 65 = 258,111.0...),
    # the FP16 cap for N' <= 3, 1831 at N' = 5
    assert O.qmax_direct(O.BLK_TC, 65) == 508
    assert O.qmax_direct(O.BLK_TC, 1) == 2048 and O.qmax_direct(O.BLK_TC, 3) == 2048
    assert O.qmax_direct(O.BLK_TC, 5) == 1831
    for nodd in (1, 3, 5, 17, 65, 257, 1025, 4097):
        q = O.qmax_direct(O.BLK_TC, nodd)
        assert nodd * q * q <= 1 << 24 and q <= 2048
        assert q == 2048 or nodd * (q + 1) * (q + 1) > 1 << 24
        assert O.exact_ok(O.BLK_TC, nodd, q, q) and not O.exact_ok(O.BLK_TC, nodd, q + 1, q + 1)


def test_tc_operands_exact_in_fp16():
    """Every integer of magnitude up to 2048 is an FP16 value; 2049 is not."""
    x = np.arange(-2048, 2049)
    assert np.array_equal(x.astype(np.float16).astype(np.int64), x)
    assert int(np.float16(2049)) != 2049


@pytest.mark.parametrize("nodd", [65, 257, 1025])
def test_tc_bound_is_tight_for_fp32_sums(nodd):
    """At Q the extreme sums (every product +Q^2, or alternating signs) stay
    exact when accumulated in FP32 in any order; one step beyond the bound the
    all-positive sum of odd products passes 2^24 at an odd value and rounds."""
    q = O.qmax_direct(O.BLK_TC, nodd)
    rng = np.random.default_rng(nodd)
    for prods in (np.full(nodd, q * q, np.int64),
                  np.array([q * q * (1 if i % 2 == 0 else -1) for i in range(nodd)], np.int64),
                  rng.choice([-1, 1], nodd) * rng.integers(0, q + 1, nodd) * q):
        want = int(prods.sum())
        for order in (np.arange(nodd), np.arange(nodd)[::-1], rng.permutation(nodd)):
            acc = np.float32(0)
            for v in prods[order]:
                acc = np.float32(acc + np.float32(v))  # products of FP16 integers are exact in FP32
            assert int(acc) == want
    q1 = q + 1 if (q + 1) % 2 == 1 else q + 2  # odd, beyond the bound
    acc = np.float32(0)
    for _ in range(nodd):
        acc = np.float32(acc + np.float32(q1 * q1))
    assert nodd * q1 * q1 > 1 << 24 and int(acc) != nodd * q1 * q1


def _tc_case(seed, dist, L, N, Wb, target, op=O.OP_CONV):
    s = wl.random_signal(seed, L, dist, 0.1 if dist == "laplace" else 1.0)
    s = (s * np.linspace(0.1, 2.0, L) ** 3).astype(np.float32)  # blocks of very different statistics
    k = wl.random_signal(seed + 1, N, "uniform")
    mode = op | O.CORE_TC | O.PACK_AUTO
    r, rq, st, rc = O.apx_conv(s, k, Wb, mode, snr_db=target, nthreads=0)
    assert rc == 0
    return s, k, mode, r, rq, O.stats_arrays(st)


@pytest.mark.parametrize("dist,L,N,Wb,op", [("normal", 30000, 64, 1024, O.OP_CONV),
                                           ("laplace", 20000, 255, 2048, O.OP_XCORR),
                                           ("uniform", 9000, 17, 512, O.OP_CONV)])
def test_tc_block_integers_are_the_companded_convolution(dist, L, N, Wb, op):
    """Every CORE_TC block's integers equal numpy's integer convolution of its
    own companded window with the companded kernel, and its outputs equal them
    times (c_s c_k)^-1 (Eq. 16)."""
    s, k, mode, r, rq, st = _tc_case(7, dist, L, N, Wb, 40.0, op)
    kk = k[::-1].copy() if op == O.OP_XCORR else k
    p = O.plan(L, N, Wb, False)
    Q = O.qmax_direct(O.BLK_TC, p.Nodd)
    Mk = O.maxabs(kk)
    ck = O.compand_factor(Q, Mk)
    kq = O.compand(kk, ck).astype(np.int64)
    ntc = 0
    for b in range(p.P):
        st0 = O.block_start(p, b)
        lo, hi = O.block_out_range(p, b)
        win = np.array([s[g] if 0 <= g < L else 0.0 for g in range(st0, st0 + Wb)], np.float32)
        if st["mode"][b] != O.BLK_TC:
            continue
        ntc += 1
        assert st["Sq"][b] == Q and st["Kq"][b] == Q
        cs = O.compand_factor(Q, O.maxabs(win))
        assert np.float32(st["cs"][b]) == cs
        sq = O.compand(win, cs).astype(np.int64)
        full = np.convolve(sq, kq)[:Wb]
        gi = np.arange(st0 + lo, st0 + hi)
        keep = (gi >= 0) & (gi < L + N - 1)
        j = np.arange(lo, hi)[keep]
        assert np.array_equal(rq[gi[keep]], full[j]), b
        want = (full[j].astype(np.float64) / (np.float64(cs) * np.float64(ck))).astype(np.float32)
        assert np.array_equal(r[gi[keep]], want), b
    assert ntc > 0


@pytest.mark.parametrize("target", [30.0, 45.0, 55.0])
def test_tc_selection_meets_the_target(target):
    """Section IV.D with the margin: every block the selector puts on the
    tensor-core core measures at least the target (its kept outputs against
    Eq. (1) in FP64); the others are full precision and equal Eq. (1)."""
    rng = np.random.default_rng(int(target))
    tc = full = 0
    for trial in range(6):
        dist = ("normal", "laplace", "uniform")[trial % 3]
        N = int(rng.choice([9, 64, 200]))
        Wb = int(rng.choice([512, 1024, 2048]))
        s, k, mode, r, rq, st = _tc_case(100 + trial, dist, 12000, N, Wb, target)
        ref = O.conv_ref(s.astype(np.float64), k.astype(np.float64))
        p = O.plan(len(s), N, Wb, False)
        for b in range(p.P):
            st0 = O.block_start(p, b)
            lo, hi = O.block_out_range(p, b)
            gi = np.arange(st0 + lo, st0 + hi)
            gi = gi[(gi >= 0) & (gi < len(r))]
            if st["mode"][b] == O.BLK_TC:
                tc += 1
                assert st["snr_pred_db"][b] >= target + O.snr_margin_db(p.W) - 1e-9
                err = r[gi].astype(np.float64) - ref[gi]
                snr = 10 * np.log10(np.sum(ref[gi] ** 2) / np.sum(err ** 2))
                assert snr >= target, (trial, b, snr)
            elif st["mode"][b] == O.BLK_FULL:
                full += 1
                np.testing.assert_allclose(r[gi], ref[gi], rtol=1e-5, atol=1e-6 * np.abs(ref).max())
    assert tc > 0 and (target < 50 or full > 0)


def test_tc_modes():
    s = wl.random_signal(3, 5000, "normal")
    k = wl.random_signal(4, 33, "uniform")
    r, rq, st, rc = O.apx_conv(s, k, 1024, O.CORE_TC | O.PACK_NONE, nthreads=0)
    assert rc == 0 and all(x.mode == O.BLK_FULL for x in st)
    for pack in (O.PACK_SYM, O.PACK_ASYM2, O.PACK_ASYM3):
        assert O.apx_conv(s, k, 1024, O.CORE_TC | pack, Sq=15, Kq=15, nthreads=0)[3] == O.ERR_ARG
