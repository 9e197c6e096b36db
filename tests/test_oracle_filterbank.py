"""Pins of the oracle's exact-integer filterbank (Eq. (1) on the companded
values of Eq. (2), inverse companding Eq. (16), per block of T outputs)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1201_3018_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_exact_when_quantization_is_lossless():
    # integer inputs whose maximum is S_q (and K_q for every filter): c_s = c_k = 1,
    # so the method reduces to Eq. (1), which numpy computes exactly on integers
    g = np.random.default_rng(1)
    L, N, F, T, Q = 3000, 37, 3, 256, 100
    s = g.integers(-Q, Q + 1, L).astype(np.float32)
    s[::T] = Q          # every window holds the maximum
    k = g.integers(-Q, Q + 1, (F, N)).astype(np.float32)
    k[:, 0] = Q
    y, yq, cs = O.filterbank(s, k, T, Q, Q)
    assert np.all(cs == 1.0)
    for f in range(F):
        ref = np.convolve(s.astype(np.int64), k[f].astype(np.int64))
        np.testing.assert_array_equal(yq[f], ref)
        np.testing.assert_array_equal(y[f], ref.astype(np.float32))


def test_integer_domain_matches_blockwise_brute_force():
    # every block: numpy's integer convolution of the block's own quantized window
    g = np.random.default_rng(2)
    L, N, F, T, Sq, Kq = 1500, 20, 2, 128, 90, 70
    s = (g.standard_normal(L) * np.linspace(0.1, 5.0, L)).astype(np.float32)
    k = g.uniform(-1, 1, (F, N)).astype(np.float32)
    y, yq, cs = O.filterbank(s, k, T, Sq, Kq)
    out_len = L + N - 1
    for f in range(F):
        ck = np.float32(Kq) / np.float32(np.abs(k[f]).max())
        kq = np.rint(ck * k[f]).astype(np.int64)
        for b in range((out_len + T - 1) // T):
            t0 = b * T
            idx = np.arange(t0 - N + 1, t0 + T)
            w = np.where((idx >= 0) & (idx < L), s[np.clip(idx, 0, L - 1)], 0).astype(np.float32)
            c = np.float32(Sq) / np.float32(np.abs(w).max())
            assert cs[b] == c
            q = np.rint(c * w).astype(np.int64)
            full = np.convolve(q, kq)          # index u + n
            t1 = min(t0 + T, out_len)
            # output t uses q[t - t0 + N - 1 - n] k[n]: full-conv index t - t0 + N - 1
            np.testing.assert_array_equal(yq[f, t0:t1], full[N - 1:N - 1 + t1 - t0])


def test_error_within_quantization_bound():
    # |y - conv(s, k)| <= sum_n (|k_n| d_s + |s| d_k + d_s d_k) + FP32 rounding,
    # d_s = 1 / (2 c_s), d_k = 1 / (2 c_k): a dropped term or a wrong scale fails
    g = np.random.default_rng(3)
    L, N, F, T, Sq, Kq = 4000, 64, 2, 512, 127, 127
    s = g.standard_normal(L).astype(np.float32)
    k = g.uniform(-1, 1, (F, N)).astype(np.float32)
    y, yq, cs = O.filterbank(s, k, T, Sq, Kq)
    out_len = L + N - 1
    for f in range(F):
        exact = O.conv_ref(s, k[f])
        ck = np.float32(Kq) / np.float32(np.abs(k[f]).max())
        for b in range((out_len + T - 1) // T):
            t0, t1 = b * T, min(b * T + T, out_len)
            ds, dk = 0.5 / float(cs[b]), 0.5 / float(ck)
            ms = np.abs(s).max()
            bound = N * (np.abs(k[f]).max() * ds + ms * dk + ds * dk)
            err = np.abs(y[f, t0:t1] - exact[t0:t1])
            assert np.all(err <= bound + 1e-6 * np.abs(exact[t0:t1]) + 1e-30)


def test_zero_window_and_zero_filter():
    s = np.zeros(2000, np.float32)
    s[1500:1510] = 1.0
    k = np.ones((2, 5), np.float32)
    k[1] = 0.0
    y, yq, cs = O.filterbank(s, k, 256, 50, 50)
    assert cs[0] == 0.0 and cs[1] == 0.0          # windows that see no sample
    assert np.all(y[1] == 0) and np.all(yq[1] == 0)
    np.testing.assert_allclose(y[0], np.convolve(s, k[0]), rtol=1e-6)


def test_block_range_equals_slice_of_full_run():
    g = np.random.default_rng(4)
    s = g.laplace(0, 0.1, 5000).astype(np.float32)
    k = g.uniform(-1, 1, (3, 40)).astype(np.float32)
    y, yq, cs = O.filterbank(s, k, 256, 127, 127)
    y2, yq2, cs2 = O.filterbank(s, k, 256, 127, 127, blocks=(5, 9))
    np.testing.assert_array_equal(yq2[:, 5 * 256:9 * 256], yq[:, 5 * 256:9 * 256])
    assert np.all(yq2[:, :5 * 256] == 0) and np.all(yq2[:, 9 * 256:] == 0)


def test_measured_snr_matches_paper_quantization_pin():
    # Section IV.A settings (iid U[-128, 128] inputs, N = 800, S_q = K_q = 16):
    # quantization alone gives the SNR the paper measures for the packed modes
    gold = GOLD["snr_measured_db"]["symmetric_Sq16"]
    g = np.random.default_rng(5)
    L, N = 1 << 16, 800
    s = g.uniform(-128, 128, L).astype(np.float32)
    k = g.uniform(-128, 128, (1, N)).astype(np.float32)
    y, _, _ = O.filterbank(s, k, 3 * N + 1, 16, 16)
    ref = O.conv_ref(s, k[0])
    snr = 10 * math.log10(np.sum(ref ** 2) / np.sum((y[0] - ref) ** 2))
    assert abs(snr - gold) < 0.6, snr


def test_nonfinite_rejected():
    s = np.ones(100, np.float32)
    s[7] = np.inf
    with pytest.raises(ArithmeticError):
        O.filterbank(s, np.ones((1, 3), np.float32), 64, 10, 10)
