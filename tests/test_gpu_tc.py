"""Tensor-core filterbank (apx_filterbank) against the oracle's exact-integer
filterbank: the integer outputs bit for bit, the per-block c_s bit for bit,
the dequantised outputs within 1e-6 relative (one FP32 rounding of
(c_s c_k)^-1 on the GPU against the oracle's single FP64 division)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1201_3018_gb300 import apx
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = apx.Context(0)
    yield c
    c.close()


def run_gpu(ctx, s, kb, Sq, Kq, pad=0):
    F, N = kb.shape
    L = len(s)
    out_len = L + N - 1
    ldy = (out_len + 3) // 4 * 4 + pad
    T, nb = apx.filterbank_blocks(L, F, N, Sq, Kq)
    sd = torch.from_numpy(s).cuda()
    kd = torch.from_numpy(np.ascontiguousarray(kb)).cuda()
    y = torch.full((F, ldy), float("nan"), device="cuda")
    yq = torch.full((F, ldy), -7, dtype=torch.int32, device="cuda")
    cs = torch.empty(nb, device="cuda")
    ctx.apx_filterbank(sd, kd, Sq, Kq, y, yq, cs)
    assert ctx.apx_sync() == 0
    y, yq, cs = y.cpu().numpy(), yq.cpu().numpy(), cs.cpu().numpy()
    # nothing written past the outputs
    assert np.all(np.isnan(y[:, out_len:])) and np.all(yq[:, out_len:] == -7)
    return y[:, :out_len], yq[:, :out_len].astype(np.int64), cs, T, nb


def check_blocks(y, yq, cs, yo, yqo, cso, T, blocks):
    for b in blocks:
        sl = slice(b * T, (b + 1) * T)
        np.testing.assert_array_equal(yq[:, sl], yqo[:, sl])
        assert cs[b] == cso[b]
        np.testing.assert_allclose(y[:, sl], yo[:, sl], rtol=1e-6, atol=0)


CASES = [  # L, F, N, Sq, Kq (S_q, K_q <= 16: FP8 operands)
    (20000, 5, 100, 127, 127),     # P = 64, three blocks, ragged tail, partial kernel group
    (50000, 5, 100, 16, 16),       # FP8: P = 128, partial group of two
    (70000, 1, 300, 16, 9),        # FP8, one kernel: P = 256
    (40000, 2, 1023, 12, 16),      # FP8, two kernels, N + P - 1 not a multiple of 128
    (20000, 3, 16384, 16, 16),     # FP8, the longest kernel
    (70000, 1, 300, 200, 200),     # P = 256
    (5000, 2, 1, 2048, 2048),      # P = 128, one tap
    (9000, 3, 1023, 127, 127),     # N + P - 1 not a multiple of 64
    (40000, 9, 64, 500, 500),      # three kernel groups, the last partial
    (3, 4, 2, 16, 16),             # shorter than a row
    (20000, 1, 16384, 32, 32),     # the longest kernel
]


@pytest.mark.parametrize("L,F,N,Sq,Kq", CASES)
def test_filterbank_matches_oracle(ctx, L, F, N, Sq, Kq):
    s = wl.random_signal(L + 11, L, "normal")
    s = (s * np.linspace(0.1, 4.0, L)).astype(np.float32)   # blocks with different c_s
    kb = np.stack([wl.random_signal(1000 + f, N, "uniform") for f in range(F)])
    y, yq, cs, T, nb = run_gpu(ctx, s, kb, Sq, Kq)
    yo, yqo, cso = O.filterbank(s, kb, T, Sq, Kq)
    check_blocks(y, yq, cs, yo, yqo, cso, T, range(nb))


def test_padded_rows_and_zero_kernel_and_silence(ctx):
    L, F, N = 30000, 6, 200
    s = wl.random_signal(5, L, "laplace", 0.1)
    s[8000:] = 0.0               # blocks whose windows are silent
    kb = np.stack([wl.random_signal(50 + f, N, "uniform") for f in range(F)])
    kb[2] = 0.0
    y, yq, cs, T, nb = run_gpu(ctx, s, kb, 127, 127, pad=36)
    yo, yqo, cso = O.filterbank(s, kb, T, 127, 127)
    check_blocks(y, yq, cs, yo, yqo, cso, T, range(nb))
    assert np.all(yq[2] == 0) and np.all(y[2] == 0)
    assert 0.0 in cs


def test_filterbank_full_size_sampled(ctx):
    """2^22 N(0,1) samples through 32 Hann-windowed-sinc band-pass kernels of
    1024 taps (log-spaced bands, 50 Hz - 20 kHz at 44.1 kHz), S_q = K_q = 127:
    the first, a middle and the last block against the oracle; the SNR of the
    dequantised outputs against Eq. (1) in FP64 on sampled outputs."""
    s, kb = wl.filterbank()
    F, N = kb.shape
    y, yq, cs, T, nb = run_gpu(ctx, s, kb, 127, 127)
    for b in (0, nb // 2, nb - 1):
        yo, yqo, cso = O.filterbank(s, kb, T, 127, 127, blocks=(b, b + 1))
        check_blocks(y, yq, cs, yo, yqo, cso, T, [b])
    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(len(s) + N - 1, 2000, replace=False))
    snrs = []
    for f in (0, 8, 16, 31):
        ref = O.conv_ref_at(s, kb[f], idx)
        snrs.append(10 * math.log10(np.sum(ref ** 2) / np.sum((y[f, idx] - ref) ** 2)))
    assert min(snrs) > 15.0, snrs


def test_filterbank_errors(ctx):
    s = torch.zeros(1000, device="cuda")
    kb = torch.zeros(4, 100, device="cuda")
    y = torch.zeros(4, 1100, device="cuda")
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_filterbank(s, kb, 2048, 2048, y)     # 100 * 2048^2 > 2^24
    assert e.value.status == apx.APX_ERR_RANGE
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_filterbank(s, kb, 4096, 1, y)        # beyond exact FP16 integers
    assert e.value.status == apx.APX_ERR_RANGE
    y_short = torch.zeros(4, 1096, device="cuda")     # ldy < L + N - 1
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_filterbank(s, kb, 16, 16, y_short)
    assert e.value.status == apx.APX_ERR_ARG
