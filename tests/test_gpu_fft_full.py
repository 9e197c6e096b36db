"""The FFT core's full-precision kernel on a pair of CTAs (a call with no
packing candidate and no per-block records: one block per two-CTA cluster,
exchanging data through distributed shared memory) against the general block
kernel, which runs when the caller asks for per-block records: the same bits,
for single calls of many or few blocks and batched calls, with zero and
non-finite blocks and with input and output pointers off the 8-byte alignment
of the paired loads and stores; and against Eq. (1) in FP64."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1201_3018_gb300 import apx
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = apx.Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _pair(ctx, s, k, Wb, mode, snr, r_off=0):
    """(full-only kernel result, general kernel result) of one call."""
    L, N = s.numel(), k.numel()
    P, _ = apx.plan_blocks(L, N, Wb, mode)
    buf = torch.full((L + N - 1 + r_off,), float("nan"), device="cuda")
    r = buf[r_off:]
    ctx.apx_conv(s, k, Wb, mode, snr, r)
    st = torch.empty(P * apx.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    r2 = torch.full((L + N - 1,), float("nan"), device="cuda")
    ctx.apx_conv(s, k, Wb, mode, snr, r2, None, st)
    status = 0
    try:
        ctx.apx_sync()
    except apx.ApxError as e:
        status = e.status
    modes = np.frombuffer(st.cpu().numpy().tobytes(), dtype=apx.STATS_DTYPE)["mode"]
    return r.cpu().numpy(), r2.cpu().numpy(), modes, status


@pytest.mark.parametrize("L,N,Wb,op", [(1 << 20, 4096, 8192, apx.OP_XCORR),   # the matching workload, one launch
                                       (300000, 1000, 4096, apx.OP_CONV),
                                       (40000, 700, 2048, apx.OP_XCORR),      # fewer than 64 blocks: three launches
                                       (5000, 63, 1024, apx.OP_CONV),
                                       (200000, 8191, 16384, apx.OP_CONV)])
@pytest.mark.parametrize("off", [0, 1])
def test_full_only_kernel_equals_general_kernel(ctx, L, N, Wb, op, off):
    s = wl.random_signal(L + 61 + off, L + off, "laplace", 0.1)
    k = wl.random_signal(N + 62, N, "uniform")
    sd = _dev(s)[off:]  # off = 1: the window loads lose their 8-byte alignment
    kd = _dev(k)
    mode = op | apx.CORE_FFT | apx.PACK_NONE
    got, gen, modes, status = _pair(ctx, sd, kd, Wb, mode, 0.0, r_off=off)
    assert status == 0 and np.all(modes == apx.BLK_FULL)
    np.testing.assert_array_equal(got, gen)
    idx = np.random.default_rng(N).choice(L + N - 1, 3000, replace=False)
    kk = k[::-1].copy() if op == apx.OP_XCORR else k
    ref = O.conv_ref_at(s[off:], kk, idx)
    err = np.linalg.norm(got[idx] - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err


def test_full_only_kernel_special_blocks(ctx):
    """Zero blocks give zeros, a non-finite sample NaN for its blocks and
    APX_ERR_NONFINITE, as the general kernel; and an all-zero kernel zeros."""
    L, N, Wb = 200000, 500, 2048
    s = wl.random_signal(71, L, "normal")
    s[20000:60000] = 0.0
    s[123456] = np.inf
    k = wl.random_signal(72, N, "uniform")
    mode = apx.CORE_FFT | apx.PACK_NONE
    got, gen, modes, status = _pair(ctx, _dev(s), _dev(k), Wb, mode, 0.0)
    assert status == apx.APX_ERR_NONFINITE
    assert np.array_equal(np.isnan(got), np.isnan(gen)) and np.isnan(got).any()
    fin = ~np.isnan(gen)
    np.testing.assert_array_equal(got[fin], gen[fin])
    assert (modes == apx.BLK_ZERO).sum() > 5 and (modes == apx.BLK_NONFINITE).sum() >= 1
    got, gen, modes, status = _pair(ctx, _dev(wl.random_signal(73, L, "normal")), _dev(np.zeros(N, np.float32)), Wb,
                                    mode, 0.0)
    assert status == 0 and np.all(got == 0) and np.all(gen == 0)


def test_full_only_kernel_batched(ctx):
    """A batch whose requests keep no packing candidate (the general kernel)
    equals, request by request, the single calls of the two-CTA kernel."""
    items = []
    g = np.random.default_rng(5)
    for i in range(12):
        L = int(2 ** g.uniform(14, 19))
        N = int(g.choice([100, 255, 1024, 3000]))
        Wb = int(g.choice([1024, 2048, 4096, 8192]))
        if Wb - (N | 1) - 1 < 2:
            Wb = 8192
        s = _dev(wl.random_signal(500 + i, L, "laplace", 0.1))
        k = _dev(wl.random_signal(600 + i, N, "uniform"))
        items.append(dict(s=s, k=k, r=torch.full((L + N - 1,), float("nan"), device="cuda"),
                          mode=(i % 2) | apx.CORE_FFT | apx.PACK_NONE, W_block=Wb))
    ctx.apx_conv_batch(ctx.make_requests(items))
    assert ctx.apx_sync() == 0
    for it in items:
        L, N = it["s"].numel(), it["k"].numel()
        r2 = torch.empty(L + N - 1, device="cuda")
        ctx.apx_conv(it["s"], it["k"], it["W_block"], it["mode"], 0.0, r2)
        assert ctx.apx_sync() == 0
        np.testing.assert_array_equal(it["r"].cpu().numpy(), r2.cpu().numpy())
