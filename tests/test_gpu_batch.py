"""Batched calls and captured graphs against single calls: each request's
result must equal the single call's (integer domain exactly, FP32 outputs
within rounding), whatever else is in the batch."""
import numpy as np
import pytest
import torch

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


def _mixed_requests(seed, count):
    g = np.random.default_rng(seed)
    items = []
    for i in range(count):
        L = int(2 ** g.uniform(10, 16))
        N = int(g.choice([1, 7, 64, 65, 256, 300, 1024]))
        core = [apx.CORE_DIRECT, apx.CORE_FFT, apx.CORE_AUTO][i % 3]
        op = apx.OP_XCORR if i % 2 else apx.OP_CONV
        pack = [apx.PACK_AUTO, apx.PACK_NONE, apx.PACK_ASYM2][i % 3 if i % 5 else 0]
        target = float(g.choice([12.0, 30.0, 45.0, 60.0]))
        Nodd = N | 1
        Wb = 0 if i % 4 == 0 else int(2 ** g.integers(max(6, int(np.ceil(np.log2(Nodd + 3))) + 1), 14))
        if core == apx.CORE_DIRECT and Wb == 0:
            Wb = 0
        s = wl.random_signal(seed * 1000 + i, L, "laplace", 0.1)
        k = wl.random_signal(seed * 1000 + 500 + i, N, "uniform")
        items.append(dict(s=_dev(s), k=_dev(k), r=torch.zeros(L + N - 1, device="cuda"), mode=op | core | pack,
                          W_block=Wb, snr_db=target))
    return items


def _single(ctx, it):
    mode = it["mode"]
    core = mode & 0xF0
    Nodd = it["k"].numel() | 1
    if core == apx.CORE_AUTO:
        core = apx.CORE_FFT if Nodd > 64 else apx.CORE_DIRECT
    Wb = it["W_block"]
    if Wb == 0:
        Wb = 1024
        while Wb < 4 * Nodd and Wb < 16384:
            Wb *= 2
    r, _, _ = ctx.conv(it["s"], it["k"], Wb, (mode & ~0xF0) | core, snr_db=it["snr_db"])
    return r


def test_batch_equals_single_calls(ctx):
    items = _mixed_requests(7, 24)
    reqs = ctx.make_requests(items)
    ctx.apx_conv_batch(reqs)
    ctx.apx_sync()
    for it in items:
        ref = _single(ctx, it).cpu().numpy()
        got = it["r"].cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-6 * max(1.0, float(np.abs(ref).max())))


def test_graph_replays_with_new_inputs(ctx):
    items = _mixed_requests(11, 12)
    reqs = ctx.make_requests(items)
    g = ctx.graph(reqs)
    assert g.launch_count() >= 1
    for rep in range(2):
        for j, it in enumerate(items):  # new contents in the same buffers
            it["s"].copy_(_dev(wl.random_signal(900 + 31 * rep + j, it["s"].numel(), "laplace", 0.1)))
            it["r"].zero_()
        g.launch()
        torch.cuda.synchronize()
        for it in items:
            ref = _single(ctx, it).cpu().numpy()
            got = it["r"].cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-6 * max(1.0, float(np.abs(ref).max())))
    g.close()


def test_batch_rejects_bad_request(ctx):
    items = _mixed_requests(3, 2)
    items[1]["W_block"] = 33  # odd
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv_batch(ctx.make_requests(items))
    assert e.value.status == apx.APX_ERR_WBLOCK
