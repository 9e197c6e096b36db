"""Prepared kernels (apx_kernel_create / apx_conv_prepared): the kernel's
statistics and spectra computed once and kept resident give the same bits as
preparing them in every call, for any number of calls and signals."""
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


CASES = [
    # L, N, W_block, op | pack, target (dB): blocks full precision, blocks packed, the full-precision twin
    (1 << 20, 4096, 8192, apx.OP_XCORR | apx.PACK_AUTO, 45.0),
    (300000, 255, 2048, apx.OP_CONV | apx.PACK_AUTO, 12.0),
    (200000, 1000, 4096, apx.OP_CONV | apx.PACK_NONE, 0.0),
]


@pytest.mark.parametrize("L,N,Wb,bits,snr", CASES)
def test_prepared_kernel_equals_per_call_preparation(ctx, L, N, Wb, bits, snr):
    mode = bits | apx.CORE_FFT
    k = _dev(wl.random_signal(wl.SEED_BASE + 610 + N, N, "uniform"))
    kp = ctx.prepare_kernel(k, Wb, mode)
    k_saved = k.clone()
    k.fill_(float("nan"))  # the handle keeps its own copy of the taps
    try:
        for rep in range(3):  # packed spectra built by the first call, reused by the next ones
            s = _dev(wl.random_signal(wl.SEED_BASE + 620 + rep, L, "laplace", 0.1))
            got = torch.empty(L + N - 1, device="cuda")
            rq = torch.empty(L + N - 1, dtype=torch.int32, device="cuda")
            n0 = ctx.launch_count()
            ctx.apx_conv_prepared(kp, s, snr, got, rq)
            assert ctx.launch_count() - n0 == 1
            assert ctx.apx_sync() == 0
            ref, rq_ref, _ = ctx.conv(s, k_saved, Wb, mode, snr_db=snr, want_int=(bits & 0xF00) != apx.PACK_NONE)
            assert ctx.apx_sync() == 0
            assert torch.equal(got, ref), rep
            if rq_ref is not None:
                assert torch.equal(rq, rq_ref), rep
    finally:
        kp.close()


def test_prepared_kernel_targets_and_rejections(ctx):
    """One handle serves calls with different targets; other cores and fixed
    packings are rejected."""
    N, Wb, L = 255, 2048, 100000
    k = _dev(wl.random_signal(wl.SEED_BASE + 630, N, "uniform"))
    s = _dev(wl.random_signal(wl.SEED_BASE + 631, L, "laplace", 0.1))
    mode = apx.OP_CONV | apx.CORE_FFT | apx.PACK_AUTO
    kp = ctx.prepare_kernel(k, Wb, mode)
    try:
        for snr in (12.0, 45.0, 20.0):
            got = torch.empty(L + N - 1, device="cuda")
            ctx.apx_conv_prepared(kp, s, snr, got)
            ref, _, _ = ctx.conv(s, k, Wb, mode, snr_db=snr)
            assert ctx.apx_sync() == 0
            assert torch.equal(got, ref), snr
    finally:
        kp.close()
    for bad in (apx.CORE_DIRECT | apx.PACK_AUTO, apx.CORE_FFT | apx.PACK_ASYM2, apx.CORE_FFT | apx.PACK_SYM):
        with pytest.raises(apx.ApxError) as e:
            ctx.prepare_kernel(k, Wb, bad)
        assert e.value.status == apx.APX_ERR_ARG


@pytest.mark.parametrize("taps", ["nan", "zero", "one"])
def test_prepared_kernel_degenerate_kernels(ctx, taps):
    """A non-finite, an all-zero and a one-tap kernel: the prepared call gives
    what the per-call preparation gives, status included."""
    N = 1 if taps == "one" else 300
    k = _dev(wl.random_signal(wl.SEED_BASE + 640, N, "uniform"))
    if taps == "nan":
        k[N // 2] = float("nan")
    elif taps == "zero":
        k.zero_()
    s = _dev(wl.random_signal(wl.SEED_BASE + 641, 150000, "laplace", 0.1))
    mode = apx.OP_XCORR | apx.CORE_FFT | apx.PACK_AUTO
    Wb = 1024
    status = []
    outs = []
    kp = ctx.prepare_kernel(k, Wb, mode)
    try:
        for prepared in (True, False):
            r = torch.empty(s.numel() + N - 1, device="cuda")
            if prepared:
                ctx.apx_conv_prepared(kp, s, 30.0, r)
            else:
                ctx.apx_conv(s, k, Wb, mode, 30.0, r)
            try:
                status.append(ctx.apx_sync())
            except apx.ApxError as e:
                status.append(e.status)
            outs.append(r.cpu().numpy())
    finally:
        kp.close()
    assert status[0] == status[1]
    assert np.array_equal(outs[0], outs[1], equal_nan=True)
    if taps == "nan":
        assert status[0] == apx.APX_ERR_NONFINITE and np.isnan(outs[0]).all()
    if taps == "zero":
        assert status[0] == apx.APX_OK and not outs[0].any()


@pytest.mark.parametrize("L", [1, 100, 5000, 65537])
def test_prepared_kernel_short_signals(ctx, L):
    """Signals shorter than the kernel and than one block (the FFT core's head
    blocks and partial last blocks) through a prepared kernel."""
    N, Wb = 4096, 16384
    mode = apx.OP_XCORR | apx.CORE_FFT | apx.PACK_AUTO
    k = _dev(wl.random_signal(wl.SEED_BASE + 650, N, "uniform"))
    kp = ctx.prepare_kernel(k, Wb, mode)
    try:
        s = _dev(wl.random_signal(wl.SEED_BASE + 651 + L, L, "laplace", 0.1))
        got = torch.empty(L + N - 1, device="cuda")
        ctx.apx_conv_prepared(kp, s, 30.0, got)
        ref, _, _ = ctx.conv(s, k, Wb, mode, snr_db=30.0)
        assert ctx.apx_sync() == 0
        assert torch.equal(got, ref)
    finally:
        kp.close()
