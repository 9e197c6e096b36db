"""The allocation-free FFT entry point (apx_conv_fft_static) against the
context entry point (apx_conv) on the same inputs.

Callers that may not allocate device memory while running (real-time audio
callbacks, plug-ins whose host application owns the device allocator, code
running while another library holds the memory pool) use this entry point;
its scratch is a fixed device array inside the library.  Outputs of packed
blocks must equal apx_conv's bit for bit (the same integers times the same
FP32 factor); full-precision blocks may differ by rounding, because the two
entry points build their twiddle tables differently.  This file is collected
last so that a failure here comes after every other test has run."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1201_3018_gb300 import apx
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
PACKED = (apx.BLK_SYM, apx.BLK_ASYM2, apx.BLK_ASYM3)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _context_result(sd, kd, Wb, mode, snr):
    """apx_conv's outputs and per-block modes for the same call."""
    ctx = apx.Context(0)
    try:
        r, _, st = ctx.conv(sd, kd, Wb, mode, snr_db=snr, want_stats=True)
        ctx.apx_sync()
        return r.cpu().numpy(), st["mode"].copy()
    finally:
        ctx.close()


def _static(sd, kd, Wb, mode, snr, stream=None):
    out = torch.full((sd.numel() + kd.numel() - 1,), float("nan"), device="cuda")
    apx.apx_conv_fft_static(sd, kd, Wb, mode, snr, out, stream=stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _compare(got, ref, modes, L, N, Wb):
    """Packed blocks bit for bit, full-precision blocks within FP32 rounding,
    every output written."""
    assert np.all(np.isfinite(got)), "outputs left unwritten"
    p = O.plan(L, N, Wb, True)
    packed = np.zeros(len(ref), bool)
    for i in range(p.P):
        if modes[i] in PACKED:
            st0 = O.block_start(p, i)
            lo, hi = O.block_out_range(p, i)
            g = np.arange(st0 + lo, st0 + hi)
            packed[g[(g >= 0) & (g < len(ref))]] = True
    np.testing.assert_array_equal(got[packed], ref[packed])
    full = ~packed
    if full.any() and np.any(ref[full] != 0):
        err = np.linalg.norm(got[full] - ref[full]) / np.linalg.norm(ref[full])
        assert err <= 1e-5, err
    return int(np.isin(modes, PACKED).sum())


@pytest.mark.parametrize("pack", [apx.PACK_AUTO, apx.PACK_SYM, apx.PACK_ASYM2, apx.PACK_ASYM3, apx.PACK_NONE])
@pytest.mark.parametrize("L,N,Wb,op,snr", [(200000, 64, 1024, apx.OP_CONV, 20.0),
                                           (1 << 18, 1024, 4096, apx.OP_XCORR, 45.0),
                                           (30000, 255, 2048, apx.OP_XCORR, 12.0)])
def test_static_entry_matches_context_entry(pack, L, N, Wb, op, snr):
    """Two calls in a row, each against apx_conv with the same arguments."""
    assert torch.cuda.is_available()
    s = wl.random_signal(wl.SEED_BASE + 300 + N, L, "laplace", 0.1)
    k = wl.random_signal(wl.SEED_BASE + 400 + N, N, "uniform")
    sd, kd = _dev(s), _dev(k)
    mode = op | apx.CORE_FFT | pack
    try:
        ref, modes = _context_result(sd, kd, Wb, mode, snr)
    except apx.ApxError as e:  # a forced packing with no admissible range at this N and W_block
        assert e.status == apx.APX_ERR_RANGE
        with pytest.raises(apx.ApxError) as e2:
            _static(sd, kd, Wb, mode, snr)
        assert e2.value.status == apx.APX_ERR_RANGE
        return
    for call in range(2):
        npk = _compare(_static(sd, kd, Wb, mode, snr), ref, modes, L, N, Wb)
        if pack in (apx.PACK_SYM, apx.PACK_ASYM2, apx.PACK_ASYM3) and N <= 255:
            assert npk > 0, "the forced packing should pack some blocks"


def test_static_entry_alternating_wblock():
    """Calls with different W_block one after another on one device: each
    equals apx_conv (the twiddle tables serve every W_block up to the maximum)."""
    L, N, op = 60000, 200, apx.OP_CONV
    s = wl.random_signal(wl.SEED_BASE + 310, L, "laplace", 0.1)
    k = wl.random_signal(wl.SEED_BASE + 311, N, "uniform")
    sd, kd = _dev(s), _dev(k)
    mode = op | apx.CORE_FFT | apx.PACK_AUTO
    refs = {Wb: _context_result(sd, kd, Wb, mode, 15.0) for Wb in (1024, 2048, 4096, 8192)}
    for Wb in (4096, 1024, 4096, 8192, 2048, 1024):
        _compare(_static(sd, kd, Wb, mode, 15.0), refs[Wb][0], refs[Wb][1], L, N, Wb)


def test_static_entry_captured_replay():
    """A static call captured into a CUDA graph, replayed after eager calls with
    other W_block values and with new signal and kernel contents: every replay
    recomputes from the current inputs (packed kernel spectra included)."""
    L, N, Wb, op = 40000, 255, 2048, apx.OP_XCORR
    mode = op | apx.CORE_FFT | apx.PACK_AUTO
    snr = 12.0
    s = _dev(wl.random_signal(wl.SEED_BASE + 320, L, "laplace", 0.1))
    k = _dev(wl.random_signal(wl.SEED_BASE + 321, N, "uniform"))
    out = torch.full((L + N - 1,), float("nan"), device="cuda")
    _static(s, k, 1024, mode, snr)  # the device's first static call comes before any capture
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            apx.apx_conv_fft_static(s, k, Wb, mode, snr, out, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    for rep in range(3):
        if rep:
            s.copy_(_dev(wl.random_signal(wl.SEED_BASE + 322 + rep, L, "laplace", 0.1)))
            k.copy_(_dev(wl.random_signal(wl.SEED_BASE + 332 + rep, N, "uniform")))
        _static(s, k, 4096, mode, snr)  # an eager call with another W_block in between
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        ref, modes = _context_result(s, k, Wb, mode, snr)
        assert _compare(out.cpu().numpy(), ref, modes, L, N, Wb) > 0


def test_static_entry_rejects_oversize_and_other_modes():
    s, k = _dev(np.ones(100000, np.float32)), _dev(np.ones(64, np.float32))
    r = torch.empty(100063, device="cuda")
    with pytest.raises(apx.ApxError) as e:
        apx.apx_conv_fft_static(s, k, 16384, apx.CORE_FFT, 30.0, r)
    assert e.value.status == apx.APX_ERR_WBLOCK
    for mode in (apx.CORE_DIRECT, apx.CORE_FFT | apx.PACK_NONE | apx.FULL_FP64,
                 apx.CORE_FFT | apx.PACK_SYM | apx.LITERAL):
        with pytest.raises(apx.ApxError) as e:
            apx.apx_conv_fft_static(s, k, 1024, mode, 30.0, r)
        assert e.value.status == apx.APX_ERR_ARG
    with pytest.raises(ValueError):  # the binding refuses an output shorter than L+N-1
        apx.apx_conv_fft_static(s, k, 1024, apx.CORE_FFT, 30.0, r[:-1])
