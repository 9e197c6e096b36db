"""The allocation-free FFT entry point (apx_conv_fft_static) against the
context entry point (apx_conv) on the same inputs, on two calls in a row.

Callers that may not allocate device memory while running (real-time audio
callbacks, plug-ins whose host owns the device allocator) use this entry
point; its scratch is a fixed device array inside the library.  This file is
collected last so that a failure here comes after every other test has run."""
import numpy as np
import pytest
import torch

from paper_1201_3018_gb300 import apx
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("L,N,Wb,op,snr", [(200000, 64, 1024, apx.OP_CONV, 20.0),
                                           (1 << 18, 1024, 4096, apx.OP_XCORR, 45.0),
                                           (30000, 255, 2048, apx.OP_XCORR, 12.0)])
def test_static_entry_matches_context_entry(L, N, Wb, op, snr):
    assert torch.cuda.is_available()
    s = wl.random_signal(wl.SEED_BASE + 300 + N, L, "laplace", 0.1)
    k = wl.random_signal(wl.SEED_BASE + 400 + N, N, "uniform")
    sd, kd = _dev(s), _dev(k)
    mode = op | apx.CORE_FFT | apx.PACK_AUTO
    ctx = apx.Context(0)
    ref = torch.empty(L + N - 1, device="cuda")
    ctx.apx_conv(sd, kd, Wb, mode, snr, ref)
    ctx.apx_sync()
    ref = ref.cpu().numpy()
    ctx.close()
    for call in range(2):
        out = torch.full((L + N - 1,), float("nan"), device="cuda")
        apx.apx_conv_fft_static(sd, kd, Wb, mode, snr, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), "call %d left outputs unwritten" % call
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (call, err)


def test_static_entry_rejects_oversize_and_direct_core():
    s, k = _dev(np.ones(100000, np.float32)), _dev(np.ones(64, np.float32))
    r = torch.empty(100063, device="cuda")
    with pytest.raises(apx.ApxError) as e:
        apx.apx_conv_fft_static(s, k, 16384, apx.CORE_FFT, 30.0, r)
    assert e.value.status == apx.APX_ERR_WBLOCK
    with pytest.raises(apx.ApxError) as e:
        apx.apx_conv_fft_static(s, k, 1024, apx.CORE_DIRECT, 30.0, r)
    assert e.value.status == apx.APX_ERR_ARG
