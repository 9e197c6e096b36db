"""Eq. (17) stores at every output alignment: the epilogues write 16 bytes at
a time between the 16-byte boundaries of r and single outputs at the ragged
ends, and the direct cores' windows load 16 bytes at a time where the signal
allows it.  Outputs (and integers) written through r and rq offset by 0-3
elements, from inputs offset by 0-3 elements, must equal the aligned call's
bit for bit, with nothing written outside [r, r + L + N - 1)."""
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


CASES = [
    (apx.CORE_DIRECT | apx.PACK_AUTO, 20000, 64, 1024, 45.0),   # packed FP64 (asymmetric) blocks
    (apx.CORE_DIRECT | apx.PACK_NONE, 20000, 65, 1024, 0.0),    # FP32 full precision
    (apx.CORE_TC | apx.PACK_AUTO, 20000, 64, 1024, 45.0),       # tensor-core blocks
    (apx.CORE_FFT | apx.PACK_AUTO, 50000, 255, 2048, 20.0),     # FFT core, packed and full blocks
    (apx.CORE_FFT | apx.PACK_NONE, 50000, 4096, 8192, 0.0),     # the two-CTA full-precision kernel
]


@pytest.mark.parametrize("mode,L,N,Wb,snr", CASES)
def test_offsets_equal_aligned(ctx, mode, L, N, Wb, snr):
    s = wl.random_signal(71, L, "laplace", 0.1)
    s = (s * np.linspace(0.1, 2.0, L) ** 2).astype(np.float32)
    k = wl.random_signal(72, N, "uniform")
    out = L + N - 1
    base_s = torch.from_numpy(np.concatenate([np.zeros(4, np.float32), s, np.zeros(4, np.float32)])).cuda()
    kd = torch.from_numpy(k).cuda()
    want_int = (mode & 0xF00) != apx.PACK_NONE
    ref = None
    for so in range(4):
        for ro in range(4):
            r = torch.full((out + 8,), float("nan"), device="cuda")
            rq = torch.full((out + 8,), -7, dtype=torch.int32, device="cuda") if want_int else None
            sv = base_s[so:so + L]
            sv.copy_(torch.from_numpy(s).cuda())
            ctx.apx_conv(sv, kd, Wb, mode, snr, r[ro:ro + out], rq[ro:ro + out] if want_int else None)
            assert ctx.apx_sync() == 0
            got = r.cpu().numpy()
            gotq = rq.cpu().numpy() if want_int else None
            # nothing outside the output range
            assert np.isnan(got[:ro]).all() and np.isnan(got[ro + out:]).all()
            if want_int:
                assert (gotq[:ro] == -7).all() and (gotq[ro + out:] == -7).all()
            cur = (got[ro:ro + out].copy(), gotq[ro:ro + out].copy() if want_int else None)
            if ref is None:
                ref = cur
                assert np.isfinite(ref[0]).all()
                continue
            assert np.array_equal(cur[0].view(np.uint32), ref[0].view(np.uint32)), (so, ro)
            if want_int:
                assert np.array_equal(cur[1], ref[1]), (so, ro)
