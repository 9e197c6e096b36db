"""Section IV.D decisions at the threshold: the kernels screen the Table 1
model in FP32 and evaluate it in FP64 only when the FP32 comparison is within
its rounding margin of the threshold.  Here each target is set so that one
block's model SNR lies on the threshold to within FP64 rounding, which the
screen must leave to the FP64 comparison; every block's decision, and every
packed block's integers, must then equal the oracle's exactly."""
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


def _signal(seed, L):
    s = wl.random_signal(seed, L, "laplace", 0.1)
    return (s * np.linspace(0.05, 3.0, L) ** 3).astype(np.float32)  # blocks of very different statistics


@pytest.mark.parametrize("core,L,N,Wb,base", [(apx.CORE_DIRECT, 30000, 64, 1024, 30.0),
                                              (apx.CORE_TC, 30000, 64, 1024, 30.0),
                                              (apx.CORE_FFT, 60000, 255, 2048, 20.0)])
def test_decisions_on_the_threshold(ctx, core, L, N, Wb, base):
    s = _signal(31, L)
    k = wl.random_signal(32, N, "uniform")
    mode = apx.OP_CONV | core | apx.PACK_AUTO
    _, _, st0, rc = O.apx_conv(s, k, Wb, mode, snr_db=base, nthreads=0)
    assert rc == 0
    st0 = O.stats_arrays(st0)
    packed = np.flatnonzero(np.isfinite(st0["snr_pred_db"]) & (st0["mode"] != apx.BLK_FULL))
    assert len(packed) >= 3
    W = O.plan(L, N, Wb, core == apx.CORE_FFT).W
    margin = O.snr_margin_db(W)
    checked = 0
    for b in packed[:: max(1, len(packed) // 4)][:4]:
        for eps in (-1e-12, 0.0, 1e-12):
            target = float(st0["snr_pred_db"][b]) - margin + eps
            r, rq, st = ctx.conv(_dev(s), _dev(k), Wb, mode, snr_db=target, want_int=True, want_stats=True)
            assert ctx.apx_sync() == 0
            ro, rqo, sto, rc = O.apx_conv(s, k, Wb, mode, snr_db=target, nthreads=0)
            assert rc == 0
            sto = O.stats_arrays(sto)
            np.testing.assert_array_equal(st["mode"], sto["mode"])
            np.testing.assert_array_equal(st["Sq"], sto["Sq"])
            np.testing.assert_array_equal(rq.cpu().numpy().astype(np.int64), rqo)
            checked += 1
    assert checked >= 9
