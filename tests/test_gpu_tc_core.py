"""GPU parity of the tensor-core core (APX_CORE_TC) against the oracle: the
direct core's blocks, each block's companded integers (Eq. 2) convolved on
the tensor cores in FP16 with FP32 sums.  Per-block decisions equal the
oracle's exactly; the integers bit for bit; the dequantised outputs within
1e-6 relative (Eq. 16 in FP32); full-precision blocks within 1e-5 relative L2
of Eq. (1) in FP64; every block on the tensor cores at or above the target;
batched calls equal single calls bit for bit."""
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


def _check(ctx, s, k, Wb, mode, snr, s_off=0):
    """Library against the oracle on one call; returns the per-block modes and
    the measured SNR of each tensor-core block."""
    L, N = len(s), len(k)
    buf = _dev(np.concatenate([np.zeros(s_off, np.float32), s]))
    r, rq, st = ctx.conv(buf[s_off:], _dev(k), Wb, mode, snr_db=snr, want_int=True, want_stats=True)
    assert ctx.apx_sync() == 0
    r, rq = r.cpu().numpy(), rq.cpu().numpy().astype(np.int64)
    ro, rqo, so, rc = O.apx_conv(s, k, Wb, mode, snr_db=snr, nthreads=0)
    assert rc == 0
    so = O.stats_arrays(so)
    np.testing.assert_array_equal(st["mode"], so["mode"])
    for f in ("Sq", "Kq", "b"):
        np.testing.assert_array_equal(st[f], so[f])
    np.testing.assert_array_equal(st["cs"].view(np.uint32), so["cs"].astype(np.float32).view(np.uint32))
    np.testing.assert_array_equal(st["maxabs"].view(np.uint32), so["maxabs"].astype(np.float32).view(np.uint32))
    live = (st["mode"] != apx.BLK_ZERO) & (st["mode"] != apx.BLK_NONFINITE)
    np.testing.assert_array_equal(st["sigma2"][live], so["sigma2"][live])
    np.testing.assert_array_equal(rq, rqo)  # the integers, exact
    xcorr = (mode & 0xF) == apx.OP_XCORR
    kk = k[::-1].copy() if xcorr else k
    p = O.plan(L, N, Wb, False)
    snrs = []
    full = []
    for b in range(p.P):
        st0 = O.block_start(p, b)
        lo, hi = O.block_out_range(p, b)
        g = np.arange(st0 + lo, st0 + hi)
        g = g[(g >= 0) & (g < len(r))]
        if st["mode"][b] == apx.BLK_TC:
            np.testing.assert_allclose(r[g], ro[g], rtol=1e-6, atol=0)
            ref = O.conv_ref_at(s, kk, g)
            if np.any(ref):
                snrs.append(10 * np.log10(np.sum(ref ** 2) / np.sum((r[g].astype(np.float64) - ref) ** 2)))
        elif st["mode"][b] == apx.BLK_FULL:
            full.append(g)
    if full:
        g = np.concatenate(full)
        ref = O.conv_ref_at(s, kk, g)
        assert np.linalg.norm(r[g] - ref) <= 1e-5 * max(np.linalg.norm(ref), 1e-300)
    return st["mode"], np.array(snrs)


def test_single_conv_workload(ctx):
    """The single-conv workload (65,536 N(0,1) samples, 64-tap U[-1,1] kernel,
    W_block 1024) at 45 dB: every block on the tensor cores, each at or above
    the target."""
    c = wl.single_conv()
    mode = apx.OP_CONV | apx.CORE_TC | apx.PACK_AUTO
    modes, snrs = _check(ctx, c.s, c.k, c.Wblock, mode, 45.0)
    assert np.all(modes == apx.BLK_TC)
    assert len(snrs) == len(modes) and snrs.min() >= 45.0, snrs.min()


@pytest.mark.parametrize("L,N,Wb,op", [(30000, 64, 1024, apx.OP_CONV), (20000, 255, 2048, apx.OP_XCORR),
                                       (9000, 1, 512, apx.OP_CONV), (50000, 449, 8192, apx.OP_CONV),
                                       (5000, 17, 128, apx.OP_XCORR), (70000, 129, 4096, apx.OP_XCORR),
                                       (777, 64, 1024, apx.OP_CONV)])
@pytest.mark.parametrize("target", [25.0, 45.0, 58.0])
@pytest.mark.parametrize("dist", ["normal", "laplace"])
def test_selection_grid(ctx, L, N, Wb, op, target, dist):
    """Blocks of very different statistics along the signal, so that some run
    on the tensor cores and some in full precision."""
    s = wl.random_signal(L + 11, L, dist, 0.1 if dist == "laplace" else 1.0)
    s = (s * np.linspace(0.05, 3.0, L) ** 3).astype(np.float32)
    k = wl.random_signal(N + 12, N, "uniform")
    modes, snrs = _check(ctx, s, k, Wb, op | apx.CORE_TC | apx.PACK_AUTO, target)
    assert np.all(np.isin(modes, (apx.BLK_TC, apx.BLK_FULL, apx.BLK_ZERO)))
    if len(snrs):
        assert snrs.min() >= target, snrs.min()


def test_special_blocks_and_alignment(ctx):
    """Silent stretches (zero blocks), a non-finite sample (NaN for its blocks,
    APX_ERR_NONFINITE), an input pointer off its 16-byte alignment."""
    L, N, Wb = 40000, 33, 1024
    s = wl.random_signal(21, L, "normal")
    s[5000:12000] = 0.0
    k = wl.random_signal(22, N, "uniform")
    mode = apx.OP_CONV | apx.CORE_TC | apx.PACK_AUTO
    modes, _ = _check(ctx, s, k, Wb, mode, 40.0, s_off=1)
    assert (modes == apx.BLK_ZERO).sum() >= 5 and (modes == apx.BLK_TC).sum() > 10
    s[23456] = np.nan
    r, rq, st = ctx.conv(_dev(s), _dev(k), Wb, mode, snr_db=40.0, want_int=True, want_stats=True)
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_sync()
    assert e.value.status == apx.APX_ERR_NONFINITE
    assert (st["mode"] == apx.BLK_NONFINITE).sum() >= 1 and np.isnan(r.cpu().numpy()).any()


def test_full_precision_twin(ctx):
    """APX_PACK_NONE with the tensor-core core: every block full precision (the
    direct core's FP32 path)."""
    c = wl.single_conv()
    modes, _ = _check(ctx, c.s, c.k, c.Wblock, apx.OP_CONV | apx.CORE_TC | apx.PACK_NONE, 0.0)
    assert np.all(modes == apx.BLK_FULL)


def test_batched_equals_single(ctx):
    """Tensor-core requests in one batched call with direct-core and FFT-core
    requests: each equals its single call bit for bit."""
    items, singles = [], []
    g = np.random.default_rng(9)
    for i in range(10):
        L = int(g.integers(3000, 60000))
        N = int(g.choice([8, 64, 200]))
        core = (apx.CORE_TC, apx.CORE_DIRECT, apx.CORE_FFT)[i % 3]
        Wb = 2048 if core != apx.CORE_FFT else 4096
        s = _dev(wl.random_signal(300 + i, L, "laplace", 0.1))
        k = _dev(wl.random_signal(400 + i, N, "uniform"))
        mode = (i % 2) | core | apx.PACK_AUTO
        items.append(dict(s=s, k=k, r=torch.full((L + N - 1,), float("nan"), device="cuda"), mode=mode,
                          W_block=Wb, snr_db=40.0))
        r1 = torch.empty(L + N - 1, device="cuda")
        ctx.apx_conv(s, k, Wb, mode, 40.0, r1)
        singles.append(r1)
    assert ctx.apx_sync() == 0
    ctx.apx_conv_batch(ctx.make_requests(items))
    assert ctx.apx_sync() == 0
    for it, r1 in zip(items, singles):
        assert torch.equal(it["r"], r1)
