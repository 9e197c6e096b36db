"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer-domain outputs of packed blocks must match bit for bit; the per-block
decisions (mode, S_q, K_q, b, c_s, statistics, FFT error bound) must match
exactly; dequantised outputs within 1e-6 relative (FP32 inverse companding);
full-precision outputs within 1e-5 relative L2 of the FP64 definition."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1201_3018_gb300 import apx
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
PACKED = (apx.BLK_SYM, apx.BLK_ASYM2, apx.BLK_ASYM3)


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = apx.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_both(ctx, s, k, Wb, mode, snr=None, Sq=None, Kq=None, want=None):
    r, rq, st = ctx.conv(dev(s), dev(k), Wb, mode, snr_db=snr, Sq=Sq, Kq=Kq, want_int=True, want_stats=True)
    assert ctx.apx_sync() == 0
    ro, rqo, sto, rc = O.apx_conv(s, k, Wb, mode, snr_db=snr or 0.0, Sq=Sq or 0, Kq=Kq or 0, nthreads=0,
                                  want=want)
    assert rc == 0
    return r.cpu().numpy(), rq.cpu().numpy().astype(np.int64), st, ro, rqo, O.stats_arrays(sto)


def check(r, rq, st, ro, rqo, so, s, k, mode, Wb, want=None):
    # per-block decisions
    np.testing.assert_array_equal(st["mode"], so["mode"])
    for f in ("Sq", "Kq", "b"):
        np.testing.assert_array_equal(st[f], so[f])
    np.testing.assert_array_equal(st["cs"].view(np.uint32), so["cs"].astype(np.float32).view(np.uint32))
    np.testing.assert_array_equal(st["maxabs"].view(np.uint32), so["maxabs"].astype(np.float32).view(np.uint32))
    live = (st["mode"] != apx.BLK_ZERO) & (st["mode"] != apx.BLK_NONFINITE)
    np.testing.assert_array_equal(st["sigma2"][live], so["sigma2"][live])
    np.testing.assert_array_equal(st["fft_err"], so["fft_err"])
    # integer domain: exact everywhere (zero outside packed blocks)
    np.testing.assert_array_equal(rq, rqo)
    # outputs by block kind
    xcorr = (mode & 0xF) == apx.OP_XCORR
    fft = (mode & 0xF0) == apx.CORE_FFT
    p = O.plan(len(s), len(k), Wb, fft)
    packed_mask = np.zeros(len(r), bool)
    full_mask = np.zeros(len(r), bool)
    for i in range(p.P):
        st0 = O.block_start(p, i)
        lo, hi = O.block_out_range(p, i)
        g = np.arange(st0 + lo, st0 + hi)
        g = g[(g >= 0) & (g < len(r))]
        if st["mode"][i] in PACKED:
            packed_mask[g] = True
        elif st["mode"][i] == apx.BLK_FULL:
            full_mask[g] = True
    if want is not None:
        full_mask &= want
    np.testing.assert_allclose(r[packed_mask], ro[packed_mask], rtol=1e-6, atol=0)
    if full_mask.any():
        kk = k[::-1] if xcorr else k
        idx = np.nonzero(full_mask)[0]
        ref = O.conv_ref_at(s, kk, idx)
        err = np.linalg.norm(r[idx] - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err <= 1e-5, err
    return packed_mask, full_mask


SHAPES = [(1000, 64, 256), (513, 8, 64), (5, 3, 16), (3000, 1, 64), (20000, 65, 1024), (40, 29, 32),
          (40000, 257, 2048), (9000, 1024, 4096)]


def q_for(blk, nodd, Q):
    return max(1, min(Q, O.qmax_direct(blk, nodd)))


@pytest.mark.parametrize("core", [apx.CORE_DIRECT, apx.CORE_FFT])
@pytest.mark.parametrize("op", [apx.OP_CONV, apx.OP_XCORR])
@pytest.mark.parametrize("L,N,Wb", SHAPES)
def test_full_precision(ctx, core, op, L, N, Wb):
    s = wl.random_signal(L + 1, L, "normal")
    k = wl.random_signal(N + 2, N, "uniform")
    mode = op | core | apx.PACK_NONE
    check(*run_both(ctx, s, k, Wb, mode), s, k, mode, Wb)


@pytest.mark.parametrize("core", [apx.CORE_DIRECT, apx.CORE_FFT])
@pytest.mark.parametrize("pack,blk,Q", [(apx.PACK_SYM, apx.BLK_SYM, 6), (apx.PACK_ASYM2, apx.BLK_ASYM2, 150),
                                        (apx.PACK_ASYM3, apx.BLK_ASYM3, 6), (apx.PACK_ASYM2, apx.BLK_ASYM2, 10)])
@pytest.mark.parametrize("L,N,Wb", SHAPES)
def test_fixed_packing(ctx, core, pack, blk, Q, L, N, Wb):
    s = wl.random_signal(L + 3, L, "laplace", 0.1)
    k = wl.random_signal(N + 4, N, "uniform")
    nodd = N | 1
    S = q_for(blk, nodd, Q)
    mode = apx.OP_CONV | core | pack
    r, rq, st, ro, rqo, so = run_both(ctx, s, k, Wb, mode, Sq=S, Kq=S)
    pm, fm = check(r, rq, st, ro, rqo, so, s, k, mode, Wb)
    if core == apx.CORE_DIRECT:
        assert np.all((st["mode"] == blk) | (st["mode"] == apx.BLK_ZERO))


@pytest.mark.parametrize("core", [apx.CORE_DIRECT, apx.CORE_FFT])
@pytest.mark.parametrize("target", [12.0, 25.0, 35.0, 45.0, 60.0])
@pytest.mark.parametrize("L,N,Wb,op", [(20000, 65, 1024, apx.OP_CONV), (40000, 257, 2048, apx.OP_XCORR),
                                       (3000, 7, 64, apx.OP_XCORR), (60000, 64, 4096, apx.OP_CONV)])
def test_auto_selection(ctx, core, target, L, N, Wb, op):
    s = wl.random_signal(L + 5, L, "laplace", 0.1)
    # vary the block statistics along the signal so that blocks choose differently
    s = (s * np.linspace(0.2, 3.0, L) ** 2).astype(np.float32)
    k = wl.random_signal(N + 6, N, "uniform")
    mode = op | core | apx.PACK_AUTO
    r, rq, st, ro, rqo, so = run_both(ctx, s, k, Wb, mode, snr=target)
    pm, fm = check(r, rq, st, ro, rqo, so, s, k, mode, Wb)
    packed = np.isin(st["mode"], PACKED)
    p = O.plan(len(s), len(k), Wb, core == apx.CORE_FFT)
    # the model clears the minimum by the Section IV.D margin
    assert np.all(st["snr_pred_db"][packed] >= target + O.snr_margin_db(p.W) - 1e-9)
    if pm.any():
        kk = k[::-1] if op == apx.OP_XCORR else k
        ref_all = O.conv_ref(s, kk.copy())
        idx = np.nonzero(pm)[0]
        ref = ref_all[idx]
        snr_gpu = 10 * math.log10(np.sum(ref ** 2) / np.sum((r[idx] - ref) ** 2))
        snr_or = 10 * math.log10(np.sum(ref ** 2) / np.sum((ro[idx] - ref) ** 2))
        assert abs(snr_gpu - snr_or) < 0.1
        assert snr_gpu >= target
        # and in every packed block (Section IV.D: a lower limit per block)
        for i in np.nonzero(packed)[0]:
            st0 = O.block_start(p, int(i))
            lo, hi = O.block_out_range(p, int(i))
            g = np.arange(st0 + lo, st0 + hi)
            g = g[(g >= 0) & (g < len(r))]
            num, den = np.sum(ref_all[g] ** 2), np.sum((r[g] - ref_all[g]) ** 2)
            if num > 0 and den > 0:
                assert 10 * math.log10(num / den) >= target, (i, st["snr_pred_db"][i])


def test_zero_blocks_and_zero_kernel(ctx):
    s = np.zeros(5000, np.float32)
    s[3000:3100] = wl.random_signal(9, 100, "normal")
    k = wl.random_signal(10, 33, "uniform")
    for core in (apx.CORE_DIRECT, apx.CORE_FFT):
        mode = core | apx.PACK_AUTO
        check(*run_both(ctx, s, k, 256, mode, snr=30.0), s, k, mode, 256)
        r, rq, st, ro, rqo, so = run_both(ctx, s, np.zeros(33, np.float32), 256, mode, snr=30.0)
        assert np.all(r == 0) and np.all(st["mode"] == apx.BLK_ZERO)


def test_nonfinite_input_reported(ctx):
    s = wl.random_signal(11, 4000, "normal")
    s[1234] = np.nan
    k = wl.random_signal(12, 31, "uniform")
    for core in (apx.CORE_DIRECT, apx.CORE_FFT):
        mode = core | apx.PACK_AUTO
        r, rq, st = ctx.conv(dev(s), dev(k), 256, mode, snr_db=30.0, want_int=True, want_stats=True)
        with pytest.raises(apx.ApxError) as e:
            ctx.apx_sync()
        assert e.value.status == apx.APX_ERR_NONFINITE
        ro, rqo, sto, rc = O.apx_conv(s, k, 256, mode, snr_db=30.0)
        np.testing.assert_array_equal(np.isnan(r.cpu().numpy()), np.isnan(ro))
        np.testing.assert_array_equal(st["mode"], O.stats_arrays(sto)["mode"])
        ctx.apx_sync()  # cleared


def test_error_codes(ctx):
    s, k = dev(np.ones(100, np.float32)), dev(np.ones(65, np.float32))
    r = torch.empty(164, device="cuda")
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv_fixed(s, k, 256, apx.PACK_SYM, 100, 100, r)
    assert e.value.status == apx.APX_ERR_RANGE
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv(s, k, 255, 0, 30.0, r)
    assert e.value.status == apx.APX_ERR_WBLOCK
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv(s, k, 96, 0, 30.0, r)  # W = 96 - 65 - 1 = 30 fine; FFT needs a power of two
        ctx.apx_conv(s, k, 96, apx.CORE_FFT, 30.0, r)
    assert e.value.status == apx.APX_ERR_WBLOCK
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv_fixed(s, k, 256, apx.PACK_ASYM2, 0, 5, r)
    assert e.value.status == apx.APX_ERR_ARG


def test_max_wblock(ctx):
    s = wl.random_signal(13, 70000, "laplace", 0.1)
    k = wl.random_signal(14, 8191, "uniform")
    for core, mode_pack in ((apx.CORE_FFT, apx.PACK_AUTO), (apx.CORE_DIRECT, apx.PACK_NONE)):
        mode = apx.OP_XCORR | core | mode_pack
        want = np.zeros(len(s) + len(k) - 1, bool)
        want[np.random.default_rng(0).choice(len(want), 3000, replace=False)] = True
        check(*run_both(ctx, s, k, 16384, mode, snr=20.0, want=want), s, k, mode, 16384, want=want)


@pytest.mark.parametrize("L,N,Wb,target", [(60000, 4096, 8192, 20.0), (50000, 8191, 16384, 12.0),
                                            (40000, 2500, 8192, 30.0)])
def test_direct_core_packs_long_kernels(ctx, L, N, Wb, target):
    """Per-block selection on the direct core with long kernels at large
    W_block: every packing the oracle offers fits one CTA (the taps stream
    through shared memory a chunk at a time), so decisions, integers and
    outputs match the oracle's, and blocks do pack."""
    s = wl.random_signal(L + 51, L, "laplace", 0.1)
    k = wl.random_signal(N + 52, N, "uniform")
    mode = apx.OP_CONV | apx.CORE_DIRECT | apx.PACK_AUTO
    want = np.zeros(L + N - 1, bool)
    want[np.random.default_rng(N).choice(len(want), 3000, replace=False)] = True
    r, rq, st, ro, rqo, so = run_both(ctx, s, k, Wb, mode, snr=target, want=want)
    check(r, rq, st, ro, rqo, so, s, k, mode, Wb, want=want)
    assert np.isin(st["mode"], PACKED).sum() >= 3


def test_host_entry_point_matches_device_path(ctx):
    case = wl.single_conv(L=30000)
    sh = torch.from_numpy(case.s).pin_memory()
    kh = torch.from_numpy(case.k).pin_memory()
    out = torch.empty(len(case.s) + len(case.k) - 1).pin_memory()
    ctx.apx_conv_host(sh, kh, case.Wblock, apx.PACK_ASYM2, Sq=191, Kq=191, r_host=out)
    r, _, _ = ctx.conv(dev(case.s), dev(case.k), case.Wblock, apx.PACK_ASYM2, Sq=191, Kq=191)
    np.testing.assert_array_equal(out.numpy(), r.cpu().numpy())


def test_single_conv_full_size(ctx):
    """65,536-sample N(0,1) input, 64-tap U[-1,1] kernel, W_block 1024, direct
    core: full precision and the fixed ~45 dB quantiser (asym2, S_q=K_q=191)."""
    case = wl.single_conv()
    for mode, Q in ((apx.PACK_NONE, None), (apx.PACK_ASYM2, 191)):
        r, rq, st, ro, rqo, so = run_both(ctx, case.s, case.k, case.Wblock, mode, Sq=Q, Kq=Q)
        check(r, rq, st, ro, rqo, so, case.s, case.k, mode, case.Wblock)
        if Q:
            ref = O.conv_ref(case.s, case.k)
            snr = 10 * math.log10(np.sum(ref ** 2) / np.sum((r - ref) ** 2))
            assert 44.0 < snr < 47.0, snr


def test_matching_xcorr_full_size(ctx):
    """2^20-sample Laplacian signal, 4096-tap template, FFT core W_block 8192,
    per-block selection at 45 dB: decisions exact, sampled outputs."""
    case = wl.matching_xcorr()
    mode = apx.OP_XCORR | apx.CORE_FFT | apx.PACK_AUTO
    want = np.zeros(len(case.s) + len(case.k) - 1, bool)
    want[np.random.default_rng(1).choice(len(want), 4000, replace=False)] = True
    for target in (45.0, 20.0):
        r, rq, st, ro, rqo, so = run_both(ctx, case.s, case.k, case.Wblock, mode, snr=target, want=want)
        check(r, rq, st, ro, rqo, so, case.s, case.k, mode, case.Wblock, want=want)


@pytest.mark.parametrize("op", [apx.OP_CONV, apx.OP_XCORR])
@pytest.mark.parametrize("L,N,Wb", [(1000, 64, 256), (20000, 65, 1024), (5, 3, 16), (9000, 1024, 4096), (3000, 1, 64)])
def test_full_fp64_direct(ctx, op, L, N, Wb):
    """FP64 full-precision twin: Eq. (1) in FP64 rounded once to FP32; against
    the FP64 definition the error is one FP32 rounding plus the FP64
    accumulation error N 2^-52 sum|s||k|."""
    s = wl.random_signal(L + 21, L, "normal")
    k = wl.random_signal(N + 22, N, "uniform")
    r = torch.empty(L + N - 1, device="cuda")
    ctx.apx_conv_full(dev(s), dev(k), Wb, op | apx.CORE_DIRECT | apx.PACK_NONE | apx.FULL_FP64, r)
    assert ctx.apx_sync() == 0
    kk = k[::-1].copy() if op == apx.OP_XCORR else k
    ref = O.conv_ref(s, kk)
    mag = O.conv_ref(np.abs(s), np.abs(kk))
    err = np.abs(r.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= 2.0 ** -24 * np.abs(ref) + N * 2.0 ** -52 * mag + 1e-300)


def test_full_fp64_needs_direct_core_and_no_packing(ctx):
    s, k = dev(np.ones(100, np.float32)), dev(np.ones(5, np.float32))
    r = torch.empty(104, device="cuda")
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv_full(s, k, 64, apx.CORE_FFT | apx.PACK_NONE | apx.FULL_FP64, r)
    assert e.value.status == apx.APX_ERR_ARG
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv(s, k, 64, apx.CORE_DIRECT | apx.PACK_AUTO | apx.FULL_FP64, 30.0, r)
    assert e.value.status == apx.APX_ERR_ARG


def test_bounded_wait_times_out_and_context_recovers(ctx):
    """Failure path without a GPU fault: the blocks that pick a packing wait
    for a packed spectrum nobody publishes, give up after their bounded spin,
    write NaN and report APX_ERR_TIMEOUT; the next call is normal."""
    L, N, Wb = 20000, 65, 1024
    s = wl.random_signal(L + 31, L, "laplace", 0.1)
    k = wl.random_signal(N + 32, N, "uniform")
    mode = apx.CORE_FFT | apx.PACK_AUTO
    sd, kd = dev(s), dev(k)
    ctx.test_stall_next()
    r, rq, st = ctx.conv(sd, kd, Wb, mode, snr_db=12.0, want_int=True, want_stats=True)
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_sync()
    assert e.value.status == apx.APX_ERR_TIMEOUT
    assert np.isnan(r.cpu().numpy()).any()
    r2, rq2, st2, ro, rqo, so = run_both(ctx, s, k, Wb, mode, snr=12.0)
    assert ctx.apx_sync() == 0
    check(r2, rq2, st2, ro, rqo, so, s, k, mode, Wb)


def test_large_input_indices(ctx):
    """2^30 + 12345 samples (4 GB in, 4 GB out): block origins, window loads and
    output offsets beyond 2^31 elements' bytes stay exact; outputs sampled at the
    start, the middle and the end against Eq. (1) in FP64."""
    L, N, Wb = (1 << 30) + 12345, 257, 4096
    g = torch.Generator(device="cuda").manual_seed(7)
    s = torch.randn(L, device="cuda", generator=g)
    k = dev(wl.random_signal(91, N, "uniform"))
    r = torch.empty(L + N - 1, device="cuda")
    ctx.apx_conv_full(s, k, Wb, apx.CORE_FFT | apx.PACK_NONE, r)
    assert ctx.apx_sync() == 0
    idx = np.concatenate([np.arange(0, 300), np.arange(L // 2, L // 2 + 300), np.arange(L + N - 1 - 600, L + N - 1)])
    lo, hi = int(idx.min()), int(idx.max())
    # the samples these outputs touch, gathered on the host
    kh = k.cpu().numpy()
    got = r[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    for part in (idx[:300], idx[300:600], idx[600:]):
        a, b = max(0, int(part.min()) - N + 1), min(L, int(part.max()) + 1)
        seg = s[a:b].cpu().numpy()
        ref = O.conv_ref_at(seg, kh, part - a)
        sel = np.isin(idx, part)
        err = np.linalg.norm(got[sel] - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err <= 1e-5, err
    del s, r
    torch.cuda.empty_cache()


def test_filterbank_large_input(ctx):
    """Filterbank over 2^28 samples (4 kernels, 4 GB of outputs): the first and
    the last block against the oracle."""
    L, F, N = 1 << 28, 4, 64
    g = torch.Generator(device="cuda").manual_seed(8)
    s = torch.randn(L, device="cuda", generator=g)
    kb = np.stack([wl.random_signal(200 + f, N, "uniform") for f in range(F)])
    out_len = L + N - 1
    ldy = (out_len + 3) // 4 * 4
    y = torch.empty(F, ldy, device="cuda")
    T, nb = apx.filterbank_blocks(L, F, N)
    cs = torch.empty(nb, device="cuda")
    ctx.apx_filterbank(s, torch.from_numpy(kb).cuda(), 127, 127, y, None, cs)
    assert ctx.apx_sync() == 0
    csh = cs.cpu().numpy()
    for b in (0, nb - 1):
        shift = b * T
        a1 = min(L, shift + T)
        if b == 0:
            yo, _, cso = O.filterbank(s[:a1].cpu().numpy(), kb, T, 127, 127, blocks=(0, 1))
            ref, c_ref = yo[:, :T], cso[0]
        else:
            # a shifted problem whose block 1 has this block's window: T - N + 1 zeros,
            # then s[bT - N + 1 .. a1)
            x = np.concatenate([np.zeros(T - N + 1, np.float32), s[shift - N + 1:a1].cpu().numpy()])
            yo, _, cso = O.filterbank(x, kb, T, 127, 127, blocks=(1, 2))
            ref, c_ref = yo[:, T:T + min(T, out_len - shift)], cso[1]
        assert c_ref == csh[b]
        got = y[:, shift:shift + ref.shape[1]].cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=0)
    del s, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("core,L,N,Wb,mode_bits,snr", [
    (apx.CORE_FFT, 1 << 20, 4096, 8192, apx.OP_XCORR | apx.PACK_AUTO, 45.0),   # the matching workload
    (apx.CORE_FFT, (1 << 19) + 777, 257, 2048, apx.PACK_AUTO, 20.0),           # packed blocks
    (apx.CORE_DIRECT, (1 << 19) + 3, 65, 1024, apx.PACK_AUTO, 45.0),
    (apx.CORE_DIRECT, 1 << 18, 64, 1024, apx.PACK_NONE | apx.FULL_FP64, 0.0),
])
def test_host_entry_equals_device_path_large(ctx, core, L, N, Wb, mode_bits, snr):
    """apx_conv_host equals the device-buffer call bit for bit, on calls with
    different inputs: page-locked buffers (the kernels read and write them in
    place) and pageable ones (staged through device buffers, the signal copied
    on a second stream while the kernel is prepared)."""
    for rep in range(3):
        s = wl.random_signal(L + 41 + rep, L, "laplace", 0.1)
        k = wl.random_signal(N + 42, N, "uniform")
        mode = core | mode_bits
        pinned = rep != 1
        sh, kh = torch.from_numpy(s), torch.from_numpy(k)
        out = torch.full((L + N - 1,), float("nan"))
        if pinned:
            sh, kh, out = sh.pin_memory(), kh.pin_memory(), out.pin_memory()
        ctx.apx_conv_host(sh, kh, Wb, mode, snr, 0, 0, out)
        r = torch.empty(L + N - 1, device="cuda")
        if (mode & 0xF00) == apx.PACK_NONE:
            ctx.apx_conv_full(dev(s), dev(k), Wb, mode, r)
        else:
            ctx.apx_conv(dev(s), dev(k), Wb, mode, snr, r)
        assert ctx.apx_sync() == 0
        np.testing.assert_array_equal(out.numpy(), r.cpu().numpy())


@pytest.mark.parametrize("L,N,Q,Wb,op,dist", [
    (20000, 65, 8, 1024, apx.OP_CONV, "uniform"),        # small range: the exact form's digits
    (1 << 16, 800, 16, 8192, apx.OP_CONV, "u128"),       # Section IV.A's symmetric setting, beyond the exact bound
    (30000, 257, 16, 2048, apx.OP_XCORR, "laplace"),
    (30000, 2500, 8, 8192, apx.OP_CONV, "laplace"),     # packed taps in two shared-memory chunks
])
def test_paper_literal_form_matches_oracle(ctx, L, N, Q, Wb, op, dist):
    """APX_LITERAL (Eq. 6 eps, FP64 Eqs. 11-15 with u_sys, packed convolution
    without fused multiply-adds) on the direct core: the same integers as the
    oracle's literal form, bit for bit, digits moved by rounding included."""
    g = np.random.default_rng(L + N + Q)
    if dist == "u128":
        s, k = g.uniform(-128, 128, L).astype(np.float32), g.uniform(-128, 128, N).astype(np.float32)
    else:
        s, k = wl.random_signal(L + 5, L, dist, 0.1), wl.random_signal(N + 6, N, "uniform")
    mode = op | apx.CORE_DIRECT | apx.PACK_SYM | apx.LITERAL
    check(*run_both(ctx, s, k, Wb, mode, Sq=Q, Kq=Q), s, k, mode, Wb)


def test_paper_literal_form_rejections(ctx):
    s, k = dev(np.ones(5000, np.float32)), dev(np.ones(65, np.float32))
    for mode in (apx.CORE_FFT | apx.PACK_SYM | apx.LITERAL, apx.CORE_DIRECT | apx.PACK_ASYM2 | apx.LITERAL,
                 apx.CORE_DIRECT | apx.PACK_AUTO | apx.LITERAL):
        with pytest.raises(apx.ApxError) as e:
            ctx.conv(s, k, 1024, mode, Sq=8, Kq=8)
        assert e.value.status == apx.APX_ERR_ARG
    with pytest.raises(apx.ApxError) as e:  # R_max = 65 * 2^20 * 2^20 > 2^31
        ctx.conv(s, k, 1024, apx.CORE_DIRECT | apx.PACK_SYM | apx.LITERAL, Sq=1 << 20, Kq=1 << 20)
    assert e.value.status == apx.APX_ERR_RANGE


def test_paper_literal_form_not_batched(ctx):
    s, k = dev(np.ones(5000, np.float32)), dev(np.ones(65, np.float32))
    r = torch.empty(5064, device="cuda")
    reqs = ctx.make_requests([dict(s=s, k=k, r=r, mode=apx.CORE_DIRECT | apx.PACK_SYM | apx.LITERAL, W_block=1024,
                                   Sq=8, Kq=8)])
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_conv_batch(reqs)
    assert e.value.status == apx.APX_ERR_ARG


@pytest.mark.parametrize("core,Wb", [(apx.CORE_FFT, 2048), (apx.CORE_FFT, 8192)])
def test_target_just_below_the_best_case_model_snr(ctx, core, Wb):
    """Blocks of constant magnitude (every sample +-1: sigma^2 = ||s||_inf^2,
    the window for which the Section IV.D model is largest) with the target a
    hair below the best-case model SNR of the first candidate: those blocks
    pass its model check, so its exact norm must be there for the FFT error
    bound, which then rejects it (the block is at full scale); per-block
    decisions, bounds and integers as the oracle's."""
    g = np.random.default_rng(Wb)
    N = 255
    k = g.uniform(-1, 1, N).astype(np.float32)
    s = np.where(g.random(60000) < 0.5, -1.0, 1.0).astype(np.float32)
    Mk, s2k = O.maxabs(k), O.second_moment(k)
    Q = O.qmax_fft(O.BLK_SYM, N, Wb)
    assert Q >= 1
    # the model must clear the target by the Section IV.D margin
    best_db = O.snr_model_db(1.0, 1.0, s2k, Mk, Q, Q) - O.snr_margin_db(Wb - N - 1)
    for target in (best_db - 0.02, best_db - 0.001):
        mode = apx.OP_CONV | core | apx.PACK_AUTO
        check(*run_both(ctx, s, k, Wb, mode, snr=target), s, k, mode, Wb)


@pytest.mark.parametrize("core,Wb", [(apx.CORE_DIRECT, 1024), (apx.CORE_FFT, 2048)])
def test_candidates_at_the_model_maximum(ctx, core, Wb):
    """Signal and kernel of +-1 values: both ratios sigma^2 / ||.||_inf^2 are 1,
    where the Section IV.D model is largest, so a candidate is unreachable for
    every block exactly when the target exceeds its model there -- the rule by
    which the plan leaves candidates out.  Targets a hair below, a hair above
    and well above each candidate's maximum: per-block decisions, integers and
    outputs as the oracle's, which evaluates every candidate."""
    g = np.random.default_rng(Wb + 7)
    N = 65
    k = np.where(g.random(N) < 0.5, -1.0, 1.0).astype(np.float32)
    s = np.where(g.random(40000) < 0.5, -1.0, 1.0).astype(np.float32)
    qfun = O.qmax_fft if core == apx.CORE_FFT else (lambda blk, n, w: O.qmax_direct(blk, n))
    tops = set()
    for blk in (O.BLK_SYM, O.BLK_ASYM3, O.BLK_ASYM2):
        Q = qfun(blk, N, Wb)
        if Q >= 1:
            # the highest target the candidate can serve: its model maximum less the margin
            tops.add(round(O.snr_model_db(1.0, 1.0, 1.0, 1.0, Q, Q) - O.snr_margin_db(Wb - N - 1), 6))
    assert tops
    mode = apx.OP_CONV | core | apx.PACK_AUTO
    for top in sorted(tops):
        for target in (top - 0.001, top + 0.001, top + 1.0):
            check(*run_both(ctx, s, k, Wb, mode, snr=target), s, k, mode, Wb)
