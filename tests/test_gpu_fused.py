"""The FFT core's one-launch form (a single call with at least 64 blocks: the
kernel preparation runs in ticketed CTAs of the block kernel's own launch)
against its three-launch form (preparation launches ahead of the block
kernel, which batched calls always use): the same bits, one launch instead of
three, and the ticket counter staying in step across interleaved calls."""
import numpy as np
import pytest
import torch

from paper_1201_3018_gb300 import apx
import oracle as O
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FUSE_MIN_BLOCKS = 64  # the library's threshold for the one-launch form


@pytest.fixture(scope="module")
def ctx():
    c = apx.Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _length_for_blocks(P, N, Wb, mode):
    """Smallest L whose block plan has exactly P blocks."""
    lo, hi = 1, 1 << 26
    while lo < hi:
        mid = (lo + hi) // 2
        if apx.plan_blocks(mid, N, Wb, mode)[0] >= P:
            hi = mid
        else:
            lo = mid + 1
    assert apx.plan_blocks(lo, N, Wb, mode)[0] == P
    return lo


def _launches(L, N, Wb, mode, snr, P):
    """Launches of a single call: one when it runs its kernel preparation in
    the block kernel's own launch (at least FUSE_MIN_BLOCKS blocks and some
    packing candidate left), else three; a call without any candidate runs the
    two-CTA full-precision kernel after the two preparation launches."""
    full_only = Wb >= 1024 and not apx.plan_candidates(L, N, Wb, mode, snr)
    return 3 if (full_only or P < FUSE_MIN_BLOCKS) else 1


def _single(ctx, s, k, Wb, mode, snr):
    r = torch.empty(s.numel() + k.numel() - 1, device="cuda")
    n0 = ctx.launch_count()
    if (mode & 0xF00) == apx.PACK_NONE:
        ctx.apx_conv_full(s, k, Wb, mode, r)
    else:
        ctx.apx_conv(s, k, Wb, mode, snr, r)
    assert ctx.apx_sync() == 0
    return r.cpu().numpy(), ctx.launch_count() - n0


def _batch_of_one(ctx, s, k, Wb, mode, snr):
    r = torch.empty(s.numel() + k.numel() - 1, device="cuda")
    ctx.apx_conv_batch(ctx.make_requests([dict(s=s, k=k, r=r, mode=mode, W_block=Wb, snr_db=snr)]))
    assert ctx.apx_sync() == 0
    return r.cpu().numpy()


CASES = [
    # (blocks, N, W_block, op | pack, target dB)
    (FUSE_MIN_BLOCKS - 1, 1024, 4096, apx.OP_XCORR | apx.PACK_AUTO, 45.0),
    (FUSE_MIN_BLOCKS, 1024, 4096, apx.OP_XCORR | apx.PACK_AUTO, 45.0),
    (300, 4096, 8192, apx.OP_XCORR | apx.PACK_AUTO, 45.0),
    (300, 4096, 8192, apx.OP_CONV | apx.PACK_NONE, 0.0),
    (200, 255, 2048, apx.OP_CONV | apx.PACK_AUTO, 12.0),     # blocks pick packings
    (100, 65, 1024, apx.OP_CONV | apx.PACK_ASYM2, 0.0),
    (80, 3000, 16384, apx.OP_XCORR | apx.PACK_AUTO, 30.0),
]


@pytest.mark.parametrize("P,N,Wb,bits,snr", CASES)
def test_one_launch_equals_three_launch_form(ctx, P, N, Wb, bits, snr):
    mode = bits | apx.CORE_FFT
    L = _length_for_blocks(P, N, Wb, mode)
    s = _dev(wl.random_signal(wl.SEED_BASE + 900 + P, L, "laplace", 0.1))
    k = _dev(wl.random_signal(wl.SEED_BASE + 950 + N, N, "uniform"))
    got, launches = _single(ctx, s, k, Wb, mode, snr)
    assert launches == _launches(L, N, Wb, mode, snr, P)
    ref = _batch_of_one(ctx, s, k, Wb, mode, snr)
    assert np.array_equal(got, ref)
    # and sampled outputs against Eq. (1) in FP64 (full precision blocks within FP32 rounding;
    # packed ones within the target)
    sh, kh = s.cpu().numpy(), k.cpu().numpy()
    if bits & 0xF == apx.OP_XCORR:
        kh = kh[::-1].copy()
    idx = np.linspace(0, L + N - 2, 400).astype(np.int64)
    exact = O.conv_ref_at(sh, kh, idx)
    err = np.linalg.norm(got[idx] - exact) / np.linalg.norm(exact)
    bound = 1e-5 if (bits & 0xF00) == apx.PACK_NONE else 10 ** (-max(snr, 12.0) / 20) * 3
    assert err <= bound, err


def test_tickets_stay_in_step_across_interleaved_calls(ctx):
    """One-launch calls between three-launch calls (the two-CTA kernel among
    them), batched calls and one-launch calls of another W_block: every repeat
    gives the first result's bits."""
    N, Wb, mode, snr = 1024, 4096, apx.OP_XCORR | apx.CORE_FFT | apx.PACK_AUTO, 30.0
    assert apx.plan_candidates(1 << 20, N, Wb, mode, snr) and apx.plan_candidates(1 << 20, N, 8192, mode, snr)
    L = _length_for_blocks(150, N, Wb, mode)
    s = _dev(wl.random_signal(wl.SEED_BASE + 990, L, "laplace", 0.1))
    k = _dev(wl.random_signal(wl.SEED_BASE + 991, N, "uniform"))
    small_s = _dev(wl.random_signal(wl.SEED_BASE + 992, 20000, "laplace", 0.1))
    small_k = _dev(wl.random_signal(wl.SEED_BASE + 993, 300, "uniform"))
    first, n = _single(ctx, s, k, Wb, mode, snr)
    assert n == 1
    for rep in range(4):
        _single(ctx, small_s, small_k, 2048, apx.OP_CONV | apx.CORE_FFT | apx.PACK_AUTO, 30.0)
        _batch_of_one(ctx, small_s, small_k, 4096, apx.OP_CONV | apx.CORE_FFT | apx.PACK_NONE, 0.0)
        _single(ctx, s, k, 4096, apx.OP_XCORR | apx.CORE_FFT | apx.PACK_NONE, 0.0)  # the two-CTA kernel
        _single(ctx, s, k, 8192, mode, snr)  # another W_block, also one launch
        again, n = _single(ctx, s, k, Wb, mode, snr)
        assert n == 1
        assert np.array_equal(again, first), rep


def test_captured_call_replays(ctx):
    """A single call captured into a CUDA graph (stream capture) takes the
    three-launch form, whose launches replay: each replay recomputes from the
    signal's current contents."""
    N, Wb, mode = 4096, 8192, apx.OP_XCORR | apx.CORE_FFT | apx.PACK_AUTO
    L = _length_for_blocks(150, N, Wb, mode)
    s = _dev(wl.random_signal(wl.SEED_BASE + 994, L, "laplace", 0.1))
    k = _dev(wl.random_signal(wl.SEED_BASE + 995, N, "uniform"))
    r = torch.empty(L + N - 1, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.apx_conv(s, k, Wb, mode, 45.0, r, stream=side)  # workspace allocated before capture
        side.synchronize()
        g = torch.cuda.CUDAGraph()
        n0 = ctx.launch_count()
        with torch.cuda.graph(g, stream=side):
            ctx.apx_conv(s, k, Wb, mode, 45.0, r, stream=side)
        assert ctx.launch_count() - n0 == 3
    torch.cuda.current_stream().wait_stream(side)
    for rep in range(2):
        s.copy_(_dev(wl.random_signal(wl.SEED_BASE + 996 + rep, L, "laplace", 0.1)))
        g.replay()
        torch.cuda.synchronize()
        got = r.cpu().numpy()
        want, n = _single(ctx, s, k, Wb, mode, 45.0)
        assert n == _launches(L, N, Wb, mode, 45.0, 150)
        assert np.array_equal(got, want), rep


def test_captured_packed_call_replays_with_new_kernel(ctx):
    """A captured single call whose blocks pack: its packed kernel spectra are
    built anew on every replay (the replays share the capture's call number),
    so replays after the template's taps change equal fresh calls."""
    N, Wb, mode = 255, 2048, apx.OP_XCORR | apx.CORE_FFT | apx.PACK_AUTO
    L = _length_for_blocks(40, N, Wb, mode)
    s = _dev(wl.random_signal(wl.SEED_BASE + 981, L, "laplace", 0.1))
    k = _dev(wl.random_signal(wl.SEED_BASE + 982, N, "uniform"))
    r = torch.empty(L + N - 1, device="cuda")
    st = torch.empty(apx.plan_blocks(L, N, Wb, mode)[0] * apx.STATS_DTYPE.itemsize, dtype=torch.uint8,
                     device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.apx_conv(s, k, Wb, mode, 12.0, r, stream=side)  # workspace allocated before capture
        side.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            ctx.apx_conv(s, k, Wb, mode, 12.0, r, None, st, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    for rep in range(3):
        k.copy_(_dev(wl.random_signal(wl.SEED_BASE + 983 + rep, N, "uniform")))
        if rep == 2:
            s.copy_(_dev(wl.random_signal(wl.SEED_BASE + 990, L, "laplace", 0.1)))
        g.replay()
        torch.cuda.synchronize()
        got = r.cpu().numpy()
        modes = np.frombuffer(st.cpu().numpy().tobytes(), dtype=apx.STATS_DTYPE)["mode"]
        assert np.isin(modes, (apx.BLK_SYM, apx.BLK_ASYM2, apx.BLK_ASYM3)).any()
        want, _ = _single(ctx, s, k, Wb, mode, 12.0)
        assert np.array_equal(got, want), rep


def test_ticket_fault_is_reported_and_recovered(ctx):
    """A ticket count out of step (host-injected): every CTA of the next
    one-launch call finds its ticket out of range and touches nothing,
    apx_sync reports APX_ERR_CHECK and resynchronises, and the following call
    is correct."""
    N, Wb, mode = 1024, 4096, apx.OP_CONV | apx.CORE_FFT | apx.PACK_AUTO
    L = _length_for_blocks(100, N, Wb, mode)
    s = _dev(wl.random_signal(wl.SEED_BASE + 997, L, "laplace", 0.1))
    k = _dev(wl.random_signal(wl.SEED_BASE + 998, N, "uniform"))
    want, _ = _single(ctx, s, k, Wb, mode, 30.0)
    for skew in (1 << 20, -(1 << 20)):  # every ticket below 0 or past the grid
        ctx.test_skew_tickets(skew)
        r = torch.full((L + N - 1,), float("nan"), device="cuda")
        ctx.apx_conv(s, k, Wb, mode, 30.0, r)
        with pytest.raises(apx.ApxError) as e:
            ctx.apx_sync()
        assert e.value.status == apx.APX_ERR_CHECK
        assert torch.isnan(r).all()
        again, n = _single(ctx, s, k, Wb, mode, 30.0)
        assert n == 1
        assert np.array_equal(again, want)
