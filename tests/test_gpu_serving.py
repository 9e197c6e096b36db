"""Serving loop on the GPU: every request of a Poisson trace completes, the
admission budget holds, batches overlap on the device, and each result is the
same bit for bit as the same request run alone (a batch of one on a fresh
context), whatever shared its batch and whatever ran beside it."""
import numpy as np
import pytest
import torch

from paper_1201_3018_gb300 import apx, serve
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _alone(ctx, q, s_host, k_host):
    s = s_host[q.s_off:q.s_off + q.L].cuda()
    k = k_host[q.k_id, :q.N].cuda()
    r = torch.full((q.L + q.N - 1,), float("nan"), device="cuda")
    ctx.apx_conv_batch(ctx.make_requests([dict(s=s, k=k, r=r, mode=q.mode, W_block=q.W_block, snr_db=q.target)]))
    torch.cuda.synchronize()
    return r.cpu()


@pytest.mark.parametrize("budget_mb,streams", [(48, 4), (40 << 10, 3)])
def test_serving_same_alone_and_in_mix(budget_mb, streams):
    seed = wl.SEED_BASE + 41
    pool = 1 << 20
    s_host, k_host = serve.host_pools(seed, pool=pool, ntemplates=8)
    trace = serve.make_trace(seed, rate_hz=2000.0, duration_s=0.12, pool=pool, ntemplates=8, lmax_log2=20.0)
    budget = budget_mb << 20
    srv = serve.Server(0, budget_bytes=budget, streams=streams, max_batch=16)
    try:
        kept = {}
        done = srv.run(trace, s_host, k_host, realtime=True, on_done=lambda q: kept.__setitem__(q.rid, q.out.clone()))
    finally:
        srv.close()
    assert sorted(q.rid for q in done) == list(range(len(trace)))
    biggest = max(serve.device_bytes(q) for q in trace)
    assert srv.peak_in_flight <= max(budget, biggest)
    assert srv.batches >= 2
    p50, p99 = serve.latency_ms(done)
    assert 0 < p50 <= p99
    ctx = apx.Context(0)
    try:
        assert sorted(kept) == list(range(len(trace)))
        for q in done:
            ref = _alone(ctx, q, s_host, k_host)
            assert torch.isfinite(kept[q.rid]).all()
            assert torch.equal(kept[q.rid], ref), "request %d differs from its run alone" % q.rid
    finally:
        ctx.close()


def _alone_engine(ctx, q, s_host, k_host):
    """The request alone on a fresh serving engine (or, for a kernel the engine
    does not take, alone through the batched path as the loop ran it)."""
    if q.W_block > 8192 or (q.mode & 0xF0) != apx.CORE_FFT or (q.N | 1) > 4093:
        return _alone(ctx, q, s_host, k_host)
    out = torch.full((q.L + q.N - 1,), float("nan")).pin_memory()
    srv = apx.Server(ctx, slots=2, templates=1, idle_ms=5.0)
    try:
        seq = srv.submit(s_host.data_ptr() + 4 * q.s_off, q.L, k_host.data_ptr() + 4 * k_host.stride(0) * q.k_id, q.N,
                         out.data_ptr(), q.W_block, q.mode, q.target)
        while srv.poll(seq) is None:
            pass
    finally:
        srv.close()
    return out


def test_persistent_serving_same_alone_and_in_mix():
    """The serving loop on the persistent kernel: every request of a Poisson
    trace completes, requests are in flight together, and each result equals
    bit for bit the same request alone (a fresh engine)."""
    seed = wl.SEED_BASE + 43
    pool = 1 << 20
    s_host, k_host = serve.host_pools(seed, pool=pool, ntemplates=8)
    trace = serve.make_trace(seed, rate_hz=2000.0, duration_s=0.12, pool=pool, ntemplates=8, lmax_log2=20.0)
    srv = serve.PersistentServer(0, budget_bytes=48 << 20, slots=64, templates=32, out_floats=16 << 20)
    try:
        kept = {}
        done = srv.run(trace, s_host, k_host, realtime=True, on_done=lambda q: kept.__setitem__(q.rid, q.out.clone()))
    finally:
        srv.close()
    assert sorted(q.rid for q in done) == list(range(len(trace)))
    assert srv.submitted >= 1 and srv.max_overlap >= 2
    assert all(q.status == 0 for q in done)
    p50, p99 = serve.latency_ms(done)
    assert 0 < p50 <= p99
    ctx = apx.Context(0)
    try:
        for q in done:
            ref = _alone_engine(ctx, q, s_host, k_host)
            assert torch.isfinite(kept[q.rid]).all()
            assert torch.equal(kept[q.rid], ref), "request %d differs from its run alone" % q.rid
    finally:
        ctx.close()
