"""The serving engine's persistent kernel (apx_server): requests submitted to
a running kernel through the mapped queue complete with the same bits as the
same request on a fresh engine alone, whatever else is in flight, and agree
with Eq. (1) (full-precision blocks) and the oracle (packed blocks); a
template shared by requests is prepared once; a block's bounded wait for a
preparation that never comes is reported as a timeout and the engine serves
the next request normally."""
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_1201_3018_gb300 import apx, serve
from paper_1201_3018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = apx.Context(0)
    yield c
    c.close()


def _wait(srv, seqs, timeout=30.0):
    st, t0 = {}, time.time()
    while len(st) < len(seqs):
        for s in seqs:
            if s not in st:
                r = srv.poll(s)
                if r is not None:
                    st[s] = r
        assert time.time() - t0 < timeout, "requests did not complete"
    return st


def _requests(seed, n, pool):
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = int(2 ** g.uniform(12, 17))
        N = int(g.choice([31, 64, 255, 700, 1500, 3000]))
        Wb = {31: 1024, 64: 1024, 255: 2048, 700: 4096, 1500: 8192, 3000: 8192}[N]
        mode = (apx.OP_XCORR if i % 2 else apx.OP_CONV) | apx.CORE_FFT | (apx.PACK_NONE if i % 5 == 4 else apx.PACK_AUTO)
        out.append(dict(s_off=int(g.integers(0, pool - L)), L=L, k_id=int(g.integers(0, 4)), N=N, Wb=Wb, mode=mode,
                        snr=float(g.choice([12.0, 20.0, 30.0, 45.0]))))
    return out


def _submit(srv, q, s_host, k_host, out):
    return srv.submit(s_host.data_ptr() + 4 * q["s_off"], q["L"], k_host.data_ptr() + 4 * k_host.stride(0) * q["k_id"],
                      q["N"], out.data_ptr(), q["Wb"], q["mode"], q["snr"])


def test_engine_in_mix_equals_alone_and_oracle(ctx):
    pool = 1 << 20
    s_host, k_host = serve.host_pools(wl.SEED_BASE + 51, pool=pool, ntemplates=4, nmax=4096)
    reqs = _requests(52, 40, pool)
    outs = [torch.full((q["L"] + q["N"] - 1,), float("nan")).pin_memory() for q in reqs]
    srv = apx.Server(ctx, slots=64, templates=64, idle_ms=5.0)
    try:
        seqs = []
        for q, o in zip(reqs, outs):  # all in flight together
            seq = _submit(srv, q, s_host, k_host, o)
            assert seq is not None
            seqs.append(seq)
        st = _wait(srv, seqs)
        assert all(v == apx.APX_OK for v in st.values())
        # an idle engine: the CTAs leave after idle_ms and the next submit relaunches
        time.sleep(0.05)
        n0 = srv.launch_count()
        q, o = reqs[0], torch.full_like(outs[0], float("nan")).pin_memory()
        assert _wait(srv, [_submit(srv, q, s_host, k_host, o)])
        assert srv.launch_count() == n0 + 1
        assert torch.equal(o, outs[0])
    finally:
        srv.close()
    for i, (q, o) in enumerate(zip(reqs, outs)):
        alone = torch.full_like(o, float("nan")).pin_memory()
        one = apx.Server(ctx, slots=4, templates=2, idle_ms=5.0)
        try:
            assert _wait(one, [_submit(one, q, s_host, k_host, alone)])
        finally:
            one.close()
        assert torch.isfinite(o).all() and torch.equal(o, alone), "request %d differs from its run alone" % i
        # sampled outputs: full-precision blocks against Eq. (1); packed blocks against the oracle
        s = s_host[q["s_off"]:q["s_off"] + q["L"]].numpy()
        k = k_host[q["k_id"], :q["N"]].numpy()
        kk = k[::-1].copy() if q["mode"] & apx.OP_XCORR else k
        ro, _, so, rc = O.apx_conv(s, k, q["Wb"], q["mode"], snr_db=q["snr"], nthreads=0, want_int=False,
                                   want=np.zeros(q["L"] + q["N"] - 1, np.uint8))
        assert rc == 0
        so = O.stats_arrays(so)
        p = O.plan(q["L"], q["N"], q["Wb"], True)
        got = o.numpy()
        full = []
        for b in range(p.P):
            st0 = O.block_start(p, b)
            lo, hi = O.block_out_range(p, b)
            gi = np.arange(st0 + lo, st0 + hi)
            gi = gi[(gi >= 0) & (gi < len(got))][::37]
            if so["mode"][b] in (apx.BLK_SYM, apx.BLK_ASYM2, apx.BLK_ASYM3):
                np.testing.assert_allclose(got[gi], ro[gi], rtol=1e-6, atol=0)
            elif so["mode"][b] == apx.BLK_FULL:
                full.append(gi)
        if full:
            gi = np.concatenate(full)
            ref = O.conv_ref_at(s, kk, gi)
            assert np.linalg.norm(got[gi] - ref) <= 1e-5 * np.linalg.norm(ref), i


def test_engine_bounded_wait_times_out_and_recovers(ctx):
    pool = 1 << 18
    s_host, k_host = serve.host_pools(wl.SEED_BASE + 53, pool=pool, ntemplates=2, nmax=512)
    q = dict(s_off=1000, L=50000, k_id=1, N=255, Wb=2048, mode=apx.CORE_FFT | apx.PACK_AUTO, snr=20.0)
    srv = apx.Server(ctx, slots=8, templates=4, idle_ms=5.0)
    try:
        good = torch.full((q["L"] + q["N"] - 1,), float("nan")).pin_memory()
        assert _wait(srv, [_submit(srv, q, s_host, k_host, good)]) 
        srv.test_stall_next()
        bad = torch.zeros_like(good).pin_memory()
        st = _wait(srv, [_submit(srv, q, s_host, k_host, bad)])
        assert list(st.values()) == [apx.APX_ERR_TIMEOUT]
        assert torch.isnan(bad).all()
        again = torch.full_like(good, float("nan")).pin_memory()
        st = _wait(srv, [_submit(srv, q, s_host, k_host, again)])
        assert list(st.values()) == [apx.APX_OK] and torch.equal(again, good)
    finally:
        srv.close()


def test_engine_rejections(ctx):
    srv = apx.Server(ctx, slots=2, templates=1, idle_ms=5.0)
    try:
        s = torch.zeros(5000, device="cuda")
        k = torch.zeros(100, device="cuda")
        r = torch.empty(5099, device="cuda")
        for W_block, mode, code in ((16384, apx.CORE_FFT, apx.APX_ERR_WBLOCK), (1024, apx.CORE_DIRECT, apx.APX_ERR_ARG),
                                    (1024, apx.CORE_FFT | apx.PACK_ASYM2, apx.APX_ERR_ARG)):
            with pytest.raises(apx.ApxError) as e:
                srv.submit(s.data_ptr(), 5000, k.data_ptr(), 100, r.data_ptr(), W_block, mode, 30.0)
            assert e.value.status == code
    finally:
        srv.close()
