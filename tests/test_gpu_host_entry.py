"""apx_conv_host beyond the equality cases of the parity tests: a non-finite
input reaches the returned status and only its blocks' outputs, on page-locked
(in place) and pageable (staged) buffers alike, and the staged route's copy
stream survives the batched path allocating its page-locked parameter stage."""
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


def _device_call(ctx, s, k, Wb, mode, snr, Sq=0, Kq=0):
    r = torch.empty(s.size + k.size - 1, device="cuda")
    if (mode & 0xF00) == apx.PACK_NONE:
        ctx.apx_conv_full(_dev(s), _dev(k), Wb, mode, r)
    elif Sq:
        ctx.apx_conv_fixed(_dev(s), _dev(k), Wb, mode, Sq, Kq, r)
    else:
        ctx.apx_conv(_dev(s), _dev(k), Wb, mode, snr, r)
    return r


def _host_call(ctx, s, k, Wb, mode, snr, Sq=0, Kq=0, pinned=True):
    sh, kh = torch.from_numpy(s), torch.from_numpy(k)
    out = torch.full((s.size + k.size - 1,), float("nan"))
    if pinned:
        sh, kh, out = sh.pin_memory(), kh.pin_memory(), out.pin_memory()
    ctx.apx_conv_host(sh, kh, Wb, mode, snr, Sq, Kq, out)
    return out.numpy()


@pytest.mark.parametrize("pinned", [True, False])
def test_nonfinite_input_is_reported(ctx, pinned):
    L, N, Wb, mode = 300000, 257, 2048, apx.CORE_FFT | apx.PACK_AUTO
    s = wl.random_signal(991, L, "laplace", 0.1)
    s[123457] = np.nan
    k = wl.random_signal(992, N, "uniform")
    _device_call(ctx, s, k, Wb, mode, 20.0)
    with pytest.raises(apx.ApxError) as e:
        ctx.apx_sync()
    assert e.value.status == apx.APX_ERR_NONFINITE
    with pytest.raises(apx.ApxError) as e:
        _host_call(ctx, s, k, Wb, mode, 20.0, pinned=pinned)
    assert e.value.status == apx.APX_ERR_NONFINITE
    # the status was read and cleared by the failing call: the next one is clean
    assert ctx.apx_sync() == 0


@pytest.mark.parametrize("pinned", [True, False])
def test_nonfinite_output_matches_device_call(ctx, pinned):
    L, N, Wb, mode = 300000, 257, 2048, apx.CORE_FFT | apx.PACK_AUTO
    s = wl.random_signal(993, L, "laplace", 0.1)
    s[200001] = np.inf
    k = wl.random_signal(994, N, "uniform")
    want = _device_call(ctx, s, k, Wb, mode, 20.0).cpu().numpy()
    with pytest.raises(apx.ApxError):
        ctx.apx_sync()
    sh, kh, out = torch.from_numpy(s), torch.from_numpy(k), torch.zeros(L + N - 1)
    if pinned:
        sh, kh, out = sh.pin_memory(), kh.pin_memory(), out.pin_memory()
    with pytest.raises(apx.ApxError):
        ctx.apx_conv_host(sh, kh, Wb, mode, 20.0, 0, 0, out)
    got = out.numpy()
    assert np.isnan(got).any() and np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    np.testing.assert_array_equal(got[ok], want[ok])


def test_copy_stream_survives_the_batch_stage():
    """A pageable host call (it creates the context's signal copy stream), a
    batched call (it allocates the page-locked parameter stage), then host
    calls again on the same context: the copy stream is still valid."""
    c = apx.Context(0)
    try:
        L, N, Wb, mode = 100000, 257, 2048, apx.CORE_FFT | apx.PACK_AUTO
        s = wl.random_signal(995, L, "laplace", 0.1)
        k = wl.random_signal(996, N, "uniform")
        first = _host_call(c, s, k, Wb, mode, 20.0, pinned=False)
        items = []
        for j in range(40):
            Lj = 5000 + 997 * j
            sj, kj = _dev(wl.random_signal(2000 + j, Lj, "normal")), _dev(wl.random_signal(3000 + j, 65, "uniform"))
            items.append(dict(s=sj, k=kj, r=torch.empty(Lj + 64, device="cuda"), mode=apx.CORE_FFT | apx.PACK_AUTO,
                              W_block=1024, snr_db=20.0))
        c.apx_conv_batch(c.make_requests(items))
        assert c.apx_sync() == 0
        again = _host_call(c, s, k, Wb, mode, 20.0, pinned=False)
        pinned = _host_call(c, s, k, Wb, mode, 20.0, pinned=True)
        assert np.array_equal(first, again) and np.array_equal(first, pinned)
    finally:
        c.close()
