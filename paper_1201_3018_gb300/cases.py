"""Run one benchmark case a few times through the C ABI (for profilers).

  python -m paper_1201_3018_gb300.cases CASE [REPEATS]

CASE:
  matching    the matching workload: 2^20-sample Laplacian(0, 0.1) signal
              cross-correlated with a 4096-tap template, FFT core, W_block
              8192, target 45 dB (every block full precision: the two-CTA
              block kernel after the two preparation launches)
  fft_packed  (2^19 + 777)-sample Laplacian(0, 0.1) signal, 257-tap U[-1,1]
              kernel, FFT core, W_block 2048, target 20 dB (most blocks pack
              asymmetric M = 2: the general block kernel's FP64 branch)
  direct_x1024  the single-conv workload (65,536 N(0,1) samples, 64-tap
              U[-1,1] kernel, W_block 1024, direct core, target 45 dB) as 1024
              requests of one batched call (asymmetric M = 2 on every block)
  tc_x1024    the same with the tensor-core core (every block's companded
              integers on the tensor cores)
Prints the per-block mode histogram of the last call.
"""
from __future__ import annotations

import sys

import numpy as np


def run(case: str, repeats: int = 3) -> np.ndarray:
    import torch
    from . import apx
    from . import workloads as wl
    ctx = apx.Context(torch.cuda.current_device())
    try:
        if case == "matching":
            c = wl.matching_xcorr(snr_db=45.0)
            s, k = torch.from_numpy(c.s).cuda(), torch.from_numpy(c.k).cuda()
            L, N, Wb = len(c.s), len(c.k), c.Wblock
            mode, snr = apx.OP_XCORR | apx.CORE_FFT | apx.PACK_AUTO, 45.0
        elif case == "fft_packed":
            L, N, Wb = (1 << 19) + 777, 257, 2048
            s = torch.from_numpy(wl.random_signal(5, L, "laplace", 0.1)).cuda()
            k = torch.from_numpy(wl.random_signal(6, N, "uniform")).cuda()
            mode, snr = apx.OP_CONV | apx.CORE_FFT | apx.PACK_AUTO, 20.0
        elif case in ("direct_x1024", "tc_x1024"):
            c = wl.single_conv()
            s, k = torch.from_numpy(c.s).cuda(), torch.from_numpy(c.k).cuda()
            L, N, Wb = len(c.s), len(c.k), c.Wblock
            core = apx.CORE_DIRECT if case == "direct_x1024" else apx.CORE_TC
            mode, snr = apx.OP_CONV | core | apx.PACK_AUTO, 45.0
            r = torch.empty(1024, L + N - 1, device="cuda")
            reqs = ctx.make_requests([dict(s=s, k=k, r=r[j], mode=mode, W_block=Wb, snr_db=snr) for j in range(1024)])
            for _ in range(repeats):
                ctx.apx_conv_batch(reqs)
            ctx.apx_sync()
        else:
            raise SystemExit("unknown case %r (matching, fft_packed, direct_x1024, tc_x1024)" % case)
        # one more single call with per-block records for the histogram (the
        # records select the general kernel; profile the launches before it)
        r1 = torch.empty(L + N - 1, device="cuda")
        if case not in ("direct_x1024", "tc_x1024"):
            for _ in range(repeats):
                ctx.apx_conv(s, k, Wb, mode, snr, r1)
        P, _ = apx.plan_blocks(L, N, Wb, mode)
        st = torch.empty(P * apx.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        ctx.apx_conv(s, k, Wb, mode, snr, r1, None, st)
        ctx.apx_sync()
        modes = np.frombuffer(st.cpu().numpy().tobytes(), dtype=apx.STATS_DTYPE)["mode"]
        return np.bincount(modes, minlength=7)
    finally:
        ctx.close()


if __name__ == "__main__":
    if len(sys.argv) < 2:
        raise SystemExit(__doc__)
    hist = run(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 3)
    print("%s: block modes full/sym/asym2/asym3/zero/nonfinite/tc = %s" % (sys.argv[1], hist.tolist()))
