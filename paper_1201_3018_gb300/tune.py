"""Autotuner for the block geometry and the convolution core.

For a kernel length N (and op, packing mode, SNR target) it picks the core
(direct or FFT) and W_block.  The prior is the paper's arithmetic-cost model
(Table 1: FLOPs of full-precision, symmetric and asymmetric convolution in the
time and frequency domains at W_block = 3N + 1, generalised here to any
W_block); it ranks the candidates, and the best few are then timed on the GPU
through the C ABI with CUDA events.  Results are cached per key in memory and,
if a path is given, in a JSON file.

The candidates are timed as single calls on a signal of L samples, so L sets
what is optimised: short signals (2^18, the default) the latency of one
request, as a server wants; long ones (2^20) the throughput of many blocks in
flight, as a batched launch wants.  On the batched workload (256 signals of
2^14 - 2^20 samples) the choices made at 2^20 ran 1.7x faster than those made
at 2^18 (W_block 4096 - 8192 instead of 512 - 4096, and no direct core).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

# ---------------------------------------------------------------- Table 1 cost model


def table1_flops(method: str, domain: str, N: float) -> float:
    """FLOPs for one input block of W_block = 3N + 1 samples (Table 1)."""
    lg = math.log2
    if domain == "time":
        return {"full": 4 * N * N, "sym": N * N + N, "asym2": 2.5 * N * N - N,
                "asym3": 2 * N * N - 2.0 / 3.0 * N}[method]
    return {"full": (45 * N + 15) * lg(3 * N + 1) + 3 * N + 1,
            "sym": (22.5 * N + 7.5) * lg(3 * N + 1) + 5 * N + 1,
            "asym2": (30 * N + 15) * lg(2 * N + 1) + 19.5 * N + 6.5,
            "asym3": (25 * N + 15) * lg(5.0 / 3.0 * N + 1) + 62.0 / 3.0 * N + 7}[method]


def flops_per_output(core: str, N: int, Wb: int, method: str = "full") -> float:
    """The same cost model at an arbitrary W_block: FLOPs per kept output.
    Time domain: 2 N' (multiply + add) per output and packed word; frequency
    domain: two real FFTs of the block length and the spectral product."""
    Nodd = N | 1
    W = Wb - Nodd - 1
    if W < 2:
        return float("inf")
    if core == "direct":
        # multiply-adds of the kept outputs (packed words for the packed methods)
        per_block = {"full": 2.0 * Nodd * W, "sym": 2.0 * (W / 2 + 1) * ((Nodd + 1) / 2),
                     "asym2": 2.0 * (W / 2 + Nodd) * Nodd, "asym3": 2.0 * (W / 3 + Nodd) * Nodd}[method]
    else:
        n = {"full": Wb, "sym": Wb / 2, "asym2": Wb, "asym3": Wb}[method]
        per_block = 5.0 * n * math.log2(n) + 3.0 * n
    return per_block / W


def candidates(N: int, max_wb: int = 16384, pack: int = 0):
    """(core, W_block) pairs that satisfy the block-geometry rules.  The
    tensor-core core ("tc": the direct core's blocks, the companded integers on
    the tensor cores) serves per-block selection (APX_PACK_AUTO) for kernels of
    at most 449 taps, W_block a multiple of 64 up to 8192."""
    Nodd = N | 1
    out = []
    wb = 64
    while wb <= max_wb:
        if wb - Nodd - 1 >= 2:
            out.append(("fft", wb))
            if wb <= 8192:
                out.append(("direct", wb))
                if pack == 0 and Nodd <= 449 and wb >= 128:
                    out.append(("tc", wb))
        wb *= 2
    return out


def core_bits(core: str) -> int:
    """The mode bits of a core name the tuner returns."""
    from . import apx
    return {"fft": apx.CORE_FFT, "direct": apx.CORE_DIRECT, "tc": apx.CORE_TC}[core]


# ---------------------------------------------------------------- measurement


class Tuner:
    """Measured choice of (core, W_block) per kernel length."""

    def __init__(self, ctx, cache_path: str | None = None, L: int = 1 << 18, top: int = 8, reps: int = 9):
        self.ctx = ctx
        self.cache_path = cache_path
        self.L = L
        self.top = top
        self.reps = reps
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    @staticmethod
    def key(N, op, pack, target):
        return "N=%d op=%d pack=%d target=%g" % (N, op, pack, target)

    def _time(self, s, k, r, Wb, mode, target):
        import torch
        from . import apx
        stream = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(self.reps)]
        for _ in range(2):  # warm-up (workspace, twiddles, caches)
            self.ctx.apx_conv(s, k, Wb, mode, target, r, stream=stream)
        for a, b in ev:
            a.record(stream)
            if (mode & 0xF00) == apx.PACK_NONE:
                self.ctx.apx_conv_full(s, k, Wb, mode, r, stream=stream)
            else:
                self.ctx.apx_conv(s, k, Wb, mode, target, r, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ev]))

    def choose(self, N: int, op: int = 0, pack: int = 0, target: float = 45.0, method: str = "full"):
        """Returns dict(core=..., W_block=..., ms=..., measured=[...])."""
        import torch
        from . import apx, workloads
        key = self.key(N, op, pack, target)
        if key in self.cache:
            return self.cache[key]
        cands = candidates(N, pack=pack)
        ranked = sorted(cands, key=lambda c: flops_per_output("direct" if c[0] == "tc" else c[0], N, c[1], method))
        # the model cannot see the relative efficiency of the cores (nor the cost
        # of the halo each block reloads), so keep the best few of each
        picks = []
        for name in ("fft", "direct", "tc"):
            picks += [c for c in ranked if c[0] == name][: self.top]
        s = torch.from_numpy(workloads.random_signal(workloads.SEED_BASE + 77, self.L, "laplace", 0.1)).cuda()
        k = torch.from_numpy(workloads.random_signal(workloads.SEED_BASE + 78, N, "uniform")).cuda()
        r = torch.empty(self.L + N - 1, device="cuda")
        measured = []
        for core, Wb in picks:
            mode = op | core_bits(core) | pack
            try:
                ms = self._time(s, k, r, Wb, mode, target)
            except apx.ApxError:
                continue
            measured.append(dict(core=core, W_block=Wb, ms=ms,
                                 model_flops_per_output=flops_per_output(core, N, Wb, method)))
        best = min(measured, key=lambda d: d["ms"])
        out = dict(core=best["core"], W_block=best["W_block"], ms=best["ms"], measured=measured)
        self.cache[key] = out
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1)
            os.replace(tmp, self.cache_path)
        return out


def batch_items(case, tuner, device, op: int = 0, pack: int | None = None, tensors=None):
    """Requests of a batched case (workloads.BatchCase) with the tuned core and
    W_block for each (N, target): dicts for Context.make_requests.  `tensors`
    reuses device copies of the signals and kernels (list of (s, k))."""
    import torch
    from . import apx
    pack = apx.PACK_AUTO if pack is None else pack
    items = []
    for i, (s, k, t) in enumerate(zip(case.signals, case.kernels, case.targets)):
        ch = tuner.choose(len(k), op, pack, t)
        core = core_bits(ch["core"])
        if tensors is None:
            sd, kd = torch.from_numpy(s).to(device), torch.from_numpy(k).to(device)
        else:
            sd, kd = tensors[i]
        items.append(dict(s=sd, k=kd, r=torch.empty(len(s) + len(k) - 1, dtype=torch.float32, device=device),
                          mode=op | core | pack, W_block=ch["W_block"], snr_db=t))
    return items


def method_sweep(ctx, Ns=(32, 64, 128, 256, 512, 1024, 2048, 4096, 8192), L=1 << 20, core="direct", reps=5):
    """Throughput of each packing method against kernel length on this GPU
    (Figure 3 of the paper measures this on IPP), next to the Table 1 model:
    rows of dict(N, method, gsamples, model_ratio)."""
    import torch
    from . import apx, workloads
    s = torch.from_numpy(workloads.random_signal(workloads.SEED_BASE + 81, L, "uniform", 128.0)).cuda()
    rows = []
    packs = {"full": apx.PACK_NONE, "sym": apx.PACK_SYM, "asym2": apx.PACK_ASYM2, "asym3": apx.PACK_ASYM3}
    stream = torch.cuda.current_stream()
    for N in Ns:
        k = torch.from_numpy(workloads.random_signal(workloads.SEED_BASE + 82, N, "uniform", 128.0)).cuda()
        r = torch.empty(L + N - 1, device="cuda")
        Wb = 1024
        while Wb < 4 * (N | 1) and Wb < 8192:
            Wb *= 2
        for method, pack in packs.items():
            mode = (apx.CORE_FFT if core == "fft" else apx.CORE_DIRECT) | pack
            try:
                if pack == apx.PACK_NONE:
                    ctx.apx_conv_full(s, k, Wb, mode, r, stream=stream)
                else:
                    ctx.apx_conv(s, k, Wb, mode, 0.0, r, stream=stream)
            except apx.ApxError:
                continue
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, b in ev:
                a.record(stream)
                if pack == apx.PACK_NONE:
                    ctx.apx_conv_full(s, k, Wb, mode, r, stream=stream)
                else:
                    ctx.apx_conv(s, k, Wb, mode, 0.0, r, stream=stream)
                b.record(stream)
            torch.cuda.synchronize()
            ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
            rows.append(dict(N=N, method=method, core=core, W_block=Wb, gsamples=(L + N - 1) / ms / 1e6,
                             model_ratio=table1_flops("full", "time" if core == "direct" else "freq", N)
                             / table1_flops(method, "time" if core == "direct" else "freq", N)))
    return rows


def calibrate_snr(ctx, s, k, W_block, mode, Q=8):
    """One-point calibration of the SNR model (Fig. 5 of the paper offsets the
    model by one measured SNR at S_q = K_q = 8): runs the packing `mode` with
    S_q = K_q = Q through apx_conv_fixed and the full-precision twin, and
    returns dict(offset_db = measured - model, measured_db, model_db).  The
    model value for the whole output combines the per-block predictions as
    noise powers (equal-power blocks).  A caller that wants the measured SNR to
    meet a target passes target - offset_db to apx_conv.  Optional: the
    library never applies it by itself."""
    import torch
    from . import apx
    L, N = s.numel(), k.numel()
    r = torch.empty(L + N - 1, dtype=torch.float32, device=s.device)
    ref = torch.empty_like(r)
    P, _ = apx.plan_blocks(L, N, W_block, mode)
    st = torch.empty(P * apx.STATS_DTYPE.itemsize, dtype=torch.uint8, device=s.device)
    ctx.apx_conv_fixed(s, k, W_block, mode, Q, Q, r, None, st)
    ctx.apx_conv_full(s, k, W_block, (mode & 0xFF) | apx.PACK_NONE, ref)
    rc = ctx.apx_sync()
    if rc:
        raise apx.ApxError("apx_sync", rc)
    stats = np.frombuffer(st.cpu().numpy().tobytes(), dtype=apx.STATS_DTYPE)
    packed = np.isin(stats["mode"], (apx.BLK_SYM, apx.BLK_ASYM2, apx.BLK_ASYM3))
    if not packed.any():
        raise ValueError("no block was packed at S_q = K_q = %d" % Q)
    model = -10.0 * math.log10(float(np.mean(10.0 ** (-stats["snr_pred_db"][packed] / 10.0))))
    d = (r.double() - ref.double())
    measured = float(10.0 * torch.log10((ref.double() ** 2).sum() / (d * d).sum()))
    return dict(offset_db=measured - model, measured_db=measured, model_db=model)
