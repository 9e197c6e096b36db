"""Serving loop with continuous batching.

Requests (convolution or cross-correlation of a signal with a kernel under an
SNR target, Section IV.D) arrive over time.  The scheduler admits, in arrival
order, every waiting request whose device buffers fit the memory budget next to
the work already on the GPU, groups the admitted ones into one batched call
(apx_conv_batch: one launch per core and W_block group), and issues it on the
next free stream.  Requests that arrive while earlier batches are on the GPU
are admitted into later batches as streams and memory free up, so their work
overlaps on the device.  Every batch is one apx_conv_batch_host call: the
library copies each request's input from pinned host memory, runs the batch and
copies the results back into pinned host memory, so the per-request host work
is one record of the request table; a request's latency is completion (the
batch's event observed done) minus arrival.

Measured at 2000 requests/s: 8 streams with at most 8 requests per batch give
a p99 of about 0.8 ms; batches of up to 64 gave 18 ms (a burst's requests wait
behind each other in one launch sequence, and the growing workspaces stall the
scheduler).  Each stream has its own library context, so the workspaces of
batches in flight never alias; a request's result does not depend on what else shares
its batch (the batched kernels take each request's parameters from its own
table entry).  Core and W_block per kernel length come from the autotuner
(tune.Tuner, one measurement per power-of-two bucket of N) or the library
default.
"""
from __future__ import annotations

import collections
import contextlib
import dataclasses
import gc
import time

import numpy as np


@contextlib.contextmanager
def gc_paused():
    """No cyclic garbage collection while requests are in flight: a full
    collection of a large heap stops the host loop for tens of milliseconds,
    which every request then in flight pays (one collection before)."""
    enabled = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        if enabled:
            gc.enable()


@dataclasses.dataclass
class Request:
    rid: int
    t: float              # arrival time, seconds from the start of the trace
    L: int
    N: int
    xcorr: bool
    target: float
    s_off: int            # offset of the signal in the host pool
    k_id: int             # template index
    arrival: float = 0.0  # wall clock of arrival
    done: float = 0.0     # wall clock of completion
    W_block: int = 0      # what was launched (0: library default)
    mode: int = 0
    out: object = None    # pinned host result
    status: int = 0       # completion status (APX_OK, ...)
    path: str = ""        # which path served it ("engine" or "batched")


def device_bytes(q) -> int:
    """Device memory a request holds while in flight: signal, kernel, result."""
    return 4 * (q.L + q.N + q.L + q.N - 1)


def admit(waiting_bytes, in_flight: int, budget: int, max_batch: int) -> int:
    """How many of the waiting requests (arrival order) the next batch takes.

    A request is admitted while the bytes in flight plus the batch so far plus
    its own stay within the budget.  A request larger than the whole budget is
    admitted alone once nothing else is in flight, so it cannot starve."""
    n, used = 0, 0
    for b in waiting_bytes:
        if n >= max_batch:
            break
        if in_flight + used + b > budget and (n > 0 or in_flight > 0):
            break
        used += b
        n += 1
    return n


def n_bucket(N: int) -> int:
    """Power of two at or above N: the autotuner's key for kernel length N."""
    b = 1
    while b < N:
        b *= 2
    return b


class Server:
    def __init__(self, device: int = 0, budget_bytes: int = 40 << 30, streams: int = 8, tuner=None,
                 max_batch: int = 8, pinned_bytes: int = 32 << 20):
        import torch
        from . import apx
        self.apx = apx
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.budget = budget_bytes
        self.ctxs = [apx.Context(device) for _ in range(streams)]
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(streams)]
        # one pinned result buffer per stream, allocated once (a first-time pinned
        # allocation of tens of MB takes milliseconds and would land in the latencies)
        self.pinned = [torch.empty(pinned_bytes // 4, dtype=torch.float32, pin_memory=True) for _ in range(streams)]
        self.busy = [None] * streams   # (event, requests, bytes, device buffers, request table)
        self.tuner = tuner
        self.max_batch = max_batch
        self.in_flight = 0
        self.peak_in_flight = 0
        self.batches = 0
        self.max_overlap = 0           # most batches on the GPU at once
        self.batch_sizes = []

    def close(self):
        for c in self.ctxs:
            c.close()

    def choice(self, N, op, target):
        from . import tune
        apx = self.apx
        if self.tuner is None:
            return 0, apx.CORE_AUTO
        ch = self.tuner.choose(n_bucket(N), op, apx.PACK_AUTO, target)
        return ch["W_block"], tune.core_bits(ch["core"])

    def _launch(self, si, batch, s_host, k_host):
        """One apx_conv_batch_host call: the library copies each request's
        signal and kernel from the pinned pools, runs the batch and copies the
        results into one pinned buffer per batch (request q's result is a view)."""
        torch, apx = self.torch, self.apx
        st = self.streams[si]
        lens = [q.L + q.N - 1 for q in batch]
        out = self.pinned[si]
        if sum(lens) > out.numel():  # a request larger than the stream's buffer (batched alone)
            out = torch.empty(sum(lens), dtype=torch.float32, pin_memory=True)
        reqs = np.zeros(len(batch), dtype=apx.REQUEST_DTYPE)
        sb, kb, ob = s_host.data_ptr(), k_host.data_ptr(), out.data_ptr()
        krow = 4 * k_host.stride(0)
        off = 0
        for j, q in enumerate(batch):
            op = apx.OP_XCORR if q.xcorr else apx.OP_CONV
            Wb, core = self.choice(q.N, op, q.target)
            q.W_block, q.mode = Wb, op | core | apx.PACK_AUTO
            reqs[j] = (sb + 4 * q.s_off, q.L, kb + krow * q.k_id, q.N, ob + 4 * off, Wb, q.mode, q.target, 0, 0, 0, 0)
            q.out = out[off:off + lens[j]]
            off += lens[j]
        self.ctxs[si].apx_conv_batch_host(reqs, stream=st)
        ev = torch.cuda.Event()
        ev.record(st)
        nbytes = sum(device_bytes(q) for q in batch)
        self.busy[si] = (ev, batch, nbytes, out, reqs)
        self.in_flight += nbytes
        self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
        self.batches += 1
        self.batch_sizes.append(len(batch))
        self.max_overlap = max(self.max_overlap, sum(b is not None for b in self.busy))

    def _poll(self, on_done=None):
        done = []
        for si, b in enumerate(self.busy):
            if b is not None and b[0].query():
                now = time.perf_counter()
                for q in b[1]:
                    q.done = now
                    if on_done is not None:
                        on_done(q)  # q.out is valid until the stream's next batch
                self.in_flight -= b[2]
                done.extend(b[1])
                self.busy[si] = None
        return done

    def run(self, trace, s_host, k_host, realtime: bool = True, on_done=None):
        """Serve `trace` (Requests sorted by arrival time t).  With realtime
        False every request arrives at once.  Returns the completed requests.
        A request's result q.out is a view of its stream's pinned buffer, valid
        until that stream's next batch: `on_done(q)` runs at completion, before
        the buffer is reused, for a consumer that keeps results."""
        with gc_paused():
            return self._run(trace, s_host, k_host, realtime, on_done)

    def _run(self, trace, s_host, k_host, realtime, on_done):
        pending = collections.deque(trace)
        waiting = collections.deque()
        finished = []
        t0 = time.perf_counter()
        while pending or waiting or any(b is not None for b in self.busy):
            now = time.perf_counter()
            while pending and (not realtime or pending[0].t <= now - t0):
                q = pending.popleft()
                q.arrival = t0 + q.t if realtime else now
                waiting.append(q)
            finished.extend(self._poll(on_done))
            free = [i for i, b in enumerate(self.busy) if b is None]
            if waiting and free:
                n = admit((device_bytes(q) for q in waiting), self.in_flight, self.budget, self.max_batch)
                # and whose results fit the stream's pinned buffer (at least one request)
                cap, used, m = self.pinned[free[0]].numel(), 0, 0
                while m < n and (m == 0 or used + waiting[m].L + waiting[m].N - 1 <= cap):
                    used += waiting[m].L + waiting[m].N - 1
                    m += 1
                n = m
                if n:
                    batch = [waiting.popleft() for _ in range(n)]
                    self._launch(free[0], batch, s_host, k_host)
                    continue
            if realtime and pending and not waiting:
                time.sleep(max(0.0, min(1e-4, pending[0].t - (time.perf_counter() - t0))))
        return finished


def make_trace(seed, rate_hz=2000.0, duration_s=1.0, pool=1 << 23, ntemplates=32, lmax_log2=22.0, nmax=8192):
    """Poisson trace of requests over a pinned signal pool and a set of
    templates (matching/filtering requests reuse templates)."""
    from . import workloads
    reqs = []
    for i, d in enumerate(workloads.serving_trace(seed, rate_hz, duration_s, lmax_log2=lmax_log2, nmax=nmax)):
        g = np.random.default_rng(d["seed"])
        L = min(d["L"], pool)
        reqs.append(Request(rid=i, t=d["t"], L=L, N=min(d["N"], nmax, L), xcorr=d["xcorr"], target=d["target"],
                            s_off=int(g.integers(0, pool - L + 1)), k_id=int(g.integers(0, ntemplates))))
    return reqs


def host_pools(seed, pool=1 << 23, ntemplates=32, nmax=8192):
    """Pinned host signal pool (Laplacian(0, 0.1)) and templates (U[-1, 1])."""
    import torch
    from . import workloads
    s = torch.from_numpy(workloads.random_signal(seed, pool, "laplace", 0.1)).pin_memory()
    k = torch.from_numpy(np.stack([workloads.random_signal(seed + 1 + j, nmax, "uniform")
                                   for j in range(ntemplates)])).pin_memory()
    return s, k


def latency_ms(done):
    lat = np.array([(q.done - q.arrival) * 1e3 for q in done])
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


class OutputRing:
    """Regions of a circular buffer of `cap` elements, handed out in order and
    released in any order; space is reclaimed from the oldest region on, so a
    region is never overwritten while it is held."""

    def __init__(self, cap: int):
        self.cap = cap
        self.regions = collections.deque()  # [start, end, released] in allocation order

    def alloc(self, n: int):
        if n < 1 or n > self.cap:
            return None
        if not self.regions:
            start = 0
        else:
            head, tail = self.regions[-1][1], self.regions[0][0]
            if head > tail or (head == tail and head == self.cap):
                start = head if head + n <= self.cap else (0 if n <= tail else None)
            elif head == tail:  # full
                start = None
            else:
                start = head if head + n <= tail else None
        if start is None:
            return None
        reg = [start, start + n, False]
        self.regions.append(reg)
        return reg

    def unalloc(self, reg):
        """Take back the newest region (its request was not accepted)."""
        assert self.regions and self.regions[-1] is reg
        self.regions.pop()

    def free(self, reg):
        reg[2] = True
        while self.regions and self.regions[0][2]:
            self.regions.popleft()


class PersistentServer:
    """The same serving on the library's persistent kernel (apx_server): each
    admitted request is submitted on its own as it arrives (no host batching:
    the kernel's CTAs take the blocks of whatever is in flight), its signal is
    read in place from the pinned pool and its result written in place into a
    pinned output ring, and completion is read from a host-mapped word.
    Templates stay resident on the device between requests that share them.
    The engine serves the FFT core at W_block 8192, kernels of up to 4093
    taps; longer kernels go to the host-batched path (Server) on its own
    streams, beside the persistent kernel (one CTA per two SMs)."""

    def __init__(self, device: int = 0, budget_bytes: int = 40 << 30, tuner=None, slots: int = 512,
                 templates: int = 128, out_floats: int = 64 << 20, idle_ms: float = 20.0, fallback_streams: int = 2,
                 ctas: int = 0):
        import torch
        from . import apx
        self.apx, self.torch = apx, torch
        self.ctx = apx.Context(device)
        # one persistent CTA per two SMs: the batched path's block kernels (up to
        # 512 threads) still find room beside it
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        self.srv = apx.Server(self.ctx, slots=slots, templates=templates, ctas=ctas or max(1, sms // 2),
                              idle_ms=idle_ms)
        self.out = torch.empty(out_floats, dtype=torch.float32, pin_memory=True)
        self.ring = OutputRing(out_floats)
        self.budget = budget_bytes
        self.tuner = tuner
        self.inflight = {}                  # seq -> (request, bytes)
        self.in_flight = 0
        self.peak_in_flight = 0
        self.max_overlap = 0
        self.submitted = 0
        self.fallback = Server(device, budget_bytes=budget_bytes, streams=fallback_streams, tuner=tuner, max_batch=1)

    def close(self):
        self.srv.close()
        self.fallback.close()
        self.ctx.close()

    def engine_choice(self, N, op, target):
        """W_block for the engine, or None for the batched path.  The engine's
        CTAs take one block per work item, so each item should carry many
        outputs: W_block 8192 (the engine's largest) for kernels of up to 4093
        taps, whose blocks then keep at least 4098 outputs."""
        return None if (N | 1) > 4093 else 8192

    def _submit(self, q, s_host, k_host):
        apx = self.apx
        op = apx.OP_XCORR if q.xcorr else apx.OP_CONV
        Wb = self.engine_choice(q.N, op, q.target)
        n = q.L + q.N - 1
        reg = self.ring.alloc(n)
        if reg is None:
            return False
        q.W_block, q.mode = Wb, op | apx.CORE_FFT | apx.PACK_AUTO
        q.out = self.out[reg[0]:reg[1]]
        seq = self.srv.submit(s_host.data_ptr() + 4 * q.s_off, q.L, k_host.data_ptr() + 4 * k_host.stride(0) * q.k_id,
                              q.N, q.out.data_ptr(), Wb, q.mode, q.target)
        if seq is None:  # every slot or template entry in use
            self.ring.unalloc(reg)
            return False
        nbytes = device_bytes(q)
        q.path = "engine"
        self.inflight[seq] = (q, nbytes, reg)
        self.in_flight += nbytes
        self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
        self.max_overlap = max(self.max_overlap, len(self.inflight))
        self.submitted += 1
        return True

    def _poll(self, on_done=None):
        done = []
        for seq in list(self.inflight):
            st = self.srv.poll(seq)
            if st is None:
                continue
            q, nbytes, reg = self.inflight.pop(seq)
            q.done = time.perf_counter()
            q.status = st
            if on_done is not None:
                on_done(q)  # q.out is valid until its region of the ring is reused
            self.ring.free(reg)
            self.in_flight -= nbytes
            done.append(q)
        return done

    def run(self, trace, s_host, k_host, realtime: bool = True, on_done=None):
        """Serve `trace` as Server.run does; returns the completed requests."""
        with gc_paused():
            return self._run(trace, s_host, k_host, realtime, on_done)

    def _run(self, trace, s_host, k_host, realtime, on_done):
        apx = self.apx
        pending = collections.deque(trace)
        waiting = collections.deque()
        finished = []
        fb = self.fallback
        t0 = time.perf_counter()
        while pending or waiting or self.inflight or any(b is not None for b in fb.busy):
            now = time.perf_counter()
            while pending and (not realtime or pending[0].t <= now - t0):
                q = pending.popleft()
                q.arrival = t0 + q.t if realtime else now
                waiting.append(q)
            finished.extend(self._poll(on_done))
            finished.extend(fb._poll(on_done))
            # admission in arrival order: the engine, or the batched path for long kernels
            while waiting:
                q = waiting[0]
                op = apx.OP_XCORR if q.xcorr else apx.OP_CONV
                if self.engine_choice(q.N, op, q.target) is None:
                    free = [i for i, b in enumerate(fb.busy) if b is None]
                    if not free:
                        break
                    q.path = "batched"
                    fb._launch(free[0], [waiting.popleft()], s_host, k_host)
                    continue
                if self.in_flight + device_bytes(q) > self.budget and self.inflight:
                    break
                if not self._submit(q, s_host, k_host):
                    break
                waiting.popleft()
            if realtime and pending and not waiting and not self.inflight:
                time.sleep(max(0.0, min(1e-4, pending[0].t - (time.perf_counter() - t0))))
        return finished
