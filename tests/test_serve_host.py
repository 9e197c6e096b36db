"""Host logic of the serving loop: admission by device-memory budget and the
request trace (no GPU)."""
import numpy as np

from paper_1201_3018_gb300 import serve


def test_admit_respects_budget():
    assert serve.admit([10, 10, 10], 0, 25, 64) == 2
    assert serve.admit([10, 10, 10], 10, 25, 64) == 1
    assert serve.admit([10, 10, 10], 20, 25, 64) == 0
    assert serve.admit([10, 10, 10], 0, 1000, 2) == 2
    assert serve.admit([], 0, 1000, 8) == 0


def test_admit_oversize_alone_when_idle():
    # larger than the whole budget: admitted alone, only with nothing in flight
    assert serve.admit([100, 1], 0, 50, 64) == 1
    assert serve.admit([100, 1], 1, 50, 64) == 0


def test_admit_fifo_no_overtaking():
    # a small request behind a large one waits (arrival order is kept)
    assert serve.admit([40, 1, 1], 20, 50, 64) == 0


def test_admission_never_exceeds_budget_in_simulation():
    g = np.random.default_rng(5)
    sizes = list(g.integers(1, 40, 500))
    budget, in_flight, flights = 100, 0, []
    waiting = list(sizes)
    while waiting or flights:
        n = serve.admit(waiting, in_flight, budget, 8)
        if n:
            b = sum(waiting[:n])
            flights.append(b)
            in_flight += b
            waiting = waiting[n:]
            assert in_flight <= budget
        if flights and (not n or len(flights) > 3):
            in_flight -= flights.pop(0)


def test_bucket_and_bytes():
    assert [serve.n_bucket(n) for n in (1, 2, 3, 64, 65, 8192)] == [1, 2, 4, 64, 128, 8192]
    q = serve.Request(0, 0.0, L=100, N=10, xcorr=False, target=45.0, s_off=0, k_id=0)
    assert serve.device_bytes(q) == 4 * (100 + 10 + 109)


def test_trace_shape():
    tr = serve.make_trace(12013023, rate_hz=2000.0, duration_s=0.5, pool=1 << 20, lmax_log2=20.0)
    assert 800 < len(tr) < 1200           # Poisson(1000)
    t = np.array([q.t for q in tr])
    assert np.all(np.diff(t) >= 0) and t[-1] <= 0.5
    for q in tr:
        assert 1 <= q.N <= min(8192, q.L) and q.L <= 1 << 20
        assert 0 <= q.s_off <= (1 << 20) - q.L
        assert q.target in (30.0, 45.0, 60.0)
    # mean inter-arrival close to 1 / rate
    assert abs(np.diff(t).mean() - 5e-4) < 1e-4


def test_output_ring_never_overlaps_held_regions():
    """Regions handed out in order and released in any order: no two held
    regions overlap, every region lies inside the buffer, and a request that
    cannot be placed is refused rather than placed over a held one."""
    g = np.random.default_rng(9)
    ring = serve.OutputRing(1000)
    held = []
    refused = 0
    for step in range(5000):
        if held and (g.random() < 0.45 or len(held) > 20):
            reg = held.pop(int(g.integers(0, len(held))))
            ring.free(reg)
            continue
        reg = ring.alloc(int(g.integers(1, 300)))
        if reg is None:
            refused += 1
            continue
        assert 0 <= reg[0] < reg[1] <= 1000
        for h in held:
            assert reg[1] <= h[0] or h[1] <= reg[0], (reg, h)
        held.append(reg)
    assert refused > 0 and ring.alloc(2000) is None
    for reg in held:
        ring.free(reg)
    assert ring.alloc(1000) == [0, 1000, False]
