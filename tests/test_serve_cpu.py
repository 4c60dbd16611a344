"""Host-side logic of the Poisson request loop (no GPU)."""
import math

import pytest

import numpy as np

from paper_1506_07933_gb300 import serve


def test_request_stream_is_seeded_and_has_the_stated_mix():
    a = serve.poisson_requests(2000, rate=200.0, seed=5)
    b = serve.poisson_requests(2000, rate=200.0, seed=5)
    assert [(r.arrival, r.n, r.precision) for r in a] == [(r.arrival, r.n, r.precision) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0           # exponential, mean 1/rate
    assert abs(np.mean([r.precision == "f64" for r in a]) - 0.3) < 0.05
    assert set(r.n for r in a) == {64, 128, 192, 256, 384, 512}
    assert set(r.sample for r in a) == {0, 1, 2, 3}
    assert all(x <= y for x, y in zip([r.arrival for r in a], [r.arrival for r in a][1:]))


def test_saturation_stream_arrives_at_once():
    reqs = serve.poisson_requests(10, rate=0, seed=1)
    assert all(r.arrival == 0.0 for r in reqs)


def test_percentiles_and_summary():
    assert serve._percentile([5, 1, 3, 2, 4], 50) == 3
    assert serve._percentile(list(range(1, 101)), 99) == 99
    assert math.isnan(serve._percentile([], 50))
    reqs = serve.poisson_requests(4, rate=100.0, seed=2)
    for i, r in enumerate(reqs):
        r.done = r.arrival + 0.001 * (i + 1)
        r.error = 1e-7
        r.batch = 1
    s = serve.summarize(reqs, 1.0)
    assert s["requests"] == 4 and abs(s["p50_ms"] - 2.0) < 1e-9 and abs(s["max_ms"] - 4.0) < 1e-9


def test_batch_cap_follows_the_byte_budget():
    class S(serve.PoissonServer):
        def __init__(self):
            self.max_batch_bytes = 64 << 20
            self.max_batch = 16
    s = S()
    assert s._cap(64, "f32") == 16
    assert s._cap(512, "f32") == 1
    assert s._cap(256, "f64") == 1
    assert s._cap(128, "f32") == 8
    assert s._cap(192, "f32") == 2
    # batches are powers of two no larger than what waits
    assert [s._batch(64, "f32", w) for w in (1, 2, 3, 7, 8, 40)] == [1, 2, 2, 4, 8, 16]
    assert s._batch(128, "f32", 100) == 8 and s._batch(512, "f64", 5) == 1
    # a single request is solved from its own buffer: no gathered input in its footprint
    assert s._footprint(64, "f32", 2) - 2 * s._footprint(64, "f32", 1) == 2 * 64 ** 3 * 4


def test_admission_survives_injected_allocation_failures():
    """Admission without a GPU: an allocation the device refuses (injected) evicts the idle plans
    of other sizes and retries once; a second refusal leaves the request waiting (None) and is
    counted.  The budget itself still refuses a batch that can never fit."""
    closed = []

    class FakePlan:
        def close(self):
            closed.append(self)

    srv = serve.PoissonServer.__new__(serve.PoissonServer)
    srv.budget, srv.max_batch_bytes, srv.max_batch = 1 << 40, 64 << 20, 16
    srv.plans, srv.held, srv.alloc_failures = {}, 0, 0
    refusals = {"left": 1}

    def alloc(n, prec, B):
        if refusals["left"] > 0:
            refusals["left"] -= 1
            raise MemoryError("injected allocation failure")
        return FakePlan(), None, object()

    srv.alloc = alloc
    srv.plans[(64, "f32", 1)] = [(FakePlan(), None, object())]
    srv.held = srv._footprint(64, "f32", 1)
    entry = srv._take(128, "f32", 1)
    assert entry is not None and len(closed) == 1 and srv.plans[(64, "f32", 1)] == []
    assert srv.held == srv._footprint(128, "f32", 1)
    refusals["left"] = 2
    assert srv._take(256, "f32", 1) is None and srv.alloc_failures == 1
    assert srv.held == srv._footprint(128, "f32", 1)
    srv.budget = 1 << 20
    with pytest.raises(MemoryError):
        srv._take(512, "f64", 1)
