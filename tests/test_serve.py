"""Host-side logic of the serving loop, with a simulated executor (no GPU)."""
import math
import time

import numpy as np
import pytest

from paper_2509_22684_gb300.serve import Engine, Request, footprint_bytes, percentile, serve_serial
from workloads import poisson_trace


class FakeExecutor:
    """A batch runs its requests shortest first; request k of the batch
    completes at start + overhead + per_elem * (elements of requests up to k);
    streams are independent (the engine only launches on idle streams)."""

    def __init__(self, per_elem_s=2e-9, overhead_s=2e-4):
        self.per_elem_s = per_elem_s
        self.overhead_s = overhead_s
        self.launched = []

    def launch(self, reqs, stream):
        t = time.perf_counter() + self.overhead_s
        ends = {}
        for r in sorted(reqs, key=lambda q: (q.log_n, q.rid)):
            t += self.per_elem_s * r.n
            ends[r.rid] = t
        self.launched.append((stream, [r.rid for r in reqs]))
        return (t, ends)

    def done(self, token):
        return time.perf_counter() >= token[0]

    def finished(self, token, r):
        return time.perf_counter() >= token[1][r.rid]

    def release(self, r):
        r.out = "released"


def _trace(count=300, rate=2000.0, lmin=10, lmax=16, seed=5000):
    return [Request(q.seed % 100000, q.arrival_s, "bls12_381_fr", q.log_n, q.kind)
            for q in poisson_trace(seed, count, rate, lmin, lmax)]


def test_every_request_served_once_with_causal_times():
    reqs = _trace()
    ex = FakeExecutor()
    done, st = Engine(ex, budget_bytes=1 << 30).run(reqs)
    assert st.requests == len(reqs) == len(done)
    assert sorted(r.rid for r in done) == sorted(r.rid for r in reqs)
    launched = [rid for _, rids in ex.launched for rid in rids]
    assert sorted(launched) == sorted(r.rid for r in reqs)   # each launched exactly once
    for r in done:
        assert r.arrival_s <= r.admit_s + 1e-9 <= r.launch_s + 2e-9 <= r.finish_s + 3e-9
        assert r.out == "released"


def test_admission_respects_memory_budget_and_arrival_order():
    reqs = _trace(count=200, rate=20000.0, lmin=12, lmax=16)
    budget = 4 * footprint_bytes(16)
    done, st = Engine(FakeExecutor(), budget_bytes=budget).run(reqs)
    assert st.peak_bytes <= budget
    by_arrival = sorted(done, key=lambda r: (r.arrival_s, r.rid))
    admits = [r.admit_s for r in by_arrival]
    assert admits == sorted(admits)                          # FIFO admission


def test_continuous_batching_overlaps_two_streams_and_batches_under_load():
    reqs = _trace(count=400, rate=50000.0, lmin=10, lmax=14)
    ex = FakeExecutor(per_elem_s=1e-8)
    done, st = Engine(ex, budget_bytes=1 << 30, streams=2, max_batch_jobs=16).run(reqs)
    assert st.max_inflight_batches == 2
    assert st.mean_batch_jobs > 1.5
    assert max(len(rids) for _, rids in ex.launched) <= 16
    assert {s for s, _ in ex.launched} == {0, 1}


def test_request_larger_than_budget_is_rejected():
    reqs = [Request(0, 0.0, "bls12_381_fr", 20, "ntt")]
    with pytest.raises(ValueError):
        Engine(FakeExecutor(), budget_bytes=footprint_bytes(19)).run(reqs)


def test_batching_beats_serial_on_the_same_trace():
    reqs = _trace(count=200, rate=20000.0, lmin=10, lmax=12)
    ex = FakeExecutor(per_elem_s=1e-9, overhead_s=5e-4)
    _, st = Engine(ex, budget_bytes=1 << 30).run([Request(**{k: getattr(r, k) for k in
                                                             ("rid", "arrival_s", "field", "log_n", "kind")})
                                                  for r in reqs])
    def run_one(r):
        t = time.perf_counter() + ex.overhead_s + ex.per_elem_s * r.n
        while time.perf_counter() < t:
            pass
    _, ser = serve_serial(reqs, run_one)
    assert st.wall_s < ser.wall_s
    assert st.p99_ms < ser.p99_ms


def test_percentile_matches_numpy():
    rng = np.random.default_rng(3)
    v = list(rng.exponential(size=1001))
    for q in (0.0, 0.5, 0.9, 0.99, 1.0):
        assert math.isclose(percentile(v, q), float(np.percentile(v, 100 * q)), rel_tol=1e-12)


def test_small_requests_retire_before_the_large_one_in_their_batch():
    reqs = [Request(0, 0.0, "bls12_381_fr", 18, "ntt")] + \
           [Request(i, 0.0, "bls12_381_fr", 10, "ntt") for i in range(1, 6)]
    ex = FakeExecutor(per_elem_s=2e-8, overhead_s=1e-4)
    done, st = Engine(ex, budget_bytes=1 << 30, streams=1).run(reqs)
    assert st.batches == 1
    big = [r for r in done if r.rid == 0][0]
    small = [r for r in done if r.rid != 0]
    assert all(r.finish_s < big.finish_s for r in small)


class SoloFakeExecutor(FakeExecutor):
    """FakeExecutor that also runs single requests as plain launches."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.solo = []

    def launch_solo(self, r, stream):
        self.solo.append(r.rid)
        return self.launch([r], stream)


def test_large_requests_run_solo_in_arrival_order():
    reqs = _trace(count=300, rate=50000.0, lmin=10, lmax=18)
    ex = SoloFakeExecutor(per_elem_s=1e-9, overhead_s=1e-4)
    done, st = Engine(ex, budget_bytes=1 << 32, streams=2, max_batch_jobs=16, solo_log_n=16).run(reqs)
    assert st.requests == len(reqs)
    big = {r.rid for r in reqs if r.log_n >= 16}
    assert big and big <= set(ex.solo)                      # every large one ran alone
    for _, rids in ex.launched:                             # and never inside a batch
        if len(rids) > 1:
            assert not big & set(rids)
    order = sorted((r for r in reqs if r.log_n >= 16), key=lambda r: (r.arrival_s, r.rid))
    first_launch = {rid: k for k, (_, rids) in enumerate(ex.launched) for rid in rids}
    ks = [first_launch[r.rid] for r in order]
    assert ks == sorted(ks)                                 # large ones keep arrival order
    launched = [rid for _, rids in ex.launched for rid in rids]
    assert sorted(launched) == sorted(r.rid for r in reqs)  # each launched exactly once


def test_single_request_batches_become_solo_launches():
    reqs = [Request(i, 0.01 * i, "bls12_381_fr", 10, "ntt") for i in range(5)]
    ex = SoloFakeExecutor(per_elem_s=1e-9, overhead_s=1e-5)
    done, st = Engine(ex, budget_bytes=1 << 30, streams=1).run(reqs)
    assert st.requests == 5
    assert sorted(ex.solo) == list(range(5))                # spaced arrivals: one at a time


def test_without_launch_solo_everything_is_batched():
    reqs = _trace(count=100, rate=50000.0, lmin=10, lmax=18)
    ex = FakeExecutor(per_elem_s=1e-9, overhead_s=1e-4)
    done, st = Engine(ex, budget_bytes=1 << 32, streams=2, solo_log_n=12).run(reqs)
    assert st.requests == len(reqs)


class LiveMemoryExecutor(FakeExecutor):
    """A device with a fixed amount of memory: launched requests hold their
    footprint until released; the engine sees only the live headroom."""

    def __init__(self, capacity, **kw):
        super().__init__(**kw)
        self.capacity = capacity
        self.held = 0
        self.max_held = 0

    def footprint(self, r):
        # single-pass sizes need no scratch, like a plan of one pass
        return 32 * r.n + (32 * r.n if r.log_n > 13 else 0)

    def headroom_bytes(self):
        return self.capacity - self.held

    def launch(self, reqs, stream):
        for r in reqs:
            self.held += self.footprint(r)
        self.max_held = max(self.max_held, self.held)
        return super().launch(reqs, stream)

    def release(self, r):
        self.held -= self.footprint(r)
        super().release(r)


def test_admission_follows_live_device_memory_and_the_plans_footprint():
    """With an executor that reports live headroom, admitted work never holds
    more device memory than there is, even under a far larger budget, and the
    footprint comes from the executor (the plan's own scratch), not from a
    size threshold."""
    reqs = _trace(count=200, rate=20000.0, lmin=12, lmax=16)
    ex = LiveMemoryExecutor(capacity=3 * 64 * (1 << 16))
    done, st = Engine(ex, budget_bytes=1 << 40, streams=2).run(reqs)
    assert st.requests == len(reqs)
    assert ex.max_held <= ex.capacity
    assert ex.held == 0
    assert st.peak_bytes <= ex.capacity
