"""Scheduling invariants of the serving engine over generated traces and
configurations (host logic only, simulated executor): every request is
served exactly once with causal timestamps, the memory budget is never
exceeded, admission is first-come first-served, no launch exceeds the batch
limit or mixes solo and batched work, and large requests keep their
arrival order."""
import time

import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from paper_2509_22684_gb300.serve import Engine, Request, footprint_bytes  # noqa: E402


class SimExecutor:
    """Completes a launch `cost(request)` after it starts; solo launches when
    `solo` is set, else everything goes through launch()."""

    def __init__(self, per_elem_s, solo):
        self.per_elem_s = per_elem_s
        self.launched = []     # (kind, stream, [rids])
        if solo:
            self.launch_solo = self._launch_solo

    def launch(self, reqs, stream):
        t = time.perf_counter()
        ends = {}
        for r in sorted(reqs, key=lambda q: (q.log_n, q.rid)):
            t += self.per_elem_s * r.n
            ends[r.rid] = t
        self.launched.append(("batch", stream, [r.rid for r in reqs]))
        return (t, ends)

    def _launch_solo(self, r, stream):
        tok = self.launch([r], stream)
        self.launched[-1] = ("solo", stream, [r.rid])
        return tok

    def done(self, token):
        return time.perf_counter() >= token[0]

    def finished(self, token, r):
        return time.perf_counter() >= token[1][r.rid]

    def release(self, r):
        pass


traces = st.lists(st.tuples(st.floats(0, 0.004), st.integers(8, 14)), min_size=1, max_size=60)


@settings(max_examples=40, deadline=None)
@given(trace=traces, streams=st.integers(1, 3), max_jobs=st.integers(1, 8),
       budget_units=st.integers(1, 6), solo=st.booleans(), solo_log_n=st.integers(9, 15))
def test_engine_invariants(trace, streams, max_jobs, budget_units, solo, solo_log_n):
    reqs = [Request(i, t, "bls12_381_fr", L, "ntt") for i, (t, L) in enumerate(sorted(trace))]
    budget = budget_units * footprint_bytes(14)
    ex = SimExecutor(per_elem_s=2e-9, solo=solo)
    eng = Engine(ex, budget_bytes=budget, streams=streams, max_batch_jobs=max_jobs,
                 solo_log_n=solo_log_n, idle_sleep_s=0)
    done, stats = eng.run(reqs, realtime=False)
    # exactly once, causal
    assert sorted(r.rid for r in done) == list(range(len(reqs)))
    launched = [rid for _, _, rids in ex.launched for rid in rids]
    assert sorted(launched) == list(range(len(reqs)))
    for r in done:
        assert r.admit_s <= r.launch_s + 1e-9 <= r.finish_s + 2e-9
    # memory budget and FIFO admission
    assert stats.peak_bytes <= budget
    by_arrival = sorted(done, key=lambda r: (r.arrival_s, r.rid))
    assert [r.admit_s for r in by_arrival] == sorted(r.admit_s for r in by_arrival)
    # batch limit, stream range
    for kind, stream, rids in ex.launched:
        assert 0 <= stream < streams
        assert 1 <= len(rids) <= max_jobs
    if solo:
        big = {r.rid for r in reqs if r.log_n >= solo_log_n}
        for kind, _, rids in ex.launched:
            if kind == "batch":
                assert not big & set(rids)            # large ones never batched
            if len(rids) == 1 and kind == "batch":
                pytest.fail("a single-request batch should have been a solo launch")
        first = {rid: k for k, (_, _, rids) in enumerate(ex.launched) for rid in rids}
        order = [first[r.rid] for r in by_arrival if r.log_n >= solo_log_n]
        assert order == sorted(order)                 # arrival order among large ones
    else:
        assert all(kind == "batch" for kind, _, _ in ex.launched)
