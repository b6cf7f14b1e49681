"""Serving loop: continuous batching of NTT requests on one GPU.

The paper observes that NTT work arrives in sizes that vary by application and
that host-device transfers and short, poorly configured launches dominate
existing libraries (Section IV-A); it calls for runtime adaptation (Section
V-A).  This engine keeps request vectors and plan twiddle tables resident in
device memory, admits requests while others run, and packs everything admitted
into the next persistent batch launch:

* admission: a request enters when its device footprint (output vector plus
  its plan's scratch) fits in the memory budget and, with a GPU executor, in
  the device memory free at that moment (read live, less a reserve);
  otherwise it waits, in arrival order;
* batching: whenever one of the compute streams is idle, all admitted,
  unstarted requests (up to ``max_batch_jobs``) go out as ONE
  ``zkntt_execute_batch`` launch on that stream; with two streams, a batch
  formed from late arrivals overlaps the previous one on the device;
* solo launches: a request of 2^solo_log_n elements or more (when the engine
  is given ``solo_log_n``), or a batch that would hold a single request, runs
  as a plain transform instead (an executor's ``launch_solo``): a large
  transform fills the GPU by itself and runs faster through the plain pass
  kernels, and a lone small one skips the batch launch's setup.  Large
  requests keep their arrival order among themselves; small ones behind a
  large one at the head of the queue may go out first, in the next batch;
* completion: each request retires as soon as its own transform is done (the
  launch writes a per-transform completion word to host-mapped memory), which
  returns its memory to the budget; the stream is reused once the launch's
  CUDA event completes; latency = retire time - arrival time.

Every GPU step runs in the library's kernels; this module only decides what
to launch and when.  The scheduling logic is independent of the device: the
executor is an object with ``launch(requests, stream) -> token``,
``done(token)``, ``finished(token, request)`` and ``release(request)``, so it
is tested on the CPU with a simulated executor.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass

KINDS = ("ntt", "intt", "coset_ntt", "coset_intt")


@dataclass
class Request:
    rid: int
    arrival_s: float
    field: str
    log_n: int
    kind: str
    seed: int = 0
    # filled in by the engine
    admit_s: float = math.nan
    launch_s: float = math.nan
    finish_s: float = math.nan
    out: object = None
    payload: object = None

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def latency_s(self) -> float:
        return self.finish_s - self.arrival_s


def footprint_bytes(log_n: int) -> int:
    """Device bytes a request may hold while admitted, when the executor cannot
    say exactly: its output vector plus one vector of scratch (the most a plan
    of any schedule takes from the pool)."""
    n = 1 << log_n
    return 32 * n + 32 * n


@dataclass
class ServeStats:
    requests: int
    elements: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    melem_s: float
    batches: int
    mean_batch_jobs: float
    max_inflight_batches: int
    peak_bytes: int

    def as_dict(self) -> dict:
        return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in self.__dict__.items()}


def percentile(values, q: float) -> float:
    if not values:
        return math.nan
    s = sorted(values)
    k = (len(s) - 1) * q
    lo, hi = math.floor(k), math.ceil(k)
    return s[lo] + (s[hi] - s[lo]) * (k - lo)


class Engine:
    """Continuous-batching scheduler over an executor (see module docstring)."""

    def __init__(self, executor, budget_bytes: int, streams: int = 2, max_batch_jobs: int = 64,
                 clock=time.perf_counter, idle_sleep_s: float = 20e-6, solo_log_n: int | None = None):
        if streams < 1 or max_batch_jobs < 1 or budget_bytes <= 0:
            raise ValueError("bad engine configuration")
        self.ex = executor
        self.budget = budget_bytes
        self.streams = streams
        self.max_batch_jobs = max_batch_jobs
        self.clock = clock
        self.idle_sleep_s = idle_sleep_s
        self.solo_log_n = solo_log_n
        self.can_solo = hasattr(executor, "launch_solo")

    def _footprint(self, r: Request) -> int:
        fp = getattr(self.ex, "footprint", None)
        return fp(r) if fp is not None else footprint_bytes(r.log_n)

    def _is_big(self, r: Request) -> bool:
        return self.can_solo and self.solo_log_n is not None and r.log_n >= self.solo_log_n

    def _next_launch(self, ready: deque) -> tuple[list[Request], bool]:
        """Requests for the next launch and whether it is a solo launch."""
        if self._is_big(ready[0]):
            return [ready.popleft()], True
        take, skipped = [], []
        while ready and len(take) < self.max_batch_jobs:
            r = ready.popleft()
            (skipped if self._is_big(r) else take).append(r)
        ready.extendleft(reversed(skipped))    # large ones keep their place
        return take, self.can_solo and len(take) == 1

    def run(self, requests, realtime: bool = True) -> tuple[list[Request], ServeStats]:
        """Serve `requests` (arrival times relative to the start).  With
        realtime=False, arrivals are released as fast as the loop turns (a
        closed test)."""
        arrivals = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
        for r in arrivals:
            r._fp = self._footprint(r)
            if r._fp > self.budget:
                raise ValueError(f"request {r.rid} (2^{r.log_n}) can never fit the memory budget")
        headroom = getattr(self.ex, "headroom_bytes", None)
        waiting: deque[Request] = deque()      # arrived, not admitted
        ready: deque[Request] = deque()        # admitted, not launched
        inflight: list = []     # (token, stream, requests, not yet retired) per busy stream
        free_streams = list(range(self.streams))
        used = 0
        peak = 0
        done: list[Request] = []
        batches = 0
        batch_sizes = []
        max_inflight = 0
        i = 0
        t0 = self.clock()
        while len(done) < len(arrivals):
            now = self.clock() - t0
            # arrivals
            while i < len(arrivals) and (not realtime or arrivals[i].arrival_s <= now):
                waiting.append(arrivals[i])
                i += 1
            # retire finished requests (each as soon as its own result is
            # ready), then free streams whose whole launch has completed
            still = []
            for token, stream, reqs, live in inflight:
                fin = None
                for r in list(live):
                    if self.ex.finished(token, r):
                        if fin is None:
                            fin = self.clock() - t0
                        r.finish_s = fin
                        used -= r._fp
                        self.ex.release(r)
                        done.append(r)
                        live.remove(r)
                if not live and self.ex.done(token):
                    free_streams.append(stream)
                else:
                    still.append((token, stream, reqs, live))
            inflight = still
            # admission in arrival order while memory allows: within the
            # budget, and (with a live executor) within the device memory
            # free right now, less what admitted but unlaunched requests will
            # still take
            if waiting and used + waiting[0]._fp <= self.budget:
                live = headroom() - sum(q._fp for q in ready) if headroom is not None else None
                while waiting and used + waiting[0]._fp <= self.budget and \
                        (live is None or waiting[0]._fp <= live):
                    r = waiting.popleft()
                    r.admit_s = self.clock() - t0
                    used += r._fp
                    if live is not None:
                        live -= r._fp
                    peak = max(peak, used)
                    ready.append(r)
            # launch: everything ready goes out on an idle stream
            while ready and free_streams:
                stream = free_streams.pop(0)
                take, solo = self._next_launch(ready)
                launch = self.clock() - t0
                for r in take:
                    r.launch_s = launch
                token = self.ex.launch_solo(take[0], stream) if solo else self.ex.launch(take, stream)
                inflight.append((token, stream, take, list(take)))
                batches += 1
                batch_sizes.append(len(take))
                max_inflight = max(max_inflight, len(inflight))
            if not ready and (not inflight or all(not self.ex.done(t) for t, _, _, _ in inflight)):
                if i < len(arrivals) or inflight:
                    if self.idle_sleep_s > 0:
                        time.sleep(self.idle_sleep_s)
        wall = self.clock() - t0
        lat = [r.latency_s * 1e3 for r in done]
        elems = sum(r.n for r in done)
        stats = ServeStats(
            requests=len(done), elements=elems, wall_s=wall,
            p50_ms=percentile(lat, 0.50), p99_ms=percentile(lat, 0.99),
            mean_ms=sum(lat) / len(lat) if lat else math.nan,
            melem_s=elems / wall / 1e6 if wall > 0 else math.nan,
            batches=batches, mean_batch_jobs=sum(batch_sizes) / max(1, len(batch_sizes)),
            max_inflight_batches=max_inflight, peak_bytes=peak)
        done.sort(key=lambda r: r.rid)
        return done, stats


def serve_serial(requests, run_one, clock=time.perf_counter, realtime: bool = True):
    """Baseline: one request at a time in arrival order, each as a plain
    transform (`run_one(request)` returns when the result is ready)."""
    arrivals = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
    t0 = clock()
    for r in arrivals:
        now = clock() - t0
        if realtime and r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        r.launch_s = clock() - t0
        run_one(r)
        r.finish_s = clock() - t0
    wall = clock() - t0
    lat = [r.latency_s * 1e3 for r in arrivals]
    elems = sum(r.n for r in arrivals)
    return arrivals, ServeStats(
        requests=len(arrivals), elements=elems, wall_s=wall,
        p50_ms=percentile(lat, 0.5), p99_ms=percentile(lat, 0.99),
        mean_ms=sum(lat) / max(1, len(lat)), melem_s=elems / wall / 1e6,
        batches=len(arrivals), mean_batch_jobs=1.0, max_inflight_batches=1, peak_bytes=0)


class GpuExecutor:
    """Executor over the library: resident plans and input vectors, one
    persistent batch launch per call (shortest transforms first) or one plain
    transform per solo call, per-request completion words in host-mapped
    memory for batches, a CUDA event per launch."""

    def __init__(self, device=0, streams: int = 2, input_pool=None, keep_outputs: bool = True,
                 flag_slots: int = 4096, reserve_bytes: int = 2 << 30):
        import torch

        import paper_2509_22684_gb300 as zk
        self.torch = torch
        self.zk = zk
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.plans = {}
        self.inputs = input_pool if input_pool is not None else {}
        self.keep_outputs = keep_outputs
        self.flags = zk.CompletionFlags(flag_slots)
        self.next_slot = 0
        self.epoch = 0
        self.reserve = reserve_bytes

    def footprint(self, r: Request) -> int:
        """Device bytes the request takes while admitted: its output vector and
        the scratch its own plan needs (zkntt_plan_scratch_bytes)."""
        p = self.plan(r.field, r.log_n, r.kind)
        return 32 * p.n + p.scratch_bytes()

    def headroom_bytes(self) -> int:
        """Device memory the engine may still admit against, read live: free
        device memory, plus what torch's caching allocator and the library's
        scratch pool hold but have not handed out, less a reserve."""
        torch = self.torch
        free, _ = torch.cuda.mem_get_info(self.device)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        pool_reserved, pool_used = self.zk.pool_info()
        return free + cached + (pool_reserved - pool_used) - self.reserve

    def plan(self, field_name: str, log_n: int, kind: str):
        key = (field_name, log_n, kind)
        p = self.plans.get(key)
        if p is None:
            _, g, _ = self.zk.field_info(field_name)
            p = self.zk.Plan(field_name, log_n, inverse=kind.endswith("intt"),
                             coset_shift=g if kind.startswith("coset") else None)
            self.plans[key] = p
        return p

    def input_for(self, r: Request):
        if r.payload is not None:
            return r.payload
        return self.inputs[(r.field, r.log_n)]

    def launch(self, reqs, stream_index: int):
        torch = self.torch
        s = self.streams[stream_index]
        plans, ins, outs = [], [], []
        for r in reqs:
            plans.append(self.plan(r.field, r.log_n, r.kind))
            x = self.input_for(r)
            ins.append(x)
            with torch.cuda.stream(s):
                r.out = torch.empty_like(x)
            outs.append(r.out)
        if self.next_slot + len(reqs) > self.flags.count:
            self.next_slot = 0   # slots are free again: in flight << flag_slots
        base = self.next_slot
        self.next_slot += len(reqs)
        self.epoch = (self.epoch + 1) & 0xFFFFFFFF or 1
        for i, r in enumerate(reqs):
            r._slot = base + i
            r._epoch = self.epoch
        self.zk.execute_batch_signal(plans, ins, outs, self.flags, list(range(base, base + len(reqs))),
                                     self.epoch, stream=s)
        ev = torch.cuda.Event()
        ev.record(s)
        return ev, False

    def launch_solo(self, r: Request, stream_index: int):
        """One request as a plain transform (zkntt_execute); it is finished
        when the launch's event has completed."""
        torch = self.torch
        s = self.streams[stream_index]
        x = self.input_for(r)
        with torch.cuda.stream(s):
            r.out = torch.empty_like(x)
        self.plan(r.field, r.log_n, r.kind).execute(x, r.out, stream=s)
        ev = torch.cuda.Event()
        ev.record(s)
        return ev, True

    def done(self, token) -> bool:
        return token[0].query()

    def finished(self, token, r: Request) -> bool:
        ev, solo = token
        return ev.query() if solo else self.flags[r._slot] == r._epoch

    def release(self, r: Request):
        if not self.keep_outputs:
            r.out = None  # back to the caching allocator (the stream's work is done with it)

    def close(self):
        for p in self.plans.values():
            p.close()
        self.plans.clear()
        self.flags.close()
