#!/usr/bin/env python
"""Benchmark of the NTT library on GB300.

Workload (one step): one forward NTT over BLS12-381 F_r, n = 2^24 elements
(512 MiB per vector, larger than the 129 MB L2, so no flush is needed),
natural-order input in Montgomery form, uniform random elements from a seed.
Metric: NTT Melem/s = n / time per transform.

Prints ONE JSON line (rank 0).  Under torchrun every rank runs the same
transform on its own GPU (replicas: the transforms are independent units, no
data-path collective); `value` is the sum over ranks computed from the slowest
rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

IMAD_PER_MUL = 264          # 8 x 32-bit CIOS: 8 x (16 + 1 + 16) multiply-adds
IMAD_LANES_PER_SM_CLK = 64  # 32-bit integer multiply-add issue rate per SM per clock
METRIC = "NTT Melem/s (BLS12-381 Fr, 2^24 forward) + % int/HBM roofline"
FIELD_IDS = {"bls12_381_fr": 0, "bn254_fr": 1, "bls12_377_fr": 2}
FIELD_R = {
    "bls12_381_fr": 0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001,
    "bn254_fr": 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001,
    "bls12_377_fr": 0x12AB655E9A2CA55660B44D1E5C37B00159AA76FED00000010A11800000000001,
}


def butterfly_mults(log_n: int) -> int:
    """Non-trivial twiddle multiplications of a radix-2 NTT: (n/2) log n - (n - 1)."""
    n = 1 << log_n
    return (n // 2) * log_n - (n - 1)


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# the sources the timed pass kernel is compiled from (BLS12-381 instantiation)
PASS_KERNEL_SOURCES = ("field.cuh", "ntt_pass.cuh", "kernels_bls12_381.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_22684_gb300", "csrc")
    for name in PASS_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def tuned_schedule(field_id: int, log_n: int, direction: int = 0) -> str:
    """The shipped tuned entry the plan uses (digits, columns, variant,
    twiddle mode), as a canonical string; "default" if none."""
    try:
        with open(os.path.join(ROOT, "paper_2509_22684_gb300", "zkntt_tuned.jsonl")) as f:
            for line in f:
                e = json.loads(line)
                if (e.get("field"), e.get("log_n"), e.get("dir")) == (field_id, log_n, direction):
                    p = e["passes"]
                    return json.dumps({"digits": e["digits"][:p], "log_cols": e["log_cols"][:p],
                                       "ilp": e["ilp"], "mode": e["mode"]}, sort_keys=True)
    except (OSError, ValueError, KeyError):
        pass
    return "default"


def recorded_traffic(kernel_hash: str, workload: str, schedule: str):
    """dram bytes per launch recorded from an ncu capture of the same pass
    kernel sources running the same schedule (profiles/ntt_traffic.json);
    None if absent or stale."""
    try:
        with open(os.path.join(ROOT, "profiles", "ntt_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    e = rec.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash or e.get("schedule") != schedule:
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; only the
    samples whose timestamps fall inside the timed region count (the nearest
    later one if the region is shorter than the sampling interval)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
             "timestamp")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="zkntt_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        deadline = time.time() + 3.0        # wait for the sampler's first line
        while time.time() < deadline and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(s: str):
        import datetime
        try:
            return datetime.datetime.strptime(s.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if self.t0 is not None and self.t1 is not None and rows:
            stamped = [(self._stamp(r[9]), r) for r in rows]
            inside = [r for t, r in stamped if t is not None and self.t0 <= t <= self.t1 + 0.01]
            later = [r for t, r in stamped if t is not None and t > self.t1]
            rows = inside or later[:1] or rows[-1:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    from paper_2509_22684_gb300.replicas import max_over_ranks as mor
    return mor(value, device="cuda")


def cpu_oracle_rate(field: str, log_n: int, budget_s: float, X=None):
    """The C oracle (as it stands) on the host cores: Melem/s of forward NTTs of
    2^log_n, repeated until `budget_s` is spent (at least once)."""
    from oracle import cpu
    from oracle import field as fld
    from workloads import uniform_elements
    F = fld.get(field)
    if X is None:
        X = uniform_elements(F.r, 1 << log_n, 2024)
    threads = cpu.threads_default()
    reps, t0 = 0, time.perf_counter()
    while True:
        cpu.ntt(F, X, threads=threads)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 50:
            break
    return (reps << log_n) / el / 1e6, threads, reps, el


def host_link_gbs(torch, h_in, h_out, d_buf, d_buf2, reps: int = 3):
    """Pinned host <-> device copy bandwidth (GB/s) for one vector: each
    direction alone, then both at once on two streams (aggregate), timed with
    CUDA events.  The two directions overlap only where the device has a copy
    engine for each."""
    s = torch.cuda.Stream()
    out = []
    for direction in ("h2d", "d2h"):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            for k in range(reps + 1):
                if k == 1:
                    e0.record(s)
                if direction == "h2d":
                    d_buf.copy_(h_in, non_blocking=True)
                else:
                    h_out.copy_(d_buf, non_blocking=True)
            e1.record(s)
        e1.synchronize()
        out.append(round(reps * h_in.numel() * h_in.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9, 1))
    s2 = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(s):
        for _ in range(reps):
            d_buf.copy_(h_in, non_blocking=True)
    with torch.cuda.stream(s2):
        for _ in range(reps):
            h_out.copy_(d_buf2, non_blocking=True)
    torch.cuda.synchronize()
    out.append(round(2 * reps * h_in.numel() * h_in.element_size() / (time.perf_counter() - t0) / 1e9, 1))
    return out


def timed(fn, stream, steps: int) -> float:
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def measured_imad_peak(zk, torch, sms: int, stream) -> dict:
    """The 32-bit multiply-add rate of this GPU, measured in this process with
    the library's calibration kernel (zkntt_imadbench): eight independent
    register chains per thread, 2048 threads per SM; best of three timed
    launches after a warm-up, for mad.lo.u32 (the peak) and for the other
    multiply forms a product is built from (zkntt_imadbench's modes); the
    carry-chained pair counts one step per pair."""
    blocks, threads, iters = sms * 8, 256, 1 << 16
    sink = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    out = {}
    for mode, name in ((0, "mad_lo_per_s"), (1, "mad_wide_per_s"), (2, "mul_wide_per_s"),
                       (3, "mad_hi_per_s"), (4, "mad_lo_cc_madc_hi_pairs_per_s")):
        zk.imadbench(mode, blocks, threads, iters // 16, sink, stream=stream)
        best = min(timed(lambda: zk.imadbench(mode, blocks, threads, iters, sink, stream=stream),
                         stream, 1) for _ in range(3))
        out[name] = blocks * threads * 8 * iters / (best / 1e3)
    out["config"] = f"{blocks} blocks x {threads} threads x 8 chains x {iters} steps"
    return out


def extras(zk, torch, field: str, stream, peak_imad: float, hbm_gbs: float) -> dict:
    """Other sizes, twiddle modes, and batched vs plain (rank 0, short runs)."""
    import numpy as np
    from workloads import batch_jobs, uniform_elements
    out = {}
    F_r = FIELD_R[field]
    sizes = {}
    for L in (20, 22, 26):
        X = uniform_elements(F_r, 1 << L, 3000 + L)
        x = torch.from_numpy(X.view(np.int32)).cuda()
        y = torch.empty_like(x)
        with zk.Plan(field, L) as p:
            scr = torch.empty(max(8, p.scratch_bytes() // 4), dtype=torch.int32, device="cuda")
            f = lambda: p.execute_scratch(x, y, scr, stream=stream)
            for _ in range(3):
                f()
            steps = 20 if L <= 22 else 5
            ms = timed(f, stream, steps) / steps
            sizes[f"2^{L}"] = {"melem_s": round((1 << L) / ms / 1e3, 1), "ms": round(ms, 4),
                              "alu_frac": round(butterfly_mults(L) * IMAD_PER_MUL / (ms / 1e3) / peak_imad, 4),
                              "hbm_frac": round(64 * (1 << L) / (ms / 1e3) / (hbm_gbs * 1e9), 4),
                              "digits": p.describe()["digits"]}
        del x, y, scr
    out["sizes"] = sizes
    # twiddle modes at 2^24
    L = 24
    X = uniform_elements(F_r, 1 << L, 3024)
    x = torch.from_numpy(X.view(np.int32)).cuda()
    y = torch.empty_like(x)
    modes = {}
    for mode in ("precomp", "otf"):
        with zk.Plan(field, L, twiddle_mode=mode) as p:
            scr = torch.empty(p.scratch_bytes() // 4, dtype=torch.int32, device="cuda")
            f = lambda: p.execute_scratch(x, y, scr, stream=stream)
            for _ in range(3):
                f()
            ms = timed(f, stream, 10) / 10
            modes[mode] = {"melem_s": round((1 << L) / ms / 1e3, 1), "ms": round(ms, 4),
                           "table_mib": round(p.describe()["table_bytes"] / 2**20, 1)}
    out["twiddle_modes_2^24"] = modes
    del x, y
    # Groth16 H at 2^22: seven transforms + pointwise as separate launches vs one fused launch
    L = 22
    a, b, c = (torch.from_numpy(uniform_elements(F_r, 1 << L, s).view(np.int32)).cuda()
               for s in (3001, 3002, 3003))
    h = torch.empty_like(a)
    scr = torch.empty((3 << L, 8), dtype=torch.int32, device="cuda")
    g16 = {}
    for fused in (False, True):
        f = lambda: zk.groth16_h(field, L, a, b, c, h=h, scratch=scr, fused=fused, stream=stream)
        for _ in range(3):
            f()
        ms = timed(f, stream, 10) / 10
        g16["fused_ms" if fused else "separate_ms"] = round(ms, 4)
    gs = torch.cuda.Stream()
    graph = zk.Groth16Graph(field, L, a, b, c, h, scr, stream=gs)
    f = lambda: graph.launch(stream=stream)
    for _ in range(3):
        f()
    g16["graph_ms"] = round(timed(f, stream, 10) / 10, 4)
    graph.close()
    g16["speedup"] = round(g16["separate_ms"] / g16["fused_ms"], 3)
    g16["graph_speedup"] = round(g16["separate_ms"] / g16["graph_ms"], 3)
    out["groth16_2^22"] = g16
    # small Groth16 sizes, where launch overhead matters: separate vs fused graph
    small = {}
    for Ls in (12, 16, 20):
        a2, b2, c2 = (torch.from_numpy(uniform_elements(F_r, 1 << Ls, s).view(np.int32)).cuda()
                      for s in (3001, 3002, 3003))
        h2 = torch.empty_like(a2)
        s2 = torch.empty((3 << Ls, 8), dtype=torch.int32, device="cuda")
        sep = lambda: zk.groth16_h(field, Ls, a2, b2, c2, h=h2, scratch=s2, fused=False, stream=stream)
        for _ in range(3):
            sep()
        ms_sep = timed(sep, stream, 20) / 20
        gr = zk.Groth16Graph(field, Ls, a2, b2, c2, h2, s2, stream=gs)
        fg = lambda: gr.launch(stream=stream)
        for _ in range(3):
            fg()
        ms_g = timed(fg, stream, 20) / 20
        gr.close()
        small[f"2^{Ls}"] = {"separate_ms": round(ms_sep, 4), "graph_ms": round(ms_g, 4),
                            "speedup": round(ms_sep / ms_g, 3)}
    out["groth16_small"] = small
    del a, b, c, h, scr
    # 64 uneven transforms: persistent batch vs one call per transform
    jobs = batch_jobs(4000, count=64, lmin=10, lmax=20)
    plans, xs, ys = [], [], []
    for j in jobs:
        X = uniform_elements(FIELD_R[j.field], 1 << j.log_n, j.seed)
        xs.append(torch.from_numpy(X.view(np.int32)).cuda())
        ys.append(torch.empty_like(xs[-1]))
        plans.append(zk.Plan(j.field, j.log_n, inverse=(j.kind == "intt")))
    scr = [torch.empty(max(8, p.scratch_bytes() // 4), dtype=torch.int32, device="cuda") for p in plans]

    def one_by_one():
        for p, x, y, s in zip(plans, xs, ys, scr):
            p.execute_scratch(x, y, s, stream=stream)

    def persistent():
        zk.execute_batch(plans, xs, ys, stream=stream)
    bt = {}
    for name, f in (("separate_ms", one_by_one), ("persistent_ms", persistent)):
        for _ in range(3):
            f()
        bt[name] = round(timed(f, stream, 10) / 10, 4)
    bt["elements"] = sum(1 << j.log_n for j in jobs)
    bt["speedup"] = round(bt["separate_ms"] / bt["persistent_ms"], 3)
    out["batch64_uneven"] = bt
    for p in plans:
        p.close()
    return out


def serve_bench(zk, torch, field: str, n_requests: int, loads, solo_log_n=None) -> dict:
    """Served NTT stream: Poisson arrivals, log_n uniform on 12..24, kinds
    uniform over {NTT, iNTT, coset NTT, coset iNTT}; for each offered load
    (a fraction of the measured serial capacity), continuous batching vs
    serial plain execution on the same trace."""
    import numpy as np
    from paper_2509_22684_gb300.serve import Engine, GpuExecutor, Request, serve_serial
    from workloads import KINDS, poisson_trace, uniform_elements
    F_r = FIELD_R[field]
    sizes = range(12, 25)
    pool = {(field, L): torch.from_numpy(uniform_elements(F_r, 1 << L, 5000 + L).view(np.int32)).cuda()
            for L in sizes}
    ex = GpuExecutor(streams=2, input_pool=pool, keep_outputs=False)
    cur = torch.cuda.current_stream()
    svc = {}
    for L in sizes:
        for kind in KINDS:
            ex.plan(field, L, kind)
        p = ex.plan(field, L, "ntt")
        x = pool[(field, L)]
        y = torch.empty_like(x)
        for _ in range(2):
            p.execute(x, y, stream=cur)
        svc[L] = timed(lambda: p.execute(x, y, stream=cur), cur, 5) / 5 / 1e3
    mean_svc = sum(svc.values()) / len(svc)

    def run_one(r):
        x = pool[(r.field, r.log_n)]
        ex.plan(r.field, r.log_n, r.kind).execute(x, torch.empty_like(x), stream=cur)
        cur.synchronize()
    out = {"requests": n_requests, "serial_capacity_per_s": round(1 / mean_svc, 1),
           "solo_log_n": solo_log_n}
    for load in loads:
        rate = load / mean_svc
        trace = poisson_trace(5000, n_requests, rate, 12, 24)
        mk = lambda: [Request(i, q.arrival_s, field, q.log_n, q.kind) for i, q in enumerate(trace)]
        # admission: live free device memory less a reserve (the executor's
        # headroom), within the device's total as the outer budget
        eng = Engine(ex, budget_bytes=int(torch.cuda.mem_get_info()[1]), streams=2,
                     max_batch_jobs=64, solo_log_n=solo_log_n)
        _, st = eng.run(mk())
        _, ser = serve_serial(mk(), run_one)
        out[f"load_{load}"] = {"offered_rate_per_s": round(rate, 1),
                               "batched": st.as_dict(), "serial": ser.as_dict(),
                               "p50_speedup": round(ser.p50_ms / st.p50_ms, 3),
                               "p99_speedup": round(ser.p99_ms / st.p99_ms, 3),
                               "throughput_ratio": round(st.melem_s / ser.melem_s, 3)}
    ex.close()
    return out


def groth16_only(args) -> None:
    """Groth16 H at 2^L: the fused persistent launch in a CUDA graph and the
    seven transforms + pointwise issued separately, both after warm-up, with
    CUDA events (one JSON line; rank 0 only)."""
    import numpy as np
    import torch

    import paper_2509_22684_gb300 as zk
    from workloads import uniform_elements
    field, L = args.field, args.groth16
    stream = torch.cuda.current_stream()
    a, b, c = (torch.from_numpy(uniform_elements(FIELD_R[field], 1 << L, s).view(np.int32)).cuda()
               for s in (3001, 3002, 3003))
    h = torch.empty_like(a)
    scr = torch.empty((3 << L, 8), dtype=torch.int32, device="cuda")
    gs = torch.cuda.Stream()
    graph = zk.Groth16Graph(field, L, a, b, c, h, scr, stream=gs)
    fused = lambda: graph.launch(stream=stream)
    sep = lambda: zk.groth16_h(field, L, a, b, c, h=h, scratch=scr, fused=False, stream=stream)
    out = {"workload": f"groth16_h {field} n=2^{L}", "steps": args.steps, "warmup": args.warmup}
    for name, f in (("fused_graph_ms", fused), ("separate_ms", sep)):
        for _ in range(args.warmup):
            f()
        out[name] = round(timed(f, stream, args.steps) / args.steps, 4)
    graph.close()
    zk.sync_status(stream)
    out["speedup"] = round(out["separate_ms"] / out["fused_graph_ms"], 3)
    print(json.dumps(out), flush=True)


def calibrate(args) -> None:
    """The multiply forms and the Montgomery product on their own (one JSON
    line): zkntt_imadbench's five modes and zkntt_mulbench for the field."""
    import torch

    import paper_2509_22684_gb300 as zk
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {"forms_per_s_T": {k: round(v / 1e12, 3)
                              for k, v in measured_imad_peak(zk, torch, sms, stream).items()
                              if k.endswith("_per_s")}}
    blocks, threads, iters = sms * 8, 256, 256
    sink = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    zk.mulbench(args.field, blocks, threads, 8, sink, stream=stream)
    best = min(timed(lambda: zk.mulbench(args.field, blocks, threads, iters, sink, stream=stream),
                     stream, 1) for _ in range(3))
    out["mulbench_products_per_s_G"] = round(blocks * threads * 4 * iters / (best / 1e3) / 1e9, 2)
    out["field"] = args.field
    out["library"] = os.environ.get("ZKNTT_LIB", "paper_2509_22684_gb300/libzkntt.so")
    print(json.dumps(out), flush=True)


def sharded_emulated(args) -> None:
    """One transform of 2^L split over G shards (paper_2509_22684_gb300.sharded),
    all shards run in this process on this GPU with the exchange done by
    copies, against the plain transform of the same size (one JSON line).  It
    measures the sharded algorithm's own device work on one GPU, not a
    multi-GPU run."""
    import numpy as np
    import torch

    import paper_2509_22684_gb300 as zk
    from paper_2509_22684_gb300.sharded import LibraryOps, ShardedNTT, emulate, scatter_input
    from workloads import uniform_elements
    field, L, G = args.field, args.log_n, args.sharded
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(uniform_elements(FIELD_R[field], 1 << L, 2024).view(np.int32)).cuda()
    ops = LibraryOps(field)
    shards = [ShardedNTT(field, L, G, r, ops=ops) for r in range(G)]
    xs = scatter_input(x, G)
    plan = zk.Plan(field, L)
    out = {"workload": f"{field} forward NTT n=2^{L}", "shards": G, "steps": args.steps}
    for name, f in (("plain_ms", lambda: plan.execute(x)), ("sharded_emulated_ms", lambda: emulate(shards, xs))):
        for _ in range(args.warmup):
            f()
        out[name] = round(timed(f, stream, args.steps) / args.steps, 4)
    out["ratio"] = round(out["sharded_emulated_ms"] / out["plain_ms"], 3)
    plan.close()
    ops.close()
    print(json.dumps(out), flush=True)


def sweep(args) -> None:
    """One JSON line per (field, kind, log_n, twiddle mode): the full grid of
    single-transform configurations, device-resident inputs, CUDA-event
    timing after warm-up (rank 0 only, no other output)."""
    import numpy as np
    import torch

    import paper_2509_22684_gb300 as zk
    from workloads import KINDS, uniform_elements
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak_imad = sms * IMAD_LANES_PER_SM_CLK * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    sizes = [int(v) for v in args.sweep_sizes.split(",")]
    # warm the GPU up (clocks, allocator, module load) before the first cell
    warm = torch.from_numpy(uniform_elements(FIELD_R["bls12_381_fr"], 1 << 22, 1).view(np.int32)).cuda()
    with zk.Plan("bls12_381_fr", 22) as p:
        t_end = time.time() + 1.0
        while time.time() < t_end:
            p.execute(warm)
        torch.cuda.synchronize()
    del warm
    for field in args.sweep_fields.split(","):
        _, g, _ = zk.field_info(field)
        for L in sizes:
            X = uniform_elements(FIELD_R[field], 1 << L, 2000 + L)
            x = torch.from_numpy(X.view(np.int32)).cuda()
            y = torch.empty_like(x)
            for kind in KINDS:
                for mode in ("precomp", "otf"):
                    with zk.Plan(field, L, inverse=kind.endswith("intt"),
                                 coset_shift=g if kind.startswith("coset") else None,
                                 twiddle_mode=mode) as p:
                        scr = torch.empty(max(8, p.scratch_bytes() // 4), dtype=torch.int32,
                                          device="cuda")
                        f = lambda: p.execute_scratch(x, y, scr, stream=stream)
                        for _ in range(3):
                            f()
                        steps = 20 if L <= 22 else 5
                        ms = timed(f, stream, steps) / steps
                        d = p.describe()
                        # coset and inverse add one product per element to the
                        # algorithmic count (the pre- or post-scale)
                        mults = butterfly_mults(L) + ((1 << L) if kind != "ntt" else 0)
                        print(json.dumps({"field": field, "kind": kind, "log_n": L, "mode": mode,
                                          "ms": round(ms, 4), "melem_s": round((1 << L) / ms / 1e3, 1),
                                          "alu_frac": round(mults * IMAD_PER_MUL / (ms / 1e3) / peak_imad, 4),
                                          "digits": d["digits"],
                                          "table_mib": round(d["table_bytes"] / 2**20, 1)}), flush=True)
                        del scr
            del x, y
    zk.sync_status(stream)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2509_22684_gb300 as zk
    from workloads import uniform_elements

    field, L = args.field, args.log_n
    n = 1 << L
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_imad = sms * IMAD_LANES_PER_SM_CLK * sm_max_mhz * 1e6
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    stream = torch.cuda.current_stream()

    X = uniform_elements(FIELD_R[field], n, 2024 + rank)
    x = torch.from_numpy(X.view(np.int32)).cuda()
    y = torch.empty_like(x)
    if args.variant:
        # force a pass-kernel variant on the shipped digit split and columns
        sched = json.loads(tuned_schedule(FIELD_IDS[field], L))
        plan = zk.Plan(field, L, digits=sched["digits"], cols=[1 << c for c in sched["log_cols"]],
                       ilp=args.variant, twiddle_mode={1: "precomp", 2: "otf"}[sched["mode"]])
    else:
        plan = zk.Plan(field, L)
    desc = plan.describe()
    scratch = torch.empty(plan.scratch_bytes() // 4, dtype=torch.int32, device="cuda")
    step = lambda: plan.execute_scratch(x, y, scratch, stream=stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("ZKNTT_SMI_INDEX", local)))
    clocks.start()
    clocks.mark_start()
    ms_total = timed(step, stream, args.steps)
    torch.cuda.synchronize()
    clocks.mark_end()
    clk = clocks.stop()
    barrier(world)
    ms_max = max_over_ranks(world, ms_total)
    zk.sync_status(stream)

    # end to end through the host-buffer entry point (zkntt_execute_host):
    # pinned host input and output, H2D + transform + D2H inside the timed
    # region for every step.  Steps rotate over four streams, so one step's
    # copies overlap another step's transform (the link is full duplex).
    nstreams = 4
    e2e_streams = [torch.cuda.Stream() for _ in range(nstreams)]
    xh = torch.from_numpy(X.view(np.int32)).pin_memory()
    yhs = [torch.empty_like(xh).pin_memory() for _ in range(nstreams)]
    works = [torch.empty(plan.work_bytes() // 4, dtype=torch.int32, device="cuda")
             for _ in range(nstreams)]
    k = [0]

    def e2e_step():
        i = k[0] % nstreams
        k[0] += 1
        plan.execute_host_buffered(xh, yhs[i], works[i], stream=e2e_streams[i])

    def e2e_run(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            e2e_step()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3

    e2e_run(max(3, min(args.warmup, 6)))
    barrier(world)
    e2e_steps = max(8, min(args.steps, 24))
    ms_e2e = max_over_ranks(world, e2e_run(e2e_steps))
    ok = all(bool(np.array_equal(yh.numpy().view(np.uint32), y.cpu().numpy().view(np.uint32)))
             for yh in yhs)
    link = host_link_gbs(torch, xh, yhs[0], x, y)

    imad = measured_imad_peak(zk, torch, sms, stream)
    passes = desc["passes"]
    avg_launch_s = ms_total / 1e3 / (args.steps * passes)
    alg_imad_per_launch = butterfly_mults(L) * IMAD_PER_MUL / passes
    achieved = alg_imad_per_launch / avg_launch_s
    value = world * n * args.steps / (ms_max / 1e3) / 1e6
    workload = f"{field} forward NTT n=2^{L}"
    khash = kernel_source_hash()
    traffic = None if args.variant else recorded_traffic(khash, workload,
                                                         tuned_schedule(FIELD_IDS[field], L))
    result = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "Melem/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32 (8x32-bit limb Montgomery F_r, exact)",
        "data": "synthetic (SplitMix64 uniform field elements, seed 2024+rank)",
        "config": {"workload": workload, "field": field, "log_n": L, "direction": "forward",
                   "variant": args.variant or "shipped schedule",
                   "passes": passes, "digits": desc["digits"], "twiddle_mode": desc["twiddle_mode"],
                   "l2": "inputs larger than L2 (512 MiB per vector vs 129 MB)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": round(achieved / 1e12, 3),
                     "peak": round(peak_imad / 1e12, 3), "unit": "TIMAD/s",
                     "frac": round(achieved / peak_imad, 4),
                     # against the multiply-add rate measured in this run
                     # (independent mad.lo.u32 chains; zkntt_imadbench)
                     "peak_measured": round(imad["mad_lo_per_s"] / 1e12, 3),
                     "frac_measured": round(achieved / imad["mad_lo_per_s"], 4),
                     "forms_measured_per_s": {k: round(v / 1e12, 3) for k, v in imad.items()
                                              if k.endswith("_per_s")},
                     "peak_measured_config": imad["config"],
                     "traffic": traffic,
                     "kernel": "ntt_pass_kernel (all passes of one transform)",
                     "peak_source": f"derived: {sms} SMs x {IMAD_LANES_PER_SM_CLK} IMAD/clk x {sm_max_mhz:.0f} MHz",
                     "hbm_frac": round(64 * n / (ms_max / args.steps / 1e3) / (hbm_gbs * 1e9), 4),
                     "hbm_peak_gbs": hbm_gbs},
        "e2e": {"value": round(world * n * e2e_steps / (ms_e2e / 1e3) / 1e6, 2), "unit": "Melem/s",
                "h2d_bytes_per_step": 32 * n, "d2h_bytes_per_step": 32 * n,
                "api": "zkntt_execute_host_buffered (pinned host buffers, one device work buffer per stream, steps over 4 streams)",
                "timing": "host wall clock around the steps with device synchronisation on both sides",
                "matches_device_result": ok,
                # pinned-copy bandwidth of this machine, one direction at a time: the
                # copies of a step are hidden behind its transform only while
                # 32n bytes each way take less than the transform
                "link_h2d_gbs": link[0], "link_d2h_gbs": link[1],
                "link_both_directions_gbs": link[2]},
        "gpu_launches": args.steps * passes,
        "clocks": clk,
    }
    plan.close()
    del x, y, scratch
    if rank == 0 and not args.no_cpu:
        rate, cores, reps, el = cpu_oracle_rate(field, L, args.cpu_budget, X)
        result["cpu_baseline"] = {"value": round(rate, 3), "unit": "Melem/s", "cores": cores,
                                  "kind": "oracle",
                                  "sample": f"C oracle (oracle/cpu_ntt.c) forward NTT 2^{L}, {reps} run(s), {el:.1f} s"}
    if rank == 0 and not args.no_extras:
        result["extras"] = extras(zk, torch, field, stream, peak_imad, hbm_gbs)
        loads = [float(v) for v in args.serve_loads.split(",") if v]
        result["extras"]["serving"] = serve_bench(zk, torch, field, args.serve_requests, loads,
                                                  args.serve_solo_log_n)
    if rank == 0:
        print(json.dumps(result), flush=True)


def run_reference(args, world, rank):
    """The oracle as it stands, timed on the host cores: each step is one
    forward transform of the same workload (a smaller size if the full one
    would not finish the run within a few minutes)."""
    if rank != 0:
        return
    from oracle import cpu
    from oracle import field as fld
    from workloads import uniform_elements
    field = args.field
    F = fld.get(field)
    L = args.log_n
    # one probe run sizes the sample
    X = uniform_elements(F.r, 1 << L, 2024)
    threads = cpu.threads_default()
    t0 = time.perf_counter()
    cpu.ntt(F, X, threads=threads)
    per = time.perf_counter() - t0
    total_runs = args.steps + args.warmup
    while per * total_runs > 180 and L > 16:
        L -= 2
        per /= 4.4
    if L != args.log_n:
        X = uniform_elements(F.r, 1 << L, 2024)
    for _ in range(args.warmup):
        cpu.ntt(F, X, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu.ntt(F, X, threads=threads)
    el = time.perf_counter() - t0
    value = (args.steps << L) / el / 1e6
    sample = f"C oracle forward NTT 2^{L} per step on {threads} host threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Melem/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 limbs (exact)",
        "data": "synthetic", "config": {"workload": f"{field} forward NTT n=2^{args.log_n}",
                                        "sample_log_n": L},
        "cpu_baseline": {"value": round(value, 3), "unit": "Melem/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "Melem/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--field", default="bls12_381_fr", choices=sorted(FIELD_R))
    ap.add_argument("--log-n", type=int, default=24)
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-loads", default="0.5,0.8,0.95",
                    help="offered loads, as fractions of the serial capacity")
    ap.add_argument("--serve-solo-log-n", type=int, default=20,
                    help="served requests of at least 2^this run as plain transforms")
    ap.add_argument("--sweep", action="store_true",
                    help="print one line per field x kind x size x twiddle mode instead")
    ap.add_argument("--sweep-sizes", default="16,20,22,24,26")
    ap.add_argument("--sweep-fields", default="bls12_381_fr,bn254_fr,bls12_377_fr")
    ap.add_argument("--variant", type=int, default=0,
                    help="force pass-kernel variant V on the shipped digit split (study runs)")
    ap.add_argument("--calibrate", action="store_true",
                    help="print the multiply-form and product rates instead")
    ap.add_argument("--sharded", type=int, default=0, metavar="G",
                    help="time the sharded transform's G shards emulated on this GPU instead")
    ap.add_argument("--groth16", type=int, default=0, metavar="L",
                    help="time only the Groth16 H sequence at 2^L (fused graph vs separate)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    if args.sweep:
        sweep(args)
        return
    if args.groth16:
        groth16_only(args)
        return
    if args.calibrate:
        calibrate(args)
        return
    if args.sharded:
        sharded_emulated(args)
        return
    world, rank, local = dist_init(args)
    try:
        run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
