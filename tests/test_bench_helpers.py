"""Host-side helpers of bench.py (no GPU): the traffic record is used only
for the same pass-kernel sources and schedule, the tuned-schedule lookup reads
the shipped table, clock samples are kept only inside the timed region."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_tuned_schedule_matches_shipped_table():
    sch = bench.tuned_schedule(0, 24)
    assert sch != "default"
    d = json.loads(sch)
    with open(os.path.join(ROOT, "paper_2509_22684_gb300", "zkntt_tuned.jsonl")) as f:
        rows = [json.loads(l) for l in f]
    e = [r for r in rows if (r["field"], r["log_n"], r["dir"]) == (0, 24, 0)][0]
    assert d["digits"] == e["digits"][:e["passes"]] and sum(d["digits"]) == 24
    assert bench.tuned_schedule(0, 99) == "default"


def test_recorded_traffic_requires_same_sources_and_schedule():
    h = bench.kernel_source_hash()
    sch = bench.tuned_schedule(0, 24)
    w = "bls12_381_fr forward NTT n=2^24"
    with open(os.path.join(ROOT, "profiles", "ntt_traffic.json")) as f:
        rec = json.load(f)[w]
    got = bench.recorded_traffic(h, w, sch)
    if rec["kernel_hash"] == h and rec["schedule"] == sch:
        assert got == rec["dram_bytes_per_launch"] and got > 0
    else:
        assert got is None                       # stale record: reported as null
    assert bench.recorded_traffic("0" * 16, w, sch) is None
    assert bench.recorded_traffic(h, w, "default") is None or sch == "default"
    assert bench.recorded_traffic(h, "no such workload", sch) is None


def test_kernel_source_hash_covers_the_pass_kernel_sources():
    assert bench.PASS_KERNEL_SOURCES == ("field.cuh", "ntt_pass.cuh", "kernels_bls12_381.cu")
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert bench.kernel_source_hash() == h      # deterministic


def test_clock_sampler_keeps_only_samples_inside_the_timed_region(tmp_path):
    s = bench.ClockSampler(0)
    base = 1_800_000_000.0
    import datetime

    def line(t, mhz):
        stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"0, {mhz}, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active, {stamp}\n"
    p = tmp_path / "clocks.csv"
    p.write_text(line(base - 1.0, 900) + line(base + 0.10, 2070) + line(base + 0.20, 2060)
                 + line(base + 2.0, 1000))
    s.path = str(p)

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    s.proc = Done()
    s.t0, s.t1 = base, base + 0.5
    out = s.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2065.0 and out["reasons"] == []


def test_clock_sampler_falls_back_to_the_next_sample_after_a_short_region(tmp_path):
    s = bench.ClockSampler(0)
    base = 1_800_000_000.0
    import datetime
    stamp = lambda t: datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    p = tmp_path / "clocks.csv"
    p.write_text(f"0, 1500, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active, {stamp(base - 0.3)}\n"
                 f"0, 2070, 2070, 300.0, 0x4, Not Active, Not Active, Not Active, Active, {stamp(base + 0.08)}\n")
    s.path = str(p)

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    s.proc = Done()
    s.t0, s.t1 = base, base + 0.02              # shorter than the sampling interval
    out = s.stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"]
