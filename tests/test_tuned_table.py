"""The shipped schedule table parses in the exact line format the library's
loader reads (csrc/tuner.cu reads each line with one fixed scanf format and
silently skips lines that do not match), covers every field, direction and
size 2^10..2^28 the tuner runs, and every entry is a valid schedule."""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_2509_22684_gb300", "zkntt_tuned.jsonl")
LINE = re.compile(
    r'^\{"gpu":"[^"]+","field":\d+,"log_n":\d+,"dir":\d+,"passes":\d+,'
    r'"digits":\[-?\d+,-?\d+,-?\d+,-?\d+\],"log_cols":\[-?\d+,-?\d+,-?\d+,-?\d+\],'
    r'"mode":\d+,"ilp":\d+,"ms":[0-9.eE+-]+\}$')


def test_every_line_matches_the_loader_format():
    with open(TABLE) as f:
        lines = [l.rstrip("\n") for l in f if l.strip()]
    bad = [l for l in lines if not LINE.match(l)]
    assert not bad, bad[:3]


def test_table_covers_every_field_direction_and_size():
    with open(TABLE) as f:
        rows = [json.loads(l) for l in f if l.strip()]
    keys = {(r["field"], r["dir"], r["log_n"]) for r in rows}
    assert len(keys) == len(rows)                     # no duplicates
    for field in (0, 1, 2):
        for d in (0, 1):
            for L in range(10, 29):
                assert (field, d, L) in keys, (field, d, L)


def test_every_entry_is_a_valid_schedule():
    with open(TABLE) as f:
        rows = [json.loads(l) for l in f if l.strip()]
    for r in rows:
        p = r["passes"]
        digits, cols = r["digits"][:p], r["log_cols"][:p]
        assert 1 <= p <= 4 and sum(digits) == r["log_n"], r
        assert all(1 <= k <= 11 for k in digits), r
        assert all(0 <= c <= 3 and k + c <= 11 for k, c in zip(digits, cols)), r
        assert r["mode"] in (1, 2) and 1 <= r["ilp"] <= 7 and r["ms"] > 0, r
