"""Tune transform schedules for every size on the current GPU.

Runs the library's autotuner (zkntt_tune) for every field (or --fields), both directions and
log_n in a range, and writes the winners as JSON lines to --out.  Copying that
file to ``zkntt_tuned.jsonl`` next to ``libzkntt.so`` makes every plan created
on a GPU with the same name use the tuned schedules.

    python -m paper_2509_22684_gb300.tune_all --out zkntt_tuned.jsonl
"""
from __future__ import annotations

import argparse
import os
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--lmin", type=int, default=10)
    ap.add_argument("--lmax", type=int, default=26)
    ap.add_argument("--candidates", type=int, default=40)
    ap.add_argument("--large-candidates", type=int, default=16,
                    help="candidate budget for log_n >= 25")
    ap.add_argument("--fields", default="bls12_381_fr,bn254_fr,bls12_377_fr")
    args = ap.parse_args()
    os.environ["ZKNTT_TUNE_CACHE"] = os.path.abspath(args.out)
    import paper_2509_22684_gb300 as zk
    t0 = time.time()
    for field in args.fields.split(","):
        _, _, s = zk.field_info(field)
        for inverse in (False, True):
            for L in range(args.lmin, min(args.lmax, s, 28) + 1):
                budget = args.candidates if L < 25 else args.large_candidates
                best = zk.tune(field, L, inverse=inverse, max_candidates=budget)
                print(f"{field} 2^{L} {'inv' if inverse else 'fwd'}: {best['digits']} cols "
                      f"{best['cols']} ilp {best['ilp']} {best['twiddle_mode']} "
                      f"{best['ms']:.4f} ms  ({(1 << L) / best['ms'] / 1e3:.0f} Melem/s)",
                      flush=True)
    print(f"done in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
