"""Served results equal the same transform run alone (and the oracle)."""
import numpy as np
import pytest

from oracle import cpu
from oracle import field as fld
from workloads import poisson_trace, uniform_elements

from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu
FMAP = {"bls12_381_fr": fld.BLS12_381, "bn254_fr": fld.BN254}


@pytest.mark.parametrize("solo_log_n", [None, 15])
def test_served_mix_matches_solo_and_oracle(solo_log_n):
    import paper_2509_22684_gb300 as zk
    from paper_2509_22684_gb300.serve import Engine, GpuExecutor, Request
    trace = poisson_trace(5000, 80, 20000.0, lmin=10, lmax=16)
    reqs = []
    for q in trace:
        field = "bls12_381_fr" if q.seed % 3 else "bn254_fr"
        F = FMAP[field]
        r = Request(q.seed % 100000, q.arrival_s, field, q.log_n, q.kind, seed=q.seed)
        r.payload = to_dev(uniform_elements(F.r, 1 << q.log_n, q.seed))
        reqs.append(r)
    ex = GpuExecutor(streams=2, keep_outputs=True)
    done, st = Engine(ex, budget_bytes=1 << 28, streams=2, max_batch_jobs=16,
                      solo_log_n=solo_log_n).run(reqs)
    zk.sync_status()
    assert st.requests == len(reqs)
    assert st.batches < len(reqs)          # requests were batched together
    for r in done:
        solo = to_host(ex.plan(r.field, r.log_n, r.kind).execute(r.payload))
        got = to_host(r.out)
        assert np.array_equal(got, solo), (r.rid, r.log_n, r.kind)
    # and a sample against the oracle
    for r in done[:12]:
        F = FMAP[r.field]
        X = to_host(r.payload)
        sh = F.to_mont(F.g) if r.kind.startswith("coset") else None
        want = cpu.ntt(F, X, inverse=r.kind.endswith("intt"), shift_mont=sh)
        assert np.array_equal(to_host(r.out), want), (r.rid, r.kind)
    ex.close()
