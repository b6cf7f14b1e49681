"""Persistent batch launch and the Groth16 H sequence: every result equals the
oracle's and the solo execution's, bit for bit; the bounded device wait
reports a timeout instead of hanging."""
import ctypes

import numpy as np
import pytest

from oracle import cpu
from oracle import field as fld
from oracle import ntt_ref as ref
from workloads import batch_jobs, uniform_elements

from gpu_util import first_mismatch, rand_dev, to_dev, to_host

pytestmark = pytest.mark.gpu
FMAP = {"bls12_381_fr": fld.BLS12_381, "bn254_fr": fld.BN254, "bls12_377_fr": fld.BLS12_377}


def _oracle(F, X, inverse=False, shift=None):
    if X.shape[0] <= 1 << 10:
        return ref.ntt_mont(F, X, inverse=inverse, shift_mont=shift)
    return cpu.ntt(F, X, inverse=inverse, shift_mont=shift)


@pytest.mark.parametrize("fields", [("bls12_381_fr", "bn254_fr"),
                                    ("bls12_381_fr", "bn254_fr", "bls12_377_fr")],
                         ids=["two_fields", "three_fields"])
def test_batch_uneven_mixed_fields_matches_oracle_and_solo(fields):
    import torch
    import paper_2509_22684_gb300 as zk
    jobs = batch_jobs(4000, count=64, lmin=10, lmax=20, fields=fields)
    assert {j.field for j in jobs} == set(fields)
    plans, xs, outs, hosts = [], [], [], []
    for j in jobs:
        F = FMAP[j.field]
        X = uniform_elements(F.r, 1 << j.log_n, j.seed)
        hosts.append(X)
        xs.append(to_dev(X))
        outs.append(torch.empty_like(xs[-1]))
        plans.append(zk.Plan(j.field, j.log_n, inverse=(j.kind == "intt")))
    zk.execute_batch(plans, xs, outs)
    zk.sync_status()
    for j, p, X, x, o in zip(jobs, plans, hosts, xs, outs):
        F = FMAP[j.field]
        got = to_host(o)
        want = _oracle(F, X, inverse=(j.kind == "intt"))
        assert np.array_equal(got, want), (j, first_mismatch(got, want))
        solo = to_host(p.execute(x))
        assert np.array_equal(solo, got)
    for p in plans:
        p.close()


def test_batch_in_place_and_order_independence():
    import torch
    import paper_2509_22684_gb300 as zk
    F = fld.BN254
    sizes = [14, 11, 18, 12]
    Xs = [uniform_elements(F.r, 1 << L, 90 + L) for L in sizes]
    plans = [zk.Plan(F.name, L, coset_shift=F.to_mont(F.g)) for L in sizes]
    wants = [_oracle(F, X, shift=F.to_mont(F.g)) for X in Xs]
    for order in ([0, 1, 2, 3], [3, 1, 0, 2]):
        xs = [to_dev(Xs[i]) for i in order]
        zk.execute_batch([plans[i] for i in order], xs, xs)   # in place
        for k, i in enumerate(order):
            assert np.array_equal(to_host(xs[k]), wants[i])
    for p in plans:
        p.close()


@pytest.mark.parametrize("F", [fld.BLS12_381, fld.BN254, fld.BLS12_377], ids=lambda f: f.name)
@pytest.mark.parametrize("L", [4, 10, 13, 16])
@pytest.mark.parametrize("fused", [False, True])
def test_groth16_matches_oracle(F, L, fused):
    import paper_2509_22684_gb300 as zk
    A, B, C = (uniform_elements(F.r, 1 << L, s) for s in (3001, 3002, 3003))
    a, b, c = (to_dev(v) for v in (A, B, C))
    h = zk.groth16_h(F.name, L, a, b, c, fused=fused)
    zk.sync_status()
    got = to_host(h)
    want = ref.groth16_h_mont(F, A, B, C) if L <= 10 else cpu.groth16_h(F, A, B, C)
    assert np.array_equal(got, want), first_mismatch(got, want)
    # the inputs are read only
    assert np.array_equal(to_host(a), A)


def test_groth16_2_22_fused_equals_separate_and_oracle():
    import paper_2509_22684_gb300 as zk
    F = fld.BLS12_381
    L = 22
    A, B, C = (uniform_elements(F.r, 1 << L, s) for s in (3001, 3002, 3003))
    a, b, c = (to_dev(v) for v in (A, B, C))
    h1 = to_host(zk.groth16_h(F.name, L, a, b, c, fused=True))
    h0 = to_host(zk.groth16_h(F.name, L, a, b, c, fused=False))
    assert np.array_equal(h0, h1)
    want = cpu.groth16_h(F, A, B, C)
    assert np.array_equal(h1, want), first_mismatch(h1, want)


def test_groth16_constrained_top_coefficient_zero():
    """c = a*b on the domain: h has degree <= n-2 (h[n-1] = 0)."""
    import paper_2509_22684_gb300 as zk
    F = fld.BLS12_381
    L = 16
    A, B = (uniform_elements(F.r, 1 << L, s) for s in (3101, 3102))
    a, b = to_dev(A), to_dev(B)
    c = zk.field_op(F.name, "mul", a, b)
    h = to_host(zk.groth16_h(F.name, L, a, b, c, fused=True))
    assert not h[-1].any()
    assert h[:-1].any()


def test_bounded_wait_reports_timeout():
    import torch
    from paper_2509_22684_gb300 import _native as N
    st = N.lib().zkntt_selftest_timeout(20, None)
    assert st == N.ETIMEOUT
    # the context is still usable afterwards
    F = fld.BLS12_381
    X, x = rand_dev(F, 12, 1)
    import paper_2509_22684_gb300 as zk
    with zk.Plan(F.name, 12) as p:
        assert np.array_equal(to_host(p.execute(x)), ref.ntt_mont(F, X))
    zk.sync_status()


def test_timeout_is_reported_on_its_own_stream_only():
    """Each stream has its own device-side error word: a bounded wait that
    gives up on stream A is reported by zkntt_sync_status(A), not by a
    concurrent stream B, and reading it clears it."""
    import torch
    from paper_2509_22684_gb300 import _native as N
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    ha, hb = ctypes.c_void_p(a.cuda_stream), ctypes.c_void_p(b.cuda_stream)
    assert N.lib().zkntt_inject_timeout(20, ha) == N.OK
    assert N.lib().zkntt_sync_status(hb) == N.OK
    assert N.lib().zkntt_sync_status(ha) == N.ETIMEOUT
    assert N.lib().zkntt_sync_status(ha) == N.OK


def test_plan_of_another_device_is_rejected_before_enqueue():
    """Every execute entry point returns EINVAL for a plan whose device is not
    the current one (the self-test passes each of them a copy of a real plan
    marked as another device's)."""
    from paper_2509_22684_gb300 import _native as N
    checked, rejected = ctypes.c_int(), ctypes.c_int()
    assert N.lib().zkntt_selftest_device_check(ctypes.byref(checked), ctypes.byref(rejected)) == N.OK
    assert checked.value == 7
    assert rejected.value == 7


@pytest.mark.parametrize("L", [10, 16])
def test_groth16_graph_replay_matches_oracle(L):
    import torch
    import paper_2509_22684_gb300 as zk
    F = fld.BLS12_381
    A, B, C = (uniform_elements(F.r, 1 << L, s) for s in (3201, 3202, 3203))
    a, b, c = (to_dev(v) for v in (A, B, C))
    h = torch.empty_like(a)
    scr = torch.empty((3 << L, 8), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = zk.Groth16Graph(F.name, L, a, b, c, h, scr, stream=s)
    want = ref.groth16_h_mont(F, A, B, C) if L <= 10 else cpu.groth16_h(F, A, B, C)
    for _ in range(2):
        h.zero_()
        torch.cuda.synchronize()
        g.launch(stream=s)
        s.synchronize()
        got = to_host(h)
        assert np.array_equal(got, want), first_mismatch(got, want)
    # new inputs in the same buffers are picked up by the replay
    A2 = uniform_elements(F.r, 1 << L, 3301)
    a.copy_(to_dev(A2))
    torch.cuda.synchronize()
    g.launch(stream=s)
    s.synchronize()
    want2 = ref.groth16_h_mont(F, A2, B, C) if L <= 10 else cpu.groth16_h(F, A2, B, C)
    assert np.array_equal(to_host(h), want2)
    g.close()
    zk.sync_status()


def test_signalled_batch_sets_every_flag_and_matches_oracle():
    import torch
    import paper_2509_22684_gb300 as zk
    jobs = batch_jobs(4100, count=24, lmin=8, lmax=17)
    plans, xs, outs, hosts = [], [], [], []
    for j in jobs:
        F = FMAP[j.field]
        X = uniform_elements(F.r, 1 << j.log_n, j.seed)
        hosts.append(X)
        xs.append(to_dev(X))
        outs.append(torch.empty_like(xs[-1]))
        plans.append(zk.Plan(j.field, j.log_n, inverse=(j.kind == "intt")))
    flags = zk.CompletionFlags(64)
    s = torch.cuda.Stream()
    zk.execute_batch_signal(plans, xs, outs, flags, list(range(10, 10 + len(jobs))), 7, stream=s)
    s.synchronize()
    zk.sync_status(s)
    assert [flags[i] for i in range(10, 10 + len(jobs))] == [7] * len(jobs)
    assert flags[9] == 0 and flags[10 + len(jobs)] == 0
    for j, X, o in zip(jobs, hosts, outs):
        F = FMAP[j.field]
        assert np.array_equal(to_host(o), _oracle(F, X, inverse=(j.kind == "intt")))
    for p in plans:
        p.close()
    flags.close()


def test_batch_larger_than_one_segment_table_is_split():
    """64 three-pass transforms are 192 pass segments, more than one persistent
    launch's table holds (160): the batch runs as consecutive launches and
    every result still equals the solo execution; the signalled form also
    marks every transform complete."""
    import torch
    import paper_2509_22684_gb300 as zk
    F = fld.BLS12_381
    plans, xs, outs = [], [], []
    for i in range(64):
        L = 12 + (i % 3)
        digits = (4, 4, L - 8)
        plans.append(zk.Plan(F.name, L, inverse=bool(i & 1), digits=digits))
        xs.append(to_dev(uniform_elements(F.r, 1 << L, 7000 + i)))
        outs.append(torch.empty_like(xs[-1]))
    assert sum(p.describe()["passes"] for p in plans) == 192
    zk.execute_batch(plans, xs, outs)
    zk.sync_status()
    for p, x, o in zip(plans, xs, outs):
        assert np.array_equal(to_host(o), to_host(p.execute(x)))
    flags = zk.CompletionFlags(64)
    outs2 = [torch.empty_like(x) for x in xs]
    zk.execute_batch_signal(plans, xs, outs2, flags, list(range(64)), 9)
    zk.sync_status()
    assert all(flags[i] == 9 for i in range(64))
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    flags.close()
    for p in plans:
        p.close()


def test_groth16_contract_signature_runs_the_fused_form():
    """zkntt_groth16_h with the boundary's own signature (no form argument)
    runs the fused sequence and equals the oracle (Fig. 2)."""
    import torch
    from paper_2509_22684_gb300 import _native as N
    F = fld.BN254
    L = 10
    A, B, C = (uniform_elements(F.r, 1 << L, s) for s in (3101, 3102, 3103))
    a, b, c = to_dev(A), to_dev(B), to_dev(C)
    h = torch.empty_like(a)
    scr = torch.empty((3 << L, 8), dtype=torch.int32, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = N.lib().zkntt_groth16_h(1, L, p(a), p(b), p(c), p(h), p(scr),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == N.OK
    assert np.array_equal(to_host(h), ref.groth16_h_mont(F, A, B, C))
