"""GPU transform parity against the oracle: every direction and coset kind,
both fields, single-pass and multi-pass schedules, both twiddle modes, forced
digit splits, in place and out of place.  Bit-exact comparison throughout."""
import numpy as np
import pytest

from oracle import cpu
from oracle import field as fld
from oracle import ntt_ref as ref

from gpu_util import first_mismatch, rand_dev, to_dev, to_host

pytestmark = pytest.mark.gpu
FIELDS = [fld.BLS12_381, fld.BN254, fld.BLS12_377]
KINDS = ["ntt", "intt", "coset_ntt", "coset_intt"]


def _oracle(F, X, kind):
    inverse = kind.endswith("intt")
    sh = F.to_mont(F.g) if kind.startswith("coset") else None
    if X.shape[0] <= 1 << 10:
        return ref.ntt_mont(F, X, inverse=inverse, shift_mont=sh)
    return cpu.ntt(F, X, inverse=inverse, shift_mont=sh)


def _plan(F, L, kind, **kw):
    import paper_2509_22684_gb300 as zk
    inverse = kind.endswith("intt")
    sh = F.to_mont(F.g) if kind.startswith("coset") else None
    return zk.Plan(F.name, L, inverse=inverse, coset_shift=sh, **kw)


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L", list(range(1, 15)))
def test_default_schedule(F, kind, L):
    X, x = rand_dev(F, L, 1000 * L + 7)
    with _plan(F, L, kind) as p:
        y = p.execute(x)
    got = to_host(y)
    want = _oracle(F, X, kind)
    assert np.array_equal(got, want), first_mismatch(got, want)


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mode", ["precomp", "otf"])
@pytest.mark.parametrize("digits,cols", [
    ((8, 8), None), ((4, 11), None), ((5, 6, 5), None), ((11, 5), (1, 8)),
    ((3, 4, 5, 4), None), ((6, 10), (2, 2)), ((9, 7), (4, 4)), ((4, 4, 4, 4), (8, 8, 8, 8)),
])
def test_forced_splits(F, kind, mode, digits, cols):
    L = sum(digits)
    X, x = rand_dev(F, L, 77 + L)
    with _plan(F, L, kind, twiddle_mode=mode, digits=digits, cols=cols) as p:
        assert p.describe()["digits"] == list(digits)
        y = p.execute(x)
    got = to_host(y)
    want = _oracle(F, X, kind)
    assert np.array_equal(got, want), first_mismatch(got, want)


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("L", [12, 17])
def test_in_place_and_scratch(F, L):
    import torch
    X, x = rand_dev(F, L, 5)
    want = _oracle(F, X, "coset_ntt")
    with _plan(F, L, "coset_ntt") as p:
        p.execute(x, x)   # in place
        assert np.array_equal(to_host(x), want)
        x2 = to_dev(X)
        out = torch.empty_like(x2)
        scr = torch.empty(max(1, p.scratch_bytes() // 4), dtype=torch.int32, device="cuda")
        p.execute_scratch(x2, out, scr)
        assert np.array_equal(to_host(out), want)


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("L", [16, 20, 22])
@pytest.mark.parametrize("kind", KINDS)
def test_configured_sizes_full_vector(F, L, kind):
    X, x = rand_dev(F, L, 2000 + L)
    with _plan(F, L, kind) as p:
        y = p.execute(x)
    got = to_host(y)
    want = _oracle(F, X, kind)
    assert np.array_equal(got, want), first_mismatch(got, want)


_BIG_INPUT = {}


def _big_input(F, L, seed):
    """Seeded input of 2^L elements, kept for the next test of the same field
    and size (one entry: a 2^26 vector is 2 GiB of host memory)."""
    key = (F.name, L, seed)
    if key not in _BIG_INPUT:
        _BIG_INPUT.clear()
        _BIG_INPUT[key] = rand_dev(F, L, seed)[0]
    return _BIG_INPUT[key]


# the tests of one field and size run one after the other, so the input is
# drawn once per (field, size)
_CASES_24 = [(F, kind, mode) for F in FIELDS for kind in KINDS for mode in ("precomp", "otf")]


@pytest.mark.parametrize("F,kind,mode", _CASES_24,
                         ids=[f"{F.name}-{k}-{m}" for F, k, m in _CASES_24])
def test_2_24_full_vector(F, kind, mode):
    """2^24, every kind in both twiddle modes: the whole output equals the C
    oracle's (Section II-B transform; coset kinds as in Fig. 2)."""
    L = 24
    X = _big_input(F, L, 2024)
    with _plan(F, L, kind, twiddle_mode=mode) as p:
        y = p.execute(to_dev(X))
    got = to_host(y)
    del y
    want = _oracle(F, X, kind)
    assert np.array_equal(got, want), first_mismatch(got, want)


_CASES_26 = [(F, kind, "precomp") for F in FIELDS for kind in KINDS] + \
    [(fld.BLS12_381, "coset_intt", "otf"), (fld.BN254, "ntt", "otf")]


@pytest.mark.parametrize("F,kind,mode", _CASES_26,
                         ids=[f"{F.name}-{k}-{m}" for F, k, m in _CASES_26])
def test_2_26_full_vector(F, kind, mode):
    """2^26 (the largest size of the plain-transform grid), every kind: the
    whole output equals the C oracle's.  A round trip alone would miss a
    mistake shared by a forward and an inverse plan (a wrong root, table
    index or digit split at this size); this comparison does not."""
    import torch
    L = 26
    X = _big_input(F, L, 2026)
    with _plan(F, L, kind, twiddle_mode=mode) as p:
        assert p.describe()["twiddle_mode"] == mode
        y = p.execute(to_dev(X))
        got = to_host(y)
        del y
        torch.cuda.empty_cache()
    want = _oracle(F, X, kind)
    assert np.array_equal(got, want), first_mismatch(got, want)


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
def test_2_26_sampled_outputs_and_round_trip(F):
    """2^26: outputs at sampled k against the definition (Horner in the C
    oracle), and inverse(forward(x)) == x over the whole vector."""
    L = 26
    X, x = rand_dev(F, L, 2026)
    with _plan(F, L, "ntt") as p, _plan(F, L, "intt") as q:
        y = p.execute(x)
        z = q.execute(y)
    got = to_host(y)
    w = F.root(L)
    for k in (0, 1, 3, (1 << L) - 1, 12345677):
        assert int.from_bytes(got[k].tobytes(), "little") == cpu.eval_at(F, X, F.to_mont(pow(w, k, F.r)))
    assert np.array_equal(to_host(z), X)


def test_bn254_maximum_size_2_28():
    """BN254 F_r has 2-adicity 28, so 2^28 is its largest transform (the
    field's top root of unity is used): outputs at sampled k against the
    definition (Horner in the C oracle), and inverse(forward(x)) == x over the
    whole vector, compared on the device (8 GiB per vector)."""
    import torch
    F = fld.BN254
    L = 28
    assert F.s == L
    X, x = rand_dev(F, L, 2028)
    with _plan(F, L, "ntt") as p:
        y = p.execute(x)
    w = F.root(L)
    for k in (1, (1 << L) - 1, 200000003):
        got = int.from_bytes(to_host(y[k:k + 1]).tobytes(), "little")
        assert got == cpu.eval_at(F, X, F.to_mont(pow(w, k, F.r))), k
    del X
    with _plan(F, L, "intt") as q:
        z = q.execute(y)
    assert torch.equal(z, x)


def test_round_trip_config1():
    """BLS12-381, n = 2^12, seed 1001: forward then inverse returns the input."""
    F = fld.BLS12_381
    X, x = rand_dev(F, 12, 1001)
    with _plan(F, 12, "ntt") as p, _plan(F, 12, "intt") as q:
        y = p.execute(x)
        z = q.execute(y)
    assert np.array_equal(to_host(y), ref.ntt_mont(F, X))
    assert np.array_equal(to_host(z), X)


def test_argument_errors():
    import torch
    import paper_2509_22684_gb300 as zk
    from paper_2509_22684_gb300 import ZkNttError
    with pytest.raises(ZkNttError):
        zk.Plan("bls12_381_fr", 0)
    with pytest.raises(ZkNttError):
        zk.Plan("bn254_fr", 29)
    with pytest.raises(ZkNttError):
        zk.Plan("bls12_381_fr", 10, coset_shift=0)
    with pytest.raises(ZkNttError):
        zk.Plan("bls12_381_fr", 10, coset_shift=fld.BLS12_381.r)
    with pytest.raises(ZkNttError):
        zk.Plan("bls12_381_fr", 20, digits=(10, 9))
    with zk.Plan("bls12_381_fr", 10) as p:
        buf = torch.zeros((1 << 10) * 8 + 8, dtype=torch.int32, device="cuda")
        mis = buf[1:1 + (1 << 10) * 8]   # 4-byte offset: misaligned
        with pytest.raises(ZkNttError):
            p.execute(mis, torch.empty_like(mis))
        a = torch.zeros(((1 << 10) + 2) * 8, dtype=torch.int32, device="cuda")
        with pytest.raises(ZkNttError):   # partial overlap
            p.execute(a[:(1 << 10) * 8], a[16:16 + (1 << 10) * 8])


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("digits,cols", [((8, 8), None), ((5, 6, 5), None), ((11, 5), (1, 8)),
                                         ((4, 4, 4, 4), (8, 8, 8, 8)), ((10,), None), ((3,), None),
                                         ((7, 9), (4, 2))])
def test_kernel_variants(F, kind, variant, digits, cols):
    """Every kernel variant (one or two butterflies per thread, the register
    budgets, the pipelined loop, twice the threads per tile) gives the same
    result."""
    L = sum(digits)
    X, x = rand_dev(F, L, 99 + L)
    with _plan(F, L, kind, digits=digits, cols=cols, ilp=variant) as p:
        y = p.execute(x)
    got = to_host(y)
    want = _oracle(F, X, kind)
    assert np.array_equal(got, want), first_mismatch(got, want)


def test_tuner_picks_a_schedule_that_stays_exact(tmp_path, monkeypatch):
    import paper_2509_22684_gb300 as zk
    monkeypatch.setenv("ZKNTT_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    F = fld.BN254
    L = 17
    best = zk.tune(F.name, L, inverse=True, max_candidates=6)
    assert sum(best["digits"]) == L and best["ms"] > 0
    X, x = rand_dev(F, L, 1717)
    with zk.Plan(F.name, L, inverse=True, use_tuner=True) as p:
        assert p.describe()["digits"] == best["digits"]
        got = to_host(p.execute(x))
    assert np.array_equal(got, cpu.ntt(F, X, inverse=True))


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
def test_execute_host_buffered_matches_device_execution(F):
    """Host buffers in and out with a caller-owned device work buffer: the
    result equals the device-resident execution; a too-small buffer is
    rejected before anything is enqueued."""
    import torch
    import paper_2509_22684_gb300 as zk
    from paper_2509_22684_gb300 import ZkNttError
    L = 18
    X, x = rand_dev(F, L, 1818)
    with _plan(F, L, "coset_intt") as p:
        want = to_host(p.execute(x))
        xh = torch.from_numpy(X.view(np.int32)).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        work = torch.empty(p.work_bytes() // 4, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        p.execute_host_buffered(xh, yh, work, stream=s)
        s.synchronize()
        assert np.array_equal(yh.numpy().view(np.uint32).reshape(-1, 8), want)
        with pytest.raises(ZkNttError):
            p.execute_host_buffered(xh, yh, work[:8 * (1 << L)], stream=s)


def test_bls12_381_2_30_beyond_the_tuned_sizes():
    """2^30 BLS12-381 F_r (32 GiB per vector; sizes above 2^28 run with the
    planner's default split and pick their twiddle mode by free memory):
    outputs at sampled k against the definition (Horner in the C oracle), and
    inverse(forward(x)) == x over the whole vector, compared on the device."""
    import torch
    from workloads import uniform_elements_threaded
    F = fld.BLS12_381
    L = 30
    X = uniform_elements_threaded(F.r, 1 << L, 2030)
    x = to_dev(X)
    with _plan(F, L, "ntt") as p:
        assert p.describe()["passes"] == 3
        y = p.execute(x)
        torch.cuda.synchronize()
    w = F.root(L)
    for k in (1, (1 << L) - 1, 987654321):
        got = int.from_bytes(to_host(y[k:k + 1]).tobytes(), "little")
        assert got == cpu.eval_at(F, X, F.to_mont(pow(w, k, F.r))), k
    del X
    with _plan(F, L, "intt") as q:
        q.execute(y, y)
        torch.cuda.synchronize()
    assert torch.equal(y, x)
    del x, y
    torch.cuda.empty_cache()
