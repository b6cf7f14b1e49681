"""The C oracle (4 x 64-bit limbs) against the Python oracle and the definition."""
import numpy as np
import pytest

from oracle import cpu
from oracle import field as fld
from oracle import ntt_ref as ref
from workloads import limbs_to_ints, uniform_elements

FIELDS = [fld.BLS12_381, fld.BN254, fld.BLS12_377]
IDS = [f.name for f in FIELDS]


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_constants(F):
    assert cpu.two_adicity(F) == F.s
    for L in (0, 1, 5, 17, F.s):
        assert cpu.root(F, L) == F.to_mont(F.root(L))
        assert cpu.root(F, L, inverse=True) == F.to_mont(F.root(L, inverse=True))


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_mont_mul(F):
    X = limbs_to_ints(uniform_elements(F.r, 300, 31))
    edge = [0, 1, F.r - 1, F.r - 2, F.R, F.to_mont(1), F.to_mont(F.r - 1)]
    vals = X + edge
    for i, a in enumerate(vals):
        b = vals[(7 * i + 3) % len(vals)]
        assert cpu.mont_mul(F, a, b) == F.mont_mul(a, b)


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
@pytest.mark.parametrize("L", [0, 1, 2, 3, 5, 8, 10, 12])
@pytest.mark.parametrize("kind", ["ntt", "intt", "coset_ntt", "coset_intt"])
def test_matches_python_oracle(F, L, kind):
    n = 1 << L
    X = uniform_elements(F.r, n, 40 + L)
    inverse = kind.endswith("intt")
    sh = F.to_mont(F.g) if kind.startswith("coset") else None
    want = ref.ntt_mont(F, X, inverse=inverse, shift_mont=sh)
    got = cpu.ntt(F, X, inverse=inverse, shift_mont=sh, threads=4)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_large_size_single_outputs(F):
    """2^18 full transform from the C oracle vs single outputs of the definition."""
    L = 18
    n = 1 << L
    X = uniform_elements(F.r, n, 4242)
    got = limbs_to_ints(cpu.ntt(F, X))
    ks = [0, 1, 2, n // 2, n - 1, 12345, 98765]
    w = F.to_mont(F.root(L))
    r = F.r
    for k in ks:
        # a(w^k) by the C Horner evaluator (Montgomery domain) ...
        wk = F.to_mont(pow(F.root(L), k, r))
        assert got[k] == cpu.eval_at(F, X, wk)
    # ... and one output by the Python definition
    assert got[12345] == ref.ntt_at_mont(F, X, [12345])[0]
    assert w == cpu.root(F, L)


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
@pytest.mark.parametrize("L", [3, 8])
def test_groth16(F, L):
    n = 1 << L
    A, B, C = (uniform_elements(F.r, n, s) for s in (51, 52, 53))
    want = ref.groth16_h_mont(F, A, B, C)
    got = cpu.groth16_h(F, A, B, C, threads=3)
    assert np.array_equal(got, want)


def test_threads_do_not_change_result():
    F = fld.BLS12_381
    X = uniform_elements(F.r, 1 << 14, 9)
    a = cpu.ntt(F, X, threads=1)
    b = cpu.ntt(F, X, threads=7)
    assert np.array_equal(a, b)
