"""Pins for the oracle's transform against mathematics that fixes the result:
the O(n^2) definition, closed-form special cases, the convolution theorem
against schoolbook products, round trips, the four-step identity and the
Groth16 divisibility property."""
import random

import numpy as np
import pytest

from oracle import field as fld
from oracle import ntt_ref as ref
from workloads import uniform_elements, limbs_to_ints

FIELDS = [fld.BLS12_381, fld.BN254, fld.BLS12_377]
IDS = [f.name for f in FIELDS]


def rand_vec(F, n, seed):
    return [v % F.r for v in limbs_to_ints(uniform_elements(F.r, n, seed))]


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
@pytest.mark.parametrize("L", [0, 1, 2, 3, 4, 5, 6])
def test_radix2_equals_definition(F, L):
    n = 1 << L
    a = rand_vec(F, n, 100 + L)
    w = F.root(L)
    assert ref.ntt_radix2(a, w, F.r) == ref.dft(a, w, F.r)
    wi = F.root(L, inverse=True)
    assert ref.ntt_radix2(a, wi, F.r) == ref.dft(a, wi, F.r)


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_special_cases(F):
    r = F.r
    for L in (1, 3, 6, 9):
        n = 1 << L
        w = F.root(L)
        delta0 = [1] + [0] * (n - 1)
        delta1 = [0, 1] + [0] * (n - 2)
        ones = [1] * n
        assert ref.ntt(F, delta0) == [1] * n
        assert ref.ntt(F, ones) == [n % r] + [0] * (n - 1)
        assert ref.ntt(F, delta1) == [pow(w, k, r) for k in range(n)]
        # coset NTT of delta_1 is g * w^k
        assert ref.ntt(F, delta1, shift=F.g) == [F.g * pow(w, k, r) % r for k in range(n)]
        # inverse of delta_0 is n^-1 everywhere; inverse of delta_1 is n^-1 w^-j
        ninv = pow(n, -1, r)
        assert ref.ntt(F, delta0, inverse=True) == [ninv] * n
        wi = F.root(L, inverse=True)
        assert ref.ntt(F, delta1, inverse=True) == [ninv * pow(wi, j, r) % r for j in range(n)]


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
@pytest.mark.parametrize("L", [1, 4, 8, 11])
def test_round_trips(F, L):
    n = 1 << L
    a = rand_vec(F, n, 200 + L)
    assert ref.ntt(F, ref.ntt(F, a), inverse=True) == a
    assert ref.ntt(F, ref.ntt(F, a, inverse=True)) == a
    g = F.g
    assert ref.ntt(F, ref.ntt(F, a, shift=g), inverse=True, shift=g) == a


def _schoolbook_cyclic(a, b, r):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            out[(i + j) % n] = (out[(i + j) % n] + a[i] * b[j]) % r
    return out


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
@pytest.mark.parametrize("L", [2, 5, 8])
def test_convolution_theorem(F, L):
    n = 1 << L
    r = F.r
    a = rand_vec(F, n, 300 + L)
    b = rand_vec(F, n, 400 + L)
    A, B = ref.ntt(F, a), ref.ntt(F, b)
    prod = ref.ntt(F, [x * y % r for x, y in zip(A, B)], inverse=True)
    assert prod == _schoolbook_cyclic(a, b, r)


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_linear_product_via_zero_padding(F):
    """Polynomial product of degree < n/2 inputs equals the schoolbook product."""
    r = F.r
    n = 64
    a = rand_vec(F, n // 2, 501) + [0] * (n // 2)
    b = rand_vec(F, n // 2, 502) + [0] * (n // 2)
    prod = ref.ntt(F, [x * y % r for x, y in zip(ref.ntt(F, a), ref.ntt(F, b))], inverse=True)
    school = [0] * n
    for i in range(n // 2):
        for j in range(n // 2):
            school[i + j] = (school[i + j] + a[i] * b[j]) % r
    assert prod == school


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_coset_identity(F):
    r = F.r
    L = 6
    n = 1 << L
    a = rand_vec(F, n, 600)
    g = F.g
    w = F.root(L)
    out = ref.ntt(F, a, shift=g)
    for k in range(n):
        assert out[k] == ref.eval_poly(a, g * pow(w, k, r) % r, r)


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
@pytest.mark.parametrize("n1,n2", [(4, 4), (2, 16), (8, 4), (16, 8)])
def test_four_step_identity(F, n1, n2):
    a = rand_vec(F, n1 * n2, 700 + n1)
    w = F.root((n1 * n2).bit_length() - 1)
    assert ref.four_step(F, a, n1, n2) == ref.dft(a, w, F.r)


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
@pytest.mark.parametrize("L", [3, 6, 9])
def test_groth16_constrained_h_has_zero_top_coefficient(F, L):
    """With c = a*b on the domain, A*B - C vanishes on it, so H = (AB - C)/Z
    is a polynomial of degree <= n - 2 and h(x)(x^n - 1) = A(x)B(x) - C(x)."""
    r = F.r
    n = 1 << L
    a = rand_vec(F, n, 800 + L)
    b = rand_vec(F, n, 900 + L)
    c = [x * y % r for x, y in zip(a, b)]
    h = ref.groth16_h(F, a, b, c)
    assert h[n - 1] == 0
    ap, bp, cp = (ref.ntt(F, v, inverse=True) for v in (a, b, c))
    rng = random.Random(L)
    for _ in range(4):
        x = rng.randrange(r)
        lhs = ref.eval_poly(h, x, r) * (pow(x, n, r) - 1) % r
        rhs = (ref.eval_poly(ap, x, r) * ref.eval_poly(bp, x, r) - ref.eval_poly(cp, x, r)) % r
        assert lhs == rhs


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_groth16_unconstrained_matches_coset_evaluation(F):
    """For any a, b, c: h(g w^i) = (a'(g w^i) b'(g w^i) - c'(g w^i)) / (g^n - 1)
    where a' = iNTT(a) etc., evaluated directly by Horner at the coset points."""
    r = F.r
    L = 5
    n = 1 << L
    a, b, c = (rand_vec(F, n, s) for s in (1001, 1002, 1003))
    h = ref.groth16_h(F, a, b, c)
    ap, bp, cp = (ref.ntt(F, v, inverse=True) for v in (a, b, c))
    g = F.g
    w = F.root(L)
    zinv = pow(pow(g, n, r) - 1, -1, r)
    for i in range(n):
        x = g * pow(w, i, r) % r
        want = (ref.eval_poly(ap, x, r) * ref.eval_poly(bp, x, r) - ref.eval_poly(cp, x, r)) * zinv % r
        assert ref.eval_poly(h, x, r) == want


@pytest.mark.parametrize("F", FIELDS, ids=IDS)
def test_mont_wrappers_and_single_outputs(F):
    L = 7
    n = 1 << L
    X = uniform_elements(F.r, n, 1100)
    shift = F.to_mont(F.g)
    for inverse in (False, True):
        for sh in (None, shift):
            full = limbs_to_ints(ref.ntt_mont(F, X, inverse=inverse, shift_mont=sh))
            ks = [0, 1, 5, n - 1, 77]
            assert ref.ntt_at_mont(F, X, ks, inverse=inverse, shift_mont=sh) == [full[k] for k in ks]


# ---- planted mistakes: each plausible error must trip at least one pin ------

def _pins_pass(F, ntt_fn):
    r = F.r
    try:
        for L in (2, 4):
            n = 1 << L
            w = F.root(L)
            if ntt_fn(F, [0, 1] + [0] * (n - 2)) != [pow(w, k, r) for k in range(n)]:
                return False
            a = rand_vec(F, n, 5 + L)
            if ntt_fn(F, ntt_fn(F, a), inverse=True) != a:
                return False
            if ntt_fn(F, ntt_fn(F, a, shift=F.g), inverse=True, shift=F.g) != a:
                return False
            coset = ntt_fn(F, a, shift=F.g)
            if any(coset[k] != ref.eval_poly(a, F.g * pow(w, k, r) % r, r) for k in range(n)):
                return False
    except Exception:
        return False
    return True


def test_pins_accept_the_oracle():
    assert _pins_pass(fld.BLS12_381, ref.ntt)


def test_pins_catch_planted_mistakes():
    F = fld.BLS12_381
    r = F.r

    def wrong_root(F, a, inverse=False, shift=None):       # uses w^-1 forward
        return ref.ntt(F, a, inverse=not inverse, shift=shift)

    def no_ninv(F, a, inverse=False, shift=None):          # drops n^-1
        out = ref.ntt(F, a, inverse=inverse, shift=shift)
        return [v * len(a) % r for v in out] if inverse else out

    def bitrev_out(F, a, inverse=False, shift=None):       # forgets the reordering
        out = ref.ntt(F, a, inverse=inverse, shift=shift)
        L = len(a).bit_length() - 1
        return [out[ref.bit_reverse(k, L)] for k in range(len(a))]

    def coset_sign(F, a, inverse=False, shift=None):       # g^-j instead of g^j
        s = None if shift is None else pow(shift, -1, r)
        return ref.ntt(F, a, inverse=inverse, shift=s)

    def twiddle_index(F, a, inverse=False, shift=None):    # wrong twiddle exponent
        n = len(a)
        L = n.bit_length() - 1
        w = F.root(L, inverse=inverse)
        x = list(a)
        if shift is not None and not inverse:
            x = [x[j] * pow(shift, j, r) % r for j in range(n)]
        out = [sum(x[j] * pow(w, j * k + (j & 1), r) for j in range(n)) % r for k in range(n)]
        if inverse:
            ninv = pow(n, -1, r)
            out = [v * ninv % r for v in out]
            if shift is not None:
                out = [out[j] * pow(pow(shift, -1, r), j, r) % r for j in range(n)]
        return out

    for bad in (wrong_root, no_ninv, bitrev_out, coset_sign, twiddle_index):
        assert not _pins_pass(F, bad), bad.__name__


def test_groth16_pins_catch_planted_mistakes():
    F = fld.BN254
    r = F.r
    L = 4
    n = 1 << L
    a = rand_vec(F, n, 21)
    b = rand_vec(F, n, 22)
    c = [x * y % r for x, y in zip(a, b)]

    def dropped_c(F, a, b, c):
        return ref.groth16_h(F, a, b, [0] * len(c))

    def no_zinv(F, a, b, c):
        g = F.g
        zl = (pow(g, len(a), r) - 1) % r
        return [v * zl % r for v in ref.groth16_h(F, a, b, c)]

    for bad in (dropped_c, no_zinv):
        h = bad(F, a, b, c)
        ap, bp, cp = (ref.ntt(F, v, inverse=True) for v in (a, b, c))
        x = 123456789
        lhs = ref.eval_poly(h, x, r) * (pow(x, n, r) - 1) % r
        rhs = (ref.eval_poly(ap, x, r) * ref.eval_poly(bp, x, r) - ref.eval_poly(cp, x, r)) % r
        assert h[n - 1] != 0 or lhs != rhs, bad.__name__


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("n", [8, 64, 256])
def test_shift_theorem(F, n):
    """A cyclic shift of the input by s multiplies output k by w^(s k) (a
    property of the DFT that pins the sign of the exponent and the index
    convention independently of the oracle's own formulas)."""
    r = F.r
    rng = random.Random(90 + n)
    a = [rng.randrange(r) for _ in range(n)]
    w = F.root(n.bit_length() - 1)
    A = ref.ntt(F, a)
    for s in (1, 3, n // 2, n - 1):
        shifted = [a[(j - s) % n] for j in range(n)]
        B = ref.ntt(F, shifted)
        assert B == [A[k] * pow(w, s * k, r) % r for k in range(n)], s


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
def test_linearity(F):
    """NTT(alpha a + beta b) = alpha NTT(a) + beta NTT(b), forward, inverse and
    coset (the coset and inverse scales are linear too)."""
    r = F.r
    rng = random.Random(91)
    n = 128
    a = [rng.randrange(r) for _ in range(n)]
    b = [rng.randrange(r) for _ in range(n)]
    alpha, beta = rng.randrange(r), rng.randrange(r)
    mix = [(alpha * x + beta * y) % r for x, y in zip(a, b)]
    for kw in ({}, {"inverse": True}, {"shift": F.g}, {"inverse": True, "shift": F.g}):
        A, B, M = ref.ntt(F, a, **kw), ref.ntt(F, b, **kw), ref.ntt(F, mix, **kw)
        assert M == [(alpha * x + beta * y) % r for x, y in zip(A, B)], kw


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
def test_c_oracle_shift_theorem_at_larger_size(F):
    """The shift theorem on the C oracle at 2^14 (sizes the Python oracle is
    slow for): output k of the shifted input equals output k times w^(s k)."""
    from oracle import cpu
    L = 14
    n = 1 << L
    X = uniform_elements(F.r, n, 92)
    s = 12345
    Xs = np.roll(X, s, axis=0)           # Xs[j] = X[j - s]
    A = limbs_to_ints(cpu.ntt(F, X))
    B = limbs_to_ints(cpu.ntt(F, Xs))
    w = F.root(L)
    for k in (0, 1, 7, n // 3, n - 1):
        # Montgomery forms: B_k = A_k * w^(s k)  <=>  B~_k = A~_k * w^(s k) (plain factor)
        assert B[k] == A[k] * pow(w, s * k, F.r) % F.r, k
