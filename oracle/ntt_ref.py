"""The NTT and the Groth16 H-polynomial sequence, written from the paper's
definitions with Python integers.

TEST INFRASTRUCTURE: see ``oracle/__init__.py`` for who may call this.

Definitions followed (arxiv 2509.22684):

* Forward transform, Section II-B: A_k = sum_{j=0}^{n-1} a_j * omega^(j*k)
  (the printed formula indexes the summand by i and runs to a_n; the reading
  used is the standard one: summand a_j, n elements a_0..a_{n-1}).
* Radix-2 Cooley-Tukey, Section II-B and Fig. 3(b): n/2 butterflies per
  stage, log2 n stages, butterfly (x, y) -> (x + y*w, x - y*w).
* Inverse transform: the paper treats it as the same computation (Section
  II-B, where NTT and INTT are discussed together); the reading used is
  omega^-1 followed by the factor
  n^-1, so that inverse(forward(a)) = a.
* Coset transforms (Groth16, Fig. 2): forward with shift g is NTT(a_j g^j);
  inverse with shift g multiplies the inverse transform's output j by g^-j.
* Groth16 H (Fig. 2 and Section IV-A, seven transforms in all): three inverse
  NTTs of the evaluation vectors a, b, c; three coset NTTs; the pointwise
  (A*B - C)/Z on the coset, where Z(x) = x^n - 1 takes the constant value
  g^n - 1 at every coset point g*omega^i; one coset inverse NTT.

All functions take and return canonical integers in [0, r) except the
``*_mont`` wrappers, which take and return [n, 8] uint32 limb arrays holding
Montgomery representatives X = x * 2^256 mod r (the layout of the library's
boundary) and convert explicitly on the way in and out.
"""
from __future__ import annotations

import numpy as np

from . import field as fld
from workloads import ints_to_limbs, limbs_to_ints


def bit_reverse(i: int, bits: int) -> int:
    """The index permutation of the radix-2 algorithm (Section II-B, Fig. 3(b):
    elements are reordered between stages; here i with its `bits` low bits
    reversed)."""
    out = 0
    for _ in range(bits):
        out = (out << 1) | (i & 1)
        i >>= 1
    return out


def dft(a: list[int], w: int, r: int) -> list[int]:
    """The definition (Section II-B, with the index typo read as a_j), O(n^2):
    A_k = sum_j a_j w^(j k) mod r."""
    n = len(a)
    return [sum(a[j] * pow(w, j * k, r) for j in range(n)) % r for k in range(n)]


def eval_poly(a: list[int], x: int, r: int) -> int:
    """sum_j a_j x^j mod r by Horner's rule: the coefficient vector read as a
    polynomial (Section II-B: the transform evaluates it at the powers of w)."""
    acc = 0
    for coef in reversed(a):
        acc = (acc * x + coef) % r
    return acc


def dft_at(a: list[int], w: int, k: int, r: int) -> int:
    """One output of the definition (Section II-B): A_k = a(w^k)."""
    return eval_poly(a, pow(w, k, r), r)


def ntt_radix2(a: list[int], w: int, r: int) -> list[int]:
    """Iterative radix-2 Cooley-Tukey, decimation in time (Fig. 3(b)).

    The input is put in bit-reversed order, then stage t (t = 1..log2 n)
    combines pairs at distance 2^(t-1) with the butterfly
    (x, y) -> (x + y*w_t^j, x - y*w_t^j), w_t = w^(n / 2^t).
    """
    n = len(a)
    bits = n.bit_length() - 1
    if 1 << bits != n:
        raise ValueError("length must be a power of two")
    x = [a[bit_reverse(i, bits)] % r for i in range(n)]
    half = 1
    while half < n:
        wt = pow(w, n // (2 * half), r)
        tw = [1] * half
        for j in range(1, half):
            tw[j] = tw[j - 1] * wt % r
        for start in range(0, n, 2 * half):
            for j in range(half):
                u = x[start + j]
                v = x[start + j + half] * tw[j] % r
                x[start + j] = (u + v) % r
                x[start + j + half] = (u - v) % r
        half *= 2
    return x


def ntt(F: fld.Field, a: list[int], inverse: bool = False, shift: int | None = None,
        use_dft: bool = False) -> list[int]:
    """Forward / inverse / coset transform of canonical values (length 2^L).

    Forward: the definition of Section II-B.  Inverse: w^-1 and the factor
    n^-1 (Section II-B treats the inverse as the same computation).  Coset
    (the Groth16 step of Fig. 2): forward multiplies a_j by shift^j first,
    inverse multiplies output j by shift^-j after.
    """
    n = len(a)
    L = n.bit_length() - 1
    r = F.r
    w = F.root(L, inverse=inverse)
    core = dft if use_dft else ntt_radix2
    if not inverse:
        x = list(a)
        if shift is not None:
            x = [x[j] * pow(shift, j, r) % r for j in range(n)]
        return core(x, w, r)
    y = core(list(a), w, r)
    ninv = pow(n, -1, r)
    y = [v * ninv % r for v in y]
    if shift is not None:
        sinv = pow(shift, -1, r)
        y = [y[j] * pow(sinv, j, r) % r for j in range(n)]
    return y


def groth16_h(F: fld.Field, a: list[int], b: list[int], c: list[int],
              shift: int | None = None) -> list[int]:
    """h coefficients from evaluation vectors a, b, c on the domain of size n.

    Steps in the order of Fig. 2: a' = iNTT(a), b' = iNTT(b), c' = iNTT(c);
    A = cosetNTT_g(a'), B = cosetNTT_g(b'), C = cosetNTT_g(c');
    H_i = (A_i B_i - C_i) * (g^n - 1)^-1;  h = cosetINTT_g(H).
    """
    r = F.r
    n = len(a)
    g = F.g if shift is None else shift
    ap = ntt(F, a, inverse=True)
    bp = ntt(F, b, inverse=True)
    cp = ntt(F, c, inverse=True)
    A = ntt(F, ap, shift=g)
    B = ntt(F, bp, shift=g)
    C = ntt(F, cp, shift=g)
    zinv = pow((pow(g, n, r) - 1) % r, -1, r)
    H = [((A[i] * B[i] - C[i]) % r) * zinv % r for i in range(n)]
    return ntt(F, H, inverse=True, shift=g)


def four_step(F: fld.Field, a: list[int], n1: int, n2: int) -> list[int]:
    """The four-step statement of the forward transform, n = n1 * n2.

    With j = j1 + n1*j2 and k = k2 + n2*k1:
    A[k2 + n2 k1] = sum_{j1} w_{n1}^(j1 k1) * w_n^(j1 k2) * sum_{j2} a[j1 + n1 j2] w_{n2}^(j2 k2).
    Used only to give the GPU's pass split an independent statement.
    """
    r = F.r
    n = n1 * n2
    assert len(a) == n
    wn = F.root(n.bit_length() - 1)
    w1 = pow(wn, n2, r)
    w2 = pow(wn, n1, r)
    inner = [[0] * n2 for _ in range(n1)]
    for j1 in range(n1):
        col = [a[j1 + n1 * j2] for j2 in range(n2)]
        inner[j1] = dft(col, w2, r)
    out = [0] * n
    for k2 in range(n2):
        row = [inner[j1][k2] * pow(wn, j1 * k2, r) % r for j1 in range(n1)]
        res = dft(row, w1, r)
        for k1 in range(n1):
            out[k2 + n2 * k1] = res[k1]
    return out


# --- Montgomery limb wrappers (the library's boundary layout) -----------------

def from_mont_limbs(F: fld.Field, X: np.ndarray) -> list[int]:
    """8 x 32-bit limbs (Section II: word-sized limbs) in Montgomery form ->
    canonical integers."""
    return [F.from_mont(v) for v in limbs_to_ints(X)]


def to_mont_limbs(F: fld.Field, x: list[int]) -> np.ndarray:
    """Canonical integers -> Montgomery-form 8 x 32-bit limbs (Section II)."""
    return ints_to_limbs([F.to_mont(v) for v in x])


def ntt_mont(F, X: np.ndarray, inverse: bool = False, shift_mont: int | None = None,
             use_dft: bool = False) -> np.ndarray:
    """Transform of Montgomery-form limbs; ``shift_mont`` is the coset shift in
    Montgomery form, as the library's plan takes it."""
    F = fld.get(F)
    x = from_mont_limbs(F, X)
    shift = None if shift_mont is None else F.from_mont(shift_mont)
    return to_mont_limbs(F, ntt(F, x, inverse=inverse, shift=shift, use_dft=use_dft))


def groth16_h_mont(F, A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """groth16_h (Fig. 2 and Section IV-A) on Montgomery-form limbs."""
    F = fld.get(F)
    a, b, c = (from_mont_limbs(F, v) for v in (A, B, C))
    return to_mont_limbs(F, groth16_h(F, a, b, c))


def ntt_at_mont(F, X: np.ndarray, ks, inverse: bool = False,
                shift_mont: int | None = None) -> list[int]:
    """Selected outputs k of the transform, each from the definition alone
    (O(n) per output), returned as Montgomery-form integers."""
    F = fld.get(F)
    x = from_mont_limbs(F, X)
    n = len(x)
    L = n.bit_length() - 1
    r = F.r
    w = F.root(L, inverse=inverse)
    shift = None if shift_mont is None else F.from_mont(shift_mont)
    out = []
    if not inverse:
        if shift is not None:
            # A_k = sum_j a_j (shift * w^k)^j
            for k in ks:
                out.append(F.to_mont(eval_poly(x, shift * pow(w, k, r) % r, r)))
        else:
            for k in ks:
                out.append(F.to_mont(dft_at(x, w, k, r)))
        return out
    ninv = pow(n, -1, r)
    for k in ks:
        v = dft_at(x, w, k, r) * ninv % r
        if shift is not None:
            v = v * pow(pow(shift, -1, r), k, r) % r
        out.append(F.to_mont(v))
    return out
