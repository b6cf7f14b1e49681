"""Pins for the oracle's field layer against number theory and the published
field definitions (tests/golden/fields.txt), not against itself."""
import os
import random

import pytest

from oracle import field as fld

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fields.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[1] == "factor":           # name factor p e (a list)
                out.setdefault(parts[0], {}).setdefault("factors", []).append(
                    (int(parts[2], 0), int(parts[3], 0)))
                continue
            name, key, val = parts
            out.setdefault(name, {})[key] = int(val, 0)
    return out


def _is_probable_prime(n, rounds=40):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    rng = random.Random(12345)
    for _ in range(rounds):
        a = rng.randrange(2, n - 1)
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


@pytest.mark.parametrize("F", [fld.BLS12_381, fld.BN254, fld.BLS12_377], ids=lambda f: f.name)
def test_modulus_matches_published_definition(F):
    g = _golden()[F.name]
    assert F.r == g["r"]
    assert F.g == g["g"]
    assert F.r.bit_length() == g["bits"]
    assert _is_probable_prime(F.r)


@pytest.mark.parametrize("F", [fld.BLS12_381, fld.BN254, fld.BLS12_377], ids=lambda f: f.name)
def test_two_adicity(F):
    g = _golden()[F.name]
    assert F.s == g["two_adicity"]
    assert (F.r - 1) % (1 << F.s) == 0
    assert ((F.r - 1) >> F.s) % 2 == 1


@pytest.mark.parametrize("F", [fld.BLS12_381, fld.BN254, fld.BLS12_377], ids=lambda f: f.name)
def test_generator_is_non_residue_and_root_has_exact_order(F):
    r = F.r
    # Euler's criterion: g is a quadratic non-residue, so g^((r-1)/2^s) has order exactly 2^s
    assert pow(F.g, (r - 1) // 2, r) == r - 1
    w = F.omega_max
    assert pow(w, 1 << F.s, r) == 1
    assert pow(w, 1 << (F.s - 1), r) == r - 1
    for L in range(0, F.s + 1):
        wl = F.root(L)
        assert pow(wl, 1 << L, r) == 1
        if L >= 1:
            assert pow(wl, 1 << (L - 1), r) == r - 1   # omega^(n/2) = -1
        assert wl * F.root(L, inverse=True) % r == 1


@pytest.mark.parametrize("F", [fld.BLS12_381, fld.BN254, fld.BLS12_377], ids=lambda f: f.name)
def test_generator_small_factor_orders(F):
    """g^((r-1)/q) != 1 for the small prime factors q of r - 1 we can find by
    trial division, so g is not confined to a subgroup of index q."""
    r = F.r
    m = r - 1
    q = 2
    found = []
    while q < 20000:
        if m % q == 0:
            found.append(q)
            while m % q == 0:
                m //= q
        q += 1
    assert 2 in found and 3 in found
    for q in found:
        assert pow(F.g, (r - 1) // q, r) != 1


@pytest.mark.parametrize("F", [fld.BLS12_381, fld.BN254, fld.BLS12_377], ids=lambda f: f.name)
def test_montgomery_constants(F):
    r = F.r
    assert F.R == (1 << 256) % r
    assert F.R * F.Rinv % r == 1
    assert (F.r * F.rprime) % (1 << 32) == (1 << 32) - 1   # r * r' = -1 mod 2^32
    g = _golden()[F.name]
    assert F.rprime == g["rprime32"]
    rng = random.Random(7)
    for _ in range(200):
        a, b = rng.randrange(r), rng.randrange(r)
        assert F.from_mont(F.to_mont(a)) == a
        # Montgomery product corresponds to the plain product under the map
        assert F.from_mont(F.mont_mul(F.to_mont(a), F.to_mont(b))) == a * b % r


def test_bls12_modulus_low_limb_structure():
    """r = 1 mod 2^32 for the BLS12-381 and BLS12-377 scalar fields (the low
    limb is 1, r' = 2^32 - 1); the GPU path is allowed to exploit this, so pin
    it."""
    for F in (fld.BLS12_381, fld.BLS12_377):
        assert F.r % (1 << 32) == 1
        assert F.rprime == 0xFFFFFFFF


def test_bls12_377_generator_has_full_order():
    """r - 1 of BLS12-377 F_r is completely factored in the golden file, so
    g = 22 is checked to generate the whole multiplicative group:
    g^((r-1)/q) != 1 for every prime q | r - 1."""
    F = fld.BLS12_377
    facs = _golden()[F.name]["factors"]
    prod = 1
    for q, e in facs:
        assert _is_probable_prime(q)
        prod *= q ** e
    assert prod == F.r - 1
    for q, _ in facs:
        assert pow(F.g, (F.r - 1) // q, F.r) != 1
    # and a non-generator is rejected by the same check (11 is a non-residue
    # of smaller order), so the check is not vacuous
    assert any(pow(11, (F.r - 1) // q, F.r) == 1 for q, _ in facs)


def test_moduli_follow_from_curve_parameters():
    g = _golden()
    x = g["bls12_381_fr"]["x"]
    assert fld.BLS12_381.r == x ** 4 - x ** 2 + 1
    u = g["bn254_fr"]["u"]
    assert fld.BN254.r == 36 * u ** 4 + 36 * u ** 3 + 18 * u ** 2 + 6 * u + 1
    x = g["bls12_377_fr"]["x"]
    assert fld.BLS12_377.r == x ** 4 - x ** 2 + 1
