"""Prime-field constants for the oracle, derived here from the modulus alone.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA path never
does.

Everything is plain Python integers (arbitrary precision).  Field operations
return values in [0, r), as the paper states for its finite fields
(Section II, background on ZKPs: results of field operations lie in [0, p)).

The paper names BLS12-381 and BLS12-377 (Section II); the scalar field F_r
of BLS12-381 is the NTT input field, BN254 F_r is the second field of the
workload, and BLS12-377 F_r the third.  Neither the generator nor the root of
unity is printed in the paper; the readings used are

* the multiplicative generator g is 7 for BLS12-381 F_r, 5 for BN254 F_r and
  22 for BLS12-377 F_r (checked by the tests: g is a quadratic non-residue,
  g^((r-1)/q) != 1 for every prime q | r - 1 that trial division finds, and
  for BLS12-377 F_r, whose r - 1 is fully factored, for every prime factor);
* the primitive 2^s-th root is omega_max = g^((r-1)/2^s) with s the 2-adicity
  of r - 1, and omega_n = omega_max^(2^(s-L)) for n = 2^L (Section II-B only
  asks only for a primitive root of unity of order n);
* Montgomery radix R = 2^256 (8 limbs of 32 bits, Section II: "word-sized
  limbs").
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field

BLS12_381_FR = 0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001
BN254_FR = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001
BLS12_377_FR = 0x12AB655E9A2CA55660B44D1E5C37B00159AA76FED00000010A11800000000001

LIMBS = 8
LIMB_BITS = 32
R_BITS = LIMBS * LIMB_BITS  # 256


def two_adicity(r: int) -> int:
    """Largest s with 2^s | r - 1: the largest power-of-two transform the
    field supports (Section II-B needs a primitive n-th root of unity)."""
    s = 0
    m = r - 1
    while m % 2 == 0:
        m //= 2
        s += 1
    return s


@dataclass(frozen=True)
class Field:
    name: str
    r: int
    g: int
    s: int = dc_field(init=False)
    R: int = dc_field(init=False)        # 2^256 mod r
    R2: int = dc_field(init=False)       # 2^512 mod r
    Rinv: int = dc_field(init=False)     # 2^-256 mod r
    rprime: int = dc_field(init=False)   # -r^-1 mod 2^32
    omega_max: int = dc_field(init=False)

    def __post_init__(self):
        r = self.r
        s = two_adicity(r)
        object.__setattr__(self, "s", s)
        object.__setattr__(self, "R", pow(2, R_BITS, r))
        object.__setattr__(self, "R2", pow(2, 2 * R_BITS, r))
        object.__setattr__(self, "Rinv", pow(2, -R_BITS, r))
        object.__setattr__(self, "rprime", (-pow(r, -1, 1 << LIMB_BITS)) % (1 << LIMB_BITS))
        object.__setattr__(self, "omega_max", pow(self.g, (r - 1) >> s, r))

    # --- plain field operations (Python big ints; results in [0, r)) -------
    def add(self, a: int, b: int) -> int:
        """FF_add (Section IV-B-1): a + b reduced to [0, r)."""
        return (a + b) % self.r

    def sub(self, a: int, b: int) -> int:
        """FF_sub (Section IV-B-1): a - b reduced to [0, r)."""
        return (a - b) % self.r

    def mul(self, a: int, b: int) -> int:
        """FF_mul (Section IV-B) by definition: a * b reduced to [0, r)."""
        return (a * b) % self.r

    def inv(self, a: int) -> int:
        """a^-1 mod r (needed for n^-1 and the coset inverse, Section II-B and
        Fig. 2)."""
        if a % self.r == 0:
            raise ZeroDivisionError("0 has no inverse")
        return pow(a, -1, self.r)

    # --- Montgomery representation (R = 2^256) --------------------------------
    def to_mont(self, x: int) -> int:
        """Montgomery form x * 2^256 mod r (the representation the paper's
        FF_mul works on, Section IV-B)."""
        return (x * self.R) % self.r

    def from_mont(self, X: int) -> int:
        """Canonical value X * 2^-256 mod r of a Montgomery-form X."""
        return (X * self.Rinv) % self.r

    def mont_mul(self, X: int, Y: int) -> int:
        """Montgomery product X*Y*R^-1 mod r, by definition."""
        return (X * Y * self.Rinv) % self.r

    # --- roots of unity ------------------------------------------------------
    def root(self, log_n: int, inverse: bool = False) -> int:
        """Primitive 2^log_n-th root omega_n = omega_max^(2^(s - log_n))."""
        if not 0 <= log_n <= self.s:
            raise ValueError(f"log_n={log_n} outside [0, {self.s}] for {self.name}")
        w = pow(self.omega_max, 1 << (self.s - log_n), self.r)
        return pow(w, -1, self.r) if inverse else w


BLS12_381 = Field("bls12_381_fr", BLS12_381_FR, 7)
BN254 = Field("bn254_fr", BN254_FR, 5)
BLS12_377 = Field("bls12_377_fr", BLS12_377_FR, 22)
FIELDS = {f.name: f for f in (BLS12_381, BN254, BLS12_377)}
FIELD_IDS = {"bls12_381_fr": 0, "bn254_fr": 1, "bls12_377_fr": 2}


def get(name_or_field) -> Field:
    if isinstance(name_or_field, Field):
        return name_or_field
    if isinstance(name_or_field, int):
        return (BLS12_381, BN254, BLS12_377)[name_or_field]
    return FIELDS[name_or_field]
