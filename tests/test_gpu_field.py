"""GPU field arithmetic (the butterfly operations) against the oracle's
definitions, on random values and edge values, through the C ABI."""
import numpy as np
import pytest

from oracle import field as fld
from workloads import ints_to_limbs, limbs_to_ints, splitmix64, uniform_elements

from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu
FIELDS = [fld.BLS12_381, fld.BN254, fld.BLS12_377]


def _edge_values(F):
    r = F.r
    base = [0, 1, 2, r - 1, r - 2, F.R, F.to_mont(1), F.to_mont(r - 1), (1 << 255) % r,
            r >> 1, (r >> 1) + 1, 0xFFFFFFFF, (1 << 32) % r, (1 << 224) - 1]
    # values whose limbs sit at 0xffffffff where r allows it
    for k in range(8):
        v = ((1 << (32 * (k + 1))) - 1) % r
        base.append(v)
    return [v % r for v in base]


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["mul", "add", "sub", "sub_lazy"])
def test_field_op(F, op):
    import paper_2509_22684_gb300 as zk
    n = 1 << 16
    A = limbs_to_ints(uniform_elements(F.r, n, 11))
    B = limbs_to_ints(uniform_elements(F.r, n, 12))
    edge = _edge_values(F)
    # every pair of edge values, placed at the front
    pairs = [(x, y) for x in edge for y in edge]
    for i, (x, y) in enumerate(pairs):
        A[i], B[i] = x, y
    a = to_dev(ints_to_limbs(A))
    b = to_dev(ints_to_limbs(B))
    c = zk.field_op(F.name, op, a, b)
    got = limbs_to_ints(to_host(c))
    r = F.r
    if op == "mul":
        want = [F.mont_mul(x, y) for x, y in zip(A, B)]
    elif op == "add":
        want = [(x + y) % r for x, y in zip(A, B)]
    elif op == "sub":
        want = [(x - y) % r for x, y in zip(A, B)]
    else:
        # the exact integer x + r - y (no reduction), in (0, 2r)
        want = [x + r - y for x, y in zip(A, B)]
        assert all(0 < w < 2 * r for w in want)
    bad = [i for i in range(n) if got[i] != want[i]]
    assert not bad, f"{len(bad)} mismatches, first at {bad[0]}: {A[bad[0]]:x} {B[bad[0]]:x}"


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
def test_mul_second_operand_any_256_bit_value(F):
    """The product's limb-scanned operand may be any value below 2^256 (the
    butterfly feeds it x + r - y unreduced); the result is still the canonical
    a b 2^-256 mod r."""
    import paper_2509_22684_gb300 as zk
    n = 1 << 14
    r = F.r
    A = limbs_to_ints(uniform_elements(r, n, 31))
    words = splitmix64(32, 0, 4 * n).reshape(n, 4)        # uniform over [0, 2^256)
    B = [int(w[0]) | int(w[1]) << 64 | int(w[2]) << 128 | int(w[3]) << 192 for w in words]
    top = (1 << 256) - 1
    edge_b = [top, top - 1, r, r + 1, 2 * r - 1, 2 * r, 2 * r + 1, top - r, 1 << 255, (1 << 255) - 1]
    edge_a = [0, 1, r - 1, r - 2, F.to_mont(1), F.to_mont(r - 1), (1 << 224) - 1]
    pairs = [(x, y) for x in edge_a for y in edge_b]
    for i, (x, y) in enumerate(pairs):
        A[i], B[i] = x, y
    got = limbs_to_ints(to_host(zk.field_op(F.name, "mul", to_dev(ints_to_limbs(A)),
                                            to_dev(ints_to_limbs(B)))))
    want = [F.mont_mul(x, y) for x, y in zip(A, B)]
    bad = [i for i in range(n) if got[i] != want[i]]
    assert not bad, f"{len(bad)} mismatches, first at {bad[0]}: {A[bad[0]]:x} {B[bad[0]]:x}"


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
def test_pointwise(F):
    import paper_2509_22684_gb300 as zk
    n = 4096
    A, B, C = (limbs_to_ints(uniform_elements(F.r, n, s)) for s in (21, 22, 23))
    z = F.to_mont(12345)
    out = zk.pointwise(F.name, *(to_dev(ints_to_limbs(v)) for v in (A, B, C)), z)
    got = limbs_to_ints(to_host(out))
    r = F.r
    want = [F.mont_mul((F.mont_mul(a, b) - c) % r, z) for a, b, c in zip(A, B, C)]
    assert got == want


def test_field_info_matches_oracle():
    import paper_2509_22684_gb300 as zk
    for F in FIELDS:
        m, g, s = zk.field_info(F.name)
        assert m == F.r and g == F.to_mont(F.g) and s == F.s
