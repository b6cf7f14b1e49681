"""The sharded transform's device steps on one GPU: all G shards run in one
process (exchange by copies; no kernel waits on another) through the
library's kernels, and the gathered result equals the C oracle's transform
of the whole vector, bit for bit.  Also the scale-by-powers kernel the
twiddle step uses, against the oracle's arithmetic."""
import numpy as np
import pytest

from oracle import cpu
from oracle import field as fld
from oracle import ntt_ref as ref
from workloads import uniform_elements

from gpu_util import first_mismatch, to_dev, to_host

pytestmark = pytest.mark.gpu
FIELDS = [fld.BLS12_381, fld.BN254, fld.BLS12_377]
KINDS = ["ntt", "intt", "coset_ntt", "coset_intt"]


def _oracle(F, X, kind):
    inverse = kind.endswith("intt")
    sh = F.to_mont(F.g) if kind.startswith("coset") else None
    if X.shape[0] <= 1 << 10:
        return ref.ntt_mont(F, X, inverse=inverse, shift_mont=sh)
    return cpu.ntt(F, X, inverse=inverse, shift_mont=sh)


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("world,L", [(1, 10), (2, 12), (4, 16), (8, 20), (8, 6)])
@pytest.mark.parametrize("kind", KINDS)
def test_emulated_shards_equal_the_oracle(F, world, L, kind):
    import torch
    from paper_2509_22684_gb300.sharded import (LibraryOps, ShardedNTT, emulate, gather_output,
                                                scatter_input)
    X = uniform_elements(F.r, 1 << L, 700 + L)
    inverse = kind.endswith("intt")
    shift = F.to_mont(F.g) if kind.startswith("coset") else None
    ops = LibraryOps(F.name)
    shards = [ShardedNTT(F.name, L, world, r, inverse=inverse, coset_shift=shift, ops=ops)
              for r in range(world)]
    xs = scatter_input(to_dev(X), world)
    outs = emulate(shards, xs)
    got = to_host(gather_output(outs, L))
    ops.close()
    want = _oracle(F, X, kind)
    assert np.array_equal(got, want), first_mismatch(got, want)


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("n", [1, 7, 1000, 1 << 16, (1 << 16) + 3])
def test_scale_powers_matches_the_oracle(F, n):
    import paper_2509_22684_gb300 as zk
    X = uniform_elements(F.r, n, 31 + n)
    c, base = uniform_elements(F.r, 2, 5 + n)
    c_m = int.from_bytes(c.tobytes(), "little")
    b_m = int.from_bytes(base.tobytes(), "little")
    x = to_dev(X)
    got = to_host(zk.scale_powers(F.name, x, c_m, b_m))
    vals = ref.from_mont_limbs(F, X)
    cv, bv = F.from_mont(c_m), F.from_mont(b_m)
    want = ref.to_mont_limbs(F, [v * cv * pow(bv, i, F.r) % F.r for i, v in enumerate(vals)])
    assert np.array_equal(got, want), first_mismatch(got, want)
    # in place, and base 1 (a constant scale)
    zk.scale_powers(F.name, x, c_m, F.to_mont(1), out=x)
    want1 = ref.to_mont_limbs(F, [v * cv % F.r for v in vals])
    assert np.array_equal(to_host(x), want1)


def test_scale_powers_argument_errors():
    import torch
    import paper_2509_22684_gb300 as zk
    from paper_2509_22684_gb300 import ZkNttError
    F = fld.BN254
    x = torch.zeros((16, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(ZkNttError):
        zk.scale_powers(F.name, x, F.r, 1)      # c not canonical
    with pytest.raises(ZkNttError):
        zk.scale_powers(F.name, x, 1, F.r + 5)  # base not canonical


@pytest.mark.parametrize("F", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("log_g", [1, 2, 3])
@pytest.mark.parametrize("inverse", [False, True])
def test_block_dft_matches_its_definition(F, log_g, inverse):
    """zkntt_block_dft against the definition, out[k b + i] = sum_r
    x[r b + i] w^(r k) with w of order G (inverse: w^-1), in place too."""
    import paper_2509_22684_gb300 as zk
    G, b = 1 << log_g, 1000
    X = uniform_elements(F.r, G * b, 41 + log_g)
    vals = ref.from_mont_limbs(F, X)
    w = F.root(log_g, inverse)
    want = ref.to_mont_limbs(F, [sum(vals[r * b + i] * pow(w, r * k, F.r) for r in range(G)) % F.r
                                 for k in range(G) for i in range(b)])
    x = to_dev(X)
    got = to_host(zk.block_dft(F.name, x, log_g, inverse=inverse))
    assert np.array_equal(got, want), first_mismatch(got, want)
    zk.block_dft(F.name, x, log_g, inverse=inverse, out=x)
    assert np.array_equal(to_host(x), want)
