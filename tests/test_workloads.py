"""The seeded generators: determinism, range, and agreement with the scalar
statement of the same stream."""
import numpy as np

from oracle import field as fld
from workloads import (batch_jobs, limbs_to_ints, poisson_trace, splitmix64,
                       splitmix64_scalar, uniform_elements, uniform_elements_scalar)


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: first outputs as published with the algorithm
    # (the same constants appear in Vigna's reference implementation notes).
    assert splitmix64_scalar(0, 0) == 0xE220A8397B1DCDAF
    assert splitmix64_scalar(0, 1) == 0x6E789E6AA1B965F4
    # the test vector usually quoted for seed 1234567
    assert splitmix64_scalar(1234567, 0) == 6457827717110365317
    v = splitmix64(0, 0, 3)
    assert [int(x) for x in v] == [splitmix64_scalar(0, i) for i in range(3)]


def test_uniform_matches_scalar_statement():
    for F in (fld.BLS12_381, fld.BN254, fld.BLS12_377):
        X = uniform_elements(F.r, 257, 77)
        assert limbs_to_ints(X) == uniform_elements_scalar(F.r, 257, 77)


def test_uniform_range_and_prefix():
    F = fld.BN254
    X = uniform_elements(F.r, 5000, 3)
    vals = limbs_to_ints(X)
    assert all(0 <= v < F.r for v in vals)
    assert max(vals) > F.r * 0.99 and min(vals) < F.r * 0.01
    Y = uniform_elements(F.r, 1000, 3)
    assert np.array_equal(X[:1000], Y)


def test_batch_and_trace_are_deterministic():
    a = batch_jobs(4000)
    b = batch_jobs(4000)
    assert a == b and len(a) == 64
    assert {j.log_n for j in a} <= set(range(10, 21))
    t = poisson_trace(5000, 200, 100.0)
    assert all(t[i].arrival_s < t[i + 1].arrival_s for i in range(len(t) - 1))
    assert {q.log_n for q in t} <= set(range(12, 25))


def test_threaded_generator_equals_the_sequential_one():
    """uniform_elements_threaded draws exactly uniform_elements' values, for
    block sizes that split the candidates many ways (including blocks smaller
    than one accepted value's share and a wave that ends mid-block)."""
    from workloads import uniform_elements_threaded
    for F in (fld.BLS12_381, fld.BN254):
        for n, block, threads in ((0, 8, 2), (1, 1, 3), (1000, 7, 4), (20000, 512, 5),
                                  (100000, 1 << 14, 16)):
            want = uniform_elements(F.r, n, 91)
            got = uniform_elements_threaded(F.r, n, 91, threads=threads, block=block)
            assert got.shape == (n, 8) and np.array_equal(got, want), (F.name, n, block)
