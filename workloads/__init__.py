"""Seeded synthetic workloads shared by the oracle side and the CUDA side.

This module draws random numbers and nothing else: it holds none of the
transform's arithmetic (no field multiplication, no roots of unity, no
Montgomery conversion).  Callers pass the field modulus in as a plain integer.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Output number i of the stream seeded with
``seed`` is ``mix(seed + (i + 1) * GAMMA)``, so any slice of the stream can be
computed without the preceding ones (a counter-based generator).

Field elements: candidate c takes stream words 4c..4c+3 as a little-endian
256-bit integer, keeps its low ``modulus.bit_length()`` bits and is accepted
iff it is below the modulus (exact rejection sampling, so accepted values are
uniform on [0, modulus)).  The accepted values are the raw 8 x 32-bit
little-endian limbs handed to the transform; since x -> x*2^256 mod r is a
bijection of [0, r), a uniform raw value is also a uniform element whatever
representation the consumer reads it in.

The paper's inputs are uniformly random field elements (Section III-B, where
test cases are generated; Section IV-C notes the inputs are uniformly random).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1

FIELD_NAMES = ("bls12_381_fr", "bn254_fr")
KINDS = ("ntt", "intt", "coset_ntt", "coset_intt")


def splitmix64_scalar(seed: int, index: int) -> int:
    """Output number ``index`` (0-based) of the SplitMix64 stream, one value."""
    z = (seed + (index + 1) * GAMMA) & _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the stream as a uint64 array."""
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + idx * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def _words_of(modulus: int) -> list[int]:
    return [(modulus >> (64 * i)) & _MASK64 for i in range(4)]


def uniform_elements(modulus: int, n: int, seed: int) -> np.ndarray:
    """n values uniform on [0, modulus) as a C-contiguous uint32 array [n, 8].

    Limb 0 is the least significant 32 bits.  Deterministic in (modulus, n,
    seed); a prefix of a longer draw equals the shorter draw.
    """
    if modulus <= 1 or modulus.bit_length() > 256:
        raise ValueError("modulus must be in (1, 2^256)")
    out = np.empty((n, 4), dtype=np.uint64)
    if n == 0:
        return out.view(np.uint32).reshape(0, 8)
    bits = modulus.bit_length()
    top_bits = bits - 192
    top_mask = np.uint64((1 << top_bits) - 1) if top_bits < 64 else np.uint64(_MASK64)
    mw = _words_of(modulus)
    accept_rate = modulus / float(1 << bits)
    filled = 0
    cand = 0
    while filled < n:
        want = n - filled
        chunk = int(want / accept_rate * 1.05) + 64
        w = splitmix64(seed, 4 * cand, 4 * chunk).reshape(chunk, 4)
        w[:, 3] &= top_mask
        # lexicographic compare from the most significant word down
        less = np.zeros(chunk, dtype=bool)
        eq = np.ones(chunk, dtype=bool)
        for k in (3, 2, 1, 0):
            mk = np.uint64(mw[k])
            less |= eq & (w[:, k] < mk)
            eq &= w[:, k] == mk
        acc = w[less]
        take = min(want, acc.shape[0])
        out[filled:filled + take] = acc[:take]
        filled += take
        cand += chunk
    return np.ascontiguousarray(out).view(np.uint32).reshape(n, 8)


def _accepted_block(modulus: int, seed: int, cand0: int, count: int) -> np.ndarray:
    """Accepted values among candidates cand0 .. cand0+count-1, in order, as
    [k, 4] uint64 words (the candidate rule of ``uniform_elements``)."""
    bits = modulus.bit_length()
    top_bits = bits - 192
    top_mask = np.uint64((1 << top_bits) - 1) if top_bits < 64 else np.uint64(_MASK64)
    mw = _words_of(modulus)
    w = splitmix64(seed, 4 * cand0, 4 * count).reshape(count, 4)
    w[:, 3] &= top_mask
    less = np.zeros(count, dtype=bool)
    eq = np.ones(count, dtype=bool)
    for k in (3, 2, 1, 0):
        mk = np.uint64(mw[k])
        less |= eq & (w[:, k] < mk)
        eq &= w[:, k] == mk
    return w[less]


def uniform_elements_threaded(modulus: int, n: int, seed: int, threads: int | None = None,
                              block: int = 1 << 20) -> np.ndarray:
    """The same values as ``uniform_elements(modulus, n, seed)``, drawn by
    several threads at once (for vectors of 2^26 elements and more): the
    candidates are cut into consecutive blocks of ``block`` candidates, each
    thread filters whole blocks, and the accepted values are concatenated in
    candidate order until n are taken."""
    import concurrent.futures as cf
    import os
    if modulus <= 1 or modulus.bit_length() > 256:
        raise ValueError("modulus must be in (1, 2^256)")
    threads = threads or min(16, os.cpu_count() or 1)
    out = np.empty((n, 4), dtype=np.uint64)
    filled, nxt = 0, 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        while filled < n:
            wave = [ex.submit(_accepted_block, modulus, seed, (nxt + i) * block, block)
                    for i in range(threads)]
            nxt += threads
            for f in wave:
                acc = f.result()
                take = min(n - filled, acc.shape[0])
                out[filled:filled + take] = acc[:take]
                filled += take
                if filled == n:
                    break
    return out.view(np.uint32).reshape(n, 8)


def uniform_elements_scalar(modulus: int, n: int, seed: int) -> list[int]:
    """Plain-Python statement of ``uniform_elements`` (for tests), as ints."""
    bits = modulus.bit_length()
    mask = (1 << bits) - 1
    vals = []
    c = 0
    while len(vals) < n:
        v = 0
        for k in range(4):
            v |= splitmix64_scalar(seed, 4 * c + k) << (64 * k)
        v &= mask
        if v < modulus:
            vals.append(v)
        c += 1
    return vals


def limbs_to_ints(x: np.ndarray) -> list[int]:
    """[n, 8] uint32 limbs -> list of Python ints (no arithmetic, a re-layout)."""
    b = np.ascontiguousarray(x, dtype=np.uint32).tobytes()
    return [int.from_bytes(b[32 * i:32 * i + 32], "little") for i in range(x.shape[0])]


def ints_to_limbs(vals) -> np.ndarray:
    """list of ints in [0, 2^256) -> [n, 8] uint32 limbs."""
    vals = list(vals)
    buf = b"".join(int(v).to_bytes(32, "little") for v in vals)
    return np.frombuffer(buf, dtype=np.uint32).reshape(len(vals), 8).copy()


def _uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of stream words."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


@dataclass(frozen=True)
class Job:
    field: str
    log_n: int
    kind: str
    seed: int


def batch_jobs(seed: int, count: int = 64, lmin: int = 10, lmax: int = 20,
               fields=FIELD_NAMES, kinds=("ntt", "intt")) -> list[Job]:
    """Uneven batch: log_n uniform over {lmin..lmax} (log-uniform sizes), field
    and kind uniform over the given lists; job i draws its elements with seed
    ``seed * 1000 + i``."""
    u = _uniform01(seed, 0, 3 * count).reshape(count, 3)
    jobs = []
    for i in range(count):
        L = lmin + min(int(u[i, 0] * (lmax - lmin + 1)), lmax - lmin)
        f = fields[min(int(u[i, 1] * len(fields)), len(fields) - 1)]
        k = kinds[min(int(u[i, 2] * len(kinds)), len(kinds) - 1)]
        jobs.append(Job(f, L, k, seed * 1000 + i))
    return jobs


@dataclass(frozen=True)
class Request:
    arrival_s: float
    log_n: int
    kind: str
    seed: int


def poisson_trace(seed: int, count: int, rate_per_s: float, lmin: int = 12,
                  lmax: int = 24, kinds=KINDS) -> list[Request]:
    """Poisson arrivals (exponential gaps with mean 1/rate), log_n uniform over
    {lmin..lmax}, kind uniform over ``kinds``."""
    if rate_per_s <= 0:
        raise ValueError("rate must be positive")
    u = _uniform01(seed, 0, 3 * count).reshape(count, 3)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log1p(-u[i, 0]) / rate_per_s
        L = lmin + min(int(u[i, 1] * (lmax - lmin + 1)), lmax - lmin)
        k = kinds[min(int(u[i, 2] * len(kinds)), len(kinds) - 1)]
        out.append(Request(t, L, k, seed * 100000 + i))
    return out
