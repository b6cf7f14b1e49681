"""The sharded transform's host logic on CPU: world-size 2 and 4 gloo process
groups run ShardedNTT (layouts, per-rank constants, the all-to-all and the
G-point combine) with its device steps replaced by an oracle-backed stand-in
defined here, and the gathered result equals the oracle's transform of the
whole vector (Section II-B; coset kinds as in Fig. 2)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import field as fld
from oracle import ntt_ref as ref
from workloads import uniform_elements

FMAP = {"bls12_381_fr": fld.BLS12_381, "bn254_fr": fld.BN254}


class OracleOps:
    """The device steps of a shard, stated with the oracle on CPU tensors."""

    def __init__(self, F):
        self.F = F

    def _vals(self, x):
        return ref.from_mont_limbs(self.F, x.numpy().view(np.uint32).reshape(-1, 8))

    def _tensor(self, vals):
        return torch.from_numpy(ref.to_mont_limbs(self.F, vals).view(np.int32).copy())

    def ntt(self, x, log_n, inverse, shift_mont):
        X = x.numpy().view(np.uint32).reshape(-1, 8)
        assert X.shape[0] == 1 << log_n
        Y = ref.ntt_mont(self.F, X, inverse=inverse, shift_mont=shift_mont)
        return torch.from_numpy(Y.view(np.int32).copy())

    def scale_powers(self, x, c_mont, base_mont):
        F = self.F
        c, base = F.from_mont(c_mont), F.from_mont(base_mont)
        out = [v * c * pow(base, i, F.r) % F.r for i, v in enumerate(self._vals(x))]
        x.copy_(self._tensor(out))
        return x

    def add(self, a, b):
        return self._tensor([(u + v) % self.F.r for u, v in zip(self._vals(a), self._vals(b))])

    def sub(self, a, b):
        return self._tensor([(u - v) % self.F.r for u, v in zip(self._vals(a), self._vals(b))])


class OracleOpsBlock(OracleOps):
    """As OracleOps, with the fused G-point step stated from its definition:
    out[k b + i] = sum_r u[r b + i] w^(r k), w of order G."""

    def block_dft(self, u, log_g, inverse):
        F, G = self.F, 1 << log_g
        vals = self._vals(u)
        b = len(vals) // G
        w = F.root(log_g, inverse)
        out = [sum(vals[r * b + i] * pow(w, r * k, F.r) for r in range(G)) % F.r
               for k in range(G) for i in range(b)]
        return self._tensor(out)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _kind_args(F, kind):
    return kind.endswith("intt"), (F.to_mont(F.g) if kind.startswith("coset") else None)


def _worker(rank, world, port, field, L, kinds, out, block=False):
    import torch.distributed as dist
    from paper_2509_22684_gb300.sharded import ShardedNTT, scatter_input
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    F = FMAP[field]
    X = uniform_elements(F.r, 1 << L, 600 + L)
    x = scatter_input(torch.from_numpy(X.view(np.int32).copy()), world)[rank]
    for kind in kinds:
        inverse, shift = _kind_args(F, kind)
        ops = OracleOpsBlock(F) if block else OracleOps(F)
        sh = ShardedNTT(field, L, world, rank, inverse=inverse, coset_shift=shift, ops=ops)
        assert torch.equal(sh.input_indices(), torch.arange(rank, 1 << L, world))
        y = sh.execute(x)
        out[(rank, kind)] = (y.numpy().tobytes(), sh.output_indices().numpy().tobytes())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("block", [False, True], ids=["butterflies", "block_step"])
@pytest.mark.parametrize("world,field,L", [(2, "bls12_381_fr", 6), (4, "bn254_fr", 6),
                                           (4, "bls12_381_fr", 7), (2, "bn254_fr", 2)])
def test_sharded_transform_over_gloo_ranks_equals_the_oracle(world, field, L, block):
    from paper_2509_22684_gb300 import build
    from paper_2509_22684_gb300.sharded import gather_output
    build.build()   # the ranks read the field constants through the library
    kinds = ["ntt", "intt", "coset_ntt", "coset_intt"]
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, field, L, kinds, out, block))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    F = FMAP[field]
    X = uniform_elements(F.r, 1 << L, 600 + L)
    for kind in kinds:
        inverse, shift = _kind_args(F, kind)
        shards = [torch.from_numpy(np.frombuffer(out[(r, kind)][0], dtype=np.int32).reshape(-1, 8).copy())
                  for r in range(world)]
        idx = np.concatenate([np.frombuffer(out[(r, kind)][1], dtype=np.int64) for r in range(world)])
        assert sorted(idx.tolist()) == list(range(1 << L))      # the shards partition the output
        got = gather_output(shards, L).numpy().view(np.uint32)
        want = ref.ntt_mont(F, X, inverse=inverse, shift_mont=shift)
        assert np.array_equal(got, want), kind
        # gather_output agrees with output_indices
        flat = np.concatenate([s.numpy().view(np.uint32) for s in shards])
        assert np.array_equal(want[idx], flat), kind


def test_sharded_arguments_are_checked():
    from paper_2509_22684_gb300 import build
    from paper_2509_22684_gb300.sharded import ShardedNTT
    build.build()
    F = fld.BLS12_381
    with pytest.raises(ValueError):
        ShardedNTT("bls12_381_fr", 8, 3, 0, ops=OracleOps(F))      # not a power of two
    with pytest.raises(ValueError):
        ShardedNTT("bls12_381_fr", 5, 8, 0, ops=OracleOps(F))      # 8^2 > 2^5
    with pytest.raises(ValueError):
        ShardedNTT("bls12_381_fr", 8, 2, 2, ops=OracleOps(F))      # rank out of range
    with pytest.raises(ValueError):
        ShardedNTT("bn254_fr", 29, 2, 0, ops=OracleOps(fld.BN254))  # above 2-adicity
