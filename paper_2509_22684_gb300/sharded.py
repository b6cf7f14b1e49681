"""One transform sharded over G ranks: the four-step decomposition with a
single all-to-all exchange.

The paper notes that a block NTT is bounded by on-chip memory, so large
transforms are split into sub-transforms joined by twiddle factors (Section
II-B).  The same split distributes a transform of n = 2^L elements over
G = 2^g GPUs (n = G * n2, n2 = n / G, b = n2 / G):

    input:   rank r holds x_r[j2] = a[r + G j2]            (j2 < n2; cyclic)
    local:   y_r = NTT_n2(x_r)                               (w_n2 = w_n^G)
    twiddle: z_r[k2] = y_r[k2] * w_n^(r k2)
    all-to-all: rank r sends z_r[s b .. (s+1) b) to rank s
    local:   for each i < b, the G-point transform over r of u_s[r][i]:
             A[k2 + n2 k1] = sum_r u_s[r][i] w_G^(r k1),   k2 = s b + i
    output:  rank s holds A[s b + i + n2 k1] as out_s[k1][i]   (k1 < G, i < b)

since w_n^((r + G j2)(k2 + n2 k1)) = w_n^(r k2) w_G^(r k1) w_n2^(j2 k2).  The
inverse runs the same steps with w^-1; its scale n^-1 = n2^-1 G^-1 is the
local inverse's n2^-1 times G^-1 folded into the twiddle step.  A coset
forward transform (input a_j g^j, Fig. 2) uses a local coset transform with
shift g^G and folds g^r into the twiddle step; a coset inverse multiplies
output k by g^-k at the end.

Every arithmetic step runs in the library's kernels (``LibraryOps``): the
local transform (zkntt_execute), the twiddle and constant scales
(zkntt_scale_powers) and the G-point transforms, one kernel over all columns
(zkntt_block_dft; with device steps that lack it, radix-2 butterflies on whole
blocks through zkntt_field_op).  The exchange is torch.distributed's all_to_all_single
(NCCL between GPUs, no multicast); ``emulate`` runs all G shards in one
process on one device with the exchange done by copies.  The host computes
only the per-rank constants (powers of w_n, g, G^-1) with Python integers.
"""
from __future__ import annotations

import torch

R_MONT = 1 << 256


class HostField:
    """The field's modulus, generator and roots from the library
    (zkntt_field_info), with the constants the sharded steps need."""

    def __init__(self, field):
        from . import field_info
        self.field = field
        self.r, g_mont, self.s = field_info(field)
        self.rinv = pow(R_MONT, -1, self.r)
        self.g = g_mont * self.rinv % self.r

    def mont(self, x: int) -> int:
        return x % self.r * R_MONT % self.r

    def root(self, log_n: int, inverse: bool = False) -> int:
        """w_n = g^((r - 1) / 2^log_n), the library's root of order n (plain)."""
        w = pow(self.g, (self.r - 1) >> log_n, self.r)
        return pow(w, -1, self.r) if inverse else w


class LibraryOps:
    """The device steps of a shard, on torch CUDA tensors of shape [m, 8]."""

    def __init__(self, field):
        self.field = field
        self._plans = {}

    def ntt(self, x: torch.Tensor, log_n: int, inverse: bool, shift_mont):
        from . import Plan
        key = (log_n, inverse, shift_mont)
        p = self._plans.get(key)
        if p is None:
            p = Plan(self.field, log_n, inverse=inverse, coset_shift=shift_mont)
            self._plans[key] = p
        return p.execute(x)

    def scale_powers(self, x: torch.Tensor, c_mont: int, base_mont: int) -> torch.Tensor:
        from . import scale_powers
        return scale_powers(self.field, x, c_mont, base_mont, out=x)

    def block_dft(self, u: torch.Tensor, log_g: int, inverse: bool) -> torch.Tensor:
        from . import block_dft
        return block_dft(self.field, u, log_g, inverse=inverse)

    def add(self, a, b):
        from . import field_op
        return field_op(self.field, "add", a, b)

    def sub(self, a, b):
        from . import field_op
        return field_op(self.field, "sub", a, b)

    def close(self):
        for p in self._plans.values():
            p.close()
        self._plans.clear()


def _rev(x: int, bits: int) -> int:
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


class ShardedNTT:
    """Rank `rank`'s part of one transform of 2^log_n elements over `world`
    ranks (a power of two, world^2 <= 2^log_n).  coset_shift: Montgomery
    form, as for Plan.  `ops` carries the device steps (LibraryOps by
    default)."""

    def __init__(self, field, log_n: int, world: int, rank: int, inverse: bool = False,
                 coset_shift: int | None = None, ops=None):
        g = world.bit_length() - 1
        if world < 1 or (1 << g) != world or not 0 <= rank < world:
            raise ValueError("world must be a power of two and 0 <= rank < world")
        if log_n < 2 * g or log_n < 1:
            raise ValueError("need world^2 <= 2^log_n")
        self.field = field
        self.F = HostField(field)
        if log_n > self.F.s:
            raise ValueError("log_n above the field's 2-adicity")
        self.L, self.G, self.g_bits, self.rank = log_n, world, g, rank
        self.n2 = 1 << (log_n - g)
        self.b = self.n2 >> g
        self.inverse = bool(inverse)
        self.shift = None
        if coset_shift is not None:
            if not 0 < coset_shift < self.F.r:
                raise ValueError("coset shift must be a nonzero canonical element")
            self.shift = coset_shift * self.F.rinv % self.F.r   # plain
        self.ops = ops if ops is not None else LibraryOps(field)

    # ---- layouts
    def input_indices(self) -> torch.Tensor:
        """Global indices j of this rank's input elements, in local order."""
        return self.rank + self.G * torch.arange(self.n2, dtype=torch.int64)

    def output_indices(self) -> torch.Tensor:
        """Global indices k of this rank's output elements, in local order
        (k1-major, then i)."""
        i = torch.arange(self.b, dtype=torch.int64)
        k1 = torch.arange(self.G, dtype=torch.int64)
        return (self.rank * self.b + i[None, :] + self.n2 * k1[:, None]).reshape(-1)

    # ---- steps
    def local_stage(self, x: torch.Tensor) -> torch.Tensor:
        """Local transform of size n2 and the twiddle scale; returns the n2
        elements whose block s goes to rank s."""
        F, r = self.F, self.rank
        fwd_coset = self.shift is not None and not self.inverse
        local_shift = F.mont(pow(self.shift, self.G, F.r)) if fwd_coset else None
        y = self.ops.ntt(x, self.L - self.g_bits, self.inverse, local_shift)
        c = pow(self.shift, r, F.r) if fwd_coset else 1
        if self.inverse:
            c = c * pow(self.G, -1, F.r) % F.r
        base = pow(F.root(self.L, self.inverse), r, F.r)
        return self.ops.scale_powers(y, F.mont(c), F.mont(base))

    def exchange(self, z: torch.Tensor, group=None) -> torch.Tensor:
        import torch.distributed as dist
        u = torch.empty_like(z)
        dist.all_to_all_single(u, z.contiguous(), group=group)
        return u

    def combine_stage(self, u: torch.Tensor) -> torch.Tensor:
        """The G-point transforms over the received blocks (one block-transform
        kernel for G <= 8, else radix-2 decimation in frequency over whole
        blocks), then the coset-inverse output scale; returns the local output
        in output_indices order."""
        F, G, b = self.F, self.G, self.b
        if 1 < G <= 8 and hasattr(self.ops, "block_dft"):
            # one kernel: every column's G-point transform, k1-major output
            out = self.ops.block_dft(u, self.g_bits, self.inverse)
            return self._coset_inverse_scale(out)
        v = [u[r * b:(r + 1) * b] for r in range(G)]
        wG = F.root(self.g_bits, self.inverse) if G > 1 else 1
        h = G >> 1
        while h >= 1:
            w2h = pow(wG, G // (2 * h), F.r)        # root of order 2h
            for g0 in range(0, G, 2 * h):
                for j in range(h):
                    x, y = v[g0 + j], v[g0 + j + h]
                    v[g0 + j] = self.ops.add(x, y)
                    d = self.ops.sub(x, y)
                    if j:
                        d = self.ops.scale_powers(d, F.mont(pow(w2h, j, F.r)), F.mont(1))
                    v[g0 + j + h] = d
            h >>= 1
        # position p holds frequency rev(p): reorder to k1-major
        out = torch.cat([v[_rev(k1, self.g_bits)] for k1 in range(G)], dim=0)
        return self._coset_inverse_scale(out)

    def _coset_inverse_scale(self, out: torch.Tensor) -> torch.Tensor:
        """Output k times g^-k (coset inverse only); out is k1-major."""
        F, G, b = self.F, self.G, self.b
        if self.shift is not None and self.inverse:
            ginv = pow(self.shift, -1, F.r)
            for k1 in range(G):
                blk = out[k1 * b:(k1 + 1) * b]
                c = pow(ginv, self.rank * b + self.n2 * k1, F.r)
                self.ops.scale_powers(blk, F.mont(c), F.mont(ginv))
        return out

    def execute(self, x: torch.Tensor, group=None) -> torch.Tensor:
        """The whole transform for this rank (a collective: every rank of the
        group calls it)."""
        if x.shape[0] != self.n2:
            raise ValueError(f"expected {self.n2} local elements")
        return self.combine_stage(self.exchange(self.local_stage(x), group))


def emulate(shards: list[ShardedNTT], xs: list[torch.Tensor]) -> list[torch.Tensor]:
    """All shards of one transform in this process (one device): the local
    stages, the exchange as block copies, the combine stages."""
    G = len(shards)
    zs = [s.local_stage(x) for s, x in zip(shards, xs)]
    b = shards[0].b
    us = [torch.cat([zs[r][s * b:(s + 1) * b] for r in range(G)], dim=0) for s in range(G)]
    return [s.combine_stage(u) for s, u in zip(shards, us)]


def scatter_input(a: torch.Tensor, world: int) -> list[torch.Tensor]:
    """Natural-order vector -> the ranks' input shards (rank r: a[r::world])."""
    return [a[r::world].contiguous() for r in range(world)]


def gather_output(outs: list[torch.Tensor], log_n: int) -> torch.Tensor:
    """The ranks' output shards -> the natural-order result."""
    world = len(outs)
    g = world.bit_length() - 1
    n2 = 1 << (log_n - g)
    b = n2 >> g
    full = torch.empty((1 << log_n, outs[0].shape[1]), dtype=outs[0].dtype, device=outs[0].device)
    for s, o in enumerate(outs):
        for k1 in range(world):
            full[s * b + n2 * k1: s * b + n2 * k1 + b] = o[k1 * b:(k1 + 1) * b]
    return full
