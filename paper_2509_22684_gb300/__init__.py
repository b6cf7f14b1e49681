"""zkntt: number-theoretic transforms over BLS12-381 F_r and BN254 F_r on GB300.

Python face of ``libzkntt.so`` (C ABI in include/zkntt.h).  Device vectors are
torch tensors of shape [n, 8] with a 4-byte integer dtype (int32 or uint32),
holding 8 little-endian 32-bit limbs per element in Montgomery form; torch
supplies device memory and streams only, every step of the transform runs in
the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N
from ._native import ZkNttError, FIELDS, TWIDDLE_MODES

__all__ = ["Plan", "ZkNttError", "FIELDS", "execute_batch", "execute_batch_signal",
           "CompletionFlags", "groth16_h", "Groth16Graph", "field_info",
           "field_op", "pointwise", "scale_powers", "block_dft", "tune", "sync_status", "mulbench", "imadbench", "pool_info",
           "new_vector"]


def _field_id(field) -> int:
    if isinstance(field, int):
        return field
    return FIELDS[field]


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.element_size() != 4 or not t.is_contiguous():
        raise ValueError("expected a contiguous tensor of 4-byte limbs")
    return ctypes.c_void_p(t.data_ptr())


def new_vector(log_n: int, device="cuda") -> torch.Tensor:
    return torch.empty((1 << log_n, 8), dtype=torch.int32, device=device)


def field_info(field):
    """(modulus, generator in Montgomery form, 2-adicity) as Python ints."""
    m = (ctypes.c_uint32 * 8)()
    g = (ctypes.c_uint32 * 8)()
    s = ctypes.c_int()
    N.check(N.lib().zkntt_field_info(_field_id(field), m, g, ctypes.byref(s)), "field_info")
    to_int = lambda a: sum(int(a[i]) << (32 * i) for i in range(8))
    return to_int(m), to_int(g), s.value


class Plan:
    """One transform size / direction / coset on the current device."""

    def __init__(self, field, log_n: int, inverse: bool = False, coset_shift: int | None = None,
                 twiddle_mode: str = "auto", digits=None, cols=None, use_tuner: bool = False,
                 ilp: int = 0):
        self.field = _field_id(field)
        self.log_n = int(log_n)
        self.inverse = bool(inverse)
        self.coset_shift = coset_shift
        opts = N.PlanOptions()
        opts.twiddle_mode = TWIDDLE_MODES[twiddle_mode]
        if digits:
            opts.num_passes = len(digits)
            for i, d in enumerate(digits):
                opts.digit_bits[i] = int(d)
        if cols:
            for i, c in enumerate(cols):
                opts.cols_per_cta[i] = int(c)
        opts.use_tuner = int(use_tuner)
        opts.ilp = int(ilp)
        shift = None if coset_shift is None else N.limbs_of(coset_shift)
        h = ctypes.c_void_p()
        N.check(N.lib().zkntt_plan_create_ex(ctypes.byref(h), self.field, self.log_n,
                                             int(self.inverse), shift, ctypes.byref(opts)),
                "zkntt_plan_create_ex")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise ValueError("plan destroyed")
        return self._h

    @property
    def n(self) -> int:
        return 1 << self.log_n

    def scratch_bytes(self) -> int:
        b = ctypes.c_size_t()
        N.check(N.lib().zkntt_plan_scratch_bytes(self.handle, ctypes.byref(b)), "scratch_bytes")
        return b.value

    def describe(self) -> dict:
        p = ctypes.c_int()
        d = (ctypes.c_int * 4)()
        m = ctypes.c_int()
        tb = ctypes.c_size_t()
        N.check(N.lib().zkntt_plan_describe(self.handle, ctypes.byref(p), d, ctypes.byref(m),
                                            ctypes.byref(tb)), "describe")
        return {"passes": p.value, "digits": list(d)[:p.value], "twiddle_mode":
                {1: "precomp", 2: "otf"}.get(m.value, "auto"), "table_bytes": tb.value}

    def _check_vec(self, t):
        if t.numel() != 8 * self.n:
            raise ValueError(f"expected {self.n} elements of 8 limbs, got {t.numel()} limbs")

    def execute(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """out = T(x) (in place when out is x); stream-ordered, asynchronous."""
        self._check_vec(x)
        if out is None:
            out = torch.empty_like(x)
        self._check_vec(out)
        N.check(N.lib().zkntt_execute(self.handle, _ptr(x), _ptr(out), _stream_handle(stream)),
                "zkntt_execute")
        return out

    def execute_scratch(self, x, out, scratch: torch.Tensor, stream=None) -> torch.Tensor:
        self._check_vec(x)
        self._check_vec(out)
        N.check(N.lib().zkntt_execute_scratch(self.handle, _ptr(x), _ptr(out), _ptr(scratch),
                                              scratch.numel() * scratch.element_size(),
                                              _stream_handle(stream)), "zkntt_execute_scratch")
        return out

    def execute_host(self, x_host: torch.Tensor, out_host: torch.Tensor, stream=None):
        """Host buffers in and out (copies inside the call); pin them for overlap."""
        self._check_vec(x_host)
        self._check_vec(out_host)
        if x_host.is_cuda or out_host.is_cuda:
            raise ValueError("execute_host takes host tensors")
        N.check(N.lib().zkntt_execute_host(self.handle, ctypes.c_void_p(x_host.data_ptr()),
                                           ctypes.c_void_p(out_host.data_ptr()),
                                           _stream_handle(stream)), "zkntt_execute_host")
        return out_host

    def work_bytes(self) -> int:
        """Device bytes execute_host_buffered needs: the vector plus scratch."""
        return 32 * self.n + self.scratch_bytes()

    def execute_host_buffered(self, x_host: torch.Tensor, out_host: torch.Tensor,
                              work: torch.Tensor, stream=None):
        """As execute_host with a caller-owned device work buffer (at least
        work_bytes() bytes): no allocation inside the call."""
        self._check_vec(x_host)
        self._check_vec(out_host)
        if x_host.is_cuda or out_host.is_cuda or not work.is_cuda:
            raise ValueError("host tensors in and out, a device work buffer")
        nbytes = work.numel() * work.element_size()
        N.check(N.lib().zkntt_execute_host_buffered(self.handle, ctypes.c_void_p(x_host.data_ptr()),
                                                    ctypes.c_void_p(out_host.data_ptr()),
                                                    _ptr(work), nbytes, _stream_handle(stream)),
                "zkntt_execute_host_buffered")
        return out_host

    def close(self):
        if getattr(self, "_h", None) is not None:
            N.lib().zkntt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def execute_batch(plans, inputs, outputs, stream=None) -> None:
    """Run len(plans) transforms as one persistent launch."""
    count = len(plans)
    if not (len(inputs) == len(outputs) == count):
        raise ValueError("plans, inputs and outputs must have the same length")
    hs = (ctypes.c_void_p * count)(*[p.handle.value for p in plans])
    ios = (N.IO * count)()
    for i in range(count):
        plans[i]._check_vec(inputs[i])
        plans[i]._check_vec(outputs[i])
        ios[i].d_in = _ptr(inputs[i]).value
        ios[i].d_out = _ptr(outputs[i]).value
    N.check(N.lib().zkntt_execute_batch(hs, ios, count, _stream_handle(stream)),
            "zkntt_execute_batch")


class CompletionFlags:
    """Pinned host words the device writes when a transform of a signalled
    batch completes (zero-copy; the host polls without synchronising)."""

    def __init__(self, count: int):
        h = ctypes.c_void_p()
        d = ctypes.c_void_p()
        N.check(N.lib().zkntt_flags_create(int(count), ctypes.byref(h), ctypes.byref(d)),
                "zkntt_flags_create")
        self.count = int(count)
        self.host = h
        self.device = d
        self.view = (ctypes.c_uint32 * self.count).from_address(h.value)

    def __getitem__(self, i: int) -> int:
        return self.view[i]

    def close(self):
        if getattr(self, "host", None) is not None:
            N.lib().zkntt_flags_destroy(self.host)
            self.host = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def execute_batch_signal(plans, inputs, outputs, flags: CompletionFlags, slots, epoch: int,
                         stream=None) -> None:
    """As execute_batch, shortest transforms first; transform i stores `epoch`
    into flags[slots[i]] when it completes.  `slots` must be consecutive
    (slots[i] = slots[0] + i) within the flag array."""
    count = len(plans)
    if not (len(inputs) == len(outputs) == len(slots) == count):
        raise ValueError("length mismatch")
    base = slots[0]
    if list(slots) != list(range(base, base + count)) or base + count > flags.count:
        raise ValueError("slots must be a consecutive range inside the flag array")
    hs = (ctypes.c_void_p * count)(*[p.handle.value for p in plans])
    ios = (N.IO * count)()
    for i in range(count):
        plans[i]._check_vec(inputs[i])
        plans[i]._check_vec(outputs[i])
        ios[i].d_in = _ptr(inputs[i]).value
        ios[i].d_out = _ptr(outputs[i]).value
    dptr = ctypes.c_void_p(flags.device.value + 4 * base)
    N.check(N.lib().zkntt_execute_batch_signal(hs, ios, count, dptr, ctypes.c_uint32(epoch),
                                               _stream_handle(stream)),
            "zkntt_execute_batch_signal")


def groth16_h(field, log_n: int, a, b, c, h=None, scratch=None, fused: bool = True,
              stream=None) -> torch.Tensor:
    """h = coset-iNTT((A*B - C)/Z) with A, B, C the coset NTTs of iNTT(a|b|c)."""
    n = 1 << log_n
    if h is None:
        h = torch.empty_like(a)
    if scratch is None:
        scratch = torch.empty((3 * n, 8), dtype=a.dtype, device=a.device)
    for t in (a, b, c, h):
        if t.numel() != 8 * n:
            raise ValueError("vector size mismatch")
    N.check(N.lib().zkntt_groth16_h_ex(_field_id(field), log_n, _ptr(a), _ptr(b), _ptr(c),
                                       _ptr(h), _ptr(scratch), int(fused), _stream_handle(stream)),
            "zkntt_groth16_h_ex")
    return h


class Groth16Graph:
    """The fused Groth16 H sequence for fixed buffers, captured once into a
    CUDA graph and replayed with ``launch()``."""

    def __init__(self, field, log_n: int, a, b, c, h, scratch, stream: torch.cuda.Stream):
        n = 1 << log_n
        for t in (a, b, c, h):
            if t.numel() != 8 * n:
                raise ValueError("vector size mismatch")
        self._bufs = (a, b, c, h, scratch)   # keep the buffers alive with the graph
        g = ctypes.c_void_p()
        N.check(N.lib().zkntt_groth16_graph_create(ctypes.byref(g), _field_id(field), log_n, _ptr(a),
                                                   _ptr(b), _ptr(c), _ptr(h), _ptr(scratch),
                                                   _stream_handle(stream)),
                "zkntt_groth16_graph_create")
        self._g = g

    def launch(self, stream=None):
        N.check(N.lib().zkntt_graph_launch(self._g, _stream_handle(stream)), "zkntt_graph_launch")

    def close(self):
        if getattr(self, "_g", None) is not None:
            N.lib().zkntt_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def field_op(field, op: str, a, b, out=None, stream=None) -> torch.Tensor:
    ops = {"mul": 0, "add": 1, "sub": 2, "sub_lazy": 3}
    out = torch.empty_like(a) if out is None else out
    N.check(N.lib().zkntt_field_op(_field_id(field), ops[op], _ptr(a), _ptr(b), _ptr(out),
                                   a.numel() // 8, _stream_handle(stream)), "zkntt_field_op")
    return out


def scale_powers(field, x, c_mont: int, base_mont: int, out=None, stream=None) -> torch.Tensor:
    """out[i] = x[i] * c * base^i (Montgomery-form c and base; in place when
    out is x)."""
    out = torch.empty_like(x) if out is None else out
    N.check(N.lib().zkntt_scale_powers(_field_id(field), _ptr(x), _ptr(out), x.numel() // 8,
                                       N.limbs_of(c_mont), N.limbs_of(base_mont),
                                       _stream_handle(stream)), "zkntt_scale_powers")
    return out


def block_dft(field, x, log_g: int, inverse: bool = False, out=None, stream=None) -> torch.Tensor:
    """G-point transforms (G = 2^log_g) over the G blocks of x: out[k*b + i] =
    sum_r x[r*b + i] w^(r k), w the root of order G (inverse: w^-1, no 1/G)."""
    out = torch.empty_like(x) if out is None else out
    n = x.numel() // 8
    if n % (1 << log_g):
        raise ValueError("the vector must hold G whole blocks")
    N.check(N.lib().zkntt_block_dft(_field_id(field), int(log_g), n >> log_g, _ptr(x), _ptr(out),
                                    int(inverse), _stream_handle(stream)), "zkntt_block_dft")
    return out


def pointwise(field, a, b, c, z_mont: int, out=None, stream=None) -> torch.Tensor:
    out = torch.empty_like(a) if out is None else out
    N.check(N.lib().zkntt_pointwise(_field_id(field), _ptr(a), _ptr(b), _ptr(c),
                                    N.limbs_of(z_mont), _ptr(out), a.numel() // 8,
                                    _stream_handle(stream)), "zkntt_pointwise")
    return out


def tune(field, log_n: int, inverse: bool = False, max_candidates: int = 24) -> dict:
    r = N.TuneResult()
    N.check(N.lib().zkntt_tune(_field_id(field), log_n, int(inverse), max_candidates,
                               ctypes.byref(r)), "zkntt_tune")
    return {"passes": r.num_passes, "digits": list(r.digit_bits)[:r.num_passes],
            "cols": list(r.cols_per_cta)[:r.num_passes],
            "twiddle_mode": {1: "precomp", 2: "otf"}.get(r.twiddle_mode, "auto"), "ilp": r.ilp,
            "ms": r.ms}


def sync_status(stream=None) -> None:
    N.check(N.lib().zkntt_sync_status(_stream_handle(stream)), "zkntt_sync_status")


def pool_info() -> tuple[int, int]:
    """(reserved, in use) bytes of the library's scratch pool on the current device."""
    r, u = ctypes.c_size_t(), ctypes.c_size_t()
    N.check(N.lib().zkntt_pool_info(ctypes.byref(r), ctypes.byref(u)), "zkntt_pool_info")
    return r.value, u.value


def imadbench(mode: int, blocks: int, threads: int, iters: int, sink: torch.Tensor, stream=None):
    """Launch the multiply-add rate calibration (mode 0 mad.lo.u32, 1
    mad.wide.u32): 8 * iters multiply-adds per thread."""
    N.check(N.lib().zkntt_imadbench(int(mode), blocks, threads, iters, _ptr(sink),
                                    _stream_handle(stream)), "zkntt_imadbench")


def mulbench(field, blocks: int, threads: int, iters: int, sink: torch.Tensor, stream=None):
    N.check(N.lib().zkntt_mulbench(_field_id(field), blocks, threads, iters, _ptr(sink),
                                   _stream_handle(stream)), "zkntt_mulbench")
