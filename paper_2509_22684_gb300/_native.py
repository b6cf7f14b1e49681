"""ctypes binding of ``libzkntt.so`` (the C ABI declared in include/zkntt.h).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  The library must have been built (``build.build()``); if it is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# ZKNTT_LIB selects another build of the library (variants built with ZKNTT_LIB_OUT)
LIB_PATH = os.environ.get("ZKNTT_LIB") or os.path.join(HERE, "libzkntt.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
FIELDS = {"bls12_381_fr": 0, "bn254_fr": 1, "bls12_377_fr": 2}
TWIDDLE_MODES = {"auto": 0, "precomp": 1, "otf": 2}


class ZkNttError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} (status {status})")


class PlanOptions(ctypes.Structure):
    _fields_ = [("twiddle_mode", ctypes.c_int), ("num_passes", ctypes.c_int),
                ("digit_bits", ctypes.c_int * 4), ("cols_per_cta", ctypes.c_int * 4),
                ("use_tuner", ctypes.c_int), ("ilp", ctypes.c_int)]


class IO(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("num_passes", ctypes.c_int), ("digit_bits", ctypes.c_int * 4),
                ("cols_per_cta", ctypes.c_int * 4), ("twiddle_mode", ctypes.c_int),
                ("ilp", ctypes.c_int), ("ms", ctypes.c_float)]


_lib = None

# every function the header declares, with its argument types
_u32p = ctypes.POINTER(ctypes.c_uint32)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
SIGNATURES = {
    "zkntt_plan_create": [ctypes.POINTER(_vp), _i, _i, _i, _u32p],
    "zkntt_plan_create_ex": [ctypes.POINTER(_vp), _i, _i, _i, _u32p, ctypes.POINTER(PlanOptions)],
    "zkntt_plan_destroy": [_vp],
    "zkntt_plan_scratch_bytes": [_vp, ctypes.POINTER(_sz)],
    "zkntt_plan_describe": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                            ctypes.POINTER(_sz)],
    "zkntt_execute": [_vp, _vp, _vp, _vp],
    "zkntt_execute_scratch": [_vp, _vp, _vp, _vp, _sz, _vp],
    "zkntt_execute_host": [_vp, _vp, _vp, _vp],
    "zkntt_execute_host_buffered": [_vp, _vp, _vp, _vp, _sz, _vp],
    "zkntt_execute_noalloc": [_vp, _vp, _vp, _vp],
    "zkntt_execute_batch": [ctypes.POINTER(_vp), ctypes.POINTER(IO), _i, _vp],
    "zkntt_execute_batch_signal": [ctypes.POINTER(_vp), ctypes.POINTER(IO), _i, _vp, ctypes.c_uint32, _vp],
    "zkntt_flags_create": [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "zkntt_flags_destroy": [_vp],
    "zkntt_groth16_h": [_i, _i, _vp, _vp, _vp, _vp, _vp, _vp],
    "zkntt_groth16_h_ex": [_i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp],
    "zkntt_groth16_graph_create": [ctypes.POINTER(_vp), _i, _i, _vp, _vp, _vp, _vp, _vp, _vp],
    "zkntt_graph_launch": [_vp, _vp],
    "zkntt_graph_destroy": [_vp],
    "zkntt_status_str": [_i],
    "zkntt_last_cuda_error": [ctypes.POINTER(_i)],
    "zkntt_sync_status": [_vp],
    "zkntt_selftest_timeout": [_i, _vp],
    "zkntt_inject_timeout": [_i, _vp],
    "zkntt_field_info": [_i, _u32p, _u32p, ctypes.POINTER(_i)],
    "zkntt_field_op": [_i, _i, _vp, _vp, _vp, _sz, _vp],
    "zkntt_pointwise": [_i, _vp, _vp, _vp, _u32p, _vp, _sz, _vp],
    "zkntt_tune": [_i, _i, _i, _i, ctypes.POINTER(TuneResult)],
    "zkntt_mulbench": [_i, _i, _i, _i, _vp, _vp],
    "zkntt_imadbench": [_i, _i, _i, _i, _vp, _vp],
    "zkntt_selftest_device_check": [ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "zkntt_pool_info": [ctypes.POINTER(_sz), ctypes.POINTER(_sz)],
    "zkntt_scale_powers": [_i, _vp, _vp, _sz, _u32p, _u32p, _vp],
    "zkntt_block_dft": [_i, _i, _sz, _vp, _vp, _i, _vp],
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libzkntt.so not built ({LIB_PATH}); run "
                              "`python -m paper_2509_22684_gb300.build` or __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "zkntt_status_str" else ctypes.c_int
        _lib = L
    return _lib


def status_str(status: int) -> str:
    return lib().zkntt_status_str(int(status)).decode()


def check(status: int, what: str) -> None:
    if status != OK:
        raise ZkNttError(status, what)


def u32_array(vals) -> ctypes.Array:
    arr = (ctypes.c_uint32 * 8)()
    for i, v in enumerate(vals):
        arr[i] = int(v) & 0xFFFFFFFF
    return arr


def limbs_of(x: int) -> ctypes.Array:
    return u32_array([(x >> (32 * i)) & 0xFFFFFFFF for i in range(8)])
