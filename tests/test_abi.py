"""The C-ABI library loads and exports every function include/zkntt.h declares;
argument validation that happens before any CUDA call works without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zkntt.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zkntt_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_22684_gb300 import build, _native
    build.build()
    return _native.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("zkntt_plan_create", "zkntt_plan_destroy", "zkntt_execute",
                     "zkntt_execute_batch", "zkntt_groth16_h", "zkntt_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2509_22684_gb300 import _native
    assert set(_declared_functions()) <= set(_native.SIGNATURES)


def test_status_strings(lib):
    from paper_2509_22684_gb300 import _native as N
    assert N.status_str(N.OK) == "ok"
    assert "invalid" in N.status_str(N.EINVAL)
    assert N.status_str(99) == "unknown status"


def test_host_side_validation_without_gpu(lib):
    from paper_2509_22684_gb300 import _native as N
    h = ctypes.c_void_p()
    # field, log_n, direction and null handle are rejected before any CUDA call
    assert lib.zkntt_plan_create(ctypes.byref(h), 7, 10, 0, None) == N.EINVAL
    assert lib.zkntt_plan_create(ctypes.byref(h), 3, 10, 0, None) == N.EINVAL
    assert lib.zkntt_plan_create(ctypes.byref(h), 2, 48, 0, None) == N.EINVAL   # above 2-adicity 47
    assert lib.zkntt_plan_create(ctypes.byref(h), 2, 33, 0, None) == N.ENOMEM   # 2^33: no device holds it
    assert lib.zkntt_plan_create(ctypes.byref(h), 0, 0, 0, None) == N.EINVAL
    assert lib.zkntt_plan_create(ctypes.byref(h), 1, 29, 0, None) == N.EINVAL
    assert lib.zkntt_plan_create(ctypes.byref(h), 0, 33, 0, None) == N.EINVAL
    assert lib.zkntt_plan_create(ctypes.byref(h), 0, 10, 2, None) == N.EINVAL
    assert lib.zkntt_plan_create(None, 0, 10, 0, None) == N.EINVAL
    zero = N.u32_array([0] * 8)
    assert lib.zkntt_plan_create(ctypes.byref(h), 0, 10, 0, zero) == N.EINVAL
    assert lib.zkntt_execute(None, None, None, None) == N.EINVAL
    assert lib.zkntt_execute_batch(None, None, -1, None) == N.EINVAL
    assert lib.zkntt_execute_batch(None, None, 0, None) == N.OK          # empty batch: no-op
    assert lib.zkntt_execute_batch(None, None, 0, None) == N.OK
    assert lib.zkntt_groth16_h(0, 10, None, None, None, None, None, None) == N.EINVAL
    assert lib.zkntt_groth16_h_ex(0, 10, None, None, None, None, None, 1, None) == N.EINVAL
    assert lib.zkntt_plan_destroy(None) == N.OK
    err = ctypes.c_int(-1)
    assert lib.zkntt_last_cuda_error(ctypes.byref(err)) == N.OK
    assert lib.zkntt_field_op(0, 5, None, None, None, 1, None) == N.EINVAL
    assert lib.zkntt_selftest_timeout(0, None) == N.EINVAL
    assert lib.zkntt_inject_timeout(0, None) == N.EINVAL
    assert lib.zkntt_inject_timeout(10001, None) == N.EINVAL
    assert lib.zkntt_imadbench(5, 1, 32, 1, ctypes.c_void_p(256), None) == N.EINVAL
    assert lib.zkntt_imadbench(0, 1, 32, 1, None, None) == N.EINVAL
    assert lib.zkntt_selftest_device_check(None, None) == N.EINVAL
    one = N.u32_array([1] + [0] * 7)
    assert lib.zkntt_scale_powers(0, None, None, 4, None, one, None) == N.EINVAL
    assert lib.zkntt_scale_powers(9, None, None, 4, one, one, None) == N.EINVAL
    assert lib.zkntt_scale_powers(0, None, None, 0, one, one, None) == N.OK    # empty: no-op
    assert lib.zkntt_block_dft(0, 4, 8, None, None, 0, None) == N.EINVAL      # G = 16
    assert lib.zkntt_block_dft(0, 0, 8, None, None, 0, None) == N.EINVAL
    assert lib.zkntt_block_dft(0, 2, 0, None, None, 0, None) == N.OK          # empty: no-op


def test_field_info_without_gpu(lib):
    from oracle import field as fld
    import paper_2509_22684_gb300 as zk
    for F in (fld.BLS12_381, fld.BN254, fld.BLS12_377):
        m, g, s = zk.field_info(F.name)
        assert m == F.r and g == F.to_mont(F.g) and s == F.s
