"""zkntt_execute_noalloc: the transform for callers that must not allocate
device memory during the call (for instance inside a host application that
keeps all device memory for itself, or in a loop that cannot afford an
allocation's synchronisation).  Called through the C ABI and compared with
zkntt_execute on two calls in a row, since the shared scratch array keeps the
previous call's contents.  The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

from oracle import field as fld
from workloads import uniform_elements

from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _noalloc(plan, x, y):
    import torch
    from paper_2509_22684_gb300 import _native as N
    st = N.lib().zkntt_execute_noalloc(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("F,L,kind,digits,single", [
    (fld.BLS12_381, 8, "ntt", None, True),     # below the tuned sizes: one pass, no scratch
    (fld.BLS12_381, 10, "ntt", (10,), True),   # forced single pass: no scratch
    (fld.BLS12_381, 10, "ntt", None, False),   # the tuned schedule has two passes
    (fld.BLS12_381, 16, "ntt", None, False),
    (fld.BN254, 18, "coset_intt", None, False),
    (fld.BLS12_381, 20, "intt", None, False),  # largest size the static scratch holds
])
def test_noalloc_matches_execute_on_two_consecutive_calls(F, L, kind, digits, single):
    import torch
    import paper_2509_22684_gb300 as zk
    from paper_2509_22684_gb300 import _native as N
    inverse = kind.endswith("intt")
    shift = F.to_mont(F.g) if kind.startswith("coset") else None
    with zk.Plan(F.name, L, inverse=inverse, coset_shift=shift, digits=digits) as p:
        assert (p.describe()["passes"] == 1) == single
        assert (p.scratch_bytes() == 0) == single
        for call, seed in enumerate((501, 502)):
            X = uniform_elements(F.r, 1 << L, seed + L)
            x = to_dev(X)
            want = to_host(p.execute(x))
            y = torch.empty_like(x)
            assert _noalloc(p, x, y) == N.OK
            got = to_host(y)
            assert np.array_equal(got, want), f"call {call}: differs from zkntt_execute"
            # in place as well
            assert _noalloc(p, x, x) == N.OK
            assert np.array_equal(to_host(x), want), f"call {call}: in place differs"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2509_22684_gb300 as zk
    from paper_2509_22684_gb300 import _native as N
    with zk.Plan("bls12_381_fr", 21) as p:
        x = torch.zeros((1 << 21, 8), dtype=torch.int32, device="cuda")
        y = torch.empty_like(x)
        assert _noalloc(p, x, y) == N.EINVAL
