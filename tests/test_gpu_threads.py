"""Plans are immutable and shared across host threads and streams: four
threads create plans concurrently (device set-up, tuned-schedule lookup and the
Groth16 plan cache run under locks), execute a shared plan on their own
streams, and run the Groth16 sequence; every result equals the serial one."""
import threading

import numpy as np
import pytest

from oracle import field as fld
from workloads import uniform_elements

from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def test_concurrent_threads_match_serial_results():
    import torch
    import paper_2509_22684_gb300 as zk
    F = fld.BLS12_381
    shared = zk.Plan(F.name, 16)
    inputs = [to_dev(uniform_elements(F.r, 1 << 16, 500 + t)) for t in range(4)]
    own = [(fld.BN254, 14), (fld.BLS12_377, 12), (fld.BLS12_381, 13), (fld.BN254, 15)]
    own_inputs = [to_dev(uniform_elements(G.r, 1 << L, 600 + t)) for t, (G, L) in enumerate(own)]
    g16 = [tuple(to_dev(uniform_elements(F.r, 1 << 12, 700 + 3 * t + i)) for i in range(3))
           for t in range(4)]
    # serial reference
    want_shared = [to_host(shared.execute(x)) for x in inputs]
    want_own = []
    for (G, L), x in zip(own, own_inputs):
        with zk.Plan(G.name, L, inverse=True) as p:
            want_own.append(to_host(p.execute(x)))
    want_g16 = [to_host(zk.groth16_h(F.name, 12, *abc)) for abc in g16]

    got = [None] * 4
    errors = []
    barrier = threading.Barrier(4)

    def work(t):
        try:
            s = torch.cuda.Stream()
            barrier.wait()
            G, L = own[t]
            p = zk.Plan(G.name, L, inverse=True)              # created concurrently
            outs = []
            with torch.cuda.stream(s):
                for _ in range(5):
                    y = shared.execute(inputs[t], stream=s)   # one plan, four streams
                z = p.execute(own_inputs[t], stream=s)
                h = zk.groth16_h(F.name, 12, *g16[t], stream=s)
            s.synchronize()
            got[t] = (to_host(y), to_host(z), to_host(h))
            p.close()
        except Exception as e:          # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert not errors, errors
    zk.sync_status()
    for t in range(4):
        y, z, h = got[t]
        assert np.array_equal(y, want_shared[t])
        assert np.array_equal(z, want_own[t])
        assert np.array_equal(h, want_g16[t])
    shared.close()
