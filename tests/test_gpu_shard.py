"""One state split into 2 and 4 shards held by one process on one GPU
(in-process loopback transport): the library's kernels apply each shard's
local gates, half-shards are exchanged for global-qubit swaps, and the
gathered state equals the FP64 oracle's.  The same plan and executor run
across processes through torch.distributed (tested on gloo CPU ranks)."""
import numpy as np
import pytest
import torch

import workloads as W
from conftest import fidelity_metrics
from paper_2106_13995_gb300 import shard as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt,g,n", [("c64", 1, 14), ("c64", 2, 20), ("c128", 2, 14)])
def test_sharded_state_on_one_gpu(svlib, oracle, dt, g, n):
    from paper_2106_13995_gb300 import _native as N
    rng = np.random.default_rng(n + g)
    c = W.random_gate_circuit(n, 120, seed=n * 3 + g)
    psi0 = W.random_state(n, rng)
    L = n - g
    states = [svlib.StateVector(L, dt).load(psi0[r << L:(r + 1) << L]) for r in range(1 << g)]
    plan = S.plan(c, g)

    def apply_local(i, sub):
        states[i].apply_circuit(sub)

    def exchanged(i):   # the amplitudes changed outside the library
        N.check(N.lib().sv_mark_modified(states[i].h))

    S.run(plan, S.LoopbackTransport([st.amps for st in states]), apply_local, on_exchange=exchanged)
    got = np.concatenate([st.numpy() for st in states]).astype(np.complex128)
    cast = psi0.astype(np.complex64 if dt == "c64" else np.complex128).astype(np.complex128)
    inf, amp = fidelity_metrics(oracle.run(c, cast), got)
    assert inf <= (1e-5 if dt == "c64" else 1e-12), inf
    print(f"{dt} n={n} over {1 << g} shards: {plan.swaps()} swaps, 1-F {inf:.2e}, max|d| {amp:.2e}")
