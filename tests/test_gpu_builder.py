"""The Python front end on the GPU: builder circuits run through the
Simulator facade (C ABI, library kernels) against the FP64 oracle --
state, expectation, samples, and the adjoint gradient of a parametrised
circuit; and the split-BF16 tensor-core mode through the same facade."""
import numpy as np
import pytest

import workloads as W
from conftest import fidelity_metrics
from paper_2106_13995_gb300 import Circuit, Simulator, X, Z, ising

pytestmark = pytest.mark.gpu


def ansatz(n, layers):
    c = Circuit(n, "builder_ansatz")
    for _ in range(layers):
        for q in range(n):
            c.ry(c.parameter(), q)
            c.rz(c.parameter(), q)
        for q in range(n - 1):
            c.cx(q, q + 1)
    return c


def test_simulator_state_expectation_samples(svlib, oracle):
    n = 10
    c = Circuit(n).h(0)
    for q in range(1, n):
        c.cx(q - 1, q)
    c.rx(0.3, 4).fsim(np.pi / 2, np.pi / 6, 2, 3).u3(0.5, 0.1, -0.2, 7, controls=(1,))
    want = oracle.run(c)
    for dt, tol in (("c64", 1e-6), ("c128", 1e-12)):
        sim = Simulator(dtype=dt)
        inf, _ = fidelity_metrics(want, sim.state_vector(c))
        assert inf <= tol * tol, (dt, inf)
        H = ising(n) + 0.25 * (X(0) * Z(9))
        assert abs(sim.expectation(c, H) - oracle.expect(want, H.terms())) <= 10 * tol
        shots = sim.sample(c, 2000, seed=5)
        assert np.array_equal(shots, oracle.sample(sim.state_vector(c), 2000, 5))
        sim.close()


def test_simulator_gradient_and_tensor_cores(svlib, oracle):
    n = 12
    c = ansatz(n, 3)
    p = W.hea_params(1, c.n_params, 9)[0]
    H = ising(n)
    sim = Simulator(dtype="c64")
    ev, g = sim.gradient(c, H, p)
    ev_o, g_o, _ = oracle.adjoint_grad(c, p, H.terms())
    assert abs(ev - ev_o) <= 1e-5 * max(1, abs(ev_o))
    assert np.max(np.abs(g - g_o)) <= 1e-5 * max(1, np.max(np.abs(g_o)))
    # split-BF16 tensor-core blocks through the same facade (state of 12 qubits)
    tc = Simulator(dtype="c64", prec="bf16x3")
    inf, amp = fidelity_metrics(oracle.run(c.bind(p)), tc.state_vector(c, p))
    assert inf <= 1e-5, inf
    sim.close()
    tc.close()
