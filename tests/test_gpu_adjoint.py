"""GPU adjoint gradients (plain and batched) against the oracle's FP64
adjoint gradient, the parameter-shift rule and central differences."""
import math

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def gtol(g_ref):
    return 1e-5 * max(1.0, float(np.max(np.abs(g_ref))))


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_small_hea_vs_oracle(svlib, oracle, dt):
    n, layers = 8, 3
    c = W.hea(n, layers)
    terms = W.tfim(n)
    P = W.hea_params(3, c.n_params, 7)
    psi, lam = svlib.StateVector(n, dt), svlib.StateVector(n, dt)
    for p in P:
        psi.set_basis(0)
        ev, g = svlib.adjoint_grad(psi, lam, c, p, terms)
        ev_o, g_o, _ = oracle.adjoint_grad(c, p, terms)
        tol = 1e-12 if dt == "c128" else None
        assert abs(ev - ev_o) <= (tol or 1e-5 * max(1, abs(ev_o)))
        assert np.max(np.abs(g - g_o)) <= (tol or gtol(g_o))
        # psi is returned to its input |0>
        back = psi.numpy()
        assert abs(abs(back[0]) - 1) <= (1e-12 if dt == "c128" else 1e-5)


def test_controlled_and_fixed_gates_mixed(svlib, oracle):
    n = 7
    c = W.Circuit(n, n_params=5)
    c.ops += [W.Op("H", (q,)) for q in range(n)]
    c.ops += [W.Op("RX", (0,), param=0), W.Op("X", (3,), (0,)), W.Op("RY", (3,), param=1),
              W.Op("FSIM", (2, 5), angles=(0.3, 0.9)), W.Op("RZ", (5,), param=2),
              W.Op("PHASE", (6,), param=3), W.Op("X", (6,), (1, 2)), W.Op("RY", (6,), param=4),
              W.Op("RX", (1,), param=0)]
    terms = [(0b1000001, 0b0000100, 0.7), (0, 0b1100000, -1.1), (0b0101010, 0b0101010, 0.4)]
    p = np.array([0.3, -1.2, 2.2, 0.5, -0.4])
    for dt, tol in (("c128", 1e-12), ("c64", 1e-5)):
        psi, lam = svlib.StateVector(n, dt).set_basis(0), svlib.StateVector(n, dt)
        ev, g = svlib.adjoint_grad(psi, lam, c, p, terms)
        ev_o, g_o, _ = oracle.adjoint_grad(c, p, terms)
        assert abs(ev - ev_o) <= tol and np.max(np.abs(g - g_o)) <= tol * 10


def test_batched_equals_plain(svlib):
    n, B = 10, 6
    c = W.hea(n, 3)
    terms = W.tfim(n)
    P = W.hea_params(B, c.n_params, 3)
    psis = [svlib.StateVector(n, "c64").set_basis(0) for _ in range(B)]
    lams = [svlib.StateVector(n, "c64") for _ in range(B)]
    ev_b, g_b = svlib.adjoint_grad_batch(psis, lams, c, P, terms)
    for b in range(B):
        psis[b].set_basis(0)
        ev, g = svlib.adjoint_grad(psis[b], lams[b], c, P[b], terms)
        assert abs(ev - ev_b[b]) <= 1e-6 and np.max(np.abs(g - g_b[b])) <= 1e-5


def test_hea_20q_full_size(svlib, oracle):
    """20-qubit, 10-layer ansatz (590 gates, 400 params), batch of 64 in one
    launch sequence; two sets checked against the oracle's FP64 adjoint and,
    for set 0, a parameter subset against the parameter-shift rule."""
    n, layers, B = 20, 10, 64
    c = W.hea(n, layers)
    terms = W.tfim(n)
    P = W.hea_params(B, c.n_params, 3)
    psis = [svlib.StateVector(n, "c64").set_basis(0) for _ in range(B)]
    lams = [svlib.StateVector(n, "c64") for _ in range(B)]
    ev_b, g_b = svlib.adjoint_grad_batch(psis, lams, c, P, terms)
    worst = 0.0
    for b in (0, 37):
        ev_o, g_o, _ = oracle.adjoint_grad(c, P[b], terms)
        err = float(np.max(np.abs(g_b[b] - g_o)))
        worst = max(worst, err / max(1, np.max(np.abs(g_o))))
        assert abs(ev_b[b] - ev_o) <= 1e-5 * max(1, abs(ev_o))
        assert err <= gtol(g_o), err
    print(f"hea 20q c64 batched: max relative gradient error {worst:.3e}")
    # parameter shift on a few parameters of set 0 (exact for exp(-i t P/2))
    for j in (0, 1, 199, 399):
        e = np.zeros(c.n_params)
        e[j] = math.pi / 2
        fp = oracle.expect(oracle.run(c, params=P[0] + e), terms)
        fm = oracle.expect(oracle.run(c, params=P[0] - e), terms)
        assert abs(g_b[0][j] - (fp - fm) / 2) <= gtol(g_b[0])


def test_autograd_function(svlib, oracle):
    n = 6
    c = W.hea(n, 2)
    terms = W.tfim(n)
    psi, lam = svlib.StateVector(n, "c128"), svlib.StateVector(n, "c128")
    theta = torch.tensor(W.hea_params(1, c.n_params, 1)[0], requires_grad=True)
    m = svlib.marshal(c)
    E = svlib.SvExpectation.apply(theta, psi, lam, m, terms, 0)
    E.backward()
    _, g_o, _ = oracle.adjoint_grad(c, theta.detach().numpy(), terms)
    assert np.max(np.abs(theta.grad.numpy() - g_o)) <= 1e-12


def test_unsupported_parametric_gate(svlib):
    from paper_2106_13995_gb300 import _native as N
    c = W.Circuit(3, [W.Op("U3", (0,), angles=(0, 0, 0), param=0)], n_params=1)
    psi, lam = svlib.StateVector(3, "c64").set_basis(0), svlib.StateVector(3, "c64")
    with pytest.raises(N.SvError, match="parametric"):
        svlib.adjoint_grad(psi, lam, c, np.zeros(1), [(0, 1, 1.0)])


def test_batched_gradient_graph_replay(svlib, oracle):
    """SV_MODE_TILED_GRAPH records the batched gradient's launch sequence once
    and replays it: every call (new parameters each time) agrees with direct
    launches to FP64 accumulation precision (the per-parameter sums are FP64
    atomics, whose order differs between any two runs) and matches the
    oracle."""
    from paper_2106_13995_gb300 import _native as N
    n, B = 12, 8
    h = W.hea(n, 3)
    terms = W.tfim(n)
    psis = [svlib.StateVector(n, "c64") for _ in range(B)]
    lams = [svlib.StateVector(n, "c64") for _ in range(B)]
    gopt = svlib.options(mode=N.SV_MODE_TILED_GRAPH)
    for seed in (1, 2, 3):
        params = W.hea_params(B, h.n_params, seed)
        for p in psis:
            p.set_basis(0)
        ev_g, g_g = svlib.adjoint_grad_batch(psis, lams, h, params, terms, opts=gopt)
        for p in psis:
            p.set_basis(0)
        ev_d, g_d = svlib.adjoint_grad_batch(psis, lams, h, params, terms)
        assert np.max(np.abs(ev_g - ev_d)) <= 1e-12 and np.max(np.abs(g_g - g_d)) <= 1e-12
        ev_o, g_o, _ = oracle.adjoint_grad(h, params[0], terms)
        assert abs(ev_g[0] - ev_o) <= 1e-5 and np.max(np.abs(g_g[0] - g_o)) <= 1e-5
