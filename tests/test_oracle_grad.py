"""Pins for the oracle's adjoint gradient: the parameter-shift rule (exact for
exp(-i theta P / 2) gates, where <H> = A cos theta + B sin theta + C) and
central differences divided by sin(h)/h, which for such f equal f'
exactly up to rounding."""
import math

import numpy as np

import workloads as W


def f_of(oracle, circ, params, terms):
    return oracle.expect(oracle.run(circ, params=params), terms)


def test_adjoint_vs_parameter_shift_and_fd(oracle):
    n, layers = 5, 3
    circ = W.hea(n, layers)
    terms = W.tfim(n)
    params = W.hea_params(2, circ.n_params, seed=3)
    for p in params:
        ev, g, psi_out = oracle.adjoint_grad(circ, p, terms)
        assert abs(ev - f_of(oracle, circ, p, terms)) <= 1e-13
        assert np.max(np.abs(psi_out - oracle.run(circ, params=p))) <= 1e-15
        shift = np.zeros_like(g)
        fd = np.zeros_like(g)
        h = 1e-3
        for j in range(circ.n_params):
            e = np.zeros_like(p)
            e[j] = math.pi / 2
            shift[j] = (f_of(oracle, circ, p + e, terms) - f_of(oracle, circ, p - e, terms)) / 2
            e[j] = h
            fd[j] = (f_of(oracle, circ, p + e, terms) - f_of(oracle, circ, p - e, terms)) / (2 * h)
        assert np.max(np.abs(g - shift)) <= 1e-12
        assert np.max(np.abs(g - fd / (math.sin(h) / h))) <= 1e-10


def test_adjoint_controlled_and_phase(oracle):
    """Controlled rotations and PHASE (generator diag(0,-2)) vs central FD."""
    n = 4
    c = W.Circuit(n, n_params=4)
    c.ops += [W.Op("H", (q,)) for q in range(n)]
    c.ops += [W.Op("RY", (1,), (0,), param=0), W.Op("PHASE", (2,), param=1),
              W.Op("RX", (3,), (1, 2), param=2), W.Op("X", (0,), (3,)), W.Op("RZ", (0,), param=3),
              W.Op("RY", (2,), param=0)]
    terms = [(0b0011, 0b0100, 0.7), (0, 0b1001, -1.3), (0b1000, 0b1000, 0.4)]
    p = np.array([0.4, -0.9, 1.7, 0.2])
    ev, g, _ = oracle.adjoint_grad(c, p, terms)
    h = 1e-5
    for j in range(4):
        e = np.zeros(4)
        e[j] = h
        fd = (f_of(oracle, c, p + e, terms) - f_of(oracle, c, p - e, terms)) / (2 * h)
        assert abs(g[j] - fd) <= 1e-8


def test_hea_structure():
    c = W.hea(20, 10)
    assert len(c.ops) == 590 and c.n_params == 400
    assert c.ops[0].name == "RY" and c.ops[1].name == "RZ" and c.ops[0].targets == c.ops[1].targets
