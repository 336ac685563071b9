"""Closed-form pins for the oracle: GHZ / Bell, QFT of a basis state,
H^n |0>, and the multiplier's a*b on basis and superposed inputs."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("n", [2, 3, 7, 12])
def test_ghz(oracle, n):
    psi = oracle.run(W.ghz(n))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - want)) <= 1e-16
    assert np.count_nonzero(psi) == 2


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_qft_of_basis_state(oracle, n):
    rng = np.random.default_rng(n)
    for x in rng.integers(0, 1 << n, size=4):
        psi = oracle.run(W.concat(W.basis_prep(n, int(x)), W.qft(n)))
        y = np.arange(1 << n)
        want = np.exp(2j * math.pi * int(x) * y / (1 << n)) / math.sqrt(1 << n)
        assert np.max(np.abs(psi - want)) <= 1e-13


def test_hadamard_all(oracle):
    for n in (1, 6, 11):
        psi = oracle.run(W.hadamard_all(n))
        assert np.max(np.abs(psi - 2 ** (-n / 2))) <= 1e-15


@pytest.mark.parametrize("nbits", [2, 3])
def test_multiplier_basis(oracle, nbits):
    circ = W.multiplier(nbits)
    n = circ.n_qubits
    assert n == 4 * nbits + 1
    for a in range(1 << nbits):
        for b in range(1 << nbits):
            psi = np.zeros(1 << n, dtype=complex)
            psi[W.multiplier_basis_index(a, b, nbits)] = 1
            out = oracle.run(circ, psi)
            idx = W.multiplier_basis_index(a, b, nbits, a * b)
            assert out[idx] == 1.0 and np.count_nonzero(out) == 1, (a, b)


def test_multiplier_superposition(oracle):
    nbits = 3
    out = oracle.run(W.multiplier(nbits, hadamard_inputs=True))
    p = np.abs(out) ** 2
    want = np.zeros_like(p)
    for a in range(8):
        for b in range(8):
            want[W.multiplier_basis_index(a, b, nbits, a * b)] = 2.0 ** (-2 * nbits)
    assert np.max(np.abs(p - want)) <= 1e-15


def test_multiplier_gate_count():
    c = W.multiplier(7)
    assert c.n_qubits == 29 and len(c.ops) == 301
    assert max(len(o.controls) for o in c.ops) == 3


def test_width_reduction_drops_gates():
    c = W.grid_random(5, 6, 20, 1)
    r = W.remove_qubits(c, 4, 101)
    assert r.n_qubits == 26
    kept = len(r.ops)
    assert kept < len(c.ops)
    r.validate()
