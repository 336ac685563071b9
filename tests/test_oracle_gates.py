"""Pins for the oracle's gate matrices (the paper fixes no convention; the
readings are the standard definitions restated here through independent
routes: matrix exponentials, squares, decompositions)."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

I2 = np.eye(2)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]])
Z = np.diag([1.0 + 0j, -1.0])

NAMED = ["I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "SX", "SY", "SW",
         "RX", "RY", "RZ", "PHASE", "U3", "CZ", "SWAP", "FSIM"]


@pytest.mark.parametrize("name", NAMED)
def test_unitary(oracle, name):
    rng = np.random.default_rng(7)
    for _ in range(5):
        U = oracle.gate_matrix(name, rng.uniform(-4, 4, size=3))
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-15, rtol=0)


def test_paulis(oracle):
    assert np.array_equal(oracle.gate_matrix("X"), X)
    assert np.array_equal(oracle.gate_matrix("Y"), Y)
    assert np.array_equal(oracle.gate_matrix("Z"), Z)
    assert np.array_equal(oracle.gate_matrix("I"), I2)


@pytest.mark.parametrize("name,P", [("RX", X), ("RY", Y), ("RZ", Z)])
def test_rotations_are_exponentials(oracle, name, P):
    for th in np.linspace(-7, 7, 29):
        assert np.allclose(oracle.gate_matrix(name, [th]), expm(-0.5j * th * P), atol=2e-15, rtol=0)


def test_square_roots(oracle):
    W = (X + Y) / math.sqrt(2)
    for name, P in [("SX", X), ("SY", Y), ("SW", W)]:
        R = oracle.gate_matrix(name)
        assert np.allclose(R @ R, P, atol=1e-15, rtol=0), name
        # Cirq's phase: P^(1/2) = e^{i pi/4} exp(-i pi/4 P)
        assert np.allclose(R, np.exp(0.25j * math.pi) * expm(-0.25j * math.pi * P), atol=1e-15, rtol=0)


def test_clifford_t_relations(oracle):
    H = oracle.gate_matrix("H")
    S, T = oracle.gate_matrix("S"), oracle.gate_matrix("T")
    assert np.allclose(H, (X + Z) / math.sqrt(2), atol=1e-16)
    assert np.allclose(S @ S, Z, atol=1e-16)
    assert np.allclose(T @ T, S, atol=1e-15)
    assert np.allclose(oracle.gate_matrix("SDG"), S.conj().T, atol=0)
    assert np.allclose(oracle.gate_matrix("TDG"), T.conj().T, atol=1e-16)


def test_u3_decomposition(oracle):
    rng = np.random.default_rng(3)
    for _ in range(20):
        th, ph, la = rng.uniform(-7, 7, size=3)
        U = oracle.gate_matrix("U3", [th, ph, la])
        rz = lambda a: expm(-0.5j * a * Z)
        ry = lambda a: expm(-0.5j * a * Y)
        assert np.allclose(U, np.exp(0.5j * (ph + la)) * rz(ph) @ ry(th) @ rz(la), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("U3", [th, 0, 0]), ry(th), atol=1e-15)
        assert np.allclose(oracle.gate_matrix("U3", [th, -math.pi / 2, math.pi / 2]),
                           expm(-0.5j * th * X), atol=1e-15)
        assert np.allclose(oracle.gate_matrix("U3", [0, 0, la]), np.diag([1, np.exp(1j * la)]), atol=1e-15)
        assert np.allclose(oracle.gate_matrix("PHASE", [la]), np.exp(0.5j * la) * rz(la), atol=1e-15)


def test_two_qubit_gates(oracle):
    assert np.array_equal(oracle.gate_matrix("CZ"), np.diag([1, 1, 1, -1]).astype(complex))
    sw = np.zeros((4, 4))
    for i in range(4):
        sw[((i & 1) << 1) | (i >> 1), i] = 1
    assert np.array_equal(oracle.gate_matrix("SWAP"), sw)
    XX, YY = np.kron(X, X), np.kron(Y, Y)
    for th in np.linspace(-3, 3, 13):
        assert np.allclose(oracle.gate_matrix("FSIM", [th, 0]), expm(-0.5j * th * (XX + YY)), atol=1e-14)
    for ph in np.linspace(-3, 3, 13):
        assert np.allclose(oracle.gate_matrix("FSIM", [0, ph]), np.diag([1, 1, 1, np.exp(-1j * ph)]), atol=1e-15)
    F = oracle.gate_matrix("FSIM", [math.pi / 2, math.pi / 6])
    assert F[1, 1] == 0 and F[2, 2] == 0          # snapped cos(pi/2)
    assert F[1, 2] == -1j and F[2, 1] == -1j
