"""The Python front end (circuit builder, Pauli sums) without a GPU: the
circuits it builds are the library's circuit format (run here through the
FP64 oracle), inverse() undoes a circuit, parameters bind as the library
binds them, and Pauli-sum products and sums equal the explicit matrices."""
import numpy as np
import pytest

import workloads as W
from paper_2106_13995_gb300 import Circuit, PauliSum, X, Y, Z, I, grid_qubit, ising


def test_builder_matches_workload_circuits(oracle):
    n = 6
    c = Circuit(n).h(0)
    for i in range(1, n):
        c.cx(0, i)
    g = W.ghz(n)
    assert [(o.name, o.targets, o.controls) for o in c.ops] == [(o.name, tuple(o.targets), tuple(o.controls))
                                                              for o in g.ops]
    psi = oracle.run(c)
    assert abs(psi[0] - 2 ** -0.5) < 1e-15 and abs(psi[-1] - 2 ** -0.5) < 1e-15
    # the 5 x 6 lattice numbering
    assert grid_qubit(2, 3, 6) == 15
    with pytest.raises(ValueError):
        grid_qubit(0, 6, 6)


def random_builder_circuit(n, rng, depth=60):
    c = Circuit(n)
    for _ in range(depth):
        kind = rng.integers(0, 12)
        q = [int(x) for x in rng.choice(n, size=4, replace=False)]
        a = float(rng.uniform(-3, 3))
        ctl = (q[3],) if rng.random() < 0.3 else ()
        if kind == 0:
            c.h(q[0], controls=ctl)
        elif kind == 1:
            c.s(q[0]).t(q[1])
        elif kind == 2:
            c.sx(q[0]).sy(q[1]).sw(q[2])
        elif kind == 3:
            c.rx(a, q[0], controls=ctl)
        elif kind == 4:
            c.ry(a, q[0]).rz(-a, q[1])
        elif kind == 5:
            c.phase(a, q[0], controls=ctl)
        elif kind == 6:
            c.u3(a, 0.4, -1.1, q[0], controls=ctl)
        elif kind == 7:
            c.cz(q[0], q[1]).swap(q[1], q[2])
        elif kind == 8:
            c.fsim(a, 0.7, q[0], q[1], controls=ctl)
        elif kind == 9:
            c.toffoli(q[0], q[1], q[2])
        elif kind == 10:
            c.unitary(W.random_unitary(2, rng), q[0], q[1], controls=ctl)
        else:
            c.sdg(q[0]).tdg(q[1]).y(q[2]).z(q[0])
    return c


def test_inverse_undoes_the_circuit(oracle):
    rng = np.random.default_rng(3)
    for n in (5, 7):
        c = random_builder_circuit(n, rng)
        psi0 = W.random_state(n, rng)
        out = oracle.run(c + c.inverse(), psi0)
        assert np.max(np.abs(out - psi0)) <= 1e-12
        # and U psi differs from psi (the check is not vacuous)
        assert np.max(np.abs(oracle.run(c, psi0) - psi0)) > 1e-3


def test_parameters_bind_like_the_library(oracle):
    c = Circuit(4)
    th = [c.parameter(f"t{i}") for i in range(3)]
    c.h(0).ry(th[0], 1).cx(1, 2).rz(th[1], 2).phase(th[2], 3).rx(0.3, 0)
    p = np.array([0.4, -1.2, 2.5])
    assert c.n_params == 3 and c.parameter_names() == ["t0", "t1", "t2"]
    a = oracle.run(c, params=p)
    b = oracle.run(c.bind(p))
    assert np.max(np.abs(a - b)) <= 1e-15
    with pytest.raises(ValueError):
        c.inverse()          # a parametric gate has no inverse in the circuit format
    assert np.max(np.abs(oracle.run(c.bind(p) + c.bind(p).inverse()) - oracle.zero_state(4))) <= 1e-12
    with pytest.raises(ValueError):
        Circuit(2).u3(0.1, th[0], 0.2, 0)    # only the first angle may be a parameter
    with pytest.raises(ValueError):
        Circuit(2).cx(0, 0)
    with pytest.raises(ValueError):
        Circuit(2).h(2)


# --- Pauli sums against explicit matrices ---------------------------------------

_P = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
      "Z": np.diag([1.0, -1.0])}


def pauli_matrix(ps: PauliSum, n: int) -> np.ndarray:
    """Sum of coeff * (tensor product of single-qubit Paulis), qubit q = bit q
    (so qubit 0 is the rightmost factor)."""
    M = np.zeros((1 << n, 1 << n), complex)
    for (x, z), c in ps.t.items():
        m = np.array([[1.0 + 0j]])
        for q in reversed(range(n)):
            k = {(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}[((x >> q) & 1, (z >> q) & 1)]
            m = np.kron(m, _P[k])
        M += c * m
    return M


def test_single_qubit_pauli_products():
    one = {"X": X(0), "Y": Y(0), "Z": Z(0)}
    for a in "XYZ":
        for b in "XYZ":
            got = pauli_matrix(one[a] * one[b], 1)
            assert np.allclose(got, _P[a] @ _P[b], atol=0), (a, b)
    assert (X(0) * Y(0)).t == {(0, 1): 1j}          # XY = iZ
    assert (Y(0) * X(0)).t == {(0, 1): -1j}         # YX = -iZ
    assert (Z(0) * Z(0)).t == {(0, 0): 1}


def test_pauli_sums_match_matrices():
    rng = np.random.default_rng(8)
    n = 3
    kinds = [X, Y, Z]
    for _ in range(20):
        A = PauliSum()
        B = PauliSum()
        for _ in range(3):
            ta = kinds[rng.integers(3)](int(rng.integers(n))) * kinds[rng.integers(3)](int(rng.integers(n)))
            tb = kinds[rng.integers(3)](int(rng.integers(n)))
            A = A + float(rng.normal()) * ta
            B = B + complex(rng.normal(), rng.normal()) * tb
        MA, MB = pauli_matrix(A, n), pauli_matrix(B, n)
        assert np.allclose(pauli_matrix(A * B, n), MA @ MB, atol=1e-12)
        assert np.allclose(pauli_matrix(A + 2.0 * B - I(), n), MA + 2 * MB - np.eye(1 << n), atol=1e-12)


def test_observable_terms_and_ising(oracle):
    n = 6
    H = ising(n)
    assert sorted(H.terms()) == sorted((x, z, c) for x, z, c in W.tfim(n))
    # <psi|H|psi> from the terms equals the explicit matrix
    psi = W.random_state(n, np.random.default_rng(1))
    want = float(np.real(np.vdot(psi, pauli_matrix(H, n) @ psi)))
    assert abs(oracle.expect(psi, H.terms()) - want) <= 1e-12
    with pytest.raises(ValueError):
        (X(0) * Y(0)).terms()     # i Z is not Hermitian
