"""Pins for the oracle's gate application (c-1): the index loop equals the
materialised 2^n x 2^n matrix, and that matrix equals independent numpy
constructions (Kronecker products for adjacent targets, tensor contraction
with control slicing for arbitrary ones)."""
import itertools

import numpy as np
import pytest

import workloads as W


def np_apply(psi, U, targets, controls=()):
    """Independent statement: reshape psi to a 2x...x2 tensor (axis a <-> qubit
    n-1-a), contract U on the target axes inside the controls=1 slice."""
    n = int(np.log2(psi.size))
    T = psi.reshape([2] * n).copy()
    k = len(targets)
    Ut = U.reshape([2] * (2 * k))          # (r_{k-1} .. r_0, c_{k-1} .. c_0)
    sl = [slice(None)] * n
    for c in controls:
        sl[n - 1 - c] = 1
    sub = T[tuple(sl)]
    # axes of the sub-tensor after removing control axes
    remaining = [a for a in range(n) if not (isinstance(sl[a], int))]
    tax = [remaining.index(n - 1 - targets[j]) for j in reversed(range(k))]   # c_{k-1}..c_0
    out = np.tensordot(Ut, sub, axes=(list(range(k, 2 * k)), tax))
    # tensordot puts the k output axes first; move them back to tax positions
    out = np.moveaxis(out, list(range(k)), tax)
    T[tuple(sl)] = out
    return T.reshape(-1)


def test_full_matrix_vs_kron(oracle):
    rng = np.random.default_rng(11)
    n = 6
    for k in (1, 2, 3):
        for t0 in range(n - k + 1):
            U = W.random_unitary(k, rng)
            M = oracle.full_matrix(n, U, list(range(t0, t0 + k)))
            ref = np.kron(np.kron(np.eye(1 << (n - t0 - k)), U), np.eye(1 << t0))
            assert np.allclose(M, ref, atol=0, rtol=0), (k, t0)


def test_full_matrix_controlled_vs_projectors(oracle):
    rng = np.random.default_rng(12)
    n = 4
    U = W.random_unitary(1, rng)
    P0, P1 = np.diag([1, 0]), np.diag([0, 1])
    # control qubit 3, target qubit 0:  |0><0| (x) I + |1><1| (x) U  on (q3, q2, q1, q0)
    ref = np.kron(np.kron(P0, np.eye(4)), np.eye(2)) + np.kron(np.kron(P1, np.eye(4)), U)
    assert np.allclose(oracle.full_matrix(n, U, [0], [3]), ref, atol=0)


@pytest.mark.parametrize("n", [1, 3, 5, 7])
def test_index_loop_equals_full_matrix(oracle, n):
    rng = np.random.default_rng(100 + n)
    for trial in range(30):
        k = int(rng.integers(1, min(3, n) + 1))
        nc = int(rng.integers(0, min(2, n - k) + 1))
        qs = [int(q) for q in rng.permutation(n)[: k + nc]]
        t, c = qs[:k], qs[k:]
        U = W.random_unitary(k, rng)
        psi = W.random_state(n, rng)
        M = oracle.full_matrix(n, U, t, c)
        want = oracle.matvec(M, psi)
        got = oracle.apply(psi.copy(), U, t, c)
        assert np.max(np.abs(got - want)) <= 1e-14
        indep = np_apply(psi, U, t, c)
        assert np.max(np.abs(indep - want)) <= 1e-14


def test_every_target_position(oracle):
    rng = np.random.default_rng(5)
    n = 8
    for k in (1, 2, 3):
        for t in itertools.permutations(range(n), k):
            if rng.random() > (1.0 if k == 1 else 0.08):
                continue
            U = W.random_unitary(k, rng)
            psi = W.random_state(n, rng)
            got = oracle.apply(psi.copy(), U, list(t))
            assert np.max(np.abs(got - np_apply(psi, U, list(t)))) <= 1e-14


def test_k6_dense(oracle):
    rng = np.random.default_rng(6)
    n = 8
    t = [7, 0, 3, 5, 1, 6]
    U = W.random_unitary(6, rng)
    psi = W.random_state(n, rng)
    assert np.max(np.abs(oracle.apply(psi.copy(), U, t) - np_apply(psi, U, t))) <= 1e-13


def test_run_matches_matrix_product(oracle):
    """A whole circuit equals the product of its per-gate full matrices."""
    circ = W.random_gate_circuit(6, 40, seed=9)
    psi = oracle.run(circ)
    M = np.eye(64, dtype=complex)
    for op in circ.ops:
        U = op.matrix if op.name == "MATRIX" else oracle.gate_matrix(op.name, op.angles)
        M = oracle.full_matrix(6, U, list(op.targets), list(op.controls)) @ M
    assert np.max(np.abs(psi - M[:, 0])) <= 1e-13


def test_norm_preserved(oracle):
    for seed in range(3):
        circ = W.random_gate_circuit(9, 60, seed=seed)
        psi = oracle.run(circ, W.random_state(9, np.random.default_rng(seed)))
        assert abs(oracle.norm2(psi) - 1) <= 1e-13
    c0 = W.random_u3_cz(12, 20, 0)
    assert abs(oracle.norm2(oracle.run(c0)) - 1) <= 1e-13


def test_config0_structure_small_via_full_matrix(oracle):
    """The 12-qubit random U3+CZ structure, run at n = 10, agrees with the
    product of materialised matrices applied one by one."""
    c = W.random_u3_cz(10, 3, 0)
    psi = oracle.run(c)
    ref = oracle.zero_state(10)
    for op in c.ops:
        U = oracle.gate_matrix(op.name, op.angles)
        ref = oracle.matvec(oracle.full_matrix(10, U, list(op.targets), list(op.controls)), ref)
    assert np.max(np.abs(psi - ref)) <= 1e-13


def test_parametric_substitution(oracle):
    c = W.Circuit(3, [W.Op("RY", (1,), param=0), W.Op("RZ", (2,), (0,), param=1)], n_params=2)
    p = np.array([0.3, -1.1])
    fixed = W.Circuit(3, [W.Op("RY", (1,), angles=(0.3,)), W.Op("RZ", (2,), (0,), angles=(-1.1,))])
    psi0 = W.random_state(3, np.random.default_rng(0))
    assert np.array_equal(oracle.run(c, psi0, p), oracle.run(fixed, psi0))
