"""GPU parity of single-gate application (K1-K5) against the FP64 oracle,
called through the C ABI on random states."""
import numpy as np
import pytest

import workloads as W
from conftest import fidelity_metrics

pytestmark = pytest.mark.gpu

TOL = {"c64": dict(infid=1e-5, amp=2e-6), "c128": dict(infid=1e-12, amp=1e-13)}


def _run_gate(svlib, oracle, n, dt, U, targets, controls, seed):
    rng = np.random.default_rng(seed)
    psi0 = W.random_state(n, rng)
    s = svlib.StateVector(n, dt).load(psi0)
    s.apply_gate(U, targets, controls)
    got = s.numpy()
    want = oracle.apply(psi0.astype(np.complex64 if dt == "c64" else np.complex128).astype(np.complex128),
                        U, targets, controls)
    s.close()
    return fidelity_metrics(want, got)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 3, 6, 11])
def test_1q_every_target(svlib, oracle, dt, n):
    rng = np.random.default_rng(n)
    for q in range(n):
        U = W.random_unitary(1, rng)
        inf, amp = _run_gate(svlib, oracle, n, dt, U, [q], [], seed=q)
        assert inf <= TOL[dt]["infid"] and amp <= TOL[dt]["amp"], (q, inf, amp)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_dense_k_with_controls(svlib, oracle, dt):
    rng = np.random.default_rng(7)
    n = 10
    for k in (1, 2, 3, 4, 5, 6):
        for nc in (0, 1, 2):
            qs = [int(x) for x in rng.permutation(n)[: k + nc]]
            U = W.random_unitary(k, rng)
            inf, amp = _run_gate(svlib, oracle, n, dt, U, qs[:k], qs[k:], seed=k * 10 + nc)
            assert inf <= TOL[dt]["infid"] and amp <= TOL[dt]["amp"] * (1 << k), (k, nc, inf, amp)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_diagonal_and_permutation(svlib, oracle, dt):
    rng = np.random.default_rng(8)
    n = 9
    for name, k in [("CZ", 2), ("T", 1), ("RZ", 1), ("PHASE", 1)]:
        U = oracle.gate_matrix(name, rng.uniform(-3, 3, 3))
        qs = [int(x) for x in rng.permutation(n)[: k + 2]]
        inf, amp = _run_gate(svlib, oracle, n, dt, U, qs[:k], qs[k:], seed=k)
        assert inf <= TOL[dt]["infid"] and amp <= TOL[dt]["amp"], name
    # permutation gates move amplitudes bit-exactly
    X = oracle.gate_matrix("X")
    psi0 = W.random_state(n, rng).astype(np.complex64 if dt == "c64" else np.complex128)
    s = svlib.StateVector(n, dt).load(psi0)
    s.apply_gate(X, [3], [0, 5]).apply_gate(oracle.gate_matrix("SWAP"), [1, 7])
    want = oracle.apply(oracle.apply(psi0.astype(np.complex128), X, [3], [0, 5]),
                        oracle.gate_matrix("SWAP"), [1, 7])
    assert np.array_equal(s.numpy().astype(np.complex128), want)


def test_adjoint_flag(svlib, oracle):
    rng = np.random.default_rng(9)
    U = W.random_unitary(2, rng)
    psi0 = W.random_state(8, rng)
    s = svlib.StateVector(8, "c128").load(psi0)
    s.apply_gate(U, [2, 6]).apply_gate(U, [2, 6], adjoint=True)
    assert np.max(np.abs(s.numpy() - psi0)) <= 1e-14


def test_set_basis_and_norm(svlib):
    for dt in ("c64", "c128"):
        s = svlib.StateVector(12, dt).set_basis(1234)
        v = s.numpy()
        assert v[1234] == 1 and np.count_nonzero(v) == 1
        assert s.norm2() == 1.0
        s2 = svlib.StateVector(5, dt).set_basis(31)
        assert s2.numpy()[31] == 1


def test_bad_arguments_report_errors(svlib):
    from paper_2106_13995_gb300 import _native as N
    s = svlib.StateVector(6, "c64").set_basis(0)
    with pytest.raises(N.SvError, match="duplicate"):
        s.apply_gate(np.eye(4), [1, 1])
    with pytest.raises(N.SvError, match="out of range"):
        s.apply_gate(np.eye(2), [6])
    with pytest.raises(N.SvError, match="duplicate"):
        s.apply_gate(np.eye(2), [2], [2])
    with pytest.raises(N.SvError):
        s.expect([(1 << 7, 0, 1.0)])
    with pytest.raises(N.SvError):
        s.set_basis(64)
    assert s.norm2() == 1.0      # the state survived every rejected call
