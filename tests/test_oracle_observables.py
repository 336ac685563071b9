"""Pins for Pauli expectations, <Z_i>, norms, sampling and the SplitMix64
counter generator."""
import math
import os
from functools import reduce

import numpy as np
import pytest
from scipy import stats

import workloads as W

P1 = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]], dtype=complex),
      "Y": np.array([[0, -1j], [1j, 0]]), "Z": np.diag([1.0 + 0j, -1.0])}


def pauli_matrix(n, xm, zm):
    """Kronecker product of single-qubit Paulis (qubit n-1 leftmost)."""
    facs = []
    for q in reversed(range(n)):
        x, z = (xm >> q) & 1, (zm >> q) & 1
        facs.append(P1["Y" if x and z else "X" if x else "Z" if z else "I"])
    return reduce(np.kron, facs)


def random_terms(n, count, rng):
    return [(int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n)), float(rng.normal()))
            for _ in range(count)]


def test_expect_vs_explicit_matrix(oracle):
    rng = np.random.default_rng(0)
    for n in (1, 3, 6):
        psi = W.random_state(n, rng)
        terms = random_terms(n, 10, rng)
        H = sum(c * pauli_matrix(n, xm, zm) for xm, zm, c in terms)
        assert abs(oracle.expect(psi, terms) - np.vdot(psi, H @ psi).real) <= 1e-13
        assert np.max(np.abs(oracle.apply_pauli_sum(psi, terms) - H @ psi)) <= 1e-13


def test_tfim_matrix(oracle):
    n = 6
    terms = W.tfim(n)
    assert len(terms) == 2 * n - 1
    Zi = lambda i: pauli_matrix(n, 0, 1 << i)
    Xi = lambda i: pauli_matrix(n, 1 << i, 0)
    H = sum(Zi(i) @ Zi(i + 1) for i in range(n - 1)) + 0.5 * sum(Xi(i) for i in range(n))
    psi = W.random_state(n, np.random.default_rng(1))
    assert abs(oracle.expect(psi, terms) - np.vdot(psi, H @ psi).real) <= 1e-13


def test_special_states(oracle):
    n = 7
    for idx in (0, 5, 127, 64):
        psi = np.zeros(1 << n, dtype=complex)
        psi[idx] = 1
        z = oracle.z_all(psi)
        assert np.array_equal(z, np.array([1.0 - 2 * ((idx >> q) & 1) for q in range(n)]))
    plus = oracle.run(W.hadamard_all(n))
    for q in range(n):
        assert abs(oracle.expect(plus, [(1 << q, 0, 1.0)]) - 1.0) <= 1e-14
    assert abs(oracle.expect(plus, [(0, 1, 1.0)])) <= 1e-15


def test_z_all_vs_matrix(oracle):
    n = 5
    psi = W.random_state(n, np.random.default_rng(2))
    z = oracle.z_all(psi)
    for q in range(n):
        assert abs(z[q] - np.vdot(psi, pauli_matrix(n, 0, 1 << q) @ psi).real) <= 1e-14
    assert abs(oracle.norm2(psi) - 1) <= 1e-14
    assert abs(oracle.norm2(2 * psi) - 4) <= 1e-13


def test_splitmix64_published_values(oracle):
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for s, hx in rows:
        assert oracle.splitmix64(0, int(s)) == int(hx, 16)


def test_sample_basis_and_ghz(oracle):
    n = 9
    psi = np.zeros(1 << n, dtype=complex)
    psi[300] = 1
    assert np.all(oracle.sample(psi, 1000, 5) == 300)
    g = oracle.run(W.ghz(n))
    s = oracle.sample(g, 20000, 7)
    assert set(np.unique(s).tolist()) <= {0, (1 << n) - 1}
    ones = int(np.sum(s == (1 << n) - 1))
    assert abs(ones - 10000) < 5 * math.sqrt(20000 * 0.25)


def test_sample_chi_square(oracle):
    n = 6
    psi = W.random_state(n, np.random.default_rng(3))
    shots = 200000
    s = oracle.sample(psi, shots, 11)
    obs = np.bincount(s.astype(np.int64), minlength=1 << n)
    exp = np.abs(psi) ** 2 * shots
    assert stats.chisquare(obs, exp).pvalue > 1e-3


def test_sample_vs_cumsum_search(oracle):
    """Brute-force restatement: cumulative sum + sorted search."""
    n = 10
    psi = W.random_state(n, np.random.default_rng(4)) * 0.7
    shots, seed = 5000, 12345
    got = oracle.sample(psi, shots, seed)
    cdf = np.cumsum(np.abs(psi) ** 2)
    u = np.array([(oracle.splitmix64(seed, s) >> 11) * 2.0 ** -53 for s in range(shots)])
    tgt = u * cdf[-1]
    want = np.searchsorted(cdf, tgt, side="right")
    near = np.min(np.abs(cdf[None, :] - tgt[:, None]), axis=1) < 1e-12
    assert np.all((got == want) | near)
