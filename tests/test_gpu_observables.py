"""GPU parity of expectations, <Z_q>, norms and sampling against the oracle."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def random_terms(n, count, rng):
    return [(int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n)), float(rng.normal()))
            for _ in range(count)]


@pytest.mark.parametrize("dt,tol", [("c64", 2e-6), ("c128", 1e-12)])
def test_expect_random_paulis(svlib, oracle, dt, tol):
    rng = np.random.default_rng(1)
    for n in (3, 12, 17):
        psi = W.random_state(n, rng)
        s = svlib.StateVector(n, dt).load(psi)
        cast = s.numpy().astype(np.complex128)
        terms = random_terms(n, 25, rng) + W.tfim(n)
        assert abs(s.expect(terms) - oracle.expect(cast, terms)) <= tol * len(terms)
        assert np.max(np.abs(s.z_all() - oracle.z_all(cast))) <= tol
        assert abs(s.norm2() - oracle.norm2(cast)) <= tol


@pytest.mark.parametrize("dt,tol", [("c64", 2e-6), ("c128", 1e-12)])
def test_expect_diagonal_groups(svlib, oracle, dt, tol):
    """Groups of Z strings only (x mask 0): random strings of weight 0..4
    over low and high bits, the same mask with several coefficients, and
    nearest-neighbour ZZ terms, at widths around the reduction kernels'
    run and chunk sizes."""
    rng = np.random.default_rng(7)
    for n in (7, 8, 9, 10, 14, 20):
        psi = W.random_state(n, rng)
        s = svlib.StateVector(n, dt).load(psi)
        cast = s.numpy().astype(np.complex128)
        terms = []
        for _ in range(40):
            w = int(rng.integers(0, 5))
            z = 0
            for q in rng.choice(n, size=min(w, n), replace=False):
                z |= 1 << int(q)
            terms.append((0, z, float(rng.normal())))
        terms += [(0, terms[3][1], 0.5), (0, terms[3][1], -0.25)]
        terms += [(0, (1 << q) | (1 << (q + 1)), 1.0) for q in range(n - 1)][:20]
        want = oracle.expect(cast, terms)
        got = s.expect(terms)
        scale = sum(abs(t[2]) for t in terms)
        assert abs(got - want) <= tol * scale, (n, got, want)
        s.close()


def test_z_all_large(svlib, oracle):
    n = 22
    c = W.random_u3_cz(n, 2, 11)
    s = svlib.StateVector(n, "c64").set_basis(0).apply_circuit(c)
    cast = s.numpy().astype(np.complex128)
    assert np.max(np.abs(s.z_all() - oracle.z_all(cast))) <= 1e-6


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_sample_matches_oracle(svlib, oracle, dt):
    rng = np.random.default_rng(3)
    # 21 and 22 qubits: 2048 and 4096 CDF chunks, a two-level prefix scan
    for n in (4, 11, 16, 21, 22):
        s = svlib.StateVector(n, dt).load(W.random_state(n, rng))
        cast = s.numpy().astype(np.complex128)
        shots, seed = 20000, 12345 + n
        got = s.sample(shots, seed)
        want = oracle.sample(cast, shots, seed)
        cdf = np.cumsum(np.abs(cast) ** 2)
        u = np.array([(oracle.splitmix64(seed, j) >> 11) * 2.0 ** -53 for j in range(shots)]) * cdf[-1]
        near = np.min(np.abs(cdf[None, :] - u[:, None]), axis=1) < 1e-9 if n <= 11 else \
            np.abs(cdf[np.searchsorted(cdf, u, side="right").clip(0, cdf.size - 1)] - u) < 1e-9
        mismatch = (got != want) & ~near
        assert not mismatch.any(), int(mismatch.sum())


def test_sample_special_states(svlib):
    s = svlib.StateVector(18, "c64").set_basis(77777)
    assert np.all(s.sample(1000, 1) == 77777)
    g = svlib.StateVector(18, "c64").set_basis(0).apply_circuit(W.ghz(18))
    x = g.sample(200000, 5)
    assert set(np.unique(x).tolist()) <= {0, (1 << 18) - 1}
    ones = int(np.sum(x != 0))
    assert abs(ones - 100000) < 5 * np.sqrt(200000 * 0.25)


def test_sample_many_shots_batches(svlib):
    """More shots than one device buffer holds: batches keep the counter."""
    s = svlib.StateVector(10, "c128").set_basis(0).apply_circuit(W.hadamard_all(10))
    a = s.sample(300000, 42)
    b = s.sample(10, 42)
    assert np.array_equal(a[:10], b)
    obs = np.bincount(a.astype(np.int64), minlength=1024)
    from scipy import stats
    assert stats.chisquare(obs).pvalue > 1e-4


def test_renormalize(svlib):
    s = svlib.StateVector(12, "c64").load(3 * W.random_state(12, np.random.default_rng(0)))
    old = s.renormalize()
    assert abs(old - 9) < 1e-4
    assert abs(s.norm2() - 1) < 1e-6
