"""Pins of the comparison metrics every parity test asserts through.

fidelity(a, b) = |<a|b>|^2 / (||a||^2 ||b||^2) and infidelity(a, b) = 1 - F
(the state is the full amplitude vector, paper Sec. II; two states that
differ by a global phase are the same physical state).  The checks use only
what the mathematics fixes: orthogonal states, global phases, a two-level
rotation with 1 - F = sin^2(eps) exactly, states with a constructed overlap,
and scale invariance.  Each planted mistake (a dropped phase removal, a
dropped ||d||^4/4 term, a missing normalisation) must fail at least one of
them, which shows the checks can see such mistakes.
"""
import numpy as np
import pytest


def _rand_state(rng, n):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def _with_overlap(rng, n, theta, alpha):
    """(psi, phi) with |<psi|phi>| = cos(theta) exactly in exact arithmetic:
    phi = e^{i alpha} (cos(theta) psi + sin(theta) chi), chi orthogonal to psi."""
    psi = _rand_state(rng, n)
    chi = _rand_state(rng, n)
    chi = chi - np.vdot(psi, chi) * psi
    chi /= np.linalg.norm(chi)
    phi = np.exp(1j * alpha) * (np.cos(theta) * psi + np.sin(theta) * chi)
    return psi, phi


def metric_failures(infid, fid):
    """Names of the pins that infid / fid violate (empty = all hold)."""
    bad = []
    rng = np.random.default_rng(11)
    # orthogonal states: 1 - F = 1, F = 0
    a = np.zeros(8, complex)
    b = np.zeros(8, complex)
    a[3], b[5] = 1.0, 1j
    if infid(a, b) != 1.0:
        bad.append("orthogonal")
    if fid(a, b) != 0.0:
        bad.append("orthogonal-F")
    # a global phase does not change the state
    for phi in (0.3, 1.7, -2.9, np.pi):
        psi = _rand_state(rng, 6)
        if not infid(psi, np.exp(1j * phi) * psi) <= 1e-28:
            bad.append(f"phase {phi}")
        if abs(fid(psi, np.exp(1j * phi) * psi) - 1.0) > 1e-14:
            bad.append(f"phase-F {phi}")
    # cos(eps)|0> + sin(eps)|1> against |0>: 1 - F = sin^2(eps), no cancellation
    for eps in (1e-1, 1e-3, 1e-5, 1e-8):
        ref = np.array([1.0, 0.0], complex)
        got = np.array([np.cos(eps), np.sin(eps)], complex)
        want = np.sin(eps) ** 2
        if abs(infid(ref, got) - want) > 1e-14 * want:
            bad.append(f"two-level {eps}")
    # unnormalised inputs: the metric normalises
    for eps in (1e-2, 1e-6):
        ref = np.array([1.0, 0.0], complex)
        got = np.array([np.cos(eps), np.sin(eps)], complex)
        want = np.sin(eps) ** 2
        if abs(infid(3.5 * ref, 0.25j * got) - want) > 1e-14 * want:
            bad.append(f"scaled {eps}")
    # constructed overlap at moderate and small angles, with a relative phase
    for theta, alpha in ((0.7, 0.4), (0.05, -1.2), (1e-4, 2.2)):
        psi, phi = _with_overlap(rng, 7, theta, alpha)
        want = np.sin(theta) ** 2
        if abs(infid(psi, phi) - want) > 1e-10 * want + 1e-15:
            bad.append(f"overlap {theta}")
        if abs(fid(2.0 * psi, 0.3 * phi) - np.cos(theta) ** 2) > 1e-13:
            bad.append(f"overlap-F {theta}")
    # the direct definition where it has no cancellation (1 - F >= 1e-3)
    for _ in range(4):
        a_, b_ = _rand_state(rng, 5), _rand_state(rng, 5)
        direct = 1 - abs(np.vdot(a_, b_)) ** 2 / (np.vdot(a_, a_).real * np.vdot(b_, b_).real)
        if abs(infid(a_, b_) - direct) > 1e-12:
            bad.append("direct")
    return bad


def test_oracle_metrics_hold(oracle):
    assert metric_failures(oracle.infidelity, oracle.fidelity) == []


def test_max_abs_err(oracle):
    a = np.array([1.0, 1j, 0.0], complex)
    b = np.array([1.0, 1j + 3e-7, 4e-7], complex)
    assert abs(oracle.max_abs_err(a, b) - 4e-7) < 1e-20


# --- planted mistakes: each must fail at least one pin -----------------------------

def _unit(v):
    return v / np.sqrt(np.vdot(v, v).real)


def _no_phase_removal(ref, got):
    r, g = _unit(np.asarray(ref, complex)), _unit(np.asarray(got, complex))
    d = g - r
    d2 = float(np.vdot(d, d).real)
    return max(0.0, d2 - d2 * d2 / 4.0)


def _no_quartic_term(ref, got):
    r, g = _unit(np.asarray(ref, complex)), _unit(np.asarray(got, complex))
    ov = np.vdot(r, g)
    d = g - (ov / abs(ov) if abs(ov) > 0 else 1.0) * r
    return max(0.0, float(np.vdot(d, d).real))


def _no_normalisation(ref, got):
    r, g = np.asarray(ref, complex), np.asarray(got, complex)
    ov = np.vdot(r, g)
    d = g - (ov / abs(ov) if abs(ov) > 0 else 1.0) * r
    d2 = float(np.vdot(d, d).real)
    return max(0.0, d2 - d2 * d2 / 4.0)


def _fid_no_normalisation(ref, got):
    return float(abs(np.vdot(ref, got)) ** 2)


@pytest.mark.parametrize("mutant", [_no_phase_removal, _no_quartic_term, _no_normalisation])
def test_planted_infidelity_mistakes_are_caught(oracle, mutant):
    assert metric_failures(mutant, oracle.fidelity) != []


def test_planted_fidelity_mistake_is_caught(oracle):
    assert metric_failures(oracle.infidelity, _fid_no_normalisation) != []


def test_fidelity_metrics_helper(oracle):
    """The helper the GPU tests call returns the oracle's 1 - F and the max
    per-amplitude error."""
    from conftest import fidelity_metrics
    ref = np.array([1.0, 0.0], complex)
    got = np.array([np.cos(1e-3), np.sin(1e-3)], complex)
    inf, mx = fidelity_metrics(ref, got)
    assert abs(inf - np.sin(1e-3) ** 2) <= 1e-14 * np.sin(1e-3) ** 2
    assert abs(mx - np.sin(1e-3)) < 1e-15
