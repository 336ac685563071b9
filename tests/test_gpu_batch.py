"""Batched execution of uneven circuits in one persistent launch (plain and
CUDA-graph replay), the autotuner, and the bounded device wait."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from conftest import fidelity_metrics

pytestmark = pytest.mark.gpu


def batch_apply(svlib, states, circs, opts=None, params=None):
    from paper_2106_13995_gb300 import _native as N
    ms = [svlib.marshal(c) for c in circs]
    B = len(states)
    hs = (C.c_void_p * B)(*[s.h.value for s in states])
    cs = (C.POINTER(N.SvCircuit) * B)(*[C.pointer(m.c) for m in ms])
    N.check(N.lib().sv_apply_circuit_batch(hs, B, cs, None, C.byref(opts) if opts else None))
    N.check(N.lib().sv_synchronize(states[0].h))
    return ms


def small_uneven(count, nmin, nmax, depth, seed):
    return W.uneven_batch(count=count, nmin=nmin, nmax=nmax, depth=depth, seed=seed)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_persistent_batch_matches_per_circuit_and_oracle(svlib, oracle, dt):
    circs = small_uneven(24, 6, 18, 8, seed=7)
    states = [svlib.StateVector(c.n_qubits, dt).set_basis(0) for c in circs]
    batch_apply(svlib, states, circs)
    for c, s in zip(circs, states):
        got = s.numpy()
        ref = svlib.StateVector(c.n_qubits, dt).set_basis(0).apply_circuit(c).numpy()
        assert np.array_equal(got, ref), c.name          # same programs, same arithmetic
        inf, _ = fidelity_metrics(oracle.run(c), got)
        assert inf <= (1e-5 if dt == "c64" else 1e-12), (c.name, inf)


def test_graph_replay(svlib):
    from paper_2106_13995_gb300 import _native as N
    circs = small_uneven(12, 8, 20, 6, seed=3)
    states = [svlib.StateVector(c.n_qubits, "c64") for c in circs]
    opts = svlib.options(mode=N.SV_MODE_TILED_GRAPH)
    outs = []
    for rep in range(3):
        for s in states:
            s.set_basis(0)
        batch_apply(svlib, states, circs, opts)
        outs.append([s.numpy() for s in states])
    for rep in (1, 2):
        for a, b in zip(outs[0], outs[rep]):
            assert np.array_equal(a, b)
    for c, s, got in zip(circs, states, outs[0]):
        ref = svlib.StateVector(c.n_qubits, "c64").set_basis(0).apply_circuit(c).numpy()
        assert np.array_equal(got, ref)


def test_uneven_256_full_size(svlib, oracle):
    """256 circuits, widths 10..24, depth 40, one persistent launch; every
    state equals its per-circuit run; a seeded subset is checked against the
    FP64 oracle (all widths <= 14 and two wider circuits)."""
    circs = W.uneven_batch()
    states = [svlib.StateVector(c.n_qubits, "c64").set_basis(0) for c in circs]
    batch_apply(svlib, states, circs)
    rng = np.random.default_rng(0)
    wide = [i for i, c in enumerate(circs) if c.n_qubits >= 20]
    check = [i for i, c in enumerate(circs) if c.n_qubits <= 14][:24] + list(rng.choice(wide, 2, replace=False))
    worst = 0.0
    for i in range(len(circs)):
        c, s = circs[i], states[i]
        if c.n_qubits <= 16 or i in check:
            got = s.numpy()
            ref = svlib.StateVector(c.n_qubits, "c64").set_basis(0).apply_circuit(c).numpy()
            assert np.array_equal(got, ref), c.name
            if i in check:
                inf, _ = fidelity_metrics(oracle.run(c), got)
                worst = max(worst, inf)
                assert inf <= 1e-5, (c.name, inf)
        s.close()
    print(f"uneven batch: worst 1-F {worst:.2e}")


def test_autotune_then_use(svlib, oracle):
    c = W.random_u3_cz(16, 10, 5)
    scratch = svlib.StateVector(16, "c64")
    from paper_2106_13995_gb300 import _native as N
    o = svlib.options()
    N.check(N.lib().sv_autotune(scratch.h, svlib.marshal(c).ref(), C.byref(o)))
    assert 2 <= o.fusion_k <= 6 and 10 <= o.tile_m <= 16
    s = svlib.StateVector(16, "c64").set_basis(0).apply_circuit(c)    # uses the tuned choice
    inf, _ = fidelity_metrics(oracle.run(c), s.numpy())
    assert inf <= 1e-5


def test_bounded_wait_times_out_and_context_survives(svlib):
    from paper_2106_13995_gb300 import _native as N
    st = torch.cuda.current_stream()
    rc = N.lib().sv_wait_selftest(C.c_void_p(st.cuda_stream), 2000)
    assert rc == N.SV_ETIMEOUT
    assert b"ran out" in N.lib().sv_last_error()
    # the context is still usable
    s = svlib.StateVector(10, "c64").set_basis(3)
    assert s.numpy()[3] == 1


def test_batch_timeout_reports_status(svlib):
    """A one-poll budget makes dependent waits run out; the launch stops and
    sv_synchronize reports SV_ETIMEOUT (or SV_OK if every wait happened to be
    satisfied at the first poll); afterwards the states work normally."""
    from paper_2106_13995_gb300 import _native as N
    circs = [W.random_u3_cz(22, 6, 1), W.random_u3_cz(21, 6, 2)]
    states = [svlib.StateVector(c.n_qubits, "c64").set_basis(0) for c in circs]
    ms = [svlib.marshal(c) for c in circs]
    hs = (C.c_void_p * 2)(*[s.h.value for s in states])
    cs = (C.POINTER(N.SvCircuit) * 2)(*[C.pointer(m.c) for m in ms])
    o = svlib.options(timeout_cycles=1)
    N.check(N.lib().sv_apply_circuit_batch(hs, 2, cs, None, C.byref(o)))
    rc = N.lib().sv_synchronize(states[0].h)
    assert rc in (N.SV_OK, N.SV_ETIMEOUT)
    assert N.lib().sv_synchronize(states[0].h) == N.SV_OK       # flag cleared
    for c, s in zip(circs, states):
        s.set_basis(0)
    batch_apply(svlib, states, circs)
    for c, s in zip(circs, states):
        ref = svlib.StateVector(c.n_qubits, "c64").set_basis(0).apply_circuit(c).numpy()
        assert np.array_equal(s.numpy(), ref)


def test_autotune_cache_leaves_tensor_core_modes_alone(svlib, oracle):
    """A CUDA-core tuning in the cache must not change what a tensor-core
    mode plans: the BF16 mode plans the same blocks as on a state with no
    tuning cached, and its result differs from the CUDA-core one only by
    split-BF16 rounding."""
    from paper_2106_13995_gb300 import _native as N
    c = W.random_u3_cz(16, 12, 9)
    m = svlib.marshal(c)
    s = svlib.StateVector(16, "c64")
    o = svlib.options()
    N.check(N.lib().sv_autotune(s.h, m.ref(), C.byref(o)))
    tc = svlib.options(prec=N.SV_PREC_TC_BF16X3)
    nb_tc, np_tc = s.plan_info(m, opts=tc)
    fresh = svlib.StateVector(16, "c64")
    assert (nb_tc, np_tc) == fresh.plan_info(m, opts=tc), o.fusion_k
    fresh.close()
    a = s.set_basis(0).apply_circuit(m).numpy()
    b = s.set_basis(0).apply_circuit(m, opts=tc).numpy()
    assert not np.array_equal(a, b)
    inf, _ = fidelity_metrics(oracle.run(c), b)
    assert inf <= 1e-5


@pytest.mark.parametrize("prec", [1, 2])
def test_uneven_circuits_tensor_core_modes(svlib, oracle, prec):
    """Per-circuit tensor-core modes on uneven widths (12..16 qubits) against
    the FP64 oracle."""
    circs = small_uneven(6, 12, 16, 12, seed=11)
    for c in circs:
        s = svlib.StateVector(c.n_qubits, "c64").set_basis(0).apply_circuit(c, opts=svlib.options(prec=prec))
        inf, _ = fidelity_metrics(oracle.run(c), s.numpy())
        assert inf <= 1e-5, (c.name, prec, inf)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_with_wide_states_on_forked_streams(svlib, oracle, prec):
    """One graph-recorded batched call over narrow states (the persistent
    queue) and several wide ones (full-grid passes spread over the library's
    forked streams; with split-BF16 the pipelined tensor-core passes), played
    twice: the narrow states match the FP64 oracle, and every state matches
    its own single-circuit run bit for bit (the kernels are deterministic,
    whatever stream runs them)."""
    from paper_2106_13995_gb300 import _native as N
    narrow = small_uneven(6, 10, 15, 12, seed=21)
    wide = small_uneven(5, 21, 22, 8, seed=22)
    circs = narrow + wide
    opts = svlib.options(prec=prec, mode=N.SV_MODE_TILED_GRAPH)
    single = svlib.options(prec=prec)
    want = []
    for c in circs:
        s = svlib.StateVector(c.n_qubits, "c64").set_basis(0).apply_circuit(c, opts=single)
        want.append(s.numpy())
        s.close()
    states = [svlib.StateVector(c.n_qubits, "c64") for c in circs]
    for rep in range(2):
        for st in states:
            st.set_basis(0)
        batch_apply(svlib, states, circs, opts)
        for i, (c, st) in enumerate(zip(circs, states)):
            got = st.numpy()
            assert np.array_equal(got, want[i]), (rep, c.name)
            if c.n_qubits <= 15:
                inf, _ = fidelity_metrics(oracle.run(c), got)
                assert inf <= (1e-5 if prec else 1e-9), (c.name, inf)
    for st in states:
        st.close()


@pytest.mark.parametrize("graph", [False, True])
def test_batch_beyond_program_cache_bound(svlib, graph):
    """A batch of more distinct circuits than the program cache holds: the
    cache evicts entries while the call still uses them, and the results
    stay bit-identical to one call per circuit."""
    from paper_2106_13995_gb300 import _native as N
    circs = [W.random_u3_cz(10, 3, seed) for seed in range(40)]
    old = N.lib().sv_program_cache_limit(8)
    try:
        states = [svlib.StateVector(10, "c64").set_basis(0) for _ in circs]
        opts = svlib.options(mode=N.SV_MODE_TILED_GRAPH) if graph else None
        for rep in range(2 if graph else 1):
            for s in states:
                s.set_basis(0)
            batch_apply(svlib, states, circs, opts)
        for c, s in zip(circs, states):
            ref = svlib.StateVector(10, "c64").set_basis(0).apply_circuit(c).numpy()
            assert np.array_equal(s.numpy(), ref), c.name
    finally:
        N.lib().sv_program_cache_limit(old)
