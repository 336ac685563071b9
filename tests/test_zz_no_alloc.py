"""sv_expect_z_all_noalloc: the <Z_q> reduction for callers that cannot
allocate device memory (graph capture, foreign allocators, allocation-free
loops).  Called through the C ABI on raw device pointers and compared with
the FP64 oracle's <Z_q> and with sv_expect_z_all, which uses a state handle
and its workspace.  Calls in a row share the library's fixed scratch array,
so each later call also shows that leftovers from the one before do not leak
into its result.  The same call recorded in a CUDA graph and replayed must
give the same values.  (States above 32 qubits, which take a second branch
of the reduction kernel, are run by the 33- and 34-qubit GHZ tests.)

This file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _out_ptr(out):
    return C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double))


def noalloc_z(N, st, stream):
    out = torch.full((st.n,), float("nan"), dtype=torch.float64, device=st.device)
    rc = N.lib().sv_expect_z_all_noalloc(C.c_void_p(st.amps.data_ptr()), st.n, st.dt, _out_ptr(out),
                                         C.c_void_p(stream.cuda_stream))
    N.check(rc)
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dt,tol", [("c64", 1e-6), ("c128", 1e-12)])
def test_noalloc_matches_oracle_and_workspace_path(svlib, oracle, dt, tol):
    from paper_2106_13995_gb300 import _native as N
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(21)
    # calls in a row: a large state (many blocks), a middle one, a small one
    for n in (22, 13, 5):
        psi0 = W.random_state(n, rng)
        circ = W.random_u3_cz(n, 2, n)
        want = oracle.z_all(oracle.run(circ, psi0))
        st = svlib.StateVector(n, dt).load(psi0)
        st.apply_circuit(circ)
        got = noalloc_z(N, st, stream)
        assert np.all(np.isfinite(got))
        err = float(np.max(np.abs(got - want)))
        print(f"n={n} {dt}: max |<Z> - oracle| = {err:.2e}")
        assert err <= tol, (n, err)
        assert np.max(np.abs(got - st.z_all())) <= tol
        st.close()


def test_noalloc_small_state_and_errors(svlib):
    from paper_2106_13995_gb300 import _native as N
    stream = torch.cuda.current_stream()
    st = svlib.StateVector(5, "c64").set_basis(0b10110)
    got = noalloc_z(N, st, stream)
    assert np.array_equal(got, np.array([1.0, -1.0, -1.0, 1.0, -1.0]))
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    op = _out_ptr(out)
    amps = C.c_void_p(st.amps.data_ptr())
    assert N.lib().sv_expect_z_all_noalloc(amps, 35, 0, op, None) == N.SV_EINVAL
    assert N.lib().sv_expect_z_all_noalloc(None, 5, 0, op, None) == N.SV_EINVAL
    assert N.lib().sv_expect_z_all_noalloc(C.c_void_p(st.amps.data_ptr() + 8), 5, 0, op, None) == N.SV_EINVAL
    # host memory is rejected before anything is launched
    host_amps = torch.zeros(64, dtype=torch.float32).pin_memory()
    host_out = torch.zeros(8, dtype=torch.float64).pin_memory()
    assert N.lib().sv_expect_z_all_noalloc(C.c_void_p(host_amps.data_ptr()), 5, 0, op, None) == N.SV_EINVAL
    assert N.lib().sv_expect_z_all_noalloc(amps, 5, 0, _out_ptr(host_out), None) == N.SV_EINVAL


def test_noalloc_in_cuda_graph(svlib, oracle):
    """Recorded once under stream capture (after a first call has done the
    per-device set-up), then replayed: the replays read the state as it is
    at replay time."""
    from paper_2106_13995_gb300 import _native as N
    n = 14
    rng = np.random.default_rng(5)
    psi_a, psi_b = W.random_state(n, rng), W.random_state(n, rng)
    st = svlib.StateVector(n, "c64").load(psi_a)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    noalloc_z(N, st, torch.cuda.current_stream())   # set-up outside capture
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        rc = N.lib().sv_expect_z_all_noalloc(C.c_void_p(st.amps.data_ptr()), n, N.SV_C64, _out_ptr(out),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(rc)
    for psi in (psi_a, psi_b, psi_a):
        st.load(psi)
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        want = oracle.z_all(np.asarray(psi, dtype=np.complex64).astype(np.complex128))
        assert np.max(np.abs(out.cpu().numpy() - want)) <= 1e-6
