"""sv_expect_z_all_noalloc: the <Z_q> reduction for callers that cannot
allocate device memory (graph capture, foreign allocators, allocation-free
loops).  Called through the C ABI on raw device pointers and compared with
sv_expect_z_all, which uses a state handle and its workspace.  Two calls in
a row share the library's fixed scratch array, so the second one also shows
that leftovers from the first do not leak into its result.

This file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def noalloc_z(N, st, stream):
    out = torch.full((st.n,), float("nan"), dtype=torch.float64, device=st.device)
    rc = N.lib().sv_expect_z_all_noalloc(C.c_void_p(st.amps.data_ptr()), st.n, st.dt,
                                         C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)),
                                         C.c_void_p(stream.cuda_stream))
    N.check(rc)
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dt,tol", [("c64", 1e-6), ("c128", 1e-12)])
def test_noalloc_matches_workspace_path(svlib, dt, tol):
    from paper_2106_13995_gb300 import _native as N
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(21)
    # two calls in a row: a large state (many blocks), then a smaller one
    for n in (22, 13):
        st = svlib.StateVector(n, dt).load(W.random_state(n, rng))
        st.apply_circuit(W.random_u3_cz(n, 2, n))
        want = st.z_all()
        got = noalloc_z(N, st, stream)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= tol, (n, np.max(np.abs(got - want)))
        st.close()


def test_noalloc_small_state_and_errors(svlib):
    from paper_2106_13995_gb300 import _native as N
    stream = torch.cuda.current_stream()
    st = svlib.StateVector(5, "c64").set_basis(0b10110)
    got = noalloc_z(N, st, stream)
    assert np.array_equal(got, np.array([1.0, -1.0, -1.0, 1.0, -1.0]))
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    op = C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double))
    assert N.lib().sv_expect_z_all_noalloc(C.c_void_p(st.amps.data_ptr()), 35, 0, op, None) == N.SV_EINVAL
    assert N.lib().sv_expect_z_all_noalloc(None, 5, 0, op, None) == N.SV_EINVAL
    assert N.lib().sv_expect_z_all_noalloc(C.c_void_p(st.amps.data_ptr() + 8), 5, 0, op, None) == N.SV_EINVAL
