"""Host <-> device moves of the whole state (sv_upload / sv_download): from
and to pageable numpy arrays (cudaMemcpyAsync), page-locked buffers (a copy
kernel reading and writing them over the GPU's host link) and page-locked
buffers off 16-byte alignment (cudaMemcpyAsync again).  Every route must
move the amplitudes bit for bit; the kernel route is the one that launches
a kernel."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _pinned(nbytes, offset):
    buf = torch.zeros(nbytes + 64, dtype=torch.uint8).pin_memory()
    return buf, buf.data_ptr() + offset


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 3, 12, 20])
def test_upload_download_routes(svlib, dt, n):
    from paper_2106_13995_gb300 import _native as N
    rng = np.random.default_rng(100 + n)
    want = W.random_state(n, rng).astype(np.complex64 if dt == "c64" else np.complex128)
    nbytes = want.nbytes
    st = svlib.StateVector(n, dt)
    lib = N.lib()
    for route, offset in (("pageable", None), ("pinned", 0), ("pinned+8", 8)):
        # upload
        if offset is None:
            src_keep, src = want, want.ctypes.data
        else:
            src_keep, src = _pinned(nbytes, offset)
            C.memmove(src, want.ctypes.data, nbytes)
        l0 = lib.sv_kernel_launch_count()
        N.check(lib.sv_upload(st.h, C.c_void_p(src), nbytes))
        launched = lib.sv_kernel_launch_count() - l0
        assert launched == (1 if route == "pinned" else 0), (route, launched)
        got = st.numpy()
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (route, "upload")
        # download
        if offset is None:
            out = np.zeros_like(want)
            N.check(lib.sv_download(st.h, C.c_void_p(out.ctypes.data), nbytes))
        else:
            dst_keep, dst = _pinned(nbytes, offset)
            N.check(lib.sv_download(st.h, C.c_void_p(dst), nbytes))
            out = np.zeros_like(want)
            C.memmove(out.ctypes.data, dst, nbytes)
        assert np.array_equal(out.view(np.uint8), want.view(np.uint8)), (route, "download")
        del src_keep
    # the size must match the state
    pin, p = _pinned(nbytes, 0)
    assert lib.sv_upload(st.h, C.c_void_p(p), nbytes - 16) == N.SV_EINVAL
    assert lib.sv_download(st.h, C.c_void_p(p), nbytes + 16) == N.SV_EINVAL
    st.close()
