"""Host-side checks of the C ABI that need no GPU: the library builds,
loads, and exports every entry point declared in include/sv_api.h."""
import ctypes as C

import pytest

import paper_2106_13995_gb300 as P
from paper_2106_13995_gb300 import _native as N


@pytest.fixture(scope="module")
def lib():
    P.build()
    return N.lib()


def test_exports_every_declared_symbol(lib):
    names = N.declared_symbols()
    assert len(names) >= 20
    missing = [s for s in names if not hasattr(lib, s)]
    assert missing == []


def test_workspace_sizes(lib):
    assert lib.sv_workspace_bytes(0, 0) == 0
    assert lib.sv_workspace_bytes(35, 0) == 0
    w20, w30 = lib.sv_workspace_bytes(20, 0), lib.sv_workspace_bytes(30, 0)
    assert 0 < w20 <= w30
    assert w30 >= (1 << 20) * 8          # CDF chunk sums for 2^30 amplitudes


def test_argument_errors_without_gpu(lib):
    h = C.c_void_p()
    assert lib.sv_create(0, 0, None, 0, None, 0, None, C.byref(h)) == N.SV_EINVAL
    assert b"n_qubits" in lib.sv_last_error()
    assert lib.sv_create(10, 7, None, 0, None, 0, None, C.byref(h)) == N.SV_EINVAL
    assert lib.sv_create(10, 0, None, 0, None, 0, None, C.byref(h)) == N.SV_EINVAL
    assert lib.sv_set_basis(None, 0) == N.SV_EINVAL
    assert lib.sv_destroy(None) == N.SV_OK
    assert lib.sv_status_string(4) == b"SV_ETIMEOUT"


def test_gate_table_matches_header():
    hdr = open(N.__file__.replace("paper_2106_13995_gb300/_native.py", "include/sv_api.h")).read()
    for name, gid in N.GATE_IDS.items():
        tok = "SV_GATE_ID" if name == "I" else f"SV_GATE_{name}"
        assert tok in hdr, name


def test_marshal_layout():
    import workloads as W
    from paper_2106_13995_gb300 import sim
    m = sim.marshal(W.random_gate_circuit(5, 30, seed=1))
    assert C.sizeof(N.SvOp) == 104          # matches static_assert in sv_api.cu
    assert m.c.n_ops == 30
