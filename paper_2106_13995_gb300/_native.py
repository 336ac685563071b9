"""ctypes binding of libsv.so: the C ABI declared in include/sv_api.h.

Argument marshalling only -- every computation happens inside the library's
CUDA kernels.  Loading fails loudly if the library has not been built; there
is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsv.so")

SV_OK, SV_EINVAL, SV_ENOMEM, SV_ECUDA, SV_ETIMEOUT, SV_EUNSUPPORTED = range(6)
SV_C64, SV_C128 = 0, 1
SV_PREC_PLAIN, SV_PREC_TC_BF16X3, SV_PREC_TC_TF32X3 = 0, 1, 2
SV_MODE_TILED, SV_MODE_PER_GATE, SV_MODE_TILED_GRAPH = 0, 1, 2

GATE_IDS = {
    "MATRIX": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8,
    "SX": 9, "SY": 10, "SW": 11, "I": 12,
    "RX": 20, "RY": 21, "RZ": 22, "PHASE": 23, "U3": 30,
    "CZ": 40, "SWAP": 41, "FSIM": 50,
}


class SvOp(C.Structure):
    _fields_ = [("gate", C.c_int32), ("n_targets", C.c_int32), ("n_controls", C.c_int32),
                ("param", C.c_int32), ("targets", C.c_int32 * 6), ("controls", C.c_int32 * 8),
                ("angles", C.c_double * 3), ("matrix_offset", C.c_int64)]


class SvCircuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_ops", C.c_int32), ("n_params", C.c_int32),
                ("reserved", C.c_int32), ("ops", C.POINTER(SvOp)), ("matrices", C.POINTER(C.c_double))]


class SvOptions(C.Structure):
    _fields_ = [("fusion_k", C.c_int32), ("tile_m", C.c_int32), ("prec", C.c_int32),
                ("mode", C.c_int32), ("timeout_cycles", C.c_uint64)]


class SvPauliTerm(C.Structure):
    _fields_ = [("x_mask", C.c_uint64), ("z_mask", C.c_uint64), ("coeff", C.c_double)]


class SvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "SV_OK", 1: "SV_EINVAL", 2: "SV_ENOMEM", 3: "SV_ECUDA", 4: "SV_ETIMEOUT", 5: "SV_EUNSUPPORTED"}
_lib = None
_lock = threading.Lock()


def lib():
    """Load libsv.so (built by ``paper_2106_13995_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2106_13995_gb300.build.build() first "
                               "(the GPU library has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, dp, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
        i32p, u64p = C.POINTER(C.c_int32), C.POINTER(C.c_uint64)
        st = C.c_int
        proto = {
            "sv_workspace_bytes": (sz, [C.c_int, C.c_int]),
            "sv_create": (st, [C.c_int, C.c_int, vp, sz, vp, sz, vp, C.POINTER(vp)]),
            "sv_destroy": (st, [vp]),
            "sv_set_basis": (st, [vp, C.c_uint64]),
            "sv_mark_modified": (st, [vp]),
            "sv_upload": (st, [vp, vp, sz]),
            "sv_download": (st, [vp, vp, sz]),
            "sv_synchronize": (st, [vp]),
            "sv_apply_gate": (st, [vp, i32p, C.c_int, i32p, C.c_int, dp, C.c_int]),
            "sv_apply_circuit": (st, [vp, C.POINTER(SvCircuit), dp, C.POINTER(SvOptions)]),
            "sv_plan_info": (st, [vp, C.POINTER(SvCircuit), dp, C.POINTER(SvOptions), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
            "sv_plan_fmas": (st, [vp, C.POINTER(SvCircuit), dp, C.POINTER(SvOptions), dp]),
            "sv_apply_circuit_batch": (st, [C.POINTER(vp), C.c_int, C.POINTER(C.POINTER(SvCircuit)),
                                            C.POINTER(dp), C.POINTER(SvOptions)]),
            "sv_expect": (st, [vp, C.POINTER(SvPauliTerm), C.c_int, dp]),
            "sv_expect_z_all": (st, [vp, dp]),
            "sv_expect_z_all_noalloc": (st, [vp, C.c_int, C.c_int, dp, vp]),
            "sv_norm": (st, [vp, dp]),
            "sv_renormalize": (st, [vp, dp]),
            "sv_sample": (st, [vp, C.c_int64, C.c_uint64, u64p]),
            "sv_adjoint_grad": (st, [vp, vp, C.POINTER(SvCircuit), dp, C.POINTER(SvPauliTerm), C.c_int,
                                     C.POINTER(SvOptions), dp, dp]),
            "sv_adjoint_grad_batch": (st, [C.POINTER(vp), C.POINTER(vp), C.c_int, C.POINTER(SvCircuit), dp,
                                           C.POINTER(SvPauliTerm), C.c_int, C.POINTER(SvOptions), dp, dp]),
            "sv_autotune": (st, [vp, C.POINTER(SvCircuit), C.POINTER(SvOptions)]),
            "sv_wait_selftest": (st, [vp, C.c_uint64]),
            "sv_kernel_launch_count": (C.c_uint64, []),
            "sv_program_cache_limit": (C.c_int64, [C.c_int64]),
            "sv_last_error": (C.c_char_p, []),
            "sv_status_string": (C.c_char_p, [C.c_int]),
        }
        for name, (res, args) in proto.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def check(status: int) -> None:
    if status != SV_OK:
        raise SvError(status, lib().sv_last_error().decode(errors="replace"))


def declared_symbols():
    """Function names declared in include/sv_api.h."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "sv_api.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(sv_[a-z_0-9]+)\s*\(", text, re.M)))
