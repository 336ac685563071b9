"""FP64 CPU oracle (ctypes wrapper around ``sv_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the GPU library never imports it.  It shares no code
with the CUDA path; the only thing both sides consume is the seeded circuit
descriptions of ``workloads``.

Every function states the definition it follows (paper Sec. I-A / Sec. II:
the state is the full vector of 2^n amplitudes and a circuit is the product
of its gate matrices applied to it).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Iterable, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    src_m = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sv_oracle.h")))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < src_m:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _OrOp(C.Structure):
    _fields_ = [("gate", C.c_int32), ("k", C.c_int32), ("nctrl", C.c_int32), ("param", C.c_int32),
                ("targets", C.c_int32 * 8), ("controls", C.c_int32 * 8),
                ("angles", C.c_double * 3), ("matrix", C.POINTER(C.c_double))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            up = C.POINTER(C.c_uint64)
            L.or_gate_id.argtypes = [C.c_char_p]
            L.or_gate_matrix.argtypes = [C.c_int, dp, dp]
            L.or_apply.argtypes = [dp, C.c_int, ip, C.c_int, ip, C.c_int, dp]
            L.or_full_matrix.argtypes = [C.c_int, ip, C.c_int, ip, C.c_int, dp, dp]
            L.or_matvec.argtypes = [C.c_int, dp, dp, dp]
            L.or_run.argtypes = [dp, C.c_int, C.POINTER(_OrOp), C.c_int, dp]
            L.or_expect.argtypes = [dp, C.c_int, up, up, dp, C.c_int]
            L.or_expect.restype = C.c_double
            L.or_apply_pauli_sum.argtypes = [dp, dp, C.c_int, up, up, dp, C.c_int]
            L.or_z_all.argtypes = [dp, C.c_int, dp]
            L.or_norm2.argtypes = [dp, C.c_int]
            L.or_norm2.restype = C.c_double
            L.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            L.or_splitmix64.restype = C.c_uint64
            L.or_sample.argtypes = [dp, C.c_int, C.c_int64, C.c_uint64, up]
            L.or_set_num_threads.argtypes = [C.c_int]
            L.or_adjoint_grad.argtypes = [dp, C.c_int, C.POINTER(_OrOp), C.c_int, dp, C.c_int,
                                          up, up, dp, C.c_int, dp, dp]
            _lib = L
    return _lib


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(t: int) -> None:
    """Thread count of later oracle calls (for timing on one core)."""
    lib().or_set_num_threads(int(t))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _up(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _as_state(psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return psi


def _nq(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.size != (1 << n):
        raise ValueError("state length must be a power of two")
    return n


# --- gates -----------------------------------------------------------------

def gate_matrix(name: str, angles: Sequence[float] = ()) -> np.ndarray:
    """Matrix of a named gate (see the per-gate readings in sv_oracle.c)."""
    g = lib().or_gate_id(name.encode())
    if g <= 0:
        raise ValueError(f"unknown named gate {name}")
    a = np.zeros(3)
    a[: len(angles)] = angles
    out = np.zeros(2 * 16)
    k = lib().or_gate_matrix(g, _dp(a), _dp(out))
    d = 1 << k
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def apply(psi: np.ndarray, U: np.ndarray, targets: Sequence[int], controls: Sequence[int] = ()) -> np.ndarray:
    """c-1 (i): in-place index-loop application; returns psi."""
    n = _nq(psi)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    t = np.asarray(targets, dtype=np.int32)
    c = np.asarray(list(controls) or [0], dtype=np.int32)
    lib().or_apply(_dp(psi.view(np.float64)), n, _ip(t), len(targets), _ip(c), len(controls),
                   _dp(U.view(np.float64)))
    return psi


def full_matrix(n: int, U: np.ndarray, targets: Sequence[int], controls: Sequence[int] = ()) -> np.ndarray:
    """c-1 (ii): the 2^n x 2^n matrix of one (controlled) gate."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    t = np.asarray(targets, dtype=np.int32)
    c = np.asarray(list(controls) or [0], dtype=np.int32)
    M = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    if lib().or_full_matrix(n, _ip(t), len(targets), _ip(c), len(controls), _dp(U.view(np.float64)),
                            _dp(M.view(np.float64))) != 0:
        raise ValueError("n too large for the full matrix")
    return M


def matvec(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    n = _nq(x)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    x = _as_state(x)
    y = np.zeros_like(x)
    lib().or_matvec(n, _dp(M.view(np.float64)), _dp(x.view(np.float64)), _dp(y.view(np.float64)))
    return y


# --- circuits ----------------------------------------------------------------

def _marshal(circ) -> Tuple[C.Array, list]:
    ops = (_OrOp * max(1, len(circ.ops)))()
    keep = []
    for i, op in enumerate(circ.ops):
        o = ops[i]
        g = lib().or_gate_id(op.name.encode())
        if g < 0:
            raise ValueError(f"unknown gate {op.name}")
        o.gate = g
        o.k = len(op.targets)
        o.nctrl = len(op.controls)
        o.param = op.param
        for j, q in enumerate(op.targets):
            o.targets[j] = q
        for j, q in enumerate(op.controls):
            o.controls[j] = q
        for j, a in enumerate(op.angles):
            o.angles[j] = a
        if op.name == "MATRIX":
            m = np.ascontiguousarray(op.matrix, dtype=np.complex128)
            keep.append(m)
            o.matrix = _dp(m.view(np.float64))
    return ops, keep


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def run(circ, psi: Optional[np.ndarray] = None, params: Optional[np.ndarray] = None) -> np.ndarray:
    """psi_out = U_G ... U_1 psi_in (|0...0> by default), complex128."""
    n = circ.n_qubits
    psi = zero_state(n) if psi is None else _as_state(psi).copy()
    if psi.size != (1 << n):
        raise ValueError("state size does not match the circuit")
    ops, keep = _marshal(circ)
    p = np.ascontiguousarray(params if params is not None else np.zeros(1), dtype=np.float64)
    if lib().or_run(_dp(psi.view(np.float64)), n, ops, len(circ.ops), _dp(p)) != 0:
        raise ValueError("malformed circuit")
    return psi


def run_inplace(circ, psi: np.ndarray, params: Optional[np.ndarray] = None) -> np.ndarray:
    """Same as run() but updates the caller's complex128 array in place."""
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.size != (1 << circ.n_qubits):
        raise ValueError("psi must be a contiguous complex128 array of 2^n entries")
    ops, keep = _marshal(circ)
    p = np.ascontiguousarray(params if params is not None else np.zeros(1), dtype=np.float64)
    if lib().or_run(_dp(psi.view(np.float64)), circ.n_qubits, ops, len(circ.ops), _dp(p)) != 0:
        raise ValueError("malformed circuit")
    return psi


# --- observables ---------------------------------------------------------------

def _terms(terms: Iterable[Tuple[int, int, float]]):
    terms = list(terms)
    xm = np.array([t[0] for t in terms] or [0], dtype=np.uint64)
    zm = np.array([t[1] for t in terms] or [0], dtype=np.uint64)
    cf = np.array([t[2] for t in terms] or [0.0], dtype=np.float64)
    return xm, zm, cf, len(terms)


def expect(psi: np.ndarray, terms) -> float:
    """sum_t c_t Re <psi| P_t |psi> for Pauli strings (x_mask, z_mask, c)."""
    psi = _as_state(psi)
    xm, zm, cf, nt = _terms(terms)
    return lib().or_expect(_dp(psi.view(np.float64)), _nq(psi), _up(xm), _up(zm), _dp(cf), nt)


def apply_pauli_sum(psi: np.ndarray, terms) -> np.ndarray:
    psi = _as_state(psi)
    out = np.zeros_like(psi)
    xm, zm, cf, nt = _terms(terms)
    lib().or_apply_pauli_sum(_dp(psi.view(np.float64)), _dp(out.view(np.float64)), _nq(psi),
                             _up(xm), _up(zm), _dp(cf), nt)
    return out


def z_all(psi: np.ndarray) -> np.ndarray:
    """<Z_q> = sum_x |psi_x|^2 (1 - 2 bit_q(x)) for every qubit q."""
    psi = _as_state(psi)
    n = _nq(psi)
    out = np.zeros(n)
    lib().or_z_all(_dp(psi.view(np.float64)), n, _dp(out))
    return out


def norm2(psi: np.ndarray) -> float:
    psi = _as_state(psi)
    return lib().or_norm2(_dp(psi.view(np.float64)), _nq(psi))


def splitmix64(seed: int, s: int) -> int:
    return int(lib().or_splitmix64(seed & (2**64 - 1), s))


def sample(psi: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Inverse-CDF sampling, u_s = (SplitMix64(seed, s) >> 11) 2^-53."""
    psi = _as_state(psi)
    out = np.zeros(max(1, shots), dtype=np.uint64)
    lib().or_sample(_dp(psi.view(np.float64)), _nq(psi), shots, seed & (2**64 - 1), _up(out))
    return out[:shots]


def adjoint_grad(circ, params: np.ndarray, terms, psi: Optional[np.ndarray] = None):
    """Adjoint-method gradient of <H> at params.  Returns (expval, grad, psi_out)."""
    n = circ.n_qubits
    psi = zero_state(n) if psi is None else _as_state(psi).copy()
    ops, keep = _marshal(circ)
    p = np.ascontiguousarray(params, dtype=np.float64)
    xm, zm, cf, nt = _terms(terms)
    ev = np.zeros(1)
    g = np.zeros(max(1, circ.n_params))
    rc = lib().or_adjoint_grad(_dp(psi.view(np.float64)), n, ops, len(circ.ops), _dp(p), circ.n_params,
                               _up(xm), _up(zm), _dp(cf), nt, _dp(ev), _dp(g))
    if rc != 0:
        raise ValueError(f"oracle adjoint failed ({rc})")
    return float(ev[0]), g[: circ.n_params], psi


# --- comparison metrics ----------------------------------------------------------

def fidelity(ref: np.ndarray, got: np.ndarray) -> float:
    """F = |<ref|got>|^2 / (||ref||^2 ||got||^2), in FP64."""
    ref = np.asarray(ref, dtype=np.complex128)
    got = np.asarray(got, dtype=np.complex128)
    ov = np.vdot(ref, got)
    return float(abs(ov) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real))


def infidelity(ref: np.ndarray, got: np.ndarray) -> float:
    """1 - F without cancellation: normalise both, remove the relative global
    phase, then 1 - F = ||d||^2 - ||d||^4 / 4 for d = got - e^{i a} ref."""
    ref = np.asarray(ref, dtype=np.complex128)
    got = np.asarray(got, dtype=np.complex128)
    r = ref / np.sqrt(np.vdot(ref, ref).real)
    g = got / np.sqrt(np.vdot(got, got).real)
    ov = np.vdot(r, g)
    ph = ov / abs(ov) if abs(ov) > 0 else 1.0
    d = g - ph * r
    d2 = float(np.vdot(d, d).real)
    return max(0.0, d2 - d2 * d2 / 4.0)


def max_abs_err(ref: np.ndarray, got: np.ndarray) -> float:
    return float(np.max(np.abs(np.asarray(got, dtype=np.complex128) - np.asarray(ref, dtype=np.complex128))))
