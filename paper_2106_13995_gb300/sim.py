"""User-facing wrapper over the C ABI.

PyTorch supplies device memory and the CUDA stream; every amplitude update,
reduction and gradient runs inside libsv.so.
"""
from __future__ import annotations

import ctypes as C
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _native as N


def _dtype_code(dtype) -> int:
    if dtype in ("c64", "complex64", torch.complex64, N.SV_C64):
        return N.SV_C64
    if dtype in ("c128", "complex128", torch.complex128, N.SV_C128):
        return N.SV_C128
    raise ValueError(f"unsupported dtype {dtype}")


def options(fusion_k: int = 0, tile_m: int = 0, prec: int = N.SV_PREC_PLAIN, mode: int = N.SV_MODE_TILED,
            timeout_cycles: int = 0) -> N.SvOptions:
    return N.SvOptions(fusion_k, tile_m, prec, mode, timeout_cycles)


class Marshalled:
    """A circuit laid out as the C ABI's sv_circuit (keeps its buffers alive)."""

    def __init__(self, circ):
        ops = (N.SvOp * max(1, len(circ.ops)))()
        mats: List[np.ndarray] = []
        moff = 0
        for i, op in enumerate(circ.ops):
            o = ops[i]
            o.gate = N.GATE_IDS[op.name]
            o.n_targets = len(op.targets)
            o.n_controls = len(op.controls)
            o.param = op.param
            for j, q in enumerate(op.targets):
                o.targets[j] = q
            for j, q in enumerate(op.controls):
                o.controls[j] = q
            for j, a in enumerate(op.angles):
                o.angles[j] = a
            o.matrix_offset = -1
            if op.name == "MATRIX":
                m = np.ascontiguousarray(op.matrix, dtype=np.complex128).reshape(-1)
                o.matrix_offset = moff
                moff += m.size
                mats.append(m)
        self.matrices = np.concatenate(mats) if mats else np.zeros(1, dtype=np.complex128)
        self.ops = ops
        self.n_qubits = circ.n_qubits
        self.n_params = circ.n_params
        self.n_ops = len(circ.ops)
        self.c = N.SvCircuit(circ.n_qubits, len(circ.ops), circ.n_params, 0, ops,
                             self.matrices.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)))

    def ref(self):
        return C.byref(self.c)


def marshal(circ) -> Marshalled:
    return circ if isinstance(circ, Marshalled) else Marshalled(circ)


def pauli_terms(terms: Iterable[Tuple[int, int, float]]):
    terms = list(terms)
    arr = (N.SvPauliTerm * max(1, len(terms)))()
    for i, (xm, zm, c) in enumerate(terms):
        arr[i] = N.SvPauliTerm(xm, zm, c)
    return arr, len(terms)


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


class StateVector:
    """2^n amplitudes in a torch CUDA tensor, wrapped by a libsv state handle."""

    def __init__(self, n: int, dtype="c64", device=None, stream: Optional[torch.cuda.Stream] = None):
        self.n = n
        self.dt = _dtype_code(dtype)
        self.device = torch.device(device if device is not None else "cuda")
        real = torch.float32 if self.dt == N.SV_C64 else torch.float64
        self.amps = torch.empty(2 << n, dtype=real, device=self.device)
        ws = N.lib().sv_workspace_bytes(n, self.dt)
        if ws == 0:
            raise ValueError("unsupported qubit count")
        self.ws = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        N.check(N.lib().sv_create(n, self.dt, self.amps.data_ptr(), self.amps.numel() * self.amps.element_size(),
                                  self.ws.data_ptr(), ws, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            N.lib().sv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbytes(self) -> int:
        return (1 << self.n) * (8 if self.dt == N.SV_C64 else 16)

    # -- state ------------------------------------------------------------
    def set_basis(self, index: int = 0):
        N.check(N.lib().sv_set_basis(self.h, index))
        return self

    def load(self, psi: np.ndarray):
        want = np.complex64 if self.dt == N.SV_C64 else np.complex128
        a = np.ascontiguousarray(psi, dtype=want)
        N.check(N.lib().sv_upload(self.h, a.ctypes.data, a.nbytes))
        return self

    def numpy(self) -> np.ndarray:
        want = np.complex64 if self.dt == N.SV_C64 else np.complex128
        out = np.empty(1 << self.n, dtype=want)
        N.check(N.lib().sv_download(self.h, out.ctypes.data, out.nbytes))
        return out

    def synchronize(self):
        N.check(N.lib().sv_synchronize(self.h))

    # -- gates ------------------------------------------------------------
    def apply_gate(self, U: np.ndarray, targets: Sequence[int], controls: Sequence[int] = (), adjoint=False):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        t = (C.c_int32 * 6)(*targets)
        c = (C.c_int32 * 8)(*controls)
        N.check(N.lib().sv_apply_gate(self.h, t, len(targets), c, len(controls),
                                      U.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)), int(adjoint)))
        return self

    def apply_circuit(self, circ, params: Optional[np.ndarray] = None, opts: Optional[N.SvOptions] = None):
        m = marshal(circ)
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
        N.check(N.lib().sv_apply_circuit(self.h, m.ref(), _dptr(p), C.byref(opts) if opts else None))
        return self

    def plan_info(self, circ, params: Optional[np.ndarray] = None, opts: Optional[N.SvOptions] = None):
        """(fused blocks, tile passes) the library plans for this circuit."""
        m = marshal(circ)
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
        nb, npass = C.c_int64(), C.c_int64()
        N.check(N.lib().sv_plan_info(self.h, m.ref(), _dptr(p), C.byref(opts) if opts else None,
                                     C.byref(nb), C.byref(npass)))
        return nb.value, npass.value

    def plan_fmas(self, circ, params: Optional[np.ndarray] = None, opts: Optional[N.SvOptions] = None) -> float:
        """Real multiply-adds per amplitude of the planned blocks."""
        m = marshal(circ)
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
        f = C.c_double()
        N.check(N.lib().sv_plan_fmas(self.h, m.ref(), _dptr(p), C.byref(opts) if opts else None, C.byref(f)))
        return f.value

    # -- observables ---------------------------------------------------------
    def expect(self, terms) -> float:
        arr, nt = pauli_terms(terms)
        out = C.c_double()
        N.check(N.lib().sv_expect(self.h, arr, nt, C.byref(out)))
        return out.value

    def z_all(self) -> np.ndarray:
        out = np.zeros(self.n)
        N.check(N.lib().sv_expect_z_all(self.h, _dptr(out)))
        return out

    def norm2(self) -> float:
        out = C.c_double()
        N.check(N.lib().sv_norm(self.h, C.byref(out)))
        return out.value

    def renormalize(self) -> float:
        out = C.c_double()
        N.check(N.lib().sv_renormalize(self.h, C.byref(out)))
        return out.value

    def sample(self, shots: int, seed: int) -> np.ndarray:
        out = np.zeros(max(1, shots), dtype=np.uint64)
        N.check(N.lib().sv_sample(self.h, shots, seed & (2**64 - 1),
                                  out.ctypes.data_as(C.POINTER(C.c_uint64))))
        return out[:shots]


def adjoint_grad(psi: StateVector, lam: StateVector, circ, params: np.ndarray, terms,
                 opts: Optional[N.SvOptions] = None):
    """<H> and d<H>/dtheta by the adjoint method; psi is reset to its input."""
    m = marshal(circ)
    p = np.ascontiguousarray(params, dtype=np.float64)
    arr, nt = pauli_terms(terms)
    ev = C.c_double()
    g = np.zeros(max(1, m.n_params))
    N.check(N.lib().sv_adjoint_grad(psi.h, lam.h, m.ref(), _dptr(p), arr, nt,
                                    C.byref(opts) if opts else None, C.byref(ev), _dptr(g)))
    return ev.value, g[: m.n_params]


def adjoint_grad_batch(psis: Sequence[StateVector], lams: Sequence[StateVector], circ, params: np.ndarray,
                       terms, opts: Optional[N.SvOptions] = None):
    """Batched adjoint gradients: params is B x n_params; returns (ev[B], grad[B, n_params])."""
    m = marshal(circ)
    B = len(psis)
    p = np.ascontiguousarray(params, dtype=np.float64).reshape(B, -1)
    arr, nt = pauli_terms(terms)
    hp = (C.c_void_p * B)(*[s.h.value for s in psis])
    hl = (C.c_void_p * B)(*[s.h.value for s in lams])
    ev = np.zeros(B)
    g = np.zeros((B, max(1, m.n_params)))
    N.check(N.lib().sv_adjoint_grad_batch(hp, hl, B, m.ref(), _dptr(p), arr, nt, C.byref(opts) if opts else None,
                                          _dptr(ev), _dptr(g)))
    return ev, g[:, : m.n_params]


def kernel_launches() -> int:
    return int(N.lib().sv_kernel_launch_count())


class SvExpectation(torch.autograd.Function):
    """E(theta) = <psi(theta)|H|psi(theta)>; backward uses the adjoint gradient.

    forward(theta, psi, lam, circ, terms, init_index): psi is reset to
    |init_index> before each evaluation.
    """

    @staticmethod
    def forward(ctx, theta, psi, lam, circ, terms, init_index=0):
        th = theta.detach().to("cpu", torch.float64).numpy()
        psi.set_basis(init_index)
        ev, g = adjoint_grad(psi, lam, circ, th, terms)
        ctx.save_for_backward(torch.from_numpy(g).to(theta.dtype))
        return theta.new_tensor(ev)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g.to(grad_out.device), None, None, None, None, None
