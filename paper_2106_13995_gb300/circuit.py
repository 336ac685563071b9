"""Python front end: a circuit builder, Pauli-sum observables and a simulator
facade over the C ABI.

The paper's point is usability from Python quantum frameworks (Sec. I: the
simulators it compares are driven through Cirq; Sec. II: QUANTIFY builds the
arithmetic circuits).  This module gives the same style of construction --
named gates, controls, symbolic parameters, grid qubits, inverse and
concatenation -- and hands the result to the library: a ``Circuit`` here is
marshalled as ``sv_circuit`` unchanged, and every amplitude update,
expectation, sample and gradient runs in libsv.so's kernels.  Nothing in this
module touches amplitudes.

Conventions are the library's (include/sv_api.h): qubit q is bit q of the
amplitude index; bit j of a k-qubit matrix's index is targets[j]; a gate acts
where all its controls are |1>.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, Iterable, List, Optional, Sequence, Tuple, Union

import numpy as np


# ---------------------------------------------------------------------------
# ops and parameters
# ---------------------------------------------------------------------------

@dataclass
class Op:
    """One gate: a named gate of the library (or "MATRIX" with ``matrix``),
    its targets, controls and angles; ``param`` >= 0 takes angle 0 from the
    parameter vector at run time."""
    name: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    angles: Tuple[float, ...] = ()
    param: int = -1
    matrix: Optional[np.ndarray] = None

    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.controls)


@dataclass(frozen=True)
class Parameter:
    """A symbolic angle: index into the parameter vector given at run time."""
    index: int
    name: str = ""


Angle = Union[float, Parameter]

# named gates: name -> (targets, angles)
_ARITY = {"H": (1, 0), "X": (1, 0), "Y": (1, 0), "Z": (1, 0), "S": (1, 0), "SDG": (1, 0), "T": (1, 0),
          "TDG": (1, 0), "SX": (1, 0), "SY": (1, 0), "SW": (1, 0), "I": (1, 0), "RX": (1, 1), "RY": (1, 1),
          "RZ": (1, 1), "PHASE": (1, 1), "U3": (1, 3), "CZ": (2, 0), "SWAP": (2, 0), "FSIM": (2, 2)}
# gates whose first angle may be a run-time parameter (the library's adjoint
# gradient differentiates RX, RY, RZ and PHASE)
_PARAMETRIC = {"RX", "RY", "RZ", "PHASE", "U3", "FSIM"}


def grid_qubit(row: int, col: int, cols: int) -> int:
    """Index of lattice site (row, col) on a grid with ``cols`` columns
    (row-major, as the 5 x 6 supremacy-style lattice is numbered)."""
    if row < 0 or col < 0 or col >= cols:
        raise ValueError("grid site out of range")
    return row * cols + col


class Circuit:
    """A gate list on ``n_qubits`` qubits, built with chained calls:

        c = Circuit(3)
        th = c.parameter("theta")
        c.h(0).cx(0, 1).ry(th, 2).toffoli(0, 1, 2)
    """

    def __init__(self, n_qubits: int, name: str = ""):
        if n_qubits < 1:
            raise ValueError("a circuit needs at least one qubit")
        self.n_qubits = n_qubits
        self.name = name
        self.ops: List[Op] = []
        self._params: List[str] = []

    # -- parameters -------------------------------------------------------------
    @property
    def n_params(self) -> int:
        return len(self._params)

    def parameter(self, name: str = "") -> Parameter:
        p = Parameter(len(self._params), name or f"p{len(self._params)}")
        self._params.append(p.name)
        return p

    def parameter_names(self) -> List[str]:
        return list(self._params)

    # -- generic append ---------------------------------------------------------
    def append(self, name: str, targets: Sequence[int], angles: Sequence[Angle] = (),
               controls: Sequence[int] = (), matrix: Optional[np.ndarray] = None) -> "Circuit":
        name = name.upper()
        targets, controls = tuple(int(q) for q in targets), tuple(int(q) for q in controls)
        if name == "MATRIX":
            d = 1 << len(targets)
            m = np.asarray(matrix, dtype=np.complex128)
            if not 1 <= len(targets) <= 6 or m.shape != (d, d):
                raise ValueError("a matrix gate acts on 1..6 targets with a 2^k x 2^k matrix")
            op = Op("MATRIX", targets, controls, (), -1, m.copy())
        else:
            if name not in _ARITY:
                raise ValueError(f"unknown gate {name}")
            k, na = _ARITY[name]
            if len(targets) != k or len(angles) != na:
                raise ValueError(f"{name} takes {k} targets and {na} angles")
            param, vals = -1, []
            for j, a in enumerate(angles):
                if isinstance(a, Parameter):
                    if j != 0 or name not in _PARAMETRIC:
                        raise ValueError("only the first angle of a rotation can be a parameter")
                    if a.index >= self.n_params:
                        raise ValueError("parameter of another circuit")
                    param, a = a.index, 0.0
                vals.append(float(a))
            op = Op(name, targets, controls, tuple(vals), param)
        q = op.qubits()
        if len(set(q)) != len(q):
            raise ValueError("a qubit appears twice in one gate")
        if any(x < 0 or x >= self.n_qubits for x in q):
            raise ValueError("qubit out of range")
        if len(controls) > 8:
            raise ValueError("at most 8 controls")
        self.ops.append(op)
        return self

    # -- named gates ------------------------------------------------------------
    def h(self, q, controls=()): return self.append("H", (q,), controls=controls)
    def x(self, q, controls=()): return self.append("X", (q,), controls=controls)
    def y(self, q, controls=()): return self.append("Y", (q,), controls=controls)
    def z(self, q, controls=()): return self.append("Z", (q,), controls=controls)
    def s(self, q, controls=()): return self.append("S", (q,), controls=controls)
    def sdg(self, q, controls=()): return self.append("SDG", (q,), controls=controls)
    def t(self, q, controls=()): return self.append("T", (q,), controls=controls)
    def tdg(self, q, controls=()): return self.append("TDG", (q,), controls=controls)
    def sx(self, q, controls=()): return self.append("SX", (q,), controls=controls)
    def sy(self, q, controls=()): return self.append("SY", (q,), controls=controls)
    def sw(self, q, controls=()): return self.append("SW", (q,), controls=controls)
    def rx(self, theta: Angle, q, controls=()): return self.append("RX", (q,), (theta,), controls)
    def ry(self, theta: Angle, q, controls=()): return self.append("RY", (q,), (theta,), controls)
    def rz(self, theta: Angle, q, controls=()): return self.append("RZ", (q,), (theta,), controls)
    def phase(self, lam: Angle, q, controls=()): return self.append("PHASE", (q,), (lam,), controls)

    def u3(self, theta: Angle, phi: float, lam: float, q, controls=()):
        return self.append("U3", (q,), (theta, phi, lam), controls)

    def cz(self, a, b, controls=()): return self.append("CZ", (a, b), controls=controls)
    def swap(self, a, b, controls=()): return self.append("SWAP", (a, b), controls=controls)

    def fsim(self, theta: Angle, phi: float, a, b, controls=()):
        return self.append("FSIM", (a, b), (theta, phi), controls)

    def cx(self, control, target): return self.append("X", (target,), controls=(control,))
    cnot = cx

    def ccx(self, c1, c2, target): return self.append("X", (target,), controls=(c1, c2))
    toffoli = ccx

    def mcx(self, controls: Sequence[int], target): return self.append("X", (target,), controls=controls)

    def unitary(self, matrix, *targets, controls=()):
        return self.append("MATRIX", targets, controls=controls, matrix=matrix)

    # -- composition ------------------------------------------------------------
    def extend(self, other: "Circuit") -> "Circuit":
        """Append another circuit's gates (its parameters become new ones)."""
        if other.n_qubits > self.n_qubits:
            raise ValueError("the appended circuit is wider")
        base = self.n_params
        self._params.extend(other._params)
        for op in other.ops:
            self.ops.append(Op(op.name, op.targets, op.controls, op.angles,
                               op.param + base if op.param >= 0 else -1,
                               None if op.matrix is None else op.matrix.copy()))
        return self

    def __add__(self, other: "Circuit") -> "Circuit":
        out = self.copy()
        out.n_qubits = max(self.n_qubits, other.n_qubits)
        return out.extend(other)

    def copy(self) -> "Circuit":
        out = Circuit(self.n_qubits, self.name)
        return out.extend(self)

    def inverse(self) -> "Circuit":
        """U^dagger: the gates reversed, each replaced by its inverse (exact:
        S <-> SDG, T <-> TDG, SX^3 for SX (SX^4 = I), rotations with negated
        angles, U3(t, p, l) -> U3(-t, -l, -p), fSim(t, p) -> fSim(-t, -p),
        conjugate-transposed matrices).  Parametric gates have no negated
        parameter in the library's circuit format and are refused."""
        out = Circuit(self.n_qubits, self.name + "_inv" if self.name else "")
        swap_names = {"S": "SDG", "SDG": "S", "T": "TDG", "TDG": "T"}
        for op in reversed(self.ops):
            if op.param >= 0:
                raise ValueError("the inverse of a parametric gate is not expressible; bind the angle first")
            if op.name == "MATRIX":
                out.unitary(op.matrix.conj().T, *op.targets, controls=op.controls)
            elif op.name in swap_names:
                out.append(swap_names[op.name], op.targets, controls=op.controls)
            elif op.name in ("SX", "SY", "SW"):
                for _ in range(3):
                    out.append(op.name, op.targets, controls=op.controls)
            elif op.name in ("RX", "RY", "RZ", "PHASE"):
                out.append(op.name, op.targets, (-op.angles[0],), op.controls)
            elif op.name == "U3":
                t, p, l = op.angles
                out.append("U3", op.targets, (-t, -l, -p), op.controls)
            elif op.name == "FSIM":
                out.append("FSIM", op.targets, (-op.angles[0], -op.angles[1]), op.controls)
            else:   # H, X, Y, Z, I, CZ, SWAP: self-inverse
                out.append(op.name, op.targets, controls=op.controls)
        return out

    def bind(self, params: Sequence[float]) -> "Circuit":
        """The same circuit with every parameter replaced by its value."""
        params = np.asarray(params, dtype=np.float64)
        if params.size != self.n_params:
            raise ValueError("one value per parameter")
        out = Circuit(self.n_qubits, self.name)
        for op in self.ops:
            ang = list(op.angles)
            if op.param >= 0:
                ang[0] = float(params[op.param])
            out.ops.append(Op(op.name, op.targets, op.controls, tuple(ang), -1,
                              None if op.matrix is None else op.matrix.copy()))
        return out

    def __len__(self) -> int:
        return len(self.ops)

    def __iter__(self):
        return iter(self.ops)

    def __repr__(self) -> str:
        return f"Circuit({self.n_qubits} qubits, {len(self.ops)} gates, {self.n_params} parameters)"


# ---------------------------------------------------------------------------
# Pauli sums (observables)
# ---------------------------------------------------------------------------

def _pc(x: int) -> int:
    return bin(x).count("1")


class PauliSum:
    """A sum of Pauli strings with complex coefficients.  A string is stored
    as (x_mask, z_mask) and means P = i^{|x & z|} X^x Z^z, the library's
    convention (Y on qubit q is x = z = bit q); products follow the Pauli
    group: P(x1, z1) P(x2, z2) = i^e P(x1 ^ x2, z1 ^ z2) with
    e = |x1&z1| + |x2&z2| - |x3&z3| + 2 |z1&x2| (mod 4), since
    Z^z X^x = (-1)^{|z&x|} X^x Z^z."""

    def __init__(self, terms: Optional[Dict[Tuple[int, int], complex]] = None):
        self.t: Dict[Tuple[int, int], complex] = {}
        for k, v in (terms or {}).items():
            if v != 0:
                self.t[k] = complex(v)

    @staticmethod
    def single(kind: str, q: int) -> "PauliSum":
        if q < 0:
            raise ValueError("negative qubit")
        b = 1 << q
        return PauliSum({{"I": (0, 0), "X": (b, 0), "Y": (b, b), "Z": (0, b)}[kind]: 1.0})

    def __add__(self, other):
        other = _as_sum(other)
        out = dict(self.t)
        for k, v in other.t.items():
            out[k] = out.get(k, 0) + v
        return PauliSum(out)

    __radd__ = __add__

    def __neg__(self):
        return PauliSum({k: -v for k, v in self.t.items()})

    def __sub__(self, other):
        return self + (-_as_sum(other))

    def __rsub__(self, other):
        return _as_sum(other) - self

    def __mul__(self, other):
        if isinstance(other, (int, float, complex, np.number)):
            return PauliSum({k: v * other for k, v in self.t.items()})
        other = _as_sum(other)
        out: Dict[Tuple[int, int], complex] = {}
        for (x1, z1), c1 in self.t.items():
            for (x2, z2), c2 in other.t.items():
                x3, z3 = x1 ^ x2, z1 ^ z2
                e = (_pc(x1 & z1) + _pc(x2 & z2) - _pc(x3 & z3) + 2 * _pc(z1 & x2)) % 4
                out[(x3, z3)] = out.get((x3, z3), 0) + c1 * c2 * (1j ** e)
        return PauliSum(out)

    def __rmul__(self, other):
        if isinstance(other, (int, float, complex, np.number)):
            return self * other
        return _as_sum(other) * self

    def terms(self, tol: float = 1e-12) -> List[Tuple[int, int, float]]:
        """(x_mask, z_mask, coeff) for sv_expect; the observable must be
        Hermitian, i.e. every coefficient real."""
        out = []
        for (x, z), c in sorted(self.t.items()):
            if abs(c.imag) > tol * max(1.0, abs(c.real)):
                raise ValueError("observable is not Hermitian (complex coefficient)")
            if c.real != 0:
                out.append((x, z, float(c.real)))
        return out

    def max_qubit(self) -> int:
        m = 0
        for x, z in self.t:
            m |= x | z
        return m.bit_length()

    def __repr__(self) -> str:
        return f"PauliSum({len(self.t)} terms)"


def _as_sum(v) -> PauliSum:
    if isinstance(v, PauliSum):
        return v
    if isinstance(v, (int, float, complex, np.number)):
        return PauliSum({(0, 0): complex(v)})
    raise TypeError(f"cannot combine a Pauli sum with {type(v).__name__}")


def X(q: int) -> PauliSum: return PauliSum.single("X", q)
def Y(q: int) -> PauliSum: return PauliSum.single("Y", q)
def Z(q: int) -> PauliSum: return PauliSum.single("Z", q)
def I() -> PauliSum: return PauliSum.single("I", 0)


def ising(n: int, j: float = 1.0, h: float = 0.5, periodic: bool = False) -> PauliSum:
    """Transverse-field Ising chain: j sum Z_i Z_{i+1} + h sum X_i."""
    H = PauliSum()
    for i in range(n - 1 + (1 if periodic and n > 2 else 0)):
        H = H + j * (Z(i) * Z((i + 1) % n))
    for i in range(n):
        H = H + h * X(i)
    return H


# ---------------------------------------------------------------------------
# simulator facade
# ---------------------------------------------------------------------------

class Simulator:
    """Runs builder circuits on one GPU through the C ABI.

        sim = Simulator(dtype="c64", prec="bf16x3")
        psi = sim.simulate(c, params)            # a StateVector (device-resident)
        e = sim.expectation(c, ising(n), params)
        e, g = sim.gradient(c, ising(n), params) # adjoint method
        shots = sim.sample(c, 1000, seed=7)
    """

    _PREC = {"plain": 0, "bf16x3": 1, "tf32x3": 2}

    def __init__(self, dtype: str = "c64", prec: str = "plain", device: str = "cuda", fusion_k: int = 0,
                 tile_m: int = 0):
        from . import sim as _sim
        if prec not in self._PREC:
            raise ValueError(f"prec must be one of {sorted(self._PREC)}")
        self._sim = _sim
        self.dtype, self.device = dtype, device
        self.opts = _sim.options(fusion_k=fusion_k, tile_m=tile_m, prec=self._PREC[prec])
        self._cache: Dict[int, object] = {}

    def _state(self, n: int):
        st = self._cache.get(n)
        if st is None:
            st = self._sim.StateVector(n, self.dtype, device=self.device)
            self._cache[n] = st
        return st

    def _params(self, circuit: Circuit, params) -> Optional[np.ndarray]:
        if circuit.n_params == 0:
            return None
        if params is None:
            raise ValueError("the circuit has parameters: pass their values")
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1)
        if p.size != circuit.n_params:
            raise ValueError("one value per parameter")
        return p

    def simulate(self, circuit: Circuit, params=None, initial_state: Union[int, np.ndarray] = 0, state=None):
        """psi = U(params) psi_0, psi_0 = |initial_state> or a given vector;
        returns the device-resident StateVector (reused per width unless
        ``state`` is given)."""
        st = state if state is not None else self._state(circuit.n_qubits)
        if isinstance(initial_state, (int, np.integer)):
            st.set_basis(int(initial_state))
        else:
            st.load(np.asarray(initial_state))
        return st.apply_circuit(circuit, self._params(circuit, params), opts=self.opts)

    def state_vector(self, circuit: Circuit, params=None, initial_state=0) -> np.ndarray:
        return self.simulate(circuit, params, initial_state).numpy()

    def expectation(self, circuit: Circuit, observable: PauliSum, params=None, initial_state=0) -> float:
        if observable.max_qubit() > circuit.n_qubits:
            raise ValueError("observable acts beyond the circuit's qubits")
        return self.simulate(circuit, params, initial_state).expect(observable.terms())

    def sample(self, circuit: Circuit, shots: int, seed: int = 0, params=None, initial_state=0) -> np.ndarray:
        return self.simulate(circuit, params, initial_state).sample(shots, seed)

    def gradient(self, circuit: Circuit, observable: PauliSum, params, initial_state: int = 0):
        """(<H>, d<H>/dparams) by the library's adjoint sweep."""
        n = circuit.n_qubits
        psi = self._state(n).set_basis(int(initial_state))
        lam_key = -n
        lam = self._cache.get(lam_key)
        if lam is None:
            lam = self._sim.StateVector(n, self.dtype, device=self.device)
            self._cache[lam_key] = lam
        return self._sim.adjoint_grad(psi, lam, circuit, self._params(circuit, params), observable.terms(),
                                      opts=self.opts)

    def close(self):
        for st in self._cache.values():
            st.close()
        self._cache.clear()
