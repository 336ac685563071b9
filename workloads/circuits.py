"""Seeded synthetic circuit workloads shared by the FP64 oracle and the GPU path.

This module only describes circuits: which named gate acts on which qubits,
with which angles, in which order.  It holds none of the simulation
arithmetic -- no gate matrix is built here (each side builds its own from the
gate name), no state is touched.  Random angles, random matchings, random
qubit removals and random test unitaries are drawn here from numpy's
``default_rng`` so both sides receive identical inputs.

Conventions (used by every consumer):
  * qubit q is bit q of the amplitude index (little-endian);
  * for a k-qubit gate, bit j of the gate's local row/column index is
    ``targets[j]``;
  * ``controls`` must all be |1> for the gate to act.

Workload shapes follow the paper's two benchmark families (Sec. III): random
"supremacy" grid circuits and quantum multipliers, plus the closed-form and
variational circuits used to pin correctness.  Non-standard widths are made
by removing random qubits and their gates from a larger circuit (Sec. II).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Named gates understood by both the oracle and the GPU library.
# name -> (number of targets, number of angles)
GATES = {
    "I": (1, 0), "X": (1, 0), "Y": (1, 0), "Z": (1, 0), "H": (1, 0),
    "S": (1, 0), "SDG": (1, 0), "T": (1, 0), "TDG": (1, 0),
    "SX": (1, 0), "SY": (1, 0), "SW": (1, 0),
    "RX": (1, 1), "RY": (1, 1), "RZ": (1, 1), "PHASE": (1, 1),
    "U3": (1, 3),
    "CZ": (2, 0), "SWAP": (2, 0), "FSIM": (2, 2),
    "MATRIX": (-1, 0),
}


@dataclass
class Op:
    """One gate of a circuit.

    ``param >= 0`` marks a parametric gate whose first angle is taken from the
    parameter vector at run time (``angles`` is then ignored for angle 0).
    ``matrix`` is only used by ``MATRIX`` ops: a 2^k x 2^k complex array.
    """
    name: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    angles: Tuple[float, ...] = ()
    param: int = -1
    matrix: Optional[np.ndarray] = None

    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.controls)


@dataclass
class Circuit:
    n_qubits: int
    ops: List[Op] = field(default_factory=list)
    n_params: int = 0
    name: str = ""

    def __len__(self) -> int:
        return len(self.ops)

    def validate(self) -> None:
        for op in self.ops:
            k, na = GATES[op.name]
            if k > 0 and len(op.targets) != k:
                raise ValueError(f"{op.name} takes {k} targets")
            q = op.qubits()
            if len(set(q)) != len(q):
                raise ValueError(f"duplicate qubit in {op}")
            if any(x < 0 or x >= self.n_qubits for x in q):
                raise ValueError(f"qubit out of range in {op}")
            if op.name == "MATRIX":
                d = 1 << len(op.targets)
                if op.matrix is None or op.matrix.shape != (d, d):
                    raise ValueError("MATRIX op needs a 2^k x 2^k matrix")
            if op.param >= self.n_params:
                raise ValueError("param index out of range")


# ---------------------------------------------------------------------------
# random inputs
# ---------------------------------------------------------------------------

def random_unitary(k: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random 2^k x 2^k unitary: QR of a complex Gaussian, phases fixed."""
    d = 1 << k
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def random_state(n: int, rng: np.random.Generator) -> np.ndarray:
    """Normalised complex Gaussian vector of length 2^n (complex128)."""
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# random U3 + CZ circuits (12-qubit parity case; uneven batch)
# ---------------------------------------------------------------------------

def random_u3_cz(n: int, layers: int, seed) -> Circuit:
    """Layers of U3 on every qubit, then CZ on a random perfect matching.

    Angles are i.i.d. uniform in [0, 2pi), drawn qubit by qubit in the order
    (theta, phi, lambda).  The matching pairs consecutive entries of a random
    permutation; for odd n the last entry idles.
    """
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"u3cz_{n}q_{layers}l")
    for _ in range(layers):
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            c.ops.append(Op("U3", (q,), angles=tuple(float(a) for a in ang[q])))
        perm = rng.permutation(n)
        for i in range(n // 2):
            a, b = int(perm[2 * i]), int(perm[2 * i + 1])
            c.ops.append(Op("CZ", (min(a, b), max(a, b))))
    return c


def block_chain(n: int, count: int, seed, span: int = 8) -> Circuit:
    """count dense 5-qubit blocks (Haar-random unitaries), each on 5 qubits
    drawn without replacement from a window of `span` consecutive qubits
    placed at random in the register, so that neighbouring blocks share
    targets and several blocks fit one tile pass."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"chain_{n}q_{count}b")
    for _ in range(count):
        lo = int(rng.integers(0, n - span + 1))
        t = tuple(int(x) for x in rng.choice(np.arange(lo, lo + span), size=5, replace=False))
        c.ops.append(Op("MATRIX", t, matrix=random_unitary(5, rng)))
    return c


# ---------------------------------------------------------------------------
# grid random ("supremacy-style") circuits
# ---------------------------------------------------------------------------

FSIM_THETA = math.pi / 2
FSIM_PHI = math.pi / 6


def grid_couplers(rows: int, cols: int):
    """Coupler sets A..D of a rows x cols lattice, qubit (r, c) -> r*cols + c.

    A: horizontal pairs starting at an even column, B: odd column,
    C: vertical pairs starting at an even row, D: odd row.  Each set is a
    matching.
    """
    A, B, C, D = [], [], [], []
    for r in range(rows):
        for c in range(cols - 1):
            (A if c % 2 == 0 else B).append((r * cols + c, r * cols + c + 1))
    for r in range(rows - 1):
        for c in range(cols):
            (C if r % 2 == 0 else D).append((r * cols + c, (r + 1) * cols + c))
    return {"A": A, "B": B, "C": C, "D": D}


def grid_random(rows: int, cols: int, cycles: int, seed) -> Circuit:
    """Random grid circuit: per cycle one of {SX, SY, SW} on every qubit (never
    the same as that qubit's previous cycle), then fSim(pi/2, pi/6) on the
    couplers of pattern ``"ABCDCDAB"[(cycle-1) mod 8]``."""
    rng = np.random.default_rng(seed)
    n = rows * cols
    cp = grid_couplers(rows, cols)
    names = ("SX", "SY", "SW")
    prev = [-1] * n
    c = Circuit(n, name=f"grid_{rows}x{cols}_{cycles}c")
    for cyc in range(1, cycles + 1):
        for q in range(n):
            if prev[q] < 0:
                g = int(rng.integers(0, 3))
            else:
                choices = [i for i in range(3) if i != prev[q]]
                g = choices[int(rng.integers(0, 2))]
            prev[q] = g
            c.ops.append(Op(names[g], (q,)))
        pat = "ABCDCDAB"[(cyc - 1) % 8]
        for a, b in cp[pat]:
            c.ops.append(Op("FSIM", (a, b), angles=(FSIM_THETA, FSIM_PHI)))
    return c


def remove_qubits(circ: Circuit, n_remove: int, seed) -> Circuit:
    """Width reduction (Sec. II): delete ``n_remove`` random qubits and every
    gate touching them, then relabel the remaining qubits densely."""
    rng = np.random.default_rng(seed)
    gone = set(int(x) for x in rng.choice(circ.n_qubits, size=n_remove, replace=False))
    keep = [q for q in range(circ.n_qubits) if q not in gone]
    relabel = {q: i for i, q in enumerate(keep)}
    out = Circuit(len(keep), n_params=circ.n_params, name=f"{circ.name}_minus{n_remove}")
    for op in circ.ops:
        if any(q in gone for q in op.qubits()):
            continue
        out.ops.append(Op(op.name, tuple(relabel[q] for q in op.targets),
                          tuple(relabel[q] for q in op.controls), op.angles, op.param, op.matrix))
    return out


# ---------------------------------------------------------------------------
# quantum multiplier (shift-and-add of controlled ripple-carry adders)
# ---------------------------------------------------------------------------

def multiplier_layout(nbits: int):
    """Register layout of the nbits x nbits multiplier: a, b, product, carry."""
    a = list(range(0, nbits))
    b = list(range(nbits, 2 * nbits))
    p = list(range(2 * nbits, 4 * nbits))
    carry = 4 * nbits
    return a, b, p, carry


def _cx(ctrls, t):
    return Op("X", (t,), tuple(ctrls))


def multiplier(nbits: int = 7, hadamard_inputs: bool = False) -> Circuit:
    """p <- a*b with a, b nbits-wide, p 2*nbits-wide, one carry ancilla.

    For each bit b_i, a ripple-carry adder (majority / un-majority-and-add
    blocks of CNOT and Toffoli) adds a into p[i .. i+nbits-1], carry out into
    p[i+nbits]; every gate of that adder gets b_i as an extra control.  Width
    4*nbits + 1.  With ``hadamard_inputs`` the circuit starts with H on every
    a and b qubit (equal-superposition inputs, Sec. III).
    """
    a, b, p, c = multiplier_layout(nbits)
    circ = Circuit(4 * nbits + 1, name=f"mult_{nbits}b" + ("_h" if hadamard_inputs else ""))
    if hadamard_inputs:
        for q in a + b:
            circ.ops.append(Op("H", (q,)))
    for i in range(nbits):
        ctl = (b[i],)
        y = p[i:i + nbits]            # sum register for this partial product
        z = p[i + nbits]              # carry out
        carry_in = [c] + a[:-1]       # MAJ chain carries ride on the a wires
        ops = []
        for j in range(nbits):        # MAJ(cin, y_j, a_j)
            cin, yj, xj = carry_in[j], y[j], a[j]
            ops += [_cx(ctl + (xj,), yj), _cx(ctl + (xj,), cin), _cx(ctl + (cin, yj), xj)]
        ops.append(_cx(ctl + (a[-1],), z))
        for j in reversed(range(nbits)):   # UMA(cin, y_j, a_j)
            cin, yj, xj = carry_in[j], y[j], a[j]
            ops += [_cx(ctl + (cin, yj), xj), _cx(ctl + (xj,), cin), _cx(ctl + (cin,), yj)]
        circ.ops.extend(ops)
    return circ


def multiplier_basis_index(a_val: int, b_val: int, nbits: int, product: int = 0) -> int:
    """Amplitude index of |a, b, product, carry=0>."""
    return a_val | (b_val << nbits) | (product << (2 * nbits))


# ---------------------------------------------------------------------------
# variational ansatz + Ising Hamiltonian
# ---------------------------------------------------------------------------

def hea(n: int = 20, layers: int = 10) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(theta) then RZ(theta) on every
    qubit (each angle its own parameter, index (layer*n + q)*2 + {0,1}), then
    a linear CNOT ladder q -> q+1."""
    c = Circuit(n, n_params=2 * n * layers, name=f"hea_{n}q_{layers}l")
    for l in range(layers):
        for q in range(n):
            c.ops.append(Op("RY", (q,), param=(l * n + q) * 2))
            c.ops.append(Op("RZ", (q,), param=(l * n + q) * 2 + 1))
        for q in range(n - 1):
            c.ops.append(Op("X", (q + 1,), (q,)))
    return c


def tfim(n: int, hx: float = 0.5) -> List[Tuple[int, int, float]]:
    """Open-chain transverse-field Ising sum_i Z_i Z_{i+1} + hx sum_i X_i as
    Pauli terms (x_mask, z_mask, coeff); a Y on qubit q sets both bits."""
    terms = [(0, (1 << i) | (1 << (i + 1)), 1.0) for i in range(n - 1)]
    terms += [(1 << i, 0, hx) for i in range(n)]
    return terms


def hea_params(batch: int, n_params: int, seed) -> np.ndarray:
    """Parameter sets, uniform in [-pi, pi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, size=(batch, n_params))


# ---------------------------------------------------------------------------
# uneven batch of random circuits
# ---------------------------------------------------------------------------

def uneven_batch(count: int = 256, nmin: int = 10, nmax: int = 24, depth: int = 40, seed=4):
    """``count`` random U3+CZ circuits with widths uniform in [nmin, nmax]."""
    ss = np.random.SeedSequence(seed)
    rng = np.random.default_rng(ss)
    widths = rng.integers(nmin, nmax + 1, size=count)
    kids = ss.spawn(count)
    return [random_u3_cz(int(w), depth, kids[i]) for i, w in enumerate(widths)]


# ---------------------------------------------------------------------------
# closed-form circuits
# ---------------------------------------------------------------------------

def ghz(n: int) -> Circuit:
    c = Circuit(n, name=f"ghz_{n}")
    c.ops.append(Op("H", (0,)))
    for i in range(1, n):
        c.ops.append(Op("X", (i,), (0,)))
    return c


def qft(n: int, with_swaps: bool = True) -> Circuit:
    """Textbook QFT on little-endian qubits: from the most significant qubit
    down, H then controlled phases pi/2^d from each lower qubit, then reverse
    the qubit order with SWAPs."""
    c = Circuit(n, name=f"qft_{n}")
    for j in reversed(range(n)):
        c.ops.append(Op("H", (j,)))
        for l in reversed(range(j)):
            c.ops.append(Op("PHASE", (j,), (l,), angles=(math.pi / (1 << (j - l)),)))
    if with_swaps:
        for q in range(n // 2):
            c.ops.append(Op("SWAP", (q, n - 1 - q)))
    return c


def basis_prep(n: int, index: int) -> Circuit:
    """X gates that turn |0...0> into |index>."""
    c = Circuit(n, name=f"basis_{index}")
    for q in range(n):
        if (index >> q) & 1:
            c.ops.append(Op("X", (q,)))
    return c


def hadamard_all(n: int) -> Circuit:
    c = Circuit(n, name=f"h_all_{n}")
    for q in range(n):
        c.ops.append(Op("H", (q,)))
    return c


def concat(*circs: Circuit) -> Circuit:
    n = max(c.n_qubits for c in circs)
    out = Circuit(n, n_params=max(c.n_params for c in circs), name="+".join(c.name for c in circs))
    for c in circs:
        out.ops.extend(c.ops)
    return out


def random_gate_circuit(n: int, count: int, seed, kmax: int = 3, cmax: int = 2,
                        names: Sequence[str] = ("H", "X", "Y", "Z", "S", "T", "SX", "SY", "SW",
                                                "RX", "RY", "RZ", "U3", "PHASE", "CZ", "SWAP",
                                                "FSIM", "MATRIX")) -> Circuit:
    """Mixed random gates (named, parametric-angle and dense random unitaries
    on up to ``kmax`` targets, with up to ``cmax`` controls) for parity tests."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"mixed_{n}q_{count}")
    for _ in range(count):
        name = names[int(rng.integers(0, len(names)))]
        k, na = GATES[name]
        if name == "MATRIX":
            k = int(rng.integers(1, min(kmax, n) + 1))
        if k > n:
            continue
        nc = int(rng.integers(0, min(cmax, n - k) + 1))
        qs = rng.permutation(n)[: k + nc]
        tg = tuple(int(x) for x in qs[:k])
        ct = tuple(int(x) for x in qs[k:])
        ang = tuple(float(a) for a in rng.uniform(-math.pi, math.pi, size=na))
        m = random_unitary(k, rng) if name == "MATRIX" else None
        c.ops.append(Op(name, tg, ct, ang, -1, m))
    return c
