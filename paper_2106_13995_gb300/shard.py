"""One state vector over several GPUs: planning and executing global-qubit
swaps.

The paper names multi-GPU simulation as the way past one device's memory
(Sec. I and Sec. IV).  A state of n qubits is split over G = 2^g ranks by
its top g index bits: rank r holds the 2^(n-g) amplitudes whose top bits
equal r.  A gate whose targets are all "local" (physical index bits below
n - g) is applied by every rank to its own shard; a control on a "global"
qubit is a condition on the rank number, so it needs no exchange.  A gate
with a global target first swaps that qubit with a local one: each rank
exchanges half of its shard (the half whose local bit differs from its own
global bit) with the partner rank whose number differs in that global bit,
after which the two qubits have traded places.  The planner tracks where
every logical qubit sits and picks the local qubit to evict whose next use
as a target is furthest away, so one swap serves many gates.

This module is orchestration only: local gates are applied by a caller's
applier (the library's kernels through ``sim.StateVector`` on GPUs) and
half-shards move through a transport -- ``torch.distributed`` point to point
between processes (NCCL on GPUs, gloo on CPUs), or an in-process loopback for
several shards held by one process.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple


@dataclass
class LocalOp:
    """A gate in physical local positions; ``rank_mask``: the rank bits that
    must all be 1 (controls on global qubits)."""
    name: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...]
    angles: Tuple[float, ...]
    param: int
    matrix: object
    rank_mask: int = 0


@dataclass
class Stage:
    """Either a run of local gates (``ops``) or one swap of global bit
    ``gbit`` (of the rank number) with local position ``lpos``."""
    kind: str                        # "local" or "swap"
    ops: List[LocalOp] = field(default_factory=list)
    gbit: int = -1
    lpos: int = -1


@dataclass
class ShardPlan:
    n: int
    g: int
    stages: List[Stage]
    final_pos: List[int]             # physical position of each logical qubit after the stages

    @property
    def local_qubits(self) -> int:
        return self.n - self.g

    def swaps(self) -> int:
        return sum(1 for s in self.stages if s.kind == "swap")


def plan(circuit, g: int, restore: bool = True) -> ShardPlan:
    """Stages that apply ``circuit`` (any object with n_qubits and ops of
    name / targets / controls / angles / param / matrix) to a state sharded
    over 2^g ranks.  With ``restore`` the layout ends as it began (logical
    qubit q at position q)."""
    n = circuit.n_qubits
    L = n - g
    if g < 0 or L < 1:
        raise ValueError("need at least one local qubit")
    pos = list(range(n))                  # logical -> physical
    at = list(range(n))                   # physical -> logical
    ops = list(circuit.ops)
    for op in ops:
        if len(op.targets) > L:
            raise ValueError("a gate has more targets than there are local qubits")
    # next use of each logical qubit as a target, from op index i on
    uses: Dict[int, List[int]] = {q: [] for q in range(n)}
    for i, op in enumerate(ops):
        for q in op.targets:
            uses[q].append(i)
    cursor = {q: 0 for q in range(n)}

    def next_use(q: int, i: int) -> int:
        lst, c = uses[q], cursor[q]
        while c < len(lst) and lst[c] < i:
            c += 1
        cursor[q] = c
        return lst[c] if c < len(lst) else 1 << 60

    stages: List[Stage] = []

    def local_stage() -> Stage:
        if not stages or stages[-1].kind != "local":
            stages.append(Stage("local"))
        return stages[-1]

    def swap(gpos: int, lpos: int):
        a, b = at[gpos], at[lpos]
        pos[a], pos[b] = lpos, gpos
        at[gpos], at[lpos] = b, a
        stages.append(Stage("swap", gbit=gpos - L, lpos=lpos))

    for i, op in enumerate(ops):
        for q in op.targets:
            if pos[q] >= L:
                busy = {pos[t] for t in op.targets if pos[t] < L}
                # evict the local qubit whose next use as a target is furthest away
                best, best_use = -1, -1
                for p in range(L):
                    if p in busy:
                        continue
                    u = next_use(at[p], i)
                    if u > best_use:
                        best, best_use = p, u
                swap(pos[q], best)
        tg = tuple(pos[q] for q in op.targets)
        lc = tuple(pos[q] for q in op.controls if pos[q] < L)
        rm = 0
        for q in op.controls:
            if pos[q] >= L:
                rm |= 1 << (pos[q] - L)
        local_stage().ops.append(LocalOp(op.name, tg, lc, tuple(op.angles), op.param,
                                         getattr(op, "matrix", None), rm))
    if restore:
        restore_layout(pos, at, L, swap, local_stage)
    return ShardPlan(n, g, stages, list(pos))


def restore_layout(pos, at, L, swap, local_stage):
    """Bring logical qubit q back to position q: global positions first (by
    swaps through local positions), then a permutation of the local ones (by
    local SWAP gates)."""
    n = len(pos)
    for P in range(L, n):
        if at[P] == P:
            continue
        if pos[P] >= L:                  # logical P sits at another global position: via a local one
            swap(pos[P], 0)
        swap(P, pos[P])
    for p in range(L):
        while at[p] != p:
            q = at[p]                     # logical q belongs at position q (< L)
            local_stage().ops.append(LocalOp("SWAP", (p, q), (), (), -1, None, 0))
            a, b = at[p], at[q]
            pos[a], pos[b] = q, p
            at[p], at[q] = b, a


# ---------------------------------------------------------------------------
# transports
# ---------------------------------------------------------------------------

def _halves(shard, lpos: int):
    """(complex view of the shard as [outer, 2, 2^lpos]) -- index 1 selects
    local bit lpos."""
    import torch
    v = shard if shard.is_complex() else torch.view_as_complex(shard.view(-1, 2))
    return v.view(-1, 2, 1 << lpos)


class LoopbackTransport:
    """Every shard held by this process (e.g. several shards on one GPU):
    a swap exchanges the halves directly."""

    def __init__(self, shards: Sequence):
        self.shards = list(shards)

    def ranks(self) -> List[int]:
        return list(range(len(self.shards)))

    def swap(self, gbit: int, lpos: int):
        for r in range(len(self.shards)):
            p = r ^ (1 << gbit)
            if p < r:
                continue
            br = (r >> gbit) & 1          # 0 for r
            a, b = _halves(self.shards[r], lpos), _halves(self.shards[p], lpos)
            tmp = a[:, 1 - br, :].clone()
            a[:, 1 - br, :] = b[:, br, :]
            b[:, br, :] = tmp


class DistTransport:
    """One shard per process; halves move by torch.distributed point-to-point
    operations (NCCL between GPUs, gloo between CPU processes)."""

    def __init__(self, shard, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.shards = [shard]

    def ranks(self) -> List[int]:
        return [self.rank]

    def swap(self, gbit: int, lpos: int):
        dist = self.dist
        partner = self.rank ^ (1 << gbit)
        b = (self.rank >> gbit) & 1
        import torch
        h = _halves(self.shards[0], lpos)
        # the half this rank gives away, as real numbers (every backend
        # carries real tensors); the partner's half lands in the same slots
        send = torch.view_as_real(h[:, 1 - b, :].contiguous())
        recv = torch.empty_like(send)
        rs = dist.isend(send, partner, group=self.group)
        rr = dist.irecv(recv, partner, group=self.group)
        rs.wait()
        rr.wait()
        h[:, 1 - b, :] = torch.view_as_complex(recv)


# ---------------------------------------------------------------------------
# execution
# ---------------------------------------------------------------------------

@dataclass
class SubCircuit:
    """The local gates one rank applies between two swaps (the library's
    circuit format, width n - g)."""
    n_qubits: int
    ops: List[LocalOp]
    n_params: int = 0


def run(plan_: ShardPlan, transport, apply_local: Callable[[int, SubCircuit], None], n_params: int = 0,
        on_exchange: Optional[Callable[[int], None]] = None):
    """Execute a plan: for each local stage, each rank of ``transport``
    applies the stage's gates whose rank conditions it meets (through
    ``apply_local(rank_index_in_transport, subcircuit)``); each swap stage
    goes through the transport.  ``on_exchange(i)`` runs after shard i was
    written by an exchange (e.g. to tell the library its amplitudes
    changed)."""
    for st in plan_.stages:
        if st.kind == "swap":
            transport.swap(st.gbit, st.lpos)
            if on_exchange:
                for i in range(len(transport.ranks())):
                    on_exchange(i)
            continue
        for i, r in enumerate(transport.ranks()):
            mine = [op for op in st.ops if (r & op.rank_mask) == op.rank_mask]
            if mine:
                apply_local(i, SubCircuit(plan_.local_qubits, mine, n_params))
