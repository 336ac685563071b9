"""One state over several ranks (global-qubit swaps), without GPUs.

The plan is checked on one full state: its local gates (with global
controls as extra controls on the rank bits) and its swaps (SWAP gates
between a rank bit and a local bit) applied by the FP64 oracle reproduce the
circuit.  Then the plan runs on 2 and 4 gloo ranks on the CPU, each holding
one shard: the ranks apply their local gates with the oracle (the test's
applier) and exchange half-shards through torch.distributed; the gathered
state equals the oracle's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2106_13995_gb300 import shard as S


def full_state_replay(oracle, plan, psi0):
    """Apply the plan's stages to the full physical state with the oracle."""
    L = plan.local_qubits
    psi = psi0.copy()
    for st in plan.stages:
        c = W.Circuit(plan.n)
        if st.kind == "swap":
            c.ops.append(W.Op("SWAP", (st.lpos, L + st.gbit)))
        else:
            for op in st.ops:
                gctl = tuple(L + j for j in range(plan.g) if (op.rank_mask >> j) & 1)
                c.ops.append(W.Op(op.name, op.targets, op.controls + gctl, op.angles, op.param, op.matrix))
        psi = oracle.run(c, psi)
    return psi


@pytest.mark.parametrize("g", [1, 2, 3])
def test_plan_replayed_on_one_state(oracle, g):
    rng = np.random.default_rng(g)
    for seed in range(4):
        n = 8
        c = W.random_gate_circuit(n, 70, seed=seed + 10 * g)
        psi0 = W.random_state(n, rng)
        p = S.plan(c, g)
        assert p.final_pos == list(range(n))
        got = full_state_replay(oracle, p, psi0)
        assert np.max(np.abs(got - oracle.run(c, psi0))) <= 1e-12
        assert p.swaps() > 0


def test_local_circuits_need_no_swap(oracle):
    c = W.random_u3_cz(6, 4, 1)
    c8 = W.Circuit(8, list(c.ops))        # gates on the low 6 of 8 qubits: all local with g = 2
    p8 = S.plan(c8, 2)
    assert p8.swaps() == 0 and len(p8.stages) == 1
    # controls on global qubits are rank conditions, not swaps
    cc = W.Circuit(8, [W.Op("X", (0,), controls=(7,)), W.Op("H", (1,), controls=(6, 2))])
    pc = S.plan(cc, 2)
    assert pc.swaps() == 0
    assert [op.rank_mask for op in pc.stages[0].ops] == [2, 1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, seed, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    g = world.bit_length() - 1
    L = n - g
    c = W.random_gate_circuit(n, 80, seed=seed)
    psi0 = W.random_state(n, np.random.default_rng(seed))
    shard = torch.from_numpy(psi0[rank << L:(rank + 1) << L].copy())

    def apply_local(i, sub):
        out = oracle.run(sub, shard.numpy())
        shard.copy_(torch.from_numpy(out))

    S.run(S.plan(c, g), S.DistTransport(shard), apply_local)
    real = torch.view_as_real(shard).contiguous()     # gloo carries real tensors
    parts = [torch.empty_like(real) for _ in range(world)] if rank == 0 else None
    dist.gather(real, parts, dst=0)
    if rank == 0:
        got = torch.view_as_complex(torch.cat(parts)).numpy()
        np.save(out_path, np.stack([got, oracle.run(c, psi0)]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_match_oracle(tmp_path, oracle, world):
    out = str(tmp_path / "res.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), 9, 5 + world, out), nprocs=world,
                       start_method="spawn", join=True)
    got, want = np.load(out)
    assert np.max(np.abs(got - want)) <= 1e-12
