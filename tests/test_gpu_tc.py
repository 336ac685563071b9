"""Fused 5-qubit dense blocks on the tensor cores (tcgen05): split-TF32 and
split-BF16 (three products, FP32 accumulation) against the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from conftest import fidelity_metrics

pytestmark = pytest.mark.gpu

MODES = {"tf32x3": 2, "bf16x3": 1}
# per-block error budget of each split mode (relative amplitude error)
AMP_TOL = {"tf32x3": 2e-6, "bf16x3": 6e-5}


def one_block_circuit(n, targets, rng):
    c = W.Circuit(n)
    c.ops.append(W.Op("MATRIX", tuple(targets), matrix=W.random_unitary(5, rng)))
    return c


# tile_m 12: the block runs inside a 12-qubit tile pass; 11: as a pass of its own
@pytest.mark.parametrize("tile_m", [12, 11])
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4), (4, 3, 2, 1, 0), (7, 2, 11, 0, 13), (13, 12, 11, 10, 9),
                                     (1, 5, 9, 12, 3)])
def test_single_block(svlib, oracle, mode, targets, tile_m):
    rng = np.random.default_rng(sum(targets))
    n = 14
    c = one_block_circuit(n, targets, rng)
    psi0 = W.random_state(n, rng)
    cast = psi0.astype(np.complex64).astype(np.complex128)
    s = svlib.StateVector(n, "c64").load(psi0)
    opts = svlib.options(prec=MODES[mode], tile_m=tile_m)
    nb, npass = s.plan_info(c, opts=opts)
    assert nb == 1 and npass == 1
    s.apply_circuit(c, opts=opts)
    got = s.numpy().astype(np.complex128)
    want = oracle.run(c, cast)
    inf, amp = fidelity_metrics(want, got)
    scale = np.max(np.abs(want))
    assert amp <= AMP_TOL[mode] * scale, (amp, scale)
    assert inf <= 1e-8


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("tile_m", [12, 11])
def test_large_state_tiles(svlib, oracle, mode, tile_m):
    """Many tiles (256 tile passes / grid-stride CTAs), 20 qubits."""
    rng = np.random.default_rng(5)
    n = 20
    c = one_block_circuit(n, (19, 3, 0, 10, 17), rng)
    psi0 = W.random_state(n, rng)
    s = svlib.StateVector(n, "c64").load(psi0)
    s.apply_circuit(c, opts=svlib.options(prec=MODES[mode], tile_m=tile_m))
    want = oracle.run(c, psi0.astype(np.complex64).astype(np.complex128))
    inf, amp = fidelity_metrics(want, s.numpy())
    assert inf <= 1e-8 and amp <= AMP_TOL[mode] * np.max(np.abs(want))


@pytest.mark.parametrize("tile_m", [12, 11])
@pytest.mark.parametrize("mode", list(MODES))
def test_circuits_with_fused_5q_blocks(svlib, oracle, mode, tile_m):
    for c in (W.random_u3_cz(16, 12, 3), W.grid_random(4, 4, 10, 2),
              W.remove_qubits(W.grid_random(5, 6, 8, 1), 10, 3)):
        opts = svlib.options(prec=MODES[mode], tile_m=tile_m)
        s = svlib.StateVector(c.n_qubits, "c64").set_basis(0)
        nb, npass = s.plan_info(c, opts=opts)
        s.apply_circuit(c, opts=opts)
        inf, amp = fidelity_metrics(oracle.run(c), s.numpy())
        assert inf <= 1e-5, (c.name, mode, inf)
        print(f"{c.name} {mode} m={tile_m}: blocks {nb}, passes {npass}, 1-F {inf:.2e}, max|d| {amp:.2e}")


def test_pipelined_layout_chains(svlib, oracle):
    """Chains of dense 5-qubit blocks with overlapping targets, split-BF16:
    the pipelined tile pass with a shared-memory layout per block (16-byte
    pair gathers and scatters), checked amplitude by amplitude against the
    FP64 oracle from a random state; the error budget grows with the
    number of blocks."""
    # 12 qubits: a single tile, so three of the CTA's four groups get none
    for seed, (n, count, span) in enumerate([(12, 10, 12), (13, 12, 7), (14, 16, 8), (16, 24, 9), (18, 20, 12)]):
        rng = np.random.default_rng(seed)
        c = W.block_chain(n, count, seed + 40, span)
        psi0 = W.random_state(n, rng)
        s = svlib.StateVector(n, "c64").load(psi0)
        opts = svlib.options(prec=MODES["bf16x3"])
        nb, npass = s.plan_info(c, opts=opts)
        s.apply_circuit(c, opts=opts)
        want = oracle.run(c, psi0.astype(np.complex64).astype(np.complex128))
        inf, amp = fidelity_metrics(want, s.numpy())
        scale = np.max(np.abs(want))
        print(f"{c.name}: blocks {nb}, passes {npass}, 1-F {inf:.2e}, max|d| {amp / scale:.2e} of max|a|")
        assert amp <= nb * AMP_TOL["bf16x3"] * scale, (c.name, amp, scale)
        assert inf <= 1e-6, (c.name, inf)
        s.close()


def test_tc_rejected_for_complex128(svlib, oracle):
    """complex128 states keep FP64 CUDA-core arithmetic in every mode."""
    c = W.random_u3_cz(13, 4, 1)
    s = svlib.StateVector(13, "c128").set_basis(0).apply_circuit(c, opts=svlib.options(prec=2))
    inf, _ = fidelity_metrics(oracle.run(c), s.numpy())
    assert inf <= 1e-12


def six_block_circuit(n, targets, rng):
    c = W.Circuit(n)
    c.ops.append(W.Op("MATRIX", tuple(targets), matrix=W.random_unitary(6, rng)))
    return c


@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4, 5), (5, 4, 3, 2, 1, 0), (7, 2, 11, 0, 13, 9),
                                     (13, 12, 11, 10, 9, 8), (1, 5, 9, 12, 3, 6)])
def test_six_qubit_block(svlib, oracle, targets):
    """A fused 6-qubit block on the tensor cores (split-BF16, a pass of its
    own: (2^(n-6) x 128) x (128 x 128) real GEMM) against the oracle, at the
    same per-amplitude budget as 5-qubit blocks."""
    rng = np.random.default_rng(sum(targets) + 6)
    n = 14
    c = six_block_circuit(n, targets, rng)
    psi0 = W.random_state(n, rng)
    s = svlib.StateVector(n, "c64").load(psi0)
    opts = svlib.options(prec=MODES["bf16x3"], fusion_k=6)
    assert s.plan_info(c, opts=opts) == (1, 1)
    l0 = svlib.kernel_launches()
    s.apply_circuit(c, opts=opts)
    assert svlib.kernel_launches() - l0 == 1
    want = oracle.run(c, psi0.astype(np.complex64).astype(np.complex128))
    inf, amp = fidelity_metrics(want, s.numpy())
    assert amp <= AMP_TOL["bf16x3"] * np.max(np.abs(want)), amp
    assert inf <= 1e-8


def test_six_qubit_blocks_many_tiles_and_circuits(svlib, oracle):
    rng = np.random.default_rng(66)
    n = 20
    c = six_block_circuit(n, (19, 3, 0, 10, 17, 7), rng)
    psi0 = W.random_state(n, rng)
    s = svlib.StateVector(n, "c64").load(psi0)
    s.apply_circuit(c, opts=svlib.options(prec=MODES["bf16x3"], fusion_k=6))
    want = oracle.run(c, psi0.astype(np.complex64).astype(np.complex128))
    inf, amp = fidelity_metrics(want, s.numpy())
    assert inf <= 1e-8 and amp <= AMP_TOL["bf16x3"] * np.max(np.abs(want))
    # whole circuits at fusion width 6: 6-qubit passes between tile passes
    for c in (W.random_u3_cz(16, 12, 3), W.grid_random(4, 4, 10, 2)):
        opts = svlib.options(prec=MODES["bf16x3"], fusion_k=6)
        st = svlib.StateVector(c.n_qubits, "c64").set_basis(0).apply_circuit(c, opts=opts)
        inf, amp = fidelity_metrics(oracle.run(c), st.numpy())
        assert inf <= 1e-5, (c.name, inf)
        print(f"{c.name} bf16x3 k<=6: blocks/passes {st.plan_info(c, opts=opts)}, 1-F {inf:.2e}, max|d| {amp:.2e}")
