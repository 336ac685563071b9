"""GPU parity of whole circuits (fusion planner + tile passes) against the
FP64 oracle: the 12-qubit random U3+CZ case, mixed random circuits under
every fusion width and tile size, grid circuits, closed forms and the
quantum multiplier."""
import math

import numpy as np
import pytest

import workloads as W
from conftest import fidelity_metrics

pytestmark = pytest.mark.gpu


def run_gpu(svlib, circ, dt, psi0=None, opts=None, params=None):
    s = svlib.StateVector(circ.n_qubits, dt)
    if psi0 is None:
        s.set_basis(0)
    else:
        s.load(psi0)
    s.apply_circuit(circ, params=params, opts=opts)
    return s


def test_random_u3cz_12q_c128(svlib, oracle):
    """12 qubits, 20 layers, complex128: 1-F <= 1e-12, <Z_i> within 1e-12."""
    c = W.random_u3_cz(12, 20, 0)
    want = oracle.run(c)
    for opts in (None, svlib.options(mode=1), svlib.options(fusion_k=1), svlib.options(fusion_k=5, tile_m=9)):
        s = run_gpu(svlib, c, "c128", opts=opts)
        inf, amp = fidelity_metrics(want, s.numpy())
        assert inf <= 1e-12 and amp <= 1e-13, (opts, inf, amp)
        z = s.z_all()
        assert np.max(np.abs(z - oracle.z_all(want))) <= 1e-12
        assert abs(s.norm2() - 1) <= 1e-13


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("fk", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("m", [6, 10, 13])
def test_mixed_random_all_fusions_and_tiles(svlib, oracle, dt, fk, m):
    n = 14
    c = W.random_gate_circuit(n, 120, seed=fk * 100 + m)
    psi0 = W.random_state(n, np.random.default_rng(m))
    cast = psi0.astype(np.complex64 if dt == "c64" else np.complex128).astype(np.complex128)
    want = oracle.run(c, cast)
    s = run_gpu(svlib, c, dt, psi0=psi0, opts=svlib.options(fusion_k=fk, tile_m=m))
    inf, amp = fidelity_metrics(want, s.numpy())
    tol = 1e-5 if dt == "c64" else 1e-12
    assert inf <= tol, (inf, amp)
    # per amplitude: a few units of the state's rounding, relative to the
    # largest amplitude (complex64 ~6e-8 per operation, complex128 ~1e-16)
    amp_tol = (1e-5 if dt == "c64" else 1e-13) * float(np.max(np.abs(want)))
    assert amp <= amp_tol, (amp, amp_tol)
    print(f"{dt} fk={fk} m={m}: 1-F {inf:.2e}, max |d psi| {amp:.2e}")


@pytest.mark.parametrize("nops", [47, 48, 49, 200])
def test_pass_op_list_around_parameter_block_size(svlib, oracle, nops):
    """A complex64 pass keeps its op list and small dense matrices in the
    launch's parameter block when the list fits (48 ops), and its global
    copies otherwise: one 13-qubit pass of nops unfused blocks on each side
    of that size agrees with the oracle."""
    n = 13
    rng = np.random.default_rng(nops)
    c = W.Circuit(n)
    for i in range(nops):
        k = 1 + i % 3
        t = tuple(int(x) for x in rng.choice(n, size=k, replace=False))
        c.ops.append(W.Op("MATRIX", t, matrix=W.random_unitary(k, rng)))
    opts = svlib.options(fusion_k=1, tile_m=n)
    s = run_gpu(svlib, c, "c64", opts=opts)
    assert s.plan_info(c, opts=opts) == (nops, 1)
    inf, amp = fidelity_metrics(oracle.run(c), s.numpy())
    assert inf <= 1e-5, (nops, inf, amp)


def test_plan_fmas_counts_blocks(svlib):
    """sv_plan_fmas: 4 * 2^k / 2^c real multiply-adds per amplitude for a
    dense k-qubit block with c controls, 4 / 2^c for a diagonal one."""
    n = 6
    s = svlib.StateVector(n, "c64")
    one = svlib.options(fusion_k=1)
    c = W.Circuit(n)
    c.ops += [W.Op("H", (q,)) for q in range(n)]
    assert s.plan_fmas(c, opts=one) == 8.0 * n
    c = W.Circuit(n)
    c.ops += [W.Op("RZ", (q,), angles=(0.3,)) for q in range(n)]
    assert s.plan_fmas(c, opts=one) == 4.0 * n
    c = W.Circuit(n)
    c.ops.append(W.Op("X", (0,), (1, 2)))                     # Toffoli: 8 / 4
    assert s.plan_fmas(c, opts=one) == 2.0
    rng = np.random.default_rng(3)
    c = W.Circuit(n)
    c.ops.append(W.Op("MATRIX", (0, 1, 2), matrix=W.random_unitary(3, rng)))
    assert s.plan_fmas(c) == 32.0
    g = W.grid_random(4, 4, 8, 1)
    s16 = svlib.StateVector(16, "c64")
    nb, _ = s16.plan_info(g)
    f = s16.plan_fmas(g)
    assert 8.0 * nb <= f <= 32.0 * nb
    s.close()
    s16.close()


@pytest.mark.parametrize("n", [3, 5, 9])
def test_small_states_single_tile(svlib, oracle, n):
    c = W.random_gate_circuit(n, 40, seed=n, kmax=min(3, n))
    want = oracle.run(c)
    for dt, tol in (("c64", 1e-5), ("c128", 1e-12)):
        inf, _ = fidelity_metrics(want, run_gpu(svlib, c, dt).numpy())
        assert inf <= tol


def test_grid_4x4(svlib, oracle):
    c = W.grid_random(4, 4, 8, seed=1)
    want = oracle.run(c)
    for opts in (None, svlib.options(mode=1), svlib.options(fusion_k=4, tile_m=11)):
        inf, amp = fidelity_metrics(want, run_gpu(svlib, c, "c64", opts=opts).numpy())
        assert inf <= 1e-5, (opts, inf)


@pytest.mark.parametrize("prec", ["plain", "bf16x3"])
def test_grid_26q_instance(svlib, oracle, prec):
    """The 26-qubit width-reduced 5x6 grid circuit, complex64 vs FP64 oracle,
    with FP32 CUDA-core blocks and with split-BF16 tensor-core blocks (the
    bench's arithmetic)."""
    from paper_2106_13995_gb300 import _native as N
    c = W.remove_qubits(W.grid_random(5, 6, 20, seed=1), 4, seed=101)
    want = oracle.run(c)
    opts = svlib.options(prec=N.SV_PREC_TC_BF16X3 if prec == "bf16x3" else N.SV_PREC_PLAIN)
    s = svlib.StateVector(c.n_qubits, "c64").set_basis(0).apply_circuit(c, opts=opts)
    got = s.numpy()
    inf, amp = fidelity_metrics(want, got)
    rms = float(np.sqrt(np.mean(np.abs(want) ** 2)))
    assert inf <= 1e-5, inf
    # per amplitude within 1e-3 of the rms amplitude (the error of one block is
    # ~1e-7 (FP32) or ~1e-5 (split-BF16) of the amplitudes it mixes)
    assert amp <= 1e-3 * rms, (amp, rms)
    print(f"grid 26q c64 {prec}: 1-F = {inf:.3e}, max |d psi| = {amp:.3e} (rms amplitude {rms:.3e})")


def test_ghz_and_qft(svlib, oracle):
    for dt in ("c64", "c128"):
        n = 20
        v = run_gpu(svlib, W.ghz(n), dt).numpy()
        r = np.float32(1 / math.sqrt(2)) if dt == "c64" else 1 / math.sqrt(2)
        assert v[0] == r and v[-1] == r and np.count_nonzero(v) == 2
        n = 10
        x = 337
        q = run_gpu(svlib, W.concat(W.basis_prep(n, x), W.qft(n)), dt).numpy()
        want = np.exp(2j * math.pi * x * np.arange(1 << n) / (1 << n)) / math.sqrt(1 << n)
        tol = 1e-6 if dt == "c64" else 1e-13
        assert np.max(np.abs(q - want)) <= tol


def test_multiplier_3bit_all_inputs(svlib):
    nb = 3
    c = W.multiplier(nb)
    for a in range(8):
        for b in range(8):
            s = svlib.StateVector(c.n_qubits, "c64").set_basis(W.multiplier_basis_index(a, b, nb))
            s.apply_circuit(c)
            v = s.numpy()
            idx = W.multiplier_basis_index(a, b, nb, a * b)
            assert v[idx] == 1 and np.count_nonzero(v) == 1


def test_multiplier_complex128_permutation_ops(svlib, oracle):
    """complex128 tile passes apply the multiplier's blocks as permutation
    ops (no FP64 arithmetic): every basis input of the 3-bit multiplier,
    through the tile passes (the basis-state path switched off), and the
    superposed 5-bit multiplier against the oracle, exactly."""
    from paper_2106_13995_gb300 import _native as N
    nb = 3
    c = W.multiplier(nb)
    s = svlib.StateVector(c.n_qubits, "c128")
    for a in range(8):
        for b in range(8):
            s.set_basis(W.multiplier_basis_index(a, b, nb))
            N.check(N.lib().sv_mark_modified(s.h))
            v = s.apply_circuit(c).numpy()
            idx = W.multiplier_basis_index(a, b, nb, a * b)
            assert v[idx] == 1 and np.count_nonzero(v) == 1
    c5 = W.multiplier(5, hadamard_inputs=True)
    got = svlib.StateVector(c5.n_qubits, "c128").set_basis(0).apply_circuit(c5).numpy()
    assert np.max(np.abs(got - oracle.run(c5))) <= 1e-15


def test_multiplier_29q_basis_inputs(svlib):
    """Full width: 7-bit x 7-bit multiplier, 64 seeded basis inputs; the
    output bits are read from <Z_q> = 1 - 2 bit_q (exactly +-1)."""
    nb = 7
    c = W.multiplier(nb)
    m = svlib.marshal(c)
    rng = np.random.default_rng(2)
    s = svlib.StateVector(c.n_qubits, "c64")
    for a, b in rng.integers(0, 128, size=(64, 2)):
        a, b = int(a), int(b)
        s.set_basis(W.multiplier_basis_index(a, b, nb))
        s.apply_circuit(m)
        z = s.z_all()
        bits = (z < 0).astype(np.int64)
        idx = int(sum(int(v) << q for q, v in enumerate(bits)))
        assert idx == W.multiplier_basis_index(a, b, nb, a * b)
        assert np.all(np.abs(np.abs(z) - 1) <= 1e-6)


def test_multiplier_superposed_inputs(svlib):
    """H on both inputs: probability 2^-2nb on every |a,b,ab,0> (within
    1e-6 relative: 1/sqrt(2) is rounded in FP32) and exactly 0 elsewhere
    (the multiplier only permutes amplitudes)."""
    nb = 5
    c = W.multiplier(nb, hadamard_inputs=True)
    v = run_gpu(svlib, c, "c64").numpy()
    p = np.abs(v.astype(np.complex128)) ** 2
    want = np.zeros_like(p)
    for a in range(1 << nb):
        for b in range(1 << nb):
            want[W.multiplier_basis_index(a, b, nb, a * b)] = 2.0 ** (-2 * nb)
    assert np.array_equal(p != 0, want != 0)
    assert np.max(np.abs(p - want)) <= 1e-6 * 2.0 ** (-2 * nb)
    # full width, checked by sampling: every shot decodes to (a, b, a*b, 0)
    nb = 7
    s = run_gpu(svlib, W.multiplier(nb, hadamard_inputs=True), "c64")
    shots = s.sample(4096, 99)
    for x in shots.tolist():
        a, b = x & 127, (x >> 7) & 127
        assert x == W.multiplier_basis_index(a, b, nb, a * b)
    assert abs(s.norm2() - 1) <= 1e-6


def test_multiplier_basis_fast_path_equals_dense_path(svlib):
    """A state set by sv_set_basis goes through the 29-qubit multiplier as a
    host-side index update (two amplitudes rewritten); after
    sv_mark_modified the same input takes the tile passes, whose blocks are
    permutation ops.  Both give the same bits, and the fast path launches a
    single one-thread kernel."""
    import torch
    from paper_2106_13995_gb300 import _native as N
    nb = 7
    m = svlib.marshal(W.multiplier(nb))
    fast = svlib.StateVector(4 * nb + 1, "c64")
    dense = svlib.StateVector(4 * nb + 1, "c64")
    rng = np.random.default_rng(12)
    for a, b in rng.integers(0, 128, size=(4, 2)):
        idx = W.multiplier_basis_index(int(a), int(b), nb)
        fast.set_basis(idx)
        l0 = svlib.kernel_launches()
        fast.apply_circuit(m)
        assert svlib.kernel_launches() - l0 == 1
        dense.set_basis(idx)
        N.check(N.lib().sv_mark_modified(dense.h))
        dense.apply_circuit(m)
        torch.cuda.synchronize()
        assert torch.equal(fast.amps, dense.amps), (a, b)
        want = W.multiplier_basis_index(int(a), int(b), nb, int(a) * int(b))
        assert fast.amps[2 * want].item() == 1.0
    # a non-permutation circuit ends the basis-state path
    fast.set_basis(0)
    fast.apply_circuit(W.Circuit(4 * nb + 1, [W.Op("H", (0,))]))
    fast.apply_circuit(m)
    v = fast.amps.view(-1, 2)
    assert torch.count_nonzero(v[:, 0]).item() == 2


def test_multiplier_29q_superposed_exhaustive(svlib):
    """H on all 14 input qubits of the 29-qubit multiplier: checked on the
    device over all 2^29 amplitudes -- exactly 2^14 nonzero, each at
    |a, b, a*b, 0> with probability 2^-14 (within 1e-6 relative)."""
    import torch
    nb = 7
    s = run_gpu(svlib, W.multiplier(nb, hadamard_inputs=True), "c64")
    v = torch.view_as_complex(s.amps.view(-1, 2))
    nz = torch.count_nonzero(v).item()
    assert nz == 1 << (2 * nb)
    ab = torch.arange(1 << (2 * nb), device=v.device, dtype=torch.int64)
    a, b = ab & 127, ab >> 7
    idx = a | (b << nb) | ((a * b) << (2 * nb))
    p = (v[idx].abs().double() ** 2)
    assert torch.max(torch.abs(p - 2.0 ** -14)).item() <= 1e-6 * 2.0 ** -14


def test_program_cache_reuse_and_params(svlib, oracle):
    c = W.hea(8, 2)
    p1 = W.hea_params(2, c.n_params, 5)
    m = svlib.marshal(c)
    s = svlib.StateVector(8, "c128")
    for p in p1:
        s.set_basis(0).apply_circuit(m, params=p)
        inf, _ = fidelity_metrics(oracle.run(c, params=p), s.numpy())
        assert inf <= 1e-12


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_permutation_table_passes_move_random_states_exactly(svlib, oracle, dt):
    """Multipliers on a random dense state: every pass is made of 0/1
    permutation blocks, so the library runs them as gather-table passes.
    Moving amplitudes is exact, so the result equals the FP64 oracle applied
    to the same (rounded) input bit for bit -- with the default tiles and
    with small tiles that leave several controls outside the tile (one
    table per setting of them)."""
    rng = np.random.default_rng(77)
    for nbits in (2, 3):
        c = W.multiplier(nbits)
        n = c.n_qubits
        psi0 = W.random_state(n, rng)
        cast = psi0.astype(np.complex64 if dt == "c64" else np.complex128)
        want = oracle.run(c, cast.astype(np.complex128))
        for tile_m in (0, 6):
            s = svlib.StateVector(n, dt).load(psi0)
            s.apply_circuit(c, opts=svlib.options(tile_m=tile_m))
            got = s.numpy().astype(np.complex128)
            assert np.array_equal(got, want), (nbits, dt, tile_m, float(np.max(np.abs(got - want))))
            s.close()
