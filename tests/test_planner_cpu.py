"""Host logic without a GPU: the library's fusion planner, tile-pass planner
and program emitter, linked from its object files into a small CPU
interpreter of the emitted programs (tests/host/plan_emulator.cu), must
reproduce the FP64 oracle for every fusion width and tile size, with
controls inside and outside the tile."""
import ctypes as C
import glob
import os
import subprocess

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def emu():
    import paper_2106_13995_gb300 as P
    import importlib
    B = importlib.import_module("paper_2106_13995_gb300.buildlib")
    P.build()
    objs = sorted(glob.glob(os.path.join(B.OUT_DIR, "*.o")))
    out_dir = os.path.join(HERE, "host", "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libplanemu.so")
    src = os.path.join(HERE, "host", "plan_emulator.cu")
    deps = [src] + objs
    if not os.path.exists(lib) or any(os.path.getmtime(d) > os.path.getmtime(lib) for d in deps):
        subprocess.check_call([B.nvcc(), *B.ARCH, "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                               "-I", os.path.join(ROOT, "include"), "-o", lib, src, *objs])
    L = C.CDLL(lib)
    L.plan_emulate.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int]
    L.check_thread_positions.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
    L.check_op_pre.argtypes = [C.c_void_p, C.c_int, C.c_int]
    return L


def run(emu, circ, fk, m, L, merge=0):
    from paper_2106_13995_gb300 import sim
    mm = sim.marshal(circ)
    psi = np.zeros(1 << circ.n_qubits, dtype=np.complex128)
    psi[0] = 1
    nb = C.c_int()
    npass = emu.plan_emulate(C.addressof(mm.c), psi.ctypes.data, fk, m, L, C.byref(nb), merge)
    assert npass > 0
    return psi, npass, nb.value


@pytest.mark.parametrize("fk", [1, 2, 3, 4, 6])
def test_mixed_circuits_every_fusion_and_tile(emu, oracle, fk):
    for seed in range(6):
        n = 9 + seed % 3
        c = W.random_gate_circuit(n, 60, seed=seed * 7 + fk)
        want = oracle.run(c)
        for m, L in ((n, 3), (7, 1), (8, 3)):
            got, npass, nb = run(emu, c, fk, m, L)
            assert oracle.infidelity(want, got) <= 1e-12, (seed, fk, m, L)


def test_grid_and_multiplier(emu, oracle):
    for c in (W.grid_random(3, 4, 8, 3), W.multiplier(2), W.random_u3_cz(11, 6, 2)):
        want = oracle.run(c)
        for fk, m in ((3, 8), (2, 6), (5, 10)):
            got, npass, nb = run(emu, c, fk, min(m, c.n_qubits), 2)
            assert oracle.infidelity(want, got) <= 1e-12, (c.name, fk, m)


def test_fusion_reduces_blocks(emu):
    """Fusion merges gates into fewer blocks (pass counts may go either way:
    wider blocks pack less freely into a tile's free slots)."""
    c = W.grid_random(4, 4, 10, 1)
    _, p1, b1 = run(emu, c, 1, 8, 3)
    _, p3, b3 = run(emu, c, 3, 8, 3)
    assert b3 < b1 == len(c.ops)
    assert p1 > 0 and p3 > 0


@pytest.mark.parametrize("fk", [2, 3, 4])
def test_merge_in_passes_matches_oracle(emu, oracle, fk):
    """Blocks of a pass that commuting lets meet merge into one block of at
    most fk qubits; the merged program still reproduces the FP64 oracle, and
    never has more blocks than the unmerged one."""
    for seed in range(6):
        n = 9 + seed % 3
        c = W.random_gate_circuit(n, 80, seed=seed * 11 + fk)
        want = oracle.run(c)
        for m, L in ((n, 3), (7, 1), (8, 3)):
            _, _, nb0 = run(emu, c, fk, m, L)
            got, npass, nb = run(emu, c, fk, m, L, merge=1)
            assert npass > 0
            assert nb <= nb0
            assert oracle.infidelity(want, got) <= 1e-12, (seed, m, L)
    g = W.grid_random(4, 4, 10, 2)
    want = oracle.run(g)
    _, _, nb0 = run(emu, g, 3, 10, 3)
    got, _, nb = run(emu, g, 3, 10, 3, merge=1)
    assert nb < nb0
    assert oracle.infidelity(want, got) <= 1e-12


def test_permutation_passes_as_tables(emu, oracle):
    """Passes whose blocks are all 0/1 permutations (the multiplier's X,
    CNOT, Toffoli and C^3X) become gather tables composed on the host, one
    per setting of the pass's global control qubits; small tiles leave many
    controls global.  Run on the CPU the programs match the oracle exactly,
    with Hadamard inputs too (the first pass then keeps its dense ops)."""
    emu.table_pass_count.restype = C.c_int
    emu.table_pass_count()
    total_h_tables = [0]
    for c in (W.multiplier(2), W.multiplier(2, hadamard_inputs=True), W.multiplier(3)):
        want = oracle.run(c)
        for fk, m in ((3, 9), (2, 6), (3, 5), (1, 4)):
            got, npass, nb = run(emu, c, fk, min(m, c.n_qubits), 2)
            tables = emu.table_pass_count()
            if not c.name.endswith("_h"):
                assert tables == npass, (c.name, fk, m, tables, npass)
            else:
                total_h_tables[0] += tables
            assert oracle.infidelity(want, got) <= 1e-12, (c.name, fk, m)
            assert np.max(np.abs(got - want)) <= 1e-12, (c.name, fk, m)
    assert total_h_tables[0] > 0   # smaller tiles split H from the permutations


def test_thread_positions_cover_every_group(emu):
    """The plan-time thread-bit positions of complex64 tile ops: with the
    trip map of the launch's thread count (and of the 512-thread persistent
    kernel) every op visits each of its groups exactly once, and most ops'
    16 lanes of a wavefront reach 16 bank rows."""
    from paper_2106_13995_gb300 import sim
    for c, fk, m in ((W.grid_random(4, 5, 10, 1), 3, 13), (W.grid_random(4, 4, 10, 2), 2, 12),
                     (W.random_gate_circuit(14, 120, seed=5), 3, 12),
                     # (Hadamard inputs: the multiplier's own passes are
                     # permutation tables and carry no tile ops)
                     (W.multiplier(3, hadamard_inputs=True), 3, 10),
                     (W.random_gate_circuit(12, 80, seed=9), 1, 9)):
        mm = sim.marshal(c)
        spread = C.c_int()
        checked = emu.check_thread_positions(C.addressof(mm.c), fk, min(m, c.n_qubits), 3, C.byref(spread))
        assert checked > 0, c.name
        assert spread.value >= 0.5 * checked, (c.name, spread.value, checked)


def test_op_setup_records_match_direct_slots(emu):
    """The per-op set-up the host puts in a tile pass's parameter block
    (member offsets, trip map, offsets of a trip's groups and of the first
    four trips) composes to the swizzled slot of every amplitude the op
    touches in those trips."""
    from paper_2106_13995_gb300 import sim
    for c, m in ((W.grid_random(4, 5, 10, 1), 13), (W.random_gate_circuit(14, 120, seed=5), 12),
                 (W.random_gate_circuit(11, 60, seed=2), 9), (W.multiplier(3, hadamard_inputs=True), 10)):
        mm = sim.marshal(c)
        assert emu.check_op_pre(C.addressof(mm.c), min(m, c.n_qubits), 3) > 0, c.name


def test_program_cache_eviction_keeps_held_programs(emu):
    """The program cache with a small bound, driven past it while an early
    entry is held (the pattern of one batched call over many circuits): the
    held program stays intact, each lookup returns its own circuit's
    program, and an evicted circuit is rebuilt to the same program."""
    from paper_2106_13995_gb300 import sim
    circs = [W.random_u3_cz(10, 2, seed) for seed in range(40)]
    ms = [sim.marshal(c) for c in circs]
    arr = (C.c_void_p * len(ms))(*[C.addressof(m.c) for m in ms])
    emu.cache_selftest.argtypes = [C.c_void_p, C.c_int, C.c_int]
    assert emu.cache_selftest(arr, len(ms), 8) == 0
    # a bound larger than the number of circuits: nothing is evicted
    assert emu.cache_selftest(arr, 5, 64) == 0


def test_split_bf16_programs_match_oracle(emu, oracle):
    """The split-BF16 tensor-core programs: small blocks padded to 5 qubits
    with idle tile qubits, targets in increasing tile position with the
    matrix permuted to match, operands packed as BF16 hi/lo parts of the
    real embedding.  Unpacked and run on the CPU they reproduce the FP64
    oracle to the split's precision (hi + lo keeps about 16 significant
    bits per entry); circuits without controlled gates take the pipelined
    kernel in every pass."""
    from paper_2106_13995_gb300 import sim
    emu.tc_program_emulate.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    cases = [(W.grid_random(3, 5, 10, 1), True), (W.random_u3_cz(14, 8, 3), True),
             (W.remove_qubits(W.grid_random(5, 6, 6, 2), 16, 7), True), (W.multiplier(3), False)]
    for c, pure in cases:
        mm = sim.marshal(c)
        psi = np.zeros(1 << c.n_qubits, dtype=np.complex128)
        psi[0] = 1
        npure, nsix = C.c_int(), C.c_int()
        npass = emu.tc_program_emulate(C.addressof(mm.c), psi.ctypes.data, C.byref(npure), 0, C.byref(nsix))
        assert npass > 0, c.name
        if pure:
            assert npure.value == npass, (c.name, npure.value, npass)
        want = oracle.run(c)
        inf = oracle.infidelity(want, psi)
        assert inf <= 1e-8, (c.name, inf)
        assert np.max(np.abs(psi - want)) <= 1e-4 * np.max(np.abs(want)), c.name


def test_pipelined_layout_chains(emu, oracle):
    """Passes of dense 5-qubit blocks whose targets overlap: every pass runs
    in the pipelined kernel, whose blocks after the first see the tile
    through their own shared-memory layout.  The emulator replays the
    kernel's address tables for every pass (each gathered member must be
    the amplitude its row and member index name, each scatter must fill
    every slot once, pair moves must be aligned 16-byte units) and runs the
    program against the FP64 oracle; over these circuits both 16-byte pair
    gathers and pair scatters must occur."""
    from paper_2106_13995_gb300 import sim
    emu.tc_program_emulate.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    emu.tc_pair_counts.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int)]
    g, sc = C.c_int(), C.c_int()
    emu.tc_pair_counts(C.byref(g), C.byref(sc))   # reset
    total_g = total_s = 0
    for seed, (n, count, span) in enumerate([(13, 12, 7), (14, 16, 8), (12, 10, 12), (15, 14, 9)]):
        c = W.block_chain(n, count, seed + 40, span)
        mm = sim.marshal(c)
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1
        npure, nsix = C.c_int(), C.c_int()
        npass = emu.tc_program_emulate(C.addressof(mm.c), psi.ctypes.data, C.byref(npure), 0, C.byref(nsix))
        assert npass > 0 and npure.value == npass, (c.name, npure.value, npass)
        emu.tc_pair_counts(C.byref(g), C.byref(sc))
        total_g += g.value
        total_s += sc.value
        want = oracle.run(c)
        assert oracle.infidelity(want, psi) <= 1e-8, c.name
        assert np.max(np.abs(psi - want)) <= 1e-4 * np.max(np.abs(want)), c.name
    assert total_g > 0 and total_s > 0, (total_g, total_s)


def test_basis_propagation_matches_oracle(emu, oracle):
    """The host-side basis-state path: through the multiplier (X, CNOT,
    Toffoli, C^3X) every basis input |a, b, 0, 0> goes to |a, b, a*b, 0> with
    amplitude exactly 1; through permutation and phase gates (SWAP, CZ, S, T,
    fSim(pi/2, phi), controlled X) the index and phase match the oracle's
    single nonzero amplitude; a Hadamard stops the path."""
    from paper_2106_13995_gb300 import sim
    emu.basis_propagate.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64), C.c_void_p]
    nb = 3
    m = sim.marshal(W.multiplier(nb))
    out = C.c_uint64()
    amp = np.zeros(2)
    for a in range(8):
        for b in range(8):
            assert emu.basis_propagate(C.addressof(m.c), W.multiplier_basis_index(a, b, nb), C.byref(out),
                                       amp.ctypes.data) == 1
            assert out.value == W.multiplier_basis_index(a, b, nb, a * b), (a, b)
            assert amp[0] == 1.0 and amp[1] == 0.0
    rng = np.random.default_rng(4)
    n = 7
    for trial in range(6):
        c = W.Circuit(n)
        for _ in range(30):
            g = rng.choice(["SWAP", "CZ", "S", "T", "FSIM", "CX", "Y", "Z"])
            q = [int(x) for x in rng.choice(n, size=3, replace=False)]
            if g in ("SWAP", "CZ"):
                c.ops.append(W.Op(g, (q[0], q[1])))
            elif g == "FSIM":
                c.ops.append(W.Op("FSIM", (q[0], q[1]), angles=(np.pi / 2, np.pi / 6)))
            elif g == "CX":
                c.ops.append(W.Op("X", (q[0],), controls=(q[1], q[2])))
            else:
                c.ops.append(W.Op(g, (q[0],)))
        idx0 = int(rng.integers(0, 1 << n))
        mm = sim.marshal(c)
        assert emu.basis_propagate(C.addressof(mm.c), idx0, C.byref(out), amp.ctypes.data) == 1
        psi0 = np.zeros(1 << n, complex)
        psi0[idx0] = 1
        want = oracle.run(c, psi0)
        nz = np.flatnonzero(np.abs(want) > 1e-12)
        assert list(nz) == [out.value]
        assert abs(want[out.value] - complex(amp[0], amp[1])) <= 1e-13
    h = W.Circuit(n, [W.Op("X", (0,)), W.Op("H", (1,))])
    assert emu.basis_propagate(C.addressof(sim.marshal(h).c), 0, C.byref(out), amp.ctypes.data) == 0


def test_split_bf16_six_qubit_blocks(emu, oracle):
    """Fusion width 6 in split-BF16: uncontrolled dense 6-qubit blocks become
    tensor-core passes of their own (their 128 x 128 real embedding packed as
    BF16 hi/lo parts), the rest stays in tile passes; unpacked and run on the
    CPU the program reproduces the FP64 oracle to the split's precision."""
    from paper_2106_13995_gb300 import sim
    emu.tc_program_emulate.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    for c in (W.grid_random(3, 5, 10, 1), W.random_u3_cz(14, 10, 5)):
        mm = sim.marshal(c)
        psi = np.zeros(1 << c.n_qubits, dtype=np.complex128)
        psi[0] = 1
        npure, nsix = C.c_int(), C.c_int()
        assert emu.tc_program_emulate(C.addressof(mm.c), psi.ctypes.data, C.byref(npure), 6, C.byref(nsix)) > 0
        assert nsix.value > 0, c.name
        want = oracle.run(c)
        assert oracle.infidelity(want, psi) <= 1e-8, c.name
        assert np.max(np.abs(psi - want)) <= 1e-4 * np.max(np.abs(want)), c.name


def test_unitarity_check_of_caller_matrices(emu, monkeypatch):
    """With SV_CHECK_UNITARY=1 a circuit's MATRIX op must be unitary to
    1e-10 (max |U^dagger U - I|) or planning stops with SV_EINVAL; without
    it the matrix is taken as given."""
    from paper_2106_13995_gb300 import sim
    from paper_2106_13995_gb300 import _native as N
    emu.build_status.argtypes = [C.c_void_p]
    rng = np.random.default_rng(1)
    good = W.random_unitary(2, rng)
    bad = good.copy()
    bad[0, 0] += 1e-6
    for m, want_checked in ((good, N.SV_OK), (bad, N.SV_EINVAL)):
        c = W.Circuit(4, [W.Op("MATRIX", (0, 2), matrix=m), W.Op("H", (1,))])
        mm = sim.marshal(c)
        monkeypatch.setenv("SV_CHECK_UNITARY", "1")
        assert emu.build_status(C.addressof(mm.c)) == want_checked
        monkeypatch.delenv("SV_CHECK_UNITARY")
        c2 = W.Circuit(4, [W.Op("MATRIX", (0, 2), matrix=m), W.Op("X", (1,))])   # a new program
        assert emu.build_status(C.addressof(sim.marshal(c2).c)) == N.SV_OK
