"""The 30-qubit grid workload at full size, in the launch configuration the
benchmark times (default options, and the two tensor-core modes).

The oracle cannot run a 30-qubit circuit in seconds, so full size is checked
two ways:
- a 30-qubit grid circuit whose couplers between lattice rows 2 and 3 are
  left out factorises into an 18-qubit and a 12-qubit state, which the
  oracle computes; the GPU state is compared with their Kronecker product
  over the whole vector (fidelity) and amplitude by amplitude on a seeded
  sample;
- the 30-qubit circuit itself is checked by properties that hold at any
  size: unit norm, agreement of the CUDA-core and tensor-core paths, and
  the inverse circuit taking the state back to |0...0>.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

N = 30
ROWS, COLS = 5, 6
CUT = 18            # qubits 0..17 are rows 0..2, qubits 18..29 rows 3..4


def factorised_grid(seed=1):
    full = W.grid_random(ROWS, COLS, 20, seed)
    low = W.Circuit(CUT, name="grid_rows012")
    high = W.Circuit(N - CUT, name="grid_rows34")
    keep = W.Circuit(N, name="grid_5x6_cut")
    for op in full.ops:
        q = op.qubits()
        if all(x < CUT for x in q):
            low.ops.append(op)
        elif all(x >= CUT for x in q):
            high.ops.append(W.Op(op.name, tuple(x - CUT for x in op.targets), (), op.angles, op.param, op.matrix))
        else:
            continue            # a coupler across the cut
        keep.ops.append(op)
    return keep, low, high


def as_complex(s):
    return torch.view_as_complex(s.amps.view(-1, 2))


def overlap_with_product(psi, a, b):
    """<a (x) b | psi> with psi[i_b * 2^len(a) + i_a]; FP64 accumulation."""
    ta = torch.from_numpy(np.conj(a)).to(psi.device)
    tb = torch.from_numpy(np.conj(b)).to(psi.device)
    M = psi.view(len(b), len(a))
    acc = torch.zeros((), dtype=torch.complex128, device=psi.device)
    step = 256
    for r in range(0, len(b), step):
        blk = M[r:r + step].to(torch.complex128)
        acc += tb[r:r + step] @ (blk @ ta)
    return complex(acc.item())


@pytest.fixture(scope="module")
def cut_case(oracle):
    keep, low, high = factorised_grid()
    return keep, oracle.run(low), oracle.run(high)


@pytest.mark.parametrize("prec", ["plain", "tf32x3", "bf16x3"])
def test_grid30_factorised_vs_oracle(svlib, cut_case, prec):
    from paper_2106_13995_gb300 import _native as Nn
    keep, a, b = cut_case
    opts = None if prec == "plain" else svlib.options(
        prec=Nn.SV_PREC_TC_TF32X3 if prec == "tf32x3" else Nn.SV_PREC_TC_BF16X3)
    s = svlib.StateVector(N, "c64").set_basis(0)
    s.apply_circuit(keep, opts=opts)
    s.synchronize()
    psi = as_complex(s)
    ov = overlap_with_product(psi, a, b)
    n2 = s.norm2()
    one_minus_f = 1.0 - abs(ov) ** 2 / n2
    assert one_minus_f <= 1e-5, one_minus_f
    # seeded sample of amplitudes, each computed from the two oracle factors
    rng = np.random.default_rng(30)
    idx = rng.integers(0, 1 << N, size=1 << 16)
    got = psi[torch.from_numpy(idx).to(psi.device)].cpu().numpy().astype(np.complex128)
    want = a[idx & ((1 << CUT) - 1)] * b[idx >> CUT]
    err = float(np.max(np.abs(got - want)))
    rms = 2.0 ** (-N / 2)
    assert err <= 1e-3 * rms, err
    print(f"grid 30q cut ({prec}): 1-F {one_minus_f:.2e}, max |d psi| on 65536 samples {err:.2e} "
          f"(rms amplitude {rms:.2e})")
    s.close()


def inverse(circ, oracle):
    out = W.Circuit(circ.n_qubits, name=circ.name + "_inv")
    for op in reversed(circ.ops):
        U = oracle.gate_matrix(op.name, op.angles) if op.name != "MATRIX" else op.matrix
        out.ops.append(W.Op("MATRIX", op.targets, op.controls, matrix=np.conj(U).T.copy()))
    return out


def test_grid30_properties(svlib, oracle):
    from paper_2106_13995_gb300 import _native as Nn
    c = W.grid_random(ROWS, COLS, 20, 1)
    s = svlib.StateVector(N, "c64").set_basis(0).apply_circuit(c)
    assert abs(s.norm2() - 1) <= 1e-5
    z = s.z_all()
    assert np.all(np.abs(z) <= 1 + 1e-6)
    ref = as_complex(s)
    for prec in (Nn.SV_PREC_TC_TF32X3, Nn.SV_PREC_TC_BF16X3):
        t = svlib.StateVector(N, "c64").set_basis(0).apply_circuit(c, opts=svlib.options(prec=prec))
        t.synchronize()
        ov = torch.vdot(ref.to(torch.complex128), as_complex(t).to(torch.complex128)).item()
        f = abs(ov) ** 2 / (s.norm2() * t.norm2())
        assert 1 - f <= 1e-5, (prec, 1 - f)
        t.close()
    s.apply_circuit(inverse(c, oracle))
    p0 = abs(complex(ref[0].item())) ** 2
    assert p0 >= 1 - 1e-5, p0
    print(f"grid 30q: |<0|U^-1 U|0>|^2 = {p0:.8f}, norm {s.norm2():.8f}")
    s.close()


@pytest.mark.parametrize("n", [33, 34])
def test_largest_states_ghz(svlib, n):
    """The largest widths the library takes (34 qubits: 128 GiB of
    complex64): GHZ = H then a CNOT chain gives <Z_q> = 0 for every q (the
    reduction's branch for qubits 32 and up included, through the workspace
    path and the no-alloc entry point), norm 1, the two nonzero amplitudes
    1/sqrt(2), and samples only at 0 and 2^n - 1."""
    import ctypes as C
    import torch
    from paper_2106_13995_gb300 import _native as N
    free, _ = torch.cuda.mem_get_info()
    if free < (8 << n) + (8 << 30):
        pytest.skip("not enough device memory for this width")
    s = svlib.StateVector(n, "c64").set_basis(0)
    c = W.ghz(n)
    N.check(N.lib().sv_mark_modified(s.h))   # take the tile passes, not the basis-state path
    s.apply_circuit(c)
    z = s.z_all()
    assert np.max(np.abs(z)) <= 1e-6, np.max(np.abs(z))
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    N.check(N.lib().sv_expect_z_all_noalloc(C.c_void_p(s.amps.data_ptr()), n, N.SV_C64,
                                            C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)),
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy())) <= 1e-6
    assert abs(s.norm2() - 1) <= 1e-6
    r = float(np.float32(2 ** -0.5))
    assert s.amps[0].item() == r and s.amps[2 * ((1 << n) - 1)].item() == r
    shots = s.sample(2000, 3)
    assert set(shots.tolist()) <= {0, (1 << n) - 1} and 700 < int(np.sum(shots == 0)) < 1300
    s.close()
    del s
    torch.cuda.empty_cache()
