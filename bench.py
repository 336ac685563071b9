#!/usr/bin/env python
"""Throughput benchmark of the GB300 state-vector simulator.

Workload (one "step"): the 30-qubit 5x6 grid random circuit (20 cycles of
random sqrt(X)/sqrt(Y)/sqrt(W) layers and fSim(pi/2, pi/6) couplers in the
ABCDCDAB pattern, 845 gates) on a complex64 state of 2^30 amplitudes (8 GiB),
covering every step of the hot path: |0...0> initialisation, the fused and
tiled gate passes, <Z_q> for all qubits, a diagonal Pauli energy, the norm
and 1000 measurement samples.  value = gates/s over the whole job.

Also reported: e2e (the same step through the C ABI starting from a pinned
host state, host<->device copies inside the timed region), the roofline of the
dominant kernel (the tile pass), single-gate passes at 30 qubits per target,
adjoint gradients of the 20-qubit ansatz batched (64 parameter sets per
launch sequence) vs plain (one call per set), and the FP64 CPU oracle timed on
this host's cores.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "gates/s + HBM GB/s at 30q vs roofline; adjoint grads/s batched vs plain"
UNIT = "gates/s"
CSRC = os.path.join(ROOT, "paper_2106_13995_gb300", "csrc")
# the dominant kernel of each arithmetic mode, its sources and its ncu traffic record
KERNELS = {
    "plain": ("k_tile_inl (tile pass; op list and 1-3 qubit matrices in the parameter block)",
              ["k_tile.cu", "tile_ops.cuh"], "k_tile_traffic.json"),
    "bf16x3": ("k_tile_tcp (pipelined tile pass of split-BF16 tensor-core blocks)",
               ["k_tile_tcp.cu", "tile_ops.cuh"], "k_tile_tcp_traffic.json"),
    "tf32x3": ("k_tile_inl and k_dense_tc (tile passes and tensor-core passes)", [], None),
}


def traffic_of(prec: str, n: int):
    """DRAM bytes per launch from the ncu record, if it was taken on the
    current sources of the kernel and for this width; else None."""
    _, srcs, rec = KERNELS[prec]
    if not rec:
        return None
    try:
        with open(os.path.join(ROOT, "profiles", rec)) as f:
            tr = json.load(f)
        h = hashlib.sha256(b"".join(open(os.path.join(CSRC, x), "rb").read() for x in srcs)).hexdigest()[:16]
        if tr.get("k_tile_sha") == h and tr.get("n_qubits") == n:
            return tr["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--qubits", type=int, default=30,
                    help="30 = the 5x6 grid; fewer = the same grid with random qubits removed")
    ap.add_argument("--prec", choices=("plain", "bf16x3", "tf32x3"), default="bf16x3",
                    help="arithmetic of the main step's fused blocks: split-BF16 tensor-core blocks "
                         "(default), plain FP32 on CUDA cores, or split-TF32")
    ap.add_argument("--sections", default="all",
                    help="comma list of step,e2e,roofline,firstcall,tc,mult,single,adjoint,uneven,widths,cpu (default all)")
    return ap.parse_args()


def workload(nq: int):
    c = W.grid_random(5, 6, 20, seed=1)
    if nq < 30:
        c = W.remove_qubits(c, 30 - nq, seed=101)
    return c


def max_over_ranks(t: float, dist, device) -> float:
    """Slowest rank's time (every rank gets it)."""
    import torch
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(units_per_rank: float, world: int, t: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time
    (replicas: every rank processes the same fixed work)."""
    return units_per_rank * world / t


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


def measured_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except Exception:
        return 1900.0, "fallback (1.9 PFLOP/s bf16 burst)"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on host cores (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def numa_nodes_with_cpus():
    """{node: set of CPUs} for the host's NUMA nodes that have CPUs."""
    out = {}
    base = "/sys/devices/system/node"
    try:
        names = sorted(x for x in os.listdir(base) if x.startswith("node") and x[4:].isdigit())
    except OSError:
        return out
    for name in names:
        try:
            txt = open(f"{base}/{name}/cpulist").read().strip()
        except OSError:
            continue
        cpus = set()
        for part in filter(None, txt.split(",")):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if cpus:
            out[int(name[4:])] = cpus
    return out


def pin_to_fastest_host_node(torch, dev):
    """Restrict this process to the CPUs of the NUMA node whose pinned memory
    copies to the GPU fastest (a 256 MiB probe per node: sysfs does not
    always name the node a GPU is attached to), so host buffers allocated
    next land there.  Returns (node, {node: probe GB/s}); the caller restores
    the affinity after allocating."""
    nodes = numa_nodes_with_cpus()
    if not nodes:
        return None, {}
    rates = {}
    dst = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    for node, cpus in nodes.items():
        try:
            os.sched_setaffinity(0, cpus)
            buf = torch.ones(64 << 20, dtype=torch.float32, pin_memory=True)
            dst.copy_(buf, non_blocking=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                dst.copy_(buf, non_blocking=True)
            torch.cuda.synchronize()
            rates[node] = 3 * buf.numel() * 4 / (time.perf_counter() - t0) / 1e9
            del buf
        except Exception:
            continue
    del dst
    if not rates:
        return None, {}
    best = max(rates, key=rates.get)
    os.sched_setaffinity(0, nodes[best])
    return best, {str(k): round(v, 1) for k, v in rates.items()}


def oracle_sample(circ, budget_s: float, max_gates=None):
    """Apply the circuit's gates one by one with the FP64 oracle to a 2^n
    complex128 state until the time budget is spent.  Returns (gates/s,
    gates done, seconds, threads, n)."""
    import oracle
    oracle.build()
    n = circ.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1
    done, t0 = 0, time.perf_counter()
    for op in circ.ops:
        oracle.run_inplace(W.Circuit(n, [op]), psi)
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_gates and done >= max_gates):
            break
    el = time.perf_counter() - t0
    return done / el, done, el, oracle.num_threads(), n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    circ = workload(args.qubits)
    # warm-up then timed steps; each step applies the first 4 gates of the
    # circuit with the FP64 oracle to a fresh 2^n complex128 state
    per_step = 4
    times = []
    for i in range(args.warmup + args.steps):
        gs, done, el, thr, n = oracle_sample(circ, 1e9, max_gates=per_step)
        if i >= args.warmup:
            times.append(el)
    total = sum(times)
    value = per_step * len(times) / total
    sample = f"first {per_step} gates of the {circ.n_qubits}-qubit grid circuit per step, FP64 oracle, complex128 state"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_of(circ, args),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def config_of(circ, args):
    return {"workload": f"grid random circuit 5x6 lattice (30 qubits{'' if circ.n_qubits == 30 else f', {30 - circ.n_qubits} removed'}),"
                        f" 20 cycles, {len(circ.ops)} gates, complex64 state",
            "n_qubits": circ.n_qubits, "gates": len(circ.ops), "state_dtype": "complex64",
            "state_bytes": (1 << circ.n_qubits) * 8,
            "l2": (f"inputs larger than L2: the state is {(1 << circ.n_qubits) * 8 / 2**20:.0f} MiB (L2 129 MB)"
                   if circ.n_qubits >= 25 else "state smaller than L2"),
            "parallelism": f"replicas x{args.gpus}"}


# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_2106_13995_gb300 as P
    if rank == 0:
        P.build()
    if world > 1:
        dist.barrier()
    from paper_2106_13995_gb300 import sim

    sections = set(args.sections.split(",")) if args.sections != "all" else \
        {"step", "e2e", "roofline", "firstcall", "tc", "mult", "single", "adjoint", "uneven", "widths", "cpu"}
    circ = workload(args.qubits)
    n = circ.n_qubits
    m = sim.marshal(circ)
    stream = torch.cuda.current_stream(dev)
    state = sim.StateVector(n, "c64", device=dev)
    from paper_2106_13995_gb300 import _native as NN
    step_opts = None if args.prec == "plain" else sim.options(
        prec=NN.SV_PREC_TC_BF16X3 if args.prec == "bf16x3" else NN.SV_PREC_TC_TF32X3)
    zz = [(0, (1 << a) | (1 << b), 1.0) for pat in W.grid_couplers(5, 6).values() for a, b in pat
          if a < n and b < n]
    shots = np.zeros(1000, dtype=np.uint64)

    def step():
        state.set_basis(0)
        state.apply_circuit(m, opts=step_opts)
        z = state.z_all()
        e = state.expect(zz)
        nrm = state.norm2()
        s = state.sample(1000, 7)
        return z, e, nrm, s

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        if world > 1:
            t = max_over_ranks(t, dist, dev)
        return t

    out = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": config_of(circ, args)}
    nblocks, npasses = state.plan_info(m, opts=step_opts)
    out["config"]["prec"] = args.prec
    out["config"]["arithmetic"] = {
        "bf16x3": "complex64 state; fused blocks of up to 5 qubits on the tensor cores as split-BF16 "
                  "(hi*hi + hi*lo + lo*hi), FP32 accumulation",
        "plain": "complex64 state; fused blocks of up to 3 qubits in FP32 on the CUDA cores",
        "tf32x3": "complex64 state; 5-qubit blocks on the tensor cores as split-TF32, FP32 accumulation"}[args.prec]
    out["config"]["fused_blocks"] = nblocks
    out["config"]["tile_passes"] = npasses

    # ---- main timed region ----------------------------------------------------
    for _ in range(args.warmup):
        step()
    l0 = sim.kernel_launches()
    with ClockSampler(local) as clk:
        t = timed(step, args.steps)
    launches = sim.kernel_launches() - l0
    out["value"] = job_value(len(circ.ops) * args.steps, world, t)
    out["ms_per_step"] = 1e3 * t / args.steps
    out["gpu_launches"] = int(launches)
    out["clocks"] = clk.summary()
    gate_bytes = 2 * (1 << n) * 8
    out["hbm_gbs_effective"] = len(circ.ops) * gate_bytes * args.steps / t / 1e9

    # ---- end to end through the C ABI from host buffers -----------------------
    if "e2e" in sections:
        aff = os.sched_getaffinity(0)
        numa, probe = pin_to_fastest_host_node(torch, dev)   # pinned pages land on that node
        host = torch.zeros(2 << n, dtype=torch.float32, pin_memory=True)
        os.sched_setaffinity(0, aff)
        host[0] = 1.0
        hp = host.data_ptr()

        def step_e2e():
            from paper_2106_13995_gb300 import _native as N
            N.check(N.lib().sv_upload(state.h, hp, state.nbytes))
            state.apply_circuit(m, opts=step_opts)
            z = state.z_all()
            e = state.expect(zz)
            s = state.sample(1000, 7)
            return z, e, s

        for _ in range(max(1, args.warmup)):
            step_e2e()
        ke = max(2, args.steps // 2)
        te = timed(step_e2e, ke)

        def upload_only():
            from paper_2106_13995_gb300 import _native as N
            N.check(N.lib().sv_upload(state.h, hp, state.nbytes))

        tu = timed(upload_only, 2) / 2
        out["e2e"] = {"value": len(circ.ops) * ke * world / te, "unit": UNIT,
                      "h2d_bytes_per_step": state.nbytes, "d2h_bytes_per_step": 8 * n + 8 + 8 * 1000,
                      "ms_per_step": 1e3 * te / ke, "h2d_gbs": state.nbytes / tu / 1e9,
                      "host_numa_node": numa, "h2d_probe_gbs_by_node": probe}
        del host

    # ---- roofline of the dominant kernel (the tile pass) -----------------------
    peak, peak_src = measured_peaks()
    if "roofline" in sections:
        reps = max(2, args.steps // 2)
        state.set_basis(0)
        tc = timed(lambda: state.apply_circuit(m, opts=step_opts), reps) / reps
        per_launch = tc / npasses
        achieved = gate_bytes / per_launch / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "traffic": traffic_of(args.prec, n),
                           "kernel": KERNELS[args.prec][0],
                           "algorithmic_bytes_per_launch": gate_bytes, "launches_per_circuit": npasses,
                           "avg_launch_ms": per_launch * 1e3, "circuit_ms": tc * 1e3, "peak_source": peak_src}
        if args.prec == "bf16x3":
            # the same passes against the tensor pipe: each 5-qubit block is a
            # (2^n/32 x 64) x (64 x 64) real GEMM done as three BF16 products,
            # 3 x 2 x 64 x 64 / 32 = 768 flops per amplitude; peak = the
            # measured dense BF16 rate (burst)
            fmas = state.plan_fmas(m, opts=step_opts)       # 128 per amplitude per 5-qubit block
            flops = 3 * 2 * fmas * (1 << n)
            tpeak, tsrc = measured_bf16()
            out["roofline_tensor"] = {"bound": "tensor", "achieved": flops / tc / 1e12, "peak": tpeak,
                                      "unit": "TFLOP/s", "frac": flops / tc / 1e12 / tpeak,
                                      "flops_per_circuit": flops, "blocks": nblocks, "peak_source": tsrc}
        # the same circuit with CUDA-core FP32 arithmetic (k_tile_inl), for comparison
        popts = sim.options()
        nb_p, np_p = state.plan_info(m, opts=popts)
        state.set_basis(0)
        state.apply_circuit(m, opts=popts)
        tp_ = timed(lambda: state.apply_circuit(m, opts=popts), reps) / reps
        fmas_p = state.plan_fmas(m, opts=popts)
        mhz = out["clocks"].get("sm_max_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        out["plain_fp32"] = {"circuit_ms": tp_ * 1e3, "gates_per_s": len(circ.ops) / tp_, "passes": np_p,
                             "blocks": nb_p, "avg_launch_ms": tp_ / np_p * 1e3,
                             "hbm_frac": gate_bytes / (tp_ / np_p) / 1e9 / peak,
                             "traffic": traffic_of("plain", n), "kernel": KERNELS["plain"][0],
                             # after fusion a CUDA-core pass does tens of multiply-adds per
                             # amplitude it moves: flops = 2 x planned multiply-adds x 2^n
                             "alu": {"bound": "alu", "achieved": 2 * fmas_p * (1 << n) / tp_ / 1e12,
                                     "peak": alu_peak, "unit": "TFLOP/s",
                                     "frac": 2 * fmas_p * (1 << n) / tp_ / 1e12 / alu_peak,
                                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz"}}

    # ---- first call of a new circuit: planning, upload, first run -----------------
    if "firstcall" in sections:
        from paper_2106_13995_gb300 import _native as NF
        fresh = sim.StateVector(n, "c64", device=dev)   # its own program cache entries
        fresh.set_basis(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fresh.plan_info(m, opts=step_opts)                # fusion and pass planning only
        t_plan = time.perf_counter() - t0
        fresh2 = sim.StateVector(n, "c64", device=dev)
        fresh2.set_basis(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fresh2.apply_circuit(m, opts=step_opts)           # plan + upload + run
        torch.cuda.synchronize()
        t_first = time.perf_counter() - t0
        t0 = time.perf_counter()
        fresh2.apply_circuit(m, opts=step_opts)           # cached program
        torch.cuda.synchronize()
        t_again = time.perf_counter() - t0
        out["first_call"] = {"plan_ms": 1e3 * t_plan, "first_apply_ms": 1e3 * t_first,
                             "cached_apply_ms": 1e3 * t_again,
                             "note": "wall clock on the host around one call each; planning fuses the gates "
                                     "(FP64 block products), plans the tile passes and packs the operands"}
        fresh.close()
        fresh2.close()
        del fresh, fresh2
        torch.cuda.empty_cache()

    # ---- the same circuit with fused 5-qubit blocks on the tensor cores ----------
    if "tc" in sections:
        # accuracy of each mode against the plain FP32 path on the same 30-qubit
        # circuit: 1 - |<psi_plain|psi_tc>|^2 / (|psi_plain|^2 |psi_tc|^2), FP64
        ref = sim.StateVector(n, "c64", device=dev)
        ref.set_basis(0)
        ref.apply_circuit(m)

        def infid(a, b):
            va = torch.view_as_complex(a.amps.view(-1, 2))
            vb = torch.view_as_complex(b.amps.view(-1, 2))
            ov = torch.zeros((), dtype=torch.complex128, device=dev)
            na = torch.zeros((), dtype=torch.float64, device=dev)
            nb = torch.zeros((), dtype=torch.float64, device=dev)
            step_ = 1 << 26
            for i in range(0, va.numel(), step_):
                x = va[i:i + step_].to(torch.complex128)
                y = vb[i:i + step_].to(torch.complex128)
                ov += torch.vdot(x, y)
                na += (x.abs() ** 2).sum()
                nb += (y.abs() ** 2).sum()
            return float(1 - abs(ov.item()) ** 2 / (na.item() * nb.item()))

        modes = {}
        arrangement = {"tf32x3": "5-qubit blocks as tensor-core passes of their own between tile passes",
                       "bf16x3": "5-qubit blocks on the tensor cores inside 12-qubit tile passes"}
        for name, code in (("tf32x3", NN.SV_PREC_TC_TF32X3), ("bf16x3", NN.SV_PREC_TC_BF16X3)):
            o = sim.options(prec=code)
            nb_, np_ = state.plan_info(m, opts=o)
            state.set_basis(0)
            state.apply_circuit(m, opts=o)
            torch.cuda.synchronize()
            one_minus_f = infid(ref, state)
            reps = max(2, args.steps // 2)
            t_ = timed(lambda: state.apply_circuit(m, opts=o), reps) / reps
            modes[name] = {"gates_per_s": len(circ.ops) / t_, "ms_per_circuit": 1e3 * t_, "fused_blocks": nb_,
                           "passes": np_, "arrangement": arrangement[name],
                           "one_minus_fidelity_vs_plain_fp32": one_minus_f,
                           "hbm_gbs_effective": len(circ.ops) * gate_bytes / t_ / 1e9}
        ref.close()
        out["tensor_core_modes"] = modes

    # ---- 29-qubit quantum multiplier: 64 basis inputs, then superposed inputs ---
    if "mult" in sections:
        mc = W.multiplier(7)
        mh = W.multiplier(7, hadamard_inputs=True)
        mmc, mmh = sim.marshal(mc), sim.marshal(mh)
        rng = np.random.default_rng(2)
        ab = rng.integers(0, 128, size=(64, 2))
        del_state = state
        ms_ = sim.StateVector(29, "c64", device=dev)

        from paper_2106_13995_gb300 import _native as NM

        def mult_all(dense: bool):
            for a_, b_ in ab:
                ms_.set_basis(W.multiplier_basis_index(int(a_), int(b_), 7))
                if dense:   # forget the basis state: tile passes of permutation ops
                    NM.check(NM.lib().sv_mark_modified(ms_.h))
                ms_.apply_circuit(mmc)

        mult_all(True)
        tm_ = timed(lambda: mult_all(True), 1)
        mult_all(False)
        tf_ = timed(lambda: mult_all(False), 1)
        ms_.set_basis(0)
        ms_.apply_circuit(mmh)
        th_ = timed(lambda: (ms_.set_basis(0), ms_.apply_circuit(mmh)), 2) / 2
        out["multiplier"] = {"n_qubits": 29, "native_ops": len(mc.ops), "basis_runs": 64,
                             "runs_per_s": 64 / tm_, "gates_per_s": 64 * len(mc.ops) / tm_,
                             "path": "tile passes composed into permutation tables (one move per amplitude, no arithmetic)",
                             "basis_fast_path": {"runs_per_s": 64 / tf_, "gates_per_s": 64 * len(mc.ops) / tf_,
                                                 "path": "basis state followed on the host, two amplitudes "
                                                         "rewritten; each run includes the 4 GiB basis-state "
                                                         "write of sv_set_basis"},
                             "superposed_run_ms": 1e3 * th_, "passes": ms_.plan_info(mmc)[1]}
        ms_.close()
        del del_state

    # ---- single-gate passes per target (K1-K3) ---------------------------------
    if "single" in sections:
        # one 1-qubit gate pass per target q = 0..n-1 (K1 for q = 0, K2 for the
        # shuffle range, K3 above), complex64 on the bench state and complex128
        # on a second 2^n state
        U = W.random_unitary(1, np.random.default_rng(0))
        res = {}
        for dt, st_, bpa in (("c64", state, 8), ("c128", None, 16)):
            if st_ is None:
                st_ = sim.StateVector(n, dt, device=dev)
                st_.set_basis(0)
            gb_ = 2 * (1 << n) * bpa
            gbs = {}
            for q in range(n):
                st_.apply_gate(U, [q])
                tq = timed(lambda: st_.apply_gate(U, [q]), 4) / 4
                gbs[q] = gb_ / tq / 1e9
            vals = list(gbs.values())
            res[dt] = {"gbs_by_target": {str(k): round(v, 1) for k, v in gbs.items()},
                       "min_gbs": min(vals), "mean_gbs": statistics.mean(vals),
                       "min_frac_of_measured": min(vals) / peak, "mean_frac_of_measured": statistics.mean(vals) / peak,
                       "gates_per_s_min": min(vals) * 1e9 / gb_}
            if dt == "c128":
                st_.close()
                del st_
                torch.cuda.empty_cache()
        out["single_gate_pass"] = res["c64"]
        out["single_gate_pass_c128"] = res["c128"]

    # ---- adjoint gradients, batched vs plain (20-qubit ansatz, 64 sets) ----------
    if "adjoint" in sections:
        del state
        torch.cuda.empty_cache()
        na, B = 20, 64
        h = W.hea(na, 10)
        hm = sim.marshal(h)
        terms = W.tfim(na)
        params = W.hea_params(B, h.n_params, 3)
        psis = [sim.StateVector(na, "c64", device=dev).set_basis(0) for _ in range(B)]
        lams = [sim.StateVector(na, "c64", device=dev) for _ in range(B)]

        gopt = sim.options(mode=NN.SV_MODE_TILED_GRAPH)

        def batched():   # one replayed launch sequence per call
            for p in psis:
                p.set_basis(0)
            return sim.adjoint_grad_batch(psis, lams, hm, params, terms, opts=gopt)

        def plain():
            for b in range(B):
                psis[b].set_basis(0)
                sim.adjoint_grad(psis[b], lams[b], hm, params[b], terms)

        for _ in range(max(1, args.warmup)):
            batched()
        plain()
        kb = max(2, args.steps // 2)
        tb = timed(batched, kb) / kb
        tp = timed(plain, 1)
        out["adjoint"] = {"grads_per_s_batched": B / tb, "grads_per_s_plain": B / tp,
                          "speedup": tp / tb, "batch": B, "n_qubits": na, "gates": len(h.ops),
                          "params": h.n_params, "state": "complex64, FP64 reductions",
                          "batched_launch": "64 parameter sets per call; the accumulator reset and every pass "
                                            "replayed from one CUDA graph (SV_MODE_TILED_GRAPH)"}
        del psis, lams

    # ---- uneven batch: 256 circuits of widths 10..24, one persistent launch -------
    if "uneven" in sections:
        import ctypes as C
        from paper_2106_13995_gb300 import _native as N
        torch.cuda.empty_cache()
        circs = W.uneven_batch()
        ums = [sim.marshal(c) for c in circs]
        ust = [sim.StateVector(c.n_qubits, "c64", device=dev) for c in circs]
        hs = (C.c_void_p * len(ust))(*[s.h.value for s in ust])
        cs = (C.POINTER(N.SvCircuit) * len(ust))(*[C.pointer(mm.c) for mm in ums])
        gopt = sim.options(mode=N.SV_MODE_TILED_GRAPH)

        def uneven_batched():
            for st_ in ust:
                st_.set_basis(0)
            N.check(N.lib().sv_apply_circuit_batch(hs, len(ust), cs, None, C.byref(gopt)))

        def uneven_plain():
            for st_, mm in zip(ust, ums):
                st_.set_basis(0)
                st_.apply_circuit(mm)

        for _ in range(max(1, args.warmup)):
            uneven_batched()
            uneven_plain()
        N.check(N.lib().sv_synchronize(ust[0].h))
        ku = max(2, args.steps // 2)
        tbu = timed(uneven_batched, ku) / ku
        N.check(N.lib().sv_synchronize(ust[0].h))
        tpu = timed(uneven_plain, ku) / ku
        # the same batched call with split-BF16 tensor-core blocks: states of
        # 12 or more qubits run the pipelined tensor-core tile passes inside
        # the same recorded launch sequence, the smaller ones the persistent
        # queue
        gopt_tc = sim.options(mode=N.SV_MODE_TILED_GRAPH, prec=N.SV_PREC_TC_BF16X3)

        def uneven_batched_tc():
            for st_ in ust:
                st_.set_basis(0)
            N.check(N.lib().sv_apply_circuit_batch(hs, len(ust), cs, None, C.byref(gopt_tc)))

        def uneven_plain_tc():
            for st_, mm in zip(ust, ums):
                st_.set_basis(0)
                st_.apply_circuit(mm, opts=sim.options(prec=N.SV_PREC_TC_BF16X3))

        uneven_batched_tc()
        uneven_plain_tc()
        N.check(N.lib().sv_synchronize(ust[0].h))
        tbu_tc = timed(uneven_batched_tc, ku) / ku
        N.check(N.lib().sv_synchronize(ust[0].h))
        tpu_tc = timed(uneven_plain_tc, ku) / ku
        # fused 5-qubit blocks on the tensor cores (split-BF16 / split-TF32)
        # vs plain complex64 per-gate passes, same batch; accuracy of each
        # against the plain tiled complex64 result (the FP64-oracle errors
        # are measured by the test suite)
        modes = {"tiled_plain": sim.options(), "tc_bf16x3": sim.options(prec=N.SV_PREC_TC_BF16X3),
                 "tc_tf32x3": sim.options(prec=N.SV_PREC_TC_TF32X3),
                 "per_gate_plain": sim.options(fusion_k=1, mode=N.SV_MODE_PER_GATE)}
        # autotuned fusion width and tile size, one sv_autotune per distinct width
        tuned = {}
        for i, c in enumerate(circs):
            if c.n_qubits not in tuned:
                o_ = sim.options()
                N.check(N.lib().sv_autotune(ust[i].h, ums[i].ref(), C.byref(o_)))
                tuned[c.n_qubits] = o_
        modes["autotuned"] = None
        ref_idx = [i for i, c in enumerate(circs) if c.n_qubits in (14, 18, 22)][:6]
        ref_states = {}
        per_mode = {}
        for name, mo in modes.items():
            def run_mode(mo=mo):
                for st_, mm, c in zip(ust, ums, circs):
                    st_.set_basis(0)
                    st_.apply_circuit(mm, opts=mo if mo is not None else tuned[c.n_qubits])
            run_mode()
            tm_ = timed(run_mode, 1)
            outs = {i: ust[i].numpy().astype(np.complex128) for i in ref_idx}
            if name == "tiled_plain":
                ref_states = outs
            errs = []
            for i in ref_idx:
                a, b_ = ref_states[i], outs[i]
                f = abs(np.vdot(a, b_)) ** 2 / (np.vdot(a, a).real * np.vdot(b_, b_).real)
                errs.append(max(0.0, 1.0 - f))
            per_mode[name] = {"circuits_per_s": len(circs) / tm_, "max_1mF_vs_tiled_c64": max(errs),
                              "median_1mF_vs_tiled_c64": statistics.median(errs)}
        per_mode["autotuned"]["choices"] = {str(k): [v.fusion_k, v.tile_m] for k, v in sorted(tuned.items())}
        out["uneven_batch"] = {"circuits_per_s_batched": len(circs) / tbu, "circuits_per_s_plain": len(circs) / tpu,
                               "speedup": tpu / tbu, "per_circuit_modes": per_mode,
                               "bf16x3": {"circuits_per_s_batched": len(circs) / tbu_tc,
                                          "circuits_per_s_per_circuit": len(circs) / tpu_tc,
                                          "speedup": tpu_tc / tbu_tc},
                               "circuits": len(circs), "widths": "10..24", "depth": 40,
                               "gates": int(sum(len(c.ops) for c in circs)),
                               "launch": "one CUDA graph per call: a persistent cooperative launch for states "
                                         "whose passes have fewer tiles than SMs, full-grid tile launches for the "
                                         "wider ones; plus one basis-state write per state"}
        del ust

    # ---- width sweep (Sec. II: random qubit removal from the 5x6 grid) ------------
    if "widths" in sections:
        sweep = {}
        for nw in range(14, 31):
            cw = W.grid_random(5, 6, 20, 1) if nw == 30 else W.remove_qubits(W.grid_random(5, 6, 20, 1), 30 - nw, 101)
            mw = sim.marshal(cw)
            sw = sim.StateVector(nw, "c64", device=dev)
            sw.set_basis(0)
            sw.apply_circuit(mw, opts=step_opts)
            nbw, npw = sw.plan_info(mw, opts=step_opts)
            kw = 3
            tw = timed(lambda: (sw.set_basis(0), sw.apply_circuit(mw, opts=step_opts)), kw) / kw
            sweep[str(nw)] = {"gates": len(cw.ops), "passes": npw, "ms": 1e3 * tw,
                              "gates_per_s": len(cw.ops) / tw,
                              "hbm_gbs_effective": len(cw.ops) * 2 * (1 << nw) * 8 / tw / 1e9}
            sw.close()
            del sw
        torch.cuda.empty_cache()
        out["width_sweep"] = sweep

    # ---- the FP64 oracle on this host's cores ------------------------------------
    if "cpu" in sections and rank == 0:
        try:
            gs, done, el, thr, nn = oracle_sample(circ, 15.0)
            # the same oracle on one core, two gates
            import oracle
            oracle.set_num_threads(1)
            gs1, done1, el1, _, _ = oracle_sample(circ, 1e9, max_gates=2)
            oracle.set_num_threads(thr)
            gb_gate = 2 * (1 << nn) * 16 / 1e9
            out["cpu_baseline"] = {"value": gs, "unit": UNIT, "cores": thr, "kind": "oracle",
                                   "sample": f"first {done} of {len(circ.ops)} gates of the same {nn}-qubit circuit "
                                             f"on a complex128 state, {el:.1f} s",
                                   "gbs": gs * gb_gate,
                                   "single_core": {"value": gs1, "unit": UNIT, "gbs": gs1 * gb_gate,
                                                   "sample": f"first {done1} gates, {el1:.1f} s"}}
        except MemoryError:
            out["cpu_baseline"] = None

    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
