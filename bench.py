#!/usr/bin/env python3
"""Benchmark: gradient evaluations per second of the 20-qubit VQE workload on GB300.

One step = one energy + full gradient evaluation (800 parameters) of the 20-qubit,
20-layer Ry.Rz + CZ-brick ansatz with the 39-term transverse-field Ising Hamiltonian:
gate materialisation, state initialisation, fused forward tile passes, expectation
fused with the adjoint seed, fused reverse passes (Algorithm 2) and the gradient
reduction, in complex64 with FP64 reductions.  The tile passes are the circuit's
specialised kernels (GBVQC_MODE_JIT, compiled during set-up, outside the timed region).
Inputs (parameters) are resident on the device; L2 (129 MB) is flushed by writing a
256 MiB buffer between timed steps.

Also reported: the end-to-end rate through the host-pointer C-ABI call, the record
interpreter (GBVQC_MODE_FUSED) and complex128 on the same workload, the plain per-gate
complex128 path, the 10-qubit plain complex128 configuration, the gate-sweep HBM
bandwidth of the 28-qubit random circuit (tile passes vs one launch per gate, both
precisions), the 512-instance batch, the 13-qubit noisy density matrix (both
precisions), the dominant kernel's roofline, clocks sampled during the timed region,
and the FP64 CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank runs an independent replica (the single-state path
does not shard); value = evaluations of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gradient evals/s (20q VQE) and gate-sweep HBM GB/s vs plain per-gate path"
UNIT = "gradient evals/s"
WORKLOAD = ("vqe_20q_hea20: 20 qubits, 20 layers of Ry.Rz on every qubit + CZ brick, "
            "800 angles U[0,2pi), H = sum Z_iZ_i+1 + sum X_i (39 terms), energy + full gradient")
FLUSH_BYTES = 256 << 20


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_tflops(sm_mhz: float, sms: int) -> float:
    """FP32 CUDA-core peak: SMs (read from the device) x 128 FP32 lanes x 2 flops (FMA) x
    SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gbvqc_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


KERNEL_SOURCES = ("fused_tile.cuh", "devmath.cuh", "common.cuh", "kernels_fused.cu", "jit.cpp", "planner.cpp",
                  "api_circuit.cu")


def kernel_src_sha() -> str:
    """Hash of the sources that define the fused tile kernels."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2406_19212_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        sha = kernel_src_sha()
        for r in rec.get("kernels", []):
            if r.get("kernel") == kernel and r.get("src_sha") == sha:
                return r.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------- oracle legs

def oracle_grad_rate(budget_s: float):
    """FP64 CPU oracle on the same workload: a full gradient evaluation if it fits the
    budget, else the first L layers (cost is linear in layers) extrapolated."""
    from oracle import oracle as O
    from paper_2406_19212_gb300 import inputs as I
    w = I.diff_20q()
    w1 = I.hea_ry_rz_cz(20, 1, 2, 1.0)
    t0 = time.perf_counter()
    O.adjoint_grad(w1.circuit, w1.theta, w1.observable)
    t_layer = time.perf_counter() - t0
    layers = int(max(1, min(20, budget_s // max(t_layer, 1e-9))))
    if layers >= 20:
        t0 = time.perf_counter()
        O.adjoint_grad(w.circuit, w.theta, w.observable)
        dt = time.perf_counter() - t0
        sample = "1 full gradient evaluation (20 layers, 800 parameters)"
        return 1.0 / dt, sample, O.num_threads()
    ws = I.hea_ry_rz_cz(20, layers, 2, 1.0)
    t0 = time.perf_counter()
    O.adjoint_grad(ws.circuit, ws.theta, ws.observable)
    dt = time.perf_counter() - t0
    sample = (f"gradient of the first {layers} of 20 layers (same 20 qubits and H), "
              f"extrapolated linearly in layers to one full evaluation")
    return (layers / 20.0) / dt, sample, O.num_threads()


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_grad_rate(budget)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, sample, cores = oracle_grad_rate(budget)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = statistics.mean(rates)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (plain C, OpenMP)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ our arm

def run_ours(args, world, rank, local):
    import torch
    import paper_2406_19212_gb300 as gb
    from paper_2406_19212_gb300 import build as gbuild
    from paper_2406_19212_gb300 import inputs as I

    torch.cuda.set_device(local)
    gbuild.build()
    pk, pk_kind = peaks()
    w = I.diff_20q()
    circ = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, w.circuit.n_qubits)
    os.environ.setdefault("GBVQC_TUNE_CACHE", "off")
    tile, low, tune_ms = circ.autotune(w.theta, obs, gb.C64)   # set-up, outside the timed region
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream(dev)
    theta = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    e_out = torch.empty(1, dtype=torch.float64, device=dev)
    g_out = torch.empty(w.circuit.n_params, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    spec = circ.specialize(gb.C64, True)   # compile the specialised passes (set-up)
    gb.grad(circ, theta, obs, gb.C64, gb.JIT, stream=stream, out=(e_out, g_out))   # load them
    torch.cuda.synchronize()
    spec["setup_s"] = time.perf_counter() - t0
    MODE = gb.JIT

    def step():
        gb.grad(circ, theta, obs, gb.C64, MODE, stream=stream, out=(e_out, g_out))

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # kernel-level profile of one evaluation (CUDA events on the launching stream)
    prof = gb.grad_profile(circ, w.theta, obs, gb.C64, MODE, stream=stream)
    # the profile times the passes alone; a step also forks one code-prefetch launch per
    # specialised pass (two directions, no barrier passes in this circuit)
    prefetch_launches = 2 * circ.plan_stats(gb.C64, True)["passes"] if MODE == gb.JIT else 0
    launches_per_step = sum(v[0] for v in prof.values()) + prefetch_launches

    # timed region: per-step events, L2 flushed between steps outside the events
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.nvtx.range_push("bench_timed")   # lets ncu restrict a capture to the timed steps
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = max_over_ranks(world, sum(step_ms) / 1e3)
    value = args.steps * world / total_s
    ms_per_step = 1e3 * total_s / args.steps

    # end to end through the host-pointer C-ABI call (H2D theta, D2H energy + gradient)
    # (theta, energy and gradient in pinned host buffers)
    n_e2e = max(5, min(args.steps, 200))
    theta_host = torch.from_numpy(np.ascontiguousarray(w.theta)).pin_memory().numpy()
    e_host = torch.empty(1, dtype=torch.float64).pin_memory().numpy()
    g_host = torch.empty(w.circuit.n_params, dtype=torch.float64).pin_memory().numpy()
    gb.grad(circ, theta_host, obs, gb.C64, MODE, out=(e_host, g_host))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        gb.grad(circ, theta_host, obs, gb.C64, MODE, out=(e_host, g_host))
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": n_e2e * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 8 * w.circuit.n_params,
           "d2h_bytes_per_step": 8 * (1 + w.circuit.n_params)}

    out = {}
    if rank == 0:
        # dominant kernel roofline
        name, (nl, ms, fl, by) = max(prof.items(), key=lambda kv: kv[1][1])
        avg_s = ms / nl / 1e3
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        alu = alu_peak_tflops(sm_mhz, sms)
        hbm = pk["hbm_gbs"]
        intensity = fl / by if by else 0.0
        ridge = alu * 1e12 / (hbm * 1e9)
        traffic = traffic_for(name)
        if intensity > ridge:
            roof = {"bound": "alu", "achieved": fl / nl / avg_s / 1e12, "peak": alu,
                    "unit": "TFLOP/s"}
            roof["peak_note"] = (f"FP32 CUDA cores: {sms} SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz "
                                 f"(derived; HBM {hbm:.0f} GB/s {pk_kind})")
        else:
            roof = {"bound": "hbm", "achieved": by / nl / avg_s / 1e9, "peak": hbm, "unit": "GB/s",
                    "peak_note": f"{pk_kind} copy bandwidth"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["traffic"] = traffic
        roof["kernel"] = name
        roof["launches_per_step"] = nl
        roof["avg_launch_us"] = avg_s * 1e6
        roof["alg_flops_per_launch"] = fl / nl
        roof["alg_bytes_per_launch"] = by / nl
        roof["hbm_frac_of_alg_bytes"] = by / nl / avg_s / 1e9 / hbm
        out["roofline"] = roof
        out["kernels"] = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in prof.items()}

    if rank == 0 and not args.no_extra:
        def rate(dtype, mode, reps):
            gb.grad(circ, theta, obs, dtype, mode, stream=stream, out=(e_out, g_out))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                gb.grad(circ, theta, obs, dtype, mode, stream=stream, out=(e_out, g_out))
            torch.cuda.synchronize()
            return reps / (time.perf_counter() - t0)
        # the same workload through the record interpreter, in complex128, and per gate
        out["interpreter_c64"] = {"value": rate(gb.C64, gb.FUSED, 50), "unit": UNIT,
                                  "mode": "fused tile passes, record interpreter (GBVQC_MODE_FUSED)"}
        circ.specialize(gb.C128, True)
        out["jit_c128"] = {"value": rate(gb.C128, gb.JIT, 20), "unit": UNIT,
                           "mode": "specialised tile passes, complex128 sweeps"}
        plain_rate = rate(gb.C128, gb.PLAIN, 3)
        out["plain_c128"] = {"value": plain_rate, "unit": UNIT,
                             "speedup_fused_c64": value / world / plain_rate}
        out["plain_10q"] = plain10_rate(gb, I, torch, dev, stream)
        out["sweep"] = gate_sweep(gb, I, torch, dev, stream, pk)
        out["batch"] = batch_rate(gb, I, torch)
        out["noisy"] = noisy_rate(gb, I, torch)
        out["heisenberg"] = heisenberg_rate(gb, I, torch, dev, stream)
    if rank == 0:
        if not args.no_cpu:
            rate, sample, cores = oracle_grad_rate(25.0)
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": sample}
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "qubits": 20, "params": w.circuit.n_params,
                       "mode": "specialised fused tile passes (GBVQC_MODE_JIT), CUDA-graph replay, "
                               "device pointers",
                       "specialised": spec,
                       "tiling": {"tile_qubits": tile, "low_qubits": low, "autotuned": True},
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clk}
    line.update(out)
    print(json.dumps(line), flush=True)
    return 0


def gate_sweep(gb, I, torch, dev, stream, pk, rows=4, cols=7):
    """Random circuit on a rows x cols grid (20 cycles; 4x7 = 28 qubits) applied in
    complex64 and complex128: specialised tile passes, the record interpreter's tile
    passes and one launch per gate; GB/s = algorithmic bytes (one read + one write of the
    state per pass or per gate) / time."""
    n = rows * cols
    w = I.grid_rqc(rows, cols, 20, 1)
    circ = gb.circuit_create(w.circuit)
    res = {"workload": f"rqc_{rows}x{cols}_c20: {n} qubits, 20 cycles of sqrt(X/Y/W) + FSIM couplers, "
                       f"{len(w.circuit.ops)} gates, complex64 ({(8 << n) >> 20} MiB state) and complex128 "
                       f"({(16 << n) >> 20} MiB)"}
    for dtype, dname, tdt, amp in ((gb.C64, "", torch.complex64, 8), (gb.C128, "c128_", torch.complex128, 16)):
        stats = circ.plan_stats(dtype, False)
        passes, tq = stats["passes"], stats["tile_qubits"]
        res[f"{dname}tile_qubits"] = tq
        res[f"{dname}fused_passes"] = passes
        circ.specialize(dtype, False)
        state = torch.zeros(1 << n, dtype=tdt, device=dev)
        state[0] = 1
        sv = gb.sv_wrap(state, n, stream=stream)
        modes = [(gb.JIT, "fused"), (gb.FUSED, "interp"), (gb.PLAIN, "plain")]
        for mode, key in modes:
            gb.apply_circuit(sv, circ, (), mode)
            torch.cuda.synchronize()
            reps = 3 if mode != gb.PLAIN else 1
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                gb.apply_circuit(sv, circ, (), mode)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            sweeps = passes if mode != gb.PLAIN else len(w.circuit.ops)
            byts = sweeps * 2 * (amp << n)
            res[f"{dname}{key}_ms"] = ms
            res[f"{dname}{key}_sweeps"] = sweeps
            res[f"{dname}{key}_gbs"] = byts / (ms / 1e3) / 1e9
            res[f"{dname}{key}_frac_hbm"] = res[f"{dname}{key}_gbs"] / pk["hbm_gbs"]
        res[f"{dname}speedup_fused_vs_plain"] = res[f"{dname}plain_ms"] / res[f"{dname}fused_ms"]
        # per-gate sweep bytes the fused passes stand in for, over the fused time
        res[f"{dname}fused_effective_gbs"] = len(w.circuit.ops) * 2 * (amp << n) / (res[f"{dname}fused_ms"] / 1e3) / 1e9
        sv.free()
        del state
        torch.cuda.empty_cache()
    res["mode"] = "fused = specialised tile passes (GBVQC_MODE_JIT); interp = record interpreter"
    return res


def plain10_rate(gb, I, torch, dev, stream):
    """The 10-qubit plain configuration: Rx.Rz.Rx + CNOT ladder, 4 layers, 120 angles,
    energy + full gradient in complex128 through the per-gate path (one launch per gate)
    and through the specialised tile passes."""
    w = I.plain_10q()
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 10)
    theta = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    e = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(w.circuit.n_params, dtype=torch.float64, device=dev)
    res = {"workload": "plain_10q: 10 qubits, 4 layers Rx.Rz.Rx + CNOT ladder, 120 angles, "
                       "H = sum Z_iZ_i+1 + 0.5 sum X_i (19 terms), complex128"}
    for mode, key in ((gb.PLAIN, "plain"), (gb.JIT, "fused")):
        for _ in range(3):
            gb.grad(c, theta, obs, gb.C128, mode, stream=stream, out=(e, g))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        reps = 50
        a.record(stream)
        for _ in range(reps):
            gb.grad(c, theta, obs, gb.C128, mode, stream=stream, out=(e, g))
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        res[f"{key}_ms"] = ms
        res[f"{key}_evals_per_s"] = 1e3 / ms
    return res


def batch_rate(gb, I, torch):
    """512 independent VQE instances (12..20 qubits, depths 4..16) per batch_grad call."""
    ws = I.batch_512()
    circs = [gb.circuit_create(w.circuit) for w in ws]
    obss = [gb.obs_create(w.observable, w.circuit.n_qubits) for w in ws]
    b = gb.batch_create(circs, obss, gb.C64)
    th = torch.tensor(np.concatenate([w.theta for w in ws]), dtype=torch.float64, device="cuda")
    e = torch.empty(len(ws), dtype=torch.float64, device="cuda")
    g = torch.empty(th.numel(), dtype=torch.float64, device="cuda")

    def time_batch():
        for _ in range(2):
            b.grad(th, out=(e, g))
        torch.cuda.synchronize()
        reps = 5
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            b.grad(th, out=(e, g))
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / reps

    ms_default = time_batch()                      # every member at the default 12-qubit tile
    t_setup = time.perf_counter()
    tiles, _ = b.autotune(np.concatenate([w.theta for w in ws]))
    tune_s = time.perf_counter() - t_setup
    ms = time_batch()
    b.free()
    hist = {}
    for t in tiles:
        hist[str(t)] = hist.get(str(t), 0) + 1
    return {"workload": "batch_512: 512 VQE instances, n ~ U{12..20}, depth ~ U{4..16}, Ry.Rz + CNOT ladder, "
                        "random-field Ising H; complex64, FP64 reductions; one CUDA-graph replay per batch",
            "ms_per_batch": ms, "gradient_evals_per_s": len(ws) * 1e3 / ms,
            "ms_per_batch_default_tiles": ms_default, "autotuned_tiles": hist, "autotune_s": tune_s,
            "amplitudes": int(sum(1 << w.circuit.n_qubits for w in ws))}


def noisy_rate(gb, I, torch):
    """13-qubit noisy density matrix (26 vectorised qubits): energy + 312-parameter gradient
    with specialised tile passes in complex64 and complex128, and per gate in complex128."""
    w = I.noisy_13q()
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 13)
    res = {"workload": "noisy_13q_hea8: density matrix, 8 layers Rx.Rz.Rx + CNOT, depolarising + amplitude "
                       "damping, 312 parameters, 2^26 amplitudes"}
    for dtype, mode, key in ((gb.C64, gb.JIT, "fused_c64"), (gb.C128, gb.JIT, "fused_c128"),
                             (gb.C128, gb.PLAIN, "plain_c128")):
        gb.grad(c, w.theta, obs, dtype, mode)
        torch.cuda.synchronize()
        reps = 3 if mode != gb.PLAIN else 1
        t0 = time.perf_counter()
        for _ in range(reps):
            gb.grad(c, w.theta, obs, dtype, mode)
        res[f"{key}_ms"] = (time.perf_counter() - t0) * 1e3 / reps
    res["speedup"] = res["plain_c128_ms"] / res["fused_c64_ms"]
    return res


def heisenberg_rate(gb, I, torch, dev, stream):
    """20-qubit random rotation circuit with the Heisenberg observable (XX/YY/ZZ + Z):
    fused complex64 energy + 200-parameter gradient, device pointers, autotuned tiling."""
    w = I.heisenberg_20q()
    c = gb.circuit_create(w.circuit)
    obs = gb.obs_create(w.observable, 20)
    c.autotune(w.theta, obs, gb.C64)
    c.specialize(gb.C64, True)
    theta = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    e = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(w.circuit.n_params, dtype=torch.float64, device=dev)
    for _ in range(3):
        gb.grad(c, theta, obs, gb.C64, gb.JIT, stream=stream, out=(e, g))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    reps = 20
    a.record(stream)
    for _ in range(reps):
        gb.grad(c, theta, obs, gb.C64, gb.JIT, stream=stream, out=(e, g))
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    return {"workload": "heisenberg_20q_rand10: 20 qubits, 10 layers of random Rx/Ry/Rz + CNOT brick, "
                        "200 parameters, H = sum Z + sum (XX + YY + ZZ) (77 terms)",
            "ms_per_eval": ms, "gradient_evals_per_s": 1e3 / ms, "l2": "warm (16 MiB states)"}


def gate_micro(gb, I, torch, n, pk):
    """Single-gate sweeps (H, Rx, CNOT, CZ) on qubit positions 0, 5, 11, 20 and n - 1 of an
    n-qubit state, one kernel per gate (per-gate path) and one tile pass (fused path):
    GB/s = algorithmic bytes / event-timed duration, the algorithmic bytes being one read
    and one write of the amplitudes the gate changes (the whole state; for CNOT the half
    with the control set and for CZ the quarter |11>, by the per-gate kernel) or of the
    whole state (tile pass).  The
    state is larger than L2 for n >= 25, so no flush is needed."""
    stream = torch.cuda.current_stream()
    rows = []
    for dtype, dname, s in ((gb.C64, "c64", 8), (gb.C128, "c128", 16)):
        sv = gb.sv_alloc(n, dtype)
        full = 2.0 * s * (1 << n)
        for gate in ("H", "RX", "CNOT", "CZ"):
            for q in sorted({0, 5, 11, 20, n - 1}):
                if q >= n:
                    continue
                if gate in ("CNOT", "CZ"):
                    op = I.Op(gate, (q, q + 1 if q + 1 < n else q - 1))
                else:
                    op = I.Op(gate, (q,), fixed=(0.3,) if gate == "RX" else ())
                c = gb.circuit_create(I.Circuit(n, [op], 0))
                row = {"dtype": dname, "gate": gate, "qubit": q}
                for mode, key in ((gb.PLAIN, "plain"), (gb.FUSED, "fused")):
                    byts = full / {"CNOT": 2, "CZ": 4}.get(gate, 1) if mode == gb.PLAIN else full
                    for _ in range(3):
                        gb.apply_circuit(sv, c, (), mode)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    reps = 20
                    a.record(stream)
                    for _ in range(reps):
                        gb.apply_circuit(sv, c, (), mode)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ms = a.elapsed_time(b) / reps
                    row[f"{key}_us"] = round(ms * 1e3, 1)
                    row[f"{key}_gbs"] = round(byts / (ms / 1e3) / 1e9, 1)
                    row[f"{key}_frac_hbm"] = round(byts / (ms / 1e3) / 1e9 / pk["hbm_gbs"], 3)
                rows.append(row)
                c.free()
        sv.free()
    return {"workload": f"single-gate sweeps on a {n}-qubit state (H, Rx(0.3), CNOT, CZ; qubits 0, 5, 11, 20, n-1)",
            "hbm_peak_gbs": pk["hbm_gbs"], "rows": rows}


def run_sweep_only(args) -> int:
    """The gate-sweep leg alone on one GPU (profiling entry point)."""
    import torch
    import paper_2406_19212_gb300 as gb
    from paper_2406_19212_gb300 import inputs as I
    rows, cols = (int(x) for x in args.sweep_grid.lower().split("x"))
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    res = gate_sweep(gb, I, torch, dev, stream, peaks()[0], rows, cols)
    print(json.dumps(res))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary legs (plain complex128, 28q sweep, batch, noisy)")
    ap.add_argument("--only-sweep", action="store_true",
                    help="run only the gate-sweep leg (fused vs per-gate) and print its JSON; "
                         "for kernel profiles on a chosen size")
    ap.add_argument("--sweep-grid", default="4x7", help="grid of the gate-sweep circuit, ROWSxCOLS")
    ap.add_argument("--gate-micro", type=int, default=0, metavar="N",
                    help="run only the single-gate sweep microbenchmark on N qubits and print its JSON")
    args = ap.parse_args()
    if args.only_sweep:
        return run_sweep_only(args)
    if args.gate_micro:
        import torch
        import paper_2406_19212_gb300 as gb
        from paper_2406_19212_gb300 import inputs as I
        torch.cuda.set_device(0)
        print(json.dumps(gate_micro(gb, I, torch, args.gate_micro, peaks()[0])))
        return 0
    world, rank, local = dist_setup()
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    else:
        rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
