#!/usr/bin/env python
"""Throughput of the GB300 noisy-MPO engine on the paper's workload.

Metric: noisy-gate MPO updates per second at chi_max = 1024 (n = 64 qubits,
Haar brickwork, two-qubit depolarising p = 0.005, seed 2). One timed step is
one brickwork layer (time step of Sec. 2.1): its n/2 or n/2-1 noisy gates,
each contraction + superoperator + truncated SVD + write-back, then the
end-of-step Schmidt sweep and entropy at every bond. Before timing, the
circuit is run until every bond sits at its cap (ramp layers, untimed), then W
warm-up layers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
                    [--impl reference]

Prints one JSON line. ``value`` is gates/s with gates already resident in HBM;
``e2e`` is the same metric through the C ABI with host gate buffers (H2D
copies inside the timed region) and the entropies read back every step.
Under torchrun each rank simulates an independent circuit (seed + rank):
a single circuit does not shard, so N GPUs run N replicas (weak scaling).
``--impl reference`` times the CPU oracle instead (test infrastructure, the
only other code path here that may run it).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # n, chi_max, p, seed, default precision
    "n64_chi1024_p0.005": dict(n=64, chi=1024, p=0.005, seed=2, precision="fp32"),
    "n32_chi256_p0.01": dict(n=32, chi=256, p=0.01, seed=1, precision="fp64"),
    "n8_chi256_p0.02": dict(n=8, chi=256, p=0.02, seed=0, precision="fp64"),
    # batching form: 256 instances, n_i in {16, 24, ..., 64}, p_i in {.005, .01,
    # .02, .05} from PCG64(4), D_i = 2 n_i, instance gates from PCG64(1000 + i)
    "batch256_chi128": dict(n=64, chi=128, p=0.02, seed=4, precision="fp32", batch=256),
}
DEFAULT_WORKLOAD = "n64_chi1024_p0.005"
METRIC = "noisy-gate MPO updates/s at chi=1024 (n=64 Haar brickwork, p=0.005)"

# FP64 and FP32 SIMT rates measured on this GPU model with an FMA-chain probe
# (8 independent chains per thread, 152 x 8 CTAs of 256 threads, CUDA events):
# the measured peaks file carries only the HBM copy and the BF16 GEMM rates.
FP64_PROBE_TFLOPS = 1.20
FP32_PROBE_TFLOPS = 74.6


def load_peaks() -> dict:
    """Roofline denominators: HBM copy and BF16 GEMM rates from the measured
    peaks file (else the documented fallback), TF32 tensor = BF16 / 2 (the
    nominal ratio), FP64 / FP32 SIMT from the probe above."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        hbm, bf16s, src = float(d["hbm_gbs"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        hbm, bf16s, src = 6800.0, 1700.0, "fallback"
    return {"hbm_gbs": hbm, "bf16_tflops": bf16s, "tf32_tflops": bf16s / 2.0, "fp64_tflops": FP64_PROBE_TFLOPS,
            "fp32_simt_tflops": FP32_PROBE_TFLOPS, "source": src}


def step_work(dims, n: int, parity: int, chi: int, prec: str, over: int, centre_only: bool) -> dict:
    """Algorithmic work of one brickwork step as the hot-path scope counts it
    (real flops, complex multiply-add = 8), from the bond dimensions dims:
    per gate theta 8 (4 chiL)(4 chiR) chiM, superoperator 2048 chiL chiR,
    Hermitian Gram of theta' 4 r^2 c, projection to the kept right factor
    8 k r c (r, c = the shorter and longer side of theta', k = min(chi, r)),
    and the Hermitian eigen-solve 13.3 m^3 with m = min(r, chi + oversample)
    (precision form) or m = r; per recorded bond of the Schmidt sweep a
    chi_b x 4 chi_{b+1} factorisation, 12 r^2 c GEMM-class + 13.3 r^3. Bytes:
    the four site tensors each gate reads or writes."""
    esz = 8 if prec == "fp32" else 16
    gemm = solve = byts = 0.0
    for l in range(1 + parity, n, 2):
        i = l - 1
        cl, cm, cr = dims[i], dims[i + 1], dims[i + 2]
        r, c = 4 * min(cl, cr), 4 * max(cl, cr)
        k = min(chi, r)
        gemm += 8.0 * (4 * cl) * (4 * cr) * cm + 2048.0 * cl * cr + 4.0 * r * r * c + 8.0 * k * r * c
        m = min(r, chi + over) if prec == "mixed" else r
        solve += 13.3 * m ** 3
        byts += 2.0 * (cl * 4 * cm + cm * 4 * cr) * esz
    bonds = [n // 2] if centre_only else range(1, n)
    for b in bonds:
        r, c = dims[b], 4 * dims[b + 1]
        gemm += 12.0 * r * r * c
        solve += 13.3 * r ** 3
    return {"gemm": gemm, "solve": solve, "bytes": byts}


def ramp_layers(n: int, chi: int) -> int:
    """Layers after which every bond can sit at its cap min(chi, 4^b, 4^(n-b))."""
    return min(n // 2, int(math.ceil(math.log(chi, 4))) + 2)


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 7:
                    self.rows.append(parts)

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_gate_sample(chi: int, p: float, seed: int, reps: int = 1) -> dict:
    """Time the CPU oracle on a bounded sample of the workload: `reps` bulk
    noisy gates at chi (theta, superoperator, truncated SVD) each with the
    two centre moves that are its share of the end-of-step sweep, on a
    synthetic saturated two-site block (random isometry + random centre)."""
    from oracle import channels
    from oracle import mpo as ompo
    from paper_2003_13163_gb300.circuits import haar_unitary, random_complex

    rng = np.random.Generator(np.random.PCG64(seed))
    A0 = np.linalg.qr(random_complex((4 * chi, chi), seed + 1))[0].reshape(chi, 4, chi)
    A1 = random_complex((chi, 4 * chi), seed + 2)
    A1 = (A1 / np.linalg.norm(A1)).reshape(chi, 4, chi)
    times = []
    for _ in range(reps):
        m = ompo.MPO(2, chi, 1e-12)
        m.A = [A0.copy(), A1.copy()]
        m.centre = 1
        M = channels.noisy_gate_superop(haar_unitary(rng), p)
        t0 = time.perf_counter()
        m.apply_superop(M, 1)
        m._move_left(1)
        m.centre = 0
        m._move_right(0)
        times.append(time.perf_counter() - t0)
    return {"seconds_per_gate": float(np.mean(times)), "reps": reps}


def cpu_threads() -> int:
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count() or 1


def run_reference(args, wl) -> None:
    """--impl reference: the CPU oracle as it stands, one bounded sample
    (one bulk gate with its sweep share) per step."""
    from paper_2003_13163_gb300 import replicas
    world, rank, _ = replicas.world()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_gate_sample(wl["chi"], wl["p"], wl["seed"])
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle_gate_sample(wl["chi"], wl["p"], wl["seed"] + i)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "gates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": wl["n"], "chi_max": wl["chi"], "p": wl["p"],
                       "step": "one bulk noisy gate at chi_max with its two sweep factorisations (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "gates/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{args.steps} bulk gates at chi={wl['chi']} on a synthetic saturated block"},
            "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, wl, prec) -> None:
    """The batching form: every instance of the ensemble advances one step per
    timed step (mpo_apply_layer_batch); value = gates of all instances / time.
    The first layers (until chi_max = 128 is reached) and W warm-up layers run
    untimed."""
    import torch
    from paper_2003_13163_gb300 import build as B
    from paper_2003_13163_gb300 import replicas
    world, rank, local = replicas.world()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    B.build()
    from paper_2003_13163_gb300 import mpo
    from paper_2003_13163_gb300.circuits import ensemble_instances

    k, chi = wl["batch"], wl["chi"]
    circs = ensemble_instances(k, seed=replicas.rank_seed(wl["seed"], rank))
    R, K, W = ramp_layers(16, chi), args.steps, args.warmup
    T = R + W + 2 * K
    assert T <= min(c.depth for c in circs)
    p_all = np.array([float(c.p[0][0]) for c in circs])
    host = []
    for t in range(1, T + 1):
        g = np.concatenate([c.gates[t - 1].reshape(-1) for c in circs])
        host.append(torch.from_numpy(g.view(np.float64).copy()).pin_memory())
    devg = [h.to(dev) for h in host]
    stream = torch.cuda.current_stream(dev)
    b = mpo.MPOBatch([c.n for c in circs], chi, prec, workers=args.workers, stream=stream.cuda_stream)
    t = 0
    t_ramp0 = time.perf_counter()
    for _ in range(R + W):
        t += 1
        b.apply_layer(t, devg[t - 1], p_all, with_trace=False)
    torch.cuda.synchronize()
    t_ramp = time.perf_counter() - t_ramp0

    def timed(gate_bufs, with_h2d):
        nonlocal t
        gates = h2d = d2h = 0
        replicas.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            t += 1
            S, _, _ = b.apply_layer(t, gate_bufs[t - 1], p_all, with_trace=False)
            gates += sum(len(c.gates[t - 1]) for c in circs)
            if with_h2d:
                h2d += gate_bufs[t - 1].numel() * 8 + p_all.nbytes
                d2h += sum(s.nbytes for s in S) + 8 * k
        e1.record(stream)
        torch.cuda.synchronize()
        replicas.barrier()
        ms = replicas.max_over_ranks(e0.elapsed_time(e1), device=dev)
        return gates * world / (ms / 1e3), ms, gates, h2d, d2h

    insts = [b.instance(i) for i in range(k)]
    for q in insts:
        q.profile(True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    value, ms, gates, _, _ = timed(devg, False)
    clk = clocks.stop()
    kern = {}
    for q in insts:
        for name, v in q.profile_read().items():
            if not name.startswith("_") and v["launches"]:
                d = kern.setdefault(name, {"ms": 0.0, "launches": 0})
                d["ms"] += v["ms"]
                d["launches"] += v["launches"]
        q.profile(False)
    e2e_value, _, _, h2d, d2h = timed(host, True)
    line = {"metric": "noisy-gate MPO updates/s, batching form (256 independent circuits, chi=128)",
            "value": value, "unit": "gates/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "instances": k,
                       "n_range": [min(c.n for c in circs), max(c.n for c in circs)],
                       "chi_max": chi, "seed": wl["seed"], "precision": prec, "workers": args.workers,
                       "parallelism": f"replicas{world}", "ramp_layers": R, "ramp_seconds": round(t_ramp, 2),
                       "gates_per_step": gates / K, "l2": "per-step working set of all instances exceeds L2"},
            "clocks": clk, "gpu_launches": int(sum(v["launches"] for v in kern.values())),
            "kernels": {name: {"ms_summed_over_streams": round(v["ms"], 1), "launches": v["launches"]}
                        for name, v in kern.items()},
            "e2e": {"value": e2e_value, "unit": "gates/s", "h2d_bytes_per_step": h2d // K,
                    "d2h_bytes_per_step": d2h // K}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--centre-only", action="store_true", help="record S at the centre bond only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workers", type=int, default=8, help="host worker threads of the batching form")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
        return
    prec = args.precision or wl["precision"]
    if "batch" in wl:
        run_batch(args, wl, prec)
        return

    import torch
    from paper_2003_13163_gb300 import replicas
    world, rank, local = replicas.world()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2003_13163_gb300 import build as B
    B.build()
    from paper_2003_13163_gb300 import mpo
    from paper_2003_13163_gb300.circuits import random_circuit

    n, chi, p = wl["n"], wl["chi"], wl["p"]
    R = ramp_layers(n, chi)
    K, W = args.steps, args.warmup
    depth = R + W + 2 * K
    circ = random_circuit(n, depth, p, replicas.rank_seed(wl["seed"], rank))
    # device-resident gates for the kernel-only number, pinned host copies for e2e
    dg = [torch.from_numpy(g.view(np.float64).copy()).to(dev) for g in circ.gates]
    dpv = [torch.from_numpy(pp.copy()).to(dev) for pp in circ.p]
    hg = [torch.from_numpy(g.view(np.float64).copy()).pin_memory() for g in circ.gates]
    hp = [torch.from_numpy(pp.copy()).pin_memory() for pp in circ.p]

    stream = torch.cuda.current_stream(dev)
    m = mpo.MPO(n, chi, prec, stream=stream.cuda_stream, centre_only=args.centre_only)
    t = 0

    def layer_dev(tt):
        m.apply_layer(circ.parity(tt), dg[tt - 1], dpv[tt - 1])

    t_ramp0 = time.perf_counter()
    for _ in range(R):
        t += 1
        layer_dev(t)
    torch.cuda.synchronize()
    t_ramp = time.perf_counter() - t_ramp0
    for _ in range(W):
        t += 1
        layer_dev(t)
    torch.cuda.synchronize()
    dims = m.bond_dims()

    barrier = replicas.barrier

    def max_over_ranks(x: float) -> float:
        return replicas.max_over_ranks(x, device=dev)

    # ---- kernel-only timed region: gates resident in HBM --------------------
    gates_timed = 0
    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    m.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        t += 1
        gates_timed += len(circ.gates[t - 1])
        layer_dev(t)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = m.profile_read()
    m.profile(False)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms)
    gates_all = gates_timed * world
    value = gates_all / (ms_max / 1e3)

    # ---- end-to-end through the C ABI with host buffers ----------------------
    barrier()
    torch.cuda.synchronize()
    h2d = d2h = 0
    gates_e2e = 0
    w0 = time.perf_counter()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(K):
        t += 1
        g, pp = hg[t - 1], hp[t - 1]
        m.apply_layer(circ.parity(t), g, pp)
        S, _, _ = m.entropy(with_trace=False)
        gates_e2e += len(circ.gates[t - 1])
        h2d += g.numel() * 8 + pp.numel() * 8
        d2h += S.nbytes + 8
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e2.elapsed_time(e3))
    e2e_value = gates_e2e * world / (e2e_ms / 1e3)
    S, tr, dw = m.entropy()

    # ---- rooflines -----------------------------------------------------------
    # (1) the dominant kernel class: its algorithmic flops (or bytes) per
    # launch as the library counts them, over its CUDA-event time on the
    # engine's stream, against the peak of the unit it runs on; (2) the whole
    # step: T_roof = F_gemm / P_gemm + F_solve / P_solve + bytes / BW over the
    # measured step time.
    peaks = load_peaks()
    classes = {k: v for k, v in prof.items() if not k.startswith("_") and v["launches"] > 0}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    d = classes[dom]
    fp64_classes = {"refine_gemm", "eig_fp64"} | ({"svd_gate", "svd_sweep", "cgemm"} if prec != "fp32" else set())
    if prec == "mixed":
        fp64_classes -= {"svd_gate", "svd_sweep"}      # the FP32 Jacobi SVD of the precision form
    tensor_classes = {"svd_gate", "svd_sweep", "cgemm", "tc_cgemm"} - fp64_classes
    if dom in fp64_classes:
        bound, pk, unit, basis = "alu", peaks["fp64_tflops"], "TFLOP/s", "FP64 FMA probe 1.20 TFLOP/s"
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
    elif dom in tensor_classes:
        bound, pk, unit = "tensor", peaks["tf32_tflops"], "TFLOP/s"
        basis = f"TF32 tensor = BF16 sustained / 2 ({peaks['source']})"
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
    else:
        bound, pk, unit, basis = "hbm", peaks["hbm_gbs"], "GB/s", f"HBM copy ({peaks['source']})"
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": pk, "unit": unit,
                "frac": achieved / pk, "traffic": None, "peak_basis": basis,
                "share_of_step": d["ms"] / ms, "launches": d["launches"], "avg_launch_ms": d["ms"] / d["launches"]}
    over = chi if prec == "mixed" else 0
    w = {"gemm": 0.0, "solve": 0.0, "bytes": 0.0}
    for tt in range(t - 2 * K + 1, t - K + 1):          # the timed steps
        sw = step_work(dims, n, circ.parity(tt), chi, prec, over, args.centre_only)
        for key in w:
            w[key] += sw[key]
    p_gemm = peaks["fp64_tflops"] if prec == "fp64" else peaks["tf32_tflops"]
    p_solve = peaks["fp32_simt_tflops"] if prec == "fp32" else peaks["fp64_tflops"]
    t_roof = w["gemm"] / (p_gemm * 1e12) + w["solve"] / (p_solve * 1e12) + w["bytes"] / (peaks["hbm_gbs"] * 1e9)
    step_roofline = {"t_roof_ms_per_step": 1e3 * t_roof / K, "measured_ms_per_step": ms / K,
                     "frac": t_roof / (ms / 1e3), "gemm_flops_per_step": w["gemm"] / K,
                     "solve_flops_per_step": w["solve"] / K, "bytes_per_step": w["bytes"] / K,
                     "p_gemm_tflops": p_gemm, "p_solve_tflops": p_solve, "hbm_gbs": peaks["hbm_gbs"],
                     "peaks": peaks["source"]}
    kernels = {k: {"ms": round(v["ms"], 3), "launches": v["launches"], "share": round(v["ms"] / ms, 4),
                   "flops": v["flops"], "bytes": v["bytes"]}
               for k, v in classes.items()}

    line = {"metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "mixed": "f32+f64"}[prec], "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "chi_max": chi, "p": p, "seed": wl["seed"],
                       "precision": prec, "entropy": "centre bond" if args.centre_only else "every bond",
                       "oversample": over, "parallelism": f"replicas{world}", "ramp_layers": R,
                       "ramp_seconds": round(t_ramp, 2), "gates_per_step": gates_timed / K,
                       "max_bond_dim": int(max(dims)), "l2": "inputs larger than L2 (site tensors "
                       f"{m.device_bytes() / 2**30:.1f} GiB)", "final_S_centre": float(S[n // 2 - 1]),
                       "final_trace": tr},
            "clocks": clk,
            "gpu_launches": int(sum(v["launches"] for v in classes.values())),
            "roofline": roofline,
            "step_roofline": step_roofline,
            "kernels": kernels,
            "svd_sweeps_per_launch": prof["_sweeps"] / max(1, sum(prof.get(k, {}).get("launches", 0)
                                                                    for k in ("svd_gate", "svd_sweep"))),
            "block_jacobi_phase_ms": {k: round(v, 1) for k, v in prof["_block_jacobi_phase_ms"].items()},
            "e2e": {"value": e2e_value, "unit": "gates/s", "h2d_bytes_per_step": h2d // K,
                    "d2h_bytes_per_step": d2h // K}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = oracle_gate_sample(chi, p, wl["seed"])
        line["cpu_baseline"] = {"value": 1.0 / smp["seconds_per_gate"], "unit": "gates/s", "cores": cpu_threads(),
                                "kind": "oracle",
                                "sample": f"1 bulk gate at chi={chi} with its 2 sweep factorisations "
                                          "(NumPy/LAPACK FP64 oracle, synthetic saturated block)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
