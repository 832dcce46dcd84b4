#!/usr/bin/env python
"""Throughput of the GB300 noisy-MPO engine on the paper's workload.

Metric: noisy-gate MPO updates per second at chi_max = 1024 (n = 64 qubits,
Haar brickwork, two-qubit depolarising p = 0.005, seed 2) in the precision
form, with its accuracy against the FP64 form. One timed step is one noisy
gate (the unit of the hot-path scope): the centre move onto its bond, the
contraction, superoperator, truncated SVD and write-back; the end-of-step
Schmidt sweep and entropy run with the last gate of each brickwork step.
Before timing, ramp layers run until the bonds reach their cap, then W
warm-up gates.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64|mixed]
                    [--workload NAME] [--impl reference]

Prints one JSON line. ``value`` is gates/s with gates already resident in HBM;
``e2e`` is the same metric through the C ABI with pinned host gate buffers
(H2D copies inside the timed region) and the entropies read back at the end
of every brickwork step. Under torchrun each rank simulates an independent
circuit (seed + rank): a single circuit does not shard, so N GPUs run N
replicas (weak scaling). ``--impl reference`` times the CPU oracle instead
(test infrastructure, the only other code path here that may run it).
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
    "n64_chi1024_p0.005": dict(n=64, chi=1024, p=0.005, seed=2, precision="mixed", centre_only=True),
    "n32_chi256_p0.01": dict(n=32, chi=256, p=0.01, seed=1, precision="fp64", centre_only=True),
    "n8_chi256_p0.02": dict(n=8, chi=256, p=0.02, seed=0, precision="fp64"),
    # batching form: 256 instances, n_i in {16, 24, ..., 64}, p_i in {.005, .01,
    # .02, .05} from PCG64(4), D_i = 2 n_i, instance gates from PCG64(1000 + i)
    "batch256_chi128": dict(n=64, chi=128, p=0.02, seed=4, precision="fp32", batch=256),
}
DEFAULT_WORKLOAD = "n64_chi1024_p0.005"
METRIC = "noisy-gate MPO updates/s at chi=1024 (mixed vs FP64, |dS|<=1e-6); % roofline"

# FP64 and FP32 SIMT rates measured on this GPU model with an FMA-chain probe
# (8 independent chains per thread, 152 x 8 CTAs of 256 threads, CUDA events):
# the measured peaks file carries only the HBM copy and the BF16 GEMM rates.
FP64_PROBE_TFLOPS = 1.20
FP32_PROBE_TFLOPS = 74.6
# DRAM bytes (read + written) per algorithmic flop of the split-BF16 GEMM,
# from an ncu capture of one 4096 x 2048 x 4096 complex product
# (dram__bytes_read.sum + dram__bytes_write.sum = 6.418e9 B for 2.749e11 flop);
# the traffic of an average launch scales with its flops
OZ_DRAM_BYTES_PER_FLOP = 6.418e9 / 2.749e11


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


MIXED_MARGIN = 64        # Ritz directions beyond chi_max in the precision form's FP64 step


def gate_work(dims, i: int, chi: int, prec: str) -> dict:
    """Algorithmic work of one noisy gate on sites (i, i+1) as the hot-path
    scope counts it (real flops, complex multiply-add = 8), from the bond
    dimensions dims: theta 8 (4 chiL)(4 chiR) chiM, superoperator
    2048 chiL chiR, Hermitian Gram of theta' 4 r^2 c, projection onto the kept
    right factor 8 k r c (r, c = the shorter and longer side of theta',
    k = min(chi, r)), the centre move onto the bond (a 4 chiM x chiM
    factorisation, 12 chiM^2 (4 chiM)); the Hermitian eigen-solve 13.3 m^3,
    m = min(r, chi + 64) in the precision form, r otherwise. Bytes: the site
    tensors the gate reads and writes."""
    esz = 8 if prec == "fp32" else 16
    cl, cm, cr = dims[i], dims[i + 1], dims[i + 2]
    r, c = 4 * min(cl, cr), 4 * max(cl, cr)
    k = min(chi, r)
    gemm = 8.0 * (4 * cl) * (4 * cr) * cm + 2048.0 * cl * cr + 4.0 * r * r * c + 8.0 * k * r * c
    gemm += 12.0 * cm * cm * (4 * cm)
    m = min(r, chi + MIXED_MARGIN) if prec == "mixed" else r
    return {"gemm": gemm, "solve": 13.3 * m ** 3, "bytes": 2.0 * (cl * 4 * cm + cm * 4 * cr) * esz}


def sweep_work(dims, n: int, centre_only: bool) -> dict:
    """The end-of-step Schmidt sweep: per recorded bond b a chi_b x 4 chi_{b+1}
    factorisation, 12 r^2 c GEMM-class + 13.3 r^3 solve."""
    gemm = solve = 0.0
    for b in ([n // 2] if centre_only else range(1, n)):
        r, c = dims[b], 4 * dims[b + 1]
        gemm += 12.0 * r * r * c
        solve += 13.3 * r ** 3
    return {"gemm": gemm, "solve": solve, "bytes": 0.0}


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


def gate_schedule(circ, n: int, t_first: int, count: int):
    """(time step, gate index, ABI bond, last gate of its step) for `count`
    consecutive gates from the first gate of step t_first."""
    out = []
    t = t_first
    while len(out) < count:
        par = circ.parity(t)
        ng = len(circ.gates[t - 1])
        for g in range(ng):
            out.append((t, g, 2 * g + par, g == ng - 1))
            if len(out) == count:
                break
        t += 1
    return out


def accuracy_checks(mpo_mod, m, circ, sched_next, chi: int) -> dict:
    """Accuracy of the precision form against the FP64 form, outside the
    timed regions: (1) |dS| at every bond after every step of a 12-step
    n = 16, chi = 64, p = 0.005 trajectory (seed 0) run through both forms;
    (2) the kept-theta relative Frobenius error of the next gate of the
    benchmark circuit itself (chi = 1024): its theta' (mpo_theta) truncated by
    both forms' SVDs (mpo_svd_truncated), compared."""
    import torch
    from paper_2003_13163_gb300.circuits import random_circuit
    out = {}
    c16 = random_circuit(16, 12, 0.005, seed=0)
    S = {}
    for prec in ("fp64", "mixed"):
        q = mpo_mod.MPO(16, 64, prec)
        rows = []
        for t in range(1, 13):
            q.apply_layer(c16.parity(t), c16.gates[t - 1], c16.p[t - 1])
            rows.append(q.entropy(with_trace=False)[0])
        q.close()
        S[prec] = np.array(rows)
    out["dS_max_n16_chi64_12steps"] = float(np.abs(S["mixed"] - S["fp64"]).max())
    t, g, b, _ = sched_next
    At = m.theta(b, circ.gates[t - 1][g], float(circ.p[t - 1][g]))   # theta' of the next gate, untruncated
    if At.shape[0] > At.shape[1]:
        At = At.conj().T.contiguous()
    At = At / torch.linalg.norm(At)
    t0 = time.perf_counter()
    U64, X64, _ = mpo_mod.svd_truncated(At, chi, "fp64", cutoff=1e-12)
    t64 = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Um, Xm, _ = mpo_mod.svd_truncated(At, chi, "mixed")
    torch.cuda.synchronize()
    tm = time.perf_counter() - t0
    ref = U64 @ X64
    err = float(torch.linalg.norm(Um @ Xm - ref) / torch.linalg.norm(ref))
    out.update({"kept_theta_rel_err_chi1024": err, "theta_shape": list(At.shape),
                "fp64_svd_seconds": round(t64, 2), "mixed_svd_seconds": round(tm, 2)})
    return out


def run_single(args, wl, prec) -> None:
    """One circuit per rank; a timed step is one noisy gate (a2-a6 on its
    bond), the end-of-step sweep and entropy charged to the step's last gate."""
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
    # App. A's schedule sweeps the whole chain (every bond) after every gate
    centre_only = (args.centre_only or wl.get("centre_only", False)) and args.update == "local"
    R = ramp_layers(n, chi)
    K, W = args.steps, args.warmup
    per_layer = n // 2 - 0.5
    depth = R + int(math.ceil((W + 2 * K + 1) / per_layer)) + 2
    circ = random_circuit(n, depth, p, replicas.rank_seed(wl["seed"], rank))
    sched = gate_schedule(circ, n, R + 1, W + 2 * K + 1)
    # device-resident gates for the kernel-only number, pinned host copies for e2e
    dg = {(t, g): torch.from_numpy(circ.gates[t - 1][g].view(np.float64).copy()).to(dev) for t, g, _, _ in sched}
    hg = {(t, g): torch.from_numpy(circ.gates[t - 1][g].view(np.float64).copy()).pin_memory()
          for t, g, _, _ in sched}

    stream = torch.cuda.current_stream(dev)
    m = mpo.MPO(n, chi, prec, stream=stream.cuda_stream, centre_only=centre_only)

    t_ramp0 = time.perf_counter()
    for t in range(1, R + 1):
        m.apply_layer(circ.parity(t), circ.gates[t - 1], circ.p[t - 1])
    torch.cuda.synchronize()
    t_ramp = time.perf_counter() - t_ramp0

    global_update = args.update == "global"

    def step(entry, bufs, read_back):
        t, g, b, last = entry
        m.apply_gate(b, bufs[(t, g)], float(circ.p[t - 1][g]))
        d2h = 0
        if last or global_update:      # App. A's schedule re-canonicalises after every gate
            m.sweep()
            if read_back:
                S, _, _ = m.entropy(with_trace=False)
                d2h = S.nbytes
        return d2h

    pos = 0
    for _ in range(W):
        step(sched[pos], dg, False)
        pos += 1
    torch.cuda.synchronize()
    dims = m.bond_dims()

    barrier = replicas.barrier

    def max_over_ranks(x: float) -> float:
        return replicas.max_over_ranks(x, device=dev)

    # ---- kernel-only timed region: gates resident in HBM --------------------
    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    m.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timed = sched[pos:pos + K]
    # the kernel-only region is the profiler range (ncu --profile-from-start off)
    torch.cuda.cudart().cudaProfilerStart()
    e0.record(stream)
    for entry in timed:
        step(entry, dg, False)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    barrier()
    pos += K
    ms = e0.elapsed_time(e1)
    prof = m.profile_read()
    m.profile(False)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms)
    value = K * world / (ms_max / 1e3)
    work = {"gemm": 0.0, "solve": 0.0, "bytes": 0.0}
    for t, g, b, last in timed:
        for key, v in gate_work(dims, b, chi, prec).items():
            work[key] += v
        if last or global_update:
            for key, v in sweep_work(dims, n, centre_only).items():
                work[key] += v

    # ---- end-to-end through the C ABI with host buffers ----------------------
    barrier()
    torch.cuda.synchronize()
    h2d = d2h = 0
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for entry in sched[pos:pos + K]:
        d2h += step(entry, hg, True)
        h2d += 32 * 8 + 8
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    pos += K
    e2e_ms = max_over_ranks(e2.elapsed_time(e3))
    e2e_value = K * world / (e2e_ms / 1e3)
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
    fp64_classes = {"refine_gemm", "eig_fp64"} | ({"svd_gate", "svd_sweep", "cgemm"} if prec == "fp64" else set())
    tensor_classes = {"cgemm", "tc_cgemm"} if prec != "fp64" else set()
    if dom == "oz_gemm":
        bound, unit = "tensor", "TFLOP/s"
        pk = peaks["bf16_tflops"] / 21.0
        basis = (f"BF16 tensor sustained ({peaks['source']}) / 21: the split scheme's BF16 products per "
                 "FP64-accurate product (6 slices, levels 2..7)")
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
    elif dom in fp64_classes:
        bound, pk, unit, basis = "alu", peaks["fp64_tflops"], "TFLOP/s", "FP64 FMA probe 1.20 TFLOP/s"
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
    elif dom in ("svd_gate", "svd_sweep"):
        bound, pk, unit = "alu", peaks["fp32_simt_tflops"], "TFLOP/s"
        basis = "FP32 FMA probe 74.6 TFLOP/s (the one-sided Jacobi runs on the FP32 pipes)"
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
    elif dom in tensor_classes:
        bound, pk, unit = "tensor", peaks["tf32_tflops"], "TFLOP/s"
        basis = f"TF32 tensor = BF16 sustained / 2 ({peaks['source']})"
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
    else:
        bound, pk, unit, basis = "hbm", peaks["hbm_gbs"], "GB/s", f"HBM copy ({peaks['source']})"
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    traffic = OZ_DRAM_BYTES_PER_FLOP * d["flops"] / d["launches"] if dom == "oz_gemm" else None
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": pk, "unit": unit,
                "frac": achieved / pk, "traffic": traffic, "peak_basis": basis,
                "traffic_basis": "ncu dram bytes of one 4096 x 2048 x 4096 launch, scaled by flops"
                if traffic is not None else None,
                "share_of_step": d["ms"] / ms, "launches": d["launches"], "avg_launch_ms": d["ms"] / d["launches"]}
    p_gemm = peaks["fp64_tflops"] if prec == "fp64" else peaks["tf32_tflops"]
    p_solve = peaks["fp32_simt_tflops"] if prec == "fp32" else peaks["fp64_tflops"]
    t_roof = work["gemm"] / (p_gemm * 1e12) + work["solve"] / (p_solve * 1e12) + work["bytes"] / (peaks["hbm_gbs"] * 1e9)
    step_roofline = {"t_roof_ms_per_step": 1e3 * t_roof / K, "measured_ms_per_step": ms / K,
                     "frac": t_roof / (ms / 1e3), "gemm_flops_per_step": work["gemm"] / K,
                     "solve_flops_per_step": work["solve"] / K, "bytes_per_step": work["bytes"] / K,
                     "p_gemm_tflops": p_gemm, "p_solve_tflops": p_solve, "hbm_gbs": peaks["hbm_gbs"],
                     "peaks": peaks["source"]}
    kernels = {k: {"ms": round(v["ms"], 3), "launches": v["launches"], "share": round(v["ms"] / ms, 4),
                   "flops": v["flops"], "bytes": v["bytes"]}
               for k, v in classes.items()}
    layers_timed = sum(1 for e in timed if e[3])
    line = {"metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "mixed": "f64 (FP32 solves + split-BF16 products)"}[prec],
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "chi_max": chi, "p": p, "seed": wl["seed"],
                       "precision": prec, "update": args.update,
                       "step": "one noisy gate (a2-a6); the end-of-step sweep and entropy with the step's last gate"
                       if args.update == "local" else "one noisy gate followed by a sweep of the whole chain (App. A)",
                       "entropy": "centre bond" if centre_only else "every bond",
                       "parallelism": f"replicas{world}", "ramp_layers": R, "ramp_seconds": round(t_ramp, 2),
                       "warmup_gates": W, "timed_gates": K, "layer_ends_timed": layers_timed,
                       "max_bond_dim": int(max(dims)), "bond_dims_min_centre": int(min(dims[n // 4: 3 * n // 4])),
                       "l2": "inputs larger than L2 (site tensors "
                       f"{m.device_bytes() / 2**30:.1f} GiB)", "final_S_centre": float(S[n // 2 - 1]),
                       "final_trace": tr},
            "clocks": clk,
            "gpu_launches": int(sum(v["launches"] for v in classes.values())),
            "roofline": roofline,
            "step_roofline": step_roofline,
            "kernels": kernels,
            "subspace_steps_per_gate": prof.get("_steps", 0) / K,
            "svd_sweeps_total": prof["_sweeps"],
            "e2e": {"value": e2e_value, "unit": "gates/s", "h2d_bytes_per_step": h2d // K,
                    "d2h_bytes_per_step": d2h // K}}
    if prec == "mixed" and rank == 0 and not args.no_accuracy:
        line["accuracy_vs_fp64"] = accuracy_checks(mpo, m, circ, sched[pos], chi)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--centre-only", action="store_true", help="record S at the centre bond only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the precision form's FP64 comparisons")
    ap.add_argument("--update", default="local", choices=["local", "global"],
                    help="local: one sweep per brickwork step (the engine's schedule); global: App. A's "
                         "re-canonicalisation of the whole chain after every gate (timed comparator)")
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

    run_single(args, wl, prec)


if __name__ == "__main__":
    main()
