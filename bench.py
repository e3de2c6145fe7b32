#!/usr/bin/env python
"""Throughput of HRKAN physics-informed training on GB300.

One step = one full-batch pass of the whole hot path over the workload's
collocation points: forward jets, residual and loss, backward (weight
gradient), cross-block reduction and Adam.  Default workload: 256 independent
2-D Poisson instances (a, b uniform in {1..4}^2), HRKAN [2,16,16,1], G=10, k=3,
m=4, interior counts uniform in [2048, 32768] and boundary = interior // 8
(seed 4), all instances in one multi-instance training step, BF16 (the hidden
layer's forward as the three-term split, weight gradient and input adjoint on
tcgen05); the plain FP32 multi-instance path of the same workload is timed
beside it (fp32_path), and both are trained 1000 steps on 8 of the instances
to compare their final relative L2 errors (equal_l2).  Inputs are synthetic and
resident in HBM when the timed region starts; L2 is flushed (a 256 MiB device
write) before every timed step, outside its events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--prec fp32|bf16|tf32]

--workload burgers_2_10_10_1 --prec fp32 times the single-network FP32
Burgers workload (viscous Burgers, nu = 0.01/pi, [2,10,10,1], G=10, 65536
interior + 4096 initial + 4096 boundary points) on the fused kernel.

--workload poisson_2_64x3_1 --prec bf16 (or tf32) times the precision workload
instead: 2-D Poisson a=b=2, HRKAN [2,64,64,64,1], G=32, 262144 interior +
16384 boundary points, the hidden layers' forward contraction and weight
gradient on the tensor cores; its roofline object is the tensor-core one
(dense contraction flops of those launches) and the FP32 path of the same
workload is timed beside it.

--impl reference times the FP64 CPU oracle (the only reference there is: the
paper ships no code) on the host cores, a bounded sample of the same workload
per step.  Under torchrun with N > 1 every rank trains its own replica (the
workload does not need a collective), and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PINN train throughput (colloc pts/s, fwd jets+bwd) vs plain FP32 at equal L2 err"
UNIT = "collocation points/s"
WORKLOAD = "poisson_batch256"
BURGERS_WORKLOAD = "burgers_2_10_10_1"
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def measured_peaks():
    """MEASURED_PEAKS.json of this machine pool, else the recipe's fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return {"bf16": float(m["bf16_tflops"]), "bf16_sustained": float(m["bf16_tflops_sustained"]),
                "hbm": float(m["hbm_gbs"]), "source": "of measured (MEASURED_PEAKS.json)",
                "hbm_source": "copy bandwidth of measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "of fallback",
                "hbm_source": "of fallback"}


def dense_tc_flops(widths, G, k, n_int, J_int, n_bnd, bf16):
    """Dense flops of the tensor-core launches of one training step, each
    2 * rows * K * O with K = I * (G + k) and rows = J * points (all K columns
    counted, zeros included): for every hidden layer the forward contraction
    (interior and boundary points) and, in BF16, the weight gradient (both
    point sets; also of the first layer) and the input adjoint G = gy W
    (interior points; the boundary's single jet row keeps the FP32 adjoint)."""
    n = G + k
    f = 0
    for l in range(1, len(widths) - 2):
        I, O = widths[l], widths[l + 1]
        fwd = 2 * (J_int * n_int + n_bnd) * I * n * O
        f += fwd
        if bf16:
            f += fwd + 2 * J_int * n_int * I * n * O
    if bf16 and 16 <= widths[1] <= 64 and widths[1] % 16 == 0:   # first layer's weight gradient
        f += 2 * (J_int * n_int + n_bnd) * widths[0] * n * widths[1]
    return f


def alg_flops_per_point(widths, k, J):
    """Algorithmic FP32 flops of one training step for one point with J jet rows.

    Sparse contraction (only the k+1 active bases per unit, Eq. 2 has compact
    support): forward 2 (k+1) I O J per layer, weight gradient the same, input
    adjoint the same for every layer but the first.  Basis evaluation: 20 flops
    per active basis in the forward (v, v', v''), 25 in the backward (+ v''').
    """
    kp = k + 1
    f = 0
    for l in range(len(widths) - 1):
        I, O = widths[l], widths[l + 1]
        mac = kp * I * O * J
        f += 2 * mac * (3 if l > 0 else 2)
        f += kp * I * (20 + 25)
    return f


# ---------------------------------------------------------------- helpers


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def emit(obj):
    print(json.dumps(obj), flush=True)


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest of one float per rank (the job takes as long as its slowest rank)."""
    if ws == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, steps: int, units_per_step: int, seconds: float) -> float:
    """Units all ranks processed per second: every rank trains its own replica of the whole
    workload (weak scaling), over the slowest rank's time."""
    return ws * steps * units_per_step / seconds


# --------------------------------------------------------------- reference


def run_reference_batched(args, w):
    """FP64 CPU oracle on the multi-instance workload, one worker process per host core: every step
    trains a bounded sample (the first instances, 256 interior + 32 boundary points of each),
    instance by instance, each instance's weights and Adam moments carried from step to step."""
    from paper_2409_14248_gb300 import inputs
    d = inputs.make_batched(w)
    P = w.n_params()
    states = []
    for i in range(w.instances):
        Wi, xi, xb, gb = _instance_sample(w, d, i)
        states.append([Wi, np.zeros(P), np.zeros(P), xi, xb, gb, w.problem(*d["ab"][i])])
    pool, cores = _oracle_pool()
    try:
        def step(k, t):
            tasks = [(w.net, st[6], st[0], st[1], st[2], st[3], w.mask_int, st[4], st[5], w.lr, t)
                     for st in states[:k]]
            pts = 0
            for st, (Wi, m1, m2, n) in zip(states, pool.map(_oracle_instance_step, tasks, chunksize=1)):
                st[0], st[1], st[2] = Wi, m1, m2
                pts += n
            return pts

        # instances per step: as many as fit ~120 s of wall time over all steps
        t0 = time.perf_counter()
        step(cores, 1)
        per_inst = (time.perf_counter() - t0) / cores
        states = []             # back to the initial weights and moments
        for i in range(w.instances):
            Wi, xi, xb, gb = _instance_sample(w, d, i)
            states.append([Wi, np.zeros(P), np.zeros(P), xi, xb, gb, w.problem(*d["ab"][i])])
        budget = 120.0
        k = int(max(1, min(w.instances, budget * cores / max(1, args.steps + args.warmup) / max(per_inst, 1e-6))))
        for t in range(1, args.warmup + 1):
            step(k, t)
        t0 = time.perf_counter()
        pts = 0
        for t in range(args.warmup + 1, args.warmup + args.steps + 1):
            pts = step(k, t)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    value = args.steps * pts / dt
    desc = (f"the first {k} of {w.instances} instances, 256 interior + 32 boundary points of each per step, "
            f"{cores} worker processes")
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
          "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": args.workload, "instances": w.instances, "widths": w.widths, "G": w.G, "k": w.k,
                     "m": w.m, "impl": f"FP64 CPU oracle (C, {cores} worker processes)"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def run_reference(args, ws, rank):
    """FP64 CPU oracle, as it stands, on a bounded sample of the workload per step."""
    if rank != 0:
        return
    import oracle
    from paper_2409_14248_gb300 import inputs
    oracle.build()
    w = inputs.WORKLOADS[args.workload]
    if w.instances > 1:
        run_reference_batched(args, w)
        return
    full = w.n_int + w.n_bnd + w.n_ic + w.n_bc
    # calibrate the oracle's rate, then size the sample so that the run takes ~2 minutes
    d = sample_data(inputs, w, 128, 16)
    Wd = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wd), np.zeros_like(Wd)
    t0 = time.perf_counter()
    oracle.train_step(w.net, w.problem(), Wd, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, 1)
    rate = 144 / (time.perf_counter() - t0)
    budget = 120.0
    per_step = int(max(64, min(full, budget / max(1, args.steps + args.warmup) * rate)))
    n_int = max(16, per_step * w.n_int // full)
    d = sample_data(inputs, w, n_int, max(4, per_step - n_int))
    Wd = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wd), np.zeros_like(Wd)
    pts = d["x_int"].shape[1] + d["x_bnd"].shape[1]
    for t in range(1, args.warmup + 1):
        oracle.train_step(w.net, w.problem(), Wd, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, t)
    t0 = time.perf_counter()
    for t in range(args.warmup + 1, args.warmup + args.steps + 1):
        oracle.train_step(w.net, w.problem(), Wd, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, t)
    dt = time.perf_counter() - t0
    value = args.steps * pts / dt
    sample = f"{d['x_int'].shape[1]} interior + {d['x_bnd'].shape[1]} boundary/initial points per step " \
             f"(of {w.n_int} + {w.n_bnd + w.n_ic + w.n_bc}), same distribution and seed"
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
          "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": args.workload, "widths": w.widths, "G": w.G, "k": w.k, "m": w.m,
                     "n_int": w.n_int, "n_bnd": w.n_bnd + w.n_ic + w.n_bc, "impl": "FP64 CPU oracle (C, 1 thread)"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ------------------------------------------------------------ many instances

LB_CHUNK_CANDIDATES = (1024, 2048, 4096, 8192, 16384)
KIND_NAMES = {5: "tc_fwd_kernel", 6: "tc_dw_kernel", 7: "tc_adj_kernel", 8: "wide_fwd_kernel",
              9: "wide_dw_kernel", 10: "wide_adjoint_kernel", 3: "lb_tail_kernel (output layer, residual, reverse)",
              1: "batch_reduce_kernel"}


def layerwise_kind_work(widths, G, k, J, n_int, n_bnd, prec, fwd_tc=True):
    """Algorithmic work of one multi-instance step on the layer-wise path per kernel kind:
    (amount, unit) with unit "flop" (dense contraction flops for the tensor-core kinds, every K
    column counted; sparse flops of the k+1 active bases for the FP32 kinds, the fused
    output-layer kernel (kind 3) included) or "byte" (the stand-alone residual of single-layer
    networks).  Interior points carry J jet rows, boundary points one.  fwd_tc False: path 2, every
    forward on the FP32 SIMT kernels."""
    n, kp = G + k, k + 1
    L = len(widths) - 1
    rows = J * n_int + n_bnd
    pts = n_int + n_bnd
    tc_ok = lambda l: prec != 0 and 0 < l < L - 1 and 16 <= widths[l + 1] <= 64 and widths[l + 1] % 16 == 0
    tc_dw_ok = lambda l: prec == 1 and (tc_ok(l) or (l == 0 and 16 <= widths[1] <= 64 and widths[1] % 16 == 0))
    w = {5: 0, 6: 0, 7: 0, 8: 0, 9: 0, 10: 0, 3: 0}
    for l in range(L):
        I, O = widths[l], widths[l + 1]
        if l == L - 1 and L >= 2:
            # the output layer runs in the fused output-layer kernel: forward and input adjoint
            # of the layer (sparse) and its weight gradient, all points
            w[3] += 2 * kp * I * O * rows * 3 + (20 + 25) * kp * I * pts
            continue
        if tc_ok(l) and fwd_tc:
            w[5] += 2 * rows * I * n * O
        else:
            w[8] += 2 * kp * I * O * rows + 20 * kp * I * pts
        if tc_dw_ok(l):
            w[6] += 2 * rows * I * n * O
        else:
            w[9] += 2 * kp * I * O * rows + 20 * kp * I * pts
        if l > 0:
            if tc_ok(l) and prec == 1:
                w[7] += 2 * J * n_int * I * n * O
                w[10] += 2 * kp * I * O * n_bnd + 25 * kp * I * n_bnd
            else:
                w[10] += 2 * kp * I * O * rows + 25 * kp * I * pts
    out = {c: (v, "flop") for c, v in w.items()}
    if L < 2:   # a single layer: the residual runs alone (coordinates, jets in, jet gradients out)
        out[3] = ((2 + 2 * J) * 4 * n_int + 3 * 4 * n_bnd, "byte")
    return out


# DRAM bytes (read + write) of one BF16 step per kernel kind, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, the mean of three steps) of the 16-instance case
# of the batching workload (293 920 interior + 36 734 boundary points; command and figures in
# profiles/batched_bf16_step_poisson_batch256.md), scaled to a run by its points.  Only valid for
# the kernels as captured: retake the capture when one of them changes.  The input adjoint
# (kind 7; 168.28 MB at that capture) has changed since, so it has no figure here.
TRAFFIC_BATCH16 = {"points": 330654,
                   "bytes": {5: 142.75e6, 6: 198.25e6, 3: 117.14e6}}


def layerwise_tc_bytes(widths, G, k, J, n_int, n_bnd, prec, fwd_tc=True):
    """Algorithmic DRAM bytes of the tensor-core kinds of one multi-instance step on the
    layer-wise path (each tensor read or written once): the forward (kind 5) reads the
    layer's input jets and writes its output jets in FP32; the weight gradient (kind 6) reads
    the input jets (the two coordinates for the first layer) and the BF16 output gradient; the
    input adjoint (kind 7, interior points) reads the input jets and the BF16 output gradient
    and writes the input gradient, in BF16 when the layer below runs on tensor cores, else
    FP32.  Interior points carry J jet rows, boundary points one; weights are not counted.
    fwd_tc False: path 2, no tensor-core forward."""
    L = len(widths) - 1
    rows = J * n_int + n_bnd
    tc_ok = lambda l: prec != 0 and 0 < l < L - 1 and 16 <= widths[l + 1] <= 64 and widths[l + 1] % 16 == 0
    tc_dw_ok = lambda l: prec == 1 and (tc_ok(l) or (l == 0 and 16 <= widths[1] <= 64 and widths[1] % 16 == 0))
    b = {5: 0, 6: 0, 7: 0}
    for l in range(L - 1):
        I, O = widths[l], widths[l + 1]
        if tc_ok(l) and fwd_tc:
            b[5] += 4 * (I + O) * rows
        if tc_dw_ok(l):
            b[6] += (8 * (n_int + n_bnd) if l == 0 else 4 * I * rows) + 2 * O * rows
        if l > 0 and tc_ok(l) and prec == 1:
            gz = 2 if tc_dw_ok(l - 1) else 4
            b[7] += (4 * I + 2 * O + gz * I) * J * n_int
    return b


def layerwise_batched_launches(widths, G, k, prec, mask, fwd_tc=True):
    """Kernels one multi-instance step of the layer-wise path launches (both point sets present):
    3 point gathers; per set the forward of every layer below the output layer (a tensor-core
    layer adds its weight conversion); the fused output-layer kernel per set; per set the
    backward of the layers below (a tensor-core weight gradient adds a BF16 conversion of its
    gradient unless the layer above wrote it in BF16; a tensor-core adjoint adds its weight
    conversion); the per-instance reduction.  Mirrors the library's kernel choice; fwd_tc False
    is path 2 (every forward on the FP32 SIMT kernels)."""
    n, L = G + k, len(widths) - 1
    J = {0x0F: 4, 0x1F: 5, 0x2F: 5}.get(mask, bin(mask).count("1"))
    np_ok = n <= 64

    def tc_fwd(l, m):
        O, Jm = widths[l + 1], (1 if m == 1 else J)
        return (fwd_tc and prec != 0 and 0 < l < L - 1 and 16 <= O <= 64 and O % 16 == 0 and Jm * O <= 320
                and np_ok and m in (0x01, 0x0F, 0x1F))

    def tc_dw(l, m):
        O = widths[l + 1]
        return prec == 1 and 16 <= O <= 64 and O % 16 == 0 and np_ok and m in (0x01, 0x0F, 0x1F)

    def tc_adj(l, m):
        return tc_dw(l, m) and m != 0x01

    def takes_bf16(l, m):
        return tc_dw(l, m) and (l == 0 or tc_adj(l, m))

    if L < 2:   # separate launches: forward, residual, weight gradient
        return 3 + 2 * 1 + 1 + 2 * 1 + 1
    count = 3 + 2 + 1            # gathers, output-layer kernels, reduction
    for m in (mask, 0x01):
        count += sum(2 if tc_fwd(l, m) else 1 for l in range(L - 1))
        bf = m != 0x01 and takes_bf16(L - 2, m)          # the output-layer kernel's gradient format
        for l in range(L - 2, -1, -1):
            count += (1 if bf else 2) if tc_dw(l, m) else 1
            if l > 0:
                count += 2 if tc_adj(l, m) else 1
                bf = tc_adj(l, m) and takes_bf16(l - 1, m)
    return count


def batched_points(d):
    return int(d["off_int"][-1]), int(d["off_bnd"][-1])


def _oracle_instance_step(task):
    """One FP64 oracle training step of one instance (runs in a worker process); returns the
    instance's updated weights and moments and the points it processed."""
    import oracle
    net, prob, W, m1, m2, xi, mask, xb, gb, lr, t = task
    oracle.train_step(net, prob, W, m1, m2, xi, mask, xb, gb, lr, t)
    return W, m1, m2, xi.shape[1] + xb.shape[1]


def _noop(_):
    return 0


def _oracle_pool():
    """A pool of worker processes, one per host core this process may use, started with "spawn"
    (this process holds a CUDA context) and warmed up outside any timing."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    pool = mp.get_context("spawn").Pool(n)
    pool.map(_noop, range(4 * n))
    return pool, n


def _instance_sample(w, d, i, per_inst=256):
    """Instance i's weights and its first per_inst interior and per_inst // 8 boundary points."""
    P = w.n_params()
    a0, a1 = int(d["off_int"][i]), int(d["off_int"][i + 1])
    b0, b1 = int(d["off_bnd"][i]), int(d["off_bnd"][i + 1])
    ni, nb = min(per_inst, a1 - a0), min(per_inst // 8, b1 - b0)
    return (d["W"][i * P:(i + 1) * P].astype(np.float64), np.ascontiguousarray(d["x_int"][:, a0:a0 + ni]),
            np.ascontiguousarray(d["x_bnd"][:, b0:b0 + nb]), np.ascontiguousarray(d["g_bnd"][b0:b0 + nb]))


def cpu_baseline_batched(w, d):
    """The FP64 oracle on the host cores, one worker process per core, instance by instance: one
    training step on a sample of each instance (the same points and weights), repeated over all
    instances until ~10 s of wall time."""
    P = w.n_params()
    tasks = []
    for i in range(w.instances):
        Wi, xi, xb, gb = _instance_sample(w, d, i)
        tasks.append((w.net, w.problem(*d["ab"][i]), Wi, np.zeros(P), np.zeros(P), xi, w.mask_int, xb, gb, w.lr, 1))
    pool, cores = _oracle_pool()
    try:
        pts, rounds = 0, 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 10.0 and rounds < 20:
            pts += sum(r[3] for r in pool.map(_oracle_instance_step, tasks, chunksize=1))
            rounds += 1
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    return {"value": pts / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one training step on each of the {w.instances} instances, 256 interior + 32 boundary "
                      f"points of each (their own points and weights), {rounds} rounds, FP64, {cores} worker "
                      f"processes"}


# --------------------------------------------------------------------- ours


def sample_data(inputs, w, n_int, n_b):
    """The workload's points with smaller counts (same distribution and seed)."""
    if w.pde == inputs.POISSON:
        return inputs.make(w, n_int=n_int, n_bnd=max(4, n_b))
    return inputs.make(w, n_int=n_int, n_ic=max(1, n_b // 2), n_bc=max(2, n_b - n_b // 2))


def cpu_baseline_leg(w):
    """The FP64 oracle on the host: full training steps of the workload when they
    take ~10 s, else one step on a bounded sample of it."""
    import oracle
    from paper_2409_14248_gb300 import inputs
    oracle.build()
    full = w.n_int + w.n_bnd + w.n_ic + w.n_bc
    d = sample_data(inputs, w, 128, 16)
    Wd = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wd), np.zeros_like(Wd)
    t0 = time.perf_counter()
    oracle.train_step(w.net, w.problem(), Wd, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, 1)
    rate = 144 / (time.perf_counter() - t0)
    if 2 * full <= 15.0 * rate:
        d, steps, what = inputs.make(w), 2, "full training steps of the workload"
    else:
        n = int(max(64, 15.0 * rate))
        d, steps, what = sample_data(inputs, w, n * w.n_int // full, max(4, n - n * w.n_int // full)), 1, \
            "training step on a sample of the workload (same distribution and seed)"
    Wd = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wd), np.zeros_like(Wd)
    t0 = time.perf_counter()
    for t in range(1, steps + 1):
        oracle.train_step(w.net, w.problem(), Wd, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, t)
    dt = time.perf_counter() - t0
    pts = d["x_int"].shape[1] + d["x_bnd"].shape[1]
    return {"value": steps * pts / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} {what} ({pts} points each), FP64, 1 thread"}


PRECS = {"fp32": 0, "bf16": 1, "tf32": 2}


def launches_per_step(widths, prec, tc_fwd, tc_dw, fused):
    """Kernels one training step launches (the layer-wise path: per layer and point
    set a forward, a weight gradient and, past the first layer, an input adjoint;
    a tensor-core call is a conversion kernel plus the contraction)."""
    if fused:
        return 2                     # fused forward+residual+backward, reduction+Adam
    L = len(widths) - 1
    per_set_fwd = sum(2 if tc_fwd(l) else 1 for l in range(L))
    per_set_bwd = sum(2 if tc_dw(l) else 1 for l in range(L)) + (L - 1)
    tc_adj = sum(1 for l in range(1, L) if tc_dw(l) and 0 < l < L - 1)   # interior set (reuses the dW's gy copy)
    return 2 * per_set_fwd + 2 * per_set_bwd + tc_adj * 1 + 2   # + w conversion; residual, reduction+Adam


def time_steps(torch, capi, h, step, first_t, steps, flush):
    """CUDA-event time of `steps` training steps (L2 flushed before each, outside the events)."""
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev_s[i].record()
        step(first_t + i)
        ev_e[i].record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(ev_s, ev_e))


def run_ours(args, ws, rank, local):
    import torch
    from paper_2409_14248_gb300 import build as pbuild
    from paper_2409_14248_gb300 import capi, inputs

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(capi.LIB_PATH):
        pbuild.build()
    if ws > 1:
        torch.distributed.barrier()
    capi.load_library()

    w = inputs.WORKLOADS[args.workload]
    prec = PRECS[args.prec]
    d = inputs.make(w)
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    pts = Ni + Nb
    J = bin(w.mask_int & 0x1F).count("1")
    p = w.problem()
    prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    W0 = dev(d["W"])
    xi, xb, gb = dev(d["x_int"]), dev(d["x_bnd"]), dev(d["g_bnd"])
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    b1, b2, eps = 0.9, 0.999, 1e-8

    def make_step(h, W):
        return lambda t: capi.hrkan_train_step(h, prob, W, xi, Ni, xb, gb, Nb, w.lr, b1, b2, eps, t, loss)

    h = capi.hrkan_init(capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, prec=prec))
    W = W0.clone()
    step = make_step(h, W)
    for t in range(1, args.warmup + 1):
        flush.fill_(0.0)
        step(t)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    capi.hrkan_profile_enable(h, True)
    for c in range(capi.HRKAN_KERNEL_CLASSES):
        capi.hrkan_profile_read(h, c, reset=True)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    total_ms = time_steps(torch, capi, h, step, args.warmup + 1, args.steps, flush)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    capi.hrkan_profile_enable(h, False)
    prof = {c: capi.hrkan_profile_read(h, c) for c in range(capi.HRKAN_KERNEL_CLASSES)}
    fused = prof[capi.HRKAN_KERNEL_FUSED][1] > 0 and prof[capi.HRKAN_KERNEL_FORWARD][1] == 0
    total_ms = max_over_ranks(total_ms, ws, "cuda")

    # end to end through the C ABI with host buffers: H2D of the inputs, the step, D2H of the loss
    pin = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32).pin_memory()
    hxi, hxb, hgb = pin(d["x_int"]), pin(d["x_bnd"]), pin(d["g_bnd"])
    hloss = torch.zeros(3, dtype=torch.float64).pin_memory()
    e2e_steps = min(args.steps, 200)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        xi.copy_(hxi, non_blocking=True)
        xb.copy_(hxb, non_blocking=True)
        gb.copy_(hgb, non_blocking=True)
        step(args.warmup + args.steps + 1 + i)
        hloss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, ws, "cuda")
    h2d = (hxi.numel() + hxb.numel() + hgb.numel()) * 4
    capi.hrkan_destroy(h)

    # the plain FP32 path of the same workload, timed beside a reduced-precision run
    fp32_path = None
    if prec != PRECS["fp32"]:
        h32 = capi.hrkan_init(capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi))
        W32 = W0.clone()
        step32 = make_step(h32, W32)
        for t in range(1, 4):
            step32(t)
        torch.cuda.synchronize()
        k32 = max(3, min(args.steps, 20))
        ms32 = max_over_ranks(time_steps(torch, capi, h32, step32, 4, k32, flush), ws, "cuda")
        capi.hrkan_destroy(h32)
        fp32_path = {"value": job_throughput(ws, k32, pts, ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32 / k32,
                     "steps": k32}

    if rank == 0:
        n = w.G + w.k
        hidden = lambda l: 0 < l < len(w.widths) - 2
        tc_ok = lambda l: hidden(l) and 16 <= w.widths[l + 1] <= 64 and w.widths[l + 1] % 16 == 0 and n <= 64
        tc_fwd = lambda l: prec != PRECS["fp32"] and tc_ok(l)
        tc_dw = lambda l: prec == PRECS["bf16"] and (tc_ok(l) or (l == 0 and 16 <= w.widths[1] <= 64
                                                                   and w.widths[1] % 16 == 0 and n <= 64))
        launches = launches_per_step(w.widths, prec, tc_fwd, tc_dw, fused) * args.steps
        if prec == PRECS["fp32"]:
            fused_ms, fused_n = prof[capi.HRKAN_KERNEL_FUSED]
            red_ms, red_n = prof[capi.HRKAN_KERNEL_REDUCE]
            flops = alg_flops_per_point(w.widths, w.k, J) * Ni + alg_flops_per_point(w.widths, w.k, 1) * Nb
            if fused:
                fused_avg_s = fused_ms / max(1, fused_n) / 1e3
                achieved = flops / fused_avg_s / 1e12
                kernel = f"narrow_grad_kernel<{w.widths}, mask {w.mask_int:#x}, TRAIN>"
                kms = fused_ms / max(1, fused_n)
            else:
                achieved = flops / (total_ms / args.steps / 1e3) / 1e12
                kernel = "layer-wise step (all kernels of one step)"
                kms = total_ms / args.steps
            # DRAM bytes of one launch of the fused kernel from one ncu capture of this workload
            # (its inputs and weights only); unknown for the other shapes
            traffic = 801365 if fused and args.workload == BURGERS_WORKLOAD else None
            roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic, "kernel": kernel, "kernel_ms": kms,
                        "reduce_adam_ms": red_ms / max(1, red_n),
                        "peak_source": FP32_PEAK_NOTE + " (derived, FP32 FMA pipe)"}
        else:
            tc_ms, tc_n = prof[capi.HRKAN_KERNEL_TENSOR]
            pk = measured_peaks()
            peak = pk["bf16_sustained"] * (1.0 if prec == PRECS["bf16"] else 0.5)
            flops = dense_tc_flops(w.widths, w.G, w.k, Ni, J, Nb, prec == PRECS["bf16"])
            achieved = flops * args.steps / (tc_ms / 1e3) / 1e12
            roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": "tc_fwd_kernel + tc_dw_kernel + tc_adj_kernel (hidden layers)"
                        if prec == PRECS["bf16"]
                        else "tc_fwd_kernel (hidden layers)",
                        "kernel_ms_per_step": tc_ms / args.steps, "launches_per_step": tc_n / args.steps,
                        "flops_per_step": flops, "peak_source": ("bf16 dense sustained " if prec == PRECS["bf16"]
                                                                 else "bf16 dense sustained x 0.5 (tf32) ")
                        + pk["source"],
                        "per_kind": {KIND_NAMES[c]: {"ms_per_step": prof[c][0] / args.steps,
                                                     "launches_per_step": prof[c][1] / args.steps}
                                     for c in (5, 6, 7, 8, 9, 10) if prof[c][1] > 0}}
        out = {"metric": METRIC, "value": job_throughput(ws, args.steps, pts, total_ms / 1e3), "unit": UNIT,
               "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
               "data": "synthetic",
               "config": {"workload": args.workload, "widths": w.widths, "G": w.G, "k": w.k, "m": w.m,
                          "n_int": Ni, "n_bnd": Nb, "precision": args.prec,
                          "parallelism": "replicas" if ws > 1 else "single",
                          "l2": "flushed before every timed step (256 MiB device write, outside the step events)"},
               "roofline": roofline, "gpu_launches": launches, "clocks": clocks,
               "e2e": {"value": job_throughput(ws, e2e_steps, pts, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": 24}}
        if fp32_path is not None:
            out["fp32_path"] = fp32_path
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_leg(w)
        emit(out)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def equal_l2_check(torch, capi, inputs, w, prec, n_inst=8, steps=1000, fp32_layerwise=False, reduced_path=1):
    """Both paths trained `steps` Adam steps from the workload's initial weights on its first
    n_inst instances, each on the kernel family the bench timed (fp32_layerwise: the FP32 one
    on the layer-wise kernels; reduced_path: hrkan_set_batch_path of the reduced-precision one);
    mean relative L2 error of u on a 100 x 100 grid against the exact solution, both evaluated
    by the FP32 path."""
    d = inputs.make_batched(w, instances=n_inst)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    probs = [capi.make_problem(w.pde, a, b, w.lam, w.nu, w.alpha) for a, b in d["ab"]]
    xi, xb, gb = dev(d["x_int"]), dev(d["x_bnd"]), dev(d["g_bnd"])
    g = np.linspace(w.lo, w.hi, 100)
    X, Y = np.meshgrid(g, g, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel()]).astype(np.float32)
    xg = dev(np.tile(grid, (1, n_inst)))
    offg = np.arange(n_inst + 1) * grid.shape[1]
    h32 = capi.hrkan_init(capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, n_instances=n_inst))
    capi.hrkan_set_batch_path(h32, 1 if fp32_layerwise else 0)
    out = {}
    try:
        for p in (PRECS["fp32"], prec):
            h = h32 if p == PRECS["fp32"] else capi.hrkan_init(
                capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, prec=p, n_instances=n_inst,
                              flags=capi.HRKAN_FLAG_LAYERWISE))
            try:
                if h is not h32:
                    capi.hrkan_set_batch_path(h, reduced_path)
                W = dev(d["W"])
                loss = torch.zeros((n_inst, 3), dtype=torch.float64, device="cuda")
                for t in range(1, steps + 1):
                    capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], w.lr, 0.9,
                                                  0.999, 1e-8, t, loss)
                u = torch.zeros((1, xg.shape[1]), device="cuda")
                capi.hrkan_forward_jets_batched(h32, W, xg, offg, 0x01, u)
                u = u.cpu().numpy()[0].astype(np.float64)
                errs = []
                for i, (a, b) in enumerate(d["ab"]):
                    want = np.sin(a * np.pi * X.ravel()) * np.sin(b * np.pi * Y.ravel())
                    errs.append(np.linalg.norm(u[offg[i]:offg[i + 1]] - want) / np.linalg.norm(want))
                out[p] = float(np.mean(errs))
            finally:
                if h is not h32:
                    capi.hrkan_destroy(h)
    finally:
        capi.hrkan_destroy(h32)
    return {"instances": n_inst, "steps": steps, "lr": w.lr, "rel_l2_fp32": out[PRECS["fp32"]],
            "rel_l2_reduced": out[prec], "ratio": out[prec] / out[PRECS["fp32"]], "bar": 1.2,
            "grid": "100 x 100 on [-1, 1]^2, u evaluated by the FP32 path"}


def run_batched(args, ws, rank, local):
    import torch
    from paper_2409_14248_gb300 import build as pbuild
    from paper_2409_14248_gb300 import capi, inputs

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(capi.LIB_PATH):
        pbuild.build()
    if ws > 1:
        torch.distributed.barrier()
    capi.load_library()

    w = inputs.WORKLOADS[args.workload]
    if args.instances:   # a K-instance case of the same recipe and seed (a smaller case, e.g. for a profiler)
        w = dataclasses.replace(w, instances=min(args.instances, w.instances))
    prec = PRECS[args.prec]
    d = inputs.make_batched(w)
    I, P = w.instances, w.n_params()
    Ni, Nb = batched_points(d)
    pts = Ni + Nb
    J = bin(w.mask_int & 0x1F).count("1")
    probs = [capi.make_problem(w.pde, a, b, w.lam, w.nu, w.alpha) for a, b in d["ab"]]
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    W0 = dev(d["W"])
    xi, xb, gb = dev(d["x_int"]), dev(d["x_bnd"]), dev(d["g_bnd"])
    loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    b1, b2, eps = 0.9, 0.999, 1e-8

    def make(p):
        flags = 0 if p == PRECS["fp32"] else capi.HRKAN_FLAG_LAYERWISE
        return capi.hrkan_init(capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, prec=p, n_instances=I,
                                             flags=flags))

    def make_step(h, W):
        return lambda t: capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], w.lr, b1,
                                                       b2, eps, t, loss)

    def tune(h, W, p):
        # the layer-wise path tunes its weight-gradient chunk, the fused path its work item;
        # the FP32 handle (a fused shape) times both kernel families and keeps the faster
        cands = LB_CHUNK_CANDIDATES if p != PRECS["fp32"] else (256, 1024, 2048, 4096, 8192)
        chosen, ms = capi.hrkan_autotune_batch(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], candidates=cands)
        path = capi.hrkan_batch_path(h)
        return {"points": chosen, "ms_per_step": ms, "path_id": path,
                "path": {0: "fused multi-instance kernel", 1: "layer-wise kernels",
                         2: "layer-wise kernels, every forward on the FP32 SIMT kernels"}[path],
                "knob": "weight-gradient chunk (points)" if path else "work item (points)"}

    h = make(prec)
    W = W0.clone()
    tuned = tune(h, W, prec)
    step = make_step(h, W)
    for t in range(1, args.warmup + 1):
        flush.fill_(0.0)
        step(t)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    total_ms = time_steps(torch, capi, h, step, args.warmup + 1, args.steps, flush)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = max_over_ranks(total_ms, ws, "cuda")

    # per-kernel times: CUDA events the library records around each launch, over a few more
    # steps of the same workload (kept out of the timed region above)
    prof_steps = min(args.steps, 10)
    capi.hrkan_profile_enable(h, True)
    for c in range(capi.HRKAN_KERNEL_CLASSES):
        capi.hrkan_profile_read(h, c, reset=True)
    time_steps(torch, capi, h, step, args.warmup + args.steps + 1, prof_steps, flush)
    capi.hrkan_profile_enable(h, False)
    prof = {c: capi.hrkan_profile_read(h, c) for c in range(capi.HRKAN_KERNEL_CLASSES)}

    # end to end through the C ABI with host buffers: H2D of the points, the step, D2H of the losses
    pin = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32).pin_memory()
    hxi, hxb, hgb = pin(d["x_int"]), pin(d["x_bnd"]), pin(d["g_bnd"])
    hloss = torch.zeros((I, 3), dtype=torch.float64).pin_memory()
    e2e_steps = min(args.steps, 50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        xi.copy_(hxi, non_blocking=True)
        xb.copy_(hxb, non_blocking=True)
        gb.copy_(hgb, non_blocking=True)
        step(args.warmup + args.steps + prof_steps + 1 + i)
        hloss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
    h2d = (hxi.numel() + hxb.numel() + hgb.numel()) * 4
    capi.hrkan_destroy(h)

    # the plain FP32 path of the same workload (autotuned over both kernel families)
    fp32_path = None
    if prec != PRECS["fp32"] and not args.no_fp32_path:
        h32 = make(PRECS["fp32"])
        W32 = W0.clone()
        tuned32 = tune(h32, W32, PRECS["fp32"])
        step32 = make_step(h32, W32)
        for t in range(1, 4):
            step32(t)
        torch.cuda.synchronize()
        k32 = max(3, min(args.steps, 20))
        ms32 = max_over_ranks(time_steps(torch, capi, h32, step32, 4, k32, flush), ws, "cuda")
        capi.hrkan_destroy(h32)
        fp32_path = {"value": job_throughput(ws, k32, pts, ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32 / k32,
                     "steps": k32, "kernel": "FP32 multi-instance step, " + tuned32["path"] + " (autotuned)",
                     "autotune": tuned32}

    if rank == 0:
        fwd_tc = tuned["path_id"] != 2
        work = layerwise_kind_work(w.widths, w.G, w.k, J, Ni, Nb, prec, fwd_tc)
        kinds = [c for c in work if prof[c][1] > 0]
        dom = max(kinds, key=lambda c: prof[c][0]) if kinds else None
        pk = measured_peaks()
        per_kind = {KIND_NAMES[c]: {"ms_per_step": prof[c][0] / prof_steps, "launches_per_step": prof[c][1] / prof_steps}
                    for c in kinds}
        roofline = None
        if dom is not None:
            amount, unit = work[dom]
            secs = prof[dom][0] / prof_steps / 1e3
            other = None
            if unit == "byte":
                achieved, peak, bound, u, src = amount / secs / 1e9, pk["hbm"], "hbm", "GB/s", pk["hbm_source"]
            elif dom in (5, 6, 7):
                # a tensor-core kind: dense flops against the tensor peak and algorithmic bytes
                # against HBM; the bound is the one whose time at peak is longer
                tpeak = pk["bf16_sustained"] * (1.0 if prec == PRECS["bf16"] else 0.5)
                nbytes = layerwise_tc_bytes(w.widths, w.G, w.k, J, Ni, Nb, prec, fwd_tc)[dom]
                t_tensor, t_hbm = amount / (tpeak * 1e12), nbytes / (pk["hbm"] * 1e9)
                tensor = {"bound": "tensor", "achieved": amount / secs / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                          "work_per_step": amount, "work_unit": "flop",
                          "peak_source": "bf16 dense sustained " + pk["source"]}
                hbm = {"bound": "hbm", "achieved": nbytes / secs / 1e9, "peak": pk["hbm"], "unit": "GB/s",
                       "work_per_step": nbytes, "work_unit": "byte", "peak_source": pk["hbm_source"]}
                first, second = (hbm, tensor) if t_hbm >= t_tensor else (tensor, hbm)
                bound, achieved, peak, u, src = (first["bound"], first["achieved"], first["peak"], first["unit"],
                                                 first["peak_source"])
                amount, unit = first["work_per_step"], first["work_unit"]
                other = dict(second, frac=second["achieved"] / second["peak"])
            else:
                achieved, peak, bound, u = amount / secs / 1e12, FP32_PEAK_TFLOPS, "alu", "TFLOP/s"
                src = FP32_PEAK_NOTE + " (derived, FP32 FMA pipe)"
            roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": u, "frac": achieved / peak,
                        "traffic": None, "kernel": KIND_NAMES[dom], "kernel_ms_per_step": secs * 1e3,
                        "launches_per_step": prof[dom][1] / prof_steps, "work_per_step": amount,
                        "work_unit": unit, "peak_source": src, "per_kind": per_kind}
            if other is not None:
                roofline["other_bound"] = other
            if args.workload == WORKLOAD and prec == PRECS["bf16"] and dom in TRAFFIC_BATCH16["bytes"]:
                roofline["traffic"] = TRAFFIC_BATCH16["bytes"][dom] * pts / TRAFFIC_BATCH16["points"]
                roofline["traffic_note"] = ("DRAM bytes per step of this kernel kind, ncu on the 16-instance case "
                                            "scaled by points (outputs partly still in L2 at that size)")
        # the fused family: the multi-instance kernel and the per-instance reduction
        per_step = 2 if tuned["path_id"] == 0 else layerwise_batched_launches(w.widths, w.G, w.k, prec, w.mask_int,
                                                                               fwd_tc)
        launches = per_step * args.steps
        out = {"metric": METRIC, "value": job_throughput(ws, args.steps, pts, total_ms / 1e3), "unit": UNIT,
               "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
               "data": "synthetic",
               "config": {"workload": args.workload, "instances": I, "widths": w.widths, "G": w.G, "k": w.k,
                          "m": w.m, "n_int": Ni, "n_bnd": Nb, "precision": args.prec,
                          "kernels": tuned["path"],
                          "parallelism": "replicas" if ws > 1 else "single",
                          "l2": "flushed before every timed step (256 MiB device write, outside the step events)"},
               "roofline": roofline, "gpu_launches": int(round(launches)), "clocks": clocks, "autotune": tuned,
               "e2e": {"value": job_throughput(ws, e2e_steps, pts, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": I * 3 * 8}}
        if fp32_path is not None:
            out["fp32_path"] = fp32_path
            if not args.no_equal_l2:
                out["equal_l2"] = equal_l2_check(torch, capi, inputs, w, prec, fp32_layerwise=tuned32["path_id"] != 0,
                                                 reduced_path=tuned["path_id"])
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_batched(w, d)
        emit(out)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="default: 200 for poisson_batch256, else 2000")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-equal-l2", action="store_true", help="skip the 1000-step equal-L2 training check")
    ap.add_argument("--no-fp32-path", action="store_true",
                    help="multi-instance workloads: skip timing the FP32 path beside the reduced-precision one "
                         "(fp32_path is then null; e.g. for a profiler)")
    ap.add_argument("--instances", type=int, default=0,
                    help="multi-instance workloads: K instances drawn by the same recipe and seed (0 = all)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="poisson_batch256 (default), burgers_2_10_10_1, poisson_2_64x3_1, burgers_2_32_32_1, "
                         "poisson_2_5_1")
    ap.add_argument("--prec", default=None, choices=sorted(PRECS),
                    help="default: bf16 for poisson_batch256, fp32 otherwise")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.prec is None:
        args.prec = "bf16" if args.workload == WORKLOAD else "fp32"
    if args.steps is None:
        args.steps = 200 if args.workload == WORKLOAD else 2000
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    from paper_2409_14248_gb300 import inputs
    if inputs.WORKLOADS[args.workload].instances > 1:
        run_batched(args, ws, rank, local)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
