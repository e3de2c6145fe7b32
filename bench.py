#!/usr/bin/env python
"""Throughput of HRKAN physics-informed training on GB300.

One step = one full-batch pass of the whole hot path over the workload's
collocation points: forward jets (u, u_x, u_t, u_xx), Burgers residual and
loss, backward (weight gradient), cross-block reduction and Adam.  Workload:
viscous Burgers u_t + u u_x = nu u_xx, nu = 0.01/pi, HRKAN [2,10,10,1], G=10,
k=3, m=4, 65536 interior + 4096 initial + 4096 boundary points (Latin
hypercube, seed 1), FP32 path.  Inputs are synthetic and resident in HBM when
the timed region starts; they are far smaller than L2, so L2 is flushed
(a 256 MiB device write) before every timed step, outside its events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference there is: the
paper ships no code) on the host cores, a bounded sample of the same workload
per step.  Under torchrun with N > 1 every rank trains its own replica (the
workload does not need a collective), and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
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
WORKLOAD = "burgers_2_10_10_1"
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


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


# --------------------------------------------------------------- reference


def run_reference(args, ws, rank):
    """FP64 CPU oracle, as it stands, on a bounded sample of the workload per step."""
    if rank != 0:
        return
    import oracle
    from paper_2409_14248_gb300 import inputs
    oracle.build()
    w = inputs.WORKLOADS[WORKLOAD]
    full = w.n_int + w.n_ic + w.n_bc
    # calibrate the oracle's rate, then size the sample so that the run takes ~2 minutes
    d = inputs.make(w, n_int=512, n_ic=32, n_bc=32)
    Wd = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wd), np.zeros_like(Wd)
    t0 = time.perf_counter()
    oracle.train_step(w.net, w.problem(), Wd, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, 1)
    rate = 576 / (time.perf_counter() - t0)
    budget = 120.0
    per_step = int(max(64, min(full, budget / max(1, args.steps + args.warmup) * rate)))
    n_int = max(16, per_step * w.n_int // full)
    n_b = max(2, (per_step - n_int) // 2)
    d = inputs.make(w, n_int=n_int, n_ic=n_b, n_bc=n_b)
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
    sample = f"{d['x_int'].shape[1]} interior + {d['x_bnd'].shape[1]} initial/boundary points per step " \
             f"(of {w.n_int} + {w.n_ic + w.n_bc}), same distribution and seed"
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
          "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": WORKLOAD, "widths": w.widths, "G": w.G, "k": w.k, "m": w.m,
                     "n_int": w.n_int, "n_bnd": w.n_ic + w.n_bc, "impl": "FP64 CPU oracle (C, 1 thread)"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# --------------------------------------------------------------------- ours


def cpu_baseline_leg(w):
    """The FP64 oracle on the host: 2 full steps of the same workload (~10 s)."""
    import oracle
    from paper_2409_14248_gb300 import inputs
    oracle.build()
    d = inputs.make(w)
    Wd = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wd), np.zeros_like(Wd)
    steps = 2
    t0 = time.perf_counter()
    for t in range(1, steps + 1):
        oracle.train_step(w.net, w.problem(), Wd, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, t)
    dt = time.perf_counter() - t0
    pts = d["x_int"].shape[1] + d["x_bnd"].shape[1]
    return {"value": steps * pts / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} full training steps of the workload ({pts} points each), FP64, 1 thread"}


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

    w = inputs.WORKLOADS[WORKLOAD]
    d = inputs.make(w)
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    pts = Ni + Nb
    cfg = capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi)
    h = capi.hrkan_init(cfg)
    p = w.problem()
    prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    W = dev(d["W"])
    xi, xb, gb = dev(d["x_int"]), dev(d["x_bnd"]), dev(d["g_bnd"])
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    b1, b2, eps = 0.9, 0.999, 1e-8

    def step(t):
        capi.hrkan_train_step(h, prob, W, xi, Ni, xb, gb, Nb, w.lr, b1, b2, eps, t, loss)

    for t in range(1, args.warmup + 1):
        flush.fill_(0.0)
        step(t)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    capi.hrkan_profile_enable(h, True)
    for c in range(5):
        capi.hrkan_profile_read(h, c, reset=True)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.fill_(float(i))
        ev_s[i].record()
        step(args.warmup + 1 + i)
        ev_e[i].record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    capi.hrkan_profile_enable(h, False)
    total_ms = sum(a.elapsed_time(b) for a, b in zip(ev_s, ev_e))
    fused_ms, fused_n = capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_FUSED)
    red_ms, red_n = capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_REDUCE)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    launches = fused_n + red_n

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
    if ws > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = (hxi.numel() + hxb.numel() + hgb.numel()) * 4
    capi.hrkan_destroy(h)

    if rank == 0:
        J = 4
        flops = alg_flops_per_point(w.widths, w.k, J) * Ni + alg_flops_per_point(w.widths, w.k, 1) * Nb
        fused_avg_s = fused_ms / max(1, fused_n) / 1e3
        achieved = flops / fused_avg_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                    "kernel": "narrow_grad_kernel<[2,10,10,1], mask 0x0F, TRAIN>",
                    "kernel_ms": fused_ms / max(1, fused_n), "reduce_adam_ms": red_ms / max(1, red_n),
                    "peak_source": FP32_PEAK_NOTE + " (derived, FP32 FMA pipe)"}
        out = {"metric": METRIC, "value": ws * args.steps * pts / (total_ms / 1e3), "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "widths": w.widths, "G": w.G, "k": w.k, "m": w.m, "n_int": Ni,
                          "n_bnd": Nb, "precision": "fp32", "parallelism": "replicas" if ws > 1 else "single",
                          "l2": "flushed before every timed step (256 MiB device write, outside the step events)"},
               "roofline": roofline, "gpu_launches": launches, "clocks": clocks,
               "e2e": {"value": ws * e2e_steps * pts / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": 24}}
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_leg(w)
        emit(out)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
