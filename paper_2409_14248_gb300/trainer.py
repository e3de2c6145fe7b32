"""Training driver with metrics logging and checkpoints.

Runs full-batch Adam steps (Section 4) of one workload through
hrkan_train_step, and every `log_every` steps appends one JSON line:

    {"step": t, "loss": L, "loss_pde": L_pde, "loss_bnd": L_bnd,
     "points_per_s": ..., "ms_per_step": ..., "test_rel_l2": ...}

test_rel_l2 is the relative L2 error of u on a test grid against the exact
solution: sin(a pi x) sin(b pi y) for Poisson; for Burgers with lam = 1 on
x in [-1, 1], t in [0, 1] and u(x, 0) = -sin(pi x) the Cole-Hopf solution
(truth.burgers_sine); null otherwise.

`checkpoint_every` writes a checkpoint (hrkan_save: weights, Adam moments, step
count) and `resume` continues from one, so an interrupted run can be restarted
with the same step numbering and optimiser state.  Every step, loss and error
evaluation runs in libhrkan.so; torch only holds device memory and the timing
events.
"""
from __future__ import annotations

import json

import numpy as np

from . import capi, inputs, truth


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


class Trainer:
    def __init__(self, workload: inputs.Workload | str, prec: int = capi.HRKAN_FP32, flags: int = 0,
                 data: dict | None = None, test_grid: int = 64):
        import torch
        self.w = inputs.WORKLOADS[workload] if isinstance(workload, str) else workload
        self.d = data if data is not None else inputs.make(self.w)
        self.cfg = capi.make_cfg(self.w.widths, self.w.G, self.w.k, self.w.m, self.w.lo, self.w.hi, prec=prec,
                                 flags=flags)
        self.h = capi.hrkan_init(self.cfg)
        p = self.w.problem()
        self.prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
        self.W = _dev(self.d["W"])
        self.x_int, self.x_bnd, self.g_bnd = _dev(self.d["x_int"]), _dev(self.d["x_bnd"]), _dev(self.d["g_bnd"])
        self.n_int, self.n_bnd = self.d["x_int"].shape[1], self.d["x_bnd"].shape[1]
        self.loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        self.t = 0
        self.x_test = self.u_test = None
        g = np.linspace(self.w.lo, self.w.hi, test_grid)
        if self.w.pde == inputs.POISSON:
            X, Y = np.meshgrid(g, g, indexing="ij")
            pts = np.stack([X.ravel(), Y.ravel()]).astype(np.float32)
            self.u_test = truth.poisson(pts[0], pts[1], self.w.a, self.w.b)
            self.x_test = _dev(pts)
        elif self.w.pde == inputs.BURGERS and self.w.lam == 1.0 and (self.w.lo, self.w.hi) == (-1.0, 1.0):
            X, T = np.meshgrid(g, np.linspace(0.0, 1.0, test_grid), indexing="ij")
            pts = np.stack([X.ravel(), T.ravel()]).astype(np.float32)
            self.u_test = truth.burgers_sine(pts[0], pts[1], self.w.nu)
            self.x_test = _dev(pts)

    def test_rel_l2(self):
        """Relative L2 error of u on the test grid (None without an exact solution)."""
        import torch
        if self.x_test is None:
            return None
        u = torch.zeros((1, self.x_test.shape[1]), device="cuda")
        capi.hrkan_forward_jets(self.h, self.W, self.x_test, self.x_test.shape[1], 0x01, u)
        got = u.cpu().numpy()[0].astype(np.float64)
        return float(np.linalg.norm(got - self.u_test) / np.linalg.norm(self.u_test))

    def step(self, lr: float | None = None):
        self.t += 1
        capi.hrkan_train_step(self.h, self.prob, self.W, self.x_int, self.n_int, self.x_bnd, self.g_bnd, self.n_bnd,
                              self.w.lr if lr is None else lr, 0.9, 0.999, 1e-8, self.t, self.loss)

    def run(self, steps: int, log_path: str | None = None, log_every: int = 100, checkpoint_path: str | None = None,
            checkpoint_every: int = 0, lr: float | None = None) -> list:
        """`steps` more steps; returns the logged records (also appended to log_path as JSON lines)."""
        import torch
        records = []
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        last_t = self.t
        start.record()
        for _ in range(steps):
            self.step(lr)
            if checkpoint_path and checkpoint_every and self.t % checkpoint_every == 0:
                capi.hrkan_save(self.h, self.W, self.t, checkpoint_path)
            if self.t % log_every == 0 or self.t == last_t + steps:
                stop.record()
                stop.synchronize()
                n = self.t - (records[-1]["step"] if records else last_t)
                ms = start.elapsed_time(stop) / max(n, 1)
                capi.hrkan_sync_status(self.h)   # raises on a non-finite loss or a device timeout
                loss = self.loss.cpu().numpy()
                rec = {"step": self.t, "loss": float(loss[0]), "loss_pde": float(loss[1]),
                       "loss_bnd": float(loss[2]), "ms_per_step": ms,
                       "points_per_s": (self.n_int + self.n_bnd) / (ms * 1e-3), "test_rel_l2": self.test_rel_l2()}
                records.append(rec)
                if log_path:
                    with open(log_path, "a") as f:
                        f.write(json.dumps(rec) + "\n")
                start.record()
        return records

    def resume(self, checkpoint_path: str):
        """Load weights, Adam moments and the step count from a checkpoint."""
        self.t = capi.hrkan_load(self.h, self.W, checkpoint_path)

    def close(self):
        if self.h is not None:
            capi.hrkan_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def read_log(path: str) -> list:
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


__all__ = ["Trainer", "read_log"]
