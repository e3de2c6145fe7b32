"""The paper's Poisson experiment (Section 4.1) on this library.

Problem (Section 4.1): laplacian(u) = -2 pi^2 sin(pi x) sin(pi y) on [-1, 1]^2,
u = 0 on the boundary, exact solution u* = sin(pi x) sin(pi y).  Training set:
960 interior points drawn uniformly at random and 30 evenly spaced points on
each of the 4 edges; loss L = alpha L_pde + L_bc with alpha = 0.05; a [2,2,1]
network with g = 5, k = 3; Adam for 3000 epochs (full batch); test set: the
100 x 100 grid.  The paper reports the mean and standard deviation of the test
MSE over 10 runs and the mean training time (Table 1, HRKAN column, and the
ReLU-KAN column, which is the m = 2 case of Eq. 2).  It does not state the
learning rate, the Adam constants or the initial weights: they are parameters
here (defaults lr = 1e-3, betas (0.9, 0.999), eps 1e-8, N(0, 0.1^2)).

Everything runs in libhrkan.so (hrkan_train_step on the layer-wise path for
this width, hrkan_forward_jets for the test set); torch only holds device
memory.
"""
from __future__ import annotations

import time

import numpy as np

from . import capi, inputs


def poisson_sets(seed: int):
    """(x_int [2, 960], x_bnd [2, 120], g_bnd [120], x_test [2, 10000], u_test [10000]) of Section 4.1."""
    rng = np.random.default_rng(seed)
    x_int = rng.uniform(-1.0, 1.0, (2, 960))
    t = np.linspace(-1.0, 1.0, 30)
    one = np.ones(30)
    x_bnd = np.concatenate([np.stack([-one, t]), np.stack([one, t]), np.stack([t, -one]), np.stack([t, one])], axis=1)
    g = np.linspace(-1.0, 1.0, 100)
    X, Y = np.meshgrid(g, g, indexing="ij")
    x_test = np.stack([X.ravel(), Y.ravel()])
    u_test = np.sin(np.pi * x_test[0]) * np.sin(np.pi * x_test[1])
    return (x_int.astype(np.float32), x_bnd.astype(np.float32), np.zeros(x_bnd.shape[1], np.float32),
            x_test.astype(np.float32), u_test)


def train_poisson(m: int = 4, seed: int = 0, epochs: int = 3000, lr: float = 1e-3, alpha: float = 0.05,
                  sigma: float = 0.1, widths=(2, 2, 1), G: int = 5) -> dict:
    """One run: returns test MSE (as a fraction, the paper prints percent), the final
    training loss and the wall-clock training seconds (device synchronised)."""
    import torch
    x_int, x_bnd, g_bnd, x_test, u_test = poisson_sets(seed)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    cfg = capi.make_cfg(list(widths), G, 3, m, -1.0, 1.0)
    P = capi.hrkan_param_count(cfg)
    W0 = inputs.init_weights(P, 1000 + seed, sigma=sigma)
    prob = capi.make_problem(capi.HRKAN_POISSON, 1.0, 1.0, 1.0, 0.0, alpha)
    h = capi.hrkan_init(cfg)
    try:
        W = dev(W0)
        xi, xb, gb = dev(x_int), dev(x_bnd), dev(g_bnd)
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(1, epochs + 1):
            capi.hrkan_train_step(h, prob, W, xi, x_int.shape[1], xb, gb, x_bnd.shape[1], lr, 0.9, 0.999, 1e-8, t,
                                  loss)
        torch.cuda.synchronize()
        seconds = time.perf_counter() - t0
        u = torch.zeros((1, x_test.shape[1]), device="cuda")
        capi.hrkan_forward_jets(h, W, dev(x_test), x_test.shape[1], 0x01, u)
        pred = u.cpu().numpy()[0].astype(np.float64)
        final = loss.cpu().numpy()
    finally:
        capi.hrkan_destroy(h)
    return {"test_mse": float(np.mean((pred - u_test) ** 2)), "train_loss": float(final[0]), "seconds": seconds,
            "m": m, "seed": seed, "lr": lr}


def table(runs: int = 10, m: int = 4, **kw) -> dict:
    """Mean / std of the test MSE (percent) and mean training seconds over `runs` seeds, as in Table 1."""
    res = [train_poisson(m=m, seed=s, **kw) for s in range(runs)]
    mse = np.array([r["test_mse"] for r in res]) * 100.0
    return {"mean_mse_pct": float(mse.mean()), "std_mse_pct": float(mse.std()),
            "median_mse_pct": float(np.median(mse)), "mean_seconds": float(np.mean([r["seconds"] for r in res])),
            "runs": res}
