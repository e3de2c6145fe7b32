"""The paper's two experiments (Sections 4.1 and 4.2) on this library.

Poisson (Section 4.1): laplacian(u) = -2 pi^2 sin(pi x) sin(pi y) on [-1, 1]^2,
u = 0 on the boundary, exact solution u* = sin(pi x) sin(pi y).  Training set:
960 interior points drawn uniformly at random and 30 evenly spaced points on
each of the 4 edges; loss L = alpha L_pde + L_bc with alpha = 0.05; a [2,2,1]
network with g = 5, k = 3; Adam for 3000 epochs (full batch); test set: the
100 x 100 grid.

Burgers (Section 4.2): u_t + u u_x - nu u_xx = 0 on [-5, 5] x [0, 2.5] with
nu = 0.001, u(+-5, t) = 0 and u(x, 0) = sech(x), solved after the change of
variable y = (x + 5) / 4 on the square [0, 2.5]^2, where it reads
u_t + (1/4) u u_y - (nu/16) u_yy = 0 (Eq. 7; the library's Burgers residual with
lam = 1/4 and nu/16), u(0, t) = u(2.5, t) = 0, u(y, 0) = sech(4y - 5).
Training set: 10000 interior points drawn uniformly at random, 100 evenly
spaced points on each of the two boundaries and on the initial line, one
pooled boundary mean in the loss (Eq. 8) with alpha = 0.05; a [2,3,3,3,1]
network with g = 7, k = 3; Adam for 3000 epochs; test set: the 200 x 200 grid.
The paper's reference solution comes from a Fourier solver; here it is the
Cole-Hopf solution of the same initial value problem on the whole line
(`burgers_truth`, by truth.burgers_sech).  At y = 0 and y = 2.5 it keeps the
initial value's tail (sech 5 = 0.0135) instead of the Dirichlet zero, which
moves the test MSE by about 2e-6 (0.0002 %).

The paper reports the mean and standard deviation of the test MSE over 10
runs and the mean training time (Tables 1 and 2; the ReLU-KAN column is the
m = 2 case of Eq. 2).  It does not state the learning rate, the Adam constants
or the initial weights: they are parameters here (defaults lr = 1e-3, betas
(0.9, 0.999), eps 1e-8, N(0, 0.1^2)).

Every training step and the test-set forward run in libhrkan.so
(hrkan_train_step on the layer-wise path for these widths, hrkan_forward_jets);
torch only holds device memory.
"""
from __future__ import annotations

import functools
import time

import numpy as np

from . import capi, inputs, truth

BURGERS_NU = 1e-3
BURGERS_SIDE = 2.5


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


def burgers_truth(y, t, nu: float = BURGERS_NU):
    """Reference solution of the rescaled problem (Eq. 7) at (y, t) in [0, 2.5]^2: u(4y - 5, t)."""
    return truth.burgers_sech(4.0 * np.asarray(y, np.float64) - 5.0, t, nu)


def burgers_sets(seed: int, n_test: int = 200):
    """(x_int [2, 10000], x_bnd [2, 300], g_bnd [300], x_test [2, n_test^2], u_test) of Section 4.2.

    Coordinates are (y, t).  x_bnd holds the 100 points of y = 0, then the 100
    of y = 2.5 (t evenly spaced on [0, 2.5]), then the 100 initial points
    (y evenly spaced, t = 0) with target sech(4y - 5)."""
    rng = np.random.default_rng(seed)
    L = BURGERS_SIDE
    x_int = rng.uniform(0.0, L, (2, 10000))
    s = np.linspace(0.0, L, 100)
    z = np.zeros(100)
    x_bnd = np.concatenate([np.stack([z, s]), np.stack([z + L, s]), np.stack([s, z])], axis=1)
    g_bnd = np.concatenate([z, z, 1.0 / np.cosh(4.0 * s - 5.0)])
    x_test, u_test = _burgers_test_grid(n_test)
    return (x_int.astype(np.float32), x_bnd.astype(np.float32), g_bnd.astype(np.float32), x_test.copy(),
            u_test.copy())


@functools.lru_cache(maxsize=4)
def _burgers_test_grid(n_test: int):
    """The n_test x n_test test grid and the truth there (the same for every seed, so computed once)."""
    g = np.linspace(0.0, BURGERS_SIDE, n_test)
    Y, T = np.meshgrid(g, g, indexing="ij")
    x_test = np.stack([Y.ravel(), T.ravel()]).astype(np.float32)   # the truth at the coordinates the net sees
    return x_test, burgers_truth(x_test[0], x_test[1])


def _train(cfg, prob, sets, seed: int, epochs: int, lr: float, sigma: float) -> dict:
    """Full-batch Adam through hrkan_train_step, then the test-set forward.

    Returns the test MSE (a fraction; the paper prints percent), the final
    training loss and the wall-clock training seconds (device synchronised)."""
    import torch
    x_int, x_bnd, g_bnd, x_test, u_test = sets
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    W0 = inputs.init_weights(capi.hrkan_param_count(cfg), 1000 + seed, sigma=sigma)
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
            "seed": seed, "lr": lr}


def train_poisson(m: int = 4, seed: int = 0, epochs: int = 3000, lr: float = 1e-3, alpha: float = 0.05,
                  sigma: float = 0.1, widths=(2, 2, 1), G: int = 5) -> dict:
    """One run of the Poisson experiment (Section 4.1)."""
    cfg = capi.make_cfg(list(widths), G, 3, m, -1.0, 1.0)
    prob = capi.make_problem(capi.HRKAN_POISSON, 1.0, 1.0, 1.0, 0.0, alpha)
    return dict(_train(cfg, prob, poisson_sets(seed), seed, epochs, lr, sigma), m=m)


def train_burgers(m: int = 4, seed: int = 0, epochs: int = 3000, lr: float = 1e-3, alpha: float = 0.05,
                  sigma: float = 0.1, widths=(2, 3, 3, 3, 1), G: int = 7, sets=None) -> dict:
    """One run of the Burgers experiment (Section 4.2, Eq. 7-8); `sets` defaults to burgers_sets(seed)."""
    cfg = capi.make_cfg(list(widths), G, 3, m, 0.0, BURGERS_SIDE)
    prob = capi.make_problem(capi.HRKAN_BURGERS, 1.0, 1.0, 0.25, BURGERS_NU / 16.0, alpha)
    return dict(_train(cfg, prob, burgers_sets(seed) if sets is None else sets, seed, epochs, lr, sigma), m=m)


def _summary(res: list) -> dict:
    mse = np.array([r["test_mse"] for r in res]) * 100.0
    return {"mean_mse_pct": float(mse.mean()), "std_mse_pct": float(mse.std()),
            "median_mse_pct": float(np.median(mse)), "mean_seconds": float(np.mean([r["seconds"] for r in res])),
            "runs": res}


def table(runs: int = 10, m: int = 4, **kw) -> dict:
    """Mean / std of the Poisson test MSE (percent) and mean training seconds over `runs` seeds (Table 1)."""
    return _summary([train_poisson(m=m, seed=s, **kw) for s in range(runs)])


def burgers_table(runs: int = 10, m: int = 4, **kw) -> dict:
    """The same statistics for the Burgers experiment (Table 2)."""
    return _summary([train_burgers(m=m, seed=s, **kw) for s in range(runs)])
