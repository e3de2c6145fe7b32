"""Seeded synthetic workloads for HRKAN physics-informed training.

This module draws the random numbers of a run (collocation points, initial
weights) and states the boundary data of each problem.  It holds none of the
method's arithmetic (no basis, no network, no residual), so both the CUDA path
and the FP64 oracle consume the very same arrays.

Every array is float32 (what the GPU path takes); the oracle converts to
float64.  Coordinates are structure-of-arrays, shape [D, N], D = 2: (x, y)
for Poisson, (x, t) for Burgers.

Workloads (sizes, seeds, learning rates and steps of the five benchmark
configurations):

* ``poisson_2_5_1``    2-D Poisson on [-1,1]^2, u* = sin(pi x) sin(pi y),
  widths [2,5,1], G=5, 1024 interior + 256 boundary points, uniform, seed 0.
* ``burgers_2_10_10_1`` viscous Burgers, nu = 0.01/pi, x in [-1,1], t in [0,1],
  u(x,0) = -sin(pi x), u(+-1,t) = 0, widths [2,10,10,1], G=10,
  65536 interior + 4096 initial + 4096 boundary points, Latin hypercube, seed 1.
* ``poisson_2_64x3_1`` Poisson with a = b = 2, widths [2,64,64,64,1], G=32,
  262144 interior + 16384 boundary points, uniform, seed 0.
* ``burgers_2_32_32_1`` Burgers as above, widths [2,32,32,1], G=20,
  131072 interior + 4096 + 4096 points, Latin hypercube, seed 1.
* ``poisson_batch256`` 256 independent Poisson instances, (a, b) uniform in
  {1..4}^2, widths [2,16,16,1], G=10, interior counts uniform in
  [2048, 32768], boundary count = interior // 8 split over the 4 edges, seed 4.

All use k = 3, order m = 4, grid [-1, 1] for every layer and initial weights
N(0, 0.1^2).  The paper's own experiments (Section 4) use 960 + 120 Poisson
points and 10000 + 300 Burgers points with the same kind of sampling
(uniform-random interior, boundary points spread over the edges); these
workloads keep that structure at GPU scale.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

POISSON = 0
BURGERS = 1

# jet-row masks, D = 2: bit 0 = u, bit 1+d = du/dx_d, bit 3+d = d2u/dx_d^2
MASK_U = 0x1
MASK_POISSON = 0x1F   # u, u_x, u_y, u_xx, u_yy
MASK_BURGERS = 0x0F   # u, u_x, u_t, u_xx


@dataclass
class Workload:
    name: str
    widths: list
    G: int
    k: int = 3
    m: int = 4
    lo: float = -1.0
    hi: float = 1.0
    pde: int = POISSON
    a: float = 1.0
    b: float = 1.0
    lam: float = 1.0
    nu: float = 0.0
    alpha: float = 1.0
    n_int: int = 0
    n_bnd: int = 0          # Poisson: total boundary points (split over 4 edges)
    n_ic: int = 0           # Burgers: initial-condition points
    n_bc: int = 0           # Burgers: boundary points (half at x=-1, half at x=+1)
    sampling: str = "uniform"
    seed: int = 0
    steps: int = 100
    lr: float = 1e-2
    sigma: float = 0.1
    instances: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def net(self):
        return dict(widths=list(self.widths), G=self.G, k=self.k, m=self.m, lo=self.lo, hi=self.hi)

    @property
    def mask_int(self):
        return MASK_POISSON if self.pde == POISSON else MASK_BURGERS

    def problem(self, a=None, b=None):
        return dict(kind=self.pde, a=self.a if a is None else a, b=self.b if b is None else b,
                    lam=self.lam, nu=self.nu, alpha=self.alpha)

    def n_params(self):
        n = self.G + self.k
        return sum(self.widths[l] * self.widths[l + 1] * n for l in range(len(self.widths) - 1))


WORKLOADS = {
    "poisson_2_5_1": Workload("poisson_2_5_1", [2, 5, 1], G=5, pde=POISSON, n_int=1024, n_bnd=256,
                              sampling="uniform", seed=0, steps=100, lr=1e-2),
    "burgers_2_10_10_1": Workload("burgers_2_10_10_1", [2, 10, 10, 1], G=10, pde=BURGERS, nu=0.01 / math.pi,
                                  n_int=65536, n_ic=4096, n_bc=4096, sampling="lhs", seed=1, steps=2000,
                                  lr=1e-3),
    "poisson_2_64x3_1": Workload("poisson_2_64x3_1", [2, 64, 64, 64, 1], G=32, pde=POISSON, a=2.0, b=2.0,
                                 n_int=262144, n_bnd=16384, sampling="uniform", seed=0, steps=100, lr=1e-2),
    "burgers_2_32_32_1": Workload("burgers_2_32_32_1", [2, 32, 32, 1], G=20, pde=BURGERS, nu=0.01 / math.pi,
                                  n_int=131072, n_ic=4096, n_bc=4096, sampling="lhs", seed=1, steps=5000,
                                  lr=1e-3),
    "poisson_batch256": Workload("poisson_batch256", [2, 16, 16, 1], G=10, pde=POISSON, sampling="uniform",
                                 seed=4, steps=1000, lr=1e-2, instances=256,
                                 extra=dict(count_lo=2048, count_hi=32768)),
}


def _lhs(rng, n, lo, hi):
    """One Latin-hypercube coordinate: a random permutation of n strata, jittered."""
    u = (rng.permutation(n) + rng.uniform(0.0, 1.0, n)) / n
    return lo + (hi - lo) * u


def _poisson_points(rng, n_int, n_bnd, lo=-1.0, hi=1.0):
    x_int = rng.uniform(lo, hi, size=(2, n_int))
    per = [n_bnd // 4 + (1 if e < n_bnd % 4 else 0) for e in range(4)]
    cols = []
    for e, c in enumerate(per):
        t = rng.uniform(lo, hi, size=c)
        fixed = np.full(c, lo if e % 2 == 0 else hi)
        cols.append(np.stack([fixed, t]) if e < 2 else np.stack([t, fixed]))
    x_bnd = np.concatenate(cols, axis=1) if cols else np.zeros((2, 0))
    g_bnd = np.zeros(x_bnd.shape[1])   # u* = sin(a pi x) sin(b pi y) vanishes on the edges
    return x_int, x_bnd, g_bnd


def _burgers_points(rng, n_int, n_ic, n_bc, sampling):
    if sampling == "lhs":
        x_int = np.stack([_lhs(rng, n_int, -1.0, 1.0), _lhs(rng, n_int, 0.0, 1.0)])
        x_ic = _lhs(rng, n_ic, -1.0, 1.0)
        t_bc = _lhs(rng, n_bc, 0.0, 1.0)
    else:
        x_int = np.stack([rng.uniform(-1.0, 1.0, n_int), rng.uniform(0.0, 1.0, n_int)])
        x_ic = rng.uniform(-1.0, 1.0, n_ic)
        t_bc = rng.uniform(0.0, 1.0, n_bc)
    ic = np.stack([x_ic, np.zeros(n_ic)])
    side = np.where(np.arange(n_bc) < n_bc // 2, -1.0, 1.0)
    bc = np.stack([side, t_bc])
    x_bnd = np.concatenate([ic, bc], axis=1)
    g_bnd = np.concatenate([-np.sin(np.pi * x_ic), np.zeros(n_bc)])   # u(x,0) = -sin(pi x), u(+-1,t) = 0
    return x_int, x_bnd, g_bnd


def init_weights(n_params, seed, sigma=0.1, instances=1):
    """Initial weights ~ N(0, sigma^2), float32, shape [instances * n_params]."""
    rng = np.random.default_rng([seed, 0x5EED])
    return (sigma * rng.standard_normal(instances * n_params)).astype(np.float32)


def make(w: Workload | str, n_int=None, n_bnd=None, n_ic=None, n_bc=None):
    """Points, boundary data and initial weights of a single-instance workload.

    Optional counts override the workload's (a smaller case with the same
    distribution and seed).  Returns a dict of float32 arrays:
    x_int [2, N_int], x_bnd [2, N_bnd], g_bnd [N_bnd], W [P].
    """
    if isinstance(w, str):
        w = WORKLOADS[w]
    rng = np.random.default_rng(w.seed)
    if w.pde == POISSON:
        x_int, x_bnd, g_bnd = _poisson_points(rng, w.n_int if n_int is None else n_int,
                                              w.n_bnd if n_bnd is None else n_bnd, w.lo, w.hi)
    else:
        x_int, x_bnd, g_bnd = _burgers_points(rng, w.n_int if n_int is None else n_int,
                                              w.n_ic if n_ic is None else n_ic,
                                              w.n_bc if n_bc is None else n_bc, w.sampling)
    W = init_weights(w.n_params(), w.seed, w.sigma)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(x_int=f32(x_int), x_bnd=f32(x_bnd), g_bnd=f32(g_bnd), W=W)


def make_batched(w: Workload | str, instances=None, count_lo=None, count_hi=None, counts=None, bnd_counts=None):
    """Ragged multi-instance Poisson workload.

    counts / bnd_counts: explicit per-instance interior / boundary counts
    (else interior counts are drawn uniformly and boundary = interior // 8).

    Returns dict with per-instance (a, b) [inst, 2] float64, interior and
    boundary offsets (int32, [inst+1]), concatenated x_int [2, sum N_int],
    x_bnd [2, sum N_bnd], g_bnd, and W [inst * P].
    """
    if isinstance(w, str):
        w = WORKLOADS[w]
    inst = w.instances if instances is None else instances
    lo_c = w.extra.get("count_lo", 2048) if count_lo is None else count_lo
    hi_c = w.extra.get("count_hi", 32768) if count_hi is None else count_hi
    rng = np.random.default_rng(w.seed)
    if counts is not None:
        inst = len(counts)
    ab = rng.integers(1, 5, size=(inst, 2)).astype(np.float64)
    drawn = rng.integers(lo_c, hi_c + 1, size=inst)
    counts = drawn if counts is None else np.asarray(counts)
    bnd_counts = [int(c) // 8 for c in counts] if bnd_counts is None else list(bnd_counts)
    xi, xb, gb = [], [], []
    for c, cb in zip(counts, bnd_counts):
        a_, b_, g_ = _poisson_points(rng, int(c), int(cb), w.lo, w.hi)
        xi.append(a_); xb.append(b_); gb.append(g_)
    off_i = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    off_b = np.concatenate([[0], np.cumsum([x.shape[1] for x in xb])]).astype(np.int32)
    W = init_weights(w.n_params(), w.seed, w.sigma, instances=inst)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(ab=ab, off_int=off_i, off_bnd=off_b, x_int=f32(np.concatenate(xi, axis=1)),
                x_bnd=f32(np.concatenate(xb, axis=1)), g_bnd=f32(np.concatenate(gb)), W=W)


def layer_jets(I, N, mask, seed, lo=-1.0, hi=1.0):
    """Random input jets [J][I][N] for testing one layer: values uniform on
    [lo, hi] (the grid range), first derivatives N(0, 1), second N(0, 3^2)."""
    rng = np.random.default_rng([seed, 0x1A7E])
    J = bin(mask & 0x1F).count("1")
    z = np.empty((J, I, N))
    z[0] = rng.uniform(lo, hi, (I, N))
    r = 1
    for bit in range(1, 5):
        if mask & (1 << bit):
            z[r] = rng.standard_normal((I, N)) * (1.0 if bit <= 2 else 3.0)
            r += 1
    return np.ascontiguousarray(z, dtype=np.float32)
