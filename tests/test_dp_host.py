"""Data-parallel split of the training step (points sharded across ranks,
weights replicated; one all-reduce of the gradient and the loss terms, then
the same Adam step on every replica), run as world-size-2 gloo process groups
on the CPU.

The library is replaced by a fake whose partial step and Adam update are the
FP64 oracle's (test infrastructure; the product module calls libhrkan.so,
whose partial step is checked on the GPU against the full step).  The checks:
the shards cover every point once; two ranks' summed gradients and loss equal
one rank's over all points; after three steps the replicas hold identical
weights, equal to the oracle's single-process training."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2409_14248_gb300 import capi, dp, inputs

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

W_NET = inputs.WORKLOADS["burgers_2_10_10_1"]


class _Handle:
    def __init__(self, P):
        self.P = P


class FakeLibrary:
    """Partial step: the oracle's residual gradient at the shard's points with the means taken
    over the totals, then the oracle's backward; Adam: the oracle's."""

    def __init__(self, w):
        self.w = w
        P = w.n_params()
        self.m1, self.m2 = np.zeros(P), np.zeros(P)

    def hrkan_train_step_partial(self, h, prob, W, x_int, N_int, x_bnd, g_bnd, N_bnd, Ni_tot, Nb_tot, loss, dW):
        w, Wd = self.w, W.numpy().astype(np.float64)
        p = w.problem()
        xi, xb, gb = x_int.numpy()[:, :N_int], x_bnd.numpy()[:, :N_bnd], g_bnd.numpy()[:N_bnd]
        jets = oracle.forward(w.net, Wd, xi, w.mask_int)
        ub = oracle.forward(w.net, Wd, xb, 0x01)[0]
        lo, dj, du = oracle.residual_loss(p, xi, w.mask_int, jets, ub, gb)
        # the oracle's means are over this shard; rescale them (and the gradient) to the totals
        fi, fb = N_int / Ni_tot, N_bnd / Nb_tot
        g = oracle.backward(w.net, Wd, xi, w.mask_int, dj * fi) + oracle.backward(w.net, Wd, xb, 0x01, du[None] * fb)
        terms = np.array([p["alpha"] * lo[1] * fi + lo[2] * fb, lo[1] * fi, lo[2] * fb])
        dW.copy_(torch.from_numpy(g.astype(np.float32)))
        loss.copy_(torch.from_numpy(terms))

    def adam_step(self, h, W, dW, lr, b1, b2, eps, t):
        Wd = W.numpy().astype(np.float64)
        oracle.adam(Wd, dW.numpy().astype(np.float64), self.m1, self.m2, lr, b1, b2, eps, t)
        W.copy_(torch.from_numpy(Wd.astype(np.float32)))


def _data():
    d = inputs.make(W_NET, n_int=301, n_ic=17, n_bc=20)
    return d


def _worker(rank, world, init_file, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"file://{init_file}", rank=rank, world_size=world)
    try:
        lib = FakeLibrary(W_NET)
        capi.hrkan_train_step_partial = lib.hrkan_train_step_partial
        capi.adam_step = lib.adam_step
        d = _data()
        p = W_NET.problem()
        prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
        step = dp.DataParallelStep(_Handle(W_NET.n_params()), prob, torch.from_numpy(d["x_int"]),
                                   torch.from_numpy(d["x_bnd"]), torch.from_numpy(d["g_bnd"]))
        W = torch.from_numpy(d["W"].copy())
        losses, grads = [], []
        for t in (1, 2, 3):
            losses.append(step(W, W_NET.lr, t).numpy().copy())
            grads.append(step.dW.numpy().copy())
        np.savez(f"{out}_{rank}.npz", W=W.numpy(), losses=np.array(losses), grads=np.array(grads),
                 n_int=step.x_int.shape[1], n_bnd=step.x_bnd.shape[1])
    finally:
        dist.destroy_process_group()


def _run(world):
    with tempfile.TemporaryDirectory() as tmp:
        init = os.path.join(tmp, "init")
        out = os.path.join(tmp, "res")
        mp.start_processes(_worker, args=(world, init, out), nprocs=world, join=True, start_method="spawn")
        return [dict(np.load(f"{out}_{r}.npz")) for r in range(world)]


def test_shards_cover_every_point_once():
    for n in (0, 1, 7, 301, 4096):
        for world in (1, 2, 3, 8):
            parts = [dp.shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def test_two_ranks_equal_one_rank_and_the_oracle():
    one = _run(1)[0]
    two = _run(2)
    assert two[0]["n_int"] + two[1]["n_int"] == 301 and two[0]["n_bnd"] + two[1]["n_bnd"] == 37
    # replicas identical after every all-reduce and Adam step
    np.testing.assert_array_equal(two[0]["W"], two[1]["W"])
    np.testing.assert_array_equal(two[0]["losses"], two[1]["losses"])
    # the sharded sums equal the single-rank step (float32 gradient: summation order only, which
    # moves the float32 weights, and so the later losses, in their last bits)
    np.testing.assert_allclose(two[0]["losses"][0], one["losses"][0], rtol=1e-12)
    np.testing.assert_allclose(two[0]["losses"], one["losses"], rtol=1e-7)
    for t in range(3):
        g1, g2 = one["grads"][t], two[0]["grads"][t]
        assert np.linalg.norm(g2 - g1) / np.linalg.norm(g1) < 1e-6, t
    np.testing.assert_allclose(two[0]["W"], one["W"], rtol=0, atol=1e-6)
    # and the oracle's own training over all points
    d = _data()
    Wd = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wd), np.zeros_like(Wd)
    for t in (1, 2, 3):
        lo, _ = oracle.train_step(W_NET.net, W_NET.problem(), Wd, m1, m2, d["x_int"], W_NET.mask_int, d["x_bnd"],
                                  d["g_bnd"], W_NET.lr, t)
        np.testing.assert_allclose(two[0]["losses"][t - 1], lo, rtol=1e-6)
    np.testing.assert_allclose(two[0]["W"], Wd, rtol=0, atol=1e-5)
