"""hrkan_train_step_partial, the per-shard step of the data-parallel split:
on one GPU, the shards' loss contributions and gradients summed equal the
full training step's (fused and layer-wise paths, FP32 and BF16), and Adam
on the summed gradient gives the full step's weights; an empty shard
contributes zeros."""
import numpy as np
import pytest

from gpu_util import TOL_D, problem_of, relerr
from paper_2409_14248_gb300 import build, capi, dp, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


CASES = [("burgers_2_10_10_1", capi.HRKAN_FP32, 0, 1e-5), ("burgers_2_32_32_1", capi.HRKAN_FP32, 0, 1e-5),
         ("burgers_2_32_32_1", capi.HRKAN_BF16, 0, 1e-5)]


@pytest.mark.parametrize("wname,prec,flags,tol", CASES)
@pytest.mark.parametrize("world", [2, 3])
def test_shard_sums_equal_the_full_step(wname, prec, flags, tol, world):
    w = inputs.WORKLOADS[wname]
    d = inputs.make(w, n_int=5000, n_ic=300, n_bc=313)
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    h = capi.hrkan_init(capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, prec=prec, flags=flags))
    try:
        prob = problem_of(w)
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        # the full step (its loss and gradient at W, then Adam)
        W_full = _dev(d["W"])
        loss_full = torch.zeros(3, dtype=torch.float64, device="cuda")
        dW_full = torch.zeros(w.n_params(), device="cuda")
        capi.hrkan_train_step(h, prob, W_full, xi, Ni, xb, gb, Nb, w.lr, 0.9, 0.999, 1e-8, 1, loss_full, dW_full)
        capi.hrkan_reset_moments(h)
        # the shards
        W = _dev(d["W"])
        loss_sum = torch.zeros(3, dtype=torch.float64, device="cuda")
        dW_sum = torch.zeros(w.n_params(), device="cuda")
        for r in range(world):
            a, b = dp.shard(Ni, r, world)
            c, e = dp.shard(Nb, r, world)
            loss = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            dW = torch.full((w.n_params(),), float("nan"), device="cuda")
            capi.hrkan_train_step_partial(h, prob, W, xi[:, a:b].contiguous(), b - a, xb[:, c:e].contiguous(),
                                          gb[c:e].contiguous(), e - c, Ni, Nb, loss, dW)
            loss_sum += loss
            dW_sum += dW
        np.testing.assert_array_equal(W.cpu().numpy(), d["W"])      # read only
        np.testing.assert_allclose(loss_sum.cpu().numpy(), loss_full.cpu().numpy(), rtol=tol)
        assert relerr(dW_sum.cpu().numpy(), dW_full.cpu().numpy()) < TOL_D / 10
        capi.adam_step(h, W, dW_sum, w.lr, 0.9, 0.999, 1e-8, 1)
        g = dW_full.cpu().numpy()
        big = np.abs(g) > 1e-3 * np.abs(g).max()       # the first step moves each weight by lr sign(g)
        np.testing.assert_allclose(W.cpu().numpy()[big], W_full.cpu().numpy()[big], rtol=0, atol=1e-6)
    finally:
        capi.hrkan_destroy(h)


def test_empty_shard_writes_zeros_and_bad_totals_are_refused():
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    h = capi.hrkan_init(capi.make_cfg(w.widths, w.G))
    try:
        W = torch.zeros(w.n_params(), device="cuda")
        loss = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
        dW = torch.full((w.n_params(),), 7.0, device="cuda")
        x = torch.zeros((2, 4), device="cuda")
        capi.hrkan_train_step_partial(h, problem_of(w), W, x, 0, x, x[0], 0, 100, 10, loss, dW)
        assert not loss.cpu().numpy().any() and not dW.cpu().numpy().any()
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_train_step_partial(h, problem_of(w), W, x, 4, x, x[0], 4, 3, 10, loss, dW)   # 4 > 3
        assert ei.value.code == capi.HRKAN_EINVAL
    finally:
        capi.hrkan_destroy(h)
