"""HR order m of Eq. 2 other than 4 on the layer-wise FP32 path, vs the FP64 oracle.

The layer-wise kernels are compiled once per order m = 2..6; the fused narrow
kernels and the tensor-core kernels are built for m = 4 only, so a handle with
m != 4 always takes the layer-wise path.  Shapes: Burgers [2,32,32,1] G=20
(mask u, u_x, u_t, u_xx) and Poisson [2,24,24,1] G=12 (all five jet rows),
with points spread over several 128-point tiles and a ragged tail.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, conditioned_tolerances, fp32_floor, layer_slices, oracle_step, relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ORDERS = [2, 3, 5, 6]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _workload(name, m):
    if name == "poisson":
        base = dataclasses.replace(inputs.WORKLOADS["poisson_2_64x3_1"], widths=[2, 24, 24, 1], G=12)
    else:
        base = inputs.WORKLOADS["burgers_2_32_32_1"]
    return dataclasses.replace(base, m=m)


def _cfg(w):
    return capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi)


@pytest.mark.parametrize("m", ORDERS)
@pytest.mark.parametrize("name", ["burgers", "poisson"])
def test_order_m_forward_matches_oracle(name, m):
    w = _workload(name, m)
    N = 333
    d = inputs.make(w, n_int=N, n_bnd=40, n_ic=20, n_bc=20)
    mask = 0x1F if name == "poisson" else w.mask_int
    J = oracle.n_rows(mask)
    h = capi.hrkan_init(_cfg(w))
    try:
        jets = torch.full((J, N), float("nan"), device="cuda")
        capi.hrkan_forward_jets(h, _dev(d["W"]), _dev(d["x_int"]), N, mask, jets)
        want = oracle.forward(w.net, d["W"], d["x_int"], mask)
        got = jets.cpu().numpy()
        for r, tol in enumerate(conditioned_tolerances(w, d["W"], d["x_int"], mask)):
            assert relerr(got[r], want[r]) < tol, (r, relerr(got[r], want[r]), tol)
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("m", ORDERS)
def test_order_m_backward_stored_and_recomputed_match_oracle(m):
    w = _workload("burgers", m)
    N = 333
    d = inputs.make(w, n_int=N, n_bnd=40, n_ic=20, n_bc=20)
    mask = w.mask_int
    J = oracle.n_rows(mask)
    g = np.random.default_rng(90 + m).standard_normal((J, N)).astype(np.float32)
    want = oracle.backward(w.net, d["W"], d["x_int"], mask, g)
    tol = max(TOL_D, 8.0 * fp32_floor(w, d["W"], d["x_int"], mask).max())
    h = capi.hrkan_init(_cfg(w))
    try:
        W, x = _dev(d["W"]), _dev(d["x_int"])
        tape = torch.zeros(capi.hrkan_tape_floats(h, N, mask), device="cuda")
        capi.hrkan_forward_jets(h, W, x, N, mask, torch.zeros((J, N), device="cuda"), tape)
        for tp in (tape, None):
            dW = torch.full((w.n_params(),), float("nan"), device="cuda")
            capi.hrkan_backward(h, W, x, N, mask, tp, _dev(g), dW)
            got = dW.cpu().numpy()
            for sl in layer_slices(w.widths, w.G):
                assert relerr(got[sl], want[sl]) < tol, (sl, relerr(got[sl], want[sl]), tol)
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("m", ORDERS)
def test_order_m_train_step_matches_oracle(m):
    """One hrkan_train_step (jets, residual loss, backward, Adam) vs the oracle's step."""
    w = _workload("poisson", m)
    d = inputs.make(w, n_int=700, n_bnd=130, n_ic=20, n_bc=20)
    lr = 1e-3
    loss_w, dW_w, W_w, _, _ = oracle_step(w, d["W"], d["x_int"], d["x_bnd"], d["g_bnd"], lr)
    p = w.problem()
    prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
    h = capi.hrkan_init(_cfg(w))
    try:
        W = _dev(d["W"])
        dW = torch.zeros_like(W)
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        capi.hrkan_train_step(h, prob, W, _dev(d["x_int"]), 700, _dev(d["x_bnd"]), _dev(d["g_bnd"]), 130, lr, 0.9,
                              0.999, 1e-8, 1, loss, dW)
        assert loss[0].item() == pytest.approx(loss_w[0], rel=1e-4)
        tol = max(TOL_D, 8.0 * fp32_floor(w, d["W"], d["x_int"], 0x1F).max())
        for sl in layer_slices(w.widths, w.G):
            assert relerr(dW.cpu().numpy()[sl], dW_w[sl]) < tol
        # Adam's first step moves each weight by about lr * sign(dW): compare where dW is not negligible
        big = np.abs(dW_w) > 1e-3 * np.abs(dW_w).max()
        np.testing.assert_allclose(W.cpu().numpy()[big], W_w[big], rtol=1e-5, atol=1e-6)
    finally:
        capi.hrkan_destroy(h)

