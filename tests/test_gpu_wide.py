"""Layer-wise path (wide networks) vs the FP64 oracle, and vs the fused path.

Shapes: [2,64,64,64,1] G=32 (Poisson a=b=2) and [2,32,32,1] G=20 (Burgers).
Covers stored layer jets (tape) and recomputation under an HBM budget.
"""
import numpy as np
import pytest

import oracle
from gpu_util import (STRESS, TOL_D, TOL_U, conditioned_tolerances, fp32_floor, layer_slices, oracle_step,
                      problem_of, random_weights, relerr, assert_close, PT_FACTOR)
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WIDE = ["poisson_2_64x3_1", "burgers_2_32_32_1"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _cfg(w, **kw):
    return capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, **kw)


def _pts(w, n):
    return inputs.make(w, n_int=n, n_bnd=max(4, n // 8), n_ic=max(2, n // 16), n_bc=max(2, n // 16))


@pytest.mark.parametrize("wname", WIDE)
@pytest.mark.parametrize("mask", [0x01, 0x0F, 0x1F])
def test_wide_forward_matches_oracle(wname, mask):
    w = inputs.WORKLOADS[wname]
    h = capi.hrkan_init(_cfg(w))
    try:
        N = 300
        d = _pts(w, N)
        J = oracle.n_rows(mask)
        for W, scale in ((d["W"], 1.0), (random_weights(w, 31, sigma=0.3), STRESS)):
            jets = torch.full((J, N), float("nan"), device="cuda")
            capi.hrkan_forward_jets(h, _dev(W), _dev(d["x_int"]), N, mask, jets)
            want = oracle.forward(w.net, W, d["x_int"], mask)
            got = jets.cpu().numpy()
            tols = conditioned_tolerances(w, W, d["x_int"], mask, scale)
            print(f"\n{wname} mask {mask:#x} scale {scale}: effective FP32 bar per row {tols}")
            for r, tol in enumerate(tols):
                assert_close(got[r], want[r], tol, PT_FACTOR * tol, what=f"row {r}")
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("wname", WIDE)
def test_wide_backward_stored_and_recomputed_match_oracle(wname):
    w = inputs.WORKLOADS[wname]
    h = capi.hrkan_init(_cfg(w))
    try:
        N = 300
        d = _pts(w, N)
        mask = w.mask_int
        J = oracle.n_rows(mask)
        W = _dev(d["W"])
        x = _dev(d["x_int"])
        g = np.random.default_rng(32).standard_normal((J, N)).astype(np.float32)
        want = oracle.backward(w.net, d["W"], d["x_int"], mask, g)
        tape = torch.zeros(capi.hrkan_tape_floats(h, N, mask), device="cuda")
        jets = torch.zeros((J, N), device="cuda")
        capi.hrkan_forward_jets(h, W, x, N, mask, jets, tape)
        # gradients inherit the forward's float32 floor (largest over the jet rows)
        tol = max(TOL_D, 8.0 * fp32_floor(w, d["W"], d["x_int"], mask).max())
        for tp in (tape, None):
            dW = torch.full((w.n_params(),), float("nan"), device="cuda")
            capi.hrkan_backward(h, W, x, N, mask, tp, _dev(g), dW)
            got = dW.cpu().numpy()
            for sl in layer_slices(w.widths, w.G):
                assert relerr(got[sl], want[sl]) < tol, (relerr(got[sl], want[sl]), tol)
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("budget", [0, 1])
def test_wide_train_step_matches_oracle(budget):
    """budget 0 keeps the layer jets; 1 byte forces their recomputation in the backward."""
    w = inputs.WORKLOADS["burgers_2_32_32_1"]
    h = capi.hrkan_init(_cfg(w, hbm_budget_bytes=budget))
    try:
        d = _pts(w, 600)
        Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
        W = _dev(d["W"])
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        dW = torch.zeros(w.n_params(), device="cuda")
        capi.hrkan_train_step(h, problem_of(w), W, _dev(d["x_int"]), Ni, _dev(d["x_bnd"]), _dev(d["g_bnd"]), Nb,
                              w.lr, 0.9, 0.999, 1e-8, 1, loss, dW)
        wl, wdW, wW, _, _ = oracle_step(w, d["W"], d["x_int"], d["x_bnd"], d["g_bnd"], w.lr)
        np.testing.assert_allclose(loss.cpu().numpy(), wl, rtol=TOL_U)
        got = dW.cpu().numpy()
        for sl in layer_slices(w.widths, w.G):
            assert relerr(got[sl], wdW[sl]) < TOL_D
        big = np.abs(wdW) > 1e-3 * np.abs(wdW).max()
        np.testing.assert_allclose(W.cpu().numpy()[big], wW[big], rtol=1e-5, atol=1e-6)
    finally:
        capi.hrkan_destroy(h)


def test_layerwise_path_equals_fused_path_on_a_narrow_net():
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    d = _pts(w, 3000)
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    out = []
    for flags in (0, capi.HRKAN_FLAG_LAYERWISE):
        h = capi.hrkan_init(_cfg(w, flags=flags))
        try:
            W = _dev(d["W"])
            loss = torch.zeros(3, dtype=torch.float64, device="cuda")
            dW = torch.zeros(w.n_params(), device="cuda")
            for t in range(1, 4):
                capi.hrkan_train_step(h, problem_of(w), W, _dev(d["x_int"]), Ni, _dev(d["x_bnd"]), _dev(d["g_bnd"]),
                                      Nb, w.lr, 0.9, 0.999, 1e-8, t, loss, dW)
            out.append((loss.cpu().numpy(), dW.cpu().numpy(), W.cpu().numpy()))
        finally:
            capi.hrkan_destroy(h)
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-5)
    assert relerr(out[0][1], out[1][1]) < 1e-4
    assert relerr(out[0][2], out[1][2]) < 1e-5


def test_wide_full_size_forward_sampled_against_oracle():
    """[2,64,64,64,1] at its full 262144 interior points; 128 sampled points checked one by one."""
    w = inputs.WORKLOADS["poisson_2_64x3_1"]
    h = capi.hrkan_init(_cfg(w))
    try:
        d = inputs.make(w)
        N = d["x_int"].shape[1]
        jets = torch.zeros((5, N), device="cuda")
        capi.hrkan_forward_jets(h, _dev(d["W"]), _dev(d["x_int"]), N, 0x1F, jets)
        idx = np.random.default_rng(33).choice(N, 128, replace=False)
        idx[:2] = [0, N - 1]
        xs = d["x_int"][:, idx]
        want = oracle.forward(w.net, d["W"], xs, 0x1F)
        got = jets.cpu().numpy()[:, idx]
        tols = conditioned_tolerances(w, d["W"], xs, 0x1F)
        print(f"\neffective FP32 bar per row {tols}")
        for r, tol in enumerate(tols):
            assert_close(got[r], want[r], tol, PT_FACTOR * tol, what=f"row {r}")
    finally:
        capi.hrkan_destroy(h)
