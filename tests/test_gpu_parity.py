"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs.

Every call goes through the C ABI (libhrkan.so) via the ctypes binding.
Sizes span several 128-point tiles and a ragged tail; the full-size Burgers
workload (65536 + 8192 points) is checked in the launch configuration the
benchmark times.
"""
import numpy as np
import pytest

import oracle
from gpu_util import (STRESS, TOL_D, TOL_U, cfg_of, layer_slices, oracle_step, problem_of, random_weights,
                      relerr, row_tolerances, assert_close, PT_FACTOR)
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NARROW = ["poisson_2_5_1", "burgers_2_10_10_1", "poisson_batch256"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


@pytest.fixture(scope="module")
def handles():
    hs = {}
    yield hs
    for h in hs.values():
        capi.hrkan_destroy(h)


def _handle(handles, w):
    if w.name not in handles:
        handles[w.name] = capi.hrkan_init(cfg_of(w))
    return handles[w.name]


def _t(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _points(w, n, seed):
    d = inputs.make(w, n_int=n, n_bnd=max(4, n // 8), n_ic=max(2, n // 16), n_bc=max(2, n // 16))
    return d


@pytest.mark.parametrize("wname", NARROW)
@pytest.mark.parametrize("mask", [0x01, 0x0F, 0x1F])
@pytest.mark.parametrize("N", [130, 1000])
def test_forward_jets_match_oracle(handles, wname, mask, N):
    w = inputs.WORKLOADS[wname]
    h = _handle(handles, w)
    d = _points(w, N, 0)
    for W, scale in ((d["W"], 1.0), (random_weights(w, 1), STRESS)):
        J = oracle.n_rows(mask)
        jets = torch.full((J, N), float("nan"), device="cuda")
        capi.hrkan_forward_jets(h, _t(W), _t(d["x_int"]), N, mask, jets)
        torch.cuda.synchronize()
        want = oracle.forward(w.net, W, d["x_int"], mask)
        got = jets.cpu().numpy()
        for r, tol in enumerate(row_tolerances(mask, scale)):
            assert_close(got[r], want[r], tol, PT_FACTOR * tol, what=f"row {r}")


@pytest.mark.parametrize("wname", NARROW)
def test_forward_single_point_equals_batch(handles, wname):
    """A point's jets do not depend on the batch it is evaluated in (bit-exact),
    and one point alone matches the oracle on the scale of the batch."""
    w = inputs.WORKLOADS[wname]
    h = _handle(handles, w)
    N = 1000
    d = _points(w, N, 0)
    W = random_weights(w, 1)
    jets = torch.zeros((5, N), device="cuda")
    capi.hrkan_forward_jets(h, _t(W), _t(d["x_int"]), N, 0x1F, jets)
    batch = jets.cpu().numpy()
    want = oracle.forward(w.net, W, d["x_int"], 0x1F)
    for p in (0, 127, 128, 999):
        one = torch.zeros((5, 1), device="cuda")
        capi.hrkan_forward_jets(h, _t(W), _t(d["x_int"][:, p:p + 1]), 1, 0x1F, one)
        one = one.cpu().numpy()[:, 0]
        assert np.array_equal(one, batch[:, p])
        scale = np.sqrt(np.mean(want ** 2, axis=1))
        tol = np.array(row_tolerances(0x1F, STRESS))
        assert np.all(np.abs(one - want[:, p]) <= tol * scale), (one, want[:, p])


def test_forward_dead_inputs_and_empty(handles):
    """Coordinates outside [s_0, e_{n-1}] touch no basis; N = 0 is a no-op."""
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    h = _handle(handles, w)
    W = random_weights(w, 2)
    x = np.array([[5.0, -7.0, 0.3, 1e30], [0.2, 9.0, -3.0, -1e30]], dtype=np.float32)
    jets = torch.zeros((5, 4), device="cuda")
    capi.hrkan_forward_jets(h, _t(W), _t(x), 4, 0x1F, jets)
    want = oracle.forward(w.net, W, x, 0x1F)
    got = jets.cpu().numpy()
    for r, tol in enumerate(row_tolerances(0x1F, STRESS)):
        assert_close(got[r], want[r], tol, PT_FACTOR * tol, what=f"row {r}")
    assert np.all(got[1:, [1, 3]] == 0.0)      # both coordinates dead: no input derivative at all
    assert np.all(got[[1, 3], 0] == 0.0)       # x dead: no x-derivatives
    assert np.all(got[[2, 4], 2] == 0.0)       # y dead: no y-derivatives
    capi.hrkan_forward_jets(h, _t(W), _t(x), 0, 0x1F, jets)
    torch.cuda.synchronize()


def test_bad_masks_are_rejected(handles):
    w = inputs.WORKLOADS["poisson_2_5_1"]
    h = _handle(handles, w)
    W, x = _t(random_weights(w, 3)), _t(np.zeros((2, 4), np.float32))
    jets = torch.zeros((5, 4), device="cuda")
    for mask, code in ((0x0, capi.HRKAN_EINVAL), (0x09, capi.HRKAN_EINVAL), (0x20, capi.HRKAN_EINVAL),
                       (0x03, capi.HRKAN_EUNSUPPORTED)):
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_forward_jets(h, W, x, 4, mask, jets)
        assert ei.value.code == code


@pytest.mark.parametrize("wname", ["poisson_2_5_1", "burgers_2_10_10_1"])
def test_residual_loss_matches_oracle(handles, wname):
    w = inputs.WORKLOADS[wname]
    h = _handle(handles, w)
    d = _points(w, 3000, 0)
    W = random_weights(w, 4)
    mask = w.mask_int
    jets = oracle.forward(w.net, W, d["x_int"], mask).astype(np.float32)
    ub = oracle.forward(w.net, W, d["x_bnd"], 0x1)[0].astype(np.float32)
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    dj = torch.zeros((oracle.n_rows(mask), Ni), device="cuda")
    du = torch.zeros(Nb, device="cuda")
    capi.pinn_residual_loss(h, problem_of(w), _t(d["x_int"]), Ni, mask, _t(jets), _t(ub), _t(d["g_bnd"]), Nb,
                            loss, dj, du)
    wl, wdj, wdu = oracle.residual_loss(w.problem(), d["x_int"], mask, jets, ub, d["g_bnd"])
    np.testing.assert_allclose(loss.cpu().numpy(), wl, rtol=TOL_U)
    assert relerr(dj.cpu().numpy(), wdj) < TOL_U
    assert relerr(du.cpu().numpy(), wdu) < TOL_U


def test_residual_rejects_mask_without_needed_rows(handles):
    w = inputs.WORKLOADS["poisson_2_5_1"]
    h = _handle(handles, w)
    z = torch.zeros((5, 4), device="cuda")
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.HRKANError) as ei:
        capi.pinn_residual_loss(h, problem_of(w), z[:2].contiguous(), 4, 0x0F, z[:4].contiguous(), None, None, 0,
                                loss)
    assert ei.value.code == capi.HRKAN_EINVAL


@pytest.mark.parametrize("wname", NARROW)
@pytest.mark.parametrize("mask", [0x01, 0x0F, 0x1F])
def test_backward_matches_oracle(handles, wname, mask):
    w = inputs.WORKLOADS[wname]
    h = _handle(handles, w)
    N = 777
    d = _points(w, N, 0)
    J = oracle.n_rows(mask)
    g = np.random.default_rng(6).standard_normal((J, N)).astype(np.float32)
    dW = torch.full((w.n_params(),), float("nan"), device="cuda")
    for W, scale in ((d["W"], 1.0), (random_weights(w, 5), STRESS)):
        capi.hrkan_backward(h, _t(W), _t(d["x_int"]), N, mask, None, _t(g), dW, accumulate=False)
        want = oracle.backward(w.net, W, d["x_int"], mask, g)
        got = dW.cpu().numpy()
        for sl in layer_slices(w.widths, w.G):
            assert_close(got[sl], want[sl], TOL_D * scale, PT_FACTOR * TOL_D * scale, what=f"layer {sl}")
    # accumulate = 1 adds a second copy
    capi.hrkan_backward(h, _t(W), _t(d["x_int"]), N, mask, None, _t(g), dW, accumulate=True)
    assert relerr(dW.cpu().numpy(), 2 * want) < TOL_D * STRESS


def test_adam_matches_oracle(handles):
    w = inputs.WORKLOADS["poisson_2_5_1"]
    h = _handle(handles, w)
    capi.hrkan_reset_moments(h)
    rng = np.random.default_rng(7)
    W0 = rng.standard_normal(w.n_params()).astype(np.float32)
    Wg = _t(W0)
    Wo, m1, m2 = W0.astype(np.float64), np.zeros(w.n_params()), np.zeros(w.n_params())
    for t in range(1, 6):
        g = rng.standard_normal(w.n_params()).astype(np.float32)
        capi.adam_step(h, Wg, _t(g), 1e-2, 0.9, 0.999, 1e-8, t)
        oracle.adam(Wo, g, m1, m2, 1e-2, 0.9, 0.999, 1e-8, t)
    np.testing.assert_allclose(Wg.cpu().numpy(), Wo, rtol=1e-6, atol=1e-7)
    capi.hrkan_reset_moments(h)


@pytest.mark.parametrize("wname", NARROW)
def test_train_step_matches_oracle(handles, wname):
    w = inputs.WORKLOADS[wname]
    h = _handle(handles, w)
    capi.hrkan_reset_moments(h)
    d = _points(w, 2000, 0)
    W = random_weights(w, 8, sigma=0.3)
    Wg = _t(W)
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    dW = torch.zeros(w.n_params(), device="cuda")
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    capi.hrkan_train_step(h, problem_of(w), Wg, _t(d["x_int"]), Ni, _t(d["x_bnd"]), _t(d["g_bnd"]), Nb, w.lr,
                          0.9, 0.999, 1e-8, 1, loss, dW)
    wl, wdW, wW, _, _ = oracle_step(w, W, d["x_int"], d["x_bnd"], d["g_bnd"], w.lr)
    np.testing.assert_allclose(loss.cpu().numpy(), wl, rtol=TOL_U)
    got = dW.cpu().numpy()
    for sl in layer_slices(w.widths, w.G):
        assert_close(got[sl], wdW[sl], TOL_D, PT_FACTOR * TOL_D, what=f"layer {sl}")
    # first Adam step moves each weight by lr * g/(|g|+eps): compare where |g| is not tiny
    big = np.abs(wdW) > 1e-3 * np.abs(wdW).max()
    np.testing.assert_allclose(Wg.cpu().numpy()[big], wW[big], rtol=1e-5, atol=1e-6)
    capi.hrkan_reset_moments(h)


def test_train_step_without_boundary_points(handles):
    w = inputs.WORKLOADS["poisson_2_5_1"]
    h = _handle(handles, w)
    capi.hrkan_reset_moments(h)
    d = _points(w, 300, 0)
    W = random_weights(w, 9)
    Wg = _t(W)
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    capi.hrkan_train_step(h, problem_of(w), Wg, _t(d["x_int"]), 300, None, None, 0, 1e-2, 0.9, 0.999, 1e-8, 1,
                          loss)
    x0 = np.zeros((2, 0))
    wl, _, _, _, _ = oracle_step(w, W, d["x_int"], x0, np.zeros(0), 1e-2)
    np.testing.assert_allclose(loss.cpu().numpy(), wl, rtol=TOL_U)
    capi.hrkan_reset_moments(h)


def test_train_trajectory_poisson_2_5_1_full_size(handles):
    """30 steps of the full 1024 + 256 point Poisson workload track the oracle."""
    w = inputs.WORKLOADS["poisson_2_5_1"]
    h = _handle(handles, w)
    capi.hrkan_reset_moments(h)
    d = inputs.make(w)
    Wg = _t(d["W"])
    Wo = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(Wo), np.zeros_like(Wo)
    xi, xb, gb = _t(d["x_int"]), _t(d["x_bnd"]), _t(d["g_bnd"])
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    for t in range(1, 31):
        capi.hrkan_train_step(h, problem_of(w), Wg, xi, Ni, xb, gb, Nb, w.lr, 0.9, 0.999, 1e-8, t, loss)
        wl, _ = oracle.train_step(w.net, w.problem(), Wo, m1, m2, d["x_int"], w.mask_int, d["x_bnd"], d["g_bnd"],
                                  w.lr, t)
        assert loss.cpu().numpy()[0] == pytest.approx(wl[0], rel=1e-3)
    assert relerr(Wg.cpu().numpy(), Wo) < 1e-3
    capi.hrkan_reset_moments(h)


def test_train_step_full_size_burgers_matches_oracle(handles):
    """Burgers [2,10,10,1], 65536 interior + 4096 + 4096 points: one step, same launch as the benchmark."""
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    h = _handle(handles, w)
    capi.hrkan_reset_moments(h)
    d = inputs.make(w)
    Wg = _t(d["W"])
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    dW = torch.zeros(w.n_params(), device="cuda")
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    capi.hrkan_train_step(h, problem_of(w), Wg, _t(d["x_int"]), Ni, _t(d["x_bnd"]), _t(d["g_bnd"]), Nb, w.lr,
                          0.9, 0.999, 1e-8, 1, loss, dW)
    wl, wdW, _, _, _ = oracle_step(w, d["W"], d["x_int"], d["x_bnd"], d["g_bnd"], w.lr)
    np.testing.assert_allclose(loss.cpu().numpy(), wl, rtol=TOL_U)
    got = dW.cpu().numpy()
    for sl in layer_slices(w.widths, w.G):
        assert relerr(got[sl], wdW[sl]) < TOL_D
    capi.hrkan_reset_moments(h)


def test_separate_calls_equal_fused_step(handles):
    """forward + residual + backward (+ Adam) through the separate calls equals hrkan_train_step."""
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    h = _handle(handles, w)
    d = _points(w, 4000, 0)
    W = random_weights(w, 10, sigma=0.3)
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    xi, xb, gb = _t(d["x_int"]), _t(d["x_bnd"]), _t(d["g_bnd"])
    mask = w.mask_int
    jets = torch.zeros((4, Ni), device="cuda")
    ub = torch.zeros((1, Nb), device="cuda")
    capi.hrkan_forward_jets(h, _t(W), xi, Ni, mask, jets)
    capi.hrkan_forward_jets(h, _t(W), xb, Nb, 0x1, ub)
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    dj = torch.zeros_like(jets)
    du = torch.zeros((1, Nb), device="cuda")
    capi.pinn_residual_loss(h, problem_of(w), xi, Ni, mask, jets, ub, gb, Nb, loss, dj, du)
    dW = torch.zeros(w.n_params(), device="cuda")
    capi.hrkan_backward(h, _t(W), xi, Ni, mask, None, dj, dW)
    capi.hrkan_backward(h, _t(W), xb, Nb, 0x1, None, du, dW, accumulate=True)
    loss2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    dW2 = torch.zeros(w.n_params(), device="cuda")
    capi.hrkan_reset_moments(h)
    capi.hrkan_train_step(h, problem_of(w), _t(W), xi, Ni, xb, gb, Nb, 1e-3, 0.9, 0.999, 1e-8, 1, loss2, dW2)
    np.testing.assert_allclose(loss.cpu().numpy(), loss2.cpu().numpy(), rtol=1e-6)
    assert relerr(dW.cpu().numpy(), dW2.cpu().numpy()) < 1e-5
    capi.hrkan_reset_moments(h)


def test_layerwise_flag_gives_a_bit_reproducible_step():
    """The fused narrow kernel sums its weight gradient with shared-memory atomics (order-dependent
    in the last bits); the same network on a HRKAN_FLAG_LAYERWISE handle sums in a fixed order, so
    two steps from the same weights and moments give the same loss and the same updated weights,
    bit for bit."""
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    h = capi.hrkan_init(capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, flags=capi.HRKAN_FLAG_LAYERWISE))
    try:
        d = _points(w, 20000, 0)
        W0 = random_weights(w, 11)
        out = []
        for _ in range(2):
            capi.hrkan_reset_moments(h)
            W = _t(W0)
            loss = torch.zeros(3, dtype=torch.float64, device="cuda")
            capi.hrkan_train_step(h, problem_of(w), W, _t(d["x_int"]), d["x_int"].shape[1], _t(d["x_bnd"]),
                                  _t(d["g_bnd"]), d["x_bnd"].shape[1], 1e-3, 0.9, 0.999, 1e-8, 1, loss)
            out.append((loss.cpu().numpy(), W.cpu().numpy()))
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1])
        assert not np.array_equal(out[0][1], W0.astype(np.float32))   # the step moved the weights
    finally:
        capi.hrkan_destroy(h)


def test_loss_is_reproducible(handles):
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    h = _handle(handles, w)
    d = _points(w, 5000, 0)
    W = random_weights(w, 11)
    out = []
    for _ in range(2):
        capi.hrkan_reset_moments(h)
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        capi.hrkan_train_step(h, problem_of(w), _t(W), _t(d["x_int"]), d["x_int"].shape[1], _t(d["x_bnd"]),
                              _t(d["g_bnd"]), d["x_bnd"].shape[1], 1e-3, 0.9, 0.999, 1e-8, 1, loss)
        out.append(loss.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    capi.hrkan_reset_moments(h)
