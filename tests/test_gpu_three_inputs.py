"""Three-input networks (D = 3) vs the FP64 oracle: the jets u, u_x, u_y, u_z,
u_xx, u_yy, u_zz (run as two passes of the two-direction layer kernels: x and
y, then z) and the backward, on [3,16,16,1] G=8 with points in [-1, 1]^3; a
3-D Poisson residual built in torch on the autograd wrapper; the library's own
residual, training step and data-parallel partial step for the Poisson kind in
three coordinates; and the calls a three-input handle refuses."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, TOL_U, layer_slices, relerr
from gpu_util import assert_close
from paper_2409_14248_gb300 import build, capi, dp, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WIDTHS, G = [3, 16, 16, 1], 8
NET = dict(widths=WIDTHS, G=G, k=3, m=4, lo=-1.0, hi=1.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _data(N, seed):
    P = oracle.param_count(NET)
    W = inputs.init_weights(P, seed, sigma=0.1)
    x = np.random.default_rng(seed + 1).uniform(-1, 1, (3, N)).astype(np.float32)
    return W, x


@pytest.mark.parametrize("mask", [0x7F, 0x0F, 0x49, 0x13])
def test_three_input_forward_matches_oracle(mask):
    N = 700
    W, x = _data(N, 51)
    J = bin(mask).count("1")
    h = capi.hrkan_init(capi.make_cfg(WIDTHS, G))
    try:
        jets = torch.full((J, N), float("nan"), device="cuda")
        capi.hrkan_forward_jets(h, _dev(W), _dev(x), N, mask, jets)
        got = jets.cpu().numpy()
    finally:
        capi.hrkan_destroy(h)
    want = oracle.forward(NET, W, x, mask)
    assert want.shape == got.shape
    for r in range(J):
        assert relerr(got[r], want[r]) < (TOL_U if r == 0 else TOL_D), (r, relerr(got[r], want[r]))


def test_three_input_backward_matches_oracle():
    N = 700
    W, x = _data(N, 52)
    g = np.random.default_rng(53).standard_normal((7, N)).astype(np.float32)
    h = capi.hrkan_init(capi.make_cfg(WIDTHS, G))
    try:
        dW = torch.full((oracle.param_count(NET),), float("nan"), device="cuda")
        capi.hrkan_backward(h, _dev(W), _dev(x), N, 0x7F, None, _dev(g), dW)
        got = dW.cpu().numpy()
        # accumulate adds a second copy
        capi.hrkan_backward(h, _dev(W), _dev(x), N, 0x7F, None, _dev(g), dW, accumulate=True)
        twice = dW.cpu().numpy()
    finally:
        capi.hrkan_destroy(h)
    want = oracle.backward(NET, W, x, 0x7F, g)
    for sl in layer_slices(WIDTHS, G):
        assert relerr(got[sl], want[sl]) < TOL_D
    np.testing.assert_allclose(twice, 2 * got, rtol=1e-6, atol=1e-7 * np.abs(got).max())


def test_three_dimensional_poisson_residual_through_autograd():
    """r = u_xx + u_yy + u_zz + 3 pi^2 sin(pi x) sin(pi y) sin(pi z) (u* = the product of sines):
    the torch loss and its weight gradient equal the oracle's."""
    from paper_2409_14248_gb300.autograd import HRKAN
    N = 900
    W, x = _data(N, 54)
    xd = x.astype(np.float64)
    f = 3 * np.pi ** 2 * np.sin(np.pi * xd[0]) * np.sin(np.pi * xd[1]) * np.sin(np.pi * xd[2])
    net = HRKAN(WIDTHS, G)
    try:
        Wt = torch.tensor(W, device="cuda", requires_grad=True)
        jets = net(Wt, _dev(x), 0x7F)
        r = jets[4].double() + jets[5].double() + jets[6].double() + torch.tensor(f, device="cuda")
        loss = (r ** 2).mean()
        loss.backward()
        got = Wt.grad.cpu().numpy()
    finally:
        net.close()
    J = oracle.forward(NET, W, x, 0x7F)
    r = J[4] + J[5] + J[6] + f
    assert loss.item() == pytest.approx(float((r ** 2).mean()), rel=1e-4)
    dL = np.zeros((7, N))
    dL[4] = dL[5] = dL[6] = 2.0 * r / N
    want = oracle.backward(NET, W, x, 0x7F, dL)
    for sl in layer_slices(WIDTHS, G):
        assert relerr(got[sl], want[sl]) < TOL_D


def test_three_input_handle_refuses_the_two_dimensional_calls():
    N = 64
    W, x = _data(N, 55)
    h = capi.hrkan_init(capi.make_cfg(WIDTHS, G))
    try:
        jets = torch.zeros((7, N), device="cuda")
        for bad in (0x11, 0x21, 0x41, 0x80 | 0x01):   # a second derivative without its first; unknown bit
            with pytest.raises(capi.HRKANError) as ei:
                capi.hrkan_forward_jets(h, _dev(W), _dev(x), N, bad, jets)
            assert ei.value.code == capi.HRKAN_EINVAL
        assert capi.hrkan_tape_floats(h, N, 0x7F) == 0
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        prob = capi.make_problem(capi.HRKAN_POISSON, 1.0, 1.0, 1.0, 0.0, 1.0)
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_train_step(h, prob, _dev(W), _dev(x), N, _dev(x), torch.zeros(N, device="cuda"), N, 1e-3,
                                  0.9, 0.999, 1e-8, 1, loss)
        assert ei.value.code == capi.HRKAN_EUNSUPPORTED
    finally:
        capi.hrkan_destroy(h)


# Eq. 3 in three coordinates: u* = sin(pi x) sin(2 pi y) sin(pi z) (a, b, c = 1, 2, 1; c in lam)
P3 = dict(kind=oracle.POISSON3, a=1.0, b=2.0, lam=1.0, alpha=0.8)


def _prob3():
    return capi.make_problem(capi.HRKAN_POISSON3, P3["a"], P3["b"], P3["lam"], 0.0, P3["alpha"])


def _boundary(N, seed):
    """N points on the faces of [-1, 1]^3 and the exact solution there."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (3, N))
    face = rng.integers(0, 3, N)
    x[face, np.arange(N)] = rng.choice([-1.0, 1.0], N)
    x = x.astype(np.float32)
    xd = x.astype(np.float64)
    g = np.sin(P3["a"] * np.pi * xd[0]) * np.sin(P3["b"] * np.pi * xd[1]) * np.sin(P3["lam"] * np.pi * xd[2])
    return x, g.astype(np.float32)


def test_poisson3_residual_matches_oracle():
    """pinn_residual_loss on a three-input handle (mask 0x7F) against the oracle's residual on the
    same jets: loss terms at 1e-5, dL/d(u_xx, u_yy, u_zz) normwise and per point at 1e-5, the
    lower rows exactly zero, the boundary gradient at 1e-6."""
    N, Nb = 900, 200
    W, x = _data(N, 56)
    xb, gb = _boundary(Nb, 57)
    jets = oracle.forward(NET, W, x, 0x7F).astype(np.float32)
    ub = np.random.default_rng(58).normal(0, 0.1, Nb).astype(np.float32)
    h = capi.hrkan_init(capi.make_cfg(WIDTHS, G))
    try:
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        dL = torch.full((7, N), float("nan"), device="cuda")
        dLb = torch.full((Nb,), float("nan"), device="cuda")
        capi.pinn_residual_loss(h, _prob3(), _dev(x), N, 0x7F, _dev(jets), _dev(ub), _dev(gb), Nb, loss, dL, dLb)
        got_l, got_d, got_b = loss.cpu().numpy(), dL.cpu().numpy(), dLb.cpu().numpy()
    finally:
        capi.hrkan_destroy(h)
    want_l, want_d, want_b = oracle.residual_loss(P3, x.astype(np.float64), 0x7F, jets.astype(np.float64),
                                                  ub.astype(np.float64), gb.astype(np.float64))
    np.testing.assert_allclose(got_l, want_l, rtol=1e-5)
    assert np.all(got_d[:4] == 0.0)
    for r in (4, 5, 6):
        assert_close(got_d[r], want_d[r], 1e-5, what=f"dL row {r}")
    assert_close(got_b, want_b, 1e-6, what="boundary gradient")


def test_poisson3_train_step_matches_oracle():
    """hrkan_train_step on [3,16,16,1]: two steps against the oracle's trajectory on the same points
    (loss terms at 1e-5, the weight gradient of every layer at the FP32 derivative bar 1e-4
    normwise and per point, the weights after each Adam step at 1e-5), both calls with t = 0 (the
    handle's device step counter: 1, then 2)."""
    N, Nb = 1500, 300
    W, x = _data(N, 59)
    xb, gb = _boundary(Nb, 60)
    P = oracle.param_count(NET)
    Wo, m1, m2 = W.astype(np.float64), np.zeros(P), np.zeros(P)
    h = capi.hrkan_init(capi.make_cfg(WIDTHS, G))
    try:
        Wd = _dev(W)
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        dW = torch.full((P,), float("nan"), device="cuda")
        for t in (1, 2):
            capi.hrkan_train_step(h, _prob3(), Wd, _dev(x), N, _dev(xb), _dev(gb), Nb, 1e-3, 0.9, 0.999, 1e-8,
                                  0, loss, dW)
            capi.hrkan_sync_status(h)
            wl, wg = oracle.train_step(NET, P3, Wo, m1, m2, x.astype(np.float64), 0x7F, xb.astype(np.float64),
                                       gb.astype(np.float64), 1e-3, t)
            np.testing.assert_allclose(loss.cpu().numpy(), wl, rtol=1e-5, err_msg=f"step {t}")
            g = dW.cpu().numpy()
            for li, sl in enumerate(layer_slices(WIDTHS, G)):
                assert_close(g[sl], wg[sl], TOL_D, what=f"step {t} layer {li} gradient")
            assert relerr(Wd.cpu().numpy(), Wo) < 1e-5, t
    finally:
        capi.hrkan_destroy(h)


def test_poisson3_partial_steps_sum_to_the_full_step():
    """The data-parallel split on a three-input network: two shards' hrkan_train_step_partial
    (means over the global totals) sum to the full step's loss and gradient."""
    N, Nb = 1200, 240
    W, x = _data(N, 61)
    xb, gb = _boundary(Nb, 62)
    P = oracle.param_count(NET)
    h = capi.hrkan_init(capi.make_cfg(WIDTHS, G))
    try:
        xi, xbd, gbd = _dev(x), _dev(xb), _dev(gb)
        loss_full = torch.zeros(3, dtype=torch.float64, device="cuda")
        dW_full = torch.zeros(P, device="cuda")
        capi.hrkan_train_step(h, _prob3(), _dev(W), xi, N, xbd, gbd, Nb, 1e-3, 0.9, 0.999, 1e-8, 1, loss_full,
                              dW_full)
        loss_sum = torch.zeros(3, dtype=torch.float64, device="cuda")
        dW_sum = torch.zeros(P, device="cuda")
        for r in range(2):
            a, b = dp.shard(N, r, 2)
            c, e = dp.shard(Nb, r, 2)
            loss = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            dW = torch.full((P,), float("nan"), device="cuda")
            capi.hrkan_train_step_partial(h, _prob3(), _dev(W), xi[:, a:b].contiguous(), b - a,
                                          xbd[:, c:e].contiguous(), gbd[c:e].contiguous(), e - c, N, Nb, loss, dW)
            loss_sum += loss
            dW_sum += dW
        np.testing.assert_allclose(loss_sum.cpu().numpy(), loss_full.cpu().numpy(), rtol=1e-6)
        assert relerr(dW_sum.cpu().numpy(), dW_full.cpu().numpy()) < TOL_D / 10
    finally:
        capi.hrkan_destroy(h)


def test_kind_and_input_count_must_match():
    """The Poisson kind in three coordinates needs a three-input network and the other kinds a
    two-input one: both mismatches are refused with HRKAN_EUNSUPPORTED before any launch."""
    N = 64
    h = capi.hrkan_init(capi.make_cfg([2, 8, 1], 5, flags=capi.HRKAN_FLAG_LAYERWISE))
    try:
        W = torch.zeros(capi.hrkan_param_count(capi.make_cfg([2, 8, 1], 5)), device="cuda")
        x = torch.zeros((2, N), device="cuda")
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_train_step(h, _prob3(), W, x, N, x, torch.zeros(N, device="cuda"), N, 1e-3, 0.9, 0.999,
                                  1e-8, 1, loss)
        assert ei.value.code == capi.HRKAN_EUNSUPPORTED
        jets = torch.zeros((5, N), device="cuda")
        with pytest.raises(capi.HRKANError) as ei:
            capi.pinn_residual_loss(h, _prob3(), x, N, 0x1F, jets, None, None, 0, loss)
        assert ei.value.code == capi.HRKAN_EUNSUPPORTED
    finally:
        capi.hrkan_destroy(h)
