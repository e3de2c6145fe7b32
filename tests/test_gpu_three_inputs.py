"""Three-input networks (D = 3) vs the FP64 oracle: the jets u, u_x, u_y, u_z,
u_xx, u_yy, u_zz (run as two passes of the two-direction layer kernels: x and
y, then z) and the backward, on [3,16,16,1] G=8 with points in [-1, 1]^3; a
3-D Poisson residual built in torch on the autograd wrapper; and the calls a
three-input handle refuses."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, TOL_U, layer_slices, relerr
from paper_2409_14248_gb300 import build, capi, inputs

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
