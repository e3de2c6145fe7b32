"""The hand-written backward behind torch.autograd.Function, on the
differentiation workload's network (Burgers [2,32,32,1], G=20): the gradient
of a PINN loss built in torch on top of the jets equals the oracle gradient and
central finite differences (h = 1e-6, FP64, on the oracle) at 64 random
weights, with the layer jets stored (tape) or recomputed."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, layer_slices, relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _torch_loss(net, W, d, w):
    from paper_2409_14248_gb300.autograd import HRKAN  # noqa: F401
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    jets = net(W, dev(d["x_int"]), inputs.MASK_BURGERS)
    u, ux, ut, uxx = jets[0], jets[1], jets[2], jets[3]
    r = ut + w.lam * u * ux - w.nu * uxx
    ub = net(W, dev(d["x_bnd"]), inputs.MASK_U)[0]
    return w.alpha * (r.double() ** 2).mean() + ((ub - dev(d["g_bnd"])).double() ** 2).mean()


def _oracle_loss(w, Wd, d):
    jets = oracle.forward(w.net, Wd, d["x_int"], inputs.MASK_BURGERS)
    ub = oracle.forward(w.net, Wd, d["x_bnd"], inputs.MASK_U)[0]
    return oracle.residual_loss(w.problem(), d["x_int"], inputs.MASK_BURGERS, jets, ub, d["g_bnd"])[0][0]


@pytest.mark.parametrize("budget", [0, 1])
def test_autograd_gradient_matches_oracle_and_finite_differences(budget):
    from paper_2409_14248_gb300.autograd import HRKAN
    w = inputs.WORKLOADS["burgers_2_32_32_1"]
    d = inputs.make(w, n_int=400, n_ic=32, n_bc=32)
    net = HRKAN(w.widths, w.G, hbm_budget_bytes=budget)
    try:
        W = torch.tensor(d["W"], device="cuda", requires_grad=True)
        loss = _torch_loss(net, W, d, w)
        loss.backward()
        g = W.grad.cpu().numpy().astype(np.float64)
    finally:
        net.close()
    Wd = d["W"].astype(np.float64)
    _, want = oracle.train_step(w.net, w.problem(), Wd.copy(), np.zeros_like(Wd), np.zeros_like(Wd), d["x_int"],
                                w.mask_int, d["x_bnd"], d["g_bnd"], w.lr, 1)
    assert loss.item() == pytest.approx(_oracle_loss(w, Wd, d), rel=1e-5)
    for sl in layer_slices(w.widths, w.G):
        assert relerr(g[sl], want[sl]) < TOL_D
    # central differences of the FP64 oracle loss at 64 random weights
    idx = np.random.default_rng(61).choice(Wd.size, 64, replace=False)
    h = 1e-6
    scale = np.abs(want).max()
    for i in idx:
        Wp, Wm = Wd.copy(), Wd.copy()
        Wp[i] += h
        Wm[i] -= h
        fd = (_oracle_loss(w, Wp, d) - _oracle_loss(w, Wm, d)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-4 * scale + 1e-3 * abs(fd), (i, g[i], fd)


def test_autograd_on_a_fused_shape_equals_the_fused_training_gradient():
    """Narrow shape (no tape: the fused kernel recomputes): autograd dW == hrkan_train_step's dW."""
    from paper_2409_14248_gb300.autograd import HRKAN
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    d = inputs.make(w, n_int=3000, n_ic=200, n_bc=200)
    net = HRKAN(w.widths, w.G)
    try:
        W = torch.tensor(d["W"], device="cuda", requires_grad=True)
        _torch_loss(net, W, d, w).backward()
        dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
        dW = torch.zeros_like(W)
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        p = w.problem()
        prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
        capi.hrkan_train_step(net.handle, prob, dev(d["W"]), dev(d["x_int"]), 3000, dev(d["x_bnd"]), dev(d["g_bnd"]),
                              400, 1e-3, 0.9, 0.999, 1e-8, 1, loss, dW)
        assert relerr(W.grad.cpu().numpy(), dW.cpu().numpy()) < 1e-5
    finally:
        net.close()
