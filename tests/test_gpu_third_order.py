"""Third-derivative jet rows (mask bits 5, 6: u_x0x0x0, u_x1x1x1) and the mixed
derivative (bit 7: u_x0x1) on the layer-wise FP32 path vs the FP64 oracle:
network forward and backward (stored and recomputed layer jets), the
single-layer calls, a KdV-type and an anisotropic second-order residual built
in torch on top of the autograd wrapper, and the masks the other paths refuse.
Shapes: Burgers [2,32,32,1] G=20 (m = 4) and a [2,24,24,1] G=12 net with m = 6
(Section 3: a larger order for higher derivatives), points over several
256-point blocks with a ragged tail."""
import dataclasses

import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, conditioned_tolerances, fp32_floor, layer_slices, relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MASKS = [0x2F, 0x7F, 0x87, 0xFF]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _workload(name):
    if name == "m6":
        return dataclasses.replace(inputs.WORKLOADS["poisson_2_64x3_1"], widths=[2, 24, 24, 1], G=12, m=6)
    return inputs.WORKLOADS["burgers_2_32_32_1"]


def _cfg(w, **kw):
    return capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, **kw)


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("name", ["burgers", "m6"])
def test_third_order_forward_matches_oracle(name, mask):
    w = _workload(name)
    N = 777
    d = inputs.make(w, n_int=N, n_bnd=40, n_ic=20, n_bc=20)
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


@pytest.mark.parametrize("name", ["burgers", "m6"])
def test_third_order_backward_stored_and_recomputed_match_oracle(name):
    w = _workload(name)
    N = 777
    mask = 0xFF
    d = inputs.make(w, n_int=N, n_bnd=40, n_ic=20, n_bc=20)
    J = oracle.n_rows(mask)
    g = np.random.default_rng(95).standard_normal((J, N)).astype(np.float32)
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


def test_third_order_single_layer_calls_match_oracle():
    """hrkan_layer_jets / _dw / _adjoint of a hidden 32 -> 32 layer under mask 0xFF."""
    w = _workload("burgers")
    I = O = 32
    N = 600
    mask = 0xFF
    J = oracle.n_rows(mask)
    rng = np.random.default_rng(96)
    z = rng.normal(0, 0.4, (J, I, N)).astype(np.float32)
    z[0] = rng.uniform(-1.1, 1.1, (I, N))
    gy = rng.normal(0, 1, (J, O, N)).astype(np.float32)
    Wl = rng.normal(0, 0.1, O * I * (w.G + 3)).astype(np.float32)
    h = capi.hrkan_init(_cfg(w))
    try:
        Wd = _dev(Wl)   # the layer's own weights [O][I][n]
        y = torch.zeros((J, O, N), device="cuda")
        capi.hrkan_layer_jets(h, 1, Wd, _dev(z), N, mask, y)
        want = oracle.layer_forward(I, O, w.G, 3, w.m, w.lo, w.hi, Wl, z, mask)
        for r in range(J):
            assert relerr(y.cpu().numpy()[r], want[r]) < 1e-5, r
        dW = torch.zeros(O * I * (w.G + 3), device="cuda")
        capi.hrkan_layer_dw(h, 1, _dev(z), _dev(gy), N, mask, dW)
        want = oracle.layer_dw(I, O, w.G, 3, w.m, w.lo, w.hi, z, gy, mask)
        assert relerr(dW.cpu().numpy(), want) < 1e-5
        gz = torch.zeros((J, I, N), device="cuda")
        capi.hrkan_layer_adjoint(h, 1, Wd, _dev(z), _dev(gy), N, mask, gz)
        want = oracle.layer_adjoint(I, O, w.G, 3, w.m, w.lo, w.hi, Wl, z, gy, mask)
        for r in range(J):
            assert relerr(gz.cpu().numpy()[r], want[r]) < 1e-5, r
    finally:
        capi.hrkan_destroy(h)


def test_kdv_residual_gradient_through_autograd_matches_oracle():
    """A KdV-type residual r = u_t + u u_x + delta u_xxx (coordinates (x, t), mask 0x2F) built in
    torch on the autograd wrapper: the loss and its weight gradient equal the oracle's."""
    from paper_2409_14248_gb300.autograd import HRKAN
    w = _workload("burgers")
    N, delta = 900, 0.0025
    d = inputs.make(w, n_int=N, n_bnd=40, n_ic=20, n_bc=20)
    net = HRKAN(w.widths, w.G, m=w.m)
    try:
        W = torch.tensor(d["W"], device="cuda", requires_grad=True)
        jets = net(W, _dev(d["x_int"]), 0x2F)   # u, u_x, u_t, u_xx, u_xxx
        r = jets[2] + jets[0] * jets[1] + delta * jets[4]
        loss = (r.double() ** 2).mean()
        loss.backward()
        got = W.grad.cpu().numpy()
    finally:
        net.close()
    J = oracle.forward(w.net, d["W"], d["x_int"], 0x2F)
    r = J[2] + J[0] * J[1] + delta * J[4]
    assert loss.item() == pytest.approx(float((r ** 2).mean()), rel=1e-4)
    g = 2.0 * r / N
    dL = np.stack([g * J[1], g * J[0], g, np.zeros(N), delta * g])
    want = oracle.backward(w.net, d["W"], d["x_int"], 0x2F, dL)
    tol = max(TOL_D, 8.0 * fp32_floor(w, d["W"], d["x_int"], 0x2F).max())
    for sl in layer_slices(w.widths, w.G):
        assert relerr(got[sl], want[sl]) < tol


def test_mixed_derivative_residual_gradient_through_autograd_matches_oracle():
    """An anisotropic second-order residual r = u_xx + u_yy + c u_xy + f (mask 0xFF rows) built in
    torch on the autograd wrapper: loss and weight gradient equal the oracle's."""
    from paper_2409_14248_gb300.autograd import HRKAN
    w = _workload("m6")
    N, c = 800, 0.7
    d = inputs.make(w, n_int=N, n_bnd=40)
    x = d["x_int"].astype(np.float64)
    f = np.sin(np.pi * x[0]) * np.cos(np.pi * x[1])
    net = HRKAN(w.widths, w.G, m=w.m)
    try:
        W = torch.tensor(d["W"], device="cuda", requires_grad=True)
        jets = net(W, _dev(d["x_int"]), 0xFF)
        r = jets[3].double() + jets[4].double() + c * jets[7].double() + torch.tensor(f, device="cuda")
        loss = (r ** 2).mean()
        loss.backward()
        got = W.grad.cpu().numpy()
    finally:
        net.close()
    J = oracle.forward(w.net, d["W"], d["x_int"], 0xFF)
    r = J[3] + J[4] + c * J[7] + f
    assert loss.item() == pytest.approx(float((r ** 2).mean()), rel=1e-4)
    g = 2.0 * r / N
    dL = np.zeros((8, N))
    dL[3], dL[4], dL[7] = g, g, c * g
    want = oracle.backward(w.net, d["W"], d["x_int"], 0xFF, dL)
    tol = max(TOL_D, 8.0 * fp32_floor(w, d["W"], d["x_int"], 0xFF).max())
    for sl in layer_slices(w.widths, w.G):
        assert relerr(got[sl], want[sl]) < tol


def test_third_order_masks_are_checked_and_refused_where_unsupported():
    w = inputs.WORKLOADS["burgers_2_10_10_1"]   # a fused narrow shape
    d = inputs.make(w, n_int=300, n_ic=20, n_bc=20)
    h = capi.hrkan_init(_cfg(w))
    try:
        jets = torch.zeros((5, 300), device="cuda")
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_forward_jets(h, _dev(d["W"]), _dev(d["x_int"]), 300, 0x2F, jets)
        assert ei.value.code == capi.HRKAN_EUNSUPPORTED
        # a third-derivative bit without the second-derivative bit of its dimension, the mixed
        # bit without both first-derivative bits, a bit past the mixed one
        for bad in (0x23, 0x47, 0x83, 0x85, 0x100 | 0x1F):
            with pytest.raises(capi.HRKANError) as ei:
                capi.hrkan_forward_jets(h, _dev(d["W"]), _dev(d["x_int"]), 300, bad, jets)
            assert ei.value.code == capi.HRKAN_EINVAL
    finally:
        capi.hrkan_destroy(h)
    # the same shape on the layer-wise path takes the mask
    h = capi.hrkan_init(_cfg(w, flags=capi.HRKAN_FLAG_LAYERWISE))
    try:
        jets = torch.zeros((5, 300), device="cuda")
        capi.hrkan_forward_jets(h, _dev(d["W"]), _dev(d["x_int"]), 300, 0x2F, jets)
        want = oracle.forward(w.net, d["W"], d["x_int"], 0x2F)
        assert relerr(jets.cpu().numpy()[4], want[4]) < TOL_D
    finally:
        capi.hrkan_destroy(h)
