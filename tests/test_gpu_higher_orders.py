"""Fourth and fifth derivative jet rows (mask bits 8 and 10: u_x0x0x0x0 and
u_x0x0x0x0x0; Section 3 picks m = 6 for a fifth derivative) on the layer-wise
FP32 path against the FP64 oracle, whose rows are pinned by sympy and finite
differences: network forward, backward with the stored and the recomputed
layer jets, and the single-layer calls.  Masks 0x12F (u, u_x, u_t, u_xx,
u_xxx, u_xxxx: the rows of a Kuramoto-Sivashinsky-type residual) and 0x52F
(also u_xxxxx).  Shapes: Burgers [2,32,32,1] G=20 (m = 4) and a
[2,24,24,1] G=12 net with m = 6, 777 points (several blocks, a ragged tail).
The FP32 bars are those of the other rows: 1e-5 on u and 1e-4 on derivative
rows and weight gradients (normwise, per row / per layer; 4x per point),
or 8x the network's float32 floor where that is higher."""
import dataclasses

import numpy as np
import pytest

import oracle
from gpu_util import PT_FACTOR, TOL_D, assert_close, conditioned_tolerances, fp32_floor, layer_slices
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MASKS = [0x12F, 0x52F]


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
def test_higher_order_forward_matches_oracle(name, mask):
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
        tols = conditioned_tolerances(w, d["W"], d["x_int"], mask)
        print(f"\n{name} mask {mask:#x}: effective FP32 bar per row {tols}")
        for r, tol in enumerate(tols):
            assert_close(got[r], want[r], tol, PT_FACTOR * tol, what=f"row {r}")
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("name", ["burgers", "m6"])
def test_higher_order_backward_stored_and_recomputed_match_oracle(name, mask):
    """The weight gradient of sum(g * jets) through the fourth and fifth rows (reverse mode through
    the sixth basis derivative), per layer, with the forward's tape kept and recomputed."""
    w = _workload(name)
    N = 777
    d = inputs.make(w, n_int=N, n_bnd=40, n_ic=20, n_bc=20)
    J = oracle.n_rows(mask)
    g = np.random.default_rng(97).standard_normal((J, N)).astype(np.float32)
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
                assert_close(got[sl], want[sl], tol, PT_FACTOR * tol, what=f"layer {sl}, tape {tp is not None}")
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("mask", MASKS)
def test_higher_order_single_layer_calls_match_oracle(mask):
    """hrkan_layer_jets / _dw / _adjoint of a hidden 24 -> 24 layer, m = 6, on seeded random
    input jets."""
    w = _workload("m6")
    I = O = 24
    N = 600
    J = oracle.n_rows(mask)
    rng = np.random.default_rng(98)
    z = rng.normal(0, 0.4, (J, I, N)).astype(np.float32)
    z[0] = rng.uniform(-1.1, 1.1, (I, N))
    gy = rng.normal(0, 1, (J, O, N)).astype(np.float32)
    Wl = rng.normal(0, 0.1, O * I * (w.G + 3)).astype(np.float32)
    h = capi.hrkan_init(_cfg(w))
    try:
        Wd = _dev(Wl)
        y = torch.zeros((J, O, N), device="cuda")
        capi.hrkan_layer_jets(h, 1, Wd, _dev(z), N, mask, y)
        want = oracle.layer_forward(I, O, w.G, 3, w.m, w.lo, w.hi, Wl, z, mask)
        for r in range(J):
            assert_close(y.cpu().numpy()[r], want[r], 1e-5, 4e-5, what=f"forward row {r}")
        dW = torch.zeros(O * I * (w.G + 3), device="cuda")
        capi.hrkan_layer_dw(h, 1, _dev(z), _dev(gy), N, mask, dW)
        want = oracle.layer_dw(I, O, w.G, 3, w.m, w.lo, w.hi, z, gy, mask)
        assert_close(dW.cpu().numpy(), want, 1e-5, 4e-5, what="weight gradient")
        gz = torch.zeros((J, I, N), device="cuda")
        capi.hrkan_layer_adjoint(h, 1, Wd, _dev(z), _dev(gy), N, mask, gz)
        want = oracle.layer_adjoint(I, O, w.G, 3, w.m, w.lo, w.hi, Wl, z, gy, mask)
        for r in range(J):
            assert_close(gz.cpu().numpy()[r], want[r], 1e-5, 4e-5, what=f"adjoint row {r}")
    finally:
        capi.hrkan_destroy(h)


def test_higher_order_masks_are_checked_and_refused_where_unsupported():
    """A fourth-derivative bit needs the third of its input and a fifth the fourth (HRKAN_EINVAL);
    the fused narrow shapes and masks without a layer kernel return HRKAN_EUNSUPPORTED."""
    w = _workload("burgers")
    d = inputs.make(w, n_int=300, n_ic=20, n_bc=20)
    h = capi.hrkan_init(_cfg(w))
    try:
        jets = torch.zeros((12, 300), device="cuda")
        for bad in (0x10F, 0x42F, 0x21F):   # u_xxxx without u_xxx; u_xxxxx without u_xxxx; bit 9 without bit 6
            with pytest.raises(capi.HRKANError) as ei:
                capi.hrkan_forward_jets(h, _dev(d["W"]), _dev(d["x_int"]), 300, bad, jets)
            assert ei.value.code == capi.HRKAN_EINVAL, hex(bad)
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_forward_jets(h, _dev(d["W"]), _dev(d["x_int"]), 300, 0x3FF, jets)   # valid, no kernel
        assert ei.value.code == capi.HRKAN_EUNSUPPORTED
    finally:
        capi.hrkan_destroy(h)
    wn = inputs.WORKLOADS["burgers_2_10_10_1"]      # a fused narrow shape
    h = capi.hrkan_init(_cfg(wn))
    try:
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_forward_jets(h, _dev(d["W"][:wn.n_params()]), _dev(d["x_int"]), 300, 0x12F,
                                    torch.zeros((6, 300), device="cuda"))
        assert ei.value.code == capi.HRKAN_EUNSUPPORTED
    finally:
        capi.hrkan_destroy(h)
