"""Tensor-core (tcgen05) forward of the hidden layers in BF16 / TF32 vs the
FP64 oracle, error reported per jet order (value, first, second derivatives).

Bar for BF16 jets: 2e-2 relative (normwise per jet row).  TF32 keeps 10
mantissa bits instead of BF16's 7, so its bar is 8x tighter (2.5e-3).
"""
import numpy as np
import pytest

import oracle
from gpu_util import relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {capi.HRKAN_BF16: 2e-2, capi.HRKAN_TF32: 2.5e-3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _forward(w, prec, W, x, mask, flags=0):
    h = capi.hrkan_init(capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi, prec=prec, flags=flags))
    try:
        N = x.shape[1]
        jets = torch.full((oracle.n_rows(mask), N), float("nan"), device="cuda")
        capi.hrkan_forward_jets(h, _dev(W), _dev(x), N, mask, jets)
        capi.hrkan_sync_status(h)
        return jets.cpu().numpy()
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("prec", [capi.HRKAN_BF16, capi.HRKAN_TF32])
@pytest.mark.parametrize("mask", [0x01, 0x1F])
def test_tc_forward_per_jet_order_error(prec, mask):
    w = inputs.WORKLOADS["poisson_2_64x3_1"]
    d = inputs.make(w, n_int=300, n_bnd=40)
    got = _forward(w, prec, d["W"], d["x_int"], mask)
    want = oracle.forward(w.net, d["W"], d["x_int"], mask)
    errs = [relerr(got[r], want[r]) for r in range(want.shape[0])]
    print("per-jet-order relative error", prec, mask, errs)
    assert np.all(np.isfinite(got))
    assert max(errs) < TOL[prec], errs


@pytest.mark.parametrize("prec", [capi.HRKAN_BF16, capi.HRKAN_TF32])
def test_tc_forward_burgers_32_and_ragged_tile(prec):
    """[2,32,32,1], G=20 (n = 23, several units per K step), 389 points (ragged last tile)."""
    w = inputs.WORKLOADS["burgers_2_32_32_1"]
    d = inputs.make(w, n_int=389, n_ic=8, n_bc=8)
    got = _forward(w, prec, d["W"], d["x_int"], 0x0F)
    want = oracle.forward(w.net, d["W"], d["x_int"], 0x0F)
    errs = [relerr(got[r], want[r]) for r in range(4)]
    assert max(errs) < TOL[prec], errs
