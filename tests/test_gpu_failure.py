"""Failure detection without a GPU fault.  A non-finite loss (a NaN boundary
target) is recorded on the device and reported by hrkan_sync_status as
HRKAN_ENONFINITE; a short bounded-wait limit makes the tensor-core kernels'
waits give up on purpose, which they report as HRKAN_ETIMEOUT after draining
their own copies and MMAs and freeing their tensor memory; in both cases the
next normal call on the same handle gives the normal result."""
import numpy as np
import pytest

from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("flags", [0, capi.HRKAN_FLAG_LAYERWISE])
def test_nan_target_is_reported_as_a_nonfinite_loss(flags):
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    d = inputs.make(w, n_int=2048, n_ic=128, n_bc=128)
    g_bad = d["g_bnd"].copy()
    g_bad[3] = np.nan   # (a NaN coordinate only deactivates that point's bases: its jets stay finite)
    p = w.problem()
    prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
    h = capi.hrkan_init(capi.make_cfg(w.widths, w.G, flags=flags))
    try:
        loss = torch.zeros(3, dtype=torch.float64, device="cuda")
        tail = (w.lr, 0.9, 0.999, 1e-8, 1, loss)
        nb = d["x_bnd"].shape[1]
        capi.hrkan_train_step(h, prob, _dev(d["W"]), _dev(d["x_int"]), 2048, _dev(d["x_bnd"]), _dev(g_bad), nb, *tail)
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_sync_status(h)
        assert ei.value.code == capi.HRKAN_ENONFINITE
        assert not np.isfinite(loss.cpu().numpy()[0])
        capi.hrkan_sync_status(h)   # the record was cleared
        capi.hrkan_reset_moments(h)
        capi.hrkan_train_step(h, prob, _dev(d["W"]), _dev(d["x_int"]), 2048, _dev(d["x_bnd"]), _dev(d["g_bnd"]), nb,
                              *tail)
        capi.hrkan_sync_status(h)
        assert np.all(np.isfinite(loss.cpu().numpy()))
    finally:
        capi.hrkan_destroy(h)


def test_forced_wait_timeout_is_reported_and_the_handle_stays_usable():
    """BF16 [2,64,64,1] G=32: the hidden layer's forward, weight gradient and adjoint run on the
    tensor cores; with a 1-cycle wait limit their first unready wait gives up."""
    widths, G, N = [2, 64, 64, 1], 32, 4096
    cfg = capi.make_cfg(widths, G, prec=capi.HRKAN_BF16)
    P = capi.hrkan_param_count(cfg)
    W = _dev(inputs.init_weights(P, 71))
    x = _dev(np.random.default_rng(72).uniform(-1, 1, (2, N)))
    g = _dev(np.random.default_rng(73).standard_normal((5, N)))
    h = capi.hrkan_init(cfg)
    try:
        ref = torch.zeros((5, N), device="cuda")
        capi.hrkan_forward_jets(h, W, x, N, 0x1F, ref)
        dW_ref = torch.zeros(P, device="cuda")
        capi.hrkan_backward(h, W, x, N, 0x1F, None, g, dW_ref)
        capi.hrkan_sync_status(h)
        capi.hrkan_set_wait_cycles(h, 1)
        for call in ("forward", "backward"):
            out = torch.zeros((5, N), device="cuda")
            dW = torch.zeros(P, device="cuda")
            if call == "forward":
                capi.hrkan_forward_jets(h, W, x, N, 0x1F, out)
            else:
                capi.hrkan_backward(h, W, x, N, 0x1F, None, g, dW)
            with pytest.raises(capi.HRKANError) as ei:
                capi.hrkan_sync_status(h)
            assert ei.value.code == capi.HRKAN_ETIMEOUT, call
        capi.hrkan_set_wait_cycles(h, 0)
        out = torch.zeros((5, N), device="cuda")
        capi.hrkan_forward_jets(h, W, x, N, 0x1F, out)
        dW = torch.zeros(P, device="cuda")
        capi.hrkan_backward(h, W, x, N, 0x1F, None, g, dW)
        capi.hrkan_sync_status(h)
        assert torch.equal(out, ref)
        np.testing.assert_allclose(dW.cpu().numpy(), dW_ref.cpu().numpy(), rtol=0,
                                   atol=1e-6 * float(dW_ref.abs().max()))
    finally:
        capi.hrkan_destroy(h)
