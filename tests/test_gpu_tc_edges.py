"""Edge cases of the tensor-core layer kernels (BF16): single units, the
smallest output width, one point, ragged single tiles, empty inputs, and a
CUDA-graph-captured BF16 training step of the layer-wise path (every launch of
the step, tensor-core ones included, replayed from the graph) against the same
steps run eagerly."""
import numpy as np
import pytest

import oracle
from gpu_util import relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _knot_case(I, O, G, N, seed):
    """Knot inputs and 7-bit weights / gradients: BF16 rounding is a no-op (see test_gpu_tc)."""
    lo, hi = -1.0, 1.0
    h = (hi - lo) / G
    n = G + 3
    rng = np.random.default_rng(seed)
    z = np.zeros((5, I, N), np.float32)
    z[0] = lo + rng.integers(-5, G + 5, (I, N)) * h
    z[1:3] = rng.choice([-0.5, 0.5], (2, I, N))
    z[3:5] = rng.choice([0.0, -2.0, 2.0, -4.0, 4.0], (2, I, N))
    gy = (rng.integers(-127, 128, (5, O, N)) / 8.0).astype(np.float32)
    Wl = (rng.integers(-127, 128, O * I * n) / 128.0).astype(np.float32)
    return z, gy, Wl


@pytest.mark.parametrize("I,O,G,N", [(1, 16, 16, 1), (1, 16, 16, 129), (3, 48, 16, 127), (2, 64, 8, 257),
                                     (9, 32, 32, 300)])
def test_tc_layer_kernels_on_edge_shapes(I, O, G, N):
    """Forward, weight gradient and input adjoint of one BF16 layer on exactly representable
    inputs equal the exact oracle (float32 accumulation only)."""
    z, gy, Wl = _knot_case(I, O, G, N, seed=I * 100 + N)
    cfg = capi.make_cfg([2, I, O, 1], G, prec=capi.HRKAN_BF16, flags=capi.HRKAN_FLAG_LAYERWISE)
    h = capi.hrkan_init(cfg)
    try:
        y = torch.full((5, O, N), float("nan"), device="cuda")
        dW = torch.full((O * I * (G + 3),), float("nan"), device="cuda")
        gz = torch.full((5, I, N), float("nan"), device="cuda")
        capi.hrkan_profile_enable(h, True)
        capi.hrkan_layer_jets(h, 1, _dev(Wl), _dev(z), N, 0x1F, y)
        capi.hrkan_layer_dw(h, 1, _dev(z), _dev(gy), N, 0x1F, dW)
        capi.hrkan_layer_adjoint(h, 1, _dev(Wl), _dev(z), _dev(gy), N, 0x1F, gz)
        capi.hrkan_sync_status(h)
        assert capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_TENSOR)[1] == 3
        y, dW, gz = y.cpu().numpy(), dW.cpu().numpy(), gz.cpu().numpy()
    finally:
        capi.hrkan_destroy(h)
    ey = oracle.layer_forward(I, O, G, 3, 4, -1.0, 1.0, Wl, z, 0x1F)
    edw = oracle.layer_dw(I, O, G, 3, 4, -1.0, 1.0, z, gy, 0x1F)
    egz = oracle.layer_adjoint(I, O, G, 3, 4, -1.0, 1.0, Wl, z, gy, 0x1F)
    for r in range(5):
        assert np.abs(y[r] - ey[r]).max() <= 1e-6 * max(1.0, np.abs(ey[r]).max()), r
        assert np.abs(gz[r] - egz[r]).max() <= 1e-5 * max(1.0, np.abs(egz[r]).max()), r
    assert np.abs(dW - edw).max() <= 1e-5 * max(1.0, np.abs(edw).max())


def test_tc_layer_entry_points_with_no_points():
    """N = 0: the forward and adjoint are no-ops, the weight gradient is zero."""
    cfg = capi.make_cfg([2, 32, 32, 1], 20, prec=capi.HRKAN_BF16, flags=capi.HRKAN_FLAG_LAYERWISE)
    h = capi.hrkan_init(cfg)
    try:
        W = torch.zeros(32 * 32 * 23, device="cuda")
        z = torch.zeros((5, 32, 1), device="cuda")
        y = torch.full((5, 32, 1), 7.0, device="cuda")
        dW = torch.full((32 * 32 * 23,), 7.0, device="cuda")
        capi.hrkan_layer_jets(h, 1, W, z, 0, 0x1F, y)
        capi.hrkan_layer_adjoint(h, 1, W, z, z, 0, 0x1F, y)
        capi.hrkan_layer_dw(h, 1, z, y, 0, 0x1F, dW)
        capi.hrkan_sync_status(h)
        assert torch.all(y == 7.0)
        assert torch.all(dW == 0.0)
    finally:
        capi.hrkan_destroy(h)


def test_graph_captured_bf16_layerwise_steps_equal_eager_steps():
    """Burgers [2,32,32,1] G=20 in BF16 (forward, weight gradient and adjoint of the hidden
    layer on the tensor cores): six steps replayed from one captured step equal six eager
    steps; the kernels are deterministic, so the results agree to rounding noise or better."""
    w = inputs.WORKLOADS["burgers_2_32_32_1"]
    d = inputs.make(w, n_int=2000, n_ic=100, n_bc=100)
    cfg = capi.make_cfg(w.widths, w.G, prec=capi.HRKAN_BF16)
    h = capi.hrkan_init(cfg)
    try:
        p = w.problem()
        prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        Ni, Nb = xi.shape[1], xb.shape[1]
        W_e = _dev(d["W"])
        loss_e = torch.zeros(3, dtype=torch.float64, device="cuda")
        K = 6
        capi.hrkan_profile_enable(h, True)
        for t in range(1, K + 1):
            capi.hrkan_train_step(h, prob, W_e, xi, Ni, xb, gb, Nb, 1e-3, 0.9, 0.999, 1e-8, t, loss_e)
        capi.hrkan_sync_status(h)
        assert capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_TENSOR)[1] > 0
        capi.hrkan_profile_enable(h, False)
        capi.hrkan_reset_moments(h)
        torch.cuda.synchronize()
        W_g = _dev(d["W"])
        loss_g = torch.zeros(3, dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            capi.hrkan_train_step(h, prob, W_g, xi, Ni, xb, gb, Nb, 1e-3, 0.9, 0.999, 1e-8, 0, loss_g, stream=s)
        for _ in range(K):
            g.replay()
        torch.cuda.synchronize()
        capi.hrkan_sync_status(h)
        np.testing.assert_allclose(loss_g.cpu().numpy(), loss_e.cpu().numpy(), rtol=1e-6)
        assert relerr(W_g.cpu().numpy(), W_e.cpu().numpy()) < 1e-6
    finally:
        capi.hrkan_destroy(h)
