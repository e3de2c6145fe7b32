"""hrkan_backward_noalloc: the backward for callers that cannot allocate device
memory (they cannot create a handle, whose workspace hrkan_init allocates).

It must give the same weight gradient as hrkan_backward, within the FP32
gradient tolerance of the other parity tests, on two calls in a row (the
second call reuses the static scratch the first one left behind).  The file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, cfg_of, random_weights, relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


@pytest.mark.parametrize("wname,mask", [("burgers_2_10_10_1", inputs.MASK_BURGERS),
                                        ("poisson_batch256", inputs.MASK_POISSON),
                                        ("poisson_2_5_1", inputs.MASK_U)])
def test_noalloc_backward_matches_handle_backward(wname, mask):
    w = inputs.WORKLOADS[wname]
    cfg = cfg_of(w)
    h = capi.hrkan_init(cfg)
    try:
        N = 5000
        d = inputs.make(w, n_int=N, n_bnd=8, n_ic=4, n_bc=4)
        J = bin(mask).count("1")
        dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
        W, x = dev(random_weights(w, 21, sigma=0.3)), dev(d["x_int"])
        rng = np.random.default_rng(22)
        for call in range(2):
            g = dev(rng.standard_normal((J, N)).astype(np.float32))
            want = torch.zeros(w.n_params(), device="cuda")
            capi.hrkan_backward(h, W, x, N, mask, None, g, want)
            got = torch.full((w.n_params(),), float("nan"), device="cuda")
            capi.hrkan_backward_noalloc(cfg, W, x, N, mask, g, got)
            torch.cuda.synchronize()
            assert relerr(got.cpu().numpy(), want.cpu().numpy()) < TOL_D, call
            # accumulate = 1 adds onto what is there
            capi.hrkan_backward_noalloc(cfg, W, x, N, mask, g, got, accumulate=True)
            torch.cuda.synchronize()
            assert relerr(got.cpu().numpy(), 2 * want.cpu().numpy()) < TOL_D, call
    finally:
        capi.hrkan_destroy(h)


def test_noalloc_rejects_bad_arguments():
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    cfg = cfg_of(w)
    z = torch.zeros(16, device="cuda")
    with pytest.raises(capi.HRKANError) as ei:
        capi.hrkan_backward_noalloc(cfg, z, z, 4, 0x09, z, z)      # u_xx without u_x
    assert ei.value.code == capi.HRKAN_EINVAL
    big = capi.make_cfg([2, 64, 64, 64, 1], 32)                      # 293440 weights, no fused kernel
    with pytest.raises(capi.HRKANError) as ei:
        capi.hrkan_backward_noalloc(big, z, z, 4, 0x1, z, z)
    assert ei.value.code == capi.HRKAN_EUNSUPPORTED


def test_noalloc_row_cap_matches_handle_backward_and_oracle():
    """[2,16,16,1] with G = 20 has P = 6992 weights, so only 149 partial rows fit the static
    scratch: with 38400 points (300 blocks of 128) the grid is capped below the occupancy grid
    (one block per SM on 152 SMs at this shape's shared memory), and each block walks several
    point blocks.  Two calls in a row equal hrkan_backward, and the oracle's gradient at the FP32
    bar.  (At G = 30, 104 rows, the float32 formulas themselves land at 1.4e-4 of the oracle,
    on the CPU as on the GPU: steep bases make that network too ill-conditioned for the bar.)"""
    w = inputs.WORKLOADS["poisson_batch256"]
    G, N, mask = 20, 128 * 300, inputs.MASK_POISSON
    cfg = capi.make_cfg(w.widths, G, w.k, w.m, w.lo, w.hi)
    P = capi.hrkan_param_count(cfg)
    assert P == 6992 and (1 << 20) // P == 149
    h = capi.hrkan_init(cfg)
    try:
        rng = np.random.default_rng(31)
        Wn = (0.1 * rng.standard_normal(P)).astype(np.float32)
        x = rng.uniform(-1, 1, (2, N)).astype(np.float32)
        dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
        W, xd = dev(Wn), dev(x)
        for call in range(2):
            g = rng.standard_normal((5, N)).astype(np.float32)
            want = torch.zeros(P, device="cuda")
            capi.hrkan_backward(h, W, xd, N, mask, None, dev(g), want)
            got = torch.full((P,), float("nan"), device="cuda")
            capi.hrkan_backward_noalloc(cfg, W, xd, N, mask, dev(g), got)
            torch.cuda.synchronize()
            assert relerr(got.cpu().numpy(), want.cpu().numpy()) < TOL_D, call
            if call == 0:   # the oracle on a 2048-point prefix (the same entry point, fewer points)
                n = 2048
                sub = torch.full((P,), float("nan"), device="cuda")
                capi.hrkan_backward_noalloc(cfg, W, dev(x[:, :n]), n, mask, dev(g[:, :n]), sub)
                torch.cuda.synchronize()
                net = dict(w.net, G=G)
                ref = oracle.backward(net, Wn.astype(np.float64), x[:, :n], mask, g[:, :n])
                assert relerr(sub.cpu().numpy(), ref) < TOL_D, relerr(sub.cpu().numpy(), ref)
    finally:
        capi.hrkan_destroy(h)


def test_noalloc_refuses_networks_above_the_scratch_size():
    """[2,16,16,1] with G = 4096: 1.3 M weights exceed the 1 Mi floats of static scratch; the
    call is refused on the host, before anything is enqueued."""
    cfg = capi.make_cfg([2, 16, 16, 1], 4096)
    assert capi.hrkan_param_count(cfg) > (1 << 20)
    z = torch.zeros(16, device="cuda")
    with pytest.raises(capi.HRKANError) as ei:
        capi.hrkan_backward_noalloc(cfg, z, z, 4, 0x1F, z, z)
    assert ei.value.code == capi.HRKAN_EINVAL
