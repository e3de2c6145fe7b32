"""Multi-instance training on the layer-wise path: every instance's points in
whole blocks of 256, one launch per layer kernel over all instances, the
hidden layer on the tensor cores in BF16 (forward as the three-term split,
weight gradient and input adjoint with one BF16 rounding).

Checked per instance against the FP64 oracle: the FP32 variant of the same
path at the FP32 bars (the batching itself: instance tables, padding, chunk
rows, per-instance loss and Adam), the BF16 path at the 2e-2 bar (jets
normwise and per point, loss and weight gradient), ragged and empty
instances, and a captured CUDA graph of the step."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, TOL_U, assert_close, maxrel, problem_of, relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W_BATCH = inputs.WORKLOADS["poisson_batch256"]
BAR = 2e-2
# ragged: one point, a part-filled block, several 4096-point chunks, no interior points,
# an exact multiple of the block, no boundary points
COUNTS = [1, 130, 9000, 0, 512, 2500]
BND = [4, 16, 375, 12, 64, 0]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _setup(prec, counts=COUNTS, bnd=BND, items=4096):
    d = inputs.make_batched(W_BATCH, counts=counts, bnd_counts=bnd)
    I = len(counts)
    cfg = capi.make_cfg(W_BATCH.widths, W_BATCH.G, n_instances=I, prec=prec, flags=capi.HRKAN_FLAG_LAYERWISE)
    h = capi.hrkan_init(cfg)
    capi.hrkan_set_batch_items(h, items)
    probs = [problem_of(W_BATCH, a, b) for a, b in d["ab"]]
    return d, I, h, probs


def _inst(d, i):
    P = W_BATCH.n_params()
    return (d["W"][i * P:(i + 1) * P].astype(np.float64), d["x_int"][:, d["off_int"][i]:d["off_int"][i + 1]],
            d["x_bnd"][:, d["off_bnd"][i]:d["off_bnd"][i + 1]], d["g_bnd"][d["off_bnd"][i]:d["off_bnd"][i + 1]])


def _step(h, probs, d, W, t, loss, dW=None):
    capi.hrkan_train_step_batched(h, probs, W, _dev(d["x_int"]), d["off_int"], _dev(d["x_bnd"]), _dev(d["g_bnd"]),
                                  d["off_bnd"], W_BATCH.lr, 0.9, 0.999, 1e-8, t, loss, dW)


@pytest.mark.parametrize("prec", [capi.HRKAN_FP32, capi.HRKAN_BF16])
def test_layerwise_batched_forward_matches_oracle(prec):
    """Output jets of every instance at its own points (scattered back from the padded layout):
    FP32 at 1e-5 / 1e-4, BF16 at 2e-2, normwise and per point."""
    d, I, h, probs = _setup(prec)
    try:
        N = int(d["off_int"][-1])
        jets = torch.full((5, N), float("nan"), device="cuda")
        capi.hrkan_profile_enable(h, True)
        capi.hrkan_forward_jets_batched(h, _dev(d["W"]), _dev(d["x_int"]), d["off_int"], 0x1F, jets)
        capi.hrkan_sync_status(h)
        tc = capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_TENSOR)[1]
        assert (tc > 0) == (prec == capi.HRKAN_BF16)     # the hidden layer ran on the tensor cores
        got = jets.cpu().numpy()
        assert np.all(np.isfinite(got))
        for i in range(I):
            Wi, xi, _, _ = _inst(d, i)
            if xi.shape[1] == 0:
                continue
            want = oracle.forward(W_BATCH.net, Wi, xi, 0x1F)
            g = got[:, d["off_int"][i]:d["off_int"][i + 1]]
            for r in range(5):
                bar = BAR if prec == capi.HRKAN_BF16 else (TOL_U if r == 0 else TOL_D)
                assert_close(g[r], want[r], bar, what=f"instance {i} row {r}")
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("prec", [capi.HRKAN_FP32, capi.HRKAN_BF16])
def test_layerwise_batched_step_matches_oracle(prec):
    """One training step: per-instance loss terms and weight gradient against the oracle's
    step on that instance's points (FP32: 1e-5 on the loss, 1e-4 on dW; BF16: 2e-2), then two
    more steps on the FP32 path against the oracle's trajectory.  Instances without interior or
    without boundary points included."""
    d, I, h, probs = _setup(prec)
    try:
        P = W_BATCH.n_params()
        W = _dev(d["W"])
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        dW = torch.full((I * P,), float("nan"), device="cuda")
        _step(h, probs, d, W, 1, loss, dW)
        capi.hrkan_sync_status(h)
        got_l, got_g = loss.cpu().numpy(), dW.cpu().numpy()
        tol_l = 1e-5 if prec == capi.HRKAN_FP32 else BAR
        tol_g = TOL_D if prec == capi.HRKAN_FP32 else BAR
        states = []
        for i in range(I):
            Wi, xi, xb, gb = _inst(d, i)
            m1, m2 = np.zeros(P), np.zeros(P)
            wl, wg = oracle.train_step(W_BATCH.net, W_BATCH.problem(*d["ab"][i]), Wi, m1, m2, xi, 0x1F, xb, gb,
                                       W_BATCH.lr, 1)
            states.append((Wi, m1, m2))
            np.testing.assert_allclose(got_l[i], wl, rtol=tol_l, atol=1e-12, err_msg=f"instance {i}")
            assert relerr(got_g[i * P:(i + 1) * P], wg) < tol_g, (i, relerr(got_g[i * P:(i + 1) * P], wg))
        if prec != capi.HRKAN_FP32:
            return
        for t in (2, 3):
            _step(h, probs, d, W, t, loss)
            got_l = loss.cpu().numpy()
            for i in range(I):
                Wi, m1, m2 = states[i]
                _, xi, xb, gb = _inst(d, i)
                wl, _ = oracle.train_step(W_BATCH.net, W_BATCH.problem(*d["ab"][i]), Wi, m1, m2, xi, 0x1F, xb, gb,
                                          W_BATCH.lr, t)
                np.testing.assert_allclose(got_l[i], wl, rtol=1e-4, atol=1e-12, err_msg=f"instance {i} step {t}")
        Wg = W.cpu().numpy()
        for i in range(I):
            assert relerr(Wg[i * P:(i + 1) * P], states[i][0]) < 1e-5, i
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("path", [1, 2])
def test_layerwise_batched_bf16_graph_replay_equals_eager(path):
    """The BF16 multi-instance step with the device step counter (t = 0), captured once in a
    CUDA graph and replayed (the capture includes the boundary set's fork onto the side stream
    and its join), gives the same weights and losses as the same number of eager steps."""
    res = []
    for graph in (False, True):
        d, I, h, probs = _setup(capi.HRKAN_BF16)
        try:
            capi.hrkan_set_batch_path(h, path)
            W = _dev(d["W"])
            loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
            xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
            step = lambda: capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"],
                                                         W_BATCH.lr, 0.9, 0.999, 1e-8, 0, loss, None)
            step()                 # warm-up: builds the layout, allocates the workspace
            torch.cuda.synchronize()
            if graph:
                s = torch.cuda.Stream()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.stream(s):
                    with torch.cuda.graph(g, stream=s):
                        capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"],
                                                      W_BATCH.lr, 0.9, 0.999, 1e-8, 0, loss, None,
                                                      stream=s.cuda_stream)
                for _ in range(4):
                    g.replay()
            else:
                for _ in range(4):
                    step()
            torch.cuda.synchronize()
            capi.hrkan_sync_status(h)
            res.append((W.cpu().numpy(), loss.cpu().numpy()))
        finally:
            capi.hrkan_destroy(h)
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])


def test_path_2_runs_the_forward_in_fp32_and_the_backward_on_tensor_cores():
    """Path 2 (hrkan_set_batch_path) on a BF16 handle: every layer's forward on the FP32 SIMT
    kernels, the weight gradient and the input adjoint on the tensor cores.  The forward jets then
    meet the FP32 bars (1e-5 / 1e-4, normwise and per point), the step's loss terms the FP32 one,
    and its gradient the BF16 bar (the backward still rounds its inputs once); no tensor-core
    forward runs, the tensor-core weight gradient does.  Paths outside 0..2 are refused."""
    d, I, h, probs = _setup(capi.HRKAN_BF16)
    try:
        assert capi.hrkan_batch_path(h) == 1
        capi.hrkan_set_batch_path(h, 2)
        assert capi.hrkan_batch_path(h) == 2
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_set_batch_path(h, 3)
        assert ei.value.code == capi.HRKAN_EINVAL
        assert capi.hrkan_batch_path(h) == 2
        capi.hrkan_profile_enable(h, True)
        for c in range(capi.HRKAN_KERNEL_CLASSES):
            capi.hrkan_profile_read(h, c, reset=True)
        N = int(d["off_int"][-1])
        jets = torch.full((5, N), float("nan"), device="cuda")
        capi.hrkan_forward_jets_batched(h, _dev(d["W"]), _dev(d["x_int"]), d["off_int"], 0x1F, jets)
        capi.hrkan_sync_status(h)
        assert capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_TC_FWD)[1] == 0
        got = jets.cpu().numpy()
        for i in range(I):
            Wi, xi, _, _ = _inst(d, i)
            if xi.shape[1] == 0:
                continue
            want = oracle.forward(W_BATCH.net, Wi, xi, 0x1F)
            g = got[:, d["off_int"][i]:d["off_int"][i + 1]]
            for r in range(5):
                assert_close(g[r], want[r], TOL_U if r == 0 else TOL_D, what=f"instance {i} row {r}")
        P = W_BATCH.n_params()
        W = _dev(d["W"])
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        dW = torch.full((I * P,), float("nan"), device="cuda")
        _step(h, probs, d, W, 1, loss, dW)
        capi.hrkan_sync_status(h)
        assert capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_TC_FWD)[1] == 0
        assert capi.hrkan_profile_read(h, capi.HRKAN_KERNEL_TC_DW)[1] > 0
        got_l, got_g = loss.cpu().numpy(), dW.cpu().numpy()
        for i in range(I):
            Wi, xi, xb, gb = _inst(d, i)
            wl, wg = oracle.train_step(W_BATCH.net, W_BATCH.problem(*d["ab"][i]), Wi, np.zeros(P), np.zeros(P), xi,
                                       0x1F, xb, gb, W_BATCH.lr, 1)
            np.testing.assert_allclose(got_l[i], wl, rtol=1e-5, atol=1e-12, err_msg=f"instance {i}")
            assert relerr(got_g[i * P:(i + 1) * P], wg) < BAR, (i, relerr(got_g[i * P:(i + 1) * P], wg))
    finally:
        capi.hrkan_destroy(h)


@pytest.mark.parametrize("path", [1, 2])
def test_boundary_set_on_the_side_stream_equals_the_step_in_order(path):
    """The layer-wise step runs the boundary set's kernels on the handle's side stream, overlapping
    the interior set's; with kernel timing on it runs both sets in order on one stream.  Three steps
    either way give the same weights and losses bit for bit (the two chains write no common
    buffer)."""
    res = []
    for timed in (False, True):
        d, I, h, probs = _setup(capi.HRKAN_BF16)
        try:
            capi.hrkan_set_batch_path(h, path)
            capi.hrkan_profile_enable(h, timed)
            W = _dev(d["W"])
            loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
            for t in (1, 2, 3):
                _step(h, probs, d, W, t, loss)
            torch.cuda.synchronize()
            capi.hrkan_sync_status(h)
            res.append((W.cpu().numpy(), loss.cpu().numpy()))
        finally:
            capi.hrkan_destroy(h)
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])


def test_layerwise_batched_chunk_size_changes_only_summation_order():
    """The weight-gradient chunk size (the knob hrkan_autotune_batch tunes on this path) moves the
    gradient only by the order of float32 sums; the loss not at all."""
    res = []
    for items in (256, 4096, 16384):
        d, I, h, probs = _setup(capi.HRKAN_BF16, items=items)
        try:
            W = _dev(d["W"])
            loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
            dW = torch.zeros(I * W_BATCH.n_params(), device="cuda")
            _step(h, probs, d, W, 1, loss, dW)
            res.append((loss.cpu().numpy(), dW.cpu().numpy()))
        finally:
            capi.hrkan_destroy(h)
    for loss, dW in res[1:]:
        np.testing.assert_array_equal(loss, res[0][0])
        assert relerr(dW, res[0][1]) < 1e-5


def _grid_rel_l2(h_eval, W, ab, n=100):
    """Relative L2 error of every instance's u on an n x n grid of [-1, 1]^2 against
    sin(a pi x) sin(b pi y), evaluated by the FP32 path of h_eval."""
    I = len(ab)
    g = np.linspace(-1.0, 1.0, n)
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()]).astype(np.float32)
    x = np.tile(pts, (1, I))
    off = np.arange(I + 1) * pts.shape[1]
    u = torch.zeros((1, x.shape[1]), device="cuda")
    capi.hrkan_forward_jets_batched(h_eval, W, _dev(x), off, 0x01, u)
    u = u.cpu().numpy()[0].astype(np.float64)
    out = []
    for i, (a, b) in enumerate(ab):
        want = np.sin(a * np.pi * X.ravel()) * np.sin(b * np.pi * Y.ravel())
        got = u[off[i]:off[i + 1]]
        out.append(np.linalg.norm(got - want) / np.linalg.norm(want))
    return np.array(out)


def test_bf16_batched_training_reaches_fp32_l2_error():
    """The metric's equal-L2 condition on the batching workload's own instances: 8 of the 256
    instances of 2-D Poisson (their (a, b) and point counts drawn by the workload's generator,
    seed 4), [2,16,16,1] G=10, the workload's N(0, 0.1^2) initial weights, 1000 Adam steps at
    lr 1e-2 on every path.  The plain FP32 path (the fused multi-instance kernel) and the BF16
    tensor-core path, on path 1 (split forward on the tensor cores) and on path 2 (FP32 forward,
    tensor-core backward), end with mean relative L2 errors (100 x 100 grid, evaluated in FP32)
    whose ratio BF16 / FP32 is at most 1.2."""
    I, steps = 8, 1000
    d = inputs.make_batched(W_BATCH, instances=I)
    probs = [problem_of(W_BATCH, a, b) for a, b in d["ab"]]
    xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
    finals = {}
    h32 = capi.hrkan_init(capi.make_cfg(W_BATCH.widths, W_BATCH.G, n_instances=I))
    try:
        for arm in ("fp32", 1, 2):
            if arm == "fp32":
                h = h32
            else:
                h = capi.hrkan_init(capi.make_cfg(W_BATCH.widths, W_BATCH.G, n_instances=I, prec=capi.HRKAN_BF16,
                                                  flags=capi.HRKAN_FLAG_LAYERWISE))
                capi.hrkan_set_batch_path(h, arm)
            try:
                W = _dev(d["W"])
                loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
                for t in range(1, steps + 1):
                    capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], W_BATCH.lr,
                                                  0.9, 0.999, 1e-8, t, loss)
                capi.hrkan_sync_status(h)
                finals[arm] = (loss.cpu().numpy()[:, 0], _grid_rel_l2(h32, W, d["ab"]))
            finally:
                if h is not h32:
                    capi.hrkan_destroy(h)
    finally:
        capi.hrkan_destroy(h32)
    l32, e32 = finals["fp32"]
    assert np.all(np.isfinite(e32))
    print(f"\nfinal loss FP32 {l32}\nrel-L2 FP32 {e32} mean {e32.mean():.4f}")
    for path in (1, 2):
        l16, e16 = finals[path]
        print(f"final loss BF16 path {path} {l16}\nrel-L2 BF16 path {path} {e16} mean {e16.mean():.4f} "
              f"ratio {e16.mean() / e32.mean():.3f}")
        assert np.all(np.isfinite(e16))
        assert e16.mean() <= 1.2 * e32.mean(), path


def test_layerwise_batched_autotune_picks_a_chunk_and_trains_like_untuned():
    """hrkan_autotune_batch on the layer-wise BF16 path times the candidate weight-gradient chunk
    sizes on path 1 and path 2 (lr = 0), keeps one pair and resets the Adam state: the tuned
    handle's first step then equals an untuned handle's with that chunk size and path set by
    hand."""
    cands = [256, 1024, 4096]
    d, I, h, probs = _setup(capi.HRKAN_BF16, items=1024)
    try:
        W = _dev(d["W"])
        chosen, ms = capi.hrkan_autotune_batch(h, probs, W, _dev(d["x_int"]), d["off_int"], _dev(d["x_bnd"]),
                                               _dev(d["g_bnd"]), d["off_bnd"], candidates=cands, reps=2)
        assert chosen in cands and ms > 0
        path = capi.hrkan_batch_path(h)
        assert path in (1, 2)
        np.testing.assert_array_equal(W.cpu().numpy(), d["W"])      # lr = 0 left W as it was
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        _step(h, probs, d, W, 1, loss)
        tuned = (W.cpu().numpy(), loss.cpu().numpy())
    finally:
        capi.hrkan_destroy(h)
    d, I, h, probs = _setup(capi.HRKAN_BF16, items=chosen)
    try:
        capi.hrkan_set_batch_path(h, path)
        W = _dev(d["W"])
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        _step(h, probs, d, W, 1, loss)
        np.testing.assert_array_equal(tuned[0], W.cpu().numpy())
        np.testing.assert_array_equal(tuned[1], loss.cpu().numpy())
    finally:
        capi.hrkan_destroy(h)


# n = G + 3 bases: 13, 15, 9 (the output layer's gradient summed over 16 slots), 23 (32 slots),
# 43 (walk over the warp's distinct cells), and a single layer (separate launches)
@pytest.mark.parametrize("widths,G,m", [([2, 16, 1], 10, 4), ([2, 24, 24, 1], 12, 3), ([2, 8, 8, 8, 1], 6, 6),
                                        ([2, 16, 16, 1], 20, 4), ([2, 8, 8, 1], 40, 4), ([2, 1], 5, 4)])
def test_layerwise_batched_step_other_shapes_match_oracle(widths, G, m):
    """The FP32 layer-wise multi-instance step on other depths and HR orders (the fused output-layer
    kernel for two or more layers, the separate launches for a single layer): per-instance loss
    terms and weight gradient against the oracle at the FP32 bars (the loss squares a residual of
    second-derivative rows, whose bar is 1e-4: 2e-4)."""
    import dataclasses
    w = dataclasses.replace(W_BATCH, widths=widths, G=G, m=m)
    d = inputs.make_batched(w, counts=[700, 1, 300, 0], bnd_counts=[50, 4, 0, 9])
    I, P = 4, w.n_params()
    h = capi.hrkan_init(capi.make_cfg(widths, G, 3, m, n_instances=I, flags=capi.HRKAN_FLAG_LAYERWISE))
    try:
        probs = [problem_of(w, a, b) for a, b in d["ab"]]
        W = _dev(d["W"])
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        dW = torch.full((I * P,), float("nan"), device="cuda")
        capi.hrkan_train_step_batched(h, probs, W, _dev(d["x_int"]), d["off_int"], _dev(d["x_bnd"]),
                                      _dev(d["g_bnd"]), d["off_bnd"], w.lr, 0.9, 0.999, 1e-8, 1, loss, dW)
        capi.hrkan_sync_status(h)
        got_l, got_g = loss.cpu().numpy(), dW.cpu().numpy()
        for i in range(I):
            Wi, xi, xb, gb = (d["W"][i * P:(i + 1) * P].astype(np.float64),
                              d["x_int"][:, d["off_int"][i]:d["off_int"][i + 1]],
                              d["x_bnd"][:, d["off_bnd"][i]:d["off_bnd"][i + 1]],
                              d["g_bnd"][d["off_bnd"][i]:d["off_bnd"][i + 1]])
            wl, wg = oracle.train_step(w.net, w.problem(*d["ab"][i]), Wi, np.zeros(P), np.zeros(P), xi, 0x1F, xb, gb,
                                       w.lr, 1)
            np.testing.assert_allclose(got_l[i], wl, rtol=2 * TOL_D, atol=1e-12, err_msg=f"instance {i}")
            assert relerr(got_g[i * P:(i + 1) * P], wg) < TOL_D, (i, relerr(got_g[i * P:(i + 1) * P], wg))
    finally:
        capi.hrkan_destroy(h)


def test_fused_shape_runs_either_kernel_family_and_autotune_picks_one():
    """A fused-shape FP32 handle ([2,16,16,1]) runs the multi-instance step on the fused kernel
    (path 0) or on the layer-wise kernels (path 1, hrkan_set_batch_path); both match the oracle per
    instance, and hrkan_autotune_batch times both families and keeps one.  A shape without a fused
    kernel refuses path 0."""
    d = inputs.make_batched(W_BATCH, counts=COUNTS, bnd_counts=BND)
    I, P = len(COUNTS), W_BATCH.n_params()
    h = capi.hrkan_init(capi.make_cfg(W_BATCH.widths, W_BATCH.G, n_instances=I))
    try:
        probs = [problem_of(W_BATCH, a, b) for a, b in d["ab"]]
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        assert capi.hrkan_batch_path(h) == 0
        want = []
        for i in range(I):
            Wi, x_i, x_b, g_b = _inst(d, i)
            want.append(oracle.train_step(W_BATCH.net, W_BATCH.problem(*d["ab"][i]), Wi, np.zeros(P), np.zeros(P),
                                          x_i, 0x1F, x_b, g_b, W_BATCH.lr, 1))
        for path in (0, 1):
            capi.hrkan_set_batch_path(h, path)
            assert capi.hrkan_batch_path(h) == path
            capi.hrkan_reset_moments(h)
            W = _dev(d["W"])
            loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
            dW = torch.full((I * P,), float("nan"), device="cuda")
            capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], W_BATCH.lr, 0.9,
                                          0.999, 1e-8, 1, loss, dW)
            got_l, got_g = loss.cpu().numpy(), dW.cpu().numpy()
            for i in range(I):
                np.testing.assert_allclose(got_l[i], want[i][0], rtol=1e-5, atol=1e-12, err_msg=f"path {path} {i}")
                assert relerr(got_g[i * P:(i + 1) * P], want[i][1]) < TOL_D, (path, i)
        W = _dev(d["W"])
        chosen, ms = capi.hrkan_autotune_batch(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"],
                                               candidates=[256, 2048], reps=2)
        assert chosen in (256, 2048) and ms > 0 and capi.hrkan_batch_path(h) in (0, 1)
        np.testing.assert_array_equal(W.cpu().numpy(), d["W"])
    finally:
        capi.hrkan_destroy(h)
    h = capi.hrkan_init(capi.make_cfg([2, 24, 24, 1], 12, n_instances=2))     # no fused kernel
    try:
        assert capi.hrkan_batch_path(h) == 1
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_set_batch_path(h, 0)
        assert ei.value.code == capi.HRKAN_EUNSUPPORTED
    finally:
        capi.hrkan_destroy(h)


def test_full_batching_workload_step_on_sampled_instances():
    """The full batching workload (256 instances, 4 603 954 interior + 575 384 boundary points)
    in the launch configuration the bench times (BF16 handle, path 2, 2048-point weight-gradient
    chunks, the boundary set on the side stream): one training step checked against the oracle
    on three instances (the fewest points, the most, and one between: loss terms at the FP32 bar
    1e-5, the forward being FP32 on this path; the weight gradient at the BF16 bar, normwise and
    per point), every instance's loss and gradient finite, and the step repeated from the same
    weights and moments bit-identical."""
    d = inputs.make_batched(W_BATCH)
    I, P = W_BATCH.instances, W_BATCH.n_params()
    h = capi.hrkan_init(capi.make_cfg(W_BATCH.widths, W_BATCH.G, n_instances=I, prec=capi.HRKAN_BF16,
                                      flags=capi.HRKAN_FLAG_LAYERWISE))
    try:
        capi.hrkan_set_batch_items(h, 2048)
        capi.hrkan_set_batch_path(h, 2)
        probs = [problem_of(W_BATCH, a, b) for a, b in d["ab"]]
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        res = []
        for _ in range(2):
            capi.hrkan_reset_moments(h)
            W = _dev(d["W"])
            loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
            dW = torch.full((I * P,), float("nan"), device="cuda")
            capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], W_BATCH.lr, 0.9,
                                          0.999, 1e-8, 1, loss, dW)
            capi.hrkan_sync_status(h)
            res.append((loss.cpu().numpy(), dW.cpu().numpy(), W.cpu().numpy()))
    finally:
        capi.hrkan_destroy(h)
    got_l, got_g, _ = res[0]
    assert np.all(np.isfinite(got_l)) and np.all(np.isfinite(got_g))
    for first, again in zip(res[0], res[1]):
        np.testing.assert_array_equal(first, again)
    counts = np.diff(d["off_int"])
    for i in sorted({int(np.argmin(counts)), int(np.argmax(counts)), 137}):
        Wi, x_i, x_b, g_b = _inst(d, i)
        wl, wg = oracle.train_step(W_BATCH.net, W_BATCH.problem(*d["ab"][i]), Wi, np.zeros(P), np.zeros(P), x_i,
                                   0x1F, x_b, g_b, W_BATCH.lr, 1)
        np.testing.assert_allclose(got_l[i], wl, rtol=1e-5, atol=1e-12, err_msg=f"instance {i}")
        assert_close(got_g[i * P:(i + 1) * P], wg, BAR, what=f"instance {i} gradient")
