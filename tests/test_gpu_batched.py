"""Multi-instance training step (one persistent launch over ragged instances)
and CUDA-graph capture, against the FP64 oracle run per instance."""
import numpy as np
import pytest

import oracle
from gpu_util import PT_FACTOR, TOL_D, TOL_U, assert_close, cfg_of, problem_of, relerr
from paper_2409_14248_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W_BATCH = inputs.WORKLOADS["poisson_batch256"]
# ragged: one point, a ragged tile, several items, no boundary points, no interior points
COUNTS = [1, 130, 3000, 777, 0, 2500]
BND = [4, 16, 375, 0, 12, 312]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def _dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _setup(items_points=1024):
    d = inputs.make_batched(W_BATCH, counts=COUNTS, bnd_counts=BND)
    I = len(COUNTS)
    cfg = capi.make_cfg(W_BATCH.widths, W_BATCH.G, n_instances=I)
    h = capi.hrkan_init(cfg)
    capi.hrkan_set_batch_items(h, items_points)
    probs = [problem_of(W_BATCH, a, b) for a, b in d["ab"]]
    return d, I, h, probs


def _oracle_steps(d, I, steps, lr):
    P = W_BATCH.n_params()
    out = []
    for i in range(I):
        Wi = d["W"][i * P:(i + 1) * P].astype(np.float64)
        m1, m2 = np.zeros(P), np.zeros(P)
        xi = d["x_int"][:, d["off_int"][i]:d["off_int"][i + 1]]
        xb = d["x_bnd"][:, d["off_bnd"][i]:d["off_bnd"][i + 1]]
        gb = d["g_bnd"][d["off_bnd"][i]:d["off_bnd"][i + 1]]
        losses = []
        for t in range(1, steps + 1):
            loss, _ = oracle.train_step(W_BATCH.net, W_BATCH.problem(*d["ab"][i]), Wi, m1, m2, xi, 0x1F, xb, gb, lr, t)
            losses.append(loss)
        out.append((np.array(losses), Wi))
    return out


def test_batched_step_matches_oracle_per_instance():
    d, I, h, probs = _setup()
    try:
        W = _dev(d["W"])
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        dW = torch.zeros(I * W_BATCH.n_params(), device="cuda")
        steps = 3
        hist = []
        for t in range(1, steps + 1):
            capi.hrkan_train_step_batched(h, probs, W, _dev(d["x_int"]), d["off_int"], _dev(d["x_bnd"]),
                                          _dev(d["g_bnd"]), d["off_bnd"], W_BATCH.lr, 0.9, 0.999, 1e-8, t, loss,
                                          dW if t == 1 else None)
            hist.append(loss.cpu().numpy().copy())
        g1 = dW.cpu().numpy()
        P0 = W_BATCH.n_params()
        for i in range(I):
            Wi = d["W"][i * P0:(i + 1) * P0].astype(np.float64)
            xi = d["x_int"][:, d["off_int"][i]:d["off_int"][i + 1]]
            xb = d["x_bnd"][:, d["off_bnd"][i]:d["off_bnd"][i + 1]]
            gb = d["g_bnd"][d["off_bnd"][i]:d["off_bnd"][i + 1]]
            _, gw = oracle.train_step(W_BATCH.net, W_BATCH.problem(*d["ab"][i]), Wi, np.zeros(P0), np.zeros(P0), xi,
                                      0x1F, xb, gb, W_BATCH.lr, 1)
            assert relerr(g1[i * P0:(i + 1) * P0], gw) < TOL_D, i
        want = _oracle_steps(d, I, steps, W_BATCH.lr)
        P = W_BATCH.n_params()
        Wg = W.cpu().numpy()
        for i in range(I):
            np.testing.assert_allclose(hist[0][i], want[i][0][0], rtol=TOL_U, atol=1e-12)
            for t in range(steps):
                np.testing.assert_allclose(hist[t][i], want[i][0][t], rtol=1e-4, atol=1e-12)
            assert relerr(Wg[i * P:(i + 1) * P], want[i][1]) < 1e-5, i
    finally:
        capi.hrkan_destroy(h)


def test_batched_result_does_not_depend_on_item_size():
    res = []
    for ip in (128, 1024, 5000):
        d, I, h, probs = _setup(ip)
        try:
            W = _dev(d["W"])
            loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
            dW = torch.zeros(I * W_BATCH.n_params(), device="cuda")
            capi.hrkan_train_step_batched(h, probs, W, _dev(d["x_int"]), d["off_int"], _dev(d["x_bnd"]),
                                          _dev(d["g_bnd"]), d["off_bnd"], 1e-2, 0.9, 0.999, 1e-8, 1, loss, dW)
            res.append((loss.cpu().numpy(), dW.cpu().numpy()))
        finally:
            capi.hrkan_destroy(h)
    # the gradients differ only by the order of float32 sums
    for loss, dW in res[1:]:
        np.testing.assert_allclose(loss, res[0][0], rtol=1e-6, atol=1e-14)
        assert relerr(dW, res[0][1]) < 1e-5


def test_batched_forward_matches_oracle():
    d, I, h, probs = _setup()
    try:
        N = int(d["off_int"][-1])
        jets = torch.zeros((5, N), device="cuda")
        capi.hrkan_forward_jets_batched(h, _dev(d["W"]), _dev(d["x_int"]), d["off_int"], 0x1F, jets)
        got = jets.cpu().numpy()
        P = W_BATCH.n_params()
        for i in range(I):
            a, b = d["off_int"][i], d["off_int"][i + 1]
            if a == b:
                continue
            want = oracle.forward(W_BATCH.net, d["W"][i * P:(i + 1) * P], d["x_int"][:, a:b], 0x1F)
            for r, tol in enumerate([TOL_U] + [TOL_D] * 4):
                assert_close(got[r, a:b], want[r], tol, PT_FACTOR * tol, what=f"instance {i} row {r}")
    finally:
        capi.hrkan_destroy(h)


def test_graph_captured_batched_steps_equal_eager_steps():
    """One captured step with the device step counter (t = 0), replayed, equals eager steps t = 1..K."""
    K = 5
    d, I, h, probs = _setup()
    try:
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        W_e = _dev(d["W"])
        loss_e = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        for t in range(1, K + 1):
            capi.hrkan_train_step_batched(h, probs, W_e, xi, d["off_int"], xb, gb, d["off_bnd"], 1e-2, 0.9, 0.999,
                                          1e-8, t, loss_e)
        capi.hrkan_reset_moments(h)
        W_g = _dev(d["W"])
        loss_g = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            # warm-up call (builds the work list), then undo it
            W_tmp = W_g.clone()
            capi.hrkan_train_step_batched(h, probs, W_tmp, xi, d["off_int"], xb, gb, d["off_bnd"], 1e-2, 0.9, 0.999,
                                          1e-8, 0, loss_g, stream=s)
        torch.cuda.synchronize()
        capi.hrkan_reset_moments(h)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            capi.hrkan_train_step_batched(h, probs, W_g, xi, d["off_int"], xb, gb, d["off_bnd"], 1e-2, 0.9, 0.999,
                                          1e-8, 0, loss_g, stream=s)
        for _ in range(K):
            g.replay()
        torch.cuda.synchronize()
        np.testing.assert_allclose(loss_g.cpu().numpy(), loss_e.cpu().numpy(), rtol=1e-5, atol=1e-14)
        assert relerr(W_g.cpu().numpy(), W_e.cpu().numpy()) < 1e-5
    finally:
        capi.hrkan_destroy(h)


def test_graph_captured_single_network_steps_equal_eager_steps():
    w = inputs.WORKLOADS["burgers_2_10_10_1"]
    d = inputs.make(w, n_int=4096, n_ic=256, n_bc=256)
    h = capi.hrkan_init(cfg_of(w))
    try:
        prob = problem_of(w)
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        Ni, Nb = xi.shape[1], xb.shape[1]
        W_e = _dev(d["W"])
        loss_e = torch.zeros(3, dtype=torch.float64, device="cuda")
        K = 6
        for t in range(1, K + 1):
            capi.hrkan_train_step(h, prob, W_e, xi, Ni, xb, gb, Nb, 1e-3, 0.9, 0.999, 1e-8, t, loss_e)
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
        np.testing.assert_allclose(loss_g.cpu().numpy(), loss_e.cpu().numpy(), rtol=1e-5)
        assert relerr(W_g.cpu().numpy(), W_e.cpu().numpy()) < 1e-5
    finally:
        capi.hrkan_destroy(h)


def test_batched_rejects_inconsistent_problems():
    d, I, h, probs = _setup()
    try:
        bad = list(probs)
        bad[2] = capi.make_problem(capi.HRKAN_POISSON, 1, 1, alpha=0.5)
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_train_step_batched(h, bad, _dev(d["W"]), _dev(d["x_int"]), d["off_int"], _dev(d["x_bnd"]),
                                          _dev(d["g_bnd"]), d["off_bnd"], 1e-2, 0.9, 0.999, 1e-8, 1, loss)
        assert ei.value.code == capi.HRKAN_EINVAL
        off = np.array(d["off_int"]); off[2] = off[3] + 1
        with pytest.raises(capi.HRKANError):
            capi.hrkan_train_step_batched(h, probs, _dev(d["W"]), _dev(d["x_int"]), off, _dev(d["x_bnd"]),
                                          _dev(d["g_bnd"]), d["off_bnd"], 1e-2, 0.9, 0.999, 1e-8, 1, loss)
    finally:
        capi.hrkan_destroy(h)



def test_batched_calls_on_a_single_layerwise_network_equal_the_single_calls():
    """A layer-wise handle with one instance runs the batched calls on the layer-wise
    multi-instance path (points gathered into 256-point blocks): its forward jets equal
    hrkan_forward_jets bit for bit (the same kernels per point), and its training step's loss
    and gradient equal hrkan_train_step's up to the order of float32 sums."""
    w = W_BATCH
    h = capi.hrkan_init(capi.make_cfg(w.widths, w.G, flags=capi.HRKAN_FLAG_LAYERWISE))
    try:
        d = inputs.make(w, n_int=700, n_bnd=90)
        Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
        W = _dev(d["W"])
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        jets = torch.zeros((5, Ni), device="cuda")
        capi.hrkan_forward_jets(h, W, xi, Ni, 0x1F, jets)
        jets_b = torch.zeros((5, Ni), device="cuda")
        capi.hrkan_forward_jets_batched(h, W, xi, np.array([0, Ni]), 0x1F, jets_b)
        np.testing.assert_array_equal(jets.cpu().numpy(), jets_b.cpu().numpy())
        prob = problem_of(w)
        res = []
        for batched in (False, True):
            capi.hrkan_reset_moments(h)
            Wt = _dev(d["W"])
            loss = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
            dW = torch.zeros(w.n_params(), device="cuda")
            if batched:
                capi.hrkan_train_step_batched(h, [prob], Wt, xi, np.array([0, Ni]), xb, gb, np.array([0, Nb]), w.lr,
                                              0.9, 0.999, 1e-8, 1, loss, dW)
            else:
                capi.hrkan_train_step(h, prob, Wt, xi, Ni, xb, gb, Nb, w.lr, 0.9, 0.999, 1e-8, 1, loss[0], dW)
            res.append((loss.cpu().numpy()[0], dW.cpu().numpy()))
        np.testing.assert_allclose(res[1][0], res[0][0], rtol=1e-6)
        assert relerr(res[1][1], res[0][1]) < 1e-5
    finally:
        capi.hrkan_destroy(h)


def test_autotune_picks_a_candidate_and_leaves_weights_and_moments_fresh():
    """hrkan_autotune_batch times each item size (on this fused shape: with both kernel
    families) with lr = 0 (W keeps its values), keeps the fastest and resets the Adam state:
    the next step equals a fresh handle's step set to the same family and size."""
    d, I, h, probs = _setup()
    h2 = None
    try:
        W = _dev(d["W"])
        xi, xb, gb = _dev(d["x_int"]), _dev(d["x_bnd"]), _dev(d["g_bnd"])
        cands = [256, 512, 1024]
        chosen, ms = capi.hrkan_autotune_batch(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], cands, reps=2)
        assert chosen in cands and ms > 0.0
        assert np.array_equal(W.cpu().numpy(), d["W"])
        loss = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        capi.hrkan_train_step_batched(h, probs, W, xi, d["off_int"], xb, gb, d["off_bnd"], W_BATCH.lr, 0.9, 0.999,
                                      1e-8, 1, loss)
        _, _, h2, _ = _setup(chosen)
        capi.hrkan_set_batch_path(h2, capi.hrkan_batch_path(h))
        W2 = _dev(d["W"])
        loss2 = torch.zeros((I, 3), dtype=torch.float64, device="cuda")
        capi.hrkan_train_step_batched(h2, probs, W2, xi, d["off_int"], xb, gb, d["off_bnd"], W_BATCH.lr, 0.9, 0.999,
                                      1e-8, 1, loss2)
        # the loss is reduced in a fixed order; the gradient's shared-memory float atomics are not
        # ordered, so the updated weights agree to rounding (stale moments would differ by O(lr))
        assert np.array_equal(loss.cpu().numpy(), loss2.cpu().numpy())
        assert relerr(W.cpu().numpy(), W2.cpu().numpy()) < 1e-6
    finally:
        capi.hrkan_destroy(h)
        if h2 is not None:
            capi.hrkan_destroy(h2)
