"""Checkpoint / resume of the training state (weights, Adam moments, step counts).

CPU: the file format round-trips bit for bit, and every malformed file or
mismatched shape is rejected.  GPU: a run interrupted after k steps, saved,
loaded into a fresh handle and continued equals the uninterrupted run — bit
for bit on the layer-wise path (its reductions run in a fixed order), and with
the device step counter (t = 0) on the fused path, where the bias correction of
the resumed steps must continue from the stored count."""
import os

import numpy as np
import pytest

from paper_2409_14248_gb300 import build, capi, inputs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load_library()


def _state(P, n_inst, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(P * n_inst).astype(np.float32), rng.standard_normal(P * n_inst),
            rng.random(P * n_inst))


def test_checkpoint_round_trip_is_bit_exact(lib, tmp_path):
    P, n_inst = 1690, 3
    W, m, v = _state(P, n_inst, 1)
    path = str(tmp_path / "state.ck")
    capi.hrkan_checkpoint_write(path, P, n_inst, 123, 45, W, m, v)
    assert not os.path.exists(path + ".part")
    assert os.path.getsize(path) == 40 + P * n_inst * (4 + 8 + 8)
    t, td, W2, m2, v2 = capi.hrkan_checkpoint_read(path, P, n_inst)
    assert (t, td) == (123, 45)
    assert W2.tobytes() == W.tobytes() and m2.tobytes() == m.tobytes() and v2.tobytes() == v.tobytes()


def test_checkpoint_rejects_other_shapes_and_damaged_files(lib, tmp_path):
    P, n_inst = 100, 1
    W, m, v = _state(P, n_inst, 2)
    path = str(tmp_path / "s.ck")
    capi.hrkan_checkpoint_write(path, P, n_inst, 1, 0, W, m, v)
    for args, code in (((P + 1, n_inst), capi.HRKAN_EINVAL), ((P, 2), capi.HRKAN_EINVAL)):
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_checkpoint_read(path, *args)
        assert ei.value.code == code
    raw = open(path, "rb").read()
    cases = {"missing": None, "truncated": raw[:-8], "trailing": raw + b"\0", "magic": b"X" + raw[1:],
             "version": raw[:8] + b"\x02" + raw[9:]}
    for name, data in cases.items():
        bad = str(tmp_path / f"{name}.ck")
        if data is not None:
            open(bad, "wb").write(data)
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_checkpoint_read(bad, P, n_inst)
        assert ei.value.code == capi.HRKAN_EIO, name
    # a failed write leaves no file under the target name
    with pytest.raises(capi.HRKANError) as ei:
        capi.hrkan_checkpoint_write(str(tmp_path / "no_such_dir" / "x.ck"), P, n_inst, 1, 0, W, m, v)
    assert ei.value.code == capi.HRKAN_EIO


def _train(h, w, d, W, steps, t0, loss):
    import torch
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    p = w.problem()
    prob = capi.make_problem(p["kind"], p["a"], p["b"], p["lam"], p["nu"], p["alpha"])
    xi, xb, gb = dev(d["x_int"]), dev(d["x_bnd"]), dev(d["g_bnd"])
    Ni, Nb = d["x_int"].shape[1], d["x_bnd"].shape[1]
    for k in range(steps):
        t = 0 if t0 == 0 else t0 + k
        capi.hrkan_train_step(h, prob, W, xi, Ni, xb, gb, Nb, w.lr, 0.9, 0.999, 1e-8, t, loss)


@pytest.mark.gpu
@pytest.mark.parametrize("wname,t_device,exact", [("burgers_2_32_32_1", False, True),
                                                  ("burgers_2_10_10_1", True, False)])
def test_resume_equals_uninterrupted_run(lib, tmp_path, wname, t_device, exact):
    torch = pytest.importorskip("torch")
    w = inputs.WORKLOADS[wname]
    d = inputs.make(w, n_int=2000, n_ic=100, n_bc=100)
    cfg = capi.make_cfg(w.widths, w.G, w.k, w.m, w.lo, w.hi)
    t0 = 0 if t_device else 1
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    # uninterrupted: 6 steps
    h = capi.hrkan_init(cfg)
    try:
        W_ref = torch.tensor(d["W"], device="cuda")
        _train(h, w, d, W_ref, 6, t0, loss)
        loss_ref = loss.cpu().numpy().copy()
    finally:
        capi.hrkan_destroy(h)
    # 3 steps, save, fresh handle, load, 3 more
    path = str(tmp_path / "run.ck")
    h = capi.hrkan_init(cfg)
    try:
        W = torch.tensor(d["W"], device="cuda")
        _train(h, w, d, W, 3, t0, loss)
        capi.hrkan_save(h, W, 3, path)
    finally:
        capi.hrkan_destroy(h)
    h = capi.hrkan_init(cfg)
    try:
        W2 = torch.zeros_like(W)
        assert capi.hrkan_load(h, W2, path) == 3
        assert torch.equal(W2, W)
        _train(h, w, d, W2, 3, 0 if t_device else 4, loss)
        got, got_loss = W2.cpu().numpy(), loss.cpu().numpy()
    finally:
        capi.hrkan_destroy(h)
    want = W_ref.cpu().numpy()
    if exact:
        assert got.tobytes() == want.tobytes()
        assert got_loss.tobytes() == loss_ref.tobytes()
    else:
        # block-local float atomics: equal to rounding; a lost step count would move W by ~lr
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-6 * max(1.0, np.abs(want).max()))
        np.testing.assert_allclose(got_loss, loss_ref, rtol=1e-6)


@pytest.mark.gpu
def test_load_rejects_a_checkpoint_of_another_network(lib, tmp_path):
    torch = pytest.importorskip("torch")
    path = str(tmp_path / "other.ck")
    P = capi.hrkan_param_count(capi.make_cfg([2, 5, 1], 5))
    W, m, v = _state(P, 1, 3)
    capi.hrkan_checkpoint_write(path, P, 1, 7, 0, W, m, v)
    h = capi.hrkan_init(capi.make_cfg([2, 10, 10, 1], 10))
    try:
        Wd = torch.full((capi.hrkan_param_count(capi.make_cfg([2, 10, 10, 1], 10)),), 2.0, device="cuda")
        with pytest.raises(capi.HRKANError) as ei:
            capi.hrkan_load(h, Wd, path)
        assert ei.value.code == capi.HRKAN_EINVAL
        assert torch.all(Wd == 2.0)   # unchanged
    finally:
        capi.hrkan_destroy(h)
