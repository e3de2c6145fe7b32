"""Host logic of the experiment drivers (Sections 4.1 and 4.2) and of the
training driver's test error, on the CPU.

The library is replaced by a fake that records every call and carries out the
training step and the forward with the FP64 oracle (test infrastructure; the
product module calls libhrkan.so).  The checks: each driver hands the library
the network, domain and problem constants its section states (for Burgers the
rescaled coefficients 1/4 and nu/16 of Eq. 7), the training set sizes,
Adam steps t = 1, 2, ... in order, the seeded initial weights, and it reports
the final loss and the test MSE of the weights it trained."""
import numpy as np
import pytest

import oracle
from paper_2409_14248_gb300 import capi, inputs, replica, trainer, truth

torch = pytest.importorskip("torch")

MASK = {capi.HRKAN_POISSON: 0x1F, capi.HRKAN_BURGERS: 0x0F}


def _net(cfg):
    return dict(widths=list(cfg.widths[:cfg.n_widths]), G=cfg.G, k=cfg.k, m=cfg.m, lo=cfg.grid_lo, hi=cfg.grid_hi)


class FakeLibrary:
    def __init__(self):
        self.steps, self.forwards, self.destroyed, self.W0 = [], [], 0, None

    def hrkan_param_count(self, cfg):
        return oracle.param_count(_net(cfg))

    def hrkan_init(self, cfg):
        self.net = _net(cfg)
        P = oracle.param_count(self.net)
        self.m1, self.m2 = np.zeros(P), np.zeros(P)
        return "handle"

    def hrkan_destroy(self, h):
        assert h == "handle"
        self.destroyed += 1

    def hrkan_train_step(self, h, prob, W, x_int, N_int, x_bnd, g_bnd, N_bnd, lr, b1, b2, eps, t, loss):
        if self.W0 is None:
            self.W0 = W.numpy().copy()
        p = dict(kind=prob.kind, a=prob.a, b=prob.b, lam=prob.lam, nu=prob.nu, alpha=prob.alpha)
        self.prob = p
        self.steps.append(dict(t=t, N_int=N_int, N_bnd=N_bnd, lr=lr, b1=b1, b2=b2, eps=eps))
        Wd = W.numpy().astype(np.float64)
        got, _ = oracle.train_step(self.net, p, Wd, self.m1, self.m2, x_int.numpy()[:, :N_int], MASK[prob.kind],
                                   x_bnd.numpy()[:, :N_bnd], g_bnd.numpy()[:N_bnd], lr, t, b1, b2, eps)
        W.copy_(torch.from_numpy(Wd.astype(np.float32)))
        loss.copy_(torch.from_numpy(np.asarray(got, np.float64)))

    def hrkan_forward_jets(self, h, W, x, N, mask, jets):
        self.forwards.append(dict(N=N, mask=mask))
        jets.copy_(torch.from_numpy(oracle.forward(self.net, W.numpy(), x.numpy()[:, :N], mask).astype(np.float32)))


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLibrary()
    for name in ("hrkan_param_count", "hrkan_init", "hrkan_destroy", "hrkan_train_step", "hrkan_forward_jets"):
        monkeypatch.setattr(capi, name, getattr(lib, name))
    # the driver allocates on cuda; here the tensors stay in host memory
    real_tensor, real_zeros = torch.tensor, torch.zeros
    monkeypatch.setattr(torch, "tensor", lambda *a, device=None, **k: real_tensor(*a, **k))
    monkeypatch.setattr(torch, "zeros", lambda *a, device=None, **k: real_zeros(*a, **k))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    return lib


def _check_result(lib, res, sets, epochs, lr, seed):
    assert [s["t"] for s in lib.steps] == list(range(1, epochs + 1))
    assert all(s["lr"] == lr and (s["b1"], s["b2"], s["eps"]) == (0.9, 0.999, 1e-8) for s in lib.steps)
    x_int, x_bnd, g_bnd, x_test, u_test = sets
    assert all(s["N_int"] == x_int.shape[1] and s["N_bnd"] == x_bnd.shape[1] for s in lib.steps)
    np.testing.assert_array_equal(lib.W0, inputs.init_weights(oracle.param_count(lib.net), 1000 + seed, sigma=0.1))
    assert lib.forwards == [dict(N=x_test.shape[1], mask=0x01)] and lib.destroyed == 1
    assert res["seed"] == seed and res["lr"] == lr and res["seconds"] >= 0.0
    return x_test, u_test


def test_burgers_driver_passes_section_4_2_set_up(fake):
    sets = replica.burgers_sets(3, n_test=12)
    res = replica.train_burgers(m=4, seed=3, epochs=3, lr=1e-2, sets=sets)
    assert fake.net == dict(widths=[2, 3, 3, 3, 1], G=7, k=3, m=4, lo=0.0, hi=2.5)
    assert fake.prob["kind"] == capi.HRKAN_BURGERS and fake.prob["alpha"] == 0.05
    assert fake.prob["lam"] == 0.25 and fake.prob["nu"] == pytest.approx(1e-3 / 16, rel=1e-15)
    assert sets[0].shape[1] == 10000 and sets[1].shape[1] == 300
    x_test, u_test = _check_result(fake, res, sets, 3, 1e-2, 3)
    # the reported error is that of the trained weights against the Cole-Hopf truth
    W = inputs.init_weights(oracle.param_count(fake.net), 1003, sigma=0.1).astype(np.float64)
    m1, m2 = np.zeros_like(W), np.zeros_like(W)
    for t in (1, 2, 3):
        loss, _ = oracle.train_step(fake.net, fake.prob, W, m1, m2, sets[0], 0x0F, sets[1], sets[2], 1e-2, t)
        W = W.astype(np.float32).astype(np.float64)
    assert res["train_loss"] == pytest.approx(loss[0], rel=1e-5)
    pred = oracle.forward(fake.net, W, x_test, 0x01)[0]
    assert res["test_mse"] == pytest.approx(np.mean((pred - u_test) ** 2), rel=1e-4)
    assert res["m"] == 4


def test_poisson_driver_passes_section_4_1_set_up(fake):
    res = replica.train_poisson(m=2, seed=1, epochs=2, lr=1e-2)
    assert fake.net == dict(widths=[2, 2, 1], G=5, k=3, m=2, lo=-1.0, hi=1.0)
    assert fake.prob["kind"] == capi.HRKAN_POISSON and fake.prob["alpha"] == 0.05
    assert (fake.prob["a"], fake.prob["b"]) == (1.0, 1.0)
    _check_result(fake, res, replica.poisson_sets(1), 2, 1e-2, 1)
    assert res["m"] == 2 and np.isfinite(res["test_mse"])


def test_tables_summarise_runs_in_percent(fake):
    t = replica.burgers_table(runs=2, m=4, epochs=1, lr=1e-2, sets=replica.burgers_sets(0, n_test=4))
    mse = np.array([r["test_mse"] for r in t["runs"]]) * 100
    assert [r["seed"] for r in t["runs"]] == [0, 1]
    assert t["mean_mse_pct"] == pytest.approx(mse.mean()) and t["std_mse_pct"] == pytest.approx(mse.std())
    assert t["median_mse_pct"] == pytest.approx(np.median(mse))


@pytest.mark.parametrize("name", ["burgers_2_10_10_1", "poisson_2_5_1"])
def test_trainer_test_error_is_against_the_exact_solution(fake, name):
    """At the initial weights the Trainer's test_rel_l2 is the oracle network's relative L2 error
    against the exact solution on the grid: for Burgers (x, t) in [-1, 1] x [0, 1] against the
    Cole-Hopf solution with u(x, 0) = -sin(pi x), for Poisson against sin(pi x) sin(pi y)."""
    w = inputs.WORKLOADS[name]
    data = inputs.make(w, n_int=64, n_bnd=16, n_ic=8, n_bc=8)
    tr = trainer.Trainer(w, data=data, test_grid=12)
    g = np.linspace(-1.0, 1.0, 12)
    if w.pde == inputs.BURGERS:
        A, B = np.meshgrid(g, np.linspace(0.0, 1.0, 12), indexing="ij")
        exact = truth.burgers_sine(A.ravel(), B.ravel(), w.nu)
    else:
        A, B = np.meshgrid(g, g, indexing="ij")
        exact = np.sin(np.pi * A.ravel()) * np.sin(np.pi * B.ravel())
    pts = np.stack([A.ravel(), B.ravel()]).astype(np.float32)
    pred = oracle.forward(w.net, data["W"], pts, 0x01)[0]
    want = np.linalg.norm(pred - exact) / np.linalg.norm(exact)
    assert tr.test_rel_l2() == pytest.approx(want, rel=1e-5)
    assert fake.forwards[-1] == dict(N=144, mask=0x01)
