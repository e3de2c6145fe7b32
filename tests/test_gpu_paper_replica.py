"""The paper's Poisson experiment (Section 4.1, Table 1) run through the library:
[2,2,1], g = 5, k = 3, alpha = 0.05, 960 random interior + 4 x 30 evenly spaced
boundary points, Adam for 3000 epochs, test MSE on the 100 x 100 grid, 10 seeds.

The paper does not state the learning rate or the initial weights (here 1e-2
and N(0, 0.1^2)), so its numbers are context only; what is checked is its
qualitative claim: the HR basis of order m = 4 trains to a lower test error
than the square-of-ReLU basis (ReLU-KAN, the m = 2 case of Eq. 2), and the
best runs reach the paper's reported order (a test MSE below 0.1 %).  The
layer-wise kernels reduce in a fixed order, so every run is reproducible."""
import numpy as np
import pytest

from paper_2409_14248_gb300 import build, capi, replica

def test_sets_follow_section_4_1():
    x_int, x_bnd, g_bnd, x_test, u_test = replica.poisson_sets(0)
    assert x_int.shape == (2, 960) and np.all(np.abs(x_int) <= 1.0)
    assert x_bnd.shape == (2, 120) and np.all(g_bnd == 0.0)
    on_edge = (np.abs(np.abs(x_bnd[0]) - 1.0) < 1e-7) | (np.abs(np.abs(x_bnd[1]) - 1.0) < 1e-7)
    assert np.all(on_edge)
    assert x_test.shape == (2, 10000)
    np.testing.assert_allclose(u_test, np.sin(np.pi * x_test[0]) * np.sin(np.pi * x_test[1]), atol=1e-6)


@pytest.mark.gpu
def test_hr_basis_beats_square_of_relu_on_the_poisson_experiment():
    pytest.importorskip("torch")
    build.build()
    capi.load_library()
    hr = replica.table(runs=10, m=4, lr=1e-2)
    relu = replica.table(runs=10, m=2, lr=1e-2)
    assert hr["median_mse_pct"] < relu["median_mse_pct"]
    assert hr["mean_mse_pct"] < relu["mean_mse_pct"]
    assert min(r["test_mse"] for r in hr["runs"]) * 100.0 < 0.1
    # every run trains: the loss ends 10x below its starting value (about alpha * mean f^2 = 0.05 pi^4 = 4.9)
    assert all(r["train_loss"] < 0.49 for r in hr["runs"])


@pytest.mark.gpu
def test_burgers_experiment_trains_to_the_papers_error_level():
    """The Burgers experiment (Section 4.2, Eq. 7-8, [2,3,3,3,1], g = 7, 3000 epochs) for 4 seeds at
    lr 1e-2.  The FP64 oracle, run on the same sets and initial weights, ends at test MSE 0.088-0.156 %
    (mean 0.119 %; the paper's HRKAN mean is 0.229 %) and training loss 2e-5 to 1.3e-4; FP32 runs
    follow other trajectories, so the bounds are medians with a margin of 2.5x and more."""
    pytest.importorskip("torch")
    build.build()
    capi.load_library()
    t = replica.burgers_table(runs=4, m=4, lr=1e-2)
    assert t["median_mse_pct"] < 0.3, t
    assert np.median([r["train_loss"] for r in t["runs"]]) < 1e-3, t
    assert all(np.isfinite(r["test_mse"]) for r in t["runs"])
