"""Reference solutions of the Burgers problems, and the data sets of the
experiment of Section 4.2, pinned on the CPU.

The solutions are the Cole-Hopf formula for u_t + u u_x = nu u_xx evaluated
by quadrature (truth.burgers_sech: u(x, 0) = sech x, the experiment;
truth.burgers_sine: u(x, 0) = -sin(pi x) on [-1, 1], the Burgers workloads).
They are checked against things they share no code with: an explicit
finite-difference solver written here (central differences in x, the
three-stage SSP Runge-Kutta method in t), the conservation of the mass
integral u dx, the PDE residual taken by central differences (for the
experiment in its rescaled form, Eq. 7, which vanishes with the coefficients
1/4 and nu/16 and not with the unscaled ones), symmetry, and the published
maximum slope of the sine problem at nu = 0.01/pi (Basdevant et al., Computers
& Fluids 14, 1986: |u_x| peaks at 152.00516 at x = 0, t = 1.6037/pi)."""
import math

import numpy as np
import pytest

from paper_2409_14248_gb300 import replica, truth

NU = replica.BURGERS_NU
NU_SINE = 0.01 / math.pi


def _fd_solve(nu, T, dx, L=5.0, u0=lambda x: 1.0 / np.cosh(x)):
    """u(x, T) on [-L, L] by central differences and SSP-RK3, ends held at u0(+-L)."""
    x = np.linspace(-L, L, int(round(2 * L / dx)) + 1)
    u = u0(x)
    dt = min(0.2 * dx * dx / nu, 0.4 * dx)
    steps = int(np.ceil(T / dt))
    dt = T / steps

    def rhs(v):
        r = np.zeros_like(v)
        f = 0.5 * v * v
        r[1:-1] = -(f[2:] - f[:-2]) / (2 * dx) + nu * (v[2:] - 2 * v[1:-1] + v[:-2]) / (dx * dx)
        return r

    for _ in range(steps):
        a = u + dt * rhs(u)
        b = 0.75 * u + 0.25 * (a + dt * rhs(a))
        u = u / 3.0 + (2.0 / 3.0) * (b + dt * rhs(b))
    return x, u


def test_initial_values_are_the_sech_profile():
    x = np.linspace(-5, 5, 101)
    np.testing.assert_array_equal(truth.burgers_sech(x, 0.0), 1.0 / np.cosh(x))
    # as t -> 0 the quadrature tends to the initial profile
    np.testing.assert_allclose(truth.burgers_sech(x, 1e-6), 1.0 / np.cosh(x), atol=2e-6)
    y = np.linspace(0, 2.5, 51)
    np.testing.assert_allclose(replica.burgers_truth(y, 0.0), 1.0 / np.cosh(4 * y - 5), rtol=1e-15)


@pytest.mark.parametrize("nu,T,dx,max_tol,rms_tol", [
    (1e-2, 2.5, 4e-3, 5e-4, 1e-4),     # smooth throughout
    (NU, 1.0, 2e-3, 2e-5, 5e-6),       # the experiment's viscosity before the shock forms (t = 2)
    (NU, 2.5, 1e-3, 1e-2, 5e-4),       # the experiment's final time, with the shock
])
def test_cole_hopf_agrees_with_a_finite_difference_solver(nu, T, dx, max_tol, rms_tol):
    x, u = _fd_solve(nu, T, dx)
    inner = np.abs(x) < 4.5            # away from the solver's fixed ends
    err = truth.burgers_sech(x[inner], T, nu) - u[inner]
    assert np.abs(err).max() < max_tol
    assert np.sqrt(np.mean(err ** 2)) < rms_tol


@pytest.mark.parametrize("T", [0.7, 2.5])
def test_mass_is_conserved(T):
    """integral of u over the line stays integral of sech = pi (the flux u^2/2 - nu u_x vanishes at +-inf)."""
    x = np.linspace(-12.0, 12.0, 24001)
    u = truth.burgers_sech(x, T)
    tails = 4.0 * np.exp(-12.0)        # integral of sech beyond |x| = 12, to leading order
    assert abs(np.trapezoid(u, x) + tails - np.pi) < 1e-5


def test_rescaled_equation_residual_vanishes():
    """u_t + (1/4) u u_y - (nu/16) u_yy = 0 (Eq. 7) by central differences at smooth points (t < 2)."""
    rng = np.random.default_rng(0)
    y, t = rng.uniform(0.3, 2.2, 200), rng.uniform(0.2, 1.5, 200)
    h = 2.5e-4
    U = lambda dy, dt: replica.burgers_truth(y + dy, t + dt)
    u = U(0, 0)
    uy = (U(h, 0) - U(-h, 0)) / (2 * h)
    uyy = (U(h, 0) - 2 * u + U(-h, 0)) / h ** 2
    ut = (U(0, h) - U(0, -h)) / (2 * h)
    r = lambda lam, nu: np.abs(ut + lam * u * uy - nu * uyy).max()
    assert r(0.25, NU / 16) < 2e-5
    # the viscous term is resolved: dropping it, or the unscaled coefficients, leave a residual
    assert r(0.25, 0.0) > 1e-3
    assert r(0.25, NU) > 1e-2
    assert r(1.0, NU / 16) > 1.0


def test_burgers_sets_follow_section_4_2():
    x_int, x_bnd, g_bnd, x_test, u_test = replica.burgers_sets(0, n_test=20)
    L = replica.BURGERS_SIDE
    assert x_int.shape == (2, 10000) and x_int.min() >= 0.0 and x_int.max() <= L
    assert x_bnd.shape == (2, 300) and g_bnd.shape == (300,)
    left, right, init = slice(0, 100), slice(100, 200), slice(200, 300)
    assert np.all(x_bnd[0, left] == 0.0) and np.all(x_bnd[0, right] == np.float32(L))
    assert np.all(g_bnd[:200] == 0.0)
    np.testing.assert_allclose(x_bnd[1, left], np.linspace(0, L, 100), rtol=1e-6)
    assert np.all(x_bnd[1, init] == 0.0)
    np.testing.assert_allclose(g_bnd[init], 1.0 / np.cosh(4.0 * x_bnd[0, init].astype(np.float64) - 5.0),
                               rtol=1e-6)
    assert x_test.shape == (2, 400) and u_test.shape == (400,)
    np.testing.assert_allclose(u_test, replica.burgers_truth(x_test[0], x_test[1]), rtol=1e-12)


def _fall_width(t):
    """Distance in y over which u(., t) falls from 0.9 to 0.3 behind its peak."""
    y = np.linspace(1.0, 2.5, 15001)
    u = replica.burgers_truth(y, t)
    i = int(u.argmax())
    return y[i + int(np.argmax(u[i:] < 0.3))] - y[i + int(np.argmax(u[i:] < 0.9))]


def test_the_wave_steepens_into_a_shock():
    """sech falls at most with slope 1/2, so characteristics first cross at t = 2: before that the
    front is spread over tenths of a unit in y; at t = 2.5 it is a viscous shock under 0.02 wide."""
    assert _fall_width(1.0) > 0.15
    assert _fall_width(2.5) < 0.02


def _sine(x, t, **kw):
    return truth.burgers_sine(x, t, NU_SINE, **kw)


def test_sine_problem_matches_the_published_maximum_slope():
    ts = np.linspace(1.59, 1.62, 61) / np.pi
    _, ux = _sine(np.zeros_like(ts), ts, slope=True)
    i = int(np.argmin(ux))
    assert abs(ts[i] * np.pi - 1.6037) < 1e-3
    assert abs(-ux[i] - 152.00516) < 2e-3


def test_sine_problem_is_odd_and_vanishes_at_the_walls():
    x = np.linspace(-1.0, 1.0, 201)
    for t in (0.0, 0.2, 0.5, 1.0):
        u = _sine(x, t)
        np.testing.assert_allclose(u, -u[::-1], atol=1e-12)
        assert abs(u[0]) < 1e-12 and abs(u[-1]) < 1e-12 and abs(u[100]) < 1e-12


def _sine_fd_error(T, dx):
    x, u = _fd_solve(NU_SINE, T, dx, L=1.0, u0=lambda x: -np.sin(np.pi * x))
    err = _sine(x, T) - u
    return np.abs(err).max(), np.sqrt(np.mean(err ** 2))


def test_finite_differences_converge_to_the_sine_solution_at_second_order():
    """t = 0.3, as the front steepens (slope about -55): halving dx cuts the gap to the
    quadrature by 4, as it must for a second-order scheme converging to the same function."""
    coarse, fine = _sine_fd_error(0.3, 2e-3), _sine_fd_error(0.3, 1e-3)
    for c, f in zip(coarse, fine):
        assert 3.5 < c / f < 4.5
    assert fine[0] < 2e-4
    assert max(_sine_fd_error(0.15, 2e-3)) < 2e-5        # smooth: close already on the coarse grid


def test_sine_problem_agrees_with_a_finite_difference_solver_across_the_shock():
    worst, rms = _sine_fd_error(1.0, 5e-4)
    assert worst < 2e-2 and rms < 1e-3


def test_sine_problem_residual_vanishes():
    """u_t + u u_x - nu u_xx = 0 by central differences away from the shock."""
    rng = np.random.default_rng(1)
    x, t = rng.uniform(0.2, 0.9, 100) * rng.choice([-1, 1], 100), rng.uniform(0.05, 0.9, 100)
    h = 2.5e-4
    U = lambda dx, dt: _sine(x + dx, t + dt)
    u = U(0, 0)
    ux = (U(h, 0) - U(-h, 0)) / (2 * h)
    uxx = (U(h, 0) - 2 * u + U(-h, 0)) / h ** 2
    ut = (U(0, h) - U(0, -h)) / (2 * h)
    assert np.abs(ut + u * ux - NU_SINE * uxx).max() < 1e-4
    assert np.abs(ut + u * ux).max() > 1e-3        # the viscous term is resolved


@pytest.mark.parametrize("which", ["sech", "sine"])
def test_slope_from_the_quadrature_moments_equals_differences_of_u(which):
    f = (lambda x, t, **k: truth.burgers_sech(x, t, NU, **k)) if which == "sech" else _sine
    rng = np.random.default_rng(2)
    x, t = rng.uniform(-0.9, 0.9, 100), rng.uniform(0.1, 0.9, 100)
    h = 1e-5
    u, ux = f(x, t, slope=True)
    np.testing.assert_allclose(u, f(x, t), rtol=0, atol=1e-14)
    fd = (f(x + h, t) - f(x - h, t)) / (2 * h)
    assert np.abs(ux - fd).max() < 1e-5 * max(1.0, np.abs(ux).max())


def test_poisson_truth():
    x, y = np.meshgrid(np.linspace(-1, 1, 9), np.linspace(-1, 1, 9))
    np.testing.assert_allclose(truth.poisson(x, y, 2.0, 3.0), np.sin(2 * np.pi * x) * np.sin(3 * np.pi * y))
    assert truth.poisson(0.5, 0.5) == pytest.approx(1.0)
