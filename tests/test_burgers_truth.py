"""The reference solution of the Burgers experiment (Section 4.2) and its data
sets, pinned on the CPU.

The solution is the Cole-Hopf formula for u_t + u u_x = nu u_xx with
u(x, 0) = sech x, evaluated by quadrature.  It is checked against things it
does not share code with: an explicit finite-difference solver written here
(central differences in x, the three-stage SSP Runge-Kutta method in t), the
conservation of the total mass integral u dx = pi, and the residual of the
rescaled equation (Eq. 7) taken by central differences, which vanishes with the
coefficients 1/4 and nu/16 and not with the unscaled ones."""
import numpy as np
import pytest

from paper_2409_14248_gb300 import replica

NU = replica.BURGERS_NU


def _fd_solve(nu, T, dx, L=5.0):
    """u(x, T) on [-L, L] by central differences and SSP-RK3, ends held at sech(+-L)."""
    x = np.linspace(-L, L, int(round(2 * L / dx)) + 1)
    u = 1.0 / np.cosh(x)
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
    np.testing.assert_array_equal(replica.cole_hopf_sech(x, 0.0), 1.0 / np.cosh(x))
    # as t -> 0 the quadrature tends to the initial profile
    np.testing.assert_allclose(replica.cole_hopf_sech(x, 1e-6), 1.0 / np.cosh(x), atol=2e-6)
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
    err = replica.cole_hopf_sech(x[inner], T, nu) - u[inner]
    assert np.abs(err).max() < max_tol
    assert np.sqrt(np.mean(err ** 2)) < rms_tol


@pytest.mark.parametrize("T", [0.7, 2.5])
def test_mass_is_conserved(T):
    """integral of u over the line stays integral of sech = pi (the flux u^2/2 - nu u_x vanishes at +-inf)."""
    x = np.linspace(-12.0, 12.0, 24001)
    u = replica.cole_hopf_sech(x, T)
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
