"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
closed forms (golden files), a polynomial expansion of Eq. 2 differentiated by
numpy, the ReLU-KAN basis of Eq. 1 (the m = 2 case), symbolic differentiation
(sympy) of a small network, central finite differences, manufactured PDE
solutions with zero residual, and torch.optim.Adam in float64.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2409_14248_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ support


def test_support_matches_bspline_supports_g5_k3():
    """Section 2.1-2.2: n = g + k = 8 supports of B_{5,3} on [-1, 1]."""
    gold = np.loadtxt(os.path.join(GOLD, "support_g5_k3.txt"))
    s, e = oracle.support(5, 3, -1.0, 1.0)
    assert len(s) == 8
    np.testing.assert_allclose(s, gold[:, 1], atol=1e-15)
    np.testing.assert_allclose(e, gold[:, 2], atol=1e-15)


def test_every_interior_point_lies_in_k_plus_1_supports():
    s, e = oracle.support(10, 3, -1.0, 1.0)
    xs = np.random.default_rng(0).uniform(-1, 1, 500)
    for x in xs:
        assert np.sum((x > s) & (x < e)) == 4


# -------------------------------------------------------------------- basis


def test_basis_golden_values_m4():
    """Section 3, Eq. 2: hand-derived exact values of v_{4,4} and derivatives."""
    gold = np.loadtxt(os.path.join(GOLD, "hr_basis_m4.txt"))
    for row in gold:
        got = oracle.hr_basis(4, -0.6, 1.0, row[0])[:4]
        np.testing.assert_allclose(got, row[1:], rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_basis_peak_one_at_midpoint_and_zero_outside(m):
    """Eq. 2: c_m normalises the height of each basis to 1 at the midpoint."""
    s, e = -0.3, 0.9
    assert oracle.hr_basis(m, s, e, 0.3)[0] == pytest.approx(1.0, rel=1e-14)
    for x in (-1.0, s, e, 2.0):
        assert oracle.hr_basis(m, s, e, x)[0] == 0.0


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_basis_matches_polynomial_expansion(m):
    """Eq. 2 inside (s, e) is c_m ((e-x)(x-s))^m; numpy expands and differentiates it."""
    s, e = -1.4, 0.2
    c = (2.0 / (e - s)) ** (2 * m)
    p = np.polynomial.Polynomial([-e * s, e + s, -1.0])  # (e-x)(x-s)
    P = c * p ** m
    ders = [P, P.deriv(1), P.deriv(2), P.deriv(3), P.deriv(4)]
    # the monomial expansion cancels near the knots: compare on each derivative's own scale
    scale = np.array([np.abs(d(np.linspace(s, e, 401))).max() for d in ders])
    for x in np.random.default_rng(m).uniform(s + 1e-3, e - 1e-3, 40):
        got = oracle.hr_basis(m, s, e, x)
        want = np.array([d(x) for d in ders])
        np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-10 * scale.max())
        assert np.all(np.abs(got - want) <= 1e-10 * scale)


def test_m2_equals_relu_kan_square_of_relu():
    """Eq. 1 (ReLU-KAN): r_i = [ReLU(e-x) ReLU(x-s)]^2 * 16/(e-s)^4 is the m = 2 case."""
    s, e = -0.6, 1.0
    for x in np.linspace(-1.0, 1.4, 97):
        r = (max(e - x, 0.0) * max(x - s, 0.0)) ** 2 * 16.0 / (e - s) ** 4
        assert oracle.hr_basis(2, s, e, x)[0] == pytest.approx(r, rel=1e-14, abs=1e-300)


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_basis_integral_closed_form(m):
    """int v = (e-s) 2^{2m} (m!)^2 / (2m+1)!  (Beta integral of (1-u^2)^m)."""
    from scipy.integrate import quad
    s, e = -0.2, 1.4
    val, _ = quad(lambda x: oracle.hr_basis(m, s, e, x)[0], s, e, epsabs=1e-14, epsrel=1e-13)
    want = (e - s) * 2 ** (2 * m) * math.factorial(m) ** 2 / math.factorial(2 * m + 1)
    assert val == pytest.approx(want, rel=1e-11)


def test_basis_symmetry_and_smoothness_at_knots():
    """v(s+e-x) = v(x); for m = 4 the derivatives up to order 3 vanish at the knots
    (Section 3: smooth, C^{m-1} at the ends of the support)."""
    m, s, e = 4, -0.6, 1.0
    for x in np.random.default_rng(1).uniform(s, e, 30):
        a = oracle.hr_basis(m, s, e, x)
        b = oracle.hr_basis(m, s, e, s + e - x)
        np.testing.assert_allclose(a * np.array([1, -1, 1, -1, 1]), b, rtol=1e-10, atol=1e-10)
    # the r-th derivative vanishes like delta^{m-r} next to each knot
    for knot, sign in ((s, 1.0), (e, -1.0)):
        a = np.abs(oracle.hr_basis(m, s, e, knot + sign * 1e-6))
        b = np.abs(oracle.hr_basis(m, s, e, knot + sign * 1e-7))
        # (the fourth derivative tends to a nonzero constant: m - 4 = 0)
        np.testing.assert_allclose(a / b, [1e4, 1e3, 1e2, 1e1, 1.0], rtol=1e-4)


def test_m2_second_derivative_jumps_at_support_end():
    """Section 3: the square-of-ReLU second derivative jumps at the end points; HR (m=4) does not."""
    s, e = -0.6, 1.0
    inside = oracle.hr_basis(2, s, e, s + 1e-9)[2]
    assert inside == pytest.approx(2 * 16.0 / (e - s) ** 2, rel=1e-6)
    assert abs(oracle.hr_basis(4, s, e, s + 1e-9)[2]) < 1e-12


# ------------------------------------------------------------------ network


def _sympy_network_at(widths, G, k, m, lo, hi, W, point):
    """The network of Sections 1-3 as a sympy expression in (x, y), valid near `point`:
    each basis of Eq. 2 enters as its polynomial piece c_m ((e-z)(x-s))^m where its ReLUs
    are active at the point, and not at all where it is zero there."""
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x0:%d" % widths[0], real=True)
    h = (hi - lo) / G
    n = G + k
    z = list(X)
    zn = [float(v) for v in point]
    off = 0
    for l in range(len(widths) - 1):
        I, O = widths[l], widths[l + 1]
        Wl = W[off: off + O * I * n].reshape(O, I, n)
        off += O * I * n
        out, outn = [], []
        for o in range(O):
            expr, val = 0, 0.0
            for j in range(I):
                for i in range(n):
                    s = lo + (i - k) * h
                    e = lo + (i + 1) * h
                    if s < zn[j] < e:
                        c = (2.0 / (e - s)) ** (2 * m)
                        expr += float(Wl[o, j, i]) * c * ((e - z[j]) * (z[j] - s)) ** m
                        val += float(Wl[o, j, i]) * c * ((e - zn[j]) * (zn[j] - s)) ** m
            out.append(sp.expand(expr) if l == 0 else expr)
            outn.append(val)
        z, zn = out, outn
    return X, z[0]


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_forward_jets_match_symbolic_differentiation(m):
    """Brute force on 8 points: jets of a [2,2,1] net vs sympy derivatives of its definition,
    for each HR order m the layer-wise kernels accept."""
    sp = pytest.importorskip("sympy")
    net = dict(widths=[2, 2, 1], G=5, k=3, m=m, lo=-1.0, hi=1.0)
    P = oracle.param_count(net)
    W = np.random.default_rng(3).normal(0, 0.5, P)
    x = np.random.default_rng(4).uniform(-1, 1, (2, 8))
    jets = oracle.forward(net, W, x, 0x1F)
    for p in range(8):
        X, u = _sympy_network_at(net["widths"], 5, 3, m, -1.0, 1.0, W, x[:, p])
        exprs = [u, sp.diff(u, X[0]), sp.diff(u, X[1]), sp.diff(u, X[0], 2), sp.diff(u, X[1], 2)]
        sub = {X[0]: x[0, p], X[1]: x[1, p]}
        want = np.array([float(e.evalf(subs=sub)) for e in exprs])
        np.testing.assert_allclose(jets[:, p], want, rtol=1e-9, atol=1e-9)


def test_single_layer_net_is_weighted_basis_sum():
    """A [1,1] net is u(x) = sum_i w_i v_i(x), here with v_i from the polynomial expansion."""
    net = dict(widths=[1, 1], G=4, k=3, m=4, lo=-1.0, hi=1.0)
    n = 7
    w = np.random.default_rng(5).normal(size=n)
    s, e = -1.0 + (np.arange(n) - 3) * 0.5, -1.0 + (np.arange(n) + 1) * 0.5
    x = np.random.default_rng(6).uniform(-1, 1, (1, 50))
    jets = oracle.forward(net, w, x, 0b111)
    want = np.zeros((3, 50))
    for i in range(n):
        c = (2.0 / (e[i] - s[i])) ** 8
        P = c * np.polynomial.Polynomial([-e[i] * s[i], e[i] + s[i], -1.0]) ** 4
        inside = (x[0] > s[i]) & (x[0] < e[i])
        for r in range(3):
            want[r] += w[i] * np.where(inside, P.deriv(r)(x[0]), 0.0)
    np.testing.assert_allclose(jets, want, rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("widths,G", [([2, 3, 1], 5), ([2, 4, 3, 1], 7)])
def test_forward_jets_match_central_differences(widths, G):
    net = dict(widths=widths, G=G, k=3, m=4, lo=-1.0, hi=1.0)
    W = np.random.default_rng(7).normal(0, 0.3, oracle.param_count(net))
    x = np.random.default_rng(8).uniform(-0.9, 0.9, (2, 16))
    jets = oracle.forward(net, W, x, 0x1F)
    u = lambda xx: oracle.forward(net, W, xx, 0x1)[0]
    for d in range(2):
        h1, h2 = 1e-6, 1e-4
        e = np.zeros((2, 1)); e[d] = 1.0
        fd1 = (u(x + h1 * e) - u(x - h1 * e)) / (2 * h1)
        fd2 = (u(x + h2 * e) - 2 * u(x) + u(x - h2 * e)) / h2 ** 2
        np.testing.assert_allclose(jets[1 + d], fd1, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(jets[3 + d], fd2, rtol=1e-4, atol=1e-4 * np.abs(fd2).max())


@pytest.mark.parametrize("m", [3, 6])
def test_third_order_jets_match_symbolic_differentiation(m):
    """Third derivatives (mask bits 5, 6) and the mixed derivative (bit 7) of a [2,2,1] net
    vs sympy on the polynomial pieces."""
    sp = pytest.importorskip("sympy")
    net = dict(widths=[2, 2, 1], G=5, k=3, m=m, lo=-1.0, hi=1.0)
    W = np.random.default_rng(30 + m).normal(0, 0.5, oracle.param_count(net))
    x = np.random.default_rng(31).uniform(-1, 1, (2, 3))
    jets = oracle.forward(net, W, x, 0xFF)
    for p in range(3):
        X, u = _sympy_network_at(net["widths"], 5, 3, m, -1.0, 1.0, W, x[:, p])
        exprs = [u, sp.diff(u, X[0]), sp.diff(u, X[1]), sp.diff(u, X[0], 2), sp.diff(u, X[1], 2),
                 sp.diff(u, X[0], 3), sp.diff(u, X[1], 3), sp.diff(u, X[0], X[1])]
        sub = {X[0]: x[0, p], X[1]: x[1, p]}
        want = np.array([float(e.evalf(subs=sub)) for e in exprs])
        # sympy evaluates the expanded degree-2m(m+1) pieces in floating point: ~1e-9 cancellation
        np.testing.assert_allclose(jets[:, p], want, rtol=1e-8, atol=1e-8)


def test_third_order_jets_match_central_differences():
    """u_ddd and u_01 equal central differences of the oracle's own u_dd and u_0 (a check
    independent of sympy)."""
    net = dict(widths=[2, 4, 3, 1], G=6, k=3, m=4, lo=-1.0, hi=1.0)
    W = np.random.default_rng(32).normal(0, 0.3, oracle.param_count(net))
    x = np.random.default_rng(33).uniform(-0.9, 0.9, (2, 16))
    jets = oracle.forward(net, W, x, 0xFF)
    h = 1e-5
    for d in range(2):
        e = np.zeros((2, 1)); e[d] = 1.0
        udd = lambda xx: oracle.forward(net, W, xx, 0x1F)[3 + d]
        fd = (udd(x + h * e) - udd(x - h * e)) / (2 * h)
        np.testing.assert_allclose(jets[5 + d], fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    e1 = np.array([[0.0], [1.0]])
    ux = lambda xx: oracle.forward(net, W, xx, 0x07)[1]
    fd = (ux(x + h * e1) - ux(x - h * e1)) / (2 * h)
    np.testing.assert_allclose(jets[7], fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())


@pytest.mark.parametrize("m", [4, 6])
def test_third_order_weight_gradient_matches_central_differences(m):
    """Backward through the third-derivative rows (which needs the basis's fourth derivative) and
    the mixed row vs central FD of L(W) = sum(R * jets) over all eight rows, on 48 random weights."""
    net = dict(widths=[2, 3, 3, 1], G=5, k=3, m=m, lo=-1.0, hi=1.0)
    rng = np.random.default_rng(34 + m)
    W = rng.normal(0, 0.4, oracle.param_count(net))
    x = rng.uniform(-1, 1, (2, 25))
    R = rng.normal(0, 1, (8, 25))
    dW = oracle.backward(net, W, x, 0xFF, R)
    loss = lambda Wv: float((R * oracle.forward(net, Wv, x, 0xFF)).sum())
    h = 1e-6
    for i in rng.choice(W.size, 48, replace=False):
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += h; Wm[i] -= h
        fd = (loss(Wp) - loss(Wm)) / (2 * h)
        assert dW[i] == pytest.approx(fd, rel=2e-5, abs=2e-8 * max(1.0, np.abs(dW).max()))


def test_third_order_rows_leave_lower_rows_unchanged():
    """Adding bits 5, 6 to a mask appends rows; the value, first and second rows are unchanged."""
    net = dict(widths=[2, 3, 1], G=5, k=3, m=4, lo=-1.0, hi=1.0)
    W = np.random.default_rng(36).normal(0, 0.3, oracle.param_count(net))
    x = np.random.default_rng(37).uniform(-1, 1, (2, 9))
    full = oracle.forward(net, W, x, 0x7F)
    np.testing.assert_array_equal(oracle.forward(net, W, x, 0x1F), full[:5])
    np.testing.assert_array_equal(oracle.forward(net, W, x, 0x2F), full[[0, 1, 2, 3, 5]])
    mixed = oracle.forward(net, W, x, 0xFF)
    np.testing.assert_array_equal(mixed[:7], full)
    np.testing.assert_array_equal(oracle.forward(net, W, x, 0x87), mixed[[0, 1, 2, 7]])


def test_three_input_jets_match_symbolic_differentiation():
    """D = 3 (a [3,2,1] net): u, the three first and three second derivatives (mask bits
    0, 1+d, 4+d) vs sympy on the polynomial pieces."""
    sp = pytest.importorskip("sympy")
    net = dict(widths=[3, 2, 1], G=4, k=3, m=4, lo=-1.0, hi=1.0)
    W = np.random.default_rng(38).normal(0, 0.5, oracle.param_count(net))
    x = np.random.default_rng(39).uniform(-1, 1, (3, 3))
    jets = oracle.forward(net, W, x, 0x7F)
    for p in range(3):
        X, u = _sympy_network_at(net["widths"], 4, 3, 4, -1.0, 1.0, W, x[:, p])
        exprs = [u] + [sp.diff(u, X[d]) for d in range(3)] + [sp.diff(u, X[d], 2) for d in range(3)]
        sub = {X[d]: x[d, p] for d in range(3)}
        want = np.array([float(e.evalf(subs=sub)) for e in exprs])
        np.testing.assert_allclose(jets[:, p], want, rtol=1e-8, atol=1e-8)


def test_three_input_weight_gradient_matches_central_differences():
    """D = 3 backward vs central FD of L(W) = sum(R * jets) over the seven rows."""
    net = dict(widths=[3, 4, 3, 1], G=5, k=3, m=4, lo=-1.0, hi=1.0)
    rng = np.random.default_rng(40)
    W = rng.normal(0, 0.4, oracle.param_count(net))
    x = rng.uniform(-1, 1, (3, 20))
    R = rng.normal(0, 1, (7, 20))
    dW = oracle.backward(net, W, x, 0x7F, R)
    loss = lambda Wv: float((R * oracle.forward(net, Wv, x, 0x7F)).sum())
    h = 1e-6
    for i in rng.choice(W.size, 40, replace=False):
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += h; Wm[i] -= h
        fd = (loss(Wp) - loss(Wm)) / (2 * h)
        assert dW[i] == pytest.approx(fd, rel=2e-5, abs=2e-8 * max(1.0, np.abs(dW).max()))


def test_mask_selects_rows_in_bit_order():
    net = dict(widths=[2, 3, 1], G=5, k=3, m=4, lo=-1.0, hi=1.0)
    W = np.random.default_rng(9).normal(0, 0.3, oracle.param_count(net))
    x = np.random.default_rng(10).uniform(-1, 1, (2, 5))
    full = oracle.forward(net, W, x, 0x1F)
    np.testing.assert_array_equal(oracle.forward(net, W, x, inputs.MASK_BURGERS), full[[0, 1, 2, 3]])
    np.testing.assert_array_equal(oracle.forward(net, W, x, 0x1 | 0x4 | 0x10), full[[0, 2, 4]])


def test_points_outside_extended_grid_are_dead():
    """Inputs beyond [lo - k h, hi + k h] touch no basis: the first layer outputs 0, so two
    such points share one output value and every input derivative is exactly zero."""
    net = dict(widths=[2, 3, 1], G=5, k=3, m=4, lo=-1.0, hi=1.0)
    W = np.random.default_rng(11).normal(0, 0.3, oracle.param_count(net))
    x = np.array([[2.3, -2.5, -2.21], [-3.0, 3.0, 2.5]])
    jets = oracle.forward(net, W, x, 0x1F)
    assert np.all(jets[1:] == 0.0)
    assert jets[0, 0] == jets[0, 1] == jets[0, 2]
    single = oracle.forward(dict(net, widths=[3, 1]), W[48:], np.zeros((3, 1)), 0x1)
    assert jets[0, 0] == pytest.approx(single[0, 0], rel=1e-15)


# --------------------------------------------------------------------- loss


def test_poisson_residual_zero_on_manufactured_solution():
    """Eq. 3-4: the exact jets of u* = sin(a pi x) sin(b pi y) give r = 0."""
    rng = np.random.default_rng(12)
    for a, b in [(1, 1), (2, 2), (3, 1)]:
        x = rng.uniform(-1, 1, (2, 64))
        su, sv = np.sin(a * np.pi * x[0]), np.sin(b * np.pi * x[1])
        cu, cv = np.cos(a * np.pi * x[0]), np.cos(b * np.pi * x[1])
        jets = np.stack([su * sv, a * np.pi * cu * sv, b * np.pi * su * cv,
                         -(a * np.pi) ** 2 * su * sv, -(b * np.pi) ** 2 * su * sv])
        prob = dict(kind=oracle.POISSON, a=a, b=b, alpha=0.05)
        loss, dj, _ = oracle.residual_loss(prob, x, 0x1F, jets, np.zeros(4), np.zeros(4))
        assert loss[1] < 1e-24
        assert np.abs(dj).max() < 1e-12


def test_poisson3_residual_zero_on_manufactured_solution():
    """The Poisson equation in three dimensions: the exact jets of
    u* = sin(a pi x) sin(b pi y) sin(c pi z) (c in lam) give r = 0, rows u, u_x, u_y, u_z,
    u_xx, u_yy, u_zz of mask 0x7F."""
    rng = np.random.default_rng(41)
    for a, b, c in [(1, 1, 1), (2, 1, 3)]:
        x = rng.uniform(-1, 1, (3, 64))
        s = [np.sin(k * np.pi * x[d]) for d, k in enumerate((a, b, c))]
        co = [np.cos(k * np.pi * x[d]) for d, k in enumerate((a, b, c))]
        u = s[0] * s[1] * s[2]
        jets = np.stack([u, a * np.pi * co[0] * s[1] * s[2], b * np.pi * s[0] * co[1] * s[2],
                         c * np.pi * s[0] * s[1] * co[2], -(a * np.pi) ** 2 * u, -(b * np.pi) ** 2 * u,
                         -(c * np.pi) ** 2 * u])
        prob = dict(kind=oracle.POISSON3, a=a, b=b, lam=c, alpha=0.5)
        loss, dj, _ = oracle.residual_loss(prob, x, 0x7F, jets, np.zeros(4), np.zeros(4))
        assert loss[1] < 1e-24
        assert np.abs(dj).max() < 1e-12


def test_poisson3_zero_network_loss_and_jet_gradient():
    """u = 0 (zero jets): L_pde = mean(f^2) with f = (a^2+b^2+c^2) pi^2 sin sin sin written out,
    L = alpha L_pde + mean(g^2); dL/d(u_xx) = dL/d(u_yy) = dL/d(u_zz) = 2 alpha f / N, and the other
    rows get nothing.  Central differences of L in single jet entries agree (L is quadratic in
    the jets, so a central difference is exact for any step)."""
    rng = np.random.default_rng(42)
    a, b, c, alpha, N = 2.0, 1.0, 3.0, 0.3, 40
    x = rng.uniform(-1, 1, (3, N))
    g = rng.normal(0, 1, 9)
    f = (a * a + b * b + c * c) * np.pi ** 2 * np.sin(a * np.pi * x[0]) * np.sin(b * np.pi * x[1]) * \
        np.sin(c * np.pi * x[2])
    prob = dict(kind=oracle.POISSON3, a=a, b=b, lam=c, alpha=alpha)
    jets = np.zeros((7, N))
    loss, dj, du = oracle.residual_loss(prob, x, 0x7F, jets, np.zeros(9), g)
    assert loss[1] == pytest.approx(np.mean(f * f), rel=1e-13)
    assert loss[0] == pytest.approx(alpha * np.mean(f * f) + np.mean(g * g), rel=1e-13)
    for r in (4, 5, 6):
        np.testing.assert_allclose(dj[r], 2 * alpha * f / N, rtol=1e-13)
    assert np.all(dj[:4] == 0.0)
    np.testing.assert_allclose(du, -2 * g / 9, rtol=1e-13)
    jets = rng.normal(0, 1, (7, N))
    _, dj, _ = oracle.residual_loss(prob, x, 0x7F, jets, np.zeros(9), g)
    h = 1e-2
    for r, p in [(4, 3), (5, 17), (6, 29), (0, 5)]:
        jp, jm = jets.copy(), jets.copy()
        jp[r, p] += h; jm[r, p] -= h
        fd = (oracle.residual_loss(prob, x, 0x7F, jp, np.zeros(9), g)[0][0] -
              oracle.residual_loss(prob, x, 0x7F, jm, np.zeros(9), g)[0][0]) / (2 * h)
        assert dj[r, p] == pytest.approx(fd, rel=1e-8, abs=1e-9)


def test_poisson3_train_step_gradient_matches_central_differences():
    """A D = 3 training step ([3,4,1], mask 0x7F): the gradient it applies equals central
    differences of its loss in the weights, and its Adam update is the first-step closed form
    w - lr g / (|g| + eps)."""
    net = dict(widths=[3, 4, 1], G=4, k=3, m=4, lo=-1.0, hi=1.0)
    rng = np.random.default_rng(43)
    P = oracle.param_count(net)
    W0 = rng.normal(0, 0.4, P)
    xi = rng.uniform(-1, 1, (3, 30))
    xb = rng.uniform(-1, 1, (3, 12))
    gb = rng.normal(0, 0.5, 12)
    prob = dict(kind=oracle.POISSON3, a=1.0, b=2.0, lam=1.0, alpha=0.7)
    W = W0.copy()
    loss, dW = oracle.train_step(net, prob, W, np.zeros(P), np.zeros(P), xi, 0x7F, xb, gb, 1e-3, 1)

    def L(Wv):
        jets = oracle.forward(net, Wv, xi, 0x7F)
        ub = oracle.forward(net, Wv, xb, 0x1)[0]
        return oracle.residual_loss(prob, xi, 0x7F, jets, ub, gb)[0][0]

    assert loss[0] == pytest.approx(L(W0), rel=1e-13)
    h = 1e-6
    for i in rng.choice(P, 25, replace=False):
        Wp, Wm = W0.copy(), W0.copy()
        Wp[i] += h; Wm[i] -= h
        assert dW[i] == pytest.approx((L(Wp) - L(Wm)) / (2 * h), rel=2e-5, abs=1e-8 * max(1.0, np.abs(dW).max()))
    np.testing.assert_allclose(W, W0 - 1e-3 * dW / (np.abs(dW) + 1e-8), rtol=1e-12, atol=1e-15)


def test_burgers_residual_zero_on_cole_hopf_solution():
    """Eq. 6-8 form: u = 2 nu pi e^{-nu pi^2 t} sin(pi x) / (a0 + e^{-nu pi^2 t} cos(pi x))
    solves u_t + u u_x = nu u_xx exactly (Cole-Hopf); sympy supplies its jets."""
    sp = pytest.importorskip("sympy")
    X, T = sp.symbols("x t", real=True)
    nu, a0 = 0.05, 2.0
    E = sp.exp(-nu * sp.pi ** 2 * T)
    u = 2 * nu * sp.pi * E * sp.sin(sp.pi * X) / (a0 + E * sp.cos(sp.pi * X))
    fs = [sp.lambdify((X, T), f, "numpy") for f in (u, sp.diff(u, X), sp.diff(u, T), sp.diff(u, X, 2))]
    x = np.random.default_rng(13).uniform([[-1], [0]], [[1], [1]], (2, 64))
    jets = np.stack([f(x[0], x[1]) for f in fs])
    prob = dict(kind=oracle.BURGERS, lam=1.0, nu=nu, alpha=1.0)
    loss, _, _ = oracle.residual_loss(prob, x, inputs.MASK_BURGERS, jets, np.zeros(1), np.zeros(1))
    assert loss[1] < 1e-26


def test_kdv_residual_zero_on_the_soliton():
    """u = (c/2) sech^2(sqrt(c)/2 (x - c t - x0)) solves u_t + 6 u u_x + u_xxx = 0 exactly
    (the KdV soliton); sympy supplies its jets (u, u_x, u_t, u_xx, u_xxx: mask 0x2F)."""
    sp = pytest.importorskip("sympy")
    X, T = sp.symbols("x t", real=True)
    c, x0 = 1.7, 0.2
    u = c / 2 * sp.sech(sp.sqrt(c) / 2 * (X - c * T - x0)) ** 2
    fs = [sp.lambdify((X, T), f, "numpy")
          for f in (u, sp.diff(u, X), sp.diff(u, T), sp.diff(u, X, 2), sp.diff(u, X, 3))]
    x = np.random.default_rng(16).uniform([[-1], [0]], [[1], [1]], (2, 64))
    jets = np.stack([f(x[0], x[1]) for f in fs])
    prob = dict(kind=oracle.KDV, lam=6.0, nu=1.0, alpha=1.0)
    loss, _, _ = oracle.residual_loss(prob, x, 0x2F, jets, np.zeros(1), np.zeros(1))
    assert loss[1] < 1e-24
    # a wrong coefficient leaves a residual of the size of the dropped term
    bad, _, _ = oracle.residual_loss(dict(prob, lam=5.0), x, 0x2F, jets, np.zeros(1), np.zeros(1))
    assert bad[1] > 1e-4


def test_loss_of_zero_network_is_mean_source_squared():
    """W = 0 gives u = 0: L = alpha mean(f^2) + mean(g^2)."""
    w = inputs.WORKLOADS["poisson_2_5_1"]
    d = inputs.make(w, n_int=200, n_bnd=40)
    net = w.net
    W = np.zeros(oracle.param_count(net))
    x = d["x_int"].astype(np.float64)
    g = np.random.default_rng(14).normal(size=40)
    jets = oracle.forward(net, W, x, 0x1F)
    ub = oracle.forward(net, W, d["x_bnd"], 0x1)[0]
    alpha = 0.05
    loss, _, _ = oracle.residual_loss(dict(kind=oracle.POISSON, a=1, b=1, alpha=alpha), x, 0x1F, jets, ub, g)
    f = 2 * np.pi ** 2 * np.sin(np.pi * x[0]) * np.sin(np.pi * x[1])
    assert loss[0] == pytest.approx(alpha * np.mean(f ** 2) + np.mean(g ** 2), rel=1e-13)


@pytest.mark.parametrize("kind", [oracle.POISSON, oracle.BURGERS, oracle.KDV])
def test_loss_gradient_wrt_jets_matches_central_differences(kind):
    rng = np.random.default_rng(15)
    mask = {oracle.POISSON: 0x1F, oracle.BURGERS: inputs.MASK_BURGERS, oracle.KDV: 0x2F}[kind]
    J = oracle.n_rows(mask)
    x = rng.uniform(-1, 1, (2, 12))
    jets = rng.normal(size=(J, 12))
    ub, gb = rng.normal(size=6), rng.normal(size=6)
    prob = dict(kind=kind, a=2, b=1, lam=0.7, nu=0.3, alpha=0.4)
    _, dj, du = oracle.residual_loss(prob, x, mask, jets, ub, gb)
    h = 1e-6
    for r in range(J):
        for p in range(0, 12, 5):
            jp, jm = jets.copy(), jets.copy()
            jp[r, p] += h; jm[r, p] -= h
            fd = (oracle.residual_loss(prob, x, mask, jp, ub, gb)[0][0]
                  - oracle.residual_loss(prob, x, mask, jm, ub, gb)[0][0]) / (2 * h)
            assert dj[r, p] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for p in range(6):
        up, um = ub.copy(), ub.copy()
        up[p] += h; um[p] -= h
        fd = (oracle.residual_loss(prob, x, mask, jets, up, gb)[0][0]
              - oracle.residual_loss(prob, x, mask, jets, um, gb)[0][0]) / (2 * h)
        assert du[p] == pytest.approx(fd, rel=1e-6, abs=1e-9)


# ----------------------------------------------------------------- backward


def _total_loss(net, prob, W, x_int, mask, x_bnd, g_bnd):
    jets = oracle.forward(net, W, x_int, mask)
    ub = oracle.forward(net, W, x_bnd, 0x1)[0]
    loss, dj, du = oracle.residual_loss(prob, x_int, mask, jets, ub, g_bnd)
    return loss[0], dj, du


@pytest.mark.parametrize("case,m", [("poisson", 4), ("burgers", 4), ("poisson", 3), ("burgers", 6)])
def test_weight_gradient_matches_central_differences(case, m):
    """Hand-written backward vs central FD (h = 1e-6, FP64) on 64 random weights."""
    rng = np.random.default_rng(16)
    if case == "poisson":
        net = dict(widths=[2, 4, 3, 1], G=5, k=3, m=m, lo=-1.0, hi=1.0)
        prob = dict(kind=oracle.POISSON, a=1, b=2, alpha=0.5)
        mask = 0x1F
        x_int = rng.uniform(-1, 1, (2, 40))
        x_bnd = np.stack([rng.choice([-1.0, 1.0], 12), rng.uniform(-1, 1, 12)])
    else:
        net = dict(widths=[2, 3, 3, 1], G=6, k=3, m=m, lo=-1.0, hi=1.0)
        prob = dict(kind=oracle.BURGERS, lam=1.0, nu=0.01 / np.pi, alpha=1.0)
        mask = inputs.MASK_BURGERS
        x_int = np.stack([rng.uniform(-1, 1, 40), rng.uniform(0, 1, 40)])
        x_bnd = np.stack([rng.uniform(-1, 1, 12), np.zeros(12)])
    g_bnd = rng.normal(0, 0.3, x_bnd.shape[1])
    P = oracle.param_count(net)
    W = rng.normal(0, 0.4, P)
    _, dj, du = _total_loss(net, prob, W, x_int, mask, x_bnd, g_bnd)
    dW = oracle.backward(net, W, x_int, mask, dj)
    oracle.backward(net, W, x_bnd, 0x1, du[None, :], dW)
    idx = rng.choice(P, size=min(64, P), replace=False)
    h = 1e-6
    for i in idx:
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += h; Wm[i] -= h
        fd = (_total_loss(net, prob, Wp, x_int, mask, x_bnd, g_bnd)[0]
              - _total_loss(net, prob, Wm, x_int, mask, x_bnd, g_bnd)[0]) / (2 * h)
        assert dW[i] == pytest.approx(fd, rel=2e-5, abs=2e-8 * max(1.0, np.abs(dW).max()))


def test_backward_accumulate_flag():
    net = dict(widths=[2, 3, 1], G=5, k=3, m=4, lo=-1.0, hi=1.0)
    rng = np.random.default_rng(17)
    W = rng.normal(0, 0.3, oracle.param_count(net))
    x = rng.uniform(-1, 1, (2, 10))
    g = rng.normal(size=(1, 10))
    a = oracle.backward(net, W, x, 0x1, g)
    b = oracle.backward(net, W, x, 0x1, g, a.copy())
    np.testing.assert_allclose(b, 2 * a, rtol=1e-12, atol=1e-300)


# --------------------------------------------------------------------- adam


def test_adam_first_step_closed_form():
    """Step 1: the bias corrections cancel, so w1 = w0 - lr g / (|g| + eps)."""
    rng = np.random.default_rng(18)
    W0 = rng.normal(size=50)
    g = rng.normal(size=50)
    W, m1, m2 = W0.copy(), np.zeros(50), np.zeros(50)
    oracle.adam(W, g, m1, m2, 1e-2, 0.9, 0.999, 1e-8, 1)
    np.testing.assert_allclose(W, W0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14)


def test_adam_matches_torch_optim_adam_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(19)
    W0 = rng.normal(size=30)
    grads = rng.normal(size=(6, 30))
    p = torch.nn.Parameter(torch.tensor(W0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    W, m1, m2 = W0.copy(), np.zeros(30), np.zeros(30)
    for t in range(6):
        p.grad = torch.tensor(grads[t], dtype=torch.float64)
        opt.step()
        oracle.adam(W, grads[t], m1, m2, 3e-3, 0.9, 0.999, 1e-8, t + 1)
    np.testing.assert_allclose(W, p.detach().numpy(), rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------- train step


def test_train_step_equals_composition_and_loss_decreases():
    w = inputs.WORKLOADS["poisson_2_5_1"]
    d = inputs.make(w, n_int=256, n_bnd=64)
    net, prob = w.net, w.problem()
    W = d["W"].astype(np.float64)
    m1, m2 = np.zeros_like(W), np.zeros_like(W)
    loss0, dj, du = _total_loss(net, prob, W, d["x_int"], 0x1F, d["x_bnd"], d["g_bnd"])
    g = oracle.backward(net, W, d["x_int"], 0x1F, dj)
    oracle.backward(net, W, d["x_bnd"], 0x1, du[None], g)
    Wc = W.copy()
    loss, dW = oracle.train_step(net, prob, W, m1, m2, d["x_int"], 0x1F, d["x_bnd"], d["g_bnd"], 1e-2, 1)
    assert loss[0] == pytest.approx(loss0, rel=1e-14)
    np.testing.assert_allclose(dW, g, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(W, Wc - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-13)
    losses = [loss[0]]
    for t in range(2, 30):
        losses.append(oracle.train_step(net, prob, W, m1, m2, d["x_int"], 0x1F, d["x_bnd"], d["g_bnd"],
                                        1e-2, t)[0][0])
    assert losses[-1] < 0.5 * losses[0]


# ------------------------------------------------------- reduced precision


def test_rounding_matches_torch_bfloat16_and_tf32_definition():
    """BF16: round to nearest even on the top 16 bits (torch.bfloat16 does the same);
    TF32: 10 explicit mantissa bits, ties away from zero."""
    torch = pytest.importorskip("torch")
    xs = np.random.default_rng(40).standard_normal(2000) * np.exp(np.random.default_rng(41).uniform(-20, 20, 2000))
    want = torch.tensor(xs, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_to(x, oracle.BF16) for x in xs])
    np.testing.assert_array_equal(got, want)
    # TF32: exact on numbers with <= 11 significant bits, ties away from zero
    assert oracle.round_to(1.0 + 2.0 ** -10, oracle.TF32) == 1.0 + 2.0 ** -10
    assert oracle.round_to(1.0 + 2.0 ** -11, oracle.TF32) == 1.0 + 2.0 ** -10     # tie -> away
    assert oracle.round_to(-(1.0 + 2.0 ** -11), oracle.TF32) == -(1.0 + 2.0 ** -10)
    assert oracle.round_to(1.0 + 2.0 ** -12, oracle.TF32) == 1.0
    rel = np.abs([oracle.round_to(x, oracle.TF32) / np.float32(x) - 1 for x in xs])
    assert rel.max() <= 2.0 ** -11 * (1 + 1e-6)


def test_forward_rounded_exact_mode_and_rounding_effect():
    net = dict(widths=[2, 4, 4, 1], G=6, k=3, m=4, lo=-1.0, hi=1.0)
    W = np.random.default_rng(42).normal(0, 0.3, oracle.param_count(net))
    x = np.random.default_rng(43).uniform(-1, 1, (2, 50))
    exact = oracle.forward(net, W, x, 0x1F)
    np.testing.assert_array_equal(oracle.forward_rounded(net, W, x, 0x1F, set(), oracle.BF16), exact)
    bf = oracle.forward_rounded(net, W, x, 0x1F, {1}, oracle.BF16)
    tf = oracle.forward_rounded(net, W, x, 0x1F, {1}, oracle.TF32)
    e_bf = np.linalg.norm(bf[0] - exact[0]) / np.linalg.norm(exact[0])
    e_tf = np.linalg.norm(tf[0] - exact[0]) / np.linalg.norm(exact[0])
    assert 0 < e_tf < e_bf < 5e-2      # TF32 keeps 3 more bits than BF16
    # a single-layer net with weights and points that BF16 represents exactly is unaffected
    net1 = dict(widths=[1, 1], G=4, k=3, m=4, lo=-1.0, hi=1.0)
    w1 = np.array([0.5, -1.0, 2.0, 0.25, 1.5, -0.75, 1.0])
    x1 = np.array([[-0.5, 0.0, 0.5]])   # u = +-0.5, 0 inside the supports: v = (3/4)^4, 1 exactly
    np.testing.assert_array_equal(oracle.forward_rounded(net1, w1, x1, 0x1, {0}, oracle.BF16)[0],
                                  oracle.forward(net1, w1, x1, 0x1)[0])


def test_layer_forward_composes_to_the_network_forward():
    """Applying layer_forward layer by layer (from coordinate jets) equals forward."""
    net = dict(widths=[2, 4, 3, 1], G=6, k=3, m=4, lo=-1.0, hi=1.0)
    n = 9
    W = np.random.default_rng(44).normal(0, 0.4, oracle.param_count(net))
    x = np.random.default_rng(45).uniform(-1, 1, (2, 20))
    z = np.zeros((5, 2, 20))
    z[0] = x
    z[1, 0] = 1.0     # dx/dx
    z[2, 1] = 1.0     # dy/dy
    off = 0
    for l in range(3):
        I, O = net["widths"][l], net["widths"][l + 1]
        z = oracle.layer_forward(I, O, 6, 3, 4, -1.0, 1.0, W[off: off + O * I * n], z, 0x1F)
        off += O * I * n
    np.testing.assert_allclose(z[:, 0, :], oracle.forward(net, W, x, 0x1F), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("mask", [0x1F, 0x7F, 0xFF])
def test_layer_dw_matches_central_differences(mask):
    """layer_dw is the gradient of sum(gy * layer_forward) w.r.t. the layer weights: the
    layer output is linear in W, so central differences are exact up to rounding."""
    I, O, G, N = 3, 4, 5, 7
    n = G + 3
    J = oracle.n_rows(mask)
    rng = np.random.default_rng(70)
    z = rng.normal(0, 0.5, (J, I, N))
    gy = rng.normal(0, 1, (J, O, N))
    W = rng.normal(0, 0.3, O * I * n)
    dw = oracle.layer_dw(I, O, G, 3, 4, -1.0, 1.0, z, gy, mask)

    def f(Wv):
        return float((gy * oracle.layer_forward(I, O, G, 3, 4, -1.0, 1.0, Wv, z, mask)).sum())

    h = 1e-3
    for i in rng.choice(W.size, 24, replace=False):
        e = np.zeros_like(W)
        e[i] = h
        assert abs((f(W + e) - f(W - e)) / (2 * h) - dw[i]) <= 1e-9 * (1 + abs(dw[i]))


def test_layer_dw_of_last_layer_equals_network_backward():
    """For [2, I, 1], the network backward's last-layer block equals layer_dw of the hidden
    jets (layer_forward of the coordinate jets) with gy = dL/d(output jets)."""
    net = dict(widths=[2, 5, 1], G=6, k=3, m=4, lo=-1.0, hi=1.0)
    n = 9
    W = np.random.default_rng(71).normal(0, 0.4, oracle.param_count(net))
    x = np.random.default_rng(72).uniform(-1, 1, (2, 30))
    g = np.random.default_rng(73).normal(0, 1, (5, 30))
    full = oracle.backward(net, W, x, 0x1F, g)
    z = np.zeros((5, 2, 30))
    z[0] = x
    z[1, 0] = 1.0
    z[2, 1] = 1.0
    hid = oracle.layer_forward(2, 5, 6, 3, 4, -1.0, 1.0, W[: 5 * 2 * n], z, 0x1F)
    last = oracle.layer_dw(5, 1, 6, 3, 4, -1.0, 1.0, hid, g[:, None, :], 0x1F)
    np.testing.assert_allclose(last, full[5 * 2 * n:], rtol=1e-12, atol=1e-12)


def test_layer_dw_rounding_is_a_no_op_on_representable_inputs():
    """Knot inputs (cell offset 0, h = 1/8, jets +-1/2 and 0/+-2/+-4) give basis-matrix entries
    with at most 8 significant bits and gy multiples of 1/8 below 16: rounding to BF16/TF32
    changes nothing, and a value off the format's grid does change."""
    I, O, G, lo, hi = 4, 3, 16, -1.0, 1.0
    h = (hi - lo) / G
    rng = np.random.default_rng(74)
    N = 50
    z = np.zeros((5, I, N))
    z[0] = lo + rng.integers(-4, G + 4, (I, N)) * h
    z[1:3] = rng.choice([-0.5, 0.5], (2, I, N))
    z[3:5] = rng.choice([0.0, -2.0, 2.0, -4.0, 4.0], (2, I, N))
    gy = rng.integers(-127, 128, (5, O, N)) / 8.0
    exact = oracle.layer_dw(I, O, G, 3, 4, lo, hi, z, gy, 0x1F)
    for fmt in (oracle.BF16, oracle.TF32):
        np.testing.assert_array_equal(oracle.layer_dw(I, O, G, 3, 4, lo, hi, z, gy, 0x1F, fmt), exact)
    gy2 = gy.copy()
    gy2[0, 0, 0] = 1.0 + 2.0 ** -12
    assert not np.array_equal(oracle.layer_dw(I, O, G, 3, 4, lo, hi, z, gy2, 0x1F, oracle.BF16),
                              oracle.layer_dw(I, O, G, 3, 4, lo, hi, z, gy2, 0x1F))


@pytest.mark.parametrize("mask", [0x01, 0x0F, 0x1F, 0x2F, 0x7F, 0x87, 0xFF])
def test_layer_adjoint_matches_central_differences(mask):
    """layer_adjoint is the gradient of sum(gy * layer_forward(z)) w.r.t. the input jets z."""
    I, O, G, N = 3, 4, 5, 6
    n = G + 3
    J = oracle.n_rows(mask)
    rng = np.random.default_rng(80 + mask)
    z = rng.normal(0, 0.5, (J, I, N))
    gy = rng.normal(0, 1, (J, O, N))
    W = rng.normal(0, 0.3, O * I * n)
    gz = oracle.layer_adjoint(I, O, G, 3, 4, -1.0, 1.0, W, z, gy, mask)

    def f(zz):
        return float((gy * oracle.layer_forward(I, O, G, 3, 4, -1.0, 1.0, W, zz, mask)).sum())

    h = 1e-6
    for idx in [(r, j, p) for r in range(J) for j in range(I) for p in range(0, N, 2)]:
        e = np.zeros_like(z)
        e[idx] = h
        fd = (f(z + e) - f(z - e)) / (2 * h)
        assert abs(fd - gz[idx]) <= 1e-6 * (1 + abs(gz[idx])), (idx, fd, gz[idx])


def test_layer_adjoint_chains_to_the_network_backward():
    """For [2, 4, 3, 1]: the network backward's first-layer block equals layer_dw of the
    coordinate jets with gy = the layer adjoint of the last two layers chained."""
    net = dict(widths=[2, 4, 3, 1], G=6, k=3, m=4, lo=-1.0, hi=1.0)
    n = 9
    W = np.random.default_rng(81).normal(0, 0.4, oracle.param_count(net))
    x = np.random.default_rng(82).uniform(-1, 1, (2, 25))
    g = np.random.default_rng(83).normal(0, 1, (5, 25))
    full = oracle.backward(net, W, x, 0x1F, g)
    z0 = np.zeros((5, 2, 25))
    z0[0] = x
    z0[1, 0] = 1.0
    z0[2, 1] = 1.0
    W0, W1, W2 = W[:4 * 2 * n], W[4 * 2 * n: 4 * 2 * n + 3 * 4 * n], W[4 * 2 * n + 3 * 4 * n:]
    z1 = oracle.layer_forward(2, 4, 6, 3, 4, -1.0, 1.0, W0, z0, 0x1F)
    z2 = oracle.layer_forward(4, 3, 6, 3, 4, -1.0, 1.0, W1, z1, 0x1F)
    g2 = oracle.layer_adjoint(3, 1, 6, 3, 4, -1.0, 1.0, W2, z2, g[:, None, :], 0x1F)
    g1 = oracle.layer_adjoint(4, 3, 6, 3, 4, -1.0, 1.0, W1, z1, g2, 0x1F)
    first = oracle.layer_dw(2, 4, 6, 3, 4, -1.0, 1.0, z0, g1, 0x1F)
    np.testing.assert_allclose(first, full[:4 * 2 * n], rtol=1e-11, atol=1e-11)


def test_bf16_weight_split_mode():
    """ORC_BF16W2 (BF16 operands, each weight as bf16 hi + bf16 lo): (a) weights exactly
    representable in BF16 give the BF16 mode bit for bit; (b) weights with at most 16 significant
    bits are carried exactly, so the layer output is the exact weights applied to BF16-rounded
    basis-matrix entries, read out one by one with one-hot weights (the layer is linear in W)."""
    I, O, G, N = 2, 1, 4, 5
    n = G + 3
    rng = np.random.default_rng(90)
    z = rng.normal(0, 0.4, (1, I, N))
    w_bf = np.array([oracle.round_to(v, oracle.BF16) for v in rng.normal(0, 0.5, O * I * n)])
    lf = lambda W, fmt: oracle.layer_forward(I, O, G, 3, 4, -1.0, 1.0, W, z, 0x01, fmt)
    np.testing.assert_array_equal(lf(w_bf, oracle.BF16W2), lf(w_bf, oracle.BF16))
    # 16-bit weights: integers below 2^16 scaled by a power of two
    w16 = rng.integers(-(1 << 15), 1 << 15, O * I * n) / float(1 << 17)
    A = np.stack([lf(np.eye(O * I * n)[c], oracle.EXACT)[0, 0] for c in range(O * I * n)])     # [I*n][N]
    A_bf = np.vectorize(lambda v: oracle.round_to(v, oracle.BF16))(A)
    np.testing.assert_allclose(lf(w16, oracle.BF16W2)[0, 0], w16 @ A_bf, rtol=1e-14, atol=1e-15)
    assert not np.allclose(lf(w16, oracle.BF16)[0, 0], w16 @ A_bf, rtol=1e-6, atol=0)   # plain BF16 rounds W too


def test_bf16_three_term_split_mode():
    """ORC_BF16X3 (each factor as bf16 hi + bf16 lo, products hi*hi + hi*lo + lo*hi; a precision
    variant of the contraction, not from the paper).  Read out with one-hot weights (the layer is
    linear in W, so a one-hot weight of 1 returns the exact basis-matrix entries A):
    (a) entries and weights exact in BF16: the mode equals the exact layer bit for bit;
    (b) BF16-exact entries (one-hot readouts use the value row of knot inputs, 81/256, 1, 0) with
        16-bit weights, and (c) 16-bit entries with BF16-exact weights: the split carries both
        factors exactly and only the lo*lo term is dropped, which is zero here, so the output is
        exact, while one BF16 rounding of each factor is not;
    (d) general inputs: every product is within 2^-15 of its exact value relative to |a w|
        (hi + lo carries a float32 value to 2^-17; the dropped lo*lo term is below 2^-16), so
        |out - exact| <= 2^-15 sum |a| |w| per output, far inside the 2^-8 of a dropped cross term."""
    I, O, G, N = 2, 1, 4, 7
    n = G + 3
    rng = np.random.default_rng(91)
    h = 2.0 / G
    lf = lambda W, z, fmt, mask=0x01: oracle.layer_forward(I, O, G, 3, 4, -1.0, 1.0, W, z, mask, fmt)
    onehot = lambda z, mask: np.stack([lf(np.eye(O * I * n)[c], z, oracle.EXACT, mask)[:, 0]
                                       for c in range(O * I * n)])    # [I*n][J][N]
    # (a) knot inputs (value row entries 81/256, 1, 81/256, 0) and BF16 weights
    zk = (-1.0 + rng.integers(-3, G + 3, (1, I, N)) * h)
    w_bf = np.array([oracle.round_to(v, oracle.BF16) for v in rng.normal(0, 0.5, O * I * n)])
    np.testing.assert_array_equal(lf(w_bf, zk, oracle.BF16X3), lf(w_bf, zk, oracle.EXACT))
    # (b) the same entries with 16-bit weights
    w16 = rng.integers(-(1 << 15), 1 << 15, O * I * n) / float(1 << 17)
    np.testing.assert_array_equal(lf(w16, zk, oracle.BF16X3), lf(w16, zk, oracle.EXACT))
    assert not np.allclose(lf(w16, zk, oracle.BF16), lf(w16, zk, oracle.EXACT), rtol=1e-6, atol=0)
    # (c) first-derivative entries v'(z) z_d with 16 significant bits: knot inputs (v' = +-27/(8a)
    #     with a = 2h = 1, five bits) times z_d = k / 2^11 (11 bits), BF16-exact weights
    J = 3
    zc = np.zeros((J, I, N))
    zc[0] = zk[0]
    zc[1:] = rng.integers(-(1 << 11), 1 << 11, (2, I, N)) / float(1 << 11)
    A = onehot(zc, 0x07)
    assert any(oracle.round_to(a, oracle.BF16) != a for a in A[:, 1].ravel())   # entries need the lo part
    np.testing.assert_array_equal(lf(w_bf, zc, oracle.BF16X3, 0x07), lf(w_bf, zc, oracle.EXACT, 0x07))
    assert not np.allclose(lf(w_bf, zc, oracle.BF16, 0x07)[1:], lf(w_bf, zc, oracle.EXACT, 0x07)[1:],
                           rtol=1e-6, atol=0)
    # (d) general inputs and weights: the error bound
    zg = np.zeros((J, I, N))
    zg[0] = rng.uniform(-1.2, 1.2, (I, N))
    zg[1:] = rng.normal(0, 1.0, (2, I, N))
    wg = rng.normal(0, 0.5, O * I * n)
    A = onehot(zg, 0x07)                                       # [I*n][J][N]
    bound = 2.0 ** -15 * np.einsum("c,cjn->jn", np.abs(wg), np.abs(A))
    err = np.abs(lf(wg, zg, oracle.BF16X3, 0x07)[:, 0] - lf(wg, zg, oracle.EXACT, 0x07)[:, 0])
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    err1 = np.abs(lf(wg, zg, oracle.BF16, 0x07)[:, 0] - lf(wg, zg, oracle.EXACT, 0x07)[:, 0])
    assert np.any(err1 > 10 * bound)        # one BF16 rounding per factor is far outside it
