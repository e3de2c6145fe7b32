"""Pins of the oracle's fourth- and fifth-derivative jets (Section 3 motivates
the HR order m by the derivative order a PDE needs and picks m = 6 for a fifth
derivative).  Mask bits, D = 2: 8 + d the fourth and 10 + d the fifth
derivative along input d; D = 3: 10 + d and 13 + d.

What pins them, none of it sharing code with the oracle: numpy's polynomial
derivatives of Eq. 2 (the basis up to its sixth derivative), sympy
differentiation of the network's polynomial pieces, central differences of
the oracle's own lower-order rows, and central differences of the loss in the
weights and in a layer's input jets (the backward, through the basis's sixth
derivative)."""
import numpy as np
import pytest

import oracle

ALL2 = 0xFFF      # D = 2: u, orders 1-3, mixed, orders 4-5 (12 rows)
ALL3 = 0xFFFF     # D = 3: u, orders 1-5 (16 rows)


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6])
def test_basis_derivatives_to_sixth_order_match_the_polynomial(m):
    """Inside (s, e) Eq. 2 is c_m ((e-x)(x-s))^m; numpy expands and differentiates it six times."""
    s, e = -0.6, 0.9
    c = (2.0 / (e - s)) ** (2 * m)
    P = c * np.polynomial.Polynomial([-e * s, e + s, -1.0]) ** m
    ders = [P.deriv(r) if r else P for r in range(7)]
    scale = np.array([np.abs(d(np.linspace(s, e, 401))).max() + 1e-300 for d in ders])
    for x in np.random.default_rng(m).uniform(s + 1e-3, e - 1e-3, 30):
        got = oracle.hr_basis6(m, s, e, x)
        want = np.array([d(x) for d in ders])
        assert np.all(np.abs(got - want) <= 1e-11 * scale), (x, got, want)
        np.testing.assert_allclose(got[:5], oracle.hr_basis(m, s, e, x), rtol=1e-12, atol=1e-12 * scale.max())
    for x in (s - 0.1, s, e, e + 0.3):
        assert np.all(oracle.hr_basis6(m, s, e, x) == 0.0)
    # (1-u^2)^m has degree 2m: the (2m+1)-th derivative and beyond vanish, the 2m-th is constant
    if 2 * m <= 6:
        x = np.random.default_rng(9).uniform(s, e, 5)
        top = [oracle.hr_basis6(m, s, e, xx)[2 * m] for xx in x]
        np.testing.assert_allclose(top, top[0], rtol=1e-12)
        assert all(np.all(oracle.hr_basis6(m, s, e, xx)[2 * m + 1:] == 0.0) for xx in x)


def _sympy_net(widths, G, m, W, point):
    """The network as a sympy expression in the inputs near `point` (each basis of Eq. 2 as its
    polynomial piece where its ReLUs are active at the point)."""
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x0:%d" % widths[0], real=True)
    lo, hi, k = -1.0, 1.0, 3
    h, n = (hi - lo) / G, G + k
    z, zn, off = list(X), [float(v) for v in point], 0
    for l in range(len(widths) - 1):
        I, O = widths[l], widths[l + 1]
        Wl = W[off: off + O * I * n].reshape(O, I, n)
        off += O * I * n
        out, outn = [], []
        for o in range(O):
            expr, val = 0, 0.0
            for j in range(I):
                for i in range(n):
                    s, e = lo + (i - k) * h, lo + (i + 1) * h
                    if s < zn[j] < e:
                        c = (2.0 / (e - s)) ** (2 * m)
                        expr += float(Wl[o, j, i]) * c * ((e - z[j]) * (z[j] - s)) ** m
                        val += float(Wl[o, j, i]) * c * ((e - zn[j]) * (zn[j] - s)) ** m
            out.append(sp.expand(expr) if l == 0 else expr)
            outn.append(val)
        z, zn = out, outn
    return X, z[0]


def test_fourth_and_fifth_order_jets_match_symbolic_differentiation():
    """m = 6, the order Section 3 picks for a fifth derivative, on a [2,1,1] net (its hidden unit
    depends on both inputs, so the fifth derivatives run through the composition of two layers);
    one point, as sympy differentiates the degree-144 composition five times."""
    sp = pytest.importorskip("sympy")
    m = 6
    net = dict(widths=[2, 1, 1], G=5, k=3, m=m, lo=-1.0, hi=1.0)
    W = np.random.default_rng(50 + m).normal(0, 0.5, oracle.param_count(net))
    x = np.random.default_rng(51).uniform(-1, 1, (2, 1))
    jets = oracle.forward(net, W, x, 0xF00 | 0x01)     # u, u_x0^(4), u_x1^(4), u_x0^(5), u_x1^(5)
    for p in range(1):
        X, u = _sympy_net(net["widths"], 5, m, W, x[:, p])
        exprs = [u, sp.diff(u, X[0], 4), sp.diff(u, X[1], 4), sp.diff(u, X[0], 5), sp.diff(u, X[1], 5)]
        sub = {X[0]: x[0, p], X[1]: x[1, p]}
        want = np.array([float(e.evalf(subs=sub)) for e in exprs])
        scale = np.abs(want).max()
        np.testing.assert_allclose(jets[:, p], want, rtol=1e-7, atol=1e-9 * scale)


@pytest.mark.parametrize("widths,mask,lower,higher", [
    ([2, 4, 3, 1], ALL2, [5, 6, 8, 9], [8, 9, 10, 11]),            # D = 2: bit 8+d from 5+d, 10+d from 8+d
    ([3, 4, 1], ALL3, [7, 8, 9, 10, 11, 12], [10, 11, 12, 13, 14, 15]),
])
def test_each_order_is_the_derivative_of_the_one_below(widths, mask, lower, higher):
    """Central differences of the oracle's own order-(r-1) rows give its order-r rows."""
    D = widths[0]
    net = dict(widths=widths, G=6, k=3, m=6, lo=-1.0, hi=1.0)
    W = np.random.default_rng(52 + D).normal(0, 0.3, oracle.param_count(net))
    x = np.random.default_rng(53).uniform(-0.9, 0.9, (D, 12))
    row = lambda bit: bin(mask & ((1 << bit) - 1)).count("1")
    jets = oracle.forward(net, W, x, mask)
    h = 1e-5
    for lo_bit, hi_bit in zip(lower, higher):
        d = (hi_bit - (8 if D == 2 else 10)) % D
        e = np.zeros((D, 1))
        e[d] = 1.0
        f = lambda xx: oracle.forward(net, W, xx, mask)[row(lo_bit)]
        fd = (f(x + h * e) - f(x - h * e)) / (2 * h)
        got = jets[row(hi_bit)]
        np.testing.assert_allclose(got, fd, rtol=2e-5, atol=2e-6 * np.abs(fd).max())


def test_higher_rows_leave_the_other_rows_unchanged():
    """Bits 8-11 append rows: every lower row is bit for bit the one of the smaller mask."""
    net = dict(widths=[2, 3, 2, 1], G=5, k=3, m=6, lo=-1.0, hi=1.0)
    W = np.random.default_rng(54).normal(0, 0.3, oracle.param_count(net))
    x = np.random.default_rng(55).uniform(-1, 1, (2, 9))
    full = oracle.forward(net, W, x, ALL2)
    np.testing.assert_array_equal(oracle.forward(net, W, x, 0xFF), full[:8])
    np.testing.assert_array_equal(oracle.forward(net, W, x, 0x12F), full[[0, 1, 2, 3, 5, 8]])
    net3 = dict(widths=[3, 3, 1], G=5, k=3, m=6, lo=-1.0, hi=1.0)
    W3 = np.random.default_rng(56).normal(0, 0.3, oracle.param_count(net3))
    x3 = np.random.default_rng(57).uniform(-1, 1, (3, 9))
    full3 = oracle.forward(net3, W3, x3, ALL3)
    np.testing.assert_array_equal(oracle.forward(net3, W3, x3, 0x3FF), full3[:10])


@pytest.mark.parametrize("widths,mask", [([2, 3, 3, 1], ALL2), ([2, 3, 1], 0xC01), ([3, 3, 1], ALL3)])
def test_weight_gradient_through_the_higher_rows_matches_central_differences(widths, mask):
    """Backward through the fourth and fifth rows (the basis's sixth derivative) vs central FD of
    L(W) = sum(R * jets)."""
    D = widths[0]
    net = dict(widths=widths, G=5, k=3, m=6, lo=-1.0, hi=1.0)
    rng = np.random.default_rng(58 + mask % 97)
    W = rng.normal(0, 0.4, oracle.param_count(net))
    x = rng.uniform(-1, 1, (D, 15))
    J = oracle.n_rows(mask, D)
    R = rng.normal(0, 1, (J, 15))
    dW = oracle.backward(net, W, x, mask, R)
    loss = lambda Wv: float((R * oracle.forward(net, Wv, x, mask)).sum())
    h = 1e-6
    for i in rng.choice(W.size, min(40, W.size), replace=False):
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += h
        Wm[i] -= h
        fd = (loss(Wp) - loss(Wm)) / (2 * h)
        assert dW[i] == pytest.approx(fd, rel=5e-5, abs=5e-8 * max(1.0, np.abs(dW).max()))


def test_layer_forward_composes_to_the_network_forward_with_all_rows():
    net = dict(widths=[2, 4, 3, 1], G=6, k=3, m=6, lo=-1.0, hi=1.0)
    n = 9
    W = np.random.default_rng(59).normal(0, 0.4, oracle.param_count(net))
    x = np.random.default_rng(60).uniform(-1, 1, (2, 10))
    z = np.zeros((12, 2, 10))
    z[0] = x
    z[1, 0] = 1.0
    z[2, 1] = 1.0
    off = 0
    for l in range(3):
        I, O = net["widths"][l], net["widths"][l + 1]
        z = oracle.layer_forward(I, O, 6, 3, 6, -1.0, 1.0, W[off: off + O * I * n], z, ALL2)
        off += O * I * n
    want = oracle.forward(net, W, x, ALL2)
    np.testing.assert_allclose(z[:, 0, :], want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("mask", [0x3FF, ALL2])
def test_layer_dw_and_adjoint_with_higher_rows_match_central_differences(mask):
    I, O, G, N, m = 3, 4, 5, 5, 6
    n = G + 3
    J = oracle.n_rows(mask)
    rng = np.random.default_rng(61 + mask % 89)
    z = rng.normal(0, 0.5, (J, I, N))
    gy = rng.normal(0, 1, (J, O, N))
    W = rng.normal(0, 0.3, O * I * n)
    f = lambda Wv, zz: float((gy * oracle.layer_forward(I, O, G, 3, m, -1.0, 1.0, Wv, zz, mask)).sum())
    dw = oracle.layer_dw(I, O, G, 3, m, -1.0, 1.0, z, gy, mask)
    h = 1e-3      # the output is linear in W
    for i in rng.choice(W.size, 20, replace=False):
        e = np.zeros_like(W)
        e[i] = h
        assert abs((f(W + e, z) - f(W - e, z)) / (2 * h) - dw[i]) <= 1e-8 * (1 + abs(dw[i]))
    gz = oracle.layer_adjoint(I, O, G, 3, m, -1.0, 1.0, W, z, gy, mask)
    # |f| reaches 4e4 with the fifth-order rows, so the rounding noise eps |f| / h of a smaller
    # step would exceed the bar; h = 1e-5 keeps both it and the truncation error below 1e-6
    h = 1e-5
    for idx in [(r, j, p) for r in range(J) for j in range(I) for p in (0, 3)]:
        e = np.zeros_like(z)
        e[idx] = h
        fd = (f(W, z + e) - f(W, z - e)) / (2 * h)
        assert abs(fd - gz[idx]) <= 2e-6 * (1 + abs(gz[idx])), (idx, fd, gz[idx])
