"""Reference solutions of the PDEs the workloads and experiments train on.

These are the ground truth for test errors (the quantity the paper reports
in Tables 1 and 2), evaluated in float64 numpy.  They are not a step of the
training path, which runs entirely in libhrkan.so.

Poisson (Section 4.1, Eq. 3): u* = sin(a pi x) sin(b pi y).

Viscous Burgers u_t + u u_x = nu u_xx (Section 4.2, Eq. 6): the Cole-Hopf
substitution u = -2 nu (log phi)_x turns it into the heat equation for phi,
with phi(s, 0) = exp(-F(s) / (2 nu)) and F an antiderivative of the initial
profile u0.  Averaging over the heat kernel gives, on the whole line,

    u(x, t)   = <d> / t,
    u_x(x, t) = 1 / t - Var(d) / (2 nu t^2),

where d = x - s and <.> is the average over s with weights exp(-E(s)),
E(s) = F(s) / (2 nu) + d^2 / (4 nu t).  E is smallest where s + t u0(s) = x
(the characteristic through x), so with |u0| <= 1 the weights live on
[x - t, x + t] widened by 12 sigma, sigma = sqrt(2 nu t), on each side
(beyond that they are below exp(-70)).  The average is a sum over equally
spaced nodes, shifted by min E so that nothing underflows.

Two initial profiles are used:
* u0 = sech(x) (the experiment of Section 4.2), F(s) = atan(sinh s);
* u0 = -sin(pi x) on [-1, 1] (the Burgers workloads), F(s) = (cos(pi s) - 1)/pi.
  That solution is odd and 2-periodic, so it vanishes at x = +-1 for all t and
  the whole-line formula is the exact solution of the Dirichlet problem.
"""
from __future__ import annotations

import math

import numpy as np


def poisson(x, y, a: float = 1.0, b: float = 1.0):
    """u* = sin(a pi x) sin(b pi y)."""
    return np.sin(a * np.pi * np.asarray(x, np.float64)) * np.sin(b * np.pi * np.asarray(y, np.float64))


def _cole_hopf(x, t, nu, F, u0, nodes, slope):
    x, t = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(t, np.float64))
    u = u0(x)
    ux = np.full(x.shape, np.nan) if slope else None
    pos = t > 0
    xs, ts = x[pos], t[pos]
    sig = np.sqrt(2.0 * nu * ts)
    lo, hi = xs - ts - 12.0 * sig, xs + ts + 12.0 * sig
    frac = np.linspace(0.0, 1.0, nodes)
    mean = np.empty(xs.size)
    var = np.empty(xs.size)
    chunk = max(1, (1 << 22) // nodes)
    for a in range(0, xs.size, chunk):
        sl = slice(a, a + chunk)
        s = lo[sl, None] + (hi[sl] - lo[sl])[:, None] * frac[None, :]
        d = xs[sl, None] - s
        E = F(s) / (2.0 * nu) + d * d / (4.0 * nu * ts[sl, None])
        w = np.exp(-(E - E.min(axis=1, keepdims=True)))
        w /= w.sum(axis=1, keepdims=True)
        mean[sl] = (w * d).sum(axis=1)
        var[sl] = (w * (d - mean[sl, None]) ** 2).sum(axis=1)
    u[pos] = mean / ts
    if slope:
        ux[pos] = 1.0 / ts - var / (2.0 * nu * ts * ts)
        return u, ux
    return u


def burgers_sech(x, t, nu: float = 1e-3, nodes: int = 3001, slope: bool = False):
    """Whole-line Burgers solution with u(x, 0) = sech(x) (and u_x if slope; nan at t = 0)."""
    return _cole_hopf(x, t, nu, lambda s: np.arctan(np.sinh(s)), lambda s: 1.0 / np.cosh(s), nodes, slope)


def burgers_sine(x, t, nu: float = 0.01 / math.pi, nodes: int = 3001, slope: bool = False):
    """Burgers solution on [-1, 1] with u(x, 0) = -sin(pi x), u(+-1, t) = 0 (and u_x if slope)."""
    return _cole_hopf(x, t, nu, lambda s: (np.cos(np.pi * s) - 1.0) / np.pi, lambda s: -np.sin(np.pi * s), nodes,
                      slope)
