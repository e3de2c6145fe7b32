"""FP64 CPU oracle for HRKAN physics-informed training.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2409_14248_gb300``) never does.  It shares no code with the CUDA
path.  The arithmetic lives in ``hrkan_oracle.c`` (plain C, double
precision); this module only compiles it with gcc and marshals numpy arrays.

What each function follows (paper sections/equations):
  support        Section 2.1-2.2 (n = g + k bases, B-spline supports)
  hr_basis       Section 3, Eq. 2 and its derivatives (hr_basis6: up to the sixth)
  forward        KAN layer as a matrix operation (Sections 1-3) + chain-rule jets
  residual_loss  Eq. 3-4 (Poisson), Eq. 6-8 (Burgers)
  backward       reverse mode of forward (training with Adam, Section 4)
  forward_rounded  forward with the contraction inputs of chosen layers rounded
                 to BF16 / TF32 (the tensor-core variants; not from the paper)
  adam           Adam update (Section 4)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hrkan_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc_hrkan.so")
_lock = threading.Lock()
_lib = None

POISSON = 0
BURGERS = 1
KDV = 2
POISSON3 = 3   # three-input networks; the third frequency c travels in "lam"
EXACT, BF16, TF32, BF16W2 = 0, 1, 2, 3   # BF16W2: BF16 operands, weights as bf16 hi + lo
BF16X3 = 4   # both factors as bf16 hi + lo, products hi*hi + hi*lo + lo*hi


def build(force: bool = False) -> str:
    """Compile hrkan_oracle.c into liborc_hrkan.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_support.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
            lib.orc_hr_basis.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
            lib.orc_hr_basis6.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
            lib.orc_param_count.argtypes = [ctypes.c_int, _ip, ctypes.c_int, ctypes.c_int]
            lib.orc_param_count.restype = ctypes.c_long
            net = [ctypes.c_int, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.orc_forward.argtypes = net + [_dp, _dp, ctypes.c_long, ctypes.c_uint, _dp]
            lib.orc_forward_rounded.argtypes = net + [_dp, _dp, ctypes.c_long, ctypes.c_uint, _dp, ctypes.c_uint,
                                                      ctypes.c_int]
            lib.orc_layer_forward.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double] * 2 + [_dp, _dp, ctypes.c_long,
                                                                                        ctypes.c_uint, _dp,
                                                                                        ctypes.c_int]
            lib.orc_layer_dw.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double] * 2 + [_dp, _dp, ctypes.c_long,
                                                                                   ctypes.c_uint, _dp, ctypes.c_int]
            lib.orc_layer_adjoint.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double] * 2 + [_dp, _dp, _dp,
                                                                                        ctypes.c_long, ctypes.c_uint,
                                                                                        _dp, ctypes.c_int]
            lib.orc_round.argtypes = [ctypes.c_double, ctypes.c_int]
            lib.orc_round.restype = ctypes.c_double
            lib.orc_backward.argtypes = net + [_dp, _dp, ctypes.c_long, ctypes.c_uint, _dp, _dp, ctypes.c_int]
            prob = [ctypes.c_int] + [ctypes.c_double] * 5
            lib.orc_residual_loss.argtypes = prob + [_dp, ctypes.c_long, ctypes.c_uint, _dp, _dp, _dp,
                                                     ctypes.c_long, _dp, _dp, _dp]
            lib.orc_adam.argtypes = [ctypes.c_long, _dp, _dp, _dp, _dp] + [ctypes.c_double] * 4 + [ctypes.c_int]
            lib.orc_train_step.argtypes = (net + prob + [_dp, _dp, _dp, _dp, ctypes.c_long, ctypes.c_uint, _dp, _dp,
                                                         ctypes.c_long] + [ctypes.c_double] * 4
                                           + [ctypes.c_int, _dp, _dp])
            _lib = lib
    return _lib


def _d(a):
    """Contiguous float64 copy/view and its pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _net_args(net):
    w = np.ascontiguousarray(net["widths"], dtype=np.int32)
    return w, [len(w), w.ctypes.data_as(_ip), int(net["G"]), int(net["k"]), int(net["m"]),
               float(net["lo"]), float(net["hi"])]


def support(G, k, lo, hi):
    """(s, e) arrays of the n = G + k basis supports."""
    lib = _load()
    s = np.zeros(G + k)
    e = np.zeros(G + k)
    lib.orc_support(G, k, lo, hi, s.ctypes.data_as(_dp), e.ctypes.data_as(_dp))
    return s, e


def hr_basis(m, s, e, x):
    """Value and first to fourth derivatives of the order-m HR basis on [s, e] at x (Eq. 2)."""
    lib = _load()
    out = np.zeros(5)
    lib.orc_hr_basis(int(m), float(s), float(e), float(x), out.ctypes.data_as(_dp))
    return out


def hr_basis6(m, s, e, x):
    """Value and first to sixth derivatives of the order-m HR basis on [s, e] at x (Eq. 2, from its
    expansion in the support coordinate)."""
    lib = _load()
    out = np.zeros(7)
    lib.orc_hr_basis6(int(m), float(s), float(e), float(x), out.ctypes.data_as(_dp))
    return out


def param_count(net):
    lib = _load()
    w, args = _net_args(net)
    return int(lib.orc_param_count(args[0], args[1], args[2], args[3]))


def n_rows(mask, D=2):
    """Rows a mask selects: D = 2 has 12 jet bits (u, three orders of pure derivatives, the mixed
    u_x0x1, then the fourth and fifth orders), D = 3 has 16 (u and five orders)."""
    return bin(int(mask) & ((1 << (12 if D == 2 else 1 + 5 * D)) - 1)).count("1")


def forward(net, W, x, mask):
    """jets[J, N] at points x[D, N] for the rows selected by mask."""
    lib = _load()
    w, args = _net_args(net)
    W, Wp = _d(W)
    x, xp = _d(x)
    N = x.shape[1]
    jets = np.zeros((n_rows(mask, x.shape[0]), N))
    rc = lib.orc_forward(*args, Wp, xp, N, int(mask), jets.ctypes.data_as(_dp))
    if rc:
        raise ValueError("orc_forward: bad arguments")
    return jets


def round_to(x, fmt):
    """x rounded to float32 and then to BF16 (nearest even) or TF32 (nearest, ties away)."""
    return _load().orc_round(float(x), int(fmt))


def forward_rounded(net, W, x, mask, round_layers, fmt):
    """forward() with the basis-matrix entries and weights of the layers in
    round_layers (a set of layer indices) rounded to fmt before each product;
    accumulation stays in float64 (the tensor cores accumulate in FP32)."""
    lib = _load()
    w, args = _net_args(net)
    W, Wp = _d(W)
    x, xp = _d(x)
    N = x.shape[1]
    jets = np.zeros((n_rows(mask, x.shape[0]), N))
    bits = sum(1 << int(l) for l in round_layers)
    rc = lib.orc_forward_rounded(*args, Wp, xp, N, int(mask), jets.ctypes.data_as(_dp), bits, int(fmt))
    if rc:
        raise ValueError("orc_forward_rounded: bad arguments")
    return jets


def layer_forward(I, O, G, k, m, lo, hi, Wl, zin, mask, fmt=EXACT):
    """One KAN layer on given input jets zin[J, I, N] (rows of mask) -> [J, O, N]."""
    lib = _load()
    Wl, Wp = _d(Wl)
    z, zp = _d(zin)
    J, _, N = z.shape
    out = np.zeros((J, O, N))
    rc = lib.orc_layer_forward(int(I), int(O), int(G), int(k), int(m), float(lo), float(hi), Wp, zp, N, int(mask),
                               out.ctypes.data_as(_dp), int(fmt))
    if rc:
        raise ValueError("orc_layer_forward: bad arguments")
    return out


def layer_dw(I, O, G, k, m, lo, hi, zin, gy, mask, fmt=EXACT):
    """Weight gradient [O*I*n] of one KAN layer for input jets zin[J, I, N] and
    output-jet gradients gy[J, O, N]; fmt rounds the basis-matrix entries and gy."""
    lib = _load()
    z, zp = _d(zin)
    g, gp = _d(gy)
    J, _, N = z.shape
    out = np.zeros(O * I * (G + k))
    rc = lib.orc_layer_dw(int(I), int(O), int(G), int(k), int(m), float(lo), float(hi), zp, gp, N, int(mask),
                          out.ctypes.data_as(_dp), int(fmt))
    if rc:
        raise ValueError("orc_layer_dw: bad arguments")
    return out


def layer_adjoint(I, O, G, k, m, lo, hi, Wl, zin, gy, mask, fmt=EXACT):
    """dL/d(input jets) [J, I, N] of one KAN layer for output-jet gradients gy[J, O, N];
    fmt rounds gy and the weights."""
    lib = _load()
    Wl, Wp = _d(Wl)
    z, zp = _d(zin)
    g, gp = _d(gy)
    J, _, N = z.shape
    out = np.zeros((J, I, N))
    rc = lib.orc_layer_adjoint(int(I), int(O), int(G), int(k), int(m), float(lo), float(hi), Wp, zp, gp, N,
                               int(mask), out.ctypes.data_as(_dp), int(fmt))
    if rc:
        raise ValueError("orc_layer_adjoint: bad arguments")
    return out


def backward(net, W, x, mask, dL_djets, dW=None):
    """dW of sum(dL_djets * jets); accumulates into dW when it is given."""
    lib = _load()
    w, args = _net_args(net)
    W, Wp = _d(W)
    x, xp = _d(x)
    g, gp = _d(dL_djets)
    acc = dW is not None
    if dW is None:
        dW = np.zeros(param_count(net))
    assert dW.dtype == np.float64 and dW.flags.c_contiguous
    rc = lib.orc_backward(*args, Wp, xp, x.shape[1], int(mask), gp, dW.ctypes.data_as(_dp), int(acc))
    if rc:
        raise ValueError("orc_backward: bad arguments")
    return dW


def _prob_args(prob):
    return [int(prob["kind"]), float(prob.get("a", 1.0)), float(prob.get("b", 1.0)),
            float(prob.get("lam", 1.0)), float(prob.get("nu", 0.0)), float(prob.get("alpha", 1.0))]


def residual_loss(prob, x_int, mask, jets_int, u_bnd, g_bnd):
    """(loss[3] = [L, L_pde, L_bnd], dL_djets_int[J, N_int], dL_du_bnd[N_bnd])."""
    lib = _load()
    x, xp = _d(x_int)
    j, jp = _d(jets_int)
    ub, ubp = _d(u_bnd)
    gb, gbp = _d(g_bnd)
    loss = np.zeros(3)
    dj = np.zeros_like(j)
    du = np.zeros_like(ub)
    rc = lib.orc_residual_loss(*_prob_args(prob), xp, x.shape[1], int(mask), jp, ubp, gbp, ub.shape[0],
                               loss.ctypes.data_as(_dp), dj.ctypes.data_as(_dp), du.ctypes.data_as(_dp))
    if rc:
        raise ValueError("orc_residual_loss: bad arguments")
    return loss, dj, du


def adam(W, g, m1, m2, lr, b1, b2, eps, t):
    """In-place Adam on float64 arrays W, m1, m2."""
    lib = _load()
    for a in (W, m1, m2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g, gp = _d(g)
    lib.orc_adam(W.size, W.ctypes.data_as(_dp), gp, m1.ctypes.data_as(_dp), m2.ctypes.data_as(_dp),
                 lr, b1, b2, eps, int(t))


def train_step(net, prob, W, m1, m2, x_int, mask_int, x_bnd, g_bnd, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One full-batch step in place on float64 W, m1, m2; returns (loss[3], dW)."""
    lib = _load()
    w, args = _net_args(net)
    for a in (W, m1, m2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    xi, xip = _d(x_int)
    xb, xbp = _d(x_bnd)
    gb, gbp = _d(g_bnd)
    loss = np.zeros(3)
    dW = np.zeros_like(W)
    rc = lib.orc_train_step(*args, *_prob_args(prob), W.ctypes.data_as(_dp), m1.ctypes.data_as(_dp),
                            m2.ctypes.data_as(_dp), xip, xi.shape[1], int(mask_int), xbp, gbp, xb.shape[1],
                            lr, b1, b2, eps, int(t), loss.ctypes.data_as(_dp), dW.ctypes.data_as(_dp))
    if rc:
        raise ValueError("orc_train_step: bad arguments")
    return loss, dW
