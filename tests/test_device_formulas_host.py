"""The kernels' basis and jet-row formulas (csrc/hr_device.cuh), compiled for
the host by nvcc and run on the CPU, against the FP64 oracle.

tests/device_host/hr_device_host.cu prints, in float32:
* B lines: the k + 1 active bases of Active<3, m, 6> (v and its first six
  derivatives) for m = 2..6 at points across and beyond the grid;
* W lines: the same reverse taken one jet row of dA at a time (Jet::row_adjoint, the
  tensor-core adjoint's form) for masks 0x1F, 0x0F (m = 4), 0x07 (m = 3) and 0x01;
* R lines: the basis-matrix rows of one input unit (Jet<mask>::rows_b) and
  their reverse (adjoint_b) for masks 0x1F, 0x0F, 0xFF (m = 4 and 6), 0x2F
  (m = 3), 0x12F (fourth derivative along x0, m = 5), 0x52F (fourth and fifth,
  m = 6), 0x3FF (fourth along both inputs, m = 4) and 0xFFF (every row, m = 6),
  with given jets and a rank-1 dA = gy[r] w[i].

The oracle gives the same quantities: hr_basis / hr_basis6 for the bases (a
term-by-term expansion of (1 - u^2)^m, where the kernels use powers of
1 - u^2), a one-input,
one-output oracle layer with one-hot weights for each row entry, and its
input adjoint for the reverse.  At a support end the derivatives of order >= m
jump (the kernels take the limit from inside, the oracle takes 0), so those
orders are compared only away from the knots."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2409_14248_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G, K, LO, HI = 6, 3, -1.0, 1.0
H = (HI - LO) / G
KNOTS = LO + H * np.arange(-K, G + K + 1)
ZR = [0.0, 0.7, -1.3, 0.45, -0.8, 2.1, -0.6, 0.35, -1.7, 0.9, 2.4, -0.55]
GY = [0.9, -0.4, 1.7, 0.25, -1.1, 0.6, 1.3, -0.75, 0.5, -0.95, 0.3, 1.15]
NDER = 6


def wv(i):
    return np.float32(0.5 - 0.17 * i + 0.03 * i * i)


def near_knot(z):
    return np.abs(KNOTS - z).min() < 1e-5


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not installed")
    exe = str(tmp_path_factory.mktemp("hdh") / "hr_device_host")
    src = os.path.join(ROOT, "tests", "device_host", "hr_device_host.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", *build.ARCH, src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0
    return [ln.split() for ln in out.stdout.splitlines()]


def test_basis_values_and_derivatives_match_the_oracle(lines):
    s, e = oracle.support(G, K, LO, HI)
    blines = [ln for ln in lines if ln[0] == "B"]
    assert len(blines) == 5 * 15
    for m in range(2, 7):
        rows = [ln for ln in blines if int(ln[1]) == m]
        got_all, want_all, keep_all = [], [], []
        for ln in rows:
            z, c = float(ln[2]), int(ln[3])
            vals = np.array(ln[4:], dtype=np.float64).reshape(NDER + 1, K + 1)     # [order][q]
            for q in range(K + 1):
                i = c + q
                if not 0 <= i < G + K:
                    assert np.all(vals[:, q] == 0.0)
                    continue
                want = np.concatenate([oracle.hr_basis(m, s[i], e[i], z), oracle.hr_basis6(m, s[i], e[i], z)[5:]])
                keep = np.array([r < m or not near_knot(z) for r in range(NDER + 1)])
                got_all.append(vals[:, q]); want_all.append(want); keep_all.append(keep)
        got, want, keep = np.array(got_all), np.array(want_all), np.array(keep_all)
        for r in range(NDER + 1):
            scale = np.abs(want[:, r]).max()
            if scale == 0.0:                       # derivatives above 2m vanish
                assert np.all(got[:, r] == 0.0), (m, r)
                continue
            err = np.abs(got[keep[:, r], r] - want[keep[:, r], r]).max()
            assert err <= 2e-5 * scale, (m, r, err, scale)


def _tol(z):
    """float32 evaluation error of the kernels' formulas: 2e-5 of the row scale, and near a support
    end the resolution of z itself, ulp(z) over the distance to the end (Q = 1 - u^2 is that small)."""
    d = np.abs(KNOTS - z).min()
    return max(2e-5, 4.0 * np.spacing(np.float32(z)) / max(d, 1e-12))


def test_jet_rows_and_their_reverse_match_the_oracle(lines):
    rlines = [ln for ln in lines if ln[0] == "R"]
    assert len(rlines) == 9 * 15
    n = G + K
    for ln in rlines:
        mask, m, z0, c = int(ln[1]), int(ln[2]), float(ln[3]), int(ln[4])
        bits = [b for b in range(12) if mask >> b & 1]
        J = len(bits)
        A = np.array(ln[5: 5 + J * (K + 1)], dtype=np.float64).reshape(J, K + 1)
        gz = np.array(ln[5 + J * (K + 1): 5 + J * (K + 1) + J], dtype=np.float64)
        order = {0: 0, 1: 1, 2: 1, 3: 2, 4: 2, 7: 2, 5: 3, 6: 3, 8: 4, 9: 4, 10: 5, 11: 5}
        max_order = 1 + max(order[b] for b in bits)   # the reverse needs one more basis derivative
        if max_order >= m and near_knot(z0):
            continue
        zin = np.array([[[z0 if b == 0 else ZR[b]]] for b in bits], dtype=np.float64)     # [J][1][1]
        zin = zin.astype(np.float32).astype(np.float64)
        tol = _tol(z0)
        for q in range(K + 1):
            i = c + q
            if not 0 <= i < n:
                continue
            onehot = np.zeros(n)
            onehot[i] = 1.0
            want = oracle.layer_forward(1, 1, G, K, m, LO, HI, onehot, zin, mask)[:, 0, 0]
            scale = max(1.0, np.abs(want).max())
            assert np.abs(A[:, q] - want).max() <= tol * scale, (mask, m, z0, q, A[:, q], want)
        w = np.array([wv(i) for i in range(n)], dtype=np.float64)
        gy = np.array([[[np.float32(GY[r])]] for r in range(J)], dtype=np.float64)
        want = oracle.layer_adjoint(1, 1, G, K, m, LO, HI, w, zin, gy, mask)[:, 0, 0]
        scale = max(1.0, np.abs(want).max())
        assert np.abs(gz - want).max() <= tol * scale, (mask, m, z0, gz, want)



def test_residuals_and_their_jet_gradients_match_the_oracle(lines):
    """P lines: the kernels' residual r and gu = dL/d(jets) of one point (L = alpha r^2, so gu is
    the oracle's dL_djets for a one-point set) for Poisson (Eq. 3), Burgers (Eq. 6) and the KdV
    residual, on the residual's own mask and on wider ones.  The oracle's gradient of the
    residual's first row (u_xx for Poisson, u_t otherwise) is 2 alpha r, which gives its r."""
    plines = [ln for ln in lines if ln[0] == "P"]
    assert len(plines) == 6 * 5
    alpha = 0.5
    for ln in plines:
        kind, mask = int(ln[1]), int(ln[2])
        x0, x1, u0, r = (float(v) for v in ln[3:7])
        bits = [b for b in range(12) if mask >> b & 1]
        gu = np.array(ln[7:], dtype=np.float64)
        assert gu.size == len(bits)
        jets = np.array([[u0 if b == 0 else float(np.float32(ZR[b]))] for b in bits])
        prob = dict(kind=kind, a=2.0, b=3.0, lam=1.0 if kind == 1 else 6.0,
                    nu=0.01 / np.pi if kind == 1 else 1.0, alpha=alpha)
        _, dj, _ = oracle.residual_loss(prob, np.array([[x0], [x1]]), mask, jets, np.zeros(0), np.zeros(0))
        dj = dj[:, 0]
        first = bits.index(3 if kind == 0 else 2)
        r_want = dj[first] / (2.0 * alpha)
        # float32 evaluation: a few ulps of the residual's largest term
        terms = np.abs(jets[:, 0]).max() * max(1.0, prob["lam"] * np.abs(jets[:, 0]).max(), prob["nu"])
        scale = terms + (13.0 * np.pi ** 2 if kind == 0 else 0.0)
        assert abs(r - r_want) <= 2e-6 * scale, (kind, mask, r, r_want)
        dr = np.abs(dj) / (2.0 * alpha * max(abs(r_want), 1e-30))      # |dr/d jet row|
        tol = 2.0 * alpha * (2e-6 * scale * dr + 2e-6 * abs(r_want) * dr) + 1e-30
        assert np.all(np.abs(gu - dj) <= tol), (kind, mask, gu, dj)
        assert np.all((gu == 0.0) == (dj == 0.0)), (kind, mask, gu, dj)


def test_row_by_row_reverse_matches_the_oracle(lines):
    """The reverse of the jet rows summed one row of dA at a time (as the tensor-core input
    adjoint applies it, no row kept) equals the oracle's input adjoint of the same one-unit
    layer, and the kernels' all-rows reverse (R lines) to float32 rounding."""
    wlines = [ln for ln in lines if ln[0] == "W"]
    assert len(wlines) == 4 * 15
    rl = {(int(ln[1]), int(ln[2]), ln[3]): ln for ln in lines if ln[0] == "R"}
    n = G + K
    seen_r = 0
    for ln in wlines:
        mask, m, z0, c = int(ln[1]), int(ln[2]), float(ln[3]), int(ln[4])
        bits = [b for b in range(12) if mask >> b & 1]
        J = len(bits)
        gz = np.array(ln[5: 5 + J], dtype=np.float64)
        assert gz.size == J
        order = {0: 0, 1: 1, 2: 1, 3: 2, 4: 2}
        if 1 + max(order[b] for b in bits) >= m and near_knot(z0):
            continue
        zin = np.array([[[z0 if b == 0 else ZR[b]]] for b in bits], dtype=np.float64)
        zin = zin.astype(np.float32).astype(np.float64)
        w = np.array([wv(i) for i in range(n)], dtype=np.float64)
        gy = np.array([[[np.float32(GY[r])]] for r in range(J)], dtype=np.float64)
        want = oracle.layer_adjoint(1, 1, G, K, m, LO, HI, w, zin, gy, mask)[:, 0, 0]
        scale = max(1.0, np.abs(want).max())
        assert np.abs(gz - want).max() <= _tol(z0) * scale, (mask, m, z0, gz, want)
        key = (mask, m, ln[3])
        if key in rl:
            seen_r += 1
            r_ln = rl[key]
            gz_r = np.array(r_ln[5 + J * (K + 1): 5 + J * (K + 1) + J], dtype=np.float64)
            assert np.abs(gz - gz_r).max() <= 1e-5 * max(1.0, np.abs(gz_r).max()), (mask, z0, gz, gz_r)
    assert seen_r == 2 * 15            # 0x1F and 0x0F at m = 4 are also R lines

