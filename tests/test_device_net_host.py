"""Whole-network float32 jets composed from the kernels' own formulas, on the CPU,
against the FP64 oracle.

tests/device_host/hr_net_host.cu runs a network forward with the device code of
csrc/hr_device.cuh (Active basis evaluation, Jet rows) compiled for the host, in
the order the layer-wise forward kernel accumulates (per output and row: over
input units, then the k+1 active bases, one fmaf each), first-layer jets seeded
as the kernels seed them.  This checks that the float32 formulas compose through
several layers to the FP32 bar (1e-5 on u, 1e-4 on every derivative row,
normwise per row) for the PDE masks, the third/mixed-derivative masks and the
fourth/fifth-derivative masks (0x12F, 0x52F, 0xFFF) that no kernel is
instantiated for yet.  The backward takes seeded output-jet gradients through
the same formulas in reverse (Jet::adjoint_b for the input adjoint, the rows
for the weight gradient) and meets the 1e-4 weight-gradient bar per layer.
Shapes: Burgers [2,32,32,1] G=20 m=4 and a [2,24,24,1] G=12 m=6 net (Section 3 picks m = 6 for a fifth derivative), workload weights
N(0, 0.1^2), 300 interior points.

A three-input network runs, as the library runs it, as two passes of the
two-direction formulas with first-layer seeds (x, y) and then (z, none); their
rows put together give u, u_x, u_y, u_z, u_xx, u_yy, u_zz, and the weight
gradient is the sum of both passes' (the u row's gradient in the first)."""
import dataclasses
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from gpu_util import TOL_D, TOL_U, layer_slices, relerr
from paper_2409_14248_gb300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MASKS = [0x0F, 0x1F, 0x2F, 0xFF, 0x12F, 0x52F, 0xFFF]


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not installed")
    path = str(tmp_path_factory.mktemp("hnh") / "hr_net_host")
    src = os.path.join(ROOT, "tests", "device_host", "hr_net_host.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", *build.ARCH, src, "-o", path], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return path


def _workload(name):
    if name == "m6":
        return dataclasses.replace(inputs.WORKLOADS["poisson_2_64x3_1"], widths=[2, 24, 24, 1], G=12, m=6)
    return inputs.WORKLOADS["burgers_2_32_32_1"]


def _run(exe, tmp_path, w, W, x, mask, gy=None, seeds=(0, 1)):
    N = x.shape[1]
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        f.write(np.array([w.m, mask, len(w.widths), *w.widths, w.G, N, *seeds], dtype=np.int32).tobytes())
        f.write(np.array([w.lo, w.hi], dtype=np.float32).tobytes())
        f.write(np.ascontiguousarray(W, dtype=np.float32).tobytes())
        f.write(np.ascontiguousarray(x, dtype=np.float32).tobytes())
        if gy is not None:
            f.write(np.ascontiguousarray(gy, dtype=np.float32).tobytes())
    r = subprocess.run([exe, fin, fout] + ([] if gy is None else ["bwd"]), capture_output=True, timeout=120)
    assert r.returncode == 0, r.returncode
    if gy is not None:
        return np.fromfile(fout, dtype=np.float64)
    return np.fromfile(fout, dtype=np.float32).reshape(oracle.n_rows(mask), N)


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("name", ["burgers", "m6"])
def test_float32_network_jets_reach_the_fp32_bar(exe, tmp_path, name, mask):
    w = _workload(name)
    d = inputs.make(w, n_int=300, n_bnd=40, n_ic=20, n_bc=20)
    x = np.asarray(d["x_int"], dtype=np.float32)
    got = _run(exe, tmp_path, w, d["W"], x, mask)
    want = oracle.forward(w.net, np.asarray(d["W"], dtype=np.float64), x.astype(np.float64), mask)
    for r in range(want.shape[0]):
        tol = TOL_U if r == 0 else TOL_D
        assert relerr(got[r], want[r]) < tol, (name, hex(mask), r, relerr(got[r], want[r]))
        assert relerr(got[r], want[r]) > 0.0       # float32 arithmetic, not a copy of the oracle


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("name", ["burgers", "m6"])
def test_float32_network_weight_gradient_reaches_the_fp32_bar(exe, tmp_path, name, mask):
    w = _workload(name)
    d = inputs.make(w, n_int=300, n_bnd=40, n_ic=20, n_bc=20)
    x = np.asarray(d["x_int"], dtype=np.float32)
    gy = np.random.default_rng(5).standard_normal((oracle.n_rows(mask), x.shape[1])).astype(np.float32)
    got = _run(exe, tmp_path, w, d["W"], x, mask, gy)
    want = oracle.backward(w.net, np.asarray(d["W"], dtype=np.float64), x.astype(np.float64), mask,
                           gy.astype(np.float64))
    for l, sl in enumerate(layer_slices(w.widths, w.G)):
        assert 0.0 < relerr(got[sl], want[sl]) < TOL_D, (name, hex(mask), l, relerr(got[sl], want[sl]))


NET3 = dict(widths=[3, 16, 16, 1], G=8, k=3, m=4, lo=-1.0, hi=1.0)


def _three_inputs(N=400, seed=51):
    w = dataclasses.replace(inputs.WORKLOADS["burgers_2_32_32_1"], widths=NET3["widths"], G=NET3["G"], m=4,
                            lo=-1.0, hi=1.0)
    W = inputs.init_weights(oracle.param_count(NET3), seed, sigma=0.1)
    x = np.random.default_rng(seed + 1).uniform(-1, 1, (3, N)).astype(np.float32)
    return w, W, x


def test_three_input_jets_from_two_seeded_passes(exe, tmp_path):
    w, W, x = _three_inputs()
    a = _run(exe, tmp_path, w, W, x, 0x1F, seeds=(0, 1))      # u, u_x, u_y, u_xx, u_yy
    b = _run(exe, tmp_path, w, W, x, 0x1F, seeds=(2, -1))     # u, u_z, 0, u_zz, 0
    assert np.array_equal(a[0], b[0])
    assert not b[2].any() and not b[4].any()
    got = np.stack([a[0], a[1], a[2], b[1], a[3], a[4], b[3]])
    want = oracle.forward(NET3, np.asarray(W, dtype=np.float64), x.astype(np.float64), 0x7F)
    for r in range(7):
        assert 0.0 < relerr(got[r], want[r]) < (TOL_U if r == 0 else TOL_D), (r, relerr(got[r], want[r]))


def test_three_input_weight_gradient_from_two_seeded_passes(exe, tmp_path):
    w, W, x = _three_inputs(seed=52)
    g = np.random.default_rng(53).standard_normal((7, x.shape[1])).astype(np.float32)
    zero = np.zeros_like(g[0])
    ga = np.stack([g[0], g[1], g[2], g[4], g[5]])             # rows of the (x, y) pass
    gb = np.stack([zero, g[3], zero, g[6], zero])             # rows of the (z, none) pass
    got = _run(exe, tmp_path, w, W, x, 0x1F, ga, seeds=(0, 1)) + _run(exe, tmp_path, w, W, x, 0x1F, gb, seeds=(2, -1))
    want = oracle.backward(NET3, np.asarray(W, dtype=np.float64), x.astype(np.float64), 0x7F, g.astype(np.float64))
    for l, sl in enumerate(layer_slices(NET3["widths"], NET3["G"])):
        assert 0.0 < relerr(got[sl], want[sl]) < TOL_D, (l, relerr(got[sl], want[sl]))
