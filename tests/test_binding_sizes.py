"""The Python binding's buffer-size checks, on the CPU.

The C ABI takes bare pointers, so the binding checks every tensor's element
count against the layout the header documents before the call reaches a
kernel.  Here the library is a fake whose entry points all succeed and the
tensors live in host memory: every call must accept buffers of exactly the
documented size and refuse, with HRKAN_EINVAL, one element fewer.  The sizes
below are written out by hand for concrete shapes from the header's layouts
(x [2][N], jets [J][N], single-layer jets [J][I][N] or for layer 0 the
coordinates [2][N], weights [O][I][G+k] per layer, batched arrays per
instance)."""
import ctypes

import numpy as np
import pytest

from paper_2409_14248_gb300 import capi

torch = pytest.importorskip("torch")


class FakeLibrary:
    """Every entry point returns HRKAN_OK; hrkan_param_count and hrkan_tape_floats follow the header."""

    def hrkan_param_count(self, cfg_ref):
        c = cfg_ref._obj
        w = [c.widths[i] for i in range(c.n_widths)]
        return sum(a * b for a, b in zip(w, w[1:])) * (c.G + c.k)

    def hrkan_tape_floats(self, h, N, mask):
        return bin(mask & 0xFF).count("1") * sum(h.widths[1:-1]) * N    # inputs of layers 1 .. L-1

    def hrkan_last_error(self):
        return b""

    def __getattr__(self, name):
        return lambda *a: capi.HRKAN_OK


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLibrary()
    monkeypatch.setattr(capi, "load_library", lambda *a, **k: lib)
    monkeypatch.setattr(capi, "_ptr", lambda t, dtype=None: None if t is None else ctypes.c_void_p(t.data_ptr()))
    monkeypatch.setattr(capi, "_stream", lambda s: None)
    return lib


def f32(n):
    return torch.zeros(max(n, 0), dtype=torch.float32)


def f64(n):
    return torch.zeros(max(n, 0), dtype=torch.float64)


def _refuses(call):
    with pytest.raises(capi.HRKANError) as ei:
        call()
    assert ei.value.code == capi.HRKAN_EINVAL


def _exact_and_short(call, sizes):
    """call(**buffers) passes with the given sizes and fails when any one buffer is one element short."""
    call(**{k: mk(n) for k, (mk, n) in sizes.items()})
    for short in sizes:
        if sizes[short][1] == 0:
            continue
        bufs = {k: mk(n - (k == short)) for k, (mk, n) in sizes.items()}
        _refuses(lambda: call(**bufs))


# [2,32,32,1], G = 20, k = 3: 23 bases per unit, P = (2*32 + 32*32 + 32*1) * 23 = 25760
NET = dict(widths=[2, 32, 32, 1], G=20)
P = 25760


def _handle(widths=NET["widths"], G=NET["G"], n_instances=1):
    return capi.hrkan_init(capi.make_cfg(widths, G, n_instances=n_instances))


def test_handle_carries_its_shape(fake):
    h = _handle()
    assert (h.P, h.D, h.n, h.n_inst, h.widths) == (P, 2, 23, 1, [2, 32, 32, 1])
    h3 = _handle([3, 8, 1], 5)
    assert (h3.P, h3.D) == ((3 * 8 + 8) * 8, 3)


def test_forward_and_backward_sizes(fake):
    h = _handle()
    N, mask = 100, 0x1F          # J = 5; the tape holds 5 x (32 + 32) x 100 floats
    _exact_and_short(lambda W, x, jets, tape: capi.hrkan_forward_jets(h, W, x, N, mask, jets, tape),
                     dict(W=(f32, P), x=(f32, 200), jets=(f32, 500), tape=(f32, 32000)))
    _exact_and_short(lambda W, x, tape, g, dW: capi.hrkan_backward(h, W, x, N, mask, tape, g, dW),
                     dict(W=(f32, P), x=(f32, 200), tape=(f32, 32000), g=(f32, 500), dW=(f32, P)))
    # third-order and mixed rows: mask 0xFF has J = 8
    _exact_and_short(lambda jets: capi.hrkan_forward_jets(h, f32(P), f32(200), N, 0xFF, jets),
                     dict(jets=(f32, 800)))
    # N = 0: the forward touches nothing, the backward still clears dW
    capi.hrkan_forward_jets(h, f32(0), f32(0), 0, mask, f32(0))
    _exact_and_short(lambda dW: capi.hrkan_backward(h, f32(0), f32(0), 0, mask, None, f32(0), dW),
                     dict(dW=(f32, P)))


def test_three_input_sizes(fake):
    h = _handle([3, 16, 1], 6)     # P = (3*16 + 16) * 9 = 576; x [3][N]; mask 0x7F has J = 7
    _exact_and_short(lambda W, x, jets: capi.hrkan_forward_jets(h, W, x, 10, 0x7F, jets),
                     dict(W=(f32, 576), x=(f32, 30), jets=(f32, 70)))


def test_residual_and_training_step_sizes(fake):
    h = _handle()
    prob = capi.make_problem(capi.HRKAN_BURGERS, lam=1.0, nu=0.01)
    Ni, Nb, mask = 50, 20, 0x0F    # J = 4
    _exact_and_short(lambda x, j, u, g, loss, dj, du: capi.pinn_residual_loss(h, prob, x, Ni, mask, j, u, g, Nb, loss,
                                                                              dj, du),
                     dict(x=(f32, 100), j=(f32, 200), u=(f32, 20), g=(f32, 20), loss=(f64, 3), dj=(f32, 200),
                          du=(f32, 20)))
    _exact_and_short(lambda W, xi, xb, gb, loss, dW: capi.hrkan_train_step(h, prob, W, xi, Ni, xb, gb, Nb, 1e-3, 0.9,
                                                                           0.999, 1e-8, 1, loss, dW),
                     dict(W=(f32, P), xi=(f32, 100), xb=(f32, 40), gb=(f32, 20), loss=(f64, 3), dW=(f32, P)))
    _exact_and_short(lambda W, dW: capi.adam_step(h, W, dW, 1e-3), dict(W=(f32, P), dW=(f32, P)))


def test_single_layer_sizes(fake):
    h = _handle()
    N, mask = 30, 0x1F             # J = 5
    for layer, I, O in ((0, 2, 32), (1, 32, 32), (2, 32, 1)):
        Wl = O * I * 23
        zin = 2 * N if layer == 0 else 5 * I * N    # the first layer takes the coordinates [2][N]
        _exact_and_short(lambda W, z, y: capi.hrkan_layer_jets(h, layer, W, z, N, mask, y),
                         dict(W=(f32, Wl), z=(f32, zin), y=(f32, 5 * O * N)))
        _exact_and_short(lambda z, gy, dW: capi.hrkan_layer_dw(h, layer, z, gy, N, mask, dW),
                         dict(z=(f32, zin), gy=(f32, 5 * O * N), dW=(f32, Wl)))
        if layer > 0:
            _exact_and_short(lambda W, z, gy, gz: capi.hrkan_layer_adjoint(h, layer, W, z, gy, N, mask, gz),
                             dict(W=(f32, Wl), z=(f32, 5 * I * N), gy=(f32, 5 * O * N), gz=(f32, 5 * I * N)))
    # an out-of-range layer is left to the library, which reports it
    capi.hrkan_layer_jets(h, 7, f32(1), f32(1), N, mask, f32(1))


def test_batched_sizes(fake):
    h = _handle([2, 16, 16, 1], 10, n_instances=4)   # P = (32 + 256 + 16) * 13 = 3952 per instance
    Pi = 3952
    probs = [capi.make_problem(capi.HRKAN_POISSON)] * 4
    oi = np.array([0, 10, 30, 30, 60])
    ob = np.array([0, 2, 4, 6, 8])
    _exact_and_short(lambda W, xi, xb, gb, loss, dW: capi.hrkan_train_step_batched(h, probs, W, xi, oi, xb, gb, ob,
                                                                                   1e-2, 0.9, 0.999, 1e-8, 1, loss,
                                                                                   dW),
                     dict(W=(f32, 4 * Pi), xi=(f32, 120), xb=(f32, 16), gb=(f32, 8), loss=(f64, 12), dW=(f32, 4 * Pi)))
    _exact_and_short(lambda W, x, jets: capi.hrkan_forward_jets_batched(h, W, x, oi, 0x0F, jets),
                     dict(W=(f32, 4 * Pi), x=(f32, 120), jets=(f32, 240)))
    # the host arrays: one problem per instance, n_instances + 1 offsets
    args = (f32(4 * Pi), f32(120))
    _refuses(lambda: capi.hrkan_train_step_batched(h, probs[:3], *args, oi, f32(16), f32(8), ob, 1e-2, 0.9, 0.999,
                                                   1e-8, 1, f64(12)))
    _refuses(lambda: capi.hrkan_train_step_batched(h, probs, *args, oi[:4], f32(16), f32(8), ob, 1e-2, 0.9, 0.999,
                                                   1e-8, 1, f64(12)))
    _refuses(lambda: capi.hrkan_forward_jets_batched(h, *args, oi[:4], 0x0F, f32(240)))
    _exact_and_short(lambda W: capi.hrkan_save(h, W, 5, "unused"), dict(W=(f32, 4 * Pi)))
