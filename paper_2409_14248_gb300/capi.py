"""Thin Python binding of the C ABI in include/hrkan.h (ctypes).

Argument marshalling only: every computation runs in libhrkan.so's CUDA
kernels.  Functions carry the C names and take torch CUDA tensors (float32
or float64 as the header states), which must be contiguous; the stream
defaults to torch's current stream.  Any non-OK status raises HRKANError with
the library's message.  There is no CPU fallback: if libhrkan.so has not been
built (``paper_2409_14248_gb300.build.build()``) loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhrkan.so")

HRKAN_OK, HRKAN_EINVAL, HRKAN_ENOMEM, HRKAN_ECUDA, HRKAN_EUNSUPPORTED, HRKAN_ETIMEOUT, HRKAN_ENONFINITE, HRKAN_EIO = \
    0, -1, -2, -3, -4, -5, -6, -7
HRKAN_FP32, HRKAN_BF16, HRKAN_TF32 = 0, 1, 2
HRKAN_POISSON, HRKAN_BURGERS, HRKAN_KDV, HRKAN_POISSON3 = 0, 1, 2, 3   # POISSON3: c in lam
HRKAN_MAX_WIDTHS = 8

# every symbol include/hrkan.h declares
EXPORTS = ("hrkan_param_count", "hrkan_init", "hrkan_destroy", "hrkan_last_error", "hrkan_tape_floats",
           "hrkan_forward_jets", "pinn_residual_loss", "hrkan_backward", "adam_step", "hrkan_reset_moments",
           "hrkan_train_step", "hrkan_profile_enable", "hrkan_profile_read", "hrkan_backward_noalloc",
           "hrkan_train_step_batched", "hrkan_forward_jets_batched", "hrkan_set_batch_items", "hrkan_sync_status",
           "hrkan_layer_jets", "hrkan_layer_dw", "hrkan_layer_adjoint", "hrkan_autotune_batch",
           "hrkan_checkpoint_write", "hrkan_checkpoint_read", "hrkan_save", "hrkan_load", "hrkan_set_wait_cycles",
           "hrkan_train_step_partial", "hrkan_set_batch_path", "hrkan_batch_path")
HRKAN_KERNEL_FUSED, HRKAN_KERNEL_REDUCE, HRKAN_KERNEL_FORWARD, HRKAN_KERNEL_RESIDUAL, HRKAN_KERNEL_TENSOR = 0, 1, 2, 3, 4
HRKAN_KERNEL_TC_FWD, HRKAN_KERNEL_TC_DW, HRKAN_KERNEL_TC_ADJ = 5, 6, 7
HRKAN_KERNEL_LAYER_FWD, HRKAN_KERNEL_LAYER_DW, HRKAN_KERNEL_LAYER_ADJ = 8, 9, 10
HRKAN_KERNEL_CLASSES = 11


class HRKANError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"status {code}: {msg}")
        self.code = code


class hrkan_cfg(ctypes.Structure):
    _fields_ = [("n_widths", ctypes.c_int), ("widths", ctypes.c_int * HRKAN_MAX_WIDTHS), ("G", ctypes.c_int),
                ("k", ctypes.c_int), ("m", ctypes.c_int), ("prec", ctypes.c_int), ("grid_lo", ctypes.c_double),
                ("grid_hi", ctypes.c_double), ("n_instances", ctypes.c_int), ("flags", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t)]


class pinn_problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("reserved", ctypes.c_int), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("lam", ctypes.c_double), ("nu", ctypes.c_double),
                ("alpha", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_vp, _i64, _u32, _i32, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint, ctypes.c_int, ctypes.c_double


def load_library(path: str = LIB_PATH):
    """Load libhrkan.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        lib.hrkan_param_count.argtypes = [ctypes.POINTER(hrkan_cfg)]
        lib.hrkan_param_count.restype = _i64
        lib.hrkan_init.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(hrkan_cfg)]
        lib.hrkan_destroy.argtypes = [_vp]
        lib.hrkan_destroy.restype = None
        lib.hrkan_last_error.restype = ctypes.c_char_p
        lib.hrkan_tape_floats.argtypes = [_vp, _i64, _u32]
        lib.hrkan_tape_floats.restype = _i64
        lib.hrkan_forward_jets.argtypes = [_vp, _vp, _vp, _i64, _u32, _vp, _vp, _vp]
        lib.pinn_residual_loss.argtypes = [_vp, ctypes.POINTER(pinn_problem), _vp, _i64, _u32, _vp, _vp, _vp, _i64,
                                           _vp, _vp, _vp, _vp]
        lib.hrkan_backward.argtypes = [_vp, _vp, _vp, _i64, _u32, _vp, _vp, _vp, _i32, _vp]
        lib.adam_step.argtypes = [_vp, _vp, _vp, _d, _d, _d, _d, _i32, _vp]
        lib.hrkan_reset_moments.argtypes = [_vp, _vp]
        lib.hrkan_train_step.argtypes = [_vp, ctypes.POINTER(pinn_problem), _vp, _vp, _i64, _vp, _vp, _i64, _d, _d,
                                         _d, _d, _i32, _vp, _vp, _vp]
        lib.hrkan_train_step_partial.argtypes = [_vp, ctypes.POINTER(pinn_problem), _vp, _vp, _i64, _vp, _vp, _i64,
                                                 _i64, _i64, _vp, _vp, _vp]
        lib.hrkan_backward_noalloc.argtypes = [ctypes.POINTER(hrkan_cfg), _vp, _vp, _i64, _u32, _vp, _vp, _i32, _vp]
        _i64p = ctypes.POINTER(_i64)
        lib.hrkan_autotune_batch.argtypes = [_vp, ctypes.POINTER(pinn_problem), _vp, _vp, _i64p, _vp, _vp, _i64p,
                                             ctypes.POINTER(ctypes.c_int), _i32, _i32, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double), _vp]
        lib.hrkan_train_step_batched.argtypes = [_vp, ctypes.POINTER(pinn_problem), _vp, _vp, _i64p, _vp, _vp, _i64p,
                                                 _d, _d, _d, _d, _i32, _vp, _vp, _vp]
        lib.hrkan_forward_jets_batched.argtypes = [_vp, _vp, _vp, _i64p, _u32, _vp, _vp]
        lib.hrkan_set_batch_items.argtypes = [_vp, _i32]
        lib.hrkan_set_batch_path.argtypes = [_vp, _i32]
        lib.hrkan_batch_path.argtypes = [_vp]
        lib.hrkan_sync_status.argtypes = [_vp]
        lib.hrkan_layer_jets.argtypes = [_vp, _i32, _vp, _vp, _i64, _u32, _vp, _vp]
        lib.hrkan_layer_dw.argtypes = [_vp, _i32, _vp, _vp, _i64, _u32, _vp, _vp]
        lib.hrkan_layer_adjoint.argtypes = [_vp, _i32, _vp, _vp, _vp, _i64, _u32, _vp, _vp]
        lib.hrkan_profile_enable.argtypes = [_vp, _i32]
        lib.hrkan_profile_read.argtypes = [_vp, _i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]
        lib.hrkan_checkpoint_write.argtypes = [ctypes.c_char_p, _i64, _i32, _i64, _i64, _vp, _vp, _vp]
        lib.hrkan_checkpoint_read.argtypes = [ctypes.c_char_p, _i64, _i32, _i64p, _i64p, _vp, _vp, _vp]
        lib.hrkan_save.argtypes = [_vp, _vp, _i64, ctypes.c_char_p, _vp]
        lib.hrkan_load.argtypes = [_vp, _vp, _i64p, ctypes.c_char_p, _vp]
        lib.hrkan_set_wait_cycles.argtypes = [_vp, _i64]
        for name in EXPORTS:
            if name not in ("hrkan_destroy", "hrkan_last_error", "hrkan_param_count", "hrkan_tape_floats"):
                getattr(lib, name).restype = _i32
        _lib = lib
        return lib


def _check(rc):
    if rc != HRKAN_OK:
        raise HRKANError(rc, load_library().hrkan_last_error().decode())


def _ptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


HRKAN_FLAG_LAYERWISE = 1


def make_cfg(widths, G, k=3, m=4, lo=-1.0, hi=1.0, prec=HRKAN_FP32, n_instances=1, hbm_budget_bytes=0, flags=0):
    c = hrkan_cfg()
    c.n_widths = len(widths)
    for i, w in enumerate(widths):
        c.widths[i] = int(w)
    c.G, c.k, c.m, c.prec = int(G), int(k), int(m), int(prec)
    c.grid_lo, c.grid_hi = float(lo), float(hi)
    c.n_instances, c.hbm_budget_bytes, c.flags = int(n_instances), int(hbm_budget_bytes), int(flags)
    return c


def make_problem(kind, a=1.0, b=1.0, lam=1.0, nu=0.0, alpha=1.0):
    return pinn_problem(int(kind), 0, float(a), float(b), float(lam), float(nu), float(alpha))


def hrkan_param_count(cfg):
    return int(load_library().hrkan_param_count(ctypes.byref(cfg)))


class Handle(ctypes.c_void_p):
    """An hrkan_t together with the network shape.  The C ABI sees bare pointers, so the
    wrappers below check each tensor's element count against what the call reads or writes
    and raise HRKANError(HRKAN_EINVAL) before a short buffer reaches a kernel."""


def hrkan_init(cfg):
    h = Handle()
    _check(load_library().hrkan_init(ctypes.byref(h), ctypes.byref(cfg)))
    h.widths = [int(cfg.widths[i]) for i in range(cfg.n_widths)]
    h.D = h.widths[0]
    h.n = int(cfg.G) + int(cfg.k)
    h.P = hrkan_param_count(cfg)
    h.n_inst = int(cfg.n_instances)
    return h


def _jets(mask):
    return bin(int(mask) & 0xFFF).count("1")


def _need(t, n, what):
    """Raise unless tensor (or array) t is absent or holds at least n elements."""
    if t is not None and t.numel() < n:
        raise HRKANError(HRKAN_EINVAL, f"{what} holds {t.numel()} elements, the call needs {n}")


def _shaped(h):
    return getattr(h, "P", None) is not None


def _layer_in(h, layer, J, N):
    """Floats of a single-layer call's input: jets [J][I][N], for layer 0 the coordinates [2][N]."""
    return 2 * N if int(layer) == 0 else J * h.widths[int(layer)] * N


def _layer_io(h, layer):
    """(I, O) of layer `layer`, or None when the index is out of range (the library reports it)."""
    L = len(h.widths) - 1
    return (h.widths[layer], h.widths[layer + 1]) if 0 <= int(layer) < L else None


def hrkan_destroy(h):
    load_library().hrkan_destroy(h)


def hrkan_tape_floats(h, N, jet_mask):
    return int(load_library().hrkan_tape_floats(h, int(N), int(jet_mask)))


def hrkan_forward_jets(h, W, x, N, jet_mask, jets, tape=None, stream=None):
    import torch
    if _shaped(h) and N > 0:
        _need(W, h.P, "W")
        _need(x, h.D * N, "x")
        _need(jets, _jets(jet_mask) * N, "jets")
        if tape is not None:
            _need(tape, hrkan_tape_floats(h, N, jet_mask), "tape")
    _check(load_library().hrkan_forward_jets(h, _ptr(W, torch.float32), _ptr(x, torch.float32), int(N),
                                             int(jet_mask), _ptr(jets, torch.float32), _ptr(tape, torch.float32),
                                             _stream(stream)))


def pinn_residual_loss(h, prob, x_int, N_int, jet_mask, jets_int, u_bnd, g_bnd, N_bnd, loss, dL_djets_int=None,
                       dL_du_bnd=None, stream=None):
    import torch
    f = torch.float32
    if _shaped(h):
        J = _jets(jet_mask)
        _need(loss, 3, "loss")
        if N_int > 0:
            _need(x_int, h.D * N_int, "x_int")
            _need(jets_int, J * N_int, "jets_int")
            _need(dL_djets_int, J * N_int, "dL_djets_int")
        if N_bnd > 0:
            _need(u_bnd, N_bnd, "u_bnd")
            _need(g_bnd, N_bnd, "g_bnd")
            _need(dL_du_bnd, N_bnd, "dL_du_bnd")
    _check(load_library().pinn_residual_loss(h, ctypes.byref(prob), _ptr(x_int, f), int(N_int), int(jet_mask),
                                             _ptr(jets_int, f), _ptr(u_bnd, f), _ptr(g_bnd, f), int(N_bnd),
                                             _ptr(loss, torch.float64), _ptr(dL_djets_int, f), _ptr(dL_du_bnd, f),
                                             _stream(stream)))


def hrkan_backward(h, W, x, N, jet_mask, tape, dL_djets, dW, accumulate=False, stream=None):
    import torch
    f = torch.float32
    if _shaped(h):
        _need(dW, h.P, "dW")
        if N > 0:
            _need(W, h.P, "W")
            _need(x, h.D * N, "x")
            _need(dL_djets, _jets(jet_mask) * N, "dL_djets")
            if tape is not None:
                _need(tape, hrkan_tape_floats(h, N, jet_mask), "tape")
    _check(load_library().hrkan_backward(h, _ptr(W, f), _ptr(x, f), int(N), int(jet_mask), _ptr(tape, f),
                                         _ptr(dL_djets, f), _ptr(dW, f), int(bool(accumulate)), _stream(stream)))


def adam_step(h, W, dW, lr, b1=0.9, b2=0.999, eps=1e-8, t=1, stream=None):
    import torch
    if _shaped(h):
        _need(W, h.P, "W")
        _need(dW, h.P, "dW")
    _check(load_library().adam_step(h, _ptr(W, torch.float32), _ptr(dW, torch.float32), float(lr), float(b1),
                                    float(b2), float(eps), int(t), _stream(stream)))


def hrkan_set_wait_cycles(h, cycles):
    """Limit of the tensor-core kernels' bounded waits (0 = default); for fault-injection tests."""
    _check(load_library().hrkan_set_wait_cycles(h, ctypes.c_int64(int(cycles))))


def hrkan_reset_moments(h, stream=None):
    _check(load_library().hrkan_reset_moments(h, _stream(stream)))


def hrkan_checkpoint_write(path, P, n_instances, t, t_device, W, m, v):
    """Write a checkpoint from host arrays (W float32, m and v float64, n_instances * P each)."""
    import numpy as np
    W = np.ascontiguousarray(W, dtype=np.float32)
    m = np.ascontiguousarray(m, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    n = int(P) * int(n_instances)
    if W.size != n or m.size != n or v.size != n:
        raise ValueError("W, m and v need n_instances * P elements")
    _check(load_library().hrkan_checkpoint_write(os.fsencode(path), ctypes.c_int64(int(P)), int(n_instances),
                                                 ctypes.c_int64(int(t)), ctypes.c_int64(int(t_device)),
                                                 W.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p),
                                                 v.ctypes.data_as(ctypes.c_void_p)))


def hrkan_checkpoint_read(path, P, n_instances):
    """Read a checkpoint into new host arrays: returns (t, t_device, W, m, v)."""
    import numpy as np
    n = int(P) * int(n_instances)
    W = np.empty(n, dtype=np.float32)
    m = np.empty(n, dtype=np.float64)
    v = np.empty(n, dtype=np.float64)
    t, td = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load_library().hrkan_checkpoint_read(os.fsencode(path), ctypes.c_int64(int(P)), int(n_instances),
                                                ctypes.byref(t), ctypes.byref(td), W.ctypes.data_as(ctypes.c_void_p),
                                                m.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p)))
    return t.value, td.value, W, m, v


def hrkan_save(h, W, t, path, stream=None):
    """Save the weights (device tensor), the handle's Adam moments and step counts."""
    import torch
    if _shaped(h):
        _need(W, h.n_inst * h.P, "W")
    _check(load_library().hrkan_save(h, _ptr(W, torch.float32), ctypes.c_int64(int(t)), os.fsencode(path),
                                     _stream(stream)))


def hrkan_load(h, W, path, stream=None):
    """Load a checkpoint into W (device tensor) and the handle; returns the stored step count t."""
    import torch
    if _shaped(h):
        _need(W, h.n_inst * h.P, "W")
    t = ctypes.c_int64(0)
    _check(load_library().hrkan_load(h, _ptr(W, torch.float32), ctypes.byref(t), os.fsencode(path), _stream(stream)))
    return t.value


def hrkan_train_step(h, prob, W, x_int, N_int, x_bnd, g_bnd, N_bnd, lr, b1, b2, eps, t, loss, dW=None,
                     stream=None):
    import torch
    f = torch.float32
    if _shaped(h):
        _need(W, h.P, "W")
        _need(dW, h.P, "dW")
        _need(loss, 3, "loss")
        if N_int > 0:
            _need(x_int, h.D * N_int, "x_int")
        if N_bnd > 0:
            _need(x_bnd, h.D * N_bnd, "x_bnd")
            _need(g_bnd, N_bnd, "g_bnd")
    _check(load_library().hrkan_train_step(h, ctypes.byref(prob), _ptr(W, f), _ptr(x_int, f), int(N_int),
                                           _ptr(x_bnd, f), _ptr(g_bnd, f), int(N_bnd), float(lr), float(b1),
                                           float(b2), float(eps), int(t), _ptr(loss, torch.float64),
                                           _ptr(dW, f), _stream(stream)))


def hrkan_train_step_partial(h, prob, W, x_int, N_int, x_bnd, g_bnd, N_bnd, N_int_total, N_bnd_total, loss, dW,
                             stream=None):
    """One shard's loss contributions and gradient (means over the totals of all shards), no Adam."""
    import torch
    f = torch.float32
    if _shaped(h):
        _need(W, h.P, "W")
        _need(dW, h.P, "dW")
        _need(loss, 3, "loss")
        if N_int > 0:
            _need(x_int, h.D * N_int, "x_int")
        if N_bnd > 0:
            _need(x_bnd, h.D * N_bnd, "x_bnd")
            _need(g_bnd, N_bnd, "g_bnd")
    _check(load_library().hrkan_train_step_partial(h, ctypes.byref(prob), _ptr(W, f), _ptr(x_int, f), int(N_int),
                                                   _ptr(x_bnd, f), _ptr(g_bnd, f), int(N_bnd), int(N_int_total),
                                                   int(N_bnd_total), _ptr(loss, torch.float64), _ptr(dW, f),
                                                   _stream(stream)))


def hrkan_profile_enable(h, enable=True):
    _check(load_library().hrkan_profile_enable(h, int(bool(enable))))


def hrkan_profile_read(h, kernel_class, reset=True):
    """(total milliseconds, launches) of one kernel class since the last reset."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(load_library().hrkan_profile_read(h, int(kernel_class), ctypes.byref(ms), ctypes.byref(n), int(reset)))
    return ms.value, n.value


def hrkan_backward_noalloc(cfg, W, x, N, jet_mask, dL_djets, dW, accumulate=False, stream=None):
    """hrkan_backward for callers that cannot allocate: no handle, static device scratch."""
    import torch
    f = torch.float32
    _check(load_library().hrkan_backward_noalloc(ctypes.byref(cfg), _ptr(W, f), _ptr(x, f), int(N), int(jet_mask),
                                                 _ptr(dL_djets, f), _ptr(dW, f), int(bool(accumulate)),
                                                 _stream(stream)))


def _i64_array(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _batch_sizes(h, probs, offsets, what):
    """The library reads n_instances problems and n_instances + 1 offsets from host memory."""
    I = h.n_inst
    if probs is not None and len(probs) < I:
        raise HRKANError(HRKAN_EINVAL, f"{len(probs)} problems for {I} instances")
    for name, off in zip(what, offsets):
        if len(off) < I + 1:
            raise HRKANError(HRKAN_EINVAL, f"{name} has {len(off)} entries, {I + 1} are needed")


def _check_batched_train(h, probs, W, x_int, oi, x_bnd, g_bnd, ob, loss, dW):
    _batch_sizes(h, probs, (oi, ob), ("off_int", "off_bnd"))
    I = h.n_inst
    n0, n1 = int(oi[I]), int(ob[I])
    _need(W, I * h.P, "W")
    _need(dW, I * h.P, "dW")
    _need(loss, 3 * I, "loss")
    if n0 > 0:
        _need(x_int, 2 * n0, "x_int")
    if n1 > 0:
        _need(x_bnd, 2 * n1, "x_bnd")
        _need(g_bnd, n1, "g_bnd")


def hrkan_train_step_batched(h, probs, W, x_int, off_int, x_bnd, g_bnd, off_bnd, lr, b1, b2, eps, t, loss,
                             dW=None, stream=None):
    """probs: sequence of pinn_problem (one per instance); offsets: host int arrays [I+1]."""
    import torch
    f = torch.float32
    arr = (pinn_problem * len(probs))(*probs)
    oi, oip = _i64_array(off_int)
    ob, obp = _i64_array(off_bnd)
    if _shaped(h):
        _check_batched_train(h, probs, W, x_int, oi, x_bnd, g_bnd, ob, loss, dW)
    _check(load_library().hrkan_train_step_batched(h, arr, _ptr(W, f), _ptr(x_int, f), oip, _ptr(x_bnd, f),
                                                   _ptr(g_bnd, f), obp, float(lr), float(b1), float(b2), float(eps),
                                                   int(t), _ptr(loss, torch.float64), _ptr(dW, f), _stream(stream)))


def hrkan_forward_jets_batched(h, W, x, offsets, jet_mask, jets, stream=None):
    import torch
    f = torch.float32
    o, op = _i64_array(offsets)
    if _shaped(h):
        _batch_sizes(h, None, (o,), ("offsets",))
        n = int(o[h.n_inst])
        _need(W, h.n_inst * h.P, "W")
        if n > 0:
            _need(x, 2 * n, "x")
            _need(jets, _jets(jet_mask) * n, "jets")
    _check(load_library().hrkan_forward_jets_batched(h, _ptr(W, f), _ptr(x, f), op, int(jet_mask), _ptr(jets, f),
                                                     _stream(stream)))


def hrkan_autotune_batch(h, probs, W, x_int, off_int, x_bnd, g_bnd, off_bnd, candidates=None, reps=3,
                         stream=None):
    """Times the multi-instance step for each item size (lr = 0: W unchanged), keeps the
    fastest, resets the Adam moments.  Returns (points per item, ms per step)."""
    import torch
    f = torch.float32
    arr = (pinn_problem * len(probs))(*probs)
    oi, oip = _i64_array(off_int)
    ob, obp = _i64_array(off_bnd)
    if _shaped(h):
        _check_batched_train(h, probs, W, x_int, oi, x_bnd, g_bnd, ob, None, None)
    cand = None if candidates is None else (ctypes.c_int * len(candidates))(*[int(c) for c in candidates])
    chosen, ms = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load_library().hrkan_autotune_batch(h, arr, _ptr(W, f), _ptr(x_int, f), oip, _ptr(x_bnd, f),
                                               _ptr(g_bnd, f), obp, cand, 0 if cand is None else len(candidates),
                                               int(reps), ctypes.byref(chosen), ctypes.byref(ms), _stream(stream)))
    return chosen.value, ms.value


def hrkan_set_batch_items(h, points_per_item):
    _check(load_library().hrkan_set_batch_items(h, int(points_per_item)))


def hrkan_set_batch_path(h, path):
    """Kernel family of the multi-instance calls: 0 fused, 1 layer-wise, 2 layer-wise with every
    layer's forward on the FP32 SIMT kernels (tensor cores for the backward only)."""
    _check(load_library().hrkan_set_batch_path(h, int(path)))


def hrkan_batch_path(h):
    """The multi-instance calls' kernel family: 0 fused, 1 layer-wise, 2 layer-wise with the FP32
    forward."""
    rc = load_library().hrkan_batch_path(h)
    if rc < 0:
        _check(rc)
    return rc


def hrkan_sync_status(h):
    """Synchronise; raise HRKANError(HRKAN_ETIMEOUT / HRKAN_ENONFINITE) for a recorded device-side failure."""
    _check(load_library().hrkan_sync_status(h))


def hrkan_layer_dw(h, layer, z, gy, N, jet_mask, dW, stream=None):
    """Weight gradient [O][I][n] of one layer from input jets z [J][I][N] and gy [J][O][N]."""
    import torch
    f = torch.float32
    io = _layer_io(h, layer) if _shaped(h) else None
    if io is not None:
        I, O = io
        J = _jets(jet_mask)
        _need(dW, O * I * h.n, "dW")
        if N > 0:
            _need(z, _layer_in(h, layer, J, N), "z")
            _need(gy, J * O * N, "gy")
    _check(load_library().hrkan_layer_dw(h, int(layer), _ptr(z, f), _ptr(gy, f), int(N), int(jet_mask), _ptr(dW, f),
                                         _stream(stream)))


def hrkan_layer_adjoint(h, layer, W_layer, z, gy, N, jet_mask, gz, stream=None):
    """Input adjoint gz [J][I][N] of layer >= 1 from z [J][I][N] and gy [J][O][N]."""
    import torch
    f = torch.float32
    io = _layer_io(h, layer) if _shaped(h) else None
    if io is not None and N > 0:
        I, O = io
        J = _jets(jet_mask)
        _need(W_layer, O * I * h.n, "W_layer")
        _need(z, J * I * N, "z")
        _need(gy, J * O * N, "gy")
        _need(gz, J * I * N, "gz")
    _check(load_library().hrkan_layer_adjoint(h, int(layer), _ptr(W_layer, f), _ptr(z, f), _ptr(gy, f), int(N),
                                              int(jet_mask), _ptr(gz, f), _stream(stream)))


def hrkan_layer_jets(h, layer, W_layer, z, N, jet_mask, y, stream=None):
    """One layer on given input jets z [J][I][N] -> y [J][O][N]."""
    import torch
    f = torch.float32
    io = _layer_io(h, layer) if _shaped(h) else None
    if io is not None and N > 0:
        I, O = io
        J = _jets(jet_mask)
        _need(W_layer, O * I * h.n, "W_layer")
        _need(z, _layer_in(h, layer, J, N), "z")
        _need(y, J * O * N, "y")
    _check(load_library().hrkan_layer_jets(h, int(layer), _ptr(W_layer, f), _ptr(z, f), int(N), int(jet_mask),
                                           _ptr(y, f), _stream(stream)))
