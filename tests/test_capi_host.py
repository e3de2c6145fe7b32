"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, exports every function include/hrkan.h declares, and rejects bad
configurations before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2409_14248_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load_library()


def _header_functions():
    src = open(os.path.join(ROOT, "include", "hrkan.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|int64_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return set(names)


def test_header_and_binding_agree():
    assert _header_functions() == set(capi.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _header_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_struct_layout_matches_header(lib):
    # int n_widths; int widths[8]; int G, k, m, prec; double lo, hi; int n_inst, reserved; size_t budget
    assert ctypes.sizeof(capi.hrkan_cfg) == 88
    assert capi.hrkan_cfg.grid_lo.offset == 56
    assert ctypes.sizeof(capi.pinn_problem) == 48


def test_param_count(lib):
    assert capi.hrkan_param_count(capi.make_cfg([2, 10, 10, 1], 10)) == 1690
    assert capi.hrkan_param_count(capi.make_cfg([2, 64, 64, 64, 1], 32)) == 293440
    assert capi.hrkan_param_count(capi.make_cfg([2, 16, 16, 1], 10)) == 3952
    assert capi.hrkan_param_count(capi.make_cfg([2, 5, 0, 1], 5)) == 0


@pytest.mark.parametrize("kw,code", [
    (dict(widths=[2, 5, 2], G=5), capi.HRKAN_EINVAL),          # two outputs
    (dict(widths=[2], G=5), capi.HRKAN_EINVAL),                # no layer
    (dict(widths=[2, 5, 1], G=0), capi.HRKAN_EINVAL),          # no grid interval
    (dict(widths=[2, 5, 1], G=5, lo=1.0, hi=-1.0), capi.HRKAN_EINVAL),
    (dict(widths=[2, 5, 1], G=5, n_instances=0), capi.HRKAN_EINVAL),
    (dict(widths=[2, 5, 1], G=5, prec=7), capi.HRKAN_EINVAL),
    (dict(widths=[4, 5, 1], G=5), capi.HRKAN_EUNSUPPORTED),    # D = 4
    (dict(widths=[3, 5, 1], G=5, prec=capi.HRKAN_BF16), capi.HRKAN_EUNSUPPORTED),   # D = 3 runs in FP32
    (dict(widths=[2, 5, 1], G=5, m=7), capi.HRKAN_EUNSUPPORTED),   # HR orders 2..6 are built
    (dict(widths=[2, 5, 1], G=5, m=1), capi.HRKAN_EUNSUPPORTED),   # u_xx needs m >= 2
    (dict(widths=[2, 5, 1], G=5, m=0), capi.HRKAN_EINVAL),
    (dict(widths=[2, 64, 1], G=5, m=6, prec=capi.HRKAN_BF16), capi.HRKAN_EUNSUPPORTED),  # tensor cores: m = 4
    (dict(widths=[3, 10, 1], G=5, n_instances=4), capi.HRKAN_EUNSUPPORTED),  # several instances: two inputs
])
def test_bad_configuration_is_rejected_before_the_device(lib, kw, code):
    with pytest.raises(capi.HRKANError) as ei:
        capi.hrkan_init(capi.make_cfg(**kw))
    assert ei.value.code == code
    assert lib.hrkan_last_error().decode()


# entry points whose first argument is an hrkan_t
HANDLE_CALLS = sorted(set(capi.EXPORTS) - {"hrkan_param_count", "hrkan_init", "hrkan_destroy", "hrkan_last_error",
                                           "hrkan_tape_floats", "hrkan_backward_noalloc", "hrkan_checkpoint_write",
                                           "hrkan_checkpoint_read"})


def _zero_args(fn):
    """NULL for every pointer, 0 for every number, in the order of the function's argtypes."""
    out = []
    for t in fn.argtypes:
        if t in (ctypes.c_int, ctypes.c_uint, ctypes.c_int64, ctypes.c_size_t):
            out.append(0)
        elif t is ctypes.c_double:
            out.append(0.0)
        else:
            out.append(None)
    return out


@pytest.mark.parametrize("name", HANDLE_CALLS)
def test_null_handle_is_rejected(lib, name):
    """Every call taking a handle returns HRKAN_EINVAL for a NULL one, with a message, before any device work."""
    fn = getattr(lib, name)
    assert fn(*_zero_args(fn)) == capi.HRKAN_EINVAL
    assert lib.hrkan_last_error().decode()


def test_null_handle_calls_without_a_status():
    lib = capi.load_library()
    lib.hrkan_destroy(None)
    assert lib.hrkan_tape_floats(None, 100, 0x1F) == 0


@pytest.mark.parametrize("cfg,mask,W,code", [
    (None, 0x1, 1, capi.HRKAN_EINVAL),                                                   # no configuration
    (dict(widths=[2, 10, 10, 1], G=10, m=6), 0x1, 1, capi.HRKAN_EUNSUPPORTED),           # fused kernels: m = 4
    (dict(widths=[2, 32, 32, 1], G=20), 0x1, 1, capi.HRKAN_EUNSUPPORTED),                # no fused kernel
    (dict(widths=[2, 10, 10, 1], G=10), 0x09, 1, capi.HRKAN_EINVAL),                     # u_xx without u_x
    (dict(widths=[2, 10, 10, 1], G=10), 0x2F, 1, capi.HRKAN_EINVAL),                     # third order: not here
    (dict(widths=[2, 10, 10, 1], G=10), 0x1F, None, capi.HRKAN_EINVAL),                  # NULL weights
])
def test_noalloc_backward_rejects_arguments_before_the_device(lib, cfg, mask, W, code):
    c = None if cfg is None else ctypes.byref(capi.make_cfg(**cfg))
    buf = (ctypes.c_float * 65536)()                   # a real host buffer; validation fails before any use
    w = None if W is None else ctypes.cast(buf, ctypes.c_void_p)
    assert lib.hrkan_backward_noalloc(c, w, w, 4, mask, w, w, 0, None) == code
    assert lib.hrkan_last_error().decode().startswith("hrkan_backward_noalloc")
