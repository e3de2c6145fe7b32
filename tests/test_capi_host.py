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
    (dict(widths=[2, 10, 1], G=5, m=3, n_instances=4), capi.HRKAN_EUNSUPPORTED),  # batched: fused m = 4 only
])
def test_bad_configuration_is_rejected_before_the_device(lib, kw, code):
    with pytest.raises(capi.HRKANError) as ei:
        capi.hrkan_init(capi.make_cfg(**kw))
    assert ei.value.code == code
    assert lib.hrkan_last_error().decode()


def test_null_handle_is_rejected(lib):
    assert lib.hrkan_forward_jets(None, None, None, 0, 1, None, None, None) == capi.HRKAN_EINVAL
    assert lib.hrkan_backward(None, None, None, 0, 1, None, None, None, 0, None) == capi.HRKAN_EINVAL
    assert lib.adam_step(None, None, None, 1e-3, 0.9, 0.999, 1e-8, 1, None) == capi.HRKAN_EINVAL
    lib.hrkan_destroy(None)
