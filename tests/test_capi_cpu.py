"""The C ABI library loads and exports every entry point that
include/grav.h declares; argument checks that never reach the device."""
import ctypes
import os
import re

import pytest

from paper_2005_10160_gb300 import capi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "grav.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grav_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(capi.EXPORTED)


def test_library_exports_every_declared_symbol(gravlib):
    for name in declared_functions():
        assert hasattr(gravlib, name), name
        assert ctypes.cast(getattr(gravlib, name), ctypes.c_void_p).value


@pytest.mark.parametrize(
    "args,needle",
    [
        ((0, 4, 4, 1.0, 1.0, 1.0, 1.0, 1), "mesh size"),
        ((4, 4, 4, 1.0, 1.0, 1.0, 0.0, 1), "station height"),
        ((4, 4, 4, 1.0, -1.0, 1.0, 1.0, 1), "cell sizes"),
        ((4, 4, 4, 1.0, 1.0, 1.0, 1.0, 0), "component"),
        ((4, 4, 4, 1.0, 1.0, 1.0, 1.0, 1 << 20), "component"),
        ((4, 4, 4, 1.0, 1.0, 1.0, 1.0, 1 << 9), "component"),
        ((4, 4, 4, 1.0, 1.0, 1.0, 1.0, 0x1FF), "more than 8 components"),
        ((capi.GRAV_MAX_NX + 1, 4, 4, 1.0, 1.0, 1.0, 1.0, 1), "mesh size"),
        ((4, capi.GRAV_MAX_NY + 1, 4, 1.0, 1.0, 1.0, 1.0, 1), "mesh size"),
        ((4, 4, 4, float("nan"), 1.0, 1.0, 1.0, 1), "cell sizes"),
    ],
)
def test_plan_create_rejects_bad_arguments(gravlib, args, needle):
    with pytest.raises(capi.GravError) as ei:
        capi.grav_plan_create(*args)
    assert ei.value.code == capi.GRAV_EINVAL
    assert needle in str(ei.value)


def test_null_plan_and_buffers_are_rejected(gravlib):
    L = gravlib
    assert L.grav_forward(None, None, None, None) == capi.GRAV_EINVAL
    assert "null" in capi.grav_last_error()
    assert L.grav_adjoint(None, None, None, None) == capi.GRAV_EINVAL
    assert L.grav_plan_bytes(None) == 0
    assert L.grav_plan_info(None, None) == capi.GRAV_EINVAL
    L.grav_plan_destroy(None)
    assert L.grav_kernel_values(4, 4, 1, 1.0, 1.0, 1.0, 1.0, 1, None, None) == capi.GRAV_EINVAL
    assert L.grav_kernel_values(4, 4, 1, 1.0, 1.0, 1.0, -1.0, 1, None, None) == capi.GRAV_EINVAL
    assert L.grav_plan_check(None) == capi.GRAV_EINVAL
    assert L.grav_plan_set_timing(None, 1) == capi.GRAV_EINVAL
    assert L.grav_forward_static_scratch(None, None, None, None) == capi.GRAV_EINVAL
    rc, _ = capi.grav_selftest_bounded_wait(0.0)
    assert rc == capi.GRAV_EINVAL
