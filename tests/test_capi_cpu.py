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
    assert L.grav_forward3d(None, None, None, None) == capi.GRAV_EINVAL
    assert L.grav_adjoint3d(None, None, None, None) == capi.GRAV_EINVAL


@pytest.mark.parametrize(
    "args,needle",
    [
        ((0, 4, 4, 1.0, 1.0, 1.0, 1), "mesh size"),
        ((4, 4, 4, 1.0, 0.0, 1.0, 1), "cell sizes"),
        ((4, 4, 4, 1.0, 1.0, 1.0, 0), "component"),
        ((4, 4, 4, 1.0, 1.0, 1.0, 0x1FF), "more than 8 components"),
        ((1025, 4, 4, 1.0, 1.0, 1.0, 1), "equal-dimension mesh"),
        ((4, 4, 513, 1.0, 1.0, 1.0, 1), "equal-dimension mesh"),
    ],
)
def test_plan_create3d_rejects_bad_arguments(gravlib, args, needle):
    """Argument checks of the equal-dimension plan, before any device call."""
    with pytest.raises(capi.GravError) as ei:
        capi.grav_plan_create3d(*args)
    assert ei.value.code == capi.GRAV_EINVAL
    assert needle in str(ei.value)


def _c_values(tmp_path, body):
    """Compile a C program against include/grav.h with gcc and return what it
    prints as name -> integer."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "abi.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "grav.h"\nint main(void) {\n' + body +
                   "return 0; }\n")
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


CONSTANTS = ["GRAV_GZ", "GRAV_GXX", "GRAV_GXY", "GRAV_GXZ", "GRAV_GYY", "GRAV_GYZ", "GRAV_GZZ", "GRAV_GX", "GRAV_GY",
             "GRAV_ALL6", "GRAV_FP64_SPECTRAL", "GRAV_OK", "GRAV_EINVAL", "GRAV_ENOMEM", "GRAV_ECUDA",
             "GRAV_ETIMEOUT", "GRAV_MAX_NX", "GRAV_MAX_NY", "GRAV_STATIC_SCRATCH_BYTES"]


def test_binding_constants_equal_the_header(tmp_path):
    """Every constant of include/grav.h, as a C compiler sees it, equals the
    Python binding's."""
    body = "".join(f'printf("{n} %lld\\n", (long long)({n}));\n' for n in CONSTANTS)
    c = _c_values(tmp_path, body)
    for n in CONSTANTS:
        assert c[n] == getattr(capi, n), n
    assert capi.GRAV_COMP_BITS == c["GRAV_GZ"] | c["GRAV_GXX"] | c["GRAV_GXY"] | c["GRAV_GXZ"] | c["GRAV_GYY"] | \
        c["GRAV_GYZ"] | c["GRAV_GZZ"] | c["GRAV_GX"] | c["GRAV_GY"]


def test_plan_info_struct_layout_equals_the_header(tmp_path):
    """grav_plan_info_t has the same size and field offsets in C and in the
    ctypes mirror the binding passes to grav_plan_info."""
    fields = [f[0] for f in capi.grav_plan_info_t._fields_]
    body = 'printf("sizeof %zu\\n", sizeof(grav_plan_info_t));\n' + "".join(
        f'printf("{f} %zu\\n", offsetof(grav_plan_info_t, {f}));\n' for f in fields)
    c = _c_values(tmp_path, body)
    assert c["sizeof"] == ctypes.sizeof(capi.grav_plan_info_t)
    for f in fields:
        assert c[f] == getattr(capi.grav_plan_info_t, f).offset, f


def _prototypes():
    """name -> (return type, [parameter types]) of every function in grav.h."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \t\*]*?)\s*\b(grav_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", text):
        plist = [] if params.strip() in ("", "void") else [q.strip() for q in params.split(",")]
        types = []
        for q in plist:
            # pointers and array parameters (which decay to pointers); else drop the name
            types.append("pointer" if ("*" in q or "[" in q) else " ".join(q.split()[:-1]))
        protos[name] = (" ".join(ret.replace("*", " * ").split()), types)
    return protos


def _kind(ctype):
    if ctype is None:
        return "void"
    if ctype in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(ctype, ctypes._Pointer):
        return "pointer"
    return {ctypes.c_int: "int", ctypes.c_uint: "unsigned", ctypes.c_double: "double",
            ctypes.c_size_t: "size_t", ctypes.c_longlong: "long long"}[ctype]


def test_binding_signatures_equal_the_header(gravlib):
    """The ctypes argument and return types the binding sets match the
    header's prototypes parameter by parameter (count and kind)."""
    capi.lib()
    protos = _prototypes()
    assert sorted(protos) == sorted(capi.EXPORTED)
    for name, (ret, params) in protos.items():
        fn = getattr(gravlib, name)
        want = ["unsigned" if t in ("unsigned", "unsigned int") else t for t in params]
        assert [_kind(t) for t in fn.argtypes] == want, name
        want_ret = "pointer" if "*" in ret else ret.replace("const ", "")
        assert _kind(fn.restype) == want_ret, (name, ret)
