"""ctypes binding of ``include/grav.h``: the same entry points, argument
marshalling only.  Every computation runs in ``libgravfft.so``; if the
library has not been built this module raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgravfft.so")

GRAV_GZ, GRAV_GXX, GRAV_GXY, GRAV_GXZ, GRAV_GYY, GRAV_GYZ, GRAV_GZZ = 1, 2, 4, 8, 16, 32, 64
GRAV_GX, GRAV_GY = 128, 256
GRAV_ALL6 = 63
GRAV_COMP_BITS = 0x1FF  # every component bit
GRAV_MAX_PLAN_COMPONENTS = 8
GRAV_FP64_SPECTRAL = 1 << 16
GRAV_OK, GRAV_EINVAL, GRAV_ENOMEM, GRAV_ECUDA, GRAV_ETIMEOUT = 0, -1, -2, -3, -4
GRAV_MAX_NX, GRAV_MAX_NY = 2048, 1024
GRAV_STATIC_SCRATCH_BYTES = 16 << 20

COMPONENT_NAMES = ("gz", "gxx", "gxy", "gxz", "gyy", "gyz", "gzz")

# Every function the header declares; the CPU test checks the library
# exports each of them.
EXPORTED = (
    "grav_plan_create",
    "grav_forward",
    "grav_adjoint",
    "grav_plan_destroy",
    "grav_last_error",
    "grav_plan_bytes",
    "grav_plan_info",
    "grav_kernel_values",
    "grav_plan_set_timing",
    "grav_plan_stage_times",
    "grav_forward_static_scratch",
    "grav_plan_check",
    "grav_selftest_bounded_wait",
    "grav_workspace_bytes",
    "grav_forward_batch",
    "grav_adjoint_batch",
    "grav_plan_create3d",
    "grav_forward3d",
    "grav_adjoint3d",
    "grav_forward_batch_plans",
    "grav_adjoint_batch_plans",
)


class GravError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class grav_plan_info_t(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("px", ctypes.c_int), ("py", ctypes.c_int),
        ("ncomp", ctypes.c_int), ("fp64", ctypes.c_int),
        ("spectra_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
        ("pz", ctypes.c_int), ("equal_dim", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with paper_2005_10160_gb300.build.build() "
                    "(there is no fallback implementation)")
            L = ctypes.CDLL(LIB_PATH)
            i, u, d, p, sz = ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
            L.grav_plan_create.argtypes = [i, i, i, d, d, d, d, u]
            L.grav_plan_create.restype = p
            L.grav_forward.argtypes = [p, p, p, p]
            L.grav_forward.restype = i
            L.grav_adjoint.argtypes = [p, p, p, p]
            L.grav_adjoint.restype = i
            L.grav_plan_destroy.argtypes = [p]
            L.grav_plan_destroy.restype = None
            L.grav_last_error.argtypes = []
            L.grav_last_error.restype = ctypes.c_char_p
            L.grav_plan_bytes.argtypes = [p]
            L.grav_plan_bytes.restype = sz
            L.grav_plan_info.argtypes = [p, ctypes.POINTER(grav_plan_info_t)]
            L.grav_plan_info.restype = i
            L.grav_kernel_values.argtypes = [i, i, i, d, d, d, d, u, p, p]
            L.grav_kernel_values.restype = i
            L.grav_plan_set_timing.argtypes = [p, i]
            L.grav_plan_set_timing.restype = i
            L.grav_plan_stage_times.argtypes = [p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
            L.grav_plan_stage_times.restype = i
            L.grav_forward_static_scratch.argtypes = [p, p, p, p]
            L.grav_forward_static_scratch.restype = i
            L.grav_plan_check.argtypes = [p]
            L.grav_plan_check.restype = i
            L.grav_selftest_bounded_wait.argtypes = [d, ctypes.POINTER(ctypes.c_double)]
            L.grav_selftest_bounded_wait.restype = i
            L.grav_workspace_bytes.argtypes = [p]
            L.grav_workspace_bytes.restype = sz
            L.grav_forward_batch.argtypes = [p, i, p, p, p, p]
            L.grav_forward_batch.restype = i
            L.grav_adjoint_batch.argtypes = [p, i, p, p, p, p]
            L.grav_adjoint_batch.restype = i
            L.grav_forward_batch_plans.argtypes = [i, ctypes.POINTER(p), p, p, p, p]
            L.grav_forward_batch_plans.restype = i
            L.grav_adjoint_batch_plans.argtypes = [i, ctypes.POINTER(p), p, p, p, p]
            L.grav_adjoint_batch_plans.restype = i
            L.grav_plan_create3d.argtypes = [i, i, i, d, d, d, u]
            L.grav_plan_create3d.restype = p
            L.grav_forward3d.argtypes = [p, p, p, p]
            L.grav_forward3d.restype = i
            L.grav_adjoint3d.argtypes = [p, p, p, p]
            L.grav_adjoint3d.restype = i
            _lib = L
    return _lib


def grav_last_error() -> str:
    return lib().grav_last_error().decode(errors="replace")


def _check(rc: int) -> int:
    if rc != GRAV_OK:
        raise GravError(rc, grav_last_error())
    return rc


def grav_plan_create(nx, ny, nz, dx, dy, dz, h, components) -> int:
    """Returns the opaque plan handle (an int); raises GravError on failure."""
    ptr = lib().grav_plan_create(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), float(h),
                                 int(components))
    if not ptr:
        msg = grav_last_error()
        code = GRAV_ENOMEM if ("memory" in msg or "cudaMalloc" in msg) else GRAV_EINVAL
        raise GravError(code, msg)
    return ptr


def grav_forward(plan, rho_ptr, out_ptr, stream=0) -> int:
    return _check(lib().grav_forward(plan, rho_ptr, out_ptr, stream or None))


def grav_adjoint(plan, r_ptr, grad_ptr, stream=0) -> int:
    return _check(lib().grav_adjoint(plan, r_ptr, grad_ptr, stream or None))


def grav_plan_destroy(plan) -> None:
    if plan:
        lib().grav_plan_destroy(plan)


def grav_plan_bytes(plan) -> int:
    return int(lib().grav_plan_bytes(plan))


def grav_plan_info(plan) -> grav_plan_info_t:
    info = grav_plan_info_t()
    _check(lib().grav_plan_info(plan, ctypes.byref(info)))
    return info


def grav_kernel_values(nx, ny, nz, dx, dy, dz, h, components, K_ptr, stream=0) -> int:
    return _check(lib().grav_kernel_values(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), float(h),
                                           int(components), K_ptr, stream or None))


def comp_list(components: int) -> list[int]:
    return [c for c in range(9) if components & (1 << c)]


def grav_plan_set_timing(plan, enable: bool) -> int:
    return _check(lib().grav_plan_set_timing(plan, 1 if enable else 0))


STAGES = ("forward_rows", "forward_columns", "forward_inverse_rows",
          "adjoint_rows", "adjoint_columns", "adjoint_inverse_rows")


def grav_plan_stage_times(plan):
    """(ms per stage as a dict, forward calls, adjoint calls) since the last read."""
    ms = (ctypes.c_double * 6)()
    calls = (ctypes.c_longlong * 2)()
    _check(lib().grav_plan_stage_times(plan, ms, calls))
    return dict(zip(STAGES, list(ms))), int(calls[0]), int(calls[1])


def grav_forward_static_scratch(plan, rho_ptr, out_ptr, stream=0) -> int:
    """grav_forward without the plan's workspaces: scratch comes from the
    library's static device array (for callers that cannot allocate)."""
    return _check(lib().grav_forward_static_scratch(plan, rho_ptr, out_ptr, stream or None))


def grav_plan_check(plan) -> int:
    """Raises GravError(GRAV_ETIMEOUT) if a bounded wait of an earlier call ran out."""
    return _check(lib().grav_plan_check(plan))


def grav_selftest_bounded_wait(limit_ms: float):
    """(status code, milliseconds waited) of the bounded-wait self-test."""
    waited = ctypes.c_double(0.0)
    rc = lib().grav_selftest_bounded_wait(float(limit_ms), ctypes.byref(waited))
    return rc, waited.value


def grav_workspace_bytes(plan) -> int:
    return int(lib().grav_workspace_bytes(plan))


def grav_forward_batch(plan, batch, rho_ptr, out_ptr, ws_ptr, stream=0) -> int:
    return _check(lib().grav_forward_batch(plan, int(batch), rho_ptr, out_ptr, ws_ptr or None, stream or None))


def grav_adjoint_batch(plan, batch, r_ptr, grad_ptr, ws_ptr, stream=0) -> int:
    return _check(lib().grav_adjoint_batch(plan, int(batch), r_ptr, grad_ptr, ws_ptr or None, stream or None))


def grav_plan_create3d(nx, ny, nz, dx, dy, dz, components) -> int:
    """Equal-dimension plan (a station at every cell centre); raises GravError on failure."""
    ptr = lib().grav_plan_create3d(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), int(components))
    if not ptr:
        msg = grav_last_error()
        code = GRAV_ENOMEM if ("memory" in msg or "cudaMalloc" in msg) else GRAV_EINVAL
        raise GravError(code, msg)
    return ptr


def grav_forward3d(plan, rho_ptr, out_ptr, stream=0) -> int:
    return _check(lib().grav_forward3d(plan, rho_ptr, out_ptr, stream or None))


def grav_adjoint3d(plan, r_ptr, grad_ptr, stream=0) -> int:
    return _check(lib().grav_adjoint3d(plan, r_ptr, grad_ptr, stream or None))


def _plan_array(plans):
    arr = (ctypes.c_void_p * len(plans))()
    for i, h in enumerate(plans):
        arr[i] = h
    return arr


def grav_forward_batch_plans(plans, rho_ptr, out_ptr, ws_ptr, stream=0) -> int:
    """One batched forward over requests on different plans of equal sizes and
    components (request b on plans[b])."""
    return _check(lib().grav_forward_batch_plans(len(plans), _plan_array(plans), rho_ptr, out_ptr, ws_ptr or None,
                                                 stream or None))


def grav_adjoint_batch_plans(plans, r_ptr, grad_ptr, ws_ptr, stream=0) -> int:
    return _check(lib().grav_adjoint_batch_plans(len(plans), _plan_array(plans), r_ptr, grad_ptr, ws_ptr or None,
                                                 stream or None))
