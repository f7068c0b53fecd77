"""Plant mistakes in a copy of the oracle (on the CPU) and check that the pins
catch every one of them.

Each mutant is the oracle's C source with one plausible error: a dropped
term, a wrong sign, swapped axes, a wrong corner sign, a wrong cell or
station index.  It is compiled into a temporary library and run against the
same independent references the pins use (quadrature of one prism and the
closed form of a whole box built from cells).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from quadrature import prism_quadrature

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "prism_oracle.c")

MUTANTS = {
    "drop_atan_term_gz": ("- zk * t_z);", ");"),
    "swap_asinh_gz": ("xi * a_y + yj * a_x", "xi * a_x + yj * a_y"),
    "sign_gxy": ("acc[2] += mu * -a_z;", "acc[2] += mu * a_z;"),
    "gxz_uses_gyz_form": ("acc[3] += mu * -a_y;", "acc[3] += mu * -a_x;"),
    "corner_sign": ("? -1.0 : 1.0", "? 1.0 : -1.0"),
    "station_minus_sign": ("x - xi1, x - xi2", "xi1 - x, xi2 - x"),
    "station_x_offset": ("(p + 0.5) * g->dx", "(p + 1.0) * g->dx"),
    "cell_y_uses_dx": ("m * g->dy, (m + 1) * g->dy", "m * g->dx, (m + 1) * g->dx"),
    "layer_index": ("n * g->dz, (n + 1) * g->dz", "(n + 1) * g->dz, (n + 2) * g->dz"),
    "rho_index_swapped": ("rho[((size_t)n * g->ny + m) * g->nx + l]", "rho[((size_t)n * g->nx + l) * g->ny + m]"),
    "atan_gxx_gyy_swapped": ("acc[1] += mu * t_x;", "acc[1] += mu * t_y;"),
    "sign_gx_atan": ("- xi * t_x);", "+ xi * t_x);"),
    "gy_asinh_swapped": ("zk * a_x + xi * a_z", "zk * a_z + xi * a_x"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, name
    mutated = src.replace(old, new)
    c_path = tmp_path / f"{name}.c"
    so_path = tmp_path / f"{name}.so"
    c_path.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so_path), str(c_path), "-lm", "-lpthread"], check=True)
    lib = ctypes.CDLL(str(so_path))
    d, i, u, p = ctypes.c_double, ctypes.c_int, ctypes.c_uint, ctypes.c_void_p
    lib.orc_prism.argtypes = [d] * 9 + [p]
    lib.orc_forward.argtypes = [i, i, i, d, d, d, d, u, p, i, p, p, i]
    lib.orc_forward.restype = i
    return lib


def _pins_pass(lib):
    """True when the library passes the quadrature and superposition pins."""
    for station, box in [((13.0, -4.0, -7.0), (0.0, 10.0, 0.0, 20.0, 0.0, 15.0)),
                         ((2.0, 30.0, -3.0), (0.0, 10.0, 0.0, 20.0, 0.0, 15.0))]:
        out = np.zeros(9)
        lib.orc_prism(*station, *box, out.ctypes.data_as(ctypes.c_void_p))
        ref = prism_quadrature(station, box, nsub=4, order=16)
        if np.abs(out - ref).max() > 1e-9 * np.abs(ref).max():
            return False
    # superposition: an off-centre box of cells versus the whole-box closed form
    nx, ny, nz, dx, dy, dz, h = 6, 5, 4, 10.0, 12.0, 9.0, 3.0
    rho = np.zeros((nz, ny, nx))
    rho[1:3, 1:4, 2:5] = 1.0
    idx = np.arange(nx * ny, dtype=np.int32)
    got = np.zeros((7, nx * ny))
    lib.orc_forward(nx, ny, nz, dx, dy, dz, h, 0x7F, rho.ctypes.data_as(ctypes.c_void_p), nx * ny,
                    idx.ctypes.data_as(ctypes.c_void_p), got.ctypes.data_as(ctypes.c_void_p), 1)
    for s in range(nx * ny):
        p_, q_ = s % nx, s // nx
        station = ((p_ + 0.5) * dx, (q_ + 0.5) * dy, -h)
        box = (2 * dx, 5 * dx, 1 * dy, 4 * dy, 1 * dz, 3 * dz)
        ref = prism_quadrature(station, box, nsub=2, order=12) if s % 7 == 0 else None
        if ref is not None and np.abs(got[:, s] - ref[:7]).max() > 1e-7 * np.abs(ref[:7]).max():
            return False
    return True


def test_unmutated_oracle_passes(tmp_path):
    lib = _build(tmp_path, "original", "#include <math.h>", "#include <math.h>")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    assert not _pins_pass(lib), f"planted mistake {name} was not caught"
