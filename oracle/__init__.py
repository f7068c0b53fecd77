"""CPU FP64 oracle for the prism gravity / gravity-gradient forward model.

Test infrastructure, not product code.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` import this
package.  It shares no code with the CUDA library and never imports it.

It computes the plain definition d = G M (Eqs. 3-4, Sec. 2.1): each
station/cell kernel value from the eight-corner closed form (Eq. 2 for gz,
the standard prism forms for the gradient components), summed directly.
The arithmetic lives in ``prism_oracle.c``; this module only compiles it with
gcc and marshals numpy arrays.

Component bits (ascending bit order is the row order of every output):
1 gz, 2 gxx, 4 gxy, 8 gxz, 16 gyy, 32 gyz, 64 gzz, 128 gx, 256 gy.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prism_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_prism_oracle.so")
_lock = threading.Lock()
_lib = None

COMPONENTS = ("gz", "gxx", "gxy", "gxz", "gyy", "gyz", "gzz", "gx", "gy")
UPSILON = 6.672e-11


_CMD = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared"]


def _stamp() -> str:
    h = hashlib.sha256(platform.machine().encode() + " ".join(_CMD).encode())
    with open(_SRC, "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile ``prism_oracle.c`` into ``_prism_oracle.so`` (plain -O2, IEEE,
    no fast-math) unless a build for this machine and source exists."""
    stamp_path = _LIB_PATH + ".stamp"
    if not force and os.path.exists(_LIB_PATH) and os.path.exists(stamp_path):
        with open(stamp_path) as fh:
            if fh.read().strip() == _stamp():
                return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(_CMD + ["-o", tmp, _SRC, "-lm", "-lpthread"], check=True)
    os.replace(tmp, _LIB_PATH)
    with open(stamp_path, "w") as fh:
        fh.write(_stamp())
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d, i, u = ctypes.c_double, ctypes.c_int, ctypes.c_uint
            p = ctypes.c_void_p
            lib.orc_prism.argtypes = [d] * 9 + [p]
            lib.orc_prism.restype = None
            lib.orc_forward.argtypes = [i, i, i, d, d, d, d, u, p, i, p, p, i]
            lib.orc_forward.restype = i
            lib.orc_adjoint.argtypes = [i, i, i, d, d, d, d, u, p, i, p, p, i]
            lib.orc_adjoint.restype = i
            lib.orc_gmatrix.argtypes = [i, i, i, d, d, d, d, u, p]
            lib.orc_gmatrix.restype = i
            lib.orc_forward3d.argtypes = [i, i, i, d, d, d, u, p, i, p, p, i]
            lib.orc_forward3d.restype = i
            lib.orc_adjoint3d.argtypes = [i, i, i, d, d, d, u, p, i, p, p, i]
            lib.orc_adjoint3d.restype = i
            lib.orc_gmatrix3d.argtypes = [i, i, i, d, d, d, u, p]
            lib.orc_gmatrix3d.restype = i
            _lib = lib
    return _lib


def comp_list(comps: int) -> list[int]:
    """Component indices selected by a bit mask, in ascending bit order."""
    return [c for c in range(len(COMPONENTS)) if comps & (1 << c)]


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def prism(station, box) -> np.ndarray:
    """Kernel per unit density of one prism at one station, all 9 components.

    station = (x, y, z); box = (xi1, xi2, eta1, eta2, zeta1, zeta2); z positive
    down.  Returns [gz, gxx, gxy, gxz, gyy, gyz, gzz] in SI units (Eq. 2 and
    the standard gradient forms)."""
    lib = _load()
    out = np.zeros(len(COMPONENTS), dtype=np.float64)
    lib.orc_prism(*[float(v) for v in station], *[float(v) for v in box],
                  out.ctypes.data_as(ctypes.c_void_p))
    return out


def _geom(mesh):
    nx, ny, nz, dx, dy, dz, h = mesh
    return int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), float(h)


def forward(mesh, comps: int, rho: np.ndarray, stations=None, nthreads=None) -> np.ndarray:
    """Direct summation d_c(i) = sum_j G_c(i, j) rho_j (Eq. 3).

    mesh = (nx, ny, nz, dx, dy, dz, h); rho is [nz][ny][nx]; ``stations`` is
    an optional list of station indices p + nx q (all stations if None).
    Returns [ncomp][n_stations] float64 (or [ncomp][ny][nx] for all)."""
    lib = _load()
    nx, ny, nz, dx, dy, dz, h = _geom(mesh)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(nz, ny, nx)
    full = stations is None
    idx = np.arange(nx * ny, dtype=np.int32) if full else np.ascontiguousarray(stations, dtype=np.int32)
    nc = len(comp_list(comps))
    out = np.zeros((nc, idx.size), dtype=np.float64)
    rc = lib.orc_forward(nx, ny, nz, dx, dy, dz, h, comps,
                         rho.ctypes.data_as(ctypes.c_void_p), int(idx.size),
                         idx.ctypes.data_as(ctypes.c_void_p),
                         out.ctypes.data_as(ctypes.c_void_p),
                         int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("orc_forward: invalid arguments")
    return out.reshape(nc, ny, nx) if full else out


def adjoint(mesh, comps: int, resid: np.ndarray, cells=None, nthreads=None) -> np.ndarray:
    """(G^T r)_j = sum_c sum_i G_c(i, j) r_c(i), the transpose of Eq. 4.

    resid is [ncomp][ny][nx]; ``cells`` an optional list of cell indices
    l + nx m + nx ny n.  Returns [nz][ny][nx] (all cells) or [n_cells]."""
    lib = _load()
    nx, ny, nz, dx, dy, dz, h = _geom(mesh)
    nc = len(comp_list(comps))
    resid = np.ascontiguousarray(resid, dtype=np.float64).reshape(nc, ny, nx)
    full = cells is None
    idx = np.arange(nx * ny * nz, dtype=np.int32) if full else np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros(idx.size, dtype=np.float64)
    rc = lib.orc_adjoint(nx, ny, nz, dx, dy, dz, h, comps,
                         resid.ctypes.data_as(ctypes.c_void_p), int(idx.size),
                         idx.ctypes.data_as(ctypes.c_void_p),
                         out.ctypes.data_as(ctypes.c_void_p),
                         int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("orc_adjoint: invalid arguments")
    return out.reshape(nz, ny, nx) if full else out


def gmatrix(mesh, comps: int) -> np.ndarray:
    """Explicit kernel matrix G[c][i][j] (Eqs. 3-5) for tiny meshes."""
    lib = _load()
    nx, ny, nz, dx, dy, dz, h = _geom(mesh)
    nc = len(comp_list(comps))
    nd, nm = nx * ny, nx * ny * nz
    if nc * nd * nm > 50_000_000:
        raise ValueError("gmatrix is for tiny meshes only")
    G = np.zeros((nc, nd, nm), dtype=np.float64)
    rc = lib.orc_gmatrix(nx, ny, nz, dx, dy, dz, h, comps, G.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("orc_gmatrix: invalid arguments")
    return G


def box_field(mesh, comps: int, box_cells, density: float, stations=None) -> np.ndarray:
    """Field of one uniform box made of whole cells, from a single prism
    evaluation per station (superposition of Eq. 3 over the box's cells).

    box_cells = (l0, l1, m0, m1, n0, n1), half-open cell ranges.  Returns
    [ncomp][n_stations] (all stations, flattened p + nx q, if None)."""
    nx, ny, nz, dx, dy, dz, h = _geom(mesh)
    l0, l1, m0, m1, n0, n1 = box_cells
    lst = comp_list(comps)
    idx = np.arange(nx * ny) if stations is None else np.asarray(stations)
    out = np.zeros((len(lst), idx.size))
    box = (l0 * dx, l1 * dx, m0 * dy, m1 * dy, n0 * dz, n1 * dz)
    for s, st in enumerate(idx):
        p, q = int(st) % nx, int(st) // nx
        v = prism(((p + 0.5) * dx, (q + 0.5) * dy, -h), box)
        out[:, s] = v[lst] * density
    return out


def forward3d(mesh, comps: int, rho: np.ndarray, stations=None, nthreads=None) -> np.ndarray:
    """Equal-dimension variant (Sec. 2.2, Eqs. 10-11): direct summation with
    a station at the centre of every cell.  mesh = (nx, ny, nz, dx, dy, dz,
    h), h unused; rho is [nz][ny][nx]; ``stations`` an optional list of
    station indices p + nx q + nx ny t.  Returns [ncomp][nz][ny][nx] (all
    stations) or [ncomp][n_stations]."""
    lib = _load()
    nx, ny, nz, dx, dy, dz, _ = _geom(mesh)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(nz, ny, nx)
    full = stations is None
    idx = np.arange(nx * ny * nz, dtype=np.int32) if full else np.ascontiguousarray(stations, dtype=np.int32)
    nc = len(comp_list(comps))
    out = np.zeros((nc, idx.size), dtype=np.float64)
    rc = lib.orc_forward3d(nx, ny, nz, dx, dy, dz, comps, rho.ctypes.data_as(ctypes.c_void_p), int(idx.size),
                           idx.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                           int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("orc_forward3d: invalid arguments")
    return out.reshape(nc, nz, ny, nx) if full else out


def adjoint3d(mesh, comps: int, resid: np.ndarray, cells=None, nthreads=None) -> np.ndarray:
    """Equal-dimension variant: (G^T r)_j = sum_c sum_i G_c(i, j) r_c(i) over
    the stations at cell centres.  resid is [ncomp][nz][ny][nx]; ``cells`` an
    optional list of cell indices.  Returns [nz][ny][nx] or [n_cells]."""
    lib = _load()
    nx, ny, nz, dx, dy, dz, _ = _geom(mesh)
    nc = len(comp_list(comps))
    resid = np.ascontiguousarray(resid, dtype=np.float64).reshape(nc, nz, ny, nx)
    full = cells is None
    idx = np.arange(nx * ny * nz, dtype=np.int32) if full else np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros(idx.size, dtype=np.float64)
    rc = lib.orc_adjoint3d(nx, ny, nz, dx, dy, dz, comps, resid.ctypes.data_as(ctypes.c_void_p), int(idx.size),
                           idx.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                           int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("orc_adjoint3d: invalid arguments")
    return out.reshape(nz, ny, nx) if full else out


def gmatrix3d(mesh, comps: int) -> np.ndarray:
    """Equal-dimension variant: explicit G[c][i][j], station i at the centre
    of cell i, for tiny meshes."""
    lib = _load()
    nx, ny, nz, dx, dy, dz, _ = _geom(mesh)
    nc = len(comp_list(comps))
    nm = nx * ny * nz
    if nc * nm * nm > 50_000_000:
        raise ValueError("gmatrix3d is for tiny meshes only")
    G = np.zeros((nc, nm, nm), dtype=np.float64)
    rc = lib.orc_gmatrix3d(nx, ny, nz, dx, dy, dz, comps, G.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("orc_gmatrix3d: invalid arguments")
    return G
