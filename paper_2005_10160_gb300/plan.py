"""Torch-facing wrapper of the C ABI: a plan object whose forward and
adjoint take and return CUDA tensors.  It validates shapes, dtypes and
devices, then passes raw pointers and the current CUDA stream to
``libgravfft.so``; all arithmetic happens there.
"""
from __future__ import annotations

import torch

from . import capi


class Plan:
    """Resident kernel spectra of one mesh (Eqs. 19, 22) on the current CUDA
    device.

    mesh: (nx, ny, nz, dx, dy, dz, h) or an object with those attributes.
    components: OR of capi.GRAV_GZ ... GRAV_GY (at most 8).
    fp64: FP64 spectra and arithmetic (float64 tensors) instead of FP32.
    """

    def __init__(self, mesh, components: int = capi.GRAV_ALL6, fp64: bool = False):
        if hasattr(mesh, "tuple"):
            mesh = mesh.tuple()
        nx, ny, nz, dx, dy, dz, h = mesh
        self.mesh = (int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), float(h))
        self.components = int(components) & capi.GRAV_COMP_BITS
        self.fp64 = bool(fp64)
        if not torch.cuda.is_available():
            raise RuntimeError("libgravfft needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device())
        flags = self.components | (capi.GRAV_FP64_SPECTRAL if fp64 else 0)
        self._h = capi.grav_plan_create(*self.mesh, flags)
        self.ncomp = len(capi.comp_list(self.components))
        self.dtype = torch.float64 if fp64 else torch.float32
        info = capi.grav_plan_info(self._h)
        self.px, self.py = info.px, info.py
        self.spectra_bytes = int(info.spectra_bytes)
        self.workspace_bytes = int(info.workspace_bytes)
        self.nbytes = capi.grav_plan_bytes(self._h)

    @property
    def handle(self):
        return self._h

    @property
    def nx(self):
        return self.mesh[0]

    @property
    def ny(self):
        return self.mesh[1]

    @property
    def nz(self):
        return self.mesh[2]

    def _check(self, t: torch.Tensor, shape, name):
        if not isinstance(t, torch.Tensor) or t.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if t.dtype != self.dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous {self.dtype} of shape {tuple(shape)}, "
                             f"got {t.dtype} {tuple(t.shape)}")

    def _stream(self, stream):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def forward(self, rho: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """d_c = sum_n G_{c,n} rho_n (Eq. 21); rho [nz][ny][nx] -> [ncomp][ny][nx]."""
        nx, ny, nz = self.mesh[:3]
        self._check(rho, (nz, ny, nx), "rho")
        if out is None:
            out = torch.empty((self.ncomp, ny, nx), dtype=self.dtype, device=self.device)
        self._check(out, (self.ncomp, ny, nx), "out")
        capi.grav_forward(self._h, rho.data_ptr(), out.data_ptr(), self._stream(stream))
        return out

    def adjoint(self, r: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """sum_c G_c^T r_c; r [ncomp][ny][nx] -> [nz][ny][nx]."""
        nx, ny, nz = self.mesh[:3]
        self._check(r, (self.ncomp, ny, nx), "r")
        if out is None:
            out = torch.empty((nz, ny, nx), dtype=self.dtype, device=self.device)
        self._check(out, (nz, ny, nx), "out")
        capi.grav_adjoint(self._h, r.data_ptr(), out.data_ptr(), self._stream(stream))
        return out

    def close(self):
        if getattr(self, "_h", None):
            capi.grav_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan3D(Plan):
    """Equal-dimension plan (Sec. 2.2, Eqs. 10-11): a station at the centre
    of every cell; three-level circulant spectra resident on the current
    CUDA device.  mesh: (nx, ny, nz, dx, dy, dz[, h]) or an object with those
    attributes (h, if given, is not used)."""

    def __init__(self, mesh, components: int = capi.GRAV_ALL6, fp64: bool = False):
        if hasattr(mesh, "tuple"):
            mesh = mesh.tuple()
        nx, ny, nz, dx, dy, dz = mesh[:6]
        self.mesh = (int(nx), int(ny), int(nz), float(dx), float(dy), float(dz), 0.0)
        self.components = int(components) & capi.GRAV_COMP_BITS
        self.fp64 = bool(fp64)
        if not torch.cuda.is_available():
            raise RuntimeError("libgravfft needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device())
        flags = self.components | (capi.GRAV_FP64_SPECTRAL if fp64 else 0)
        self._h = capi.grav_plan_create3d(*self.mesh[:6], flags)
        self.ncomp = len(capi.comp_list(self.components))
        self.dtype = torch.float64 if fp64 else torch.float32
        info = capi.grav_plan_info(self._h)
        self.px, self.py, self.pz = info.px, info.py, info.pz
        self.spectra_bytes = int(info.spectra_bytes)
        self.workspace_bytes = int(info.workspace_bytes)
        self.nbytes = capi.grav_plan_bytes(self._h)

    def forward(self, rho: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """d_c at every cell centre; rho [nz][ny][nx] -> [ncomp][nz][ny][nx]."""
        nx, ny, nz = self.mesh[:3]
        self._check(rho, (nz, ny, nx), "rho")
        if out is None:
            out = torch.empty((self.ncomp, nz, ny, nx), dtype=self.dtype, device=self.device)
        self._check(out, (self.ncomp, nz, ny, nx), "out")
        capi.grav_forward3d(self._h, rho.data_ptr(), out.data_ptr(), self._stream(stream))
        return out

    def adjoint(self, r: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """sum_c G_c^T r_c; r [ncomp][nz][ny][nx] -> [nz][ny][nx]."""
        nx, ny, nz = self.mesh[:3]
        self._check(r, (self.ncomp, nz, ny, nx), "r")
        if out is None:
            out = torch.empty((nz, ny, nx), dtype=self.dtype, device=self.device)
        self._check(out, (nz, ny, nx), "out")
        capi.grav_adjoint3d(self._h, r.data_ptr(), out.data_ptr(), self._stream(stream))
        return out


def kernel_values(mesh, components: int, device=None, stream=None) -> torch.Tensor:
    """The FP64 kernel over the offset grid, [ncomp][nz][2ny-1][2nx-1] (Eq. 10)."""
    if hasattr(mesh, "tuple"):
        mesh = mesh.tuple()
    nx, ny, nz = (int(v) for v in mesh[:3])
    device = device or torch.device("cuda", torch.cuda.current_device())
    nc = len(capi.comp_list(components))
    K = torch.empty((nc, nz, 2 * ny - 1, 2 * nx - 1), dtype=torch.float64, device=device)
    s = stream if stream is not None else torch.cuda.current_stream(device)
    capi.grav_kernel_values(*mesh, components, K.data_ptr(), s.cuda_stream)
    return K
