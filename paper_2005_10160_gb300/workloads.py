"""Seeded synthetic density meshes.

This module only draws inputs: meshes, densities, boxes and noise.  It holds
none of the forward model's arithmetic, so both the CUDA path and the CPU
oracle can consume what it makes.  Every generator is seeded (NumPy PCG64,
seed 20051016 + workload index) and returns NumPy arrays; densities are in
kg/m^3 with layout [nz][ny][nx] (x fastest, the cell order of Sec. 2.2).

Workloads (the paper's experiments are all synthetic, Secs. 3.1-3.2):

* ``small16``   16x16x4 cells of 10 m, stations 1 m above the top, density
                U(-500, 500) plus +800 on cells l, m in [6, 10), n in [1, 3).
* ``boxes256``  256x256x32 cells of 25x25x20 m, stations 5 m up, 20 random
                boxes of +-300 plus N(0, 20^2) noise.
* ``grf1024``   1024x1024x100 cells of 50x50x25 m, stations 10 m up, a
                smooth Gaussian random field (std 200, correlation length 20
                cells) stored as float32.
* ``boxes1024`` the grf1024 mesh with three seeded boxes of +300, -200 and
                +150 (a field known in closed form at every station).
* ``boxes512``  512x512x64 cubes of 20 m, stations 10 m up, three boxes of
                +400, -300 and +250.
* ``cube40``    the accuracy model of Sec. 3.1: a 300 m cube with its top at
                500 m and bottom at 800 m, +300 kg/m^3, on a 40x40x20 mesh
                of 50 m cells, stations 50 m above ground.
* serving meshes 64^2x16, 128^2x32, 256^2x32, 512^2x64 of 20 m cubes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 20051016


@dataclass(frozen=True)
class Mesh:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    h: float

    def tuple(self):
        return (self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.h)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_stations(self) -> int:
        return self.nx * self.ny


def rng_for(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


def random_boxes(mesh: Mesh, n_boxes: int, rng: np.random.Generator, magnitude=300.0):
    """Axis-aligned boxes of whole cells: uniform integer corner, extent in
    [1, n/4] per axis (clipped to the mesh), sign +-.  Returns a list of
    (l0, l1, m0, m1, n0, n1, density) with half-open cell ranges."""
    boxes = []
    dims = (mesh.nx, mesh.ny, mesh.nz)
    for _ in range(n_boxes):
        lo_hi = []
        for n in dims:
            ext = int(rng.integers(1, max(1, n // 4) + 1))
            c0 = int(rng.integers(0, n))
            lo_hi += [c0, min(n, c0 + ext)]
        sign = 1.0 if rng.random() < 0.5 else -1.0
        boxes.append((*lo_hi, sign * magnitude))
    return boxes


def paint_boxes(mesh: Mesh, boxes, dtype=np.float64) -> np.ndarray:
    rho = np.zeros((mesh.nz, mesh.ny, mesh.nx), dtype=np.float64)
    for (l0, l1, m0, m1, n0, n1, d) in boxes:
        rho[n0:n1, m0:m1, l0:l1] += d
    return rho.astype(dtype)


def small16():
    mesh = Mesh(16, 16, 4, 10.0, 10.0, 10.0, 1.0)
    rng = rng_for(1)
    rho = rng.uniform(-500.0, 500.0, size=(4, 16, 16))
    rho[1:3, 6:10, 6:10] += 800.0
    return mesh, rho


def boxes256(noise=True):
    mesh = Mesh(256, 256, 32, 25.0, 25.0, 20.0, 5.0)
    rng = rng_for(2)
    boxes = random_boxes(mesh, 20, rng, 300.0)
    rho = paint_boxes(mesh, boxes)
    if noise:
        rho += rng.normal(0.0, 20.0, size=rho.shape)
    return mesh, rho, boxes


def grf_mesh(nx=1024, ny=1024, nz=100):
    return Mesh(nx, ny, nz, 50.0, 50.0, 25.0, 10.0)


def grf1024(nx=1024, ny=1024, nz=100, corr_cells=20.0, std=200.0, device="cpu"):
    """Smooth Gaussian random field in float32: white N(0,1) noise, a
    separable Gaussian filter of standard deviation corr/sqrt(2) cells along
    each axis (applied spectrally, periodic), rescaled to the requested
    standard deviation.  Returns (mesh, torch.float32 tensor on ``device``)."""
    import torch

    mesh = grf_mesh(nx, ny, nz)
    rng = rng_for(3)
    white = rng.standard_normal(size=(nz, ny, nx), dtype=np.float32)
    t = torch.from_numpy(white).to(device)
    sig = corr_cells / np.sqrt(2.0)
    spec = torch.fft.rfftn(t)
    fz = torch.fft.fftfreq(nz, device=device, dtype=torch.float32)
    fy = torch.fft.fftfreq(ny, device=device, dtype=torch.float32)
    fx = torch.fft.rfftfreq(nx, device=device, dtype=torch.float32)
    c = -2.0 * (np.pi ** 2) * sig ** 2
    spec *= torch.exp(c * fz * fz)[:, None, None]
    spec *= torch.exp(c * fy * fy)[None, :, None]
    spec *= torch.exp(c * fx * fx)[None, None, :]
    field = torch.fft.irfftn(spec, s=(nz, ny, nx))
    field = field - field.mean()
    field = field * (std / field.std())
    return mesh, field.to(torch.float32).contiguous()


def boxes1024():
    """The grf1024 mesh (1024x1024x100 cells of 50x50x25 m, stations 10 m
    up) holding three seeded boxes of +300, -200 and +150 kg/m^3 (extents up
    to a quarter of each axis): a density whose field at every station is the
    sum of three whole-box closed forms."""
    mesh = grf_mesh()
    rng = rng_for(6)
    boxes = []
    for d in (300.0, -200.0, 150.0):
        b = random_boxes(mesh, 1, rng, 1.0)[0]
        boxes.append((*b[:6], d))
    return mesh, paint_boxes(mesh, boxes, np.float32), boxes


def boxes512():
    mesh = Mesh(512, 512, 64, 20.0, 20.0, 20.0, 10.0)
    rng = rng_for(4)
    boxes = []
    for d in (400.0, -300.0, 250.0):
        b = random_boxes(mesh, 1, rng, 1.0)[0]
        boxes.append((*b[:6], d))
    return mesh, paint_boxes(mesh, boxes), boxes


def cube40():
    """Sec. 3.1: cube of 300 m, top 500 m, bottom 800 m, +300 kg/m^3, centred
    under the middle of a 40x40 station grid (50 m spacing, 50 m up)."""
    mesh = Mesh(40, 40, 20, 50.0, 50.0, 50.0, 50.0)
    box = (17, 23, 17, 23, 10, 16, 300.0)
    return mesh, paint_boxes(mesh, [box]), [box]


SERVING_SHAPES = ((64, 64, 16), (128, 128, 32), (256, 256, 32), (512, 512, 64))


def serving_mesh(i: int) -> Mesh:
    nx, ny, nz = SERVING_SHAPES[i]
    return Mesh(nx, ny, nz, 20.0, 20.0, 20.0, 10.0)


def serving_density(mesh: Mesh, rng: np.random.Generator, dtype=np.float32):
    return paint_boxes(mesh, random_boxes(mesh, 20, rng, 300.0), dtype)


def station_subset(mesh: Mesh, n: int, rng: np.random.Generator) -> np.ndarray:
    """n station indices p + nx q including the four corners and the centre."""
    nx, ny = mesh.nx, mesh.ny
    fixed = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, (ny // 2) * nx + nx // 2]
    fixed = list(dict.fromkeys(fixed))
    rest = rng.choice(nx * ny, size=max(0, n - len(fixed)), replace=False)
    out = list(fixed) + [int(v) for v in rest if int(v) not in fixed]
    return np.asarray(out[:n], dtype=np.int32)


def random_mesh_density(mesh: Mesh, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(-500.0, 500.0, size=(mesh.nz, mesh.ny, mesh.nx))
