"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

This module holds no arithmetic of the LDG method: it only lays out meshes
(vertex coordinates, vertex ids, element order) and draws seeded random vectors
and parameter sets. Both the product path and the oracle receive exactly these
arrays and build everything else (connectivity, geometry, bases) themselves.

Mesh convention
---------------
* ``xyz``  float64 ``[E][nv][nd]``: each element's own vertex coordinates. On a
  periodic mesh the elements across the seam keep unwrapped coordinates.
* ``vid``  int64 ``[E][nv]``: topological vertex ids; on periodic meshes the
  vertices that the period identifies share one id, which is how face
  neighbours across the seam are found.
* Vertex order: quadrilaterals and hexahedra list their vertices in
  lexicographic (tensor) order, x fastest; triangles counter-clockwise.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TRI, QUAD, HEX = 0, 1, 2
NV = {TRI: 3, QUAD: 4, HEX: 8}
ND = {TRI: 2, QUAD: 2, HEX: 3}


@dataclass
class Mesh:
    etype: int
    xyz: np.ndarray      # [E][nv][nd] float64
    vid: np.ndarray      # [E][nv] int64
    name: str = ""

    @property
    def n_elem(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def nd(self) -> int:
        return ND[self.etype]


def _grid_ids(n, periodic):
    """Vertex id of grid point (i, j[, k]) with periodic identification."""
    dims = [ni if per else ni + 1 for ni, per in zip(n, periodic)]

    def vid(*ijk):
        idx = 0
        stride = 1
        for a, (ni, per) in enumerate(zip(n, periodic)):
            ia = ijk[a] % ni if per else ijk[a]
            idx += ia * stride
            stride *= dims[a]
        return idx
    return vid


def quad_box(n: int | tuple, lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(False, False),
             affine: np.ndarray | None = None) -> Mesh:
    """n[0] x n[1] uniform quadrilaterals of the box [lo, hi], x fastest.

    ``affine`` (2x2) optionally shears the whole mesh; elements stay parallelograms.
    """
    nx, ny = (n, n) if np.isscalar(n) else n
    hx = (hi[0] - lo[0]) / nx
    hy = (hi[1] - lo[1]) / ny
    vid = _grid_ids((nx, ny), periodic)
    xyz = np.empty((nx * ny, 4, 2))
    ids = np.empty((nx * ny, 4), dtype=np.int64)
    e = 0
    for j in range(ny):
        for i in range(nx):
            for v, (di, dj) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
                xyz[e, v] = (lo[0] + (i + di) * hx, lo[1] + (j + dj) * hy)
                ids[e, v] = vid(i + di, j + dj)
            e += 1
    if affine is not None:
        xyz = xyz @ np.asarray(affine, dtype=np.float64).T
    return Mesh(QUAD, xyz, ids, f"quad{nx}x{ny}")


def hex_box(n: int | tuple, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
            periodic=(False, False, False), affine: np.ndarray | None = None) -> Mesh:
    """n^3 uniform hexahedra of the box [lo, hi], x fastest then y then z."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    h = [(hi[a] - lo[a]) / m for a, m in enumerate((nx, ny, nz))]
    vid = _grid_ids((nx, ny, nz), periodic)
    E = nx * ny * nz
    # vectorised layout of the same definition as quad_box
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    xyz = np.empty((E, 8, 3))
    ids = np.empty((E, 8), dtype=np.int64)
    dims = [m if per else m + 1 for m, per in zip((nx, ny, nz), periodic)]
    for v in range(8):
        di, dj, dk = v & 1, (v >> 1) & 1, (v >> 2) & 1
        xyz[:, v, 0] = lo[0] + (i + di) * h[0]
        xyz[:, v, 1] = lo[1] + (j + dj) * h[1]
        xyz[:, v, 2] = lo[2] + (k + dk) * h[2]
        ii = (i + di) % nx if periodic[0] else i + di
        jj = (j + dj) % ny if periodic[1] else j + dj
        kk = (k + dk) % nz if periodic[2] else k + dk
        ids[:, v] = ii + dims[0] * (jj + dims[1] * kk)
    if affine is not None:
        xyz = xyz @ np.asarray(affine, dtype=np.float64).T
    del vid
    return Mesh(HEX, xyz, ids, f"hex{nx}x{ny}x{nz}")


def tri_square(n: int, lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(False, False),
               affine: np.ndarray | None = None) -> Mesh:
    """n x n squares of [lo, hi], each split along its (x_i, y_j)-(x_{i+1}, y_{j+1})
    diagonal into two counter-clockwise triangles: 2 n^2 elements."""
    hx = (hi[0] - lo[0]) / n
    hy = (hi[1] - lo[1]) / n
    vid = _grid_ids((n, n), periodic)
    xyz = np.empty((2 * n * n, 3, 2))
    ids = np.empty((2 * n * n, 3), dtype=np.int64)
    e = 0
    for j in range(n):
        for i in range(n):
            a, b, c, d = (i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)
            for tri in ((a, b, c), (a, c, d)):
                for v, (ii, jj) in enumerate(tri):
                    xyz[e, v] = (lo[0] + ii * hx, lo[1] + jj * hy)
                    ids[e, v] = vid(ii, jj)
                e += 1
    if affine is not None:
        xyz = xyz @ np.asarray(affine, dtype=np.float64).T
    return Mesh(TRI, xyz, ids, f"tri{n}x{n}")


def random_vector(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded N(0, scale^2) float64 vector (numpy PCG64)."""
    return np.random.default_rng(seed).standard_normal(n) * scale


def random_euler_state(n_elem: int, npe: int, seed: int, amp: float = 0.1) -> np.ndarray:
    """Seeded conservative Euler state [E][4][npe]: density and pressure near 1,
    velocity near (1, 1), perturbed by ``amp``-sized uniform noise (gamma = 1.4)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + amp * rng.uniform(-1, 1, (n_elem, npe))
    vx = 1.0 + amp * rng.uniform(-1, 1, (n_elem, npe))
    vy = 1.0 + amp * rng.uniform(-1, 1, (n_elem, npe))
    pr = 1.0 + amp * rng.uniform(-1, 1, (n_elem, npe))
    u = np.empty((n_elem, 4, npe))
    u[:, 0] = rho
    u[:, 1] = rho * vx
    u[:, 2] = rho * vy
    u[:, 3] = pr / 0.4 + 0.5 * rho * (vx * vx + vy * vy)
    return u.reshape(-1)


def batch_instances(n_inst: int = 256, seed: int = 20221):
    """Parameter draws of the batched convection-diffusion sweep: kappa log-uniform
    on [1e-3, 1e-1], beta angle uniform on [0, 2 pi) with |beta| = 1, quad mesh side
    uniform in {8, 16, 32, 64} and p uniform in {2, 3, 4}."""
    rng = np.random.default_rng(seed)
    kappa = 10.0 ** rng.uniform(-3, -1, n_inst)
    ang = rng.uniform(0, 2 * np.pi, n_inst)
    side = rng.choice([8, 16, 32, 64], n_inst)
    p = rng.choice([2, 3, 4], n_inst)
    return [dict(kappa=float(kappa[i]), beta=(float(np.cos(ang[i])), float(np.sin(ang[i]))),
                 side=int(side[i]), p=int(p[i])) for i in range(n_inst)]
