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

Curved elements additionally carry
* ``pg``   the degree of the element map, and
* ``xgeo`` float64 ``[E][(pg+1)^2][2]`` (quadrilaterals): the physical positions of the
  (pg+1)^2 equispaced reference points (-1 + 2a/pg, -1 + 2b/pg), a fastest; or
  ``[E][(pg+1)(pg+2)/2][2]`` (triangles): the equispaced points (-1 + 2i/pg,
  -1 + 2j/pg), i + j <= pg, row by row (j outer); the element map is their
  degree-pg Lagrange interpolant. Shared edges are images of the same points,
  so neighbouring maps agree along them.
* ``bc``   uint8 ``[E][4]``: kind of each boundary face, 1 = solid wall,
  0 = data (Dirichlet or far field); ignored on interior faces.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TRI, QUAD, HEX, TET = 0, 1, 2, 3
NV = {TRI: 3, QUAD: 4, HEX: 8, TET: 4}
ND = {TRI: 2, QUAD: 2, HEX: 3, TET: 3}


@dataclass
class Mesh:
    etype: int
    xyz: np.ndarray      # [E][nv][nd] float64
    vid: np.ndarray      # [E][nv] int64
    name: str = ""
    pg: int = 0                       # curved elements: degree of the element map
    xgeo: np.ndarray | None = None    # [E][points][2] map points
    bc: np.ndarray | None = None      # [E][4] uint8 boundary kinds

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


def tri_annulus(n_r: int, n_t: int, pg: int, r0: float = 0.5, r1: float = 1.0) -> Mesh:
    """The annulus r0 <= r <= r1 as curved triangles of map degree pg: the (rho, theta)
    parameter grid of n_r layers by n_t sectors (theta periodic), each cell split along its
    diagonal into two triangles that are counter-clockwise in (rho, theta) and hence in
    the plane, each mapped by (rho, theta) -> (rho cos theta, rho sin theta) at its
    degree-pg lattice points. Shared edges are images of the same parameter points, so
    neighbouring maps agree along them. 2 n_r n_t elements; the corners' coordinates are
    the mapped vertices (no unwrapping: the seam's positions coincide)."""
    G = lambda P: np.stack([P[..., 0] * np.cos(P[..., 1]), P[..., 0] * np.sin(P[..., 1])], -1)
    vid = _grid_ids((n_r, n_t), (False, True))
    lat = [(i, j) for j in range(pg + 1) for i in range(pg + 1 - j)]   # the degree-pg node order
    E = 2 * n_r * n_t
    xyz = np.empty((E, 3, 2))
    ids = np.empty((E, 3), dtype=np.int64)
    xgeo = np.empty((E, len(lat), 2))
    par = lambda i, j: np.array([r0 + (r1 - r0) * i / n_r, 2.0 * np.pi * j / n_t])
    e = 0
    for j in range(n_t):
        for i in range(n_r):
            a, b, c, d = (i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)
            for tri in ((a, b, c), (a, c, d)):
                P = [par(*v) for v in tri]
                for v in range(3):
                    xyz[e, v] = G(P[v])
                    ids[e, v] = vid(*tri[v])
                pts = np.array([P[0] + (li / pg) * (P[1] - P[0]) + (lj / pg) * (P[2] - P[0]) for li, lj in lat])
                xgeo[e] = G(pts)
                e += 1
    return Mesh(TRI, xyz, ids, f"tri_annulus{n_r}x{n_t}", pg=pg, xgeo=xgeo)


def tri_unstructured(n: int, seed: int = 0, jitter: float = 0.25) -> Mesh:
    """Seeded triangle mesh of [0, 1]^2 with unstructured topology and shapes: n x n
    squares, each split along a diagonal drawn at random (vertex degrees 3 to 8), interior
    vertices moved by up to jitter cell sizes in each direction, each triangle's vertex
    list rotated at random (still counter-clockwise, so neighbours see their shared edge
    under every local numbering), and the elements shuffled: 2 n^2 affine triangles."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    pts = np.stack(np.meshgrid(np.linspace(0.0, 1.0, n + 1), np.linspace(0.0, 1.0, n + 1), indexing="ij"), -1)
    move = rng.uniform(-jitter * h, jitter * h, pts.shape)
    move[0, :] = move[-1, :] = 0.0
    move[:, 0] = move[:, -1] = 0.0
    pts = pts + move
    tris = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = (i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)
            pair = ((a, b, c), (a, c, d)) if rng.random() < 0.5 else ((a, b, d), (b, c, d))
            for t in pair:
                r = int(rng.integers(3))
                tris.append(t[r:] + t[:r])
    order = rng.permutation(len(tris))
    xyz = np.empty((len(tris), 3, 2))
    ids = np.empty((len(tris), 3), dtype=np.int64)
    for e, k in enumerate(order):
        for v, (ii, jj) in enumerate(tris[k]):
            xyz[e, v] = pts[ii, jj]
            ids[e, v] = ii + (n + 1) * jj
    return Mesh(TRI, xyz, ids, f"tri_unstructured{n}_s{seed}")


def _curved_quads(params, node_id, n0, n1, G, pg, bc_of, name):
    """Quadrilaterals of a structured n0 x n1 grid of parameter points: element (i, j)
    (i fastest) has corners params[i..i+1, j..j+1]; its map sends reference point
    (xi, eta) to G of the bilinear blend of its corner parameters, sampled at the
    equispaced points of degree pg."""
    t = np.linspace(-1.0, 1.0, pg + 1)
    a = np.tile(t, pg + 1)                  # first reference coordinate, fastest
    b = np.repeat(t, pg + 1)
    w = np.stack([(1 - a) * (1 - b), (1 + a) * (1 - b), (1 - a) * (1 + b), (1 + a) * (1 + b)], 1) / 4
    E = n0 * n1
    xyz = np.empty((E, 4, 2))
    ids = np.empty((E, 4), dtype=np.int64)
    xgeo = np.empty((E, (pg + 1) ** 2, 2))
    bc = np.zeros((E, 4), dtype=np.uint8)
    e = 0
    for j in range(n1):
        for i in range(n0):
            cor = [(i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1)]
            P = np.array([params[c] for c in cor])            # [4][2] parameters
            xyz[e] = G(P)
            ids[e] = [node_id(*c) for c in cor]
            xgeo[e] = G(w @ P)
            bc[e] = bc_of(i, j)
            e += 1
    return Mesh(QUAD, xyz, ids, name, pg=pg, xgeo=xgeo, bc=bc)


def warped_box(n: int | tuple, pg: int, lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(False, False),
               amp: float = 0.1) -> Mesh:
    """n[0] x n[1] curved quadrilaterals of the box [lo, hi]: the uniform grid moved by
    the smooth displacement amp L / (2 pi) sin(2 pi X) sin(2 pi Y) in each direction
    (X, Y the box coordinates scaled to [0, 1]). The displacement vanishes on the box
    boundary and is periodic, so periodic meshes stay periodic."""
    nx, ny = (n, n) if np.isscalar(n) else n
    L = np.array(hi, dtype=np.float64) - np.array(lo, dtype=np.float64)
    params = {(i, j): (lo[0] + i * L[0] / nx, lo[1] + j * L[1] / ny) for j in range(ny + 1) for i in range(nx + 1)}

    def G(P):
        P = np.atleast_2d(P)
        X = (P[:, 0] - lo[0]) / L[0]
        Y = (P[:, 1] - lo[1]) / L[1]
        s = amp / (2 * np.pi) * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
        return np.stack([P[:, 0] + L[0] * s, P[:, 1] + L[1] * s], 1)
    vid = _grid_ids((nx, ny), periodic)
    return _curved_quads(params, vid, nx, ny, G, pg, lambda i, j: (0, 0, 0, 0), f"warped{nx}x{ny}")


def o_grid(n_r: int, n_theta: int, pg: int, r0: float = 0.5, outer=("rect", (-10.0, 30.0, -10.0, 10.0)),
           first: float | None = None, jitter: float = 0.0, seed: int = 7, wall: bool = True,
           outer_wall: bool = False) -> Mesh:
    """Curved quadrilaterals between the circle of radius r0 about the origin and an
    outer boundary: ("circle", R) or ("rect", (x0, x1, y0, y1)) around the origin.

    Parameter grid: s_j in [0, 1] across the layer (j = 0 on the circle) and the angle
    theta_i = 2 pi i / n_theta. A point (s, theta) lies on the ray at angle theta,
    a fraction s of the way from the circle to the outer boundary. With ``first`` the
    s-spacing grows geometrically from a first layer of that physical thickness
    (advancing layers); otherwise it is uniform. ``jitter`` moves every parameter
    point off both boundaries by up to +- jitter/2 of the local spacing in each
    direction (seeded, numpy PCG64). The first reference axis runs across the layer
    (outward), the second along theta, so every element is positively oriented.
    Faces on the circle are walls when ``wall`` is set; outer faces carry data unless
    ``outer_wall`` is set."""
    kind, spec = outer

    def radius(th):
        c, s = np.cos(th), np.sin(th)
        if kind == "circle":
            return np.full_like(th, float(spec))
        x0, x1, y0, y1 = spec
        with np.errstate(divide="ignore", invalid="ignore"):
            tx = np.where(c > 0, x1 / c, np.where(c < 0, x0 / c, np.inf))
            ty = np.where(s > 0, y1 / s, np.where(s < 0, y0 / s, np.inf))
        return np.minimum(tx, ty)

    if first is None:
        sj = np.linspace(0.0, 1.0, n_r + 1)
    else:
        # thickness of the layer along the ray with the smallest span sets the growth
        span = float(radius(np.linspace(0, 2 * np.pi, 721)).min() - r0)
        h0 = first / span
        lo_g, hi_g = 1.0 + 1e-12, 2.0
        for _ in range(200):   # bisection for the ratio g with h0 (g^n - 1) / (g - 1) = 1
            g = 0.5 * (lo_g + hi_g)
            if h0 * (g ** n_r - 1) / (g - 1) > 1.0:
                hi_g = g
            else:
                lo_g = g
        sj = np.concatenate([[0.0], np.cumsum(h0 * g ** np.arange(n_r))])
        sj /= sj[-1]
    rng = np.random.default_rng(seed)
    params = {}
    for j in range(n_r + 1):
        ds = (sj[min(j + 1, n_r)] - sj[max(j - 1, 0)]) / 2
        for i in range(n_theta):
            s, th = sj[j], 2 * np.pi * i / n_theta
            if jitter and 0 < j < n_r:
                s += jitter * ds * (rng.uniform() - 0.5)
                th += jitter * (2 * np.pi / n_theta) * (rng.uniform() - 0.5)
            params[(j, i)] = (s, th)
    for j in range(n_r + 1):      # the seam: the same points one turn on
        s, th = params[(j, 0)]
        params[(j, n_theta)] = (s, th + 2 * np.pi)

    def G(P):
        P = np.atleast_2d(P)
        s, th = P[:, 0], P[:, 1]
        r = r0 + s * (radius(th) - r0)
        return np.stack([r * np.cos(th), r * np.sin(th)], 1)

    def node_id(j, i):
        return (i % n_theta) + n_theta * j
    # element (j, i): first reference axis across the layer (j), second along theta (i)
    par = {(j, i): params[(j, i)] for j in range(n_r + 1) for i in range(n_theta + 1)}
    m = _curved_quads(par, node_id, n_r, n_theta, G, pg,
                      lambda j, i: (1 if (wall and j == 0) else 0, 1 if (outer_wall and j == n_r - 1) else 0, 0, 0),
                      f"ogrid{n_r}x{n_theta}")
    # elements ordered with theta fastest for locality along the layers
    order = np.arange(n_r * n_theta).reshape(n_theta, n_r).T.ravel()
    return Mesh(QUAD, m.xyz[order], m.vid[order], m.name, pg=pg, xgeo=m.xgeo[order], bc=m.bc[order])


def cylinder_mesh(n_r: int = 100, n_theta: int = 400, pg: int = 3, seed: int = 7) -> Mesh:
    """Flow past a cylinder: radius 0.5 about the origin in [-10, 30] x [-10, 10],
    n_r x n_theta curved quadrilaterals (40,000 by default) in advancing layers from a
    first layer of thickness 0.01, interior nodes jittered by +- 10% of the spacing."""
    return o_grid(n_r, n_theta, pg, 0.5, ("rect", (-10.0, 30.0, -10.0, 10.0)), first=0.01, jitter=0.2,
                  seed=seed)


def tet_cube(n: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic=(False, False, False),
             affine: np.ndarray | None = None) -> Mesh:
    """n^3 cubes of the box [lo, hi], each split into the 6 tetrahedra that share its
    (0,0,0)-(1,1,1) diagonal (one per monotone path along the cube's edges), so that
    neighbouring cubes' faces match: 6 n^3 elements. Each tetrahedron's vertices are
    ordered so that its three edges from the first vertex are right-handed."""
    h = [(hi[a] - lo[a]) / n for a in range(3)]
    vid = _grid_ids((n, n, n), periodic)
    paths = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    E = 6 * n ** 3
    xyz = np.empty((E, 4, 3))
    ids = np.empty((E, 4), dtype=np.int64)
    e = 0
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for path in paths:
                    corner = [0, 0, 0]
                    verts = [tuple(corner)]
                    for ax in path:
                        corner[ax] += 1
                        verts.append(tuple(corner))
                    pts = [np.array([lo[0] + (i + a) * h[0], lo[1] + (j + b) * h[1], lo[2] + (k + c) * h[2]])
                           for a, b, c in verts]
                    vv = [vid(i + a, j + b, k + c) for a, b, c in verts]
                    if np.linalg.det(np.stack([pts[1] - pts[0], pts[2] - pts[0], pts[3] - pts[0]])) < 0:
                        pts[1], pts[2] = pts[2], pts[1]
                        vv[1], vv[2] = vv[2], vv[1]
                    xyz[e] = pts
                    ids[e] = vv
                    e += 1
    if affine is not None:
        xyz = xyz @ np.asarray(affine, dtype=np.float64).T
    return Mesh(TET, xyz, ids, f"tet{n}")


def tet_unstructured(n: int, seed: int = 0, jitter: float = 0.15) -> Mesh:
    """Seeded tetrahedral mesh of [0, 1]^3 with distorted shapes and no element order:
    tet_cube(n) with every interior vertex moved by up to jitter cell sizes in each
    direction (right-handed vertex order restored where needed) and the elements
    shuffled: 6 n^3 affine tetrahedra."""
    rng = np.random.default_rng(seed)
    base = tet_cube(n)
    pos = {}
    for e in range(base.n_elem):
        for v in range(4):
            pos.setdefault(int(base.vid[e, v]), base.xyz[e, v].copy())
    h = 1.0 / n
    moved = {}
    for vid_ in sorted(pos):
        x = pos[vid_]
        inner = np.all((x > 0.5 * h) & (x < 1.0 - 0.5 * h))
        moved[vid_] = x + (rng.uniform(-jitter * h, jitter * h, 3) if inner else 0.0)
    order = rng.permutation(base.n_elem)
    xyz = np.empty((base.n_elem, 4, 3))
    ids = np.empty((base.n_elem, 4), dtype=np.int64)
    for e, k in enumerate(order):
        vv = [int(t) for t in base.vid[k]]
        pts = [moved[t] for t in vv]
        if np.linalg.det(np.stack([pts[1] - pts[0], pts[2] - pts[0], pts[3] - pts[0]])) < 0:
            pts[1], pts[2] = pts[2], pts[1]
            vv[1], vv[2] = vv[2], vv[1]
        xyz[e] = pts
        ids[e] = vv
    return Mesh(TET, xyz, ids, f"tet_unstructured{n}_s{seed}")


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
