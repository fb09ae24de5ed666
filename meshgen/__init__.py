"""Seeded synthetic triangle meshes for the sBHA/sBMDS pipeline.

This module only builds inputs: vertex positions (float64, n x 3, row-major) and
triangles (int32, f x 3).  It holds none of the method's arithmetic (no edge
lengths, cotangents, operators or distances) so that both the CUDA path and the
CPU oracle can be fed from it without sharing any of the method's code.

The paper evaluates on scanned meshes (Brain, Bunny, Dragon, TOSCA) that are not
available here; the generators below are synthetic stand-ins with the same
structure: closed or open 2-manifold triangle surfaces of valence about 6, with
seeded noise so that no two distances tie by symmetry.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64), which gives
the same stream on every platform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Mesh",
    "icosphere",
    "geodesic_sphere",
    "torus",
    "sphere_patch_bumps",
    "flat_grid",
    "mesh_batch",
    "workload",
    "WORKLOADS",
]


@dataclass
class Mesh:
    """A triangle mesh: ``xyz`` float64 (n, 3) and ``faces`` int32 (f, 3)."""

    xyz: np.ndarray
    faces: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def f(self) -> int:
        return int(self.faces.shape[0])

    def __post_init__(self):
        self.xyz = np.ascontiguousarray(self.xyz, dtype=np.float64)
        self.faces = np.ascontiguousarray(self.faces, dtype=np.int32)


def _icosahedron():
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # faces = convex hull of the 12 vertices, oriented outward
    from scipy.spatial import ConvexHull

    hull = ConvexHull(v)
    faces = []
    for tri in hull.simplices:
        a, b, c = (int(t) for t in tri)
        nrm = np.cross(v[b] - v[a], v[c] - v[a])
        if np.dot(nrm, v[a] + v[b] + v[c]) < 0:
            b, c = c, b
        faces.append((a, b, c))
    faces.sort()
    return v, np.array(faces, dtype=np.int64)


def icosphere(level: int, noise: float = 0.0, seed: int = 0) -> Mesh:
    """Recursive midpoint-subdivided icosahedron (n = 10*4^level + 2).

    Each level splits every triangle into four through its edge midpoints, which
    are pushed back onto the unit sphere.  ``noise`` is the standard deviation of
    a per-vertex radial factor r = 1 + N(0, noise) drawn from ``seed``.
    """
    v, faces = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            m = cache.get(key)
            if m is None:
                p = np.add(verts[a], verts[b]) * 0.5
                p = p / np.linalg.norm(p)
                verts.append(tuple(p))
                m = len(verts) - 1
                cache[key] = m
            return m

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = np.array(nf, dtype=np.int64)
    xyz = np.array(verts, dtype=np.float64)
    if noise > 0:
        rng = np.random.default_rng(seed)
        xyz = xyz * (1.0 + rng.normal(0.0, noise, size=(xyz.shape[0], 1)))
    return Mesh(xyz, faces.astype(np.int32), f"icosphere{level}")


def geodesic_sphere(freq: int, noise: float = 0.0, seed: int = 0) -> Mesh:
    """Class-I geodesic sphere of frequency ``freq`` (n = 10*freq^2 + 2).

    Every icosahedron face is cut into freq^2 triangles on a barycentric grid and
    the grid points are projected onto the unit sphere.  Points on shared edges
    are keyed by their exact integer barycentric weights over the icosahedron's
    vertex ids, so they are created once.
    """
    v0, f0 = _icosahedron()
    index: dict[tuple, int] = {}
    pts: list[np.ndarray] = []

    def vid(weights: dict[int, int]) -> int:
        key = tuple(sorted((k, w) for k, w in weights.items() if w))
        i = index.get(key)
        if i is None:
            p = sum(w * v0[k] for k, w in key) / float(freq)
            pts.append(p / np.linalg.norm(p))
            i = len(pts) - 1
            index[key] = i
        return i

    faces = []
    for a, b, c in f0:
        grid = {}
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                k = freq - i - j
                w: dict[int, int] = {}
                for vtx, wt in ((a, i), (b, j), (c, k)):
                    w[int(vtx)] = w.get(int(vtx), 0) + wt
                grid[(i, j)] = vid(w)
        for i in range(freq):
            for j in range(freq - i):
                p, q, r = grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]
                faces.append((p, q, r))
                if i + j + 1 < freq:
                    s = grid[(i + 1, j + 1)]
                    faces.append((q, s, r))
    xyz = np.array(pts, dtype=np.float64)
    faces = np.array(faces, dtype=np.int64)
    # orient outward
    nrm = np.cross(xyz[faces[:, 1]] - xyz[faces[:, 0]], xyz[faces[:, 2]] - xyz[faces[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, xyz[faces].sum(axis=1)) < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    if noise > 0:
        rng = np.random.default_rng(seed)
        xyz = xyz * (1.0 + rng.normal(0.0, noise, size=(xyz.shape[0], 1)))
    return Mesh(xyz, faces.astype(np.int32), f"geosphere{freq}")


def _grid_faces(nu: int, nv: int, wrap_u: bool, wrap_v: bool) -> np.ndarray:
    """Triangulate an nu x nv vertex grid (vertex id = i*nv + j), one diagonal per quad."""
    iu = nu if wrap_u else nu - 1
    iv = nv if wrap_v else nv - 1
    i, j = np.meshgrid(np.arange(iu), np.arange(iv), indexing="ij")
    i, j = i.ravel(), j.ravel()
    i1, j1 = (i + 1) % nu, (j + 1) % nv
    a, b, c, d = i * nv + j, i1 * nv + j, i1 * nv + j1, i * nv + j1
    f = np.empty((2 * a.size, 3), dtype=np.int64)
    f[0::2] = np.stack([a, b, c], axis=1)
    f[1::2] = np.stack([a, c, d], axis=1)
    return f


def _mean_incident_edge(xyz: np.ndarray, faces: np.ndarray) -> np.ndarray:
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    ln = np.linalg.norm(xyz[e[:, 0]] - xyz[e[:, 1]], axis=1)
    s = np.zeros(xyz.shape[0])
    c = np.zeros(xyz.shape[0])
    np.add.at(s, e[:, 0], ln)
    np.add.at(s, e[:, 1], ln)
    np.add.at(c, e[:, 0], 1)
    np.add.at(c, e[:, 1], 1)
    return s / c


def torus(nu: int = 250, nv: int = 200, R: float = 1.0, r: float = 0.3, jitter: float = 0.2, seed: int = 0) -> Mesh:
    """Torus on an nu x nv parameter grid, jittered per vertex.

    Vertex (i, j) sits at angles u = 2*pi*i/nu, v = 2*pi*j/nv.  Each vertex then moves
    by an isotropic 3-D Gaussian with standard deviation ``jitter`` times the mean
    length of its incident edges on the unjittered grid.
    """
    u = 2.0 * np.pi * np.arange(nu) / nu
    v = 2.0 * np.pi * np.arange(nv) / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    xyz = np.stack([(R + r * np.cos(V)) * np.cos(U), (R + r * np.cos(V)) * np.sin(U), r * np.sin(V)], axis=-1)
    xyz = xyz.reshape(-1, 3)
    faces = _grid_faces(nu, nv, True, True)
    if jitter > 0:
        h = _mean_incident_edge(xyz, faces)
        rng = np.random.default_rng(seed)
        xyz = xyz + rng.normal(0.0, 1.0, size=xyz.shape) * (jitter * h)[:, None]
    return Mesh(xyz, faces.astype(np.int32), f"torus{nu}x{nv}")


def sphere_patch_bumps(N: int = 448, nbumps: int = 20, seed: int = 2) -> Mesh:
    """Open, non-rigidly deformed surface: a gnomonic cube-face patch of the unit sphere.

    Grid point (i, j) has parameters u, v in [-pi/4, pi/4] and lies at
    normalize(tan u, tan v, 1).  ``nbumps`` Gaussian bumps push it along the normal:
    radius = 1 + sum_k a_k exp(-|p - c_k|^2 / (2 w_k^2)), amplitude a_k ~ U(0, 0.3),
    width w_k ~ U(0.05, 0.2), centres c_k drawn uniformly on the patch.
    """
    rng = np.random.default_rng(seed)
    t = np.linspace(-np.pi / 4, np.pi / 4, N)
    U, V = np.meshgrid(t, t, indexing="ij")
    p = np.stack([np.tan(U), np.tan(V), np.ones_like(U)], axis=-1).reshape(-1, 3)
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    amp = rng.uniform(0.0, 0.3, nbumps)
    wid = rng.uniform(0.05, 0.2, nbumps)
    cu = rng.uniform(-np.pi / 4, np.pi / 4, nbumps)
    cv = rng.uniform(-np.pi / 4, np.pi / 4, nbumps)
    c = np.stack([np.tan(cu), np.tan(cv), np.ones(nbumps)], axis=-1)
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    rad = np.ones(p.shape[0])
    for k in range(nbumps):
        d2 = np.sum((p - c[k]) ** 2, axis=1)
        rad += amp[k] * np.exp(-d2 / (2.0 * wid[k] ** 2))
    xyz = p * rad[:, None]
    faces = _grid_faces(N, N, False, False)
    return Mesh(xyz, faces.astype(np.int32), f"patch{N}")


def flat_grid(nx: int, ny: int, h: float = 1.0, jitter: float = 0.0, seed: int = 0) -> Mesh:
    """Flat nx x ny grid in the z = 0 plane with spacing ``h`` (open mesh, one diagonal per quad).

    ``jitter`` moves each vertex in-plane by N(0, jitter*h); z stays 0.
    """
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    xyz = np.stack([i.ravel() * h, j.ravel() * h, np.zeros(nx * ny)], axis=1).astype(np.float64)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        xyz[:, :2] += rng.normal(0.0, jitter * h, size=(nx * ny, 2))
    faces = _grid_faces(nx, ny, False, False)
    return Mesh(xyz, faces.astype(np.int32), f"grid{nx}x{ny}")


def mesh_batch(count: int = 64, nmin: int = 5000, nmax: int = 100000, seed: int = 1):
    """Meshes of uneven size: sizes log-uniform in [nmin, nmax] from ``seed``.

    Even positions are geodesic spheres (n = 10 f^2 + 2), odd positions tori with an
    aspect ratio of 5:4; each has its own noise seed (seed*1000 + position).
    """
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(nmin), np.log(nmax), count))
    out = []
    for k, s in enumerate(sizes):
        if k % 2 == 0:
            freq = max(2, int(round(math.sqrt((s - 2) / 10.0))))
            out.append(geodesic_sphere(freq, noise=0.01, seed=seed * 1000 + k))
        else:
            nv = max(8, int(round(math.sqrt(s * 0.8))))
            nu = max(8, int(round(s / nv)))
            out.append(torus(nu, nv, 1.0, 0.3, 0.2, seed=seed * 1000 + k))
    return out


def knn_graph(n: int, k: int = 6, seed: int = 0, dim: int = 2):
    """A generic graph: n points uniform in the unit square (or cube), each joined to its k nearest
    neighbours, edges made symmetric; lengths are the Euclidean distances.  Returns
    (rowptr int32, col int32, length float64, xyz float64 [n x 3])."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, dim))
    d2 = np.sum((pts[:, None, :] - pts[None, :, :]) ** 2, axis=2)
    np.fill_diagonal(d2, np.inf)
    nbr = np.argsort(d2, axis=1, kind="stable")[:, :k]
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in nbr[i]:
            adj[i].add(int(j))
            adj[int(j)].add(i)
    rowptr = np.zeros(n + 1, np.int32)
    cols, lens = [], []
    for i in range(n):
        js = sorted(adj[i])
        rowptr[i + 1] = rowptr[i] + len(js)
        cols += js
        lens += [float(np.sqrt(np.sum((pts[i] - pts[j]) ** 2))) for j in js]
    xyz = np.zeros((n, 3))
    xyz[:, :dim] = pts
    return rowptr, np.array(cols, np.int32), np.array(lens), xyz


def grid_graph(nx: int, ny: int):
    """The nx x ny 4-neighbour grid graph (vertex i + nx j), without lengths."""
    n = nx * ny
    rowptr = np.zeros(n + 1, np.int32)
    cols = []
    for j in range(ny):
        for i in range(nx):
            v = i + nx * j
            nb = []
            if j > 0:
                nb.append(v - nx)
            if i > 0:
                nb.append(v - 1)
            if i < nx - 1:
                nb.append(v + 1)
            if j < ny - 1:
                nb.append(v + nx)
            cols += nb
            rowptr[v + 1] = rowptr[v] + len(nb)
    return rowptr, np.array(cols, np.int32)


# Named workloads: the method's parameters with their meshes.  l = landmarks,
# p_row = operator nonzeros kept per row, k = embedding dimension.
WORKLOADS = {
    "icosphere3_l32": dict(mesh=lambda: icosphere(3, noise=0.01, seed=0), l=32, p_row=8, k=3, first=0),
    "torus250x200_l500": dict(mesh=lambda: torus(250, 200, 1.0, 0.3, 0.2, seed=0), l=500, p_row=16, k=3, first=0),
    "patch448_l2000": dict(mesh=lambda: sphere_patch_bumps(448, 20, seed=2), l=2000, p_row=16, k=3, first=0),
}


def workload(name: str):
    """Return (mesh, params) for a named workload."""
    w = dict(WORKLOADS[name])
    mesh = w.pop("mesh")()
    mesh.name = name
    return mesh, w
