"""Triangle surface meshes for collocation BEM workloads.

Every mesh is returned as flat panels: vertices ``tri[N,3,3]`` (panel, corner,
xyz), collocation points ``centroid[N,3]`` and flat-triangle ``area[N]``, all
float64 and in a fixed, documented panel order.  The paper's own test model
(three conducting spheres plus their three image spheres, 64,800 triangles,
Section 4.1.2) is not available; these spheres and cubes of the same geometry
class stand in for it.
"""
from dataclasses import dataclass
import math
import numpy as np


@dataclass
class Mesh:
    tri: np.ndarray        # (N, 3, 3) float64 corners, outward orientation
    centroid: np.ndarray   # (N, 3) float64 collocation points (flat-triangle centroids)
    area: np.ndarray       # (N,) float64 flat-triangle areas
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.area.shape[0])


def _finish(tri: np.ndarray, name: str) -> Mesh:
    tri = np.ascontiguousarray(tri, dtype=np.float64)
    a, b, c = tri[:, 0, :], tri[:, 1, :], tri[:, 2, :]
    # centroid summed in a fixed order so every consumer sees the same doubles
    centroid = ((a + b) + c) / 3.0
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.sqrt((cr[:, 0] * cr[:, 0] + cr[:, 1] * cr[:, 1]) + cr[:, 2] * cr[:, 2])
    return Mesh(tri=tri, centroid=np.ascontiguousarray(centroid),
                area=np.ascontiguousarray(area), name=name)


def _icosahedron():
    """12 unit vertices (0,+-1,+-phi), (+-1,+-phi,0), (+-phi,0,+-1) in that order and
    the 20 faces, found as the vertex triples at mutual edge distance 2 (before
    normalisation), oriented outward and sorted lexicographically."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (1.0, -1.0):
        for s2 in (1.0, -1.0):
            v.append((0.0, s1, s2 * phi))
    for s1 in (1.0, -1.0):
        for s2 in (1.0, -1.0):
            v.append((s1, s2 * phi, 0.0))
    for s1 in (1.0, -1.0):
        for s2 in (1.0, -1.0):
            v.append((s1 * phi, 0.0, s2))
    v = np.array(v, dtype=np.float64)
    n = len(v)
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    adj = np.abs(d2 - 4.0) < 1e-9
    faces = []
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    a, b, c = v[i], v[j], v[k]
                    if np.dot(np.cross(b - a, c - a), a + b + c) > 0:
                        faces.append((i, j, k))
                    else:
                        faces.append((i, k, j))
    assert len(faces) == 20
    faces.sort()
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    return v, faces


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)) -> Mesh:
    """Unit icosphere refined ``level`` times, N = 20 * 4**level flat panels.

    Each refinement splits (a, b, c) into [a, ab, ca], [ab, b, bc], [ca, bc, c],
    [ab, bc, ca] with the edge midpoints pushed out to the unit sphere; children
    follow their parent's order.  The result is scaled by ``radius`` and shifted to
    ``center``."""
    if level < 0:
        raise ValueError("level must be >= 0")
    v, faces = _icosahedron()
    tri = np.stack([np.stack([v[a], v[b], v[c]]) for a, b, c in faces])  # (20,3,3)
    for _ in range(level):
        a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]

        def mid(p, q):
            m = 0.5 * (p + q)
            return m / np.linalg.norm(m, axis=1, keepdims=True)

        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        kids = np.stack([np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
                         np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1)], 1)
        tri = kids.reshape(-1, 3, 3)
    tri = tri * float(radius) + np.asarray(center, dtype=np.float64)[None, None, :]
    return _finish(tri, f"icosphere_L{level}")


def two_spheres(level: int, distance: float = 3.0) -> Mesh:
    """Two unit icospheres of the same level centred at (0,0,0) and (distance,0,0);
    sphere 1's panels come first."""
    s1 = icosphere(level)
    s2 = icosphere(level, center=(distance, 0.0, 0.0))
    return _finish(np.concatenate([s1.tri, s2.tri], 0), f"two_spheres_L{level}_d{distance:g}")


def _cube_faces_grid(n: int, lo: float, hi: float):
    """Six faces of the cube [lo,hi]^3, each an n x n grid of squares split along the
    diagonal from grid corner (i,j) to (i+1,j+1) into two right triangles, outward."""
    t = np.linspace(lo, hi, n + 1)
    out = []
    for axis in range(3):
        for side, val in ((0, lo), (1, hi)):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            for i in range(n):
                for j in range(n):
                    def P(ii, jj):
                        p = np.zeros(3)
                        p[axis] = val
                        p[u_ax] = t[ii]
                        p[v_ax] = t[jj]
                        return p
                    p00, p10, p11, p01 = P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)
                    for tri in ((p00, p10, p11), (p00, p11, p01)):
                        a, b, c = tri
                        nrm = np.cross(b - a, c - a)
                        outward = nrm[axis] * (1.0 if side == 1 else -1.0)
                        out.append((a, b, c) if outward > 0 else (a, c, b))
    return np.array(out, dtype=np.float64)


def unit_cube(n: int) -> Mesh:
    """Surface of the unit cube [0,1]^3, N = 12 n^2 right triangles."""
    if n < 1:
        raise ValueError("n must be >= 1")
    return _finish(_cube_faces_grid(n, 0.0, 1.0), f"unit_cube_n{n}")


def cube_sphere(n: int) -> Mesh:
    """The n x n-per-face grid of the cube [-1,1]^3 with every vertex pushed onto the
    unit sphere (N = 12 n^2 flat triangles)."""
    tri = _cube_faces_grid(n, -1.0, 1.0)
    tri = tri / np.linalg.norm(tri, axis=2, keepdims=True)
    return _finish(tri, f"cube_sphere_n{n}")


def uneven_batch_specs(count: int = 48, seed: int = 20191101, n_lo: int = 1280, n_hi: int = 20480):
    """Specs of an uneven batch of independent problems: N_target drawn log-uniformly
    in [n_lo, n_hi], a cube-surface or a cube-sphere with Bernoulli(1/2), and grid
    n = round(sqrt(N_target / 12)) so that N = 12 n^2."""
    from .rhs import splitmix64_uniform
    u = splitmix64_uniform(2 * count, seed)
    specs = []
    for k in range(count):
        nt = math.exp(math.log(n_lo) + u[2 * k] * (math.log(n_hi) - math.log(n_lo)))
        n = max(1, int(round(math.sqrt(nt / 12.0))))
        kind = "cube" if u[2 * k + 1] < 0.5 else "sphere"
        specs.append((kind, n))
    return specs


def mesh_from_spec(spec) -> Mesh:
    kind, n = spec
    return unit_cube(n) if kind == "cube" else cube_sphere(n)
