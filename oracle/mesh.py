"""Oracle of the per-phase interface meshes (the paper's isosurface output of each phase,
Section 3.2), in plain numpy, FP64.

TEST INFRASTRUCTURE ONLY: loaded by the tests, never by the product library; it shares no code
with the CUDA path.

The isosurface phi_a = iso of one phase field is extracted by marching tetrahedra over the grid of
cell centres:

* a cube has the 8 cell centres (i + a, j + b, k + c), a, b, c in {0, 1}, as corners; corner n =
  a + 2 b + 4 c.  Cubes wrap periodically in x and y (the corner value of i + 1 = nx is that of
  column 0, its position stays nx) and not in z: nx * ny * (nz - 1) cubes, in the order
  c = (k ny + j) nx + i.
* each cube is cut into the six tetrahedra of its Kuhn triangulation: for each permutation
  (s1, s2, s3) of the axes, the tetrahedron corner 0 -> + e_s1 -> + e_s2 -> corner 7, the
  permutations in lexicographic order.  Neighbouring cubes cut their shared faces the same way, so
  the surface has no cracks.
* a corner is inside when its value is >= iso.  A tetrahedron with 1 (or 3) inside corners gives one
  triangle through the three edges from the lone corner to the others (taken in increasing corner
  order); with 2 inside corners a, b (a < b) and outside c, d (c < d), the quad through the edges
  a-c, a-d, b-d, b-c, as the triangles (ac, ad, bd) and (ac, bd, bc).  On an edge from an inside
  corner p_in to an outside corner p_out the vertex is p_in + t (p_out - p_in), t = (iso - f_in) /
  (f_out - f_in).
* a triangle is oriented so that its normal (v1 - v0) x (v2 - v0) points from the tetrahedron's
  inside corners to its outside ones (toward lower phi_a): if the normal's product with (mean of the
  outside corners - mean of the inside corners) is negative, v1 and v2 are swapped.

Positions are in units of dx, the cell centre of cell (i, j, k) at (i + 1/2, j + 1/2, k + 1/2 + off)
with off the window offset.  Output: triangles (T, 3, 3), ordered by cube, then tetrahedron, then
triangle within the tetrahedron.
"""
from __future__ import annotations

import itertools

import numpy as np

# corner positions (a, b, c) of corner n = a + 2b + 4c
CORNERS = np.array([[n & 1, (n >> 1) & 1, (n >> 2) & 1] for n in range(8)], dtype=np.int64)
# the six Kuhn tetrahedra: corner 0, then the axes of a permutation added one by one
TETS = []
for perm in itertools.permutations(range(3)):
    v = [0]
    pos = [0, 0, 0]
    for ax in perm:
        pos[ax] = 1
        v.append(pos[0] + 2 * pos[1] + 4 * pos[2])
    TETS.append(v)
TETS = np.array(TETS, dtype=np.int64)


def tet_triangles(p, f, iso):
    """Triangles of one tetrahedron: corner positions p (4, 3), values f (4,) -> list of (3, 3)
    arrays (the rules of the module docstring)."""
    inside = [q for q in range(4) if f[q] >= iso]
    outside = [q for q in range(4) if f[q] < iso]

    def vert(a, b):  # a inside, b outside
        t = (iso - f[a]) / (f[b] - f[a])
        return p[a] + t * (p[b] - p[a])

    tris = []
    if len(inside) == 1:
        s = inside[0]
        tris.append([vert(s, o) for o in outside])
    elif len(inside) == 3:
        s = outside[0]
        tris.append([vert(q, s) for q in inside])
    elif len(inside) == 2:
        a, b = inside
        c, d = outside
        ac, ad, bd, bc = vert(a, c), vert(a, d), vert(b, d), vert(b, c)
        tris.append([ac, ad, bd])
        tris.append([ac, bd, bc])
    if tris:
        ci = p[inside].mean(axis=0)
        co = p[outside].mean(axis=0)
        out = []
        for tr in tris:
            v0, v1, v2 = (np.asarray(x, dtype=np.float64) for x in tr)
            nrm = np.cross(v1 - v0, v2 - v0)
            if np.dot(nrm, co - ci) < 0:
                v1, v2 = v2, v1
            out.append(np.stack([v0, v1, v2]))
        return out
    return []


def _corner_values(f: np.ndarray, k0: int, k1: int) -> np.ndarray:
    """Corner values (8, k1 - k0, ny, nx) of the cubes of layers k0 .. k1-1."""
    nz, ny, nx = f.shape
    cv = np.empty((8, k1 - k0, ny, nx))
    for n, (a, b, c) in enumerate(CORNERS):
        cv[n] = np.roll(np.roll(f[k0 + c:k1 + c], -b, axis=1), -a, axis=2)
    return cv


def _cube_triangles(vals, base, iso):
    tris = []
    for tet in TETS:
        p = base[None, :] + CORNERS[tet].astype(np.float64)
        tris.extend(tet_triangles(p, vals[tet], iso))
    return tris


def interface_mesh(field: np.ndarray, iso: float = 0.5, off: float = 0.0) -> np.ndarray:
    """Triangles (T, 3, 3) of the isosurface field = iso of a (nz, ny, nx) scalar field (one phase
    field), by the rules of the module docstring.  Plain loops over the cubes that the surface
    crosses; the crossing test itself is vectorised."""
    f = np.asarray(field, dtype=np.float64)
    nz, ny, nx = f.shape
    if nz < 2:
        return np.zeros((0, 3, 3))
    cv = _corner_values(f, 0, nz - 1)
    ins = cv >= iso
    crossed = ins.any(axis=0) & ~ins.all(axis=0)
    tris = []
    for k, j, i in zip(*np.nonzero(crossed)):  # C order: the cube order c = (k ny + j) nx + i
        tris.extend(_cube_triangles(cv[:, k, j, i], np.array([i + 0.5, j + 0.5, k + 0.5 + off]), iso))
    return np.array(tris).reshape(-1, 3, 3)


def cube_triangles(field: np.ndarray, iso: float, off: float, i: int, j: int, k: int) -> np.ndarray:
    """Triangles (t, 3, 3) of the single cube (i, j, k), 0 <= k < nz - 1: the entries of
    interface_mesh that this cube contributes, in the same order."""
    f = np.asarray(field, dtype=np.float64)
    nz, ny, nx = f.shape
    vals = np.array([f[k + c, (j + b) % ny, (i + a) % nx] for a, b, c in CORNERS])
    return np.array(_cube_triangles(vals, np.array([i + 0.5, j + 0.5, k + 0.5 + off]), iso)).reshape(-1, 3, 3)


def cube_counts(field: np.ndarray, iso: float, planes_per_chunk: int = 64) -> np.ndarray:
    """Triangles per cube, (nz - 1, ny, nx) int64: for each tetrahedron, 1 with one or three inside
    corners, 2 with two, 0 otherwise (the counts of tet_triangles, vectorised over the cubes and
    taken a few layers at a time so that large fields fit in memory)."""
    f = np.asarray(field)
    nz, ny, nx = f.shape
    out = np.zeros((max(nz - 1, 0), ny, nx), dtype=np.int64)
    for k0 in range(0, nz - 1, planes_per_chunk):
        k1 = min(nz - 1, k0 + planes_per_chunk)
        ins = _corner_values(np.asarray(f[k0:k1 + 1], dtype=np.float64), 0, k1 - k0) >= iso
        for tet in TETS:
            n_in = ins[tet].sum(axis=0)
            out[k0:k1] += np.where(n_in == 2, 2, np.where((n_in == 1) | (n_in == 3), 1, 0))
    return out


def mesh_area(tris: np.ndarray) -> float:
    return float(0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1).sum())


def mesh_volume(tris: np.ndarray) -> float:
    """Signed enclosed volume by the divergence theorem (positive for outward normals)."""
    return float(np.einsum("ij,ij->i", tris[:, 0], np.cross(tris[:, 1], tris[:, 2])).sum() / 6.0)


def weld(tris: np.ndarray, decimals: int = 9):
    """Vertices merged by their rounded coordinates: (vertex array, (T, 3) index array)."""
    flat = np.round(tris.reshape(-1, 3), decimals)
    verts, idx = np.unique(flat, axis=0, return_inverse=True)
    return verts, idx.reshape(-1, 3)
