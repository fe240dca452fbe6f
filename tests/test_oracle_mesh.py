"""Pins of the interface-mesh oracle (oracle/mesh.py: marching tetrahedra over the cell centres).

Each check is fixed by geometry, not by the oracle itself: the Kuhn tetrahedra tile the cube; every
vertex lies where the linear interpolant of the field equals iso; a planar front gives a flat mesh
of exactly the domain's cross-section; a sphere gives a closed, consistently outward-oriented
surface of Euler characteristic 2 whose enclosed volume and area approach the sphere's.
"""
import itertools

import numpy as np

from oracle import mesh as M


def test_kuhn_tetrahedra_tile_the_cube():
    assert M.TETS.shape == (6, 4)
    for tet in M.TETS:
        assert tet[0] == 0 and tet[3] == 7
        # a path of unit steps from corner 0 to corner 7: 6 such paths, one per axis order
        for a, b in zip(tet[:-1], tet[1:]):
            assert bin(int(a) ^ int(b)).count("1") == 1 and b > a
        p = M.CORNERS[tet]
        assert abs(round(np.linalg.det((p[1:] - p[0]).astype(float)))) == 1  # volume 1/6 each
    assert len({tuple(t) for t in M.TETS}) == 6
    # they tile the cube: random points lie in exactly one of them
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 1, size=(2000, 3))
    hits = np.zeros(len(pts), dtype=int)
    for tet in M.TETS:
        p = M.CORNERS[tet].astype(float)
        T = np.concatenate([p.T, np.ones((1, 4))])
        lam = np.linalg.solve(T, np.concatenate([pts.T, np.ones((1, len(pts)))]))
        hits += (lam > 0).all(axis=0)
    assert (hits == 1).all()


def test_every_inside_outside_pattern_of_a_tetrahedron():
    rng = np.random.default_rng(0)
    p = rng.uniform(0, 1, size=(4, 3))
    for pattern in itertools.product([False, True], repeat=4):
        f = np.where(pattern, rng.uniform(0.6, 1.0, 4), rng.uniform(0.0, 0.4, 4))
        tris = M.tet_triangles(p, f, 0.5)
        n_in = sum(pattern)
        assert len(tris) == {0: 0, 1: 1, 2: 2, 3: 1, 4: 0}[n_in]
        # the barycentric (linear) interpolant of f equals iso at every vertex
        T = np.concatenate([p.T, np.ones((1, 4))])
        for tr in tris:
            for v in tr:
                lam = np.linalg.solve(T, np.append(v, 1.0))
                assert abs(lam @ f - 0.5) < 1e-12
                assert lam.min() > -1e-12  # on the tetrahedron
            # oriented from the inside corners towards the outside ones
            nrm = np.cross(tr[1] - tr[0], tr[2] - tr[0])
            ci = p[np.array(pattern)].mean(axis=0)
            co = p[~np.array(pattern)].mean(axis=0)
            assert nrm @ (co - ci) >= 0


def test_planar_front_gives_a_flat_mesh_of_the_cross_section():
    nx, ny, nz, z0 = 7, 5, 12, 5.3
    zc = np.arange(nz) + 0.5
    f = np.clip((zc - z0) / 4.0 + 0.5, 0.0, 1.0)[:, None, None] * np.ones((nz, ny, nx))
    tris = M.interface_mesh(f, 0.5, off=0.0)
    assert len(tris) > 0
    assert np.abs(tris[:, :, 2] - z0).max() < 1e-12
    assert abs(M.mesh_area(tris) - nx * ny) < 1e-9
    # phi grows with z: the normals point down, towards lower phi
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert (nrm[:, 2] < 0).all()
    # the window offset moves the mesh rigidly
    tris2 = M.interface_mesh(f, 0.5, off=40.0)
    assert np.array_equal(tris2[:, :, :2], tris[:, :, :2]) and np.allclose(tris2[:, :, 2], tris[:, :, 2] + 40.0)


def test_front_across_the_periodic_boundary():
    nx, ny, nz = 16, 4, 6
    xc = np.arange(nx) + 0.5
    f = np.cos(2 * np.pi * xc / nx)[None, None, :] * np.ones((nz, ny, nx))
    tris = M.interface_mesh(f, 0.0)
    # two planes x = nx/4 and x = 3 nx/4 (the wrap cubes i = nx-1 reach x = nx + 1/2), each of area
    # ny * (nz - 1)
    assert abs(M.mesh_area(tris) - 2 * ny * (nz - 1)) < 1e-9
    xs = np.unique(np.round(tris[:, :, 0], 9))
    assert np.allclose(sorted(xs), [nx / 4, 3 * nx / 4])
    # the same across y
    yc = np.arange(ny * 4) + 0.5
    g = np.cos(2 * np.pi * yc / (ny * 4))[None, :, None] * np.ones((nz, ny * 4, 3))
    tris = M.interface_mesh(g, 0.0)
    assert abs(M.mesh_area(tris) - 2 * 3 * (nz - 1)) < 1e-9
    assert np.allclose(sorted(np.unique(np.round(tris[:, :, 1], 9))), [ny, 3 * ny])


def test_sphere_is_closed_outward_and_approaches_the_sphere():
    n, R, w = 28, 7.0, 3.0
    c = (n / 2.0, n / 2.0, n / 2.0)
    zz, yy, xx = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.sqrt((xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2)
    f = np.clip(0.5 - (r - R) / w, 0.0, 1.0)
    tris = M.interface_mesh(f, 0.5)
    verts, idx = M.weld(tris)
    edges = np.sort(np.concatenate([idx[:, [0, 1]], idx[:, [1, 2]], idx[:, [2, 0]]]), axis=1)
    _, counts = np.unique(edges, axis=0, return_counts=True)
    assert (counts == 2).all()  # closed, no cracks
    E = len(counts)
    assert len(verts) - E + len(idx) == 2  # a sphere's Euler characteristic
    # consistently oriented: every directed edge once, its reverse in the neighbouring triangle
    directed = np.concatenate([idx[:, [0, 1]], idx[:, [1, 2]], idx[:, [2, 0]]])
    dset = {tuple(e) for e in directed}
    assert len(dset) == len(directed)
    assert all((b, a) in dset for a, b in dset)
    vol = M.mesh_volume(tris)
    assert vol > 0  # normals outward (towards lower phi)
    assert abs(vol / (4.0 / 3.0 * np.pi * R ** 3) - 1) < 0.02
    assert abs(M.mesh_area(tris) / (4 * np.pi * R ** 2) - 1) < 0.05


def test_cube_counts_and_single_cubes_agree_with_the_whole_mesh():
    # a random smooth field: many crossing patterns, several chunks of layers, a ragged last chunk
    rng = np.random.default_rng(5)
    nz, ny, nx = 11, 6, 7
    f = rng.uniform(0, 1, size=(nz, ny, nx))
    tris = M.interface_mesh(f, 0.45, off=3.0)
    cnt = M.cube_counts(f, 0.45, planes_per_chunk=4)
    assert cnt.shape == (nz - 1, ny, nx)
    assert cnt.sum() == len(tris)
    assert ((cnt >= 0) & (cnt <= 12)).all()
    # the entries of the whole mesh, cube by cube in the order (k ny + j) nx + i
    start = np.concatenate([[0], np.cumsum(cnt.ravel())])
    for c in rng.choice(cnt.size, 25, replace=False):
        k, j, i = np.unravel_index(c, cnt.shape)
        one = M.cube_triangles(f, 0.45, 3.0, i, j, k)
        assert len(one) == cnt[k, j, i]
        assert np.array_equal(one, tris[start[c]:start[c + 1]])
    # layers that are all inside or all outside give nothing; a single layer has no cubes
    assert M.cube_counts(np.ones((4, 3, 3)), 0.5).sum() == 0
    assert M.cube_counts(f[:1], 0.5).shape == (0, ny, nx) and len(M.interface_mesh(f[:1], 0.5)) == 0


def test_vertical_cylinder_is_an_open_tube_ending_on_the_first_and_last_planes():
    # no cubes across z: a phase column through the whole domain meshes to a tube whose boundary
    # edges (each in one triangle only) lie on the first and last cell-centre planes, Euler
    # characteristic 0, area approaching the cylinder's
    n, nz, R, w, off = 30, 9, 7.0, 3.0, 11.0
    c = n / 2.0
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.sqrt((xx - c) ** 2 + (yy - c) ** 2)
    f = np.clip(0.5 - (r - R) / w, 0.0, 1.0)
    tris = M.interface_mesh(f, 0.5, off=off)
    verts, idx = M.weld(tris)
    edges = np.sort(np.concatenate([idx[:, [0, 1]], idx[:, [1, 2]], idx[:, [2, 0]]]), axis=1)
    uniq, counts = np.unique(edges, axis=0, return_counts=True)
    assert set(counts.tolist()) == {1, 2}
    bz = verts[uniq[counts == 1]][:, :, 2]
    assert np.all((np.abs(bz - (off + 0.5)) < 1e-9) | (np.abs(bz - (off + nz - 0.5)) < 1e-9))
    assert len(verts) - len(uniq) + len(idx) == 0
    assert abs(M.mesh_area(tris) / (2 * np.pi * R * (nz - 1)) - 1) < 0.05
