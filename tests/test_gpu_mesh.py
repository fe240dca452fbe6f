"""Interface meshes on the GPU (the paper's per-phase isosurface output, Section 3.2) against the
oracle (oracle/mesh.py), through pf_interface_mesh.

Both sides classify corners (value >= iso) in the simulation's precision: the oracle is given the
field the GPU holds (read back exactly) and iso rounded to that precision, so the triangle count,
the cubes they come from and their order must agree exactly.  Vertices: the GPU interpolates in
the field's precision, forms positions in FP64 and stores FP32.  With t = (iso - f_a) / (f_b - f_a)
from exact inputs (relative error <= 3 u of the field's precision, t in [0, 1]) and the FP32 store
(half an ulp of the coordinate), a coordinate differs from the oracle's FP64 by at most
3 u + 2^-24 |x|: the tests allow 4e-7 + 2^-23 |x| for FP32 fields and 1e-12 + 2^-23 |x| for FP64.
The orientation is a sign decision on the normal; for triangles of area below 1e-6 (a vertex at a
corner) the two may legitimately differ, so there v1 and v2 are compared as a set.
"""
import numpy as np
import pytest

from oracle import mesh as M
from paper_1506_01684_gb300 import pf
from paper_1506_01684_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.lib()


def _iso(precision, iso):
    return float(np.float32(iso)) if precision.startswith("fp32") else float(iso)


def _tol(precision, ref):
    base = 4e-7 if precision.startswith("fp32") else 1e-12
    return base + 2.0 ** -23 * np.abs(ref)


def _compare(gpu, ref, precision):
    assert gpu.shape == ref.shape
    if len(ref) == 0:
        return
    tol = _tol(precision, ref)
    g = gpu.astype(np.float64)
    # v0 always; v1, v2 in order where the triangle has an area, as a set where it is degenerate
    assert (np.abs(g[:, 0] - ref[:, 0]) <= tol[:, 0]).all()
    area = 0.5 * np.linalg.norm(np.cross(ref[:, 1] - ref[:, 0], ref[:, 2] - ref[:, 0]), axis=1)
    same = (np.abs(g[:, 1:] - ref[:, 1:]) <= tol[:, 1:]).all(axis=(1, 2))
    swapped = (np.abs(g[:, [2, 1]] - ref[:, 1:]) <= tol[:, 1:]).all(axis=(1, 2))
    assert (same | ((area < 1e-6) & swapped)).all()
    assert same[area >= 1e-6].all()


def _run(nx, ny, nz, precision, steps, seed=1, window=0.0, grains=6):
    p = W.symmetric_params(n_grains=grains, window_trigger_z=window)
    p["seed_layers"] = min(10, nz - 2)
    sim = pf.Simulation(nx, ny, nz, p, precision)
    sim.init(seed)
    sim.step(steps)
    return sim


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mesh_of_every_phase_matches_the_oracle(precision):
    # 37 x 13 x 24: 11 063 cubes in 299 row segments of 37 (one counting chunk of 23 layers), the window moved (offset
    # and ring base non-zero), grains of all three solids
    nx, ny, nz = 37, 13, 24
    sim = _run(nx, ny, nz, precision, steps=400, window=8.0)
    st = sim.stats()
    assert st["window_offset"] > 0
    phi, _ = sim.fields()
    for a in range(4):
        for iso in (0.5, 0.27):
            iso_r = _iso(precision, iso)
            ref = M.interface_mesh(phi[a], iso_r, off=st["window_offset"])
            gpu = sim.interface_mesh(a, iso)
            assert len(ref) > 0, (a, iso)
            _compare(gpu, ref, precision)
    sim.close()


def test_rows_wider_than_one_segment():
    # nx = 300: two segments of cubes per row (256 + a ragged 44, the row's last cube wrapping to
    # column 0 across the segment boundary), 13 layers (a ragged counting chunk)
    nx, ny, nz = 300, 6, 14
    sim = _run(nx, ny, nz, "fp32", steps=60, grains=9)
    phi, _ = sim.fields()
    for a in (0, 3):
        ref = M.interface_mesh(phi[a], 0.5)
        assert len(ref) > 0
        _compare(sim.interface_mesh(a, 0.5), ref, "fp32")
    sim.close()


def test_degenerate_cases():
    sim = _run(20, 9, 16, "fp32", steps=20)
    # a level no value reaches, and one every value reaches: no triangles
    assert len(sim.interface_mesh(3, 2.0)) == 0
    assert len(sim.interface_mesh(0, -1.0)) == 0
    # a count query, a too-small buffer, bad arguments
    import ctypes
    n = ctypes.c_size_t()
    assert pf.lib().pf_interface_mesh(sim.h, 3, 0.5, None, 0, ctypes.byref(n)) == pf.PF_OK
    assert n.value > 0
    buf = np.zeros((n.value - 1) * 9, dtype=np.float32)
    fp = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    assert pf.lib().pf_interface_mesh(sim.h, 3, 0.5, fp, n.value - 1, ctypes.byref(n)) == pf.PF_E_INVAL
    assert (buf == 0).all()
    for phase, iso in ((4, 0.5), (-1, 0.5), (0, float("nan")), (0, float("inf"))):
        assert pf.lib().pf_interface_mesh(sim.h, phase, iso, None, 0, ctypes.byref(n)) == pf.PF_E_INVAL
    assert pf.lib().pf_interface_mesh(sim.h, 0, 0.5, None, 0, None) == pf.PF_E_INVAL
    sim.close()
    # one plane: no cubes
    one = pf.Simulation(8, 8, 1, W.symmetric_params(), "fp64")
    phi = np.zeros((4, 1, 8, 8))
    phi[0, :, :, :4] = 1.0
    phi[3, :, :, 4:] = 1.0
    one.set_fields(phi, np.zeros((2, 1, 8, 8)))
    assert len(one.interface_mesh(0, 0.5)) == 0
    one.close()
    # two planes, a front across x that wraps (nx = 2: a cell's x neighbours are the same cell)
    two = pf.Simulation(2, 3, 2, W.symmetric_params(), "fp64")
    phi = np.zeros((4, 2, 3, 2))
    phi[0, :, :, 0] = 1.0
    phi[3, :, :, 1] = 1.0
    two.set_fields(phi, np.zeros((2, 2, 3, 2)))
    _compare(two.interface_mesh(0, 0.5), M.interface_mesh(phi[0], 0.5), "fp64")
    two.close()


def test_mesh_of_the_large_domain_on_sampled_cubes():
    # 256 x 256 x 1024 FP32, 64 grains (the benchmark's domain) after 300 steps: the exact count per
    # cube from the oracle's vectorised counts, and the triangles of 400 sampled crossed cubes
    nx, ny, nz = 256, 256, 1024
    p = W.symmetric_params(n_grains=64, window_trigger_z=512.0)
    sim = pf.Simulation(nx, ny, nz, p, "fp32")
    sim.init(0)
    sim.step(300)
    off = sim.stats()["window_offset"]
    phi, _ = sim.fields()
    rng = np.random.default_rng(11)
    for a in (0, 3):
        field = phi[a]
        gpu = sim.interface_mesh(a, 0.5)
        cnt = M.cube_counts(field, 0.5)
        assert len(gpu) == int(cnt.sum()) > 0
        start = np.concatenate([[0], np.cumsum(cnt.ravel())])
        crossed = np.flatnonzero(cnt.ravel())
        for c in rng.choice(crossed, min(400, len(crossed)), replace=False):
            k, j, i = np.unravel_index(c, cnt.shape)
            ref = M.cube_triangles(field, 0.5, off, i, j, k)
            _compare(gpu[start[c]:start[c + 1]], ref, "fp32")
        # the mesh lies in the domain: x, y within the periodic cubes, z inside the cell centres
        assert gpu[:, :, 0].min() >= 0.5 and gpu[:, :, 0].max() <= nx + 0.5
        assert gpu[:, :, 2].min() >= off + 0.5 and gpu[:, :, 2].max() <= off + nz - 0.5
    sim.close()
