"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds parameter values, grid shapes and seeded random draws only; it
holds none of the method's arithmetic (no time step, no stability limit, no
thermodynamics).  The paper's Ag-Al-Cu coefficients are not printed in the paper,
so every workload uses the symmetric stand-in set described below.

Symmetric parameter set (Section 2 model, readings R1/R3/R12):
  * N = 4 phases (alpha, beta, gamma solid; phase 3 liquid), K = 3 components,
    so mu has K-1 = 2 entries.
  * dx = 1, eps = 4 dx, tau = 1; dt <= 0 asks the library/oracle for
    0.5 x the explicit stability limit.
  * gamma_ab = 1 for all pairs, gamma_abd = 15 for all triples.
  * parabolic grand potentials with equal curvature A = 1; solid equilibrium
    compositions alpha (0.8, 0.1), beta (0.1, 0.8), gamma (0.1, 0.1); liquid
    (1/3, 1/3); TE = 1; s = 1 for solids, 0 for the liquid; kT = 0 for solids,
    (0.1, 0.1) for the liquid; D = 1 in the liquid, 0 in the solids.
  * frozen gradient T = T0 + G (z - v t) with G = 1e-3, v = 1e-2 and
    T0 = TE - G H - DT0: the top of the H = 8 seed layers starts DT0 = 0.15
    below TE (the eutectic isotherm lies DT0/G = 150 cells above the seeds).
    With DT0 = 0 the seeds, thinner than the diffuse interface (about 10 cells
    at eps = 4), melt back completely within about 2000 steps; at 0.15 they
    survive and the front advances.
"""
from __future__ import annotations

import copy

import numpy as np

SEED_LAYERS = 8
INITIAL_UNDERCOOLING = 0.15


def symmetric_params(G: float = 1e-3, v: float = 1e-2, n_grains: int = 12,
                     window_trigger_z: float = 0.0, dt: float = 0.0) -> dict:
    TE = 1.0
    H = SEED_LAYERS
    return {
        "dx": 1.0, "eps": 4.0, "tau": 1.0, "dt": dt,
        "gamma2": [1.0] * 6, "gamma3": [15.0] * 4,
        "A": [1.0, 1.0, 1.0, 1.0],
        "cE": [[0.8, 0.1], [0.1, 0.8], [0.1, 0.1], [1.0 / 3.0, 1.0 / 3.0]],
        "kT": [[0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [0.1, 0.1]],
        "s": [1.0, 1.0, 1.0, 0.0],
        "D": [0.0, 0.0, 0.0, 1.0],
        "TE": TE, "T0": TE - G * H - INITIAL_UNDERCOOLING, "G": G, "v": v,
        "seed_layers": H, "n_grains": n_grains,
        "window_trigger_z": window_trigger_z,
    }


def general_params(G: float = 1e-3, v: float = 1e-2, n_grains: int = 12,
                   window_trigger_z: float = 0.0, dt: float = 0.0) -> dict:
    """The symmetric set with general parabolic thermodynamics (the Ag-Al-Cu-shaped variant, whose
    coefficients the paper does not print): the Gibbs-energy curvature of each phase a symmetric
    positive-definite 2x2 matrix A_a = [[a11, a12], [a12, a22]] with unequal diagonal entries and a
    cross term ("Am": a11, a12, a22), and a relaxation time per phase pair ("tau_ab", pairs 01 02 03
    12 13 23).  Everything else as symmetric_params."""
    p = symmetric_params(G=G, v=v, n_grains=n_grains, window_trigger_z=window_trigger_z, dt=dt)
    p["Am"] = [[1.2, 0.3, 0.8], [0.7, -0.2, 1.5], [1.0, 0.4, 1.1], [0.9, 0.15, 1.3]]
    p["tau_ab"] = [2.0, 1.6, 1.0, 1.8, 0.8, 1.2]
    return p


def with_(p: dict, **kw) -> dict:
    q = copy.deepcopy(p)
    q.update(kw)
    return q


# ---------------------------------------------------------------------------
# the benchmark configurations (grid sizes, grains, steps, seeds)
# ---------------------------------------------------------------------------

CONFIGS = {
    # plain FP64 method, small: the case the oracle finishes in seconds
    "c0_32x32x64": dict(nx=32, ny=32, nz=64, n_grains=12, steps=200, seed=0),
    # single large domain: FP32 vs FP64, window trigger at z = 512
    "c1_256x256x1024": dict(nx=256, ny=256, nz=1024, n_grains=64, steps=2000, seed=0,
                            window_trigger_z=512.0),
    # precision study
    "c2_128x128x512": dict(nx=128, ny=128, nz=512, n_grains=20, steps=20000, seed=0),
}


def batched_domains(n: int = 64, seed: int = 0):
    """64 uneven domains: x,y in {32,64,96,128}, z in {128,256,512}, v in [5e-3,2e-2],
    G in [5e-4,2e-3] (numpy PCG64 stream seeded with ``seed``)."""
    rng = np.random.default_rng(seed)
    xy = [32, 64, 96, 128]
    zs = [128, 256, 512]
    out = []
    for q in range(n):
        nx = int(rng.choice(xy))
        ny = int(rng.choice(xy))
        nz = int(rng.choice(zs))
        v = float(rng.uniform(5e-3, 2e-2))
        G = float(rng.uniform(5e-4, 2e-3))
        out.append(dict(nx=nx, ny=ny, nz=nz, v=v, G=G, seed=int(rng.integers(0, 2**31))))
    return out


def serving_requests(n: int = 500, seed: int = 0, big_fraction: float = 0.1,
                     steps_range=(500, 5000)):
    """Poisson arrival stream: sizes as in ``batched_domains`` plus ``big_fraction`` at
    256x256x512; steps uniform in ``steps_range``; random v, G and seed.  Arrival times are
    returned in units of the mean inter-arrival gap (scale them to the wanted rate)."""
    rng = np.random.default_rng(seed + 1)
    xy = [32, 64, 96, 128]
    zs = [128, 256, 512]
    gaps = rng.exponential(1.0, size=n)
    arr = np.cumsum(gaps)
    out = []
    for q in range(n):
        if rng.uniform() < big_fraction:
            nx, ny, nz = 256, 256, 512
        else:
            nx, ny, nz = int(rng.choice(xy)), int(rng.choice(xy)), int(rng.choice(zs))
        out.append(dict(arrival=float(arr[q]), nx=nx, ny=ny, nz=nz,
                        v=float(rng.uniform(5e-3, 2e-2)), G=float(rng.uniform(5e-4, 2e-3)),
                        steps=int(rng.integers(steps_range[0], steps_range[1] + 1)),
                        seed=int(rng.integers(0, 2**31))))
    return out


def random_simplex_field(rng: np.random.Generator, nx: int, ny: int, nz: int, sharp: float = 0.3):
    """Random phase fields on the Gibbs simplex: a mix of one-hot cells and random interior
    points (Dirichlet draws), shape (4, nz, ny, nx)."""
    x = rng.dirichlet([0.5] * 4, size=(nz, ny, nx))
    onehot = rng.uniform(size=(nz, ny, nx)) < sharp
    k = rng.integers(0, 4, size=(nz, ny, nx))
    x[onehot] = np.eye(4)[k[onehot]]
    return np.ascontiguousarray(np.moveaxis(x, -1, 0))


def random_mu(rng: np.random.Generator, nx: int, ny: int, nz: int, scale: float = 0.05):
    return np.ascontiguousarray(rng.uniform(-scale, scale, size=(2, nz, ny, nx)))


def planar_front(nx: int, ny: int, nz: int, z0: float, width: float, solid: int = 0):
    """Phase field of a flat solid(`solid`)/liquid front at height z0 with a sine profile
    of the given width, shape (4, nz, ny, nx); exactly one-hot outside the profile."""
    phi = np.zeros((4, nz, ny, nx))
    for k in range(nz):
        s = (k - z0) / width * np.pi
        if s <= -np.pi / 2:
            f = 1.0
        elif s >= np.pi / 2:
            f = 0.0
        else:
            f = 0.5 * (1.0 - np.sin(s))
        phi[solid, k] = f
        phi[3, k] = 1.0 - f
    return phi


def _voronoi_labels(points, seeds, box):
    """Index of the nearest seed for every point (periodic in x and y over box[:2], open in z;
    ties to the lowest index), through scipy's k-d tree."""
    from scipy.spatial import cKDTree

    bx, by, bz = box
    tree = cKDTree(seeds, boxsize=[bx, by, 4.0 * bz])
    _, idx = tree.query(points, k=1)
    return idx


REGION_KINDS = ("liquid", "solid", "interface")


def region_fields(kind: str, nx: int, ny: int, nz: int, seed: int = 0):
    """Initial fields of the three block compositions of the paper's performance section
    (Section 4: liquid, solid and interface blocks), shape (4, nz, ny, nx) and (2, nz, ny, nx):
      * liquid: pure liquid, mu uniform in [-1e-3, 1e-3];
      * solid: 3D Voronoi grains of the three solid phases, about 48 cells across (bulk
        dominated), mu as above;
      * interface: the solidification front crossing the block -- columnar grains (x-y Voronoi,
        about 12 cells across, phases drawn uniformly from the three solids) below z = nz/2,
        liquid above, mu as above.
    Interfaces start sharp; a few steps give them their diffuse profile.  numpy PCG64 stream
    seeded with ``seed``."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-1e-3, 1e-3, size=(2, nz, ny, nx))
    lab = np.full((nz, ny, nx), 3, dtype=np.int64)
    if kind == "solid":
        ng = max(4, int(nx * ny * nz / 48.0 ** 3))
        seeds = rng.uniform(0, 1, size=(ng, 3)) * [nx, ny, nz]
        phase = rng.integers(0, 3, size=ng)
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        pts = np.stack([i.ravel() + 0.5, j.ravel() + 0.5, k.ravel() + 0.5], axis=1)
        lab = phase[_voronoi_labels(pts, seeds, (nx, ny, nz))].reshape(nz, ny, nx)
    elif kind == "interface":
        ng = max(3, int(nx * ny / 12.0 ** 2))
        seeds = np.concatenate([rng.uniform(0, 1, size=(ng, 2)) * [nx, ny], np.zeros((ng, 1))], axis=1)
        phase = rng.integers(0, 3, size=ng)
        j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        pts = np.stack([i.ravel() + 0.5, j.ravel() + 0.5, np.zeros(i.size)], axis=1)
        cols = phase[_voronoi_labels(pts, seeds, (nx, ny, 1))].reshape(ny, nx)
        lab[: nz // 2] = cols[None]
    elif kind != "liquid":
        raise ValueError(kind)
    phi = np.zeros((4, nz, ny, nx))
    for a in range(4):
        phi[a][lab == a] = 1.0
    return phi, mu
