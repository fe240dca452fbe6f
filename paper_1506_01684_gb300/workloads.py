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
    T0 = TE - G H so that the eutectic isotherm starts at the top of the
    H = 8 seed layers.
"""
from __future__ import annotations

import copy

import numpy as np

SEED_LAYERS = 8


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
        "TE": TE, "T0": TE - G * H, "G": G, "v": v,
        "seed_layers": H, "n_grains": n_grains,
        "window_trigger_z": window_trigger_z,
    }


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


def interface_block(n: int, seed: int = 0):
    """Region micro-benchmarks of the paper's performance section (liquid, solid, interface)
    at n^3: returns dict name -> (phi, mu) initial data or None when the library's own
    initial condition (Voronoi) is used."""
    rng = np.random.default_rng(seed)
    liquid_phi = np.zeros((4, n, n, n))
    liquid_phi[3] = 1.0
    liquid_mu = rng.uniform(-1e-3, 1e-3, size=(2, n, n, n))
    return {"liquid": (liquid_phi, liquid_mu)}
