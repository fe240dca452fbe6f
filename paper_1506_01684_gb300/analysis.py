"""Host-side analysis of simulation results (not part of the time step).

lamella_count: reading R14 of the paper's "lamella" observable -- for each solid phase, the number
of 4-connected components of {phi_a > 1/2} in one x-y plane, with periodic boundaries in x and y
(a lamella crossing the domain edge is one lamella).
"""
from __future__ import annotations

import numpy as np


def _components_periodic(mask: np.ndarray) -> int:
    """Number of 4-connected components of a 2D boolean mask with periodic wrap in both axes."""
    ny, nx = mask.shape
    parent = np.arange(ny * nx)

    def find(a):
        root = a
        while parent[root] != root:
            root = parent[root]
        while parent[a] != root:
            parent[a], a = root, parent[a]
        return root

    def union(a, b):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)

    idx = np.arange(ny * nx).reshape(ny, nx)
    for axis in (0, 1):
        nb_mask = np.roll(mask, -1, axis=axis)
        nb_idx = np.roll(idx, -1, axis=axis)
        both = mask & nb_mask
        for a, b in zip(idx[both], nb_idx[both]):
            union(int(a), int(b))
    roots = {find(int(a)) for a in idx[mask]}
    return len(roots)


def lamella_count(phi: np.ndarray, h_int: float, depth: int = 8) -> list:
    """phi: (4, nz, ny, nx).  Counts per solid phase in the plane z = max(0, floor(h_int) - depth)."""
    nz = phi.shape[1]
    z = min(max(0, int(np.floor(h_int)) - depth), nz - 1)
    return [_components_periodic(phi[a, z] > 0.5) for a in range(3)]
