"""Lamella count (reading R14): periodic 4-connected components, checked on hand-made planes."""
import numpy as np

from paper_1506_01684_gb300.analysis import _components_periodic, lamella_count


def test_components_wrap_around_the_periodic_edges():
    m = np.zeros((6, 8), bool)
    m[:, 0] = True
    m[:, 7] = True  # touches column 0 through the x wrap: one lamella
    assert _components_periodic(m) == 1
    m2 = np.zeros((6, 8), bool)
    m2[1, 1] = m2[4, 5] = True
    assert _components_periodic(m2) == 2
    m3 = np.zeros((6, 8), bool)
    m3[0, 2] = m3[5, 2] = True  # y wrap
    m3[2, 4] = True
    m3[3, 5] = True  # diagonal only: not 4-connected
    assert _components_periodic(m3) == 3
    assert _components_periodic(np.ones((3, 3), bool)) == 1
    assert _components_periodic(np.zeros((3, 3), bool)) == 0


def test_lamella_count_reads_the_plane_below_the_interface():
    phi = np.zeros((4, 20, 6, 8))
    phi[3] = 1.0
    # stripes of phase 0 and 1 at z = 4 (h = 12.x -> plane 12 - 8 = 4)
    phi[:, 4] = 0.0
    phi[0, 4, :, 0:2] = 1.0
    phi[1, 4, :, 2:5] = 1.0
    phi[2, 4, :, 5:8] = 1.0
    assert lamella_count(phi, 12.7) == [1, 1, 1]
    phi[0, 4, :, 6] = 1.0
    phi[2, 4, :, 6] = 0.0  # splits the phase-2 stripe and adds a second phase-0 stripe
    assert lamella_count(phi, 12.7) == [2, 1, 2]
