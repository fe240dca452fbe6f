"""Pins for the oracle's pointwise model functions (no GPU).

Each derivative the oracle uses is checked against central finite differences of
the function it differentiates, and each energy against a closed form that the
model fixes in a special case:
  * gradient energy a (reading R3): on a two-phase 1D profile with
    phi_a + phi_l = 1, q = -phi_a', so a = gamma (phi_a')^2;
  * obstacle potential: two-phase value (16/pi^2) gamma x (1 - x), triple point;
  * grand potentials (R1): equal at (mu = 0, T = TE); c^a = -d psi_a/d mu;
  * h (R2): partition of unity, one-hot at bulk points;
  * simplex projection (R6): brute-force search over all supports (the KKT
    solution of the small QP), idempotence, fixed points.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1506_01684_gb300 import workloads as W

P = W.symmetric_params()


def _random_params(rng):
    """A non-symmetric parameter set so that index mix-ups cannot cancel."""
    p = W.symmetric_params()
    p["gamma2"] = list(rng.uniform(0.5, 2.0, 6))
    p["gamma3"] = list(rng.uniform(5.0, 20.0, 4))
    p["A"] = list(rng.uniform(0.5, 2.0, 4))
    p["cE"] = [list(rng.uniform(0, 1, 2)) for _ in range(4)]
    p["kT"] = [list(rng.uniform(-0.2, 0.2, 2)) for _ in range(4)]
    p["s"] = list(rng.uniform(-1, 1, 4))
    p["D"] = list(rng.uniform(0, 1, 4))
    return p


def _fd(f, x, hstep=1e-5):
    x = np.array(x, dtype=float)
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy()
        xm = x.copy()
        xp[idx] += hstep
        xm[idx] -= hstep
        g[idx] = (f(xp) - f(xm)) / (2 * hstep)
    return g


@pytest.mark.parametrize("seed", range(6))
def test_gradient_energy_derivatives_match_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = _random_params(rng)
    for _ in range(4):
        phi = rng.dirichlet([1.0] * 4)
        g = rng.normal(size=(4, 3))
        dphi = oracle.dadphi(p, phi, g)
        dgrad = oracle.dadgrad(p, phi, g)
        fd_phi = _fd(lambda x: oracle.a_energy(p, x, g), phi)
        fd_grad = _fd(lambda x: oracle.a_energy(p, phi, x), g)
        scale = max(1.0, np.abs(fd_phi).max(), np.abs(fd_grad).max())
        assert np.abs(dphi - fd_phi).max() <= 1e-8 * scale
        assert np.abs(dgrad - fd_grad).max() <= 1e-8 * scale


@pytest.mark.parametrize("seed", range(6))
def test_obstacle_and_driving_force_derivatives_match_finite_differences(seed):
    rng = np.random.default_rng(100 + seed)
    p = _random_params(rng)
    for _ in range(4):
        phi = rng.dirichlet([1.0] * 4)
        mu = rng.normal(scale=0.3, size=2)
        T = rng.uniform(0.9, 1.1)
        np.testing.assert_allclose(oracle.domega(p, phi), _fd(lambda x: oracle.omega(p, x), phi),
                                   rtol=1e-8, atol=1e-8)
        np.testing.assert_allclose(oracle.dpsi(p, phi, mu, T), _fd(lambda x: oracle.psi(p, x, mu, T), phi),
                                   rtol=1e-8, atol=1e-8)
        for a in range(4):
            # c^a = -d psi_a / d mu
            fd = -_fd(lambda m: oracle.psi_alpha(p, a, m, T), mu)
            np.testing.assert_allclose(oracle.c_alpha(p, a, mu, T), fd, rtol=1e-8, atol=1e-9)
            # dc^a/dT = kT_a
            dT = (oracle.c_alpha(p, a, mu, T + 1e-5) - oracle.c_alpha(p, a, mu, T - 1e-5)) / 2e-5
            np.testing.assert_allclose(dT, p["kT"][a], rtol=1e-7, atol=1e-9)
            # dc^a/dmu = 1/(2 A_a)
            dm = (oracle.c_alpha(p, a, mu + [1e-5, 0], T) - oracle.c_alpha(p, a, mu - [1e-5, 0], T)) / 2e-5
            np.testing.assert_allclose(dm, [1 / (2 * p["A"][a]), 0.0], rtol=1e-7, atol=1e-9)


def test_gradient_energy_two_phase_profile_closed_form():
    # phi = (x, 0, 0, 1-x), grad phi = (g, 0, 0, -g) e_z  =>  q_03 = -g e_z, a = gamma_03 g^2
    rng = np.random.default_rng(7)
    p = _random_params(rng)
    for x, gz in [(0.3, 0.7), (0.5, -1.3), (0.9, 0.05)]:
        phi = [x, 0, 0, 1 - x]
        g = np.zeros((4, 3))
        g[0, 2] = gz
        g[3, 2] = -gz
        assert oracle.a_energy(p, phi, g) == pytest.approx(p["gamma2"][2] * gz * gz, rel=1e-14)
    # a vanishes for any uniform field and for any field where all phases share one gradient direction
    # with proportional profiles (q = 0): phi_b = lambda_b f, grad phi_b = lambda_b grad f
    lam = rng.dirichlet([1] * 4)
    f, gf = 0.8, rng.normal(size=3)
    phi = lam * f
    g = np.outer(lam, gf)
    assert abs(oracle.a_energy(p, phi, g)) < 1e-15


def test_obstacle_potential_closed_forms():
    gam = 1.3
    p = W.with_(P, gamma2=[gam] * 6, gamma3=[11.0] * 4)
    for x in [0.1, 0.25, 0.5, 0.77]:
        assert oracle.omega(p, [x, 0, 0, 1 - x]) == pytest.approx(16 / math.pi**2 * gam * x * (1 - x), rel=1e-14)
    # triple point of three phases: 3 pairs at 1/9 each plus one triple at 1/27
    third = 1.0 / 3.0
    assert oracle.omega(p, [third, third, 0, third]) == pytest.approx(
        16 / math.pi**2 * gam * 3 / 9 + 11.0 / 27, rel=1e-14)
    # bulk: no potential
    for a in range(4):
        e = np.eye(4)[a]
        assert oracle.omega(p, e) == 0.0


def test_grand_potentials_and_interpolation():
    # all grand potentials coincide at the eutectic point (mu = 0, T = TE) ...
    vals = [oracle.psi_alpha(P, a, [0, 0], P["TE"]) for a in range(4)]
    assert max(vals) == min(vals) == 0.0
    # ... and solids are favoured below TE (the symmetric set has s_solid = 1, s_liquid = 0)
    T = P["TE"] - 0.01
    assert all(oracle.psi_alpha(P, a, [0, 0], T) < oracle.psi_alpha(P, 3, [0, 0], T) for a in range(3))
    # equilibrium compositions at mu = 0, T = TE
    for a in range(4):
        np.testing.assert_allclose(oracle.c_alpha(P, a, [0, 0], P["TE"]), P["cE"][a], rtol=0, atol=1e-16)
    rng = np.random.default_rng(3)
    for _ in range(20):
        phi = rng.dirichlet([0.7] * 4)
        hh = oracle.h(phi)
        assert hh.sum() == pytest.approx(1.0, abs=5e-16)
        assert (hh >= 0).all()
    for a in range(4):
        assert (oracle.h(np.eye(4)[a]) == np.eye(4)[a]).all()
    # dpsi vanishes at bulk points (h is flat there)
    for a in range(4):
        assert np.all(oracle.dpsi(P, np.eye(4)[a], [0.3, -0.2], 0.97) == 0.0)


def _project_brute(u):
    """Minimise |x - u|^2 over the simplex by enumerating supports (KKT on each)."""
    best, bestd = None, np.inf
    for r in range(1, 5):
        for S in itertools.combinations(range(4), r):
            x = np.zeros(4)
            lam = (sum(u[i] for i in S) - 1.0) / r
            for i in S:
                x[i] = u[i] - lam
            if (x >= -1e-15).all():
                d = ((x - u) ** 2).sum()
                if d < bestd:
                    best, bestd = np.maximum(x, 0), d
    return best


def test_simplex_projection_matches_brute_force_and_is_idempotent():
    rng = np.random.default_rng(11)
    cases = [rng.normal(scale=s, size=4) + o for s in (0.01, 0.3, 2.0) for o in (0.0, 0.25, 1.0)
             for _ in range(40)]
    cases += [np.array([1.0, 0, 0, 0]), np.array([0.25] * 4), np.array([0.5, 0.5, 0, 0]),
              np.array([2.0, 2.0, -1.0, 0.3]), np.array([0.3, 0.3, 0.3, 0.3])]
    for u in cases:
        x = oracle.project(u)
        assert abs(x.sum() - 1.0) <= 1e-15
        assert (x >= 0).all()
        np.testing.assert_allclose(x, _project_brute(u), rtol=0, atol=2e-15)
        np.testing.assert_allclose(oracle.project(x), x, rtol=0, atol=5e-16)
    # points already on the simplex are fixed; one-hot bulk points exactly
    for _ in range(50):
        s = rng.dirichlet([0.5] * 4)
        np.testing.assert_allclose(oracle.project(s), s, rtol=0, atol=4e-16)
    for a in range(4):
        assert (oracle.project(np.eye(4)[a]) == np.eye(4)[a]).all()


def test_splitmix64_matches_published_vector():
    import os
    here = os.path.dirname(__file__)
    want = [int(line, 16) for line in open(os.path.join(here, "golden", "splitmix64_seed0.txt"))
            if line.strip() and not line.startswith("#")]
    assert oracle.splitmix64(0, len(want)) == want


def test_default_dt_is_half_the_explicit_limit():
    # 32x32x64, G = 1e-3, T0 = TE - 8 G - 0.15: T_max = T0 + 63 G = 0.905, gamma_max = 1, D_max = 1
    dt = oracle.default_dt(P, 64)
    Tmax = 1.0 - 8e-3 - 0.15 + 63e-3
    assert dt == pytest.approx(0.5 * min(1.0 / (12 * Tmax), 1.0 / 6.0), rel=1e-15)
    assert dt == pytest.approx(0.0460, abs=1e-4)
