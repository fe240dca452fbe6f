"""Pins of the oracle's general parabolic thermodynamics (reading R17: the Gibbs-energy curvature
A_a of each phase a symmetric 2x2 matrix, K_a = dc^a/dmu = (1/2) A_a^{-1}, chi = sum h_a K_a,
M = sum D_a h_a K_a, and a relaxation time interpolated over the phase pairs).

Each check is fixed by something other than the oracle: numpy's matrix inverse, finite
differences, the exact discrete solution of a diffusion equation with a constant matrix
coefficient, exact scaling of the phi increment, exact solute conservation, and the reduction to
the scalar form.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1506_01684_gb300 import workloads as W


def _A(p, a):
    a11, a12, a22 = p["Am"][a]
    return np.array([[a11, a12], [a12, a22]])


def _fd(f, x, h=1e-5):
    g = np.zeros_like(x, dtype=float)
    for i in range(len(x)):
        e = np.zeros_like(x, dtype=float)
        e[i] = h
        g[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def test_k_is_half_the_inverse_curvature():
    p = W.general_params()
    for a in range(4):
        np.testing.assert_allclose(oracle.kmat(p, a), 0.5 * np.linalg.inv(_A(p, a)), rtol=1e-15, atol=1e-16)
    q = W.symmetric_params()
    q["A"] = [1.0, 1.3, 0.8, 1.1]
    for a in range(4):
        assert (oracle.kmat(q, a) == np.eye(2) / (2 * q["A"][a])).all()


def test_c_is_minus_the_mu_gradient_of_a_concave_grand_potential():
    p = W.general_params()
    rng = np.random.default_rng(4)
    for _ in range(5):
        mu = rng.normal(scale=0.3, size=2)
        T = rng.uniform(0.9, 1.1)
        for a in range(4):
            fd = -_fd(lambda m: oracle.psi_alpha(p, a, m, T), mu)
            np.testing.assert_allclose(oracle.c_alpha(p, a, mu, T), fd, rtol=1e-8, atol=1e-9)
            # dc/dmu = (1/2) A^{-1}, column by column
            J = np.stack([(oracle.c_alpha(p, a, mu + e, T) - oracle.c_alpha(p, a, mu - e, T)) / 2e-5
                          for e in (np.array([1e-5, 0.0]), np.array([0.0, 1e-5]))], axis=1)
            np.testing.assert_allclose(J, 0.5 * np.linalg.inv(_A(p, a)), rtol=1e-7, atol=1e-9)
    # equal grand potentials at the eutectic point, whatever the curvatures
    assert max(abs(oracle.psi_alpha(p, a, [0.0, 0.0], p["TE"])) for a in range(4)) == 0.0


@pytest.mark.parametrize("mix", [(0.6, 0.0, 0.0, 0.4), (0.2, 0.5, 0.0, 0.3), (0.1, 0.2, 0.3, 0.4),
                                 (0.0, 0.0, 0.0, 1.0)])
def test_matrix_diffusion_in_a_uniform_mixture_follows_the_discrete_solution(mix):
    # phi uniform (frozen: tau huge), mu = cos(2 pi m x / nx) v: div(M grad mu) = -lam M mu with
    # lam = 4 sin^2(pi m / nx) / dx^2, so mu^n = cos(...) (I - dt lam chi^{-1} M)^n v exactly, with
    # chi = sum h_a K_a and M = sum D_a h_a K_a built here from numpy's inverse of A_a
    nx, ny, nz, m, n = 16, 2, 3, 3, 20
    p = W.general_params(G=0.0)
    p["D"] = [0.3, 0.0, 0.1, 1.0]
    p["tau"] = 1e30
    p["tau_ab"] = [1e30] * 6
    p["dt"] = 0.1
    st = oracle.State(p, nx, ny, nz)
    st.phi = np.array(mix, dtype=float)[:, None, None, None] * np.ones((4, nz, ny, nx))
    v = np.array([0.02, -0.035])
    x = np.arange(nx)
    wave = np.cos(2 * np.pi * m * x / nx)
    st.mu = v[:, None, None, None] * wave[None, None, None, :] * np.ones((2, nz, ny, nx))
    st.step(n)
    phi = np.array(mix, dtype=float)
    h = phi ** 2 / (phi ** 2).sum()
    K = [0.5 * np.linalg.inv(_A(p, a)) for a in range(4)]
    chi = sum(h[a] * K[a] for a in range(4))
    M = sum(p["D"][a] * h[a] * K[a] for a in range(4))
    lam = 4 * math.sin(math.pi * m / nx) ** 2 / p["dx"] ** 2
    step = np.eye(2) - p["dt"] * lam * np.linalg.solve(chi, M)
    want = np.linalg.matrix_power(step, n) @ v
    assert np.abs(want).max() > 0.05 * np.abs(v).max()  # still a clear signal
    for c in range(2):
        np.testing.assert_allclose(st.mu[c], want[c] * wave[None, None, :] * np.ones((nz, ny, nx)),
                                   rtol=0, atol=1e-12 * np.abs(v).max())
    assert np.abs(st.phi - phi[:, None, None, None]).max() <= 1e-15


def test_relaxation_time_of_a_cell_is_that_of_its_phase_pairs():
    # phi* - phi^n = -(dt/(tau(phi) eps)) (rhs - mean): with tau_ab distinct per pair, a cell holding
    # exactly two phases a, b moves by 1/tau_ab of the move at tau = 1; a single-phase cell by 1/tau
    rng = np.random.default_rng(9)
    n = 8
    phi = np.zeros((4, n, n, n))
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    labels = rng.integers(0, 10, size=(n, n, n))
    x = rng.uniform(0.1, 0.9, size=(n, n, n))
    for idx, (a, b) in enumerate(pairs):
        sel = labels == idx
        phi[a][sel] = x[sel]
        phi[b][sel] = 1 - x[sel]
    three = (labels >= 6) & (labels <= 8)
    w = rng.dirichlet([1.0] * 3, size=int(three.sum()))
    for q, a in enumerate((0, 1, 3)):
        phi[a][three] = w[:, q]
    one = labels == 9
    phi[:, one] = 0.0
    phi[2][one] = 1.0
    mu = W.random_mu(rng, n, n, n)
    base = oracle.resolve_params(W.symmetric_params(), n)
    gen = dict(base, tau_ab=[2.0, 1.6, 1.0, 1.8, 0.8, 1.2], tau=1.7)
    _, s0 = oracle.phi_sweep(base, phi, mu, want_star=True)
    _, s1 = oracle.phi_sweep(gen, phi, mu, want_star=True)
    d0, d1 = s0 - phi, s1 - phi
    for idx, (a, b) in enumerate(pairs):
        sel = labels == idx
        np.testing.assert_allclose(d1[:, sel], d0[:, sel] / gen["tau_ab"][idx], rtol=1e-12, atol=1e-17)
    np.testing.assert_allclose(d1[:, one], d0[:, one] / 1.7, rtol=1e-12, atol=1e-17)
    # three phases 0, 1, 3: the pair-weighted mean of tau_01, tau_03, tau_13
    p0, p1, p3 = phi[0][three], phi[1][three], phi[3][three]
    wts = np.stack([p0 * p1, p0 * p3, p1 * p3])
    tau3 = (np.array([2.0, 1.0, 0.8])[:, None] * wts).sum(0) / wts.sum(0)
    np.testing.assert_allclose(d1[:, three], d0[:, three] / tau3, rtol=1e-12, atol=1e-17)
    assert oracle.tau(gen, [0.0, 0.0, 1.0, 0.0]) == 1.7


@pytest.mark.parametrize("G", [0.0, 2e-3])
def test_solute_is_conserved_with_general_thermodynamics(G):
    nx, ny, nz = 16, 12, 24
    p = W.general_params(G=G, v=0.05, n_grains=6)
    p["seed_layers"] = 12
    p["D"] = [0.2, 0.0, 0.1, 1.0]  # diffusion in two solids too: cross-phase fluxes with M a matrix
    st = oracle.State(p, nx, ny, nz).init(3)
    rng = np.random.default_rng(1)
    st.mu = rng.uniform(-0.05, 0.05, size=st.mu.shape)
    _, so0, _, _ = st.reduce()
    for _ in range(4):
        st.step(50)
        fr, so, _, bad = st.reduce()
        assert not bad
        assert np.abs(so - so0).max() <= 1e-12 * np.abs(so0).max()
    assert np.abs(st.phi.sum(0) - 1).max() <= 4e-16 and st.phi.min() >= 0.0


def test_isotropic_matrices_and_equal_pair_times_reduce_to_the_scalar_form():
    nx, ny, nz = 12, 10, 16
    q = W.symmetric_params(G=1e-3, n_grains=5)
    q["A"] = [1.0, 1.3, 0.8, 1.1]
    q["seed_layers"] = 8
    g = dict(q, Am=[[q["A"][a], 0.0, q["A"][a]] for a in range(4)], tau_ab=[q["tau"]] * 6)
    a = oracle.State(q, nx, ny, nz).init(2)
    b = oracle.State(g, nx, ny, nz).init(2)
    assert a.params["dt"] == b.params["dt"]
    a.step(20)
    b.step(20)
    assert np.abs(a.phi - b.phi).max() <= 1e-13
    assert np.abs(a.mu - b.mu).max() <= 1e-13 * max(np.abs(a.mu).max(), 1e-8)


def _relaxed_profile_error(p, eps=4.0, nz=48, steps=4000):
    # a flat two-phase alpha / liquid front at TE, mu = 0: the stationary profile is the obstacle sine
    # 1/2 (1 - sin(4 z / (pi eps))) whatever the curvatures and relaxation times (all grand potentials
    # vanish at mu = 0, T = TE); returns the largest deviation from it and the state
    p = dict(p, eps=eps, T0=p["TE"])
    st = oracle.State(p, 1, 1, nz)
    st.phi = W.planar_front(1, 1, nz, nz / 2 + 0.3, 0.6 * math.pi ** 2 * eps / 4)
    st.mu = np.zeros((2, nz, 1, 1))
    st.step(steps)
    prof = st.phi[0, :, 0, 0]
    k = np.where((prof[:-1] >= 0.5) & (prof[1:] < 0.5))[0][0]
    zc = k + (prof[k] - 0.5) / (prof[k] - prof[k + 1])
    s = 4 * (np.arange(nz) - zc) / (math.pi * eps)
    ref = np.where(s <= -math.pi / 2, 1.0, np.where(s >= math.pi / 2, 0.0, 0.5 * (1 - np.sin(np.clip(s, -7, 7)))))
    return np.abs(prof - ref).max(), st


def test_general_thermodynamics_keep_the_two_phase_equilibrium_profile():
    e_sym, _ = _relaxed_profile_error(W.symmetric_params(G=0.0))
    for p in (W.general_params(G=0.0), dict(W.general_params(G=0.0), tau_ab=[2.0, 1.6, 2.0, 1.8, 0.8, 1.2])):
        e, st = _relaxed_profile_error(p)
        assert e < 1.1 * e_sym and e < 0.007, (e, e_sym)
        assert (st.phi[1] == 0).all() and (st.phi[2] == 0).all()  # the front stays two-phase
