"""Pins for the oracle's sweeps, step, reductions, window and initial condition (no GPU).

What pins what:
  * phi-sweep rhs (Eq. 2): on smooth fields the discrete rhs converges at second order
    to the continuum rhs, which is built here from the definitions of a, omega and psi
    with sympy's own derivatives (not the oracle's hand-derived ones) and a 4th-order
    numerical divergence of the exact flux.
  * mu face fluxes (Eq. 3 flux, Eq. 4): the same second-order convergence against the
    continuum M grad mu - J_at at face centres.
  * mu update (Eq. 3 with reading R10): exact discrete eigen-decay of a Fourier mode in
    pure liquid, the closed-form drift from dc/dT dT/dt, and solute conservation to
    roundoff in a closed box (any wrong term in the update breaks it).
  * phi update (Eq. 1): Lagrange term sums to zero, bulk cells are fixed points, a flat
    front stays flat, the 1D two-phase equilibrium profile converges to
    1/2 (1 - sin(4 z/(pi eps))), the free energy decreases (reading R4's sign).
  * symmetries: periodic translation in x/y (bitwise), the (alpha<->beta, mu_0<->mu_1)
    symmetry of the symmetric parameter set.
  * window (R11), Voronoi initial condition (R13) and reductions: brute force.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_1506_01684_gb300 import workloads as W

P = W.symmetric_params()


# ---------------------------------------------------------------------------
# continuum reference built with sympy
# ---------------------------------------------------------------------------

def _sym_model(p):
    """Pointwise functions from the model definitions, differentiated by sympy."""
    ph = sp.symbols("p0:4", real=True)
    g = [[sp.Symbol(f"g{a}{d}", real=True) for d in range(3)] for a in range(4)]
    m = sp.symbols("m0:2", real=True)
    T = sp.Symbol("T", real=True)
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    triples = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
    a_expr = sum(p["gamma2"][q] * sum((ph[a] * g[b][d] - ph[b] * g[a][d]) ** 2 for d in range(3))
                 for q, (a, b) in enumerate(pairs))
    om = (16 / sp.pi ** 2) * sum(p["gamma2"][q] * ph[a] * ph[b] for q, (a, b) in enumerate(pairs)) + \
        sum(p["gamma3"][q] * ph[a] * ph[b] * ph[c] for q, (a, b, c) in enumerate(triples))
    S = sum(x * x for x in ph)
    psis = []
    for a in range(4):
        chat = [p["cE"][a][i] + p["kT"][a][i] * (T - p["TE"]) for i in range(2)]
        psis.append(-(m[0] ** 2 + m[1] ** 2) / (4 * p["A"][a]) - (m[0] * chat[0] + m[1] * chat[1])
                    + p["s"][a] * (T - p["TE"]))
    psi = sum(ph[a] ** 2 / S * psis[a] for a in range(4))
    gflat = [x for row in g for x in row]
    args = list(ph) + gflat
    dadp = sp.lambdify(args, [sp.diff(a_expr, ph[a]) for a in range(4)], "numpy")
    dadg = sp.lambdify(args, [[sp.diff(a_expr, g[a][d]) for d in range(3)] for a in range(4)], "numpy")
    domega = sp.lambdify(list(ph), [sp.diff(om, ph[a]) for a in range(4)], "numpy")
    dpsi = sp.lambdify(list(ph) + list(m) + [T], [sp.diff(psi, ph[a]) for a in range(4)], "numpy")
    return dadp, dadg, domega, dpsi


def _sym_fields(L, Lz):
    """Smooth phase fields on the simplex (softmax of trigonometric polynomials), periodic in
    x and y with period L, time dependent, and a smooth mu field."""
    x, y, z, t = sp.symbols("x y z t", real=True)
    kx, kz = 2 * sp.pi / L, 2 * sp.pi / Lz
    f = [0.6 * sp.sin(kx * x + 0.3) * sp.cos(kx * y) + 0.4 * sp.sin(kz * z) + 0.3 * t,
         0.5 * sp.cos(kx * x) * sp.sin(kx * y + 0.7) - 0.3 * sp.cos(kz * z + 0.2) - 0.2 * t,
         0.4 * sp.sin(kx * (x + y)) + 0.2 * sp.sin(2 * kz * z + 1.0) + 0.1 * t * sp.cos(kx * x),
         0.5 * sp.cos(kx * (x - y) + 0.4) + 0.5 * sp.cos(kz * z)]
    e = [sp.exp(fi) for fi in f]
    Z = sum(e)
    Phi = [ei / Z for ei in e]
    mu = [0.1 * sp.sin(kx * x + 0.5) * sp.cos(kz * z) + 0.05 * sp.cos(kx * y),
          -0.08 * sp.cos(kx * x) * sp.sin(kx * y) + 0.06 * sp.sin(kz * z + 0.1)]
    X = (x, y, z)
    Phi_f = sp.lambdify((x, y, z, t), Phi, "numpy")
    gPhi_f = sp.lambdify((x, y, z, t), [[sp.diff(Phi[a], X[d]) for d in range(3)] for a in range(4)], "numpy")
    mu_f = sp.lambdify((x, y, z), mu, "numpy")
    gmu_f = sp.lambdify((x, y, z), [[sp.diff(mu[c], X[d]) for d in range(3)] for c in range(2)], "numpy")
    return Phi_f, gPhi_f, mu_f, gmu_f


def _bcast(v, shape):
    return np.broadcast_to(np.asarray(v, dtype=float), shape)


def _grid(n, nz, dx):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    return i * dx, j * dx, k * dx


def _phi_on(Phi_f, X, Y, Z, t):
    return np.ascontiguousarray(np.stack([_bcast(v, X.shape) for v in Phi_f(X, Y, Z, t)]))


def _continuum_rhs(p, fields, model, X, Y, Z, t):
    Phi_f, gPhi_f, mu_f, _ = fields
    dadp, dadg, domega, dpsi = model
    shp = X.shape

    def state(x, y, z):
        ph = [_bcast(v, shp) for v in Phi_f(x, y, z, t)]
        gr = [[_bcast(v, shp) for v in row] for row in gPhi_f(x, y, z, t)]
        return ph, [v for row in gr for v in row]

    ph, gflat = state(X, Y, Z)
    # divergence of da/d(grad phi) by 4th-order central differences of the exact flux
    hh = 1e-3
    div = [np.zeros(shp) for _ in range(4)]
    for d in range(3):
        acc = [np.zeros(shp) for _ in range(4)]
        for w, s in [(-1.0, 2.0), (8.0, 1.0), (-8.0, -1.0), (1.0, -2.0)]:
            off = [X, Y, Z]
            off = [o + (s * hh if dd == d else 0.0) for dd, o in enumerate(off)]
            php, gp = state(*off)
            F = dadg(*php, *gp)
            for a in range(4):
                acc[a] = acc[a] + w * _bcast(F[a][d], shp)
        for a in range(4):
            div[a] += acc[a] / (12 * hh)
    T = p["T0"] + p["G"] * (Z - p["v"] * t)
    mu = [_bcast(v, shp) for v in mu_f(X, Y, Z)]
    A = dadp(*ph, *gflat)
    O = domega(*ph)
    S = dpsi(*ph, *mu, T)
    return np.stack([p["eps"] * T * (_bcast(A[a], shp) - div[a]) + T / p["eps"] * _bcast(O[a], shp)
                     + _bcast(S[a], shp) for a in range(4)])


def _conv_params():
    # a non-trivial parameter set (unequal gammas, curvatures, slopes) to expose index errors
    p = W.symmetric_params(G=0.02, v=0.05)
    p.update(gamma2=[1.0, 1.3, 0.8, 1.1, 0.9, 1.2], gamma3=[15.0, 12.0, 9.0, 14.0],
             A=[1.0, 1.2, 0.8, 1.1], D=[0.1, 0.2, 0.15, 1.0],
             kT=[[0.01, -0.02], [0.0, 0.03], [0.02, 0.0], [0.1, 0.12]],
             s=[1.0, 0.9, 1.1, 0.0], dt=0.01)
    return p


def test_phi_rhs_converges_to_continuum_at_second_order():
    p = _conv_params()
    model = _sym_model(p)
    L = 16.0
    fields = _sym_fields(L, L)
    errs = []
    for n in (16, 32):
        dx = L / n
        q = W.with_(p, dx=dx)
        X, Y, Z = _grid(n, n, dx)
        t = 0.7
        phi = _phi_on(fields[0], X, Y, Z, t)
        mu = np.ascontiguousarray(np.stack([_bcast(v, X.shape) for v in fields[2](X, Y, Z)]))
        _, rhs = oracle.phi_sweep(q, phi, mu, t=t, off=0.0, want_rhs=True)
        ref = _continuum_rhs(q, fields, model, X, Y, Z, t)
        kk = slice(2, n - 2)  # z interior (mirror boundaries are not part of the continuum problem)
        errs.append(np.abs(rhs[:, kk] - ref[:, kk]).max())
        scale = np.abs(ref).max()
    assert errs[1] < 0.02 * scale
    assert errs[0] / errs[1] > 3.3, errs  # second order: ratio -> 4


def _continuum_face_flux(p, fields, X, Y, Z, t0, t1, d):
    Phi_f, gPhi_f, mu_f, gmu_f = fields
    shp = X.shape
    ph = np.stack([_bcast(v, shp) for v in Phi_f(X, Y, Z, t1)])
    ph0 = np.stack([_bcast(v, shp) for v in Phi_f(X, Y, Z, t0)])
    gr = np.stack([np.stack([_bcast(v, shp) for v in row]) for row in gPhi_f(X, Y, Z, t1)])  # (4,3,...)
    mu = np.stack([_bcast(v, shp) for v in mu_f(X, Y, Z)])
    gmu = np.stack([np.stack([_bcast(v, shp) for v in row]) for row in gmu_f(X, Y, Z)])
    pdot = (ph - ph0) / (t1 - t0)
    # faces where every |grad phi| is well away from zero (the unit normal of Eq. 4 is
    # ill-conditioned at critical points of phi, where no fixed-order error bound holds)
    good = np.sqrt((gr ** 2).sum(1)).min(0) > 0.01
    S = (ph ** 2).sum(0)
    h = ph ** 2 / S
    M = sum(p["D"][a] * h[a] / (2 * p["A"][a]) for a in range(4))
    T = p["T0"] + p["G"] * (Z - p["v"] * t0)
    out = np.stack([M * gmu[c, d] for c in range(2)])
    nl = gr[3] / np.sqrt((gr[3] ** 2).sum(0))
    for a in range(3):
        na = gr[a] / np.sqrt((gr[a] ** 2).sum(0))
        ndot = (na * nl).sum(0)
        pref = math.pi * p["eps"] / 4 * ph[a] * h[3] / np.sqrt(ph[a] * ph[3]) * pdot[a] * ndot
        for c in range(2):
            cl = mu[c] / (2 * p["A"][3]) + p["cE"][3][c] + p["kT"][3][c] * (T - p["TE"])
            ca = mu[c] / (2 * p["A"][a]) + p["cE"][a][c] + p["kT"][a][c] * (T - p["TE"])
            out[c] = out[c] - pref * (cl - ca) * na[d]
    return out, good


def test_mu_face_flux_converges_to_continuum_at_second_order():
    # steep temperature dependence (G, kT) and a large dt: a face temperature taken at the
    # wrong height or phi taken at the wrong time level would leave an error that does not
    # shrink at second order
    p = _conv_params()
    p.update(G=0.3, dt=0.25, kT=[[0.1, -0.05], [0.0, 0.12], [0.08, 0.0], [0.5, 0.6]])
    L = 16.0
    fields = _sym_fields(L, L)
    t0 = 0.4
    errs = []
    for n in (32, 64):
        dx = L / n
        q = W.with_(p, dx=dx)
        t1 = t0 + q["dt"]
        X, Y, Z = _grid(n, n, dx)
        pold = _phi_on(fields[0], X, Y, Z, t0)
        pnew = _phi_on(fields[0], X, Y, Z, t1)
        mu = np.ascontiguousarray(np.stack([_bcast(v, X.shape) for v in fields[2](X, Y, Z)]))
        v = oracle.face_flux_field(q, pold, pnew, mu, t=t0, off=0.0)
        kk = slice(2, n - 2)
        e = 0.0
        sc = 0.0
        for d in range(3):
            sh = [0.0, 0.0, 0.0]
            sh[d] = 0.5 * dx
            ref, good = _continuum_face_flux(q, fields, X + sh[0], Y + sh[1], Z + sh[2], t0, t1, d)
            gk = good[kk]
            assert gk.mean() > 0.5
            e = max(e, np.abs(v[:, d, kk] - ref[:, kk])[:, gk].max())
            sc = max(sc, np.abs(ref).max())
        errs.append(e)
    assert errs[1] < 0.02 * sc
    assert errs[0] / errs[1] > 3.3, errs


def test_antitrapping_is_skipped_without_liquid_and_without_motion():
    # solid/solid face: J_at = 0 so v = M grad mu exactly; static field: J_at = 0 too
    rng = np.random.default_rng(5)
    p = _conv_params()
    n = 6
    phi = np.zeros((4, n, n, n))
    phi[0] = rng.uniform(0.2, 0.8, (n, n, n))
    phi[1] = 1.0 - phi[0]
    mu = rng.normal(scale=0.1, size=(2, n, n, n))
    v = oracle.face_flux_field(p, phi, phi, mu)
    for pn, po in [(phi, phi)]:
        vv = oracle.face_flux_field(p, po, pn, mu)
        np.testing.assert_array_equal(v, vv)
    # v along x equals M(phi_bar) (mu_R - mu_L)/dx computed by brute force
    pb = 0.5 * (phi + np.roll(phi, -1, axis=3))
    h = pb ** 2 / (pb ** 2).sum(0)
    M = sum(p["D"][a] * h[a] / (2 * p["A"][a]) for a in range(4))
    want = M * (np.roll(mu, -1, axis=3) - mu) / p["dx"]
    np.testing.assert_allclose(v[:, 0], want, rtol=1e-15, atol=1e-17)
    # a static three-phase field with liquid: dphi/dt = 0, so again no anti-trapping current
    phi3 = W.random_simplex_field(rng, n, n, n, sharp=0.0)
    v3 = oracle.face_flux_field(p, phi3, phi3, mu)
    pb = 0.5 * (phi3 + np.roll(phi3, -1, axis=3))
    h = pb ** 2 / (pb ** 2).sum(0)
    M = sum(p["D"][a] * h[a] / (2 * p["A"][a]) for a in range(4))
    np.testing.assert_allclose(v3[:, 0], M * (np.roll(mu, -1, axis=3) - mu) / p["dx"], rtol=1e-14, atol=1e-17)


def test_antitrapping_flux_points_into_the_liquid_for_a_growing_solid():
    # 1D alpha (below) / liquid (above) front moving up: the current carries the rejected
    # solute (c^l > c^alpha in component 1 of the symmetric set) into the liquid: v_z < 0 part
    # from J_at, i.e. J_z > 0 where c^l - c^alpha > 0.
    p = W.symmetric_params(G=0.0)
    p["dt"] = 0.01
    nz = 40
    old = W.planar_front(1, 1, nz, 20.0, 10.0)
    new = W.planar_front(1, 1, nz, 20.05, 10.0)
    mu = np.zeros((2, nz, 1, 1))
    v = oracle.face_flux_field(p, old, new, mu)
    # M grad mu = 0 here, so v = -J.  c^l - c^alpha = (1/3 - 0.8, 1/3 - 0.1) = (-, +)
    vz = v[:, 2, :, 0, 0]
    inside = slice(16, 24)
    assert (vz[1, inside] < 0).all() and (vz[0, inside] > 0).all()


# ---------------------------------------------------------------------------
# mu update: closed forms and conservation
# ---------------------------------------------------------------------------

def _liquid(nx, ny, nz):
    phi = np.zeros((4, nz, ny, nx))
    phi[3] = 1.0
    return phi


@pytest.mark.parametrize("m", [1, 3])
def test_mu_fourier_mode_decays_with_the_discrete_eigenvalue(m):
    nx, ny, nz = 24, 4, 3
    p = oracle.resolve_params(W.symmetric_params(G=0.0), nz)
    st = oracle.State(p, nx, ny, nz)
    st.phi = _liquid(nx, ny, nz)
    x = np.arange(nx)
    a = 0.01
    st.mu = np.zeros((2, nz, ny, nx))
    st.mu[0] = a * np.cos(2 * np.pi * m * x / nx)
    st.mu[1] = -2 * a * np.cos(2 * np.pi * m * x / nx)
    n = 60
    st.step(n)
    D, dt, dx = p["D"][3], p["dt"], p["dx"]
    lam = 1 - 4 * D * dt * math.sin(math.pi * m / nx) ** 2 / dx ** 2
    np.testing.assert_allclose(st.mu[0], a * lam ** n * np.cos(2 * np.pi * m * x / nx) + 0 * st.mu[0],
                               rtol=0, atol=1e-12 * a)
    np.testing.assert_allclose(st.mu[1], -2 * a * lam ** n * np.cos(2 * np.pi * m * x / nx) + 0 * st.mu[1],
                               rtol=0, atol=2e-12 * a)
    assert (st.phi == _liquid(nx, ny, nz)).all()


def test_mu_stability_threshold_of_the_checkerboard_mode():
    # pure liquid, x-y checkerboard (uniform in z, so the mirror boundary plays no part):
    # the discrete factor per step is 1 - 8 D dt / dx^2, which crosses -1 at dt = dx^2/(4 D)
    nx = ny = nz = 4
    cb = 1e-3 * (-1.0) ** np.indices((nz, ny, nx))[1:].sum(0)
    for frac, grows in [(0.95, False), (1.05, True)]:
        p = W.symmetric_params(G=0.0, dt=frac / 4.0)
        st = oracle.State(p, nx, ny, nz)
        st.phi = _liquid(nx, ny, nz)
        st.mu = np.stack([cb, cb])
        st.step(40)
        amp = np.abs(st.mu).max()
        assert (amp > 1e-3) == grows
        np.testing.assert_allclose(st.mu[0], cb * (1 - 8 * frac / 4.0) ** 40, rtol=1e-12)


def test_dc_dT_source_gives_the_closed_form_drift():
    nx, ny, nz = 4, 4, 4
    p = oracle.resolve_params(W.symmetric_params(G=2e-3, v=0.05), nz)
    st = oracle.State(p, nx, ny, nz)
    st.phi = _liquid(nx, ny, nz)
    st.mu = np.full((2, nz, ny, nx), 0.01)
    n = 50
    st.step(n)
    # chi = 1/(2 A_l);  dmu = -(2 A_l) kT_l (-G v dt) per step
    want = 0.01 + n * 2 * p["A"][3] * np.array(p["kT"][3]) * p["G"] * p["v"] * p["dt"]
    for c in range(2):
        np.testing.assert_allclose(st.mu[c], want[c], rtol=1e-13)


@pytest.mark.parametrize("G", [0.0, 2e-3])
def test_solute_is_conserved_to_roundoff_in_a_closed_box(G):
    nx, ny, nz = 16, 12, 24
    p = W.symmetric_params(G=G, v=0.05, n_grains=6)
    p["seed_layers"] = 12
    # unequal curvatures make chi = sum h_a/(2 A_a) depend on phi (with equal A it is constant)
    p["A"] = [1.0, 1.3, 0.8, 1.1]
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


# ---------------------------------------------------------------------------
# phi update
# ---------------------------------------------------------------------------

def test_lagrange_term_sums_to_zero_and_bulk_cells_are_fixed_points():
    rng = np.random.default_rng(2)
    n = 10
    phi = W.random_simplex_field(rng, n, n, n, sharp=0.6)
    phi[:, :3] = 0.0
    phi[3, :3] = 1.0  # a bulk liquid slab
    mu = W.random_mu(rng, n, n, n)
    p = oracle.resolve_params(W.symmetric_params(), n)
    new, star = oracle.phi_sweep(p, phi, mu, want_star=True)
    assert np.abs((star - phi).sum(0)).max() <= 1e-15
    # cells whose 7-point neighbourhood is one identical one-hot vector do not change
    bulk = np.ones((n, n, n), bool)
    for ax in (1, 2, 3):
        for s in (1, -1):
            nb = np.roll(phi, s, axis=ax)
            if ax == 1:  # mirror in z
                nb = phi.copy()
                if s == 1:
                    nb[:, 1:] = phi[:, :-1]
                else:
                    nb[:, :-1] = phi[:, 1:]
            bulk &= (nb == phi).all(0)
    bulk &= (phi == 1.0).any(0)
    assert bulk.sum() > 100
    assert (new[:, bulk] == phi[:, bulk]).all()


def test_flat_front_stays_flat_bitwise():
    nx, ny, nz = 12, 10, 40
    p = W.symmetric_params()
    st = oracle.State(p, nx, ny, nz)
    st.phi = W.planar_front(nx, ny, nz, 12.3, 9.0, solid=1)
    st.mu = np.zeros((2, nz, ny, nx))
    st.mu[0] += 0.01 * np.linspace(0, 1, nz)[:, None, None]
    st.step(100)
    for f in (st.phi, st.mu):
        assert (f == f[:, :, :1, :1]).all()


def test_periodic_translation_invariance_is_bitwise():
    nx, ny, nz = 16, 12, 20
    p = W.symmetric_params(n_grains=5)
    a = oracle.State(p, nx, ny, nz).init(7)
    b = oracle.State(p, nx, ny, nz)
    b.phi = np.roll(a.phi, (3, 5), axis=(2, 3)).copy()
    b.mu = np.roll(a.mu, (3, 5), axis=(2, 3)).copy()
    a.step(30)
    b.step(30)
    assert (np.roll(a.phi, (3, 5), axis=(2, 3)) == b.phi).all()
    assert (np.roll(a.mu, (3, 5), axis=(2, 3)) == b.mu).all()


def test_alpha_beta_and_component_swap_symmetry():
    nx, ny, nz = 12, 12, 20
    p = W.symmetric_params(n_grains=5)
    a = oracle.State(p, nx, ny, nz).init(9)
    rng = np.random.default_rng(0)
    a.mu = rng.uniform(-0.02, 0.02, a.mu.shape)
    b = oracle.State(p, nx, ny, nz)
    b.phi = a.phi[[1, 0, 2, 3]].copy()
    b.mu = a.mu[[1, 0]].copy()
    a.step(40)
    b.step(40)
    np.testing.assert_allclose(b.phi, a.phi[[1, 0, 2, 3]], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b.mu, a.mu[[1, 0]], rtol=0, atol=1e-12)


def _relax_profile(eps, nz, steps):
    p = W.symmetric_params(G=0.0)
    p.update(eps=eps, T0=1.0)
    st = oracle.State(p, 1, 1, nz)
    z0 = nz / 2 + 0.3
    st.phi = W.planar_front(1, 1, nz, z0, 0.6 * math.pi ** 2 * eps / 4)
    st.mu = np.zeros((2, nz, 1, 1))
    st.step(steps)
    prof = st.phi[0, :, 0, 0]
    # centre of the relaxed profile: where phi crosses 1/2 (linear interpolation)
    k = np.where((prof[:-1] >= 0.5) & (prof[1:] < 0.5))[0][0]
    zc = k + (prof[k] - 0.5) / (prof[k] - prof[k + 1])
    z = np.arange(nz)
    s = 4 * (z - zc) / (math.pi * eps)
    ref = np.where(s <= -math.pi / 2, 1.0, np.where(s >= math.pi / 2, 0.0, 0.5 * (1 - np.sin(np.clip(s, -7, 7)))))
    return np.abs(prof - ref).max(), st


def test_two_phase_equilibrium_profile_converges_to_the_obstacle_sine():
    # relaxation time grows with the profile width squared, hence 4x the steps for 2x eps
    e1, st1 = _relax_profile(4.0, 48, 4000)
    e2, st2 = _relax_profile(8.0, 64, 16000)
    # second-phase fields stay exactly zero (the projection keeps the profile two-phase)
    assert (st2.phi[1] == 0).all() and (st2.phi[2] == 0).all()
    assert e2 < 0.003
    assert e1 / e2 > 3.0, (e1, e2)


def _free_energy(p, phi):
    # F = sum over cells of eps T a(phi, grad phi) + (T/eps) omega(phi), central gradients,
    # evaluated in numpy independently of the oracle's sweep
    g = np.stack([np.gradient(phi, axis=ax) for ax in (3, 2, 1)], axis=1)  # (4,3,z,y,x)
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    a = sum(((phi[i] * g[j] - phi[j] * g[i]) ** 2).sum(0) for i, j in pairs)
    om = 16 / math.pi ** 2 * sum(phi[i] * phi[j] for i, j in pairs) + \
        15.0 * sum(phi[i] * phi[j] * phi[k] for i, j, k in [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)])
    return (p["eps"] * a + om / p["eps"]).sum()


def test_free_energy_decreases_at_the_eutectic_temperature():
    n = 16
    p = W.symmetric_params(G=0.0)
    p["T0"] = 1.0
    st = oracle.State(p, n, n, n)
    rng = np.random.default_rng(4)
    raw = rng.uniform(size=(4, n, n, n)) ** 4
    for _ in range(3):  # smooth a little
        raw = sum(np.roll(raw, s, axis=ax) for ax in (1, 2, 3) for s in (-1, 0, 1)) / 9
    st.phi = raw / raw.sum(0)
    st.mu = np.zeros((2, n, n, n))
    F = [_free_energy(p, st.phi)]
    for _ in range(6):
        st.step(10)
        F.append(_free_energy(p, st.phi))
    assert all(F[i + 1] < F[i] for i in range(len(F) - 1)), F


# ---------------------------------------------------------------------------
# window, initial condition, reductions
# ---------------------------------------------------------------------------

def test_window_shift_semantics():
    rng = np.random.default_rng(8)
    nx, ny, nz = 6, 5, 20
    p = W.symmetric_params(window_trigger_z=7.5)
    st = oracle.State(p, nx, ny, nz)
    phi = W.random_simplex_field(rng, nx, ny, nz)
    phi[:, 12:] = 0.0
    phi[3, 12:] = 1.0
    mu = W.random_mu(rng, nx, ny, nz)
    fr, so, h, bad = oracle.reduce(p, phi, mu)
    assert h == pytest.approx((1 - phi[3]).sum() / (nx * ny))
    import ctypes
    off = ctypes.c_double(2.0)
    ph2, mu2 = phi.copy(), mu.copy()
    s = oracle.lib().orc_window_shift(ctypes.byref(oracle.make_params(p)), nx, ny, nz, h, ctypes.byref(off),
                                      oracle._dp(ph2), oracle._dp(mu2))
    want_s = min(int(math.floor(h - 7.5)) + 1, nz - 1) if h >= 7.5 else 0
    assert s == want_s and s > 0
    assert off.value == 2.0 + s
    np.testing.assert_array_equal(ph2[:, : nz - s], phi[:, s:])
    np.testing.assert_array_equal(mu2[:, : nz - s], mu[:, s:])
    assert (ph2[3, nz - s:] == 1).all() and (ph2[:3, nz - s:] == 0).all()
    for k in range(nz - s, nz):
        np.testing.assert_array_equal(mu2[:, k], mu[:, nz - 1])
    # below the trigger nothing moves
    off2 = ctypes.c_double(0.0)
    q = W.with_(p, window_trigger_z=h + 0.01)
    s2 = oracle.lib().orc_window_shift(ctypes.byref(oracle.make_params(q)), nx, ny, nz, h, ctypes.byref(off2),
                                       oracle._dp(ph2), oracle._dp(mu2))
    assert s2 == 0 and off2.value == 0.0


def test_window_moves_in_a_step_and_temperature_follows_the_offset():
    nx, ny, nz = 8, 8, 24
    p = W.symmetric_params(window_trigger_z=9.0, n_grains=4)
    p["seed_layers"] = 10
    st = oracle.State(p, nx, ny, nz).init(1)
    st.step(1)
    assert st.shifts >= 1 and st.off == float(st.shifts)
    # after the shift the state equals an unshifted run's fields moved down by s planes
    ref = oracle.State(W.with_(p, window_trigger_z=0.0), nx, ny, nz).init(1)
    ref.step(1)
    s = st.shifts
    np.testing.assert_array_equal(st.phi[:, : nz - s], ref.phi[:, s:])
    np.testing.assert_array_equal(st.mu[:, : nz - s], ref.mu[:, s:])
    assert oracle.temperature(st.params, (0 + st.off) * p["dx"], st.t) == \
        oracle.temperature(ref.params, (s + ref.off) * p["dx"], ref.t)


def test_voronoi_initial_condition_is_the_nearest_seed():
    nx, ny, nz = 20, 14, 16
    p = W.symmetric_params(n_grains=9)
    st = oracle.State(p, nx, ny, nz).init(123)
    seeds = oracle.voronoi_seeds(nx, ny, 8, 9, 123)
    # seeds follow the splitmix64 stream: 4 draws per grain, u = (x >> 11) 2^-53
    raw = oracle.splitmix64(123, 36)
    u = np.array([(x >> 11) * 2.0 ** -53 for x in raw]).reshape(9, 4)
    np.testing.assert_array_equal(seeds[:, 0], u[:, 0] * nx)
    np.testing.assert_array_equal(seeds[:, 1], u[:, 1] * ny)
    np.testing.assert_array_equal(seeds[:, 2], u[:, 2] * 8)
    np.testing.assert_array_equal(seeds[:, 3], np.floor(3 * u[:, 3]))
    k, j, i = np.meshgrid(np.arange(8), np.arange(ny), np.arange(nx), indexing="ij")
    best_d = np.full(k.shape, np.inf)
    for g in range(9):
        dx = np.abs(i + 0.5 - seeds[g, 0])
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(j + 0.5 - seeds[g, 1])
        dy = np.minimum(dy, ny - dy)
        dz = np.abs(k + 0.5 - seeds[g, 2])
        best_d = np.minimum(best_d, dx * dx + dy * dy + dz * dz)
    gr = st.grain[:8]
    dsel = np.zeros(k.shape)
    for g in range(9):
        m = gr == g
        dx = np.abs(i + 0.5 - seeds[g, 0])
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(j + 0.5 - seeds[g, 1])
        dy = np.minimum(dy, ny - dy)
        dz = np.abs(k + 0.5 - seeds[g, 2])
        dsel[m] = (dx * dx + dy * dy + dz * dz)[m]
    np.testing.assert_allclose(dsel, best_d, rtol=1e-15)
    ph = seeds[gr, 3].astype(int)
    onehot = np.moveaxis(np.eye(4)[ph], -1, 0)
    np.testing.assert_array_equal(st.phi[:, :8], onehot)
    assert (st.phi[3, 8:] == 1).all() and (st.grain[8:] == -1).all()
    assert (st.mu == 0).all()


def test_reductions_match_brute_force():
    rng = np.random.default_rng(12)
    nx, ny, nz = 7, 9, 11
    p = W.symmetric_params(G=3e-3)
    phi = W.random_simplex_field(rng, nx, ny, nz)
    mu = W.random_mu(rng, nx, ny, nz)
    t, off = 1.7, 3.0
    fr, so, h, bad = oracle.reduce(p, phi, mu, t, off)
    np.testing.assert_allclose(fr, phi.reshape(4, -1).mean(1), rtol=1e-14)
    assert h == pytest.approx((1 - phi[3]).sum() / (nx * ny), rel=1e-14)
    T = p["T0"] + p["G"] * ((np.arange(nz) + off)[:, None, None] - p["v"] * t)
    hh = phi ** 2 / (phi ** 2).sum(0)
    want = [sum(hh[a] * (mu[c] / 2 + p["cE"][a][c] + p["kT"][a][c] * (T - 1.0)) for a in range(4)).sum()
            for c in range(2)]
    np.testing.assert_allclose(so, want, rtol=1e-13)
    assert not bad
    mu[1, 3, 4, 5] = np.nan
    assert oracle.reduce(p, phi, mu, t, off)[3]
