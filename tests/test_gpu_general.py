"""General parabolic thermodynamics on the GPU (matrix curvatures A_a, the 2x2 susceptibility
inverse, the matrix mobility and pair relaxation times) against the oracle, through the C ABI.

Tolerances as for the symmetric set: FP64 1e-12 (phi absolute; mu relative to max(|mu_ref|_inf,
1e-8)), FP32 2e-5.  Every kernel path runs: the two sweeps, the fused step (odd nx), the lean
kernel beside the general planes (even nx), the compensated FP32 sweeps, the batch and the
moving window.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1506_01684_gb300 import pf
from paper_1506_01684_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.lib()


def _mu_err(mu, ref):
    return np.abs(mu - ref).max() / max(np.abs(ref).max(), 1e-8)


def _params(**kw):
    p = W.general_params(**kw)
    p["D"] = [0.2, 0.0, 0.1, 1.0]  # two solids diffuse too: interfaces with a full matrix mobility
    return p


def test_effective_dt_takes_the_smallest_pair_time():
    p = _params()
    sim = pf.Simulation(8, 8, 64, p)
    assert sim.params.dt == oracle.default_dt(p, 64)
    assert sim.params.dt < oracle.default_dt(W.symmetric_params(), 64)
    sim.close()


@pytest.mark.parametrize("variant", ["unfused", "fused", "auto"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_grains_match_the_oracle(variant, precision, tol):
    # 36 x 20 x 40 (even nx: the auto path runs the lean kernel beside the general planes),
    # 9 grains, 120 steps
    nx, ny, nz = 36, 20, 40
    p = _params(G=2e-3, n_grains=9)
    p["seed_layers"] = 10
    sim = pf.Simulation(nx, ny, nz, p, precision, variant=variant)
    ref = oracle.State(p, nx, ny, nz)
    sim.init(4)
    ref.init(4)
    sim.step(120)
    ref.step(120)
    phi, mu = sim.fields()
    e_phi, e_mu = np.abs(phi - ref.phi).max(), _mu_err(mu, ref.mu)
    print(f"{precision} {variant}: max|dphi| = {e_phi:.3e}, |dmu|/scale = {e_mu:.3e}")
    assert e_phi <= tol and e_mu <= tol
    if precision == "fp64":
        st = sim.stats()
        fr, so, h, _ = ref.reduce()
        np.testing.assert_allclose(st["solute"], so, rtol=1e-12)
    sim.close()


@pytest.mark.parametrize("shape", [(37, 21, 19), (2, 3, 5), (64, 8, 3)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("variant", ["unfused", "fused"])
def test_random_states_match_the_oracle(shape, precision, tol, variant):
    # diffuse cells with up to four phases everywhere (every matrix and pair-time term active)
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + nz)
    p = _params(G=2e-3)
    phi0 = W.random_simplex_field(rng, nx, ny, nz, sharp=0.4)
    mu0 = W.random_mu(rng, nx, ny, nz, scale=0.05)
    if precision == "fp32":
        phi0 = phi0.astype(np.float32).astype(np.float64)
        mu0 = mu0.astype(np.float32).astype(np.float64)
    sim = pf.Simulation(nx, ny, nz, p, precision, variant=variant)
    ref = oracle.State(p, nx, ny, nz)
    sim.set_fields(phi0, mu0)
    ref.phi, ref.mu = phi0.copy(), mu0.copy()
    sim.step(5)
    ref.step(5)
    phi, mu = sim.fields()
    assert np.abs(phi - ref.phi).max() <= tol
    assert _mu_err(mu, ref.mu) <= tol
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_lean_kernel_with_matrix_curvatures(precision, tol):
    # pure liquid with a thin front in the middle and a temperature drift: the lean kernel's
    # constants C1 = dt D_l / dx^2, C0 = -K_l^{-1} k_l dT
    nx, ny, nz = 40, 13, 60
    rng = np.random.default_rng(3)
    p = _params(G=5e-3, v=0.05)
    phi0 = np.zeros((4, nz, ny, nx))
    phi0[3] = 1.0
    phi0[:, nz // 2] = W.random_simplex_field(rng, nx, ny, 1, sharp=0.5)[:, 0]
    mu0 = rng.uniform(-0.05, 0.05, size=(2, nz, ny, nx))
    if precision == "fp32":
        phi0 = phi0.astype(np.float32).astype(np.float64)
        mu0 = mu0.astype(np.float32).astype(np.float64)
    sim = pf.Simulation(nx, ny, nz, p, precision, variant="fused")
    ref = oracle.State(p, nx, ny, nz)
    sim.set_fields(phi0, mu0)
    ref.phi, ref.mu = phi0.copy(), mu0.copy()
    sim.step(8)
    ref.step(8)
    assert "lean_step" in sim.step_bytes()
    phi, mu = sim.fields()
    assert np.abs(phi - ref.phi).max() <= tol
    assert _mu_err(mu, ref.mu) <= tol
    sim.close()


@pytest.mark.parametrize("variant", ["unfused", "fused"])
def test_moving_window_with_general_thermodynamics(variant):
    p = _params(window_trigger_z=7.0)
    p["seed_layers"] = 10
    nx, ny, nz = 32, 16, 48
    sim = pf.Simulation(nx, ny, nz, p, "fp64", variant=variant)
    ref = oracle.State(p, nx, ny, nz)
    sim.init(3)
    ref.init(3)
    sim.step(60)
    ref.step(60)
    assert ref.shifts > 0 and sim.shifts() == ref.shifts
    phi, mu = sim.fields()
    assert np.abs(phi - ref.phi).max() <= 1e-12
    assert _mu_err(mu, ref.mu) <= 1e-12
    sim.close()


def test_compensated_fp32_with_general_thermodynamics():
    # the compensated state against the FP64 GPU path, at the FP32 tolerance
    nx, ny, nz = 24, 16, 32
    p = _params(G=2e-3, n_grains=6)
    out = {}
    for prec in ("fp64", "fp32c"):
        sim = pf.Simulation(nx, ny, nz, p, prec)
        sim.init(2)
        sim.step(100)
        out[prec] = sim.fields()
        sim.close()
    assert np.abs(out["fp32c"][0] - out["fp64"][0]).max() <= 2e-5
    assert _mu_err(out["fp32c"][1], out["fp64"][1]) <= 2e-5


def test_batch_of_general_and_symmetric_domains_equals_single_runs():
    shapes = [(32, 16, 40), (24, 24, 24), (33, 8, 30)]
    params = [_params(n_grains=5), W.symmetric_params(n_grains=4), _params(n_grains=3, window_trigger_z=9.0)]
    for q in params:
        q["seed_layers"] = 10
    b = pf.Batch(shapes, params, "fp32")
    b.init([1, 2, 3])
    b.step(40)
    got = [b.fields(d) for d in range(len(shapes))]
    b.close()
    for d, ((nx, ny, nz), q) in enumerate(zip(shapes, params)):
        sim = pf.Simulation(nx, ny, nz, q, "fp32", variant="fused")  # the kernels a batched domain takes
        sim.init(d + 1)
        sim.step(40)
        phi, mu = sim.fields()
        sim.close()
        # FP32: the batched and single kernels are separate instantiations whose multiply-adds the
        # compiler may contract differently, and after a window shift the two may refresh their
        # liquid maps at different points: equal to FP32 rounding (both match the oracle,
        # test_odd_width_domain_with_a_moving_window_in_a_batch)
        assert np.abs(got[d][0] - phi).max() <= 1e-6, d
        assert _mu_err(got[d][1], mu) <= 1e-6, d


def test_invalid_general_parameters_are_refused():
    L = pf.lib()
    h = ctypes.c_void_p()
    for change in ({"Am": [[1.0, 2.0, 1.0]] + [[0.0, 0.0, 0.0]] * 3},       # not positive definite
                   {"Am": [[1.0, 0.1, -1.0]] + [[0.0, 0.0, 0.0]] * 3},      # negative a22
                   {"tau_ab": [1.0, 1.0, 0.0, 1.0, 1.0, 1.0]}):             # some pairs without a time
        p = pf.params_from_dict(dict(W.symmetric_params(), **change))
        assert L.pf_create(8, 8, 8, ctypes.byref(p), None, ctypes.byref(h)) == pf.PF_E_INVAL
