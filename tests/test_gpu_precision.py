"""Compensated FP32 (PF_FP32_COMP): the state is kept as hi + lo FP32 pairs; increments formed in
FP32 are accumulated without loss.  Checked against the oracle and against closed forms."""
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


def test_compensated_state_keeps_increments_below_the_fp32_spacing():
    # pure liquid, uniform mu = 1: each step adds 2 A kT G v dt (the dc/dT dT/dt source, Eq. 3),
    # about 7.9e-8, less than half the FP32 spacing at 1.0 -- plain FP32 rounds every step
    nx = ny = nz = 8
    p = W.symmetric_params(G=1e-3, v=1e-2)
    phi = np.zeros((4, nz, ny, nx))
    phi[3] = 1.0
    mu = np.ones((2, nz, ny, nx))
    n = 1000
    res = {}
    for prec in ("fp32", "fp32c", "fp64"):
        sim = pf.Simulation(nx, ny, nz, p, prec)
        sim.set_fields(phi, mu)
        sim.step(n)
        res[prec] = sim.fields()[1]
        dt = sim.params.dt
        sim.close()
    q = oracle.resolve_params(p, nz)
    assert q["dt"] == dt
    want = 1.0 + n * 2 * 1.0 * 0.1 * p["G"] * p["v"] * dt
    err = {k: np.abs(v - want).max() / (want - 1.0) for k, v in res.items()}
    print("relative error of the accumulated drift:", err)
    # FP64 accumulates ~1000 half-ulp roundings of 1.0 against a drift of ~8e-5: ~1e-9 relative;
    # compensated FP32 keeps every increment (its error is the FP32 rounding of the increment);
    # plain FP32 rounds each increment to a whole spacing of 1.0
    assert err["fp64"] < 1e-8
    assert err["fp32c"] < 1e-7
    assert err["fp32"] > 1e4 * err["fp32c"]


# "fused" takes the lean path wherever it can run: (32, 32, 64) and (40, 24, 48) run the plan, the lean
# kernel and the general planes' sweeps in compensated form; an odd nx or nx = 1 has no tensor map for
# the lean kernel and runs the two whole-domain sweeps, as does the explicit "unfused" variant; "auto"
# chooses between the two from the state
@pytest.mark.parametrize("variant", ["auto", "fused", "unfused"])
@pytest.mark.parametrize("shape", [(32, 32, 64), (40, 24, 48), (37, 21, 19), (1, 1, 16)])
def test_compensated_path_matches_the_oracle(shape, variant):
    nx, ny, nz = shape
    p = W.symmetric_params(n_grains=6)
    sim = pf.Simulation(nx, ny, nz, p, "fp32c", variant=variant)
    ref = oracle.State(p, nx, ny, nz)
    sim.init(7)
    ref.init(7)
    sim.step(100)
    ref.step(100)
    phi, mu = sim.fields()
    e_phi = np.abs(phi - ref.phi).max()
    e_mu = np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8)
    print(f"fp32c vs oracle {shape}: {e_phi:.3e} {e_mu:.3e}")
    assert e_phi <= 2e-5 and e_mu <= 2e-5
    # the compensated state sums to one far below the FP32 spacing
    assert np.abs(phi.sum(0) - 1).max() <= 1e-12 and phi.min() >= 0


def test_compensated_fields_round_trip_through_the_host():
    rng = np.random.default_rng(4)
    nx, ny, nz = 9, 7, 5
    phi = W.random_simplex_field(rng, nx, ny, nz)
    mu = W.random_mu(rng, nx, ny, nz)
    sim = pf.Simulation(nx, ny, nz, W.symmetric_params(), "fp32c")
    sim.set_fields(phi, mu)
    phi2, mu2 = sim.fields()
    # hi + lo carries 48 significant bits
    assert np.abs(phi2 - phi).max() <= 1e-14
    assert np.abs(mu2 - mu).max() <= 1e-14


def test_compensated_window_shift_matches_the_oracle():
    p = W.symmetric_params(window_trigger_z=7.0)
    p["seed_layers"] = 10
    sim = pf.Simulation(32, 32, 64, p, "fp32c")
    ref = oracle.State(p, 32, 32, 64)
    sim.init(3)
    ref.init(3)
    sim.step(60)
    ref.step(60)
    assert ref.shifts > 0 and sim.shifts() == ref.shifts
    phi, mu = sim.fields()
    assert np.abs(phi - ref.phi).max() <= 2e-5
    assert np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8) <= 2e-5


def test_compensated_lean_kernel_moves_the_low_words():
    # pure liquid: every plane is lean; the lean kernel's tally is mu^n in and mu^{n+1} out with their
    # low words, 32 bytes a cell (16 in plain FP32), once phi^{n+1} = e_l is known to be stored
    nx, ny, nz = 64, 32, 48
    p = W.symmetric_params()
    phi = np.zeros((4, nz, ny, nx))
    phi[3] = 1.0
    rng = np.random.default_rng(2)
    mu = rng.uniform(-1e-3, 1e-3, (2, nz, ny, nx))
    for prec, per_cell in (("fp32", 16.0), ("fp32c", 32.0)):
        sim = pf.Simulation(nx, ny, nz, p, prec)
        sim.set_fields(phi, mu)
        sim.step(4)
        b = sim.step_bytes()
        assert set(b) == {"lean_step"}, b
        assert b["lean_step"] == per_cell * nx * ny * nz
        sim.close()


def test_compensated_lean_and_sweeps_agree_over_a_growing_front():
    # the lean path (its general planes included) and the whole-domain sweeps compute the same step
    # in compensated form: after 300 steps of a growing front they agree far inside the FP32 tolerance
    nx, ny, nz = 64, 32, 64
    p = W.symmetric_params(n_grains=8, G=2e-3)
    out = {}
    for variant in ("fused", "unfused"):
        sim = pf.Simulation(nx, ny, nz, p, "fp32c", variant=variant)
        sim.init(11)
        sim.step(300)
        if variant == "fused":
            assert "lean_step" in sim.step_bytes()
        out[variant] = sim.fields()
        sim.close()
    (pa, ma), (pu, mu_) = out["fused"], out["unfused"]
    assert np.abs(pa - pu).max() <= 2e-6
    assert np.abs(ma - mu_).max() / max(np.abs(mu_).max(), 1e-8) <= 2e-6


@pytest.mark.parametrize("variant", ["auto", "unfused"])
def test_compensated_state_stays_within_tolerance_across_the_pair_tau_jump(variant):
    # The general set's relaxation time is the phi-weighted mean of the pair values on a mixed cell
    # and the single tau on a single-phase cell, so it jumps where a phase starts to appear.  On this
    # domain phase 0 grows into a phase-1 cell at step 12: FP64 reaches step 11 with that cell exactly
    # single-phase, plain FP32 with a rounding residue of ~4e-8 in phase 0, which selects the pair
    # value (twice the single tau) and halves that step's growth -- a departure of ~1e-4, above the
    # 2e-5 tolerance.  The compensated state carries the residue's value exactly enough to take the
    # same side as FP64 and the oracle.
    rng = np.random.default_rng(201)
    p = W.general_params(G=float(rng.uniform(5e-4, 2e-3)), v=float(rng.uniform(5e-3, 2e-2)),
                         n_grains=int(rng.integers(2, 9)))
    shape, seed, steps = (37, 21, 40), 13, 25
    ref = oracle.State(p, *shape).init(seed)
    ref.step(steps)
    err = {}
    for prec in ("fp64", "fp32c", "fp32"):
        sim = pf.Simulation(*shape, p, prec, variant=variant)
        sim.init(seed)
        sim.step(steps)
        phi, mu = sim.fields()
        err[prec] = (float(np.abs(phi - ref.phi).max()),
                     float(np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8)))
        sim.close()
    print(variant, "max |dphi|, |dmu|/scale against the oracle:", err)
    assert err["fp64"][0] <= 1e-12 and err["fp64"][1] <= 1e-12
    assert err["fp32c"][0] <= 2e-5 and err["fp32c"][1] <= 2e-5


@pytest.mark.parametrize("thermo", ["symmetric", "general"])
def test_fp32_forms_stay_within_tolerance_of_fp64_over_seeds(thermo):
    # 32x32x64, 12 grains, 200 steps, sixteen Voronoi seeds: both FP32 forms against the FP64 path
    # (itself within 1e-12 of the oracle, test_gpu_parity.py).  Runs are bitwise reproducible, so
    # the worst seed is fixed; over 64 seeds the worst plain-FP32 errors were 5.2e-6 (symmetric) and
    # 1.0e-5 (general), the compensated ones 1.3e-6 and 7.0e-7.
    f = W.symmetric_params if thermo == "symmetric" else W.general_params
    p = f()
    worst = {"fp32": 0.0, "fp32c": 0.0}
    for seed in range(16):
        out = {}
        for prec in ("fp64", "fp32", "fp32c"):
            sim = pf.Simulation(32, 32, 64, p, prec)
            sim.init(seed)
            sim.step(200)
            out[prec] = sim.fields()
            sim.close()
        phi64, mu64 = out["fp64"]
        scale = max(np.abs(mu64).max(), 1e-8)
        for prec in ("fp32", "fp32c"):
            phi, mu = out[prec]
            e = max(float(np.abs(phi - phi64).max()), float(np.abs(mu - mu64).max() / scale))
            worst[prec] = max(worst[prec], e)
            assert e <= 2e-5, (prec, seed, e)
    print(thermo, "worst over 16 seeds:", worst)
