"""The fused step's pure-liquid shortcut (the paper's Section 3.3 shortcuts) against the oracle.

On a plane whose phi^n neighbourhood is pure liquid the fused step neither loads phi^n (the
liquid map says it is e_l) nor stores phi^{n+1} where the destination buffer already holds pure
liquid (its own map, which describes the field two steps back).  Results must not depend on
what the destination buffer held: these cases make that content differ from the new field
(host writes between steps, melting solid, window shifts) and compare with the oracle at the
FP64 tolerance (1e-12; mu relative to max(|mu_ref|_inf, 1e-8)).  The per-step byte tally the
kernels report is checked against the design's word counts.
"""
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


def _liquid(nx, ny, nz, rng, scale=1e-3):
    phi = np.zeros((4, nz, ny, nx))
    phi[3] = 1.0
    return phi, rng.uniform(-scale, scale, size=(2, nz, ny, nx))


@pytest.mark.parametrize("shape", [(70, 21, 40), (32, 8, 24)])
def test_host_writes_between_fused_steps_match_the_oracle(shape):
    # run a solid/liquid front, then overwrite the state with pure liquid: the buffer the next
    # step writes still holds solid cells where the new field is liquid
    nx, ny, nz = shape
    rng = np.random.default_rng(7)
    p = W.symmetric_params(G=2e-3)
    sim = pf.Simulation(nx, ny, nz, p, "fp64", variant="fused")
    phi0, mu0 = W.region_fields("interface", nx, ny, nz, seed=3)
    sim.set_fields(phi0, mu0)
    sim.step(3)
    phi1, mu1 = _liquid(nx, ny, nz, rng)
    phi1[:, nz - 4:] = phi0[:, : 4]  # a few solid planes at the top, so both paths run
    sim.set_fields(phi1, mu1)
    ref = oracle.State(p, nx, ny, nz)
    ref.phi, ref.mu = phi1.copy(), mu1.copy()
    ref.t = sim.stats()["t"]
    sim.step(5)
    ref.step(5)
    phi, mu = sim.fields()
    assert np.abs(phi - ref.phi).max() <= 1e-12
    assert _mu_err(mu, ref.mu) <= 1e-12
    sim.close()


def test_melting_solid_matches_the_oracle():
    # thin solid columns well above the eutectic temperature melt: after the interfaces have
    # spread, cells turn pure liquid again while the destination buffer still holds their
    # diffuse state from two steps back.  FP64, where the shortcut must be exact to 1e-12 (the
    # shortcut's logic is the same template in both precisions; this forced melt drives phi far
    # harder than the solidification runs the FP32 tolerance is stated for)
    precision, tol = "fp64", 1e-12
    nx, ny, nz = 40, 24, 32
    p = W.symmetric_params(G=0.0)
    p["T0"] = 1.2  # above TE = 1 everywhere
    phi0, mu0 = W.region_fields("interface", nx, ny, nz, seed=1)
    phi0[:, 4:] = 0.0  # solid columns in planes 0..3 only, liquid above
    phi0[3, 4:] = 1.0
    sim = pf.Simulation(nx, ny, nz, p, precision, variant="fused")
    sim.set_fields(phi0, mu0)
    ref = oracle.State(p, nx, ny, nz)
    ref.phi, ref.mu = phi0.copy(), mu0.copy()
    for _ in range(2):
        sim.step(150)
        ref.step(150)
        phi, mu = sim.fields()
        assert np.abs(phi - ref.phi).max() <= tol
        assert _mu_err(mu, ref.mu) <= tol
        if _ == 0:
            liquid_mid = (ref.phi[3] == 1.0).mean()
    assert (ref.phi[3] == 1.0).mean() > liquid_mid + 0.02  # cells did turn pure liquid
    sim.close()


def test_step_bytes_follow_the_design_word_counts():
    nx, ny, nz = 64, 40, 48
    cells = nx * ny * nz
    rng = np.random.default_rng(0)
    phi_l, mu_l = _liquid(nx, ny, nz, rng)
    p = W.symmetric_params()
    # two sweeps: 10 + 12 words a cell, 18 + 16 with the compensated low words
    for prec, w, kp, km in (("fp32", 4, 10, 12), ("fp64", 8, 10, 12), ("fp32c", 4, 18, 16)):
        sim = pf.Simulation(nx, ny, nz, p, prec, variant="unfused")
        sim.set_fields(phi_l, mu_l)
        assert sim.step_bytes() == {}
        sim.step(2)
        assert sim.step_bytes() == {"phi_sweep": kp * w * cells, "mu_sweep": km * w * cells}, prec
        sim.close()
    # fused step on pure liquid (nx even: the lean kernel takes every plane): mu in and out only
    # (4 words a cell) once the destination holds pure liquid too
    for prec, w in (("fp32", 4), ("fp64", 8)):
        sim = pf.Simulation(nx, ny, nz, p, prec, variant="fused")
        sim.set_fields(phi_l, mu_l)
        sim.step(3)
        assert sim.step_bytes() == {"lean_step": 4 * w * cells}, prec
        sim.close()
    # odd nx: the fused kernel runs the pure-liquid planes itself
    sim = pf.Simulation(nx - 1, ny, nz, p, "fp32", variant="fused")
    sim.set_fields(phi_l[:, :, :, 1:], mu_l[:, :, :, 1:])
    sim.step(3)
    assert sim.step_bytes() == {"fused_step": 16 * (nx - 1) * ny * nz}
    sim.close()
    # a solidification front: the general planes run as the two sweeps (22 words a cell), the
    # pure-liquid planes in the lean kernel (4 words a cell)
    sim = pf.Simulation(nx, ny, nz, p, "fp32", variant="fused")
    phi_i, mu_i = W.region_fields("interface", nx, ny, nz, seed=0)
    sim.set_fields(phi_i, mu_i)
    sim.step(3)
    b = sim.step_bytes()
    assert set(b) == {"general_sweeps", "lean_step"}
    assert b["general_sweeps"] % (88 * nx) == 0  # whole tile rows of 22 words a cell
    assert 16 * cells < sum(b.values()) < 88 * cells
    sim.close()


def test_lean_kernel_matches_the_oracle_on_wrapping_and_ragged_tiles():
    # even nx (the lean kernel's tensor copies), tiles that wrap in x and y, a ragged last tile in
    # x (nx = 40: 32 + 8) and y (ny = 13), nx = 2 (a cell's x neighbours are the same cell), a
    # thin front so that both kernels run, FP64 and FP32
    for (nx, ny, nz) in ((40, 13, 70), (2, 9, 33), (64, 8, 20)):
        rng = np.random.default_rng(nx + ny)
        p = W.symmetric_params(G=1e-3)
        phi0, mu0 = _liquid(nx, ny, nz, rng, scale=0.05)
        phi0[:, nz // 2] = W.random_simplex_field(rng, nx, ny, 1, sharp=0.5)[:, 0]
        for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
            a, m = phi0, mu0
            if prec == "fp32":
                a = a.astype(np.float32).astype(np.float64)
                m = m.astype(np.float32).astype(np.float64)
            sim = pf.Simulation(nx, ny, nz, p, prec, variant="fused")
            sim.set_fields(a, m)
            ref = oracle.State(p, nx, ny, nz)
            ref.phi, ref.mu = a.copy(), m.copy()
            sim.step(6)
            ref.step(6)
            assert "lean_step" in sim.step_bytes()
            phi, mu = sim.fields()
            assert np.abs(phi - ref.phi).max() <= tol, (nx, ny, nz, prec)
            assert _mu_err(mu, ref.mu) <= tol, (nx, ny, nz, prec)
            sim.close()
