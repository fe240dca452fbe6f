"""PF_VARIANT_AUTO chooses the step's path from the state: the lean path (plan, lean kernel, general
planes' sweeps) where the current field's liquid map is mostly pure liquid, the two whole-domain
sweeps of Algorithm 1 elsewhere.  The measure is the fraction f of exactly pure-liquid (tile, plane)
entries; the lean path needs f >= 0.6 on domains of 2^20 to 2^23 cells, f >= 0.45 on larger ones, and
is always kept below 2^20 cells.  The choice is made from the state on the first step after the state
is set, so two runs from one state choose alike, and it travels in checkpoints, so a resumed run
continues on the same path."""
import numpy as np
import pytest

from paper_1506_01684_gb300 import pf
from paper_1506_01684_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.lib()


def _path(sim):
    # the lean path tallies its lean kernel and its general planes' sweeps (a domain without pure-
    # liquid planes has only the latter); the two whole-domain sweeps tally phi_sweep and mu_sweep
    b = sim.step_bytes()
    if set(b) & {"lean_step", "general_sweeps"}:
        assert not set(b) & {"phi_sweep", "mu_sweep"}, b
        return "lean"
    assert set(b) == {"phi_sweep", "mu_sweep"}, b
    return "sweeps"


def _sim(nx, ny, nz, layers, precision="fp32"):
    p = W.symmetric_params(n_grains=12)
    p["seed_layers"] = layers
    sim = pf.Simulation(nx, ny, nz, p, precision)
    sim.init(5)
    return sim


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_auto_takes_the_lean_path_on_a_liquid_dominated_domain(precision):
    # 128^2 x 128 (2^21 cells), Voronoi seeds in the bottom 8 planes: ~90 % pure-liquid map entries
    sim = _sim(128, 128, 128, 8, precision)
    sim.step(4)
    assert _path(sim) == "lean"


def test_auto_takes_the_sweeps_on_a_solid_dominated_domain():
    # seeds filling 48 of 64 planes: f ~ 0.2
    sim = _sim(128, 128, 64, 48)
    sim.step(4)
    assert _path(sim) == "sweeps"


def test_auto_keeps_the_lean_path_on_small_domains():
    # 32 x 32 x 64 (2^16 cells): the lean path whatever the composition (10 or 60 seeded planes)
    for layers in (10, 60):
        sim = _sim(32, 32, 64, layers)
        sim.step(4)
        assert _path(sim) == "lean", layers


def test_auto_on_a_large_domain_takes_the_lower_threshold():
    # 256 x 256 x 128 (2^23 cells): half the planes seeded (f ~ 0.5) keeps the lean path, three
    # quarters (f ~ 0.25) take the sweeps
    for layers, want in ((64, "lean"), (96, "sweeps")):
        sim = _sim(256, 256, 128, layers)
        sim.step(4)
        assert _path(sim) == want, layers
        sim.close()


def test_the_choice_travels_in_a_checkpoint(tmp_path):
    path = str(tmp_path / "auto.pfc")
    a = _sim(128, 128, 64, 48)  # chooses the sweeps
    a.step(3)
    a.checkpoint(path)
    b = _sim(128, 128, 128 // 2, 4)  # a liquid state of the same grid: would choose the lean path
    b.step(3)
    assert _path(b) == "lean"
    b.restore(path)
    b.step(3)
    assert _path(b) == "sweeps"
    a.step(3)
    pa, ma = a.fields()
    pb, mb = b.fields()
    assert np.array_equal(pa, pb) and np.array_equal(ma, mb)
    # new fields: AUTO chooses again from the state at the next step
    b.set_fields(*_sim(128, 128, 64, 4).fields())
    b.step(3)
    assert _path(b) == "lean"
