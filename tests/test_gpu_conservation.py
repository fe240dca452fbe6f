"""Solute conservation on the GPU paths: in a closed box (periodic in x and y, zero flux through the
mirror planes in z, no window shift) Eq. 3 changes the total solute only by the divergence of the face
fluxes, which cancels between neighbouring cells, so the total of c = sum_a h_a c^a(mu, T) stays
constant to roundoff -- also under the frozen temperature gradient, whose dc/dT term the mu-update
takes into account.  Checked with the library's FP64 reduction (pf_stats) on every kernel path."""
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


def _drift(precision, variant, thermo, G, steps=300):
    f = W.symmetric_params if thermo == "symmetric" else W.general_params
    p = f(n_grains=8, G=G)  # no window trigger: the box stays closed
    sim = pf.Simulation(48, 40, 64, p, precision, variant=variant)
    sim.init(3)
    s0 = np.array(sim.stats()["solute"])
    sim.step(steps)
    s1 = np.array(sim.stats()["solute"])
    path = sorted(sim.step_bytes())
    sim.close()
    return np.abs(s1 - s0).max() / np.abs(s0).max(), path


@pytest.mark.parametrize("G", [0.0, 1e-3])
@pytest.mark.parametrize("thermo", ["symmetric", "general"])
@pytest.mark.parametrize("variant", ["auto", "unfused", "fused"])
def test_fp64_paths_conserve_solute_to_roundoff(variant, thermo, G):
    drift, path = _drift("fp64", variant, thermo, G)
    print(f"fp64 {variant} {thermo} G={G}: relative solute drift {drift:.2e} over 300 steps ({path})")
    assert drift <= 1e-12


@pytest.mark.parametrize("precision,bound", [("fp32c", 5e-10), ("fp32", 1e-8)])
def test_fp32_paths_conserve_solute_to_their_rounding(precision, bound):
    # compensated FP32 carries every increment; plain FP32 rounds each stored value
    for variant in ("auto", "unfused"):
        drift, path = _drift(precision, variant, "symmetric", 1e-3)
        print(f"{precision} {variant}: relative solute drift {drift:.2e} over 300 steps ({path})")
        assert drift <= bound
