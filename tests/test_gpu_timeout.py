"""Failure path of the bounded device waits, tested without a GPU fault.

Every wait of the lean kernel (the fused step's pure-liquid planes) on an mbarrier gives up after
about 2^31 clock cycles, raises the CTA's abort flag and returns; the step then reports
PF_E_TIMEOUT through pf_sync instead of hanging.  A test hook makes the kernel's producer issue
none of its copies, so the consumers' waits run out; afterwards the context must still be usable.
"""
import time

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


def test_a_wait_that_runs_out_reports_a_timeout_and_the_context_recovers():
    nx, ny, nz = 32, 8, 24  # one tile, pure liquid: every plane is the lean kernel's
    p = W.symmetric_params()
    rng = np.random.default_rng(5)
    phi = np.zeros((4, nz, ny, nx))
    phi[3] = 1.0
    mu = rng.uniform(-1e-3, 1e-3, size=(2, nz, ny, nx)).astype(np.float32).astype(np.float64)
    sim = pf.Simulation(nx, ny, nz, p, "fp32", variant="fused")
    sim.set_fields(phi, mu)
    pf.pf_test_withhold_copies(sim.h, True)
    t0 = time.perf_counter()
    sim.step(1)
    with pytest.raises(pf.PfError) as e:
        sim.sync()
    assert e.value.status == pf.PF_E_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    # normal steps again, from a state written anew (a timed-out step leaves its planes undefined)
    pf.pf_test_withhold_copies(sim.h, False)
    sim.set_fields(phi, mu)
    t = sim.stats()["t"]
    sim.step(3)
    sim.sync()
    ref = oracle.State(p, nx, ny, nz)
    ref.phi, ref.mu, ref.t = phi.copy(), mu.copy(), t
    ref.step(3)
    phi1, mu1 = sim.fields()
    assert np.abs(phi1 - ref.phi).max() <= 2e-5
    assert np.abs(mu1 - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8) <= 2e-5
    sim.close()
