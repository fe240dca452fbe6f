"""pf_split: one domain cut into y-slabs with ghost rows (Section 3.1), stepped with Algorithm 1's
exchanges after each sweep and Algorithm 2's overlap of the mu exchange with the phi-sweep, on
one GPU.  Each slab runs the same sweep kernels as an undivided domain with PF_VARIANT_UNFUSED, so
the assembled fields must equal that run bit for bit, through window shifts; in FP64 both are also
checked against the oracle."""
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


def _params(thermo="symmetric"):
    f = W.symmetric_params if thermo == "symmetric" else W.general_params
    p = f(n_grains=8, window_trigger_z=7.0)
    p["seed_layers"] = 10  # the window starts moving in the first step
    return p


# one slab (its own neighbour), even and ragged cuts, an odd nx, one row per slab
CASES = [((32, 30, 64), 1), ((32, 30, 64), 3), ((32, 30, 64), 4), ((37, 21, 19), 2), ((16, 6, 24), 6)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,nslabs", CASES)
def test_split_equals_the_undivided_domain_bit_for_bit(precision, shape, nslabs):
    nx, ny, nz = shape
    p = _params()
    whole = pf.Simulation(nx, ny, nz, p, precision, variant="unfused").init(3)
    sp = pf.Split(nx, ny, nz, p, nslabs, precision).init(3)
    pw, mw = whole.fields()
    ps, ms = sp.fields()
    assert np.array_equal(ps, pw) and np.array_equal(ms, mw)  # the same initial state
    for n in (1, 5, 24):
        whole.step(n)
        sp.step(n)
        pw, mw = whole.fields()
        ps, ms = sp.fields()
        assert np.array_equal(ps, pw), (n, np.abs(ps - pw).max())
        assert np.array_equal(ms, mw), (n, np.abs(ms - mw).max())
        a, b = whole.stats(), sp.stats()
        assert b["t"] == a["t"] and b["window_offset"] == a["window_offset"]
        assert b["shifts"] == whole.shifts()
        # the interface height: the same cells summed in another order
        assert b["h_int"] == pytest.approx(a["h_int"], rel=1e-12, abs=1e-12)
    assert sp.stats()["shifts"] > 0
    whole.close()
    sp.close()


@pytest.mark.parametrize("thermo", ["symmetric", "general"])
def test_split_matches_the_oracle_in_fp64(thermo):
    nx, ny, nz = 24, 20, 32
    p = _params(thermo)
    sp = pf.Split(nx, ny, nz, p, 3, "fp64").init(9)
    ref = oracle.State(p, nx, ny, nz).init(9)
    sp.step(40)
    ref.step(40)
    phi, mu = sp.fields()
    assert ref.shifts > 0 and sp.stats()["shifts"] == ref.shifts
    assert np.abs(phi - ref.phi).max() <= 1e-12
    assert np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8) <= 1e-12
    sp.close()


def test_split_rejects_what_it_cannot_do():
    p = _params()
    for nslabs in (0, 31):
        with pytest.raises(pf.PfError) as e:
            pf.Split(32, 30, 64, p, nslabs, "fp64")
        assert e.value.status == pf.PF_E_INVAL
    with pytest.raises(pf.PfError) as e:
        pf.Split(32, 30, 64, p, 2, "fp32c")
    assert e.value.status == pf.PF_E_INVAL
