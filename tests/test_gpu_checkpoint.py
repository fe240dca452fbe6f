"""Checkpoint and restart (the paper's field checkpoints, Section 3.2) through the C ABI.

A run resumed from a checkpoint of its own precision must continue bitwise as the uninterrupted
run: same fields, clock, window offset and shift count.  The configuration shifts the moving
window before the checkpoint, so that the restored window offset and clock decide the plane
constants of the resumed steps.
"""
import os

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


def _params():
    p = W.symmetric_params(window_trigger_z=7.0)
    p["seed_layers"] = 10
    return p


# bytes per value slot: the compensated state stores its two FP32 words
@pytest.mark.parametrize("precision,elem", [("fp32", 4), ("fp64", 8), ("fp32c", 8)])
@pytest.mark.parametrize("variant", ["auto", "unfused"])
def test_resumed_run_equals_the_uninterrupted_run_bitwise(tmp_path, precision, elem, variant):
    nx, ny, nz = 32, 32, 64
    p = _params()
    path = str(tmp_path / f"ck_{precision}_{variant}.pfc")
    a = pf.Simulation(nx, ny, nz, p, precision, variant=variant)
    a.init(3)
    a.step(25)
    a.checkpoint(path)
    st_ck = a.stats()
    assert os.path.getsize(path) == 64 + nz * 6 * nx * ny * elem
    a.step(30)
    pa, ma = a.fields()
    sa = a.stats()
    b = pf.Simulation(nx, ny, nz, p, precision, variant=variant)
    b.init(99)  # a different state, overwritten by the checkpoint
    b.step(3)
    b.restore(path)
    sb0 = b.stats()
    assert sb0["t"] == st_ck["t"] and sb0["window_offset"] == st_ck["window_offset"]
    b.step(30)
    pb, mb = b.fields()
    sbb = b.stats()
    assert st_ck["window_offset"] > 0  # the window had moved: the restored offset sets the plane constants
    assert (pa == pb).all() and (ma == mb).all()
    assert sa["t"] == sbb["t"] and sa["window_offset"] == sbb["window_offset"]
    assert a.shifts() == b.shifts()
    a.close()
    b.close()


def test_fp32_checkpoint_restores_into_fp64(tmp_path):
    nx, ny, nz = 24, 16, 20
    p = W.symmetric_params(n_grains=5)
    path = str(tmp_path / "ck32.pfc")
    a = pf.Simulation(nx, ny, nz, p, "fp32")
    a.init(1)
    a.step(5)
    a.checkpoint(path)
    pa, ma = a.fields()
    b = pf.Simulation(nx, ny, nz, p, "fp64")
    b.restore(path)
    pb, mb = b.fields()
    assert (pa == pb).all() and (ma == mb).all()  # FP32 values are exact in FP64
    assert b.stats()["t"] == a.stats()["t"]
    a.close()
    b.close()


def test_compensated_checkpoint_holds_both_words(tmp_path):
    # the pairs' words go to the file as they are: a compensated reader gets the same pairs (the
    # next steps agree bitwise), an FP64 reader the value of each pair
    nx, ny, nz = 24, 16, 20
    p = W.symmetric_params(n_grains=5)
    path = str(tmp_path / "ckc.pfc")
    a = pf.Simulation(nx, ny, nz, p, "fp32c")
    a.init(1)
    a.step(40)
    a.checkpoint(path)
    pa, ma = a.fields()
    b = pf.Simulation(nx, ny, nz, p, "fp64")
    b.restore(path)
    pb, mb = b.fields()
    assert (pa == pb).all() and (ma == mb).all()
    c = pf.Simulation(nx, ny, nz, p, "fp32c")
    c.restore(path)
    a.step(20)
    c.step(20)
    (pa2, ma2), (pc2, mc2) = a.fields(), c.fields()
    assert (pa2 == pc2).all() and (ma2 == mc2).all()
    for s in (a, b, c):
        s.close()


def test_checkpoint_errors(tmp_path):
    p = W.symmetric_params(n_grains=3)
    a = pf.Simulation(16, 8, 12, p, "fp32")
    a.init(0)
    path = str(tmp_path / "ck.pfc")
    a.checkpoint(path)
    # another grid
    b = pf.Simulation(16, 8, 13, p, "fp32")
    with pytest.raises(pf.PfError) as e:
        b.restore(path)
    assert e.value.status == pf.PF_E_INVAL
    # missing and truncated files
    with pytest.raises(pf.PfError):
        a.restore(str(tmp_path / "missing.pfc"))
    data = open(path, "rb").read()
    short = str(tmp_path / "short.pfc")
    open(short, "wb").write(data[: len(data) // 2])
    with pytest.raises(pf.PfError):
        a.restore(short)
    bad = str(tmp_path / "bad.pfc")
    open(bad, "wb").write(b"NOTACKPT" + data[8:])
    with pytest.raises(pf.PfError):
        a.restore(bad)
    # an unwritable path
    with pytest.raises(pf.PfError):
        a.checkpoint(str(tmp_path / "no_such_dir" / "ck.pfc"))
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_single_precision_checkpoint_of_a_high_precision_run(tmp_path, precision):
    # Section 3.2: the run in double precision, the checkpoint in single.  The resumed run starts
    # from the state rounded once to FP32 and stays within the FP32 tolerance of the uninterrupted
    # run; the file is half an FP64 checkpoint
    nx, ny, nz = 32, 32, 64
    p = _params()
    path = str(tmp_path / f"ck32_{precision}.pfc")
    a = pf.Simulation(nx, ny, nz, p, precision)
    a.init(3)
    a.step(25)
    p0, m0 = a.fields()
    a.checkpoint(path, single=True)
    st_ck = a.stats()
    assert os.path.getsize(path) == 64 + nz * 6 * nx * ny * 4
    b = pf.Simulation(nx, ny, nz, p, precision)
    b.restore(path)
    pb0, mb0 = b.fields()
    # the restored state is the FP32 rounding of the checkpointed one
    assert np.array_equal(pb0, p0.astype(np.float32).astype(np.float64))
    assert np.array_equal(mb0, m0.astype(np.float32).astype(np.float64))
    assert b.stats()["t"] == st_ck["t"] and b.stats()["window_offset"] == st_ck["window_offset"]
    n = 200
    a.step(n)
    b.step(n)
    pa, ma = a.fields()
    pb, mb = b.fields()
    e_phi = np.abs(pa - pb).max()
    e_mu = np.abs(ma - mb).max() / max(np.abs(ma).max(), 1e-8)
    print(f"{precision}: resume error after {n} steps from the single-precision checkpoint: "
          f"max|dphi| {e_phi:.3e}, |dmu|/scale {e_mu:.3e}")
    assert 0 < max(e_phi, e_mu)
    assert e_phi <= 2e-5 and e_mu <= 2e-5
    assert a.shifts() == b.shifts() and a.stats()["window_offset"] == b.stats()["window_offset"]
