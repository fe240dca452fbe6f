"""Host I/O of the fields with FP32 host buffers (pf_read_fields_f32 / pf_write_fields_f32) against the
FP64 forms: exact where FP32 holds the values, one rounding otherwise."""
import ctypes

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


def _state(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    return W.random_simplex_field(rng, nx, ny, nz, sharp=0.4), W.random_mu(rng, nx, ny, nz, scale=0.05)


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32c"])
def test_fp32_host_buffers_round_trip(precision):
    # 37 x 21 x 150: several staging chunks are not needed, but ragged tiles and an odd width are
    nx, ny, nz = 37, 21, 150
    p = W.symmetric_params(G=2e-3)
    phi, mu = _state(nx, ny, nz, 3)
    sim = pf.Simulation(nx, ny, nz, p, precision)
    sim.set_fields(phi, mu)
    sim.step(4)
    phi64, mu64 = sim.fields()
    phi32, mu32 = sim.fields_f32()
    # read: the state's value rounded once to FP32 (exact for an FP32 state)
    assert (phi32 == phi64.astype(np.float32)).all() and (mu32 == mu64.astype(np.float32)).all()
    if precision == "fp32":
        assert (phi32.astype(np.float64) == phi64).all() and (mu32.astype(np.float64) == mu64).all()
    # write: FP32 values are exact in every precision
    sim.set_fields_f32(phi32, mu32)
    back_phi, back_mu = sim.fields()
    assert (back_phi == phi32.astype(np.float64)).all() and (back_mu == mu32.astype(np.float64)).all()
    sim.close()


def test_a_state_written_in_fp32_steps_as_the_same_state_written_in_fp64():
    nx, ny, nz = 40, 24, 48
    p = W.symmetric_params(G=2e-3, n_grains=6)
    phi, mu = _state(nx, ny, nz, 5)
    phi = phi.astype(np.float32)
    mu = mu.astype(np.float32)
    a = pf.Simulation(nx, ny, nz, p, "fp32").set_fields(phi.astype(np.float64), mu.astype(np.float64))
    b = pf.Simulation(nx, ny, nz, p, "fp32").set_fields_f32(phi, mu)
    a.step(10)
    b.step(10)
    (pa, ma), (pb, mb) = a.fields(), b.fields()
    assert (pa == pb).all() and (ma == mb).all()
    a.close()
    b.close()


def test_fp32_host_io_errors():
    sim = pf.Simulation(8, 8, 8, W.symmetric_params(), "fp32")
    L = pf.lib()
    fp = ctypes.POINTER(ctypes.c_float)
    buf = np.zeros(4 * 8 * 8 * 8, dtype=np.float32)
    assert L.pf_read_fields_f32(sim.h, buf.ctypes.data_as(fp), None, 8 * 8 * 8 - 1) == pf.PF_E_INVAL
    assert L.pf_read_fields_f32(sim.h, None, None, 8 * 8 * 8) == pf.PF_OK
    assert L.pf_write_fields_f32(sim.h, buf.ctypes.data_as(fp), None) == pf.PF_E_INVAL
    assert L.pf_write_fields_f32(None, buf.ctypes.data_as(fp), buf.ctypes.data_as(fp)) == pf.PF_E_INVAL
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32c"])
@pytest.mark.parametrize("host", ["f32", "f64"])
def test_pinned_host_buffers_take_the_direct_path_with_the_same_result(precision, host):
    # pinned (device-addressable) host buffers are read and written by the pack / unpack kernels
    # directly; pageable ones go through the staging chunks: the values are the same
    import torch
    nx, ny, nz = 64, 40, 300  # more than one staging chunk (2^22 cells) would need nz > 1638
    phi, mu = _state(nx, ny, nz, 11)
    dt = np.float32 if host == "f32" else np.float64
    write = pf.pf_write_fields_f32 if host == "f32" else pf.pf_write_fields
    read = pf.pf_read_fields_f32 if host == "f32" else pf.pf_read_fields
    out = {}
    for kind in ("pageable", "pinned"):
        sim = pf.Simulation(nx, ny, nz, W.symmetric_params(), precision)
        if kind == "pinned":
            hp = torch.from_numpy(phi.astype(dt)).pin_memory()
            hm = torch.from_numpy(mu.astype(dt)).pin_memory()
            sp, sm = hp.numpy(), hm.numpy()
            op = torch.empty(phi.shape, dtype=hp.dtype).pin_memory().numpy()
            om = torch.empty(mu.shape, dtype=hm.dtype).pin_memory().numpy()
        else:
            sp, sm = phi.astype(dt), mu.astype(dt)
            op, om = np.empty(phi.shape, dtype=dt), np.empty(mu.shape, dtype=dt)
        write(sim.h, np.ascontiguousarray(sp), np.ascontiguousarray(sm))
        sim.step(5)
        read(sim.h, op, om)
        out[kind] = (op.copy(), om.copy())
        sim.close()
    assert np.array_equal(out["pinned"][0], out["pageable"][0])
    assert np.array_equal(out["pinned"][1], out["pageable"][1])
