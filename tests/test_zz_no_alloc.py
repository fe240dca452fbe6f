"""The allocation-free step (pf_step_noalloc) against the regular entry points.

pf_step_noalloc exists for callers that cannot allocate device memory (their device memory
belongs to another allocator's budget, or they must not pay cudaMalloc's implicit device
synchronisation).  Here the caller's fields are torch tensors; the library allocates nothing
for the call and keeps its scratch in a fixed device array.  Two calls in a row are compared
with pf_step through a pf_sim on the same state; both run the same kernels, so the results
agree within the tests' tolerances (in practice bit for bit).

This file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_1506_01684_gb300 import pf
from paper_1506_01684_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.lib()
    return t


def _aos(torch, soa, dtype):
    # host SoA (c, z, y, x) -> device array of cells (z, y, x, c)
    return torch.from_numpy(np.ascontiguousarray(np.moveaxis(soa, 0, -1))).to("cuda", dtype).contiguous()


def _soa(t):
    return np.moveaxis(t.double().cpu().numpy(), -1, 0)


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-12)])
@pytest.mark.parametrize("thermo", ["symmetric", "general"])
def test_noalloc_step_matches_pf_step_on_two_calls_in_a_row(torch, precision, tol, thermo):
    nx, ny, nz = 48, 40, 36
    # the general set (matrix curvatures, pair relaxation times) runs the kernels' general branches
    p = W.symmetric_params(n_grains=7) if thermo == "symmetric" else W.general_params(n_grains=7)
    # a state with diffuse interfaces: 10 steps from the Voronoi start through the regular path
    ref = pf.Simulation(nx, ny, nz, p, precision)
    ref.init(5)
    ref.step(10)
    phi0, mu0 = ref.fields()
    st0 = ref.stats()
    # restart the reference from exactly this state at t, offset of the state
    ref.set_fields(phi0, mu0)
    params = ref.params  # effective parameters (dt resolved)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    stream = torch.cuda.current_stream()
    src_phi, src_mu = _aos(torch, phi0, dtype), _aos(torch, mu0, dtype)
    dst_phi, dst_mu = torch.empty_like(src_phi), torch.empty_like(src_mu)
    t = st0["t"]
    off = st0["window_offset"]
    for call in range(2):
        free_before = torch.cuda.mem_get_info()[0]
        h = pf.pf_step_noalloc(nx, ny, nz, params, t, off, src_phi.data_ptr(), src_mu.data_ptr(),
                               dst_phi.data_ptr(), dst_mu.data_ptr(), True, stream)
        if call == 1:
            # after the first call's one-time set-up the call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        ref.step(1)
        phi_r, mu_r = ref.fields()
        phi_n, mu_n = _soa(dst_phi), _soa(dst_mu)
        assert np.abs(phi_n - phi_r).max() <= tol
        assert np.abs(mu_n - mu_r).max() / max(np.abs(mu_r).max(), 1e-8) <= tol
        # h = sum (1 - phi_l) / (nx ny) from each path's own fields: the two differ by at most nz
        # times the largest phi_l difference (FP32: the two kernel paths may round differently)
        h_ref = ref.stats()["h_int"]
        assert abs(h - h_ref) <= nz * np.abs(phi_n[3] - phi_r[3]).max() + 1e-12 * abs(h_ref)
        # next call: the new state is the input
        src_phi, dst_phi = dst_phi, src_phi
        src_mu, dst_mu = dst_mu, src_mu
        t = t + params.dt
    ref.close()


def test_noalloc_step_rejects_what_it_cannot_do(torch):
    p = pf.params_from_dict(W.symmetric_params(), pf.PF_FP32)
    a = torch.zeros(64, dtype=torch.float32, device="cuda")
    L = pf.lib()
    ptr = a.data_ptr()
    # a grid whose scratch exceeds the fixed array: 2 * nz plane-table entries alone are too many
    assert L.pf_step_noalloc(1, 1, 1 << 17, p, 0.0, 0.0, ptr, ptr, ptr, ptr, None, None) == pf.PF_E_INVAL
    # compensated FP32 is not offered here; null and misaligned fields are rejected before any launch
    q = pf.params_from_dict(W.symmetric_params(), pf.PF_FP32_COMP)
    assert L.pf_step_noalloc(4, 4, 4, q, 0.0, 0.0, ptr, ptr, ptr, ptr, None, None) == pf.PF_E_INVAL
    assert L.pf_step_noalloc(4, 4, 4, p, 0.0, 0.0, None, ptr, ptr, ptr, None, None) == pf.PF_E_INVAL
    assert L.pf_step_noalloc(4, 4, 4, p, 0.0, 0.0, ptr + 4, ptr, ptr, ptr, None, None) == pf.PF_E_INVAL


def noalloc_scratch_bytes(nx, ny, nz, word):
    """The scratch a grid needs, by the formula the header states for pf_step_noalloc."""
    gx, gy = -(-nx // 32), -(-ny // 8)
    zc = min(nz, max(8, min(64, -(-nz // -(-2432 // (gx * gy))))))
    gz = -(-nz // zc)
    table = -(-(2 * nz * 16 * word) // 256) * 256
    return 256 + table + 32 * gx * gy * gz


def test_noalloc_scratch_limit_is_exact(torch):
    limit = 8 * 1024 * 1024
    # the header's example
    assert noalloc_scratch_bytes(256, 256, 1024, 4) == 262400
    # a 1 x 1 column whose scratch is just under the limit runs; one plane more is rejected
    nz = 64000
    while noalloc_scratch_bytes(1, 1, nz + 1, 4) <= limit:
        nz += 1
    assert noalloc_scratch_bytes(1, 1, nz, 4) <= limit < noalloc_scratch_bytes(1, 1, nz + 1, 4)
    p = pf.params_from_dict(W.symmetric_params(G=0.0), pf.PF_FP32)
    phi = torch.zeros((nz + 1, 4), dtype=torch.float32, device="cuda")
    phi[:, 3] = 1.0  # pure liquid: a fixed point apart from the temperature drift (none at G = 0)
    mu = torch.zeros((nz + 1, 2), dtype=torch.float32, device="cuda")
    phi_o, mu_o = torch.empty_like(phi), torch.empty_like(mu)
    L = pf.lib()
    stream = torch.cuda.current_stream()
    h = pf.pf_step_noalloc(1, 1, nz, p, 0.0, 0.0, phi.data_ptr(), mu.data_ptr(), phi_o.data_ptr(),
                           mu_o.data_ptr(), True, stream)
    assert h == 0.0
    assert torch.equal(phi_o[:nz], phi[:nz]) and torch.equal(mu_o[:nz], mu[:nz])
    assert L.pf_step_noalloc(1, 1, nz + 1, p, 0.0, 0.0, phi.data_ptr(), mu.data_ptr(), phi_o.data_ptr(),
                             mu_o.data_ptr(), None, None) == pf.PF_E_INVAL
