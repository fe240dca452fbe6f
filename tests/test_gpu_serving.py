"""Serving loop: continuous batching, admission by device-memory footprint, results independent
of the mix a request ran in."""
import time

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


def _requests(n=8):
    rng = np.random.default_rng(9)
    out = []
    for q in range(n):
        nx, ny = int(rng.choice([16, 32, 48])), int(rng.choice([16, 24, 32]))
        nz = int(rng.choice([40, 64, 96]))
        p = W.symmetric_params(G=float(rng.uniform(5e-4, 2e-3)), v=float(rng.uniform(5e-3, 2e-2)),
                               n_grains=int(rng.integers(2, 8)))
        out.append(dict(nx=nx, ny=ny, nz=nz, p=p, seed=int(rng.integers(1, 1000)), steps=int(rng.integers(20, 150))))
    return out


def _wait(srv, ticket, nx, ny, timeout=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = pf.pf_poll(srv, ticket, nx, ny)
        if r is not None:
            return r
        time.sleep(0.002)
    raise TimeoutError(ticket)


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = _requests()
    # in the mix: staggered arrivals, so later requests join while earlier ones run
    srv = pf.pf_server_create(0, 0, 16)
    tickets = []
    for r in reqs:
        tickets.append(pf.pf_submit(srv, r["nx"], r["ny"], r["nz"], pf.params_from_dict(r["p"], pf.PF_FP32),
                                    r["seed"], r["steps"]))
        time.sleep(0.003)
    mixed = [_wait(srv, t, r["nx"], r["ny"]) for t, r in zip(tickets, reqs)]
    stats = pf.pf_server_stats(srv)
    assert stats["running"] == 0 and stats["queued"] == 0 and stats["used_bytes"] == 0 and stats["mlups"] > 0
    pf.pf_server_destroy(srv)
    # alone: each request on its own server, nothing else running
    for r, (fr, slab, lat) in zip(reqs, mixed):
        s1 = pf.pf_server_create(0, 0, 16)
        t = pf.pf_submit(s1, r["nx"], r["ny"], r["nz"], pf.params_from_dict(r["p"], pf.PF_FP32), r["seed"],
                         r["steps"])
        fr1, slab1, _ = _wait(s1, t, r["nx"], r["ny"])
        pf.pf_server_destroy(s1)
        assert (fr1 == fr).all() and (slab1 == slab).all()
        assert lat > 0
        # and the same as the plain simulation API, up to rounding order: served runs take the
        # batched fused tile, a simulation of even nx the lean kernel and the two sweeps (same
        # expressions, another order; phi agrees to ~1e-7, so a mean of phi to well below 1e-6)
        sim = pf.Simulation(r["nx"], r["ny"], r["nz"], r["p"], "fp32", variant="fused")
        sim.init(r["seed"])
        sim.step(r["steps"])
        np.testing.assert_allclose(sim.fractions(), fr, rtol=0, atol=1e-6)
        sim.close()


def test_admission_respects_the_device_memory_budget():
    reqs = _requests(6)
    # a budget that holds only about two of these requests at a time
    one = 2 * max(r["nx"] * r["ny"] * r["nz"] for r in reqs) * 24 + 64 * 1024
    srv = pf.pf_server_create(int(2.2 * one), 0, 8)
    ts = [pf.pf_submit(srv, r["nx"], r["ny"], r["nz"], pf.params_from_dict(r["p"], pf.PF_FP32), r["seed"], r["steps"])
          for r in reqs]
    peak = 0
    pending = set(range(len(ts)))
    t0 = time.time()
    while pending and time.time() - t0 < 120:
        st = pf.pf_server_stats(srv)
        peak = max(peak, st["used_bytes"])
        for i in list(pending):
            if pf.pf_poll(srv, ts[i], reqs[i]["nx"], reqs[i]["ny"]) is not None:
                pending.discard(i)
        time.sleep(0.001)
    assert not pending
    assert 0 < peak <= int(2.2 * one)
    # a request larger than the whole budget is refused at submission
    with pytest.raises(pf.PfError) as e:
        pf.pf_submit(srv, 512, 512, 512, pf.params_from_dict(reqs[0]["p"], pf.PF_FP32), 1, 10)
    assert e.value.status == pf.PF_E_NOMEM
    pf.pf_server_destroy(srv)


def test_cancel_and_unknown_ticket():
    r = _requests(1)[0]
    srv = pf.pf_server_create(0, 0, 4)
    t = pf.pf_submit(srv, r["nx"], r["ny"], r["nz"], pf.params_from_dict(r["p"], pf.PF_FP32), r["seed"], 100000)
    time.sleep(0.05)
    pf.pf_cancel(srv, t)
    t0 = time.time()
    while True:
        st = pf.lib().pf_poll(srv, t, None, None, None)
        if st != pf.PF_E_PENDING or time.time() - t0 > 60:
            break
        time.sleep(0.002)
    assert st == pf.PF_E_CANCELLED
    assert pf.lib().pf_poll(srv, 987654321, None, None, None) == pf.PF_E_INVAL
    assert pf.pf_server_stats(srv)["used_bytes"] == 0
    pf.pf_server_destroy(srv)
