"""The block decomposition on CPU ranks: two gloo processes each own a y-slab of the domain with
one ghost row on either side (Section 3.1), exchange the new phi rows after the phi-sweep and the
new mu rows after the mu-sweep (Algorithm 1), and agree on the moving window through one sum of
the interface height (Section 3.3).  Every cell update is the oracle's; the decomposition alone is
under test: the assembled slabs must equal the undivided oracle run exactly.

The same schedule runs on one GPU as pf_split (slabs on streams, ghost rows by device copies); this
file checks the exchange logic with real messages between processes."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

NX, NY, NZ, STEPS, SEED = 12, 10, 16, 12, 5


def _params():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_1506_01684_gb300 import workloads as W
    p = W.symmetric_params(n_grains=5, window_trigger_z=5.0)
    p["seed_layers"] = 8
    return oracle, oracle.resolve_params(p, NZ)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _exchange(f, nys, world):
    """Ghost rows of the extended slab f (..., nys + 2, nx) from the neighbours' boundary rows:
    row 0 takes the previous rank's last own row, row nys + 1 the next rank's first own row."""
    mine = torch.from_numpy(np.ascontiguousarray(np.stack([f[..., 1, :], f[..., nys, :]])))
    got = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(got, mine)
    r = dist.get_rank()
    f[..., 0, :] = got[(r - 1) % world][1].numpy()
    f[..., nys + 1, :] = got[(r + 1) % world][0].numpy()


def _rank(rank, world, port, out, skip_phi_exchange=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle, d = _params()
    whole = oracle.State(d, NX, NY, NZ).init(SEED)
    y0, y1 = rank * NY // world, (rank + 1) * NY // world
    nys = y1 - y0
    rows = [(y0 - 1 + j) % NY for j in range(nys + 2)]  # own rows and one ghost row on either side
    phi = np.ascontiguousarray(whole.phi[:, :, rows, :])
    mu = np.ascontiguousarray(whole.mu[:, :, rows, :])
    t = off = 0.0
    shifts = 0
    for _ in range(STEPS):
        pn = oracle.phi_sweep(d, phi, mu, t, off)
        if not skip_phi_exchange:
            _exchange(pn, nys, world)  # phi^{n+1} ghost rows before the mu-sweep reads them
        mn = oracle.mu_sweep(d, phi, pn, mu, t, off)
        _exchange(mn, nys, world)  # mu^{n+1} ghost rows for the next phi- and mu-sweeps
        phi, mu = pn, mn
        t += d["dt"]
        # one window decision for the whole domain: the interface height from every rank's own rows
        liq = torch.tensor([float(np.sum(1.0 - phi[3][:, 1:nys + 1, :]))], dtype=torch.float64)
        dist.all_reduce(liq)
        s, off = oracle.window_shift(d, phi, mu, float(liq[0]) / (NX * NY), off)
        shifts += s
    own = (slice(None), slice(None), slice(1, nys + 1), slice(None))
    out.put((rank, y0, phi[own].copy(), mu[own].copy(), t, off, shifts))
    dist.barrier()
    dist.destroy_process_group()


def _run(skip_phi_exchange=False):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, skip_phi_exchange)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_two_gloo_ranks_step_slabs_with_ghost_rows_like_the_whole_domain():
    res = _run()
    oracle, d = _params()
    ref = oracle.State(d, NX, NY, NZ).init(SEED)
    ref.step(STEPS)
    assert ref.shifts > 0  # the window moved during the run
    phi = np.empty_like(ref.phi)
    mu = np.empty_like(ref.mu)
    for rank, y0, ph, m, t, off, shifts in res:
        phi[:, :, y0:y0 + ph.shape[2], :] = ph
        mu[:, :, y0:y0 + m.shape[2], :] = m
        assert t == ref.t and off == ref.off and shifts == ref.shifts
    # each cell's update reads the same neighbours in the same order: the slabs reproduce the
    # undivided run exactly
    assert np.array_equal(phi, ref.phi)
    assert np.array_equal(mu, ref.mu)


def test_without_the_phi_exchange_the_slabs_drift_from_the_whole_domain():
    # the mu-sweep reads phi^{n+1} across the slab boundary (the anti-trapping current and the
    # phi rate): with stale ghost rows there the slabs no longer reproduce the whole domain
    res = _run(skip_phi_exchange=True)
    oracle, d = _params()
    ref = oracle.State(d, NX, NY, NZ).init(SEED)
    ref.step(STEPS)
    mu = np.empty_like(ref.mu)
    for rank, y0, ph, m, t, off, shifts in res:
        mu[:, :, y0:y0 + m.shape[2], :] = m
    assert np.abs(mu - ref.mu).max() > 1e-6
