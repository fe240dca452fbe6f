"""Batched launch of uneven domains (one persistent fused kernel per step)."""
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


SHAPES = [(32, 32, 64), (37, 21, 40), (64, 16, 96), (8, 40, 33), (1, 3, 20)]


def _params(i, window=0.0):
    rng = np.random.default_rng(100 + i)
    p = W.symmetric_params(G=float(rng.uniform(5e-4, 2e-3)), v=float(rng.uniform(5e-3, 2e-2)),
                           n_grains=int(rng.integers(2, 9)), window_trigger_z=window)
    return p


@pytest.mark.parametrize("nsteps", [7, 30])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_domains_equal_their_own_fused_runs(nsteps, precision):
    # a batched domain runs the kernels its own fused run takes (even nx: the plan, the general
    # planes' two sweeps and the lean kernel; odd nx: the fused tile), over the same chunks.  FP64
    # is compiled without multiply-add contraction: bitwise.  In FP32 the batched and the single
    # kernels are separate instantiations whose multiply-adds the compiler may contract
    # differently: equal to FP32 rounding.
    params = [_params(i) for i in range(len(SHAPES))]
    seeds = [11 * i + 1 for i in range(len(SHAPES))]
    b = pf.Batch(SHAPES, params, precision)
    b.init(seeds)
    b.step(nsteps)
    b.sync()
    for d, (shape, p) in enumerate(zip(SHAPES, params)):
        sim = pf.Simulation(*shape, p, precision, variant="fused")
        sim.init(seeds[d])
        sim.step(nsteps)
        a_phi, a_mu = b.fields(d)
        s_phi, s_mu = sim.fields()
        if precision == "fp64":
            assert (a_phi == s_phi).all() and (a_mu == s_mu).all(), d
        else:
            assert np.abs(a_phi - s_phi).max() <= 1e-6, d
            assert np.abs(a_mu - s_mu).max() <= 1e-6 * max(np.abs(s_mu).max(), 1e-8), d
        assert b.stats(d)["t"] == sim.stats()["t"]
        sim.close()
    b.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-12)])
def test_batched_domains_match_the_oracle(precision, tol):
    params = [_params(i, window=9.0 if i == 0 else 0.0) for i in range(len(SHAPES))]
    params[0]["seed_layers"] = 12
    seeds = [3 * i + 5 for i in range(len(SHAPES))]
    b = pf.Batch(SHAPES, params, precision)
    b.init(seeds)
    b.step(25)
    b.sync()
    for d, (shape, p) in enumerate(zip(SHAPES, params)):
        ref = oracle.State(p, *shape).init(seeds[d])
        ref.step(25)
        phi, mu = b.fields(d)
        assert np.abs(phi - ref.phi).max() <= tol, d
        assert np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8) <= tol, d
        assert b.shifts(d) == ref.shifts, d
    assert b.shifts(0) > 0  # the window of domain 0 moved inside the batch
    b.close()


def test_autotune_restores_the_state_and_keeps_results():
    params = [_params(i) for i in range(len(SHAPES))]
    seeds = list(range(1, len(SHAPES) + 1))
    b = pf.Batch(SHAPES, params, "fp32")
    b.init(seeds)
    b.step(3)
    before = [b.fields(d) for d in range(len(SHAPES))]
    t_before = [b.stats(d)["t"] for d in range(len(SHAPES))]
    zc, ms = pf.pf_batch_autotune(b.h, 4)
    assert zc in (16, 32, 64, 128, 256, 512) and ms > 0
    for d in range(len(SHAPES)):
        phi, mu = b.fields(d)
        assert (phi == before[d][0]).all() and (mu == before[d][1]).all()
        assert b.stats(d)["t"] == t_before[d]
    # results after tuning agree with the oracle (the z chunk only changes the schedule)
    b.step(10)
    for d, (shape, p) in enumerate(zip(SHAPES, params)):
        ref = oracle.State(p, *shape).init(seeds[d])
        ref.step(13)
        phi, mu = b.fields(d)
        assert np.abs(phi - ref.phi).max() <= 2e-5
    b.close()


def test_a_domain_stepped_on_its_own_is_refused():
    # the batch adopts each domain's buffers when it builds its work table (first step); a domain
    # stepped on its own after that would desynchronise the table and is refused
    b = pf.Batch(SHAPES[:2], [_params(0), _params(1)], "fp32")
    b.init([1, 2])
    b.step(1)
    pf.pf_step(b.domain(1), 1)
    with pytest.raises(pf.PfError) as e:
        b.step(2)
    assert e.value.status == pf.PF_E_INVAL
    b.close()


@pytest.mark.parametrize("general", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_odd_width_domain_with_a_moving_window_in_a_batch(general, precision, tol):
    # an odd-nx domain (the fused tile, no tensor copies) whose window shifts, beside an even one
    shapes = [(33, 8, 30), (32, 16, 24)]
    base = W.general_params if general else W.symmetric_params
    params = [base(n_grains=3, window_trigger_z=9.0), base(n_grains=4)]
    for q in params:
        q["seed_layers"] = 10
    b = pf.Batch(shapes, params, precision)
    b.init([1, 2])
    b.step(40)
    for d, (shape, q) in enumerate(zip(shapes, params)):
        ref = oracle.State(q, *shape).init(d + 1)
        ref.step(40)
        phi, mu = b.fields(d)
        assert b.shifts(d) == ref.shifts, d
        assert np.abs(phi - ref.phi).max() <= tol, d
        assert np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8) <= tol, d
        sim = pf.Simulation(*shape, q, precision, variant="fused")
        sim.init(d + 1)
        sim.step(40)
        s_phi, s_mu = sim.fields()
        print(d, precision, general, "batch vs single:", np.abs(phi - s_phi).max(), np.abs(mu - s_mu).max(),
              "single vs oracle:", np.abs(s_phi - ref.phi).max())
        assert np.abs(s_phi - ref.phi).max() <= tol, d
        sim.close()
    assert b.shifts(0) > 0
    b.close()


def test_batch_step_bytes_tally_each_domains_cells():
    # two pure-liquid domains on the lean path: the lean kernel moves mu^n in and mu^{n+1} out, 16
    # bytes a cell, once phi^{n+1} = e_l is known to be stored; the same domains with a front add
    # the general planes' 88 bytes a general cell
    shapes = [(64, 32, 48), (32, 32, 64)]
    p = W.symmetric_params()
    b = pf.Batch(shapes, [p, p], "fp32")
    rng = np.random.default_rng(3)
    for d, (nx, ny, nz) in enumerate(shapes):
        phi = np.zeros((4, nz, ny, nx))
        phi[3] = 1.0
        pf.pf_write_fields(b.domain(d), phi, rng.uniform(-1e-3, 1e-3, (2, nz, ny, nx)))
    b.step(4)
    b.sync()
    cells = sum(x * y * z for x, y, z in shapes)
    got = pf.pf_batch_step_bytes(b.h)
    assert got == {"general_and_fused": 0.0, "lean_step": 16.0 * cells}
    b.init([1, 2])
    b.step(4)
    got = pf.pf_batch_step_bytes(b.h)
    assert got["general_and_fused"] > 0 and got["general_and_fused"] % 88.0 == 0
    assert 0 < got["lean_step"] < 16.0 * cells
    b.close()


def test_autotune_restores_the_plane_tables_too():
    # FP64: a batch that tuned its launch shape (its state put back afterwards, plane tables
    # included) steps on as one that never tuned: a stale plane table (the temperature of the last
    # trial's clock) would show as a ~1e-7 relative error in mu after the first step; the schedule
    # itself leaves the FP64 results equal up to rounding order
    params = [_params(i, window=7.0) for i in range(len(SHAPES))]
    seeds = list(range(1, len(SHAPES) + 1))
    a = pf.Batch(SHAPES, params, "fp64")
    b = pf.Batch(SHAPES, params, "fp64")
    for x in (a, b):
        x.init(seeds)
        x.step(3)
    zc, ms = pf.pf_batch_autotune(b.h, 4)
    cfg = pf.pf_batch_config(b.h)
    assert cfg["zchunk"] == zc and cfg["general_ctas_per_sm"] in (1, 2) and cfg["lean_split"] in (1, 2, 4) \
        and cfg["lean_tile_rows"] in (8, 4)
    a.step(10)
    b.step(10)
    for d in range(len(SHAPES)):
        pa, ma = a.fields(d)
        pb, mb = b.fields(d)
        assert np.abs(pa - pb).max() <= 1e-13
        assert np.abs(ma - mb).max() <= 1e-13 * max(np.abs(ma).max(), 1e-8)
        assert a.stats(d)["t"] == b.stats(d)["t"]
    a.close()
    b.close()


# launch shapes: (z chunk, general CTAs an SM, lean split, lean tile rows)
LAUNCH_SHAPES = [(0, 2, 1, 8), (0, 2, 1, 4), (16, 1, 2, 4), (32, 2, 4, 8), (64, 1, 4, 4)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_launch_shape_gives_the_same_fields(precision):
    # a cell's update is the same arithmetic under any tile, z-chunk or z-block shape: FP64 (no
    # multiply-add contraction) is bitwise; FP32 kernels of other tile shapes are other instantiations
    # whose multiply-adds the compiler may contract differently: equal to FP32 rounding.  Domain 0's
    # window moves; ny = 21 and 3 leave ragged 32x4 and 32x8 row blocks.
    params = [_params(i, window=9.0 if i == 0 else 0.0) for i in range(len(SHAPES))]
    params[0]["seed_layers"] = 12
    seeds = [5 * i + 2 for i in range(len(SHAPES))]
    runs = []
    for shape in LAUNCH_SHAPES:
        b = pf.Batch(SHAPES, params, precision)
        pf.pf_batch_set_config(b.h, *shape)
        assert tuple(pf.pf_batch_config(b.h).values()) == shape
        b.init(seeds)
        b.step(3)
        b.step(24)  # graph-replayed
        b.sync()
        runs.append([b.fields(d) for d in range(len(SHAPES))] + [b.shifts(0)])
        b.close()
    assert runs[0][-1] > 0
    for shape, run in zip(LAUNCH_SHAPES[1:], runs[1:]):
        assert run[-1] == runs[0][-1], shape
        for d in range(len(SHAPES)):
            (p0, m0), (p1, m1) = runs[0][d], run[d]
            if precision == "fp64":
                assert (p0 == p1).all() and (m0 == m1).all(), (shape, d)
            else:
                assert np.abs(p0 - p1).max() <= 1e-6, (shape, d)
                assert np.abs(m0 - m1).max() <= 1e-6 * max(np.abs(m0).max(), 1e-8), (shape, d)


def test_half_height_lean_tiles_match_the_oracle():
    params = [_params(i, window=9.0 if i == 0 else 0.0) for i in range(len(SHAPES))]
    params[0]["seed_layers"] = 12
    seeds = [7 * i + 3 for i in range(len(SHAPES))]
    b = pf.Batch(SHAPES, params, "fp32")
    pf.pf_batch_set_config(b.h, 16, 2, 2, 4)
    b.init(seeds)
    b.step(25)
    b.sync()
    assert pf.pf_batch_step_bytes(b.h)["lean_step"] > 0  # the half-height lean kernel ran
    for d, (shape, p) in enumerate(zip(SHAPES, params)):
        ref = oracle.State(p, *shape).init(seeds[d])
        ref.step(25)
        phi, mu = b.fields(d)
        assert np.abs(phi - ref.phi).max() <= 2e-5, d
        assert np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8) <= 2e-5, d
        assert b.shifts(d) == ref.shifts, d
    b.close()


def test_set_config_rejects_shapes_it_cannot_run():
    b = pf.Batch(SHAPES[:2], [_params(0), _params(1)], "fp32")
    for bad in [(-1, 2, 1, 8), (0, 3, 1, 8), (0, 2, 3, 8), (0, 2, 1, 2), (0, 0, 1, 8)]:
        with pytest.raises(pf.PfError) as e:
            pf.pf_batch_set_config(b.h, *bad)
        assert e.value.status == pf.PF_E_INVAL
    b.close()


def test_general_parameter_set_matches_the_oracle_under_every_launch_shape():
    # matrix curvatures and pair relaxation times take other branches in every batched kernel, the
    # lean kernel's liquid constants included; each launch shape (half-height lean tiles, split z
    # chunks) must reach the oracle's fields.  Domain 0's window moves.  FP64 only: in plain FP32 a
    # rounding residue can tip a single-phase cell across the jump of the pair relaxation time (the
    # cases and the compensated state's answer are in test_gpu_precision.py).
    precision, tol = "fp64", 1e-12
    params = []
    for i in range(len(SHAPES)):
        rng = np.random.default_rng(200 + i)
        q = W.general_params(G=float(rng.uniform(5e-4, 2e-3)), v=float(rng.uniform(5e-3, 2e-2)),
                             n_grains=int(rng.integers(2, 9)), window_trigger_z=9.0 if i == 0 else 0.0)
        params.append(q)
    params[0]["seed_layers"] = 12
    seeds = [4 * i + 9 for i in range(len(SHAPES))]
    refs = []
    for d, (shape, q) in enumerate(zip(SHAPES, params)):
        ref = oracle.State(q, *shape).init(seeds[d])
        ref.step(25)
        refs.append(ref)
    assert refs[0].shifts > 0
    for launch in [(0, 2, 1, 4), (16, 1, 2, 4), (32, 2, 4, 8)]:
        b = pf.Batch(SHAPES, params, precision)
        pf.pf_batch_set_config(b.h, *launch)
        b.init(seeds)
        b.step(25)
        b.sync()
        for d, ref in enumerate(refs):
            phi, mu = b.fields(d)
            assert b.shifts(d) == ref.shifts, (launch, d)
            assert np.abs(phi - ref.phi).max() <= tol, (launch, d)
            assert np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8) <= tol, (launch, d)
        b.close()
