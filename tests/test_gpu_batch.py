"""Batched domains (tiled form: one launch per time step over the tiles of every domain;
dataflow form: many time steps in one persistent launch): each domain must evolve exactly as
the same domain run alone, and, for FP64 storage, as the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    return tv


SIZES = [(64, 48), (128, 64), (40, 72), (96, 96), (33, 17)]  # includes ragged tiles
TAUS = [0.6, 0.8, 1.3, 0.55, 0.9]


@pytest.mark.parametrize("storage", ["fp32_dev", "fp16_dev"])
@pytest.mark.parametrize("config", [0, 1, 2, 3])
def test_batch_equals_single_domain_runs(tv, storage, config):
    nx = [s[0] for s in SIZES]
    ny = [s[1] for s in SIZES]
    b = tv.Batch(nx, ny, TAUS, "D2Q16", storage=storage)
    b.set_tile(config)
    fields = [workloads.random_smooth(x, y, seed=40 + d, amp_u=0.06, amp_T=0.06) for d, (x, y) in enumerate(SIZES)]
    for d, f in enumerate(fields):
        b.init_moments(d, *f)
    b.step(45)  # graph replay (32) + direct launches
    for d, (x, y) in enumerate(SIZES):
        s = tv.Simulation(x, y, "D2Q16", tau=TAUS[d], storage=storage, form="tiled")
        s.set_tile(config)
        s.init_moments(*fields[d])
        s.step(45)
        assert np.array_equal(b.populations_f64(d), s.populations_f64()), (d, config)
        s.close()
    b.close()


FLOW_SIZES = [(64, 48), (128, 64), (192, 96), (64, 32), (256, 16)]  # multiples of every tile shape


@pytest.mark.parametrize("storage", ["fp32_dev", "fp16_dev", "fp64"])
@pytest.mark.parametrize("config", [0, 1, 2, 3])
def test_batch_flow_equals_single_domain_runs(tv, storage, config):
    """The persistent multi-step launch (captured on the first call of each start parity,
    replayed after, launched directly for another step count) gives every domain the populations
    of the same domain run alone in the tiled form, bit for bit."""
    nx = [s[0] for s in FLOW_SIZES]
    ny = [s[1] for s in FLOW_SIZES]
    taus = [0.6, 0.8, 1.3, 0.55, 0.9]
    b = tv.Batch(nx, ny, taus, "D2Q16", storage=storage)
    b.set_tile(config)
    b.set_form("flow")
    fields = [workloads.random_smooth(x, y, seed=80 + d, amp_u=0.06, amp_T=0.06) for d, (x, y) in enumerate(FLOW_SIZES)]
    for d, f in enumerate(fields):
        b.init_moments(d, *f)
    b.step(21)  # captured (start parity 0)
    b.step(21)  # captured (start parity 1)
    b.step(21)  # replayed
    b.step(5)   # another count: a direct launch
    for d, (x, y) in enumerate(FLOW_SIZES):
        s = tv.Simulation(x, y, "D2Q16", tau=taus[d], storage=storage, form="tiled")
        s.set_tile(config)
        s.init_moments(*fields[d])
        s.step(68)
        assert np.array_equal(b.populations_f64(d), s.populations_f64()), (d, config)
        s.close()
    assert all(b.conserved_sums(d)[4] == 0 for d in range(len(FLOW_SIZES)))
    b.close()


def test_batch_flow_rejections(tv):
    nx = [s[0] for s in SIZES]
    ny = [s[1] for s in SIZES]
    b = tv.Batch(nx, ny, TAUS, "D2Q16", storage="fp32_dev")
    with pytest.raises(tv.TvlbmError) as e:
        b.set_form("flow")  # ragged domains
    assert e.value.code == tv.TVLBM_EINVAL
    b.close()
    b = tv.Batch([64, 128], [24, 64], [0.7, 0.8], "D2Q16", storage="fp32_dev")
    cfg8 = [k for k in range(b.tile_count()) if tuple(b.tile_shape(k))[:2] == (32, 8)][0]
    cfg16 = [k for k in range(b.tile_count()) if tuple(b.tile_shape(k))[:2] == (32, 16)][0]
    b.set_tile(cfg8)
    b.set_form("flow")
    with pytest.raises(tv.TvlbmError):
        b.set_tile(cfg16)  # 16-row tiles do not cover 24 rows
    b.close()


def test_batch_fp64_matches_oracle(tv):
    nx = [s[0] for s in SIZES[:3]]
    ny = [s[1] for s in SIZES[:3]]
    b = tv.Batch(nx, ny, TAUS[:3], "D2Q36", storage="fp64")
    fields = [workloads.random_smooth(x, y, seed=60 + d) for d, (x, y) in enumerate(SIZES[:3])]
    for d, f in enumerate(fields):
        b.init_moments(d, *f)
    b.step(20)
    for d, (x, y) in enumerate(SIZES[:3]):
        ref = oracle.Oracle(x, y, "D2Q36", tau=TAUS[d])
        ref.init_moments(*fields[d])
        ref.run(20)
        got = b.populations_f64(d)
        assert np.max(np.abs(got - ref.f)) / np.max(np.abs(ref.f)) < 1e-11, d
    b.close()


def test_batch_conservation_per_domain(tv):
    nx = [128, 256, 64]
    ny = [128, 64, 192]
    b = tv.Batch(nx, ny, [0.7, 1.1, 0.58], "D2Q16", storage="fp32_dev")
    for d in range(3):
        b.init_moments(d, *workloads.random_smooth(nx[d], ny[d], seed=70 + d, amp_u=0.1, amp_T=0.1))
    s0 = [b.conserved_sums(d) for d in range(3)]
    b.step(300)
    for d in range(3):
        s1 = b.conserved_sums(d)
        assert np.all(np.abs(s1[:4] - s0[d][:4]) < 2e-8 * s0[d][0]), (d, s1 - s0[d])
    b.close()


@pytest.mark.slow
@pytest.mark.parametrize("form", ["tiled", "flow"])
def test_batch_full_size_bench_workload(tv, form):
    """The batched workload as the bench runs it: 256 periodic D2Q16 domains (sides from
    {128 .. 1024}, tau ~ U[0.55, 1.5], seeded Gaussian bump + random flow at each domain's Mach
    number), FP32 deviation storage, the 64 x 16 tile, one bench step of 20 time steps, in both
    forms (the bench's autotuner picks the faster).  The smallest, a middle and the largest domain equal the same domain run
    alone bit for bit (single-domain runs are checked against the oracle elsewhere), and every
    domain conserves mass, momentum and energy to FP32 rounding."""
    specs = workloads.batched_domains(256, seed=3)
    n = [s["n"] for s in specs]
    b = tv.Batch(n, n, [s["tau"] for s in specs], "D2Q16", storage="fp32_dev")
    cfg = [k for k in range(b.tile_count()) if tuple(b.tile_shape(k)) == (64, 16, 4)][0]
    b.set_tile(cfg)
    b.set_form(form)

    def fields(s):
        return workloads.gaussian_bump_random_flow(s["n"], s["n"], seed=s["seed"], amp_u=s["mach"], sigma=s["n"] / 16.0)

    for d, s in enumerate(specs):
        b.init_moments(d, *fields(s))
    s0 = [b.conserved_sums(d) for d in range(len(specs))]
    b.step(20)
    for d in range(len(specs)):
        s1 = b.conserved_sums(d)
        assert s1[4] == 0, d
        assert np.all(np.abs(s1[:4] - s0[d][:4]) < 1e-7 * s0[d][0]), (d, s1 - s0[d])
    order = sorted(range(len(specs)), key=lambda d: specs[d]["n"])
    for d in (order[0], order[len(order) // 2], order[-1]):
        s = specs[d]
        sim = tv.Simulation(s["n"], s["n"], "D2Q16", tau=s["tau"], storage="fp32_dev", form="tiled")
        sim.set_tile(cfg)
        sim.init_moments(*fields(s))
        sim.step(20)
        assert np.array_equal(b.populations_f64(d), sim.populations_f64()), d
        sim.close()
    b.close()
