"""GPU parity of the multi-step dataflow form (TVLBM_FORM_FLOW).

The dataflow launch runs the same per-tile gather/collide/store as the tiled form, so for the
same tile configuration its populations must equal the tiled form's bit for bit, for any step
count and any split of the steps into calls; FP64 storage is also compared with the oracle
element by element.  Domains that the form cannot run (walls, tiles that do not cover the
domain) must be refused."""
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


def tile_of(tv, velset, storage, cfg):
    sim = tv.Simulation(64, 64, velset, storage=storage)
    shape = tv.tvlbm_tile_shape(sim.ctx, cfg)
    sim.close()
    return shape[0], shape[1]


def run(tv, nx, ny, velset, storage, form, cfg, fields, splits, tau=0.7, dt=1.0):
    sim = tv.Simulation(nx, ny, velset, tau=tau, dt=dt, storage=storage)
    sim.set_tile(cfg)
    sim.set_form(form)
    sim.init_moments(*fields)
    for n in splits:
        sim.step(n)
    out = sim.raw_populations()
    sums = sim.conserved_sums()
    sim.close()
    return out, sums


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp32_dev", "fp16_dev", "bf16_dev"])
@pytest.mark.parametrize("cfg", [0, 1, 2, 3])
def test_flow_equals_tiled_bit_exact(tv, storage, cfg):
    """D2Q16, 3 x 5 tiles of configuration cfg, 37 steps in uneven calls."""
    tx, ty = tile_of(tv, "D2Q16", storage, cfg)
    nx, ny = 3 * tx, 5 * ty
    fields = workloads.random_smooth(nx, ny, seed=40 + cfg, amp_u=0.05, amp_T=0.03)
    a, sa = run(tv, nx, ny, "D2Q16", storage, "tiled", cfg, fields, [37])
    b, sb = run(tv, nx, ny, "D2Q16", storage, "flow", cfg, fields, [1, 7, 29])
    assert np.array_equal(a, b)
    assert np.array_equal(sa, sb)


@pytest.mark.parametrize("velset,dt", [("D2Q9", 1.0 / np.sqrt(3.0)), ("D2Q9", 0.8), ("D2Q36", 0.45), ("D2Q36", 1.0)])
def test_flow_equals_tiled_other_sets(tv, velset, dt):
    tx, ty = tile_of(tv, velset, "fp32_dev", 0)
    nx, ny = 4 * tx, 3 * ty
    fields = workloads.random_smooth(nx, ny, seed=50, amp_u=0.04, amp_T=0.02)
    a, _ = run(tv, nx, ny, velset, "fp32_dev", "tiled", 0, fields, [24], dt=dt)
    b, _ = run(tv, nx, ny, velset, "fp32_dev", "flow", 0, fields, [24], dt=dt)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("tiles", [(1, 1), (1, 2), (2, 1), (2, 2), (1, 7), (6, 1)])
def test_flow_degenerate_tile_grids(tv, tiles):
    """One or two tiles per direction: a tile is its own (or its only) periodic neighbour."""
    tx, ty = tile_of(tv, "D2Q16", "fp32", 0)
    nx, ny = tiles[0] * tx, tiles[1] * ty
    fields = workloads.random_smooth(nx, ny, seed=60, amp_u=0.05)
    a, _ = run(tv, nx, ny, "D2Q16", "fp32", "tiled", 0, fields, [19])
    b, _ = run(tv, nx, ny, "D2Q16", "fp32", "flow", 0, fields, [19])
    assert np.array_equal(a, b)


def test_flow_fp64_matches_oracle(tv):
    """FP64, D2Q16, 4 x 8 tiles, 60 steps: element-wise against the oracle (rounding order)."""
    tx, ty = tile_of(tv, "D2Q16", "fp64", 0)
    nx, ny = 4 * tx, 8 * ty
    fields = workloads.random_smooth(nx, ny, seed=61, amp_u=0.05, amp_T=0.03)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=0.8, dt=1.0, storage="fp64", form="flow")
    sim.init_moments(*fields)
    sim.step(60)
    ref = oracle.Oracle(nx, ny, "D2Q16", tau=0.8, dt=1.0)
    ref.init_moments(*fields)
    ref.run(60)
    got = sim.populations_f64()
    assert float(np.max(np.abs(got - ref.f)) / np.max(np.abs(ref.f))) < 1e-11
    sim.close()


def test_flow_full_size_bench_configuration(tv):
    """The 1024 x 1024 D2Q16 FP32 workload, every tile configuration that covers it: the
    dataflow launch of 100 steps equals 100 tiled launches bit for bit."""
    nx = ny = 1024
    fields = workloads.gaussian_bump_random_flow(nx, ny, seed=1)
    for cfg in range(4):
        a, _ = run(tv, nx, ny, "D2Q16", "fp32_dev", "tiled", cfg, fields, [100])
        b, _ = run(tv, nx, ny, "D2Q16", "fp32_dev", "flow", cfg, fields, [100])
        assert np.array_equal(a, b), "tile configuration %d" % cfg


def test_flow_refuses_walls_and_ragged(tv):
    sim = tv.Simulation(64, 40, "D2Q16", storage="fp32", walls=(0.0, 1.0, 0.0, 1.0))
    with pytest.raises(tv.TvlbmError):
        sim.set_form("flow")
    sim.close()
    tx, ty = tile_of(tv, "D2Q16", "fp32", 0)
    sim = tv.Simulation(3 * tx + 1, 2 * ty, "D2Q16", storage="fp32")
    with pytest.raises(tv.TvlbmError):
        sim.set_form("flow")
    sim.close()
    # in the dataflow form, a tile configuration that leaves a ragged tile is refused and the
    # current one stays selected
    shapes = [tile_of(tv, "D2Q16", "fp32", c) for c in range(4)]
    nx, ny = shapes[0][0], shapes[0][1]
    bad = [c for c, (x, y) in enumerate(shapes) if nx % x or ny % y]
    sim = tv.Simulation(nx, ny, "D2Q16", storage="fp32", form="flow")
    for c in bad:
        with pytest.raises(tv.TvlbmError):
            sim.set_tile(c)
    sim.step(3)
    sim.close()


def test_flow_zero_steps_and_conservation(tv):
    tx, ty = tile_of(tv, "D2Q16", "fp64", 0)
    nx, ny = 2 * tx, 3 * ty
    fields = workloads.random_smooth(nx, ny, seed=62, amp_u=0.05, amp_T=0.03)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=0.6, storage="fp64", form="flow")
    sim.init_moments(*fields)
    before = sim.raw_populations()
    s0 = sim.conserved_sums()
    sim.step(0)
    assert np.array_equal(before, sim.raw_populations())
    sim.step(45)
    s1 = sim.conserved_sums()
    assert s1[4] == 0.0
    for k in range(4):
        assert abs(s1[k] - s0[k]) <= 1e-12 * max(1.0, abs(s0[0]))
    sim.close()
