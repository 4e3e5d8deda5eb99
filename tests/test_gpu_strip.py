"""GPU parity of the strip form (TVLBM_FORM_STRIP).

Each CTA walks a run of rows of a 128-column strip (one column per thread) with the previous row
carried in registers, its source rows arriving in a ring of TMA row-chunk copies.  The per-row
arithmetic (x-interpolation, y-interpolation against the carried row, collision, stores with
periodic images) is the tiled form's, so the two must give the same populations bit for bit, for
any domain shape -- runs that cross from one strip into the next, a last strip narrower than 128
columns, fewer rows than CTAs, walls and per-row references included -- and FP64 storage must
match the oracle element by element."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

WALLS = (0.0, 1.0, 0.1, 1.1)


@pytest.fixture(scope="module")
def tv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    return tv


def run(tv, nx, ny, velset, storage, form, fields, splits, tau=0.7, dt=1.0, walls=None, rows=None, refresh=0):
    sim = tv.Simulation(nx, ny, velset, tau=tau, dt=dt, storage=storage, walls=walls)
    sim.set_form(form)
    if rows is not None:
        sim.set_reference_rows(*rows)
        if refresh:
            sim.set_reference_refresh(refresh, kind="mean")
    sim.init_moments(*fields)
    for n in splits:
        sim.step(n)
    out = sim.raw_populations()
    sums = sim.conserved_sums()
    sim.close()
    return out, sums


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp32_dev", "fp16_dev", "bf16_dev"])
@pytest.mark.parametrize("nx,ny", [(300, 37), (256, 64), (96, 40), (77, 53), (5, 3), (33, 1), (1, 70)])
def test_strip_equals_tiled_periodic(tv, storage, nx, ny):
    """D2Q16, periodic: whole and ragged strips, a single narrow strip, one row, one column."""
    fields = workloads.random_smooth(nx, ny, seed=70, amp_u=0.05, amp_T=0.03)
    a, sa = run(tv, nx, ny, "D2Q16", storage, "tiled", fields, [23])
    b, sb = run(tv, nx, ny, "D2Q16", storage, "strip", fields, [1, 5, 17])
    assert np.array_equal(a, b)
    assert np.array_equal(sa, sb)


@pytest.mark.parametrize("velset,dt", [("D2Q9", 1.0 / np.sqrt(3.0)), ("D2Q9", 0.8), ("D2Q36", 0.45), ("D2Q36", 1.0),
                                       ("D2Q16", 0.6)])
@pytest.mark.parametrize("walls", [None, WALLS])
def test_strip_equals_tiled_sets_and_walls(tv, velset, dt, walls):
    nx, ny = 270, 45
    fields = workloads.random_smooth(nx, ny, seed=71, amp_u=0.04, amp_T=0.02)
    a, _ = run(tv, nx, ny, velset, "fp32_dev", "tiled", fields, [19], dt=dt, walls=walls)
    b, _ = run(tv, nx, ny, velset, "fp32_dev", "strip", fields, [19], dt=dt, walls=walls)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["fp32_dev", "fp16_dev", "bf16_dev"])
def test_strip_equals_tiled_row_reference(tv, storage):
    """D2Q36 channel with the per-row reference refreshed from the rows' mean populations every 5
    steps (the channel workload's arrangement, 300 x 48)."""
    nx, ny = 300, 48
    _, ux, uy, T = workloads.couette_linear(1, ny, WALLS[1], WALLS[3])
    rows = (ux[:, 0], uy[:, 0], T[:, 0])
    fields = workloads.couette_linear(nx, ny, WALLS[1], WALLS[3])
    a, sa = run(tv, nx, ny, "D2Q36", storage, "tiled", fields, [23], tau=0.9, walls=WALLS, rows=rows, refresh=5)
    b, sb = run(tv, nx, ny, "D2Q36", storage, "strip", fields, [23], tau=0.9, walls=WALLS, rows=rows, refresh=5)
    assert np.array_equal(a, b)
    assert np.array_equal(sa, sb)


@pytest.mark.parametrize("velset,walls", [("D2Q16", None), ("D2Q36", WALLS), ("D2Q9", None)])
def test_strip_fp64_matches_oracle(tv, velset, walls):
    """FP64, 150 x 38, 40 steps: element-wise against the oracle (rounding order only)."""
    nx, ny, steps = 150, 38, 40
    fields = workloads.random_smooth(nx, ny, seed=72, amp_u=0.05, amp_T=0.03)
    sim = tv.Simulation(nx, ny, velset, tau=0.8, dt=1.0, storage="fp64", walls=walls, form="strip")
    sim.init_moments(*fields)
    sim.step(steps)
    ref = oracle.Oracle(nx, ny, velset, tau=0.8, dt=1.0, walls=walls)
    ref.init_moments(*fields)
    ref.run(steps)
    got = sim.populations_f64()
    assert float(np.max(np.abs(got - ref.f)) / np.max(np.abs(ref.f))) < 1e-11
    s0 = sim.conserved_sums()
    assert s0[4] == 0
    sim.close()


def test_strip_zero_steps_and_conservation(tv):
    nx, ny = 64, 50
    fields = workloads.random_smooth(nx, ny, seed=73, amp_u=0.05, amp_T=0.03)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=0.6, storage="fp64", form="strip")
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


def test_strip_full_size_channel_equals_tiled(tv):
    """The 4096 x 512 D2Q36 FP16-deviation channel (row-mean reference refreshed every 100 steps),
    150 steps: the strip form equals the tiled form bit for bit at the size the bench times."""
    nx, ny = 4096, 512
    _, ux, uy, T = workloads.couette_linear(1, ny, WALLS[1], WALLS[3])
    rows = (ux[:, 0], uy[:, 0], T[:, 0])
    fields = workloads.couette_linear(nx, ny, WALLS[1], WALLS[3])
    a, _ = run(tv, nx, ny, "D2Q36", "fp16_dev", "tiled", fields, [150], tau=0.9, walls=WALLS, rows=rows, refresh=100)
    b, _ = run(tv, nx, ny, "D2Q36", "fp16_dev", "strip", fields, [150], tau=0.9, walls=WALLS, rows=rows, refresh=100)
    assert np.array_equal(a, b)


def test_strip_full_size_periodic_equals_tiled(tv):
    """The 1024 x 1024 D2Q16 FP32-deviation workload, 100 steps, strip against tiled."""
    nx = ny = 1024
    fields = workloads.gaussian_bump_random_flow(nx, ny, seed=1)
    a, _ = run(tv, nx, ny, "D2Q16", "fp32_dev", "tiled", fields, [100])
    b, _ = run(tv, nx, ny, "D2Q16", "fp32_dev", "strip", fields, [100])
    assert np.array_equal(a, b)


def test_batch_refuses_strip(tv):
    b = tv.Batch([64, 96], [64, 32], [0.7, 0.8], "D2Q16", storage="fp32_dev")
    with pytest.raises(tv.TvlbmError):
        b.set_form("strip")
    b.close()
