"""The 4096 x 4096 D2Q16 FP32-deviation workload at full size, in the launch configuration the
bench times there (tiled form, 64 x 16 tiles): against the FP64 oracle on the whole grid after a
few steps (moments and populations), and every sweep form that can run it -- tiled with each
tile shape, dataflow, strip -- bit-identical to that configuration over more steps."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

N = 4096


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    fields = workloads.gaussian_bump_random_flow(N, N, seed=1, sigma=64.0 * N / 1024)
    return tv, fields


def bench_config(tv):
    sim = tv.Simulation(N, N, "D2Q16", tau=0.7, storage="fp32_dev")
    cfg = [k for k in range(tv.tvlbm_tile_count(sim.ctx)) if tuple(tv.tvlbm_tile_shape(sim.ctx, k)) == (64, 16, 4)][0]
    sim.set_tile(cfg)
    sim.set_form("tiled")
    return sim, cfg


def test_full_size_matches_oracle(setup):
    tv, fields = setup
    steps = 3
    sim, _ = bench_config(tv)
    sim.init_moments(*fields)
    sim.step(steps)
    got = sim.populations_f64()
    mom = sim.moments()
    sums = sim.conserved_sums()
    sim.close()
    ref = oracle.Oracle(N, N, "D2Q16", tau=0.7, dt=1.0)
    ref.init_moments(*fields)
    ref.run(steps)
    # FP32 deviation storage: populations to the storage's rounding relative to the rest weights
    assert float(np.max(np.abs(got - ref.f)) / np.max(np.abs(ref.f))) < 1e-6
    want = ref.moments()
    for g, w, name in zip(mom, want, ("rho", "ux", "uy", "T")):
        assert float(np.max(np.abs(g - w)) / np.max(np.abs(w))) < 1e-5, name
    ref_sums = ref.conserved_sums()
    assert sums[4] == 0
    assert abs(sums[0] - ref_sums[0]) <= 1e-7 * ref_sums[0]


def test_full_size_forms_bit_identical(setup):
    tv, fields = setup
    steps = 20
    sim, cfg = bench_config(tv)
    sim.init_moments(*fields)
    sim.step(steps)
    want = sim.raw_populations()
    sim.close()
    runs = []
    for c in range(4):
        runs.append(("tiled", c))
        runs.append(("flow", c))
    runs.append(("strip", 0))
    for form, c in runs:
        if (form, c) == ("tiled", cfg):
            continue
        s = tv.Simulation(N, N, "D2Q16", tau=0.7, storage="fp32_dev")
        s.set_tile(c)
        s.set_form(form)
        s.init_moments(*fields)
        s.step(steps)
        assert np.array_equal(s.raw_populations(), want), (form, c)
        s.close()
