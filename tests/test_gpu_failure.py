"""Failure detection on the GPU, in the forms that leave the device usable: a bounded device wait
that is made to run out (a completion count no tile reaches, through the test hook
tvlbm_set_flow_wait) must end the launch early with the status word set, be reported as
TVLBM_ETIMEOUT by the next synchronising call, and leave a context that recovers once its
populations are restored; non-finite populations written in from the host must be counted by
the conserved sums and reported as TVLBM_ENONFINITE.  Nothing here faults, traps or hangs."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    return tv


def test_flow_wait_timeout_is_reported_and_the_context_recovers(tv):
    n = 64
    sim = tv.Simulation(n, n, "D2Q16", tau=0.7, storage="fp32_dev", form="flow")
    sim.init_moments(*workloads.random_smooth(n, n, seed=21))
    sim.step(3)
    snap = sim.raw_populations()
    tv.tvlbm_set_flow_wait(sim.ctx, 1e-3, unmet=True)
    sim.step(20)  # asynchronous: the launch gives up its first neighbourhood wait after 1 ms
    with pytest.raises(tv.TvlbmError) as e:
        sim.conserved_sums()
    assert e.value.code == tv.TVLBM_ETIMEOUT
    sim.moments()  # the status was cleared: the next synchronising call succeeds
    # restore and run again with the default wait: same populations as an undisturbed context
    tv.tvlbm_set_flow_wait(sim.ctx, 2.0, unmet=False)
    sim.set_raw_populations(snap)
    sim.step(20)
    ref = tv.Simulation(n, n, "D2Q16", tau=0.7, storage="fp32_dev", form="flow")
    ref.set_raw_populations(snap)
    ref.step(20)
    assert np.array_equal(sim.raw_populations(), ref.raw_populations())
    assert sim.conserved_sums()[4] == 0
    sim.close()
    ref.close()


def test_flow_wait_hook_rejects_bad_limits(tv):
    sim = tv.Simulation(32, 32, "D2Q16", storage="fp32_dev")
    for bad in (0.0, -1.0, 3.0, float("nan")):
        with pytest.raises(tv.TvlbmError) as e:
            tv.tvlbm_set_flow_wait(sim.ctx, bad)
        assert e.value.code == tv.TVLBM_EINVAL
    sim.close()


@pytest.mark.parametrize("storage", ["fp32", "fp32_dev", "bf16_dev", "fp64"])
def test_nonfinite_populations_are_reported(tv, storage):
    nx, ny = 40, 24
    sim = tv.Simulation(nx, ny, "D2Q16", tau=0.8, storage=storage)
    sim.init_moments(*workloads.random_smooth(nx, ny, seed=22))
    assert sim.conserved_sums()[4] == 0
    raw = sim.raw_populations()
    if raw.dtype == np.uint16:  # half storage: the raw bit patterns of NaN and +inf
        nan_bits, inf_bits = (0x7FC0, 0x7F80) if storage == "bf16_dev" else (0x7E00, 0x7C00)
        raw[5, 7, 11] = nan_bits
        raw[9, 3, 2] = inf_bits
    else:
        raw[5, 7, 11] = np.nan
        raw[9, 3, 2] = np.inf
    sim.set_raw_populations(raw)
    with pytest.raises(tv.TvlbmError) as e:
        sim.conserved_sums()
    assert e.value.code == tv.TVLBM_ENONFINITE
    assert sim.conserved_sums(allow_nonfinite=True)[4] == 2
    sim.step(2)  # the stream carries them into the neighbouring cells
    assert sim.conserved_sums(allow_nonfinite=True)[4] > 2
    sim.close()
