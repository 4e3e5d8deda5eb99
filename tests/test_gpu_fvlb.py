"""GPU parity of the finite-volume scheme (TVLBM_SCHEME_FVLB) against the FP64 oracle
(oracle/fvlb.py): element-wise populations in FP64 storage (rounding order only), FP32 storage
within its rounding, every velocity set without the Prandtl term and D2Q16 with it; exact
conservation; the viscosity ratio the Prandtl term sets."""
import math

import numpy as np
import pytest

import workloads
from oracle import fvlb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    return tv


def pair(tv, nx, ny, velset, storage, tau, tau_g, dt, seed):
    fields = workloads.random_smooth(nx, ny, seed=seed, amp_u=0.05, amp_T=0.03)
    sim = tv.Simulation(nx, ny, velset, tau=tau, dt=dt, storage=storage)
    sim.set_scheme("fvlb", tau_g)
    sim.init_moments(*fields)
    ref = fvlb.FVLB(nx, ny, velset, tau=tau, tau_g=tau_g, dt=dt)
    ref.init_moments(*fields)
    return sim, ref


@pytest.mark.parametrize("velset,tau_g", [("D2Q9", np.inf), ("D2Q16", np.inf), ("D2Q36", np.inf),
                                          ("D2Q16", 2.0), ("D2Q16", -1.0)])
def test_fp64_matches_oracle(tv, velset, tau_g):
    dt = {"D2Q9": 0.05, "D2Q16": 0.02, "D2Q36": 0.01}[velset]
    sim, ref = pair(tv, 37, 29, velset, "fp64", 0.5, tau_g, dt, 17)
    sim.step(40)
    ref.step(40)
    got = sim.populations_f64()
    assert np.max(np.abs(got - ref.f)) <= 1e-12 * np.max(np.abs(ref.f))
    sim.close()


@pytest.mark.parametrize("velset,storage,tau_g,pscale", [
    ("D2Q9", "fp64", np.inf, False), ("D2Q16", "fp64", 2.0, True), ("D2Q36", "fp64", -1.0, False),
    ("D2Q9", "fp32", 2.0, False), ("D2Q16", "fp32", 2.0, False), ("D2Q16", "fp32", np.inf, True),
    ("D2Q36", "fp32", 2.0, False)])
@pytest.mark.parametrize("nx,ny", [(37, 29), (97, 45)])
def test_fused_equals_two_kernels(tv, velset, storage, tau_g, pscale, nx, ny):
    """One fused kernel per step (the collision term of each block in shared memory, recomputed
    on the block's ring of halo cells) gives the two-kernel form's populations bit for bit, on
    grids that leave ragged blocks in both directions."""
    dt = {"D2Q9": 0.05, "D2Q16": 0.02, "D2Q36": 0.01}[velset]
    fields = workloads.random_smooth(nx, ny, seed=23, amp_u=0.05, amp_T=0.03)
    out = []
    for fused in (True, False):
        sim = tv.Simulation(nx, ny, velset, tau=0.5, dt=dt, storage=storage)
        sim.set_scheme("fvlb", tau_g)
        if pscale:
            sim.set_fv_pressure_scaling(True)
        sim.set_fv_fused(fused)
        sim.init_moments(*fields)
        sim.step(25)
        out.append(sim.populations_f64())
        sim.close()
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1])


def test_fp32_matches_oracle(tv):
    sim, ref = pair(tv, 40, 24, "D2Q16", "fp32", 0.5, 2.0, 0.02, 18)
    sim.step(50)
    ref.step(50)
    got = sim.moments()
    want = ref.moments()
    for k in range(4):
        assert np.max(np.abs(got[k] - want[k])) <= 1e-5 * max(np.max(np.abs(want[k])), 1e-3), k
    sim.close()


@pytest.mark.parametrize("tau_g", [np.inf, 2.0])
def test_conserves(tv, tau_g):
    sim, _ = pair(tv, 64, 48, "D2Q16", "fp64", 0.5, tau_g, 0.02, 19)
    s0 = sim.conserved_sums()
    sim.step(200)
    s1 = sim.conserved_sums()
    for k in range(4):
        assert abs(s1[k] - s0[k]) <= 1e-12 * abs(s0[0])
    sim.close()


def test_prandtl_term_sets_the_viscosity_ratio(tv):
    """Shear-wave decay on the GPU: nu(tau_g) / nu(inf) = tau_g / (tau_g - 2 tau)."""
    ny, nx, tau, dt = 64, 32, 0.5, 0.02
    k = 2 * math.pi / ny
    y = np.arange(ny, dtype=float).reshape(-1, 1) * np.ones((1, nx))

    def rate(tau_g):
        sim = tv.Simulation(nx, ny, "D2Q16", tau=tau, dt=dt, storage="fp64")
        sim.set_scheme("fvlb", tau_g)
        sim.init_moments(*workloads.shear_wave(nx, ny, eps=0.01))
        sim.step(250)
        a0 = np.mean(sim.moments()[1] * np.sin(k * y))
        sim.step(1500)
        a1 = np.mean(sim.moments()[1] * np.sin(k * y))
        sim.close()
        return math.log(a0 / a1) / (1500 * dt)

    base = rate(np.inf)
    assert abs(base / (tau * k * k) - 1) < 0.02
    for tau_g in (4 * tau, -2 * tau):
        r = rate(tau_g) / base
        assert abs(r / (tau_g / (tau_g - 2 * tau)) - 1) < 0.03, (tau_g, r)


def test_scheme_rejections(tv):
    s = tv.Simulation(32, 32, "D2Q16", storage="fp32_dev")
    with pytest.raises(tv.TvlbmError):
        s.set_scheme("fvlb", 2.0)
    s.close()
    # a channel takes the scheme, but steps only once its walls are configured
    s = tv.Simulation(32, 32, "D2Q16", storage="fp64", walls=(0.0, 1.0, 0.0, 1.0))
    s.set_scheme("fvlb")
    with pytest.raises(tv.TvlbmError):
        s.step(1)
    s.close()
    s = tv.Simulation(32, 32, "D2Q16", storage="fp64")
    with pytest.raises(tv.TvlbmError):
        s.set_scheme("fvlb", 0.0)
    s.set_scheme("fvlb", 1.0)
    s.set_scheme("volumetric")  # back to the default scheme
    s.step(2)
    s.close()
