"""Per-row deviation reference of a channel (tvlbm_set_reference_rows): row y stores
d_l = f_l / w_l - R_l(y) with R_l(y) the equilibrium of a (u, T) profile across the channel.
In exact arithmetic the time step is the same as with one reference (the gather adds the
reference's own gather shift, the collision takes the row's reference moments), so FP32
deviation storage must match the FP64 oracle as tightly as before, and half storage gains
because the stored deviations no longer carry the channel's temperature gradient.  The channel
(walls T = 1.0 / 1.1, top wall u = 0.1) starts at rest with T linear across it; the moving wall's
shear stays within a thin layer over 1000 steps, so the profile is that start: u = 0, T linear."""
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


def field_errors(got, want):
    """(rho, u, T) max errors, each against the field's own max |value| (u: both components
    against max |u_ref|)."""
    e_rho = float(np.max(np.abs(got[0] - want[0])) / np.max(np.abs(want[0])))
    umax = max(np.max(np.abs(want[1])), np.max(np.abs(want[2])), 1e-300)
    e_u = float(max(np.max(np.abs(got[1] - want[1])), np.max(np.abs(got[2] - want[2]))) / umax)
    e_T = float(np.max(np.abs(got[3] - want[3])) / np.max(np.abs(want[3])))
    return e_rho, e_u, e_T


def couette_profile(ny):
    _, ux, uy, T = workloads.couette_linear(1, ny, WALLS[1], WALLS[3])
    return ux[:, 0], uy[:, 0], T[:, 0]


def perturbed_couette(nx, ny, seed):
    rho, ux, uy, T = workloads.couette_linear(nx, ny, WALLS[1], WALLS[3])
    pert = workloads.random_smooth(nx, ny, seed=seed, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    return rho * pert[0], ux + pert[1], uy + pert[2], T * pert[3]


def gpu_run(tv, nx, ny, velset, storage, form, fields, steps, rows=True, tau=0.9):
    sim = tv.Simulation(nx, ny, velset, tau=tau, walls=WALLS, storage=storage, form=form)
    if rows:
        sim.set_reference_rows(*couette_profile(ny))
    else:
        sim.set_reference(0.05, 0.0, 1.05)
    sim.init_moments(*fields)
    sim.step(steps)
    return sim


def oracle_run(nx, ny, velset, fields, steps, tau=0.9):
    ref = oracle.Oracle(nx, ny, velset, tau=tau, walls=WALLS)
    ref.init_moments(*fields)
    ref.run(steps)
    return ref


@pytest.mark.parametrize("velset", ["D2Q16", "D2Q36"])
@pytest.mark.parametrize("form", ["plain", "tiled"])
def test_fp32_dev_matches_oracle(tv, velset, form):
    nx, ny, steps = 64, 48, 300
    fields = perturbed_couette(nx, ny, 41)
    sim = gpu_run(tv, nx, ny, velset, "fp32_dev", form, fields, steps)
    errs = field_errors(sim.moments(), oracle_run(nx, ny, velset, fields, steps).moments())
    print("row reference fp32_dev", velset, form, "errors (rho, u, T):", errs)
    assert max(errs) < 1e-5, errs
    sim.close()


@pytest.mark.parametrize("storage,bound", [("fp16_dev", 1e-3), ("bf16_dev", 3e-2)])
@pytest.mark.parametrize("form", ["plain", "tiled"])
def test_half_storage_walls_d2q36(tv, storage, bound, form):
    """96 x 64, 1000 steps, the x-varying perturbation of the single-reference test (u and T
    perturbed by 2 %, which no row reference follows: it dominates the deviations here, so both
    references end at similar errors).  FP16 meets the 1e-3 bar; BF16's bound is a regression
    check at its measured level (its 8-bit significand resolves a 2 % x-varying perturbation only
    to ~1e-2), not a parity claim: BF16 parity is claimed on the channel workload below."""
    nx, ny = 96, 64
    fields = perturbed_couette(nx, ny, 8)
    want = oracle_run(nx, ny, "D2Q36", fields, 1000).moments()
    errs = {}
    for rows in (True, False):
        sim = gpu_run(tv, nx, ny, "D2Q36", storage, form, fields, 1000, rows=rows)
        errs[rows] = field_errors(sim.moments(), want)
        sim.close()
    print("half storage walls 96x64 1000 steps", storage, form, "row / mean reference:", errs[True], errs[False])
    assert max(errs[True]) < bound, errs


# The half-storage parity claims on the channel workload (bar 1e-3 after 1000 steps): the per-row
# reference refreshed from the rows' mean populations (kind "mean"), which leaves only the
# departures from the row averages since the last refresh in the stored deviations -- every 20
# or 40 steps for BF16 (the bench's channel: 40), every 20 or 100 steps for FP16 (the bench's:
# 100) -- and FP16 with the rows' mean equilibria refreshed every 100 steps.
C2_PARITY = [("bf16_dev", 20, "mean"), ("bf16_dev", 40, "mean"), ("fp16_dev", 20, "mean"), ("fp16_dev", 100, "mean"),
             ("fp16_dev", 100, "equilibrium")]
# Regression checks at measured levels with margin, not parity claims: with the start's profile
# held fixed (refresh 0) the top wall's shear layer, where u climbs to 0.1 against u_ref = 0,
# dominates the FP16 u error; BF16 against the rows' mean equilibria keeps their non-equilibrium
# part in the deviations (4.1e-3 measured).
C2_REGRESSION = [("fp16_dev", 0, "equilibrium", 2e-3), ("bf16_dev", 100, "equilibrium", 1e-2),
                 ("bf16_dev", 0, "equilibrium", 1e-2)]


def c2_run(tv, storage, refresh, kind, steps=1000):
    nx, ny = 4096, 512
    sim = tv.Simulation(nx, ny, "D2Q36", tau=0.9, walls=WALLS, storage=storage, form="tiled")
    sim.set_reference_rows(*couette_profile(ny))
    sim.init_moments(*workloads.couette_linear(nx, ny, WALLS[1], WALLS[3]))
    sim.set_reference_refresh(refresh, kind=kind)
    sim.step(steps)
    got = sim.moments()
    ref = oracle_run(8, ny, "D2Q36", workloads.couette_linear(8, ny, WALLS[1], WALLS[3]), steps)
    want = [np.broadcast_to(a[:, :1], (ny, nx)) for a in ref.moments()]
    errs = field_errors(got, want)
    assert sim.conserved_sums()[4] == 0
    sim.close()
    return errs


@pytest.mark.parametrize("storage,refresh,kind", C2_PARITY)
def test_c2_channel_full_width(tv, storage, refresh, kind):
    """4096 x 512 D2Q36 thermal Couette channel, tau = 0.9, 1000 steps (the tiled form the bench
    times).  The flow is x-invariant, so the oracle runs an 8 x 512 strip; every column must
    match it to the half-storage bar 1e-3."""
    errs = c2_run(tv, storage, refresh, kind)
    print("C2 4096x512 1000 steps row reference", storage, kind, "refresh", refresh, "errors (rho, u, T):", errs)
    assert max(errs) < 1e-3, errs


@pytest.mark.parametrize("storage,refresh,kind,bound", C2_REGRESSION)
def test_c2_channel_regression(tv, storage, refresh, kind, bound):
    errs = c2_run(tv, storage, refresh, kind)
    print("C2 4096x512 1000 steps (regression)", storage, kind, "refresh", refresh, "errors (rho, u, T):", errs)
    assert max(errs) < bound, errs


@pytest.mark.parametrize("kind", ["equilibrium", "mean"])
@pytest.mark.parametrize("form,every", [("plain", 7), ("tiled", 7), ("tiled", 40)])
def test_refresh_is_a_reencoding(tv, form, every, kind):
    """FP32 deviation storage: a run whose reference is refreshed every 7 steps (single launches)
    or every 40 (a captured 32-step graph and single launches between refreshes) matches the
    oracle as tightly as one with a fixed reference; turning the refresh on without a row
    reference takes the state's own row averages.  Kind "mean" takes the rows' mean
    populations, whose density is the row's own (not rho0): the reference's mass enters the
    collision's density and every diagnostic."""
    nx, ny, steps = 64, 48, 100
    fields = perturbed_couette(nx, ny, 44)
    sim = tv.Simulation(nx, ny, "D2Q36", tau=0.9, walls=WALLS, storage="fp32_dev", form=form)
    sim.init_moments(*fields)
    sim.set_reference_refresh(every, kind=kind)
    sim.step(steps)
    errs = field_errors(sim.moments(), oracle_run(nx, ny, "D2Q36", fields, steps).moments())
    print("refresh every", every, "steps fp32_dev", form, "errors (rho, u, T):", errs)
    assert max(errs) < 1e-5, errs
    sim.set_reference_refresh(0)
    sim.step(3)
    sim.close()


@pytest.mark.parametrize("storage,tol", [("fp32_dev", 2e-6), ("fp16_dev", 2e-3)])
def test_row_reference_is_a_reencoding(tv, storage, tol):
    """Setting a row reference mid-run, and going back to a single reference, re-expresses the
    state: moments unchanged to the storage precision; a run with the row reference from the
    start agrees with one that switched to it."""
    nx, ny = 48, 40
    fields = perturbed_couette(nx, ny, 52)
    prof = couette_profile(ny)
    a = tv.Simulation(nx, ny, "D2Q16", tau=0.8, walls=WALLS, storage=storage)
    a.init_moments(*fields)
    a.step(20)
    m0 = a.moments()
    a.set_reference_rows(*prof)
    m1 = a.moments()
    assert max(field_errors(m1, m0)) < tol
    b = tv.Simulation(nx, ny, "D2Q16", tau=0.8, walls=WALLS, storage=storage)
    b.set_reference_rows(*prof)
    b.init_moments(*fields)
    b.step(20)
    a.step(30)
    b.step(30)
    assert max(field_errors(a.moments(), b.moments())) < tol
    m2 = a.moments()
    a.set_reference(0.0, 0.0, 1.0)  # back to the default single reference
    assert max(field_errors(a.moments(), m2)) < tol
    a.step(5)
    b.step(5)
    assert max(field_errors(a.moments(), b.moments())) < tol
    a.close()
    b.close()


def test_populations_round_trip(tv):
    """FP64 populations read out through the row reference equal the oracle's initial state;
    populations written in go through the same rows (the oracle's state after 10 steps, read
    back within FP32 rounding of the deviations)."""
    nx, ny = 40, 24
    fields = perturbed_couette(nx, ny, 60)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=0.8, walls=WALLS, storage="fp32_dev")
    sim.set_reference_rows(*couette_profile(ny))
    sim.init_moments(*fields)
    ref = oracle.Oracle(nx, ny, "D2Q16", tau=0.8, walls=WALLS)
    ref.init_moments(*fields)
    scale = np.max(np.abs(ref.f))
    assert np.max(np.abs(sim.populations_f64() - ref.f)) <= 1e-7 * scale
    ref.run(10)
    sim.set_populations_f64(ref.f)
    assert np.max(np.abs(sim.populations_f64() - ref.f)) <= 1e-7 * scale
    sim.close()


def test_mass_conserved_fp32_dev(tv):
    """Diffuse walls conserve mass; with the row reference FP32 deviation storage keeps it to
    FP32 rounding over 500 steps."""
    nx, ny = 64, 48
    sim = gpu_run(tv, nx, ny, "D2Q16", "fp32_dev", "tiled", perturbed_couette(nx, ny, 70), 0)
    s0 = sim.conserved_sums()
    sim.step(500)
    s1 = sim.conserved_sums()
    assert abs(s1[0] - s0[0]) <= 1e-6 * abs(s0[0]), (s0, s1)
    sim.close()


def test_rejections(tv):
    prof = couette_profile(32)
    s = tv.Simulation(32, 32, "D2Q16", storage="fp32_dev")  # periodic
    with pytest.raises(tv.TvlbmError) as e:
        s.set_reference_rows(*prof)
    assert e.value.code == tv.TVLBM_EINVAL
    s.close()
    s = tv.Simulation(32, 32, "D2Q16", walls=WALLS, storage="fp32")  # full-f storage
    with pytest.raises(tv.TvlbmError):
        s.set_reference_rows(*prof)
    s.close()
    s = tv.Simulation(32, 32, "D2Q16", walls=WALLS, storage="fp16_dev")
    bad = (prof[0], prof[1], np.where(np.arange(32) == 5, 0.0, prof[2]))
    with pytest.raises(tv.TvlbmError):
        s.set_reference_rows(*bad)  # T <= 0 in one row
    s.set_reference_rows(*prof)
    with pytest.raises(tv.TvlbmError):
        s.set_reference_refresh(-1)
    s.step(2)
    s.close()
    s = tv.Simulation(32, 32, "D2Q16", storage="fp16_dev")  # periodic
    with pytest.raises(tv.TvlbmError):
        s.set_reference_refresh(10)
    s.set_reference_refresh(0)  # off is always accepted
    with pytest.raises(tv.TvlbmError):
        tv.tvlbm_set_reference_kind(s.ctx, tv.REFERENCE_KINDS["mean"])  # periodic
    s.close()
    s = tv.Simulation(32, 32, "D2Q16", walls=WALLS, storage="bf16_dev")
    with pytest.raises(tv.TvlbmError) as e:
        tv.tvlbm_set_reference_kind(s.ctx, 7)
    assert e.value.code == tv.TVLBM_EINVAL
    s.close()


def test_mass_conserved_mean_reference(tv):
    """The mean-population reference carries each row's own density: refreshing it every 7 steps
    (FP32 deviations) keeps the channel's mass to FP32 rounding over 500 steps."""
    nx, ny = 64, 48
    sim = tv.Simulation(nx, ny, "D2Q36", tau=0.9, walls=WALLS, storage="fp32_dev", form="tiled")
    sim.init_moments(*perturbed_couette(nx, ny, 71))
    s0 = sim.conserved_sums()
    sim.set_reference_refresh(7, kind="mean")
    sim.step(500)
    s1 = sim.conserved_sums()
    assert abs(s1[0] - s0[0]) <= 1e-6 * abs(s0[0]), (s0, s1)
    sim.close()
