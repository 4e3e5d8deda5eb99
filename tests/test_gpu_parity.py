"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element,
on the same seeded inputs.  Tolerances: FP64 storage 1e-11 (rounding order only), FP32
storage 1e-5 and half-deviation storage 1e-3 (max relative error of rho, u, T, each measured
against the field's own max |value|)."""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FORMS = ["plain", "tiled"]


@pytest.fixture(scope="module")
def tv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    return tv


def forms_for(tv, storage):
    out = ["plain"]
    sim = tv.Simulation(8, 9, "D2Q16", storage=storage)
    try:
        sim.set_form("tiled")
        out.append("tiled")
    except tv.TvlbmError:
        pass
    sim.close()
    return out


def rel_err(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


def field_errors(got, want):
    """(rho, u, T) errors; u combines both components against max |u_ref|."""
    e_rho = rel_err(got[0], want[0])
    umax = max(np.max(np.abs(want[1])), np.max(np.abs(want[2])), 1e-300)
    e_u = max(np.max(np.abs(got[1] - want[1])), np.max(np.abs(got[2] - want[2]))) / umax
    e_T = rel_err(got[3], want[3])
    return e_rho, float(e_u), e_T


def run_pair(tv, nx, ny, velset, tau, dt, walls, storage, fields, steps, form="plain", graphs=True):
    sim = tv.Simulation(nx, ny, velset, tau=tau, dt=dt, walls=walls, storage=storage, form=form, graphs=graphs)
    sim.init_moments(*fields)
    sim.step(steps)
    ref = oracle.Oracle(nx, ny, velset, tau=tau, dt=dt, walls=walls)
    ref.init_moments(*fields)
    ref.run(steps)
    return sim, ref


# ---------------------------------------------------------------------------------------------
# FP64 storage: element-wise population parity (differences are rounding order only)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("form", FORMS)
def test_c0_shear_wave_fp64(tv, form):
    """64x64 periodic D2Q16, FP64, tau=0.8, dt=1, u_x = 0.01 sin(2 pi y/64), 200 steps."""
    if form not in forms_for(tv, "fp64"):
        pytest.skip("form not built for this storage")
    fields = workloads.shear_wave(64, 64, eps=0.01)
    sim, ref = run_pair(tv, 64, 64, "D2Q16", 0.8, 1.0, None, "fp64", fields, 200, form=form)
    f = sim.populations_f64()
    assert rel_err(f, ref.f) < 1e-11
    for e in field_errors(sim.moments(), ref.moments()):
        assert e < 1e-11


@pytest.mark.parametrize("velset,nx,ny", [("D2Q16", 37, 29), ("D2Q36", 45, 23), ("D2Q9", 33, 35),
                                          ("D2Q16", 1, 12), ("D2Q16", 2, 3), ("D2Q36", 3, 5)])
@pytest.mark.parametrize("form", FORMS)
def test_periodic_ragged_fp64(tv, velset, nx, ny, form):
    if form not in forms_for(tv, "fp64"):
        pytest.skip("form not built for this storage")
    fields = workloads.random_smooth(nx, ny, seed=nx * 100 + ny, amp_u=0.08, amp_T=0.08)
    sim, ref = run_pair(tv, nx, ny, velset, 0.75, 1.0, None, "fp64", fields, 30, form=form)
    assert rel_err(sim.populations_f64(), ref.f) < 1e-11


@pytest.mark.parametrize("velset", ["D2Q16", "D2Q36"])
@pytest.mark.parametrize("form", FORMS)
def test_walls_fp64(tv, velset, form):
    if form not in forms_for(tv, "fp64"):
        pytest.skip("form not built for this storage")
    nx, ny = 29, 21
    walls = (0.0, 1.0, 0.1, 1.1)
    fields = workloads.random_smooth(nx, ny, seed=17, amp_u=0.05, amp_T=0.05)
    sim, ref = run_pair(tv, nx, ny, velset, 0.9, 1.0, walls, "fp64", fields, 40, form=form)
    assert rel_err(sim.populations_f64(), ref.f) < 1e-11


@pytest.mark.parametrize("dt", [0.37, 1.2])
def test_other_time_steps_fp64(tv, dt):
    fields = workloads.random_smooth(20, 18, seed=2)
    sim, ref = run_pair(tv, 20, 18, "D2Q16", 0.9, dt, None, "fp64", fields, 25)
    assert rel_err(sim.populations_f64(), ref.f) < 1e-11


# ---------------------------------------------------------------------------------------------
# Exact integer shift: D2Q9 with dt = 1/sqrt(3) streams as an exact lattice shift; with
# tau = inf (no collision) the stored populations must be np.roll of the initial ones, bit for bit.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp32_dev", "bf16_dev", "fp16_dev"])
@pytest.mark.parametrize("walls", [False, True])
def test_integer_shift_bit_exact(tv, storage, walls):
    nx, ny = 19, 13
    wl = (0.0, 1.0, 0.0, 1.0) if walls else None
    sim = tv.Simulation(nx, ny, "D2Q9", tau=math.inf, dt=1.0 / math.sqrt(3.0), walls=wl, storage=storage)
    sim.init_moments(*workloads.random_smooth(nx, ny, seed=4, amp_u=0.2, amp_T=0.2))
    f0 = sim.raw_populations()
    steps = 3
    sim.step(steps)
    f1 = sim.raw_populations()
    sx, sy, ax, ay = tv.tvlbm_stream_table(9, 1.0 / math.sqrt(3.0))
    assert np.all(ax == 0) and np.all(ay == 0)
    for l in range(9):
        want = np.roll(f0[l], shift=(steps * int(sy[l]), steps * int(sx[l])), axis=(0, 1))
        if walls:
            # rows fed from beyond a wall are not a roll; compare the rows that stayed inside
            k = steps * abs(int(sy[l]))
            rows = slice(k, ny) if sy[l] > 0 else slice(0, ny - k)
            assert np.array_equal(f1[l][rows].view(np.uint8), want[rows].view(np.uint8)), l
        else:
            assert np.array_equal(f1[l].view(np.uint8), want.view(np.uint8)), l


# ---------------------------------------------------------------------------------------------
# FP32 and half-deviation storage against the FP64 oracle
# ---------------------------------------------------------------------------------------------

# FP32 storage, both forms, bar 1e-5: scaled deviations (fp32_dev, the shipped form) and raw f
# (fp32, the plain form), whose arithmetic splits the rest populations off exactly so that only
# the store rounds relative to f.
FP32_BOUND = {"fp32_dev": 1e-5, "fp32": 1e-5}


@pytest.mark.parametrize("storage", ["fp32", "fp32_dev"])
@pytest.mark.parametrize("form", FORMS)
def test_c1_recipe_reduced_fp32(tv, storage, form):
    """The 1024^2 recipe (T bump, random Fourier flow, tau=0.7) at 256^2 with sigma scaled
    to 16 cells, 300 steps."""
    if form not in forms_for(tv, storage):
        pytest.skip("form not built for this storage")
    n = 256
    fields = workloads.gaussian_bump_random_flow(n, n, seed=1, sigma=16.0)
    sim, ref = run_pair(tv, n, n, "D2Q16", 0.7, 1.0, None, storage, fields, 300, form=form)
    errs = field_errors(sim.moments(), ref.moments())
    print("C1 recipe 256^2 300 steps", storage, form, "errors (rho, u, T):", errs)
    assert max(errs) < FP32_BOUND[storage], errs


# Half-deviation storage after 1000 steps with ONE reference, the flow's mean state.  FP16
# (11-bit significand) meets the 1e-3 bar on the 96 x 64 walls case (measured 6.9e-4).  These are
# not the half-storage parity claims on the channel workload -- those take a per-row reference
# (tests/test_gpu_reference_rows.py, bar 1e-3 for both FP16 and BF16) -- but regression checks of
# the single-reference encoding at its measured levels with margin: on the 4096 x 512 channel FP16
# reaches 1.4e-3, and BF16 (8-bit significand) rounds 8x coarser than FP16 (1.6e-2 measured).
HALF_BOUND = {"fp16_dev": 1e-3, "bf16_dev": 3e-2}
HALF_BOUND_C2 = {"fp16_dev": 2e-3, "bf16_dev": 3e-2}


@pytest.mark.parametrize("storage", ["bf16_dev", "fp16_dev"])
@pytest.mark.parametrize("form", FORMS)
def test_half_storage_walls_d2q36(tv, storage, form):
    """Thermal Couette start (walls T = 1.0 / 1.1, top wall u = 0.1, tau = 0.9), D2Q36,
    with an x-varying perturbation, 96 x 64, 1000 steps."""
    if form not in forms_for(tv, storage):
        pytest.skip("form not built for this storage")
    nx, ny = 96, 64
    walls = (0.0, 1.0, 0.1, 1.1)
    rho, ux, uy, T = workloads.couette_linear(nx, ny, 1.0, 1.1)
    pert = workloads.random_smooth(nx, ny, seed=8, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    fields = (rho * pert[0], ux + pert[1], uy + pert[2], T * pert[3])
    sim = tv.Simulation(nx, ny, "D2Q36", tau=0.9, walls=walls, storage=storage, form=form)
    sim.set_reference(0.05, 0.0, 1.05)  # the channel's mean state
    sim.init_moments(*fields)
    sim.step(1000)
    ref = oracle.Oracle(nx, ny, "D2Q36", tau=0.9, walls=walls)
    ref.init_moments(*fields)
    ref.run(1000)
    errs = field_errors(sim.moments(), ref.moments())
    print("half storage walls 96x64 1000 steps", storage, form, "errors (rho, u, T):", errs)
    assert max(errs) < HALF_BOUND[storage], errs


@pytest.mark.parametrize("storage", ["bf16_dev", "fp16_dev"])
def test_c2_single_reference_regression(tv, storage):
    """4096 x 512 D2Q36 channel (walls T = 1.0 / 1.1, top wall u = 0.1, tau = 0.9), half
    storage against one mean-state reference, 1000 steps (a regression check, see HALF_BOUND).
    The flow is x-invariant, so the oracle runs an 8 x 512 periodic strip and every GPU column
    must match it."""
    nx, ny, steps = 4096, 512, 1000
    walls = (0.0, 1.0, 0.1, 1.1)
    sim = tv.Simulation(nx, ny, "D2Q36", tau=0.9, walls=walls, storage=storage)
    sim.set_reference(0.05, 0.0, 1.05)
    sim.init_moments(*workloads.couette_linear(nx, ny, 1.0, 1.1))
    sim.step(steps)
    got = sim.moments()
    ref = oracle.Oracle(8, ny, "D2Q36", tau=0.9, walls=walls)
    ref.init_moments(*workloads.couette_linear(8, ny, 1.0, 1.1))
    ref.run(steps)
    want = [np.broadcast_to(a[:, :1], (ny, nx)) for a in ref.moments()]
    errs = field_errors(got, want)
    print("C2 4096x512 1000 steps", storage, "errors (rho, u, T):", errs)
    assert max(errs) < HALF_BOUND_C2[storage], errs
    m = sim.conserved_sums()
    assert m[4] == 0


@pytest.mark.slow
@pytest.mark.parametrize("storage,form", [("fp32_dev", "tiled"), ("fp32", "plain")])
def test_c1_full_size_fp32(tv, storage, form):
    """1024 x 1024 periodic D2Q16, FP32 populations, tau = 0.7, T = 1 + 0.05 Gaussian bump
    (sigma = 64 cells), random Fourier flow (|k| <= 8, amplitude 0.02), 1000 steps, against the
    FP64 oracle: max relative rho/u/T error <= 1e-5 (shipped form) and conservation."""
    if form not in forms_for(tv, storage):
        pytest.skip("form not built for this storage")
    n, steps = 1024, 1000
    fields = workloads.gaussian_bump_random_flow(n, n, seed=1)
    sim = tv.Simulation(n, n, "D2Q16", tau=0.7, storage=storage, form=form)
    sim.init_moments(*fields)
    s0 = sim.conserved_sums()
    sim.step(steps)
    s1 = sim.conserved_sums()
    got = sim.moments()
    ref = _c1_reference(fields, steps)
    errs = field_errors(got, ref)
    drift = (s1[:4] - s0[:4]) / s0[0]
    print("C1 1024^2 1000 steps", storage, form, "errors (rho, u, T):", errs, "drift (M, Px, Py, E)/M:", drift)
    assert max(errs) < FP32_BOUND[storage], errs
    assert np.all(np.abs(drift) < 1e-7), drift


_C1_REF = {}


def _c1_reference(fields, steps):
    if steps not in _C1_REF:
        ref = oracle.Oracle(1024, 1024, "D2Q16", tau=0.7)
        ref.init_moments(*fields)
        ref.run(steps)
        _C1_REF[steps] = ref.moments()
    return _C1_REF[steps]


# ---------------------------------------------------------------------------------------------
# Diagnostics, checkpoint, graphs
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("storage,tol", [("fp64", 1e-13), ("fp32", 1e-7), ("fp32_dev", 2e-8), ("fp16_dev", 1e-5)])
def test_conservation_on_gpu(tv, storage, tol):
    n = 96
    sim = tv.Simulation(n, n, "D2Q16", tau=0.7, storage=storage)
    sim.init_moments(*workloads.random_smooth(n, n, seed=6, amp_u=0.1, amp_T=0.1))
    s0 = sim.conserved_sums()
    sim.step(500)
    s1 = sim.conserved_sums()
    scale = s0[0]
    print("conservation 96^2 500 steps", storage, "drift/M:", (s1[:4] - s0[:4]) / scale)
    assert np.all(np.abs(s1[:4] - s0[:4]) <= tol * scale), (s1 - s0)
    assert s1[4] == 0


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16_dev"])
def test_diagnostics_match_oracle_on_same_state(tv, storage):
    nx, ny = 23, 17
    ref = oracle.Oracle(nx, ny, "D2Q36")
    ref.init_moments(*workloads.random_smooth(nx, ny, seed=3))
    ref.run(5)
    sim = tv.Simulation(nx, ny, "D2Q36", storage=storage)
    sim.set_populations_f64(ref.f)
    tol = {"fp64": 1e-14, "fp32": 1e-6, "bf16_dev": 5e-3}[storage]
    f = sim.populations_f64()
    assert rel_err(f, ref.f) < tol
    errs = field_errors(sim.moments(), ref.moments(f))  # moments of the stored state, both sides
    assert max(errs) < 1e-12, errs
    s = sim.conserved_sums()
    np.testing.assert_allclose(s[:4], ref.conserved_sums(f), rtol=0, atol=1e-12 * abs(s[0]))


@pytest.mark.parametrize("storage", ["fp32_dev", "fp16_dev"])
def test_reference_is_a_reencoding(tv, storage):
    """Setting the deviation reference re-expresses the state: moments unchanged to the storage
    precision, and runs with either reference agree."""
    nx, ny = 48, 40
    fields = workloads.random_smooth(nx, ny, seed=31, amp_u=0.05, amp_T=0.05)
    a = tv.Simulation(nx, ny, "D2Q16", storage=storage)
    a.init_moments(*fields)
    a.step(20)
    m0 = a.moments()
    a.set_reference(0.03, -0.02, 1.04)  # re-encodes the current state
    m1 = a.moments()
    tol = {"fp32_dev": 2e-6, "fp16_dev": 2e-3}[storage]
    assert max(field_errors(m1, m0)) < tol
    b = tv.Simulation(nx, ny, "D2Q16", storage=storage)
    b.set_reference(0.03, -0.02, 1.04)
    b.init_moments(*fields)
    b.step(20)
    a.step(30)
    b.step(30)
    assert max(field_errors(a.moments(), b.moments())) < tol


def test_reference_rejected_for_full_storage(tv):
    sim = tv.Simulation(8, 8, "D2Q16", storage="fp32")
    with pytest.raises(tv.TvlbmError) as e:
        sim.set_reference(0.1, 0.0, 1.0)
    assert e.value.code == tv.TVLBM_EINVAL


def test_checkpoint_resume_bit_identical(tv):
    nx, ny = 50, 40
    fields = workloads.random_smooth(nx, ny, seed=12)
    a = tv.Simulation(nx, ny, "D2Q16", storage="bf16_dev")
    a.init_moments(*fields)
    a.step(10)
    b = tv.Simulation(nx, ny, "D2Q16", storage="bf16_dev")
    b.init_moments(*fields)
    b.step(4)
    snap = b.raw_populations()
    c = tv.Simulation(nx, ny, "D2Q16", storage="bf16_dev")
    c.set_raw_populations(snap)
    c.step(6)
    assert np.array_equal(a.raw_populations(), c.raw_populations())


@pytest.mark.parametrize("storage", ["fp32", "fp16_dev"])
def test_graphs_equal_direct_launches(tv, storage):
    nx, ny = 64, 48
    fields = workloads.random_smooth(nx, ny, seed=13)
    a = tv.Simulation(nx, ny, "D2Q16", storage=storage, graphs=True)
    b = tv.Simulation(nx, ny, "D2Q16", storage=storage, graphs=False)
    for s in (a, b):
        s.init_moments(*fields)
        s.step(70)
        s.step(33)
    assert np.array_equal(a.raw_populations(), b.raw_populations())


def test_init_rejects_nonpositive_fields(tv):
    sim = tv.Simulation(8, 8, "D2Q16")
    rho, ux, uy, T = workloads.random_smooth(8, 8, seed=1)
    T = T.copy()
    T[3, 3] = -1.0
    with pytest.raises(tv.TvlbmError) as e:
        sim.init_moments(rho, ux, uy, T)
    assert e.value.code == tv.TVLBM_EINVAL


def test_create_in_rejects_small_memory(tv):
    import torch
    need = tv.tvlbm_memory_bytes(32, 32, 16, None, tv.TVLBM_FP32)
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(tv.TvlbmError) as e:
        tv.tvlbm_create_in(32, 32, 16, 0.8, 1.0, None, tv.TVLBM_FP32, 1.0, buf.data_ptr(), need - 256)
    assert e.value.code == tv.TVLBM_ENOMEM
