"""GPU parity of the volumetric step on a mesh non-uniform in y (tvlbm_set_y_faces) against the
FP64 oracle (oracle/mesh.py): populations element by element in FP64 storage, periodic and
with walls, every velocity set, ragged launch blocks; moments within 1e-5 in FP32-deviation
storage over 200 steps; unit cells equal the uniform scheme; the height-weighted sums conserved;
the calls the mesh refuses."""
import numpy as np
import pytest

import workloads
from oracle.mesh import MeshOracle
from workloads import random_faces, tanh_faces

pytestmark = pytest.mark.gpu

WALLS = (0.02, 1.0, -0.03, 1.05)


@pytest.fixture(scope="module")
def tv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    return tv


def pair(tv, nx, faces, velset, storage, walls, tau=0.7, dt=0.5, seed=3):
    ny = len(faces) - 1
    fields = workloads.random_smooth(nx, ny, seed=seed, amp_u=0.04, amp_T=0.03)
    sim = tv.Simulation(nx, ny, velset, tau=tau, dt=dt, storage=storage, walls=walls)
    sim.set_y_faces(faces)
    sim.init_moments(*fields)
    ref = MeshOracle(nx, faces, velset, tau=tau, dt=dt, walls=walls)
    ref.init_moments(*fields)
    return sim, ref


@pytest.mark.parametrize("velset", ["D2Q9", "D2Q16", "D2Q36"])
@pytest.mark.parametrize("walls", [None, WALLS])
def test_fp64_matches_oracle(tv, velset, walls):
    ny = 19
    faces = random_faces(ny, seed=4) if walls is None else tanh_faces(ny, 19.0, 1.6)
    sim, ref = pair(tv, 37, faces, velset, "fp64", walls)
    sim.step(12)
    ref.step(12)
    got = sim.populations_f64()
    assert np.max(np.abs(got - ref.f)) <= 1e-12 * np.max(np.abs(ref.f))
    sim.close()


def _pattern(heights, ny):
    return np.concatenate([[0.0], np.cumsum(np.resize(np.asarray(heights, dtype=np.float64), ny))])


# longest row lists of 2, 3, 4 entries (the unrolled gathers) and 5 and 8 (the general loop), by
# the mesh oracle's tables: near-unit cells, random cells, and a tall cell among shorter ones,
# periodic and with walls
@pytest.mark.parametrize("faces,walls", [
    (random_faces(21, 4, 0.9, 1.1), None),
    (random_faces(21, 4), WALLS),
    (_pattern([2.0, 0.5, 0.5, 0.5], 21), None),
    (_pattern([2.5, 0.3, 0.3, 0.3, 0.3], 21), WALLS),
    (_pattern([3.0, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25], 21), None)])
def test_every_row_length_matches_oracle(tv, faces, walls):
    sim, ref = pair(tv, 29, faces, "D2Q16", "fp64", walls, dt=1.0 if walls is None else 0.5)
    sim.step(10)
    ref.step(10)
    got = sim.populations_f64()
    assert np.max(np.abs(got - ref.f)) <= 1e-12 * np.max(np.abs(ref.f))
    sim.close()


def test_fp32_deviation_matches_oracle_over_200_steps(tv):
    faces = tanh_faces(24, 24.0, 1.8)
    sim, ref = pair(tv, 40, faces, "D2Q16", "fp32_dev", WALLS, seed=5)
    sim.step(200)
    ref.step(200)
    got, want = sim.moments(), ref.moments()
    for k, name in enumerate(("rho", "ux", "uy", "T")):
        if name in ("ux", "uy"):
            err = np.max(np.abs(got[1] - want[1]) + np.abs(got[2] - want[2])) / np.max(np.hypot(want[1], want[2]))
        else:
            err = np.max(np.abs(got[k] - want[k])) / np.max(np.abs(want[k]))
        assert err <= 1e-5, (name, err)
    sim.close()


@pytest.mark.parametrize("walls", [None, WALLS])
def test_unit_cells_equal_the_uniform_scheme(tv, walls):
    nx, ny = 33, 17
    fields = workloads.random_smooth(nx, ny, seed=6, amp_u=0.04, amp_T=0.03)
    out = []
    for faces in (np.arange(ny + 1, dtype=np.float64) - 0.5, None):
        sim = tv.Simulation(nx, ny, "D2Q16", tau=0.8, storage="fp64", walls=walls)
        if faces is not None:
            sim.set_y_faces(faces)
        else:
            sim.set_form("plain")
        sim.init_moments(*fields)
        sim.step(20)
        out.append(sim.populations_f64())
        sim.close()
    assert np.max(np.abs(out[0] - out[1])) <= 1e-13 * np.max(np.abs(out[1]))


def test_height_weighted_sums_are_conserved(tv):
    faces = tanh_faces(30, 30.0, 2.0)
    sim, ref = pair(tv, 24, faces, "D2Q16", "fp64", WALLS)
    s0 = sim.conserved_sums()
    assert abs(s0[0] - ref.mass()) <= 1e-12 * ref.mass()
    sim.step(100)
    s1 = sim.conserved_sums()
    assert abs(s1[0] - s0[0]) <= 1e-12 * abs(s0[0])
    # periodic: mass, momentum and energy
    sim2, ref2 = pair(tv, 24, random_faces(26, seed=9), "D2Q16", "fp64", None)
    a = sim2.conserved_sums()
    assert np.max(np.abs(a[:4] - ref2.conserved_sums())) <= 1e-12 * abs(a[0])
    sim2.step(100)
    b = sim2.conserved_sums()
    assert np.max(np.abs(b[:4] - a[:4])) <= 1e-12 * abs(a[0])
    sim.close()
    sim2.close()


def test_faces_none_returns_to_unit_cells(tv):
    nx, ny = 20, 14
    fields = workloads.random_smooth(nx, ny, seed=7)
    out = []
    for twice in (True, False):
        sim = tv.Simulation(nx, ny, "D2Q16", tau=0.8, storage="fp64")
        sim.set_form("plain")
        if twice:
            sim.set_y_faces(random_faces(ny, seed=1))
            sim.set_y_faces(None)
        sim.init_moments(*fields)
        sim.step(10)
        out.append(sim.populations_f64())
        sim.close()
    assert np.array_equal(out[0], out[1])


def test_refusals(tv):
    faces = np.arange(15, dtype=np.float64)
    s = tv.Simulation(16, 14, "D2Q16", storage="fp16_dev")
    with pytest.raises(tv.TvlbmError):
        s.set_y_faces(faces)  # half storage
    s.close()
    s = tv.Simulation(16, 14, "D2Q16", storage="fp64")
    bad = faces.copy()
    bad[5] = bad[4]
    with pytest.raises(tv.TvlbmError):
        s.set_y_faces(bad)  # not increasing
    bad[5] = np.nan
    with pytest.raises(tv.TvlbmError):
        s.set_y_faces(bad)
    s.set_y_faces(faces)
    with pytest.raises(tv.TvlbmError):
        s.set_form("tiled")  # the mesh runs the plain form only
    with pytest.raises(tv.TvlbmError):
        s.set_scheme("fvlb", 2.0)
    s.step(2)
    s.close()
    # one tall cell among 79 thin ones: its shifted interval would cover every thin cell
    s = tv.Simulation(16, 80, "D2Q16", storage="fp64")
    tall = np.concatenate([[0.0], np.cumsum(np.concatenate([np.full(79, 1e-3), [10.0]]))])
    with pytest.raises(tv.TvlbmError):
        s.set_y_faces(tall)
    s.close()
