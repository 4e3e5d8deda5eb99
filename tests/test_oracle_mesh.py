"""Pins of the non-uniform-mesh oracle (oracle/mesh.py) against facts that do not come from it:
unit cells are the uniform scheme (the pinned Oracle, periodic and with walls); dyadic cells
moved by a whole period of their pattern land on whole rows (an exact roll); every row's
weights sum to one and agree with a sampled measure of the shifted interval; the mass
sum_y h_y f_y of each velocity survives streaming on a periodic mesh, the total mass with
walls; the shifted slab reaches beyond a wall by exactly |s|."""
import numpy as np
import pytest

import workloads
from oracle import Oracle
from oracle.mesh import MeshOracle, beyond_walls, y_overlaps
from workloads import random_faces as _random_faces, tanh_faces

WALLS = (0.02, 1.0, -0.03, 1.05)


def unit_faces(ny):
    return np.arange(ny + 1, dtype=np.float64) - 0.5


def random_faces(ny, seed, lo=0.3, hi=1.7):
    return _random_faces(ny, seed, lo, hi)


@pytest.mark.parametrize("velset", ["D2Q9", "D2Q16", "D2Q36"])
@pytest.mark.parametrize("walls", [None, WALLS])
def test_unit_cells_are_the_uniform_scheme(velset, walls):
    nx, ny = 12, 10
    fields = workloads.random_smooth(nx, ny, seed=5, amp_u=0.05, amp_T=0.03)
    ref = Oracle(nx, ny, velset, tau=0.8, walls=walls)
    ref.init_moments(*fields)
    got = MeshOracle(nx, unit_faces(ny), velset, tau=0.8, walls=walls)
    got.init_moments(*fields)
    ref.run(6)
    got.step(6)
    assert np.max(np.abs(got.f - ref.f)) <= 1e-13 * np.max(np.abs(ref.f))


def test_dyadic_cells_move_by_whole_rows():
    # heights 0.25, 0.75 repeating: a shift by one pattern period (1.0) maps cell y onto cell y + 2
    ny = 8
    faces = np.concatenate([[0.0], np.cumsum(np.tile([0.25, 0.75], ny // 2))])
    for s, d in ((1.0, 2), (-1.0, -2), (2.0, 4)):
        tab = y_overlaps(faces, s, periodic=True)
        for y in range(ny):
            assert tab[y] == {(y - d) % ny: 1.0}
    f = np.random.default_rng(1).normal(size=ny)
    tab = y_overlaps(faces, 1.0, periodic=True)
    moved = np.array([sum(w * f[r] for r, w in tab[y].items()) for y in range(ny)])
    assert np.array_equal(moved, np.roll(f, 2))


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("s", [0.37, -0.81, 2.6, -3.3])
def test_weights_sum_to_one_and_match_sampling(periodic, s):
    faces = random_faces(14, seed=3)
    F = faces
    period = F[-1] - F[0]
    tab = y_overlaps(faces, s, periodic)
    rng = np.random.default_rng(11)
    for y, ent in enumerate(tab):
        assert abs(sum(ent.values()) - 1.0) <= 1e-14
        # sampled measure of the shifted destination interval in each source cell
        pts = rng.uniform(F[y] - s, F[y + 1] - s, 20000)
        if periodic:
            pts = F[0] + np.mod(pts - F[0], period)
            rows = np.searchsorted(F, pts, side="right") - 1
        else:
            rows = np.where(pts < F[0], -1, np.where(pts > F[-1], len(F) - 1, np.searchsorted(F, pts, side="right") - 1))
        for r, w in ent.items():
            assert abs(np.mean(rows == r) - w) < 0.02


def test_mass_of_each_velocity_survives_streaming():
    nx, ny = 6, 16
    faces = random_faces(ny, seed=7)
    m = MeshOracle(nx, faces, "D2Q16", dt=1.0)
    f = np.random.default_rng(2).uniform(0.5, 1.5, size=(m.Q, ny, nx))
    out = m.stream(f)
    h = np.diff(faces)[None, :, None]
    before = np.sum(f * h, axis=(1, 2))
    after = np.sum(out * h, axis=(1, 2))
    assert np.max(np.abs(after - before)) <= 1e-13 * np.max(before)
    # a state that is uniform in space stays uniform
    u = np.ones_like(f) * np.arange(1, m.Q + 1)[:, None, None]
    assert np.max(np.abs(m.stream(u) - u)) <= 1e-14 * m.Q


@pytest.mark.parametrize("velset", ["D2Q16", "D2Q36"])
def test_channel_conserves_total_mass(velset):
    nx, ny = 5, 20
    faces = tanh_faces(ny, 24.0, 1.8)
    m = MeshOracle(nx, faces, velset, tau=0.7, dt=0.5, walls=WALLS)
    m.init_moments(*workloads.random_smooth(nx, ny, seed=8, amp_u=0.04, amp_T=0.02))
    m0 = m.mass()
    for _ in range(10):
        m.step(1)
        assert abs(m.mass() - m0) <= 1e-13 * m0


def test_shifted_slab_reaches_beyond_a_wall_by_the_shift():
    faces = tanh_faces(18, 10.0, 2.0)
    for s in (-0.3, -2.2, 0.45, 3.1):
        assert abs(beyond_walls(faces, s).sum() - abs(s)) <= 1e-14 * 10
    # only the cells within the shift of the wall cross it
    b = beyond_walls(faces, -0.7)
    assert np.all(b[faces[:-1] >= faces[0] + 0.7] == 0.0)
    assert np.all(b[faces[:-1] < faces[0] + 0.7] > 0.0)


def test_tanh_faces_cover_the_channel_and_crowd_at_the_walls():
    F = tanh_faces(20, 6.0, 1.5)
    assert F[0] == 0.0 and abs(F[-1] - 6.0) < 1e-14
    h = np.diff(F)
    assert np.all(h > 0)
    assert h[0] < h[10] and h[-1] < h[10]
    assert np.allclose(h, h[::-1], rtol=0, atol=1e-14 * 6.0)
