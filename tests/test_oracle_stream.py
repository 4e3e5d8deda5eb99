"""Pins of the oracle's volumetric streaming (each population moves by c dt and is shared among
the cells its shifted cell volume overlaps; the Introduction's volumetric, conservative form)."""
import math

import numpy as np
import pytest

import oracle


def overlap_1d(lo_a, hi_a, lo_b, hi_b):
    return max(0.0, min(hi_a, hi_b) - max(lo_a, lo_b))


def brute_force_stream(f, cx, cy, dt, nx, ny):
    """Explicit area overlap of every shifted source square with every destination square,
    summed over periodic images; no floor/alpha bookkeeping."""
    Q = f.shape[0]
    out = np.zeros_like(f)
    for l in range(Q):
        sx, sy = cx[l] * dt, cy[l] * dt
        for j in range(ny):
            for i in range(nx):
                for b in range(ny):
                    ly = sum(overlap_1d(j + sy - 0.5, j + sy + 0.5, b + k * ny - 0.5, b + k * ny + 0.5)
                             for k in range(-4, 5))
                    if ly == 0.0:
                        continue
                    for a in range(nx):
                        lx = sum(overlap_1d(i + sx - 0.5, i + sx + 0.5, a + k * nx - 0.5, a + k * nx + 0.5)
                                 for k in range(-4, 5))
                        out[l, b, a] += lx * ly * f[l, j, i]
    return out


@pytest.mark.parametrize("name,dt", [("D2Q16", 1.0), ("D2Q16", 0.37), ("D2Q36", 1.0), ("D2Q9", 0.8)])
def test_stream_equals_brute_force_overlap(name, dt):
    nx, ny = 5, 3
    o = oracle.Oracle(nx, ny, name, tau=0.8, dt=dt)
    rng = np.random.default_rng(11)
    f = rng.uniform(0.0, 1.0, size=(o.Q, ny, nx))
    got = o.stream_only(f)
    want = brute_force_stream(f, o.vs["cx"], o.vs["cy"], dt, nx, ny)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_integer_shift_is_exact_roll():
    """D2Q9 nodes are 0 and +-sqrt(3); with dt = 1/sqrt(3) every shift is an integer and the
    volumetric streaming must be the exact lattice shift, bit for bit."""
    nx, ny = 13, 9
    o = oracle.Oracle(nx, ny, "D2Q9", tau=0.8, dt=1.0 / math.sqrt(3.0))
    assert np.all(o.ax == 0.0) and np.all(o.ay == 0.0)
    rng = np.random.default_rng(3)
    f = rng.uniform(0.0, 1.0, size=(o.Q, ny, nx))
    got = o.stream_only(f)
    for l in range(o.Q):
        want = np.roll(f[l], shift=(int(o.sy[l]), int(o.sx[l])), axis=(0, 1))
        assert np.array_equal(got[l], want), l


@pytest.mark.parametrize("name", ["D2Q16", "D2Q36"])
def test_stream_conserves_each_population(name):
    nx, ny = 17, 11
    o = oracle.Oracle(nx, ny, name)
    rng = np.random.default_rng(5)
    f = rng.uniform(0.0, 1.0, size=(o.Q, ny, nx))
    got = o.stream_only(f)
    np.testing.assert_allclose(got.sum(axis=(1, 2)), f.sum(axis=(1, 2)), rtol=1e-14)


def test_stream_moves_mass_centre_by_c_dt():
    """The centre of mass of a population moves by exactly c dt (overlap weights have mean s)."""
    nx, ny = 40, 40
    o = oracle.Oracle(nx, ny, "D2Q16", dt=1.0)
    f = np.zeros((o.Q, ny, nx))
    f[:, 20, 20] = 1.0
    g = o.stream_only(f)
    ys, xs = np.mgrid[0:ny, 0:nx]
    for l in range(o.Q):
        mx = np.sum(xs * g[l]) - 20.0
        my = np.sum(ys * g[l]) - 20.0
        assert abs(mx - o.vs["cx"][l]) < 1e-13 and abs(my - o.vs["cy"][l]) < 1e-13
