"""The learned closure's training targets (paper_1004_5059_gb300.closure.TargetSolver) against a
dense solve in real space built only from the oracle.

TargetSolver works per wavevector: the conserved moments that streaming gives the basis
corrections w psi_k form a 4 x active matrix K(k) (the gather's Fourier symbol, from the stream
table), and the target is o(k) = K^H (K K^H + lambda s I)^-1 r(k), s = mean tr(K K^H) / 4.
Here the same map is assembled column by column in real space -- the oracle's correction
w sum_k o_k psi_k of a unit coefficient in one cell, the oracle's pull-gather streaming of it,
then its conserved moments (mass, momentum, energy) per cell -- and the regularised
minimum-norm solution o = L^T (L L^T + lambda s I)^-1 r, s = tr(L L^T) / (4 N), is solved
densely.  The two must agree to rounding: any slip in the solver's shifts, overlap fractions,
basis or moment weights changes L's Fourier blocks and fails here.  No GPU: the solver only
reads the library's host-side velocity set and stream table.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closure as ocl


def _dense_map(n, active):
    """L[4 N][active N]: coefficient o_k at cell c -> conserved moments of the streamed
    correction, cells row-major (c = y n + x), moments (mass, P_x, P_y, E = sum |c|^2 f / 2)."""
    vs = oracle.velocity_set("D2Q16")
    o_ = oracle.Oracle(n, n, "D2Q16", tau=math.inf)
    phi = np.stack([np.ones(16), vs["cx"], vs["cy"], 0.5 * (vs["cx"] ** 2 + vs["cy"] ** 2)])
    N = n * n
    L = np.zeros((4 * N, active * N))
    for k in range(active):
        for c in range(N):
            o = np.zeros((n, n, 12))
            o[c // n, c % n, k] = 1.0
            g = o_.stream_only(ocl.correction(o, vs))
            L[:, k * N + c] = np.tensordot(phi, g, axes=([1], [0])).reshape(-1)
    return L


@pytest.mark.parametrize("active", [2, 6])
def test_targets_equal_dense_regularised_solve(active):
    from paper_1004_5059_gb300 import closure as C
    n, lam = 12, 1e-2
    solver = C.TargetSolver(n, lam, active)
    L = _dense_map(n, active)
    N = n * n
    s = np.trace(L @ L.T) / (4 * N)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((4, n, n)) * np.array([1e-3, 2e-3, 2e-3, 3e-3])[:, None, None]
    rv = r.reshape(-1)
    want = L.T @ np.linalg.solve(L @ L.T + lam * s * np.eye(4 * N), rv)
    got = solver.solve(r)
    assert got.shape == (12, n, n)
    assert np.all(got[active:] == 0.0)
    got_v = got[:active].reshape(-1)
    assert np.max(np.abs(got_v - want)) <= 1e-10 * np.max(np.abs(want))
    # the oracle's step with the solver's correction leaves the regularised residual
    resid = rv - L @ got_v
    assert np.max(np.abs(resid - lam * s * np.linalg.solve(L @ L.T + lam * s * np.eye(4 * N), rv))) <= \
        1e-10 * np.max(np.abs(rv))


def test_unregularised_target_reproduces_the_mismatch():
    """With lambda -> 0 and all 12 vectors active the conserved mismatch of a smooth field is
    reproduced exactly by the streamed correction (K has full row rank away from k = 0, where
    streaming conserves everything and only a zero mismatch is reachable)."""
    from paper_1004_5059_gb300 import closure as C
    n = 12
    solver = C.TargetSolver(n, 1e-12, 12)
    L = _dense_map(n, 12)
    y, x = np.mgrid[0:n, 0:n]
    r = np.stack([np.sin(2 * np.pi * (x + 2 * y) / n) * a for a in (1e-3, 2e-3, -1e-3, 5e-4)])
    o = solver.solve(r)
    back = (L @ o.reshape(-1)).reshape(4, n, n)
    assert np.max(np.abs(back - r)) <= 1e-8 * np.max(np.abs(r))
