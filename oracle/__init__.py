"""FP64 CPU oracle of the TVLBM time step: plain, slow and written from the paper.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
(and its `--impl reference` arm) may import this package.  The CUDA library never imports,
loads or calls it, and it shares no code with the library: its velocity set comes from
Golub-Welsch (numpy eigensolver on the Jacobi matrix), its streaming table, equilibrium,
moments, BGK step and wall treatment are its own (tvlbm_oracle.c and the functions below).

Pins: every function here is checked in tests/test_oracle_*.py against facts the paper or
mathematics fix (quadrature exactness, Gaussian moments, Appendix A, conservation, exact
integer shifts, brute-force overlap areas, linear-theory decay rates, closed forms).
"""
from __future__ import annotations

import ctypes
import math
import os
from itertools import product

import numpy as np

from . import build as _build

_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_create.restype = _P
        lib.oracle_create.argtypes = [_I, _I, _I, _I, _DP, _DP, _DP, _IP, _IP, _DP, _DP, _D, _D, _I, _D, _D, _D, _D]
        lib.oracle_destroy.argtypes = [_P]
        lib.oracle_set_threads.argtypes = [_P, _I]
        lib.oracle_equilibrium.argtypes = [_P, _D, _D, _D, _D, _DP]
        lib.oracle_equilibrium_appendix_a.argtypes = [_P, _D, _D, _D, _D, _DP]
        lib.oracle_init.argtypes = [_P, _DP, _DP, _DP, _DP, _DP]
        lib.oracle_run.argtypes = [_P, _DP, _DP, _I]
        lib.oracle_stream.argtypes = [_P, _DP, _DP]
        lib.oracle_collide.argtypes = [_P, _DP, _DP]
        lib.oracle_moments.argtypes = [_P, _DP, _DP, _DP, _DP, _DP]
        lib.oracle_conserved_sums.argtypes = [_P, _DP, _DP]
        lib.oracle_ghosts.argtypes = [_P, _DP]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


# ----------------------------------------------------------------------------------------------
# Velocity sets (Sec. "The TVLBM model": velocities on the roots of Hermite polynomials)
# ----------------------------------------------------------------------------------------------

def gauss_hermite(n: int):
    """n-point Gauss quadrature for the standard normal weight exp(-x^2/2)/sqrt(2 pi)
    (probabilists' Hermite polynomials He_n), by Golub-Welsch: the nodes are the eigenvalues
    of the symmetric Jacobi matrix of the recurrence x He_k = He_{k+1} + k He_{k-1}
    (zero diagonal, off-diagonal sqrt(k)); each weight is the squared first component of the
    normalised eigenvector (the weight function has unit mass).  Returned sorted ascending."""
    J = np.zeros((n, n))
    for k in range(1, n):
        J[k, k - 1] = J[k - 1, k] = math.sqrt(k)
    vals, vecs = np.linalg.eigh(J)
    w = vecs[0, :] ** 2
    order = np.argsort(vals)
    x = vals[order]
    w = w[order]
    # the node set is symmetric about 0; symmetrise away eigensolver noise
    x = 0.5 * (x - x[::-1])
    w = 0.5 * (w + w[::-1])
    w = w / w.sum()
    return x, w


VELSETS = {"D2Q9": 3, "D2Q16": 4, "D2Q36": 6}


def velocity_set(name: str):
    """Tensor-product set: c_l = (x_i, x_j), w_l = w_i w_j, ordered l = i + n j (i along x).
    Hermite truncation order N = n - 1, the largest total degree whose equilibrium moments
    the n-point rule integrates exactly (2N <= 2n - 1)."""
    n = VELSETS[name]
    x, w1 = gauss_hermite(n)
    cx = np.array([x[i] for j in range(n) for i in range(n)])
    cy = np.array([x[j] for j in range(n) for i in range(n)])
    w = np.array([w1[i] * w1[j] for j in range(n) for i in range(n)])
    return dict(name=name, n=n, Q=n * n, N=n - 1, x=x, w1=w1, cx=cx, cy=cy, w=w)


def stream_table(c: np.ndarray, dt: float, dx: float = 1.0):
    """Shift of one velocity component over one step, in cells: s = c dt/dx = n + alpha with
    n = floor(s), 0 <= alpha < 1.  A shift within 1e-12 of an integer is taken as that integer
    (alpha = 0), so a space-filling velocity streams as an exact shift."""
    s = np.asarray(c, dtype=np.float64) * dt / dx
    r = np.round(s)
    snap = np.abs(s - r) < 1e-12
    n = np.where(snap, r, np.floor(s))
    a = np.where(snap, 0.0, s - n)
    return n.astype(np.int32), a


# ----------------------------------------------------------------------------------------------
# Pure-Python tensor equilibrium (small cases; the C core has its own copy of the same definition)
# ----------------------------------------------------------------------------------------------

def _pairings(idx, k):
    """All ways of choosing k disjoint pairs of positions of idx with equal entries; yields the
    tuple of unpaired entries (Grad notation: each pair is a Kronecker delta)."""
    n = len(idx)

    def rec(pos, used, left, singles):
        while pos < n and used[pos]:
            pos += 1
        if pos == n:
            if left == 0:
                yield tuple(singles)
            return
        used[pos] = True
        yield from rec(pos + 1, used, left, singles + [idx[pos]])
        if left > 0:
            for q in range(pos + 1, n):
                if not used[q] and idx[q] == idx[pos]:
                    used[q] = True
                    yield from rec(pos + 1, used, left - 1, singles)
                    used[q] = False
        used[pos] = False

    yield from rec(0, [False] * n, k, [])


def _grad(idx, k, v):
    return sum(math.prod(v[s] for s in singles) for singles in _pairings(idx, k))


def equilibrium_tensor(rho, ux, uy, T, cx, cy, w, N):
    """f_eq_l = w_l sum_{n<=N} (1/n!) a^(n)_0 : H^(n)(c_l) with a^(n) = rho sum_k (T-1)^k
    [delta^k u^(n-2k)] and H^(n) = sum_k (-1)^k [delta^k c^(n-2k)] (Sec. "The TVLBM model")."""
    u = (ux, uy)
    out = np.zeros(len(w))
    for l in range(len(w)):
        c = (cx[l], cy[l])
        s = 0.0
        for n in range(N + 1):
            sn = 0.0
            for idx in product(range(2), repeat=n):
                a = rho * sum((T - 1.0) ** k * _grad(idx, k, u) for k in range(n // 2 + 1))
                H = sum((-1.0) ** k * _grad(idx, k, c) for k in range(n // 2 + 1))
                sn += a * H
            s += sn / math.factorial(n)
        out[l] = w[l] * s
    return out


# ----------------------------------------------------------------------------------------------
# The oracle simulation (C core)
# ----------------------------------------------------------------------------------------------

class Oracle:
    """FP64 TVLBM on an nx-by-ny grid: periodic, or with diffuse walls at y = -1/2 and
    y = ny - 1/2 (walls=(u_lo, T_lo, u_hi, T_hi)).  State = post-collision populations
    f[Q][ny][nx]."""

    def __init__(self, nx, ny, velset="D2Q16", tau=0.8, dt=1.0, walls=None, threads=0):
        self.nx, self.ny = int(nx), int(ny)
        self.vs = velocity_set(velset) if isinstance(velset, str) else velset
        self.Q, self.N = self.vs["Q"], self.vs["N"]
        self.tau, self.dt = float(tau), float(dt)
        sx, ax = stream_table(self.vs["cx"], dt)
        sy, ay = stream_table(self.vs["cy"], dt)
        self.sx, self.sy, self.ax, self.ay = sx, sy, ax, ay
        wl = walls if walls is not None else (0.0, 1.0, 0.0, 1.0)
        lib = _load()
        self._keep = [np.ascontiguousarray(a) for a in (self.vs["cx"], self.vs["cy"], self.vs["w"], ax, ay)]
        self._ikeep = [np.ascontiguousarray(a, dtype=np.int32) for a in (sx, sy)]
        self._h = lib.oracle_create(self.nx, self.ny, self.Q, self.N,
                                    _dp(self._keep[0]), _dp(self._keep[1]), _dp(self._keep[2]),
                                    self._ikeep[0].ctypes.data_as(_IP), self._ikeep[1].ctypes.data_as(_IP),
                                    _dp(self._keep[3]), _dp(self._keep[4]), self.tau, self.dt,
                                    1 if walls is not None else 0, *[float(v) for v in wl])
        if not self._h:
            raise ValueError("oracle_create rejected the arguments")
        lib.oracle_set_threads(self._h, int(threads))
        self.f = np.zeros((self.Q, self.ny, self.nx))
        self._work = np.zeros_like(self.f)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_destroy(self._h)
            self._h = None

    def set_threads(self, threads: int):
        _load().oracle_set_threads(self._h, int(threads))

    def equilibrium(self, rho, ux, uy, T):
        out = np.zeros(self.Q)
        _load().oracle_equilibrium(self._h, rho, ux, uy, T, _dp(out))
        return out

    def equilibrium_appendix_a(self, rho, ux, uy, T):
        out = np.zeros(self.Q)
        _load().oracle_equilibrium_appendix_a(self._h, rho, ux, uy, T, _dp(out))
        return out

    def init_moments(self, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, T)]
        for a in arrs:
            assert a.shape == (self.ny, self.nx)
        _load().oracle_init(self._h, *[_dp(a) for a in arrs], _dp(self.f))

    def set_populations(self, f):
        self.f[...] = f

    def run(self, nsteps: int):
        _load().oracle_run(self._h, _dp(self.f), _dp(self._work), int(nsteps))

    def stream_only(self, f=None):
        fin = np.ascontiguousarray(self.f if f is None else f, dtype=np.float64)
        out = np.zeros_like(fin)
        _load().oracle_stream(self._h, _dp(fin), _dp(out))
        return out

    def collide_only(self, f=None):
        fin = np.ascontiguousarray(self.f if f is None else f, dtype=np.float64)
        out = np.zeros_like(fin)
        _load().oracle_collide(self._h, _dp(fin), _dp(out))
        return out

    def moments(self, f=None):
        fin = np.ascontiguousarray(self.f if f is None else f, dtype=np.float64)
        outs = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        _load().oracle_moments(self._h, _dp(fin), *[_dp(o) for o in outs])
        return tuple(outs)

    def conserved_sums(self, f=None):
        fin = np.ascontiguousarray(self.f if f is None else f, dtype=np.float64)
        out = np.zeros(4)
        _load().oracle_conserved_sums(self._h, _dp(fin), _dp(out))
        return out

    def ghosts(self):
        out = np.zeros((2, self.Q, self.nx))
        _load().oracle_ghosts(self._h, _dp(out))
        return out
