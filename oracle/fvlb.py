"""The paper's own evolution scheme: finite-volume update with the Prandtl-number term.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import
this module; the CUDA library shares no code with it.

Plain FP64 numpy, on a uniform periodic grid (Delta x = Delta y = 1), written from Sec. "The
TVLBM Evolution scheme" and Sec. "The TVLBM model":

* collision term (Eq. OMEGAFVLB): Omega_l = -(f_l - f_eq_l) / tau + (1 / tau_g) f_eq_l / (rho T^2)
  Pi : (c_l - u)(c_l - u), with Pi_ij = sum_l (f_l - f_eq_l)(c_l - u)_i (c_l - u)_j (the second
  term is left out when tau_g is infinite).  The second term carries no mass, momentum or
  energy for an exact Maxwellian; the truncated equilibrium of a finite velocity set leaves an
  O(u^2 Pi) energy residue, so the term is applied with its components along the collision
  invariants removed: its projection on the 12 non-conserved Hermite vectors (D2Q16), which
  keeps its traceless stress 2 Pi / tau_g;
* explicit Euler step of length dt (Eq. FVLB): f(t + dt) = f + dt (Omega_bar - c . grad f);
* the second-order stencils on the eight neighbours P1..P8 of P0 (P1 east, P2 north, P3 west,
  P4 south, P5 north-east, P6 north-west, P7 south-west, P8 south-east):
    d_x f ~ 3/8 (f1 - f3) + 1/16 (f5 - f6 - f7 + f8),
    d_y f ~ 3/8 (f2 - f4) + 1/16 (f5 + f6 - f7 - f8),
    Omega_bar ~ 9/16 Omega(0) + 3/32 (Omega(1) + .. + Omega(4)) + 1/64 (Omega(5) + .. + Omega(8)).
The equilibrium at each cell's own moments comes from the oracle's C core (its BGK collision
with dt / tau = 1 returns exactly f_eq).
"""
from __future__ import annotations

import numpy as np

from . import Oracle
from .closure import correction, project


def _at(a: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """Value at (x + dx, y + dy) of every cell of a [Q][ny][nx] (or [ny][nx]) periodic field."""
    return np.roll(a, shift=(-dy, -dx), axis=(-2, -1))


def grad_x(f: np.ndarray) -> np.ndarray:
    return 3.0 / 8.0 * (_at(f, 1, 0) - _at(f, -1, 0)) + 1.0 / 16.0 * (
        _at(f, 1, 1) - _at(f, -1, 1) - _at(f, -1, -1) + _at(f, 1, -1))


def grad_y(f: np.ndarray) -> np.ndarray:
    return 3.0 / 8.0 * (_at(f, 0, 1) - _at(f, 0, -1)) + 1.0 / 16.0 * (
        _at(f, 1, 1) + _at(f, -1, 1) - _at(f, -1, -1) - _at(f, 1, -1))


def average9(w: np.ndarray) -> np.ndarray:
    return (9.0 / 16.0 * w + 3.0 / 32.0 * (_at(w, 1, 0) + _at(w, 0, 1) + _at(w, -1, 0) + _at(w, 0, -1))
            + 1.0 / 64.0 * (_at(w, 1, 1) + _at(w, -1, 1) + _at(w, -1, -1) + _at(w, 1, -1)))


class FVLB:
    """FP64 finite-volume TVLBM on an nx x ny periodic grid; state f[Q][ny][nx]."""

    def __init__(self, nx, ny, velset="D2Q16", tau=0.5, tau_g=np.inf, dt=0.01):
        self.nx, self.ny = int(nx), int(ny)
        self.tau, self.tau_g, self.dt = float(tau), float(tau_g), float(dt)
        # the oracle's collision with dt / tau = 1 gives f_eq at each cell's moments
        self._eq = Oracle(nx, ny, velset, tau=1.0, dt=1.0)
        self.vs = self._eq.vs
        self.Q = self.vs["Q"]
        self.f = np.zeros((self.Q, self.ny, self.nx))

    def init_moments(self, rho, ux, uy, T):
        self._eq.init_moments(rho, ux, uy, T)
        self.f[...] = self._eq.f

    def equilibrium(self, f=None) -> np.ndarray:
        return self._eq.collide_only(self.f if f is None else f)

    def omega(self, f=None) -> np.ndarray:
        """Omega_l of every cell (Eq. OMEGAFVLB)."""
        f = self.f if f is None else f
        feq = self.equilibrium(f)
        om = -(f - feq) / self.tau
        if np.isfinite(self.tau_g):
            om += self.prandtl_term(f, feq)
        return om

    def prandtl_term(self, f, feq) -> np.ndarray:
        """(1 / tau_g) f_eq / (rho T^2) Pi : (c - u)(c - u)."""
        cx = self.vs["cx"].reshape(-1, 1, 1)
        cy = self.vs["cy"].reshape(-1, 1, 1)
        rho, ux, uy, T = self._eq.moments(f)
        dx, dy = cx - ux, cy - uy
        neq = f - feq
        pxx = (neq * dx * dx).sum(axis=0)
        pxy = (neq * dx * dy).sum(axis=0)
        pyy = (neq * dy * dy).sum(axis=0)
        contr = pxx * dx * dx + 2.0 * pxy * dx * dy + pyy * dy * dy
        raw = feq / (rho * T * T) * contr / self.tau_g
        return correction(project(raw, self.vs), self.vs)

    def step(self, n: int = 1):
        cx = self.vs["cx"].reshape(-1, 1, 1)
        cy = self.vs["cy"].reshape(-1, 1, 1)
        for _ in range(n):
            f = self.f
            self.f = f + self.dt * (average9(self.omega(f)) - cx * grad_x(f) - cy * grad_y(f))

    def moments(self, f=None):
        return self._eq.moments(self.f if f is None else f)

    def conserved_sums(self, f=None):
        return self._eq.conserved_sums(self.f if f is None else f)
