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

    def __init__(self, nx, ny, velset="D2Q16", tau=0.5, tau_g=np.inf, dt=0.01, pressure_scaled=False):
        self.nx, self.ny = int(nx), int(ny)
        self.tau, self.tau_g, self.dt = float(tau), float(tau_g), float(dt)
        # tau -> tau / p and tau_g -> tau_g / p, p = rho T, for a viscosity and a conductivity
        # that do not vary with the local state (Sec. "Boundary Conditions: Avoiding temperature
        # and velocity slip")
        self.pressure_scaled = bool(pressure_scaled)
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
        p = 1.0
        if self.pressure_scaled:
            rho, _, _, T = self._eq.moments(f)
            p = rho * T
        om = -(f - feq) * p / self.tau
        if np.isfinite(self.tau_g):
            om += p * self.prandtl_term(f, feq)
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


# ----------------------------------------------------------------------------------------------
# Channel: wall nodes (Eq. FVLB2), diffuse-reflection imposition (Eq. IMPOSITION), the
# Newton-Raphson correction of the wall equilibrium (App. B), non-uniform node spacing in y
# (Eqs. NONUNI1-2)
# ----------------------------------------------------------------------------------------------

def tanh_nodes(ny: int, L: float, beta: float) -> np.ndarray:
    """Node positions y_j = L/2 (1 + tanh(beta phi_j) / tanh(beta)), phi_j = 1 - 2 (j-1)/(N-1),
    j = 1..N (Eq. NONUNI2), returned ascending."""
    j = np.arange(1, ny + 1)
    phi = 1.0 - 2.0 * (j - 1) / (ny - 1)
    return np.sort(0.5 * L * (1.0 + np.tanh(beta * phi) / np.tanh(beta)))


class FVLBChannel(FVLB):
    """Finite-volume TVLBM between two walls: periodic in x (spacing 1), node rows j = 0 .. ny-1
    at positions y[j], walls on the nodes j = 0 (normal +y) and j = ny - 1 (normal -y) with
    velocities u_lo, u_hi and temperatures T_lo, T_hi.  exact=False: the outgoing populations of
    a wall node are the diffuse-reflection Maxwellian at the wall's (u, T) (Eq. IMPOSITION);
    exact=True: at a wall equilibrium (u_eq, T_eq) found by Newton-Raphson (App. B) so that the
    wall node's velocity and temperature are the wall's."""

    def __init__(self, nx, ny, y, walls, velset="D2Q16", tau=0.5, tau_g=np.inf, dt=0.01, exact=False,
                 nr_iters=32, pressure_scaled=False):
        super().__init__(nx, ny, velset, tau=tau, tau_g=tau_g, dt=dt, pressure_scaled=pressure_scaled)
        self.y = np.asarray(y, dtype=np.float64)
        assert self.y.shape == (ny,) and np.all(np.diff(self.y) > 0)
        self.walls = [float(v) for v in walls]  # u_lo, T_lo, u_hi, T_hi
        self.exact, self.nr_iters = bool(exact), int(nr_iters)
        # per wall and column: the wall equilibrium (u_eq, T_eq) of the last imposition; the
        # paper's Newton-Raphson neglects the density's dependence on it (linear convergence)
        self.wall_eq = [[[self.walls[0], self.walls[1]] for _ in range(self.nx)],
                        [[self.walls[2], self.walls[3]] for _ in range(self.nx)]]

    # -- wall imposition --------------------------------------------------------------------
    def _feq1(self, u, T):
        """Equilibrium of unit density at velocity (u, 0) and temperature T."""
        return self._eq.equilibrium(1.0, u, 0.0, T)

    def impose(self):
        cx, cy = self.vs["cx"], self.vs["cy"]
        for side, j in ((0, 0), (1, self.ny - 1)):
            cn = cy if side == 0 else -cy  # c . n, n pointing into the fluid
            out = cn > 0
            uw, Tw = self.walls[2 * side], self.walls[2 * side + 1]
            for x in range(self.nx):
                f = self.f[:, j, x]
                incoming = np.sum(np.abs(cn[~out]) * f[~out])
                ue, Te = (uw, Tw) if not self.exact else self.wall_eq[side][x]
                for it in range(self.nr_iters + 1 if self.exact else 1):
                    feq = self._feq1(ue, Te)
                    S = np.sum(np.abs(cn[out]) * feq[out])
                    f[out] = incoming / S * feq[out]
                    if not self.exact or it == self.nr_iters:
                        break  # the last iterate's imposition stays
                    rho = f.sum()
                    F1 = rho * uw - np.sum(f * cx)
                    F2 = 2.0 * rho * Tw + rho * uw * uw - np.sum(f * (cx * cx + cy * cy))
                    # App. B: A, B, C, D from the derivatives of the wall equilibrium
                    h = 1e-6
                    du = (self._feq1(ue + h, Te) - self._feq1(ue - h, Te)) / (2 * h)
                    dT = (self._feq1(ue, Te + h) - self._feq1(ue, Te - h)) / (2 * h)
                    c2 = cx * cx + cy * cy
                    wn = np.abs(cn)

                    def coef(g, dfe):
                        return np.sum(g[out] * dfe[out]) - np.sum(wn[out] * dfe[out]) * np.sum(g[out] * feq[out]) / S
                    A, B = coef(cx, du), coef(cx, dT)
                    C, D = coef(c2, du), coef(c2, dT)
                    pref = S / ((A * D - B * C) * incoming)
                    ue += pref * (D * F1 - B * F2)
                    Te += pref * (-C * F1 + A * F2)
                if self.exact:
                    self.wall_eq[side][x] = [ue, Te]

    # -- the update ---------------------------------------------------------------------------
    def step(self, n: int = 1):
        cx = self.vs["cx"].reshape(-1, 1)
        cy = self.vs["cy"].reshape(-1, 1)
        dy = np.diff(self.y)
        ny = self.ny
        for _ in range(n):
            self.impose()
            f = self.f
            om = self.omega(f)
            new = f.copy()
            xs = lambda a, d: np.roll(a, -d, axis=-1)  # value at x + d
            for j in range(ny):
                if 0 < j < ny - 1:
                    fN, fS, fC = f[:, j + 1], f[:, j - 1], f[:, j]
                    gx = 3 / 8 * (xs(fC, 1) - xs(fC, -1)) + 1 / 16 * (xs(fN, 1) - xs(fN, -1) - xs(fS, -1) + xs(fS, 1))
                    gy = (3 / 8 * (fN - fS) + 1 / 16 * (xs(fN, 1) + xs(fN, -1) - xs(fS, -1) - xs(fS, 1))) * (
                        2.0 / (dy[j] + dy[j - 1]))
                    oN, oS, oC = om[:, j + 1], om[:, j - 1], om[:, j]
                    ob = (9 / 16 * oC + 3 / 32 * (xs(oC, 1) + oN + xs(oC, -1) + oS)
                          + 1 / 64 * (xs(oN, 1) + xs(oN, -1) + xs(oS, -1) + xs(oS, 1)))
                    new[:, j] = fC + self.dt * (ob - cx * gx - cy * gy)
                else:
                    bottom = j == 0
                    fC = f[:, j]
                    fI = f[:, 1] if bottom else f[:, ny - 2]  # the fluid-side neighbour row
                    dyw = dy[0] if bottom else dy[-1]
                    gx = 3 / 8 * (xs(fC, 1) - xs(fC, -1)) + 1 / 8 * (xs(fI, 1) - xs(fI, -1))
                    s = 1.0 if bottom else -1.0  # d_y f = s * (one-sided difference into the fluid)
                    gy = s * (2.0 / dyw) * (3 / 8 * (fI - fC) + 1 / 16 * (xs(fI, 1) + xs(fI, -1) - xs(fC, 1) - xs(fC, -1)))
                    oC, oI = om[:, j], om[:, 1] if bottom else om[:, ny - 2]
                    ob = (9 / 16 * oC + 3 / 32 * (xs(oC, 1) + xs(oC, -1)) + 3 / 16 * oI
                          + 1 / 32 * (xs(oI, 1) + xs(oI, -1)))
                    upd = fC + self.dt * (ob - cx * gx - cy * gy)
                    cn = (cy if bottom else -cy).ravel()
                    ingoing = cn <= 0
                    new[ingoing, j] = upd[ingoing]
            self.f = new

    def profile(self):
        """x-averaged (rho, u_x, u_y, T) per node row."""
        return tuple(a.mean(axis=1) for a in self.moments())
