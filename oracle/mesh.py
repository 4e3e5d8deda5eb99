"""FP64 oracle of the volumetric (area-overlap) step on a mesh that is non-uniform in y.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import it.

The grid refinement of Sec. "Grid Refinement for simple unidirectional flows" (Eqs. NONUNI1-2:
cells crowded near the walls, e.g. a tanh stretching) taken to the volumetric scheme: cell y
is the interval [F_y, F_{y+1}] of height h_y (x stays uniform, dx = 1).  A population moves
rigidly by s = c dt in one step, so destination cell y pulls, per velocity,

    f_y  <-  sum_r  |[F_y - s, F_{y+1} - s]  intersected with cell r| / h_y  *  f_r        (1)

(the shifted destination interval, a union of pieces of source cells; with unit cells this is
the (1 - a, a) overlap of the uniform scheme).  The mass sum_y h_y f_y of each velocity is
unchanged on a periodic mesh.  With walls at F_0 and F_ny the part of the shifted interval
beyond a wall is filled from the wall: per column x the wall re-emits what the outgoing
velocities carry beyond it, M_out(x) = sum_l sum_r f~_l(x, r) |image of cell r beyond the wall|
(f~ the populations after the x part of the gather), as A(x) f_eq_l(1, u_w, T_w) for the
incoming velocities, A = M_out / sum_in |c_y dt| f_eq_l (Eq. IMPOSITION, the uniform scheme's
ghost-row rule, which is this rule on unit cells).  The collision is the pinned oracle's
(Oracle.collide_only); the step is stream (with the wall fill) then collide, so the state is
the post-collision populations, as in Oracle.

Pins (tests/test_oracle_mesh.py): unit cells reproduce Oracle (periodic and walls); dyadic
cells shifted by a whole period of their pattern move by whole rows (bit-exact roll); every
row's weights sum to one; the mass sum h_y f_y of each velocity is conserved (periodic), the
total mass with walls.
"""
from __future__ import annotations

import math

import numpy as np

from . import Oracle, stream_table


def y_overlaps(faces, s, periodic):
    """Gather weights of Eq. (1): for each destination row y a dict {source row: weight}.
    Periodic: the mesh repeats with period F_ny - F_0.  Walls: the part beyond the bottom wall is
    keyed -1, beyond the top wall ny."""
    F = np.asarray(faces, dtype=np.float64)
    ny = len(F) - 1
    h = np.diff(F)
    period = F[-1] - F[0]
    rows = []
    for y in range(ny):
        lo, hi = F[y] - s, F[y + 1] - s
        ent = {}
        if periodic:
            m0 = math.floor((lo - F[0]) / period) - 1
            m1 = math.floor((hi - F[0]) / period) + 1
            for m in range(m0, m1 + 1):
                for r in range(ny):
                    a = max(lo, F[r] + m * period)
                    b = min(hi, F[r + 1] + m * period)
                    if b > a:
                        ent[r] = ent.get(r, 0.0) + (b - a)
        else:
            for r in range(ny):
                a = max(lo, F[r])
                b = min(hi, F[r + 1])
                if b > a:
                    ent[r] = ent.get(r, 0.0) + (b - a)
            if lo < F[0]:
                ent[-1] = min(hi, F[0]) - lo
            if hi > F[-1]:
                ent[ny] = hi - max(lo, F[-1])
        rows.append({r: v / h[y] for r, v in ent.items()})
    return rows


def beyond_walls(faces, s):
    """Length of each fluid cell's image, moved by s, below the bottom wall (s < 0) or above the
    top wall (s > 0): array [ny]."""
    F = np.asarray(faces, dtype=np.float64)
    ny = len(F) - 1
    out = np.zeros(ny)
    for r in range(ny):
        lo, hi = F[r] + s, F[r + 1] + s
        if s < 0:
            out[r] = max(0.0, min(hi, F[0]) - lo)
        elif s > 0:
            out[r] = max(0.0, hi - max(lo, F[-1]))
    return out


class MeshOracle:
    """Volumetric TVLBM on nx uniform columns and the y cells of `faces` (ny + 1 increasing
    values): periodic in y, or walls=(u_lo, T_lo, u_hi, T_hi) at F_0 and F_ny."""

    def __init__(self, nx, faces, velset="D2Q16", tau=0.8, dt=1.0, walls=None):
        self.faces = np.asarray(faces, dtype=np.float64)
        self.nx, self.ny = int(nx), len(self.faces) - 1
        self.h = np.diff(self.faces)
        self.core = Oracle(self.nx, self.ny, velset, tau=tau, dt=dt)  # collision, equilibrium
        self.vs = self.core.vs
        self.Q, self.n1 = self.vs["Q"], int(round(math.sqrt(self.vs["Q"])))
        self.dt = float(dt)
        self.walls = walls
        xnodes = self.vs["cx"][: self.n1]  # l = i + n1 j: the first n1 entries run over i
        self.sx, self.ax = stream_table(xnodes, self.dt)
        self.sy = xnodes * self.dt  # y shift of node j (exact, not split into integer + fraction)
        periodic = walls is None
        self.tables = [y_overlaps(self.faces, self.sy[j], periodic) for j in range(self.n1)]
        self.beyond = [beyond_walls(self.faces, self.sy[j]) for j in range(self.n1)]
        if walls is not None:
            u_lo, T_lo, u_hi, T_hi = walls
            self.feq_w = [self.core.equilibrium(1.0, u_lo, 0.0, T_lo), self.core.equilibrium(1.0, u_hi, 0.0, T_hi)]
        self.f = np.zeros((self.Q, self.ny, self.nx))

    def init_moments(self, rho, ux, uy, T):
        self.core.init_moments(rho, ux, uy, T)
        self.f = self.core.f.copy()

    def _xgather(self, g, i):
        """x part of the gather for x-node i: g(x - s) with s = sx + ax (periodic columns)."""
        return (1.0 - self.ax[i]) * np.roll(g, self.sx[i], axis=-1) + self.ax[i] * np.roll(g, self.sx[i] + 1, axis=-1)

    def stream(self, f):
        n1, ny = self.n1, self.ny
        fx = np.empty_like(f)
        for l in range(self.Q):
            fx[l] = self._xgather(f[l], l % n1)
        ghost = {}
        if self.walls is not None:
            for side in (0, 1):
                out_l = [l for l in range(self.Q) if (self.sy[l // n1] < 0) == (side == 0) and self.sy[l // n1] != 0]
                in_l = [l for l in range(self.Q) if (self.sy[l // n1] > 0) == (side == 0) and self.sy[l // n1] != 0]
                m_out = np.zeros(self.nx)
                for l in out_l:
                    m_out += np.tensordot(self.beyond[l // n1], fx[l], axes=(0, 0))
                den = sum(abs(self.sy[l // n1]) * self.feq_w[side][l] for l in in_l)
                amp = m_out / den
                for l in in_l:  # the wall value after the x part of the gather
                    ghost[(side, l)] = self._xgather(amp * self.feq_w[side][l], l % n1)
        out = np.zeros_like(f)
        for l in range(self.Q):
            j = l // n1
            for y in range(ny):
                acc = np.zeros(self.nx)
                for r, w in self.tables[j][y].items():
                    if r < 0:
                        acc += w * ghost[(0, l)]
                    elif r >= ny:
                        acc += w * ghost[(1, l)]
                    else:
                        acc += w * fx[l, r]
                out[l, y] = acc
        return out

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            self.f = self.core.collide_only(self.stream(self.f))

    def moments(self):
        return self.core.moments(self.f)

    def mass(self, f=None):
        """sum_y h_y sum_l f (the conserved mass of the mesh)."""
        f = self.f if f is None else f
        return float(np.sum(f.sum(axis=0) * self.h[:, None]))

    def conserved_sums(self, f=None):
        """(M, P_x, P_y, E) weighted by the cell heights."""
        f = self.f if f is None else f
        cx, cy = self.vs["cx"], self.vs["cy"]
        hw = self.h[None, :, None]
        m = np.sum(f * hw)
        px = np.sum(cx[:, None, None] * f * hw)
        py = np.sum(cy[:, None, None] * f * hw)
        e = 0.5 * np.sum((cx * cx + cy * cy)[:, None, None] * f * hw)
        return np.array([m, px, py, e])
