"""Linearised one-step operator of the TVLBM step about the rest state, assembled from first
principles for the oracle pins (independent of the oracle's code).

State = post-collision populations.  One step = volumetric gather, then BGK collision.
For a Fourier mode exp(i k y) the gather of velocity l multiplies by
    S_l(k) = (1 - alpha_l) exp(-i k n_l) + alpha_l exp(-i k (n_l + 1)),   s_l = c_l,y dt = n_l + alpha_l,
and the collision about rest (rho=1, u=0, T=1) is C = (1 - omega) I + omega J with
    J_lm = d f_eq_l / d f_m = w_l [1 + c_l.c_m + (|c_l|^2 - D)/2 (|c_m|^2/D - 1)]
(the first-order Hermite terms: d rho = sum df, d u = sum c df, d T = sum |c|^2 df / D - d rho).
One step is f -> C S f.
"""
import math

import numpy as np
from numpy.polynomial.hermite_e import hermegauss


def velocity_set(n):
    x, w = hermegauss(n)
    w = w / w.sum()
    cx = np.array([x[i] for j in range(n) for i in range(n)])
    cy = np.array([x[j] for j in range(n) for i in range(n)])
    W = np.array([w[i] * w[j] for j in range(n) for i in range(n)])
    return cx, cy, W, x, w


def step_matrix(n, tau, dt, k):
    cx, cy, W, _, _ = velocity_set(n)
    D = 2.0
    c2 = cx ** 2 + cy ** 2
    J = (np.outer(W, np.ones_like(W)) + np.outer(W * cx, cx) + np.outer(W * cy, cy)
         + np.outer(W * (c2 - D) / 2.0, c2 / D - 1.0))
    om = dt / tau
    C = (1.0 - om) * np.eye(len(W)) + om * J
    s = cy * dt
    nn = np.floor(s)
    a = s - nn
    S = (1.0 - a) * np.exp(-1j * k * nn) + a * np.exp(-1j * k * (nn + 1.0))
    return C @ np.diag(S), cx, cy, W


def modes(n, tau, dt, k):
    """Eigen-decomposition; returns (lam, vecs, cx, cy, W, shear_index, heat_index)."""
    M, cx, cy, W = step_matrix(n, tau, dt, k)
    lam, V = np.linalg.eig(M)
    # modes with k along y split by parity in c_x: the shear mode is odd in c_x
    mirror = np.array([np.argmin(np.abs(cx + cx[l]) + np.abs(cy - cy[l])) for l in range(len(cx))])
    odd = np.array([np.linalg.norm(V[:, m] + V[mirror, m]) < 1e-8 * np.linalg.norm(V[:, m]) for m in range(len(lam))])
    real = np.abs(np.angle(lam)) < 1e-9
    shear = max((m for m in range(len(lam)) if odd[m] and real[m]), key=lambda m: abs(lam[m]))
    heat = max((m for m in range(len(lam)) if (not odd[m]) and real[m]), key=lambda m: abs(lam[m]))
    return lam, V, cx, cy, W, shear, heat


def numerical_viscosity(n, dt=1.0):
    """Leading-order diffusion of the area-overlap gather: per axis the kernel has variance
    alpha(1-alpha), so nu_num = sum_b w_b alpha_b (1 - alpha_b) / 2 over the 1-D nodes."""
    _, _, _, x, w = velocity_set(n)
    s = x * dt
    a = s - np.floor(s)
    return float(np.sum(w * a * (1.0 - a) / 2.0))
