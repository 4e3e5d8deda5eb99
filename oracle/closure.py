"""Learned coarse-grid closure: the plain FP64 definitions the GPU path is checked against.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import
this module; the CUDA library shares no code with it.

The paper has no learned part: this is the extension the method is carried to (a coarse D2Q16
run whose collision is corrected by a small network), and each function below is the plain
definition written out, numpy in FP64:

* nonconserved_basis -- the D2Q16 Hermite tensor basis He_a(c_x) He_b(c_y) / sqrt(a! b!)
  (a, b <= 3; probabilists' Hermite polynomials, the velocity nodes of Sec. "The TVLBM model")
  with the collision invariants 1, c_x, c_y, |c|^2 taken out: 12 vectors psi_k, orthonormal in
  the quadrature inner product <g, h> = sum_l w_l g_l h_l and orthogonal to the invariants.
* correction(o) -- Delta f_l = w_l sum_k o_k psi_k(c_l): it adds no mass, momentum or energy.
* project(R) -- o_k = sum_l R_l psi_k(c_l): the o whose correction is closest to a population
  residual R in the metric sum_l R_l^2 / w_l.
* block_average -- a coarse cell's populations are the mean over the m x m fine cells it covers.
* cell_features -- (rho, u_x, u_y, T, Pi^neq_xy, Pi^neq_xx - Pi^neq_yy) of every cell, from
  the moment definitions of Sec. "The TVLBM model" (D = 2).
* neighbourhood -- the normalised features of the 3 x 3 periodic neighbourhood, 54 per cell.
* MLP 54 -> 128 -> 128 -> 12 with the exact GELU z Phi(z); forward, mean squared loss and its
  gradient by the chain rule.
* noneq_coefficients -- n_k = sum_l (f - f_eq)_l psi_k(c_l), f_eq at each cell's own moments:
  the non-equilibrium part of a state in the basis.
* closure_step -- one learned coarse step: stream, then every cell becomes f_eq(rho, u, T)
  + w sum_k o_k psi_k with the network's o computed from the streamed state (the conserved
  moments come from the streaming, the non-conserved ones from the network).
* bf16_round -- round to the nearest bfloat16 (ties to even), the encoding the GPU network's
  operands use.
"""
from __future__ import annotations

import math

import numpy as np

from . import velocity_set

N_IN, N_HID, N_OUT = 54, 128, 12
N_FEAT = 6


# ----------------------------------------------------------------------------------------------
# Hermite basis of the non-conserved moments (D2Q16)
# ----------------------------------------------------------------------------------------------

def hermite_e(n: int, x: np.ndarray) -> np.ndarray:
    """Probabilists' Hermite polynomial He_n(x): He_0 = 1, He_1 = x, He_{k+1} = x He_k - k He_{k-1}."""
    h0, h1 = np.ones_like(x), np.asarray(x, dtype=np.float64)
    if n == 0:
        return h0
    for k in range(1, n):
        h0, h1 = h1, x * h1 - k * h0
    return h1


# (a, b) pairs of the basis, in the fixed order the library uses too (see the header).  The
# first vector is the normal-stress difference, built from (2, 0) and (0, 2).
BASIS_ORDER = [("diff", None), (1, 1), (3, 0), (2, 1), (1, 2), (0, 3), (3, 1), (2, 2), (1, 3), (3, 2), (2, 3), (3, 3)]


def nonconserved_basis(vs=None) -> np.ndarray:
    """psi[k][l], k < 12, l < 16 (l = i + 4 j)."""
    vs = vs or velocity_set("D2Q16")
    assert vs["Q"] == 16
    cx, cy = vs["cx"], vs["cy"]
    psi = np.zeros((12, 16))
    for k, (a, b) in enumerate(BASIS_ORDER):
        if a == "diff":
            psi[k] = (hermite_e(2, cx) - hermite_e(2, cy)) / 2.0  # norm^2 = (2 + 2) / 4
        else:
            psi[k] = hermite_e(a, cx) * hermite_e(b, cy) / math.sqrt(math.factorial(a) * math.factorial(b))
    return psi


def correction(o: np.ndarray, vs=None) -> np.ndarray:
    """o[..., 12] -> Delta f[16, ...]: w_l sum_k o_k psi_k(c_l)."""
    vs = vs or velocity_set("D2Q16")
    psi = nonconserved_basis(vs)
    d = np.tensordot(o, psi, axes=([-1], [0]))  # [..., 16]
    return np.moveaxis(d, -1, 0) * vs["w"].reshape((16,) + (1,) * (d.ndim - 1))


def project(R: np.ndarray, vs=None) -> np.ndarray:
    """R[16, ...] -> o[..., 12]: o_k = sum_l R_l psi_k(c_l)."""
    psi = nonconserved_basis(vs)
    return np.moveaxis(np.tensordot(psi, R, axes=([1], [0])), 0, -1)


# ----------------------------------------------------------------------------------------------
# Coarse graining and per-cell features
# ----------------------------------------------------------------------------------------------

def block_average(f: np.ndarray, m: int) -> np.ndarray:
    """f[Q, ny, nx] -> [Q, ny/m, nx/m]: mean over each m x m block of cells."""
    Q, ny, nx = f.shape
    assert ny % m == 0 and nx % m == 0
    return f.reshape(Q, ny // m, m, nx // m, m).mean(axis=(2, 4))


def cell_features(f: np.ndarray, vs=None) -> np.ndarray:
    """f[16, ny, nx] -> [6, ny, nx]: rho, u_x, u_y, T, Pi^neq_xy, Pi^neq_xx - Pi^neq_yy, with
    rho = sum f, rho u = sum f c, rho (|u|^2 + 2 T) = sum f |c|^2 and Pi^neq = sum f c c - rho u u."""
    vs = vs or velocity_set("D2Q16")
    cx = vs["cx"].reshape(-1, 1, 1)
    cy = vs["cy"].reshape(-1, 1, 1)
    rho = f.sum(axis=0)
    ux = (f * cx).sum(axis=0) / rho
    uy = (f * cy).sum(axis=0) / rho
    e2 = (f * (cx * cx + cy * cy)).sum(axis=0)
    T = 0.5 * (e2 / rho - (ux * ux + uy * uy))
    pxy = (f * cx * cy).sum(axis=0) - rho * ux * uy
    nd = (f * (cx * cx - cy * cy)).sum(axis=0) - rho * (ux * ux - uy * uy)
    return np.stack([rho, ux, uy, T, pxy, nd])


def neighbourhood(feat: np.ndarray, mu=None, inv_sigma=None) -> np.ndarray:
    """feat[6, ny, nx] -> X[ny * nx, 54] (row = y * nx + x): entry ((dy + 1) * 3 + dx + 1) * 6 + q
    holds feature q of cell (x + dx, y + dy), periodic, normalised as (value - mu_q) * inv_sigma_q."""
    F, ny, nx = feat.shape
    mu = np.zeros(F) if mu is None else np.asarray(mu, dtype=np.float64)
    inv_sigma = np.ones(F) if inv_sigma is None else np.asarray(inv_sigma, dtype=np.float64)
    norm = (feat - mu.reshape(-1, 1, 1)) * inv_sigma.reshape(-1, 1, 1)
    X = np.zeros((ny, nx, 9 * F))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            # value at (x + dx, y + dy): roll the field by (-dy, -dx)
            shifted = np.roll(norm, shift=(-dy, -dx), axis=(1, 2))
            k = (dy + 1) * 3 + (dx + 1)
            X[:, :, k * F:(k + 1) * F] = np.moveaxis(shifted, 0, -1)
    return X.reshape(ny * nx, 9 * F)


# ----------------------------------------------------------------------------------------------
# The network
# ----------------------------------------------------------------------------------------------

def gelu(z):
    """Exact GELU: z Phi(z), Phi the standard normal CDF."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


_erf = np.vectorize(math.erf, otypes=[np.float64])


PARAM_SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
                ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
PARAM_COUNT = sum(int(np.prod(s)) for _, s in PARAM_SHAPES)


def unpack(theta: np.ndarray) -> dict:
    """Flat parameter vector (W1, b1, W2, b2, W3, b3; matrices row-major, [out][in]) -> dict."""
    out, k = {}, 0
    for name, shape in PARAM_SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    assert k == theta.size
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in PARAM_SHAPES])


def forward(p: dict, X: np.ndarray):
    """Y = W3 g(W2 g(W1 x + b1) + b2) + b3 for every row x of X; returns Y and the intermediates."""
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = gelu(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (Z1, H1, Z2, H2)


def loss(Y: np.ndarray, Ystar: np.ndarray) -> float:
    """Mean over rows and outputs of (Y - Y*)^2."""
    return float(np.mean((Y - Ystar) ** 2))


def loss_and_grad(p: dict, X: np.ndarray, Ystar: np.ndarray):
    """The loss and its gradient with respect to every parameter (chain rule, layer by layer)."""
    Y, (Z1, H1, Z2, H2) = forward(p, X)
    M = X.shape[0]
    dY = 2.0 * (Y - Ystar) / (M * Y.shape[1])
    g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
    dZ2 = (dY @ p["W3"]) * gelu_grad(Z2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_grad(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return loss(Y, Ystar), g


def init_params(seed: int, scale: float = 1.0) -> dict:
    """Seeded random parameters (uniform, fan-in scaled), for tests."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in PARAM_SHAPES:
        fan_in = shape[-1] if len(shape) == 2 else N_HID
        p[name] = rng.uniform(-1.0, 1.0, size=shape) * scale / math.sqrt(fan_in)
    return p


# ----------------------------------------------------------------------------------------------
# bfloat16 encoding
# ----------------------------------------------------------------------------------------------

def bf16_round(a) -> np.ndarray:
    """Nearest bfloat16 value (ties to even) of each element, returned as float64.  The value is
    first rounded to binary32 (as the GPU path holds it), then its low 16 bits are rounded off."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(x)
    out[nan] = np.nan
    return out.reshape(np.shape(a))


# ----------------------------------------------------------------------------------------------
# One learned coarse step
# ----------------------------------------------------------------------------------------------

def equilibrium_field(oracle, f: np.ndarray) -> np.ndarray:
    """f_eq(rho, u, T) of every cell, at the cell's own moments (the oracle's equilibrium)."""
    rho, ux, uy, T = oracle.moments(f)
    out = np.empty_like(f)
    for y in range(f.shape[1]):
        for x in range(f.shape[2]):
            out[:, y, x] = oracle.equilibrium(rho[y, x], ux[y, x], uy[y, x], T[y, x])
    return out


def noneq_coefficients(oracle, f=None) -> np.ndarray:
    """n[ny * nx, 12]: projection of f - f_eq(moments of f) on the basis."""
    f = oracle.f if f is None else f
    return project(f - equilibrium_field(oracle, f), oracle.vs).reshape(-1, N_OUT)


def closure_coefficients(oracle, p: dict, mu, inv_sigma, out_scale, f=None, bf16=False) -> np.ndarray:
    """o[ny * nx, 12] = out_scale * MLP(normalised 3 x 3 features of the stored state f).
    With bf16, the network's inputs and hidden activations are rounded to BF16 where a BF16
    network stores them (everything else in FP64), so that a BF16 implementation can be held
    to the rounding of its accumulations rather than to that of its storage."""
    f = oracle.f if f is None else f
    X = neighbourhood(cell_features(f, oracle.vs), mu, inv_sigma)
    if bf16:
        X = bf16_round(X)
        H1 = bf16_round(gelu(X @ p["W1"].T + p["b1"]))
        H2 = bf16_round(gelu(H1 @ p["W2"].T + p["b2"]))
        Y = H2 @ p["W3"].T + p["b3"]
    else:
        Y, _ = forward(p, X)
    return Y * np.asarray(out_scale, dtype=np.float64)


def closure_step(oracle, p: dict, mu, inv_sigma, out_scale, bf16=False) -> np.ndarray:
    """Advance oracle.f by one learned coarse step: stream; the coefficients come from the
    streamed state; each cell becomes f_eq(its moments) + the correction.  Returns the
    coefficients used.  bf16: as closure_coefficients."""
    streamed = oracle.stream_only()
    o = closure_coefficients(oracle, p, mu, inv_sigma, out_scale, f=streamed, bf16=bf16)
    nxt = equilibrium_field(oracle, streamed) + correction(o.reshape(oracle.ny, oracle.nx, N_OUT), oracle.vs)
    oracle.f[...] = nxt
    return o
