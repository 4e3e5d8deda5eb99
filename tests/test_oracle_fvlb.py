"""Pins of the finite-volume oracle (oracle/fvlb.py, Sec. "The TVLBM Evolution scheme") against
what the mathematics fixes: the stencils are exact on quadratics and the collision average
keeps constants; the update conserves mass, momentum and energy on a periodic grid; the Prandtl
term adds no mass, momentum or energy and changes the stress by 2 Pi / tau_g; shear waves then
decay with nu = T tau tau_g / (tau_g - 2 tau) while heat modes do not feel tau_g."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import fvlb


def test_stencils_exact_on_quadratics():
    ny, nx = 24, 24
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    for a, b, c, d in [(0.3, -0.2, 0.0, 0.0), (0.0, 0.0, 0.05, -0.03)]:
        f = a * xx + b * yy + c * xx * xx + d * yy * yy + 0.01 * xx * yy
        gx, gy = fvlb.grad_x(f), fvlb.grad_y(f)
        inner = (slice(2, -2), slice(2, -2))
        assert np.allclose(gx[inner], (a + 2 * c * xx + 0.01 * yy)[inner], atol=1e-12)
        assert np.allclose(gy[inner], (b + 2 * d * yy + 0.01 * xx)[inner], atol=1e-12)
    assert np.allclose(fvlb.average9(np.full((5, 7), 3.5)), 3.5, atol=1e-15)
    lin = 0.2 * xx + 0.1 * yy
    assert np.allclose(fvlb.average9(lin)[2:-2, 2:-2], lin[2:-2, 2:-2], atol=1e-12)


@pytest.mark.parametrize("tau_g", [np.inf, 2.0, -1.0])
def test_update_conserves(tau_g):
    nx = ny = 12
    s = fvlb.FVLB(nx, ny, tau=0.5, tau_g=tau_g, dt=0.02)
    s.init_moments(*workloads.random_smooth(nx, ny, seed=14, amp_u=0.05, amp_T=0.03))
    s.step(5)  # develop a non-equilibrium part
    s0 = s.conserved_sums()
    s.step(20)
    s1 = s.conserved_sums()
    assert np.max(np.abs(s1 - s0)) < 1e-12 * abs(s0[0])


def test_prandtl_term_moments():
    """At rest, on a perturbed state: the term has zero mass, momentum and energy and its second
    central moment is 2 Pi / tau_g (there the raw formula needs no projection: checked too)."""
    nx, ny = 4, 3
    s = fvlb.FVLB(nx, ny, tau=0.5, tau_g=1.7)
    rng = np.random.default_rng(15)
    s.init_moments(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), np.ones((ny, nx)))
    vs = s.vs
    from oracle import closure as cl
    psi = cl.nonconserved_basis(vs)
    # a non-equilibrium part along the stress vectors only (u, rho, T unchanged)
    a = rng.normal(size=(ny, nx, 2)) * 1e-3
    f = s.f + cl.correction(np.concatenate([a, np.zeros((ny, nx, 10))], axis=-1), vs)
    feq = s.equilibrium(f)
    term = s.prandtl_term(f, feq)
    cx = vs["cx"].reshape(-1, 1, 1)
    cy = vs["cy"].reshape(-1, 1, 1)
    for m in (np.ones_like(cx), cx, cy, cx * cx + cy * cy):
        assert np.max(np.abs((term * m).sum(axis=0))) < 1e-15
    neq = f - feq
    pxy = (neq * cx * cy).sum(axis=0)
    pd = (neq * (cx * cx - cy * cy)).sum(axis=0)
    assert np.allclose((term * cx * cy).sum(axis=0), 2 * pxy / 1.7, atol=1e-16)
    assert np.allclose((term * (cx * cx - cy * cy)).sum(axis=0), 2 * pd / 1.7, atol=1e-16)
    rho, ux, uy, T = s.moments(f)
    raw = feq / (rho * T * T) * ((neq * cx * cx).sum(0) * cx * cx + 2 * pxy * cx * cy
                                 + (neq * cy * cy).sum(0) * cy * cy) / 1.7
    assert np.max(np.abs(raw - term)) < 1e-11 * np.max(np.abs(raw))


def test_prandtl_term_energy_residue_is_removed_away_from_rest():
    """With u != 0 the raw formula's energy moment is not zero on D2Q16; the applied term's is."""
    nx, ny = 6, 5
    s = fvlb.FVLB(nx, ny, tau=0.5, tau_g=1.3, dt=0.02)
    s.init_moments(*workloads.random_smooth(nx, ny, seed=16, amp_u=0.2, amp_T=0.05))
    s.step(3)
    f = s.f
    feq = s.equilibrium(f)
    term = s.prandtl_term(f, feq)
    cx = s.vs["cx"].reshape(-1, 1, 1)
    cy = s.vs["cy"].reshape(-1, 1, 1)
    for m in (np.ones_like(cx), cx, cy, cx * cx + cy * cy):
        assert np.max(np.abs((term * m).sum(axis=0))) < 1e-16


def _decay_rate(s, field, k, y, t0_steps, t1_steps):
    """Rate of the sin(k y) amplitude of a moment field between two times."""
    s.step(t0_steps)
    a0 = np.mean(field(s) * np.sin(k * y))
    s.step(t1_steps - t0_steps)
    a1 = np.mean(field(s) * np.sin(k * y))
    return math.log(a0 / a1) / ((t1_steps - t0_steps) * s.dt)


def _shear(tau_g):
    ny, nx = 32, 2
    s = fvlb.FVLB(nx, ny, tau=0.5, tau_g=tau_g, dt=0.02)
    s.init_moments(*workloads.shear_wave(nx, ny, eps=0.01))
    k = 2 * math.pi / ny
    y = np.arange(ny, dtype=float).reshape(-1, 1) * np.ones((1, nx))
    return _decay_rate(s, lambda q: q.moments()[1], k, y, 250, 1000)


def _heat(tau_g):
    ny, nx = 64, 2
    s = fvlb.FVLB(nx, ny, tau=0.5, tau_g=tau_g, dt=0.02)
    rho, ux, uy, T = workloads.heat_mode(nx, ny, eps=0.01)
    s.init_moments(rho, ux, uy, T)
    k = 2 * math.pi / ny
    y = np.arange(ny, dtype=float).reshape(-1, 1) * np.ones((1, nx))
    return _decay_rate(s, lambda q: q.moments()[3] - 1.0, k, y, 250, 1000)


@pytest.mark.slow
def test_prandtl_term_scales_viscosity_not_conduction():
    tau = 0.5
    base = _shear(np.inf)
    k = 2 * math.pi / 32
    # BGK: nu = T tau (no numerical diffusion in the finite-volume update), within 2 %
    assert abs(base / (tau * k * k) - 1) < 0.02
    for tau_g in (4 * tau, -2 * tau):
        ratio = _shear(tau_g) / base
        assert abs(ratio / (tau_g / (tau_g - 2 * tau)) - 1) < 0.03, (tau_g, ratio)
    # heat modes: tau_g moves the rate only through the O(k^4) coupling of the thermal mode to the
    # viscous stress (k = 2 pi / 64 here).  (Their absolute rate is not T tau k^2 on D2Q16: its
    # third-order equilibrium lacks the fourth moments the heat-flux relaxation needs.)
    h0 = _heat(np.inf)
    for tau_g in (4 * tau, -2 * tau):
        assert abs(_heat(tau_g) / h0 - 1) < 0.02, (tau_g, _heat(tau_g) / h0)
