"""Pins of the oracle's diffuse-reflection walls (Sec. 'Boundary Condition: Diffuse Scattering
Kernel', Eq. IMPOSITION: the re-emitted flux equals the flux hitting the wall, in the shape of
the wall equilibrium; Sec. 'Slip and Temperature Jump for Couette Flows', Eq. PRED)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


@pytest.mark.parametrize("name", ["D2Q16", "D2Q36"])
def test_gas_in_equilibrium_with_walls_is_a_fixed_point(name):
    """Gas at the walls' own (u_w, T_w): the outgoing and re-emitted fluxes match velocity by
    velocity, so the state must not change."""
    nx, ny = 3, 20
    uw, Tw = 0.05, 1.07
    o = oracle.Oracle(nx, ny, name, tau=0.9, walls=(uw, Tw, uw, Tw))
    one = np.ones((ny, nx))
    o.init_moments(one, uw * one, 0 * one, Tw * one)
    f0 = o.f.copy()
    o.run(5)
    np.testing.assert_allclose(o.f, f0, rtol=0, atol=5e-15)


@pytest.mark.parametrize("name", ["D2Q16", "D2Q36"])
def test_wall_mass_conservation(name):
    nx, ny = 5, 24
    o = oracle.Oracle(nx, ny, name, tau=0.9, walls=(0.0, 1.0, 0.1, 1.1))
    o.init_moments(*workloads.random_smooth(nx, ny, seed=4, amp_u=0.05, amp_T=0.05))
    m0 = o.conserved_sums()[0]
    o.run(300)
    m1 = o.conserved_sums()[0]
    assert abs(m1 - m0) < 1e-13 * m0


def test_zero_net_normal_flux_each_step():
    """The ghost rows re-emit exactly the mass the gather moves past the wall: with the wall
    at rest the y-momentum of a symmetric state stays zero."""
    nx, ny = 2, 24
    o = oracle.Oracle(nx, ny, "D2Q16", tau=0.9, walls=(0.0, 1.0, 0.0, 1.0))
    rho, ux, uy, T = workloads.couette_linear(nx, ny, 1.0, 1.0)
    T = T + 0.02 * np.cos(2 * math.pi * (np.arange(ny)[:, None] + 0.5) / ny)
    o.init_moments(rho, ux, uy, T)
    m0 = o.conserved_sums()[0]
    for _ in range(20):
        o.run(1)
        assert abs(o.conserved_sums()[0] - m0) < 1e-13


def _fit(y, v):
    A = np.vstack([np.ones_like(y), y]).T
    coef, *_ = np.linalg.lstsq(A, v, rcond=None)
    return coef, np.max(np.abs(A @ coef - v))


def test_isothermal_couette_linear_profile_with_bounded_slip():
    """Steady Couette flow: linear velocity in the bulk; the wall slip is of the order of the
    diffuse-reflection slip 1.43684 tau (Eq. PRED), far below one channel width."""
    nx, ny, tau, U = 1, 32, 0.9, 0.01
    o = oracle.Oracle(nx, ny, "D2Q16", tau=tau, walls=(0.0, 1.0, U, 1.0))
    o.init_moments(*workloads.couette_linear(nx, ny, 1.0, 1.0))
    o.run(12000)
    rho, ux, uy, T = (a[:, 0] for a in o.moments())
    y = np.arange(ny) + 0.5  # distance from the lower wall
    bulk = slice(6, ny - 6)
    (a, b), res = _fit(y[bulk], ux[bulk])
    assert res < 2e-4 * U
    slip_lo = a  # extrapolated gas velocity at the lower wall
    slip_hi = U - (a + b * ny)
    c = GOLD["slip_coefficient"]["value"]
    # slip length = slip / gradient, positive and of the order of c * tau (mean free path)
    for s in (slip_lo, slip_hi):
        L = s / b
        assert 0.2 * c * tau < L < 3.0 * c * tau, (L, c * tau)
    # the cell-centre y-momentum differs from the (zero) face flux only by the overlap gather's
    # diffusion of the population gradients: tiny against the wall speed
    assert np.max(np.abs(uy)) < 1e-4 * U


def test_thermal_couette_viscous_heating():
    """Thermal Couette with a moving wall (Sec. 'Avoiding temperature and velocity slip'): in the
    bulk T = a + b eta + (U_eff^2 / 4) eta (1 - eta)  (unit Prandtl number, c_P = 2 in D = 2, so
    mu/(2k) = 1/(2 c_P)), with U_eff the extrapolated velocity difference across the channel."""
    nx, ny, tau, U = 1, 32, 0.9, 0.2
    o = oracle.Oracle(nx, ny, "D2Q36", tau=tau, walls=(0.0, 1.0, U, 1.05))
    o.init_moments(*workloads.couette_linear(nx, ny, 1.0, 1.05))
    o.run(12000)
    rho, ux, uy, T = (a[:, 0] for a in o.moments())
    y = np.arange(ny) + 0.5
    bulk = slice(5, ny - 5)
    (a, b), _ = _fit(y[bulk], ux[bulk])
    U_eff = b * ny
    eta = y / ny
    A = np.vstack([np.ones_like(eta), eta, eta * (1 - eta)]).T[bulk]
    coef, *_ = np.linalg.lstsq(A, T[bulk], rcond=None)
    cP = GOLD["specific_heats_D2"]["c_P"]
    want = U_eff ** 2 / (2.0 * cP)
    assert abs(coef[2] - want) / want < 0.05, (coef[2], want)
    # pressure is uniform across the channel in the steady state
    p = rho * T
    assert np.max(np.abs(p[bulk] - p[bulk].mean())) < 1e-3 * p.mean()
