"""Pins of the finite-volume channel oracle (oracle/fvlb.py: FVLBChannel): the tanh mesh against
the spacings the paper quotes (Sec. "Grid Refinement for simple unidirectional flows": beta =
2.3, 60 spacings over L = 10, from 0.016631 at the walls to 0.391 in the middle); a gas at rest
in equilibrium with both walls stays put; the Newton-Raphson imposition (App. B) makes the wall
nodes' velocity and temperature the walls'; the diffuse imposition balances the mass fluxes at
the wall (Eq. IMPOSITION); the isothermal Couette profile is linear on uniform and tanh meshes,
without slip in the exact mode and with slip in the diffuse one."""
import numpy as np
import pytest

import oracle
from oracle import fvlb


def test_tanh_mesh_matches_the_quoted_spacings():
    y = fvlb.tanh_nodes(61, 10.0, 2.3)
    d = np.diff(y)
    assert y[0] == 0.0 and abs(y[-1] - 10.0) < 1e-12
    assert 0 <= d.min() - 0.016631 < 1e-6  # quoted to six decimals (truncated)
    assert abs(d.max() - 0.391) < 2e-3
    assert np.allclose(d, d[::-1], rtol=1e-12)  # symmetric about the centre


def _channel(exact, y, walls, tau=0.5, dt=0.01, nx=2):
    ny = len(y)
    s = fvlb.FVLBChannel(nx, ny, y, walls, tau=tau, dt=dt, exact=exact)
    return s


def test_rest_state_with_matching_walls_is_a_fixed_point():
    y = np.linspace(0.0, 4.0, 9)
    s = _channel(False, y, (0.0, 1.0, 0.0, 1.0))
    ones = np.ones((9, 2))
    s.init_moments(ones, 0 * ones, 0 * ones, ones)
    f0 = s.f.copy()
    s.step(20)
    assert np.max(np.abs(s.f - f0)) < 1e-14


def test_newton_raphson_sets_the_wall_velocity_and_temperature():
    y = np.linspace(0.0, 4.0, 9)
    s = _channel(True, y, (0.05, 1.02, -0.03, 0.97))
    ny, nx = 9, 2
    yy = np.linspace(0, 1, ny).reshape(-1, 1) * np.ones((1, nx))
    s.init_moments(np.ones((ny, nx)), 0.02 * np.sin(3 * yy), 0 * yy, 1.0 + 0.01 * yy)
    s.step(3)
    s.impose()
    rho, ux, uy, T = s.moments()
    # the paper's Newton-Raphson neglects the wall density's dependence on the corrections, so it
    # converges linearly (ratio ~ 0.6): 32 iterations per imposition reach ~1e-12
    assert np.max(np.abs(ux[0] - 0.05)) < 1e-10 and np.max(np.abs(T[0] - 1.02)) < 1e-10
    assert np.max(np.abs(ux[-1] + 0.03)) < 1e-10 and np.max(np.abs(T[-1] - 0.97)) < 1e-10


def test_diffuse_imposition_balances_the_wall_mass_flux():
    y = np.linspace(0.0, 4.0, 9)
    s = _channel(False, y, (0.05, 1.0, 0.0, 1.1))
    ny, nx = 9, 2
    yy = np.linspace(0, 1, ny).reshape(-1, 1) * np.ones((1, nx))
    s.init_moments(np.ones((ny, nx)), 0.02 * yy, 0 * yy, 1.0 + 0.05 * yy)
    s.step(2)
    s.impose()
    cy = s.vs["cy"]
    for j in (0, ny - 1):
        flux = np.sum(s.f[:, j, :] * cy.reshape(-1, 1), axis=0)  # normal mass flux of the wall node
        assert np.max(np.abs(flux)) < 1e-15


@pytest.mark.slow
@pytest.mark.parametrize("mesh", ["uniform", "tanh"])
def test_isothermal_couette_profile_without_slip(mesh):
    """Steady isothermal Couette flow (walls at -U and +U, started from the linear profile, 1000
    steps of dt = 0.02 ~ 3 viscous times of the 6-unit gap): the exact-mode wall nodes move with
    the walls and the interior profile is linear with nearly the full shear (a kinetic layer one
    node wide takes ~3 % of the velocity jump at tau = 0.5); the diffuse mode slips (~14 %) and
    shears the bulk less."""
    ny, L, U = 13, 6.0, 0.05
    y = np.linspace(0.0, L, ny) if mesh == "uniform" else fvlb.tanh_nodes(ny, L, 1.5)
    nx = 2
    prof = (-U + 2 * U * y / L).reshape(-1, 1) * np.ones((1, nx))
    ones = np.ones((ny, nx))
    res = {}
    for exact in (True, False):
        s = _channel(exact, y, (-U, 1.0, U, 1.0), tau=0.5, dt=0.02)
        s.init_moments(ones, prof, 0 * ones, ones)
        s.step(1000)
        rho, ux, uy, T = s.profile()
        inner = slice(2, ny - 2)
        c = np.polyfit(y[inner], ux[inner], 1)
        res[exact] = dict(wall=ux[0] / -U, fit=np.max(np.abs(np.polyval(c, y[inner]) - ux[inner])) / U,
                          slope=c[0] / (2 * U / L), centre=abs(ux[ny // 2]) / U)
    ex, di = res[True], res[False]
    assert abs(ex["wall"] - 1) < 1e-7 and ex["fit"] < 1e-2 and ex["slope"] > 0.95 and ex["centre"] < 1e-10, ex
    assert di["wall"] < 0.95 and di["slope"] < 0.9 and di["centre"] < 1e-10, di
