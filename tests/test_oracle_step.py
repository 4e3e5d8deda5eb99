"""Pins of the oracle's full time step: conservation (Abstract, Introduction, Conclusions: exact
conservation of density, momentum and energy), linear theory and the decay closed forms of the
transport-coefficient experiments (Sec. 'Measuring the transport coefficients')."""
import math

import numpy as np
import pytest

import oracle
import workloads
from linear_theory import modes, numerical_viscosity


@pytest.mark.parametrize("name,tau", [("D2Q16", 0.8), ("D2Q36", 0.9)])
def test_conservation_over_steps(name, tau):
    nx, ny = 24, 20
    o = oracle.Oracle(nx, ny, name, tau=tau)
    o.init_moments(*workloads.random_smooth(nx, ny, seed=7, amp_u=0.08, amp_T=0.08))
    s0 = o.conserved_sums()
    for _ in range(4):
        o.run(50)
        s = o.conserved_sums()
        scale = s0[0]
        assert np.all(np.abs(s - s0) <= 1e-13 * scale), (s - s0)


@pytest.mark.parametrize("name", ["D2Q16", "D2Q36"])
def test_collision_conserves_per_cell_and_rest_is_fixed(name):
    nx, ny = 6, 5
    o = oracle.Oracle(nx, ny, name, tau=0.7)
    rng = np.random.default_rng(2)
    o.init_moments(*workloads.random_smooth(nx, ny, seed=1))
    f = o.f * (1.0 + 0.05 * rng.uniform(-1, 1, size=o.f.shape))  # off equilibrium
    g = o.collide_only(f)
    cx, cy = o.vs["cx"][:, None, None], o.vs["cy"][:, None, None]
    for wgt in (1.0, cx, cy, cx * cx + cy * cy):
        np.testing.assert_allclose((wgt * g).sum(0), (wgt * f).sum(0), rtol=0, atol=2e-14)
    o.init_moments(np.full((ny, nx), 1.3), np.zeros((ny, nx)), np.zeros((ny, nx)), np.ones((ny, nx)))
    f0 = o.f.copy()
    o.run(3)
    np.testing.assert_allclose(o.f, f0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name,n,tau,which", [("D2Q16", 4, 0.8, "shear"), ("D2Q16", 4, 0.8, "heat"),
                                               ("D2Q36", 6, 0.9, "shear"), ("D2Q36", 6, 0.9, "heat")])
def test_linear_eigenmode_evolves_exactly(name, n, tau, which):
    """A small-amplitude eigenmode of the linearised step, f = f_rest + eps Re(v e^{iky}), must be
    multiplied by its eigenvalue every step (to O(eps^2))."""
    nx, ny = 2, 32
    k = 2 * math.pi / ny
    lam, V, cx, cy, W, sh, ht = modes(n, tau, 1.0, k)
    m = sh if which == "shear" else ht
    v = V[:, m] / np.max(np.abs(V[:, m]))
    eps = 1e-7
    y = np.arange(ny)
    pert = eps * np.real(v[:, None] * np.exp(1j * k * y)[None, :])  # (Q, ny)
    o = oracle.Oracle(nx, ny, name, tau=tau)
    f0 = W[:, None, None] + pert[:, :, None] * np.ones((1, 1, nx))
    o.set_populations(f0)
    steps = 40
    o.run(steps)
    want = W[:, None, None] + (lam[m].real ** steps) * pert[:, :, None]
    dev_got = o.f - W[:, None, None]
    dev_want = want - W[:, None, None]
    err = np.max(np.abs(dev_got - dev_want)) / np.max(np.abs(dev_want))
    assert err < 1e-5, err


def _decay_rate(o, field_index, k, t0, t1):
    o.run(t0)
    a0 = _amp(o, field_index, k)
    o.run(t1 - t0)
    a1 = _amp(o, field_index, k)
    return -math.log(a1 / a0) / ((t1 - t0) * k * k)


def _amp(o, field_index, k):
    fld = o.moments()[field_index].mean(axis=1)
    y = np.arange(len(fld))
    if field_index == 3:
        fld = fld - fld.mean()
    s = 2 * np.mean(fld * np.sin(k * y))
    c = 2 * np.mean(fld * np.cos(k * y))
    return math.hypot(s, c)


def test_shear_wave_closed_form_config_c0():
    """64x64 D2Q16, tau=0.8, dt=1, u_x = 0.01 sin(2 pi y/64): the amplitude decays as
    exp(-nu k^2 t) with nu = T(tau - 1/2) + nu_num (nu_num: the overlap gather's diffusion)."""
    nx = ny = 64
    k = 2 * math.pi / ny
    o = oracle.Oracle(nx, ny, "D2Q16", tau=0.8)
    o.init_moments(*workloads.shear_wave(nx, ny, eps=0.01))
    nu = _decay_rate(o, 1, k, 20, 200)
    nu_pred = (0.8 - 0.5) + numerical_viscosity(4)
    assert abs(nu - nu_pred) / nu_pred < 0.01, (nu, nu_pred)
    lam, *_ , sh, _ = modes(4, 0.8, 1.0, k)
    nu_lin = -math.log(abs(lam[sh])) / k ** 2
    assert abs(nu - nu_lin) / nu_lin < 2e-3, (nu, nu_lin)


def test_heat_mode_closed_form_d2q16():
    """T = 1 + 0.01 sin(2 pi y/64), rho = 1/T: the temperature mode decays as exp(-chi k^2 t)
    with chi = kappa/(rho c_P) = T (tau - 1/2) + numerical part (unit Prandtl number of BGK)."""
    nx, ny = 2, 64
    k = 2 * math.pi / ny
    o = oracle.Oracle(nx, ny, "D2Q16", tau=0.8)
    o.init_moments(*workloads.heat_mode(nx, ny, eps=0.01))
    chi = _decay_rate(o, 3, k, 20, 200)
    chi_pred = (0.8 - 0.5) + numerical_viscosity(4)
    assert abs(chi - chi_pred) / chi_pred < 0.01, (chi, chi_pred)
