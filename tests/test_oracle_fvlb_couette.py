"""Pins of the finite-volume channel oracle with the pressure-scaled relaxation times of the
thermal Couette experiments (Sec. "Boundary Conditions: Avoiding temperature and velocity slip":
tau -> tau / p, tau_g -> tau_g / p, p = rho T, Newton-Raphson walls, Pr swept through tau_g).

With the scaling the dynamic viscosity is mu = tau Pr, Pr = tau_g / (tau_g - 2 tau), whatever
the density and temperature.  A sine perturbation of the Couette velocity, eps sin(pi y / L),
between the no-slip walls then decays at the rate nu (pi / L)^2, nu = tau Pr / rho; measured
between t = 0.5 and 1.5 (after the stress has built up from the equilibrium start) the oracle's
rate must match it for Pr = 1, 1/2 and 1/3 (tau_g = inf, -2 tau, -tau) within 3 %: the stress
follows the strain with a lag of the relaxation time (a (1 - tau_eff rate) ~ 1 % effect) and the
wall nodes carry a kinetic layer one node thick."""
import numpy as np
import pytest

from oracle import fvlb

U, TC, TAU, DT, L, NY, NX = 0.2, 1.0, 0.1, 0.005, 10.0 / 3.0, 41, 2
DTW = U ** 2 / 2.0  # Eckert number U^2 / (c_v dT) = 2 with c_v = 1


def _tau_g(pr):
    return np.inf if pr == 1.0 else 2.0 * TAU * pr / (pr - 1.0)


@pytest.mark.parametrize("pr", [1.0, 0.5, 1.0 / 3.0])
def test_pressure_scaled_viscosity_with_the_prandtl_term(pr):
    y = np.linspace(0.0, L, NY)
    eta = (y / L).reshape(-1, 1) * np.ones((1, NX))
    T = TC + DTW * (eta + pr / 2.0 * eta * (1.0 - eta))
    amps = []
    for eps in (0.0, 0.01):
        s = fvlb.FVLBChannel(NX, NY, y, (0.0, TC, U, TC + DTW), tau=TAU, tau_g=_tau_g(pr), dt=DT, exact=True,
                             nr_iters=8, pressure_scaled=True)
        s.init_moments(1.0 / T, U * eta + eps * np.sin(np.pi * eta), 0.0 * eta, T)
        a = []
        for _ in range(2):
            s.step(100 if not a else 200)
            a.append(s.profile())
        amps.append(a)
    c = NY // 2
    A = [(amps[1][k][1][c] - amps[0][k][1][c]) / 0.01 for k in range(2)]
    rho = amps[0][0][0][c]
    rate = -np.log(A[1] / A[0]) / (200 * DT)
    want = TAU * pr / rho * np.pi ** 2 / L ** 2
    assert abs(rate / want - 1.0) < 0.03, (rate, want)


def test_pressure_scaling_changes_only_the_rates():
    """The scaled collision term is the unscaled one times each cell's own p = rho T (both parts,
    BGK and Prandtl term): near p = 1 and near p = 2."""
    y = np.linspace(0.0, 2.0, 9)
    ny, nx = 9, 4
    yy = np.linspace(0, 1, ny).reshape(-1, 1) * np.ones((1, nx))
    for p in (1.0, 2.0):
        T = 1.0 + 0.02 * yy
        rho = p / T
        st = [fvlb.FVLBChannel(nx, ny, y, (0.0, 1.0, 0.0, 1.0), tau=0.5, tau_g=-1.5, dt=0.01, exact=False,
                               pressure_scaled=ps) for ps in (False, True)]
        for s in st:
            s.init_moments(rho, 0.03 * np.sin(3 * yy), 0.0 * yy, T)
            s.f += 1e-4 * np.cos(np.arange(16)).reshape(-1, 1, 1) * s.f  # a non-equilibrium part
        o0, o1 = st[0].omega(), st[1].omega()
        r, _, _, t = st[0].moments()
        assert abs(np.mean(r * t) - p) < 1e-3 * p
        assert np.max(np.abs(o1 - (r * t) * o0)) <= 1e-13 * np.max(np.abs(o1))
