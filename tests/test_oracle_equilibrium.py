"""Pins of the oracle's Hermite equilibrium (Sec. 'The TVLBM model'; Appendix A)."""
import math

import numpy as np
import pytest

import oracle


def gaussian_raw_moment(k, u, T):
    """E[(u + sqrt(T) Z)^k], Z standard normal (closed form)."""
    s = 0.0
    for j in range(0, k // 2 + 1):
        dfact = 1
        for m in range(2 * j - 1, 0, -2):
            dfact *= m
        s += math.comb(k, 2 * j) * u ** (k - 2 * j) * T ** j * dfact
    return s


def _cases(seed, count=6):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        yield rng.uniform(0.5, 2.0), rng.normal() * 0.2, rng.normal() * 0.2, rng.uniform(0.8, 1.25)


@pytest.mark.parametrize("name", ["D2Q9", "D2Q16", "D2Q36"])
def test_tensor_form_equals_appendix_a(name):
    o = oracle.Oracle(4, 4, name)
    for rho, ux, uy, T in _cases(1):
        a = o.equilibrium(rho, ux, uy, T)
        b = o.equilibrium_appendix_a(rho, ux, uy, T)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * rho)


@pytest.mark.parametrize("name", ["D2Q9", "D2Q16", "D2Q36"])
def test_moments_of_equilibrium_are_gaussian(name):
    """The truncated Hermite expansion reproduces the Maxwellian moments of total degree <= N:
    sum_l f_eq cx^a cy^b = rho E[(ux+sqrt(T)Z)^a] E[(uy+sqrt(T)Z)^b].  This fixes every order
    of a^(n):H^(n) up to N (a dropped or mis-signed term moves some moment)."""
    o = oracle.Oracle(4, 4, name)
    vs, N = o.vs, o.N
    for rho, ux, uy, T in _cases(2):
        f = o.equilibrium(rho, ux, uy, T)
        for a in range(N + 1):
            for b in range(N + 1 - a):
                got = np.sum(f * vs["cx"] ** a * vs["cy"] ** b)
                want = rho * gaussian_raw_moment(a, ux, T) * gaussian_raw_moment(b, uy, T)
                assert abs(got - want) < 1e-13 * max(1.0, abs(want)), (name, a, b, got, want)
        # conserved moments with the paper's definitions: rho, rho u, (D/2) rho T + rho u^2/2
        assert abs(f.sum() - rho) < 1e-14
        e = 0.5 * np.sum((vs["cx"] ** 2 + vs["cy"] ** 2) * f)
        assert abs(e - (rho * T + 0.5 * rho * (ux * ux + uy * uy))) < 1e-13


def test_truncation_is_real():
    """Degree N+1 moments are NOT those of the Maxwellian (the set's order is the cut)."""
    o = oracle.Oracle(4, 4, "D2Q16")
    vs = o.vs
    f = o.equilibrium(1.0, 0.2, 0.1, 1.1)
    got = np.sum(f * vs["cx"] ** 4)
    want = gaussian_raw_moment(4, 0.2, 1.1)
    assert abs(got - want) > 1e-4


@pytest.mark.parametrize("name", ["D2Q16", "D2Q36"])
def test_rest_state(name):
    o = oracle.Oracle(4, 4, name)
    np.testing.assert_allclose(o.equilibrium(1.7, 0.0, 0.0, 1.0), 1.7 * o.vs["w"], rtol=1e-15, atol=0)


def test_c_core_matches_python_tensor_definition():
    o = oracle.Oracle(4, 4, "D2Q16")
    vs = o.vs
    for rho, ux, uy, T in _cases(3, 3):
        a = o.equilibrium(rho, ux, uy, T)
        b = oracle.equilibrium_tensor(rho, ux, uy, T, vs["cx"], vs["cy"], vs["w"], vs["N"])
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name", ["D2Q16", "D2Q36"])
def test_init_then_moments_roundtrip(name):
    import workloads
    o = oracle.Oracle(9, 7, name)
    fields = workloads.random_smooth(9, 7, seed=5)
    o.init_moments(*fields)
    got = o.moments()
    for g, w in zip(got, fields):
        np.testing.assert_allclose(g, w, rtol=0, atol=1e-13)
