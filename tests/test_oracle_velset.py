"""Pins of the oracle's velocity sets: Gauss-Hermite quadrature (the paper builds its velocity
sets on Hermite roots, Sec. 'The TVLBM model' and Introduction)."""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gauss_hermite_closed_forms.json")


def _dfact(k):
    return 1 if k <= 0 else k * _dfact(k - 2)


def gaussian_moment(k):
    """E[Z^k] for a standard normal Z: (k-1)!! for even k, 0 for odd k."""
    return 0.0 if k % 2 else float(_dfact(k - 1))


@pytest.mark.parametrize("n", [3, 4])
def test_closed_form_nodes_and_weights(n):
    g = json.load(open(GOLD))["n%d" % n]
    x, w = oracle.gauss_hermite(n)
    np.testing.assert_allclose(x, g["nodes"], rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, g["weights"], rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_matches_library_rule(n):
    xr, wr = hermegauss(n)
    x, w = oracle.gauss_hermite(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=5e-15)
    np.testing.assert_allclose(w, wr / wr.sum(), rtol=0, atol=5e-15)


@pytest.mark.parametrize("name", ["D2Q9", "D2Q16", "D2Q36"])
def test_quadrature_exactness_brute_force(name):
    """sum_l w_l cx^a cy^b = E[Z^a] E[Z^b] for all a, b <= 2n-1, and the rule fails at degree 2n."""
    vs = oracle.velocity_set(name)
    n = vs["n"]
    for a in range(2 * n):
        for b in range(2 * n):
            terms = vs["w"] * vs["cx"] ** a * vs["cy"] ** b
            want = gaussian_moment(a) * gaussian_moment(b)
            # odd moments cancel between large symmetric terms: compare against their size
            scale = max(1.0, np.sum(np.abs(terms)))
            assert abs(np.sum(terms) - want) <= 1e-14 * scale, (a, b, np.sum(terms), want)
    got = np.sum(vs["w"] * vs["cx"] ** (2 * n))
    assert abs(got - gaussian_moment(2 * n)) > 1e-3


def test_ordering_and_truncation_order():
    vs = oracle.velocity_set("D2Q16")
    assert vs["Q"] == 16 and vs["N"] == 3
    # l = i + n j : x varies fastest
    assert vs["cx"][1] > vs["cx"][0] and vs["cy"][1] == vs["cy"][0]
    assert vs["cy"][4] > vs["cy"][0]
    assert oracle.velocity_set("D2Q36")["N"] == 5
    assert oracle.velocity_set("D2Q9")["N"] == 2


def test_stream_table():
    n, a = oracle.stream_table(np.array([-2.3344142183389773, -0.741963784302726, 0.741963784302726, 2.5]), 1.0)
    assert list(n) == [-3, -1, 0, 2]
    np.testing.assert_allclose(a, [1 - 0.3344142183389773, 1 - 0.741963784302726, 0.741963784302726, 0.5], atol=1e-15)
    # space-filling shift: sqrt(3) * (1/sqrt(3)) snaps to exactly 1
    n, a = oracle.stream_table(np.array([-math.sqrt(3), 0.0, math.sqrt(3)]), 1.0 / math.sqrt(3))
    assert list(n) == [-1, 0, 1] and list(a) == [0.0, 0.0, 0.0]
