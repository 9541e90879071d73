"""Pins of the oracle's Grunwald-Letnikov weights (Section 2.1) to closed forms.

psi(g, m) = (-1)^m binom(1-g, m) (eq. psidefinition) is evaluated independently
in 50-digit arithmetic (mpmath) and by its Gamma-function form; the partial
sums and the generating function are standard binomial-series identities:
  sum_{m<=M} psi_m = Gamma(M+g) / (Gamma(g) M!),   sum_m psi_m z^m = (1-z)^{1-g}.
"""
import math

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 50

GAMMAS = [0.3, 0.5, 0.6, 0.7, 0.8, 0.95, 1.0, 1.4]


def mp_psi(g, m):
    return (-1) ** m * mpmath.binomial(1 - mpmath.mpf(g), m)


@pytest.mark.parametrize("g", GAMMAS)
def test_weights_match_binomial(g):
    n = 3000
    psi = oracle.weights(g, n)
    for m in list(range(0, 40)) + list(range(40, n, 97)) + [n - 1]:
        ref = float(mp_psi(g, m))
        if ref == 0.0:
            assert psi[m] == 0.0
        else:
            assert abs(psi[m] - ref) <= 5e-14 * abs(ref) * max(1.0, math.log(m + 1)), (m, psi[m], ref)


def test_weights_gamma_form_large_m():
    # psi_m = Gamma(m-1+g) / (Gamma(g-1) m!)  (eq. psidefinition with Gamma(n+1-m) reflected)
    g = 0.7
    n = 100001
    psi = oracle.weights(g, n)
    for m in (1000, 10000, 50000, 100000):
        ref = mpmath.gamma(m - 1 + mpmath.mpf(g)) / (mpmath.gamma(mpmath.mpf(g) - 1) * mpmath.factorial(m))
        assert abs(psi[m] / float(ref) - 1.0) < 1e-11


@pytest.mark.parametrize("g", [0.3, 0.6, 0.8, 0.95])
def test_partial_sums_closed_form(g):
    n = 20001
    psi = oracle.weights(g, n)
    ps = np.cumsum(psi)
    for M in (0, 1, 5, 100, 1000, 20000):
        ref = float(mpmath.gamma(M + mpmath.mpf(g)) / (mpmath.gamma(mpmath.mpf(g)) * mpmath.factorial(M)))
        assert ps[M] > 0
        assert abs(ps[M] - ref) < 1e-12 * max(1.0, M ** 0.5) * ref + 1e-15


@pytest.mark.parametrize("g", [0.5, 0.8, 1.3])
def test_generating_function(g):
    psi = oracle.weights(g, 200)
    for z in (0.5, -0.5, -1.0 + 1e-9):
        if abs(z) > 0.99:
            continue
        s = math.fsum(psi * z ** np.arange(200))
        assert abs(s - (1 - z) ** (1 - g)) < 1e-13


@pytest.mark.parametrize("g", [0.3, 0.5, 0.8, 0.95])
def test_sign_and_monotone_subdiffusion(g):
    psi = oracle.weights(g, 5000)
    assert psi[0] == 1.0
    assert np.all(psi[1:] < 0)
    assert np.all(np.abs(psi[2:]) < np.abs(psi[1:-1]))


def test_gamma_one_is_heat():
    psi = oracle.weights(1.0, 100)
    assert psi[0] == 1.0 and np.all(psi[1:] == 0.0)


@pytest.mark.parametrize("g", [0.35, 0.65, 0.7, 0.9])
def test_derivative_matches_digamma_form(g):
    # d psi_m / dg = psi_m [digamma(m-1+g) - digamma(g-1)]  (from the Gamma form)
    n = 4001
    psi, dpsi = oracle.weights(g, n, with_derivative=True)
    assert dpsi[0] == 0.0
    for m in (1, 2, 3, 10, 100, 1000, 4000):
        ref = mp_psi(g, m) * (mpmath.digamma(m - 1 + mpmath.mpf(g)) - mpmath.digamma(mpmath.mpf(g) - 1))
        assert abs(dpsi[m] - float(ref)) <= 1e-12 * abs(float(ref)) + 1e-18, m
    # and against a numerical derivative of the 50-digit binomial
    for m in (1, 7, 250):
        ref = mpmath.diff(lambda gg: mp_psi(gg, m), mpmath.mpf(g))
        assert abs(dpsi[m] - float(ref)) <= 1e-12 * abs(float(ref)) + 1e-18
