"""Pins of the oracle's frequency sampler (Eqs. Blinear, kg, App. A).

The CDF is checked against numerical integration of the linear density built
independently from the textbook Planck shape nu^3/(e^{nu/T}-1); the inverse
by G(nu(eta)) = eta; the distribution by a chi-square test."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O


def _planck(nu, T):
    return nu ** 3 / math.expm1(nu / T)


def _linear_density(nlo, nhi, T):
    mid = 0.5 * (nlo + nhi)
    dnu = nhi - nlo
    Bm = _planck(mid, T)
    k = (_planck(nhi, T) - _planck(nlo, T)) / dnu
    k = max(-2 * Bm / dnu, min(2 * Bm / dnu, k))
    return lambda nu: Bm + k * (nu - mid)


CASES = [(0.1, 0.13, 1.0), (1.0, 1.36, 0.3), (2.0, 2.7, 0.05), (0.01, 0.0136, 1.0),
         (5.0, 6.8, 1.0), (0.2, 0.9, 2.0)]


@pytest.mark.parametrize("nlo,nhi,T", CASES)
def test_cdf_matches_integrated_density(nlo, nhi, T):
    f = _linear_density(nlo, nhi, T)
    tot = integrate.quad(f, nlo, nhi, epsabs=0, epsrel=1e-13)[0]
    for nu in np.linspace(nlo, nhi, 9):
        want = integrate.quad(f, nlo, nu, epsabs=0, epsrel=1e-13)[0] / tot if nu > nlo else 0.0
        assert abs(O.nu_cdf(nlo, nhi, T, nu) - want) < 1e-13


@pytest.mark.parametrize("nlo,nhi,T", CASES)
def test_inverse(nlo, nhi, T):
    for eta in [1e-12, 1e-6, 0.1, 0.37, 0.5, 0.9, 1 - 1e-9]:
        nu = O.sample_nu(nlo, nhi, T, eta)
        assert nlo <= nu <= nhi
        assert abs(O.nu_cdf(nlo, nhi, T, nu) - eta) < 1e-14
    # where the clamped density vanishes at an end the CDF is quadratic there,
    # so the end is only resolved to ~sqrt(machine eps) of the group width
    assert abs(O.sample_nu(nlo, nhi, T, 0.0) - nlo) < 1e-7 * (nhi - nlo)
    assert abs(O.sample_nu(nlo, nhi, T, 1.0) - nhi) < 1e-7 * (nhi - nlo)


def test_clamped_slope_in_wien_tail():
    # at nu/T ~ 100 the Planck shape falls by e^-30 over the group: the line is
    # clamped to reach zero at nu+, density 2 (nhi - nu)/dnu^2
    nlo, nhi, T = 3.0, 3.3, 0.01
    for nu in [3.0, 3.1, 3.2, 3.3]:
        u = (nu - nlo) / (nhi - nlo)
        assert abs(O.nu_cdf(nlo, nhi, T, nu) - (2 * u - u * u)) < 1e-13
    # and with the Planck values far below the double range (x ~ 1e4)
    nu = O.sample_nu(9.0, 10.0, 1e-3, 0.75)
    assert abs(nu - (9.0 + 1.0 * (1 - math.sqrt(0.25)))) < 1e-12


def test_histogram_chi2():
    nlo, nhi, T = 1.0, 1.8, 0.4
    f = _linear_density(nlo, nhi, T)
    tot = integrate.quad(f, nlo, nhi)[0]
    rng = np.random.Generator(np.random.Philox(7))
    etas = rng.random(40000)
    nus = np.array([O.sample_nu(nlo, nhi, T, e) for e in etas])
    edges = np.linspace(nlo, nhi, 21)
    obs, _ = np.histogram(nus, edges)
    expv = np.array([integrate.quad(f, a, b)[0] / tot for a, b in zip(edges[:-1], edges[1:])]) * len(nus)
    chi2 = ((obs - expv) ** 2 / expv).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4
