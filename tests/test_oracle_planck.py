"""Pins of the oracle's Planck group integrals and group opacity.

b_g(T) = (15/pi^4) int t^3/(e^t-1) dt over the group (Sec. 2.1: the group
integral of B with int int B = a c T^4).  Pinned by the pi^4/15 identity, the
small-x and large-x closed forms, arbitrary-precision quadrature, and the
T-derivative by finite differences."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def test_partition_of_unity():
    edges = np.concatenate([[1e-7], np.geomspace(1e-3, 60.0, 80), [800.0]])
    s = sum(O.planck_integral(a, b) for a, b in zip(edges[:-1], edges[1:]))
    assert abs(s - 1.0) < 2e-14


def test_small_x_limit():
    # t^3/(e^t-1) = t^2 - t^3/2 + t^4/12 - t^6/720 + ...
    for a, b in [(1e-4, 2e-4), (1e-3, 1.5e-3), (0.01, 0.02)]:
        F = lambda x: x ** 3 / 3 - x ** 4 / 8 + x ** 5 / 60 - x ** 7 / 5040
        exact = 15 / math.pi ** 4 * (F(b) - F(a))
        assert abs(O.planck_integral(a, b) - exact) <= 1e-13 * exact


def test_large_x_closed_form():
    # for x >= 40 only the n = 1 term of the Bose series survives:
    # int_x^inf t^3 e^-t dt = e^-x (x^3 + 3x^2 + 6x + 6)
    P = lambda x: math.exp(-x) * (x ** 3 + 3 * x ** 2 + 6 * x + 6)
    for a, b in [(40.0, 45.0), (50.0, 80.0), (100.0, 101.0), (600.0, 800.0), (683.3, 928.8)]:
        exact = 15 / math.pi ** 4 * (P(a) - P(b))
        assert abs(O.planck_integral(a, b) - exact) <= 1e-13 * exact


def test_against_arbitrary_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    f = lambda t: t ** 3 / mp.expm1(t)
    for a, b in [(0.05, 0.07), (0.7, 1.1), (2.0, 2.7), (3.0, 9.0), (12.0, 16.0), (0.2, 30.0)]:
        exact = float(15 / mp.pi ** 4 * mp.quad(f, [a, b]))
        assert abs(O.planck_integral(a, b) - exact) <= 1e-14 * exact


def test_derivative_integral_identity():
    # int_0^inf t^4 e^t/(e^t-1)^2 dt = 4 pi^4/15 (by parts)
    edges = [1e-7, 0.5, 2.0, 10.0, 50.0, 800.0]
    s = sum(O.planck_dintegral(a, b) for a, b in zip(edges[:-1], edges[1:]))
    assert abs(s - 4.0) < 1e-13


def test_dphi_is_derivative_of_phi():
    p = I.multigroup_slab(nx=4, G=8)
    op = O.OracleProblem(p)
    for T in [0.003, 0.05, 0.3, 1.0, 2.5]:
        for g in range(p.G):
            xmax = max(1.0, p.nu_edges[g + 1] / T)
            h = 1e-4 * T / xmax          # keeps the O((h x/T)^2) truncation small
            fd = (O.phi(op, g, T + h) - O.phi(op, g, T - h)) / (2 * h)
            d = O.dphi(op, g, T)
            if O.phi(op, g, T) < 1e-250:
                continue
            assert abs(d - fd) <= 1e-7 * abs(d) + 1e-300, (T, g, d, fd)


def test_phi_sums_to_acT4_over_full_groups():
    p = I.multigroup_slab(nx=2, G=40)
    p.nu_edges = np.geomspace(1e-9, 1e4, 41)
    p.a, p.c = 0.7, 3.0
    op = O.OracleProblem(p)
    for T in [0.01, 0.3, 1.0, 7.0]:
        tot = sum(O.phi(op, g, T) for g in range(p.G))
        assert abs(tot - p.a * p.c * T ** 4) <= 1e-13 * p.a * p.c * T ** 4


def test_grey_phi():
    p = I.grey_slab(nx=2)
    op = O.OracleProblem(p)
    assert O.phi(op, 0, 0.5) == p.a * p.c * 0.5 ** 4
    assert O.dphi(op, 0, 0.5) == 4 * p.a * p.c * 0.5 ** 3


def test_simpson_group_opacity():
    p = I.multigroup_slab(nx=3, G=5)
    p.sigma0 = np.array([2.0, 3.0, 5.0])
    p.sig_cap = 0.0
    # p = 2: Simpson's rule is exact for the group average of nu^2
    p.sig_p, p.sig_q = 2.0, 0.0
    op = O.OracleProblem(p)
    for g in range(p.G):
        a, b = p.nu_edges[g], p.nu_edges[g + 1]
        avg = 3.0 * (b ** 3 - a ** 3) / (3 * (b - a))
        assert abs(O.sigma_group(op, 1, g, 0.7) - avg) <= 1e-14 * avg
    # p = 0, q = -1/2: constant in nu
    p.sig_p, p.sig_q = 0.0, -0.5
    op = O.OracleProblem(p)
    assert abs(O.sigma_group(op, 2, 3, 0.25) - 5.0 * 2.0) < 1e-14
    # the cap is applied pointwise before averaging
    p.sig_p, p.sig_q, p.sig_cap = -3.0, 0.0, 1e6
    p.nu_edges = np.array([0.001, 0.01, 0.1, 1.0, 10.0, 100.0])
    op = O.OracleProblem(p)
    a, b = 0.001, 0.01
    m = 0.5 * (a + b)
    pts = [min(2.0 * v ** -3, 1e6) for v in (a, m, b)]
    assert abs(O.sigma_group(op, 0, 0, 1.0) - (pts[0] + 4 * pts[1] + pts[2]) / 6) < 1e-9
    assert O.sigma(op, 0, 0.001, 1.0) == 1e6
