"""Pins of the time-integrated flux coefficients.

C2 is the time average of c_2(t) = (t + tau) e^{-t/tau} - tau (Eq. C2Formula),
C4 and C5 the time averages of e^{-t/tau} and -t e^{-t/tau} (UGKS free flux,
Sec. 2.2).  The oracle returns C2/tau, C4 - e, (C5 + dt e/2)/tau and C4 at
x = dt/tau.  Pinned by direct quadrature of those time integrals, by
40-digit evaluation of the closed forms, and by the thin/thick limits."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O

XS = [1e-9, 1e-6, 1e-4, 1e-3, 0.01, 0.1, 0.3, 0.49, 0.5, 0.51, 1.0, 3.0, 10.0, 100.0, 1e4]


def _quad_coefs(x):
    tau, dt = 1.0, x
    c2 = lambda t: (t + tau) * math.exp(-t / tau) - tau
    C2 = integrate.quad(c2, 0, dt, epsabs=0, epsrel=1e-13)[0] / dt
    C4 = integrate.quad(lambda t: math.exp(-t / tau), 0, dt, epsabs=0, epsrel=1e-13)[0] / dt
    C5 = -integrate.quad(lambda t: t * math.exp(-t / tau), 0, dt, epsabs=0, epsrel=1e-13)[0] / dt
    e = math.exp(-x)
    return C2 / tau, C4 - e, (C5 + dt * e / 2) / tau, C4


@pytest.mark.parametrize("x", [0.05, 0.2, 0.7, 2.0, 8.0, 30.0])
def test_time_integral_quadrature(x):
    want = _quad_coefs(x)
    got = O.coefs(x)
    for w, g in zip(want, got):
        assert abs(g - w) <= 1e-9 * abs(w), (x, want, got)


@pytest.mark.parametrize("x", XS)
def test_closed_forms_high_precision(x):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    X = mp.mpf(x)
    e = mp.e ** (-X)
    f2 = (2 / X) * (1 - e) - 1 - e
    c4 = (1 - e) / X
    f4 = c4 - e
    f5 = e * (1 + X / 2) - (1 - e) / X
    got = O.coefs(x)
    for w, g in zip((f2, f4, f5, c4), got):
        w = float(w)
        assert abs(g - w) <= 2e-15 * abs(w) + 1e-300, (x, w, g)


def test_limits():
    # thin: C2 -> 0, C4 -> 1, C5 -> -dt/2 ; thick: C2 -> -tau, C4 -> 0, C5 -> 0
    f2, f4, f5, c4 = O.coefs(1e-10)
    assert abs(f2) < 1e-19 and abs(c4 - 1) < 1e-9 and abs(f4) < 1e-9
    x = 1e-8
    f2, f4, f5, c4 = O.coefs(x)
    C5 = -f4  # C5/tau when e_eff = 0
    assert abs(C5 / x + 0.5) < 1e-8  # C5 / dt -> -1/2
    f2, f4, f5, c4 = O.coefs(1e6)
    assert abs(f2 + 1.0) < 1e-5 and c4 < 1e-5 and abs(f4) < 1e-5 and abs(f5) < 1e-5


def test_c5_identity():
    # C5 = tau e - (tau^2/dt)(1-e) = -tau (C4 - e)
    for x in [0.2, 1.0, 5.0]:  # the naive double forms below cancel for small x
        e = math.exp(-x)
        C5 = e - (1 - e) / x
        f2, f4, f5, c4 = O.coefs(x)
        assert abs(C5 + f4) <= 1e-13 * abs(C5)
        assert abs(f5 - (C5 + x * e / 2)) <= 1e-12 * abs(f5) + 1e-17
