"""The CUDA path's coefficient tables, checked on the CPU: the committed
headers are exactly what their generator writes, and the device's evaluation
of them (one Horner pass, emulated here in float64 with the same operation
order) gives the Planck group fractions b_g(T) and their T-derivative
(Sec. 2.1) to the accuracy of the oracle's quadrature, the equilibrium flux
coefficient C2 (Eq. C2Formula) to that of the oracle's series and closed
forms, and the FP64 particle kernel's -ln u of a free-time draw (Eq.
particle-tf-formula) to about an ulp of the library logarithm."""
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2312_16981_gb300", "csrc")
HEADER = os.path.join(CSRC, "ugkwp_planck_table.h")
C2HEADER = os.path.join(CSRC, "ugkwp_c2_table.h")
LOGHEADER = os.path.join(CSRC, "ugkwp_log_table.h")


def table():
    txt = open(HEADER).read()
    body = txt[txt.index("kPlanckTab["):]
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-f.]+p[-+]?\d+", body)]
    deg = int(re.search(r"kPlanckDeg = (\d+)", txt).group(1))
    rows = int(re.search(r"kPlanckRows = (\d+)", txt).group(1))
    lower = int(re.search(r"kPlanckLowerRows = (\d+)", txt).group(1))
    return np.array(vals).reshape(rows + 1, deg + 1, 2), rows, lower


TAB, ROWS, LOWER = table()
PI4_15 = math.pi ** 4 / 15


def edge(x):
    """(V, g4, lower) as the device computes them."""
    if not x > 0:
        return 0.0, 0.0, True
    if x > 740.0:
        return 0.0, 0.0, False
    tail = x >= 40.0
    j = ROWS if tail else int(x * 2.0)
    s = x if tail else (x - (0.25 + 0.5 * j)) * 4.0
    p1, p2 = TAB[j, -1]
    for k in range(TAB.shape[1] - 2, -1, -1):
        p1 = p1 * s + TAB[j, k, 0]
        p2 = p2 * s + TAB[j, k, 1]
    lower = j < LOWER
    m = x * x * x if lower else (math.exp(-x) if tail else 1.0)
    return m * p1, m * p2, lower


def fraction(x1, x2):
    lo, hi = edge(x1), edge(x2)
    if hi[2]:
        I_ = hi[0] - lo[0]
    elif not lo[2]:
        I_ = lo[0] - hi[0]
    else:
        I_ = (PI4_15 - lo[0]) - hi[0]
    b = I_ / PI4_15
    return b, 4.0 * b + (lo[1] - hi[1]) / PI4_15


def c2_table():
    txt = open(C2HEADER).read()
    body = txt[txt.index("kC2Tab["):]
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-f.]+p[-+]?\d+", body)]
    return np.array(vals).reshape(ROWS + 1, TAB.shape[1])


C2TAB = c2_table()


def g2(x, ix):
    """f2(x)/x as the device computes it."""
    tail = x >= 40.0
    j = ROWS if tail else int(x * 2.0)
    s = ix if tail else (x - (0.25 + 0.5 * j)) * 4.0
    p = C2TAB[j, -1]
    for k in range(C2TAB.shape[1] - 2, -1, -1):
        p = p * s + C2TAB[j, k]
    return p * x if j < LOWER else p


def test_headers_are_generator_output(tmp_path):
    subprocess.run([sys.executable, os.path.join(CSRC, "gen_tables.py"), str(tmp_path)], check=True,
                   capture_output=True)
    assert (tmp_path / "ugkwp_planck_table.h").read_text() == open(HEADER).read()
    assert (tmp_path / "ugkwp_c2_table.h").read_text() == open(C2HEADER).read()
    assert (tmp_path / "ugkwp_log_table.h").read_text() == open(LOGHEADER).read()


def _log_table():
    txt = open(LOGHEADER).read()
    body = txt[txt.index("kLogTab["):]
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-f.]+p[-+]?\d+", body)]
    jmin = int(re.search(r"kLogJMin = (-?\d+)", txt).group(1))
    return np.array(vals).reshape(-1, 2), jmin


LOGTAB, LOGJMIN = _log_table()
LN2_HI, LN2_LO = float.fromhex("0x1.62e42fefa3800p-1"), float.fromhex("0x1.ef35793c76730p-45")


def neg_log(u):
    """-ln u as the FP64 particle kernel computes it (same operations)."""
    if u > 0.5:
        x, kd = u - 1.0, 0.0
    else:
        b = int(np.float64(u).view(np.int64))
        k = ((b >> 52) & 0x7FF) - 1023
        mb = (b & 0x000FFFFFFFFFFFFF) | 0x3FF0000000000000
        if mb > 0x3FF6A09E667F3BCD:
            mb -= 0x0010000000000000
            k += 1
        x = float(np.int64(mb).view(np.float64)) - 1.0
        kd = float(k)
    jd = float(np.rint(x * 128.0))
    ic, lc = LOGTAB[int(jd) - LOGJMIN]
    r = (x - jd * (1.0 / 128.0)) * ic
    p = 1.0 / 7.0
    for c in (-1.0 / 6.0, 1.0 / 5.0, -0.25, 1.0 / 3.0, -0.5):
        p = math.fma(p, r, c) if hasattr(math, "fma") else p * r + c
    l1p = (r * r) * p + r
    return -(kd * LN2_HI + (lc + (kd * LN2_LO + l1p)))


def test_log_table_entries():
    for j in range(LOGJMIN, LOGJMIN + len(LOGTAB)):
        c = 1.0 + j / 128.0
        ic, lc = LOGTAB[j - LOGJMIN]
        assert abs(ic * c - 1.0) <= 2.3e-16
        assert abs(lc - math.log(c)) <= 1.2e-16 * max(abs(lc), 1e-300) + 1e-300


def test_neg_log_within_an_ulp_or_two():
    rng = np.random.default_rng(7)
    # draws as the kernel forms them: (m + 1/2) 2^-52, never 0 or 1
    m = rng.integers(0, 1 << 52, size=20000, dtype=np.int64)
    us = list((m.astype(np.float64) + 0.5) * 2.0 ** -52)
    us += [2.0 ** -53, (2 ** 52 - 0.5) * 2.0 ** -52, 0.5, 0.5 + 2 ** -53, 0.25, 2 ** -0.5, 0.75, 1e-300 ** 0 * 0.9999]
    for u in us:
        want = -math.log(u)
        assert abs(neg_log(u) - want) <= 4.5e-16 * want, (u, neg_log(u), want)


def test_c2_table_matches_oracle_coefficients():
    # the oracle's f2 = C2/tau from its own series / closed forms
    for x in np.concatenate([np.geomspace(1e-9, 1e4, 500), [0.5, 1.999999, 2.0, 39.999, 40.0]]):
        want = O.coefs(x)[0] / x
        got = g2(x, 1.0 / x)
        assert abs(got - want) <= 3e-14 * abs(want), (x, got, want)


def test_c2_tail_row_is_the_exact_expansion():
    np.testing.assert_array_equal(C2TAB[ROWS, :3], [0.0, -1.0, 2.0])
    assert not C2TAB[ROWS, 3:].any()


def test_tail_row_is_the_exact_polynomials():
    np.testing.assert_array_equal(TAB[ROWS, :5, 0], [6.0, 6.0, 3.0, 1.0, 0.0])
    np.testing.assert_array_equal(TAB[ROWS, :5, 1], [0.0, 0.0, 0.0, 0.0, 1.0])
    assert not TAB[ROWS, 5:].any()


def test_rows_are_continuous_at_their_joints():
    # adjacent interpolants meet at the shared end point (s = +1 / s = -1)
    for j in range(ROWS - 1):
        a1 = np.polynomial.polynomial.polyval(1.0, TAB[j, :, 0])
        b1 = np.polynomial.polynomial.polyval(-1.0, TAB[j + 1, :, 0])
        if j + 1 == LOWER:      # L/x^3 against U: L(2) = pi^4/15 - U(2)
            assert abs(8.0 * a1 - (PI4_15 - b1)) < 1e-15 * PI4_15
        else:
            assert abs(a1 - b1) <= 1e-15 * abs(b1)


def test_group_fractions_match_quadrature():
    edges = I.log_groups(30, 1e-3, 10.0)
    worst_b = worst_d = 0.0
    for T in np.geomspace(1e-4, 20.0, 41):
        for g in range(30):
            x1, x2 = edges[g] / T, edges[g + 1] / T
            b, d = fraction(x1, x2)
            wb, wd = O.planck_integral(x1, x2), O.planck_dintegral(x1, x2)
            if wb > 1e-300:
                worst_b = max(worst_b, abs(b - wb) / wb)
            if wd > 1e-300:
                worst_d = max(worst_d, abs(d - wd) / wd)
    assert worst_b < 2e-13, worst_b
    assert worst_d < 2e-12, worst_d


@pytest.mark.parametrize("x", [1e-6, 0.3, 1.999999, 2.0, 2.000001, 7.77, 39.99, 40.0, 123.0, 700.0])
def test_single_edges_against_quadrature(x):
    # lower part against [0, x], upper part against [x, 800]
    V, g4, lower = edge(x)
    if lower:
        want = O.planck_integral(1e-300, x) * PI4_15
    else:
        want = O.planck_integral(x, 800.0) * PI4_15
    assert abs(V - want) <= 1e-14 * want
    assert abs(g4 - x ** 4 / math.expm1(x)) <= 1e-15 * g4
