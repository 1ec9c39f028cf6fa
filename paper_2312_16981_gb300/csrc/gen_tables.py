#!/usr/bin/env python
"""Write the CUDA path's coefficient tables: ugkwp_planck_table.h
(piecewise polynomial interpolants of the Planck edge functions used by the
group fractions b_g(T)), ugkwp_c2_table.h (the same for the equilibrium
flux coefficient C2 of the source-iteration faces) and ugkwp_log_table.h
(the breakpoints of the FP64 particle kernel's logarithm).

The group fraction (15/pi^4) int_{x_lo}^{x_hi} t^3/(e^t - 1) dt and its
T-derivative need, per group edge x = nu/T, the lower or upper partial
integral and the integrand times x, x^4/(e^x - 1).  This script evaluates
them in 60-digit decimal arithmetic from their series:

  lower part  L(x) = int_0^x t^3/(e^t-1) dt
                   = x^3/3 - x^4/8 + sum_{m>=1} B_2m x^{2m+3}/((2m+3)(2m)!)   (|x| < 2 pi),
  upper part  U(x) = int_x^inf t^3/(e^t-1) dt
                   = sum_{n>=1} e^{-nx} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4)  (x > 0),

(B_2m the Bernoulli numbers, exact rationals), and fits, on each interval of
width 1/2, the Chebyshev interpolant of degree 10 at the Chebyshev nodes,
re-expanded in powers of s = (x - centre)/(1/4) in [-1, 1]:

  rows 0..3   (0 <= x < 2):  L(x)/x^3 and x/(e^x - 1)   (the x^3 factor is applied
                             on the device, so both stay accurate as x -> 0);
  rows 4..79  (2 <= x < 40): U(x) and x^4/(e^x - 1) themselves;
  row 80      (x >= 40):     x^3 + 3x^2 + 6x + 6 and x^4 in powers of x
                             (times e^{-x} on the device; the next Bose term
                             is below e^{-40} of the first).

Each row stores 11 coefficient pairs (first function, second function),
constant term first.  The script also checks, in double-precision Horner
evaluation as the device does it, the worst relative error over 21 points
per interval and refuses to write a table worse than 1e-15.

The C2 table holds g2(x) = C2/(tau x) = f2(x)/x at x = dt/tau, with
f2(x) = 2 (1 - e^{-x})/x - 1 - e^{-x} (Eq. C2Formula divided by tau), on the
same intervals: rows 0..3 hold f2(x)/x^2 (-> -1/6 at x = 0; the device
multiplies by x), rows 4..79 g2 itself, and row 80 (x >= 40) g2 = (2/x - 1)/x
in powers of s = 1/x (the e^{-x} terms are below e^{-40} of it).

The log table serves a table-driven ln(1 + x) for x in [-1/2, 0.42]
(the method of P. T. P. Tang, "Table-driven implementation of the logarithm
function in IEEE floating-point arithmetic", ACM TOMS 16 (1990)): breakpoints
c_j = 1 + j/128, j = -64..54, with 1/c_j and ln c_j rounded to double from 60
digits; on the device ln(1 + x) = ln c_j + ln(1 + r), r = (x - j/128)/c_j,
|r| <= 1/128, by a degree-7 series.

Usage: python gen_tables.py [directory]   (default: this file's directory).
The committed headers are this script's output.
"""
from __future__ import annotations

import math
import os
import sys
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60
DEG = 10
WIDTH = Fraction(1, 2)
N_LOWER = 4          # rows on [0, 2)
N_ROWS = 80          # rows on [0, 40)
PI = Decimal("3.14159265358979323846264338327950288419716939937510582097494459")
TINY = Decimal(10) ** -58


def bernoulli(nmax):
    b = [Fraction(0)] * (nmax + 1)
    b[0] = Fraction(1)
    for m in range(1, nmax + 1):
        b[m] = -sum(math.comb(m + 1, k) * b[k] for k in range(m)) / (m + 1)
    return b


BERN = bernoulli(130)


def lower_over_x3(x: Decimal) -> Decimal:
    s = Decimal(1) / 3 - x / 8
    y, p = x * x, Decimal(1)
    for m in range(1, 64):
        p *= y
        bm = BERN[2 * m]
        t = Decimal(bm.numerator) / Decimal(bm.denominator) / ((2 * m + 3) * Decimal(math.factorial(2 * m))) * p
        s += t
        if abs(t) < TINY:
            return s
    raise RuntimeError("lower series did not converge at x = %s" % x)


def x_over_expm1(x: Decimal) -> Decimal:
    return Decimal(1) if x == 0 else x / (x.exp() - 1)


def upper(x: Decimal) -> Decimal:
    s, n = Decimal(0), 1
    while True:
        t = (-n * x).exp() * (x ** 3 / n + 3 * x * x / n ** 2 + 6 * x / n ** 3 + Decimal(6) / n ** 4)
        s += t
        if t < TINY * s:
            return s
        n += 1


def x4_over_expm1(x: Decimal) -> Decimal:
    return x ** 4 / (x.exp() - 1)


def cos_dec(a: Decimal) -> Decimal:
    s = t = Decimal(1)
    k = 0
    while True:
        k += 2
        t = -t * a * a / (k * (k - 1))
        s += t
        if abs(t) < TINY:
            return s


def cheb_powers(n):
    """Coefficients of T_0..T_{n-1} in powers of s."""
    tm = [[Fraction(1)], [Fraction(0), Fraction(1)]]
    for m in range(2, n):
        a = [Fraction(0)] + [2 * v for v in tm[m - 1]]
        b = tm[m - 2] + [Fraction(0)] * (len(a) - len(tm[m - 2]))
        tm.append([p - q for p, q in zip(a, b)])
    return tm[:n]


TPOW = cheb_powers(DEG + 1)


def fit(f, lo: Fraction, hi: Fraction):
    """Degree-DEG Chebyshev interpolant of f on [lo, hi] in powers of s."""
    n = DEG + 1
    c = Decimal(lo.numerator) / lo.denominator + Decimal((hi - lo).numerator) / (2 * (hi - lo).denominator)
    r = Decimal((hi - lo).numerator) / (2 * (hi - lo).denominator)
    ang = [PI * (Decimal(k) + Decimal("0.5")) / n for k in range(n)]
    fv = [f(c + r * cos_dec(a)) for a in ang]
    ch = []
    for m in range(n):
        ch.append(sum(fv[k] * cos_dec(m * ang[k]) for k in range(n)) * 2 / n)
    ch[0] /= 2
    mono = [Decimal(0)] * n
    for m in range(n):
        for j, v in enumerate(TPOW[m]):
            if v:
                mono[j] += ch[m] * Decimal(v.numerator) / v.denominator
    return [float(v) for v in mono]


def horner(coef, s):
    p = 0.0
    for a in reversed(coef):
        p = p * s + a
    return p


def f2_over_x2(x: Decimal) -> Decimal:
    if x == 0:
        return Decimal(-1) / 6
    e = (-x).exp()
    return (2 * (1 - e) / x - 1 - e) / (x * x)


def g2(x: Decimal) -> Decimal:
    e = (-x).exp()
    return (2 * (1 - e) / x - 1 - e) / x


def build_c2():
    rows = []
    worst = 0.0
    for j in range(N_ROWS):
        lo, hi = j * WIDTH, (j + 1) * WIDTH
        f = f2_over_x2 if j < N_LOWER else g2
        a = fit(f, lo, hi)
        centre = float(lo + WIDTH / 2)
        for k in range(21):
            x = float(lo) + float(WIDTH) * k / 20
            got = horner(a, (x - centre) * 4.0)
            want = f(Decimal(x))
            worst = max(worst, float(abs(Decimal(got) - want) / abs(want)))
        rows.append(a)
    rows.append([0.0, -1.0, 2.0] + [0.0] * (DEG - 2))
    return rows, worst


def build():
    rows = []
    worst = 0.0
    for j in range(N_ROWS):
        lo, hi = j * WIDTH, (j + 1) * WIDTH
        f1, f2 = (lower_over_x3, x_over_expm1) if j < N_LOWER else (upper, x4_over_expm1)
        a1, a2 = fit(f1, lo, hi), fit(f2, lo, hi)
        centre = float(lo + WIDTH / 2)
        for k in range(21):
            x = float(lo) + float(WIDTH) * k / 20
            s = (x - centre) * 4.0
            for coef, f in ((a1, f1), (a2, f2)):
                want = f(Decimal(x))
                got = horner(coef, s)
                worst = max(worst, float(abs(Decimal(got) - want) / abs(want)))
        rows.append((a1, a2))
    tail1 = [6.0, 6.0, 3.0, 1.0] + [0.0] * (DEG - 3)
    tail2 = [0.0, 0.0, 0.0, 0.0, 1.0] + [0.0] * (DEG - 4)
    rows.append((tail1, tail2))
    return rows, worst


def write(path):
    rows, worst = build()
    if not worst < 1e-15:
        raise RuntimeError("interpolation error %.3g exceeds 1e-15" % worst)
    lines = [
        "// ugkwp_planck_table.h -- written by gen_tables.py (do not edit).",
        "// Piecewise degree-%d interpolants of the Planck edge functions on intervals" % DEG,
        "// of width 1/2: rows 0..3 (x < 2) L(x)/x^3 and x/(e^x - 1); rows 4..79",
        "// (2 <= x < 40) U(x) and x^4/(e^x - 1); row 80 (x >= 40) x^3 + 3x^2 + 6x + 6",
        "// and x^4 in powers of x.  Per row: %d pairs (first, second function) of" % (DEG + 1),
        "// coefficients of s^0 .. s^%d, s = 4 (x - centre) (row 80: s = x)." % DEG,
        "// Worst relative error of the double-precision Horner evaluation: %.2e." % worst,
        "#pragma once",
        "",
        "namespace ugkwp {",
        "",
        "constexpr int kPlanckDeg = %d;" % DEG,
        "constexpr int kPlanckRows = %d;    // rows on [0, 40); one more for x >= 40" % N_ROWS,
        "constexpr int kPlanckLowerRows = %d;" % N_LOWER,
        "",
        "static __device__ __align__(16) const double kPlanckTab[%d] = {" % (len(rows) * (DEG + 1) * 2),
    ]
    for j, (a1, a2) in enumerate(rows):
        vals = []
        for k in range(DEG + 1):
            vals += [a1[k].hex(), a2[k].hex()]
        lines.append("    // row %d" % j)
        for i in range(0, len(vals), 4):
            lines.append("    " + ", ".join(vals[i:i + 4]) + ",")
    lines += ["};", "", "}  // namespace ugkwp", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))
    return worst


def write_c2(path):
    rows, worst = build_c2()
    if not worst < 1e-15:
        raise RuntimeError("interpolation error %.3g exceeds 1e-15" % worst)
    lines = [
        "// ugkwp_c2_table.h -- written by gen_tables.py (do not edit).",
        "// Piecewise degree-%d interpolants of g2(x) = f2(x)/x, f2 = C2/tau at" % DEG,
        "// x = dt/tau, on intervals of width 1/2: rows 0..3 (x < 2) f2(x)/x^2; rows",
        "// 4..79 (2 <= x < 40) g2(x); row 80 (x >= 40) (2/x - 1)/x in powers of 1/x.",
        "// Per row: %d coefficients of s^0 .. s^%d, s = 4 (x - centre) (row 80: s = 1/x)." % (DEG + 1, DEG),
        "// Worst relative error of the double-precision Horner evaluation: %.2e." % worst,
        "#pragma once",
        "",
        "namespace ugkwp {",
        "",
        "static __device__ __align__(16) const double kC2Tab[%d] = {" % (len(rows) * (DEG + 1)),
    ]
    for j, a in enumerate(rows):
        vals = [v.hex() for v in a]
        lines.append("    // row %d" % j)
        for i in range(0, len(vals), 4):
            lines.append("    " + ", ".join(vals[i:i + 4]) + ",")
    lines += ["};", "", "}  // namespace ugkwp", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))
    return worst


LOG_JMIN, LOG_JMAX = -64, 54


def write_log(path):
    lines = [
        "// ugkwp_log_table.h -- written by gen_tables.py (do not edit).",
        "// Breakpoints c_j = 1 + j/128, j = %d..%d, of the table-driven ln(1 + x):" % (LOG_JMIN, LOG_JMAX),
        "// pairs (1/c_j, ln c_j) rounded to double from 60-digit values.",
        "#pragma once",
        "",
        "namespace ugkwp {",
        "",
        "constexpr int kLogJMin = %d, kLogJMax = %d;" % (LOG_JMIN, LOG_JMAX),
        "",
        "static __device__ __align__(16) const double kLogTab[%d] = {" % (2 * (LOG_JMAX - LOG_JMIN + 1)),
    ]
    for j in range(LOG_JMIN, LOG_JMAX + 1):
        c = 1 + Decimal(j) / 128
        lines.append("    %s, %s,  // j = %d" % (float(1 / c).hex(), float(c.ln()).hex(), j))
    lines += ["};", "", "}  // namespace ugkwp", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.dirname(os.path.abspath(__file__))
    print("Planck table: worst relative error %.3e" % write(os.path.join(out, "ugkwp_planck_table.h")))
    print("C2 table:     worst relative error %.3e" % write_c2(os.path.join(out, "ugkwp_c2_table.h")))
    write_log(os.path.join(out, "ugkwp_log_table.h"))
    print("log table written")
