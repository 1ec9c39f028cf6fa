"""Brute-force single-particle traces on 3-cell (and 2x2-cell) inputs with
hand-derived positions and times for fixed uniforms.

Cases: cross then collide, reflect (no t_f reset at a wall), reset into a
thick cell, escape through a vacuum side, the strict-inequality tie at a
face, and in 2D an x-face then y-face crossing and a corner tie.  The rule
under test is the streaming of Algorithm 1 with the t_f reset of the
interface remark: t_f2 = min(-tau_i ln eta, dt - t_tra)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def slab3(sig, dt=10.0, bc_right=I.BC_VACUUM):
    p = I.Problem(dim=1, nx=3, ny=1, dx=1.0, dy=1.0, G=1, grey=1, nu_edges=np.array([0.0, 1.0]),
                  sigma0=np.array(sig, dtype=float), cv=np.ones(3), T0=np.ones(3), dt=dt,
                  sig_p=0.0, sig_q=0.0, sig_cap=0.0,
                  bc=[I.BC_REFLECT, bc_right, I.BC_REFLECT, I.BC_REFLECT])
    return p, O.OracleProblem(p)


def run(op, p, x, mu, cell, newborn, draws, y=0.0, oy=0.0, w=1.0):
    tal = O.Tallies(p)
    r = O.stream_particle(op, np.ones(p.ncell), 0, x, y, mu, oy, 1.0, w, 0, cell, 0, newborn, 0,
                          np.array(draws, dtype=float), tal)
    return r, tal


def test_cross_then_collide():
    p, op = slab3([1.0, 1.0, 1.0])
    r, tal = run(op, p, 0.5, 0.5, 0, True, [math.exp(-0.5)])
    # face x=1 after (1-0.5)/0.5 = 1; in cell 1 t_f2 = 0.5 < 9: collide at x = 1 + 0.5*0.5
    assert r["fate"] == O.ABSORBED and r["cell"] == 1 and r["nseg"] == 2
    np.testing.assert_allclose(r["trace_x"], [1.0, 1.25], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r["trace_t"], [1.0, 1.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(tal.W, [-1.0, 1.0, 0.0])
    assert tal.E_abs[1] == 1.0 and tal.E_surv.sum() == 0.0


def test_reflect_reset_escape():
    p, op = slab3([0.1, 1e-3, 1e-6])
    r, tal = run(op, p, 0.5, -1.0, 0, False, [math.exp(-0.2), 0.999, 0.5], w=2.0)
    # t_f = 0.2/0.1 = 2: wall at t=0.5 (reflect, no reset), face 1 at t=1.5,
    # t_f2 = -ln(0.999)/1e-3 = 1.0005 > 1, face 2 at t=2.5, t_f3 = ln2/1e-6 > 7.5,
    # right wall (vacuum) at t = 3.5
    assert r["fate"] == O.ESCAPED and r["nseg"] == 4
    np.testing.assert_allclose(r["trace_x"], [0.0, 1.0, 2.0, 3.0], atol=1e-15)
    np.testing.assert_allclose(r["trace_t"], [0.5, 1.5, 2.5, 3.5], atol=1e-14)
    assert r["ox"] == 1.0
    np.testing.assert_allclose(tal.W, [-2.0, 0.0, 0.0])
    assert tal.esc[1] == 2.0


def test_reset_into_thick_cell():
    p, op = slab3([1.0, 1e6, 1.0])
    r, tal = run(op, p, 0.9, 1.0, 0, True, [0.5])
    tc = math.log(2.0) / 1e6
    assert r["fate"] == O.ABSORBED and r["cell"] == 1
    assert abs(r["x"] - (1.0 + tc)) < 1e-15 and abs(r["t_end"] - (0.1 + tc)) < 1e-15


def test_survivor_stays_and_tie_is_not_a_crossing():
    p, op = slab3([1e-9, 1e-9, 1e-9], dt=1.0)
    # reaches the face x=2 exactly at t = dt: ends on the face, stays in cell 1
    r, tal = run(op, p, 1.5, 0.5, 1, True, [])
    assert r["fate"] == O.SURVIVED and r["cell"] == 1 and r["x"] == 2.0 and r["nseg"] == 1
    assert tal.E_surv[1] == 1.0 and not tal.W.any()


def test_survivor_collides_in_own_cell():
    p, op = slab3([2.0, 2.0, 2.0], dt=1.0)
    r, _ = run(op, p, 1.2, -0.25, 1, False, [math.exp(-0.4)])
    # t_f = 0.4/2 = 0.2 < dt: collide at x = 1.2 - 0.25*0.2
    assert r["fate"] == O.ABSORBED and abs(r["x"] - 1.15) < 1e-15 and abs(r["t_end"] - 0.2) < 1e-16


def test_missing_draw_is_reported():
    p, op = slab3([1.0, 1.0, 1.0])
    r, _ = run(op, p, 0.5, 0.5, 0, True, [])
    assert r["fate"] == -1


def square2(sig=1e-9, dt=10.0):
    p = I.Problem(dim=2, nx=2, ny=2, dx=1.0, dy=1.0, G=1, grey=1, nu_edges=np.array([0.0, 1.0]),
                  sigma0=np.full(4, sig), cv=np.ones(4), T0=np.ones(4), dt=dt,
                  sig_p=0.0, sig_q=0.0, sig_cap=0.0,
                  bc=[I.BC_REFLECT, I.BC_REFLECT, I.BC_REFLECT, I.BC_VACUUM])
    return p, O.OracleProblem(p)


def test_2d_x_then_y_then_escape():
    p, op = square2()
    r, tal = run(op, p, 0.5, 0.6, 0, True, [0.5, 0.5], y=0.25, oy=0.8)
    t1 = 0.5 / 0.6
    y1 = 0.25 + 0.8 * t1
    t2 = t1 + (1.0 - y1) / 0.8
    x2 = 1.0 + 0.6 * (t2 - t1)
    t3 = t2 + 1.0 / 0.8
    assert r["fate"] == O.ESCAPED and r["nseg"] == 3 and r["cell"] == 3
    np.testing.assert_allclose(r["trace_t"], [t1, t2, t3], rtol=1e-14)
    np.testing.assert_allclose(r["trace_x"], [1.0, x2, x2 + 0.6 * 1.25], rtol=1e-14)
    assert r["y"] == 2.0
    np.testing.assert_allclose(tal.W, [-1.0, 0.0, 0.0, 0.0], atol=1e-15)
    assert tal.esc[3] == 1.0


def test_2d_corner_tie_takes_x_first():
    p, op = square2()
    s = math.sqrt(0.5)
    r, tal = run(op, p, 0.5, s, 0, True, [0.5, 0.5, 0.5], y=0.5, oy=s)
    # x-face first (cell 1), then the y-face at (almost) the same time (cell 3)
    assert r["trace_x"][0] == 1.0
    assert r["nseg"] >= 3 and r["fate"] == O.ESCAPED
    assert abs(r["trace_t"][0] - 0.5 / s) < 1e-15 and abs(r["trace_t"][1] - 0.5 / s) < 1e-15
