"""Pins of the oracle's pathwise derivative (tangent) with respect to the
per-cell log-opacity scales s_c (sigma0_c -> sigma0_c e^{s_c}).

Every piece is compared with central finite differences of the oracle's own
forward functions, which the other oracle tests pin to the paper: the
coefficient derivatives, the Simpson group opacity, the wave flux, the
converged source iteration, and whole steps under common random numbers
(same seed, so every Monte Carlo decision is the same in the + and - runs;
the tests check that it is).  A dropped term, a wrong sign or a transposed
index in the tangent shows up as a mismatch far above the FD error."""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def test_dcoefs_matches_fd_both_branches():
    for x in [1e-6, 1e-3, 0.05, 0.3, 0.49, 0.499999, 0.5, 0.500001, 0.8, 2.0, 7.5, 30.0]:
        h = 1e-6 * max(x, 1e-2)
        cp, cm = np.array(O.coefs(x + h)), np.array(O.coefs(x - h))
        fd = (cp - cm) / (2 * h)
        d = np.array(O.dcoefs(x))
        np.testing.assert_allclose(d, fd, rtol=2e-7, atol=1e-9, err_msg="x=%g" % x)


def test_dcoefs_limits_and_identities():
    # x -> 0: c4 = 1 - x/2 + ..., f4 = x/2 - x^2/3 + ..., f2 = -x^2/6 + ..., f5 = -x^2/6 + ...
    df2, df4, df5, dc4 = O.dcoefs(1e-12)
    assert abs(dc4 + 0.5) < 1e-11 and abs(df4 - 0.5) < 1e-11
    assert abs(df2) < 1e-11 and abs(df5) < 1e-11
    # f4 = c4 - e and f2 = 2 c4 - 1 - e, so f4' - c4' = e and f2' - 2 c4' = e on both branches
    for x in [0.01, 0.2, 0.45, 0.6, 3.0]:
        df2, df4, df5, dc4 = O.dcoefs(x)
        assert abs((df4 - dc4) - np.exp(-x)) < 1e-14
        assert abs((df2 - 2 * dc4) - np.exp(-x)) < 1e-14


def test_dsigma_group_matches_fd_and_cap():
    p = I.small_multigroup(nx=4, G=6)
    p.sigma0 = np.array([1e2, 3.0, 1e5, 0.5])
    prob = O.OracleProblem(p)
    for c, T in [(0, 0.3), (1, 1.0), (2, 0.02), (3, 2.0)]:
        for g in range(p.G):
            for ds, dT in [(1.0, 0.0), (0.0, 1.0), (0.7, -0.4)]:
                h = 1e-7
                pp = O.OracleProblem(O.with_log_opacity(p, np.where(np.arange(4) == c, h * ds, 0.0)))
                pm = O.OracleProblem(O.with_log_opacity(p, np.where(np.arange(4) == c, -h * ds, 0.0)))
                fd = (O.sigma_group(pp, c, g, T + h * dT * T) - O.sigma_group(pm, c, g, T - h * dT * T)) / (2 * h)
                d = O.dsigma_group(prob, c, g, T, ds, dT * T)
                assert abs(d - fd) <= 1e-6 * abs(O.sigma_group(prob, c, g, T)) + 1e-12, (c, T, g)
    # every Simpson point under the cap: no dependence on s at all
    q = p.replace(sig_cap=1.0)
    q.sigma0 = np.full(4, 1e6)
    assert O.dsigma_group(O.OracleProblem(q), 0, 0, 0.01, 1.0, 0.3) == 0.0


def _wave_case(p, seed):
    rng = np.random.default_rng(seed)
    T = 0.2 + rng.random(p.ncell)
    rho_h = rng.random(p.ncell * p.G) * 0.3 + 0.05
    e_eff = np.zeros((p.ncell + 4) * p.G)
    # sampled fraction: e of the cell's group opacity where "particles were born"
    prob = O.OracleProblem(p)
    for c in range(p.ncell):
        for g in range(p.G):
            if rng.random() < 0.7:
                e_eff[c * p.G + g] = np.exp(-p.dt * p.c / p.eps ** 2 * O.sigma_group(prob, c, g, T[c]))
    for side in range(2):
        if p.dim == 1 and p.bc[side] == I.BC_BLACKBODY:
            cin = 0 if side == 0 else p.nx - 1
            for g in range(p.G):
                e_eff[(p.ncell + side) * p.G + g] = np.exp(
                    -p.dt * p.c / p.eps ** 2 * O.sigma_group(prob, cin, g, p.bcT[side]))
    return T, rho_h, e_eff


@pytest.mark.parametrize("case", ["bb_order2", "bb_order1", "vacuum", "reflect_2d", "vacuum_2d"])
def test_wave_flux_tangent_matches_fd(case):
    if case.startswith("bb"):
        p = I.small_multigroup(nx=9, G=4)
        p.wave_order = 2 if case == "bb_order2" else 1
    elif case == "vacuum":
        p = I.small_multigroup(nx=9, G=4)
        p.bc = [I.BC_VACUUM, I.BC_VACUUM, 0, 0]
    else:
        p = I.small_checkerboard(n=6, G=3)
        if case == "vacuum_2d":
            p.bc = [I.BC_VACUUM, I.BC_REFLECT, I.BC_VACUUM, I.BC_VACUUM]
    p.dt = 0.02 * p.dx
    rng = np.random.default_rng(3)
    p.sigma0 = 10 ** rng.uniform(-1, 2, p.ncell)
    T, rho_h, e_eff = _wave_case(p, 5)
    ds = rng.normal(size=p.ncell)
    dT = rng.normal(size=p.ncell) * T
    drho_h = rng.normal(size=p.ncell * p.G) * rho_h
    d = O.wave_flux_tangent(O.OracleProblem(p), T, dT, ds, rho_h, drho_h, e_eff)
    h = 1e-7

    def F(sgn):
        q = O.with_log_opacity(p, sgn * h * ds)
        # e_eff is the upwind cell's e, a function of its opacity: recompute it
        prob = O.OracleProblem(q)
        Tq = T + sgn * h * dT
        e = e_eff.copy()
        for c in range(p.ncell):
            for g in range(p.G):
                if e_eff[c * p.G + g] > 0:
                    e[c * p.G + g] = np.exp(-p.dt * p.c / p.eps ** 2 * O.sigma_group(prob, c, g, Tq[c]))
        for side in range(2):
            if p.dim == 1 and p.bc[side] == I.BC_BLACKBODY:
                cin = 0 if side == 0 else p.nx - 1
                for g in range(p.G):
                    e[(p.ncell + side) * p.G + g] = np.exp(
                        -p.dt * p.c / p.eps ** 2 * O.sigma_group(prob, cin, g, p.bcT[side]))
        return O.wave_flux(prob, Tq, rho_h + sgn * h * drho_h, e)
    fd = (F(1) - F(-1)) / (2 * h)
    scale = np.max(np.abs(fd))
    assert scale > 0
    np.testing.assert_allclose(d, fd, rtol=0, atol=2e-6 * scale)


@pytest.mark.parametrize("dim", [1, 2])
def test_source_iteration_tangent_matches_fd(dim):
    if dim == 1:
        p = I.small_multigroup(nx=10, G=4)
        p.bc = [I.BC_BLACKBODY, I.BC_VACUUM, 0, 0]
    else:
        p = I.small_checkerboard(n=6, G=3)
    p.si_tol = 1e-14
    p.si_max_iters = 2000
    rng = np.random.default_rng(11)
    p.sigma0 = 10 ** rng.uniform(0, 2.5, p.ncell)
    T_n = 0.3 + rng.random(p.ncell)
    prob = O.OracleProblem(p)
    rho_n = np.array([O.phi(prob, g, T_n[c]) * (0.5 + rng.random()) for c in range(p.ncell) for g in range(p.G)])
    R = rho_n * (1.0 + 0.1 * rng.normal(size=rho_n.size))
    ds = rng.normal(size=p.ncell)
    dT_n = rng.normal(size=p.ncell) * T_n
    dR = rng.normal(size=R.size) * R
    st, T, rho, _, it = O.source_iteration(prob, T_n, rho_n, R)
    assert st == 0
    st, dT, drho, it2 = O.source_iteration_tangent(prob, dT_n, ds, dR, T, rho)
    assert st == 0 and it2 < 2000
    h = 1e-6

    def S(sgn):
        q = O.OracleProblem(O.with_log_opacity(p, sgn * h * ds))
        s, Tq, rq, _, _ = O.source_iteration(q, T_n + sgn * h * dT_n, rho_n, R + sgn * h * dR)
        assert s == 0
        return Tq, rq
    (Tp, rp), (Tm, rm) = S(1), S(-1)
    np.testing.assert_allclose(dT, (Tp - Tm) / (2 * h), rtol=0, atol=1e-6 * np.max(np.abs(dT)))
    np.testing.assert_allclose(drho, (rp - rm) / (2 * h), rtol=0, atol=1e-6 * np.max(np.abs(drho)))


def _step_case(name):
    if name == "multigroup":
        return I.small_multigroup(nx=12, G=4, omega_ref=2e-6), 4
    if name == "multigroup_order1":
        p = I.small_multigroup(nx=12, G=4, omega_ref=2e-6)
        p.wave_order = 1
        return p, 4
    if name == "grey_blackbody":
        return I.grey_slab(nx=20, omega_ref=2.5e-6), 5
    if name == "vacuum":
        p = I.small_multigroup(nx=10, G=3, omega_ref=2e-6)
        p.bc = [I.BC_BLACKBODY, I.BC_VACUUM, 0, 0]
        return p, 4
    return I.small_checkerboard(n=8, G=3, omega_ref=2e-6), 3


@pytest.mark.parametrize("name", ["multigroup", "multigroup_order1", "grey_blackbody", "vacuum", "checkerboard"])
def test_step_tangent_matches_crn_finite_differences(name):
    p, steps = _step_case(name)
    rng = np.random.default_rng(0)
    s = rng.normal(0, 0.1, p.ncell)
    v = rng.normal(0, 1, p.ncell)
    _, stt, _ = O.misfit(O.with_log_opacity(p, rng.normal(0, 0.1, p.ncell)), steps, np.zeros(p.ncell))
    L, dL, st = O.misfit_tangent(O.with_log_opacity(p, s), steps, stt.T, v)
    assert st.particles.n > 100
    h = 1e-6
    Lp, _, rp = O.misfit(O.with_log_opacity(p, s + h * v), steps, stt.T, records=True)
    Lm, _, rm = O.misfit(O.with_log_opacity(p, s - h * v), steps, stt.T, records=True)
    # common random numbers: the same decisions in both runs
    for a, b in zip(rp, rm):
        assert len(a) == len(b)
        assert np.array_equal(a["fate"], b["fate"]) and np.array_equal(a["cell1"], b["cell1"])
        assert np.array_equal(a["id"], b["id"])
    fd = (Lp - Lm) / (2 * h)
    assert abs(dL - fd) <= 1e-6 * abs(fd), (dL, fd)


def test_step_tangent_is_linear_in_the_direction():
    p, steps = _step_case("multigroup")
    rng = np.random.default_rng(4)
    s = rng.normal(0, 0.1, p.ncell)
    Tt = np.full(p.ncell, 0.05)
    v1, v2 = rng.normal(size=p.ncell), rng.normal(size=p.ncell)
    q = O.with_log_opacity(p, s)
    _, d1, _ = O.misfit_tangent(q, steps, Tt, v1)
    _, d2, _ = O.misfit_tangent(q, steps, Tt, v2)
    _, d12, _ = O.misfit_tangent(q, steps, Tt, 2.0 * v1 - 3.0 * v2)
    assert abs(d12 - (2.0 * d1 - 3.0 * d2)) <= 1e-10 * (abs(d1) + abs(d2))
