"""Pins of the numerical collision time used for sampling at thin/thick
joints (Sec. 3.2, heterogeneous Marshak and Larsen cases):
tau_num = tau + C J dt, J the temperature contrast across the cell's faces.
Checked against what the definition fixes: it reduces to tau when C = 0 or
where T is uniform, it never samples fewer particles than tau does, it
grows the sampled fraction towards 1 as C grows, and a step with it still
conserves energy exactly."""
import numpy as np

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def _joint_slab(C):
    p = I.small_multigroup(nx=16, G=4, omega_ref=2e-6)
    sig0 = np.full(p.nx, 10.0)
    sig0[8:] = 1e4            # thin | thick joint between cells 7 and 8
    p.sigma0 = sig0
    p.tau_num_C = C
    return p


def _T():
    T = np.full(16, 1e-3)
    T[:8] = 0.5              # uniform hot side: the only contrast is at the joint
    return T


def test_reduces_to_tau_without_C_or_contrast():
    T = _T()
    for C in (0.0, 1e3):
        prob = O.OracleProblem(_joint_slab(C))
        rate = 1.0
        for c in (0, 7, 8, 15):
            for g in range(4):
                x = prob.p.dt * rate * O.sigma_group(prob, c, g, T[c])
                xn = O.x_num(prob, T, c, g)
                if C == 0.0:
                    assert xn == x
                else:
                    assert 0.0 < xn <= x
    # uniform temperature: no contrast, tau_num = tau for any C
    prob = O.OracleProblem(_joint_slab(1e5))
    Tu = np.full(16, 0.5)
    for c in range(16):
        for g in range(4):
            assert O.x_num(prob, Tu, c, g) == prob.p.dt * O.sigma_group(prob, c, g, 0.5)


def test_sampled_fraction_grows_with_C_at_a_joint():
    T = _T()
    c, g = 7, 0          # hot thin side of the joint, next to the cold cell 8
    prev = None
    for C in (0.0, 1e1, 1e3, 1e5, 1e9):
        prob = O.OracleProblem(_joint_slab(C))
        e = np.exp(-O.x_num(prob, T, c, g))
        if prev is not None:
            assert e >= prev
        prev = e
    assert prev > 0.999          # C -> infinity: the whole wave part is sampled
    # tau_num - tau equals C J dt with J = |T_c - T_n|/(T_c + T_n) of the sharpest face
    prob = O.OracleProblem(_joint_slab(1e3))
    x = prob.p.dt * O.sigma_group(prob, c, g, T[c])
    xn = O.x_num(prob, T, c, g)
    J = abs(T[c] - T[c + 1]) / (T[c] + T[c + 1])
    assert abs((prob.p.dt / xn - prob.p.dt / x) - 1e3 * J * prob.p.dt) <= 1e-12 * (prob.p.dt / xn)


def test_step_with_tau_num_conserves_energy_and_samples_more_at_the_joint():
    res = {}
    for C in (0.0, 1e3):
        p = _joint_slab(C)
        p.bc = [I.BC_BLACKBODY, I.BC_REFLECT, 0, 0]
        prob = O.OracleProblem(p)
        st = O.initial_state(prob)
        st = O.State(p, _T(), st.rho, st.rho.copy(), st.particles, 0)
        rho = np.array([O.phi(prob, g, st.T[c]) for c in range(16) for g in range(4)])
        st = O.State(p, st.T, rho, rho.copy(), st.particles, 0)
        st2, tal, _, status = O.step(prob, st)
        assert status == 0
        E0, E1 = tal.c.E_rad0 + tal.c.E_mat0, tal.c.E_rad1 + tal.c.E_mat1
        r = E1 - E0 - (tal.c.bnd_in_macro + tal.c.bnd_in_part - tal.c.bnd_out_part + tal.c.src_in)
        assert abs(r) <= 1e-12 * E1
        res[C] = tal.N.reshape(-1, 4)[:16].copy()
    # more particles sampled in the joint cells, the same elsewhere
    assert res[1e3][7].sum() > res[0.0][7].sum()
    assert np.array_equal(res[1e3][:5], res[0.0][:5])
