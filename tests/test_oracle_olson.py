"""Pins of the Olson carbon-hydrogen foam materials (Sec. 3.5) in the oracle:
the heat capacity of Eq. cvolson against its material energy (the closed
antiderivative e(T) = K [T + (T + chi) alpha] checked by quadrature of
rho C_v, which also checks the paper's alpha' against alpha), its limits, the
structure of the three-band opacity kappa(nu, T) (exact power laws in nu and
in the T factors, the 1e7 cap of the low band), the converged source
iteration against the material equation with the T-dependent heat capacity,
the energy ledger with the time-limited source, and a Planck equilibrium
held fixed."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def _op(**kw):
    p = I.olson_slab(G=12)
    for k, v in kw.items():
        setattr(p, k, v)
    return p, O.OracleProblem(p)


def test_material_energy_is_the_antiderivative_of_the_heat_capacity():
    p, op = _op()
    for T1, T2 in [(1e-3, 0.01), (0.01, 0.05), (0.05, 0.2), (0.2, 1.0), (1.0, 5.0)]:
        q, err = integrate.quad(lambda T: O.heat_capacity(op, 0, T), T1, T2, epsabs=0, epsrel=1e-13, limit=200)
        de = O.mat_energy(op, 0, T2) - O.mat_energy(op, 0, T1)
        assert abs(de - q) <= 1e-11 * abs(q), (T1, T2, de, q)


def test_heat_capacity_limits():
    p, op = _op()
    K = p.cv[0]
    # T -> 0: alpha and alpha' vanish (alpha ~ e^{-chi/2T}); e -> 0
    assert abs(O.heat_capacity(op, 0, 1e-3) - K) <= 1e-12 * K
    assert O.mat_energy(op, 0, 1e-3) == pytest.approx(K * 1e-3, rel=1e-12)
    # T -> infinity: alpha -> (sqrt 5 - 1)/2, alpha' -> 0
    golden = (math.sqrt(5.0) - 1.0) / 2.0
    assert O.heat_capacity(op, 0, 1e4) == pytest.approx(K * (1.0 + golden), rel=1e-4)
    # and the constant law is unchanged
    q = O.OracleProblem(p.replace(cv_law=0))
    assert O.mat_energy(q, 0, 0.7) == K * 0.7 and O.heat_capacity(q, 0, 0.7) == K


def test_opacity_bands_follow_their_power_laws():
    p, op = _op()
    rho = p.sigma0[0]
    # low band: 1e9 T^2, capped at 1e7 (T >= 0.1), independent of nu
    for T in (0.01, 0.05):
        assert O.sigma(op, 0, 0.004, T) == pytest.approx(rho * 1e9 * T * T, rel=1e-14)
        assert O.sigma(op, 0, 0.002, T) == O.sigma(op, 0, 0.004, T)
    assert O.sigma(op, 0, 0.004, 0.5) == pytest.approx(rho * 1e7, rel=1e-15)
    # middle band: nu^-2, and kappa (1 + 200 T^1.5) independent of T
    T = 0.07
    assert O.sigma(op, 0, 0.1, T) / O.sigma(op, 0, 0.05, T) == pytest.approx(0.25, rel=1e-14)
    k1 = O.sigma(op, 0, 0.1, 0.02) * (1 + 200 * 0.02 ** 1.5)
    k2 = O.sigma(op, 0, 0.1, 0.3) * (1 + 200 * 0.3 ** 1.5)
    assert k1 == pytest.approx(k2, rel=1e-14)
    # upper band: both terms go as nu^-2.5, so at any fixed T the band is one power law
    for T in (0.0, 0.05, 0.4):
        r = O.sigma(op, 0, 2.0, T) / O.sigma(op, 0, 1.0, T)
        assert r == pytest.approx(2.0 ** -2.5, rel=1e-14)
    # the band edges are where the paper puts them: 0.008 and 0.3 keV
    assert O.sigma(op, 0, 0.008, 0.05) == O.sigma(op, 0, 0.001, 0.05)
    assert O.sigma(op, 0, 0.3, 0.05) == pytest.approx(O.sigma(op, 0, 0.15, 0.05) / 4.0, rel=1e-14)


def test_source_iteration_satisfies_the_material_equation():
    # no particles (wave part only), a hot/cold profile, one step: the
    # converged T^{n+1} satisfies e(T^{n+1}) - e(T^n) = dt sum_g sigma_g (rho_g - Phi_g)
    p, op = _op(omega_ref=0.0, src_on=0.0)
    p.T0 = np.linspace(0.3, 0.01, p.nx)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    st, tal, _, status = O.step(op, st)
    assert status == 0 and tal.c.si_iters > 1
    G, n = p.G, p.nx
    T1, rho1 = st.T, st.rho.reshape(n, G)
    for c in range(0, n, 7):
        em = sum(p.dt / p.eps ** 2 * O.sigma_group(op, c, g, T1[c]) * (rho1[c, g] - O.phi(op, g, T1[c]))
                 for g in range(G))
        e1, e0 = O.mat_energy(op, c, T1[c]), O.mat_energy(op, c, p.T0[c])
        assert abs(e1 - (e0 + em)) <= 1e-9 * e1, (c, e1, e0 + em)


def test_olson_steps_conserve_energy_and_the_source_stops():
    p = I.olson_slab(G=12, omega_frac=1e-5)
    p.src_t_end = 3 * p.dt          # source on for steps 0, 1, 2
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for n in range(5):
        st, tal, _, status = O.step(op, st)
        assert status == 0
        c = tal.c
        E0, E1 = c.E_rad0 + c.E_mat0, c.E_rad1 + c.E_mat1
        r = E1 - E0 - (c.bnd_in_macro + c.bnd_in_part - c.bnd_out_part + c.src_in)
        assert abs(r) <= 1e-12 * E1
        assert (c.src_in > 0.0) == (n < 3)
    assert st.particles.n > 1000
    assert st.T[0] > 0.01 and np.all(st.T > 0.0)


def test_equilibrium_held_with_the_foam_heat_capacity():
    p, op = _op(omega_ref=0.0, src_on=0.0)
    p.T0 = np.full(p.nx, 0.2)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(2):
        st, _, _, status = O.step(op, st)
        assert status == 0
    np.testing.assert_allclose(st.T, 0.2, rtol=1e-12)
