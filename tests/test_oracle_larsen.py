"""Pins of the Larsen opacity law sigma = gamma0 (1 - e^{-nu/T}) nu^-3
(Sec. 3.3, photo-ionisation absorption) and of the Larsen problem set-up:
the limits the factor fixes (nu >> T: the bare nu^-3 law; nu << T: gamma0
nu^-2/T; nu = T ln 2: half of it), the cap, the Simpson group opacity
reducing to the pointwise value in a narrow group, and energy conservation
of steps through the thin/thick/thin slab with a free right side."""
import math

import numpy as np

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def _prob(**kw):
    p = I.larsen_slab()
    for k, v in kw.items():
        setattr(p, k, v)
    return O.OracleProblem(p)


def test_pointwise_limits_of_the_photo_ionisation_factor():
    prob = _prob()
    c = 0                    # gamma0 = 1 there
    for T in (1e-3, 0.1, 1.0):
        nu = 40.0 * T
        assert abs(O.sigma(prob, c, nu, T) - nu ** -3) <= 1e-15 * nu ** -3 + 1e-300
        nu = 1e-6 * T
        s = O.sigma(prob, c, nu, T)
        if s < 1e6:          # below the cap
            assert abs(s - nu ** -2 / T) <= 1e-6 * nu ** -2 / T
        nu = T * math.log(2.0)
        s = O.sigma(prob, c, nu, T)
        if s < 1e6:
            assert abs(s - 0.5 * nu ** -3) <= 1e-14 * nu ** -3
    # the cap applies after the factor
    prob = _prob(sig_cap=10.0)
    assert O.sigma(prob, 100, 0.01, 1.0) == 10.0


def test_power_law_unchanged_without_the_factor():
    p = I.larsen_slab()
    q = p.replace(sig_law=0)
    a, b = O.OracleProblem(p), O.OracleProblem(q)
    for nu, T in [(0.5, 0.2), (3.0, 1.0), (0.05, 0.01)]:
        assert O.sigma(a, 0, nu, T) == O.sigma(b, 0, nu, T) * -math.expm1(-nu / T)


def test_group_opacity_of_a_narrow_group_is_pointwise():
    p = I.larsen_slab(G=24)
    edges = np.array([0.999, 1.001])
    p = p.replace(G=1, nu_edges=edges)
    prob = O.OracleProblem(p)
    T = 0.3
    sg = O.sigma_group(prob, 0, 0, T)
    s_mid = O.sigma(prob, 0, 1.0, T)
    assert abs(sg - s_mid) <= 1e-5 * s_mid


def test_larsen_steps_conserve_energy():
    p = I.larsen_slab(G=12, omega_frac=2e-5)
    prob = O.OracleProblem(p)
    st = O.initial_state(prob)
    for n in range(6):
        st, tal, _, status = O.step(prob, st)
        assert status == 0
        E0, E1 = tal.c.E_rad0 + tal.c.E_mat0, tal.c.E_rad1 + tal.c.E_mat1
        r = E1 - E0 - (tal.c.bnd_in_macro + tal.c.bnd_in_part - tal.c.bnd_out_part + tal.c.src_in)
        assert abs(r) <= 1e-12 * E1
    assert st.particles.n > 100
    assert st.T[0] > 1e-3 and np.all(st.T > 0.0)
