"""Pins of the oracle's UGKP variant (Sec. 2.2: the specific intensity fully
represented by particles -- every step samples all of the wave part I^h, and
each newborn draws its own free time, instead of the collisionless fraction
e^{-dt/tau} I^h with t_f = dt of UGKWP).

Pinned by what the method fixes: the newborns' collision probability is
1 - e^{-dt/tau} (binomial bounds); in the optically thin limit nothing
collides and UGKP and UGKWP take the same paths; in the thick limit both
leave free transport to the equilibrium flux and agree to O(tau/dt); the
energy ledger closes to roundoff; and a sampled half carries no wave flux."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def one_cell(method, x, n_particles=200_000, seed=3):
    """One grey cell between mirror walls at equilibrium T = 1, dt/tau = x."""
    p = I.grey_slab(nx=1, omega_ref=1.0, seed=seed)
    p.bc = [I.BC_REFLECT] * 4
    p.T0 = np.ones(1)
    p.sigma0 = np.full(1, x / p.dt)        # c = eps = 1: dt/tau = dt sigma
    p.omega_ref = p.dx * 1.0 / n_particles  # rho = a c T^4 = 1
    p.method = method
    p.particle_capacity = 2 * n_particles
    return p


def test_ugkp_newborns_collide_with_probability_one_minus_e():
    x = 0.7
    p = one_cell(I.UGKP, x)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    _, tal, _, status = O.step(op, st)
    assert status == 0
    n = tal.c.n_born
    assert abs(n - 200_000) <= 1
    q = 1.0 - math.exp(-x)
    k = tal.c.n_absorbed
    assert abs(k - n * q) <= 5.0 * math.sqrt(n * q * (1 - q)), (k, n * q)
    assert tal.c.n_survived == n - k          # mirror walls: nobody escapes


def test_ugkwp_newborns_never_collide_in_their_birth_cell():
    # the same cell in UGKWP: only the collisionless fraction e N is born,
    # with t_f = dt, and a single cell has no interface to reset at
    x = 0.7
    p = one_cell(I.UGKWP, x)
    op = O.OracleProblem(p)
    _, tal, _, status = O.step(op, O.initial_state(op))
    assert status == 0
    assert abs(tal.c.n_born - round(200_000 * math.exp(-x))) <= 1
    assert tal.c.n_absorbed == 0


def _run(p, n):
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    tals = []
    for _ in range(n):
        st, tal, _, status = O.step(op, st)
        assert status == 0
        tals.append(tal)
    return st, tals


def test_thin_limit_ugkp_equals_ugkwp():
    # sigma -> 0: e = 1 - O(1e-12), no collisions, the same particles and paths
    base = I.grey_slab(nx=20, omega_ref=2e-5)
    base.sigma0 = np.full(base.nx, 1e-9)
    a, ta = _run(base, 3)
    b, tb = _run(base.replace(method=I.UGKP), 3)
    for x, y in zip(ta, tb):
        assert x.c.n_born == y.c.n_born and x.c.n_absorbed == y.c.n_absorbed == 0
        assert x.c.n_segments == y.c.n_segments
    np.testing.assert_allclose(b.T, a.T, rtol=1e-9)
    np.testing.assert_allclose(b.rho, a.rho, rtol=1e-9, atol=1e-12 * a.rho.max())
    np.testing.assert_allclose(b.particles.view()["x"], a.particles.view()["x"], rtol=0, atol=1e-15)


def test_thick_limit_ugkp_equals_ugkwp_to_tau_over_dt():
    # e ~ 0: UGKWP samples nothing; UGKP samples everything, and it collides
    # in its birth cell within ~tau; both leave the flux to F^eq
    base = I.grey_slab(nx=20, omega_ref=1e-5)
    base.sigma0 = np.full(base.nx, 1e5)       # tau/dt = 1e-2 at dt = 1e-3
    base.T0 = np.linspace(1.0, 0.3, base.nx)
    a, ta = _run(base, 2)
    b, tb = _run(base.replace(method=I.UGKP), 2)
    assert sum(t.c.n_born for t in ta) == 0
    assert sum(t.c.n_born for t in tb) > 20_000
    np.testing.assert_allclose(b.T, a.T, rtol=2e-3)


@pytest.mark.parametrize("make", [
    lambda: I.small_multigroup(nx=16, G=5, omega_ref=5e-6),
    lambda: I.small_checkerboard(n=8, G=3, omega_ref=1e-6),
])
def test_ugkp_energy_ledger_closes(make):
    p = make().replace(method=I.UGKP)
    _, tals = _run(p, 3)
    for tal in tals:
        c = tal.c
        dE = (c.E_rad1 + c.E_mat1) - (c.E_rad0 + c.E_mat0)
        r = dE - (c.bnd_in_macro + c.bnd_in_part - c.bnd_out_part + c.src_in)
        assert abs(r) <= 1e-13 * (c.E_rad1 + c.E_mat1)
    assert sum(t.c.n_absorbed for t in tals) > 0


def test_sampled_half_carries_no_wave_flux():
    # interior bins all sampled (e_eff = -1 marks UGKP's whole wave part):
    # every face between two sampled halves carries no wave flux, and a
    # face whose halves are unsampled (e_eff = 0) carries the UGKS flux
    p = I.small_multigroup(nx=10, G=3)
    p.bc = [I.BC_REFLECT] * 4
    op = O.OracleProblem(p)
    T = np.linspace(0.3, 1.0, p.nx)
    rng = np.random.default_rng(0)
    rho_h = rng.random(p.ncell * p.G)
    e_all = np.full(p.nbins, -1.0)
    F = O.wave_flux(op, T, rho_h, e_all)
    assert not F.any()
    F0 = O.wave_flux(op, T, rho_h, np.zeros(p.nbins))
    assert np.abs(F0).max() > 0
