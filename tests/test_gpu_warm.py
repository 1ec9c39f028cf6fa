"""FP32 warm start of the mixed-precision source iteration (App. B,
Algorithm 2): FP32 iterates from T^n, then FP64 iterates to si_tol.  The
fixed point is the FP64 iteration's, so one step from the same state gives
the temperatures and radiation energies of the FP64-only iteration to within
the iteration's convergence (both stop within si_tol = 1e-12 of the fixed
point); the particle phase is the same in both.  Also: the counts of FP32
and FP64 iterates, the default switch on problem size, ensembles, and the
energy ledger."""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_RTOL = 1e-10


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def evolved_state(p, steps):
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(steps):
        st, _, _, _ = O.step(op, st)
    return st


def one_step(B, p, st, warm):
    q = p.replace(precision=I.MIXED, si_warm32=warm)
    sim = B.Simulation(q)
    sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=st.step)
    sim.step(1)
    return sim.tallies(), sim.get_state()


def ledger_residual(t):
    E0, E1 = t["E_rad0"] + t["E_mat0"], t["E_rad1"] + t["E_mat1"]
    return E1 - E0 - (t["bnd_in_macro"] + t["bnd_in_part"] - t["bnd_out_part"] + t["src_in"]), E1


def check_same_fixed_point(p, ton, gon, toff, goff):
    assert ton["status_bits"] == 0 and toff["status_bits"] == 0
    assert ton["si_iters32"] > 0 and toff["si_iters32"] == 0
    assert ton["n_born"] == toff["n_born"] and gon["n"] == goff["n"]
    np.testing.assert_allclose(gon["T"], goff["T"], rtol=T_RTOL, atol=0)
    rs = np.abs(goff["rho"].reshape(p.ncell, p.G)).sum(1, keepdims=True)
    assert (np.abs(gon["rho"] - goff["rho"]).reshape(p.ncell, p.G) <= T_RTOL * rs + 1e-300).all()
    for t in (ton, toff):
        r, E1 = ledger_residual(t)
        assert abs(r) <= 1e-12 * E1


def test_warm_start_slab(B):
    p = I.small_multigroup(nx=24, G=6, omega_ref=1e-6)
    st = evolved_state(p, 3)
    ton, gon = one_step(B, p, st, 1)
    toff, goff = one_step(B, p, st, -1)
    check_same_fixed_point(p, ton, gon, toff, goff)
    # and the oracle's FP64 step (mixed-precision tolerance of T)
    st2, _, _, status = O.step(O.OracleProblem(p), st)
    assert status == 0
    np.testing.assert_allclose(gon["T"], st2.T, rtol=1e-5)


def test_warm_start_larsen_photoionisation(B):
    # sig_law 1: the photo-ionisation factor in the FP32 opacity
    p = I.larsen_slab(G=12, omega_frac=2e-5)
    st = evolved_state(p, 4)
    check_same_fixed_point(p, *one_step(B, p, st, 1), *one_step(B, p, st, -1))


def test_warm_start_olson_foam(B):
    # sig_law 2 and the T-dependent heat capacity (cv_law 1)
    p = I.olson_slab(G=10, omega_frac=1e-3)
    st = evolved_state(p, 2)
    check_same_fixed_point(p, *one_step(B, p, st, 1), *one_step(B, p, st, -1))


def test_warm_start_checkerboard_2d(B):
    # the face pass of 2D in FP32
    p = I.small_checkerboard(n=16, G=4, omega_ref=2e-7)
    st = evolved_state(p, 2)
    check_same_fixed_point(p, *one_step(B, p, st, 1), *one_step(B, p, st, -1))


def test_warm_start_checkerboard_3d(B):
    p = I.checkerboard_3d(n=8, G=8, block=2, patch=2, omega_ref=5e-8)
    p.particle_capacity = 1 << 18
    st = evolved_state(p, 2)
    check_same_fixed_point(p, *one_step(B, p, st, 1), *one_step(B, p, st, -1))


def test_warm_start_ensemble(B):
    probs = []
    for m in range(3):
        p = I.small_multigroup(nx=[12, 20, 7][m], G=[4, 6, 3][m], omega_ref=[1e-6, 2e-6, 5e-7][m])
        p.sigma0 = np.full(p.nx, [1e2, 30.0, 3e2][m])
        p.instance = m
        p.seed = 7
        probs.append(p)
    out = {}
    for warm in (1, -1):
        ens = B.Simulation([p.replace(precision=I.MIXED, si_warm32=warm) for p in probs])
        ens.step(1)
        out[warm] = [(ens.tallies(member=m), ens.get_state(member=m)) for m in range(3)]
    for m, p in enumerate(probs):
        check_same_fixed_point(p, *out[1][m], *out[-1][m])


def test_warm_start_default_follows_problem_size(B):
    # 2^17 (cell, group) pairs and more: on by default in mixed precision;
    # never in FP64
    big = I.checkerboard_2d(n=128, G=30)
    big.particle_capacity = 1 << 21
    s = I.synthetic_state(big, 200000, seed=3, front=0.35)
    for prec, want in ((I.MIXED, True), (I.FP64, False)):
        sim = B.Simulation(big.replace(precision=prec))
        sim.set_state(s["T"], s["rho"], s["rho_h"], s["particles"], step=s["step"])
        sim.step(1)
        t = sim.tallies()
        assert t["status_bits"] == 0
        assert (t["si_iters32"] > 0) == want
        assert t["si_iters"] >= 2
    small = I.small_multigroup(nx=24, G=6).replace(precision=I.MIXED)
    sim = B.Simulation(small)
    sim.step(1)
    assert sim.tallies()["si_iters32"] == 0
