"""Ensembles of independent problems advanced together in one step.

Members differ in cells, groups, opacity scale, boundary temperature,
reference weight and instance number; each member must reproduce the same
problem run alone (same particle identities and random streams, so the same
births, survivors and temperatures up to the summation order of FP64
atomics), and its energy ledger must close.  Also the oracle agrees with a
member directly."""
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


def slab_members(k, precision=I.FP64):
    probs = []
    for m in range(k):
        j = m % 4
        p = I.small_multigroup(nx=[12, 20, 7, 31][j], G=[4, 6, 3, 8][j],
                               omega_ref=[1e-6, 2e-6, 5e-7, 3e-6][j])
        p.sigma0 = np.full(p.nx, [1e2, 30.0, 3e2, 10.0][j])
        p.bcT = [[1.0, 0.7, 1.5, 0.9][j], 0, 0, 0]
        p.instance = m
        p.seed = 7
        p.precision = precision
        probs.append(p)
    return probs


def compare_member_with_alone(B, probs, steps, T_rtol=T_RTOL):
    ens = B.Simulation(probs)
    ens.step(steps)
    for m, p in enumerate(probs):
        alone = B.Simulation(p)
        alone.step(steps)
        a, e = alone.get_state(), ens.get_state(member=m)
        ta, te = alone.tallies(), ens.tallies(member=m)
        assert te["status_bits"] == 0 and ta["status_bits"] == 0
        assert e["n"] == a["n"] and te["n_born"] == ta["n_born"]
        np.testing.assert_allclose(e["T"], a["T"], rtol=T_rtol)
        ia, ie = np.argsort(a["particles"]["id"]), np.argsort(e["particles"]["id"])
        np.testing.assert_array_equal(a["particles"]["id"][ia], e["particles"]["id"][ie])
        np.testing.assert_allclose(e["particles"]["x"][ie], a["particles"]["x"][ia], rtol=0, atol=1e-12)
        E0, E1 = te["E_rad0"] + te["E_mat0"], te["E_rad1"] + te["E_mat1"]
        r = E1 - E0 - (te["bnd_in_macro"] + te["bnd_in_part"] - te["bnd_out_part"] + te["src_in"])
        assert abs(r) <= 1e-12 * E1
    return ens


def test_ensemble_members_equal_single_runs_fp64(B):
    compare_member_with_alone(B, slab_members(5), 4)


def test_ensemble_members_equal_single_runs_mixed(B):
    compare_member_with_alone(B, slab_members(4, I.MIXED), 3)


def test_ensemble_2d_members(B):
    probs = [I.small_checkerboard(n=8, G=3, omega_ref=1e-6), I.small_checkerboard(n=12, G=4, omega_ref=4e-7)]
    for m, p in enumerate(probs):
        p.instance = m
    compare_member_with_alone(B, probs, 2)


def test_ensemble_member_matches_oracle(B):
    probs = slab_members(3)
    ens = B.Simulation(probs)
    m = 1
    op = O.OracleProblem(probs[m])
    st = O.initial_state(op)
    for _ in range(3):
        ens.step(1)
        st, _, _, status = O.step(op, st)
        assert status == 0
    g = ens.get_state(member=m)
    np.testing.assert_allclose(g["T"], st.T, rtol=1e-9)
    assert g["n"] == st.particles.n


def test_ensemble_of_uneven_members_many(B):
    # many members with very different particle counts in one launch
    probs = []
    for m in range(24):
        p = I.small_multigroup(nx=8 + 5 * m, G=3 + (m % 5), omega_ref=10 ** (-5 - (m % 3)))
        p.instance = m
        probs.append(p)
    ens = B.Simulation(probs)
    ens.step(3)
    counts = [ens.get_state(member=m)["n"] for m in range(len(probs))]
    assert max(counts) > 20 * max(1, min(counts))
    for m in (0, 7, 23):
        alone = B.Simulation(probs[m])
        alone.step(3)
        np.testing.assert_allclose(ens.get_state(member=m)["T"], alone.get_state()["T"], rtol=T_RTOL)
