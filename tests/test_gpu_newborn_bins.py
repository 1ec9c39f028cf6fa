"""Newborn bins of the slab survivor kernel against the oracle.

The kernel finds a newborn's bin (the largest b with off[b] <= j for its
birth ordinal j, Eq. IhpFormula's counts scanned) from a shared-memory table
of every 32nd offset and one warp-wide load of a 32-bin segment; above
32768 bins it searches the offsets in global memory.  Both are checked on
states whose births are spread thinly over many segments, so a warp's 32
ordinals span several segments and many bins have no newborn: every
newborn's identity (step, bin, ordinal in the bin) and its birth state must
equal the oracle's, particle by particle, and the step must stay within the
mixed build's stated error."""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def one_step(B, p, s):
    op = O.OracleProblem(p)
    st = O.State(p, s["T"], s["rho"], s["rho_h"], O.ParticleSet.from_arrays(s["particles"]), s["step"])
    pm = p.replace(precision=I.MIXED)
    sim = B.Simulation(pm)
    sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=st.step)
    _, n_new, _ = O.birth_counts(op, st.T, st.rho_h)
    sim.attach_records(st.particles.n + n_new + 8)
    sim.step(1)
    t = sim.tallies()
    rg = sim.records(t["n_in"] + t["n_born"])
    st2, tal, ro, status = O.step(op, st, records=True)
    assert status == 0 and t["status_bits"] == 0
    return t, sim.get_state(), rg, st2, tal, ro, n_new


def check(p, t, g, rg, st2, tal, ro, n_new, min_bins):
    assert t["n_born"] == tal.c.n_born == n_new
    np.testing.assert_array_equal(rg["id"], ro["id"])
    born = rg["id"] >> np.uint64(44) == np.uint64(st2.step - 1)
    assert born.sum() == n_new
    bins = (rg["id"][born] >> np.uint64(20)) & np.uint64((1 << 24) - 1)
    assert len(np.unique(bins)) >= min_bins   # births spread over many bins
    same = (rg["fate"] == ro["fate"]) & (rg["cell1"] == ro["cell1"]) & (rg["nseg"] == ro["nseg"])
    assert (~same).sum() <= max(2, 2e-3 * len(rg))
    nb = born & same
    assert np.abs(rg["x"][nb] - ro["x"][nb]).max() <= 2e-5 * p.nx * p.dx
    np.testing.assert_allclose(rg["nu"][nb], ro["nu"][nb], rtol=1e-5)
    np.testing.assert_allclose(rg["w"][born], ro["w"][born], rtol=1e-7)
    np.testing.assert_allclose(g["T"], st2.T, rtol=1e-5)


def sparse_state(p, n_particles, seed):
    # a hot region over most of the slab and a thin wave part: a few
    # newborns in each of many bins, none in most
    s = I.synthetic_state(p, n_particles, seed=seed, front=0.9, wave_fraction=0.002)
    return s


def test_newborn_bins_many_segments(B):
    # 200 x 30 bins: 188 segments of 32 in the shared-memory table
    p = I.multigroup_slab(nx=200, G=30, omega_ref=3e-7)
    p.particle_capacity = 1 << 20
    s = sparse_state(p, 20000, seed=5)
    check(p, *one_step(B, p, s), min_bins=200)


def test_newborn_bins_global_search(B):
    # 2048 x 20 = 40960 cell bins: above the table's 32768, the search runs on
    # the offsets in global memory (v dt / dx = 0.2 keeps the survivor kernel)
    p = I.multigroup_slab(nx=2048, G=20, omega_ref=3e-7)
    p.particle_capacity = 1 << 20
    s = sparse_state(p, 20000, seed=6)
    check(p, *one_step(B, p, s), min_bins=200)
