"""Mixed precision (FP32 particle state and arithmetic, FP64 tallies, FP64
source iteration) against the FP64 oracle, one step from identical states.

Stated error of the mixed build: unflipped particles end within 2e-5 of the
slab length (positions), 1e-5 relative (frequency, time) and 1e-5 (direction cosines);
at most 2e-3 of the particles take a different event (an FP32 near-tie);
T after the step within 1e-5 relative; the energy ledger still closes to
roundoff because every tally uses the particle's own (FP32) weight."""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FLIPS = 2e-3
X_TOL = 2e-5
REL_TOL = 1e-5
T_TOL = 1e-5
DIR_TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def run_gpu(B, p, st, op, shape=None):
    pm = p.replace(precision=I.MIXED)
    sim = B.Simulation(pm)
    if shape is not None:
        sim.set_launch(*shape)
    sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=st.step)
    _, n_new, _ = O.birth_counts(op, st.T, st.rho_h)
    sim.attach_records(st.particles.n + n_new + 8)
    sim.step(1)
    t = sim.tallies()
    g = sim.get_state()
    rg = sim.records(t["n_in"] + t["n_born"])
    assert t["status_bits"] == 0
    return t, g, rg


def run_pair(B, p, st, op, shape=None):
    t, g, rg = run_gpu(B, p, st, op, shape)
    st2, tal, ro, status = O.step(op, st, records=True)
    assert status == 0
    return t, g, rg, st2, tal, ro


def check(p, t, g, rg, st2, tal, ro):
    assert t["n_born"] == tal.c.n_born
    np.testing.assert_array_equal(rg["id"], ro["id"])
    same = (rg["fate"] == ro["fate"]) & (rg["cell1"] == ro["cell1"]) & (rg["nseg"] == ro["nseg"])
    flips = int((~same).sum())
    assert flips <= max(2, FLIPS * len(rg)), (flips, len(rg))
    L = p.nx * p.dx
    assert np.abs(rg["x"][same] - ro["x"][same]).max() <= X_TOL * L
    if p.dim >= 2:
        assert np.abs(rg["y"][same] - ro["y"][same]).max() <= X_TOL * L
    if p.dim == 3:
        assert np.abs(rg["z"][same] - ro["z"][same]).max() <= X_TOL * L
        assert np.abs(rg["oz"][same] - ro["oz"][same]).max() <= DIR_TOL
    assert np.abs(rg["ox"][same] - ro["ox"][same]).max() <= DIR_TOL
    if p.dim >= 2:
        assert np.abs(rg["oy"][same] - ro["oy"][same]).max() <= DIR_TOL
    if not p.grey:
        np.testing.assert_allclose(rg["nu"][same], ro["nu"][same], rtol=REL_TOL)
    np.testing.assert_allclose(rg["w"], ro["w"], rtol=1e-7)
    assert np.abs(rg["t_end"][same] - ro["t_end"][same]).max() <= REL_TOL * p.dt
    np.testing.assert_allclose(g["T"], st2.T, rtol=T_TOL)
    E0, E1 = t["E_rad0"] + t["E_mat0"], t["E_rad1"] + t["E_mat1"]
    resid = E1 - E0 - (t["bnd_in_macro"] + t["bnd_in_part"] - t["bnd_out_part"] + t["src_in"])
    assert abs(resid) <= 1e-12 * E1
    return flips


def test_mixed_multigroup_slab(B):
    p = I.small_multigroup(nx=24, G=6, omega_ref=1e-6)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(3):
        st, _, _, _ = O.step(op, st)
    check(p, *run_pair(B, p, st, op))


def test_mixed_checkerboard_2d(B):
    p = I.small_checkerboard(n=16, G=4, omega_ref=2e-7)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(2):
        st, _, _, _ = O.step(op, st)
    check(p, *run_pair(B, p, st, op))


def test_mixed_larsen_slab(B):
    # photo-ionisation opacity (Sec. 3.3), paper units, tau_num at the joints
    p = I.larsen_slab(G=12, omega_frac=2e-5)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(4):
        st, _, _, _ = O.step(op, st)
    check(p, *run_pair(B, p, st, op))


@pytest.fixture(scope="module")
def full_size_slab():
    # the 200x30 slab from the benchmark's 1e6-particle synthetic state, and
    # the oracle's step from it (computed once for every launch shape)
    p = I.multigroup_slab()
    s = I.synthetic_state(p, 1_000_000, seed=3)
    op = O.OracleProblem(p)
    st = O.State(p, s["T"], s["rho"], s["rho_h"], O.ParticleSet.from_arrays(s["particles"]), s["step"])
    st2, tal, ro, status = O.step(op, st, records=True)
    assert status == 0
    return p, op, st, st2, tal, ro


# the default shape and those the autotuner picks on this workload (the
# benchmark times the one it picks)
@pytest.mark.parametrize("shape", [None, (512, 4, 0), (256, 2, 0), (128, 1, 0)])
def test_mixed_full_size_slab(B, full_size_slab, shape):
    p, op, st, st2, tal, ro = full_size_slab
    t, g, rg = run_gpu(B, p, st, op, shape)
    flips = check(p, t, g, rg, st2, tal, ro)
    assert flips < 2000


@pytest.mark.parametrize("case", ["slab", "checkerboard"])
def test_mixed_wave_flux_fp32(B, case):
    # the mixed build's wave-part flux is computed in FP32 from FP32 copies of
    # its inputs: within 2e-5 of the oracle's FP64 flux relative to the
    # largest flux of the group (C5's closed form cancels near x = 1 and the
    # van Leer slopes difference neighbouring rho^h)
    if case == "slab":
        p = I.small_multigroup(nx=24, G=6, omega_ref=1e-6)
    else:
        p = I.small_checkerboard(n=16, G=4, omega_ref=2e-7)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(3):
        st, _, _, _ = O.step(op, st)
    sim = B.Simulation(p.replace(precision=I.MIXED))
    sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=st.step)
    sim.step(1)
    _, tal, _, status = O.step(op, st)
    assert status == 0
    Fg = sim.device_array("Fwave").cpu().numpy().reshape(-1, p.G)
    Fo = tal.Fwave.reshape(-1, p.G)
    scale = np.abs(Fo).max(0, keepdims=True) + 1e-300
    assert (np.abs(Fg - Fo) <= 2e-5 * scale).all(), np.abs((Fg - Fo) / scale).max()


def test_mixed_energy_conserved_over_steps(B):
    p = I.small_checkerboard(n=16, G=4, omega_ref=2e-7).replace(precision=I.MIXED)
    p.src_on = 0.0
    p.T0 = np.linspace(0.2, 1.0, p.ncell)
    p.particle_capacity = 1 << 21      # ~5.7e5 births in the first step
    sim = B.Simulation(p)
    for _ in range(4):
        sim.step(1)
        t = sim.tallies()
        assert t["status_bits"] == 0
        E0, E1 = t["E_rad0"] + t["E_mat0"], t["E_rad1"] + t["E_mat1"]
        assert abs(E1 - E0) <= 1e-12 * E0
    assert t["n_in"] > 1000


def test_mixed_steps_across_the_survivor_sort(B):
    # every step sorts the survivors by bin: after 8 steps the particles
    # still match the oracle's one by one (by identity: position, direction,
    # frequency, weight, cell)
    p = I.small_multigroup(nx=24, G=6, omega_ref=1e-6).replace(precision=I.MIXED)
    p.particle_capacity = 1 << 20
    op = O.OracleProblem(p.replace(precision=I.FP64))
    st = O.initial_state(op)
    sim = B.Simulation(p)
    for n in range(8):
        sim.step(1)
        st, tal, _, status = O.step(op, st)
        assert status == 0 and sim.tallies()["status_bits"] == 0
    g = sim.get_state()
    np.testing.assert_allclose(g["T"], st.T, rtol=T_TOL * 10)
    pg, po = g["particles"], st.particles.view()
    assert abs(g["n"] - st.particles.n) <= max(2, FLIPS * st.particles.n)
    common, ig, io = np.intersect1d(pg["id"], po["id"], return_indices=True)
    assert len(common) >= (1 - FLIPS) * st.particles.n and len(common) > 1000
    assert (pg["cell"][ig] == po["cell"][io]).mean() > 1 - FLIPS
    same = pg["cell"][ig] == po["cell"][io]
    L = p.nx * p.dx
    assert np.abs(pg["x"][ig][same] - po["x"][io][same]).max() <= 10 * X_TOL * L
    np.testing.assert_allclose(pg["ox"][ig], po["ox"][io], rtol=0, atol=10 * DIR_TOL)
    np.testing.assert_allclose(pg["nu"][ig], po["nu"][io], rtol=10 * REL_TOL)
    np.testing.assert_allclose(pg["w"][ig], po["w"][io], rtol=REL_TOL)   # scaled survivors: the bin factor to mixed precision
    # the survivors are held in bin order after every step
    key = pg["cell"] * p.G + pg["grp"]
    assert (np.diff(key) >= 0).all()


def test_capacity_overflow_across_sorting_steps_stays_consistent(B):
    # more particles than the particle buffers hold: the step is flagged
    # (status bit), a particle without a slot is dropped (its energy stays
    # with the wave part) and the sort moves only the stored survivors, so
    # the live particles stay a consistent set (valid bins, bin order, no
    # slot left unwritten)
    p = I.small_checkerboard(n=16, G=4, omega_ref=2e-7).replace(precision=I.MIXED)
    p.src_on = 0.0
    p.T0 = np.linspace(0.2, 1.0, p.ncell)
    p.particle_capacity = 1 << 16
    sim = B.Simulation(p)
    bits = 0
    for _ in range(8):
        sim.step(1)
        bits |= sim.tallies()["status_bits"]
    assert bits & 1   # UGKWP_ST_CAPACITY
    g = sim.get_state()
    assert 0 < g["n"] <= p.particle_capacity
    par = g["particles"]
    assert (par["cell"] >= 0).all() and (par["cell"] < p.ncell).all()
    assert (par["grp"] >= 0).all() and (par["grp"] < p.G).all()
    assert np.isfinite(par["w"]).all() and (par["w"] > 0).all()
    assert len(np.unique(par["id"])) == g["n"]
    assert (np.diff(par["cell"] * p.G + par["grp"]) >= 0).all()
    assert np.isfinite(g["T"]).all() and (g["T"] > 0).all()
