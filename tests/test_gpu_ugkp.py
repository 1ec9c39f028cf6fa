"""The UGKP variant (Sec. 2.2: all of the wave part sampled, newborns draw
their own free time, sampled halves carry no wave flux) on the GPU against
the oracle through the C ABI: one step from identical states with
per-particle records (FP64: element by element with event flips counted;
mixed precision: to its stated error), and a few steps from the initial
state (T to the FP64 tolerance)."""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

from test_gpu_step import check_step, oracle_run, T_RTOL
import test_gpu_mixed as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def warm_slab(omega_ref=5e-5):
    # a warm medium, so the interior wave part (not only the black-body
    # side) is sampled: step 0 samples all of it, later steps the remainder
    p = I.small_multigroup(nx=24, G=6, omega_ref=omega_ref).replace(method=I.UGKP)
    p.T0 = np.linspace(1.0, 0.2, p.nx)
    return p


@pytest.mark.parametrize("before", [0, 2])
def test_ugkp_step_parity_multigroup_slab(B, before):
    t, tal = check_step(B, warm_slab(), before)
    assert t["n_born"] > (4000 if before == 0 else 200) and t["n_absorbed"] > 100


def test_ugkp_step_parity_checkerboard_2d(B):
    p = I.small_checkerboard(n=16, G=4, omega_ref=4e-7).replace(method=I.UGKP)
    t, tal = check_step(B, p, 2)
    assert t["n_born"] > 1000 and t["n_absorbed"] > 100


def test_ugkp_wave_flux_matches_oracle(B):
    # the flux of the unsampled remainder, with sampled halves contributing none
    p = warm_slab()
    op, st = oracle_run(p, 0)
    sim = B.Simulation(p)
    sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=st.step)
    sim.step(1)
    _, tal, _, _ = O.step(op, st)
    Fw = sim.device_array("Fwave").cpu().numpy()
    scale = np.abs(tal.Fwave).max() + 1e-300
    assert np.abs(Fw - tal.Fwave).max() <= 1e-12 * scale
    # bins with particles on both sides of an interior face: no wave flux
    N = tal.N[: p.ncell * p.G].reshape(p.nx, p.G)
    both = (N[:-1] > 0) & (N[1:] > 0)
    inner = Fw.reshape(p.nx + 1, p.G)[1:-1]
    assert both.any() and not inner[both].any()


@pytest.mark.parametrize("before", [0, 2])
def test_ugkp_mixed_precision_slab(B, before):
    p = warm_slab()
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(before):
        st, _, _, _ = O.step(op, st)
    M.check(p, *M.run_pair(B, p, st, op))


def test_ugkp_steps_from_initial_state(B):
    p = warm_slab(2e-4)
    _, st = oracle_run(p, 4)
    sim = B.Simulation(p)
    sim.step(4)
    g = sim.get_state()
    assert sim.tallies()["status_bits"] == 0
    np.testing.assert_allclose(g["T"], st.T, rtol=T_RTOL)


def test_ugkp_adjoint_is_refused(B):
    p = I.small_multigroup(nx=8, G=3).replace(method=I.UGKP)
    sim = B.Simulation(p)
    with pytest.raises(Exception, match="UGKWP"):
        sim.tape_buffer(16)
