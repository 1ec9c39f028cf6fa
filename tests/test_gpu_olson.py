"""The Olson carbon-hydrogen foam (Sec. 3.5: three-band opacity kappa(nu, T),
the heat capacity of Eq. cvolson, the source B(0.5 keV) e^{-693 x^3} for
ct <= 2) on the GPU against the oracle through the C ABI: one step from an
identical state with per-particle records (FP64: element by element with
event flips counted; mixed precision: to its stated error), and steps from
the initial state across the source's end time (T to the FP64 tolerance,
energy ledger closed, no source energy after the end time)."""
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


def foam(**kw):
    p = I.olson_slab(G=12, omega_frac=1e-5)
    p.particle_capacity = 1 << 18
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_olson_step_parity(B):
    t, tal = check_step(B, foam(), 3)
    assert t["n_in"] > 500


def test_olson_step_parity_warm(B):
    # a warm foam: the middle and upper opacity bands and the heat capacity's
    # alpha terms all matter, and more particles are sampled
    p = foam(T0=np.linspace(0.5, 0.05, 128))
    t, tal = check_step(B, p, 0)
    assert t["n_born"] > 10000


def test_olson_mixed_precision(B):
    p = foam(T0=np.linspace(0.5, 0.05, 128))
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    M.check(p, *M.run_pair(B, p, st, op))


def test_olson_steps_across_the_source_end(B):
    p = foam(src_t_end=3 * I.olson_slab().dt)
    _, st = oracle_run(p, 5)
    sim = B.Simulation(p)
    for n in range(5):
        sim.step(1)
        t = sim.tallies()
        assert t["status_bits"] == 0
        E0, E1 = t["E_rad0"] + t["E_mat0"], t["E_rad1"] + t["E_mat1"]
        resid = E1 - E0 - (t["bnd_in_macro"] + t["bnd_in_part"] - t["bnd_out_part"] + t["src_in"])
        assert abs(resid) <= 1e-12 * E1
        assert (t["src_in"] > 0.0) == (n < 3)
    np.testing.assert_allclose(sim.get_state()["T"], st.T, rtol=T_RTOL)


def test_olson_adjoint_is_refused(B):
    sim = B.Simulation(foam(sig_law=0, sig_p=-3.0, sig_q=-0.5))
    with pytest.raises(Exception, match="heat capacity"):
        sim.tape_buffer(16)
