"""Failure detection on the GPU without a GPU fault: each failure is made on
the host (an impossible wait injected through the C ABI, an iteration cap of
one, a non-finite input) and must come back as a status the host reads, with
the device context still usable afterwards."""
import time

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


def small():
    return I.small_multigroup(nx=16, G=4, omega_ref=5e-6)


@pytest.mark.parametrize("make", [small, lambda: I.small_checkerboard(n=8, G=3, omega_ref=1e-6)])
def test_barrier_wait_runs_out_and_is_reported(B, make):
    sim = B.Simulation(make())
    sim.step(1)
    assert sim.tallies()["status_bits"] == 0
    # every barrier also waits for an arrival that never comes: each wait
    # gives up after its bounded number of polls
    sim.set_wait_limit(spins=2000, extra_arrivals=1)
    t0 = time.perf_counter()
    sim.step(1)
    t = sim.tallies()
    assert time.perf_counter() - t0 < 10.0
    assert t["status_bits"] & B.ST_TIMEOUT
    sim.close()
    # the context is still usable
    sim2 = B.Simulation(make())
    sim2.step(2)
    assert sim2.tallies()["status_bits"] == 0
    sim2.close()


def test_wait_limit_alone_does_not_fail_a_step(B):
    sim = B.Simulation(small())
    sim.set_wait_limit(spins=1 << 20, extra_arrivals=0)
    sim.step(2)
    assert sim.tallies()["status_bits"] == 0


def test_iteration_cap_is_reported(B):
    p = small()
    p.si_max_iters = 1
    p.T0 = np.linspace(1.0, 0.05, p.nx)
    sim = B.Simulation(p)
    sim.step(1)
    t = sim.tallies()
    assert t["status_bits"] & B.ST_NOCONV and t["si_iters"] == 1


def test_non_finite_state_is_reported(B):
    p = small()
    T0 = np.full(p.nx, 0.1)
    T0[5] = np.nan
    p.T0 = T0
    try:
        sim = B.Simulation(p)
    except B.UGKWPError:
        return                     # refused at set-up: also a reported failure
    sim.step(1)
    assert sim.tallies()["status_bits"] & B.ST_NONFINITE


def test_tally_log_is_json_lines(B, tmp_path):
    import json
    path = tmp_path / "steps.jsonl"
    sim = B.Simulation(small())
    for k in range(3):
        sim.step(1)
        sim.log_tallies(str(path), run="log-test")
    rows = [json.loads(line) for line in path.read_text().splitlines()]
    assert [r["step"] for r in rows] == [1, 2, 3]
    for r in rows:
        assert r["status_bits"] == 0 and r["run"] == "log-test"
        assert abs(r["ledger_residual"]) <= 1e-12 * (r["E_rad1"] + r["E_mat1"])


def test_identity_space_limit_is_flagged(B):
    # a newborn's identity holds its birth step in 20 bits: step 2^20 - 1 still
    # samples; the next step samples nothing and sets the status bit (the
    # oracle does the same); a state may not be set past the limit
    p = I.small_multigroup(nx=12, G=4, omega_ref=1e-6)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    st, _, _, _ = O.step(op, st)
    sim = B.Simulation(p)
    last = (1 << 20) - 1
    sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=last)
    sim.step(1)
    t = sim.tallies()
    assert t["n_born"] > 100 and not (t["status_bits"] & B.ST_IDSPACE)
    sim.step(1)
    t = sim.tallies()
    assert t["n_born"] == 0 and (t["status_bits"] & B.ST_IDSPACE)
    with pytest.raises(Exception):
        sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=1 << 20)
