"""Run-to-run reproducibility: the particle tallies W and E_surv are summed
in fixed point with integer atomics, so two runs of the same problem give
bitwise-identical temperatures and radiation, whatever order the threads
add in (FP64 and mixed precision, 1D and 2D, single and batched).  The
finite-difference check of the adjoint relies on it."""
import numpy as np
import pytest

from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def _run(B, p, steps, graph=True):
    sim = B.Simulation(p)
    if graph:
        sim.step(steps)
    else:
        for _ in range(steps):
            sim.step_timed()
    st = sim.get_state(cap=0)
    t = sim.tallies()
    sim.close()
    assert t["status_bits"] == 0
    return st


@pytest.mark.parametrize("prec", [I.FP64, I.MIXED])
def test_two_runs_are_bitwise_identical_1d(B, prec):
    p = I.multigroup_slab(nx=120, G=12, omega_ref=2e-8).replace(precision=prec, particle_capacity=1 << 21)
    a = _run(B, p, 40)
    b = _run(B, p, 40, graph=False)
    assert a["n"] == b["n"] and a["n"] > 10000
    assert np.array_equal(a["T"], b["T"])
    assert np.array_equal(a["rho"], b["rho"])


def test_two_runs_are_bitwise_identical_2d(B):
    p = I.adjoint_grid(n=48, G=8, patch=8, omega_ref=5e-8).replace(particle_capacity=1 << 21)
    a = _run(B, p, 30)
    b = _run(B, p, 30)
    assert a["n"] > 10000
    assert np.array_equal(a["T"], b["T"])
    assert np.array_equal(a["rho_h"], b["rho_h"])
