"""Full-size parity in the benchmark's launch configuration, on sampled
outputs the oracle can compute one by one and on properties that hold at
any size:

* the 2D 256x256x30 checkerboard from a 2e7-particle synthetic state (FP64
  and mixed precision): the first 200k particles processed in the GPU step
  are streamed one by one by the oracle at the same T^n with the same
  Philox streams (fates, end cells, segment counts, positions), and the
  step's energy ledger closes;
* the 256-member slab ensemble after 100 steps from cold starts: every
  member's ledger closes and every member's status is clean.
"""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SAMPLE = 200_000
EVERY = 20          # stream every 20th sampled particle in the oracle (10k particles)


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def _ledger_residual(t):
    E0, E1 = t["E_rad0"] + t["E_mat0"], t["E_rad1"] + t["E_mat1"]
    return E1 - E0 - (t["bnd_in_macro"] + t["bnd_in_part"] - t["bnd_out_part"] + t["src_in"]), E1


@pytest.mark.parametrize("prec", [I.FP64, I.MIXED])
def test_checkerboard_full_size_sampled_particles_and_ledger(B, prec):
    n = 20_000_000
    p = I.checkerboard_2d().replace(precision=prec)
    p.particle_capacity = int(1.6 * n)
    s = I.synthetic_state(p, n, seed=3, front=0.35)
    sim = B.Simulation(p)
    sim.set_state(s["T"], s["rho"], s["rho_h"], s["particles"], step=s["step"])
    sim.attach_records(N_SAMPLE)
    sim.step(1)
    t = sim.tallies()
    assert t["status_bits"] == 0 and t["n_in"] == n
    rec = sim.records(N_SAMPLE)
    r, E1 = _ledger_residual(t)
    assert abs(r) <= 1e-12 * E1
    op = O.OracleProblem(p.replace(precision=I.FP64))
    parts = s["particles"]
    L = p.nx * p.dx
    x_tol = 1e-9 * L if prec == I.FP64 else 2e-5 * L
    flip_budget = 1e-4 if prec == I.FP64 else 2e-3
    idx = np.arange(0, N_SAMPLE, EVERY)
    flips = 0
    for i in idx:
        o = O.stream_particle(op, s["T"], s["step"], parts["x"][i], parts["y"][i], parts["ox"][i],
                              parts["oy"][i], parts["nu"][i], parts["w"][i], int(parts["id"][i]),
                              int(parts["cell"][i]), int(parts["grp"][i]), newborn=False)
        g = rec[i]
        assert g["id"] == parts["id"][i]
        if g["fate"] != o["fate"] or g["cell1"] != o["cell"] or g["nseg"] != o["nseg"]:
            flips += 1
            continue
        assert abs(g["x"] - o["x"]) <= x_tol and abs(g["y"] - o["y"]) <= x_tol
    assert flips <= max(1, flip_budget * len(idx)), flips


def test_ensemble_of_256_slabs_after_100_steps(B):
    probs = I.ensemble_slabs(256, steps=100)
    for q in probs:
        q.precision = I.MIXED
        q.particle_capacity = int(2.0 * 0.25 * q.bcT[0] ** 4 * q.dt * 100 / q.omega_ref) + 65536
    ens = B.Simulation(probs)
    ens.step(100)
    alive = 0
    for m in range(len(probs)):
        t = ens.tallies(member=m)
        assert t["status_bits"] == 0, (m, t["status_bits"])
        r, E1 = _ledger_residual(t)
        assert abs(r) <= 1e-11 * E1, (m, r, E1)
        alive += t["n_particles"]
    assert alive > 1e7
