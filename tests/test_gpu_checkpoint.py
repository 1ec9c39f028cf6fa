"""Checkpoint/restore of the whole state (device-to-device) and the launch
shape autotuner.  A restored run repeats the same steps: identities and
counter-based streams are part of the state, so births, survivors and
temperatures agree with the first pass up to the summation order of FP64
atomics.  Every launch shape gives the same physics."""
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


@pytest.mark.parametrize("precision", [I.FP64, I.MIXED])
def test_restore_repeats_the_same_steps(B, precision):
    p = I.small_multigroup(nx=20, G=5, omega_ref=1e-6).replace(precision=precision)
    sim = B.Simulation(p)
    sim.step(3)
    buf = sim.checkpoint_buffer()
    sim.checkpoint(buf)
    sim.step(4)
    first = sim.get_state()
    t1 = sim.tallies()
    sim.restore(buf)
    assert sim.tallies()["step"] == 3
    sim.step(4)
    second = sim.get_state()
    t2 = sim.tallies()
    assert t1["step"] == t2["step"] == 7 and first["n"] == second["n"]
    np.testing.assert_allclose(second["T"], first["T"], rtol=1e-10)
    np.testing.assert_array_equal(np.sort(first["particles"]["id"]), np.sort(second["particles"]["id"]))


@pytest.mark.parametrize("precision", [I.FP64, I.MIXED])
def test_restore_repeats_the_steps_bitwise(B, precision):
    # a step starts its source iteration from the state the previous step's
    # last iterate left (T^n's opacities and Planck values); a restore or a
    # set_state drops it and the state is re-evaluated, to the same bits
    p = I.small_multigroup(nx=20, G=5, omega_ref=1e-6).replace(precision=precision)
    sim = B.Simulation(p)
    sim.step(3)
    buf = sim.checkpoint_buffer()
    sim.checkpoint(buf)
    sim.step(4)
    first = sim.get_state()
    sim.restore(buf)
    sim.step(4)
    second = sim.get_state()
    np.testing.assert_array_equal(second["T"], first["T"])
    np.testing.assert_array_equal(second["rho"], first["rho"])


def test_set_state_mid_run_gives_the_same_step(B):
    p = I.small_multigroup(nx=20, G=5, omega_ref=1e-6)
    a = B.Simulation(p)
    a.step(3)
    st = a.get_state()
    b = B.Simulation(p)
    b.set_state(st["T"], st["rho"], st["rho_h"], st["particles"], step=a.tallies()["step"])
    a.step(1)
    b.step(1)
    np.testing.assert_array_equal(b.get_state()["T"], a.get_state()["T"])


def test_checkpoint_of_an_ensemble(B):
    probs = [I.small_multigroup(nx=10 + 7 * m, G=3 + m, omega_ref=1e-6) for m in range(3)]
    for m, p in enumerate(probs):
        p.instance = m
    sim = B.Simulation(probs)
    sim.step(2)
    buf = sim.checkpoint_buffer()
    sim.checkpoint(buf)
    sim.step(3)
    first = [sim.get_state(member=m)["T"] for m in range(3)]
    sim.restore(buf)
    sim.step(3)
    for m in range(3):
        np.testing.assert_allclose(sim.get_state(member=m)["T"], first[m], rtol=1e-10)


@pytest.mark.parametrize("shape", [(128, 1, 0), (512, 2, 0), (256, 2, 2), (256, 4, 0)])
def test_launch_shapes_give_the_same_physics(B, shape):
    p = I.small_multigroup(nx=24, G=6, omega_ref=5e-7).replace(precision=I.MIXED)
    ref = B.Simulation(p)
    ref.step(3)
    sim = B.Simulation(p)
    sim.set_launch(*shape)
    sim.step(3)
    a, b = ref.get_state(), sim.get_state()
    assert a["n"] == b["n"]
    np.testing.assert_allclose(b["T"], a["T"], rtol=1e-10)


def test_autotune_keeps_state_and_caches(B, tmp_path):
    p = I.small_multigroup(nx=24, G=6, omega_ref=5e-7)
    sim = B.Simulation(p)
    sim.step(2)
    before = sim.get_state()
    cache = str(tmp_path / "tune.json")
    out = sim.autotune(steps=1, cache=cache)
    assert out["block"] in (128, 256, 512) and out["particles_per_thread"] in (1, 2, 4) and not out["cached"]
    after = sim.get_state()
    np.testing.assert_array_equal(after["T"], before["T"])
    assert after["n"] == before["n"] and sim.tallies()["step"] == 2
    again = B.Simulation(p)
    again.step(2)
    out2 = again.autotune(steps=1, cache=cache)
    assert out2["cached"] and out2["block"] == out["block"]
