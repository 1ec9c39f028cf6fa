"""The CUDA adjoint (pathwise gradient of L = sum (T - T_target)^2 with
respect to the per-cell log-opacity scales) against

* the oracle's tangent: the directional derivative dL.v along random and
  unit directions, on the same seed (the GPU and the oracle take the same
  Monte Carlo decisions at these sizes, so both differentiate the same
  path; the tangent is forward mode written independently of the adjoint);
* central finite differences with common random numbers on the GPU;
* itself with different checkpoint spacings, and through the
  torch.autograd.Function.
"""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-6       # GPU adjoint vs oracle tangent (same path, different summation order)


@pytest.fixture(scope="module")
def A():
    from paper_2312_16981_gb300 import adjoint, binding
    binding.load()
    return adjoint


def _case(name):
    if name == "multigroup":
        return I.small_multigroup(nx=12, G=4, omega_ref=2e-6), 4
    if name == "multigroup_order1":
        p = I.small_multigroup(nx=12, G=4, omega_ref=2e-6)
        p.wave_order = 1
        return p, 4
    if name == "grey_blackbody":
        return I.grey_slab(nx=20, omega_ref=2.5e-6), 5
    if name == "vacuum":
        p = I.small_multigroup(nx=10, G=3, omega_ref=2e-6)
        p.bc = [I.BC_BLACKBODY, I.BC_VACUUM, 0, 0]
        return p, 4
    if name == "checkerboard":
        return I.small_checkerboard(n=8, G=3, omega_ref=2e-6), 3
    if name == "source_patch_2d":
        p = I.adjoint_grid(n=10, G=4, patch=4, omega_ref=3e-8)
        p.particle_capacity = 1 << 18
        return p, 3
    raise KeyError(name)


def _setup(p, steps, seed=0):
    rng = np.random.default_rng(seed)
    s = rng.normal(0, 0.1, p.ncell)
    tgt = O.with_log_opacity(p.replace(seed=p.seed + 1), rng.normal(0, 0.1, p.ncell))
    _, st, _ = O.misfit(tgt, steps, np.zeros(p.ncell))
    return s, st.T


@pytest.mark.parametrize("name", ["multigroup", "multigroup_order1", "grey_blackbody", "vacuum",
                                  "checkerboard", "source_patch_2d"])
def test_adjoint_matches_oracle_tangent(A, name):
    p, steps = _case(name)
    s, Tt = _setup(p, steps)
    L, g = A.misfit_and_gradient(p, s, steps, Tt, ckpt_every=2)
    rng = np.random.default_rng(1)
    q = O.with_log_opacity(p, s)
    # a random direction and the unit directions of the cells with the
    # largest and a middling sensitivity (cold cells far from the front have
    # gradients below 1e-90: compared on the scale of the whole gradient)
    order = np.argsort(-np.abs(g))
    for v in [rng.normal(size=p.ncell), np.eye(p.ncell)[order[0]], np.eye(p.ncell)[order[p.ncell // 4]]]:
        Lo, dLo, _ = O.misfit_tangent(q, steps, Tt, v)
        assert abs(L - Lo) <= 1e-8 * abs(Lo)
        scale = np.sum(np.abs(g * v)) + 1e-9 * np.max(np.abs(g))
        assert abs(float(g @ v) - dLo) <= REL * scale, (name, float(g @ v), dLo)


def test_adjoint_matches_crn_finite_differences_on_gpu(A):
    p = I.small_multigroup(nx=40, G=8, omega_ref=5e-7)
    p.sigma0 = np.full(p.ncell, 30.0)
    steps = 12
    s, Tt = _setup(p, steps, seed=3)
    L, g = A.misfit_and_gradient(p, s, steps, Tt, ckpt_every=5)
    cells = [0, 7, 19, 33]
    fd = A.crn_finite_differences(p, s, steps, Tt, cells, h=1e-6)
    for c, f in zip(cells, fd):
        assert abs(g[c] - f) <= 1e-4 * max(abs(f), 1e-3 * np.max(np.abs(g))), (c, g[c], f)


def test_checkpoint_spacing_does_not_change_the_gradient(A):
    # survivors are compacted in a thread-order-dependent order, so the
    # particles of a checkpoint and of the recomputed segment before it are
    # matched by identity; every spacing must give the same gradient
    p, steps = _case("checkerboard")
    steps = 6
    s, Tt = _setup(p, steps, seed=5)
    _, g1 = A.misfit_and_gradient(p, s, steps, Tt, ckpt_every=1)
    _, g6 = A.misfit_and_gradient(p, s, steps, Tt, ckpt_every=6)
    _, g4 = A.misfit_and_gradient(p, s, steps, Tt, ckpt_every=4)
    np.testing.assert_allclose(g6, g1, rtol=0, atol=1e-9 * np.max(np.abs(g1)))
    np.testing.assert_allclose(g4, g1, rtol=0, atol=1e-9 * np.max(np.abs(g1)))


def test_autograd_function(A):
    p, steps = _case("multigroup")
    s, Tt = _setup(p, steps, seed=7)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    L = A.log_opacity_misfit(st, p, steps, Tt, ckpt_every=3)
    L.backward()
    L2, g = A.misfit_and_gradient(p, s, steps, Tt, ckpt_every=3)
    assert abs(L.item() - L2) <= 1e-10 * L2
    np.testing.assert_allclose(st.grad.numpy(), g, rtol=0, atol=1e-9 * np.max(np.abs(g)))


def test_adjoint_rejects_mixed_precision_and_small_tapes(A):
    from paper_2312_16981_gb300 import binding as B
    p, steps = _case("multigroup")
    sim = B.Simulation(p.replace(precision=I.MIXED))
    with pytest.raises(B.UGKWPError):
        sim.adjoint_buffer()
    sim.close()
    sim = B.Simulation(p)
    sim.step(2)
    tape = sim.tape_buffer(8)                # far fewer than the step's particles
    sim.step_taped(tape, 8)
    assert sim.tallies()["status_bits"] & 1
    sim.close()
