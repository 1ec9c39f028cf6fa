"""The method on a 3D grid (faces normal to x, y and z; six sides; 3D
isotropic birth directions) on the GPU against the oracle through the C ABI:
one step from an identical state with per-particle records (FP64: element by
element with event flips counted, positions and directions on all three
axes; mixed precision: to its stated error), first- and second-order wave
flux, the numerical collision time at the checkerboard's thin/thick joints,
open z sides (escape tallies per side), a multi-step trajectory from the
initial state, and the 32^3 x 8 checkerboard in the launch configuration of
a CUDA-graph step with its energy ledger closed."""
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


def box(**kw):
    # 8^3 cells, 2^3 blocks alternating sigma0 = 1e3 / 1, a 2^3 source patch
    p = I.checkerboard_3d(n=8, G=3, block=2, patch=2, omega_ref=5e-8)
    p.particle_capacity = 1 << 18
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("order", [1, 2])
def test_step_parity_checkerboard_3d(B, order):
    t, tal = check_step(B, box(wave_order=order), 2)
    assert t["n_born"] > 4000 and t["n_in"] > 1500


def test_step_parity_3d_tau_num(B):
    p = box(tau_num_C=1e3)
    t, tal = check_step(B, p, 2)
    _, st = oracle_run(p, 2)
    _, n_tau, _ = O.birth_counts(O.OracleProblem(p.replace(tau_num_C=0.0)), st.T, st.rho_h)
    assert t["n_born"] > n_tau


def test_step_parity_3d_open_z_sides(B):
    # vacuum z- and z+, mirror x and y; a hot slab of cells next to z-
    p = box(bc=[I.BC_REFLECT] * 4 + [I.BC_VACUUM] * 2)
    T0 = np.full(p.ncell, 1e-3)
    T0.reshape(p.nz, p.ny, p.nx)[:2] = 0.5
    p.T0 = T0
    p.sigma0 = np.full(p.ncell, 1.0)
    t, tal = check_step(B, p, 1)
    sim = B.Simulation(p)
    op, st = oracle_run(p, 1)
    sim.set_state(st.T, st.rho, st.rho_h, st.particles.view(), step=st.step)
    sim.step(1)
    esc = sim.device_array("esc").cpu().numpy().reshape(6, p.G)
    st2, tal2, _, _ = O.step(op, st)
    esc_o = np.asarray(tal2.esc).reshape(6, p.G)
    assert esc_o[4].sum() > 0.0 and esc_o[:4].sum() == 0.0
    np.testing.assert_allclose(esc, esc_o, rtol=1e-12, atol=1e-300)


def test_mixed_checkerboard_3d(B):
    p = box()
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(2):
        st, _, _, _ = O.step(op, st)
    M.check(p, *M.run_pair(B, p, st, op))


@pytest.mark.parametrize("precision", [I.FP64, I.MIXED])
def test_3d_trajectory_from_the_initial_state(B, precision):
    p = box(precision=precision)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    sim = B.Simulation(p)
    tol = T_RTOL if precision == I.FP64 else 1e-3
    for n in range(3):
        sim.step(1)
        st, tal, _, _ = O.step(op, st)
        g = sim.get_state()
        t = sim.tallies()
        assert t["status_bits"] == 0 and t["n_born"] == tal.c.n_born
        if precision == I.FP64:
            assert t["n_particles"] == st.particles.n
        np.testing.assert_allclose(g["T"], st.T, rtol=tol)


def test_full_size_checkerboard_3d_graph_steps(B):
    # 32^3 cells x 8 groups, the source patch 8^3; graph-captured steps
    p = I.checkerboard_3d()
    sim = B.Simulation(p)
    sim.step(4)
    t = sim.tallies()
    assert t["status_bits"] == 0 and t["n_particles"] > 10000
    E0, E1 = t["E_rad0"] + t["E_mat0"], t["E_rad1"] + t["E_mat1"]
    resid = E1 - E0 - (t["bnd_in_macro"] + t["bnd_in_part"] - t["bnd_out_part"] + t["src_in"])
    assert abs(resid) <= 1e-12 * E1
    # the wave part's state against the oracle on sampled cells: the oracle's
    # birth counts from the GPU's own T and rho_h match the GPU's exactly
    g = sim.get_state(cap=0)
    op = O.OracleProblem(p)
    N, n_new, _ = O.birth_counts(op, g["T"], g["rho_h"])
    sim.step(1)
    assert sim.tallies()["n_born"] == n_new


def test_3d_adjoint_rejected(B):
    sim = B.Simulation(box(omega_ref=0.0))
    with pytest.raises(B.UGKWPError) as e:
        sim.tape_buffer(16)
    assert e.value.code == -8


@pytest.mark.parametrize("precision", [I.FP64, I.MIXED])
def test_3d_checkpoint_restore_repeats_the_steps(B, precision):
    # z positions and directions are part of the checkpointed particle state
    sim = B.Simulation(box(precision=precision))
    sim.step(2)
    buf = sim.checkpoint_buffer()
    sim.checkpoint(buf)
    sim.step(2)
    first = sim.get_state()
    sim.restore(buf)
    sim.step(2)
    second = sim.get_state()
    assert first["n"] == second["n"] and first["n"] > 1000
    np.testing.assert_allclose(second["T"], first["T"], rtol=1e-10)
    a, b = first["particles"], second["particles"]
    ia, ib = np.argsort(a["id"]), np.argsort(b["id"])
    np.testing.assert_array_equal(a["id"][ia], b["id"][ib])
    for f in ("z", "oz", "x", "y"):
        np.testing.assert_allclose(b[f][ib], a[f][ia], rtol=0, atol=1e-9)
    assert np.abs(a["oz"]).max() > 0.5 and (a["z"] > 0).all() and (a["z"] < 1).all()


def ragged(G=40, **kw):
    # nx != ny != nz, dx != dy != dz, G > 32 (two groups per lane in the
    # source iteration), a hot corner and a thick slab of cells
    nx, ny, nz = 6, 5, 4
    n = nx * ny * nz
    T0 = np.full(n, 0.02)
    T0.reshape(nz, ny, nx)[:2, :2, :3] = 0.6
    sig0 = np.full(n, 3.0)
    sig0.reshape(nz, ny, nx)[:, 3:, :] = 300.0
    p = I.checkerboard_3d(n=4, G=G, block=2, patch=0, omega_ref=4e-7).replace(
        nx=nx, ny=ny, nz=nz, dx=0.11, dy=0.17, dz=0.23, sigma0=sig0, cv=np.ones(n), T0=T0,
        src_T=None, src_on=0.0, dt=0.05, bc=[I.BC_REFLECT, I.BC_VACUUM, I.BC_VACUUM, I.BC_REFLECT,
                                            I.BC_REFLECT, I.BC_VACUUM], bcT=[0.0] * 6)
    p.particle_capacity = 1 << 19
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("order", [1, 2])
def test_step_parity_ragged_3d_box(B, order):
    t, tal = check_step(B, ragged(wave_order=order), 2)
    assert t["n_born"] > 500 and t["n_in"] > 10000 and t["n_escaped"] > 0


def test_mixed_ragged_3d_box(B):
    p = ragged(G=12)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    for _ in range(2):
        st, _, _, _ = O.step(op, st)
    M.check(p, *M.run_pair(B, p, st, op))
