"""Pins of the oracle in 3D (the paper's method on a third axis: faces
normal to z, six sides, 3D isotropic directions).  A 3D problem uniform
along y and z between mirror walls is the 1D problem (wave part and source
iteration, no particles: to roundoff); the energy ledger closes with
particles; free streaming in a nearly transparent box moves each particle
by (c/eps) Omega dt, reflecting at the walls; newborn directions are
isotropic (moments against 1/3); and a Planck equilibrium is held fixed."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I


def _run(p, n, st=None):
    op = O.OracleProblem(p)
    st = st or O.initial_state(op)
    tals = []
    for _ in range(n):
        st, tal, _, status = O.step(op, st)
        assert status == 0
        tals.append(tal)
    return op, st, tals


def test_uniform_in_y_and_z_is_the_1d_problem():
    p1 = I.small_multigroup(nx=12, G=4, omega_ref=0.0, dt=5e-3)
    p1.bc = [I.BC_REFLECT] * 4
    p1.T0 = np.linspace(1.0, 0.05, p1.nx)
    ny, nz = 2, 3
    p3 = p1.replace(dim=3, ny=ny, nz=nz, dy=0.3, dz=0.7, bc=[I.BC_REFLECT] * 6, bcT=[0.0] * 6,
                    sigma0=np.tile(p1.sigma0, ny * nz), cv=np.tile(p1.cv, ny * nz), T0=np.tile(p1.T0, ny * nz))
    _, s1, _ = _run(p1, 2)
    _, s3, _ = _run(p3, 2)
    T3 = s3.T.reshape(nz, ny, p1.nx)
    for iz in range(nz):
        for iy in range(ny):
            np.testing.assert_allclose(T3[iz, iy], s1.T, rtol=1e-14)
    np.testing.assert_allclose(s3.rho.reshape(nz * ny, -1), np.tile(s1.rho, (nz * ny, 1)), rtol=1e-13)


def test_3d_energy_ledger_closes():
    p = I.checkerboard_3d(n=8, G=3, block=2, patch=2, omega_ref=2e-7)
    p.T0 = np.linspace(0.2, 1.0, p.ncell)
    p.src_on = 0.0
    _, st, tals = _run(p, 3)
    E0 = tals[0].c.E_rad0 + tals[0].c.E_mat0
    for tal in tals:
        c = tal.c
        assert abs(c.E_rad1 + c.E_mat1 - E0) <= 1e-13 * E0   # mirror walls, no source
    assert st.particles.n > 1000 and sum(t.c.n_absorbed for t in tals) > 0


def test_free_streaming_in_a_transparent_box():
    n = 4
    p = I.checkerboard_3d(n=n, G=1, block=1, patch=0, omega_ref=0.0).replace(grey=1, sig_p=0.0, sig_q=0.0)
    p.sigma0 = np.full(p.ncell, 1e-12)
    p.nu_edges = np.array([0.0, 1.0])
    p.src_on = 0.0
    rng = np.random.default_rng(3)
    m = 500
    pos = rng.uniform(0.05, 0.95, size=(m, 3))
    mu = rng.uniform(-1, 1, m)
    ph = rng.uniform(0, 2 * np.pi, m)
    om = np.stack([np.sqrt(1 - mu ** 2) * np.cos(ph), np.sqrt(1 - mu ** 2) * np.sin(ph), mu], 1)
    idx = np.minimum((pos / p.dx).astype(int), n - 1)
    cell = (idx[:, 2] * n + idx[:, 1]) * n + idx[:, 0]
    parts = {"x": pos[:, 0], "y": pos[:, 1], "z": pos[:, 2], "ox": om[:, 0], "oy": om[:, 1], "oz": om[:, 2],
             "nu": np.zeros(m), "w": np.full(m, 1e-6), "id": np.arange(m, dtype=np.uint64) + 7,
             "cell": cell.astype(np.int32), "grp": np.zeros(m, dtype=np.int32)}
    op = O.OracleProblem(p)
    st0 = O.initial_state(op)
    st0.particles = O.ParticleSet.from_arrays(parts, cap=2 * m)
    st1, tal, rec, status = O.step(op, st0, records=True)
    assert status == 0 and tal.c.n_survived == m
    L = p.c / p.eps * p.dt
    for k in range(m):
        # unfolded straight line, folded back by the mirror walls at 0 and 1
        for a, key in enumerate(("x", "y", "z")):
            u = pos[k, a] + L * om[k, a]
            u = u % 2.0
            want = u if u <= 1.0 else 2.0 - u
            assert abs(rec[key][k] - want) <= 1e-12
        i3 = [min(int(rec[key][k] / p.dx), n - 1) for key in ("x", "y", "z")]
        assert rec["cell1"][k] == (i3[2] * n + i3[1]) * n + i3[0] or \
            any(abs(rec[key][k] / p.dx - round(rec[key][k] / p.dx)) < 1e-12 for key in ("x", "y", "z"))


def test_newborn_directions_are_isotropic_in_3d():
    p = I.checkerboard_3d(n=4, G=1, block=1, patch=0, omega_ref=1e-7).replace(grey=1, sig_p=0.0, sig_q=0.0)
    p.nu_edges = np.array([0.0, 1.0])
    p.sigma0 = np.full(p.ncell, 1e-12)
    p.T0 = np.full(p.ncell, 0.5)
    p.src_on = 0.0
    op = O.OracleProblem(p)
    st, tal, rec, status = O.step(op, O.initial_state(op), records=True)
    assert status == 0
    n = len(rec)
    assert n > 50_000
    o = np.stack([rec["ox"], rec["oy"], rec["oz"]], 1)
    np.testing.assert_allclose(np.linalg.norm(o, axis=1), 1.0, atol=1e-12)
    for a in range(3):
        assert abs(np.mean(o[:, a])) < 5.0 / math.sqrt(3 * n)
        assert abs(np.mean(o[:, a] ** 2) - 1.0 / 3.0) < 5.0 * math.sqrt(4.0 / 45.0 / n)


def test_3d_equilibrium_held_without_particles():
    p = I.checkerboard_3d(n=6, G=3, block=3, patch=0, omega_ref=0.0)
    p.T0 = np.full(p.ncell, 0.3)
    p.src_on = 0.0
    _, st, _ = _run(p, 2)
    np.testing.assert_allclose(st.T, 0.3, rtol=1e-12)
