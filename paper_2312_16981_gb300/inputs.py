"""Problem descriptions and seeded synthetic workloads.

This module holds no arithmetic of the method: it only lays out the inputs a
user supplies -- the grid, the group edges, per-cell opacity scale and heat
capacity, the initial temperature, boundary conditions, the reference particle
weight and the seed.  Both the CUDA path and the CPU oracle consume the same
``Problem``; nothing here evaluates opacities, Planck integrals or fluxes.

Workloads are synthetic stand-ins shaped like the paper's Marshak-wave
(Sec. 3.1, Eq. sigmaMarsharkMF) and Olson-type (Sec. 3.5-3.6) set-ups, in
normalised units a = c = h = k = 1, eps = 1.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

BC_REFLECT, BC_VACUUM, BC_BLACKBODY = 0, 1, 2
FP64, MIXED = 0, 1
UGKWP, UGKP = 0, 1


@dataclass
class Problem:
    """One UGKWP problem: a 1D slab or a 2D rectangle of uniform cells."""

    dim: int
    nx: int
    ny: int
    dx: float
    dy: float
    G: int
    nu_edges: np.ndarray          # [G+1], increasing, > 0 (unused when grey)
    sigma0: np.ndarray            # [ncell] opacity scale
    cv: np.ndarray                # [ncell] heat capacity
    T0: np.ndarray                # [ncell] initial material temperature
    dt: float
    sig_p: float = -3.0           # sigma = sigma0 * nu^p * T^q, capped
    sig_q: float = -0.5
    sig_cap: float = 1e6
    grey: int = 0
    a: float = 1.0
    c: float = 1.0
    eps: float = 1.0
    bc: List[int] = field(default_factory=lambda: [BC_REFLECT] * 4)
    bcT: List[float] = field(default_factory=lambda: [0.0] * 4)
    src_T: Optional[np.ndarray] = None   # [ncell] source temperature, 0 = none
    src_on: float = 0.0
    src_amp: Optional[np.ndarray] = None  # [ncell] source profile factor (None: 1)
    src_t_end: float = 0.0   # the source acts while t^n < src_t_end (<= 0: always)
    cv_law: int = 0          # 0: constant cv; 1: Olson CH foam heat capacity (Eq. cvolson)
    cv_chi: float = 0.0      # chi of cv_law 1
    tau_num_C: float = 0.0   # thin/thick joint sampling constant C of tau_num (0: off)
    sig_law: int = 0         # 0: sigma0 nu^p T^q; 1: times (1 - e^{-nu/T}) (Larsen case)
    split_literal: int = 0   # 1: I^h = I^{n+1} - I^p as written (no survivor weight scaling)
    si_warm32: int = 0       # mixed precision: FP32 iterates before the FP64 ones (0 auto, 1 on, -1 off)
    si_pair: int = 0         # small 1D grids: two warps per cell in the source iteration (0 auto, -1 off)
    method: int = 0          # 0: UGKWP (sample the collisionless part); 1: UGKP (sample all of I^h)
    nz: int = 1              # 3D: cells along z (dim 3); sides 4, 5 of bc/bcT are z- and z+
    dz: float = 1.0
    omega_ref: float = 1e-6
    seed: int = 0
    instance: int = 0
    si_tol: float = 1e-12
    si_max_iters: int = 500
    wave_order: int = 2
    precision: int = FP64
    particle_capacity: int = 1 << 20
    n_steps: int = 1
    name: str = "problem"

    @property
    def ncell(self) -> int:
        return self.nx * (self.ny if self.dim >= 2 else 1) * (self.nz if self.dim == 3 else 1)

    @property
    def nface(self) -> int:
        ny = self.ny if self.dim >= 2 else 1
        nz = self.nz if self.dim == 3 else 1
        n = (self.nx + 1) * ny * nz
        if self.dim >= 2:
            n += self.nx * (ny + 1) * nz
        if self.dim == 3:
            n += self.nx * ny * (nz + 1)
        return n

    @property
    def nbins(self) -> int:
        return (self.ncell + 4) * self.G

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def log_groups(G: int, nu_min: float, nu_max: float) -> np.ndarray:
    """Logarithmically spaced group edges (Sec. 3, numerical set-up)."""
    return np.geomspace(nu_min, nu_max, G + 1)


# ----------------------------------------------------------------------------
# The five workloads.  Unstated fields take the readings listed in the design
# document (slab length 1, reflecting far side, Cv = 1, CFL-1 time steps for
# the 2D cases, nu in [1e-3, 10] with cap 1e6).

def grey_slab(nx: int = 100, steps: int = 100, omega_ref: float = 2.5e-7,
              seed: int = 0) -> Problem:
    """Grey 1D slab: sigma = 10, T0 = 0.01, black body T = 1 at x = 0,
    reflecting at x = 1, Cv = 1, dt = 1e-3 (about 1e5 particles per step)."""
    n = nx
    return Problem(
        dim=1, nx=n, ny=1, dx=1.0 / n, dy=1.0, G=1, grey=1,
        nu_edges=np.array([0.0, 1.0]), sigma0=np.full(n, 10.0), cv=np.ones(n),
        T0=np.full(n, 0.01), dt=1e-3, sig_p=0.0, sig_q=0.0, sig_cap=0.0,
        bc=[BC_BLACKBODY, BC_REFLECT, BC_REFLECT, BC_REFLECT], bcT=[1.0, 0.0, 0.0, 0.0],
        omega_ref=omega_ref, seed=seed, n_steps=steps, name="grey_slab_100x1",
        particle_capacity=1 << 19)


def multigroup_slab(nx: int = 200, G: int = 30, steps: int = 500,
                    omega_ref: float = 1e-8, sigma0: float = 1e2,
                    seed: int = 0, dt: float = 1e-4) -> Problem:
    """Frequency-dependent 1D slab (Marshak-wave shape): sigma =
    sigma0 nu^-3 T^-1/2 capped at 1e6, G log groups on [1e-3, 10], T = 1 black
    body at x = 0 into T = 1e-3, reflecting at x = 1, dt = 1e-4."""
    return Problem(
        dim=1, nx=nx, ny=1, dx=1.0 / nx, dy=1.0, G=G, grey=0,
        nu_edges=log_groups(G, 1e-3, 10.0), sigma0=np.full(nx, sigma0), cv=np.ones(nx),
        T0=np.full(nx, 1e-3), dt=dt,
        bc=[BC_BLACKBODY, BC_REFLECT, BC_REFLECT, BC_REFLECT], bcT=[1.0, 0.0, 0.0, 0.0],
        omega_ref=omega_ref, seed=seed, n_steps=steps,
        name="multigroup_slab_%dx%d" % (nx, G), particle_capacity=1 << 22)


def checkerboard_2d(n: int = 256, G: int = 30, block: int = 16, patch: int = 32,
                    steps: int = 100, omega_ref: float = 1e-9, seed: int = 0,
                    precision: int = FP64) -> Problem:
    """2D [0,1]^2 checkerboard of block x block cells alternating sigma0 = 1e3
    and 1, same nu^-3 T^-1/2 law, G groups, isotropic T_s = 1 source in a
    central patch x patch square, T0 = 1e-3, reflecting walls, dt = dx/c."""
    ix, iy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    thick = ((ix // block) + (iy // block)) % 2 == 0
    sig0 = np.where(thick, 1e3, 1.0).reshape(-1).astype(np.float64)
    lo, hi = n // 2 - patch // 2, n // 2 + patch // 2
    src = np.zeros((n, n))
    src[lo:hi, lo:hi] = 1.0
    dx = 1.0 / n
    return Problem(
        dim=2, nx=n, ny=n, dx=dx, dy=dx, G=G, grey=0,
        nu_edges=log_groups(G, 1e-3, 10.0), sigma0=sig0, cv=np.ones(n * n),
        T0=np.full(n * n, 1e-3), dt=dx, src_T=src.reshape(-1), src_on=1.0,
        bc=[BC_REFLECT] * 4, bcT=[0.0] * 4, omega_ref=omega_ref, seed=seed,
        n_steps=steps, precision=precision, name="checkerboard_%dx%dx%d" % (n, n, G),
        particle_capacity=1 << 25)


def checkerboard_3d(n: int = 32, G: int = 8, block: int = 8, patch: int = 8,
                    steps: int = 20, omega_ref: float = 1e-8, seed: int = 0,
                    precision: int = FP64) -> Problem:
    """3D [0,1]^3 checkerboard of block^3 cells alternating sigma0 = 1e3 and 1
    (the 2D checkerboard's law, groups and source extended by a z axis):
    central patch^3 T_s = 1 source, T0 = 1e-3, reflecting walls on all six
    sides, dt = dx/c."""
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    thick = ((ix // block) + (iy // block) + (iz // block)) % 2 == 0
    # cell order c = (iz n + iy) n + ix
    sig0 = np.where(thick, 1e3, 1.0).transpose(2, 1, 0).reshape(-1).astype(np.float64)
    lo, hi = n // 2 - patch // 2, n // 2 + patch // 2
    src = np.zeros((n, n, n))
    src[lo:hi, lo:hi, lo:hi] = 1.0
    dx = 1.0 / n
    return Problem(
        dim=3, nx=n, ny=n, nz=n, dx=dx, dy=dx, dz=dx, G=G, grey=0,
        nu_edges=log_groups(G, 1e-3, 10.0), sigma0=sig0, cv=np.ones(n ** 3),
        T0=np.full(n ** 3, 1e-3), dt=dx, src_T=src.reshape(-1), src_on=1.0,
        bc=[BC_REFLECT] * 6, bcT=[0.0] * 6, omega_ref=omega_ref, seed=seed,
        n_steps=steps, precision=precision, name="checkerboard3d_%dx%dx%dx%d" % (n, n, n, G),
        particle_capacity=1 << 22)


def adjoint_grid(n: int = 128, G: int = 16, patch: int = 16, steps: int = 200,
                 omega_ref: float = 1e-9, seed: int = 0) -> Problem:
    """2D [0,1]^2 grid for the opacity-gradient workload: n x n cells, G log
    groups on [1e-3, 10], base sigma0 = 1e2 (sigma = sigma0 e^{s_c} nu^-3
    T^-1/2, capped at 1e6; the per-cell scales s_c are the parameters),
    isotropic T_s = 1 source in a central patch x patch square, T0 = 1e-3,
    reflecting walls, dt = dx/c."""
    lo, hi = n // 2 - patch // 2, n // 2 + patch // 2
    src = np.zeros((n, n))
    src[lo:hi, lo:hi] = 1.0
    dx = 1.0 / n
    return Problem(
        dim=2, nx=n, ny=n, dx=dx, dy=dx, G=G, grey=0,
        nu_edges=log_groups(G, 1e-3, 10.0), sigma0=np.full(n * n, 1e2), cv=np.ones(n * n),
        T0=np.full(n * n, 1e-3), dt=dx, src_T=src.reshape(-1), src_on=1.0,
        bc=[BC_REFLECT] * 4, bcT=[0.0] * 4, omega_ref=omega_ref, seed=seed,
        n_steps=steps, name="adjoint_grid_%dx%dx%d" % (n, n, G), particle_capacity=1 << 23)


def larsen_slab(G: int = 24, omega_frac: float = 1e-4, steps: int = 1349) -> Problem:
    """The Larsen test problem (Sec. 3.3) in the paper's units (cm, ns, keV,
    GJ; c = 29.98 cm/ns, a = 0.01372 GJ/(cm^3 keV^4)): [0, 4] cm, 200 cells,
    sigma = gamma0 (1 - e^{-nu/T})/nu^3 with gamma0 = 1, 1000, 1 keV^3/cm on
    [0, 2], (2, 3], (3, 4] cm, C_v = 0.05109 GJ/(cm^3 keV), T0 = 1e-3 keV,
    a T_r = 1 keV black body at x = 0, a free (vacuum) side at x = 4, G log
    groups on [1e-2, 1e2] keV, dt = dx/c (CFL 1), tau_num with C = 1e3 at the
    thin/thick joints, reference weight omega_frac x V in rho V units
    (rho = c x energy density); t = 0.9 ns after `steps` steps."""
    nx, L = 200, 4.0
    dx = L / nx
    xc = (np.arange(nx) + 0.5) * dx
    gamma0 = np.where((xc > 2.0) & (xc <= 3.0), 1000.0, 1.0)
    c, a = 29.98, 0.01372
    return Problem(
        dim=1, nx=nx, ny=1, dx=dx, dy=1.0, G=G, grey=0, nu_edges=log_groups(G, 1e-2, 1e2),
        sigma0=gamma0, cv=np.full(nx, 0.05109), T0=np.full(nx, 1e-3), dt=dx / c,
        sig_p=-3.0, sig_q=0.0, sig_cap=1e6, sig_law=1, a=a, c=c, eps=1.0,
        bc=[BC_BLACKBODY, BC_VACUUM, BC_REFLECT, BC_REFLECT], bcT=[1.0, 0.0, 0.0, 0.0],
        omega_ref=omega_frac * dx * c, tau_num_C=1e3, n_steps=steps, name="larsen_%dx%d" % (nx, G),
        particle_capacity=1 << 22)


def olson_slab(G: int = 30, omega_frac: float = 1e-4, steps: int = 107) -> Problem:
    """The Olson 1D carbon-hydrogen foam (Sec. 3.5), normalised a = c = 1,
    T and h nu in keV: [0, 4.8] cm in 128 cells (dx = 0.0375), sigma = rho
    kappa(nu, T) with rho = 1e-3 g/cc (sig_law 2), heat capacity of Eq.
    cvolson with a T_keV^3 H = 0.1 and chi = 0.1 (cv_law 1), T0 = 0.01,
    reflecting walls, source B(0.5 keV) e^{-693 x^3} (cell centres) for
    ct <= 2, dt = dx/c (107 steps reach ct = 4); G log groups on
    [1e-3, 10] keV (covering both breaks of kappa); reference weight
    1e-4 c V."""
    n = 128
    dx = 4.8 / n
    xc = (np.arange(n) + 0.5) * dx
    return Problem(
        dim=1, nx=n, ny=1, dx=dx, dy=1.0, G=G, grey=0,
        nu_edges=log_groups(G, 1e-3, 10.0), sigma0=np.full(n, 1e-3), cv=np.full(n, 0.1),
        T0=np.full(n, 0.01), dt=dx, sig_p=0.0, sig_q=0.0, sig_cap=0.0, sig_law=2,
        cv_law=1, cv_chi=0.1,
        bc=[BC_REFLECT] * 4, bcT=[0.0] * 4,
        src_T=np.full(n, 0.5), src_amp=np.exp(-693.0 * xc ** 3), src_on=1.0, src_t_end=2.0,
        omega_ref=omega_frac * dx, n_steps=steps, name="olson_slab_128x%d" % G,
        particle_capacity=1 << 21)


def ensemble_slabs(n_instances: int = 256, seed: int = 0, steps: int = 100) -> List[Problem]:
    """Ensemble of independent 1D slabs with uneven sizes: cells U{64..1024},
    G in {8,16,32,64}, sigma0 log-U[1, 1e4], black-body T U[0.5, 2], target
    particle counts log-U[1e4, 1e6].  Drawn from a seeded numpy generator."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for k in range(n_instances):
        nx = int(rng.integers(64, 1025))
        G = int(rng.choice([8, 16, 32, 64]))
        s0 = float(10.0 ** rng.uniform(0.0, 4.0))
        Tb = float(rng.uniform(0.5, 2.0))
        target = float(10.0 ** rng.uniform(4.0, 6.0))
        p = multigroup_slab(nx=nx, G=G, steps=steps, sigma0=s0, seed=seed)
        p.bcT = [Tb, 0.0, 0.0, 0.0]
        p.instance = k
        # reference weight scaled with the energy a black body at Tb feeds in
        p.omega_ref = 0.25 * Tb ** 4 * p.dt * steps / target
        p.name = "ensemble_%d" % k
        out.append(p)
    return out


def small_multigroup(nx: int = 24, G: int = 6, omega_ref: float = 2e-6, dt: float = 2e-3,
                     seed: int = 0) -> Problem:
    """A small multigroup slab that the oracle finishes in seconds but that
    still spans several tiles of particles and a ragged tail."""
    p = multigroup_slab(nx=nx, G=G, steps=10, omega_ref=omega_ref, seed=seed, dt=dt)
    p.name = "small_multigroup_%dx%d" % (nx, G)
    p.particle_capacity = 1 << 18
    return p


def small_checkerboard(n: int = 16, G: int = 4, omega_ref: float = 2e-6, seed: int = 0) -> Problem:
    p = checkerboard_2d(n=n, G=G, block=4, patch=4, steps=5, omega_ref=omega_ref, seed=seed)
    p.name = "small_checkerboard_%dx%dx%d" % (n, n, G)
    p.particle_capacity = 1 << 18
    return p


def synthetic_state(p: Problem, n_particles: int, seed: int = 1, front: float = 0.2,
                    step: int = 0, wave_fraction: float = 0.02) -> dict:
    """A seeded mid-run state shaped like a Marshak front, for full-size runs
    that both the CUDA path and the oracle start from.

    Pure input generation: a temperature profile falling from 1 to T0 over
    `front` of the slab (1D) or of the distance from the domain centre (2D,
    the source patch sits there); a spectral shape T^4 x (log-normal bump near
    nu ~ 3T); n_particles particles placed in (cell, group) bins in
    proportion to that shape, uniform in the cell, isotropic (3D directions
    projected on the plane in 2D), with frequency uniform in the group and
    weight omega_ref * U(0.5, 1.5); the wave part rho_h = wave_fraction x the
    shape, and rho = rho_h + the particles' energy per volume (so most of the
    radiation is carried by particles, as in a running problem).
    """
    rng = np.random.Generator(np.random.Philox(seed))
    T0 = float(np.min(p.T0))
    if p.dim == 1:
        L = p.nx * p.dx
        dist = (np.arange(p.nx) + 0.5) * p.dx
        V = p.dx
    else:
        L = 0.5 * min(p.nx * p.dx, p.ny * p.dy)
        xc = (np.arange(p.nx) + 0.5) * p.dx - 0.5 * p.nx * p.dx
        yc = (np.arange(p.ny) + 0.5) * p.dy - 0.5 * p.ny * p.dy
        dist = np.hypot(xc[None, :], yc[:, None]).reshape(-1)
        V = p.dx * p.dy
    ncell = p.ncell
    T = T0 + (1.0 - T0) * np.sqrt(np.clip(1.0 - dist / (front * L), 0.0, None))
    if p.grey:
        shape = np.ones((ncell, 1))
    else:
        lnu = np.log(np.sqrt(p.nu_edges[:-1] * p.nu_edges[1:]))
        shape = np.exp(-0.5 * ((lnu[None, :] - np.log(3.0 * T[:, None])) / 0.7) ** 2)
        shape /= shape.sum(1, keepdims=True)
    field = ((T[:, None] ** 4) * shape).reshape(-1)
    prob = field / field.sum()
    bins = rng.choice(ncell * p.G, size=n_particles, p=prob)
    bins.sort()
    cell = (bins // p.G).astype(np.int32)
    grp = (bins % p.G).astype(np.int32)
    if p.dim == 1:
        x = (cell + rng.random(n_particles)) * p.dx
        y = np.zeros(n_particles)
        ox = 2.0 * rng.random(n_particles) - 1.0
        oy = np.zeros(n_particles)
    else:
        x = (cell % p.nx + rng.random(n_particles)) * p.dx
        y = (cell // p.nx + rng.random(n_particles)) * p.dy
        muz = 2.0 * rng.random(n_particles) - 1.0
        phi = 2.0 * np.pi * rng.random(n_particles)
        sxy = np.sqrt(np.maximum(0.0, 1.0 - muz * muz))
        ox, oy = sxy * np.cos(phi), sxy * np.sin(phi)
    if p.grey:
        nu = np.zeros(n_particles)
    else:
        lo, hi = p.nu_edges[grp], p.nu_edges[grp + 1]
        nu = lo + (hi - lo) * rng.random(n_particles)
    w = p.omega_ref * (0.5 + rng.random(n_particles))
    # unique identities (birth step 0): bin and rank within the bin
    first = np.searchsorted(bins, bins, side="left")
    k = np.arange(n_particles) - first
    pid = (np.uint64(step) << np.uint64(44)) | (bins.astype(np.uint64) << np.uint64(20)) | k.astype(np.uint64)
    parts = dict(x=x, y=y, ox=ox, oy=oy, nu=nu, w=w, id=pid, cell=cell, grp=grp)
    rho_p = np.bincount(bins, weights=w, minlength=ncell * p.G) / V
    rho_h = wave_fraction * field
    return dict(T=T, rho=rho_h + rho_p, rho_h=rho_h, particles=parts, step=step + 1)
