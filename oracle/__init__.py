"""CPU FP64 oracle of the UGKWP particle phase, wave flux and source iteration.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never calls it and shares no code with it: the oracle is a plain C
restatement of the paper (``ugkwp_oracle.c``) behind this ctypes binding.

Every function of the C file cites the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

SURVIVED, ABSORBED, ESCAPED, REMOVED = 0, 1, 2, 3
# step status codes of ugkwp_oracle.h (OR_ERR_IDSPACE: a step past the 20
# bits of the birth step in a particle identity samples nothing)
OR_ERR_CAPACITY, OR_ERR_NOCONV, OR_ERR_NONFINITE, OR_ERR_IDSPACE = -3, -4, -5, -9

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint64)


class CProblem(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("G", C.c_int32),
        ("grey", C.c_int32), ("wave_order", C.c_int32), ("si_max_iters", C.c_int32),
        ("bc", C.c_int32 * 4), ("sig_law", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double),
        ("sig_p", C.c_double), ("sig_q", C.c_double), ("sig_cap", C.c_double),
        ("a", C.c_double), ("c", C.c_double), ("eps", C.c_double), ("dt", C.c_double),
        ("omega_ref", C.c_double), ("si_tol", C.c_double), ("src_on", C.c_double),
        ("tau_num_C", C.c_double),
        ("bcT", C.c_double * 4),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("method", C.c_int32),
        ("nu_edges", _dp), ("sigma0", _dp), ("cv", _dp), ("src_T", _dp),
        ("src_amp", _dp), ("src_t_end", C.c_double), ("cv_law", C.c_int32), ("_pad2", C.c_int32),
        ("cv_chi", C.c_double),
        ("nz", C.c_int32), ("bc_z", C.c_int32 * 2), ("_pad3", C.c_int32), ("dz", C.c_double),
        ("bcT_z", C.c_double * 2), ("split_literal", C.c_int32), ("_pad4", C.c_int32),
    ]


class CParticles(C.Structure):
    _fields_ = [("x", _dp), ("y", _dp), ("ox", _dp), ("oy", _dp), ("nu", _dp), ("w", _dp),
                ("id", _up), ("cell", _ip), ("grp", _ip), ("z", _dp), ("oz", _dp)]


RECORD_DTYPE = np.dtype([
    ("id", np.uint64), ("fate", np.int32), ("cell0", np.int32), ("cell1", np.int32),
    ("grp", np.int32), ("nseg", np.int32), ("_pad", np.int32),
    ("x", np.float64), ("y", np.float64), ("ox", np.float64), ("oy", np.float64),
    ("nu", np.float64), ("w", np.float64), ("t_end", np.float64),
    ("z", np.float64), ("oz", np.float64)])


class CTallies(C.Structure):
    _fields_ = [
        ("W", _dp), ("E_surv", _dp), ("E_abs", _dp), ("esc", _dp), ("inflow", _dp),
        ("Fwave", _dp), ("Feq", _dp), ("N", _ip), ("omega", _dp), ("e_eff", _dp),
        ("n_in", C.c_int64), ("n_born", C.c_int64), ("n_survived", C.c_int64),
        ("n_absorbed", C.c_int64), ("n_escaped", C.c_int64), ("n_removed", C.c_int64),
        ("n_segments", C.c_int64), ("si_iters", C.c_int32), ("status", C.c_int32),
        ("E_rad0", C.c_double), ("E_mat0", C.c_double), ("E_rad1", C.c_double),
        ("E_mat1", C.c_double), ("bnd_in_macro", C.c_double), ("bnd_out_macro", C.c_double),
        ("bnd_in_part", C.c_double), ("bnd_out_part", C.c_double), ("src_in", C.c_double),
        ("n_scaled_bins", C.c_int64),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.or_uniform.argtypes = [C.c_uint32, C.c_uint32]
        L.or_uniform.restype = C.c_double
        L.or_draw.argtypes = [C.POINTER(CProblem), C.c_uint64, C.c_int64, C.c_int64]
        L.or_draw.restype = C.c_double
        L.or_sigma.argtypes = [C.POINTER(CProblem), C.c_int, C.c_double, C.c_double]
        L.or_sigma.restype = C.c_double
        L.or_sigma_group.argtypes = [C.POINTER(CProblem), C.c_int, C.c_int, C.c_double]
        L.or_sigma_group.restype = C.c_double
        for f in ("or_mat_energy", "or_heat_capacity"):
            getattr(L, f).argtypes = [C.POINTER(CProblem), C.c_int, C.c_double]
            getattr(L, f).restype = C.c_double
        for n in ("or_planck_integral", "or_planck_dintegral"):
            getattr(L, n).argtypes = [C.c_double, C.c_double]
            getattr(L, n).restype = C.c_double
        for n in ("or_phi", "or_dphi"):
            getattr(L, n).argtypes = [C.POINTER(CProblem), C.c_int, C.c_double]
            getattr(L, n).restype = C.c_double
        L.or_coefs.argtypes = [C.c_double, _dp, _dp, _dp, _dp]
        L.or_nu_cdf.argtypes = [C.c_double] * 4
        L.or_nu_cdf.restype = C.c_double
        L.or_sample_nu.argtypes = [C.c_double] * 4
        L.or_sample_nu.restype = C.c_double
        L.or_stream_particle.argtypes = [
            C.POINTER(CProblem), _dp, C.c_int64, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
            C.c_uint64, _ip, C.c_int32, C.c_int, C.c_int64, _dp, C.c_int64, C.POINTER(CTallies),
            _ip, _dp, _dp, _dp, C.c_int, _ip]
        L.or_stream_particle.restype = C.c_int
        L.or_birth_counts.argtypes = [C.POINTER(CProblem), _dp, _dp, C.POINTER(CTallies),
                                      C.POINTER(C.c_int64)]
        L.or_wave_flux.argtypes = [C.POINTER(CProblem), _dp, _dp, _dp, _dp]
        L.or_source_iteration.argtypes = [C.POINTER(CProblem), _dp, _dp, _dp, _dp, _dp, _dp,
                                          C.POINTER(C.c_int)]
        L.or_step.argtypes = [
            C.POINTER(CProblem), C.c_int64, _dp, _dp, _dp, C.c_int64, C.POINTER(CParticles),
            _dp, _dp, _dp, _dp, C.POINTER(CParticles), C.c_int64, C.POINTER(C.c_int64),
            C.c_void_p, C.c_int64, C.POINTER(CTallies)]
        L.or_init_rho.argtypes = [C.POINTER(CProblem), _dp, _dp]
        L.or_x_num.argtypes = [C.POINTER(CProblem), _dp, C.c_int, C.c_int]
        L.or_x_num.restype = C.c_double
        L.or_dsigma_group.argtypes = [C.POINTER(CProblem), C.c_int, C.c_int, C.c_double,
                                      C.c_double, C.c_double]
        L.or_dsigma_group.restype = C.c_double
        L.or_dcoefs.argtypes = [C.c_double, _dp, _dp, _dp, _dp]
        L.or_wave_flux_tangent.argtypes = [C.POINTER(CProblem), _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_source_iteration_tangent.argtypes = [C.POINTER(CProblem), _dp, _dp, _dp, _dp, _dp,
                                                  _dp, _dp, C.POINTER(C.c_int)]
        L.or_step_tangent.argtypes = [
            C.POINTER(CProblem), C.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, _dp, C.c_int64,
            C.POINTER(CParticles), _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
            C.POINTER(CParticles), _dp, C.c_int64, C.POINTER(C.c_int64), C.POINTER(CTallies)]
        _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


class OracleProblem:
    """Keeps the numpy arrays alive that the C struct points to."""

    def __init__(self, p):
        self.p = p
        self.nu_edges = np.ascontiguousarray(p.nu_edges, dtype=np.float64)
        self.sigma0 = np.ascontiguousarray(p.sigma0, dtype=np.float64)
        self.cv = np.ascontiguousarray(p.cv, dtype=np.float64)
        self.src_T = None if p.src_T is None else np.ascontiguousarray(p.src_T, dtype=np.float64)
        s = CProblem()
        s.dim, s.nx, s.ny, s.G = p.dim, p.nx, (p.ny if p.dim >= 2 else 1), p.G
        s.grey, s.wave_order, s.si_max_iters = p.grey, p.wave_order, p.si_max_iters
        for i in range(4):
            s.bc[i] = int(p.bc[i])
            s.bcT[i] = float(p.bcT[i])
        s.dx, s.dy = p.dx, p.dy
        s.sig_p, s.sig_q, s.sig_cap = p.sig_p, p.sig_q, p.sig_cap
        s.a, s.c, s.eps, s.dt = p.a, p.c, p.eps, p.dt
        s.omega_ref, s.si_tol, s.src_on = p.omega_ref, p.si_tol, p.src_on
        s.tau_num_C = float(getattr(p, "tau_num_C", 0.0))
        s.sig_law = int(getattr(p, "sig_law", 0))
        s.seed, s.instance = p.seed & 0xFFFFFFFFFFFFFFFF, p.instance
        s.method = int(getattr(p, "method", 0))
        s.nu_edges, s.sigma0, s.cv = _d(self.nu_edges), _d(self.sigma0), _d(self.cv)
        s.src_T = _d(self.src_T) if self.src_T is not None else None
        amp = getattr(p, "src_amp", None)
        self.src_amp = None if amp is None else np.ascontiguousarray(amp, dtype=np.float64)
        s.src_amp = _d(self.src_amp) if self.src_amp is not None else None
        s.src_t_end = float(getattr(p, "src_t_end", 0.0))
        s.cv_law = int(getattr(p, "cv_law", 0))
        s.cv_chi = float(getattr(p, "cv_chi", 0.0))
        s.nz = int(getattr(p, "nz", 1))
        s.dz = float(getattr(p, "dz", 1.0))
        bc = list(p.bc) + [0] * (6 - len(p.bc))
        bcT = list(p.bcT) + [0.0] * (6 - len(p.bcT))
        s.bc_z[0], s.bc_z[1] = int(bc[4]), int(bc[5])
        s.bcT_z[0], s.bcT_z[1] = float(bcT[4]), float(bcT[5])
        s.split_literal = int(getattr(p, "split_literal", 0))
        self.s = s

    @property
    def ref(self):
        return C.byref(self.s)


# ---------------------------------------------------------------------------
# building blocks

def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(wa: int, wb: int) -> float:
    return lib().or_uniform(wa, wb)


def draw(prob: OracleProblem, pid: int, step: int, j: int) -> float:
    return lib().or_draw(prob.ref, pid, step, j)


def sigma(prob: OracleProblem, c: int, nu: float, T: float) -> float:
    return lib().or_sigma(prob.ref, c, nu, T)


def mat_energy(prob: OracleProblem, c: int, T: float) -> float:
    return lib().or_mat_energy(prob.ref, c, T)


def heat_capacity(prob: OracleProblem, c: int, T: float) -> float:
    return lib().or_heat_capacity(prob.ref, c, T)


def sigma_group(prob: OracleProblem, c: int, g: int, T: float) -> float:
    return lib().or_sigma_group(prob.ref, c, g, T)


def planck_integral(x1: float, x2: float) -> float:
    return lib().or_planck_integral(x1, x2)


def planck_dintegral(x1: float, x2: float) -> float:
    return lib().or_planck_dintegral(x1, x2)


def phi(prob: OracleProblem, g: int, T: float) -> float:
    return lib().or_phi(prob.ref, g, T)


def dphi(prob: OracleProblem, g: int, T: float) -> float:
    return lib().or_dphi(prob.ref, g, T)


def coefs(x: float):
    """(C2/tau, C4 - e, (C5 + dt e/2)/tau, C4) at x = dt/tau."""
    a, b, c, d = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    lib().or_coefs(x, C.byref(a), C.byref(b), C.byref(c), C.byref(d))
    return a.value, b.value, c.value, d.value


def nu_cdf(nlo, nhi, T, nu) -> float:
    return lib().or_nu_cdf(nlo, nhi, T, nu)


def sample_nu(nlo, nhi, T, eta) -> float:
    return lib().or_sample_nu(nlo, nhi, T, eta)


def init_rho(prob: OracleProblem, T0: np.ndarray) -> np.ndarray:
    p = prob.p
    rho = np.zeros(p.ncell * p.G)
    lib().or_init_rho(prob.ref, _d(np.ascontiguousarray(T0, dtype=np.float64)), _d(rho))
    return rho


class Tallies:
    def __init__(self, p):
        n = p.ncell * p.G
        self.W = np.zeros(n)
        self.E_surv = np.zeros(n)
        self.E_abs = np.zeros(n)
        self.esc = np.zeros(6 * p.G)
        self.inflow = np.zeros(6 * p.G)
        self.Fwave = np.zeros(p.nface * p.G)
        self.Feq = np.zeros(p.nface * p.G)
        self.N = np.zeros(p.nbins, dtype=np.int32)
        self.omega = np.zeros(p.nbins)
        self.e_eff = np.zeros(p.nbins)
        t = CTallies()
        t.W, t.E_surv, t.E_abs = _d(self.W), _d(self.E_surv), _d(self.E_abs)
        t.esc, t.inflow, t.Fwave, t.Feq = _d(self.esc), _d(self.inflow), _d(self.Fwave), _d(self.Feq)
        t.N = self.N.ctypes.data_as(_ip)
        t.omega, t.e_eff = _d(self.omega), _d(self.e_eff)
        self.c = t

    def scalars(self) -> Dict[str, float]:
        return {k: getattr(self.c, k) for k, _ in CTallies._fields_[10:]}


def stream_particle(prob: OracleProblem, T: np.ndarray, step: int, x: float, y: float,
                    ox: float, oy: float, nu: float, w: float, pid: int, cell: int, g: int,
                    newborn: bool, first_draw: int = 0, draws: Optional[np.ndarray] = None,
                    tallies: Optional[Tallies] = None, trace_cap: int = 64):
    """Stream one particle; returns a dict with the end state and the trace."""
    px, py, pox, poy = C.c_double(x), C.c_double(y), C.c_double(ox), C.c_double(oy)
    pc = C.c_int32(cell)
    nseg = C.c_int32(0)
    tend = C.c_double(0.0)
    tx = np.zeros(trace_cap)
    tt = np.zeros(trace_cap)
    ntr = C.c_int(0)
    T = np.ascontiguousarray(T, dtype=np.float64)
    dr = None if draws is None else np.ascontiguousarray(draws, dtype=np.float64)
    fate = lib().or_stream_particle(
        prob.ref, _d(T), step, C.byref(px), C.byref(py), C.byref(pox), C.byref(poy), nu, w, pid,
        C.byref(pc), g, int(newborn), first_draw, None if dr is None else _d(dr),
        0 if dr is None else len(dr), None if tallies is None else C.byref(tallies.c),
        C.byref(nseg), C.byref(tend), _d(tx), _d(tt), trace_cap, C.byref(ntr))
    n = ntr.value
    return dict(fate=fate, x=px.value, y=py.value, ox=pox.value, oy=poy.value, cell=pc.value,
                nseg=nseg.value, t_end=tend.value, trace_x=tx[:n].copy(), trace_t=tt[:n].copy())


def birth_counts(prob: OracleProblem, T: np.ndarray, rho_h: np.ndarray):
    tal = Tallies(prob.p)
    n = C.c_int64(0)
    st = lib().or_birth_counts(prob.ref, _d(np.ascontiguousarray(T, dtype=np.float64)),
                               _d(np.ascontiguousarray(rho_h, dtype=np.float64)), C.byref(tal.c),
                               C.byref(n))
    return st, n.value, tal


def wave_flux(prob: OracleProblem, T, rho_h, e_eff) -> np.ndarray:
    p = prob.p
    F = np.zeros(p.nface * p.G)
    lib().or_wave_flux(prob.ref, _d(np.ascontiguousarray(T, dtype=np.float64)),
                       _d(np.ascontiguousarray(rho_h, dtype=np.float64)),
                       _d(np.ascontiguousarray(e_eff, dtype=np.float64)), _d(F))
    return F


def source_iteration(prob: OracleProblem, T_n, rho_n, R):
    p = prob.p
    T_out = np.zeros(p.ncell)
    rho_out = np.zeros(p.ncell * p.G)
    Feq = np.zeros(p.nface * p.G)
    it = C.c_int(0)
    st = lib().or_source_iteration(prob.ref, _d(np.ascontiguousarray(T_n, dtype=np.float64)),
                                   _d(np.ascontiguousarray(rho_n, dtype=np.float64)),
                                   _d(np.ascontiguousarray(R, dtype=np.float64)),
                                   _d(T_out), _d(rho_out), _d(Feq), C.byref(it))
    return st, T_out, rho_out, Feq, it.value


class ParticleSet:
    """Structure-of-arrays particles (numpy), in the oracle's layout."""

    FIELDS = ("x", "y", "ox", "oy", "nu", "w", "z", "oz")

    def __init__(self, cap: int):
        self.cap = cap
        for f in self.FIELDS:
            setattr(self, f, np.zeros(cap))
        self.id = np.zeros(cap, dtype=np.uint64)
        self.cell = np.zeros(cap, dtype=np.int32)
        self.grp = np.zeros(cap, dtype=np.int32)
        self.n = 0

    def cstruct(self) -> CParticles:
        s = CParticles()
        for f in self.FIELDS:
            setattr(s, f, _d(getattr(self, f)))
        s.id = self.id.ctypes.data_as(_up)
        s.cell = self.cell.ctypes.data_as(_ip)
        s.grp = self.grp.ctypes.data_as(_ip)
        return s

    def view(self) -> Dict[str, np.ndarray]:
        d = {f: getattr(self, f)[: self.n].copy() for f in self.FIELDS}
        d["id"] = self.id[: self.n].copy()
        d["cell"] = self.cell[: self.n].copy()
        d["grp"] = self.grp[: self.n].copy()
        return d

    @staticmethod
    def from_arrays(d: Dict[str, np.ndarray], cap: Optional[int] = None) -> "ParticleSet":
        n = len(d["id"])
        ps = ParticleSet(max(cap or 0, n, 1))
        for f in ParticleSet.FIELDS:
            if f in d:
                getattr(ps, f)[:n] = d[f]
        ps.id[:n] = d["id"]
        ps.cell[:n] = d["cell"]
        ps.grp[:n] = d["grp"]
        ps.n = n
        return ps


class State:
    def __init__(self, p, T, rho, rho_h, particles: ParticleSet, step: int = 0):
        self.p, self.T, self.rho, self.rho_h, self.particles, self.step = p, T, rho, rho_h, particles, step


def initial_state(prob: OracleProblem) -> State:
    p = prob.p
    T = np.ascontiguousarray(p.T0, dtype=np.float64).copy()
    rho = init_rho(prob, T)
    return State(p, T, rho, rho.copy(), ParticleSet(16), 0)


def step(prob: OracleProblem, st: State, records: bool = False, cap_out: Optional[int] = None):
    """One time step; returns (new_state, tallies, records or None, status)."""
    p = prob.p
    pin = st.particles
    cap = cap_out if cap_out is not None else max(p.particle_capacity, 16)
    pout = ParticleSet(cap)
    T_out = np.zeros(p.ncell)
    rho_out = np.zeros(p.ncell * p.G)
    rho_h_out = np.zeros(p.ncell * p.G)
    rho_p_out = np.zeros(p.ncell * p.G)
    tal = Tallies(p)
    n_out = C.c_int64(0)
    rec = None
    rec_cap = 0
    if records:
        # the number of newborns is known only after the birth counts; size
        # generously from a dry count
        stb, n_new, _ = birth_counts(prob, st.T, st.rho_h)
        rec_cap = pin.n + n_new
        rec = np.zeros(max(rec_cap, 1), dtype=RECORD_DTYPE)
    cin = pin.cstruct()
    cout = pout.cstruct()
    status = lib().or_step(
        prob.ref, st.step, _d(st.T), _d(st.rho), _d(st.rho_h), pin.n, C.byref(cin),
        _d(T_out), _d(rho_out), _d(rho_h_out), _d(rho_p_out), C.byref(cout), cap,
        C.byref(n_out), None if rec is None else rec.ctypes.data, rec_cap, C.byref(tal.c))
    pout.n = min(n_out.value, cap)
    new = State(p, T_out, rho_out, rho_h_out, pout, st.step + 1)
    new.rho_p = rho_p_out
    if rec is not None:
        rec = rec[:rec_cap]
    return new, tal, rec, status


# ---------------------------------------------------------------------------
# pathwise derivative (tangent) with respect to the per-cell log-opacity scales

def dsigma_group(prob: OracleProblem, c: int, g: int, T: float, ds: float, dT: float) -> float:
    return lib().or_dsigma_group(prob.ref, c, g, T, ds, dT)


def dcoefs(x: float):
    """x-derivatives (f2', f4', f5', c4') of the flux coefficients."""
    o = [C.c_double() for _ in range(4)]
    lib().or_dcoefs(x, *[C.byref(v) for v in o])
    return tuple(v.value for v in o)


def wave_flux_tangent(prob: OracleProblem, T, dT, ds, rho_h, drho_h, e_eff) -> np.ndarray:
    p = prob.p
    out = np.zeros(p.nface * p.G)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (T, dT, ds, rho_h, drho_h, e_eff)]
    lib().or_wave_flux_tangent(prob.ref, *[_d(v) for v in a], _d(out))
    return out


def source_iteration_tangent(prob: OracleProblem, dT_n, ds, dR, T, rho):
    p = prob.p
    dT = np.zeros(p.ncell)
    drho = np.zeros(p.ncell * p.G)
    it = C.c_int()
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (dT_n, ds, dR, T, rho)]
    st = lib().or_source_iteration_tangent(prob.ref, *[_d(v) for v in a], _d(dT), _d(drho), C.byref(it))
    return st, dT, drho, it.value


class Tangent:
    """Tangent of a state: dT, drho, drho_h and one weight tangent per particle."""

    def __init__(self, p, dT, drho, drho_h, dw):
        self.dT, self.drho, self.drho_h, self.dw = dT, drho, drho_h, dw

    @staticmethod
    def zero(st: State) -> "Tangent":
        p = st.p
        return Tangent(p, np.zeros(p.ncell), np.zeros(p.ncell * p.G), np.zeros(p.ncell * p.G),
                       np.zeros(max(st.particles.cap, 1)))


def step_tangent(prob: OracleProblem, st: State, tg: Tangent, ds, cap_out: Optional[int] = None):
    """One step and its tangent along ds (log-opacity scales) and tg.
    Returns (new_state, new_tangent, tallies, status)."""
    p = prob.p
    pin = st.particles
    cap = cap_out if cap_out is not None else max(p.particle_capacity, 16)
    pout = ParticleSet(cap)
    ncg = p.ncell * p.G
    T_out, dT_out = np.zeros(p.ncell), np.zeros(p.ncell)
    rho_out, drho_out = np.zeros(ncg), np.zeros(ncg)
    rho_h_out, drho_h_out, rho_p_out = np.zeros(ncg), np.zeros(ncg), np.zeros(ncg)
    dw_out = np.zeros(cap)
    dw_in = np.ascontiguousarray(tg.dw, dtype=np.float64)
    if len(dw_in) < max(pin.n, 1):
        raise ValueError("weight tangents shorter than the particle set")
    tal = Tallies(p)
    n_out = C.c_int64(0)
    cin, cout = pin.cstruct(), pout.cstruct()
    ds = np.ascontiguousarray(ds, dtype=np.float64)
    status = lib().or_step_tangent(
        prob.ref, st.step, _d(ds), _d(st.T), _d(tg.dT), _d(st.rho), _d(tg.drho), _d(st.rho_h),
        _d(tg.drho_h), pin.n, C.byref(cin), _d(dw_in), _d(T_out), _d(dT_out), _d(rho_out),
        _d(drho_out), _d(rho_h_out), _d(drho_h_out), _d(rho_p_out), C.byref(cout), _d(dw_out), cap,
        C.byref(n_out), C.byref(tal.c))
    pout.n = min(n_out.value, cap)
    new = State(p, T_out, rho_out, rho_h_out, pout, st.step + 1)
    new.rho_p = rho_p_out
    return new, Tangent(p, dT_out, drho_out, drho_h_out, dw_out), tal, status


def with_log_opacity(p, s):
    """The problem with sigma0_c scaled by exp(s_c)."""
    return p.replace(sigma0=np.asarray(p.sigma0, dtype=np.float64) * np.exp(np.asarray(s, dtype=np.float64)))


def misfit(p, steps: int, T_target, cap: Optional[int] = None, records: bool = False):
    """L = sum_c (T_c - T_target_c)^2 after `steps` oracle steps from the
    initial state; also the per-step records (decisions) when asked."""
    prob = OracleProblem(p)
    st = initial_state(prob)
    recs = []
    for _ in range(steps):
        st, _, rec, status = step(prob, st, records=records, cap_out=cap)
        if status != 0:
            raise RuntimeError("oracle step failed with status %d" % status)
        recs.append(rec)
    return float(np.sum((st.T - T_target) ** 2)), st, recs


def misfit_tangent(p, steps: int, T_target, ds, cap: Optional[int] = None):
    """(L, dL) with dL the pathwise directional derivative of L along ds."""
    prob = OracleProblem(p)
    st = initial_state(prob)
    tg = Tangent.zero(st)
    for _ in range(steps):
        st, tg, _, status = step_tangent(prob, st, tg, ds, cap_out=cap)
        if status != 0:
            raise RuntimeError("oracle tangent step failed with status %d" % status)
    r = st.T - T_target
    return float(np.sum(r * r)), float(np.sum(2.0 * r * tg.dT)), st


def x_num(prob: OracleProblem, T, c: int, g: int) -> float:
    """Delta t / tau_num of cell c, group g at temperatures T."""
    return lib().or_x_num(prob.ref, _d(np.ascontiguousarray(T, dtype=np.float64)), c, g)
