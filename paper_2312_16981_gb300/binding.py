"""ctypes binding of ``libugkwp.so`` (C ABI in ``include/ugkwp.h``).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library.  PyTorch supplies the device workspace and the stream.  There
is no CPU fallback: if the library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

from .inputs import Problem

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libugkwp.so")
_lib = None

OK = 0
ERRORS = {-1: "ARG", -2: "CUDA", -3: "CAPACITY", -4: "NOCONV", -5: "NONFINITE", -6: "TIMEOUT",
          -7: "WORKSPACE", -8: "UNSUPPORTED"}
ST_CAPACITY, ST_NOCONV, ST_NONFINITE, ST_TIMEOUT, ST_IDSPACE = 1, 2, 4, 8, 16

_dp = C.POINTER(C.c_double)


class UGKWPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("ugkwp error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


class CProblem(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("G", C.c_int32),
        ("grey", C.c_int32), ("wave_order", C.c_int32), ("si_max_iters", C.c_int32),
        ("precision", C.c_int32), ("bc", C.c_int32 * 4), ("sig_law", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double),
        ("sig_p", C.c_double), ("sig_q", C.c_double), ("sig_cap", C.c_double),
        ("a", C.c_double), ("c", C.c_double), ("eps", C.c_double), ("dt", C.c_double),
        ("omega_ref", C.c_double), ("si_tol", C.c_double), ("src_on", C.c_double),
        ("tau_num_C", C.c_double),
        ("bcT", C.c_double * 4), ("seed", C.c_uint64), ("instance", C.c_uint32),
        ("method", C.c_int32), ("particle_capacity", C.c_int64),
        ("nu_edges", _dp), ("sigma0", _dp), ("cv", _dp), ("T0", _dp), ("rho0", _dp),
        ("src_T", _dp),
        ("src_amp", _dp), ("src_t_end", C.c_double), ("cv_law", C.c_int32), ("_pad2", C.c_int32),
        ("cv_chi", C.c_double),
        ("nz", C.c_int32), ("bc_z", C.c_int32 * 2), ("_pad3", C.c_int32), ("dz", C.c_double),
        ("bcT_z", C.c_double * 2), ("split_literal", C.c_int32), ("si_warm32", C.c_int32),
        ("si_pair", C.c_int32), ("_pad6", C.c_int32),
    ]


class CTallyReport(C.Structure):
    _fields_ = [
        ("T", C.c_void_p), ("rho", C.c_void_p), ("rho_h", C.c_void_p), ("rho_p", C.c_void_p),
        ("W", C.c_void_p), ("Fwave", C.c_void_p), ("Feq", C.c_void_p), ("esc", C.c_void_p),
        ("inflow", C.c_void_p),
        ("step", C.c_int64), ("n_particles", C.c_int64), ("n_in", C.c_int64), ("n_born", C.c_int64),
        ("n_survived", C.c_int64), ("n_absorbed", C.c_int64), ("n_escaped", C.c_int64),
        ("n_removed", C.c_int64), ("n_segments", C.c_int64), ("si_iters", C.c_int32),
        ("status_bits", C.c_uint32),
        ("E_rad0", C.c_double), ("E_mat0", C.c_double), ("E_rad1", C.c_double), ("E_mat1", C.c_double),
        ("bnd_in_macro", C.c_double), ("bnd_in_part", C.c_double), ("bnd_out_part", C.c_double),
        ("src_in", C.c_double), ("n_scaled_bins", C.c_int64), ("si_iters32", C.c_int32),
        ("_pad5", C.c_int32),
    ]


class CParticlesHost(C.Structure):
    _fields_ = [("x", _dp), ("y", _dp), ("ox", _dp), ("oy", _dp), ("nu", _dp), ("w", _dp),
                ("id", C.POINTER(C.c_uint64)), ("cell", C.POINTER(C.c_int32)),
                ("grp", C.POINTER(C.c_int32)), ("z", _dp), ("oz", _dp)]


RECORD = np.dtype([
    ("id", np.uint64), ("fate", np.int32), ("cell0", np.int32), ("cell1", np.int32),
    ("grp", np.int32), ("nseg", np.int32), ("_pad", np.int32),
    ("x", np.float64), ("y", np.float64), ("ox", np.float64), ("oy", np.float64),
    ("nu", np.float64), ("w", np.float64), ("t_end", np.float64),
    ("z", np.float64), ("oz", np.float64)])

FUNCTIONS = {
    "ugkwp_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "ugkwp_init": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "ugkwp_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "ugkwp_step_timed": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_float)]),
    "ugkwp_tallies": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ugkwp_get_state": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _dp, C.c_void_p, C.c_int64,
                                  C.POINTER(C.c_int64), C.c_void_p]),
    "ugkwp_set_state": (C.c_int, [C.c_void_p, _dp, _dp, _dp, C.c_void_p, C.c_int64, C.c_int64,
                                  C.c_void_p]),
    "ugkwp_set_records": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "ugkwp_workspace_size_ensemble": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]),
    "ugkwp_init_ensemble": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                      C.POINTER(C.c_void_p)]),
    "ugkwp_tallies_member": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "ugkwp_get_state_member": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, C.c_void_p, C.c_int64,
                                         C.POINTER(C.c_int64), C.c_void_p]),
    "ugkwp_set_state_member": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, C.c_void_p, C.c_int64,
                                         C.c_int64, C.c_void_p]),
    "ugkwp_last_error": (C.c_char_p, [C.c_void_p]),
    "ugkwp_checkpoint_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "ugkwp_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ugkwp_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ugkwp_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "ugkwp_set_wait_limit": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p]),
    "ugkwp_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p,
                                 C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "ugkwp_tape_size": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_size_t)]),
    "ugkwp_step_taped": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int64, C.c_void_p]),
    "ugkwp_adjoint_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "ugkwp_adjoint_seed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "ugkwp_adjoint_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int64, C.c_void_p,
                                     C.c_size_t, C.c_void_p]),
    "ugkwp_adjoint_remap": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                                      C.c_void_p]),
    "ugkwp_adjoint_result": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_uint32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_uint64), C.c_void_p]),
    "ugkwp_destroy": (None, [C.c_void_p]),
    "ugkwp_philox": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_int64, C.c_void_p]),
    "ugkwp_planck": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    "ugkwp_coefs": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ugkwp_sample_nu": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_double,
                                  C.c_void_p, C.c_void_p]),
    "ugkwp_exclusive_scan": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t,
                                       C.c_void_p]),
    "ugkwp_exclusive_scan_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
}


def scan_scratch_bytes(n: int) -> int:
    return 4 * ((n + 4095) // 4096) + 4


def load(path: str = LIB_PATH):
    """Load the CUDA library (built by ``paper_2312_16981_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libugkwp.so is not built (%s); run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        for name, (res, args) in FUNCTIONS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, handle=None):
    if code != OK:
        msg = load().ugkwp_last_error(handle)
        raise UGKWPError(code, msg.decode() if msg else "")


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr())


class _HostProblem:
    """C problem struct plus the host arrays it points to."""

    def __init__(self, p: Problem, rho0: Optional[np.ndarray] = None):
        keep = {}

        def arr(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            if a.size < n:
                raise ValueError("array of %d values where the problem needs %d" % (a.size, n))
            keep[id(a)] = a
            return a.ctypes.data_as(_dp)

        s = CProblem()
        s.dim, s.nx, s.ny, s.G = p.dim, p.nx, (p.ny if p.dim >= 2 else 1), p.G
        s.grey, s.wave_order, s.si_max_iters, s.precision = p.grey, p.wave_order, p.si_max_iters, p.precision
        for i in range(4):
            s.bc[i] = int(p.bc[i])
            s.bcT[i] = float(p.bcT[i])
        s.dx, s.dy = p.dx, p.dy
        s.sig_p, s.sig_q, s.sig_cap = p.sig_p, p.sig_q, p.sig_cap
        s.a, s.c, s.eps, s.dt = p.a, p.c, p.eps, p.dt
        s.omega_ref, s.si_tol, s.src_on = p.omega_ref, p.si_tol, p.src_on
        s.tau_num_C = float(p.tau_num_C)
        s.sig_law = int(p.sig_law)
        s.seed, s.instance = p.seed & 0xFFFFFFFFFFFFFFFF, p.instance
        s.method = int(getattr(p, "method", 0))
        s.particle_capacity = int(p.particle_capacity)
        s.nu_edges = arr(p.nu_edges, p.G + 1)
        s.sigma0 = arr(p.sigma0, p.ncell)
        s.cv = arr(p.cv, p.ncell)
        s.T0 = arr(p.T0, p.ncell)
        s.rho0 = arr(rho0, p.ncell * p.G)
        s.src_T = arr(p.src_T, p.ncell)
        s.src_amp = arr(getattr(p, "src_amp", None), p.ncell)
        s.src_t_end = float(getattr(p, "src_t_end", 0.0))
        s.cv_law = int(getattr(p, "cv_law", 0))
        s.cv_chi = float(getattr(p, "cv_chi", 0.0))
        s.nz = int(p.nz) if p.dim == 3 else 1
        s.dz = float(p.dz) if p.dim == 3 else 1.0
        bc = list(p.bc) + [0] * (6 - len(p.bc))
        bcT = list(p.bcT) + [0.0] * (6 - len(p.bcT))
        s.bc_z[0], s.bc_z[1] = int(bc[4]), int(bc[5])
        s.bcT_z[0], s.bcT_z[1] = float(bcT[4]), float(bcT[5])
        s.split_literal = int(getattr(p, "split_literal", 0))
        s.si_warm32 = int(getattr(p, "si_warm32", 0))
        s.si_pair = int(getattr(p, "si_pair", 0))
        self.s = s
        self._keep = keep


def workspace_bytes(p: Problem) -> int:
    hp = _HostProblem(p)
    n = C.c_size_t()
    _check(load().ugkwp_workspace_size(C.byref(hp.s), C.byref(n)))
    return n.value


class Simulation:
    """One UGKWP problem (or an ensemble of independent ones) resident on a GPU."""

    def __init__(self, p, device: str = "cuda:0", rho0: Optional[np.ndarray] = None,
                 stream=None):
        import torch
        L = load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the UGKWP library has no CPU path")
        probs = list(p) if isinstance(p, (list, tuple)) else [p]
        self.members = probs
        self.p = probs[0]
        self.device = torch.device(device)
        self.stream = stream
        hps = [_HostProblem(q, rho0 if k == 0 else None) for k, q in enumerate(probs)]
        arr = (CProblem * len(probs))(*[hp.s for hp in hps])
        n = C.c_size_t()
        _check(L.ugkwp_workspace_size_ensemble(arr, len(probs), C.byref(n)))
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.ugkwp_init_ensemble(arr, len(probs), C.c_void_p(_ptr(self.workspace)), n.value,
                                         C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h
        self._records = None

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().ugkwp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _check(load().ugkwp_step(self.h, int(n), C.c_void_p(_stream_ptr(self.stream))), self.h)

    def step_timed(self):
        """One step; returns device milliseconds: total, birth+scan, wave flux,
        particles, source iteration, end of step."""
        ms = (C.c_float * 6)()
        _check(load().ugkwp_step_timed(self.h, C.c_void_p(_stream_ptr(self.stream)), ms), self.h)
        return list(ms)

    def tallies(self, member: int = 0) -> Dict:
        r = CTallyReport()
        _check(load().ugkwp_tallies_member(self.h, member, C.byref(r),
                                           C.c_void_p(_stream_ptr(self.stream))), self.h)
        out = {k: getattr(r, k) for k, _ in CTallyReport._fields_[9:] if not k.startswith("_")}
        out["ptr"] = {k: getattr(r, k) for k, _ in CTallyReport._fields_[:9]}
        return out

    def log_tallies(self, out, member: int = 0, **extra) -> Dict:
        """Append this step's report (counters, iterations, status bits and the
        energy ledger, with its residual) to `out` -- a path or an open text
        file -- as one JSON line; returns the record."""
        import json
        t = self.tallies(member=member)
        rec = {k: v for k, v in t.items() if k != "ptr"}
        rec["ledger_residual"] = ((t["E_rad1"] + t["E_mat1"]) - (t["E_rad0"] + t["E_mat0"])
                                  - (t["bnd_in_macro"] + t["bnd_in_part"] - t["bnd_out_part"] + t["src_in"]))
        rec["member"] = member
        rec.update(extra)
        line = json.dumps(rec) + "\n"
        if hasattr(out, "write"):
            out.write(line)
        else:
            with open(out, "a") as f:
                f.write(line)
        return rec

    def device_array(self, name: str):
        """A torch view (float64, on the device) of a tally array."""
        import torch
        r = self.tallies()
        p = self.p
        n = {"T": p.ncell, "rho": p.ncell * p.G, "rho_h": p.ncell * p.G, "rho_p": p.ncell * p.G,
             "W": p.ncell * p.G, "Fwave": p.nface * p.G, "Feq": p.nface * p.G, "esc": 6 * p.G,
             "inflow": 6 * p.G}[name]
        off = r["ptr"][name] - _ptr(self.workspace)
        return self.workspace[off: off + 8 * n].view(torch.float64)

    def get_state(self, cap: Optional[int] = None, member: int = 0) -> Dict[str, np.ndarray]:
        p = self.members[member]
        T = np.zeros(p.ncell)
        rho = np.zeros(p.ncell * p.G)
        rho_h = np.zeros_like(rho)
        rho_p = np.zeros_like(rho)
        n = C.c_int64()
        L = load()
        sp = C.c_void_p(_stream_ptr(self.stream))
        _check(L.ugkwp_get_state_member(self.h, member, T.ctypes.data_as(_dp), rho.ctypes.data_as(_dp),
                                        rho_h.ctypes.data_as(_dp), rho_p.ctypes.data_as(_dp), None, 0,
                                        C.byref(n), sp), self.h)
        m = n.value if cap is None else min(cap, n.value)
        parts = {f: np.zeros(max(m, 1)) for f in ("x", "y", "ox", "oy", "nu", "w", "z", "oz")}
        parts["id"] = np.zeros(max(m, 1), dtype=np.uint64)
        parts["cell"] = np.zeros(max(m, 1), dtype=np.int32)
        parts["grp"] = np.zeros(max(m, 1), dtype=np.int32)
        cs = CParticlesHost(*[parts[f].ctypes.data_as(_dp) for f in ("x", "y", "ox", "oy", "nu", "w")],
                            parts["id"].ctypes.data_as(C.POINTER(C.c_uint64)),
                            parts["cell"].ctypes.data_as(C.POINTER(C.c_int32)),
                            parts["grp"].ctypes.data_as(C.POINTER(C.c_int32)),
                            parts["z"].ctypes.data_as(_dp), parts["oz"].ctypes.data_as(_dp))
        if m > 0:
            _check(L.ugkwp_get_state_member(self.h, member, None, None, None, None, C.byref(cs), m,
                                            C.byref(n), sp), self.h)
        parts = {k: v[:m] for k, v in parts.items()}
        return dict(T=T, rho=rho, rho_h=rho_h, rho_p=rho_p, particles=parts, n=n.value)

    def set_state(self, T, rho, rho_h, particles: Optional[Dict[str, np.ndarray]] = None,
                  step: int = 0, member: int = 0):
        L = load()
        T = np.ascontiguousarray(T, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        rho_h = np.ascontiguousarray(rho_h, dtype=np.float64)
        n = 0 if particles is None else len(particles["id"])
        keep = []
        cs = None
        if n:
            arrs = {}
            for f in ("x", "y", "ox", "oy", "nu", "w", "z", "oz"):
                if f in particles:
                    arrs[f] = np.ascontiguousarray(particles[f], dtype=np.float64)
                else:
                    arrs[f] = np.zeros(n)
            arrs["id"] = np.ascontiguousarray(particles["id"], dtype=np.uint64)
            arrs["cell"] = np.ascontiguousarray(particles["cell"], dtype=np.int32)
            arrs["grp"] = np.ascontiguousarray(particles["grp"], dtype=np.int32)
            keep.append(arrs)
            cs = CParticlesHost(*[arrs[f].ctypes.data_as(_dp) for f in ("x", "y", "ox", "oy", "nu", "w")],
                                arrs["id"].ctypes.data_as(C.POINTER(C.c_uint64)),
                                arrs["cell"].ctypes.data_as(C.POINTER(C.c_int32)),
                                arrs["grp"].ctypes.data_as(C.POINTER(C.c_int32)),
                                arrs["z"].ctypes.data_as(_dp), arrs["oz"].ctypes.data_as(_dp))
        _check(L.ugkwp_set_state_member(self.h, member, T.ctypes.data_as(_dp), rho.ctypes.data_as(_dp),
                                        rho_h.ctypes.data_as(_dp), None if cs is None else C.byref(cs), n,
                                        int(step), C.c_void_p(_stream_ptr(self.stream))), self.h)

    def checkpoint_buffer(self):
        """A device buffer (torch uint8) large enough for one checkpoint."""
        import torch
        n = C.c_size_t()
        _check(load().ugkwp_checkpoint_size(self.h, C.byref(n)), self.h)
        return torch.empty(n.value, dtype=torch.uint8, device=self.device)

    def checkpoint(self, buf):
        _check(load().ugkwp_checkpoint(self.h, C.c_void_p(_ptr(buf)), buf.numel(),
                                       C.c_void_p(_stream_ptr(self.stream))), self.h)

    def restore(self, buf):
        _check(load().ugkwp_restore(self.h, C.c_void_p(_ptr(buf)), buf.numel(),
                                    C.c_void_p(_stream_ptr(self.stream))), self.h)

    # ---- adjoint (pathwise gradient with respect to log sigma0 per cell)
    def tape_buffer(self, rec_cap: int):
        """A device buffer for one step's tape holding up to rec_cap particles."""
        import torch
        n = C.c_size_t()
        _check(load().ugkwp_tape_size(self.h, int(rec_cap), C.byref(n)), self.h)
        return torch.empty(n.value, dtype=torch.uint8, device=self.device)

    def step_taped(self, tape, rec_cap: int):
        _check(load().ugkwp_step_taped(self.h, C.c_void_p(_ptr(tape)), tape.numel(), int(rec_cap),
                                       C.c_void_p(_stream_ptr(self.stream))), self.h)

    def adjoint_buffer(self):
        import torch
        n = C.c_size_t()
        _check(load().ugkwp_adjoint_workspace_size(self.h, C.byref(n)), self.h)
        return torch.empty(n.value, dtype=torch.uint8, device=self.device)

    def adjoint_seed(self, adj, dL_dT=None):
        """dL_dT: torch float64 tensor [ncell] on this device (None: zero)."""
        if dL_dT is not None:
            assert dL_dT.dtype.is_floating_point and dL_dT.numel() == self.p.ncell
        ptr = None if dL_dT is None else C.c_void_p(_ptr(dL_dT.contiguous()))
        _check(load().ugkwp_adjoint_seed(self.h, C.c_void_p(_ptr(adj)), adj.numel(), ptr,
                                         C.c_void_p(_stream_ptr(self.stream))), self.h)

    def adjoint_step(self, tape, rec_cap: int, adj):
        _check(load().ugkwp_adjoint_step(self.h, C.c_void_p(_ptr(tape)), tape.numel(), int(rec_cap),
                                         C.c_void_p(_ptr(adj)), adj.numel(),
                                         C.c_void_p(_stream_ptr(self.stream))), self.h)

    def adjoint_remap(self, adj, ckpt):
        """Re-index the particles' weight adjoints from checkpoint `ckpt`'s
        particle order to the current one (by particle identity)."""
        _check(load().ugkwp_adjoint_remap(self.h, C.c_void_p(_ptr(adj)), adj.numel(), C.c_void_p(_ptr(ckpt)),
                                          ckpt.numel(), C.c_void_p(_stream_ptr(self.stream))), self.h)

    def adjoint_result(self, adj):
        """(dL/ds, dL/dT of the first reversed step's input, status bits, last
        adjoint source iterations, particles unmatched across checkpoints);
        the arrays are torch float64 on the device."""
        import torch
        ds = torch.empty(self.p.ncell, dtype=torch.float64, device=self.device)
        dT = torch.empty(self.p.ncell, dtype=torch.float64, device=self.device)
        st = C.c_uint32()
        it = C.c_int32()
        um = C.c_uint64()
        _check(load().ugkwp_adjoint_result(self.h, C.c_void_p(_ptr(adj)), adj.numel(), C.c_void_p(_ptr(ds)),
                                           C.c_void_p(_ptr(dT)), C.byref(st), C.byref(it), C.byref(um),
                                           C.c_void_p(_stream_ptr(self.stream))), self.h)
        return ds, dT, st.value, it.value, um.value

    def set_launch(self, block: int, particles_per_thread: int = 1, blocks_per_sm: int = 0):
        _check(load().ugkwp_set_launch(self.h, block, particles_per_thread, blocks_per_sm), self.h)

    def set_wait_limit(self, spins: int = 0, extra_arrivals: int = 0):
        """Bound the source iteration's barrier waits to `spins` polls (0: the
        default); extra_arrivals > 0 makes every wait run out (failure
        injection for tests)."""
        _check(load().ugkwp_set_wait_limit(self.h, int(spins), int(extra_arrivals),
                                           C.c_void_p(_stream_ptr(self.stream))), self.h)

    def autotune(self, steps: int = 2, cache: Optional[str] = None):
        """Pick the particle kernel's launch shape by timing each candidate on
        identical steps (state saved and restored).  With `cache` (a JSON
        file), a shape found before for the same GPU and workload signature
        is reused without timing."""
        import json
        import torch
        key = None
        if cache:
            props = torch.cuda.get_device_properties(self.device)
            total = sum(self.get_state(cap=0, member=m)["n"] for m in range(len(self.members)))
            key = "%s|sm%d|dim%d|prec%d|members%d|particles2^%d" % (
                props.name, props.multi_processor_count, self.p.dim, self.p.precision,
                len(self.members), max(0, int(total).bit_length()))
            try:
                with open(cache) as f:
                    known = json.load(f)
            except (OSError, ValueError):
                known = {}
            if key in known:
                b, ppt, per, ms = known[key]
                self.set_launch(b, ppt, per)
                return {"block": b, "particles_per_thread": ppt, "blocks_per_sm": per, "ms": ms, "cached": True}
        buf = self.checkpoint_buffer()
        best = (C.c_int * 3)()
        ms = C.c_float()
        _check(load().ugkwp_autotune(self.h, C.c_void_p(_ptr(buf)), buf.numel(), steps,
                                     C.c_void_p(_stream_ptr(self.stream)), best, C.byref(ms)), self.h)
        out = {"block": best[0], "particles_per_thread": best[1], "blocks_per_sm": best[2],
               "ms": ms.value, "cached": False}
        if cache:
            import os
            try:
                with open(cache) as f:
                    known = json.load(f)
            except (OSError, ValueError):
                known = {}
            known[key] = [best[0], best[1], best[2], ms.value]
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(known, f, indent=1)
        return out

    def attach_records(self, cap: int):
        import torch
        self._records = torch.zeros(cap * RECORD.itemsize, dtype=torch.uint8, device=self.device)
        self._rec_cap = cap
        _check(load().ugkwp_set_records(self.h, C.c_void_p(_ptr(self._records)), cap), self.h)

    def detach_records(self):
        _check(load().ugkwp_set_records(self.h, None, 0), self.h)
        self._records = None

    def records(self, n: int) -> np.ndarray:
        import torch
        torch.cuda.synchronize(self.device)
        n = min(n, self._rec_cap)
        raw = self._records[: n * RECORD.itemsize].cpu().numpy()
        return raw.view(RECORD).copy()


# ---------------------------------------------------------------------------
# kernel-level entry points (torch tensors on the device)

def philox(ctr, k0: int, k1: int):
    """ctr: int32/uint32-valued tensor [n, 4] on the device -> [n, 4] words (int64 view)."""
    import torch
    ctr = ctr.contiguous().to(torch.int32)
    out = torch.empty_like(ctr)
    _check(load().ugkwp_philox(C.c_void_p(_ptr(ctr)), k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF,
                               C.c_void_p(_ptr(out)), ctr.shape[0], C.c_void_p(_stream_ptr())))
    return out.to(torch.int64) & 0xFFFFFFFF


def planck(T, nu_edges):
    """b_g(T) and d_g(T) for temperatures T [n] and edges [G+1] (device float64)."""
    import torch
    T = T.contiguous().to(torch.float64)
    nu = nu_edges.contiguous().to(torch.float64)
    G = nu.numel() - 1
    b = torch.empty(T.numel(), G, dtype=torch.float64, device=T.device)
    d = torch.empty_like(b)
    _check(load().ugkwp_planck(C.c_void_p(_ptr(T)), T.numel(), C.c_void_p(_ptr(nu)), G,
                               C.c_void_p(_ptr(b)), C.c_void_p(_ptr(d)), C.c_void_p(_stream_ptr())))
    return b, d


def coefs(x):
    import torch
    x = x.contiguous().to(torch.float64)
    out = torch.empty(x.numel(), 4, dtype=torch.float64, device=x.device)
    _check(load().ugkwp_coefs(C.c_void_p(_ptr(x)), x.numel(), C.c_void_p(_ptr(out)),
                              C.c_void_p(_stream_ptr())))
    return out


def sample_nu(eta, nlo: float, nhi: float, T: float):
    import torch
    eta = eta.contiguous().to(torch.float64)
    nu = torch.empty_like(eta)
    _check(load().ugkwp_sample_nu(C.c_void_p(_ptr(eta)), eta.numel(), nlo, nhi, T,
                                  C.c_void_p(_ptr(nu)), C.c_void_p(_stream_ptr())))
    return nu


def exclusive_scan(counts):
    """Exclusive prefix sum of uint32 counts (int32 tensor on the device) ->
    [n + 1] offsets (int64 view of the uint32 results)."""
    import torch
    counts = counts.contiguous().to(torch.int32)
    n = counts.numel()
    out = torch.empty(n + 1, dtype=torch.int32, device=counts.device)
    scratch = torch.empty(scan_scratch_bytes(n), dtype=torch.uint8, device=counts.device)
    _check(load().ugkwp_exclusive_scan(C.c_void_p(_ptr(counts) if n else 0), n, C.c_void_p(_ptr(out)),
                                       C.c_void_p(_ptr(scratch)), scratch.numel(),
                                       C.c_void_p(_stream_ptr())))
    return out.to(torch.int64) & 0xFFFFFFFF
