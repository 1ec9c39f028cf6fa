"""Gradient of a material-temperature misfit with respect to per-cell
log-opacity scales, through the library's adjoint.

The parameters s_c scale each cell's opacity: sigma0_c -> sigma0_c e^{s_c}.
The loss is L = sum_c (T_c - T_target_c)^2 after `steps` steps from the
problem's initial state.  The gradient is pathwise: every Monte Carlo
decision is held as the forward run took it, with the same Philox draws
(common random numbers), so it is the derivative of the sampled path, the
quantity central finite differences with common random numbers approach.

Memory: the forward run keeps a device checkpoint every `ckpt_every` steps;
the backward pass restores each checkpoint in turn, re-runs its steps with
tapes (one per step, holding per-particle start cell, end cell, output slot
and group) and reverses them.  Everything runs in the CUDA library; this
module only sequences the calls.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import binding as B
from .inputs import Problem


def with_log_opacity(p: Problem, s) -> Problem:
    """The problem with sigma0_c scaled by exp(s_c)."""
    s = np.asarray(s, dtype=np.float64).reshape(-1)
    if s.size != p.ncell:
        raise ValueError("one log-opacity scale per cell expected")
    return p.replace(sigma0=np.asarray(p.sigma0, dtype=np.float64) * np.exp(s))


@dataclass
class ForwardRun:
    sim: "B.Simulation"
    checkpoints: List[Tuple[int, object]]   # (step offset, device buffer)
    T: object                               # torch float64 [ncell] on the device
    steps: int
    ckpt_every: int
    max_processed: int                      # largest survivors-in + newborns of a step
    unmatched: int = 0                      # particles unmatched across checkpoints (backward)


def forward(p: Problem, steps: int, ckpt_every: int = 20, device: str = "cuda:0") -> ForwardRun:
    """Run `steps` steps from the initial state, checkpointing every
    `ckpt_every` steps; returns the run with T at the end."""
    if steps < 1 or ckpt_every < 1:
        raise ValueError("steps and ckpt_every must be >= 1")
    sim = B.Simulation(p, device=device)
    ckpts = []
    most = 0
    for n0 in range(0, steps, ckpt_every):
        buf = sim.checkpoint_buffer()
        sim.checkpoint(buf)
        ckpts.append((n0, buf))
        for _ in range(min(ckpt_every, steps - n0)):
            sim.step(1)
            t = sim.tallies()
            most = max(most, t["n_in"] + t["n_born"])
    t = sim.tallies()
    if t["status_bits"]:
        raise B.UGKWPError(-3, "forward run reported status bits %d" % t["status_bits"])
    return ForwardRun(sim, ckpts, sim.device_array("T").clone(), steps, ckpt_every, most)


def backward(run: ForwardRun, dL_dT, rec_cap: Optional[int] = None):
    """dL/ds for the adjoint dL/dT of the final temperature (torch float64
    on the device).  Returns (dL/ds on the device, adjoint SI iterations of the
    last reversed step)."""
    import torch
    sim = run.sim
    if rec_cap is None:
        # restored steps repeat the forward ones up to roundoff: leave a margin
        rec_cap = int(1.1 * run.max_processed) + 4096
    adj = sim.adjoint_buffer()
    sim.adjoint_seed(adj, dL_dT.to(device=sim.device, dtype=torch.float64).contiguous())
    tapes = [sim.tape_buffer(rec_cap) for _ in range(min(run.ckpt_every, run.steps))]
    later = None   # checkpoint of the segment reversed last (its particle order indexes the adjoints)
    for n0, buf in reversed(run.checkpoints):
        m = min(run.ckpt_every, run.steps - n0)
        sim.restore(buf)
        for j in range(m):
            sim.step_taped(tapes[j], rec_cap)
        if later is not None:
            sim.adjoint_remap(adj, later)
        for j in reversed(range(m)):
            sim.adjoint_step(tapes[j], rec_cap, adj)
        later = buf
    ds, _, status, iters, unmatched = sim.adjoint_result(adj)
    fwd = sim.tallies()["status_bits"]
    if status or fwd:
        raise B.UGKWPError(-3, "adjoint status bits %d, replay status bits %d" % (status, fwd))
    run.unmatched = unmatched
    return ds, iters


def misfit_and_gradient(p: Problem, s, steps: int, T_target, ckpt_every: int = 20,
                        device: str = "cuda:0"):
    """(L, dL/ds as numpy) for L = sum (T - T_target)^2 after `steps` steps."""
    import torch
    run = forward(with_log_opacity(p, s), steps, ckpt_every, device)
    Tt = torch.as_tensor(np.asarray(T_target, dtype=np.float64), device=run.T.device)
    r = run.T - Tt
    L = float((r * r).sum())
    ds, _ = backward(run, 2.0 * r)
    run.sim.close()
    return L, ds.cpu().numpy()


def misfit(p: Problem, s, steps: int, T_target, device: str = "cuda:0") -> float:
    """L alone (one forward run, CUDA-graph steps)."""
    sim = B.Simulation(with_log_opacity(p, s), device=device)
    sim.step(steps)
    T = sim.get_state(cap=0)["T"]
    st = sim.tallies()["status_bits"]
    sim.close()
    if st:
        raise B.UGKWPError(-3, "forward run reported status bits %d" % st)
    return float(np.sum((T - np.asarray(T_target)) ** 2))


def misfit_with_decisions(p: Problem, s, steps: int, T_target, device: str = "cuda:0"):
    """(L, fingerprint): the fingerprint lists, per step, the counts of births,
    collisions, escapes, survivors and flight segments -- two runs with the
    same fingerprint took the same Monte Carlo decisions (up to an exchange
    that leaves every count unchanged)."""
    sim = B.Simulation(with_log_opacity(p, s), device=device)
    fp = []
    for _ in range(steps):
        sim.step(1)
        t = sim.tallies()
        fp.append((t["n_born"], t["n_absorbed"], t["n_escaped"], t["n_survived"], t["n_segments"]))
    T = sim.get_state(cap=0)["T"]
    st = sim.tallies()["status_bits"]
    sim.close()
    if st:
        raise B.UGKWPError(-3, "forward run reported status bits %d" % st)
    return float(np.sum((T - np.asarray(T_target)) ** 2)), tuple(fp)


def crn_finite_differences(p: Problem, s, steps: int, T_target, cells: Sequence[int], h: float = 1e-6,
                           device: str = "cuda:0", retries: int = 0):
    """Central differences (L(s + h e_i) - L(s - h e_i))/2h with the same seed
    (common random numbers) for each listed cell i.

    With retries = 0, returns the differences.  With retries > 0, also checks
    that the + and - runs took the same decisions as the unperturbed run (a
    decision that flips inside [s - h, s + h] makes the difference measure a
    jump, not a derivative) and, where one flipped, tries again with h/10, up
    to `retries` times; returns (differences, h used per cell, flipped mask)."""
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros(len(cells))
    if retries <= 0:
        for k, c in enumerate(cells):
            e = np.zeros_like(s)
            e[c] = h
            out[k] = (misfit(p, s + e, steps, T_target, device) - misfit(p, s - e, steps, T_target, device)) / (2 * h)
        return out
    _, fp0 = misfit_with_decisions(p, s, steps, T_target, device)
    used = np.zeros(len(cells))
    flipped = np.zeros(len(cells), dtype=bool)
    for k, c in enumerate(cells):
        hk = h
        for attempt in range(retries + 1):
            e = np.zeros_like(s)
            e[c] = hk
            Lp, fpp = misfit_with_decisions(p, s + e, steps, T_target, device)
            Lm, fpm = misfit_with_decisions(p, s - e, steps, T_target, device)
            out[k], used[k] = (Lp - Lm) / (2 * hk), hk
            flipped[k] = fpp != fp0 or fpm != fp0
            if not flipped[k]:
                break
            hk *= 0.1
    return out, used, flipped


def _autograd():
    import torch

    class LogOpacityMisfit(torch.autograd.Function):
        """L(s) = sum_c (T_c(s) - T_target_c)^2 after `steps` UGKWP steps, with
        its pathwise gradient from the adjoint (checkpoint every `ckpt_every`
        steps).  s: float64 tensor [ncell] (any device)."""

        @staticmethod
        def forward(ctx, s, problem, steps, T_target, ckpt_every=20, device="cuda:0"):
            run = forward(with_log_opacity(problem, s.detach().cpu().numpy()), int(steps), int(ckpt_every), device)
            Tt = torch.as_tensor(np.asarray(T_target, dtype=np.float64), device=run.T.device)
            r = run.T - Tt
            ctx.run = run
            ctx.r = r
            ctx.s_meta = (s.device, s.dtype)
            return (r * r).sum().to(device=s.device, dtype=s.dtype)

        @staticmethod
        def backward(ctx, gL):
            run = ctx.run
            ds, _ = backward(run, 2.0 * ctx.r * float(gL))
            run.sim.close()
            ctx.run = None
            dev, dt = ctx.s_meta
            return ds.to(device=dev, dtype=dt), None, None, None, None, None

    return LogOpacityMisfit


_FN = None


def log_opacity_misfit(s, problem: Problem, steps: int, T_target, ckpt_every: int = 20,
                       device: str = "cuda:0"):
    """Differentiable L(s) (a torch scalar); call .backward() for dL/ds."""
    global _FN
    if _FN is None:
        _FN = _autograd()
    return _FN.apply(s, problem, steps, T_target, ckpt_every, device)
