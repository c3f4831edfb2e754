"""Gradients of the cycle-averaged electron number through the adjoint of the step.

The objective is the time average over the run of the number of electrons in the gap,

    J = (1/N) sum_{n=1..N} sum_i c_i n_e(x_i, t_n),   n_e(x_i) = m_n . F_i   (Section 2 moments),

with Clenshaw-Curtis weights c_i of the collocation points on [0, L] (bte operator "ccw"). It is
linear in every state, dJ/dF^n = g = (1/N) c (x) m_n, so the discrete adjoint runs backwards
lambda^N = g, lambda^n = S_n^T lambda^{n+1} + g (n >= 1), where S_n is the step's linear map
(bte_step_adjoint), and the parameter gradient is contracted from the sensitivities the adjoint
steps accumulate (bte_adjoint_gradient). States are recomputed per segment of `checkpoint` steps
from the checkpoints kept in the forward pass.

Parameters (theta, 8 values for the four-process workloads): the cross-section scale factor of
every process, the threshold shift [eV] of every process that has a threshold, and the RF
amplitude V0 [V]. All of it runs in libbte's FP64 kernels; this module orders the calls.
"""
from __future__ import annotations

import copy

import numpy as np

from . import bte


class CycleDensity:
    """A workload (dict as in workloads.py) whose cycle-averaged electron number is differentiated."""

    def __init__(self, cfg: dict, steps: int | None = None, checkpoint: int = 50, h_eV: float = 1e-4):
        self.cfg = copy.deepcopy(cfg)
        self.steps = int(cfg["steps"] if steps is None else steps)
        self.checkpoint = int(checkpoint)
        self.h_eV = float(h_eV)
        procs = self.cfg["processes"]
        self.threshold_of = [j for j, p in enumerate(procs) if p.get("threshold_eV", 0.0) > 0.0]
        self.n_params = len(procs) + len(self.threshold_of) + 1

    def names(self):
        procs = self.cfg["processes"]
        return ([f"scale[{j}:{p['kind']}]" for j, p in enumerate(procs)] +
                [f"threshold[{j}:{procs[j]['kind']}]" for j in self.threshold_of] + ["V0"])

    def theta0(self) -> np.ndarray:
        procs = self.cfg["processes"]
        return np.array([p.get("scale", 1.0) for p in procs] + [0.0] * len(self.threshold_of) + [self.cfg["V0"]])

    def config(self, theta) -> dict:
        """The workload with the parameters applied (scales replace, threshold shifts add)."""
        theta = np.asarray(theta, dtype=np.float64)
        c = copy.deepcopy(self.cfg)
        np_ = len(c["processes"])
        for j, p in enumerate(c["processes"]):
            p["scale"] = float(theta[j])
        for k, j in enumerate(self.threshold_of):
            c["processes"][j]["threshold_eV"] = float(self.cfg["processes"][j]["threshold_eV"] + theta[np_ + k])
        c["V0"] = float(theta[-1])
        return c

    # ------------------------------------------------------------------------------------ passes
    def _weights(self, solver):
        import torch
        c = torch.tensor(solver.operator("ccw"), dtype=torch.float64, device=solver.device)
        m = torch.tensor(solver.operator("mom_n"), dtype=torch.float64, device=solver.device)
        g = (c[:, None] * m[None, :] / self.steps).reshape(solver.nx, solver.nt, solver.nr).contiguous()
        return c, g

    def forward(self, theta):
        """J(theta) and what the adjoint pass needs (solver, checkpoints)."""
        import torch
        cfg = self.config(theta)
        s = bte.Solver(cfg, precision="fp64")
        c, g = self._weights(s)
        F = s.initial_state()
        ckpt = {0: F.clone()}
        J = torch.zeros((), dtype=torch.float64, device=s.device)
        for n in range(self.steps):
            s.step(F, n * cfg["dt_s"])
            ne, _, _ = s.moments(F)
            J += torch.dot(c, ne) / self.steps
            if (n + 1) % self.checkpoint == 0 and n + 1 < self.steps:
                ckpt[n + 1] = F.clone()
        return float(J.item()), (s, ckpt, g, cfg)

    def gradient(self, saved) -> np.ndarray:
        """dJ/dtheta by the adjoint sweep over the segments, last segment first."""
        import torch
        s, ckpt, g, cfg = saved
        dt = cfg["dt_s"]
        nv = s.nv
        SC = torch.zeros((nv, nv), dtype=torch.float64, device=s.device)
        SA = torch.zeros_like(SC)
        lam = g.clone()
        starts = sorted(ckpt)
        for a in reversed(starts):
            b = min(a + self.checkpoint, self.steps)
            states = [ckpt[a].clone()]
            for n in range(a, b - 1):
                F = states[-1].clone()
                s.step(F, n * dt)
                states.append(F)
            for n in range(b - 1, a - 1, -1):
                s.step_adjoint(states[n - a], lam, n * dt, g=g, g_weight=1.0 if n >= 1 else 0.0, SC=SC, SA=SA)
        full = s.adjoint_gradient(SC, SA, self.h_eV)
        np_ = len(cfg["processes"])
        return np.concatenate([full[:np_], full[np_ + np.array(self.threshold_of, dtype=int)], full[-1:]])


def _function():
    import torch

    class _CycleDensityFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, model):
            J, saved = model.forward(theta.detach().cpu().numpy())
            ctx.model, ctx.saved = model, saved
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            grad = ctx.model.gradient(ctx.saved)
            return torch.from_numpy(grad) * gJ.cpu(), None

    return _CycleDensityFn


_FN = None


def cycle_averaged_density(theta, model: CycleDensity):
    """J(theta) as a torch scalar whose backward runs the adjoint (theta: float64 CPU tensor)."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(theta, model)
