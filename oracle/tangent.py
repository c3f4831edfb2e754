"""FP64 CPU oracle for parameter derivatives of the cycle-averaged electron number.

TEST INFRASTRUCTURE ONLY (same rules as oracle/bte.py): only tests/ may import it; it shares no
code with the CUDA path.

The step of eqs. "bte_semi_implicit" (Section 3.4) with a specified field is linear in F,
F^{n+1} = X A_n^{-1} X F^n with A_n = I - dt (K_C(theta) + E_n(V0) K_A) per point. The functional is

    J = (1/N) sum_{n=1..N} sum_i c_i n_e(x_i, t_n),

c_i the Clenshaw-Curtis weights of the collocation points on [0, L]. Forward-mode (tangent)
derivative along one parameter theta_k, differentiating the recursion:

    dF^{n+1} = X A_n^{-1} ( X dF^n + dt (dK/dtheta_k) F*_n ),    F*_n = A_n^{-1} X F^n,
    dJ = (1/N) sum_n sum_i c_i m_n . dF^n_i,

with dK/dscale_j = process j's own K_C at unit scale, dK/dthreshold_j by a central difference of
this oracle's assembly, and dK/dV0 = (sin(2 pi f (t_n + dt/2)) / L) K_A.

Parameters theta (same order as the library's adjoint): the scale factor of every process, the
threshold shift [eV] of every process with a threshold, V0 [V].
"""
from __future__ import annotations

import copy

import numpy as np

from oracle import bte as O


def clenshaw_curtis(nx, L):
    """Weights w with sum_i w_i p(x_i) = int_0^L p dx for every polynomial of degree <= nx - 1, on
    the Chebyshev-Gauss-Lobatto points, from the moment equations in the Chebyshev basis
    (int_{-1}^{1} T_k = 2/(1 - k^2) for even k, 0 for odd k)."""
    N = nx - 1
    s = np.cos(np.pi * np.arange(nx) / N)           # s_i, x_i = (L/2)(1 - s_i)
    k = np.arange(nx)
    T = np.cos(np.outer(k, np.arccos(np.clip(s, -1.0, 1.0))))   # T[k, i] = T_k(s_i)
    mom = np.where(k % 2 == 0, 2.0 / (1.0 - k.astype(float) ** 2 + (k == 1)), 0.0)
    w = np.linalg.solve(T, mom)
    return 0.5 * L * w


def threshold_processes(cfg):
    return [j for j, p in enumerate(cfg["processes"]) if p.get("threshold_eV", 0.0) > 0.0]


def apply(cfg, theta):
    """The workload with parameters theta applied (scales replace, threshold shifts add)."""
    c = copy.deepcopy(cfg)
    procs = c["processes"]
    thr = threshold_processes(cfg)
    for j in range(len(procs)):
        procs[j]["scale"] = float(theta[j])
    for k, j in enumerate(thr):
        procs[j]["threshold_eV"] = float(cfg["processes"][j]["threshold_eV"] + theta[len(procs) + k])
    c["V0"] = float(theta[-1])
    return c


def theta0(cfg):
    procs = cfg["processes"]
    return np.array([p.get("scale", 1.0) for p in procs] + [0.0] * len(threshold_processes(cfg)) + [cfg["V0"]])


def objective(cfg, steps):
    """J of the oracle's own trajectory from the workload's initial state (t_0 = 0)."""
    ops = O.Operators(cfg)
    c = clenshaw_curtis(ops.nx, ops.L)
    F = ops.initial_state()
    J = 0.0
    for n in range(steps):
        F = ops.step(F, n * ops.dt)
        J += c @ ops.moments(F)[0] / steps
    return J


def _operator_derivative(cfg, theta, k, h_eV):
    procs = cfg["processes"]
    np_ = len(procs)
    base = apply(cfg, theta)
    if k < np_:
        one = copy.deepcopy(base)
        p = copy.deepcopy(base["processes"][k])
        p["scale"] = 1.0
        one["processes"] = [p]
        return O.Operators(one).KC, None
    if k < len(theta) - 1:
        j = threshold_processes(cfg)[k - np_]
        up, dn = copy.deepcopy(base), copy.deepcopy(base)
        up["processes"][j]["threshold_eV"] += h_eV
        dn["processes"][j]["threshold_eV"] -= h_eV
        return (O.Operators(up).KC - O.Operators(dn).KC) / (2.0 * h_eV), None
    return None, "V0"


def tangent(cfg, theta, steps, h_eV=1e-4):
    """dJ/dtheta_k for every k, one forward-mode sweep per parameter (dense per-point solves)."""
    theta = np.asarray(theta, dtype=np.float64)
    base = apply(cfg, theta)
    ops = O.Operators(base)
    c = clenshaw_curtis(ops.nx, ops.L)
    out = np.zeros(theta.size)
    for k in range(theta.size):
        dK, kind = _operator_derivative(cfg, theta, k, h_eV)
        F = ops.initial_state()
        dF = np.zeros_like(F)
        dJ = 0.0
        for n in range(steps):
            t = n * ops.dt
            E = ops.field(t + 0.5 * ops.dt)
            G = ops.x_halfstep(F)
            dG = ops.x_halfstep(dF)
            Fs = np.empty_like(G)
            rhs = np.empty_like(G)
            for i in range(ops.nx):
                Fs[i] = ops.v_solve(E[i], G[i].reshape(-1)).reshape(ops.nt, ops.nr)
                if kind == "V0":
                    dKi = np.sin(2.0 * np.pi * base["freq_Hz"] * (t + 0.5 * ops.dt)) / ops.L * ops.KA
                else:
                    dKi = dK
                src = dG[i].reshape(-1) + ops.dt * (dKi @ Fs[i].reshape(-1))
                rhs[i] = ops.v_solve(E[i], src).reshape(ops.nt, ops.nr)
            F = ops.x_halfstep(Fs)
            dF = ops.x_halfstep(rhs)
            dJ += c @ ops.moments(dF)[0] / steps
        out[k] = dJ
    return out
