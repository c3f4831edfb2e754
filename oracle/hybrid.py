"""FP64 CPU oracle for the self-consistent (hybrid) parts of the method: electrostatics, the ion
fluid step, the semi-implicit electron step with the field recomputed from the electrons, and the
fully-implicit electron step (arXiv 2502.16555, Sections 2.3 and 3.4).

TEST INFRASTRUCTURE ONLY (same rules as oracle/bte.py): only tests/ and bench.py's CPU leg may
import it; it shares no code with the CUDA path.

What it computes, in the notation of Section 3.4 (x on the Chebyshev-Gauss-Lobatto points of
oracle.bte, ascending, x_0 = 0, x_{Nx-1} = L):

  Electrostatics (eqs. "hybrid_cnt_c", "hybrid_discrete_c", "voltage_bc"): d^2V/dx^2 =
  -(e/eps0)(n_i - n_e) on the interior points, V(0) = V0 sin(2 pi f t), V(L) = 0, E = -D_x V.
  Linear in the charge: E = Lop (n_i - n_e) + V(0) E_1, with E_1 the field of a unit left voltage
  (uniform, 1/L).

  Ion step (eq. "fluid_step", flux eq. "hybrid_cnt_a_flux", wall condition eq. "fl_ion_bc"):
  (n^{n+1} - n^n)/dt + D_x J(n^{n+1}) = S with J = mu_i E^n n - D_i D_x n and the source
  S = n0 r_ion . F^n (= k_i n0 n_e, r_ion the ionization rate moment vector of oracle.bte), E^n
  the field of (n_i^n, F^n) at t_n. The wall rows carry the flux condition at the new level:
  x = 0 (outward normal -1): J(0) = n(0) max(0, -mu_i E(0)); x = L: J(L) = -n(L) max(0, mu_i E(L)).

  Semi-implicit self-consistent electron step (eqs. "bte_semi_implicit"): the x half step of
  oracle.bte, the field E^{1/2} from (n_i, u^T F^{n+1/2}) at t_n + dt/2, the velocity solves with
  that field per point, the second x half step.

  Fully-implicit electron step (eqs. "bte_fully_implicit"): F^{n+1} is the root of
  R(F) = F - F^n + dt [A_x F D_x^T - P_O C P_S F - P_O A_v P_S (E(F) . F)],
  E(F) = Lop (n_i - u^T F) + V(t_{n+1}) E_1, with the zero-inflow rows R = F at x = 0 (mu >= 0) and
  x = L (mu < 0). Per ordinate a, A_x F D_x^T is mu_a D_x F_a G^T with G = M_v^-1 G_v. Found by
  Newton's method with the dense Jacobian (small sizes only) to a relative residual of 1e-14.

Readings (the paper does not fix these): the ion wall condition enforced on the boundary rows at
the new time level with E^n; the ion source uses F^n (lagged) as eq. "fluid_step" prints; mu_i and
D_i from n0 mu_i = 4.65e21 /(V m s) and n0 D_i = 2.07e20 /(m s) of the parameter table; the
fully-implicit field at t_{n+1}.
"""
from __future__ import annotations

import numpy as np

from oracle import bte as O

EPS0 = 8.8541878128e-12      # CODATA 2018
N0_MU_I = 4.65e21            # n0 * ion mobility [1/(V m s)]
N0_D_I = 2.07e20             # n0 * ion diffusion [1/(m s)]


class Hybrid:
    """The self-consistent operators of one discharge on top of oracle.bte.Operators."""

    def __init__(self, ops: O.Operators, n0_mu_i=N0_MU_I, n0_d_i=N0_D_I):
        self.ops = ops
        nx = ops.nx
        self.mu_i = n0_mu_i / ops.n0
        self.d_i = n0_d_i / ops.n0
        # Dirichlet Laplacian: rows 0 and nx-1 are V itself
        A = ops.Dx @ ops.Dx
        A[0, :] = 0.0
        A[-1, :] = 0.0
        A[0, 0] = 1.0
        A[-1, -1] = 1.0
        self.lap = A
        # E = -D_x V, V = A^-1 rhs, rhs = -(e/eps0) rho on interior rows, V(0), V(L) on the walls
        S = -(O.E_CHARGE / EPS0) * np.eye(nx)
        S[0, :] = 0.0
        S[-1, :] = 0.0
        self.Lop = -ops.Dx @ np.linalg.solve(A, S)
        e0 = np.zeros(nx)
        e0[0] = 1.0
        self.E1 = -ops.Dx @ np.linalg.solve(A, e0)
        self.u = ops.mom_n.reshape(-1)
        ion = [j for j, p in enumerate(ops.procs) if p["kind"] == "ionization"]
        self.r_ion = ops.mom_r[ion[0]].reshape(-1) if ion else np.zeros(ops.nv)
        # G = M_v^-1 G_v = U diag(lam) U^-1 (the x-advection speed operator)
        self.Gt = ops.U @ np.diag(ops.lam) @ ops.Uinv

    # ---- electrostatics
    def v_left(self, t, V0=None, freq=None):
        V0 = self.ops.cfg["V0"] if V0 is None else V0
        freq = self.ops.cfg["freq_Hz"] if freq is None else freq
        return V0 * np.sin(2.0 * np.pi * freq * t)

    def ne(self, F):
        return F.reshape(self.ops.nx, -1) @ self.u

    def field(self, ni, F, t, V0=None, freq=None):
        """E at the collocation points for ion density ni, electron state F, time t."""
        return self.Lop @ (ni - self.ne(F)) + self.v_left(t, V0, freq) * self.E1

    # ---- ions
    def ion_step(self, ni, F, t, V0=None, freq=None):
        """n_i^{n+1} from eq. "fluid_step" with the lagged field and source."""
        ops = self.ops
        dt = ops.dt
        E = self.field(ni, F, t, V0, freq)
        D = ops.Dx
        flux = self.mu_i * D * E[None, :] - self.d_i * (D @ D)   # (D_x J)(n) as a matrix
        A = np.eye(ops.nx) / dt + flux
        rhs = ni / dt + ops.n0 * (F.reshape(ops.nx, -1) @ self.r_ion)
        Jrow = self.mu_i * np.diag(E) - self.d_i * D             # J(n) rows
        A[0, :] = Jrow[0, :]
        A[0, 0] -= max(0.0, -self.mu_i * E[0])
        A[-1, :] = Jrow[-1, :]
        A[-1, -1] += max(0.0, self.mu_i * E[-1])
        rhs[0] = 0.0
        rhs[-1] = 0.0
        # the flux rows are ~1e-9 of the interior rows (1/dt) in scale: equilibrate them (same
        # solution) so the wall values are not left to the rounding of a badly scaled system
        for w in (0, -1):
            A[w, :] *= (1.0 / dt) / np.max(np.abs(A[w, :]))
        return np.linalg.solve(A, rhs)

    # ---- electrons, semi-implicit with the electrostatics update
    def sc_step(self, F, ni, t, V0=None, freq=None):
        ops = self.ops
        F1 = ops.x_halfstep(F)
        E = self.field(ni, F1, t + 0.5 * ops.dt, V0, freq)
        F2 = ops.v_step(F1, E)
        return ops.x_halfstep(F2), E

    # ---- electrons, fully implicit
    def _inflow_mask(self):
        ops = self.ops
        m = np.zeros((ops.nx, ops.nt, ops.nr), dtype=bool)
        for a in range(ops.nt):
            m[ops.inflow_row(a), a, :] = True
        return m

    def x_operator(self, F):
        """A_x F D_x^T: per ordinate a, mu_a D_x F_a G^T."""
        ops = self.ops
        out = np.empty_like(F)
        for a in range(ops.nt):
            out[:, a, :] = ops.mu[a] * (ops.Dx @ F[:, a, :] @ self.Gt.T)
        return out

    def v_operator(self, F, E):
        """P_O (C + E_i A_v) P_S F at every point i."""
        ops = self.ops
        Ff = F.reshape(ops.nx, -1)
        out = Ff @ ops.KC.T + E[:, None] * (Ff @ ops.KA.T)
        return out.reshape(F.shape)

    def implicit_residual(self, F, Fn, ni, t1, V0=None, freq=None):
        ops = self.ops
        E = self.field(ni, F, t1, V0, freq)
        R = F - Fn + ops.dt * (self.x_operator(F) - self.v_operator(F, E))
        m = self._inflow_mask()
        R[m] = F[m]
        return R

    def implicit_jacobian(self, F, ni, t1, V0=None, freq=None):
        """Dense dR/dF in the flattened (x, a, k) order (small sizes only)."""
        ops = self.ops
        nx, nv = ops.nx, ops.nv
        D = nx * nv
        E = self.field(ni, F, t1, V0, freq)
        J = np.eye(D)
        # x part: block (i,a,:) <- (j,a,:) = dt mu_a Dx[i,j] G
        Jx = np.zeros((nx, ops.nt, ops.nr, nx, ops.nt, ops.nr))
        for a in range(ops.nt):
            Jx[:, a, :, :, a, :] = ops.mu[a] * np.einsum("ij,km->ikjm", ops.Dx, self.Gt)
        J += ops.dt * Jx.reshape(D, D)
        # v part at frozen E: block diagonal -dt (KC + E_i KA)
        for i in range(nx):
            J[i * nv:(i + 1) * nv, i * nv:(i + 1) * nv] -= ops.dt * (ops.KC + E[i] * ops.KA)
        # field linearisation: dE_i/dF[j, v] = -Lop[i, j] u[v]
        KAF = F.reshape(nx, nv) @ ops.KA.T                  # (KA F_i) per point
        J += ops.dt * np.einsum("iv,ij,w->ivjw", KAF, self.Lop, self.u).reshape(D, D)
        m = self._inflow_mask().reshape(-1)
        J[m, :] = 0.0
        J[m, m] = 1.0
        return J

    def implicit_step(self, Fn, ni, t, V0=None, freq=None, tol=1e-14, max_newton=30):
        """F^{n+1} of eqs. "bte_fully_implicit" by Newton with the dense Jacobian."""
        t1 = t + self.ops.dt
        F = Fn.copy()
        scale = np.linalg.norm(Fn)
        for it in range(max_newton):
            R = self.implicit_residual(F, Fn, ni, t1, V0, freq)
            if np.linalg.norm(R) <= tol * scale:
                return F, it
            J = self.implicit_jacobian(F, ni, t1, V0, freq)
            F = F - np.linalg.solve(J, R.reshape(-1)).reshape(F.shape)
        raise RuntimeError("Newton did not converge")
