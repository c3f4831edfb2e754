"""Pins of the oracle's parameter tangent (oracle/tangent.py) and of the Clenshaw-Curtis weights,
on the CPU."""
import numpy as np
import pytest

from oracle import bte as O
from oracle import tangent as T
from paper_2502_16555_gb300 import workloads as W
from tests._lib import ensure_built


@pytest.mark.parametrize("nx", [5, 8, 17])
def test_clenshaw_curtis_exact_on_polynomials(nx):
    L = 0.0254
    x = O.cheb_points(nx, L)
    w = T.clenshaw_curtis(nx, L)
    for k in range(nx):
        exact = L ** (k + 1) / (k + 1)
        assert abs(w @ x**k - exact) <= 1e-13 * exact * (k + 1)
    assert np.all(w > 0)


def test_library_clenshaw_curtis_weights_match_definition():
    ensure_built()
    from paper_2502_16555_gb300 import bte
    for nx in (6, 9, 32):
        cfg = W.scaled(W.SMALL, nx=nx, nr=6, ntheta=4)
        s = bte.Solver(cfg, host_only=True)
        w = s.operator("ccw")
        x = s.operator("x")
        for k in range(nx):
            exact = cfg["L_m"] ** (k + 1) / (k + 1)
            assert abs(w @ x**k - exact) <= 1e-12 * exact * (k + 1)


def tiny():
    return W.scaled(W.ADJOINT, nx=5, nr=6, ntheta=4, dt_s=W.ADJOINT["dt_s"] * 20)


def test_tangent_matches_central_differences_of_the_oracle():
    """Every component of the forward-mode tangent against (J(th + h) - J(th - h)) / 2h of the
    oracle's own objective (h relative 1e-4, thresholds 1e-4 eV). |J| is about 1e13 and some
    components are 100 times below the largest, so h = 1e-6 left the central difference at the
    roundoff floor (1e-5 off); with 1e-4 every component agrees to 1e-7."""
    cfg = tiny()
    steps = 6
    th = T.theta0(cfg)
    g = T.tangent(cfg, th, steps)
    for k in range(th.size):
        h = 1e-4 if (len(cfg["processes"]) <= k < th.size - 1) else 1e-4 * max(1.0, abs(th[k]))
        up, dn = th.copy(), th.copy()
        up[k] += h
        dn[k] -= h
        fd = (T.objective(T.apply(cfg, up), steps) - T.objective(T.apply(cfg, dn), steps)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g).max()), (k, g[k], fd)
