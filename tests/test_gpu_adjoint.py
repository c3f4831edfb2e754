"""Adjoint of the step on the GPU (bte_step_adjoint, bte_adjoint_gradient, the autograd wrapper)
against the transposition identity, central finite differences and the oracle's tangent."""
import numpy as np
import pytest

from oracle import tangent as T
from paper_2502_16555_gb300 import workloads as W
from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_step_adjoint_is_the_transpose():
    """<lam, S F> = <S^T lam, F> for random F, lam (ragged LU panels: nv = 7 * 11 = 77)."""
    from paper_2502_16555_gb300 import bte
    cfg = W.scaled(W.ADJOINT, nx=9, nr=11, ntheta=7)
    s = bte.Solver(cfg, "fp64")
    rng = np.random.default_rng(3)
    F = torch.from_numpy(rng.standard_normal((9, 7, 11))).cuda()
    lam = torch.from_numpy(rng.standard_normal((9, 7, 11))).cuda()
    t = 0.37 / W.RF_FREQ_HZ
    SF = F.clone()
    s.step(SF, t)
    StL = lam.clone()
    s.step_adjoint(F, StL, t)
    a = float(torch.sum(lam * SF))
    b = float(torch.sum(StL * F))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b)), (a, b)


def tiny():
    return W.scaled(W.ADJOINT, nx=6, nr=8, ntheta=4, dt_s=W.ADJOINT["dt_s"] * 10)


def test_gradient_against_central_differences_and_oracle_tangent():
    from paper_2502_16555_gb300 import adjoint
    cfg = tiny()
    steps = 24
    m = adjoint.CycleDensity(cfg, steps=steps, checkpoint=5)
    th = m.theta0()
    J, saved = m.forward(th)
    g = m.gradient(saved)
    assert g.shape == (8,)
    assert abs(J - T.objective(T.apply(cfg, th), steps)) <= 1e-10 * abs(J)
    fd = np.zeros(th.size)
    for k in range(th.size):
        h = 1e-6 * max(1.0, abs(th[k]))
        up, dn = th.copy(), th.copy()
        up[k] += h
        dn[k] -= h
        fd[k] = (m.forward(up)[0] - m.forward(dn)[0]) / (2 * h)
    # normwise: a central difference with h = 1e-6 of an FP64 trajectory carries rounding noise of
    # about |J| 1e-14 / h, which the smallest components feel; the tangent below has none
    assert np.abs(g - fd).max() <= 1e-5 * np.abs(g).max(), (m.names(), g, fd)
    ref = T.tangent(cfg, th, steps)
    assert np.allclose(g, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max()), (g, ref)


def test_autograd_function_backward():
    from paper_2502_16555_gb300 import adjoint
    cfg = tiny()
    m = adjoint.CycleDensity(cfg, steps=10, checkpoint=4)
    th = torch.tensor(m.theta0(), dtype=torch.float64, requires_grad=True)
    J = adjoint.cycle_averaged_density(th, m)
    J.backward()
    _, saved = m.forward(m.theta0())
    assert np.allclose(th.grad.numpy(), m.gradient(saved), rtol=1e-12, atol=0.0)


def test_gradient_at_the_adjoint_workload_size():
    """The adjoint workload's grid (Nx=64, Nr=32, Ntheta=16, Nv=512, 1 Torr, 100 V, four
    processes), 100 steps with a checkpoint every 50: the adjoint gradient with respect to V0 and
    the elastic cross-section scale against central differences of the forward run (h = 1e-6
    relative), each component to 1e-5."""
    from paper_2502_16555_gb300 import adjoint
    cfg = W.ADJOINT
    m = adjoint.CycleDensity(cfg, steps=100, checkpoint=50)
    th = m.theta0()
    J, saved = m.forward(th)
    g = m.gradient(saved)
    names = m.names()
    for k in (0, th.size - 1):
        h = 1e-6 * max(1.0, abs(th[k]))
        up, dn = th.copy(), th.copy()
        up[k] += h
        dn[k] -= h
        fd = (m.forward(up)[0] - m.forward(dn)[0]) / (2 * h)
        print("%s: adjoint %.10e  central difference %.10e" % (names[k], g[k], fd))
        assert abs(g[k] - fd) <= 1e-5 * abs(fd), (names[k], g[k], fd)
