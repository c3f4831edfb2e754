"""Pins of the self-consistent oracle (oracle/hybrid.py) against closed forms, an analytic decay
rate, the specified-field step it must reduce to, and the time order of the two electron schemes."""
import numpy as np
import pytest

from oracle import bte as O
from oracle import hybrid as H
from paper_2502_16555_gb300 import workloads as W


def tiny(nx=9, nr=8, nt=6, **kw):
    cfg = W.scaled(W.SMALL, nx=nx, nr=nr, ntheta=nt)
    cfg.update(kw)
    return cfg


def profile(ops, peak, shift=0.0):
    xi = 2.0 * ops.x / ops.L - 1.0
    return peak * (1.0 - xi * xi) + shift


def test_field_without_charge_is_uniform():
    """Gauss's law with no charge: V linear between the electrodes, E = V(0)/L everywhere."""
    ops = O.Operators(tiny(nx=17))
    h = H.Hybrid(ops)
    E = h.Lop @ np.zeros(ops.nx) + 37.0 * h.E1
    np.testing.assert_allclose(E, np.full(ops.nx, 37.0 / ops.L), rtol=1e-12)


@pytest.mark.parametrize("order", [0, 1])
def test_field_of_polynomial_charge_matches_closed_form(order):
    """rho = c (order 0) or c x (order 1) between V(0) = Vl and V(L) = 0:
    E = Vl/L - (e c / 2 eps0)(L - 2x), or E = -B + (e c / 2 eps0) x^2 with
    B = e c L^2 / (6 eps0) - Vl/L (the quadratic / cubic V is exact on the collocation grid)."""
    ops = O.Operators(tiny(nx=17))
    h = H.Hybrid(ops)
    x, L, Vl, k = ops.x, ops.L, 25.0, O.E_CHARGE / H.EPS0
    if order == 0:
        c = 3e14
        rho = np.full(ops.nx, c)
        exact = Vl / L - 0.5 * k * c * (L - 2.0 * x)
    else:
        c = 2e16
        rho = c * x
        B = k * c * L * L / 6.0 - Vl / L
        exact = -B + 0.5 * k * c * x * x
    E = h.Lop @ rho + Vl * h.E1
    assert np.max(np.abs(E - exact)) <= 1e-10 * np.max(np.abs(exact))


def test_ion_diffusion_mode_decays_at_the_backward_euler_rate():
    """No mobility, no electrons: n = 1 + a cos(pi x/L) keeps zero wall flux, and one implicit
    step multiplies the mode by 1/(1 + dt D pi^2/L^2) (spectral accuracy in x)."""
    # a step long enough that diffusion matters (dt D pi^2/L^2 = 0.5; ions are slow)
    cfg = tiny(nx=24)
    n0_d = H.N0_D_I / O.neutral_density(cfg["p_Torr"], cfg["T0_K"])
    cfg["dt_s"] = 0.5 * cfg["L_m"] ** 2 / (n0_d * np.pi ** 2)
    ops = O.Operators(cfg)
    h = H.Hybrid(ops, n0_mu_i=0.0)
    a = 0.3e15
    ni = 1e15 + a * np.cos(np.pi * ops.x / ops.L)
    F = np.zeros((ops.nx, ops.nt, ops.nr))
    out = h.ion_step(ni, F, 0.0)
    g = 1.0 / (1.0 + ops.dt * h.d_i * np.pi ** 2 / ops.L ** 2)
    exact = 1e15 + a * g * np.cos(np.pi * ops.x / ops.L)
    assert abs(g - 1.0 / 1.5) < 1e-12
    assert np.max(np.abs(out - exact)) <= 1e-8 * 1e15


def test_ion_step_wall_rows_hold_outflow_flux():
    """At the new level the wall rows satisfy J(0) = n max(0, -mu E) and J(L) = -n max(0, mu E)."""
    ops = O.Operators(tiny(nx=13))
    h = H.Hybrid(ops)
    ni = profile(ops, 1e15, 1e13)
    F = ops.initial_state()
    out = h.ion_step(ni, F, 0.13 / ops.cfg["freq_Hz"])
    E = h.field(ni, F, 0.13 / ops.cfg["freq_Hz"])
    J = h.mu_i * E * out - h.d_i * (ops.Dx @ out)
    # the wall rows are small next to the interior rows (1/dt), so a backward-stable solve leaves
    # them a residual of ~1e-8 of their own terms; a wrong condition would be off by O(1)
    for w, target in ((0, out[0] * max(0.0, -h.mu_i * E[0])), (-1, -out[-1] * max(0.0, h.mu_i * E[-1]))):
        terms = abs(h.mu_i * E[w] * out[w]) + h.d_i * (np.abs(ops.Dx[w]) @ np.abs(out))
        assert abs(J[w] - target) <= 1e-6 * terms, (w, J[w], target, terms)


def test_semi_implicit_step_without_space_charge_is_the_specified_field_step():
    """With the charge term removed the field is V(t)/L: the step of oracle.bte."""
    ops = O.Operators(tiny())
    h = H.Hybrid(ops)
    h.Lop = np.zeros_like(h.Lop)
    F = W.random_state(ops.nx, ops.nt, ops.nr, seed=5)
    t = 0.17 / ops.cfg["freq_Hz"]
    out, _ = h.sc_step(F, profile(ops, 1e15), t)
    ref = ops.step(F, t)
    assert np.linalg.norm(out - ref) <= 1e-13 * np.linalg.norm(ref)


def test_implicit_jacobian_matches_central_differences():
    """The dense Jacobian (including the field linearisation) against differences of R."""
    ops = O.Operators(tiny(nx=7, nr=6, nt=4))
    h = H.Hybrid(ops)
    F = ops.initial_state() * (1.0 + 0.1 * W.random_state(ops.nx, ops.nt, ops.nr, seed=2) / 1e15)
    Fn = ops.initial_state()
    ni = profile(ops, 1.2e15)
    t1 = 0.3 / ops.cfg["freq_Hz"]
    J = h.implicit_jacobian(F, ni, t1)
    X = W.random_state(ops.nx, ops.nt, ops.nr, seed=9)
    eps = 1e-6 * np.linalg.norm(F) / np.linalg.norm(X)
    fd = (h.implicit_residual(F + eps * X, Fn, ni, t1) - h.implicit_residual(F - eps * X, Fn, ni, t1)) / (2 * eps)
    jx = (J @ X.reshape(-1)).reshape(F.shape)
    assert np.linalg.norm(jx - fd) <= 1e-7 * np.linalg.norm(fd)


def test_implicit_step_converges_and_agrees_with_semi_implicit_to_second_order():
    """Both schemes are first order in dt, so after one step from the same state they differ by
    O(dt^2): halving dt divides the difference by about 4. Newton converges in a few steps."""
    diffs = []
    for frac in (2e-4, 1e-4):
        cfg = tiny(nx=9, nr=8, nt=6, dt_s=frac / W.RF_FREQ_HZ)
        ops = O.Operators(cfg)
        h = H.Hybrid(ops)
        F = ops.initial_state()
        ni = profile(ops, 1.1e15)
        t = 0.21 / cfg["freq_Hz"]
        Fi, it = h.implicit_step(F, ni, t)
        assert it <= 6
        R = h.implicit_residual(Fi, F, ni, t + ops.dt)
        assert np.linalg.norm(R) <= 1e-13 * np.linalg.norm(F)
        Fs, _ = h.sc_step(F, ni, t)
        diffs.append(np.linalg.norm(Fi - Fs) / np.linalg.norm(F))
    ratio = diffs[0] / diffs[1]
    assert 3.0 < ratio < 5.0, (diffs, ratio)


def _backward_euler_pulse(x, x0, s, v, D, dt):
    """One backward-Euler step of n_t + v n_x = D n_xx on the whole line for n = exp(-(x-x0)^2/2s^2),
    evaluated by its Fourier integral: n1_hat(k) = n0_hat(k) / (1 + dt (i k v + D k^2))."""
    k = np.linspace(-12.0 / s, 12.0 / s, 200001)
    dk = k[1] - k[0]
    g = s * np.sqrt(2.0 * np.pi) * np.exp(-0.5 * (s * k) ** 2) / (1.0 + dt * (1j * k * v + D * k * k))
    return np.array([np.real(np.sum(g * np.exp(1j * k * (xe - x0)))) * dk / (2.0 * np.pi) for xe in x])


def test_ion_drift_diffusion_of_a_pulse_matches_the_whole_line_solution():
    """Uniform field (space charge removed), no electrons: a Gaussian pulse far from both walls
    drifts at mu_i E and spreads with D_i. The collocation step must equal the exact
    backward-Euler step of the whole-line problem (Fourier integral, independent of D_x). The
    step moves the pulse by 2 % of the gap; a drift of the wrong sign or size is off by O(0.1)."""
    cfg = tiny(nx=64, nr=8, nt=4)
    ops = O.Operators(cfg)
    h = H.Hybrid(ops)
    h.Lop = np.zeros_like(h.Lop)
    V0 = 100.0
    vd = h.mu_i * V0 / ops.L                          # E = V0/L at t = T/4
    ops.dt = 0.02 * ops.L / vd
    s, x0 = ops.L / 15.0, 0.42 * ops.L
    n_old = np.exp(-0.5 * ((ops.x - x0) / s) ** 2)
    out = h.ion_step(n_old, np.zeros((ops.nx, ops.nt, ops.nr)), 0.25 / cfg["freq_Hz"], V0=V0)
    exact = _backward_euler_pulse(ops.x, x0, s, vd, h.d_i, ops.dt)
    assert np.max(np.abs(out - exact)) < 1e-8
    assert np.max(np.abs(_backward_euler_pulse(ops.x, x0, s, -vd, h.d_i, ops.dt) - exact)) > 0.1


def test_ion_source_is_the_ionization_rate_of_the_electrons():
    """No ion mobility, uniform ions and a uniform 3 eV Maxwellian electron state: the flux
    vanishes (walls included), so one step adds dt n0 k_ion n_e everywhere. k_ion is the
    Maxwellian average of v sigma_ion (sigma = 3e-21 ln(eps/15.76)/(eps/15.76) above threshold)
    by adaptive quadrature, truncated at vmax; agreement to the B-spline projection error. vmax =
    60 eV keeps the ionization tail far from vmax, where the radial functions must vanish."""
    from scipy import integrate
    cfg = tiny(nx=9, nr=48, nt=4)
    cfg["vmax_eV"] = 60.0
    ops = O.Operators(cfg)
    h = H.Hybrid(ops, n0_mu_i=0.0)
    Te, ne = 3.0, 2.0e15
    F = ne * np.broadcast_to(ops.maxwellian_coeffs(Te), (ops.nx, ops.nt, ops.nr)).copy()
    ni = np.full(ops.nx, 1.0e15)
    out = h.ion_step(ni, F, 0.1 / cfg["freq_Hz"])
    vth = np.sqrt(2.0 * O.E_CHARGE * Te / O.M_E)
    vmax, th = ops.vmax, np.sqrt(2.0 * O.E_CHARGE * 15.76 / O.M_E)

    def sigma(v):
        r = 0.5 * O.M_E * v * v / O.E_CHARGE / 15.76
        return 3e-21 * np.log(r) / r

    fM = lambda v: np.exp(-(v / vth) ** 2) * 4.0 * np.pi * v * v / (np.pi ** 1.5 * vth ** 3)
    num = integrate.quad(lambda v: sigma(v) * v * fM(v), th, vmax, epsabs=0, epsrel=1e-12, limit=200)[0]
    den = integrate.quad(fM, 0.0, vmax, epsabs=0, epsrel=1e-12, limit=200)[0]
    n_e_truncated = ne * den                      # the projected state holds the truncated density
    expect = ni + ops.dt * ops.n0 * (num / den) * n_e_truncated
    assert np.max(np.abs(out - expect)) < 1e-4 * np.max(expect - ni)
    assert np.all(out > ni)


def _clenshaw_curtis(nx, L):
    """Clenshaw-Curtis weights on the Chebyshev-Gauss-Lobatto points of [0, L] (exact for every
    polynomial of degree < nx): w_k = (c_k/N)(1 - sum_j b_j cos(2 j theta_k)/(4 j^2 - 1)),
    theta_k = pi k/N, N = nx - 1, c_k = 1 at the ends and 2 inside, b_j = 1 at j = N/2 else 2."""
    N = nx - 1
    th = np.pi * np.arange(nx) / N
    w = np.ones(nx)
    for j in range(1, N // 2 + 1):
        b = 1.0 if 2 * j == N else 2.0
        w -= b * np.cos(2 * j * th) / (4 * j * j - 1)
    c = np.full(nx, 2.0)
    c[0] = c[-1] = 1.0
    return 0.5 * L * c * w / N


def test_ion_step_conserves_ions_in_a_space_charge_field():
    """The ions are their own space charge (no electrons, no source), so E varies across the pulse.
    With the flux in conservation form, D_x(mu_i E n), the step changes the number of ions only
    through the walls, where the pulse is negligible: sum_i c_i n_i is kept (Clenshaw-Curtis
    weights, exact for the collocation polynomial). Written as mu_i E D_x n instead, it would
    change by dt mu_i int E' n, about 1e-3 of the total here."""
    cfg = tiny(nx=64, nr=8, nt=4)
    ops = O.Operators(cfg)
    h = H.Hybrid(ops)
    ops.dt = 1e-9
    n_old = 1e15 * np.exp(-0.5 * ((ops.x - 0.5 * ops.L) / (ops.L / 14.0)) ** 2)
    F = np.zeros((ops.nx, ops.nt, ops.nr))
    out = h.ion_step(n_old, F, 0.0)
    c = _clenshaw_curtis(ops.nx, ops.L)
    E = h.field(n_old, F, 0.0)
    drift_change = ops.dt * h.mu_i * abs(c @ ((ops.Dx @ E) * n_old))
    assert drift_change > 1e-4 * (c @ n_old)
    assert abs(c @ out - c @ n_old) < 1e-9 * (c @ n_old)
