"""CPU-only checks of libbte: it loads, exports every symbol of include/bte.h, validates its
arguments, and its independent C++ host assembly matches the oracle's operators."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import bte as O
from paper_2502_16555_gb300 import workloads as W
from tests._lib import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "bte.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bte_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    ensure_built()
    from paper_2502_16555_gb300 import bte
    return bte.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_2502_16555_gb300 import bte
    assert sorted(bte.EXPORTS) == names


def _solver(cfg, **kw):
    from paper_2502_16555_gb300 import bte
    return bte.Solver(cfg, host_only=True, **kw)


@pytest.mark.parametrize("name,cfg", [
    ("small", W.SMALL),
    ("nl_lt_ntheta", W.scaled(W.MEDIUM, nx=16, nr=24, ntheta=8, nl=3)),
    ("odd_ntheta", W.scaled(W.SMALL, nx=7, nr=9, ntheta=5)),
    ("nl_one", W.scaled(W.SMALL, nx=6, nr=10, ntheta=4, nl=1)),
    ("table_and_nu", dict(W.scaled(W.SMALL, nx=5, nr=12, ntheta=4), processes=[
        W.process("elastic", "table", eps_eV=[0.0, 5.0, 30.0], sigma_m2=[1e-19, 2e-19, 5e-20]),
        W.process("excitation", "table", threshold_eV=11.55, eps_eV=[11.55, 20.0, 40.0], sigma_m2=[0.0, 3e-21, 1e-21]),
        W.process("elastic", "nu", sigma0=1e-13)])),
])
def test_host_assembly_matches_oracle(name, cfg):
    s = _solver(cfg)
    ops = O.Operators(cfg)

    def rel(a, b):
        scale = np.max(np.abs(b))   # K_A is zero with one harmonic: then both must be exactly zero
        return np.max(np.abs(a - b)) / scale if scale > 0 else np.max(np.abs(a))

    assert rel(s.operator("x"), ops.x) < 1e-15
    assert rel(s.operator("Dx"), ops.Dx) < 1e-12
    assert rel(s.operator("mu"), ops.mu) < 1e-14
    assert rel(s.operator("M"), ops.M) < 1e-13
    assert rel(s.operator("lambda"), ops.lam) < 1e-12
    assert rel(s.operator("KC"), ops.KC) < 1e-11
    assert rel(s.operator("KA"), ops.KA) < 1e-11
    U, Ui, lam = s.operator("U"), s.operator("Uinv"), s.operator("lambda")
    assert rel(U @ np.diag(lam) @ Ui, np.linalg.solve(ops.M, ops.G)) < 1e-11
    assert rel(s.operator("mom_n"), ops.mom_n.ravel()) < 1e-13
    assert rel(s.operator("mom_e"), ops.mom_e.ravel()) < 1e-13
    assert rel(s.operator("mom_r"), np.array([r.ravel() for r in ops.mom_r])) < 1e-12
    # Q_ij through Algorithm 1 reproduces the oracle's x half step
    Q = s.operator("Q")
    F = W.random_state(ops.nx, ops.nt, ops.nr, seed=1)
    out = np.empty_like(F)
    for a in range(ops.nt):
        Y = F[:, a, :] @ Ui.T
        for i in range(ops.nr):
            Y[:, i] = Q[a, i] @ Y[:, i]
        out[:, a, :] = Y @ U.T
    assert rel(out, ops.x_halfstep(F)) < 1e-12


@pytest.mark.parametrize("cfg", [W.scaled(W.SMALL, nx=5, nr=12, ntheta=6),
                                 W.scaled(W.SMALL, nx=5, nr=9, ntheta=5)])
def test_unscaled_operators_of_the_factored_form(cfg):
    """The dense path factors (I (x) M_v) A_i = I (x) M_v - dt (KCg + E KAg): KCg and KAg must equal
    the oracle's mass-scaled K_C, K_A multiplied by I (x) M_v, and a handle that factors the reduced
    system does not form them."""
    from paper_2502_16555_gb300 import bte
    s = _solver(cfg)
    ops = O.Operators(cfg)
    Mh = np.kron(np.eye(ops.nt), ops.M)
    for name, K in (("KCg", ops.KC), ("KAg", ops.KA)):
        want = Mh @ K
        assert np.max(np.abs(s.operator(name) - want)) <= 1e-11 * np.max(np.abs(want)), name
    red = _solver(dict(cfg, nl=2))
    with pytest.raises(bte.BteError) as e:
        red.operator("KCg")
    assert e.value.status == bte.ESTATE


def test_create_rejects_bad_configs(lib):
    from paper_2502_16555_gb300 import bte
    bad = [dict(nx=2), dict(nr=3), dict(ntheta=1), dict(nl=9, ntheta=8), dict(dt_s=0.0), dict(p_Torr=-1.0),
           dict(nx=4097), dict(nr=881, ntheta=2), dict(nr=128, ntheta=64)]
    for kw in bad:
        cfg = W.scaled(W.SMALL, **{k: v for k, v in kw.items() if k != "nl"})
        if "nl" in kw:
            cfg["nl"] = kw["nl"]
        with pytest.raises(bte.BteError) as e:
            bte.Solver(cfg, host_only=True)
        assert e.value.status == bte.EINVAL, kw


def test_create_accepts_the_largest_grids(lib):
    """The limits themselves are accepted: nr = 880 and nr * ntheta = 7936."""
    from paper_2502_16555_gb300 import bte
    for kw in (dict(nx=3, nr=880, ntheta=2), dict(nx=3, nr=124, ntheta=64)):
        s = bte.Solver(W.scaled(W.SMALL, **kw), host_only=True)
        assert s.info()["nr"] == kw["nr"]


def test_factorisation_order_follows_the_harmonic_count(lib):
    """nl < ntheta factors the reduced matrix of order nl * nr unless BTE_FLAG_FULL_V; nl = ntheta
    factors A_i (order nv); the structured solve holds no factors."""
    from paper_2502_16555_gb300 import bte
    cfg = W.scaled(W.SMALL, nx=5, nr=12, ntheta=8, nl=3)
    assert bte.Solver(cfg, host_only=True).info()["solve_n"] == 36
    assert bte.Solver(cfg, host_only=True, full_v=True).info()["solve_n"] == 96
    assert bte.Solver(cfg, host_only=True, structured=True).info()["solve_n"] == 0
    assert bte.Solver(W.scaled(W.SMALL, nx=5, nr=12, ntheta=8), host_only=True).info()["solve_n"] == 96


def test_bad_process_lists(lib):
    from paper_2502_16555_gb300 import bte
    s = _solver(W.scaled(W.SMALL, nx=5, nr=6, ntheta=4))
    with pytest.raises(bte.BteError):
        s.set_cross_sections([W.process("excitation", "linear", 1e-21, 0.0)])
    with pytest.raises(bte.BteError):
        s.set_cross_sections([W.process("elastic", "table", eps_eV=[1.0, 0.5], sigma_m2=[1.0, 1.0])])


def test_host_only_handle_refuses_device_work(lib):
    from paper_2502_16555_gb300 import bte
    s = _solver(W.scaled(W.SMALL, nx=5, nr=6, ntheta=4))
    st = lib.bte_step(s.h, ctypes.c_void_p(1), None, 0.0, 1.0, 1.0)
    assert st == bte.ESTATE
    st = lib.bte_step(s.h, None, None, 0.0, 1.0, 1.0)
    assert st == bte.EINVAL
    assert lib.bte_destroy(None) == bte.OK


def test_static_fill_bound_and_arguments_without_device_work(lib):
    """bte_init_maxwellian_static stages at most 4096 coefficients in its file-scope array; bte_create
    already refuses nr > 880 (here nr = 4097 on a host-only handle), so no handle can reach that
    bound. Bad arguments are refused before any CUDA call."""
    import ctypes as C
    from paper_2502_16555_gb300 import bte
    with pytest.raises(bte.BteError) as e:
        bte.Solver(W.scaled(W.SMALL, nx=3, nr=4097, ntheta=2), host_only=True)
    assert e.value.status == bte.EINVAL
    s = _solver(W.scaled(W.SMALL, nx=5, nr=6, ntheta=4))
    assert lib.bte_init_maxwellian_static(s.h, None, C.c_void_p(8), 2.0) == bte.EINVAL
    assert lib.bte_init_maxwellian_static(s.h, C.c_void_p(8), None, 2.0) == bte.EINVAL
    assert lib.bte_init_maxwellian_static(s.h, C.c_void_p(8), C.c_void_p(8), -1.0) == bte.EINVAL
    assert lib.bte_init_maxwellian_static(None, C.c_void_p(8), C.c_void_p(8), 2.0) == bte.EINVAL


def test_batch_create_validates_before_any_device_work():
    """bte_batch_create refuses NULL/empty input and handles without device buffers (host-only),
    without touching a GPU."""
    import ctypes as C
    from paper_2502_16555_gb300 import bte
    lib = bte.load()
    out = C.c_void_p()
    assert lib.bte_batch_create(0, None, None, 0, C.byref(out)) == bte.EINVAL
    cfg = W.scaled(W.SMALL, nx=5, nr=6, ntheta=4)
    s1 = bte.Solver(cfg, host_only=True)
    s2 = bte.Solver(cfg, host_only=True)
    hs = (C.c_void_p * 2)(s1.h, s2.h)
    assert lib.bte_batch_create(2, hs, None, 0, C.byref(out)) == bte.ESTATE
    assert b"device buffers" in lib.bte_batch_last_error(None)
    same = (C.c_void_p * 2)(s1.h, s1.h)
    assert lib.bte_batch_create(2, same, None, 0, C.byref(out)) in (bte.EINVAL, bte.ESTATE)
    assert not out.value
    assert lib.bte_batch_destroy(None) == bte.OK


def test_structured_flag_validates_nr_without_device_work():
    import ctypes as C
    from paper_2502_16555_gb300 import bte
    lib = bte.load()
    c = bte.Config()
    cfg = W.scaled(W.SMALL, nx=5, nr=80, ntheta=4)
    c.nx, c.nr, c.ntheta, c.nl = cfg["nx"], cfg["nr"], cfg["ntheta"], 0
    c.L_m, c.vmax_eV, c.p_Torr = cfg["L_m"], cfg["vmax_eV"], cfg["p_Torr"]
    c.T0_K, c.m0_amu, c.dt_s = cfg["T0_K"], cfg["m0_amu"], cfg["dt_s"]
    c.precision, c.refine_tol, c.refine_max, c.stream = bte.FP64, 0.0, -1, None
    c.flags = bte.FLAG_STRUCTURED
    h = C.c_void_p()
    assert lib.bte_create(C.byref(c), C.byref(h)) == bte.EINVAL
    assert b"nr <= 64" in lib.bte_last_error(None)


def test_self_consistent_entry_points_validate_without_device_work(lib):
    """The field, ion and implicit entry points reject NULL arguments and bad ion coefficients,
    and refuse a host-only handle (no device buffers), before any device work."""
    import ctypes as C
    from paper_2502_16555_gb300 import bte
    s = _solver(W.scaled(W.SMALL, nx=5, nr=6, ntheta=4))
    p = C.c_void_p(1)
    assert lib.bte_set_ion_transport(s.h, -1.0, 1.0) == bte.EINVAL
    assert lib.bte_set_ion_transport(s.h, 1.0, 0.0) == bte.EINVAL
    assert lib.bte_set_ion_transport(s.h, 4.65e21, 2.07e20) == bte.OK
    assert lib.bte_field(s.h, None, None, 0.0, 1.0, 1.0, p) == bte.EINVAL
    assert lib.bte_field(s.h, p, None, 0.0, 1.0, 1.0, p) == bte.ESTATE
    assert lib.bte_ion_step(s.h, None, p, 0.0, 1.0, 1.0) == bte.EINVAL
    assert lib.bte_ion_step(s.h, p, p, 0.0, 1.0, 1.0) == bte.ESTATE
    assert lib.bte_step_sc(s.h, p, None, 0.0, 1.0, 1.0, None) == bte.EINVAL
    assert lib.bte_step_sc(s.h, p, p, 0.0, 1.0, 1.0, None) == bte.ESTATE
    o = bte.ImplicitOpts()
    assert lib.bte_step_implicit(s.h, p, None, 0.0, 1.0, 1.0, C.byref(o)) == bte.EINVAL
    assert lib.bte_step_implicit(s.h, p, p, 0.0, 1.0, 1.0, C.byref(o)) == bte.ESTATE
    assert lib.bte_step_implicit(None, p, p, 0.0, 1.0, 1.0, None) == bte.EINVAL
