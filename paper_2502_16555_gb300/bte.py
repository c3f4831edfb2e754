"""Thin ctypes binding of libbte (include/bte.h): argument marshalling only.

Every step of the method runs in the library's own CUDA kernels; PyTorch provides device memory
and the stream. There is no fallback: if libbte.so has not been built, loading raises.

    from paper_2502_16555_gb300 import bte, workloads
    s = bte.Solver(workloads.SMALL, precision="fp64")
    F = s.initial_state()                # torch.float64 on cuda, shape (nx, ntheta, nr)
    s.step(F, t=0.0)
    ne, mean_eV, rates = s.moments(F)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbte.so")

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ENOCONV, ENONFINITE, ESTATE = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESINGULAR", 5: "ENOCONV",
                6: "ENONFINITE", 7: "ESTATE"}
FP64, MIXED = 0, 1
FLAG_HOST_ONLY = 1
FLAG_SIMT_GEMM = 2
FLAG_STRUCTURED = 4
FLAG_TC_SINGLE = 8
FLAG_FULL_V = 16
FLAG_DIAG_TC_TIMEOUT = 32
FLAG_TC_ONE_CTA = 64
FLAG_PANEL_TC = 128
KINDS = {"elastic": 0, "excitation": 1, "ionization": 2}
FORMS = {"const": 0, "linear": 1, "log": 2, "table": 3, "nu": 4}
OPERATORS = {"x": 0, "Dx": 1, "mu": 2, "KC": 3, "KA": 4, "lambda": 5, "U": 6, "Uinv": 7, "Q": 8,
             "M": 9, "mom_n": 10, "mom_e": 11, "mom_r": 12, "ccw": 13, "KCg": 14, "KAg": 15}
EXPORTS = ("bte_create", "bte_set_cross_sections", "bte_init_maxwellian", "bte_step", "bte_run",
           "bte_step_host", "bte_moments", "bte_get_operator", "bte_get_info", "bte_profile",
           "bte_destroy", "bte_last_error", "bte_init_maxwellian_static", "bte_batch_create",
           "bte_batch_run", "bte_batch_get_info", "bte_batch_destroy", "bte_batch_last_error",
           "bte_step_adjoint", "bte_adjoint_gradient", "bte_set_ion_transport", "bte_field",
           "bte_ion_step", "bte_step_sc", "bte_step_implicit")
BATCH_AUTOTUNE = 1
KERNELS = ("x_to_eigen", "x_apply_q", "x_from_eigen", "v_form", "lu_panel", "lu_swap_trsm", "lu_gemm",
           "lu_solve", "residual", "other")


class Config(C.Structure):
    _fields_ = [("nx", C.c_int), ("nr", C.c_int), ("ntheta", C.c_int), ("nl", C.c_int),
                ("L_m", C.c_double), ("vmax_eV", C.c_double), ("p_Torr", C.c_double),
                ("T0_K", C.c_double), ("m0_amu", C.c_double), ("dt_s", C.c_double),
                ("precision", C.c_int), ("refine_tol", C.c_double), ("refine_max", C.c_int),
                ("stream", C.c_void_p), ("flags", C.c_uint)]


class Process(C.Structure):
    _fields_ = [("kind", C.c_int), ("form", C.c_int), ("threshold_eV", C.c_double),
                ("scale", C.c_double), ("sigma0", C.c_double), ("n_tab", C.c_int),
                ("eps_eV", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double))]


class ImplicitOpts(C.Structure):
    _fields_ = [("newton_rtol", C.c_double), ("newton_max", C.c_int), ("gmres_restart", C.c_int),
                ("gmres_rtol", C.c_double), ("gmres_max", C.c_int), ("precond", C.c_int),
                ("newton_iters", C.c_int), ("gmres_iters", C.c_int), ("residual", C.c_double)]


class Info(C.Structure):
    _fields_ = [("nx", C.c_int), ("nr", C.c_int), ("ntheta", C.c_int), ("nl", C.c_int),
                ("nv", C.c_int), ("n_proc", C.c_int), ("precision", C.c_int), ("n0_m3", C.c_double),
                ("vmax_ms", C.c_double), ("device_bytes", C.c_size_t),
                ("last_refine_sweeps", C.c_int), ("last_residual", C.c_double),
                ("last_flags", C.c_uint), ("launches", C.c_ulonglong), ("tensor_cores", C.c_int),
                ("solve_n", C.c_int), ("last_refine_evals", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Open libbte.so (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libbte.so not found at {path}: build it with "
                           "`python -m paper_2502_16555_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(path)
    vp, i, d, u = C.c_void_p, C.c_int, C.c_double, C.c_uint
    pd = C.POINTER(C.c_double)
    lib.bte_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
    lib.bte_set_cross_sections.argtypes = [vp, i, C.POINTER(Process)]
    lib.bte_init_maxwellian.argtypes = [vp, vp, vp, d]
    lib.bte_step.argtypes = [vp, vp, vp, d, d, d]
    lib.bte_run.argtypes = [vp, vp, i, d, d, d]
    lib.bte_step_host.argtypes = [vp, pd, d, d, d]
    lib.bte_moments.argtypes = [vp, vp, vp, vp, vp]
    lib.bte_get_operator.argtypes = [vp, i, pd, C.c_size_t]
    lib.bte_get_info.argtypes = [vp, C.POINTER(Info)]
    lib.bte_profile.argtypes = [vp, i, pd, C.POINTER(C.c_ulonglong)]
    lib.bte_init_maxwellian_static.argtypes = [vp, vp, vp, d]
    lib.bte_destroy.argtypes = [vp]
    lib.bte_last_error.argtypes = [vp]
    lib.bte_last_error.restype = C.c_char_p
    lib.bte_batch_create.argtypes = [i, C.POINTER(vp), vp, u, C.POINTER(vp)]
    lib.bte_batch_run.argtypes = [vp, C.POINTER(vp), i, pd, pd, pd, C.POINTER(C.c_int)]
    lib.bte_batch_get_info.argtypes = [vp, i, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.POINTER(C.c_ulonglong)]
    lib.bte_batch_destroy.argtypes = [vp]
    lib.bte_step_adjoint.argtypes = [vp, vp, vp, d, d, d, vp, d, vp, vp]
    lib.bte_adjoint_gradient.argtypes = [vp, vp, vp, d, pd]
    lib.bte_set_ion_transport.argtypes = [vp, d, d]
    lib.bte_field.argtypes = [vp, vp, vp, d, d, d, vp]
    lib.bte_ion_step.argtypes = [vp, vp, vp, d, d, d]
    lib.bte_step_sc.argtypes = [vp, vp, vp, d, d, d, vp]
    lib.bte_step_implicit.argtypes = [vp, vp, vp, d, d, d, C.POINTER(ImplicitOpts)]
    lib.bte_batch_last_error.argtypes = [vp]
    lib.bte_batch_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("bte_last_error", "bte_batch_last_error"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


class BteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _processes(procs):
    keep = []
    arr = (Process * max(1, len(procs)))()
    for j, p in enumerate(procs):
        q = arr[j]
        q.kind = KINDS[p["kind"]]
        q.form = FORMS[p["form"]]
        q.threshold_eV = p.get("threshold_eV", 0.0)
        q.scale = p.get("scale", 1.0)
        q.sigma0 = p.get("sigma0", 0.0)
        if p["form"] == "table":
            e = np.ascontiguousarray(p["eps_eV"], dtype=np.float64)
            s = np.ascontiguousarray(p["sigma_m2"], dtype=np.float64)
            keep += [e, s]
            q.n_tab = e.size
            q.eps_eV = e.ctypes.data_as(C.POINTER(C.c_double))
            q.sigma_m2 = s.ctypes.data_as(C.POINTER(C.c_double))
    return arr, keep


class Solver:
    """One discharge on one GPU: owns a libbte handle; F tensors belong to the caller."""

    def __init__(self, cfg: dict, precision: str = "fp64", refine_tol: float = 0.0,
                 refine_max: int = -1, stream=None, host_only: bool = False, device=None,
                 simt_gemm: bool = False, structured: bool = False, tc_single: bool = False,
                 full_v: bool = False, diag_tc_timeout: bool = False, tc_one_cta: bool = False,
                 panel_tc: bool = False):
        self.lib = load()
        self.cfg = dict(cfg)
        self.host_only = host_only
        self.torch = None
        if not host_only:
            import torch
            self.torch = torch
            self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
            if stream is None:
                stream = torch.cuda.current_stream(self.device)
            self.stream = stream
        c = Config()
        c.nx, c.nr, c.ntheta = cfg["nx"], cfg["nr"], cfg["ntheta"]
        c.nl = cfg.get("nl") or cfg["ntheta"]
        c.L_m, c.vmax_eV, c.p_Torr = cfg["L_m"], cfg["vmax_eV"], cfg["p_Torr"]
        c.T0_K, c.m0_amu, c.dt_s = cfg["T0_K"], cfg["m0_amu"], cfg["dt_s"]
        c.precision = {"fp64": FP64, "mixed": MIXED}[precision]
        c.refine_tol, c.refine_max = refine_tol, refine_max
        c.stream = None if host_only else C.c_void_p(stream.cuda_stream)
        c.flags = ((FLAG_HOST_ONLY if host_only else 0) | (FLAG_SIMT_GEMM if simt_gemm else 0) |
                   (FLAG_STRUCTURED if structured else 0) | (FLAG_TC_SINGLE if tc_single else 0) |
                   (FLAG_FULL_V if full_v else 0) | (FLAG_DIAG_TC_TIMEOUT if diag_tc_timeout else 0) |
                   (FLAG_TC_ONE_CTA if tc_one_cta else 0) | (FLAG_PANEL_TC if panel_tc else 0))
        h = C.c_void_p()
        st = self.lib.bte_create(C.byref(c), C.byref(h))
        if st != OK:
            raise BteError(st, self.lib.bte_last_error(None).decode())
        self.h = h
        self.nx, self.nr, self.nt = c.nx, c.nr, c.ntheta
        self.nv = self.nr * self.nt
        self.precision = precision
        self.set_cross_sections(cfg["processes"])

    # ---- life cycle
    def close(self):
        if getattr(self, "h", None):
            self.lib.bte_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise BteError(st, self.lib.bte_last_error(self.h).decode())

    # ---- entry points
    def set_cross_sections(self, procs):
        arr, keep = _processes(procs)
        self._check(self.lib.bte_set_cross_sections(self.h, len(procs), arr))
        self.n_proc = len(procs)
        del keep

    def empty_state(self):
        return self.torch.zeros((self.nx, self.nt, self.nr), dtype=self.torch.float64, device=self.device)

    def init_maxwellian(self, F, ne, Te_eV):
        self._check(self.lib.bte_init_maxwellian(self.h, _ptr(F), _ptr(ne), float(Te_eV)))
        return F

    def initial_state(self):
        """F(0) = n_e(x) f_M(v; Te), n_e = ne_peak (1 - xi^2), xi = 2x/L - 1 (workload IC)."""
        ic = self.cfg.get("ic", {"Te_eV": 2.0, "ne_peak": 1e15})
        x = self.operator("x")
        xi = 2.0 * x / self.cfg["L_m"] - 1.0
        ne = self.torch.tensor(ic["ne_peak"] * (1.0 - xi * xi), dtype=self.torch.float64, device=self.device)
        F = self.empty_state()
        return self.init_maxwellian(F, ne, ic["Te_eV"])

    def _f(self, F):
        t = self.torch
        if not (F.is_cuda and F.dtype == t.float64 and F.is_contiguous() and F.numel() == self.nx * self.nv):
            raise ValueError("F must be a contiguous float64 CUDA tensor of shape (nx, ntheta, nr)")
        return F

    def step(self, F, t: float, E=None, V0=None, freq=None):
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        if E is not None and not (E.is_cuda and E.dtype == self.torch.float64 and E.numel() == self.nx):
            raise ValueError("E must be a float64 CUDA tensor with nx entries")
        self._check(self.lib.bte_step(self.h, _ptr(self._f(F)), _ptr(E), float(t), float(V0), float(freq)))
        return F

    # ---- self-consistent field, ions, fully-implicit electrons
    def _nx_vec(self, v, name):
        if v is not None and not (v.is_cuda and v.dtype == self.torch.float64 and v.numel() == self.nx
                                  and v.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor with nx entries")
        return v

    def set_ion_transport(self, n0_mu_i: float, n0_D_i: float):
        self._check(self.lib.bte_set_ion_transport(self.h, float(n0_mu_i), float(n0_D_i)))

    def field(self, F, ni, t: float, V0=None, freq=None):
        """E = L (n_i - u^T F) + V(0, t) E_1 at the collocation points (a new CUDA tensor)."""
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        E = self.torch.empty(self.nx, dtype=self.torch.float64, device=self.device)
        self._check(self.lib.bte_field(self.h, _ptr(self._f(F)), _ptr(self._nx_vec(ni, "ni")), float(t),
                                       float(V0), float(freq), _ptr(E)))
        return E

    def ion_step(self, ni, F, t: float, V0=None, freq=None):
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        self._check(self.lib.bte_ion_step(self.h, _ptr(self._nx_vec(ni, "ni")), _ptr(self._f(F)), float(t),
                                          float(V0), float(freq)))
        return ni

    def step_sc(self, F, ni, t: float, V0=None, freq=None, E_out=None):
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        self._check(self.lib.bte_step_sc(self.h, _ptr(self._f(F)), _ptr(self._nx_vec(ni, "ni")), float(t),
                                         float(V0), float(freq), _ptr(self._nx_vec(E_out, "E_out"))))
        return F

    def step_implicit(self, F, ni, t: float, V0=None, freq=None, newton_rtol=0.0, newton_max=0,
                      gmres_restart=0, gmres_rtol=0.0, gmres_max=0, precond=0):
        """One fully-implicit step; returns (newton_iters, gmres_iters, relative residual)."""
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        o = ImplicitOpts(newton_rtol=newton_rtol, newton_max=newton_max, gmres_restart=gmres_restart,
                         gmres_rtol=gmres_rtol, gmres_max=gmres_max, precond=precond)
        self._check(self.lib.bte_step_implicit(self.h, _ptr(self._f(F)), _ptr(self._nx_vec(ni, "ni")), float(t),
                                               float(V0), float(freq), C.byref(o)))
        return o.newton_iters, o.gmres_iters, o.residual

    def run(self, F, n_steps: int, t: float, V0=None, freq=None):
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        self._check(self.lib.bte_run(self.h, _ptr(self._f(F)), int(n_steps), float(t), float(V0), float(freq)))
        return F

    def step_host(self, F_host: np.ndarray, t: float, V0=None, freq=None):
        """bte_step on a host array (copied in and out by the library)."""
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        if not (isinstance(F_host, np.ndarray) and F_host.dtype == np.float64 and F_host.flags.c_contiguous
                and F_host.size == self.nx * self.nv):
            raise ValueError("F_host must be a C-contiguous float64 array with nx*ntheta*nr entries")
        self._check(self.lib.bte_step_host(self.h, F_host.ctypes.data_as(C.POINTER(C.c_double)), float(t),
                                           float(V0), float(freq)))
        return F_host

    def moments(self, F):
        t = self.torch
        ne = t.empty(self.nx, dtype=t.float64, device=self.device)
        mean = t.empty_like(ne)
        rates = t.empty((max(self.n_proc, 1), self.nx), dtype=t.float64, device=self.device)
        self._check(self.lib.bte_moments(self.h, _ptr(self._f(F)), _ptr(ne), _ptr(mean), _ptr(rates)))
        return ne, mean, rates[: self.n_proc]

    def operator(self, name: str) -> np.ndarray:
        sizes = {"x": (self.nx,), "Dx": (self.nx, self.nx), "mu": (self.nt,), "KC": (self.nv, self.nv),
                 "KA": (self.nv, self.nv), "lambda": (self.nr,), "U": (self.nr, self.nr),
                 "Uinv": (self.nr, self.nr), "Q": (self.nt, self.nr, self.nx, self.nx), "M": (self.nr, self.nr),
                 "mom_n": (self.nv,), "mom_e": (self.nv,), "mom_r": (self.n_proc, self.nv), "ccw": (self.nx,),
                 "KCg": (self.nv, self.nv), "KAg": (self.nv, self.nv)}
        out = np.empty(sizes[name], dtype=np.float64)
        self._check(self.lib.bte_get_operator(self.h, OPERATORS[name], out.ctypes.data_as(C.POINTER(C.c_double)),
                                              out.size))
        return out

    def step_adjoint(self, F, lam, t: float, g=None, g_weight: float = 0.0, SC=None, SA=None, V0=None, freq=None):
        """lam <- S_n^T lam + g_weight g for the step from F at time t (bte_step_adjoint); adds the
        step's sensitivity products to SC / SA (nv x nv float64 CUDA tensors) when given."""
        V0 = self.cfg["V0"] if V0 is None else V0
        freq = self.cfg["freq_Hz"] if freq is None else freq
        for m in (SC, SA):
            if m is not None and not (m.is_cuda and m.dtype == self.torch.float64 and m.numel() == self.nv * self.nv
                                      and m.is_contiguous()):
                raise ValueError("SC/SA must be contiguous float64 CUDA tensors of nv x nv")
        self._check(self.lib.bte_step_adjoint(self.h, _ptr(self._f(F)), _ptr(self._f(lam)), float(t), float(V0),
                                              float(freq), _ptr(None if g is None else self._f(g)), float(g_weight),
                                              _ptr(SC), _ptr(SA)))
        return lam

    def adjoint_gradient(self, SC, SA, h_eV: float = 1e-4) -> np.ndarray:
        """[dJ/dscale_j..., dJ/dthreshold_j..., dJ/dV0] from the accumulated sensitivities."""
        out = np.empty(2 * self.n_proc + 1, dtype=np.float64)
        self._check(self.lib.bte_adjoint_gradient(self.h, _ptr(SC), _ptr(SA), float(h_eV),
                                                  out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def profile_start(self):
        """Start recording CUDA events around every kernel launch of this handle."""
        self._check(self.lib.bte_profile(self.h, 1, None, None))

    def profile_stop(self) -> dict:
        """Stop recording; returns {kernel class: (summed device ms, launches)}."""
        ms = (C.c_double * len(KERNELS))()
        cnt = (C.c_ulonglong * len(KERNELS))()
        self._check(self.lib.bte_profile(self.h, 0, ms, cnt))
        return {k: (ms[j], cnt[j]) for j, k in enumerate(KERNELS)}

    def info(self) -> dict:
        i = Info()
        self._check(self.lib.bte_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in Info._fields_}


class Batch:
    """Many Solvers (uneven grids, pressures, cross sections) stepped together through one CUDA
    graph per step (bte_batch_*). The solvers stay owned by the caller and must outlive the batch."""

    def __init__(self, solvers, autotune: bool = False, stream=None):
        self.lib = load()
        import torch
        self.torch = torch
        self.solvers = list(solvers)
        if stream is None:
            stream = torch.cuda.current_stream(self.solvers[0].device)
        n = len(self.solvers)
        hs = (C.c_void_p * n)(*[sv.h for sv in self.solvers])
        b = C.c_void_p()
        st = self.lib.bte_batch_create(n, hs, C.c_void_p(stream.cuda_stream), BATCH_AUTOTUNE if autotune else 0,
                                       C.byref(b))
        if st != OK:
            raise BteError(st, self.lib.bte_batch_last_error(None).decode())
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            self.lib.bte_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, Fs, n_steps: int, t0, V0=None, freq=None, raise_on_error: bool = True):
        """n_steps steps of every instance; t0, V0, freq: scalars or one value per instance.
        Returns the per-instance status list."""
        n = len(self.solvers)
        if len(Fs) != n:
            raise ValueError("one state per instance")
        for sv, F in zip(self.solvers, Fs):
            sv._f(F)

        def vec(v, key):
            if v is None:
                v = [sv.cfg[key] for sv in self.solvers]
            v = np.broadcast_to(np.asarray(v, dtype=np.float64), (n,)).copy()
            return v
        t0v, v0v, fv = vec(t0, None) if t0 is not None else np.zeros(n), vec(V0, "V0"), vec(freq, "freq_Hz")
        ptrs = (C.c_void_p * n)(*[F.data_ptr() for F in Fs])
        status = (C.c_int * n)()
        pd_ = C.POINTER(C.c_double)
        st = self.lib.bte_batch_run(self.b, ptrs, int(n_steps), t0v.ctypes.data_as(pd_), v0v.ctypes.data_as(pd_),
                                    fv.ctypes.data_as(pd_), status)
        if st != OK and raise_on_error:
            raise BteError(st, self.lib.bte_batch_last_error(self.b).decode())
        return list(status)

    def info(self, i: int) -> dict:
        tc, w, pr, cg, lps = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_ulonglong()
        st = self.lib.bte_batch_get_info(self.b, int(i), C.byref(tc), C.byref(w), C.byref(pr), C.byref(cg),
                                         C.byref(lps))
        if st != OK:
            raise BteError(st, self.lib.bte_batch_last_error(self.b).decode())
        return {"tensor_cores": tc.value, "panel_w": w.value, "tc_pair": pr.value, "tc_cg": cg.value,
                "launches_per_step": lps.value}
