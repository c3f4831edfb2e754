"""Synthetic workloads shaped like the paper's RF glow discharges, and seeded input draws.

This module holds plain data and random draws only -- no arithmetic of the method. Both the
CUDA path (through the binding) and the CPU oracle read their inputs from here, so a parity test
feeds the two sides exactly the same numbers.

Shapes follow the paper's discharge set-up (Table "model parameters", Section 4.3: gap
L = 2.54 cm, 13.56 MHz drive, T0 = 300 K) with analytic stand-ins for the argon cross sections
(Section 3.2, Table "three species Ar collisional model"); the LXCat data the paper uses is not
shipped with this package.
"""
from __future__ import annotations

import copy
import numpy as np

RF_FREQ_HZ = 13.56e6
GAP_M = 2.54e-2

# Cross-section forms (energy eps in eV, threshold th in eV):
#   "const"   sigma = sigma0
#   "linear"  sigma = sigma0 * (1 - th/eps)              for eps > th, else 0
#   "log"     sigma = sigma0 * ln(eps/th) / (eps/th)     for eps > th, else 0
#   "nu"      sigma = sigma0 / v   (sigma0 in m^3/s, so n0*sigma*v is a constant frequency)
#   "table"   piecewise-linear in eps through (eps_eV[i], sigma_m2[i]), 0 outside the table
FORMS = ("const", "linear", "log", "table", "nu")
KINDS = ("elastic", "excitation", "ionization")


def process(kind, form, sigma0=0.0, threshold_eV=0.0, scale=1.0, eps_eV=None, sigma_m2=None):
    assert kind in KINDS and form in FORMS
    p = dict(kind=kind, form=form, sigma0=float(sigma0), threshold_eV=float(threshold_eV),
             scale=float(scale))
    if form == "table":
        p["eps_eV"] = [float(e) for e in eps_eV]
        p["sigma_m2"] = [float(s) for s in sigma_m2]
    return p


P1_ELASTIC = process("elastic", "const", 1e-19)
P2_EXC = process("excitation", "linear", 2e-21, 11.55)
P3_ION = process("ionization", "log", 3e-21, 15.76)
P4_EXC = process("excitation", "linear", 1e-21, 13.0)


def base(nx, nr, ntheta, p_Torr, V0, dt_frac, steps, processes, nl=None):
    """One discharge. dt = dt_frac / RF_FREQ_HZ; E(t) = (V0/L) sin(2 pi f t), uniform in x."""
    return dict(nx=nx, nr=nr, ntheta=ntheta, nl=ntheta if nl is None else nl,
                L_m=GAP_M, vmax_eV=30.0, p_Torr=p_Torr, T0_K=300.0, m0_amu=39.948,
                V0=V0, freq_Hz=RF_FREQ_HZ, dt_s=dt_frac / RF_FREQ_HZ, steps=steps,
                processes=copy.deepcopy(processes),
                ic=dict(Te_eV=2.0, ne_peak=1e15))


# The five workloads: single small FP64 discharge; FP64 vs mixed at Nv = 2048; batched uneven
# discharges; adjoint-sized discharge; largest single discharge.
SMALL = base(32, 16, 16, 1.0, 100.0, 1e-3, 200, [P1_ELASTIC, P2_EXC, P3_ION])
MEDIUM = base(128, 64, 32, 0.5, 150.0, 5e-4, 2000, [P1_ELASTIC, P2_EXC, P3_ION, P4_EXC])
ADJOINT = base(64, 32, 16, 1.0, 100.0, 1e-3, 1000, [P1_ELASTIC, P2_EXC, P3_ION, P4_EXC])
LARGEST = base(256, 128, 32, 0.1, 200.0, 5e-4, 20000, [P1_ELASTIC, P2_EXC, P3_ION, P4_EXC])

WORKLOADS = {"small_nx32_nr16_nt16": SMALL, "medium_nx128_nr64_nt32": MEDIUM,
             "adjoint_nx64_nr32_nt16": ADJOINT, "largest_nx256_nr128_nt32": LARGEST}


def batched_instances(n=64, seed=20250223):
    """Uneven discharges: per instance the draw order is pressure (log-uniform in [0.1, 2] Torr),
    V0 (uniform in [50, 200] V), then Nx, Nr, Ntheta from their candidate sets."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        p = float(np.exp(rng.uniform(np.log(0.1), np.log(2.0))))
        v0 = float(rng.uniform(50.0, 200.0))
        nx = int(rng.choice([64, 96, 128, 192]))
        nr = int(rng.choice([32, 48, 64]))
        nt = int(rng.choice([16, 24, 32]))
        out.append(base(nx, nr, nt, p, v0, 1e-3, 500, [P1_ELASTIC, P2_EXC, P3_ION]))
    return out


def scaled(cfg, **kw):
    """Copy of a workload with some fields replaced (grid sizes for parity-sized cases, etc.)."""
    c = copy.deepcopy(cfg)
    c.update(kw)
    if "ntheta" in kw and "nl" not in kw:
        c["nl"] = c["ntheta"]
    return c


def random_state(nx, ntheta, nr, seed=0, scale=1e15):
    """Seeded synthetic distribution coefficients F[x][theta][r] (float64, C order).

    Smooth positive bulk plus noise: a stand-in for a mid-cycle discharge state, used where a
    test wants an input that is not the symmetric initial Maxwellian."""
    rng = np.random.default_rng(seed)
    xi = np.linspace(-1.0, 1.0, nx)
    prof = (1.0 - xi**2)[:, None, None] + 0.05
    r = np.exp(-np.linspace(0.0, 6.0, nr))[None, None, :]
    f = prof * r * (1.0 + 0.3 * rng.standard_normal((nx, ntheta, nr)))
    return np.ascontiguousarray(scale * f, dtype=np.float64)


def random_field(nx, seed=0, e0=6.0e3):
    """Seeded non-uniform field samples E[x] in V/m (for per-point parity of the velocity step)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(e0 * rng.uniform(-1.0, 1.0, nx), dtype=np.float64)
