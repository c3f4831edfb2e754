"""Benchmark of the semi-implicit BTE step on GB300: DOF-updates/s, mixed precision vs plain FP64.

Workload: one discharge with Nx=128 Chebyshev points, Nr=64 B-splines, Ntheta=32 ordinates
(Nv = 2048, 262,144 DOFs), 0.5 Torr, 150 V at 13.56 MHz, dt = T_RF/2000, four analytic processes,
synthetic Maxwellian initial state. A step is one full bte_step: x half step, per-point dense
LU solve of the velocity system (with FP64 refinement in the mixed path), x half step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank steps its own discharge (independent replicas: weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_16555_gb300 import workloads as W  # noqa: E402

WORKLOAD = "medium_nx128_nr64_nt32"
LARGEST = "largest_nx256_nr128_nt32"   # the largest single discharge: a parity and timing case
METRIC = "DOF-updates/s per bte_step (mixed vs plain FP64, same GPU) at rel-L2 <=1e-6 vs FP64"
UNIT = "DOF-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal ratio TF32 : BF16 dense tensor throughput (1.1 : 2.25 PFLOP/s) applied to the measured
# BF16 peak; TF32x3 spends three tensor products per FP32-accurate product.
TF32_OVER_BF16 = 1.1 / 2.25
# FP32 SIMT peak from unit counts and clock: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (used when the
# library FP32 GEMM measured in the run is not a plain CUDA-core GEMM).
FP32_SIMT_UNITS_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the first-panel launch (k0 = 0) of
# the kernels captured with ncu on this workload (the commands are in profiles/); the per-launch
# figure reported is scaled to the step's average launch by the algorithmic bytes. Remove an entry
# when its kernel changes.
TRAFFIC_K0 = {"lu_gemm": 2.584127e9 + 1.590629e9, "lu_panel": 402.5408e6 + 122.445056e6}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"], "src": "measured",
                "when": p.get("when")}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback", "when": None}


def library_peaks(torch, n64=4096, n32=8192):
    """cuBLAS GEMM throughput on this GPU, measured now (torch.matmul, best of several, CUDA
    events): FP64 (DGEMM, n64^3), FP32 on the CUDA cores (SGEMM without TF32, n32^3) and TF32
    (n32^3). TFLOP/s = 2 n^3 / time."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    for name, dt, tf32, n, it in (("fp64", torch.float64, False, n64, 3), ("fp32", torch.float32, False, n32, 4),
                                  ("tf32", torch.float32, True, n32, 8)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        a @ b
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(it):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name + "_tflops"] = 2.0 * n**3 / best / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def roofline_peaks(file_peaks, lib=None, clocks=None):
    """The denominators of the roofline fractions, each with where it comes from:
      hbm      copy bandwidth from MEASURED_PEAKS.json;
      tensor   TF32x3 = the TF32 library GEMM measured in this run / 3 products (the BF16 peak of
               MEASURED_PEAKS.json x 1.1/2.25 / 3 is reported beside it);
      fp64     the FP64 library GEMM measured in this run;
      fp32     the FP32 CUDA-core library GEMM measured in this run, unless it runs faster than the
               unit-count peak (then it is not a CUDA-core GEMM and the unit count is used)."""
    bf16_derived = file_peaks["bf16_tflops"] * TF32_OVER_BF16 / 3.0
    p = {"hbm_gbs": file_peaks["hbm_gbs"],
         "hbm_src": "MEASURED_PEAKS.json hbm_gbs (%s%s)" % (file_peaks["src"],
                                                           ", " + file_peaks["when"] if file_peaks.get("when") else ""),
         "tensor_tflops_bf16_derived": bf16_derived}
    run = "measured in this run (cuBLAS via torch.matmul, best of several)"
    if lib:
        p["tensor_tflops"] = lib["tf32_tflops"] / 3.0
        p["tensor_src"] = "TF32 GEMM 8192^3 %s: %.1f TFLOP/s / 3 products" % (run, lib["tf32_tflops"])
        p["fp64_tflops"] = lib["fp64_tflops"]
        p["fp64_src"] = "FP64 GEMM 4096^3 " + run
        if lib["fp32_tflops"] <= 1.15 * FP32_SIMT_UNITS_TFLOPS:
            p["fp32_tflops"] = lib["fp32_tflops"]
            p["fp32_src"] = "FP32 CUDA-core GEMM 8192^3 " + run
        else:
            p["fp32_tflops"] = FP32_SIMT_UNITS_TFLOPS
            p["fp32_src"] = ("unit counts (152 SMs x 128 lanes x 2 flop x 2.07 GHz); the FP32 library GEMM "
                             "measured %.1f TFLOP/s, above that, so not a CUDA-core GEMM" % lib["fp32_tflops"])
        p["library"] = dict(lib, clocks=clocks)
    else:
        p["tensor_tflops"] = bf16_derived
        p["tensor_src"] = "MEASURED_PEAKS.json bf16_tflops x 1.1/2.25 (TF32) / 3 products"
        p["fp64_tflops"] = 1.10
        p["fp64_src"] = "FP64 GEMM measured on a GB300 of this pool in an earlier run"
        p["fp32_tflops"] = FP32_SIMT_UNITS_TFLOPS
        p["fp32_src"] = "unit counts: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    return p


# ---------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------- work model

def tc_pairs(nv):
    """The tensor-core factorisation in panel pairs: (k0, width of the second panel, trailing
    columns right of the pair) per pair, as the library orders it."""
    out = []
    for k0 in range(0, nv, 256):
        if k0 + min(128, nv - k0) >= nv:
            break
        kb2 = min(128, nv - k0 - 128)
        out.append((k0, kb2, max(0, nv - k0 - 256)))
    return out


def algorithmic(cfg, precision, kernel, tc, pair=True):
    """(amount, unit, bound) of the algorithmic work of one step for a kernel class (per-step sums
    over its launches; per unit):
      lu_panel     read + write of every outer panel once: 2 * 4 B * (Nv - k0) * 128 per point;
      lu_gemm      trailing updates, 2 M^2 128 flop per point and panel (M = Nv - k0 - 128); on the
                   tensor cores in panel pairs: 2 M1 kb2 128 for the first panel's update of the
                   second panel's columns (M1 = Nv - k0 - 128) plus 2 M2^2 256 for the pair's update
                   (M2 = Nv - k0 - 256);
      lu_swap_trsm U12 = inv(L11) P A12, 2 * 128 * M * 128 flop per point and panel; in pairs
                   2 * 128 * kb2 * 128 plus 2 * 3 * 128^2 * M2 (the nonzero blocks of the pair's
                   inv(L11)) plus 2 * 128^3 for that inverse's off-diagonal block;
      lu_solve     per point solve: the strictly block-lower and block-upper factors and the
                   panels' two diagonal-block inverses, esz * (n^2 + n * nb) (n = the order factored);
      x_apply_q    the FP64 Q stream (8 B Nv Nx^2) plus Y in/out, per half step;
      v_form       write of the per-point matrices plus the K_C/K_A read;
      residual     FP64 flops of the structured residual (Algorithm 2) per point evaluation,
                   banded products and the banded Cholesky substitutions of M_v.
    The refinement kernels skip converged points, so those two count point-solves and point
    evaluations (the library's exact count of residual evaluations per point and step)."""
    nx, nr, nt = cfg["nx"], cfg["nr"], cfg["ntheta"]
    nv = nr * nt
    nl = cfg.get("nl") or nt
    esz = 8 if precision == "fp64" else 4
    nb = 64 if precision == "fp64" else 128
    panels = [(k0, min(nb, nv - k0)) for k0 in range(0, nv, nb)]
    if kernel == "lu_panel":
        return sum(2.0 * esz * (nv - k0) * kb for k0, kb in panels) * nx, "byte", "hbm"
    if kernel == "lu_panel_flops":
        # LU of an m x kb panel: m kb^2 - kb^3/3 flops (leading terms), m = Nv - k0
        return sum((nv - k0) * kb * kb - kb ** 3 / 3.0 for k0, kb in panels) * nx, "flop", "alu"
    if kernel == "lu_gemm":
        if tc and pair:
            return sum(2.0 * (nv - k0 - 128) * kb2 * 128 + 2.0 * m2 ** 2 * 256
                       for k0, kb2, m2 in tc_pairs(nv)) * nx, "flop", "tensor"
        return sum(2.0 * (nv - k0 - kb) ** 2 * kb for k0, kb in panels) * nx, "flop", "tensor" if tc else "alu"
    if kernel == "lu_swap_trsm":
        if tc and pair:
            return sum(2.0 * 128 * kb2 * 128 + (2.0 * 3 * 128 ** 2 * m2 + 2.0 * 128 ** 3 if m2 else 0.0)
                       for k0, kb2, m2 in tc_pairs(nv)) * nx, "flop", "tensor"
        return sum(2.0 * kb * (nv - k0 - kb) * kb for k0, kb in panels) * nx, "flop", "tensor" if tc else "alu"
    if kernel == "lu_solve":
        n = nl * nr if nl < nt else nv
        return float(esz) * (n * n + n * nb), "byte/point", "hbm"
    if kernel == "x_apply_q":
        return 2 * (8.0 * nv * nx * nx + 16.0 * nv * nx), "byte", "hbm"
    if kernel == "x_apply_q_flops":
        return 2 * (2.0 * nv * nx * nx), "flop", "alu"
    if kernel == "v_form":
        return float(esz) * nx * nv * nv + 16.0 * nv * nv, "byte", "hbm"
    if kernel == "residual":
        # P_S and P_O projections, C_0 dense, the loss band of C_l (l >= 1), the field blocks as
        # banded combinations of Dv and M1 (two neighbours), the two banded Cholesky substitutions
        # of M_v (half bandwidth w = 3 for cubic B-splines)
        w = 3
        fma = (2 * nl * nt * nr + nr * nr + (nl - 1) * nr * (2 * w + 1) + 2 * (nl - 1) * nr * (2 * w + 1)
               + 2 * nl * nr * w)
        return 2.0 * fma, "flop/point", "alu"
    return None, None, None


def traffic_per_launch(cfg, kernel, launches_per_step):
    """Measured DRAM bytes of the k0 = 0 launch scaled to the average launch of the step (both
    kernels move bytes in proportion to their algorithmic bytes, which shrink with k0)."""
    if kernel not in TRAFFIC_K0 or not launches_per_step:
        return None
    nv = cfg["nr"] * cfg["ntheta"]
    nb = 128
    if kernel == "lu_gemm":
        # the k0 = 0 pair launch (C read and written once: 2 M2^2 words) scales the pair launches by
        # M2^2 and the single-panel-column launches by their M1 x kb2 block
        per = []
        for k0, kb2, m2 in tc_pairs(nv):
            per.append((nv - k0 - 128) * kb2)
            if m2:
                per.append(m2 ** 2)
        return TRAFFIC_K0[kernel] * (sum(per) / len(per)) / (nv - 256) ** 2
    else:
        per = [nv - k0 for k0 in range(0, nv, nb)]
    return TRAFFIC_K0[kernel] * (sum(per) / len(per)) / per[0]


def roofline_of(cfg, precision, kernel, prof, steps, peaks, tc, evals=None, measured=True):
    amount, unit, bound = algorithmic(cfg, precision, kernel, tc)
    ms, launches = prof.get(kernel, (0.0, 0))
    if amount is None or launches == 0 or ms <= 0:
        return None
    if unit.endswith("/point"):
        # one solve and one residual evaluation per point and evaluation (converged points skip)
        if evals is None:
            return None
        units = steps * cfg["nx"] * evals
    else:
        units = steps
    total = amount * units
    rate = total / (ms / 1e3)
    if bound == "hbm":
        achieved, peak, u, src = rate / 1e9, peaks["hbm_gbs"], "GB/s", peaks["hbm_src"]
    elif bound == "tensor":
        achieved, peak, u, src = rate / 1e12, peaks["tensor_tflops"], "TFLOP/s", peaks["tensor_src"]
    elif precision == "fp64" or kernel == "residual":
        achieved, peak, u, src = rate / 1e12, peaks["fp64_tflops"], "TFLOP/s", peaks["fp64_src"]
    else:
        achieved, peak, u, src = rate / 1e12, peaks["fp32_tflops"], "TFLOP/s", peaks["fp32_src"]
    out = {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": u,
           "frac": achieved / peak,
           "traffic": traffic_per_launch(cfg, kernel, launches / steps) if measured else None,
           "launches_per_step": launches / steps, "ms_per_step": ms / steps, "peak_source": src}
    if unit.endswith("/point"):
        out["point_units_per_step"] = cfg["nx"] * evals
    return out


def rooflines(cfg, precision, prof, steps, peaks, tc, evals=None, measured=True):
    out = {}
    for k in prof:
        r = roofline_of(cfg, precision, k, prof, steps, peaks, tc, evals, measured)
        if r:
            out[k] = r
    dom = max(out, key=lambda k: out[k]["ms_per_step"])
    return out[dom], out


# ---------------------------------------------------------------------------------- CPU oracle leg

def oracle_sample(cfg, budget_s=20.0, name=WORKLOAD):
    """Time the oracle (as it stands) on the host: one full x half step plus the velocity solve of a
    bounded subset of points; the per-step time is 2 t_x + (Nx/k) t_v(k)."""
    from oracle import bte as O
    ops = O.Operators(cfg)
    F = ops.initial_state()
    t0 = time.perf_counter()
    F1 = ops.x_halfstep(F)
    tx = time.perf_counter() - t0
    E = ops.field(0.25 / cfg["freq_Hz"])
    k, tv = 0, 0.0
    while k < cfg["nx"] and (tv + 2 * tx) < budget_s:
        t0 = time.perf_counter()
        np.linalg.solve(ops.v_matrix(E[k]), F1[k].reshape(-1))
        tv += time.perf_counter() - t0
        k += 1
    step_s = 2 * tx + cfg["nx"] / k * tv
    dof = cfg["nx"] * cfg["nr"] * cfg["ntheta"]
    cores = len(os.sched_getaffinity(0))
    return {"value": dof / step_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{name}: 1 full x half step ({tx:.2f} s) + dense v-solves of {k}/{cfg['nx']} points "
                      f"({tv:.2f} s), extrapolated to one step = {step_s:.2f} s; numpy/LAPACK on {cores} host threads"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cfg = W.WORKLOADS[WORKLOAD]
    vals = []
    for _ in range(max(1, args.warmup)):
        oracle_sample(cfg, budget_s=3.0)
    for _ in range(args.steps):
        vals.append(oracle_sample(cfg, budget_s=8.0))
    v = float(np.median([x["value"] for x in vals]))
    base = vals[-1]
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 262144 / v * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "nx": 128, "nr": 64, "ntheta": 32},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                            "sample": base["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------------- GPU leg

def run_ours(args, rank, world):
    import torch
    from paper_2502_16555_gb300 import bte

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    name = args.workload if args.workload in (WORKLOAD, LARGEST) else WORKLOAD
    cfg = W.WORKLOADS[name]
    if args.nx:
        # fewer collocation points of the same velocity grid: the small case that profiler
        # captures use (not a bench line)
        cfg = W.scaled(cfg, nx=args.nx)
    dof = cfg["nx"] * cfg["nr"] * cfg["ntheta"]
    dt = cfg["dt_s"]
    # roofline denominators: the copy bandwidth from MEASURED_PEAKS.json, the library GEMM rates now
    with ClockSampler(local) as pclk:
        lib = library_peaks(torch)
    peaks = roofline_peaks(load_peaks(), lib, pclk.summary())

    # ---- mixed precision (the headline)
    s = bte.Solver(cfg, precision="mixed", panel_tc=args.panel_tc)
    tc = bool(s.info()["tensor_cores"])
    F = s.initial_state()
    F0 = F.clone()
    s.run(F, args.warmup, 0.0)
    launches0 = s.info()["launches"]
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        s.profile_start()
        ev0.record()
        s.run(F, args.steps, args.warmup * dt)
        ev1.record()
        barrier()
        prof = s.profile_stop()
    launches = s.info()["launches"] - launches0
    sweeps = s.info()["last_refine_sweeps"]
    evals = s.info()["last_refine_evals"]
    ms = ev0.elapsed_time(ev1) / args.steps
    # the same timing again without event bracketing of every kernel (the end-to-end leg below
    # repeats exactly these steps: same start state, same times)
    s.run(F, 1, (args.warmup + args.steps) * dt)
    Fq = F.clone()
    F_e2e = F.clone()
    t_q = (args.warmup + args.steps + 1) * dt
    barrier()
    launches1 = s.info()["launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.run(Fq, args.steps, t_q)   # replays the library's CUDA graph of one step (no event bracketing)
    e1.record()
    barrier()
    ms_plain = e0.elapsed_time(e1) / args.steps
    launches_plain = s.info()["launches"] - launches1
    if ms_plain <= ms:
        launches = launches_plain   # the kernels of the run the value is taken from
    ms = max_over_ranks(min(ms, ms_plain), dist)
    value = world * dof / (ms / 1e3)

    # ---- plain FP64 on the same GPU, same steps from the same state
    fp64 = None
    if not args.no_fp64:
        s64 = bte.Solver(cfg, precision="fp64")
        G = F0.clone()
        n64 = args.warmup + args.steps
        s64.run(G, args.warmup, 0.0)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        s64.run(G, args.steps, args.warmup * dt)
        f1.record()
        barrier()
        ms64 = f0.elapsed_time(f1) / args.steps
        # accuracy of the mixed path against FP64 after the same n64 steps
        Fm = F0.clone()
        s.run(Fm, n64, 0.0)
        ne_m, _, _ = s.moments(Fm)
        ne_d, _, _ = s64.moments(G)
        torch.cuda.synchronize()
        fp64 = {"value": world * dof / (ms64 / 1e3), "ms_per_step": ms64, "unit": UNIT,
                "accuracy_mixed_vs_fp64": {"steps": n64,
                                           "rel_l2_f": float(torch.linalg.norm(Fm - G) / torch.linalg.norm(G)),
                                           "rel_l2_ne": float(torch.linalg.norm(ne_m - ne_d) / torch.linalg.norm(ne_d))}}
        del s64

    # ---- the structure-exploiting velocity solve (block tridiagonal in l), both precisions, from the
    # same state for the same steps; accuracy against the dense FP64 state after the same steps
    structured = None
    if not args.no_structured and cfg["nr"] <= 64:
        structured = {}
        n_chk = args.warmup + args.steps
        for prec in ("mixed", "fp64"):
            ss = bte.Solver(cfg, precision=prec, structured=True)
            Gs = F0.clone()
            ss.run(Gs, args.warmup, 0.0)
            barrier()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record()
            ss.run(Gs, args.steps, args.warmup * dt)
            g1.record()
            barrier()
            mss = g0.elapsed_time(g1) / args.steps
            entry = {"value": world * dof / (mss / 1e3), "ms_per_step": mss, "unit": UNIT,
                     "refine_sweeps": ss.info()["last_refine_sweeps"]}
            if fp64 is not None:
                ne_s, _, _ = ss.moments(Gs)
                entry["rel_l2_f_vs_dense_fp64"] = float(torch.linalg.norm(Gs - G) / torch.linalg.norm(G))
                entry["rel_l2_ne_vs_dense_fp64"] = float(torch.linalg.norm(ne_s - ne_d) / torch.linalg.norm(ne_d))
                entry["steps_compared"] = n_chk
            structured[prec] = entry
            del ss

    # ---- accuracy over the configured run (one RF cycle of 2000 steps for the default discharge):
    # the mixed path against FP64. The dense FP64 path takes about 0.65 s per step here, so the
    # reference is the FP64 block-tridiagonal solve of the same systems (refined in FP64), which
    # matches the dense FP64 path to ~1e-15 over the steps compared above (structured_solve).
    cycle = None
    if not args.no_cycle and cfg["nr"] <= 64 and cfg.get("steps"):
        n_cyc = int(cfg["steps"])
        Fm = F0.clone()
        Gs = F0.clone()
        s.run(Fm, n_cyc, 0.0)
        ref = bte.Solver(cfg, precision="fp64", structured=True)
        ref.run(Gs, n_cyc, 0.0)
        ne_m, _, _ = s.moments(Fm)
        ne_r, _, _ = ref.moments(Gs)
        torch.cuda.synchronize()
        cycle = {"steps": n_cyc, "reference": "FP64 block-tridiagonal solve (BTE_FLAG_STRUCTURED), same start state",
                 "rel_l2_f": float(torch.linalg.norm(Fm - Gs) / torch.linalg.norm(Gs)),
                 "rel_l2_ne": float(torch.linalg.norm(ne_m - ne_r) / torch.linalg.norm(ne_r))}
        del ref, Fm, Gs

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region:
    # the device-timed plain run's steps again, from its start state at its times
    e2e = None
    if not args.no_e2e:
        Fh = torch.empty(F.shape, dtype=torch.float64, pin_memory=True).numpy()
        Fh[...] = F_e2e.cpu().numpy()
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            s.step_host(Fh, t_q + i * dt)
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": world * dof / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * dof,
               "d2h_bytes_per_step": 8 * dof, "ms_per_step": e2e_s * 1e3, "api": "bte_step_host",
               "steps": "the device-timed plain run's %d steps: same start state and times" % args.steps,
               "matches_device_run": bool(np.array_equal(Fh, Fq.cpu().numpy()))}

    # the measured DRAM traffic was captured on the default workload only
    measured = name == WORKLOAD and not args.nx
    rf_dom, rf_all = rooflines(cfg, "mixed", prof, args.steps, peaks, tc, evals=evals, measured=measured)
    # kernels with a flop and a byte floor are measured against the binding one: the panel's FP32
    # flops (CUDA-core peak) and the Q apply's FP64 flops (FP64 peak) take longer than their bytes
    for kern, fkey, fpeak, fsrc in (
            ("lu_panel", "lu_panel_flops", peaks["fp32_tflops"], peaks["fp32_src"]),
            ("x_apply_q", "x_apply_q_flops", peaks["fp64_tflops"], peaks["fp64_src"])):
        if kern not in prof or not prof[kern][1] or kern not in rf_all:
            continue
        fl, _, _ = algorithmic(cfg, "mixed", fkey, tc)
        by, _, _ = algorithmic(cfg, "mixed", kern, tc)
        t_alu, t_hbm = fl / (fpeak * 1e12), by / (peaks["hbm_gbs"] * 1e9)
        if t_alu <= t_hbm:
            continue
        ms_k = prof[kern][0] / args.steps
        hbm = rf_all[kern]
        rate = fl / (ms_k / 1e3) / 1e12
        rf_all[kern] = dict(hbm, bound="alu", achieved=rate, peak=fpeak, unit="TFLOP/s", frac=rate / fpeak,
                            peak_source=fsrc, hbm_frac=hbm["frac"], floor_ms={"alu": t_alu * 1e3, "hbm": t_hbm * 1e3})
        if rf_dom["kernel"] == kern:
            rf_dom = rf_all[kern]
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "fp32-panel+tf32x3+f64-refine" if prof["lu_gemm"][1] and tc else "fp32+f64-refine",
        "data": "synthetic",
        "config": {"workload": name, "nx": cfg["nx"], "nr": cfg["nr"], "ntheta": cfg["ntheta"],
                   "nv": cfg["nr"] * cfg["ntheta"], "dof": dof, "precision": "mixed",
                   "l2": "working set > L2: %.1f GB of per-point FP32 factors streamed every step"
                         % (4.0 * cfg["nx"] * (cfg["nr"] * cfg["ntheta"]) ** 2 / 1e9),
                   "parallelism": f"replicas x{world}"},
        "fp64": fp64,
        "speedup_mixed_over_fp64": (fp64["ms_per_step"] / ms) if fp64 else None,
        "structured_solve": structured,
        "cycle_accuracy": cycle,
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": rf_dom,
        "rooflines": rf_all,
        "peaks": peaks,
        "refinement": {"sweeps_rounded_up": sweeps, "residual_evals_per_point_step": evals},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
    }
    if world == 1 and not args.no_cpu:
        out["cpu_baseline"] = oracle_sample(cfg, name=name)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def max_over_ranks(x, dist, device="cuda"):
    """The largest of every rank's value (all-reduce MAX); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n, rank, world):
    """Instances of a batched workload handled by one rank: a contiguous, balanced slice (no
    data-path exchange between ranks)."""
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return list(range(lo, hi))


def run_batched(args, rank, world):
    """64 uneven discharges (per-instance grids, pressures, amplitudes drawn from a fixed seed)
    stepped together through one CUDA graph per step, autotuned per shape; instances are sharded
    across ranks. Mixed precision; with --batched-fp64 also the plain FP64 batch on the same
    instances (one timed step)."""
    import torch
    from paper_2502_16555_gb300 import bte

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    inst = W.batched_instances()
    mine = [inst[k] for k in shard(len(inst), rank, world)]

    def leg(precision, steps, warmup, sequential=False):
        sv = [bte.Solver(c, precision=precision) for c in mine]
        Fs = [s.initial_state() for s in sv]
        t_setup = time.perf_counter()
        b = bte.Batch(sv, autotune=True)
        t_setup = time.perf_counter() - t_setup
        b.run(Fs, warmup, 0.0)
        t0 = [warmup * c["dt_s"] for c in mine]
        Fseq = [F.clone() for F in Fs] if sequential else None
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record()
            b.run(Fs, steps, t0)
            e1.record()
            torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist)
        info = [b.info(i) for i in range(len(sv))]
        seq = None
        if sequential:
            # the same instances, variants, states and times, stepped one discharge after another
            # (each through bte_run on its own stream): what batching buys over a loop of handles
            per = []
            torch.cuda.synchronize()
            for k, (sk, F) in enumerate(zip(sv, Fseq)):
                q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                q0.record(sk.stream)
                sk.run(F, steps, t0[k])
                q1.record(sk.stream)
                torch.cuda.synchronize()
                per.append(q0.elapsed_time(q1) / steps)
            same = max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(Fseq, Fs))
            seq = {"ms_per_step": sum(per), "instance_ms_min": min(per), "instance_ms_max": max(per),
                   "batch_speedup": sum(per) / ms,
                   "max_rel_l2_vs_batch": same}
        ne = [s.moments(F)[0] for s, F in zip(sv, Fs)]
        b.close()
        del sv, Fs, Fseq
        torch.cuda.empty_cache()
        return ms, info, clk.summary(), t_setup, ne, seq

    dof_all = sum(c["nx"] * c["nr"] * c["ntheta"] for c in inst)

    def variant_name(i):
        if not i["tensor_cores"]:
            return "cuda-core update"
        if not i["tc_pair"]:
            return "tensor cores, single panels (K=128, 128x128 tiles)"
        return "tensor cores, panel pairs (K=256, %s)" % ("256x256 CTA-pair tiles" if i["tc_cg"] == 2
                                                        else "128x128 one-CTA tiles")
    ms, info, clocks, t_setup, ne_m, seq = leg("mixed", args.steps, args.warmup, sequential=True)
    shapes = {}
    for c, i in zip(mine, info):
        key = "nx%d_nr%d_nt%d" % (c["nx"], c["nr"], c["ntheta"])
        shapes[key] = "%s; panel block %s" % (variant_name(i), "8x8" if i["panel_w"] == 8 else "16x4")
    out = {
        "metric": METRIC, "value": dof_all / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "fp32-panel+tf32x3+f64-refine", "data": "synthetic",
        "config": {"workload": "batched64_uneven", "instances": len(inst), "dof": dof_all,
                   "graph": "one CUDA graph launch per step, instances as concurrent branches",
                   "l2": "working set > L2", "parallelism": f"instances sharded over {world} rank(s)"},
        "clocks": clocks,
        "gpu_launches": int(info[0]["launches_per_step"] * args.steps) if info else 0,
        "autotune": {"setup_s": t_setup,
                     "tensor_core_instances": sum(i["tensor_cores"] for i in info),
                     "panel_w8_instances": sum(1 for i in info if i["panel_w"] == 8),
                     "choice_per_shape": shapes},
        "sequential": seq,
    }
    if args.batched_fp64:
        ms64, _, _, _, ne_d, _ = leg("fp64", 1, 1)
        out["fp64"] = {"value": dof_all / (ms64 / 1e3), "ms_per_step": ms64, "unit": UNIT}
        out["speedup_mixed_over_fp64"] = ms64 / ms
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


HYBRID = "hybrid_nx128_nr64_nt32"


def run_hybrid(args, rank, world):
    """The self-consistent parts on the medium workload (mixed precision, ion density of the same
    parabolic shape as the electrons, 1.05e15 m^-3 peak): the ion step (eq. "fluid_step"), the
    semi-implicit step with the field recomputed from the electrons, and the fully-implicit step
    (Newton-GMRES) at the same dt and at 4 dt (the paper's comparison of the two schemes runs the
    fully-implicit one at a 4x larger step). Each leg starts from the same state; times are CUDA
    events around `steps` steps after `warmup` steps."""
    import torch
    from paper_2502_16555_gb300 import bte
    from oracle import bte as O

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if rank != 0:
        return 0
    cfg = W.WORKLOADS[WORKLOAD]
    dof = cfg["nx"] * cfg["nr"] * cfg["ntheta"]
    x = O.cheb_points(cfg["nx"], cfg["L_m"])
    ni0 = torch.from_numpy(1.05e15 * (1.0 - (2.0 * x / cfg["L_m"] - 1.0) ** 2) + 1e13).cuda()
    t0 = 0.25 / cfg["freq_Hz"]

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = [fn(i) for i in range(n)]
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n, out

    s = bte.Solver(cfg, precision="mixed")
    F0 = s.initial_state()
    out = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "data": "synthetic", "dtype": "fp32-panel+tf32x3+f64-refine",
           "config": {"workload": HYBRID, "nx": cfg["nx"], "nr": cfg["nr"], "ntheta": cfg["ntheta"],
                      "dof": dof, "precision": "mixed", "ions": "parabolic, peak 1.05e15 m^-3"}}
    # ions
    ni = ni0.clone()
    for i in range(args.warmup):
        s.ion_step(ni, F0, t0)
    ms_ion, _ = timed(lambda i: s.ion_step(ni, F0, t0 + i * cfg["dt_s"]), args.steps)
    out["ion_step"] = {"ms_per_step": ms_ion, "nx": cfg["nx"]}
    # semi-implicit, self-consistent field
    F = F0.clone()
    for i in range(args.warmup):
        s.step_sc(F, ni0, t0 + i * cfg["dt_s"])
    F = F0.clone()
    ms_sc, _ = timed(lambda i: s.step_sc(F, ni0, t0 + i * cfg["dt_s"]), args.steps)
    out["semi_implicit_sc"] = {"ms_per_step": ms_sc, "value": dof / (ms_sc / 1e3), "dt_s": cfg["dt_s"]}
    # fully implicit at dt and at 4 dt
    for tag, k in (("fully_implicit", 1), ("fully_implicit_4dt", 4)):
        c = dict(cfg)
        c["dt_s"] = k * cfg["dt_s"]
        si = s if k == 1 else bte.Solver(c, precision="mixed")
        import ctypes as C

        def implicit(i, si=si, c=c, k=k):
            # at 4 dt the iteration is capped (8 Newton x 400 GMRES): it is reported, converged or not
            o = bte.ImplicitOpts(newton_max=12 if k == 1 else 8, gmres_max=1000 if k == 1 else 400)
            st = si.lib.bte_step_implicit(si.h, bte._ptr(Fi), bte._ptr(ni0), t0 + i * c["dt_s"], float(c["V0"]),
                                          float(c["freq_Hz"]), C.byref(o))
            return st, o.newton_iters, o.gmres_iters, o.residual

        Fi = F0.clone()
        for i in range(max(1, args.warmup) if k == 1 else 0):
            implicit(i)
        Fi = F0.clone()
        ms, stats = timed(implicit, args.steps if k == 1 else 1)
        out[tag] = {"ms_per_step": ms, "value": dof / (ms / 1e3), "dt_s": c["dt_s"],
                    "converged_steps": sum(1 for st in stats if st[0] == bte.OK), "steps": len(stats),
                    "newton_per_step": sum(st[1] for st in stats) / len(stats),
                    "gmres_per_step": sum(st[2] for st in stats) / len(stats),
                    "relative_residuals": [st[3] for st in stats]}
    # cost per simulated time, semi-implicit over fully-implicit at 4 dt (> 1: the implicit wins)
    out["semi_over_fully_4dt_per_simulated_time"] = (ms_sc / cfg["dt_s"]) / (
        out["fully_implicit_4dt"]["ms_per_step"] / (4 * cfg["dt_s"]))
    out["value"] = out["semi_implicit_sc"]["value"]
    out["ms_per_step"] = ms_sc
    print(json.dumps(out), flush=True)
    return 0


HYBRID_TABLE = "hybrid_table_nt16_nl3"
# The rows of the paper's table comparing the two electron schemes in the hybrid model
# (Section 5.3, Table "performance_hybrid"): (Nr, Nx) at Ntheta = 16 ordinates and N_l = 3
# harmonics, semi-implicit at dt f = 5e-5, fully-implicit at dt f = 2e-4; the paper's step
# times on one A100 (seconds, whole hybrid step with the ions), context only.
TABLE_ROWS = [(64, 100, 3.53e-2, 6.52e-2), (128, 100, 3.61e-2, 6.55e-2), (256, 100, 3.71e-2, 6.68e-2),
              (128, 200, 3.93e-2, 2.52e-1)]


def run_hybrid_table(args, rank, world):
    """The whole hybrid step (ion step, then the electron step) on the paper's table rows, both
    electron schemes, from the workload's initial state (Maxwellian at 2 eV, n_e peak 1e15 m^-3)
    with parabolic ions (peak 1.05e15 m^-3), argon at 1 Torr with the three analytic processes,
    V0 = 100 V. Times are CUDA events around `steps` consecutive steps after `warmup` steps; the
    fully-implicit leg records its Newton and GMRES counts and whether each step converged."""
    import ctypes as C
    import torch
    from paper_2502_16555_gb300 import bte
    from oracle import bte as O

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if rank != 0:
        return 0
    f = W.RF_FREQ_HZ

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = [fn(i) for i in range(n)]
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n, out

    rows = []
    for nr, nx, paper_semi, paper_fully in TABLE_ROWS:
        row = {"nr": nr, "ntheta": 16, "nl": 3, "nx": nx, "dof": nx * nr * 16,
               "paper_a100_s": {"semi_implicit": paper_semi, "fully_implicit": paper_fully,
                                "speedup": 4 * paper_semi / paper_fully}}
        x = O.cheb_points(nx, W.GAP_M)
        ni0 = torch.from_numpy(1.05e15 * (1.0 - (2.0 * x / W.GAP_M - 1.0) ** 2) + 1e13).cuda()
        for tag, dtf in (("semi_implicit", 5e-5), ("fully_implicit", 2e-4)):
            cfg = W.scaled(W.SMALL, nx=nx, nr=nr, ntheta=16, nl=3, p_Torr=1.0, V0=100.0, dt_s=dtf / f)
            s = bte.Solver(cfg, precision="mixed")
            F, ni = s.initial_state(), ni0.clone()
            t0 = 0.25 / f
            opts = bte.ImplicitOpts(newton_max=12, gmres_max=1000)

            def step(i, s=s, F=F, ni=ni, cfg=cfg, tag=tag, opts=opts):
                t = t0 + i * cfg["dt_s"]
                s.ion_step(ni, F, t)
                if tag == "semi_implicit":
                    s.step_sc(F, ni, t)
                    return (bte.OK, 0, 0, 0.0)
                st = s.lib.bte_step_implicit(s.h, bte._ptr(F), bte._ptr(ni), t, float(cfg["V0"]),
                                             float(cfg["freq_Hz"]), C.byref(opts))
                return (st, opts.newton_iters, opts.gmres_iters, opts.residual)

            for i in range(args.warmup):
                step(i)
            n = args.steps if tag == "semi_implicit" else max(1, min(args.steps, 3))
            ms, stats = timed(lambda i: step(args.warmup + i), n)
            leg = {"ms_per_step": ms, "dt_f": dtf, "steps": n}
            if tag == "fully_implicit":
                leg.update({"converged_steps": sum(1 for st in stats if st[0] == bte.OK),
                            "newton_per_step": sum(st[1] for st in stats) / n,
                            "gmres_per_step": sum(st[2] for st in stats) / n,
                            "relative_residuals": [st[3] for st in stats]})
            row[tag] = leg
            del s, F, ni
            torch.cuda.empty_cache()
        # overall runtime for the same simulated time, semi-implicit over fully-implicit
        row["speedup"] = 4 * row["semi_implicit"]["ms_per_step"] / row["fully_implicit"]["ms_per_step"]
        row["semi_implicit_vs_paper"] = paper_semi * 1e3 / row["semi_implicit"]["ms_per_step"]
        row["fully_implicit_vs_paper"] = paper_fully * 1e3 / row["fully_implicit"]["ms_per_step"]
        rows.append(row)
    out = {"metric": "hybrid step time, semi-implicit vs fully-implicit electrons (ions included)",
           "unit": "ms/step", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "data": "synthetic", "dtype": "fp32-panel+tf32x3+f64-refine",
           "config": {"workload": HYBRID_TABLE, "precision": "mixed", "p_Torr": 1.0, "V0": 100.0,
                      "ions": "parabolic, peak 1.05e15 m^-3"},
           "rows": rows}
    print(json.dumps(out), flush=True)
    return 0


def run_adjoint(args, rank, world):
    """Gradient of the cycle-averaged electron number over one RF cycle (1000 steps, FP64,
    Nx=64, Nr=32, Ntheta=16) with respect to 8 parameters (four cross-section scales, three
    threshold shifts, V0) by the adjoint with checkpoints every 50 steps, checked against central
    differences (h = 1e-6 relative) of the same forward run."""
    import torch
    from paper_2502_16555_gb300 import adjoint

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = W.WORKLOADS["adjoint_nx64_nr32_nt16"]
    steps = cfg["steps"] if args.adjoint_steps <= 0 else args.adjoint_steps
    m = adjoint.CycleDensity(cfg, steps=steps, checkpoint=50)
    th = m.theta0()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, saved = m.forward(th)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g = m.gradient(saved)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    fd = []
    for k in range(th.size):
        h = 1e-6 * max(1.0, abs(th[k]))
        up, dn = th.copy(), th.copy()
        up[k] += h
        dn[k] -= h
        fd.append((m.forward(up)[0] - m.forward(dn)[0]) / (2 * h))
    fd = np.array(fd)
    rel = np.abs(g - fd) / np.maximum(np.abs(fd), 1e-300)
    normwise = float(np.abs(g - fd).max() / np.abs(g).max())
    dof = cfg["nx"] * cfg["nr"] * cfg["ntheta"]
    out = {"metric": "adjoint gradient of the cycle-averaged electron number", "workload": "adjoint_nx64_nr32_nt16",
           "steps": steps, "checkpoint": 50, "J": J, "params": m.names(), "grad_adjoint": g.tolist(),
           "grad_central_difference": fd.tolist(), "max_rel_deviation": float(rel.max()),
           "normwise_deviation": normwise,
           "forward_s": t1 - t0, "adjoint_s": t2 - t1,
           "forward_dof_updates_per_s": dof * steps / (t1 - t0), "dtype": "f64", "data": "synthetic"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def measure_peaks():
    """Library GEMM throughput on this GPU (cuBLAS via torch.matmul, 8192^3, best of several): the
    denominators for FP64 and TF32 work that MEASURED_PEAKS.json does not carry."""
    import torch
    out = {}
    for name, dt, tf32, it in (("fp64", torch.float64, False, 3), ("fp32_simt", torch.float32, False, 5),
                               ("tf32", torch.float32, True, 10), ("bf16", torch.bfloat16, False, 10)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(8192, 8192, device="cuda", dtype=dt)
        b = torch.randn(8192, 8192, device="cuda", dtype=dt)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(it):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name + "_tflops"] = 2 * 8192**3 / best / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-structured", action="store_true", help="skip the block-tridiagonal solve legs")
    ap.add_argument("--no-cycle", action="store_true",
                    help="skip the accuracy leg over the configured run (mixed against FP64)")
    ap.add_argument("--peaks", action="store_true", help="only measure library GEMM peaks (FP64, FP32, TF32, BF16)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, LARGEST, "batched64_uneven", "adjoint_nx64_nr32_nt16", HYBRID, HYBRID_TABLE],
                    help="the headline single discharge (default), the largest single discharge (Nv = 4096; "
                         "use a few steps: its FP64 leg takes seconds per step), the 64 uneven discharges "
                         "in one graph, the adjoint-gradient check, the self-consistent parts on the medium grid, "
                         "or the paper's semi- vs fully-implicit table rows")
    ap.add_argument("--adjoint-steps", type=int, default=0, help="adjoint workload: steps (0 = one RF cycle)")
    ap.add_argument("--batched-fp64", action="store_true", help="batched workload: also time the FP64 batch")
    ap.add_argument("--panel-tc", action="store_true",
                    help="mixed path: the panel's left-looking updates on the tensor cores (BTE_FLAG_PANEL_TC)")
    ap.add_argument("--nx", type=int, default=0,
                    help="profiling only: run the default workload with this many x points instead of 128")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.peaks:
        return measure_peaks()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched64_uneven":
        return run_batched(args, rank, world)
    if args.workload == "adjoint_nx64_nr32_nt16":
        return run_adjoint(args, rank, world)
    if args.workload == HYBRID:
        return run_hybrid(args, rank, world)
    if args.workload == HYBRID_TABLE:
        return run_hybrid_table(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
