// The handle behind the C ABI (opaque to callers): operators, device buffers and state. Shared by
// the translation units that implement entry points (bte_api.cu, bte_adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "bte_internal.h"

struct bte_handle {
  bte_config cfg{};
  bte::HostOps ops;
  std::string err;
  bool host_only = false;
  cudaStream_t st = nullptr;
  int precision = BTE_FP64;
  int nb = 64;            // outer LU panel width
  double tol = 0.0;
  int refine_max = 0;
  bool structured = false;  // block-tridiagonal velocity solve instead of the dense LU
  void* xs = nullptr;       // its per-point scratch (nx * nl * nr * nr values)
  double* xs64 = nullptr;   // mixed path: FP64 scratch of the structured solve that takes over points
                            // whose refinement with the FP32 factors stalls (nx * nl * nr * nr)
  bool reduced = false;     // dense LU of I - dt B_i (order nl * nr) instead of A_i (order nv)
  int nlu = 0;              // order of the per-point factorisation (nv, or nl * nr when reduced)
  double *yred = nullptr, *zred = nullptr;  // P_S f and the reduced solution (nx * nlu each)
  bool use_tc = false;    // tcgen05 trailing update (FP32 storage only)
  bool have_tc = false;   // the tensor-core workspace exists (use_tc may be switched on)
  int panel_w = 0;        // preferred column-block width of the panel kernel (0: by shape)
  bool tc_pair = true;    // tensor-core updates two panels at a time (K = 256)
  int tc_probe = 0;      // BTE_FLAG_DIAG_TC_TIMEOUT: tensor-core launches expire a wait first
  int tc_cg = 2;          // pair update on CTA pairs (2) or single CTAs (1)
  bool panel_tc = false;  // the panel's left-looking updates on the tensor cores
  size_t bytes = 0;
  std::vector<void*> allocs;

  // x-step operators
  double *U = nullptr, *Uinv = nullptr, *Q = nullptr;
  // velocity operators: KCg, KAg = P_O C P_S, P_O A_v P_S (Nv x Nv, before the mass scaling; the
  // dense form only), Cs, Alo, Aup the mass-scaled harmonic blocks (residual, structured solve),
  // Cg, Aglo, Agup the same blocks before the mass scaling (reduced form only), Mband the band of M
  double *KCg = nullptr, *KAg = nullptr, *Cs = nullptr, *Alo = nullptr, *Aup = nullptr;
  double *Cg = nullptr, *Aglo = nullptr, *Agup = nullptr, *Mband = nullptr;
  // the refinement residual's banded operators (bte::ResidualOps)
  double *rc0 = nullptr, *rband = nullptr, *rfband = nullptr, *rchol = nullptr, *rcinv = nullptr;
  double *TO = nullptr, *TS = nullptr;
  double *mom_n = nullptr, *mom_e = nullptr, *mom_r = nullptr;
  // work
  double *Y = nullptr, *Y2 = nullptr, *Fa = nullptr, *Fb = nullptr, *Fw = nullptr, *R = nullptr;
  double *Fhost_dev = nullptr, *coef = nullptr, *ratio = nullptr;
  void* fac = nullptr;
  void* linv = nullptr;
  void* uinv = nullptr;
  void* tcws = nullptr;
  int *piv = nullptr, *perm = nullptr, *conv = nullptr;
  unsigned* status = nullptr;
  unsigned* status_host = nullptr;  // pinned
  std::vector<bte::Process> procs;  // the cross sections of the last bte_set_cross_sections
  // transposed x-step operators for the adjoint (allocated on its first use)
  double *Ut = nullptr, *Uinvt = nullptr, *Qt = nullptr;
  // self-consistent field, ions and the fully-implicit step (allocated on their first use)
  bool hybrid = false;
  double n0_mu_i = 4.65e21, n0_D_i = 2.07e20;   // n0 times ion mobility and diffusion
  double *Lop = nullptr, *E1 = nullptr, *Dxd = nullptr, *mud = nullptr, *lamd = nullptr, *rion = nullptr;
  double *Esc = nullptr, *Ek = nullptr, *ned = nullptr, *ionA = nullptr, *ionb = nullptr;
  int gm = 0;                                   // GMRES basis size allocated
  double *Fk = nullptr, *Fn = nullptr, *Rv = nullptr, *Zx = nullptr, *VX = nullptr, *KAF = nullptr;
  double *El = nullptr, *Wv = nullptr, *Pz = nullptr, *Vb = nullptr, *part = nullptr, *dsum = nullptr;
  double* Zb = nullptr;                         // preconditioned basis Z_j = P^-1 V_j (flexible GMRES)
  double *Dl = nullptr, *Qfull = nullptr;       // Newton direction; full-step Q_ij of the preconditioner
  double* dsum_host = nullptr;                  // pinned
  int last_sweeps = 0;
  double last_evals = 0.0;   // residual evaluations per point and step of the last run
  double last_resid = 0.0;
  unsigned last_flags = 0;
  unsigned long long launches = 0;
  // bte_run's CUDA graph of one step: the field of each step comes from run_seq[*run_idx] (the
  // uniform fields of the call, uploaded from the host) through run_E; captured for the state
  // pointer run_F, dropped when the operators or the variant change
  cudaGraph_t run_graph = nullptr;
  cudaGraphExec_t run_exec = nullptr;
  double* run_F = nullptr;
  double* run_E = nullptr;
  double* run_seq = nullptr;   // run_cap doubles, owned apart from allocs (it grows)
  int run_cap = 0;
  int* run_idx = nullptr;
  unsigned long long run_launches = 0;   // kernels per replayed step
  cudaStream_t cap_st = nullptr;         // private stream the step is captured on (non-blocking)
  // profiling: events around every launch while enabled
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

