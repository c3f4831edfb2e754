// C ABI of libbte (declared in include/bte.h): handle life cycle, device buffers and the
// per-step launch sequence of the semi-implicit scheme (eqs. "bte_semi_implicit", arXiv 2502.16555).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bte_handle.h"
#include "bte_kernels.h"

using bte::HostOps;


namespace {

std::string g_create_error;

bte_status fail(bte_handle* h, bte_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return s;
}

bte_status cuda_fail(bte_handle* h, cudaError_t e, const char* what) {
  return fail(h, BTE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BTE_CUDA(h, call)                                       \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
  } while (0)

#define BTE_TRY(x)               \
  do {                           \
    const bte_status r_ = (x);   \
    if (r_ != BTE_OK) return r_; \
  } while (0)

template <typename T>
bte_status dalloc(bte_handle* h, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return fail(h, BTE_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  h->allocs.push_back(q);
  h->bytes += bytes;
  *p = static_cast<T*>(q);
  return BTE_OK;
}

template <typename T>
bte_status upload(bte_handle* h, T* dst, const std::vector<T>& src) {
  if (src.empty()) return BTE_OK;
  BTE_CUDA(h, cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->st));
  return BTE_OK;
}

// the first n elements of a host array (n > 0)
template <typename T>
bte_status upload_n(bte_handle* h, T* dst, const T* src, size_t n) {
  BTE_CUDA(h, cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, h->st));
  return BTE_OK;
}

cudaEvent_t next_event(bte_handle* h) {
  if (h->pool_used == h->pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->pool.push_back(e);
  }
  return h->pool[h->pool_used++];
}

// Brackets one launch: counts it and, while profiling, records events around it.
struct Launch {
  bte_handle* h;
  int kind;
  cudaEvent_t a = nullptr;
  Launch(bte_handle* h_, int k) : h(h_), kind(k) {
    ++h->launches;
    if (h->prof) {
      a = next_event(h);
      cudaEventRecord(a, h->st);
    }
  }
  ~Launch() {
    if (h->prof) {
      cudaEvent_t b = next_event(h);
      cudaEventRecord(b, h->st);
      h->recs.push_back({kind, a, b});
    }
  }
};
// A launch whose configuration the runtime rejects (grid, block, shared memory, cluster shape)
// fails the call at once, naming the launcher; execution errors surface at the next sync.
bte_status launch_fail(bte_handle* h, cudaError_t e, const char* what) {
  cudaGetLastError();
  std::string w(what);
  const size_t paren = w.find('(');
  return fail(h, BTE_ECUDA, "launch rejected in " + w.substr(0, paren) + ": " + cudaGetErrorString(e));
}
#define BTE_LAUNCH(kind, call)                                    \
  do {                                                            \
    {                                                             \
      Launch l_(h, kind);                                         \
      call;                                                       \
    }                                                             \
    const cudaError_t le_ = cudaPeekAtLastError();                \
    if (le_ != cudaSuccess) return launch_fail(h, le_, #call);    \
  } while (0)

bte_status device_status(bte_handle* h) {
  if (h->host_only) return fail(h, BTE_ESTATE, "handle was created with BTE_FLAG_HOST_ONLY");
  if (!h->ops.have_v) return fail(h, BTE_ESTATE, "bte_set_cross_sections has not been called");
  // a launch error left behind by earlier work in the process (ours or the caller's) is reported
  // here, not against the first launch of this call
  const cudaError_t pend = cudaGetLastError();
  if (pend != cudaSuccess)
    return fail(h, BTE_ECUDA, std::string("a CUDA error was pending before this call: ") + cudaGetErrorString(pend));
  return BTE_OK;
}

// out_i (+)= A_i^-1 in_i through the factors of the last factoring call (dense paths), at the
// points with conv[i] == 0 (conv NULL: every point). The factors are those of (I (x) M_v) A_i, so
// every solve multiplies its right-hand side by I (x) M_v first. With the reduced system
// (nl < ntheta) they are those of (I (x) M_v) G_i, G_i = I - dt B_i, and
// A_i^-1 f = f + P_O (G_i^-1 - I) P_S f (Section 3.3).
bte_status enqueue_lu_solve(bte_handle* h, const double* in, double* out, const int* conv, int accumulate) {
  const HostOps& o = h->ops;
  const int nx = o.nx, n = h->nlu, nb = h->nb;
  const bte::MassBand mass{h->Mband, o.nr, o.mw};
  cudaStream_t st = h->st;
  const double* src = in;
  double* dst = out;
  int acc = accumulate;
  if (h->reduced) {
    BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_reduce_project(in, h->TS, h->yred, conv, nx, o.nt, o.nr, o.nl, st));
    src = h->yred;
    dst = h->zred;
    acc = 0;
  }
  if (h->precision == BTE_FP64)
    BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_lu_solve<double>(static_cast<double*>(h->fac), h->piv, src, dst, nx, n, nb,
                                                            conv, acc, st, mass));
  else
    BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_lu_solve_blocked<float>(static_cast<float*>(h->fac), h->perm,
                                                                   static_cast<float*>(h->linv),
                                                                   static_cast<float*>(h->uinv), src, dst, nx, n, nb,
                                                                   conv, acc, st, mass));
  if (h->reduced)
    BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_reduce_lift(in, h->yred, h->zred, h->TO, out, conv, accumulate, nx, o.nt,
                                                       o.nr, o.nl, st));
  return BTE_OK;
}

// The per-point matrices the dense paths factor: (I (x) M_v) A_i = I (x) M_v - dt (P_O C P_S +
// E_i P_O A_v P_S), or (I (x) M_v) G_i (order nl * nr) for the reduced system. Multiplying by the
// block-diagonal mass matrix leaves the solution unchanged; LU with partial pivoting on the
// mass-scaled A_i meets element growth of order 1e15 on speed grids of a few hundred B-splines at
// fields where dt e E / (m_e dv) is near 0.8, on this form it stays of order 1.
template <typename T>
void form_v(bte_handle* h, const double* E_dev, double Eu, T* fac) {
  const HostOps& o = h->ops;
  const bte::MassBand mass{h->Mband, o.nr, o.mw};
  if (h->reduced)
    bte::launch_v_form_reduced<T>(h->Cg, h->Aglo, h->Agup, mass, E_dev, Eu, o.dt, fac, o.nx, o.nr, o.nl, h->st);
  else
    bte::launch_v_form<T>(h->KCg, h->KAg, mass, E_dev, Eu, o.dt, fac, o.nx, o.nv, h->st);
}

// Velocity step (eq. "bte_semi_implicit_vspace" / "vspace_batched_system"): out_i = A_i^-1 in_i at
// every point, A_i = I - dt (K_C + E_i K_A) with E_i = E_dev[i] (or Eu when E_dev is NULL). With
// factor the per-point matrices are formed and factored first; without it the factors of the last
// factoring call are reused (dense path; the structured solve has no factors and always runs).
bte_status enqueue_vsolve(bte_handle* h, const double* in, double* out, const double* E_dev, double Eu,
                          bool factor) {
  const HostOps& o = h->ops;
  const int nx = o.nx, nt = o.nt, nr = o.nr, nl = o.nl;
  cudaStream_t st = h->st;
  const int n = h->nlu, nb = h->nb;
  if (h->structured) {
    if (h->precision == BTE_FP64)
      BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_vsolve_struct<double>(in, out, E_dev, Eu, o.dt, h->Cs, h->Alo, h->Aup,
                                                                   h->TO, h->TS, static_cast<double*>(h->xs), nx, nt,
                                                                   nr, nl, nullptr, 0, h->status, st));
    else
      BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_vsolve_struct<float>(in, out, E_dev, Eu, o.dt, h->Cs, h->Alo, h->Aup,
                                                                  h->TO, h->TS, static_cast<float*>(h->xs), nx, nt,
                                                                  nr, nl, nullptr, 0, h->status, st));
  } else if (h->precision == BTE_FP64) {
    double* fac = static_cast<double*>(h->fac);
    if (factor) {
      BTE_LAUNCH(BTE_K_V_FORM, form_v<double>(h, E_dev, Eu, fac));
      for (int k0 = 0; k0 < n; k0 += nb) {
        const int kb = std::min(nb, n - k0);
        BTE_LAUNCH(BTE_K_LU_PANEL, bte::launch_lu_panel<double>(fac, h->piv, h->perm, static_cast<double*>(h->linv), nullptr,
                                                                nx, n, k0, kb, nb, h->status, nullptr, nullptr,
                                                                nullptr, nullptr, h->panel_w, st));
        if (k0 + kb < n) {
          BTE_LAUNCH(BTE_K_LU_SWAP_TRSM, bte::launch_lu_swap_trsm<double>(fac, h->perm, static_cast<double*>(h->linv), nx,
                                                                          n, k0, kb, nb, nullptr, nullptr, st));
          BTE_LAUNCH(BTE_K_LU_GEMM, bte::launch_lu_gemm_simt<double>(fac, nx, n, k0, kb, st));
        }
      }
    }
  } else {
    float* fac = static_cast<float*>(h->fac);
    const bool fused_uinv = bte::lu_panel_fuses_uinv<float>(n, nb, h->panel_w);
    float* linv = static_cast<float*>(h->linv);
    float* uinv = fused_uinv ? static_cast<float*>(h->uinv) : nullptr;
    if (factor) {
      BTE_LAUNCH(BTE_K_V_FORM, form_v<float>(h, E_dev, Eu, fac));
      if (h->use_tc) {
        // workspace parts (tc_ws_part): 0-1 L21 split, 2-3 (P A12)^T split, 4-5 one panel's inv(L11)
        // split, 8-9 the two-panel block's inv(L11) split (6-7, U12^T, stay inside the tc_lu_* calls)
        float* ws[10];
        for (int p = 0; p < 10; ++p) ws[p] = bte::tc_ws_part(h->tcws, nx, n, p);
        const int ks = bte::kTcKs;
        auto panel = [&](int k0, int kb) {
          // the L21 split for the tensor cores is written by lu_swap_pack
          BTE_LAUNCH(BTE_K_LU_PANEL, bte::launch_lu_panel<float>(fac, h->piv, h->perm, linv, uinv, nx, n, k0, kb, nb,
                                                                 h->status, nullptr, nullptr, ws[4], ws[5],
                                                                 h->panel_w, st, h->panel_tc));
          return BTE_OK;
        };
        // the panel at k0 applied to the next ncols columns (U12, then A22 -= L21 U12)
        auto single = [&](int k0, int ncols) {
          BTE_LAUNCH(BTE_K_LU_SWAP_TRSM, bte::launch_lu_swap_pack(fac, h->perm, nx, n, k0, nb, nb, ncols, ks, ws[2],
                                                                  ws[3], ws[0], ws[1], st));
          BTE_LAUNCH(BTE_K_LU_SWAP_TRSM, bte::tc_lu_u12(fac, nx, n, k0, ncols, h->tcws, h->status, st, h->tc_probe));
          BTE_LAUNCH(BTE_K_LU_GEMM, bte::tc_lu_gemm(fac, nx, n, k0, ncols, h->tcws, h->status, st, h->tc_probe));
          return BTE_OK;
        };
        if (!h->tc_pair) {
          for (int k0 = 0; k0 < n; k0 += nb) {
            const int kb = std::min(nb, n - k0);
            BTE_TRY(panel(k0, kb));
            if (k0 + kb < n) BTE_TRY(single(k0, n - k0 - kb));
          }
        } else {
          // panels in pairs: the first panel updates only the second panel's columns; once the
          // second panel is factored, both update the rest together (K = 256), which reads and
          // writes the trailing matrix once per pair instead of once per panel
          for (int k0 = 0; k0 < n; k0 += 2 * nb) {
            const int kb1 = std::min(nb, n - k0);
            BTE_TRY(panel(k0, kb1));
            if (k0 + kb1 == n) break;
            const int kb2 = std::min(nb, n - k0 - nb);
            BTE_TRY(single(k0, kb2));
            BTE_TRY(panel(k0 + nb, kb2));
            if (k0 + nb + kb2 == n) break;
            BTE_LAUNCH(BTE_K_LU_SWAP_TRSM, bte::launch_lu_pair_linv(fac, h->perm, linv, nx, n, k0, ws[8], ws[9], st));
            BTE_LAUNCH(BTE_K_LU_SWAP_TRSM, bte::launch_lu_swap_pack_pair(fac, h->perm, nx, n, k0, ks, ws[2], ws[3],
                                                                         ws[0], ws[1], st));
            BTE_LAUNCH(BTE_K_LU_SWAP_TRSM, bte::tc_lu_u12_pair(fac, nx, n, k0, h->tcws, h->status, st, h->tc_probe));
            BTE_LAUNCH(BTE_K_LU_GEMM, bte::tc_lu_gemm_pair(fac, nx, n, k0, h->tcws, h->status, st, h->tc_probe, h->tc_cg));
          }
        }
      } else {
        for (int k0 = 0; k0 < n; k0 += nb) {
          const int kb = std::min(nb, n - k0);
          BTE_LAUNCH(BTE_K_LU_PANEL, bte::launch_lu_panel<float>(fac, h->piv, h->perm, linv, uinv, nx, n, k0, kb, nb,
                                                                 h->status, nullptr, nullptr, nullptr, nullptr,
                                                                 h->panel_w, st));
          if (k0 + kb < n) {
            BTE_LAUNCH(BTE_K_LU_SWAP_TRSM, bte::launch_lu_swap_trsm<float>(fac, h->perm, linv, nx, n, k0, kb, nb,
                                                                           nullptr, nullptr, st));
            BTE_LAUNCH(BTE_K_LU_GEMM, bte::launch_lu_gemm_simt<float>(fac, nx, n, k0, kb, st));
          }
        }
      }
      if (!fused_uinv)
        BTE_LAUNCH(BTE_K_LU_PANEL, bte::launch_lu_uinv<float>(fac, static_cast<float*>(h->uinv), nx, n, nb, st));
    }
  }
  if (!h->structured) BTE_TRY(enqueue_lu_solve(h, in, out, nullptr, 0));
  return BTE_OK;
}

// Residual evaluations of the mixed path's FP64 escalation (the first follows the fresh FP64 solve,
// each later one a correction through it).
constexpr int kEscalationSweeps = 3;

// One semi-implicit step of F_in into F_out (F_out is written only if the status word stays 0).
bte_status enqueue_step(bte_handle* h, const double* F_in, double* F_out, const double* E_dev,
                        double t, double V0, double freq, const double* ni_dev = nullptr) {
  const HostOps& o = h->ops;
  const int nx = o.nx, nt = o.nt, nr = o.nr, nv = o.nv, nl = o.nl;
  const double Eu = V0 / o.L * std::sin(2.0 * bte::kPi * freq * (t + 0.5 * o.dt));
  cudaStream_t st = h->st;
  // a non-finite field is an input error like a non-finite state (the uniform one is known here)
  if (!E_dev && !ni_dev && !std::isfinite(Eu)) return fail(h, BTE_ENONFINITE, "non-finite field (V0, freq_Hz or t_s)");
  // x half step #1 (eq. "bte_semi_implicit_xspace0")
  BTE_LAUNCH(BTE_K_X_TO_EIGEN, bte::launch_x_to_eigen(F_in, h->Uinv, h->Y, nx, nt, nr, h->status, st));
  BTE_LAUNCH(BTE_K_X_APPLY_Q, bte::launch_x_apply_q(h->Q, h->Y, h->Y2, nx, nt, nr, st));
  BTE_LAUNCH(BTE_K_X_FROM_EIGEN, bte::launch_x_from_eigen(h->Y2, h->U, h->Fa, nx, nt, nr, nullptr, st));
  // self-consistent field (eq. "bte_semi_implicit_efield"): E^{1/2} from the ions and the electrons
  // after the first x half step
  if (ni_dev) {
    const bte_status fs = bte::enqueue_field(h, h->Fa, ni_dev, t + 0.5 * o.dt, V0, freq, h->Esc);
    if (fs != BTE_OK) return fs;
    E_dev = h->Esc;
  }
  // velocity step (eq. "bte_semi_implicit_vspace" / "vspace_batched_system"); a caller's field
  // array is checked like the state
  if (E_dev && !ni_dev) BTE_LAUNCH(BTE_K_OTHER, bte::launch_check_field(E_dev, nx, h->status, st));
  {
    const bte_status vs = enqueue_vsolve(h, h->Fa, h->Fb, E_dev, Eu, true);
    if (vs != BTE_OK) return vs;
  }
  // FP64 iterative refinement: residual through Algorithm 2, correction through the factors
  if (h->refine_max > 0) {
    bte::ResidualOps ro;
    ro.c0 = h->rc0, ro.band = h->rband, ro.fband = h->rfband, ro.chol = h->rchol, ro.cinv = h->rcinv, ro.w = o.mw;
    BTE_CUDA(h, cudaMemsetAsync(h->conv, 0, sizeof(int) * nx, st));
    for (int s = 0; s <= h->refine_max; ++s) {
      BTE_LAUNCH(BTE_K_RESIDUAL, bte::launch_residual(h->Fb, h->Fa, E_dev, Eu, o.dt, ro, h->TO, h->TS, h->R, h->ratio,
                                                      h->conv, h->tol, o.kc_inf, o.ka_inf, nx, nt, nr, nl, h->status,
                                                      st));
      if (s == h->refine_max) break;
      if (h->structured && h->precision == BTE_FP64)
        BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_vsolve_struct<double>(h->R, h->Fb, E_dev, Eu, o.dt, h->Cs, h->Alo, h->Aup,
                                                                     h->TO, h->TS, static_cast<double*>(h->xs), nx,
                                                                     nt, nr, nl, h->conv, 1, nullptr, st));
      else if (h->structured)
        BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_vsolve_struct<float>(h->R, h->Fb, E_dev, Eu, o.dt, h->Cs, h->Alo, h->Aup,
                                                                    h->TO, h->TS, static_cast<float*>(h->xs), nx, nt,
                                                                    nr, nl, h->conv, 1, nullptr, st));
      else
        BTE_TRY(enqueue_lu_solve(h, h->R, h->Fb, h->conv, 1));
    }
    if (h->xs64) {
      // points whose refinement with the FP32 factors has not converged (cond(A_i) * eps_32 near or
      // above 1: strong fields) are solved again with the FP64 block-tridiagonal solve and refined
      // through it; converged points return at once from every launch here
      BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_vsolve_struct<double>(h->Fa, h->Fb, E_dev, Eu, o.dt, h->Cs, h->Alo, h->Aup,
                                                                   h->TO, h->TS, h->xs64, nx, nt, nr, nl, h->conv, 0,
                                                                   nullptr, st));
      for (int s = 0; s < kEscalationSweeps; ++s) {
        BTE_LAUNCH(BTE_K_RESIDUAL, bte::launch_residual(h->Fb, h->Fa, E_dev, Eu, o.dt, ro, h->TO, h->TS, h->R,
                                                        h->ratio, h->conv, h->tol, o.kc_inf, o.ka_inf, nx, nt, nr, nl,
                                                        h->status, st));
        if (s + 1 == kEscalationSweeps) break;
        BTE_LAUNCH(BTE_K_LU_SOLVE, bte::launch_vsolve_struct<double>(h->R, h->Fb, E_dev, Eu, o.dt, h->Cs, h->Alo,
                                                                     h->Aup, h->TO, h->TS, h->xs64, nx, nt, nr, nl,
                                                                     h->conv, 1, nullptr, st));
      }
    }
    BTE_LAUNCH(BTE_K_OTHER, bte::launch_check_conv(h->conv, nx, h->status, st));
  }
  // x half step #2 (eq. "bte_semi_implicit_xspace1"), then commit if nothing was flagged
  BTE_LAUNCH(BTE_K_X_TO_EIGEN, bte::launch_x_to_eigen(h->Fb, h->Uinv, h->Y, nx, nt, nr, nullptr, st));
  BTE_LAUNCH(BTE_K_X_APPLY_Q, bte::launch_x_apply_q(h->Q, h->Y, h->Y2, nx, nt, nr, st));
  BTE_LAUNCH(BTE_K_X_FROM_EIGEN, bte::launch_x_from_eigen(h->Y2, h->U, h->Fw, nx, nt, nr, h->status, st));
  BTE_LAUNCH(BTE_K_OTHER, bte::launch_commit(h->Fw, F_out, static_cast<size_t>(nx) * nv, h->status, st));
  BTE_CUDA(h, cudaGetLastError());
  return BTE_OK;
}

// bte_run's graph: the step's field from the call's sequence of uniform fields, and the counter
__global__ void run_field_kernel(const double* __restrict__ seq, const int* __restrict__ idx, double* __restrict__ E,
                                 int nx) {
  const double e = seq[*idx];
  for (int x = threadIdx.x; x < nx; x += blockDim.x) E[x] = e;
}
__global__ void run_advance_kernel(int* idx) { *idx += 1; }

void release_run_graph(bte_handle* h) {
  if (h->run_exec) cudaGraphExecDestroy(h->run_exec);
  if (h->run_graph) cudaGraphDestroy(h->run_graph);
  h->run_exec = nullptr;
  h->run_graph = nullptr;
  h->run_F = nullptr;
}

// The step graph applies unless bte_profile records (per-launch events) or the caller is capturing
// the handle's stream.
bte_status graph_allowed(bte_handle* h, bool& ok) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  BTE_CUDA(h, cudaStreamIsCapturing(h->st, &cs));
  ok = !h->prof && cs == cudaStreamCaptureStatusNone;
  return BTE_OK;
}

// n_steps > 0 steps of F_dev with the uniform sinusoidal field as replays of a CUDA graph of one
// step, captured for F_dev (again when F_dev, the cross sections or the variant change). The steps'
// fields are formed exactly as enqueue_step forms them and reach the step through the per-point
// field array, which gives the same factors and residuals: the result equals the steps launched
// one kernel at a time.
bte_status enqueue_graph_steps(bte_handle* h, double* F_dev, int n_steps, double t_s, double V0, double freq_Hz) {
  const HostOps& o = h->ops;
  std::vector<double> seq(n_steps);
  for (int i = 0; i < n_steps; ++i) {
    const double t = t_s + i * o.dt;
    seq[i] = V0 / o.L * std::sin(2.0 * bte::kPi * freq_Hz * (t + 0.5 * o.dt));
    if (!std::isfinite(seq[i])) return fail(h, BTE_ENONFINITE, "non-finite field (V0, freq_Hz or t_s)");
  }
  if (!h->run_E) BTE_TRY(dalloc(h, &h->run_E, o.nx));
  if (!h->run_idx) BTE_TRY(dalloc(h, &h->run_idx, 1));
  if (h->run_cap < n_steps) {
    release_run_graph(h);
    if (h->run_seq) cudaFree(h->run_seq);
    h->run_seq = nullptr;
    h->run_cap = 0;
    const int cap = std::max(n_steps, 256);
    BTE_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&h->run_seq), sizeof(double) * cap));
    h->run_cap = cap;
  }
  if (!h->run_exec || h->run_F != F_dev) {
    release_run_graph(h);
    // captured on a private stream (the caller's may be the legacy default stream, which cannot be
    // captured); the graph is then launched on the handle's own stream
    if (!h->cap_st) BTE_CUDA(h, cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    const unsigned long long before = h->launches;
    cudaStream_t own = h->st;
    // relaxed: a launcher's first use may set a kernel attribute or encode a tensor map
    BTE_CUDA(h, cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeRelaxed));
    h->st = h->cap_st;
    run_field_kernel<<<1, 256, 0, h->st>>>(h->run_seq, h->run_idx, h->run_E, o.nx);
    const bte_status s = enqueue_step(h, F_dev, F_dev, h->run_E, 0.0, 0.0, 0.0);
    run_advance_kernel<<<1, 1, 0, h->st>>>(h->run_idx);
    h->st = own;
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(h->cap_st, &g);
    h->run_launches = h->launches - before + 2;   // the step's kernels, the field and the counter
    h->launches = before;                         // captured, not launched: counted per replay
    if (s != BTE_OK || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();   // a failed capture must not leave an error behind for the caller
      if (s != BTE_OK) return s;
      return fail(h, BTE_ECUDA, std::string("capturing the step: ") + cudaGetErrorString(ee));
    }
    h->run_graph = g;
    const cudaError_t ie = cudaGraphInstantiate(&h->run_exec, g, 0);
    if (ie != cudaSuccess) {
      release_run_graph(h);
      return fail(h, BTE_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
    h->run_F = F_dev;
  }
  BTE_CUDA(h, cudaMemcpyAsync(h->run_seq, seq.data(), sizeof(double) * n_steps, cudaMemcpyHostToDevice, h->st));
  BTE_CUDA(h, cudaMemsetAsync(h->run_idx, 0, sizeof(int), h->st));
  for (int i = 0; i < n_steps; ++i) BTE_CUDA(h, cudaGraphLaunch(h->run_exec, h->st));
  h->launches += h->run_launches * static_cast<unsigned long long>(n_steps);
  return BTE_OK;
}

bte_status read_status(bte_handle* h, int steps = 1) {
  BTE_CUDA(h, cudaMemcpyAsync(h->status_host, h->status, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
  BTE_CUDA(h, cudaStreamSynchronize(h->st));
  const unsigned f = h->status_host[0];
  h->last_flags = f;
  // status word 1 counts the residual evaluations of all points and steps since the reset: per
  // point and step one more than the correction sweeps
  if (h->refine_max > 0 && steps > 0) {
    const double per = static_cast<double>(h->status_host[1]) / (static_cast<double>(h->ops.nx) * steps);
    h->last_evals = per;
    h->last_sweeps = static_cast<int>(std::ceil(per - 1.0 - 1e-9));
    if (h->last_sweeps < 0) h->last_sweeps = 0;
  } else {
    h->last_evals = 0.0;
    h->last_sweeps = 0;
  }
  if (h->refine_max > 0) {
    std::vector<double> r(h->ops.nx);
    std::vector<int> c(h->ops.nx);
    BTE_CUDA(h, cudaMemcpy(r.data(), h->ratio, sizeof(double) * r.size(), cudaMemcpyDeviceToHost));
    double m = 0;
    for (double v : r) m = std::max(m, v);
    h->last_resid = m;
  }
  // a non-finite input explains whatever follows from it; otherwise a failed factorisation explains
  // a non-finite result
  if (f & bte::kTimeout) return fail(h, BTE_ECUDA, "a bounded device-side wait expired in the tensor-core update");
  if (f & bte::kNonFiniteIn) return fail(h, BTE_ENONFINITE, "non-finite values in the state or field handed in");
  if (f & bte::kZeroPivot) return fail(h, BTE_ESINGULAR, "zero or non-finite pivot in a per-point factorisation");
  if (f & bte::kNonFinite) return fail(h, BTE_ENONFINITE, "non-finite values in the result of a step");
  if (f & bte::kNoConv) return fail(h, BTE_ENOCONV, "iterative refinement did not converge");
  return BTE_OK;
}

bool valid_cfg(const bte_config* c, std::string& why) {
  if (!c) return why = "cfg is NULL", false;
  if (c->nx < 3) return why = "nx must be >= 3", false;
  if (c->nr < 4) return why = "nr must be >= 4", false;
  if (c->ntheta < 2) return why = "ntheta must be >= 2", false;
  const int nl = c->nl > 0 ? c->nl : c->ntheta;
  if (nl < 1 || nl > c->ntheta) return why = "nl must satisfy 1 <= nl <= ntheta", false;
  if (!(c->L_m > 0) || !(c->vmax_eV > 0) || !(c->p_Torr > 0) || !(c->T0_K > 0) || !(c->m0_amu > 0) ||
      !(c->dt_s > 0))
    return why = "L_m, vmax_eV, p_Torr, T0_K, m0_amu and dt_s must be positive", false;
  if (c->precision != BTE_FP64 && c->precision != BTE_MIXED) return why = "unknown precision", false;
  // what the kernels' shared-memory plans hold (opt-in sizes): the eigen-basis transforms stage
  // nr x 33 doubles (nr <= 880); the FP64 panel of a tall first panel stages about 28 bytes per
  // row (nv <= 7936); the structured residual and operator applies stage nv + 2 nl nr <= 3 nv
  // doubles, within 220 KB under that bound
  const double nv = static_cast<double>(c->nr) * c->ntheta;
  if (c->nr > bte::kMaxNr) return why = "nr must be <= 880", false;
  if (nv > bte::kMaxNv || c->nx > 4096) return why = "grid too large (nr*ntheta <= 7936, nx <= 4096)", false;
  return true;
}

}  // namespace

namespace bte {
bte_status handle_enqueue_step(bte_handle* h, double* F_dev, const double* E_dev, double t, double V0, double freq,
                               cudaStream_t st) {
  BTE_TRY(device_status(h));
  cudaStream_t own = h->st;
  h->st = st;
  bte_status s = enqueue_step(h, F_dev, F_dev, E_dev, t, V0, freq);
  h->st = own;
  return s;
}
bte_status handle_enqueue_sc_step(bte_handle* h, double* F_dev, const double* ni_dev, double t, double V0,
                                  double freq) {
  return enqueue_step(h, F_dev, F_dev, nullptr, t, V0, freq, ni_dev);
}
bte_status handle_enqueue_xhalf(bte_handle* h, const double* in, double* out) {
  const HostOps& o = h->ops;
  cudaStream_t st = h->st;
  BTE_LAUNCH(BTE_K_X_TO_EIGEN, bte::launch_x_to_eigen(in, h->Uinv, h->Y, o.nx, o.nt, o.nr, nullptr, st));
  BTE_LAUNCH(BTE_K_X_APPLY_Q, bte::launch_x_apply_q(h->Q, h->Y, h->Y2, o.nx, o.nt, o.nr, st));
  BTE_LAUNCH(BTE_K_X_FROM_EIGEN, bte::launch_x_from_eigen(h->Y2, h->U, out, o.nx, o.nt, o.nr, h->status, st));
  BTE_CUDA(h, cudaGetLastError());
  return BTE_OK;
}
bte_status handle_enqueue_vsolve(bte_handle* h, const double* in, double* out, const double* E_dev, bool factor) {
  return enqueue_vsolve(h, in, out, E_dev, 0.0, factor);
}
bte_status handle_reset_status(bte_handle* h, cudaStream_t st) {
  BTE_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), st));
  return BTE_OK;
}
bte_status handle_read_status(bte_handle* h) { return read_status(h); }
bte_status handle_device_status(bte_handle* h) { return device_status(h); }
bool handle_profiling(const bte_handle* h) { return h->prof; }
unsigned long long handle_launches(const bte_handle* h) { return h->launches; }
void handle_add_launches(bte_handle* h, unsigned long long n) { h->launches += n; }
bool handle_has_tc(const bte_handle* h) { return h->have_tc; }
void handle_set_variant(bte_handle* h, const Variant& v) {
  release_run_graph(h);
  h->use_tc = v.tc && h->have_tc;
  h->panel_w = v.panel_w;
  h->tc_pair = v.pair;
  h->tc_cg = v.cg == 1 ? 1 : 2;
}
Variant handle_get_variant(const bte_handle* h) {
  Variant v;
  v.tc = h->use_tc;
  v.panel_w = h->panel_w;
  v.pair = h->tc_pair;
  v.cg = h->tc_cg;
  return v;
}
const HostOps* handle_ops(const bte_handle* h) { return &h->ops; }
void* handle_stream_ptr(const bte_handle* h) { return static_cast<void*>(h->st); }
bte_status handle_fail(const bte_handle* h, bte_status s, const std::string& msg) {
  return fail(const_cast<bte_handle*>(h), s, msg);
}
}  // namespace bte

extern "C" {

bte_status bte_create(const bte_config* cfg, bte_handle** out) {
  std::string why;
  if (!out) return fail(nullptr, BTE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!valid_cfg(cfg, why)) return fail(nullptr, BTE_EINVAL, why);
  bte_handle* h = new bte_handle();
  h->cfg = *cfg;
  h->host_only = (cfg->flags & BTE_FLAG_HOST_ONLY) != 0;
  h->st = static_cast<cudaStream_t>(cfg->stream);
  h->precision = cfg->precision;
  h->nb = cfg->precision == BTE_FP64 ? 64 : 128;
  h->structured = (cfg->flags & BTE_FLAG_STRUCTURED) != 0;
  h->tc_pair = (cfg->flags & BTE_FLAG_TC_SINGLE) == 0;
  h->tc_probe = (cfg->flags & BTE_FLAG_DIAG_TC_TIMEOUT) != 0 ? 1 : 0;
  h->tc_cg = (cfg->flags & BTE_FLAG_TC_ONE_CTA) != 0 ? 1 : 2;
  h->panel_tc = (cfg->flags & BTE_FLAG_PANEL_TC) != 0;
  {
    const int nl = cfg->nl > 0 ? cfg->nl : cfg->ntheta;
    h->reduced = !h->structured && nl < cfg->ntheta && (cfg->flags & BTE_FLAG_FULL_V) == 0;
    h->nlu = h->reduced ? nl * cfg->nr : cfg->nr * cfg->ntheta;
  }
  if (h->structured) {
    const int nl = cfg->nl > 0 ? cfg->nl : cfg->ntheta;
    const size_t ts = cfg->precision == BTE_FP64 ? 8 : 4;
    if (cfg->nr > 64 || bte::struct_smem_bytes(cfg->nr, nl, ts) > 200 * 1024) {
      delete h;
      return fail(nullptr, BTE_EINVAL, "BTE_FLAG_STRUCTURED needs nr <= 64");
    }
  }
  h->tol = cfg->refine_tol > 0 ? cfg->refine_tol : (cfg->precision == BTE_FP64 ? 1e-13 : 1e-12);
  h->refine_max = cfg->refine_max >= 0 ? cfg->refine_max : (cfg->precision == BTE_FP64 ? 2 : 4);
  std::string e = bte::assemble_x(*cfg, h->ops);
  // handles that factor the Nv x Nv form keep its unscaled operators
  h->ops.want_kg = !h->reduced && !h->structured;
  if (!e.empty()) {
    delete h;
    return fail(nullptr, BTE_EINVAL, e);
  }
  if (!h->host_only) {
    const HostOps& o = h->ops;
    const size_t D = static_cast<size_t>(o.nx) * o.nv;
    const size_t nn = static_cast<size_t>(h->nlu) * h->nlu;
    // the dense P_O C P_S, P_O A_v P_S (nv x nv) serve only the full-matrix form and the adjoint,
    // the unscaled harmonic blocks only the reduced form; both forms multiply by the band of M
    const bool dense_k = !h->reduced && !h->structured;
    const size_t blk = static_cast<size_t>(o.nl) * o.nr * o.nr;
    bte_status s;
    auto chk = [&](bte_status r) { s = r; return r == BTE_OK; };
    bool ok = chk(dalloc(h, &h->U, o.U.size())) && chk(dalloc(h, &h->Uinv, o.Uinv.size())) &&
              chk(dalloc(h, &h->Q, o.Q.size())) &&
              (!dense_k || (chk(dalloc(h, &h->KCg, static_cast<size_t>(o.nv) * o.nv)) &&
                            chk(dalloc(h, &h->KAg, static_cast<size_t>(o.nv) * o.nv)))) &&
              (!h->reduced || (chk(dalloc(h, &h->Cg, blk)) && chk(dalloc(h, &h->Aglo, blk)) &&
                               chk(dalloc(h, &h->Agup, blk)))) &&
              (h->structured || chk(dalloc(h, &h->Mband, o.Mband.size()))) &&
              chk(dalloc(h, &h->rc0, static_cast<size_t>(o.nr) * o.nr)) &&
              chk(dalloc(h, &h->rband, static_cast<size_t>(o.nr) * (2 * o.mw + 1))) &&
              chk(dalloc(h, &h->rfband, static_cast<size_t>(2) * o.nl * o.nr * (2 * o.mw + 1))) &&
              chk(dalloc(h, &h->rchol, static_cast<size_t>(o.nr) * (o.mw + 1))) && chk(dalloc(h, &h->rcinv, o.nr)) &&
              chk(dalloc(h, &h->Cs, static_cast<size_t>(o.nl) * o.nr * o.nr)) &&
              chk(dalloc(h, &h->Alo, static_cast<size_t>(o.nl) * o.nr * o.nr)) &&
              chk(dalloc(h, &h->Aup, static_cast<size_t>(o.nl) * o.nr * o.nr)) &&
              chk(dalloc(h, &h->TO, o.TO.size())) && chk(dalloc(h, &h->TS, o.TS.size())) &&
              chk(dalloc(h, &h->mom_n, o.nv)) && chk(dalloc(h, &h->mom_e, o.nv)) &&
              chk(dalloc(h, &h->Y, D)) && chk(dalloc(h, &h->Y2, D)) && chk(dalloc(h, &h->Fa, D)) &&
              chk(dalloc(h, &h->Fb, D)) && chk(dalloc(h, &h->Fw, D)) && chk(dalloc(h, &h->R, D)) &&
              chk(dalloc(h, &h->Fhost_dev, D)) && chk(dalloc(h, &h->coef, o.nr)) &&
              chk(dalloc(h, &h->ratio, o.nx)) && chk(dalloc(h, &h->piv, D)) &&
              chk(dalloc(h, &h->perm, static_cast<size_t>(o.nx) * ((h->nlu + h->nb - 1) / h->nb) *
                                          bte::perm_record_ints(h->nb))) &&
              chk(dalloc(h, &h->conv, o.nx)) && chk(dalloc(h, &h->status, 2));
    if (ok && h->structured) {
      const size_t xsz = static_cast<size_t>(o.nx) * o.nl * o.nr * o.nr;
      if (h->precision == BTE_FP64) {
        double* x = nullptr;
        ok = chk(dalloc(h, &x, xsz));
        h->xs = x;
      } else {
        float* x = nullptr;
        ok = chk(dalloc(h, &x, xsz));
        h->xs = x;
        if (ok && bte::struct_smem_bytes(o.nr, o.nl, sizeof(double)) <= 200 * 1024)
          ok = chk(dalloc(h, &h->xs64, xsz));
      }
    } else if (ok) {
      // the mixed path's escalation for ill-conditioned points: the FP64 block-tridiagonal solve
      if (h->precision == BTE_MIXED && o.nr <= 64 && bte::struct_smem_bytes(o.nr, o.nl, sizeof(double)) <= 200 * 1024)
        ok = chk(dalloc(h, &h->xs64, static_cast<size_t>(o.nx) * o.nl * o.nr * o.nr));
      if (h->reduced)
        ok = chk(dalloc(h, &h->yred, static_cast<size_t>(o.nx) * h->nlu)) &&
             chk(dalloc(h, &h->zred, static_cast<size_t>(o.nx) * h->nlu));
      const size_t npan = (h->nlu + h->nb - 1) / h->nb;
      const size_t blk = static_cast<size_t>(o.nx) * npan * h->nb * h->nb;
      if (h->precision == BTE_FP64) {
        double *f = nullptr, *l = nullptr;
        ok = ok && chk(dalloc(h, &f, nn * o.nx)) && chk(dalloc(h, &l, blk));
        h->fac = f;
        h->linv = l;
      } else {
        float *f = nullptr, *l = nullptr, *u = nullptr;
        ok = ok && chk(dalloc(h, &f, nn * o.nx)) && chk(dalloc(h, &l, blk)) && chk(dalloc(h, &u, blk));
        h->fac = f;
        h->linv = l;
        h->uinv = u;
        if (ok && !(cfg->flags & BTE_FLAG_SIMT_GEMM) && bte::tc_workspace_bytes(o.nx, h->nlu, h->nb) > 0 &&
            bte::tc_available()) {
          unsigned char* w = nullptr;
          ok = chk(dalloc(h, &w, bte::tc_workspace_bytes(o.nx, h->nlu, h->nb)));
          h->tcws = w;
          h->use_tc = ok;
          h->have_tc = ok;
        }
      }
    }
    if (ok) {
      cudaError_t ce = cudaMallocHost(reinterpret_cast<void**>(&h->status_host), 2 * sizeof(unsigned));
      if (ce != cudaSuccess) ok = false, s = cuda_fail(h, ce, "cudaMallocHost");
    }
    if (ok) ok = chk(upload(h, h->U, o.U)) && chk(upload(h, h->Uinv, o.Uinv)) && chk(upload(h, h->Q, o.Q)) &&
                 chk(upload(h, h->TO, o.TO)) && chk(upload(h, h->TS, o.TS)) &&
                 (!h->Mband || chk(upload(h, h->Mband, o.Mband)));
    if (ok) {
      cudaError_t ce = cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), h->st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
      if (ce != cudaSuccess) ok = false, s = cuda_fail(h, ce, "initialising device buffers");
    }
    if (!ok) {
      g_create_error = h->err;
      bte_destroy(h);
      return s;
    }
  }
  *out = h;
  return BTE_OK;
}

bte_status bte_set_cross_sections(bte_handle* h, int n_proc, const bte_process* procs) {
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (n_proc < 0 || n_proc > 64 || (n_proc > 0 && !procs)) return fail(h, BTE_EINVAL, "bad process list");
  std::vector<bte::Process> ps;
  for (int j = 0; j < n_proc; ++j) {
    const bte_process& p = procs[j];
    if (p.kind < BTE_ELASTIC || p.kind > BTE_IONIZATION) return fail(h, BTE_EINVAL, "unknown process kind");
    if (p.form < BTE_SIGMA_CONST || p.form > BTE_SIGMA_NU) return fail(h, BTE_EINVAL, "unknown cross-section form");
    if (p.kind != BTE_ELASTIC && !(p.threshold_eV > 0))
      return fail(h, BTE_EINVAL, "inelastic processes need a positive threshold");
    if ((p.form == BTE_SIGMA_LINEAR || p.form == BTE_SIGMA_LOG) && !(p.threshold_eV > 0))
      return fail(h, BTE_EINVAL, "linear/log cross sections need a positive threshold");
    bte::Process q;
    q.kind = p.kind;
    q.form = p.form;
    q.th_eV = p.kind == BTE_ELASTIC && p.form != BTE_SIGMA_LINEAR && p.form != BTE_SIGMA_LOG ? 0.0 : p.threshold_eV;
    q.scale = p.scale;
    q.sigma0 = p.sigma0;
    if (p.form == BTE_SIGMA_TABLE) {
      if (p.n_tab < 2 || !p.eps_eV || !p.sigma_m2) return fail(h, BTE_EINVAL, "table needs n_tab >= 2 points");
      q.tab_eps.assign(p.eps_eV, p.eps_eV + p.n_tab);
      q.tab_sigma.assign(p.sigma_m2, p.sigma_m2 + p.n_tab);
      for (int i = 1; i < p.n_tab; ++i)
        if (!(q.tab_eps[i] > q.tab_eps[i - 1])) return fail(h, BTE_EINVAL, "table energies must ascend");
    }
    ps.push_back(q);
  }
  std::string e = bte::assemble_v(h->ops, ps);
  if (!e.empty()) return fail(h, BTE_EINVAL, e);
  // bte_run's graph holds the previous operators' norms as kernel arguments
  if (!h->host_only) release_run_graph(h);
  h->procs = ps;
  if (h->host_only) return BTE_OK;
  const HostOps& o = h->ops;
  if (h->mom_r) {
    cudaFree(h->mom_r);
    h->mom_r = nullptr;
  }
  if (o.n_proc > 0) {
    BTE_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&h->mom_r), sizeof(double) * o.mom_r.size()));
  }
  bte_status s;
  if ((h->KCg && (s = upload(h, h->KCg, o.KCg)) != BTE_OK) || (h->KAg && (s = upload(h, h->KAg, o.KAg)) != BTE_OK) ||
      (h->Cg && (s = upload(h, h->Cg, o.Cg)) != BTE_OK) || (h->Aglo && (s = upload(h, h->Aglo, o.Ag_lo)) != BTE_OK) ||
      (h->Agup && (s = upload(h, h->Agup, o.Ag_up)) != BTE_OK) ||
      (s = upload_n(h, h->rc0, o.Cg.data(), static_cast<size_t>(o.nr) * o.nr)) != BTE_OK ||
      (s = upload(h, h->rband, o.rband)) != BTE_OK ||
      (s = upload(h, h->rfband, o.rfband)) != BTE_OK ||
      (s = upload(h, h->rchol, o.rchol)) != BTE_OK || (s = upload(h, h->rcinv, o.rcinv)) != BTE_OK ||
      (s = upload(h, h->Cs, o.Cs)) != BTE_OK || (s = upload(h, h->Alo, o.As_lo)) != BTE_OK ||
      (s = upload(h, h->Aup, o.As_up)) != BTE_OK || (s = upload(h, h->mom_n, o.mom_n)) != BTE_OK ||
      (s = upload(h, h->mom_e, o.mom_e)) != BTE_OK || (o.n_proc > 0 && (s = upload(h, h->mom_r, o.mom_r)) != BTE_OK))
    return s;
  BTE_CUDA(h, cudaStreamSynchronize(h->st));
  return BTE_OK;
}

bte_status bte_init_maxwellian(bte_handle* h, double* F_dev, const double* ne_dev, double Te_eV) {
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev || !ne_dev || !(Te_eV > 0)) return fail(h, BTE_EINVAL, "bad arguments");
  if (h->host_only) return fail(h, BTE_ESTATE, "handle was created with BTE_FLAG_HOST_ONLY");
  std::vector<double> c = bte::maxwellian_coeffs(h->ops, Te_eV);
  bte_status s = upload(h, h->coef, c);
  if (s != BTE_OK) return s;
  bte::launch_fill_maxwellian(F_dev, ne_dev, h->coef, h->ops.nx, h->ops.nt, h->ops.nr, h->st);
  BTE_CUDA(h, cudaGetLastError());
  BTE_CUDA(h, cudaStreamSynchronize(h->st));  // keeps the host coefficient vector alive until copied
  return BTE_OK;
}

bte_status bte_step(bte_handle* h, double* F_dev, const double* E_dev, double t_s, double V0,
                    double freq_Hz) {
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev) return fail(h, BTE_EINVAL, "F_dev is NULL");
  BTE_TRY(device_status(h));
  bool graph = false;
  BTE_TRY(graph_allowed(h, graph));
  BTE_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), h->st));
  if (graph && !E_dev)
    BTE_TRY(enqueue_graph_steps(h, F_dev, 1, t_s, V0, freq_Hz));
  else
    BTE_TRY(enqueue_step(h, F_dev, F_dev, E_dev, t_s, V0, freq_Hz));
  return read_status(h);
}

bte_status bte_run(bte_handle* h, double* F_dev, int n_steps, double t_s, double V0, double freq_Hz) {
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev || n_steps < 0) return fail(h, BTE_EINVAL, "bad arguments");
  BTE_TRY(device_status(h));
  bool graph = false;
  BTE_TRY(graph_allowed(h, graph));
  BTE_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), h->st));
  if (graph && n_steps > 0) {
    BTE_TRY(enqueue_graph_steps(h, F_dev, n_steps, t_s, V0, freq_Hz));
  } else {
    for (int i = 0; i < n_steps; ++i) BTE_TRY(enqueue_step(h, F_dev, F_dev, nullptr, t_s + i * h->ops.dt, V0, freq_Hz));
  }
  return read_status(h, n_steps);
}

bte_status bte_step_host(bte_handle* h, double* F_host, double t_s, double V0, double freq_Hz) {
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_host) return fail(h, BTE_EINVAL, "F_host is NULL");
  BTE_TRY(device_status(h));
  bool graph = false;
  BTE_TRY(graph_allowed(h, graph));
  const size_t bytes = sizeof(double) * h->ops.nx * h->ops.nv;
  BTE_CUDA(h, cudaMemcpyAsync(h->Fhost_dev, F_host, bytes, cudaMemcpyHostToDevice, h->st));
  BTE_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), h->st));
  if (graph)
    BTE_TRY(enqueue_graph_steps(h, h->Fhost_dev, 1, t_s, V0, freq_Hz));
  else
    BTE_TRY(enqueue_step(h, h->Fhost_dev, h->Fhost_dev, nullptr, t_s, V0, freq_Hz));
  BTE_CUDA(h, cudaMemcpyAsync(F_host, h->Fhost_dev, bytes, cudaMemcpyDeviceToHost, h->st));
  return read_status(h);
}

bte_status bte_moments(bte_handle* h, const double* F_dev, double* ne_dev, double* mean_eV_dev,
                       double* rates_dev) {
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev) return fail(h, BTE_EINVAL, "F_dev is NULL");
  BTE_TRY(device_status(h));
  bte::launch_moments(F_dev, h->mom_n, h->mom_e, h->mom_r, rates_dev ? h->ops.n_proc : 0, ne_dev,
                      mean_eV_dev, rates_dev, h->ops.nx, h->ops.nv, h->st);
  BTE_CUDA(h, cudaGetLastError());
  return BTE_OK;
}

bte_status bte_get_operator(const bte_handle* hc, int which, double* out, size_t count) {
  bte_handle* h = const_cast<bte_handle*>(hc);
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!out) return fail(h, BTE_EINVAL, "output is NULL");
  const HostOps& o = h->ops;
  const std::vector<double>* v = nullptr;
  switch (which) {
    case 0: v = &o.x; break;
    case 1: v = &o.Dx; break;
    case 2: v = &o.mu; break;
    case 3: v = &o.KC; break;
    case 4: v = &o.KA; break;
    case 5: v = &o.lam; break;
    case 6: v = &o.U; break;
    case 7: v = &o.Uinv; break;
    case 8: v = &o.Q; break;
    case 9: v = &o.M; break;
    case 10: v = &o.mom_n; break;
    case 11: v = &o.mom_e; break;
    case 12: v = &o.mom_r; break;
    case 13: v = &o.ccw; break;
    case 14: v = &o.KCg; break;
    case 15: v = &o.KAg; break;
    default: return fail(h, BTE_EINVAL, "unknown operator id");
  }
  const bool needs_v = which == 3 || which == 4 || (which >= 10 && which <= 12) || which >= 14;
  if (needs_v && !o.have_v)
    return fail(h, BTE_ESTATE, "velocity operators not assembled yet");
  if (which >= 14 && v->empty())
    return fail(h, BTE_ESTATE, "this handle does not factor the Nv x Nv form (reduced or structured)");
  if (v->size() != count) return fail(h, BTE_EINVAL, "count does not match the operator size");
  std::memcpy(out, v->data(), count * sizeof(double));
  return BTE_OK;
}

bte_status bte_get_info(const bte_handle* hc, bte_info* info) {
  if (!hc || !info) return fail(nullptr, BTE_EINVAL, "NULL argument");
  const HostOps& o = hc->ops;
  info->nx = o.nx;
  info->nr = o.nr;
  info->ntheta = o.nt;
  info->nl = o.nl;
  info->nv = o.nv;
  info->n_proc = o.n_proc;
  info->precision = hc->precision;
  info->n0_m3 = o.n0;
  info->vmax_ms = o.vmax;
  info->device_bytes = hc->bytes;
  info->last_refine_sweeps = hc->last_sweeps;
  info->last_residual = hc->last_resid;
  info->last_flags = hc->last_flags;
  info->launches = hc->launches;
  info->tensor_cores = hc->use_tc ? 1 : 0;
  info->solve_n = hc->structured ? 0 : hc->nlu;
  info->last_refine_evals = hc->last_evals;
  return BTE_OK;
}

bte_status bte_profile(bte_handle* h, int enable, double* ms_out, unsigned long long* count_out) {
  if (!h) return fail(nullptr, BTE_EINVAL, "handle is NULL");
  if (h->host_only) return fail(h, BTE_ESTATE, "handle was created with BTE_FLAG_HOST_ONLY");
  if (enable) {
    h->recs.clear();
    h->pool_used = 0;
    h->prof = true;
    return BTE_OK;
  }
  h->prof = false;
  BTE_CUDA(h, cudaStreamSynchronize(h->st));
  double ms[BTE_NPROF] = {0};
  unsigned long long cnt[BTE_NPROF] = {0};
  for (const auto& r : h->recs) {
    float t = 0.f;
    BTE_CUDA(h, cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.kind] += t;
    cnt[r.kind] += 1;
  }
  h->recs.clear();
  h->pool_used = 0;
  for (int k = 0; k < BTE_NPROF; ++k) {
    if (ms_out) ms_out[k] = ms[k];
    if (count_out) count_out[k] = cnt[k];
  }
  return BTE_OK;
}

bte_status bte_destroy(bte_handle* h) {
  if (!h) return BTE_OK;
  if (!h->host_only) {
    cudaStreamSynchronize(h->st);
    release_run_graph(h);
    if (h->run_seq) cudaFree(h->run_seq);
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
    for (void* p : h->allocs) cudaFree(p);
    if (h->mom_r) cudaFree(h->mom_r);
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->dsum_host) cudaFreeHost(h->dsum_host);
  }
  delete h;
  return BTE_OK;
}

const char* bte_last_error(const bte_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
