// Adjoint of the semi-implicit step (declared in include/bte.h: bte_step_adjoint,
// bte_adjoint_gradient). With a specified field the step of eqs. "bte_semi_implicit"
// (arXiv 2502.16555, Section 3.4) is linear in F: F^{n+1} = S_n F^n with S_n = X V_n X, X the x half
// step (Algorithm 1) and V_n the per-point solves with A_i = I - dt (K_C + E_i K_A). Its transpose is
// S_n^T = X^T V_n^T X^T: X^T applies U^T, the transposed Q_ij blocks and U^-T in place of U^-1, Q_ij
// and U; V_n^T solves with A_i^T through the same LU factors. The factors are those of
// (I (x) M_v) A_i, so A_i^-1 g = LU^-1 (I (x) M_v) g and A_i^-T g = (I (x) M_v) LU^-T g (M_v is
// symmetric). A parameter theta enters only through
// A_i, and d(A^-1 G)/dtheta = -A^-1 (dA/dtheta) F*, so a step contributes
//     dJ/dtheta += mu^T (dt dK/dtheta) F*,   mu = A^-T X^T lambda^{n+1},  F* = A^-1 X F^n,
// per point; the library accumulates SC = sum mu F*^T (and SA with the weight dE/dV0) and contracts
// them with dK/dtheta once at the end. FP64 handles only.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "bte_handle.h"
#include "bte_kernels.h"

namespace {

bte_status afail(const bte_handle* h, bte_status s, const std::string& m) { return bte::handle_fail(h, s, m); }

#define BA_CUDA(h, call)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return afail((h), BTE_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

// SC[a][b] += P[a][b], SA[a][b] += wA P[a][b], P = sum_i mu[i][a] Fs[i][b] (32 x 32 tiles, the
// point dimension staged through shared memory in chunks of 32).
__global__ void sens_accumulate_kernel(const double* __restrict__ mu, const double* __restrict__ Fs, int nx, int nv,
                                       double* __restrict__ SC, double* __restrict__ SA, double wA) {
  __shared__ double ms[32][33], fs[32][33];
  const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads, 4 outputs each
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i0 = 0; i0 < nx; i0 += 32) {
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int ii = idx / 32, c = idx % 32;
      const bool in = i0 + ii < nx;
      ms[ii][c] = in && a0 + c < nv ? mu[static_cast<size_t>(i0 + ii) * nv + a0 + c] : 0.0;
      fs[ii][c] = in && b0 + c < nv ? Fs[static_cast<size_t>(i0 + ii) * nv + b0 + c] : 0.0;
    }
    __syncthreads();
    for (int ii = 0; ii < 32; ++ii) {
      const double f = fs[ii][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += ms[ii][ty + 8 * q] * f;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = a0 + ty + 8 * q, b = b0 + tx;
    if (a < nv && b < nv) {
      const size_t e = static_cast<size_t>(a) * nv + b;
      if (SC) SC[e] += acc[q];
      if (SA) SA[e] += wA * acc[q];
    }
  }
}

// y += w g
__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ g, double w, size_t n) {
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x)
    y[e] += w * g[e];
}

template <typename T>
bte_status dalloc(bte_handle* h, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return afail(h, BTE_ENOMEM, "cudaMalloc failed");
  h->allocs.push_back(q);
  h->bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return BTE_OK;
}

// Transposed x-step operators, uploaded on the first adjoint call.
bte_status ensure_transposed(bte_handle* h) {
  if (h->Qt) return BTE_OK;
  const bte::HostOps& o = h->ops;
  const int nr = o.nr, nx = o.nx;
  std::vector<double> ut(nr * nr), uit(nr * nr), qt(o.Q.size());
  for (int i = 0; i < nr; ++i)
    for (int k = 0; k < nr; ++k) ut[i * nr + k] = o.U[k * nr + i], uit[i * nr + k] = o.Uinv[k * nr + i];
  const size_t blocks = static_cast<size_t>(o.nt) * nr;
  for (size_t bk = 0; bk < blocks; ++bk)
    for (int r = 0; r < nx; ++r)
      for (int c = 0; c < nx; ++c) qt[bk * nx * nx + static_cast<size_t>(r) * nx + c] = o.Q[bk * nx * nx + static_cast<size_t>(c) * nx + r];
  bte_status s;
  if ((s = dalloc(h, &h->Ut, ut.size())) != BTE_OK || (s = dalloc(h, &h->Uinvt, uit.size())) != BTE_OK ||
      (s = dalloc(h, &h->Qt, qt.size())) != BTE_OK)
    return s;
  BA_CUDA(h, cudaMemcpy(h->Ut, ut.data(), sizeof(double) * ut.size(), cudaMemcpyHostToDevice));
  BA_CUDA(h, cudaMemcpy(h->Uinvt, uit.data(), sizeof(double) * uit.size(), cudaMemcpyHostToDevice));
  BA_CUDA(h, cudaMemcpy(h->Qt, qt.data(), sizeof(double) * qt.size(), cudaMemcpyHostToDevice));
  return BTE_OK;
}

}  // namespace

extern "C" {

bte_status bte_step_adjoint(bte_handle* h, const double* F_dev, double* lambda_dev, double t_s, double V0,
                            double freq_Hz, const double* g_dev, double g_weight, double* SC_dev, double* SA_dev) {
  if (!h) return afail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev || !lambda_dev) return afail(h, BTE_EINVAL, "F_dev and lambda_dev are required");
  if (h->host_only || !h->ops.have_v) return afail(h, BTE_ESTATE, "needs device buffers and cross sections");
  if (h->precision != BTE_FP64) return afail(h, BTE_ESTATE, "the adjoint is implemented for FP64 handles");
  if (h->structured) return afail(h, BTE_ESTATE, "the adjoint needs the dense factorisation (no BTE_FLAG_STRUCTURED)");
  if (h->reduced)
    return afail(h, BTE_ESTATE, "the adjoint needs the full Nv x Nv factors (BTE_FLAG_FULL_V when nl < ntheta)");
  bte_status s = ensure_transposed(h);
  if (s != BTE_OK) return s;
  const bte::HostOps& o = h->ops;
  const int nx = o.nx, nt = o.nt, nr = o.nr, nv = o.nv, n = nv, nb = h->nb;
  const size_t D = static_cast<size_t>(nx) * nv;
  cudaStream_t st = h->st;
  const double arg = 2.0 * bte::kPi * freq_Hz * (t_s + 0.5 * o.dt);
  const double Eu = V0 / o.L * std::sin(arg);
  double* fac = static_cast<double*>(h->fac);
  unsigned long long nl = 0;
  BA_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), st));
  // forward pieces of step n: G = X F^n (Fa), the factors of A_i, F* = A^-1 G (Fb)
  bte::launch_x_to_eigen(F_dev, h->Uinv, h->Y, nx, nt, nr, h->status, st);
  bte::launch_x_apply_q(h->Q, h->Y, h->Y2, nx, nt, nr, st);
  bte::launch_x_from_eigen(h->Y2, h->U, h->Fa, nx, nt, nr, nullptr, st);
  const bte::MassBand mass{h->Mband, nr, o.mw};
  bte::launch_v_form<double>(h->KCg, h->KAg, mass, nullptr, Eu, o.dt, fac, nx, nv, st);
  nl += 4;
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = std::min(nb, n - k0);
    bte::launch_lu_panel<double>(fac, h->piv, h->perm, static_cast<double*>(h->linv), nullptr, nx, n, k0, kb, nb,
                                 h->status, nullptr, nullptr, nullptr, nullptr, h->panel_w, st);
    ++nl;
    if (k0 + kb < n) {
      bte::launch_lu_swap_trsm<double>(fac, h->perm, static_cast<double*>(h->linv), nx, n, k0, kb, nb, nullptr,
                                       nullptr, st);
      bte::launch_lu_gemm_simt<double>(fac, nx, n, k0, kb, st);
      nl += 2;
    }
  }
  bte::launch_lu_solve<double>(fac, h->piv, h->Fa, h->Fb, nx, n, nb, nullptr, 0, st, mass);
  // nu = X^T lambda (R), mu = A^-T nu (Fw), sensitivities, lambda <- X^T mu + w g
  bte::launch_x_to_eigen(lambda_dev, h->Ut, h->Y, nx, nt, nr, h->status, st);
  bte::launch_x_apply_q(h->Qt, h->Y, h->Y2, nx, nt, nr, st);
  bte::launch_x_from_eigen(h->Y2, h->Uinvt, h->R, nx, nt, nr, nullptr, st);
  bte::launch_lu_solve_t(fac, h->piv, h->R, h->Fw, nx, n, nb, st, mass);
  nl += 5;
  if (SC_dev || SA_dev) {
    dim3 grid((nv + 31) / 32, (nv + 31) / 32);
    sens_accumulate_kernel<<<grid, 256, 0, st>>>(h->Fw, h->Fb, nx, nv, SC_dev, SA_dev, std::sin(arg) / o.L);
    ++nl;
  }
  bte::launch_x_to_eigen(h->Fw, h->Ut, h->Y, nx, nt, nr, nullptr, st);
  bte::launch_x_apply_q(h->Qt, h->Y, h->Y2, nx, nt, nr, st);
  bte::launch_x_from_eigen(h->Y2, h->Uinvt, lambda_dev, nx, nt, nr, h->status, st);
  nl += 3;
  if (g_dev && g_weight != 0.0) {
    axpy_kernel<<<static_cast<unsigned>(std::min<size_t>((D + 255) / 256, 4096)), 256, 0, st>>>(lambda_dev, g_dev,
                                                                                              g_weight, D);
    ++nl;
  }
  BA_CUDA(h, cudaGetLastError());
  h->launches += nl;
  BA_CUDA(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  BA_CUDA(h, cudaStreamSynchronize(st));
  const unsigned f = *h->status_host;
  h->last_flags = f;
  if (f & bte::kNonFiniteIn) return afail(h, BTE_ENONFINITE, "non-finite values in the state or adjoint handed in");
  if (f & bte::kZeroPivot) return afail(h, BTE_ESINGULAR, "zero or non-finite pivot in a per-point factorisation");
  if (f & bte::kNonFinite) return afail(h, BTE_ENONFINITE, "non-finite values in the adjoint step");
  return BTE_OK;
}

bte_status bte_adjoint_gradient(const bte_handle* h, const double* SC_dev, const double* SA_dev, double h_eV,
                                double* grad_out) {
  if (!h) return afail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!SC_dev || !SA_dev || !grad_out || !(h_eV > 0)) return afail(h, BTE_EINVAL, "bad arguments");
  if (h->host_only || !h->ops.have_v) return afail(h, BTE_ESTATE, "needs device buffers and cross sections");
  const bte::HostOps& o = h->ops;
  const size_t nn = static_cast<size_t>(o.nv) * o.nv;
  std::vector<double> SC(nn), SA(nn);
  BA_CUDA(h, cudaStreamSynchronize(h->st));
  BA_CUDA(h, cudaMemcpy(SC.data(), SC_dev, nn * sizeof(double), cudaMemcpyDeviceToHost));
  BA_CUDA(h, cudaMemcpy(SA.data(), SA_dev, nn * sizeof(double), cudaMemcpyDeviceToHost));
  auto dotS = [&](const std::vector<double>& K, const std::vector<double>& S) {
    double acc = 0.0;
    for (size_t e = 0; e < nn; ++e) acc += K[e] * S[e];
    return acc;
  };
  const int np = static_cast<int>(h->procs.size());
  for (int j = 0; j < np; ++j) {
    // scale factor: K_C is linear in it, dK_C/ds_j = the process's own K_C at unit scale
    bte::Process p = h->procs[j];
    p.scale = 1.0;
    std::vector<double> K;
    std::string e = bte::assemble_kc_only(o, {p}, K);
    if (!e.empty()) return afail(h, BTE_EINVAL, e);
    grad_out[j] = o.dt * dotS(K, SC);
    // threshold: central difference of the assembly (0 for processes without one)
    grad_out[np + j] = 0.0;
    if (h->procs[j].th_eV > 0.0) {
      bte::Process pp = h->procs[j], pm = h->procs[j];
      pp.th_eV += h_eV;
      pm.th_eV -= h_eV;
      std::vector<double> Kp, Km;
      std::string e1 = bte::assemble_kc_only(o, {pp}, Kp), e2 = bte::assemble_kc_only(o, {pm}, Km);
      if (!e1.empty() || !e2.empty()) return afail(h, BTE_EINVAL, e1 + e2);
      double acc = 0.0;
      for (size_t q = 0; q < nn; ++q) acc += (Kp[q] - Km[q]) * SC[q];
      grad_out[np + j] = o.dt * acc / (2.0 * h_eV);
    }
  }
  grad_out[2 * np] = o.dt * dotS(o.KA, SA);
  return BTE_OK;
}

}  // extern "C"
