// Self-consistent field, ion fluid step and the fully-implicit electron step of arXiv 2502.16555
// (Section 2.3, eqs. "hybrid_discrete", "voltage_bc", "fl_ion_bc"; Section 3.4, eqs. "fluid_step",
// "bte_semi_implicit_efield", "bte_fully_implicit", "1dbte_jac_action"), declared in include/bte.h.
//
//   field        E = L (n_i - u^T F) + V(0, t) E_1: n_e per point, then one dense Nx x Nx product
//                (L and E_1 from the Dirichlet Laplacian on the collocation points, host-assembled);
//   ion step     (I/dt + D_x (mu_i E^n .) - D_i D_x D_x) n^{n+1} = n^n/dt + n0 r_ion.F^n with the
//                outflow-only wall fluxes as the first and last rows, solved by one CTA (GEPP);
//   sc step      the semi-implicit step with E^{1/2} recomputed after the first x half step;
//   implicit     Newton with backtracking on R(F) = F - F^n + dt [A_x F D_x^T - P_O (C + E(F) A_v) P_S F]
//                (inflow rows R = F), each Newton system by restarted flexible GMRES on the Jacobian
//                action J X = X + dt [A_x X D_x^T - P_O (C + E(F) A_v) P_S X
//                + P_O A_v P_S ((L u^T X) . F)], right-preconditioned at the iterate's field by the
//                per-point solves (factors formed once per Newton iteration) followed by one full x
//                step (default), or by the semi-implicit step's map; the preconditioned vectors are
//                kept, so the update is exact for the basis GMRES built. Orthogonalisation by
//                classical Gram-Schmidt applied twice; the small Hessenberg least-squares problem on
//                the host. All vectors FP64 on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "bte_handle.h"
#include "bte_kernels.h"

namespace {

constexpr int kDotBlock = 256;   // threads of the reduction kernels
constexpr int kDotGrid = 304;    // blocks of the partial dot products (2 per SM)

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// out[i] = w . X_i for every point i (one CTA per point): n_e with w = u, the ionisation source
// with w = r_ion.
__global__ void point_dot_kernel(const double* __restrict__ X, const double* __restrict__ w, int nv,
                                 double* __restrict__ out) {
  __shared__ double red[32];
  const double* x = X + static_cast<size_t>(blockIdx.x) * nv;
  double s = 0.0;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) s = fma(__ldg(w + v), x[v], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// E_i = sum_j L[i][j] (ni_j - ne_j) + vleft E1_i (ni NULL: no ions), one warp per row.
__global__ void field_kernel(const double* __restrict__ Lop, const double* __restrict__ E1,
                             const double* __restrict__ ni, const double* __restrict__ ne, double vleft, int nx,
                             double* __restrict__ E) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nx) return;
  const double* l = Lop + static_cast<size_t>(warp) * nx;
  double s = 0.0;
  for (int j = lane; j < nx; j += 32) s = fma(l[j], (ni ? ni[j] : 0.0) - ne[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) E[warp] = s + vleft * E1[warp];
}

// The ion system of eq. "fluid_step", row i per CTA: A = I/dt + D_x diag(mu E) - d D_x D_x,
// b = ni/dt + src; the wall rows are the flux conditions J(0) = n max(0, -mu E(0)) and
// J(L) = -n max(0, mu E(L)) with J = mu E n - d D_x n (right-hand side 0).
__global__ void ion_assemble_kernel(const double* __restrict__ Dx, const double* __restrict__ E,
                                    const double* __restrict__ ni, const double* __restrict__ src, double mu,
                                    double d, double dt, int nx, double* __restrict__ A, double* __restrict__ b) {
  const int i = blockIdx.x;
  double* a = A + static_cast<size_t>(i) * nx;
  const double* di = Dx + static_cast<size_t>(i) * nx;
  const bool wall = i == 0 || i == nx - 1;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    double v;
    if (wall) {
      v = -d * di[j] + (i == j ? mu * E[i] : 0.0);
      if (i == j) v += i == 0 ? -fmax(0.0, -mu * E[i]) : fmax(0.0, mu * E[i]);
    } else {
      double dd = 0.0;  // (D_x D_x)[i][j]
      for (int k = 0; k < nx; ++k) dd = fma(di[k], Dx[static_cast<size_t>(k) * nx + j], dd);
      v = di[j] * mu * E[j] - d * dd + (i == j ? 1.0 / dt : 0.0);
    }
    a[j] = v;
  }
  if (threadIdx.x == 0) b[i] = wall ? 0.0 : ni[i] / dt + src[i];
  if (wall) {
    // the flux rows are ~1e-9 of the interior rows (1/dt) in scale: equilibrate them (same
    // solution) so the wall values are not left to the rounding of a badly scaled system
    __shared__ double red[32];
    __syncthreads();
    double mx = 0.0;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) mx = fmax(mx, fabs(a[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) red[0] = fmax(red[0], red[w]);
    }
    __syncthreads();
    const double sc = red[0] > 0.0 ? (1.0 / dt) / red[0] : 1.0;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) a[j] *= sc;
  }
}

// x = A^-1 b by Gaussian elimination with partial pivoting, one CTA, A and b in global memory
// (overwritten). A zero or non-finite pivot sets kZeroPivot in status.
__global__ void dense_solve_kernel(double* __restrict__ A, double* __restrict__ b, int n, double* __restrict__ x,
                                   unsigned* status) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int piv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += nt) {
      const double v = fabs(A[static_cast<size_t>(i) * n + k]);
      if (v > best) best = v, bi = i;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
    }
    if (lane == 0) rv[warp] = best, ri[warp] = bi;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < nt / 32; ++w)
        if (rv[w] > rv[0] || (rv[w] == rv[0] && ri[w] < ri[0])) rv[0] = rv[w], ri[0] = ri[w];
      piv = ri[0];
      if (!(rv[0] > 0.0) || !isfinite(rv[0])) atomicOr(status, bte::kZeroPivot);
    }
    __syncthreads();
    const int p = piv;
    if (p != k) {
      for (int j = tid; j < n; j += nt) {
        const double t = A[static_cast<size_t>(k) * n + j];
        A[static_cast<size_t>(k) * n + j] = A[static_cast<size_t>(p) * n + j];
        A[static_cast<size_t>(p) * n + j] = t;
      }
      if (tid == 0) {
        const double t = b[k];
        b[k] = b[p];
        b[p] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / A[static_cast<size_t>(k) * n + k];
    // rows below the pivot: a warp per row, lanes over the columns (lane 0 also takes b)
    for (int i = k + 1 + warp; i < n; i += nt >> 5) {
      const double l = A[static_cast<size_t>(i) * n + k] * inv;
      for (int j = k + 1 + lane; j < n; j += 32) A[static_cast<size_t>(i) * n + j] -= l * A[static_cast<size_t>(k) * n + j];
      if (lane == 0) b[i] -= l * b[k];
    }
    __syncthreads();
  }
  __shared__ double red[32];
  for (int i = n - 1; i >= 0; --i) {
    double s = 0.0;
    for (int j = i + 1 + tid; j < n; j += nt) s = fma(A[static_cast<size_t>(i) * n + j], x[j], s);
    s = block_sum(s, red);
    if (tid == 0) x[i] = (b[i] - s) / A[static_cast<size_t>(i) * n + i];
    __syncthreads();
  }
}

// The same elimination with A and b staged in shared memory (n <= kSmemSolve): one CTA, the
// pivot column scanned by warp 0, rows exchanged and updated in shared memory.
constexpr int kSmemSolve = 150;
__global__ void dense_solve_smem_kernel(const double* __restrict__ Ag, const double* __restrict__ bg, int n,
                                        double* __restrict__ x, unsigned* status) {
  extern __shared__ double sm[];
  const int ld = n + 1;          // padded rows; column n holds b
  double* A = sm;
  __shared__ int piv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  for (int i = tid >> 5; i < n; i += nt >> 5)
    for (int j = lane; j < n; j += 32) A[i * ld + j] = Ag[static_cast<size_t>(i) * n + j];
  for (int i = tid; i < n; i += nt) A[i * ld + n] = bg[i];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + lane; i < n; i += 32) {
        const double v = fabs(A[i * ld + k]);
        if (v > best) best = v, bi = i;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
      }
      if (lane == 0) {
        piv = bi;
        if (!(best > 0.0) || !isfinite(best)) atomicOr(status, bte::kZeroPivot);
      }
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int j = k + tid; j <= n; j += nt) {
        const double t = A[k * ld + j];
        A[k * ld + j] = A[p * ld + j];
        A[p * ld + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / A[k * ld + k];
    // rows below the pivot: a warp per row, lanes over the columns (column n: right-hand side)
    for (int i = k + 1 + (tid >> 5); i < n; i += nt >> 5) {
      const double l = A[i * ld + k] * inv;
      for (int j = k + 1 + lane; j <= n; j += 32) A[i * ld + j] -= l * A[k * ld + j];
    }
    __syncthreads();
  }
  // back substitution by warp 0 alone (lanes over the row, shuffle sums): no block barriers
  if (tid < 32) {
    for (int i = n - 1; i >= 0; --i) {
      double s = 0.0;
      for (int j = i + 1 + lane; j < n; j += 32) s = fma(A[i * ld + j], A[j * ld + n], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) A[i * ld + n] = (A[i * ld + n] - s) / A[i * ld + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) x[i] = A[i * ld + n];
}

// out_i = P_O (c C_s + e_i A_s) P_S X_i per point (one CTA per point): c = 1 and e_i = E[i] for
// the velocity operator at a field, c = 0 and e_i = 1 for P_O A_v P_S alone. Structured operators
// as in the refinement residual (Algorithm 2).
__global__ void v_apply_kernel(const double* __restrict__ X, const double* __restrict__ E, double c,
                               const double* __restrict__ Cs, const double* __restrict__ Alo,
                               const double* __restrict__ Aup, const double* __restrict__ TO,
                               const double* __restrict__ TS, double* __restrict__ out, int nt, int nr, int nl) {
  extern __shared__ double sm[];
  const int i = blockIdx.x, nv = nt * nr;
  double* xs = sm;             // nv
  double* xS = xs + nv;        // nl*nr
  double* g = xS + nl * nr;    // nl*nr
  const double* x = X + static_cast<size_t>(i) * nv;
  const double e = E ? E[i] : 1.0;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) xs[v] = x[v];
  __syncthreads();
  for (int idx = threadIdx.x; idx < nl * nr; idx += blockDim.x) {
    const int l = idx / nr, k = idx % nr;
    double s = 0.0;
    for (int a = 0; a < nt; ++a) s = fma(__ldg(TS + l * nt + a), xs[a * nr + k], s);
    xS[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nl * nr; idx += blockDim.x) {
    const int l = idx / nr, p = idx % nr;
    const size_t off = (static_cast<size_t>(l) * nr + p) * nr;
    double cc = 0.0, f = 0.0;
    if (c != 0.0)
      for (int k = 0; k < nr; ++k) cc = fma(__ldg(Cs + off + k), xS[l * nr + k], cc);
    if (l >= 1)
      for (int k = 0; k < nr; ++k) f = fma(__ldg(Alo + off + k), xS[(l - 1) * nr + k], f);
    if (l + 1 < nl)
      for (int k = 0; k < nr; ++k) f = fma(__ldg(Aup + off + k), xS[(l + 1) * nr + k], f);
    g[idx] = c * cc + e * f;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const int a = v / nr, p = v % nr;
    double s = 0.0;
    for (int l = 0; l < nl; ++l) s = fma(__ldg(TO + a * nl + l), g[l * nr + p], s);
    out[static_cast<size_t>(i) * nv + v] = s;
  }
}

// out = X + s0 Y0 + dt (Zx - VX) - dt El_i KAF_i  (El, KAF may be NULL), except the inflow rows of
// each ordinate (x = 0 for mu >= 0, x = L otherwise), where out = X.
__global__ void implicit_combine_kernel(const double* __restrict__ X, const double* __restrict__ Y0, double s0,
                                        const double* __restrict__ Zx, const double* __restrict__ VX,
                                        const double* __restrict__ El, const double* __restrict__ KAF,
                                        const double* __restrict__ mu, double dt, int nx, int nt, int nr,
                                        double* __restrict__ out) {
  const size_t n = static_cast<size_t>(nx) * nt * nr;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e / (static_cast<size_t>(nt) * nr));
    const int a = static_cast<int>((e / nr) % nt);
    const bool inflow = mu[a] >= 0.0 ? i == 0 : i == nx - 1;
    double v = X[e];
    if (!inflow) {
      if (Y0) v += s0 * Y0[e];
      double r = Zx[e] - VX[e];
      if (El) r -= El[i] * KAF[e];
      v += dt * r;
    }
    out[e] = v;
  }
}

// partial[blk][j] = sum over this block's elements of V_j . w, j < k (V_j = V + j ld)
__global__ void multi_dot_kernel(const double* __restrict__ V, size_t ld, int k, const double* __restrict__ w,
                                 size_t n, double* __restrict__ partial) {
  __shared__ double red[32];
  for (int j = 0; j < k; ++j) {
    const double* v = V + j * ld;
    double s = 0.0;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x)
      s = fma(v[e], w[e], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[static_cast<size_t>(blockIdx.x) * k + j] = s;
  }
}

// out[j] = sum over blocks of partial[blk][j]: one CTA per j, strided partial sums then a tree
// (a fixed order, so the result is reproducible)
__global__ void sum_partials_kernel(const double* __restrict__ partial, int nblk, int k, double* __restrict__ out) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[static_cast<size_t>(b) * k + j];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[j] = s;
}

// w = a w + sg sum_{j<k} c_j V_j   (c in device memory)
__global__ void multi_axpy_kernel(double* __restrict__ w, double a, const double* __restrict__ V, size_t ld, int k,
                                  const double* __restrict__ c, double sg, size_t n) {
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s = fma(c[j], V[j * ld + e], s);
    w[e] = (a == 0.0 ? 0.0 : a * w[e]) + sg * s;
  }
}

// y += a x
__global__ void axpy_kernel(double* __restrict__ y, double a, const double* __restrict__ x, size_t n) {
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}

// x *= a
__global__ void scale_kernel(double* __restrict__ x, double a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= a;
}

}  // namespace

namespace bte {
namespace {

bte_status hfail(const bte_handle* h, bte_status s, const std::string& m) { return handle_fail(h, s, m); }

#define BH_CUDA(h, call)                                                                          \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return hfail((h), BTE_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
bte_status halloc(bte_handle* h, T** p, size_t count) {
  void* q = nullptr;
  const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
  if (e != cudaSuccess) return hfail(h, BTE_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  h->allocs.push_back(q);
  h->bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return BTE_OK;
}

template <typename T>
bte_status hupload(bte_handle* h, T** p, const std::vector<T>& v) {
  bte_status s = halloc(h, p, v.size());
  if (s != BTE_OK) return s;
  BH_CUDA(h, cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return BTE_OK;
}

int vec_grid(size_t n) { return static_cast<int>(std::min<size_t>((n + 255) / 256, 1216)); }

// Operators of the self-consistent parts, assembled and uploaded on first use.
bte_status hybrid_setup(bte_handle* h) {
  if (h->hybrid) return BTE_OK;
  const HostOps& o = h->ops;
  if (!o.have_v) return hfail(h, BTE_ESTATE, "set the cross sections first");
  std::vector<double> Lop, E1;
  const std::string e = assemble_field(o, Lop, E1);
  if (!e.empty()) return hfail(h, BTE_EINVAL, e);
  std::vector<double> rion(o.nv, 0.0);
  for (size_t j = 0; j < h->procs.size(); ++j)
    if (h->procs[j].kind == BTE_IONIZATION) {
      std::copy(o.mom_r.begin() + j * o.nv, o.mom_r.begin() + (j + 1) * o.nv, rion.begin());
      break;
    }
  bte_status s = BTE_OK;
  if (s == BTE_OK) s = hupload(h, &h->Lop, Lop);
  if (s == BTE_OK) s = hupload(h, &h->E1, E1);
  if (s == BTE_OK) s = hupload(h, &h->Dxd, o.Dx);
  if (s == BTE_OK) s = hupload(h, &h->mud, o.mu);
  if (s == BTE_OK) s = hupload(h, &h->lamd, o.lam);
  if (s == BTE_OK) s = hupload(h, &h->rion, rion);
  if (s == BTE_OK) s = halloc(h, &h->Esc, o.nx);
  if (s == BTE_OK) s = halloc(h, &h->ned, o.nx);
  if (s == BTE_OK) s = halloc(h, &h->Ek, o.nx);
  if (s == BTE_OK) s = halloc(h, &h->ionA, static_cast<size_t>(o.nx) * o.nx);
  if (s == BTE_OK) s = halloc(h, &h->ionb, o.nx);
  if (s != BTE_OK) return s;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(v_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  h->hybrid = true;
  return BTE_OK;
}

// Work vectors of the fully-implicit step for a GMRES basis of m + 1 vectors.
bte_status implicit_setup(bte_handle* h, int m, bool full_q) {
  bte_status s = BTE_OK;
  if (full_q && !h->Qfull) {
    // Q_ij for a full step, (I + dt lam_i mu_a D_x)^-1 with the inflow rows
    std::vector<double> Q;
    if (!assemble_q(h->ops, h->ops.dt, Q)) return hfail(h, BTE_EINVAL, "a full-step x operator is singular");
    if ((s = hupload(h, &h->Qfull, Q)) != BTE_OK) return s;
  }
  if (h->gm >= m) return BTE_OK;
  const size_t D = static_cast<size_t>(h->ops.nx) * h->ops.nv;
  if (!h->Fk) {
    for (double** p : {&h->Fk, &h->Fn, &h->Rv, &h->Zx, &h->VX, &h->KAF, &h->Wv, &h->Pz, &h->Dl})
      if (s == BTE_OK) s = halloc(h, p, D);
    if (s == BTE_OK) s = halloc(h, &h->El, h->ops.nx);
  }
  if (s == BTE_OK) s = halloc(h, &h->Vb, D * (m + 1));
  if (s == BTE_OK) s = halloc(h, &h->Zb, D * m);
  if (s == BTE_OK) s = halloc(h, &h->part, static_cast<size_t>(kDotGrid) * (m + 1));
  if (s == BTE_OK) s = halloc(h, &h->dsum, 3 * (m + 1));  // two Gram-Schmidt passes and a norm
  if (s != BTE_OK) return s;
  if (h->dsum_host) cudaFreeHost(h->dsum_host);
  BH_CUDA(h, cudaMallocHost(reinterpret_cast<void**>(&h->dsum_host), 3 * (m + 1) * sizeof(double)));
  h->gm = m;
  return BTE_OK;
}

// A_x X D_x^T (per ordinate mu_a D_x X_a G^T, G = M_v^-1 G_v) through the eigen basis of G
void enqueue_xop(bte_handle* h, const double* X, double* out) {
  const HostOps& o = h->ops;
  cudaStream_t st = h->st;
  launch_x_to_eigen(X, h->Uinv, h->Y, o.nx, o.nt, o.nr, h->status, st);
  launch_x_matvec(h->Dxd, false, h->lamd, h->mud, h->Y, h->Y2, o.nx, o.nt, o.nr, st);  // lam_i mu_a D_x Y
  launch_x_from_eigen(h->Y2, h->U, out, o.nx, o.nt, o.nr, nullptr, st);
}

void enqueue_vapply(bte_handle* h, const double* X, const double* E, double c, double* out) {
  const HostOps& o = h->ops;
  const size_t smem = sizeof(double) * (static_cast<size_t>(o.nv) + 2 * o.nl * o.nr);
  v_apply_kernel<<<o.nx, 256, smem, h->st>>>(X, E, c, h->Cs, h->Alo, h->Aup, h->TO, h->TS, out, o.nt, o.nr, o.nl);
}

// out_dev[j] = V_j . w for j < k on the device (stream-ordered; no host synchronisation)
void enqueue_dots(bte_handle* h, const double* V, size_t ld, int k, const double* w, double* out_dev) {
  const size_t D = static_cast<size_t>(h->ops.nx) * h->ops.nv;
  multi_dot_kernel<<<kDotGrid, kDotBlock, 0, h->st>>>(V, ld, k, w, D, h->part);
  sum_partials_kernel<<<k, 128, 0, h->st>>>(h->part, kDotGrid, k, out_dev);
}

// dots[j] = V_j . w for j < k into the pinned host array (synchronises the stream)
bte_status host_dots(bte_handle* h, const double* V, size_t ld, int k, const double* w, std::vector<double>& out) {
  const size_t D = static_cast<size_t>(h->ops.nx) * h->ops.nv;
  multi_dot_kernel<<<kDotGrid, kDotBlock, 0, h->st>>>(V, ld, k, w, D, h->part);
  sum_partials_kernel<<<k, 128, 0, h->st>>>(h->part, kDotGrid, k, h->dsum);
  BH_CUDA(h, cudaMemcpyAsync(h->dsum_host, h->dsum, k * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  BH_CUDA(h, cudaStreamSynchronize(h->st));
  out.assign(h->dsum_host, h->dsum_host + k);
  return BTE_OK;
}

}  // namespace

bte_status enqueue_field(bte_handle* h, const double* F_dev, const double* ni_dev, double t, double V0,
                         double freq, double* E_dev) {
  const HostOps& o = h->ops;
  point_dot_kernel<<<o.nx, 256, 0, h->st>>>(F_dev, h->mom_n, o.nv, h->ned);
  const double vleft = V0 * std::sin(2.0 * kPi * freq * t);
  field_kernel<<<(o.nx * 32 + 255) / 256, 256, 0, h->st>>>(h->Lop, h->E1, ni_dev, h->ned, vleft, o.nx, E_dev);
  handle_add_launches(h, 2);
  BH_CUDA(h, cudaGetLastError());
  return BTE_OK;
}

}  // namespace bte

// ---------------------------------------------------------------------------------- entry points

using bte::hfail;

extern "C" {

bte_status bte_set_ion_transport(bte_handle* h, double n0_mu_i, double n0_D_i) {
  if (!h) return hfail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!(n0_mu_i >= 0.0) || !(n0_D_i > 0.0) || !std::isfinite(n0_mu_i) || !std::isfinite(n0_D_i))
    return hfail(h, BTE_EINVAL, "ion mobility must be >= 0 and ion diffusion > 0 (both finite)");
  h->n0_mu_i = n0_mu_i;
  h->n0_D_i = n0_D_i;
  return BTE_OK;
}

bte_status bte_field(bte_handle* h, const double* F_dev, const double* ni_dev, double t_s, double V0,
                     double freq_Hz, double* E_dev) {
  if (!h) return hfail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev || !E_dev) return hfail(h, BTE_EINVAL, "F_dev and E_dev must not be NULL");
  {
    const bte_status ds = bte::handle_device_status(h);
    if (ds != BTE_OK) return ds;
  }
  bte_status s = bte::hybrid_setup(h);
  if (s != BTE_OK) return s;
  return bte::enqueue_field(h, F_dev, ni_dev, t_s, V0, freq_Hz, E_dev);
}

bte_status bte_ion_step(bte_handle* h, double* ni_dev, const double* F_dev, double t_s, double V0,
                        double freq_Hz) {
  if (!h) return hfail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!ni_dev || !F_dev) return hfail(h, BTE_EINVAL, "ni_dev and F_dev must not be NULL");
  {
    const bte_status ds = bte::handle_device_status(h);
    if (ds != BTE_OK) return ds;
  }
  bte_status s = bte::hybrid_setup(h);
  if (s != BTE_OK) return s;
  const bte::HostOps& o = h->ops;
  cudaStream_t st = h->st;
  BH_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), st));
  // E^n from (n_i^n, F^n) at t_n, then the source n0 r_ion . F^n, the system, its solve
  s = bte::enqueue_field(h, F_dev, ni_dev, t_s, V0, freq_Hz, h->Esc);
  if (s != BTE_OK) return s;
  point_dot_kernel<<<o.nx, 256, 0, st>>>(F_dev, h->rion, o.nv, h->ned);
  scale_kernel<<<(o.nx + 255) / 256, 256, 0, st>>>(h->ned, o.n0, o.nx);
  ion_assemble_kernel<<<o.nx, 256, 0, st>>>(h->Dxd, h->Esc, ni_dev, h->ned, h->n0_mu_i / o.n0, h->n0_D_i / o.n0,
                                           o.dt, o.nx, h->ionA, h->ionb);
  if (o.nx <= kSmemSolve) {
    const size_t smem = sizeof(double) * o.nx * (o.nx + 1);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(dense_solve_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr = true;
    }
    dense_solve_smem_kernel<<<1, 1024, smem, st>>>(h->ionA, h->ionb, o.nx, h->ned, h->status);
  } else {
    dense_solve_kernel<<<1, 1024, 0, st>>>(h->ionA, h->ionb, o.nx, h->ned, h->status);
  }
  bte::launch_commit(h->ned, ni_dev, o.nx, h->status, st);
  bte::handle_add_launches(h, 5);
  BH_CUDA(h, cudaGetLastError());
  return bte::handle_read_status(h);
}

bte_status bte_step_sc(bte_handle* h, double* F_dev, const double* ni_dev, double t_s, double V0, double freq_Hz,
                       double* E_out_dev) {
  if (!h) return hfail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev || !ni_dev) return hfail(h, BTE_EINVAL, "F_dev and ni_dev must not be NULL");
  {
    const bte_status ds = bte::handle_device_status(h);
    if (ds != BTE_OK) return ds;
  }
  bte_status s = bte::hybrid_setup(h);
  if (s != BTE_OK) return s;
  BH_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), h->st));
  s = bte::handle_enqueue_sc_step(h, F_dev, ni_dev, t_s, V0, freq_Hz);
  if (s != BTE_OK) return s;
  if (E_out_dev)
    BH_CUDA(h, cudaMemcpyAsync(E_out_dev, h->Esc, h->ops.nx * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  return bte::handle_read_status(h);
}

bte_status bte_step_implicit(bte_handle* h, double* F_dev, const double* ni_dev, double t_s, double V0,
                             double freq_Hz, bte_implicit_opts* opts) {
  if (!h) return hfail(nullptr, BTE_EINVAL, "handle is NULL");
  if (!F_dev || !ni_dev) return hfail(h, BTE_EINVAL, "F_dev and ni_dev must not be NULL");
  {
    const bte_status ds = bte::handle_device_status(h);
    if (ds != BTE_OK) return ds;
  }
  double rtol = 1e-10, grtol = 1e-2;
  int newton_max = 8, m = 100, gmax = 400, precond = 0;
  if (opts) {
    if (opts->newton_rtol > 0) rtol = opts->newton_rtol;
    if (opts->gmres_rtol > 0) grtol = opts->gmres_rtol;
    if (opts->newton_max > 0) newton_max = opts->newton_max;
    if (opts->gmres_restart > 0) m = opts->gmres_restart;
    if (opts->gmres_max > 0) gmax = opts->gmres_max;
    precond = opts->precond;
    opts->newton_iters = opts->gmres_iters = 0;
    opts->residual = 0.0;
  }
  if (m > 200) return hfail(h, BTE_EINVAL, "gmres_restart must be <= 200");
  if (precond != 0 && precond != 1) return hfail(h, BTE_EINVAL, "precond must be 0 or 1");
  bte_status s = bte::hybrid_setup(h);
  if (s == BTE_OK) s = bte::implicit_setup(h, m, precond == 0);
  if (s != BTE_OK) return s;
  const bte::HostOps& o = h->ops;
  const int nx = o.nx, nt = o.nt, nr = o.nr;
  const size_t D = static_cast<size_t>(nx) * o.nv;
  const double dt = o.dt, t1 = t_s + dt;
  cudaStream_t st = h->st;
  const int vg = bte::vec_grid(D);
  unsigned long long launches = 0;

  // F^n, and the initial iterate: the semi-implicit self-consistent step from F^n (F^n itself if
  // that step flags anything)
  BH_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), st));
  BH_CUDA(h, cudaMemcpyAsync(h->Fn, F_dev, D * sizeof(double), cudaMemcpyDeviceToDevice, st));
  BH_CUDA(h, cudaMemcpyAsync(h->Fk, F_dev, D * sizeof(double), cudaMemcpyDeviceToDevice, st));
  s = bte::handle_enqueue_sc_step(h, h->Fk, ni_dev, t_s, V0, freq_Hz);
  if (s != BTE_OK) return s;
  s = bte::handle_read_status(h);
  if (s == BTE_ENONFINITE) return s;
  BH_CUDA(h, cudaMemsetAsync(h->status, 0, 2 * sizeof(unsigned), st));

  auto residual = [&](const double* X, double* R) {
    bte::enqueue_field(h, X, ni_dev, t1, V0, freq_Hz, h->Esc);
    bte::enqueue_xop(h, X, h->Zx);
    bte::enqueue_vapply(h, X, h->Esc, 1.0, h->VX);
    implicit_combine_kernel<<<vg, 256, 0, st>>>(X, h->Fn, -1.0, h->Zx, h->VX, nullptr, nullptr, h->mud, dt, nx, nt,
                                                nr, R);
    launches += 7;
  };
  auto norm = [&](const double* X, double& out) -> bte_status {
    std::vector<double> d;
    const bte_status r = bte::host_dots(h, X, 0, 1, X, d);
    out = std::sqrt(d[0]);
    launches += 2;
    return r;
  };
  // the preconditioner at the frozen field Ek, from the split step's pieces with the factors of
  // this Newton iteration. precond 0: the per-point solves, then one full x step (exact when either
  // part vanishes, also for the stiffest x modes); 1: the semi-implicit step's map (x half step,
  // solves, x half step), whose x part is (I + dt/2 A_x)^-2, far from (I + dt A_x)^-1 for x modes
  // with dt |A_x| >> 1
  auto pinv = [&](const double* in, double* out) -> bte_status {
    bte_status r = BTE_OK;
    if (precond == 0) {
      r = bte::handle_enqueue_vsolve(h, in, h->VX, h->Ek, false);
      if (r == BTE_OK) {
        bte::launch_x_to_eigen(h->VX, h->Uinv, h->Y, nx, nt, nr, nullptr, st);
        bte::launch_x_apply_q(h->Qfull, h->Y, h->Y2, nx, nt, nr, st);
        bte::launch_x_from_eigen(h->Y2, h->U, out, nx, nt, nr, nullptr, st);
        launches += 3;
      }
    } else {
      r = bte::handle_enqueue_xhalf(h, in, h->Wv);
      if (r == BTE_OK) r = bte::handle_enqueue_vsolve(h, h->Wv, h->VX, h->Ek, false);
      if (r == BTE_OK) r = bte::handle_enqueue_xhalf(h, h->VX, out);
    }
    return r;
  };
  // Jacobian action at F_k (eq. "1dbte_jac_action" with the inflow rows as identity)
  auto jac = [&](const double* X, double* out) {
    point_dot_kernel<<<nx, 256, 0, st>>>(X, h->mom_n, o.nv, h->ned);
    field_kernel<<<(nx * 32 + 255) / 256, 256, 0, st>>>(h->Lop, h->E1, nullptr, h->ned, 0.0, nx, h->El);
    bte::enqueue_xop(h, X, h->Zx);
    bte::enqueue_vapply(h, X, h->Ek, 1.0, h->VX);
    implicit_combine_kernel<<<vg, 256, 0, st>>>(X, nullptr, 0.0, h->Zx, h->VX, h->El, h->KAF, h->mud, dt, nx, nt,
                                                nr, out);
    launches += 7;
  };

  double fn = 0.0, rn = 0.0;
  if ((s = norm(h->Fn, fn)) != BTE_OK) return s;
  residual(h->Fk, h->Rv);
  if ((s = norm(h->Rv, rn)) != BTE_OK) return s;
  bool conv = rn <= rtol * fn;
  int newton = 0, gm_total = 0;
  std::vector<double> H(static_cast<size_t>(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  // forcing term of the current Newton iteration: a failed line search (no sufficient decrease
  // along a direction GMRES solved only to grtol) retries the iteration with a 100x tighter
  // linear solve, at most twice, before the step gives up
  double eta = grtol;
  int retries = 0;
  while (!conv && newton < newton_max) {
    // the iterate's field, frozen for the preconditioner and the Jacobian; factors at that field
    BH_CUDA(h, cudaMemcpyAsync(h->Ek, h->Esc, nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if ((s = bte::handle_enqueue_vsolve(h, h->Rv, h->Pz, h->Ek, true)) != BTE_OK) return s;
    bte::enqueue_vapply(h, h->Fk, nullptr, 0.0, h->KAF);
    // restarted GMRES on J delta = -R, right-preconditioned: delta accumulates in Dl; every cycle
    // solves J P^-1 y = r for the current residual r = -R - J delta
    BH_CUDA(h, cudaMemsetAsync(h->Dl, 0, D * sizeof(double), st));
    int inner = 0;
    double rc = rn;  // |r| of the current cycle
    for (int cyc = 0; inner < gmax; ++cyc) {
      if (cyc > 0) {
        jac(h->Dl, h->Vb);  // r = -R - J delta
        multi_axpy_kernel<<<vg, 256, 0, st>>>(h->Vb, -1.0, nullptr, D, 0, nullptr, 0.0, D);
        axpy_kernel<<<vg, 256, 0, st>>>(h->Vb, -1.0, h->Rv, D);
        if ((s = norm(h->Vb, rc)) != BTE_OK) return s;
        if (rc <= eta * rn) break;
        multi_axpy_kernel<<<vg, 256, 0, st>>>(h->Vb, 1.0 / rc, nullptr, D, 0, nullptr, 0.0, D);
      } else {
        BH_CUDA(h, cudaMemcpyAsync(h->Vb, h->Rv, D * sizeof(double), cudaMemcpyDeviceToDevice, st));
        multi_axpy_kernel<<<vg, 256, 0, st>>>(h->Vb, -1.0 / rn, nullptr, D, 0, nullptr, 0.0, D);
      }
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = rc;
      int k = 0;
      bool done = false;
      for (int j = 0; j < m && inner < gmax; ++j, ++inner) {
        double* Vj = h->Vb + static_cast<size_t>(j) * D;
        double* Vn = h->Vb + static_cast<size_t>(j + 1) * D;
        double* Zj = h->Zb + static_cast<size_t>(j) * D;
        if ((s = pinv(Vj, Zj)) != BTE_OK) return s;
        jac(Zj, Vn);
        // classical Gram-Schmidt twice, then the norm: the projections stay on the device (the
        // axpys read them there), so the host waits once per iteration for all three results
        const size_t stride = static_cast<size_t>(m) + 1;
        for (int pass = 0; pass < 2; ++pass) {
          double* dp = h->dsum + pass * stride;
          bte::enqueue_dots(h, h->Vb, D, j + 1, Vn, dp);
          multi_axpy_kernel<<<vg, 256, 0, st>>>(Vn, 1.0, h->Vb, D, j + 1, dp, -1.0, D);
          launches += 3;
        }
        bte::enqueue_dots(h, Vn, 0, 1, Vn, h->dsum + 2 * stride);
        launches += 2;
        BH_CUDA(h, cudaMemcpyAsync(h->dsum_host, h->dsum, 3 * stride * sizeof(double), cudaMemcpyDeviceToHost, st));
        BH_CUDA(h, cudaStreamSynchronize(st));
        for (int i = 0; i <= j; ++i) H[static_cast<size_t>(i) * m + j] += h->dsum_host[i] + h->dsum_host[stride + i];
        const double hn = std::sqrt(h->dsum_host[2 * stride]);
        H[static_cast<size_t>(j + 1) * m + j] = hn;
        if (hn > 0.0) multi_axpy_kernel<<<vg, 256, 0, st>>>(Vn, 1.0 / hn, nullptr, D, 0, nullptr, 0.0, D);
        for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
          const double a = H[static_cast<size_t>(i) * m + j], b = H[static_cast<size_t>(i + 1) * m + j];
          H[static_cast<size_t>(i) * m + j] = cs[i] * a + sn[i] * b;
          H[static_cast<size_t>(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
        }
        const double a = H[static_cast<size_t>(j) * m + j], b = H[static_cast<size_t>(j + 1) * m + j];
        const double r = std::hypot(a, b);
        cs[j] = r > 0.0 ? a / r : 1.0;
        sn[j] = r > 0.0 ? b / r : 0.0;
        H[static_cast<size_t>(j) * m + j] = r;
        H[static_cast<size_t>(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        k = j + 1;
        if (std::fabs(g[j + 1]) <= eta * rn || hn == 0.0) {
          done = true;
          ++inner;
          break;
        }
      }
      for (int i = k - 1; i >= 0; --i) {  // H y = g, upper triangular
        double v = g[i];
        for (int q = i + 1; q < k; ++q) v -= H[static_cast<size_t>(i) * m + q] * y[q];
        y[i] = v / H[static_cast<size_t>(i) * m + i];
      }
      // delta += Z y with the stored Z_j = P^-1 V_j (flexible GMRES): the Arnoldi relation
      // J Z = V H holds for whatever the preconditioner returned, so the residual the rotations
      // track is the true one even where the FP32 solves inside P^-1 are far from linear (stiff
      // velocity systems: relative rounding kappa eps_32 of order one)
      std::copy(y.begin(), y.begin() + k, h->dsum_host);
      BH_CUDA(h, cudaMemcpyAsync(h->dsum, h->dsum_host, k * sizeof(double), cudaMemcpyHostToDevice, st));
      multi_axpy_kernel<<<vg, 256, 0, st>>>(h->Dl, 1.0, h->Zb, D, k, h->dsum, 1.0, D);
      if (done) break;
    }
    gm_total += inner;
    // backtracking on |R|
    double lam = 1.0, rt = 0.0;
    bool acc = false;
    for (int ls = 0; ls < 8 && !acc; ++ls) {
      BH_CUDA(h, cudaMemcpyAsync(h->Wv, h->Fk, D * sizeof(double), cudaMemcpyDeviceToDevice, st));
      axpy_kernel<<<vg, 256, 0, st>>>(h->Wv, lam, h->Dl, D);
      residual(h->Wv, h->Rv);
      if ((s = norm(h->Rv, rt)) != BTE_OK) return s;
      if (rt <= (1.0 - 1e-4 * lam) * rn) acc = true;
      else lam *= 0.5;
    }
    if (!acc) {
      if (retries < 2 && inner > 0) {
        eta *= 1e-2;
        ++retries;
        // the residual of the iterate again (the line search overwrote Rv and the field)
        residual(h->Fk, h->Rv);
        if ((s = norm(h->Rv, rn)) != BTE_OK) return s;
        continue;
      }
      ++newton;
      break;
    }
    ++newton;
    eta = grtol;
    retries = 0;
    std::swap(h->Fk, h->Wv);
    rn = rt;
    conv = rn <= rtol * fn;
  }
  bte::handle_add_launches(h, launches);
  BH_CUDA(h, cudaGetLastError());
  if (opts) {
    opts->newton_iters = newton;
    opts->gmres_iters = gm_total;
    opts->residual = fn > 0.0 ? rn / fn : rn;
  }
  s = bte::handle_read_status(h);
  if (s != BTE_OK) return s;
  if (!conv) return hfail(h, BTE_ENOCONV, "Newton did not reach newton_rtol");
  BH_CUDA(h, cudaMemcpyAsync(F_dev, h->Fk, D * sizeof(double), cudaMemcpyDeviceToDevice, st));
  BH_CUDA(h, cudaStreamSynchronize(st));
  return BTE_OK;
}

}  // extern "C"
