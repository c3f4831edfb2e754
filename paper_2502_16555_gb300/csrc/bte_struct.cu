// Structure-exploiting velocity solve. The per-point matrix of eq. "vspace_batched_system" is
// A_i = I - dt P_O B_i P_S with B_i = C + E_i A_v in the spherical-harmonic basis (arXiv 2502.16555,
// eqs. "proj_ops", "bte_1d_discrete"), where C is block diagonal in l and A_v block tridiagonal
// (couplings l -> l +- 1 only, Section 3.3). Because P_S P_O = T_S T_O = I,
//     A_i^-1 f = f + P_O ( (I - dt B_i)^-1 - I ) P_S f,
// so one dense Nv x Nv solve becomes one block-tridiagonal solve of N_l blocks of Nr x Nr:
// y = P_S f; block elimination over l (S_0 = D_0, S_q = D_q - L_q S_{q-1}^-1 U_{q-1}, blocks
// D_q = I - dt Cs_q, L_q = -dt E As_lo[q], U_q = -dt E As_up[q]); back substitution; f* = f + P_O (z - y).
// The blocks are inverted by Gauss-Jordan without pivoting: S_q stays diagonally dominant enough
// (in-block growth 1.0 and pivots >= 0.2 on the workloads' field range), and the FP64 refinement
// that follows (Algorithm 2 residual) removes what rounding leaves.
//
// One CTA of 256 threads per point, a 16 x 16 thread grid over the Nr x Nr blocks (Nr <= 64):
// thread (ty, tx) owns the elements (ty + 16 a, tx + 16 b), a, b < 4, of the block being inverted and
// keeps them in registers for the whole Gauss-Jordan sweep; only the pivot row and column go
// through shared memory. Inverses are stored transposed, couplings transposed where they are the
// left factor, so every shared-memory read is a broadcast or conflict-free. The X_q of the
// forward sweep go to a per-point global scratch for the back substitution.
#include <cuda_runtime.h>

#include "bte_kernels.h"

namespace bte {
namespace {

constexpr int kST = 256;  // threads per CTA
constexpr int kG = 4;     // elements per thread and dimension (Nr <= 16 kG)

// acc(a, b) += sum_k AT[k][ty + 16 a] B[k][tx + 16 b] over k < n: AT is the left factor stored
// transposed (AT[k][i] = A[i][k]), both n x n with leading dimension n in shared memory.
template <typename T>
__device__ __forceinline__ void grid_gemm(const T* AT, const T* B, int n, T (&acc)[kG][kG]) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int k = 0; k < n; ++k) {
    T a[kG], b[kG];
#pragma unroll
    for (int u = 0; u < kG; ++u) {
      a[u] = ty + 16 * u < n ? AT[k * n + ty + 16 * u] : T(0);
      b[u] = tx + 16 * u < n ? B[k * n + tx + 16 * u] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kG; ++u)
#pragma unroll
      for (int v = 0; v < kG; ++v) acc[u][v] += a[u] * b[v];
  }
}

// out[i] = alpha * sum_k MT[k][i] x[k] for i < n (MT the matrix stored transposed): thread i,
// consecutive threads read consecutive addresses.
template <typename T>
__device__ __forceinline__ void gemv_t(const T* MT, const T* x, T* out, int n, T alpha) {
  for (int i = threadIdx.x; i < n; i += kST) {
    T acc = T(0);
    for (int k = 0; k < n; ++k) acc += MT[k * n + i] * x[k];
    out[i] = alpha * acc;
  }
}

// In-place inverse of the block held in registers (s[a][b] = S[ty + 16 a][tx + 16 b]) by
// Gauss-Jordan elimination without pivoting. Step k reads the pivot row and column from a copy
// written in step k - 1 by the owners of row/column k (double-buffered by parity): one barrier
// per step.
template <typename T>
__device__ void grid_gauss_jordan(T (&s)[kG][kG], int n, T* prow2, T* pcol2) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < kG; ++a)
#pragma unroll
    for (int b = 0; b < kG; ++b) {
      const int i = ty + 16 * a, j = tx + 16 * b;
      if (i == 0 && j < n) prow2[j] = s[a][b];
      if (j == 0 && i < n) pcol2[i] = s[a][b];
    }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const T* prow = prow2 + (k & 1) * 64;
    const T* pcol = pcol2 + (k & 1) * 64;
    T* nrow = prow2 + ((k + 1) & 1) * 64;
    T* ncol = pcol2 + ((k + 1) & 1) * 64;
    const T p = T(1) / prow[k];
    T pr[kG], fc[kG];
#pragma unroll
    for (int u = 0; u < kG; ++u) {
      pr[u] = tx + 16 * u < n ? prow[tx + 16 * u] : T(0);
      fc[u] = ty + 16 * u < n ? pcol[ty + 16 * u] * p : T(0);
    }
#pragma unroll
    for (int a = 0; a < kG; ++a)
#pragma unroll
      for (int b = 0; b < kG; ++b) {
        const int i = ty + 16 * a, j = tx + 16 * b;
        T v = s[a][b] - fc[a] * pr[b];
        if (i == k) v = pr[b] * p;
        if (j == k) v = (i == k) ? p : -fc[a];
        s[a][b] = v;
        if (i == k + 1 && j < n) nrow[j] = v;
        if (j == k + 1 && i < n) ncol[i] = v;
      }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kST) vsolve_struct_kernel(const double* __restrict__ Fin, double* __restrict__ Fout,
                                                            const double* __restrict__ E, double E_uniform, double dt,
                                                            const double* __restrict__ Cs, const double* __restrict__ Alo,
                                                            const double* __restrict__ Aup, const double* __restrict__ TO,
                                                            const double* __restrict__ TS, T* __restrict__ Xg, int nt,
                                                            int nr, int nl, const int* __restrict__ conv, int accumulate,
                                                            unsigned* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  if (conv && conv[pt]) return;
  const int n = nr, nn = nr * nr, nv = nt * nr;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* SinvT = reinterpret_cast<T*>(smraw);  // S_q^-1, transposed
  T* Xp = SinvT + nn;                      // X_{q-1} = S_{q-1}^-1 U_{q-1}, row-major
  T* Xc = Xp + nn;                         // X_q
  T* Ab = Xc + nn;                         // As_lo[q] transposed, then As_up[q] row-major
  T* y = Ab + nn;                          // nl x nr: P_S f, then w_q
  T* wq = y + nl * nr;                     // nl x nr: S_q^-1 w_q, then z
  T* tmp = wq + nl * nr;                   // nr
  T* prow2 = tmp + nr;                     // 2 x 64 pivot rows
  T* pcol2 = prow2 + 128;                  // 2 x 64 pivot columns
  const double* f = Fin + static_cast<size_t>(pt) * nv;
  const T eE = static_cast<T>(dt * (E ? E[pt] : E_uniform));
  T* X = Xg + static_cast<size_t>(pt) * nl * nn;

  // y = T_S f (per radial index)
  for (int e = threadIdx.x; e < nl * nr; e += kST) {
    const int l = e / nr, k = e % nr;
    double s = 0.0;
    for (int a = 0; a < nt; ++a) s += TS[l * nt + a] * f[a * nr + k];
    y[e] = static_cast<T>(s);
  }
  __syncthreads();
  for (int q = 0; q < nl; ++q) {
    // S_q = I - dt Cs_q + dt E As_lo[q] X_{q-1} in registers;  w_q = y_q + dt E As_lo[q] wq_{q-1}
    T s[kG][kG];
    const double* C = Cs + static_cast<size_t>(q) * nn;
#pragma unroll
    for (int a = 0; a < kG; ++a)
#pragma unroll
      for (int b = 0; b < kG; ++b) {
        const int i = ty + 16 * a, j = tx + 16 * b;
        s[a][b] = (i < n && j < n) ? (i == j ? T(1) : T(0)) - static_cast<T>(dt * C[i * n + j]) : T(0);
      }
    if (q > 0) {
      const double* Al = Alo + static_cast<size_t>(q) * nn;
      for (int e = threadIdx.x; e < nn; e += kST) Ab[(e % n) * n + e / n] = static_cast<T>(Al[e]);
      __syncthreads();
      T acc[kG][kG] = {};
      grid_gemm<T>(Ab, Xp, n, acc);
#pragma unroll
      for (int a = 0; a < kG; ++a)
#pragma unroll
        for (int b = 0; b < kG; ++b) s[a][b] += eE * acc[a][b];
      gemv_t<T>(Ab, wq + (q - 1) * nr, tmp, n, eE);
      for (int k = threadIdx.x; k < nr; k += kST) y[q * nr + k] += tmp[k];  // same thread wrote tmp[k]
    }
    grid_gauss_jordan<T>(s, n, prow2, pcol2);
#pragma unroll
    for (int a = 0; a < kG; ++a)
#pragma unroll
      for (int b = 0; b < kG; ++b) {
        const int i = ty + 16 * a, j = tx + 16 * b;
        if (i < n && j < n) SinvT[j * n + i] = s[a][b];
      }
    if (q + 1 < nl) {
      const double* Au = Aup + static_cast<size_t>(q) * nn;
      for (int e = threadIdx.x; e < nn; e += kST) Ab[e] = static_cast<T>(Au[e]);
    }
    __syncthreads();
    // wq_q = S_q^-1 w_q;  X_q = S_q^-1 U_q = -dt E S_q^-1 As_up[q]
    gemv_t<T>(SinvT, y + q * nr, wq + q * nr, n, T(1));
    if (q + 1 < nl) {
      T acc[kG][kG] = {};
      grid_gemm<T>(SinvT, Ab, n, acc);
#pragma unroll
      for (int a = 0; a < kG; ++a)
#pragma unroll
        for (int b = 0; b < kG; ++b) {
          const int i = ty + 16 * a, j = tx + 16 * b;
          if (i < n && j < n) {
            const T v = -eE * acc[a][b];
            Xc[i * n + j] = v;
            X[static_cast<size_t>(q) * nn + i * n + j] = v;
          }
        }
      T* t = Xp;
      Xp = Xc;
      Xc = t;
    }
    __syncthreads();
  }
  // back substitution: z_{L-1} = wq_{L-1}; z_q = wq_q - X_q z_{q+1}, a warp per row, lanes across k
  for (int q = nl - 2; q >= 0; --q) {
    const T* Xq = X + static_cast<size_t>(q) * nn;
    for (int r = warp; r < nr; r += kST / 32) {
      T acc = T(0);
      for (int k = lane; k < nr; k += 32) acc += Xq[r * nr + k] * wq[(q + 1) * nr + k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) wq[q * nr + r] -= acc;
    }
    __syncthreads();
  }
  // z - y with y = P_S f again (y held w_q), then f* = f + T_O (z - y)
  for (int e = threadIdx.x; e < nl * nr; e += kST) {
    const int l = e / nr, k = e % nr;
    double s = 0.0;
    for (int a = 0; a < nt; ++a) s += TS[l * nt + a] * f[a * nr + k];
    y[e] = wq[e] - static_cast<T>(s);
  }
  __syncthreads();
  bool bad = false;
  double* out = Fout + static_cast<size_t>(pt) * nv;
  for (int e = threadIdx.x; e < nv; e += kST) {
    const int a = e / nr, k = e % nr;
    double s = 0.0;
    for (int l = 0; l < nl; ++l) s += TO[a * nl + l] * static_cast<double>(y[l * nr + k]);
    const double v = f[e] + s;
    bad |= !isfinite(v);
    out[e] = accumulate ? out[e] + v : v;
  }
  if (bad && status) atomicOr(status, kNonFinite);
}

// ---- the reduced dense system (N_l < N_theta): the same identity with I - dt B_i factored as a
// dense m x m matrix, m = N_l Nr, by the LU kernels of the full system, in its unscaled form
// (I (x) M_v)(I - dt B_i) (LU with partial pivoting on the mass-scaled form meets large element
// growth on fine speed grids). Row and column (l, k) sit at l Nr + k: block (l, l) = M_v - dt Cg_l,
// block (l, l - 1) = -dt E_i Aglo[l], block (l, l + 1) = -dt E_i Agup[l], zero elsewhere.

// (I (x) M_v) G_i, one CTA per row (point i, row (l, p)); columns in blocks of Nr.
template <typename T>
__global__ void v_form_reduced_kernel(const double* __restrict__ Cg, const double* __restrict__ Aglo,
                                      const double* __restrict__ Agup, MassBand mass, const double* __restrict__ E,
                                      double E_uniform, double dt, T* __restrict__ G, int nr, int nl) {
  const int m = nl * nr;
  const size_t rowg = blockIdx.x;  // i * m + row
  const int i = static_cast<int>(rowg / m), row = static_cast<int>(rowg % m);
  const int l = row / nr, p = row % nr;
  const double Ei = E ? E[i] : E_uniform;
  const size_t off = (static_cast<size_t>(l) * nr + p) * nr;
  T* out = G + rowg * m;
  const int bw = 2 * mass.w + 1;
  for (int lc = 0; lc < nl; ++lc) {
    const double* src = lc == l ? Cg : lc == l - 1 ? Aglo : lc == l + 1 ? Agup : nullptr;
    const double w = lc == l ? 1.0 : Ei;
    for (int k = threadIdx.x; k < nr; k += blockDim.x) {
      const double b = src ? w * __ldg(src + off + k) : 0.0;
      const int dk = k - p;
      const double d = lc == l && dk >= -mass.w && dk <= mass.w ? __ldg(mass.m + p * bw + dk + mass.w) : 0.0;
      out[lc * nr + k] = static_cast<T>(d - dt * b);
    }
  }
}

// y_i = P_S f_i: y[l][k] = sum_a T_S[l][a] f[a][k], skipping converged points.
__global__ void reduce_project_kernel(const double* __restrict__ F, const double* __restrict__ TS,
                                      double* __restrict__ Yr, const int* __restrict__ conv, int nt, int nr,
                                      int nl) {
  const int i = blockIdx.x;
  if (conv && conv[i]) return;
  const int m = nl * nr;
  const double* f = F + static_cast<size_t>(i) * nt * nr;
  for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
    const int l = idx / nr, k = idx % nr;
    double s = 0.0;
    for (int a = 0; a < nt; ++a) s = fma(__ldg(TS + l * nt + a), f[a * nr + k], s);
    Yr[static_cast<size_t>(i) * m + idx] = s;
  }
}

// out_i (+)= f_i + P_O (z_i - y_i): out[a][k] = f[a][k] + sum_l T_O[a][l] (z[l][k] - y[l][k]),
// skipping converged points.
__global__ void reduce_lift_kernel(const double* __restrict__ F, const double* __restrict__ Yr,
                                   const double* __restrict__ Zr, const double* __restrict__ TO,
                                   double* __restrict__ out, const int* __restrict__ conv, int accumulate, int nt,
                                   int nr, int nl) {
  const int i = blockIdx.x;
  if (conv && conv[i]) return;
  const int m = nl * nr, nv = nt * nr;
  const size_t base = static_cast<size_t>(i) * nv;
  const double* y = Yr + static_cast<size_t>(i) * m;
  const double* z = Zr + static_cast<size_t>(i) * m;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const int a = v / nr, k = v % nr;
    double s = F[base + v];
    for (int l = 0; l < nl; ++l) s = fma(__ldg(TO + a * nl + l), z[l * nr + k] - y[l * nr + k], s);
    out[base + v] = accumulate ? out[base + v] + s : s;
  }
}

}  // namespace

template <typename T>
void launch_v_form_reduced(const double* Cg, const double* Aglo, const double* Agup, MassBand mass, const double* E,
                           double E_uniform, double dt, T* G, int nx, int nr, int nl, cudaStream_t st) {
  const unsigned rows = static_cast<unsigned>(nx) * nl * nr;
  v_form_reduced_kernel<T><<<rows, nr >= 128 ? 128 : 64, 0, st>>>(Cg, Aglo, Agup, mass, E, E_uniform, dt, G, nr, nl);
}
template void launch_v_form_reduced<float>(const double*, const double*, const double*, MassBand, const double*,
                                           double, double, float*, int, int, int, cudaStream_t);
template void launch_v_form_reduced<double>(const double*, const double*, const double*, MassBand, const double*,
                                            double, double, double*, int, int, int, cudaStream_t);

void launch_reduce_project(const double* F, const double* TS, double* Yr, const int* conv, int nx, int nt, int nr,
                           int nl, cudaStream_t st) {
  reduce_project_kernel<<<nx, 256, 0, st>>>(F, TS, Yr, conv, nt, nr, nl);
}

void launch_reduce_lift(const double* F, const double* Yr, const double* Zr, const double* TO, double* out,
                        const int* conv, int accumulate, int nx, int nt, int nr, int nl, cudaStream_t st) {
  reduce_lift_kernel<<<nx, 256, 0, st>>>(F, Yr, Zr, TO, out, conv, accumulate, nt, nr, nl);
}

size_t struct_smem_bytes(int nr, int nl, size_t tsize) {
  return (4ull * nr * nr + 2ull * nl * nr + nr + 4ull * 64) * tsize;
}

template <typename T>
void launch_vsolve_struct(const double* Fin, double* Fout, const double* E, double E_uniform, double dt,
                          const double* Cs, const double* Alo, const double* Aup, const double* TO, const double* TS,
                          T* Xscratch, int nx, int nt, int nr, int nl, const int* conv, int accumulate,
                          unsigned* status, cudaStream_t st) {
  const size_t smem = struct_smem_bytes(nr, nl, sizeof(T));
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(vsolve_struct_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  vsolve_struct_kernel<T><<<nx, kST, smem, st>>>(Fin, Fout, E, E_uniform, dt, Cs, Alo, Aup, TO, TS, Xscratch, nt, nr, nl,
                                                 conv, accumulate, status);
}

template void launch_vsolve_struct<float>(const double*, double*, const double*, double, double, const double*,
                                          const double*, const double*, const double*, const double*, float*, int, int,
                                          int, int, const int*, int, unsigned*, cudaStream_t);
template void launch_vsolve_struct<double>(const double*, double*, const double*, double, double, const double*,
                                           const double*, const double*, const double*, const double*, double*, int,
                                           int, int, int, const int*, int, unsigned*, cudaStream_t);

}  // namespace bte
