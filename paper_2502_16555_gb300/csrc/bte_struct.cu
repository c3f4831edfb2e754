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
// One CTA of 256 threads per point; four Nr x Nr tiles in shared memory (S^-1, the previous
// X = S^-1 U, the current X, a coupling block), the right-hand sides and intermediate vectors;
// the X_q of the forward sweep go to a per-point global scratch for the back substitution.
#include <cuda_runtime.h>

#include "bte_kernels.h"

namespace bte {
namespace {

constexpr int kST = 256;  // threads per CTA

// C = alpha * A B (+ C if accumulate) for n x n row-major tiles in shared memory (ld = n), 4 x 4
// register tiles over the 256 threads (edges masked).
template <typename T, typename TA>
__device__ void tile_gemm(const TA* A, const T* B, T* C, int n, T alpha, bool accumulate) {
  const int tn = (n + 3) / 4;
  for (int tt = threadIdx.x; tt < tn * tn; tt += kST) {
    const int ti = tt / tn, tj = tt % tn;
    T acc[4][4] = {};
    for (int k = 0; k < n; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = 4 * ti + r < n ? static_cast<T>(A[(4 * ti + r) * n + k]) : T(0);
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = 4 * tj + c < n ? B[k * n + 4 * tj + c] : T(0);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (4 * ti + r < n && 4 * tj + c < n) {
          T& o = C[(4 * ti + r) * n + 4 * tj + c];
          o = accumulate ? o + alpha * acc[r][c] : alpha * acc[r][c];
        }
      }
  }
}

// In-place inverse of the n x n tile S by Gauss-Jordan elimination without pivoting. The threads
// form a 16 x 16 grid over the tile (element (i, j) belongs to thread (i % 16, j % 16)). Per step k
// every element reads the pivot row and column of step k from a copy (double-buffered by step
// parity), and the threads owning row k + 1 and column k + 1 write those copies for the next
// step as they update them, so one barrier per step suffices.
template <typename T>
__device__ void gauss_jordan_inverse(T* S, int n, T* prow2, T* pcol2) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int j = threadIdx.x; j < n; j += kST) prow2[j] = S[j], pcol2[j] = S[j * n];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const T* prow = prow2 + (k & 1) * n;
    const T* pcol = pcol2 + (k & 1) * n;
    T* nrow = prow2 + ((k + 1) & 1) * n;
    T* ncol = pcol2 + ((k + 1) & 1) * n;
    const T p = T(1) / prow[k];
    for (int i = ty; i < n; i += 16) {
      const T fi = pcol[i] * p;
      for (int j = tx; j < n; j += 16) {
        T v;
        if (i == k) v = (j == k) ? p : prow[j] * p;
        else if (j == k) v = -fi;
        else v = S[i * n + j] - fi * prow[j];
        S[i * n + j] = v;
        if (i == k + 1) nrow[j] = v;
        if (j == k + 1) ncol[i] = v;
      }
    }
    __syncthreads();
  }
}

// y[w] (+)= alpha * sum_k M[w][k] x[k], n x n tile M, one warp-stride thread per output row.
template <typename T>
__device__ void tile_gemv(const T* M, const T* x, T* y, int n, T alpha, bool accumulate) {
  for (int i = threadIdx.x; i < n; i += kST) {
    T acc = T(0);
    for (int k = 0; k < n; ++k) acc += M[i * n + k] * x[k];
    y[i] = accumulate ? y[i] + alpha * acc : alpha * acc;
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
  const int i = blockIdx.x;
  if (conv && conv[i]) return;
  const int n = nr, nn = nr * nr, nv = nt * nr;
  T* Sinv = reinterpret_cast<T*>(smraw);
  T* Xp = Sinv + nn;        // previous X = S^-1 U
  T* Xc = Xp + nn;          // current X
  T* Ab = Xc + nn;          // coupling block
  T* y = Ab + nn;           // nl x nr: P_S f
  T* wq = y + nl * nr;      // nl x nr: S_q^-1 w_q
  T* tmp = wq + nl * nr;    // nr
  T* prow = tmp + nr;       // 2 nr (double-buffered pivot rows)
  T* pcol = prow + 2 * nr;  // 2 nr
  const double* f = Fin + static_cast<size_t>(i) * nv;
  const T eE = static_cast<T>(dt * (E ? E[i] : E_uniform));
  T* X = Xg + static_cast<size_t>(i) * nl * nn;

  // y = T_S f (per radial index)
  for (int e = threadIdx.x; e < nl * nr; e += kST) {
    const int l = e / nr, k = e % nr;
    double s = 0.0;
    for (int a = 0; a < nt; ++a) s += TS[l * nt + a] * f[a * nr + k];
    y[e] = static_cast<T>(s);
  }
  __syncthreads();
  for (int q = 0; q < nl; ++q) {
    // S_q = I - dt Cs_q - L_q X_{q-1} = I - dt Cs_q + dt E As_lo[q] X_{q-1};  w_q = y_q + dt E As_lo[q] wq_{q-1}
    const double* C = Cs + static_cast<size_t>(q) * nn;
    for (int e = threadIdx.x; e < nn; e += kST) Sinv[e] = (e / n == e % n ? T(1) : T(0)) - static_cast<T>(dt * C[e]);
    __syncthreads();
    if (q > 0) {
      const double* Al = Alo + static_cast<size_t>(q) * nn;
      for (int e = threadIdx.x; e < nn; e += kST) Ab[e] = static_cast<T>(Al[e]);
      __syncthreads();
      tile_gemm<T, T>(Ab, Xp, Sinv, n, eE, true);
      tile_gemv<T>(Ab, wq + (q - 1) * nr, tmp, n, eE, false);
      __syncthreads();
      for (int k = threadIdx.x; k < nr; k += kST) y[q * nr + k] += tmp[k];  // y_q now holds w_q
      __syncthreads();
    }
    gauss_jordan_inverse<T>(Sinv, n, prow, pcol);
    // wq_q = S_q^-1 w_q;  X_q = S_q^-1 U_q = -dt E S_q^-1 As_up[q]
    tile_gemv<T>(Sinv, y + q * nr, wq + q * nr, n, T(1), false);
    if (q + 1 < nl) {
      const double* Au = Aup + static_cast<size_t>(q) * nn;
      for (int e = threadIdx.x; e < nn; e += kST) Ab[e] = static_cast<T>(Au[e]);
      __syncthreads();
      tile_gemm<T, T>(Sinv, Ab, Xc, n, -eE, false);
      __syncthreads();
      for (int e = threadIdx.x; e < nn; e += kST) X[static_cast<size_t>(q) * nn + e] = Xc[e];
      T* t = Xp;
      Xp = Xc;
      Xc = t;
    }
    __syncthreads();
  }
  // back substitution: z_{L-1} = wq_{L-1}; z_q = wq_q - X_q z_{q+1}  (z overwrites wq)
  for (int q = nl - 2; q >= 0; --q) {
    const T* Xq = X + static_cast<size_t>(q) * nn;
    for (int e = threadIdx.x; e < nn; e += kST) Xc[e] = Xq[e];  // coalesced staging
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += kST) {
      T acc = T(0);
      for (int k = 0; k < nr; ++k) acc += Xc[r * nr + k] * wq[(q + 1) * nr + k];
      wq[q * nr + r] -= acc;
    }
    __syncthreads();
  }
  // restore y = P_S f (it held w_q) and form f* = f + T_O (z - y)
  for (int e = threadIdx.x; e < nl * nr; e += kST) {
    const int l = e / nr, k = e % nr;
    double s = 0.0;
    for (int a = 0; a < nt; ++a) s += TS[l * nt + a] * f[a * nr + k];
    y[e] = wq[e] - static_cast<T>(s);  // z - y
  }
  __syncthreads();
  bool bad = false;
  double* out = Fout + static_cast<size_t>(i) * nv;
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

}  // namespace

size_t struct_smem_bytes(int nr, int nl, size_t tsize) {
  return (4ull * nr * nr + 2ull * nl * nr + 5ull * nr) * tsize;
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
