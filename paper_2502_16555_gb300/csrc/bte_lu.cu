// Batched dense LU with partial pivoting of the per-point velocity-step matrices
// A_i = I - dt (K_C + E_i K_A)  (eq. "vspace_batched_system" of arXiv 2502.16555), and the
// triangular solves. The paper solves these systems with GMRES; a direct factorisation reaches the
// same unique solution.
//
// Right-looking blocked LU, one launch sequence per outer panel of width nb, batched over the Nx
// points (blockIdx.x / blockIdx.z = point):
//   lu_panel      factor A[k0:n, k0:k0+nb] (sub-panels of width W staged in shared memory), record
//                 the pivots, the resulting row permutation of the panel rows, and inv(L11);
//   lu_swap_trsm  apply the panel's row permutation to the trailing columns and form
//                 U12 = inv(L11) P A12;
//   gemm          A22 -= L21 U12 (SIMT here; the FP32 path has a tcgen05 tensor-core version).
// Row swaps are not applied to the columns left of a panel ("lazy" swaps): the forward solve
// applies each panel's pivots to the right-hand side just before eliminating with that panel's
// columns, which is the same elimination order the factorisation used.
#include <cuda_runtime.h>

#include <cstdint>

#include "bte_kernels.h"
#include "bte_tf32.cuh"

namespace bte {
namespace {

template <typename T>
__device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }

// Per-point panel record (ints): [0] number of displaced rows d, [1 .. nbmax] final origin row of
// panel rows k0..k0+nb-1, then d pairs (destination row >= k0+nb, origin row in [k0, k0+nb)).
__host__ __device__ constexpr int perm_stride(int nbmax) { return 1 + nbmax + 2 * nbmax; }

template <typename T>
__global__ void __launch_bounds__(512) lu_panel_kernel(T* __restrict__ fac, int* __restrict__ piv,
                                                       int* __restrict__ perm, T* __restrict__ linv,
                                                       int n, int k0, int nb, int nbmax, int W,
                                                       unsigned* status, float* __restrict__ ws_hi,
                                                       float* __restrict__ ws_lo) {
  extern __shared__ unsigned char smraw[];
  const int ld = W + 1;
  T* S = reinterpret_cast<T*>(smraw);                                 // (n-k0) x ld
  int* orig = reinterpret_cast<int*>(S + static_cast<size_t>(n - k0) * ld);  // n-k0
  __shared__ T red_v[16];
  __shared__ int red_i[16];
  __shared__ int s_pr;
  __shared__ int s_cnt;

  const int mat = blockIdx.x;
  T* A = fac + static_cast<size_t>(mat) * n * n;
  int* ip = piv + static_cast<size_t>(mat) * n;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;

  for (int r = tid; r < n - k0; r += bd) orig[r] = k0 + r;
  bool bad_pivot = false;

  for (int c0 = k0; c0 < k0 + nb; c0 += W) {
    const int w = min(W, k0 + nb - c0);
    const int m = n - c0;
    for (int idx = tid; idx < m * w; idx += bd) {
      const int r = idx / w, jj = idx % w;
      S[r * ld + jj] = A[static_cast<size_t>(c0 + r) * n + c0 + jj];
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
      // pivot: largest |S[r][j]|, r >= j; ties go to the smaller row
      T best = T(-1);
      int bi = j;
      for (int r = j + tid; r < m; r += bd) {
        const T v = tabs(S[r * ld + j]);
        if (v > best) best = v, bi = r;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
      }
      if (lane == 0) red_v[warp] = best, red_i[warp] = bi;
      __syncthreads();
      if (warp == 0) {
        best = lane < (bd >> 5) ? red_v[lane] : T(-1);
        bi = lane < (bd >> 5) ? red_i[lane] : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T ov = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
        }
        if (lane == 0) s_pr = (bi >= j && bi < m) ? bi : j;
      }
      __syncthreads();
      const int pr = s_pr;
      if (tid == 0) ip[c0 + j] = c0 + pr;
      if (pr != j) {
        for (int jj = tid; jj < w; jj += bd) {
          const T t = S[j * ld + jj];
          S[j * ld + jj] = S[pr * ld + jj];
          S[pr * ld + jj] = t;
        }
        const int nleft = c0 - k0, nright = k0 + nb - (c0 + w);
        for (int q = tid; q < nleft + nright; q += bd) {
          const int col = q < nleft ? k0 + q : c0 + w + (q - nleft);
          T* a1 = A + static_cast<size_t>(c0 + j) * n + col;
          T* a2 = A + static_cast<size_t>(c0 + pr) * n + col;
          const T t = *a1;
          *a1 = *a2;
          *a2 = t;
        }
        if (tid == 0) {
          const int t = orig[c0 + j - k0];
          orig[c0 + j - k0] = orig[c0 + pr - k0];
          orig[c0 + pr - k0] = t;
        }
      }
      __syncthreads();
      const T pv = S[j * ld + j];
      if (tid == 0 && (!(tabs(pv) > T(0)) || !isfinite(static_cast<double>(pv)))) bad_pivot = true;
      const T inv = (pv != T(0)) ? T(1) / pv : T(0);
      for (int r = j + 1 + tid; r < m; r += bd) {
        const T l = S[r * ld + j] * inv;
        S[r * ld + j] = l;
        for (int jj = j + 1; jj < w; ++jj) S[r * ld + jj] -= l * S[j * ld + jj];
      }
      __syncthreads();
    }
    for (int idx = tid; idx < m * w; idx += bd) {
      const int r = idx / w, jj = idx % w;
      A[static_cast<size_t>(c0 + r) * n + c0 + jj] = S[r * ld + jj];
    }
    __syncthreads();
    // right-looking update of the not yet factored columns of this outer panel
    const int rw = k0 + nb - (c0 + w);
    if (rw > 0) {
      const int cb = c0 + w;
      for (int col = tid; col < rw; col += bd) {
        for (int jr = 1; jr < w; ++jr) {
          T x = A[static_cast<size_t>(c0 + jr) * n + cb + col];
          for (int jj = 0; jj < jr; ++jj) x -= S[jr * ld + jj] * A[static_cast<size_t>(c0 + jj) * n + cb + col];
          A[static_cast<size_t>(c0 + jr) * n + cb + col] = x;
        }
      }
      __syncthreads();
      for (int idx = tid; idx < (m - w) * rw; idx += bd) {
        const int r = w + idx / rw, col = idx % rw;
        T acc = A[static_cast<size_t>(c0 + r) * n + cb + col];
        for (int jj = 0; jj < w; ++jj) acc -= S[r * ld + jj] * A[static_cast<size_t>(c0 + jj) * n + cb + col];
        A[static_cast<size_t>(c0 + r) * n + cb + col] = acc;
      }
      __syncthreads();
    }
  }
  if (tid == 0 && bad_pivot) atomicOr(status, kZeroPivot);

  // permutation record for the trailing columns
  int* pr_rec = perm + static_cast<size_t>(mat) * perm_stride(nbmax);
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int j = tid; j < nb; j += bd) pr_rec[1 + j] = orig[j];
  for (int r = nb + tid; r < n - k0; r += bd) {
    if (orig[r] != k0 + r) {
      const int slot = atomicAdd(&s_cnt, 1);
      pr_rec[1 + nbmax + 2 * slot] = k0 + r;
      pr_rec[1 + nbmax + 2 * slot + 1] = orig[r];
    }
  }
  __syncthreads();
  if (tid == 0) pr_rec[0] = s_cnt;

  // L21 split into TF32 head/remainder for the tensor-core trailing update ([point][row][nbmax])
  if (ws_hi) {
    const int M = n - k0 - nb;
    float* hi = ws_hi + static_cast<size_t>(mat) * (n - nbmax) * nbmax;
    float* lo = ws_lo + static_cast<size_t>(mat) * (n - nbmax) * nbmax;
    for (int idx = tid; idx < M * nb; idx += bd) {
      const int r = idx / nb, k = idx % nb;
      float h, l;
      split_tf32(static_cast<float>(A[static_cast<size_t>(k0 + nb + r) * n + k0 + k]), h, l);
      hi[static_cast<size_t>(r) * nbmax + k] = h;
      lo[static_cast<size_t>(r) * nbmax + k] = l;
    }
  }

  // inv(L11), L11 = unit lower part of A[k0:k0+nb, k0:k0+nb]
  T* X = linv + static_cast<size_t>(mat) * nbmax * nbmax;
  for (int c = tid; c < nb; c += bd) {
    for (int r = 0; r < c; ++r) X[r * nbmax + c] = T(0);
    X[c * nbmax + c] = T(1);
    for (int r = c + 1; r < nb; ++r) {
      T s = T(0);
      for (int j = c; j < r; ++j) s += A[static_cast<size_t>(k0 + r) * n + k0 + j] * X[j * nbmax + c];
      X[r * nbmax + c] = -s;
    }
  }
}

constexpr int kTrsmCols = 64;
constexpr int kTrsmLd = kTrsmCols + 1;  // padded smem row (transposed reads)

template <typename T>
__global__ void __launch_bounds__(256) lu_swap_trsm_kernel(T* __restrict__ fac, const int* __restrict__ perm,
                                                           const T* __restrict__ linv, int n, int k0,
                                                           int nb, int nbmax, float* __restrict__ ws_hi,
                                                           float* __restrict__ ws_lo) {
  extern __shared__ unsigned char smraw[];
  T* top = reinterpret_cast<T*>(smraw);                 // original panel rows, later U12   nb x ld
  T* Bs = top + static_cast<size_t>(nb) * kTrsmLd;       // permuted panel rows             nb x ld
  const int mat = blockIdx.x;
  const int C0 = k0 + nb + blockIdx.y * kTrsmCols;
  const int ncol = min(kTrsmCols, n - C0);
  T* A = fac + static_cast<size_t>(mat) * n * n;
  const int* rec = perm + static_cast<size_t>(mat) * perm_stride(nbmax);
  const T* X = linv + static_cast<size_t>(mat) * nbmax * nbmax;
  const int tid = threadIdx.x, bd = blockDim.x;
  // read phase: original panel rows, and the final content of the panel rows
  for (int idx = tid; idx < nb * kTrsmCols; idx += bd) {
    const int r = idx / kTrsmCols, c = idx % kTrsmCols;
    top[r * kTrsmLd + c] = c < ncol ? A[static_cast<size_t>(k0 + r) * n + C0 + c] : T(0);
    const int o = rec[1 + r];
    Bs[r * kTrsmLd + c] = c < ncol ? A[static_cast<size_t>(o) * n + C0 + c] : T(0);
  }
  __syncthreads();
  // write phase: rows pushed below the panel receive their original panel row
  const int d = rec[0];
  for (int idx = tid; idx < d * kTrsmCols; idx += bd) {
    const int q = idx / kTrsmCols, c = idx % kTrsmCols;
    if (c >= ncol) continue;
    const int dst = rec[1 + nbmax + 2 * q], src = rec[1 + nbmax + 2 * q + 1];
    A[static_cast<size_t>(dst) * n + C0 + c] = top[(src - k0) * kTrsmLd + c];
  }
  __syncthreads();
  // U12 = inv(L11) P A12 (inv(L11) unit lower), staged in `top`
  for (int idx = tid; idx < nb * kTrsmCols; idx += bd) {
    const int r = idx / kTrsmCols, c = idx % kTrsmCols;
    T s = Bs[r * kTrsmLd + c];
    for (int j = 0; j < r; ++j) s += X[r * nbmax + j] * Bs[j * kTrsmLd + c];
    top[r * kTrsmLd + c] = s;
  }
  __syncthreads();
  for (int idx = tid; idx < nb * kTrsmCols; idx += bd) {
    const int r = idx / kTrsmCols, c = idx % kTrsmCols;
    if (c < ncol) A[static_cast<size_t>(k0 + r) * n + C0 + c] = top[r * kTrsmLd + c];
  }
  // U12 transposed (K-major) and split for the tensor-core trailing update
  if (ws_hi) {
    const size_t off = static_cast<size_t>(mat) * (n - nbmax) * nbmax;
    for (int idx = tid; idx < kTrsmCols * nb; idx += bd) {
      const int c = idx / nb, r = idx % nb;
      if (c >= ncol) continue;
      float h, l;
      split_tf32(static_cast<float>(top[r * kTrsmLd + c]), h, l);
      const size_t o = off + static_cast<size_t>(C0 - (k0 + nb) + c) * nbmax + r;
      ws_hi[o] = h;
      ws_lo[o] = l;
    }
  }
}

// C -= A B on the trailing block: C = A22 (rows/cols k0+nb..n), A = L21, B = U12. Tile BM x BN,
// 256 threads with a 16 x 16 layout, each owning a TM x TN register tile.
template <typename T, int BM, int BN, int BK>
__global__ void __launch_bounds__(256) lu_gemm_simt_kernel(T* __restrict__ fac, int n, int k0, int nb) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  const int mat = blockIdx.z;
  T* A = fac + static_cast<size_t>(mat) * n * n;
  const int base = k0 + nb;
  const int M = n - base;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  for (int kk = 0; kk < nb; kk += BK) {
    for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
      const int r = idx / BK, k = idx % BK;
      const int gr = row0 + r, gk = kk + k;
      As[k][r] = (gr < M && gk < nb) ? A[static_cast<size_t>(base + gr) * n + k0 + gk] : T(0);
    }
    for (int idx = threadIdx.x; idx < BK * BN; idx += 256) {
      const int k = idx / BN, c = idx % BN;
      const int gc = col0 + c, gk = kk + k;
      Bs[k][c] = (gc < M && gk < nb) ? A[static_cast<size_t>(k0 + gk) * n + base + gc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = row0 + ty + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gc = col0 + tx + 16 * j;
      if (gc < M) A[static_cast<size_t>(base + gr) * n + base + gc] -= acc[i][j];
    }
  }
}

// x = A^-1 b for one point per CTA, with the lazily applied pivots; Tc is the arithmetic type.
template <typename T, typename Tc>
__global__ void __launch_bounds__(1024) lu_solve_kernel(const T* __restrict__ fac, const int* __restrict__ piv,
                                                        const double* __restrict__ b, double* __restrict__ x,
                                                        int n, int nb, const int* __restrict__ conv,
                                                        int accumulate) {
  extern __shared__ unsigned char smraw[];
  Tc* s = reinterpret_cast<Tc*>(smraw);
  const int mat = blockIdx.x;
  if (conv && conv[mat]) return;
  const T* A = fac + static_cast<size_t>(mat) * n * n;
  const int* ip = piv + static_cast<size_t>(mat) * n;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int r = tid; r < n; r += bd) s[r] = static_cast<Tc>(b[static_cast<size_t>(mat) * n + r]);
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = min(nb, n - k0);
    if (tid == 0)
      for (int j = 0; j < kb; ++j) {
        const int p = ip[k0 + j];
        if (p != k0 + j) {
          const Tc t = s[k0 + j];
          s[k0 + j] = s[p];
          s[p] = t;
        }
      }
    __syncthreads();
    for (int j0 = k0; j0 < k0 + kb; j0 += 32) {
      const int cw = min(32, k0 + kb - j0);
      if (warp == 0) {
        Tc v = lane < cw ? s[j0 + lane] : Tc(0);
        for (int jj = 0; jj < cw; ++jj) {
          const Tc xj = __shfl_sync(0xffffffffu, v, jj);
          if (lane > jj && lane < cw) v -= static_cast<Tc>(A[static_cast<size_t>(j0 + lane) * n + j0 + jj]) * xj;
        }
        if (lane < cw) s[j0 + lane] = v;
      }
      __syncthreads();
      for (int r = j0 + cw + tid; r < n; r += bd) {
        const T* a = A + static_cast<size_t>(r) * n + j0;
        Tc acc = Tc(0);
        for (int jj = 0; jj < cw; ++jj) acc += static_cast<Tc>(a[jj]) * s[j0 + jj];
        s[r] -= acc;
      }
      __syncthreads();
    }
  }
  for (int j0 = ((n - 1) / 32) * 32; j0 >= 0; j0 -= 32) {
    const int cw = min(32, n - j0);
    if (warp == 0) {
      Tc v = lane < cw ? s[j0 + lane] : Tc(0);
      for (int jj = cw - 1; jj >= 0; --jj) {
        if (lane == jj) v /= static_cast<Tc>(A[static_cast<size_t>(j0 + jj) * n + j0 + jj]);
        const Tc xj = __shfl_sync(0xffffffffu, v, jj);
        if (lane < jj) v -= static_cast<Tc>(A[static_cast<size_t>(j0 + lane) * n + j0 + jj]) * xj;
      }
      if (lane < cw) s[j0 + lane] = v;
    }
    __syncthreads();
    for (int r = tid; r < j0; r += bd) {
      const T* a = A + static_cast<size_t>(r) * n + j0;
      Tc acc = Tc(0);
      for (int jj = 0; jj < cw; ++jj) acc += static_cast<Tc>(a[jj]) * s[j0 + jj];
      s[r] -= acc;
    }
    __syncthreads();
  }
  double* xo = x + static_cast<size_t>(mat) * n;
  for (int r = tid; r < n; r += bd) xo[r] = accumulate ? xo[r] + static_cast<double>(s[r]) : static_cast<double>(s[r]);
}

}  // namespace

// sub-panel width: largest power of two <= 32 whose staging buffer fits the shared-memory budget
template <typename T>
static int panel_width(int n, int nb) {
  int w = 32;
  while (w > 1 && (static_cast<size_t>(n) * (w + 1) * sizeof(T) + n * sizeof(int)) > 200 * 1024) w >>= 1;
  return w < nb ? w : nb;
}

template <typename T>
void launch_lu_panel(T* fac, int* piv, int* perm, T* linv, int nx, int n, int k0, int nb, int nbmax,
                     unsigned* status, float* ws_hi, float* ws_lo, cudaStream_t st) {
  const int W = panel_width<T>(n, nbmax);
  const size_t smem = static_cast<size_t>(n - k0) * (W + 1) * sizeof(T) + (n - k0) * sizeof(int);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  lu_panel_kernel<T><<<nx, 512, smem, st>>>(fac, piv, perm, linv, n, k0, nb, nbmax, W, status,
                                             k0 + nb < n ? ws_hi : nullptr, ws_lo);
}

template <typename T>
void launch_lu_swap_trsm(T* fac, const int* perm, const T* linv, int nx, int n, int k0, int nb,
                         int nbmax, float* ws_hi, float* ws_lo, cudaStream_t st) {
  const int ntrail = n - k0 - nb;
  if (ntrail <= 0) return;
  dim3 grid(nx, (ntrail + kTrsmCols - 1) / kTrsmCols);
  const size_t smem = 2 * static_cast<size_t>(nb) * kTrsmLd * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_swap_trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  lu_swap_trsm_kernel<T><<<grid, 256, smem, st>>>(fac, perm, linv, n, k0, nb, nbmax, ws_hi, ws_lo);
}

template <typename T>
void launch_lu_gemm_simt(T* fac, int nx, int n, int k0, int nb, cudaStream_t st) {
  const int M = n - k0 - nb;
  if (M <= 0) return;
  if (sizeof(T) == 8) {
    dim3 grid((M + 63) / 64, (M + 63) / 64, nx);
    lu_gemm_simt_kernel<T, 64, 64, 16><<<grid, 256, 0, st>>>(fac, n, k0, nb);
  } else {
    dim3 grid((M + 127) / 128, (M + 127) / 128, nx);
    lu_gemm_simt_kernel<T, 128, 128, 8><<<grid, 256, 0, st>>>(fac, n, k0, nb);
  }
}

template <typename T>
void launch_lu_solve(const T* fac, const int* piv, const double* b, double* x, int nx, int n, int nb,
                     const int* conv, int accumulate, cudaStream_t st) {
  using Tc = T;
  const size_t smem = static_cast<size_t>(n) * sizeof(Tc);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_solve_kernel<T, Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr_set = true;
  }
  lu_solve_kernel<T, Tc><<<nx, 1024, smem, st>>>(fac, piv, b, x, n, nb, conv, accumulate);
}

int perm_record_ints(int nbmax) { return perm_stride(nbmax); }

#define BTE_INST(T)                                                                                 \
  template void launch_lu_panel<T>(T*, int*, int*, T*, int, int, int, int, int, unsigned*, float*, float*, \
                                   cudaStream_t);                                                   \
  template void launch_lu_swap_trsm<T>(T*, const int*, const T*, int, int, int, int, int, float*, float*, \
                                       cudaStream_t);                                               \
  template void launch_lu_gemm_simt<T>(T*, int, int, int, int, cudaStream_t);                       \
  template void launch_lu_solve<T>(const T*, const int*, const double*, double*, int, int, int,     \
                                   const int*, int, cudaStream_t);
BTE_INST(double)
BTE_INST(float)
#undef BTE_INST

}  // namespace bte
