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

// Shared-memory plan of lu_panel (elements of T unless noted):
//   R0   max(m0 * (W+1), 2 * nb * (nb+1))   sub-panel S (later L11 and inv(L11) staging)
//   U    W * nbmax                          U rows of the current sub-panel, right part
//   SB   2W * nbmax                         row-swap staging of the other panel columns
//   ints m0 (orig) + W (local pivots) + 2W (slot rows) + 2W (slot contents)
template <typename T>
__host__ __device__ inline size_t panel_smem_bytes(int m0, int nb, int nbmax, int W) {
  size_t r0 = static_cast<size_t>(m0) * (W + 1);
  const size_t linv = 2ull * nb * (nb + 1);
  if (linv > r0) r0 = linv;
  const size_t elems = r0 + static_cast<size_t>(W) * nbmax + 2ull * W * nbmax;
  return elems * sizeof(T) + (static_cast<size_t>(m0) + 5 * W) * sizeof(int) + 16;
}

constexpr int kColWarps = 8;  // warps running the column-by-column elimination of a sub-panel
constexpr int kLoadBatch = 8; // independent global loads in flight per thread in copy loops

// inv(L) for a unit-lower (kLower) or inv(U) for an upper triangular nb x nb matrix held in shared
// memory (row stride ldl), by row blocks R of 16: the 16 x 16 diagonal blocks are inverted first
// (one warp each, lane = column, registers), then row block by row block (downwards for L, upwards
// for U) X[R, rest] = -inv(D_RR) (D[R, between] X[between, rest]) as two parallel products.
// All threads of the block; X must not alias D.
template <typename T, bool kLower>
__device__ void tri_inverse_smem(const T* D, T* X, int nb, int ldl) {
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = bd >> 5;
  const int nblk = (nb + 15) / 16;
  for (int idx = tid; idx < nb * nb; idx += bd) X[(idx / nb) * ldl + idx % nb] = T(0);
  __syncthreads();
  // diagonal blocks: X[R,R] = inv(D[R,R]); lanes 0..15 one block, 16..31 the next
  for (int pb = warp * 2; pb < nblk; pb += nwarp * 2) {
    const int blk = pb + (lane >> 4), c = lane & 15;
    const int r0 = 16 * blk, rb = blk < nblk ? min(16, nb - r0) : 0;
    T x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = T(0);
    if (c < rb) {
      if (kLower) {
        x[c] = T(1);
#pragma unroll
        for (int r = 1; r < 16; ++r) {
          if (r > c && r < rb) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (k >= c && k < r) acc += D[(r0 + r) * ldl + r0 + k] * x[k];
            x[r] = -acc;
          }
        }
      } else {
#pragma unroll
        for (int r = 15; r >= 0; --r) {
          if (r <= c) {
            T acc = (r == c) ? T(1) : T(0);
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (k > r && k <= c) acc -= D[(r0 + r) * ldl + r0 + k] * x[k];
            x[r] = acc / D[(r0 + r) * ldl + r0 + r];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (r < rb) X[(r0 + r) * ldl + r0 + c] = x[r];
    }
  }
  __syncthreads();
  // off-diagonal row blocks; the product D[R, between] X[between, rest] is staged in T1, the rows
  // of X below (L) or above (U) the diagonal blocks' area are still zero and serve as scratch
  T* T1 = X;  // write target rows R of X directly after the second product
  (void)T1;
  for (int bi = 1; bi < nblk; ++bi) {
    const int blk = kLower ? bi : nblk - 1 - bi;
    const int r0 = 16 * blk, r1 = min(nb, r0 + 16), rb = r1 - r0;
    // columns of X in row block R still to fill: [0, r0) for L, [r1, nb) for U
    const int c_lo = kLower ? 0 : r1, c_hi = kLower ? r0 : nb, ncol = c_hi - c_lo;
    // acc[r][c] = sum over k between of D[r][k] X[k][c]; stored temporarily in X[r][c]
    for (int idx = tid; idx < rb * ncol; idx += bd) {
      const int r = r0 + idx / ncol, c = c_lo + idx % ncol;
      T acc = T(0);
      if (kLower) {
        for (int k = c; k < r0; ++k) acc += D[r * ldl + k] * X[k * ldl + c];
      } else {
        for (int k = r1; k <= c; ++k) acc += D[r * ldl + k] * X[k * ldl + c];
      }
      X[r * ldl + c] = acc;
    }
    __syncthreads();
    // X[R, cols] = -inv(D_RR) acc: each thread one column, the 16 rows in registers
    for (int c = c_lo + tid; c < c_hi; c += bd) {
      T v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = i < rb ? X[(r0 + i) * ldl + c] : T(0);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (i < rb) {
          T acc = T(0);
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (k < rb) acc += X[(r0 + i) * ldl + r0 + k] * v[k];
          X[(r0 + i) * ldl + c] = -acc;
        }
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) lu_panel_kernel(T* __restrict__ fac, int* __restrict__ piv,
                                                       int* __restrict__ perm, T* __restrict__ linv,
                                                       int n, int k0, int nb, int nbmax, int W,
                                                       unsigned* status, float* __restrict__ ws_hi,
                                                       float* __restrict__ ws_lo, float* __restrict__ li_hi,
                                                       float* __restrict__ li_lo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = W + 1;
  const int m0 = n - k0;
  size_t r0sz = static_cast<size_t>(m0) * ld;
  if (static_cast<size_t>(2) * nb * (nb + 1) > r0sz) r0sz = static_cast<size_t>(2) * nb * (nb + 1);
  T* S = reinterpret_cast<T*>(smraw);
  T* Ub = S + r0sz;
  T* SB = Ub + static_cast<size_t>(W) * nbmax;
  int* orig = reinterpret_cast<int*>(SB + static_cast<size_t>(2) * W * nbmax);
  int* lp = orig + m0;              // local pivots of the current sub-panel (relative to c0)
  int* slot_row = lp + W;           // rows of the swap slots (2W)
  int* content = slot_row + 2 * W;  // 2W
  __shared__ T red_v[kColWarps];
  __shared__ int red_i[kColWarps];
  __shared__ int s_pr, s_cnt, s_nslot;
  __shared__ int pslot[32];

  const int mat = blockIdx.x;
  T* A = fac + static_cast<size_t>(mat) * n * n;
  int* ip = piv + static_cast<size_t>(mat) * n;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int npan = (n + nbmax - 1) / nbmax, pan = k0 / nbmax;
  constexpr int kColThreads = kColWarps * 32;

  for (int r = tid; r < m0; r += bd) orig[r] = k0 + r;
  bool bad_pivot = false;

  // argmax over the column warps: larger |v| wins, ties to the smaller row; result in s_pr,
  // published by the next column barrier
  auto col_sync = []() { asm volatile("bar.sync 1, %0;" ::"r"(kColThreads) : "memory"); };
  auto col_argmax = [&](T best, int bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
    }
    if (lane == 0) red_v[warp] = best, red_i[warp] = bi;
    col_sync();
    if (warp == 0) {
      best = lane < kColWarps ? red_v[lane] : T(-1);
      bi = lane < kColWarps ? red_i[lane] : 0x7fffffff;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
      }
      if (lane == 0) s_pr = bi;
    }
  };

  for (int c0 = k0; c0 < k0 + nb; c0 += W) {
    const int w = min(W, k0 + nb - c0);
    const int m = n - c0;
    for (int base = tid; base < m * w; base += bd * kLoadBatch) {
      T v[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = base + u * bd;
        v[u] = idx < m * w ? A[static_cast<size_t>(c0 + idx / w) * n + c0 + idx % w] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = base + u * bd;
        if (idx < m * w) S[(idx / w) * ld + idx % w] = v[u];
      }
    }
    __syncthreads();
    if (warp < kColWarps) {
      {
        T best = T(-1);
        int bi = 0;
        for (int r = tid; r < m; r += kColThreads) {
          const T v = tabs(S[r * ld]);
          if (v > best) best = v, bi = r;
        }
        col_argmax(best, bi);
      }
      for (int j = 0; j < w; ++j) {
        col_sync();  // s_pr of column j is published
        int pr = s_pr;
        if (pr < j || pr >= m) pr = j;
        if (pr != j)
          for (int jj = tid; jj < w; jj += kColThreads) {
            const T t = S[j * ld + jj];
            S[j * ld + jj] = S[pr * ld + jj];
            S[pr * ld + jj] = t;
          }
        if (tid == 0) lp[j] = pr;
        col_sync();  // pivot row in place
        const T pv = S[j * ld + j];
        if (tid == 0 && (!(tabs(pv) > T(0)) || !isfinite(static_cast<double>(pv)))) bad_pivot = true;
        const T inv = (pv != T(0)) ? T(1) / pv : T(0);
        T best = T(-1);
        int bi = j + 1;
        for (int r = j + 1 + tid; r < m; r += kColThreads) {
          const T l = S[r * ld + j] * inv;
          S[r * ld + j] = l;
          for (int jj = j + 1; jj < w; ++jj) S[r * ld + jj] -= l * S[j * ld + jj];
          if (j + 1 < w) {
            const T v = tabs(S[r * ld + j + 1]);
            if (v > best) best = v, bi = r;
          }
        }
        if (j + 1 < w) col_argmax(best, bi);
      }
    }
    __syncthreads();
    for (int idx = tid; idx < m * w; idx += bd) {
      const int r = idx / w, jj = idx % w;
      A[static_cast<size_t>(c0 + r) * n + c0 + jj] = S[r * ld + jj];
    }
    // the sub-panel's row permutation, as slots: slot k < w is row c0+k, further slots are the
    // distinct pivot rows below the sub-panel; content[k] = slot whose original row ends in slot k
    if (tid == 0) {
      int ns = w;
      for (int k = 0; k < w; ++k) slot_row[k] = c0 + k;
      for (int j = 0; j < w; ++j) {
        const int p = lp[j];
        int sl = p;
        if (p >= w) {
          sl = -1;
          for (int q = w; q < ns; ++q)
            if (slot_row[q] == c0 + p) sl = q;
          if (sl < 0) slot_row[sl = ns++] = c0 + p;
        }
        pslot[j] = sl;
        ip[c0 + j] = c0 + p;
        const int a = c0 + j - k0, b = c0 + p - k0;
        const int t = orig[a];
        orig[a] = orig[b];
        orig[b] = t;
      }
      for (int k = 0; k < ns; ++k) content[k] = k;
      for (int j = 0; j < w; ++j) {
        const int t = content[j];
        content[j] = content[pslot[j]];
        content[pslot[j]] = t;
      }
      s_nslot = ns;
    }
    __syncthreads();
    // apply it to the other columns of the outer panel: [k0, c0) and [c0+w, k0+nb)
    const int nsl = s_nslot, nleft = c0 - k0, noth = nb - w;
    for (int idx = tid; idx < nsl * noth; idx += bd) {
      const int k = idx / noth, q = idx % noth;
      const int col = q < nleft ? k0 + q : c0 + w + (q - nleft);
      SB[k * noth + q] = A[static_cast<size_t>(slot_row[k]) * n + col];
    }
    __syncthreads();
    for (int idx = tid; idx < nsl * noth; idx += bd) {
      const int k = idx / noth, q = idx % noth;
      const int col = q < nleft ? k0 + q : c0 + w + (q - nleft);
      A[static_cast<size_t>(slot_row[k]) * n + col] = SB[content[k] * noth + q];
    }
    __syncthreads();
    // right-looking update of the not yet factored columns of this outer panel
    const int rw = k0 + nb - (c0 + w);
    if (rw > 0) {
      const int cb = c0 + w;
      for (int idx = tid; idx < w * rw; idx += bd) {
        const int jr = idx / rw, q = idx % rw;
        Ub[jr * nbmax + q] = A[static_cast<size_t>(c0 + jr) * n + cb + q];
      }
      __syncthreads();
      for (int q = tid; q < rw; q += bd)
        for (int jr = 1; jr < w; ++jr) {
          T x = Ub[jr * nbmax + q];
          for (int jj = 0; jj < jr; ++jj) x -= S[jr * ld + jj] * Ub[jj * nbmax + q];
          Ub[jr * nbmax + q] = x;
        }
      __syncthreads();
      for (int idx = tid; idx < w * rw; idx += bd) {
        const int jr = idx / rw, q = idx % rw;
        A[static_cast<size_t>(c0 + jr) * n + cb + q] = Ub[jr * nbmax + q];
      }
      // rows below: A[c0+r][cb+q] -= S[r][:w] . Ub[:w][q], TR x 4 register tiles
      constexpr int TR = sizeof(T) == 4 ? 8 : 4;
      const int ntr = (m - w + TR - 1) / TR, ntc = (rw + 3) / 4;
      for (int t = tid; t < ntr * ntc; t += bd) {
        const int r0 = w + TR * (t / ntc), q0 = 4 * (t % ntc);
        T acc[TR][4];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = T(0);
        for (int jj = 0; jj < w; ++jj) {
          T sv[TR], uv[4];
#pragma unroll
          for (int i = 0; i < TR; ++i) sv[i] = (r0 + i < m) ? S[(r0 + i) * ld + jj] : T(0);
#pragma unroll
          for (int c = 0; c < 4; ++c) uv[c] = (q0 + c < rw) ? Ub[jj * nbmax + q0 + c] : T(0);
#pragma unroll
          for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][c] += sv[i] * uv[c];
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
          if (r0 + i >= m) continue;
          T* row = A + static_cast<size_t>(c0 + r0 + i) * n + cb + q0;
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (q0 + c < rw) row[c] -= acc[i][c];
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0 && bad_pivot) atomicOr(status, kZeroPivot);

  // permutation record for the trailing columns
  int* pr_rec = perm + (static_cast<size_t>(mat) * npan + pan) * perm_stride(nbmax);
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int j = tid; j < nb; j += bd) pr_rec[1 + j] = orig[j];
  for (int r = nb + tid; r < m0; r += bd) {
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
    for (int base = tid; base < M * nb; base += bd * kLoadBatch) {
      float v[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = base + u * bd;
        v[u] = idx < M * nb ? static_cast<float>(A[static_cast<size_t>(k0 + nb + idx / nb) * n + k0 + idx % nb]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = base + u * bd;
        if (idx < M * nb) {
          float h, l;
          split_tf32(v[u], h, l);
          hi[static_cast<size_t>(idx / nb) * nbmax + idx % nb] = h;
          lo[static_cast<size_t>(idx / nb) * nbmax + idx % nb] = l;
        }
      }
    }
  }

  // inv(L11), L11 = unit lower part of A[k0:k0+nb, k0:k0+nb], staged in shared memory
  const int ldl = nb + 1;
  T* Ls = S;
  T* Xs = S + static_cast<size_t>(nb) * ldl;
  for (int idx = tid; idx < nb * nb; idx += bd) {
    const int r = idx / nb, c = idx % nb;
    Ls[r * ldl + c] = A[static_cast<size_t>(k0 + r) * n + k0 + c];
  }
  __syncthreads();
  tri_inverse_smem<T, true>(Ls, Xs, nb, ldl);
  T* X = linv + (static_cast<size_t>(mat) * npan + pan) * nbmax * nbmax;
  for (int idx = tid; idx < nb * nb; idx += bd) {
    const int r = idx / nb, c = idx % nb;
    X[r * nbmax + c] = Xs[r * ldl + c];
  }
  // inv(L11) split for the tensor-core formation of U12 ([point][nbmax][nbmax])
  if (li_hi) {
    for (int idx = tid; idx < nbmax * nbmax; idx += bd) {
      const int r = idx / nbmax, c = idx % nbmax;
      float h = 0.f, l = 0.f;
      if (r < nb && c < nb) split_tf32(static_cast<float>(Xs[r * ldl + c]), h, l);
      li_hi[static_cast<size_t>(mat) * nbmax * nbmax + idx] = h;
      li_lo[static_cast<size_t>(mat) * nbmax * nbmax + idx] = l;
    }
  }
}

// 16-byte vector of T
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void vload(const T* p, T* out) {
  using V = typename Vec16<T>::type;
  const V v = *reinterpret_cast<const V*>(p);
  const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
  for (int i = 0; i < Vec16<T>::n; ++i) out[i] = e[i];
}
template <typename T>
__device__ __forceinline__ void vstore(T* p, const T* in) {
  using V = typename Vec16<T>::type;
  V v;
  T* e = reinterpret_cast<T*>(&v);
#pragma unroll
  for (int i = 0; i < Vec16<T>::n; ++i) e[i] = in[i];
  *reinterpret_cast<V*>(p) = v;
}

// Register-resident panel factorisation (same contract as lu_panel_kernel). Thread t holds panel rows
// t and t + 1024 (RPT rows) of the current W-wide column block in registers. Per block: load it,
// apply the earlier blocks of this panel left-looking (U block by a W x W unit-lower solve, then the
// rank-W update of every row below, streaming the earlier L columns), eliminate column by column
// (two barriers per column: argmax partials, then the pivot/current rows through shared memory),
// store it, and apply its row swaps to the other panel columns. All global row segments move as
// 16-byte vectors. Requires n % (16/sizeof(T)) == 0, nb % W == 0 and n - k0 <= 1024 * RPT.
template <typename T, int W, int RPT>
__global__ void __launch_bounds__(1024) lu_panel_rr_kernel(T* __restrict__ fac, int* __restrict__ piv,
                                                          int* __restrict__ perm, T* __restrict__ linv,
                                                          int n, int k0, int nb, int nbmax,
                                                          unsigned* status, float* __restrict__ ws_hi,
                                                          float* __restrict__ ws_lo, float* __restrict__ li_hi,
                                                          float* __restrict__ li_lo) {
  constexpr int NT = 1024, VE = Vec16<T>::n;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int m0 = n - k0;
  T* SB = reinterpret_cast<T*>(smraw);                       // 2W x nbmax: swap staging
  int* orig = reinterpret_cast<int*>(SB + 2 * static_cast<size_t>(W) * nbmax);  // m0
  __shared__ T Ublk[W][W + 1];
  __shared__ T Lt[W][W + 1];
  __shared__ T prow[W], orow[W];
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ int lp[W], pslot[W], slot_row[2 * W], content[2 * W];
  __shared__ int s_cnt, s_nslot;

  const int mat = blockIdx.x;
  T* A = fac + static_cast<size_t>(mat) * n * n;
  int* ip = piv + static_cast<size_t>(mat) * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int npan = (n + nbmax - 1) / nbmax, pan = k0 / nbmax;
  for (int r = tid; r < m0; r += NT) orig[r] = k0 + r;
  bool bad_pivot = false;
  T a[RPT][W];

  for (int s0 = 0; s0 < nb; s0 += W) {
    const int c0 = k0 + s0;
    // load the column block, every panel row
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = tid + q * NT;
      if (r < m0) {
#pragma unroll
        for (int v = 0; v < W; v += VE) vload(A + static_cast<size_t>(k0 + r) * n + c0 + v, &a[q][v]);
      }
    }
    // left-looking: the earlier blocks of this panel
    for (int t0 = 0; t0 < s0; t0 += W) {
      const int ct = k0 + t0;
      if (tid >= t0 && tid < t0 + W) {
#pragma unroll
        for (int jj = 0; jj < W; ++jj) Ublk[tid - t0][jj] = a[0][jj];
      }
      if (tid < W * W) Lt[tid / W][tid % W] = A[static_cast<size_t>(ct + tid / W) * n + ct + tid % W];
      __syncthreads();
      if (tid < W) {
        for (int i = 1; i < W; ++i) {
          T x = Ublk[i][tid];
          for (int k = 0; k < i; ++k) x -= Lt[i][k] * Ublk[k][tid];
          Ublk[i][tid] = x;
        }
      }
      __syncthreads();
      if (tid >= t0 && tid < t0 + W) {
#pragma unroll
        for (int jj = 0; jj < W; ++jj) a[0][jj] = Ublk[tid - t0][jj];
      }
      // rows below the block: a[q][:] -= L[r][ct:ct+W] Ublk
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid + q * NT;
        if (r >= t0 + W && r < m0) {
          const T* lr = A + static_cast<size_t>(k0 + r) * n + ct;
#pragma unroll
          for (int kv = 0; kv < W; kv += VE) {
            T l[VE];
            vload(lr + kv, l);
#pragma unroll
            for (int u = 0; u < VE; ++u)
#pragma unroll
              for (int jj = 0; jj < W; ++jj) a[q][jj] -= l[u] * Ublk[kv + u][jj];
          }
        }
      }
      __syncthreads();
    }
    // column-by-column elimination of rows s0.. (panel-relative)
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const int cur = s0 + j;
      T best = T(-1);
      int bi = 0x7fffffff;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid + q * NT;
        if (r >= cur && r < m0) {
          const T v = tabs(a[q][j]);
          if (v > best || (v == best && r < bi)) best = v, bi = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
      }
      if (lane == 0) red_v[warp] = best, red_i[warp] = bi;
      __syncthreads();
      best = red_v[lane];
      bi = red_i[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
      }
      const int pr = (bi >= cur && bi < m0) ? bi : cur;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid + q * NT;
        if (r == pr) {
#pragma unroll
          for (int jj = 0; jj < W; ++jj) prow[jj] = a[q][jj];
        }
        if (r == cur) {
#pragma unroll
          for (int jj = 0; jj < W; ++jj) orow[jj] = a[q][jj];
        }
      }
      if (tid == 0) lp[j] = pr - s0;
      __syncthreads();
      const T pv = prow[j];
      if (tid == 0 && (!(tabs(pv) > T(0)) || !isfinite(static_cast<double>(pv)))) bad_pivot = true;
      const T inv = (pv != T(0)) ? T(1) / pv : T(0);
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid + q * NT;
        if (r == cur) {
#pragma unroll
          for (int jj = 0; jj < W; ++jj) a[q][jj] = prow[jj];
        } else if (r == pr) {
#pragma unroll
          for (int jj = 0; jj < W; ++jj) a[q][jj] = orow[jj];
        }
        if (r > cur && r < m0) {
          const T l = a[q][j] * inv;
          a[q][j] = l;
#pragma unroll
          for (int jj = j + 1; jj < W; ++jj) a[q][jj] -= l * prow[jj];
        }
      }
    }
    // store the column block
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = tid + q * NT;
      if (r < m0) {
#pragma unroll
        for (int v = 0; v < W; v += VE) vstore(A + static_cast<size_t>(k0 + r) * n + c0 + v, &a[q][v]);
      }
    }
    // the block's row permutation as slots (see lu_panel_kernel), applied to the other panel columns
    if (tid == 0) {
      int ns = W;
      for (int k = 0; k < W; ++k) slot_row[k] = c0 + k;
      for (int j = 0; j < W; ++j) {
        const int pl = lp[j];
        int sl = pl;
        if (pl >= W) {
          sl = -1;
          for (int q = W; q < ns; ++q)
            if (slot_row[q] == c0 + pl) sl = q;
          if (sl < 0) slot_row[sl = ns++] = c0 + pl;
        }
        pslot[j] = sl;
        ip[c0 + j] = c0 + pl;
        const int x = c0 + j - k0, y = c0 + pl - k0;
        const int t = orig[x];
        orig[x] = orig[y];
        orig[y] = t;
      }
      for (int k = 0; k < ns; ++k) content[k] = k;
      for (int j = 0; j < W; ++j) {
        const int t = content[j];
        content[j] = content[pslot[j]];
        content[pslot[j]] = t;
      }
      s_nslot = ns;
    }
    __syncthreads();
    const int nsl = s_nslot, nleft = s0, noth = nb - W;
    for (int idx = tid; idx < nsl * noth; idx += NT) {
      const int k = idx / noth, q = idx % noth;
      const int col = q < nleft ? k0 + q : c0 + W + (q - nleft);
      SB[k * noth + q] = A[static_cast<size_t>(slot_row[k]) * n + col];
    }
    __syncthreads();
    for (int idx = tid; idx < nsl * noth; idx += NT) {
      const int k = idx / noth, q = idx % noth;
      const int col = q < nleft ? k0 + q : c0 + W + (q - nleft);
      A[static_cast<size_t>(slot_row[k]) * n + col] = SB[content[k] * noth + q];
    }
    __syncthreads();
  }
  if (tid == 0 && bad_pivot) atomicOr(status, kZeroPivot);

  // permutation record for the trailing columns
  int* pr_rec = perm + (static_cast<size_t>(mat) * npan + pan) * perm_stride(nbmax);
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int j = tid; j < nb; j += NT) pr_rec[1 + j] = orig[j];
  for (int r = nb + tid; r < m0; r += NT) {
    if (orig[r] != k0 + r) {
      const int slot = atomicAdd(&s_cnt, 1);
      pr_rec[1 + nbmax + 2 * slot] = k0 + r;
      pr_rec[1 + nbmax + 2 * slot + 1] = orig[r];
    }
  }
  __syncthreads();
  if (tid == 0) pr_rec[0] = s_cnt;

}

// After lu_panel_rr: the L21 split for the tensor-core trailing update and inv(L11) (+ its split).
template <typename T>
__global__ void __launch_bounds__(1024) lu_panel_tail_kernel(const T* __restrict__ fac, T* __restrict__ linv, int n,
                                                            int k0, int nb, int nbmax, float* __restrict__ ws_hi,
                                                            float* __restrict__ ws_lo, float* __restrict__ li_hi,
                                                            float* __restrict__ li_lo) {
  constexpr int NT = 1024, VE = Vec16<T>::n;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* LX = reinterpret_cast<T*>(smraw);
  const int mat = blockIdx.x, tid = threadIdx.x;
  const T* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + nbmax - 1) / nbmax, pan = k0 / nbmax;
  // L21 split for the tensor-core trailing update ([point][row][nbmax]), 16-byte vectors
  if (ws_hi) {
    const int M = n - k0 - nb, q4 = nb / VE;
    float* hi = ws_hi + static_cast<size_t>(mat) * (n - nbmax) * nbmax;
    float* lo = ws_lo + static_cast<size_t>(mat) * (n - nbmax) * nbmax;
    for (int idx = tid; idx < M * q4; idx += NT) {
      const int r = idx / q4, k = VE * (idx % q4);
      T v[VE];
      vload(A + static_cast<size_t>(k0 + nb + r) * n + k0 + k, v);
      float h[VE], l[VE];
#pragma unroll
      for (int u = 0; u < VE; ++u) split_tf32(static_cast<float>(v[u]), h[u], l[u]);
      if (VE == 4) {
        *reinterpret_cast<float4*>(hi + static_cast<size_t>(r) * nbmax + k) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(lo + static_cast<size_t>(r) * nbmax + k) = make_float4(l[0], l[1], l[2], l[3]);
      } else {
#pragma unroll
        for (int u = 0; u < VE; ++u) {
          hi[static_cast<size_t>(r) * nbmax + k + u] = h[u];
          lo[static_cast<size_t>(r) * nbmax + k + u] = l[u];
        }
      }
    }
  }

  // inv(L11) in shared memory (+ its split for the tensor-core U12 formation)
  const int ldl = nb + 1;
  T* Ls = LX;
  T* Xs = LX + static_cast<size_t>(nb) * ldl;
  for (int idx = tid; idx < nb * nb; idx += NT) Ls[(idx / nb) * ldl + idx % nb] = A[static_cast<size_t>(k0 + idx / nb) * n + k0 + idx % nb];
  __syncthreads();
  tri_inverse_smem<T, true>(Ls, Xs, nb, ldl);
  T* X = linv + (static_cast<size_t>(mat) * npan + pan) * nbmax * nbmax;
  for (int idx = tid; idx < nb * nb; idx += NT) X[(idx / nb) * nbmax + idx % nb] = Xs[(idx / nb) * ldl + idx % nb];
  if (li_hi) {
    for (int idx = tid; idx < nbmax * nbmax; idx += NT) {
      const int r = idx / nbmax, c = idx % nbmax;
      float h = 0.f, l = 0.f;
      if (r < nb && c < nb) split_tf32(static_cast<float>(Xs[r * ldl + c]), h, l);
      li_hi[static_cast<size_t>(mat) * nbmax * nbmax + idx] = h;
      li_lo[static_cast<size_t>(mat) * nbmax * nbmax + idx] = l;
    }
  }
}


template <typename T, int W>
__host__ inline size_t panel_rr_smem_bytes(int m0, int nb, int nbmax) {
  (void)nb;
  return 2ull * W * nbmax * sizeof(T) + static_cast<size_t>(m0) * sizeof(int) + 16;
}

// inv(U11) of every panel of every point, after the factorisation (one CTA per point and panel).
template <typename T>
__global__ void __launch_bounds__(256) lu_uinv_kernel(const T* __restrict__ fac, T* __restrict__ uinv, int n,
                                                      int nbmax) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int npan = (n + nbmax - 1) / nbmax;
  const int mat = blockIdx.x / npan, pan = blockIdx.x % npan;
  const int k0 = pan * nbmax, nb = min(nbmax, n - k0), ldl = nb + 1;
  T* Us = reinterpret_cast<T*>(smraw);
  T* Xs = Us + static_cast<size_t>(nb) * ldl;
  const T* A = fac + static_cast<size_t>(mat) * n * n;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx % nb;
    Us[r * ldl + c] = A[static_cast<size_t>(k0 + r) * n + k0 + c];
  }
  __syncthreads();
  tri_inverse_smem<T, false>(Us, Xs, nb, ldl);
  T* Y = uinv + (static_cast<size_t>(mat) * npan + pan) * nbmax * nbmax;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx % nb;
    Y[r * nbmax + c] = Xs[r * ldl + c];
  }
}

constexpr int kTrsmCols = 64;
constexpr int kTrsmLd = kTrsmCols + 1;  // padded smem row (transposed reads)

template <typename T>
__host__ __device__ inline size_t trsm_smem_bytes(int nb) {
  return (2ull * nb * kTrsmLd + static_cast<size_t>(nb) * (nb + 1)) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) lu_swap_trsm_kernel(T* __restrict__ fac, const int* __restrict__ perm,
                                                           const T* __restrict__ linv, int n, int k0,
                                                           int nb, int nbmax, float* __restrict__ ws_hi,
                                                           float* __restrict__ ws_lo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* top = reinterpret_cast<T*>(smraw);                  // original panel rows, later U12   nb x ld
  T* Bs = top + static_cast<size_t>(nb) * kTrsmLd;        // permuted panel rows             nb x ld
  T* Xs = Bs + static_cast<size_t>(nb) * kTrsmLd;         // inv(L11)                        nb x (nb+1)
  const int mat = blockIdx.x;
  const int C0 = k0 + nb + blockIdx.y * kTrsmCols;
  const int ncol = min(kTrsmCols, n - C0);
  T* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + nbmax - 1) / nbmax, pan = k0 / nbmax;
  const int* rec = perm + (static_cast<size_t>(mat) * npan + pan) * perm_stride(nbmax);
  const T* X = linv + (static_cast<size_t>(mat) * npan + pan) * nbmax * nbmax;
  const int tid = threadIdx.x, bd = blockDim.x;
  // read phase: inv(L11), the original panel rows, and the final content of the panel rows
  for (int idx = tid; idx < nb * nb; idx += bd) {
    const int r = idx / nb, c = idx % nb;
    Xs[r * (nb + 1) + c] = X[r * nbmax + c];
  }
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
  // U12 = inv(L11) P A12 (inv(L11) unit lower), 4 x 4 register tiles, staged in `top`
  const int ntr = (nb + 3) / 4;
  for (int t = tid; t < ntr * (kTrsmCols / 4); t += bd) {
    const int r0 = 4 * (t / (kTrsmCols / 4)), q0 = 4 * (t % (kTrsmCols / 4));
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][c] = T(0);
    const int jmax = min(r0 + 4, nb);
    for (int j = 0; j < jmax; ++j) {
      T bv[4], xv[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[j * kTrsmLd + q0 + c];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = (r0 + i < nb && j <= r0 + i) ? Xs[(r0 + i) * (nb + 1) + j] : T(0);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] += xv[i] * bv[c];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (r0 + i < nb)
#pragma unroll
        for (int c = 0; c < 4; ++c) top[(r0 + i) * kTrsmLd + q0 + c] = acc[i][c];
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

// Tensor-core path: apply the panel's row permutation to the trailing columns (displaced rows only)
// and write (P A12)^T, split into TF32 head/remainder, as the K-major B operand of the U12 GEMM.
__global__ void __launch_bounds__(256) lu_swap_pack_kernel(float* __restrict__ fac, const int* __restrict__ perm,
                                                           int n, int k0, int nb, int nbmax,
                                                           float* __restrict__ bt_hi, float* __restrict__ bt_lo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* top = reinterpret_cast<float*>(smraw);            // original panel rows  nb x ld
  float* Bs = top + static_cast<size_t>(nb) * kTrsmLd;      // permuted panel rows nb x ld
  const int mat = blockIdx.x;
  const int C0 = k0 + nb + blockIdx.y * kTrsmCols;
  const int ncol = min(kTrsmCols, n - C0);
  float* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + nbmax - 1) / nbmax, pan = k0 / nbmax;
  const int* rec = perm + (static_cast<size_t>(mat) * npan + pan) * perm_stride(nbmax);
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int idx = tid; idx < nb * kTrsmCols; idx += bd) {
    const int r = idx / kTrsmCols, c = idx % kTrsmCols;
    top[r * kTrsmLd + c] = c < ncol ? A[static_cast<size_t>(k0 + r) * n + C0 + c] : 0.f;
    const int o = rec[1 + r];
    Bs[r * kTrsmLd + c] = c < ncol ? A[static_cast<size_t>(o) * n + C0 + c] : 0.f;
  }
  __syncthreads();
  const int d = rec[0];
  for (int idx = tid; idx < d * kTrsmCols; idx += bd) {
    const int q = idx / kTrsmCols, c = idx % kTrsmCols;
    if (c >= ncol) continue;
    const int dst = rec[1 + nbmax + 2 * q], src = rec[1 + nbmax + 2 * q + 1];
    A[static_cast<size_t>(dst) * n + C0 + c] = top[(src - k0) * kTrsmLd + c];
  }
  const size_t off = static_cast<size_t>(mat) * (n - nbmax) * nbmax;
  for (int idx = tid; idx < kTrsmCols * nbmax; idx += bd) {
    const int c = idx / nbmax, r = idx % nbmax;
    if (c >= ncol) continue;
    float h = 0.f, l = 0.f;
    if (r < nb) split_tf32(Bs[r * kTrsmLd + c], h, l);
    const size_t o = off + static_cast<size_t>(C0 - (k0 + nb) + c) * nbmax + r;
    bt_hi[o] = h;
    bt_lo[o] = l;
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
// Column chunks of 32: the 32 x 32 diagonal block is staged in shared memory and solved by one
// warp, then every thread updates whole rows below (forward) or above (backward) the chunk.
template <typename T, typename Tc>
__global__ void __launch_bounds__(1024) lu_solve_kernel(const T* __restrict__ fac, const int* __restrict__ piv,
                                                        const double* __restrict__ b, double* __restrict__ x,
                                                        int n, int nb, const int* __restrict__ conv,
                                                        int accumulate) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Tc* s = reinterpret_cast<Tc*>(smraw);
  __shared__ Tc dblk[32][33];
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
    for (int j0 = k0; j0 < k0 + kb; j0 += 32) {
      const int cw = min(32, k0 + kb - j0);
      for (int idx = tid; idx < cw * cw; idx += bd) {
        const int r = idx / cw, c = idx % cw;
        dblk[r][c] = static_cast<Tc>(A[static_cast<size_t>(j0 + r) * n + j0 + c]);
      }
      __syncthreads();
      if (warp == 0) {
        Tc v = lane < cw ? s[j0 + lane] : Tc(0);
        for (int jj = 0; jj < cw; ++jj) {
          const Tc xj = __shfl_sync(0xffffffffu, v, jj);
          if (lane > jj && lane < cw) v -= dblk[lane][jj] * xj;
        }
        if (lane < cw) s[j0 + lane] = v;
      }
      __syncthreads();
      {
        const Tc xv = lane < cw ? s[j0 + lane] : Tc(0);
        for (int r = j0 + cw + warp; r < n; r += (bd >> 5)) {
          Tc acc = lane < cw ? static_cast<Tc>(A[static_cast<size_t>(r) * n + j0 + lane]) * xv : Tc(0);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) s[r] -= acc;
        }
      }
      __syncthreads();
    }
  }
  for (int j0 = ((n - 1) / 32) * 32; j0 >= 0; j0 -= 32) {
    const int cw = min(32, n - j0);
    for (int idx = tid; idx < cw * cw; idx += bd) {
      const int r = idx / cw, c = idx % cw;
      dblk[r][c] = static_cast<Tc>(A[static_cast<size_t>(j0 + r) * n + j0 + c]);
    }
    __syncthreads();
    if (warp == 0) {
      Tc v = lane < cw ? s[j0 + lane] : Tc(0);
      for (int jj = cw - 1; jj >= 0; --jj) {
        if (lane == jj) v /= dblk[jj][jj];
        const Tc xj = __shfl_sync(0xffffffffu, v, jj);
        if (lane < jj) v -= dblk[lane][jj] * xj;
      }
      if (lane < cw) s[j0 + lane] = v;
    }
    __syncthreads();
    {
      const Tc xv = lane < cw ? s[j0 + lane] : Tc(0);
      for (int r = warp; r < j0; r += (bd >> 5)) {
        Tc acc = lane < cw ? static_cast<Tc>(A[static_cast<size_t>(r) * n + j0 + lane]) * xv : Tc(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s[r] -= acc;
      }
    }
    __syncthreads();
  }
  double* xo = x + static_cast<size_t>(mat) * n;
  for (int r = tid; r < n; r += bd) xo[r] = accumulate ? xo[r] + static_cast<double>(s[r]) : static_cast<double>(s[r]);
}

// x = A^-1 b (or x += A^-1 b) for one point per CTA with the per-panel block inverses: forward,
// per panel p: permute the right-hand side with the panel's row record, y = inv(L11_p) b_p, then
// b[below] -= L21_p y; backward, per panel from the last: y = inv(U11_p) b_p, b[above] -= U_p y.
// Rows are processed one per warp with the lanes across the panel's columns (coalesced).
template <typename T>
__global__ void __launch_bounds__(1024) lu_solve_blocked_kernel(const T* __restrict__ fac, const int* __restrict__ perm,
                                                                const T* __restrict__ linv, const T* __restrict__ uinv,
                                                                const double* __restrict__ b, double* __restrict__ x,
                                                                int n, int nb, const int* __restrict__ conv,
                                                                int accumulate) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* s = reinterpret_cast<T*>(smraw);   // n
  T* y = s + n;                          // nb
  T* tmp = y + nb;                       // 2 nb
  const int mat = blockIdx.x;
  if (conv && conv[mat]) return;
  const T* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + nb - 1) / nb;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = bd >> 5;
  for (int r = tid; r < n; r += bd) s[r] = static_cast<T>(b[static_cast<size_t>(mat) * n + r]);
  __syncthreads();
  for (int p = 0; p < npan; ++p) {
    const int k0 = p * nb, kb = min(nb, n - k0);
    const int* rec = perm + (static_cast<size_t>(mat) * npan + p) * perm_stride(nb);
    const int d = rec[0];
    for (int j = tid; j < kb; j += bd) tmp[j] = s[rec[1 + j]];
    for (int q = tid; q < d; q += bd) tmp[nb + q] = s[rec[1 + nb + 2 * q + 1]];
    __syncthreads();
    for (int j = tid; j < kb; j += bd) s[k0 + j] = tmp[j];
    for (int q = tid; q < d; q += bd) s[rec[1 + nb + 2 * q]] = tmp[nb + q];
    __syncthreads();
    const T* X = linv + (static_cast<size_t>(mat) * npan + p) * nb * nb;
    for (int r = warp; r < kb; r += nwarp) {
      T acc = T(0);
      for (int c = lane; c <= r; c += 32) acc += X[r * nb + c] * s[k0 + c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) y[r] = acc;
    }
    __syncthreads();
    for (int j = tid; j < kb; j += bd) s[k0 + j] = y[j];
    for (int r = k0 + kb + warp; r < n; r += nwarp) {
      const T* a = A + static_cast<size_t>(r) * n + k0;
      T acc = T(0);
      for (int c = lane; c < kb; c += 32) acc += a[c] * y[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) s[r] -= acc;
    }
    __syncthreads();
  }
  for (int p = npan - 1; p >= 0; --p) {
    const int k0 = p * nb, kb = min(nb, n - k0);
    const T* Y = uinv + (static_cast<size_t>(mat) * npan + p) * nb * nb;
    for (int r = warp; r < kb; r += nwarp) {
      T acc = T(0);
      for (int c = r + lane; c < kb; c += 32) acc += Y[r * nb + c] * s[k0 + c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) y[r] = acc;
    }
    __syncthreads();
    for (int j = tid; j < kb; j += bd) s[k0 + j] = y[j];
    for (int r = warp; r < k0; r += nwarp) {
      const T* a = A + static_cast<size_t>(r) * n + k0;
      T acc = T(0);
      for (int c = lane; c < kb; c += 32) acc += a[c] * y[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) s[r] -= acc;
    }
    __syncthreads();
  }
  double* xo = x + static_cast<size_t>(mat) * n;
  for (int r = tid; r < n; r += bd) xo[r] = accumulate ? xo[r] + static_cast<double>(s[r]) : static_cast<double>(s[r]);
}

}  // namespace

// sub-panel width: largest power of two <= 32 whose shared-memory plan fits the budget
template <typename T>
static int panel_width(int n, int nb) {
  int w = 32;
  while (w > 2 && panel_smem_bytes<T>(n, nb, nb, w) > 210 * 1024) w >>= 1;
  return w < nb ? w : nb;
}

template <typename T, int W, int RPT>
static void launch_rr(T* fac, int* piv, int* perm, T* linv, int nx, int n, int k0, int nb, int nbmax, unsigned* status,
                      float* ws_hi, float* ws_lo, float* li_hi, float* li_lo, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_panel_rr_kernel<T, W, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  static bool attr_tail = false;
  if (!attr_tail) {
    cudaFuncSetAttribute(lu_panel_tail_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_tail = true;
  }
  const size_t smem = panel_rr_smem_bytes<T, W>(n - k0, nb, nbmax);
  lu_panel_rr_kernel<T, W, RPT><<<nx, 1024, smem, st>>>(fac, piv, perm, linv, n, k0, nb, nbmax, status, ws_hi, ws_lo,
                                                       li_hi, li_lo);
  const size_t smem_tail = 2ull * nb * (nb + 1) * sizeof(T);
  lu_panel_tail_kernel<T><<<nx, 1024, smem_tail, st>>>(fac, linv, n, k0, nb, nbmax, ws_hi, ws_lo, li_hi, li_lo);
}

template <typename T>
void launch_lu_panel(T* fac, int* piv, int* perm, T* linv, int nx, int n, int k0, int nb, int nbmax,
                     unsigned* status, float* ws_hi, float* ws_lo, float* li_hi, float* li_lo, cudaStream_t st) {
  const bool trail = k0 + nb < n;
  float* wh = trail ? ws_hi : nullptr;
  float* lh = trail ? li_hi : nullptr;
  // register-resident kernel when the shape allows it
  constexpr int VE = 16 / sizeof(T);
  constexpr int W2 = sizeof(T) == 4 ? 16 : 8, W4 = sizeof(T) == 4 ? 8 : 4;
  if (n % VE == 0 && nbmax <= 128) {
    if (n - k0 <= 2048 && nb % W2 == 0) {
      launch_rr<T, W2, 2>(fac, piv, perm, linv, nx, n, k0, nb, nbmax, status, wh, ws_lo, lh, li_lo, st);
      return;
    }
    if (n - k0 <= 4096 && nb % W4 == 0) {
      launch_rr<T, W4, 4>(fac, piv, perm, linv, nx, n, k0, nb, nbmax, status, wh, ws_lo, lh, li_lo, st);
      return;
    }
  }
  const int W = panel_width<T>(n, nbmax);
  const size_t smem = panel_smem_bytes<T>(n - k0, nb, nbmax, W);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  lu_panel_kernel<T><<<nx, 1024, smem, st>>>(fac, piv, perm, linv, n, k0, nb, nbmax, W, status, wh, ws_lo, lh, li_lo);
}

template <typename T>
void launch_lu_swap_trsm(T* fac, const int* perm, const T* linv, int nx, int n, int k0, int nb,
                         int nbmax, float* ws_hi, float* ws_lo, cudaStream_t st) {
  const int ntrail = n - k0 - nb;
  if (ntrail <= 0) return;
  dim3 grid(nx, (ntrail + kTrsmCols - 1) / kTrsmCols);
  const size_t smem = trsm_smem_bytes<T>(nb);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_swap_trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  lu_swap_trsm_kernel<T><<<grid, 256, smem, st>>>(fac, perm, linv, n, k0, nb, nbmax, ws_hi, ws_lo);
}

void launch_lu_swap_pack(float* fac, const int* perm, int nx, int n, int k0, int nb, int nbmax, float* bt_hi,
                         float* bt_lo, cudaStream_t st) {
  const int ntrail = n - k0 - nb;
  if (ntrail <= 0) return;
  dim3 grid(nx, (ntrail + kTrsmCols - 1) / kTrsmCols);
  const size_t smem = 2ull * nb * kTrsmLd * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_swap_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  lu_swap_pack_kernel<<<grid, 256, smem, st>>>(fac, perm, n, k0, nb, nbmax, bt_hi, bt_lo);
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

template <typename T>
void launch_lu_uinv(const T* fac, T* uinv, int nx, int n, int nbmax, cudaStream_t st) {
  const int npan = (n + nbmax - 1) / nbmax;
  const size_t smem = 2ull * nbmax * (nbmax + 1) * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_uinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  lu_uinv_kernel<T><<<nx * npan, 256, smem, st>>>(fac, uinv, n, nbmax);
}

template <typename T>
void launch_lu_solve_blocked(const T* fac, const int* perm, const T* linv, const T* uinv, const double* b,
                             double* x, int nx, int n, int nb, const int* conv, int accumulate, cudaStream_t st) {
  const size_t smem = (static_cast<size_t>(n) + 3 * nb) * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_solve_blocked_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr_set = true;
  }
  lu_solve_blocked_kernel<T><<<nx, 1024, smem, st>>>(fac, perm, linv, uinv, b, x, n, nb, conv, accumulate);
}

#define BTE_INST(T)                                                                                 \
  template void launch_lu_panel<T>(T*, int*, int*, T*, int, int, int, int, int, unsigned*, float*,       \
                                   float*, float*, float*, cudaStream_t);                           \
  template void launch_lu_uinv<T>(const T*, T*, int, int, int, cudaStream_t);                        \
  template void launch_lu_solve_blocked<T>(const T*, const int*, const T*, const T*, const double*,  \
                                           double*, int, int, int, const int*, int, cudaStream_t);  \
  template void launch_lu_swap_trsm<T>(T*, const int*, const T*, int, int, int, int, int, float*, float*, \
                                       cudaStream_t);                                               \
  template void launch_lu_gemm_simt<T>(T*, int, int, int, int, cudaStream_t);                       \
  template void launch_lu_solve<T>(const T*, const int*, const double*, double*, int, int, int,     \
                                   const int*, int, cudaStream_t);
BTE_INST(double)
BTE_INST(float)
#undef BTE_INST

}  // namespace bte
