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
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

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
// X = 0, then the inverses of the 16 x 16 diagonal blocks of D into X (lanes 0..15 of a warp one block,
// 16..31 the next; lane = column, the column in registers). Ends with a barrier.
template <typename T, bool kLower>
__device__ void tri_inverse_diag16(const T* D, T* X, int nb, int ldl) {
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
}

template <typename T, bool kLower>
__device__ void tri_inverse_smem(const T* D, T* X, int nb, int ldl) {
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nblk = (nb + 15) / 16;
  tri_inverse_diag16<T, kLower>(D, X, nb, ldl);
  // off-diagonal row blocks; the product D[R, between] X[between, rest] is staged in T1, the rows
  // of X below (L) or above (U) the diagonal blocks' area are still zero and serve as scratch
  T* T1 = X;  // write target rows R of X directly after the second product
  (void)T1;
  for (int bi = 1; bi < nblk; ++bi) {
    const int blk = kLower ? bi : nblk - 1 - bi;
    const int r0 = 16 * blk, r1 = min(nb, r0 + 16), rb = r1 - r0;
    // columns of X in row block R still to fill: [0, r0) for L, [r1, nb) for U
    const int c_lo = kLower ? 0 : r1, c_hi = kLower ? r0 : nb, ncol = c_hi - c_lo;
    // acc[r][c] = sum over k between of D[r][k] X[k][c], stored temporarily in X[r][c]. Register
    // tiles of 4 rows x 2 columns (c and c + half): per k, four broadcast reads of D and two
    // conflict-free reads of X feed eight FMAs. Entries of X outside its triangle are zero, so the
    // union of the two columns' k ranges can be used.
    {
      const int half = (ncol + 1) / 2, ngrp = (rb + 3) / 4, js = (half + 31) & ~31;
      for (int t = tid; t < ngrp * js; t += bd) {
        const int g = t / js, j = t % js;
        if (j >= half) continue;
        const int ca = c_lo + j, cb = c_lo + j + half;
        const bool has_b = cb < c_hi;
        const int ra = r0 + 4 * g;
        T acc[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = T(0);
        const int k_lo = kLower ? ca : r1, k_hi = kLower ? r0 : (has_b ? cb : ca) + 1;
        for (int k = k_lo; k < k_hi; ++k) {
          const T xa = X[k * ldl + ca], xb = has_b ? X[k * ldl + cb] : T(0);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const T d = (ra + i < r1) ? D[(ra + i) * ldl + k] : T(0);
            acc[i][0] += d * xa;
            acc[i][1] += d * xb;
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (ra + i < r1) {
            X[(ra + i) * ldl + ca] = acc[i][0];
            if (has_b) X[(ra + i) * ldl + cb] = acc[i][1];
          }
        }
      }
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

// Four consecutive T from a 16-byte aligned address (one or two 16-byte loads).
template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&o)[4]) {
  using V = typename Vec16<T>::type;
  constexpr int VE = Vec16<T>::n;
#pragma unroll
  for (int v = 0; v < 4; v += VE) {
    const V x = *reinterpret_cast<const V*>(p + v);
    const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int u = 0; u < VE; ++u) o[v + u] = e[u];
  }
}

// acc[r][c] += sum_k A[r][k] B[k][c] for a 4 x 4 tile (rows of A at A + r lda, rows of B at
// B + k ldb); K, lda, ldb multiples of 4, A and B 16-byte aligned.
template <typename T>
__device__ __forceinline__ void tile4_nn(const T* A, int lda, const T* B, int ldb, int K, T (&acc)[4][4]) {
  for (int k = 0; k < K; k += 4) {
    T a[4][4], b[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) load4(A + r * lda + k, a[r]);
#pragma unroll
    for (int q = 0; q < 4; ++q) load4(B + (k + q) * ldb, b[q]);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += a[r][q] * b[q][c];
  }
}

// inv(L) (unit lower, kLower) or inv(U) (upper) of an nb x nb block in shared memory by recursive
// doubling: the 16 x 16 diagonal blocks first (tri_inverse_diag16), then for w = 16, 32, 64, ... every
// pair of neighbouring w-blocks [a, b), [b, e) is joined:
//   lower  X[b:e, a:b] = -X[b:e, b:e] (D[b:e, a:b] X[a:b, a:b])
//   upper  X[a:b, b:e] = -X[a:b, a:b] (D[a:b, b:e] X[b:e, b:e])
// each as two 4 x 4-register-tiled products over all pairs of a level at once, with the inner
// product staged in Tmp (nb * nb / 4 elements at most). Requires nb % 16 == 0, ldl % 4 == 0 and
// 16-byte aligned D, X, Tmp. X's unused triangle is zero on return. All threads of the block.
template <typename T, bool kLower>
__device__ void tri_inverse_rd(const T* D, T* X, T* Tmp, int nb, int ldl) {
  const int tid = threadIdx.x, bd = blockDim.x;
  tri_inverse_diag16<T, kLower>(D, X, nb, ldl);
  for (int w = 16; w < nb; w *= 2) {
    const int npair = (nb + 2 * w - 1) / (2 * w), tw = w / 4, tpp = tw * tw;
    // phase 1: Tmp_pair = lower: D[b:e, a:b] X[a:b, a:b]  ((e-b) x w);  upper: D[a:b, b:e] X[b:e, b:e]  (w x (e-b))
    for (int g = tid; g < npair * tpp; g += bd) {
      const int pr = g / tpp, ti = (g % tpp) / tw, tj = g % tw;
      const int a0 = 2 * w * pr, b0 = a0 + w, e0 = min(a0 + 2 * w, nb);
      if (b0 >= nb) continue;
      const int rows = kLower ? e0 - b0 : w, cols = kLower ? w : e0 - b0;
      if (4 * ti >= rows || 4 * tj >= cols) continue;
      T acc[4][4] = {};
      if (kLower)
        tile4_nn(D + (b0 + 4 * ti) * ldl + a0, ldl, X + a0 * ldl + a0 + 4 * tj, ldl, w, acc);
      else
        tile4_nn(D + (a0 + 4 * ti) * ldl + b0, ldl, X + b0 * ldl + b0 + 4 * tj, ldl, e0 - b0, acc);
      T* t = Tmp + static_cast<size_t>(pr) * w * w;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) t[(4 * ti + r) * w + 4 * tj + c] = acc[r][c];
    }
    __syncthreads();
    // phase 2: lower X[b:e, a:b] = -X[b:e, b:e] Tmp;  upper X[a:b, b:e] = -X[a:b, a:b] Tmp
    for (int g = tid; g < npair * tpp; g += bd) {
      const int pr = g / tpp, ti = (g % tpp) / tw, tj = g % tw;
      const int a0 = 2 * w * pr, b0 = a0 + w, e0 = min(a0 + 2 * w, nb);
      if (b0 >= nb) continue;
      const int rows = kLower ? e0 - b0 : w, cols = kLower ? w : e0 - b0;
      if (4 * ti >= rows || 4 * tj >= cols) continue;
      T acc[4][4] = {};
      const T* t = Tmp + static_cast<size_t>(pr) * w * w;
      T* out;
      if (kLower) {
        tile4_nn(X + (b0 + 4 * ti) * ldl + b0, ldl, t + 4 * tj, w, e0 - b0, acc);
        out = X + (b0 + 4 * ti) * ldl + a0 + 4 * tj;
      } else {
        tile4_nn(X + (a0 + 4 * ti) * ldl + a0, ldl, t + 4 * tj, w, w, acc);
        out = X + (a0 + 4 * ti) * ldl + b0 + 4 * tj;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) out[r * ldl + c] = -acc[r][c];
    }
    __syncthreads();
  }
}


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

// Elements of the product staging of tri_inverse_rd for an nb x nb block.
__host__ __device__ inline int rd_tmp_elems(int nb) {
  int m = 0;
  for (int w = 16; w < nb; w *= 2) {
    const int e = ((nb + 2 * w - 1) / (2 * w)) * w * w;
    m = e > m ? e : m;
  }
  return m;
}

// Elements of the panel kernel's product staging area (after D and X).
__host__ __device__ inline int lazy_tmp_elems(int nb) {
  const int a = rd_tmp_elems(nb), b = 16 * (nb + 4);
  return a > b ? a : b;
}

// ---- tensor-core left-looking update of the panel (FP32 factors): PTX helpers and shared state.
// The L tiles come from the matrix by TMA (128 rows x 32 columns, 128-byte swizzle, K-major), a
// converter splits them into TF32 head and remainder in shared memory, and one thread issues
// tcgen05 TF32 MMAs (M = 128 rows, N = 16 block columns, K = 8) accumulating L U in tensor memory.
constexpr int kTcllTile = 128 * 32 * 4;           // one L tile: 16 KB
constexpr int kTcllBTile = 16 * 32 * 4;           // one 32-deep chunk of U^T: 2 KB
constexpr int kTcllBChunks = 4;                   // K <= 128 - 16
constexpr long long kTcllWait = 1ll << 31;        // ~1 s of SM clock
// tensor-core state bytes in the dynamic area after the diagonal block: 1 KB alignment slack, two
// stages of (head, remainder) tiles, the U^T head and remainder chunks
constexpr size_t kTcllBytes = 1024 + 2ull * 2 * kTcllTile + 2ull * kTcllBChunks * kTcllBTile;
// instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9, 10-12 = 2), both
// K-major, N >> 3 = 2 at bits 17-22, M >> 4 = 8 at bits 24-28
constexpr uint32_t kTcllIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (2u << 17) | (8u << 24);

template <bool kTc>
struct TcllShared {};
template <>
struct TcllShared<true> {
  alignas(8) uint64_t full[2];   // L tile landed (TMA transaction count)
  uint64_t conv[2];              // tile split (four converter warps arrive)
  uint64_t empty[2];             // the MMAs that read the stage have completed
  uint64_t done;                 // every MMA of the block has completed
  uint64_t drain;
  uint32_t tmem;
  int abort;
  float Rall[128][16];           // earlier blocks' pivot rows, this block's columns
  float Uall[128][16];           // ... as U rows
};

__device__ __forceinline__ uint32_t tcll_saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void tcll_mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tcll_saddr(b)), "r"(count));
}
__device__ __forceinline__ void tcll_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tcll_saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tcll_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tcll_saddr(b)) : "memory");
}
__device__ __forceinline__ bool tcll_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(tcll_saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the phase did not complete within kTcllWait cycles (the abort flag is set
// and the status bit recorded) or another thread has aborted.
__device__ bool tcll_wait(uint64_t* b, uint32_t parity, int* abort, unsigned* status) {
  const long long t0 = clock64();
  while (!tcll_try(b, parity)) {
    if (*reinterpret_cast<volatile int*>(abort)) return false;
    if (clock64() - t0 > kTcllWait) {
      atomicExch(abort, 1);
      atomicOr(status, kTimeout);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tcll_tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(tcll_saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tcll_saddr(bar))
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t tcll_sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}
__device__ __forceinline__ void tcll_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(kTcllIdesc), "r"(accum));
}
__device__ __forceinline__ void tcll_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tcll_saddr(bar))
               : "memory");
}
__device__ __forceinline__ void tcll_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Panel factorisation with pivots as marks (same contract as lu_panel_kernel, plus inv(U11); the
// TF32 split of L21 is left to lu_swap_pack). One CTA of 1024 threads per point; thread t holds
// physical panel rows t + 1024 q (q < RPT) of the current W-wide column block in registers. Rows do
// not move while the panel is factored: choosing a pivot marks its row with the column it pivots
// (pc). Per column block:
//   load it; apply the earlier blocks left-looking (their pivot rows post the block's entries, the
//   W x W unit-lower solve goes through the precomputed inverse of that block's diagonal part, the
//   unmarked rows take the rank-W update streaming their earlier L entries);
//   eliminate column by column with ONE barrier per column: each warp posts its best unmarked
//   candidate together with the candidate's row, then every warp reduces the 32 posts itself and
//   reads the pivot row from the winning post (posts are double-buffered by column parity);
//   store it and invert the unit-lower part of its own diagonal block for the later blocks.
// Broadcast operands (pivot rows, U blocks) are read from shared memory as 16-byte vectors.
// At the end the rows are put in the order of the equivalent swap sequence (only displaced rows
// move), the panel record and the LAPACK-style pivots are written, and inv(L11) (+ split) and,
// when uinv is given, inv(U11) are formed from the final diagonal block.
// kTcLL (FP32, W = 16, 4 rows x 512 threads): the left-looking update of a column block runs on the
// tensor cores instead. The earlier blocks' pivot rows post their entries and U = inv(L11) (posted
// entries) is formed in shared memory by block forward substitution (L11: those rows' L entries in
// pivot order, copied to shared memory as each block is finished); then D = L[rows, 0:s0] U
// accumulates in tensor memory, 128 rows x 16 columns per row group, by TF32x3 MMAs (the L tiles by
// TMA from the matrix, split into head and remainder in shared memory), and every thread subtracts
// its rows of D.
template <typename T, int W, int RPT, int NT, bool kTcLL>
__global__ void __launch_bounds__(NT, 1) lu_panel_lazy_kernel(T* __restrict__ fac, int* __restrict__ piv,
                                                               int* __restrict__ perm, T* __restrict__ linv,
                                                               T* __restrict__ uinv, int n, int k0, int nb,
                                                               int nbmax, unsigned* status,
                                                               float* __restrict__ li_hi, float* __restrict__ li_lo,
                                                               const __grid_constant__ CUtensorMap mFac) {
  constexpr int VE = Vec16<T>::n, NONE = 1 << 30, MAXB = 128 / W, NW = NT / 32;
  static_assert(NT % 64 == 0 && NT <= 1024 && W * W <= NT, "block shape");
  static_assert(!kTcLL || (sizeof(T) == 4 && W == 16 && RPT == 4 && NT == 512), "tensor-core left-looking shape");
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T LinvB[MAXB][W][W + 1];             // inverse of the unit-lower part of each block's diagonal block
  __shared__ T Tb[W][W + 1];                      // the diagonal block of the block just eliminated
  __shared__ __align__(16) T Raw[W][W];           // block t's pivot rows, current block's columns
  __shared__ __align__(16) T Ub[2][W][W];         // ... after the unit-lower solve
  __shared__ T red_v[2][32];                      // candidate magnitude per warp (FP64 path)
  __shared__ unsigned red_k[2][32];               // candidate key: bits of |v| (FP32 path)
  __shared__ int red_i[2][32];
  __shared__ __align__(16) T red_row[2][32][W];
  __shared__ int pphys[128];
  __shared__ int s_cnt, s_cnt2;
  __shared__ TcllShared<kTcLL> tls;

  const int m0 = n - k0;
  int* orig = reinterpret_cast<int*>(smraw);  // logical position -> physical row (panel-relative)
  int* pos = orig + m0;                       // physical row -> logical position
  int* dl = pos + m0;                         // displaced logical positions (<= 2 nb)
  const int ldl = nb + 4;
  T* triD = reinterpret_cast<T*>(smraw + ((static_cast<size_t>(2 * m0 + 2 * nbmax) * sizeof(int) + 15) & ~size_t(15)));
  T* triX = triD + static_cast<size_t>(nb) * ldl;
  T* triT = triX + static_cast<size_t>(nb) * ldl;

  const int mat = blockIdx.x;
  T* A = fac + static_cast<size_t>(mat) * n * n;
  int* ip = piv + static_cast<size_t>(mat) * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int npan = (n + nbmax - 1) / nbmax, pan = k0 / nbmax;
  // tensor-core left-looking state: L11 in the diagonal-block area, the tiles after it (1 KB aligned)
  T* L11s = triD;
  unsigned char* tcb = nullptr;
  uint32_t tmem = 0, gt = 0, done_ph = 0;
  if constexpr (kTcLL) {
    const uint32_t x = tcll_saddr(triX);
    tcb = reinterpret_cast<unsigned char*>(triX) + (((x + 1023u) & ~1023u) - x);
    if (tid == 0) {
      for (int i = 0; i < 2; ++i) tcll_mbar_init(&tls.full[i], 1), tcll_mbar_init(&tls.conv[i], 4),
                                  tcll_mbar_init(&tls.empty[i], 1);
      tcll_mbar_init(&tls.done, 1);
      tcll_mbar_init(&tls.drain, 1);
      tls.abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(tcll_saddr(&tls.tmem)));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = tls.tmem;
  }
  for (int r = tid; r < m0; r += NT) orig[r] = r, pos[r] = r;
  int pc[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) pc[q] = NONE;
  bool bad_pivot = false;
  T a[RPT][W];
  // warps without panel rows only take part in the barriers; their posts (and the slots of warps
  // this block does not have) say "no candidate"
  const bool active = warp * 32 < m0;
  for (int i = tid; i < 64; i += NT) {
    const int w = i & 31;
    if (w >= NW || w * 32 >= m0) red_v[i >> 5][w] = T(-1), red_k[i >> 5][w] = 0u, red_i[i >> 5][w] = 0x7fffffff;
  }

  for (int b = 0; b * W < nb; ++b) {
    const int s0 = b * W, c0 = k0 + s0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = tid + q * NT;
      if (r < m0) {
#pragma unroll
        for (int v = 0; v < W; v += VE) vload(A + static_cast<size_t>(k0 + r) * n + c0 + v, &a[q][v]);
      }
    }
    if constexpr (kTcLL) {
      if (b > 0) {
        float* stage = reinterpret_cast<float*>(tcb);              // [2][head, remainder] L tiles
        float* bhi = reinterpret_cast<float*>(tcb + 4 * kTcllTile);  // U^T head, [chunk][16][32] swizzled
        float* blo = bhi + kTcllBChunks * kTcllBTile / 4;
        // (1) the earlier blocks' pivot rows post their entries; U[0:s0, :] = inv(L11) Rall by block
        //     forward substitution
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (pc[q] < s0) {
#pragma unroll
            for (int v = 0; v < W; v += VE) vstore(&tls.Rall[pc[q]][v], &a[q][v]);
          }
        }
        __syncthreads();
        for (int t = 0; t < b; ++t) {
          const int t0 = t * W;
          for (int e = tid; e < W * W; e += NT) {
            const int i = e / W, jj = e % W;
            float acc = tls.Rall[t0 + i][jj];
            for (int k = 0; k < i; ++k) acc += LinvB[t][i][k] * tls.Rall[t0 + k][jj];
            tls.Uall[t0 + i][jj] = acc;
          }
          __syncthreads();
          if (t + 1 < b) {
            const int r0 = t0 + W;
            for (int e = tid; e < (s0 - r0) * W; e += NT) {
              const int i = r0 + e / W, jj = e % W;
              const float* lr = L11s + static_cast<size_t>(i) * ldl + t0;
              float acc = tls.Rall[i][jj];
#pragma unroll
              for (int k = 0; k < W; ++k) acc -= lr[k] * tls.Uall[t0 + k][jj];
              tls.Rall[i][jj] = acc;
            }
            __syncthreads();
          }
        }
        // (2) U^T into the MMA's B operand: head and remainder, K-major, 128-byte swizzle (the 16-byte
        //     chunk j of row nn sits at j ^ (nn % 8)); pivot rows take their U rows
        for (int e = tid; e < s0 * W; e += NT) {
          const int k = e / W, nn = e % W, c = k >> 5, kk = k & 31;
          float h, l;
          split_tf32(tls.Uall[k][nn], h, l);
          const int off = c * (kTcllBTile / 4) + (nn >> 3) * 256 + (nn & 7) * 32 + ((((kk >> 2) ^ (nn & 7))) << 2) + (kk & 3);
          bhi[off] = h;
          blo[off] = l;
        }
        unsigned upd = 0u;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (pc[q] < s0) {
#pragma unroll
            for (int v = 0; v < W; v += VE) vload(&tls.Uall[pc[q]][v], &a[q][v]);
          } else if (tid + q * NT < m0) {
            upd |= 1u << q;
          }
        }
        // the tensor-core reads (TMA of the L entries this CTA stored, MMA of the U^T tiles) come after
        // every thread's ordinary writes
        asm volatile("fence.proxy.async;" ::: "memory");
        __syncthreads();
        // (3) D = L[rows, 0:s0] U: row group g (rows 128 g ..), 32-column chunk c of K per tile
        const int G = (m0 + 127) / 128, C = (s0 + 31) / 32, ntile = G * C;
        const bool run = !*reinterpret_cast<volatile int*>(&tls.abort);
        if (run) {
          if (warp == 0 && lane == 0) {
            // producer: L tiles of the matrix into the two stages
            uint32_t it = gt;
            for (int i = 0; i < ntile; ++i, ++it) {
              const int st = it & 1;
              if (!tcll_wait(&tls.empty[st], ((it >> 1) & 1u) ^ 1u, &tls.abort, status)) break;
              tcll_expect_tx(&tls.full[st], kTcllTile);
              tcll_tma_load3(stage + st * 2 * (kTcllTile / 4), &mFac, k0 + 32 * (i % C), k0 + 128 * (i / C), mat,
                             &tls.full[st]);
            }
          } else if (warp == 1 && lane == 0) {
            // MMA issuer: three TF32 products per K step (remainder x head, head x remainder, head x head)
            uint32_t it = gt;
            for (int i = 0; i < ntile; ++i, ++it) {
              const int st = it & 1;
              if (!tcll_wait(&tls.conv[st], (it >> 1) & 1u, &tls.abort, status)) break;
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const int g = i / C, c = i % C;
              const uint32_t d = tmem + 16 * g;
              const uint32_t ah = tcll_saddr(stage + st * 2 * (kTcllTile / 4)), al = ah + kTcllTile;
              const uint32_t bh = tcll_saddr(bhi) + c * kTcllBTile, bl = tcll_saddr(blo) + c * kTcllBTile;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                if (32 * c + 8 * kk >= s0) break;
                const uint32_t off = kk * 32;
                tcll_mma(d, tcll_sdesc(al + off), tcll_sdesc(bh + off), (c | kk) ? 1u : 0u);
                tcll_mma(d, tcll_sdesc(ah + off), tcll_sdesc(bl + off), 1u);
                tcll_mma(d, tcll_sdesc(ah + off), tcll_sdesc(bh + off), 1u);
              }
              tcll_commit(&tls.empty[st]);
            }
            tcll_commit(&tls.done);
          } else if (warp >= 2 && warp < 6) {
            // converters: head = TF32 rounding in place, remainder beside it
            const int ct = tid - 64;
            uint32_t it = gt;
            for (int i = 0; i < ntile; ++i, ++it) {
              const int st = it & 1;
              // one lane waits for the tile and the warp follows it, so the warp never splits
              int ok = 0;
              if (lane == 0) ok = tcll_wait(&tls.full[st], (it >> 1) & 1u, &tls.abort, status) ? 1 : 0;
              ok = __shfl_sync(0xffffffffu, ok, 0);
              __syncwarp();
              if (!ok) break;
              float4* hp = reinterpret_cast<float4*>(stage + st * 2 * (kTcllTile / 4));
              float4* lp = hp + kTcllTile / 16;
#pragma unroll
              for (int u = 0; u < kTcllTile / 16 / 128; ++u) {
                const float4 x = hp[ct + 128 * u];
                float4 h, l;
                split_tf32(x.x, h.x, l.x);
                split_tf32(x.y, h.y, l.y);
                split_tf32(x.z, h.z, l.z);
                split_tf32(x.w, h.w, l.w);
                hp[ct + 128 * u] = h;
                lp[ct + 128 * u] = l;
              }
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              __syncwarp();
              if (lane == 0) tcll_arrive(&tls.conv[st]);
            }
          }
          gt += ntile;
        }
        __syncthreads();
        if (run && tid == 0) tcll_wait(&tls.done, done_ph, &tls.abort, status);
        if (run) done_ph ^= 1u;
        __syncthreads();
        if (*reinterpret_cast<volatile int*>(&tls.abort)) {
          // an expired wait: let the copies and products in flight finish before the CTA moves on
          if (warp == 0 && lane == 0) {
            for (int st = 0; st < 2; ++st) {
              const long long t1 = clock64();
              while (!tcll_try(&tls.full[st], ((gt - 1 - st) >> 1) & 1u) && clock64() - t1 < kTcllWait) {
              }
            }
          } else if (warp == 1 && lane == 0) {
            tcll_commit(&tls.drain);
            const long long t1 = clock64();
            while (!tcll_try(&tls.drain, 0) && clock64() - t1 < kTcllWait) {
            }
          }
          __syncthreads();
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t lanes = static_cast<uint32_t>(32 * (warp & 3)) << 16;
#pragma unroll
          for (int q = 0; q < RPT; ++q) {
            float dv[16];
            tcll_ld16(tmem + lanes + 16 * ((warp >> 2) + 4 * q), dv);
            if ((upd >> q) & 1u) {
#pragma unroll
              for (int j = 0; j < W; ++j) a[q][j] -= dv[j];
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
      }
    } else {
    // left-looking: earlier blocks t of this panel
      for (int t = 0; t < b; ++t) {
        const int t0 = t * W;
  #pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (pc[q] >= t0 && pc[q] < t0 + W) {
  #pragma unroll
            for (int v = 0; v < W; v += VE) vstore(&Raw[pc[q] - t0][v], &a[q][v]);
          }
        }
        __syncthreads();
        T (*U)[W] = Ub[t & 1];
        if (tid < W * W) {
          const int i = tid / W, jj = tid % W;
          T acc = Raw[i][jj];
          for (int k = 0; k < i; ++k) acc += LinvB[t][i][k] * Raw[k][jj];
          U[i][jj] = acc;
        }
        __syncthreads();
        // pivot rows of block t take their U values; rows below block t (unmarked, or marked by a
        // later block) take the rank-W update, each U row chunk read once for all of a thread's rows.
        // A row's L entries are fetched one 32-byte sector (two 16-byte vectors) at a time.
        constexpr int KC = 32 / sizeof(T) < W ? 32 / sizeof(T) : W;
        bool upd[RPT];
        const T* lr[RPT];
  #pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int r = tid + q * NT;
          upd[q] = r < m0 && pc[q] >= t0 + W;
          lr[q] = A + static_cast<size_t>(k0 + (r < m0 ? r : 0)) * n + k0 + t0;
          if (r < m0 && pc[q] >= t0 && pc[q] < t0 + W) {
            const int i = pc[q] - t0;
  #pragma unroll
            for (int v = 0; v < W; v += VE) vload(&U[i][v], &a[q][v]);
          }
        }
        if (active) {
  #pragma unroll
          for (int kv = 0; kv < W; kv += KC) {
            T l[RPT][KC];
  #pragma unroll
            for (int q = 0; q < RPT; ++q) {
  #pragma unroll
              for (int c = 0; c < KC; c += VE) {
                if (upd[q]) vload(lr[q] + kv + c, &l[q][c]);
                else
  #pragma unroll
                  for (int u = 0; u < VE; ++u) l[q][c + u] = T(0);
              }
            }
  #pragma unroll
            for (int u = 0; u < KC; ++u) {
  #pragma unroll
              for (int v = 0; v < W; v += VE) {
                T uu[VE];
                vload(&U[kv + u][v], uu);
  #pragma unroll
                for (int q = 0; q < RPT; ++q)
  #pragma unroll
                  for (int e = 0; e < VE; ++e) a[q][v + e] -= l[q][u] * uu[e];
              }
            }
          }
        }
      }
    }
    // column-by-column elimination, one barrier per column
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const int cur = s0 + j, buf = cur & 1;
      if (!active) {
        __syncthreads();
        continue;
      }
      int bi;
      if constexpr (sizeof(T) == 4) {
        // argmax as two warp reductions over (bits of |v|, row): the magnitude's bit pattern orders
        // like the value; NaN counts as infinity, the smallest row wins a tie
        unsigned key = 0u;
        int ri = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int r = tid + q * NT;
          if (r < m0 && pc[q] == NONE) {
            unsigned k = __float_as_uint(static_cast<float>(a[q][j])) & 0x7fffffffu;
            if (k > 0x7f800000u) k = 0x7f800000u;
            if (k > key || ri == 0x7fffffff) key = k, ri = r;
          }
        }
        const unsigned wk = __reduce_max_sync(0xffffffffu, key);
        const int wi = static_cast<int>(__reduce_min_sync(0xffffffffu, key == wk ? static_cast<unsigned>(ri) : 0x7fffffffu));
        if (lane == 0) red_k[buf][warp] = wk, red_i[buf][warp] = wi;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (tid + q * NT == wi) {
#pragma unroll
            for (int v = (j / VE) * VE; v < W; v += VE) vstore(&red_row[buf][warp][v], &a[q][v]);
          }
        }
        __syncthreads();
        const unsigned pk = red_k[buf][lane];
        const int pi = red_i[buf][lane];
        const unsigned gk = __reduce_max_sync(0xffffffffu, pk);
        bi = static_cast<int>(__reduce_min_sync(0xffffffffu, pk == gk ? static_cast<unsigned>(pi) : 0x7fffffffu));
      } else {
        T best = T(-1);
        bi = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int r = tid + q * NT;
          if (r < m0 && pc[q] == NONE) {
            T v = tabs(a[q][j]);
            if (v != v) v = T(INFINITY);  // a NaN candidate wins and is reported as a bad pivot
            if (v > best || (v == best && r < bi)) best = v, bi = r;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T ov = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
        }
        if (lane == 0) red_v[buf][warp] = best, red_i[buf][warp] = bi;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (tid + q * NT == bi) {
#pragma unroll
            for (int v = (j / VE) * VE; v < W; v += VE) vstore(&red_row[buf][warp][v], &a[q][v]);
          }
        }
        __syncthreads();
        best = red_v[buf][lane];
        bi = red_i[buf][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T ov = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
        }
      }
      const T* prow = red_row[buf][(bi % NT) >> 5];
      T pr[W];
#pragma unroll
      for (int v = (j / VE) * VE; v < W; v += VE) vload(prow + v, &pr[v]);
      const T pv = pr[j];
      if (tid == 0) {
        pphys[cur] = bi;
        if (!(tabs(pv) > T(0)) || !isfinite(static_cast<double>(pv))) bad_pivot = true;
      }
      T inv = T(0);
      if (pv != T(0)) {
        if constexpr (sizeof(T) == 4) inv = __frcp_rn(pv);
        else inv = __drcp_rn(pv);
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid + q * NT;
        if (r == bi) {
          pc[q] = cur;
        } else if (r < m0 && pc[q] == NONE) {
          const T l = a[q][j] * inv;
          a[q][j] = l;
#pragma unroll
          for (int jj = j + 1; jj < W; ++jj) a[q][jj] -= l * pr[jj];
        }
      }
    }
    // store the block (physical rows)
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = tid + q * NT;
      if (r < m0) {
#pragma unroll
        for (int v = 0; v < W; v += VE) vstore(A + static_cast<size_t>(k0 + r) * n + c0 + v, &a[q][v]);
      }
      if (pc[q] >= s0 && pc[q] < s0 + W) {
#pragma unroll
        for (int jj = 0; jj < W; ++jj) Tb[pc[q] - s0][jj] = a[q][jj];
      }
    }
    __syncthreads();
    if constexpr (kTcLL) {
      if (s0 + W < nb) {
        // this block's pivot rows enter L11 for the later blocks: their entries in the panel's
        // columns 0 .. s0+W (just stored), one 16-byte vector per thread and pass
        const int nvec = (s0 + W) / VE;
        for (int idx = tid; idx < W * nvec; idx += NT) {
          const int i = idx / nvec, v = idx - i * nvec;
          *reinterpret_cast<float4*>(L11s + static_cast<size_t>(s0 + i) * ldl + v * VE) =
              *reinterpret_cast<const float4*>(A + static_cast<size_t>(k0 + pphys[s0 + i]) * n + k0 + v * VE);
        }
      }
    }
    if (tid < W) {
      // column c of the inverse of the unit-lower part of Tb, in registers
      const int c = tid;
      T x[W];
#pragma unroll
      for (int r = 0; r < W; ++r) {
        T acc = (r == c) ? T(1) : T(0);
#pragma unroll
        for (int k = 0; k < r; ++k) acc -= Tb[r][k] * x[k];
        x[r] = (r < c) ? T(0) : acc;
      }
#pragma unroll
      for (int r = 0; r < W; ++r) LinvB[b][r][c] = x[r];
    } else if (tid == 32) {
      // the swap sequence equivalent to this block's pivots: logical order and LAPACK pivots
      for (int j = 0; j < W && s0 + j < nb; ++j) {
        const int cur = s0 + j, p = pphys[cur], y = pos[p], o = orig[cur];
        ip[k0 + cur] = k0 + y;
        orig[cur] = p;
        orig[y] = o;
        pos[p] = cur;
        pos[o] = y;
      }
    }
    __syncthreads();
  }
  if (tid == 0 && bad_pivot) atomicOr(status, kZeroPivot);

  // move displaced rows (panel columns) to their logical positions, staged through the (still
  // unused) triangular-inverse area: d <= 2 nb rows of nb entries
  if (tid == 0) s_cnt = 0, s_cnt2 = 0;
  __syncthreads();
  for (int y = tid; y < m0; y += NT)
    if (orig[y] != y) dl[atomicAdd(&s_cnt, 1)] = y;
  __syncthreads();
  const int d = s_cnt, nvr = nb / VE;
  using V = typename Vec16<T>::type;
  V* stage = reinterpret_cast<V*>(triD);
  for (int idx = tid; idx < d * nvr; idx += NT) {
    const int y = dl[idx / nvr], v = idx % nvr;
    stage[idx] = *reinterpret_cast<const V*>(A + static_cast<size_t>(k0 + orig[y]) * n + k0 + v * VE);
  }
  __syncthreads();
  for (int idx = tid; idx < d * nvr; idx += NT) {
    const int y = dl[idx / nvr], v = idx % nvr;
    *reinterpret_cast<V*>(A + static_cast<size_t>(k0 + y) * n + k0 + v * VE) = stage[idx];
  }
  // panel record: origin of the top nb rows, then the displaced rows below them
  int* rec = perm + (static_cast<size_t>(mat) * npan + pan) * perm_stride(nbmax);
  for (int j = tid; j < nb; j += NT) rec[1 + j] = k0 + orig[j];
  for (int k = tid; k < d; k += NT) {
    const int y = dl[k];
    if (y >= nb) {
      const int slot = atomicAdd(&s_cnt2, 1);
      rec[1 + nbmax + 2 * slot] = k0 + y;
      rec[1 + nbmax + 2 * slot + 1] = k0 + orig[y];
    }
  }
  __syncthreads();
  if (tid == 0) rec[0] = s_cnt2;

  // inv(L11) (+ split) and inv(U11) of the final diagonal block
  for (int idx = tid; idx < nb * nb; idx += NT)
    triD[(idx / nb) * ldl + idx % nb] = A[static_cast<size_t>(k0 + idx / nb) * n + k0 + idx % nb];
  __syncthreads();
  // the 4 x 4 register tiles of the doubling inverse fit the 64-register budget in FP32 only
  if constexpr (sizeof(T) == 4) {
    if (nb % 16 == 0) tri_inverse_rd<T, true>(triD, triX, triT, nb, ldl);
    else tri_inverse_smem<T, true>(triD, triX, nb, ldl);
  } else {
    tri_inverse_smem<T, true>(triD, triX, nb, ldl);
  }
  T* X = linv + (static_cast<size_t>(mat) * npan + pan) * nbmax * nbmax;
  for (int idx = tid; idx < nb * nb; idx += NT) X[(idx / nb) * nbmax + idx % nb] = triX[(idx / nb) * ldl + idx % nb];
  if (li_hi) {
    for (int idx = tid; idx < nbmax * nbmax; idx += NT) {
      const int r = idx / nbmax, c = idx % nbmax;
      float h = 0.f, l = 0.f;
      if (r < nb && c < nb) split_tf32(static_cast<float>(triX[r * ldl + c]), h, l);
      li_hi[static_cast<size_t>(mat) * nbmax * nbmax + idx] = h;
      li_lo[static_cast<size_t>(mat) * nbmax * nbmax + idx] = l;
    }
  }
  if (uinv) {
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      if (nb % 16 == 0) tri_inverse_rd<T, false>(triD, triX, triT, nb, ldl);
      else tri_inverse_smem<T, false>(triD, triX, nb, ldl);
    } else {
      tri_inverse_smem<T, false>(triD, triX, nb, ldl);
    }
    T* Y = uinv + (static_cast<size_t>(mat) * npan + pan) * nbmax * nbmax;
    for (int idx = tid; idx < nb * nb; idx += NT) Y[(idx / nb) * nbmax + idx % nb] = triX[(idx / nb) * ldl + idx % nb];
  }
  if constexpr (kTcLL) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
    }
  }
}


// Dynamic shared memory of the panel kernel: orig/pos/displaced lists, then D and X (nb x (nb+4)
// each: the diagonal block and the inverse being built) and a product staging area (the
// doubling inverse's, and 16 rows of X's extension).
__host__ inline size_t panel_lazy_smem_bytes(int m0, int nb, int nbmax, size_t tsize) {
  const size_t ints = ((static_cast<size_t>(2 * m0 + 2 * nbmax) * sizeof(int) + 15) & ~size_t(15));
  return ints + (2ull * nb * (nb + 4) + lazy_tmp_elems(nb)) * tsize;
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

// Tensor-core path: apply the panel's row permutation to the first ncols trailing columns
// (displaced rows only) and write (P A12)^T, split into TF32 head/remainder, as the K-major B
// operand of the U12 product; split L21 (every row below the panel) into the A operand of the
// trailing update. Operand rows hold ks floats (K = nbmax of them used here).
__global__ void __launch_bounds__(256) lu_swap_pack_kernel(float* __restrict__ fac, const int* __restrict__ perm,
                                                           int n, int k0, int nb, int nbmax, int ncols, int ks,
                                                           float* __restrict__ bt_hi, float* __restrict__ bt_lo,
                                                           float* __restrict__ a_hi, float* __restrict__ a_lo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* top = reinterpret_cast<float*>(smraw);            // original panel rows  nb x ld
  float* Bs = top + static_cast<size_t>(nb) * kTrsmLd;      // permuted panel rows nb x ld
  const int mat = blockIdx.x;
  const int C0 = k0 + nb + blockIdx.y * kTrsmCols;
  const int ncol = min(kTrsmCols, k0 + nb + ncols - C0);
  float* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + nbmax - 1) / nbmax, pan = k0 / nbmax;
  const int* rec = perm + (static_cast<size_t>(mat) * npan + pan) * perm_stride(nbmax);
  const int tid = threadIdx.x, bd = blockDim.x;
  const size_t off = static_cast<size_t>(mat) * (n - nbmax) * ks;
  if (ncol > 0) {
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
    for (int idx = tid; idx < kTrsmCols * nbmax; idx += bd) {
      const int c = idx / nbmax, r = idx % nbmax;
      if (c >= ncol) continue;
      float h = 0.f, l = 0.f;
      if (r < nb) split_tf32(Bs[r * kTrsmLd + c], h, l);
      const size_t o = off + static_cast<size_t>(C0 - (k0 + nb) + c) * ks + r;
      bt_hi[o] = h;
      bt_lo[o] = l;
    }
  }
  // TF32 split of L21 rows [k0 + nb + 64 y, +64) (the A operand of the trailing update)
  const int R0 = blockIdx.y * kTrsmCols, nrow = min(kTrsmCols, n - k0 - nb - R0);
  if (!a_hi || nrow <= 0) return;
  if ((n & 3) != 0 || (nb & 3) != 0) {
    for (int idx = tid; idx < nrow * nb; idx += bd) {
      const int r = idx / nb, k = idx % nb;
      float h, l;
      split_tf32(A[static_cast<size_t>(k0 + nb + R0 + r) * n + k0 + k], h, l);
      const size_t o = off + static_cast<size_t>(R0 + r) * ks + k;
      a_hi[o] = h;
      a_lo[o] = l;
    }
  } else {
    const int q4 = nb / 4;
    for (int idx = tid; idx < nrow * q4; idx += bd) {
      const int r = idx / q4, k = 4 * (idx % q4);
      const float4 v = *reinterpret_cast<const float4*>(A + static_cast<size_t>(k0 + nb + R0 + r) * n + k0 + k);
      float4 h, l;
      split_tf32(v.x, h.x, l.x);
      split_tf32(v.y, h.y, l.y);
      split_tf32(v.z, h.z, l.z);
      split_tf32(v.w, h.w, l.w);
      const size_t o = off + static_cast<size_t>(R0 + r) * ks + k;
      *reinterpret_cast<float4*>(a_hi + o) = h;
      *reinterpret_cast<float4*>(a_lo + o) = l;
    }
  }
}

// The two 128-wide panels at k0 (P_1, L_1, L21_1) and k0 + 128 (P_2, L_2, L21_2) as one 256-wide
// step, for the columns right of and the rows below base = k0 + 256. Blocks y < ncb take 32 columns
// each:
//   A <- P_2 P_1 A on those columns (displaced rows only; the pivot rows go to the B operand);
//   (P A12)^T split over the 256 panel rows (B operand of the block's U12 product);
// blocks y >= ncb take 32 rows each of the A operand of the trailing update, [P_2 L21_1, L21_2]
// split, row i of P_2 L21_1 being the matrix row that P_2 moved to i. Both panels are full (128
// columns); n % 4 == 0, so every row segment here is whole 16-byte vectors.
constexpr int kPairP = 128, kPairCols = 32, kPairLd = kPairCols + 1;
__global__ void __launch_bounds__(256) lu_swap_pack_pair_kernel(float* __restrict__ fac, const int* __restrict__ perm,
                                                                int n, int k0, int ks, int ncb,
                                                                float* __restrict__ bt_hi, float* __restrict__ bt_lo,
                                                                float* __restrict__ a_hi, float* __restrict__ a_lo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* piv = reinterpret_cast<float*>(smraw);  // rows of P A over the pair's 256 panel rows, 256 x ld
  int* srow = reinterpret_cast<int*>(piv + 2 * kPairP * kPairLd);  // pivot rows, 2 x 128
  int* spair = srow + 2 * kPairP;                                   // displaced (dst, src), 2 x 2 x 128
  const int mat = blockIdx.x, tid = threadIdx.x;
  const int base = k0 + 2 * kPairP, M = n - base;
  float* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + kPairP - 1) / kPairP, pan = k0 / kPairP;
  const int* rec1 = perm + (static_cast<size_t>(mat) * npan + pan) * perm_stride(kPairP);
  const int* rec2 = rec1 + perm_stride(kPairP);
  const size_t off = static_cast<size_t>(mat) * (n - kPairP) * ks;
  const int d1 = rec1[0], d2 = rec2[0];
  if (static_cast<int>(blockIdx.y) < ncb) {
    const int C0 = base + blockIdx.y * kPairCols;
    const int ncol = min(kPairCols, n - C0);
    for (int q = tid; q < 2 * kPairP; q += 256) {
      const int* rec = q < kPairP ? rec1 : rec2;
      const int r = q % kPairP;
      srow[q] = rec[1 + r];
      spair[2 * q] = rec[1 + kPairP + 2 * r];
      spair[2 * q + 1] = rec[1 + kPairP + 2 * r + 1];
    }
    __syncthreads();
    const int r8 = tid / 8, c4 = 4 * (tid % 8);  // 8 threads per row, one float4 each
    const bool cok = c4 < ncol;
    for (int half = 0; half < 2; ++half) {
      // pivot rows into shared memory (all 128 loads of the half in flight together)
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r8 + 32 * u;
        v[u] = cok ? *reinterpret_cast<const float4*>(A + static_cast<size_t>(srow[half * kPairP + r]) * n + C0 + c4)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float* d = piv + (half * kPairP + r8 + 32 * u) * kPairLd + c4;
        d[0] = v[u].x, d[1] = v[u].y, d[2] = v[u].z, d[3] = v[u].w;
      }
      // every pivot row is read before a displaced row overwrites its old place
      __syncthreads();
      const int d = half ? d2 : d1;
      const int* pr = spair + half * 2 * kPairP;
      float4 w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = r8 + 32 * u;
        w[u] = q < d && cok ? *reinterpret_cast<const float4*>(A + static_cast<size_t>(pr[2 * q + 1]) * n + C0 + c4)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = r8 + 32 * u;
        if (q < d && cok) *reinterpret_cast<float4*>(A + static_cast<size_t>(pr[2 * q]) * n + C0 + c4) = w[u];
      }
      // the second permutation reads rows the first one wrote (global writes of this block are
      // visible to it after the barrier)
      __syncthreads();
    }
    // (P A12)^T split: column c of the block is operand row C0 - base + c, K = the 256 panel rows
#pragma unroll 4
    for (int idx = tid; idx < kPairCols * 2 * kPairP; idx += 256) {
      const int c = idx / (2 * kPairP), r = idx % (2 * kPairP);
      if (c >= ncol) continue;
      float h, l;
      split_tf32(piv[r * kPairLd + c], h, l);
      const size_t o = off + static_cast<size_t>(C0 - base + c) * ks + r;
      bt_hi[o] = h;
      bt_lo[o] = l;
    }
    return;
  }
  // ---- L21 operand rows [base + R0, +32)
  int* rowsrc = srow;
  const int R0 = (blockIdx.y - ncb) * kPairCols, nrow = min(kPairCols, M - R0);
  if (tid < kPairCols) rowsrc[tid] = base + R0 + tid;
  __syncthreads();
  for (int q = tid; q < d2; q += 256) {
    const int dst = rec2[1 + kPairP + 2 * q] - (base + R0);
    if (dst >= 0 && dst < nrow) rowsrc[dst] = rec2[1 + kPairP + 2 * q + 1];
  }
  __syncthreads();
  // 32 rows x 64 float4: 8 per thread, loads first
  float4 v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int f = tid + 256 * u, r = f / 64, k = 4 * (f % 64);
    const int src = k < kPairP ? rowsrc[r] : base + R0 + r;
    v[u] = r < nrow ? *reinterpret_cast<const float4*>(A + static_cast<size_t>(src) * n + k0 + k)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int f = tid + 256 * u, r = f / 64, k = 4 * (f % 64);
    if (r >= nrow) continue;
    float4 h, l;
    split_tf32(v[u].x, h.x, l.x);
    split_tf32(v[u].y, h.y, l.y);
    split_tf32(v[u].z, h.z, l.z);
    split_tf32(v[u].w, h.w, l.w);
    const size_t o = off + static_cast<size_t>(R0 + r) * ks + k;
    *reinterpret_cast<float4*>(a_hi + o) = h;
    *reinterpret_cast<float4*>(a_lo + o) = l;
  }
}

// inv(L11) of the two-panel block at k0 (see launch_lu_pair_linv), one CTA per point:
//   T = Lp inv(L_1)   (Lp = rows P_2 moved to the top of panel 2, first panel's columns),
//   X = -inv(L_2) T,
// both products over the nonzero (lower-triangular) part of the inverses only; 8 x 8 outputs per
// thread (16 x 16 threads), operands from shared memory. The diagonal blocks and the zero block are
// written alongside.
__global__ void __launch_bounds__(256) lu_pair_linv_kernel(const float* __restrict__ fac, const int* __restrict__ perm,
                                                           const float* __restrict__ linv, int n, int k0,
                                                           float* __restrict__ o_hi, float* __restrict__ o_lo) {
  constexpr int P = kPairP, LD = P + 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* Mt = reinterpret_cast<float*>(smraw);  // Lp^T, then inv(L_2)^T   [k][i]
  float* Ia = Mt + P * LD;                      // inv(L_1), upper part 0  [k][j]
  float* Ts = Ia + P * LD;                      // T                       [k][j]
  int* srow = reinterpret_cast<int*>(Ts + P * LD);
  const int mat = blockIdx.x, tid = threadIdx.x;
  const float* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + P - 1) / P, pan = k0 / P;
  const int* rec2 = perm + (static_cast<size_t>(mat) * npan + pan + 1) * perm_stride(P);
  const float* La = linv + (static_cast<size_t>(mat) * npan + pan) * P * P;
  const float* Lb = La + P * P;
  if (tid < P) srow[tid] = rec2[1 + tid];
  __syncthreads();
  // a P x P matrix into Mt transposed: thread i % 128 takes row i in 16-byte pieces; all 16 loads
  // of a thread are issued before its shared-memory stores
  auto load_t = [&](auto row_ptr) {
    float4 v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int f = tid + 256 * u, i = f % P, k = 4 * (f / P);
      v[u] = *reinterpret_cast<const float4*>(row_ptr(i) + k);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int f = tid + 256 * u, i = f % P, k = 4 * (f / P);
      Mt[k * LD + i] = v[u].x;
      Mt[(k + 1) * LD + i] = v[u].y;
      Mt[(k + 2) * LD + i] = v[u].z;
      Mt[(k + 3) * LD + i] = v[u].w;
    }
  };
  load_t([&](int i) { return A + static_cast<size_t>(srow[i]) * n + k0; });
  {
    float4 v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int f = tid + 256 * u, k = f / (P / 4), j = 4 * (f % (P / 4));
      v[u] = *reinterpret_cast<const float4*>(La + k * P + j);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int f = tid + 256 * u, k = f / (P / 4), j = 4 * (f % (P / 4));
      // inv(L_1) is lower triangular: entries above the diagonal are zero
      *reinterpret_cast<float4*>(Ia + k * LD + j) =
          make_float4(k >= j ? v[u].x : 0.f, k >= j + 1 ? v[u].y : 0.f, k >= j + 2 ? v[u].z : 0.f,
                      k >= j + 3 ? v[u].w : 0.f);
    }
  }
  __syncthreads();
  const int ti = tid / 16, tj = tid % 16;  // rows 8 ti .. +7, columns 8 tj .. +7
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  for (int k = 8 * tj; k < P; ++k) {  // inv(L_1)[k][j] = 0 for k < j
    const float4 a0 = *reinterpret_cast<const float4*>(Mt + k * LD + 8 * ti);
    const float4 a1 = *reinterpret_cast<const float4*>(Mt + k * LD + 8 * ti + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(Ia + k * LD + 8 * tj);
    const float4 b1 = *reinterpret_cast<const float4*>(Ia + k * LD + 8 * tj + 4);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float* d = Ts + (8 * ti + r) * LD + 8 * tj;
    *reinterpret_cast<float4*>(d) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    *reinterpret_cast<float4*>(d + 4) = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
  }
  __syncthreads();
  load_t([&](int i) { return Lb + static_cast<size_t>(i) * P; });
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  for (int k = 0; k <= 8 * ti + 7; ++k) {  // inv(L_2)[i][k] = 0 for k > i
    const float4 a0 = *reinterpret_cast<const float4*>(Mt + k * LD + 8 * ti);
    const float4 a1 = *reinterpret_cast<const float4*>(Mt + k * LD + 8 * ti + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(Ts + k * LD + 8 * tj);
    const float4 b1 = *reinterpret_cast<const float4*>(Ts + k * LD + 8 * tj + 4);
    const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    float av[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) av[r] = k <= 8 * ti + r ? ar[r] : 0.f;
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
  }
  constexpr int W = 2 * P;
  float* oh = o_hi + static_cast<size_t>(mat) * W * W;
  float* ol = o_lo + static_cast<size_t>(mat) * W * W;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float4 hi, lo;
      split_tf32(-acc[r][4 * h], hi.x, lo.x);
      split_tf32(-acc[r][4 * h + 1], hi.y, lo.y);
      split_tf32(-acc[r][4 * h + 2], hi.z, lo.z);
      split_tf32(-acc[r][4 * h + 3], hi.w, lo.w);
      const size_t o = static_cast<size_t>(P + 8 * ti + r) * W + 8 * tj + 4 * h;
      *reinterpret_cast<float4*>(oh + o) = hi;
      *reinterpret_cast<float4*>(ol + o) = lo;
    }
  }
  // diagonal blocks (lower triangles of the panel inverses) and the zero block: 128 rows x 32 float4
#pragma unroll 4
  for (int u = 0; u < 16; ++u) {
    const int f = tid + 256 * u, i = f / (P / 4), j = 4 * (f % (P / 4));
    const float4 a = *reinterpret_cast<const float4*>(La + i * P + j);
    const float4 b = *reinterpret_cast<const float4*>(Lb + i * P + j);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
    float ha[4], la[4], hb[4], lb[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      split_tf32(j + e <= i ? av[e] : 0.f, ha[e], la[e]);
      split_tf32(j + e <= i ? bv[e] : 0.f, hb[e], lb[e]);
    }
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(oh + static_cast<size_t>(i) * W + j) = make_float4(ha[0], ha[1], ha[2], ha[3]);
    *reinterpret_cast<float4*>(ol + static_cast<size_t>(i) * W + j) = make_float4(la[0], la[1], la[2], la[3]);
    *reinterpret_cast<float4*>(oh + static_cast<size_t>(i) * W + P + j) = z;
    *reinterpret_cast<float4*>(ol + static_cast<size_t>(i) * W + P + j) = z;
    *reinterpret_cast<float4*>(oh + static_cast<size_t>(P + i) * W + P + j) = make_float4(hb[0], hb[1], hb[2], hb[3]);
    *reinterpret_cast<float4*>(ol + static_cast<size_t>(P + i) * W + P + j) = make_float4(lb[0], lb[1], lb[2], lb[3]);
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

// ((I (x) M_v) v)[r] for one point's vector v (global or shared memory): the banded row p = r mod nr
// of M_v against the block of v that holds r.
template <typename V>
__device__ __forceinline__ double mass_row(const MassBand& mb, const V* v, int r) {
  const int p = r % mb.nr, base = r - p;
  const int k0 = max(0, p - mb.w), k1 = min(mb.nr - 1, p + mb.w);
  const double* row = mb.m + static_cast<size_t>(p) * (2 * mb.w + 1) + mb.w - p;
  double acc = 0.0;
  for (int k = k0; k <= k1; ++k) acc = fma(__ldg(row + k), static_cast<double>(v[base + k]), acc);
  return acc;
}

// x = A^-1 b for one point per CTA, with the lazily applied pivots; Tc is the arithmetic type.
// With mass.m the right-hand side is (I (x) M_v) b.
// Column chunks of 32: the 32 x 32 diagonal block is staged in shared memory and solved by one
// warp, then every thread updates whole rows below (forward) or above (backward) the chunk.
template <typename T, typename Tc>
__global__ void __launch_bounds__(1024) lu_solve_kernel(const T* __restrict__ fac, const int* __restrict__ piv,
                                                        const double* __restrict__ b, double* __restrict__ x,
                                                        int n, int nb, const int* __restrict__ conv,
                                                        int accumulate, MassBand mass) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Tc* s = reinterpret_cast<Tc*>(smraw);
  __shared__ Tc dblk[32][33];
  const int mat = blockIdx.x;
  if (conv && conv[mat]) return;
  const T* A = fac + static_cast<size_t>(mat) * n * n;
  const int* ip = piv + static_cast<size_t>(mat) * n;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const double* bp = b + static_cast<size_t>(mat) * n;
  for (int r = tid; r < n; r += bd) s[r] = static_cast<Tc>(mass.m ? mass_row(mass, bp, r) : bp[r]);
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

// y = A^-T c for one point per CTA, with the factors of the FP64 path (LAPACK-style pivots ip,
// row swaps not applied left of each panel). The forward solve is x = U^-1 E_k ... E_0 c with
// E_p = (per 32-column block: unit-lower block solve, then the update of all rows below) after the
// panel's swaps; its transpose runs the other way: U^-T (per 32 block ascending: subtract the
// column-block dots with the rows above, then the transposed triangular block), then per panel
// descending and per 32 block descending: subtract the column-block dots with the rows below,
// solve with the transposed unit-lower block, and finally undo the panel's swaps in reverse.
__device__ void colblock_dots(const double* A, int n, int j0, int cw, int r0, int r1, const double* s,
                              double (*red)[33], double* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double acc = 0.0;
  if (lane < cw)
    for (int r = r0 + warp; r < r1; r += nw) acc += A[static_cast<size_t>(r) * n + j0 + lane] * s[r];
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w][lane];
    if (lane < cw) out[lane] = t;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) lu_solve_t_kernel(const double* __restrict__ fac, const int* __restrict__ piv,
                                                          const double* __restrict__ b, double* __restrict__ x,
                                                          int n, int nb, MassBand mass) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* s = reinterpret_cast<double*>(smraw);
  __shared__ double red[32][33];
  __shared__ double dot[32];
  __shared__ double dblk[32][33];
  const int mat = blockIdx.x;
  const double* A = fac + static_cast<size_t>(mat) * n * n;
  const int* ip = piv + static_cast<size_t>(mat) * n;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int r = tid; r < n; r += bd) s[r] = b[static_cast<size_t>(mat) * n + r];
  __syncthreads();
  // z = U^-T c
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int cw = min(32, n - j0);
    if (j0 > 0) {
      colblock_dots(A, n, j0, cw, 0, j0, s, red, dot);
      for (int c = tid; c < cw; c += bd) s[j0 + c] -= dot[c];
    }
    for (int idx = tid; idx < cw * cw; idx += bd) {
      const int r = idx / cw, c = idx % cw;
      dblk[r][c] = A[static_cast<size_t>(j0 + r) * n + j0 + c];
    }
    __syncthreads();
    if (warp == 0) {
      double v = lane < cw ? s[j0 + lane] : 0.0;
      for (int c = 0; c < cw; ++c) {
        if (lane == c) v /= dblk[c][c];
        const double zc = __shfl_sync(0xffffffffu, v, c);
        if (lane > c && lane < cw) v -= dblk[c][lane] * zc;
      }
      if (lane < cw) s[j0 + lane] = v;
    }
    __syncthreads();
  }
  // panels descending: L-blocks transposed, then the swaps undone
  const int npan = (n + nb - 1) / nb;
  for (int p = npan - 1; p >= 0; --p) {
    const int k0 = p * nb, kb = min(nb, n - k0);
    for (int j0 = k0 + ((kb - 1) / 32) * 32; j0 >= k0; j0 -= 32) {
      const int cw = min(32, k0 + kb - j0);
      if (j0 + cw < n) {
        colblock_dots(A, n, j0, cw, j0 + cw, n, s, red, dot);
        for (int c = tid; c < cw; c += bd) s[j0 + c] -= dot[c];
      }
      for (int idx = tid; idx < cw * cw; idx += bd) {
        const int r = idx / cw, c = idx % cw;
        dblk[r][c] = A[static_cast<size_t>(j0 + r) * n + j0 + c];
      }
      __syncthreads();
      if (warp == 0) {
        double v = lane < cw ? s[j0 + lane] : 0.0;
        for (int c = cw - 1; c >= 0; --c) {
          const double zc = __shfl_sync(0xffffffffu, v, c);
          if (lane < c) v -= dblk[c][lane] * zc;
        }
        if (lane < cw) s[j0 + lane] = v;
      }
      __syncthreads();
    }
    if (tid == 0)
      for (int j = kb - 1; j >= 0; --j) {
        const int q = ip[k0 + j];
        if (q != k0 + j) {
          const double t = s[k0 + j];
          s[k0 + j] = s[q];
          s[q] = t;
        }
      }
    __syncthreads();
  }
  for (int r = tid; r < n; r += bd) x[static_cast<size_t>(mat) * n + r] = mass.m ? mass_row(mass, s, r) : s[r];
}


// Sum of eight per-lane partials over the warp in nine shuffles (transposing butterfly): lane
// 4 k returns row k's total (k = 0..7).
__device__ __forceinline__ float warp_sum8(const float (&p)[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  float a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = h16 ? p[4 + i] : p[i], send = h16 ? p[i] : p[4 + i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float b2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = h8 ? a[2 + i] : a[i], send = h8 ? a[i] : a[2 + i];
    b2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float keep = h4 ? b2[1] : b2[0], send = h4 ? b2[0] : b2[1];
  float u = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  u += __shfl_xor_sync(0xffffffffu, u, 2);
  u += __shfl_xor_sync(0xffffffffu, u, 1);
  return u;
}

// out(r, dot(M[r, 0:128], v)) for rows r in [r0, r1) of a row-major FP32 matrix with leading
// dimension ld (a multiple of 4, M 16-byte aligned): eight rows per warp and pass, one 16-byte
// streaming load per lane and row, so that a CTA keeps 128 KB of loads in flight. v is in shared
// memory. The total of row r0 + 8 pass + k sits in lane 4k (bits 4, 3, 2 of the lane = k).
template <typename Out>
__device__ __forceinline__ void rows_dot128(const float* __restrict__ M, size_t ld, int r0, int r1, const float* v,
                                            int warp, int nwarp, int lane, Out out) {
  const float4 vv = reinterpret_cast<const float4*>(v)[lane];
  for (int r = r0 + 8 * warp; r < r1; r += 8 * nwarp) {
    float p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      p[i] = 0.f;
      if (r + i < r1) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(M + static_cast<size_t>(r + i) * ld) + lane);
        p[i] = a.x * vv.x + a.y * vv.y + a.z * vv.z + a.w * vv.w;
      }
    }
    const float t = warp_sum8(p, lane);
    const int k = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && r + k < r1) out(r + k, t);
  }
}

// out(r, dot(M[r, 0:kb], v)) for any width: one row per warp, lanes across the columns.
template <typename T, typename Out>
__device__ __forceinline__ void rows_dot_any(const T* __restrict__ M, size_t ld, int r0, int r1, int kb, const T* v,
                                             int warp, int nwarp, int lane, Out out) {
  for (int r = r0 + warp; r < r1; r += nwarp) {
    const T* a = M + static_cast<size_t>(r) * ld;
    T acc = T(0);
    for (int c = lane; c < kb; c += 32) acc += a[c] * v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out(r, acc);
  }
}

template <typename T, typename Out>
__device__ __forceinline__ void rows_dot(const T* __restrict__ M, size_t ld, int r0, int r1, int kb, const T* v,
                                         int warp, int nwarp, int lane, Out out) {
  if constexpr (sizeof(T) == 4) {
    if (kb == 128 && (ld & 3) == 0) {
      rows_dot128(M, ld, r0, r1, v, warp, nwarp, lane, out);
      return;
    }
  }
  rows_dot_any(M, ld, r0, r1, kb, v, warp, nwarp, lane, out);
}

// x = A^-1 c (or x += A^-1 c), c = b or (I (x) M_v) b, for one point per CTA with the per-panel
// block inverses: forward,
// per panel p: permute the right-hand side with the panel's row record, y = inv(L11_p) b_p, then
// b[below] -= L21_p y; backward, per panel from the last: y = inv(U11_p) b_p, b[above] -= U_p y.
// Every product is a batch of row dot products (rows_dot): the stored inverses are zero outside
// their triangles, so full rows are used. The factors are streamed once per solve.
template <typename T>
__global__ void __launch_bounds__(1024) lu_solve_blocked_kernel(const T* __restrict__ fac, const int* __restrict__ perm,
                                                                const T* __restrict__ linv, const T* __restrict__ uinv,
                                                                const double* __restrict__ b, double* __restrict__ x,
                                                                int n, int nb, const int* __restrict__ conv,
                                                                int accumulate, MassBand mass) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* s = reinterpret_cast<T*>(smraw);   // n (rounded up to 4)
  T* y = s + ((n + 3) & ~3);             // nb
  T* tmp = y + nb;                       // 2 nb
  const int mat = blockIdx.x;
  if (conv && conv[mat]) return;
  const T* A = fac + static_cast<size_t>(mat) * n * n;
  const int npan = (n + nb - 1) / nb;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = bd >> 5;
  const double* bp = b + static_cast<size_t>(mat) * n;
  for (int r = tid; r < n; r += bd) s[r] = static_cast<T>(mass.m ? mass_row(mass, bp, r) : bp[r]);
  __syncthreads();
  auto set_y = [&](int r, T v) { y[r] = v; };
  auto sub_s = [&](int r, T v) { s[r] -= v; };
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
    rows_dot(X, nb, 0, kb, kb, s + k0, warp, nwarp, lane, set_y);
    __syncthreads();
    for (int j = tid; j < kb; j += bd) s[k0 + j] = y[j];
    __syncthreads();
    rows_dot(A + k0, n, k0 + kb, n, kb, y, warp, nwarp, lane, sub_s);
    __syncthreads();
  }
  for (int p = npan - 1; p >= 0; --p) {
    const int k0 = p * nb, kb = min(nb, n - k0);
    const T* Y = uinv + (static_cast<size_t>(mat) * npan + p) * nb * nb;
    rows_dot(Y, nb, 0, kb, kb, s + k0, warp, nwarp, lane, set_y);
    __syncthreads();
    for (int j = tid; j < kb; j += bd) s[k0 + j] = y[j];
    __syncthreads();
    rows_dot(A + k0, n, 0, k0, kb, y, warp, nwarp, lane, sub_s);
    __syncthreads();
  }
  double* xo = x + static_cast<size_t>(mat) * n;
  for (int r = tid; r < n; r += bd) xo[r] = accumulate ? xo[r] + static_cast<double>(s[r]) : static_cast<double>(s[r]);
}

}  // namespace

// dynamic shared memory cap of lu_panel_kernel
constexpr int kPanelDynSmemMax = 226 * 1024;

// sub-panel width: largest power of two <= 32 whose shared-memory plan fits the budget
template <typename T>
static int panel_width(int n, int nb) {
  int w = 32;
  while (w > 2 && panel_smem_bytes<T>(n, nb, nb, w) > 210 * 1024) w >>= 1;
  return w < nb ? w : nb;
}


template <typename T, int W, int RPT>
static void launch_lazy(T* fac, int* piv, int* perm, T* linv, T* uinv, int nx, int n, int k0, int nb, int nbmax,
                        unsigned* status, float* li_hi, float* li_lo, const CUtensorMap* map, cudaStream_t st) {
  constexpr int NT = 512;
  constexpr bool kTc = std::is_same<T, float>::value && W == 16 && RPT == 4;
  static bool attr_set = false;
  if (!attr_set) {
    // static shared memory (18 KB; 35 KB with the tensor-core state) plus this cap within 227 KB
    cudaFuncSetAttribute(lu_panel_lazy_kernel<T, W, RPT, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    if constexpr (kTc)
      cudaFuncSetAttribute(lu_panel_lazy_kernel<T, W, RPT, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           190 * 1024);
    attr_set = true;
  }
  const size_t smem = panel_lazy_smem_bytes(n - k0, nb, nbmax, sizeof(T));
  CUtensorMap m{};
  if constexpr (kTc) {
    if (map) {
      m = *map;
      lu_panel_lazy_kernel<T, W, RPT, NT, true><<<nx, NT, smem, st>>>(fac, piv, perm, linv, uinv, n, k0, nb, nbmax,
                                                                    status, li_hi, li_lo, m);
      return;
    }
  }
  lu_panel_lazy_kernel<T, W, RPT, NT, false><<<nx, NT, smem, st>>>(fac, piv, perm, linv, uinv, n, k0, nb, nbmax,
                                                                 status, li_hi, li_lo, m);
}

// The tensor map of the per-point matrices for the panel's tensor-core left-looking update (cached
// for the last (fac, nx, n)); NULL if it cannot be made.
static const CUtensorMap* panel_matrix_map(float* fac, int nx, int n) {
  static float* key_fac = nullptr;
  static int key_nx = 0, key_n = 0;
  static bool ok = false;
  static CUtensorMap m;
  if (fac != key_fac || nx != key_nx || n != key_n) {
    ok = tc_matrix_map(&m, fac, nx, n);
    key_fac = fac, key_nx = nx, key_n = n;
  }
  return ok ? &m : nullptr;
}

// Column-block width and rows per thread of the mark-pivoting panel kernel (512 threads) for a
// panel of m0 rows and width nb (W = 0: the kernel does not apply). The W x rows-per-thread block
// of the panel held in registers stays at 64 values per thread.
// w_pref selects the narrower block (W4, 8 rows per thread) where both apply; 0 picks by shape.
template <typename T>
static void lazy_shape(int n, int m0, int nb, int nbmax, int w_pref, int& W, int& rpt) {
  constexpr int VE = 16 / sizeof(T);
  constexpr int W2 = sizeof(T) == 4 ? 16 : 8, W4 = sizeof(T) == 4 ? 8 : 4;
  W = 0, rpt = 0;
  if (n % VE != 0 || nbmax > 128 || nbmax % VE != 0) return;
  if (m0 <= 2048 && nb % W2 == 0 && w_pref != W4) W = W2, rpt = 4;
  else if (m0 <= 4096 && nb % W4 == 0) W = W4, rpt = 8;
}

template <typename T>
bool lu_panel_fuses_uinv(int n, int nbmax, int w_pref) {
  for (int k0 = 0; k0 < n; k0 += nbmax) {
    int W, rpt;
    lazy_shape<T>(n, n - k0, std::min(nbmax, n - k0), nbmax, w_pref, W, rpt);
    if (!W) return false;
  }
  return true;
}

template <typename T>
void launch_lu_panel(T* fac, int* piv, int* perm, T* linv, T* uinv, int nx, int n, int k0, int nb, int nbmax,
                     unsigned* status, float* ws_hi, float* ws_lo, float* li_hi, float* li_lo, int w_pref,
                     cudaStream_t st, bool tc_ll) {
  const bool trail = k0 + nb < n;
  float* wh = trail ? ws_hi : nullptr;
  float* lh = trail ? li_hi : nullptr;
  int W, rpt;
  lazy_shape<T>(n, n - k0, nb, nbmax, w_pref, W, rpt);
  constexpr int W2 = sizeof(T) == 4 ? 16 : 8, W4 = sizeof(T) == 4 ? 8 : 4;
  if (W == W2 && rpt == 4) {
    // the tensor-core left-looking update needs a full 128-column panel (its tiles fit beside the
    // diagonal block) and 16-byte aligned matrix rows
    const CUtensorMap* map = nullptr;
    if constexpr (sizeof(T) == 4) {
      if (tc_ll && nb == 128 && nbmax == 128 && n % 4 == 0 &&
          (static_cast<size_t>(nb) * (nb + 4) + lazy_tmp_elems(nb)) * sizeof(T) >= kTcllBytes)
        map = panel_matrix_map(reinterpret_cast<float*>(fac), nx, n);
    }
    launch_lazy<T, W2, 4>(fac, piv, perm, linv, uinv, nx, n, k0, nb, nbmax, status, lh, li_lo, map, st);
    return;
  }
  if (W == W4 && rpt == 8) {
    launch_lazy<T, W4, 8>(fac, piv, perm, linv, uinv, nx, n, k0, nb, nbmax, status, lh, li_lo, nullptr, st);
    return;
  }
  const int Wf = panel_width<T>(n, nbmax);
  const size_t smem = panel_smem_bytes<T>(n - k0, nb, nbmax, Wf);
  static bool attr_set = false;
  if (!attr_set) {
    // 226 KB: with the kernel's static shared memory (a few hundred bytes) within the 227 KB a CTA
    // may opt in to. The narrowest plan (W = 2) of the largest accepted order, nv = 7936 in FP64,
    // takes 225,336 bytes.
    cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelDynSmemMax);
    attr_set = true;
  }
  lu_panel_kernel<T><<<nx, 1024, smem, st>>>(fac, piv, perm, linv, n, k0, nb, nbmax, Wf, status, wh, ws_lo, lh, li_lo);
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

void launch_lu_swap_pack(float* fac, const int* perm, int nx, int n, int k0, int nb, int nbmax, int ncols,
                         int ks, float* bt_hi, float* bt_lo, float* a_hi, float* a_lo, cudaStream_t st) {
  const int ntrail = n - k0 - nb;
  ncols = std::min(ncols, ntrail);
  if (ntrail <= 0 || ncols <= 0) return;
  const int by = (std::max(ncols, a_hi ? ntrail : 0) + kTrsmCols - 1) / kTrsmCols;
  dim3 grid(nx, by);
  const size_t smem = 2ull * nb * kTrsmLd * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_swap_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  lu_swap_pack_kernel<<<grid, 256, smem, st>>>(fac, perm, n, k0, nb, nbmax, ncols, ks, bt_hi, bt_lo, a_hi, a_lo);
}

void launch_lu_swap_pack_pair(float* fac, const int* perm, int nx, int n, int k0, int ks, float* bt_hi,
                              float* bt_lo, float* a_hi, float* a_lo, cudaStream_t st) {
  const int M = n - k0 - 2 * kPairP;
  if (M <= 0) return;
  const int ncb = (M + kPairCols - 1) / kPairCols;
  dim3 grid(nx, 2 * ncb);
  const size_t smem = 2ull * kPairP * kPairLd * sizeof(float) + 6ull * kPairP * sizeof(int);
  lu_swap_pack_pair_kernel<<<grid, 256, smem, st>>>(fac, perm, n, k0, ks, ncb, bt_hi, bt_lo, a_hi, a_lo);
}

void launch_lu_pair_linv(const float* fac, const int* perm, const float* linv, int nx, int n, int k0,
                         float* o_hi, float* o_lo, cudaStream_t st) {
  constexpr int P = kPairP;
  const size_t smem = 3ull * P * (P + 4) * sizeof(float) + P * sizeof(int);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_pair_linv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  lu_pair_linv_kernel<<<nx, 256, smem, st>>>(fac, perm, linv, n, k0, o_hi, o_lo);
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
                     const int* conv, int accumulate, cudaStream_t st, MassBand mass) {
  using Tc = T;
  const size_t smem = static_cast<size_t>(n) * sizeof(Tc);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_solve_kernel<T, Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr_set = true;
  }
  lu_solve_kernel<T, Tc><<<nx, 1024, smem, st>>>(fac, piv, b, x, n, nb, conv, accumulate, mass);
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

void launch_lu_solve_t(const double* fac, const int* piv, const double* b, double* x, int nx, int n, int nb,
                       cudaStream_t st, MassBand mass) {
  const size_t smem = sizeof(double) * n;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_solve_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  lu_solve_t_kernel<<<nx, 1024, smem, st>>>(fac, piv, b, x, n, nb, mass);
}

template <typename T>
void launch_lu_solve_blocked(const T* fac, const int* perm, const T* linv, const T* uinv, const double* b,
                             double* x, int nx, int n, int nb, const int* conv, int accumulate, cudaStream_t st,
                             MassBand mass) {
  const size_t smem = (static_cast<size_t>((n + 3) & ~3) + 3 * nb) * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lu_solve_blocked_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr_set = true;
  }
  lu_solve_blocked_kernel<T><<<nx, 1024, smem, st>>>(fac, perm, linv, uinv, b, x, n, nb, conv, accumulate, mass);
}

#define BTE_INST(T)                                                                                 \
  template void launch_lu_panel<T>(T*, int*, int*, T*, T*, int, int, int, int, int, unsigned*, float*,   \
                                   float*, float*, float*, int, cudaStream_t, bool);                      \
  template bool lu_panel_fuses_uinv<T>(int, int, int);                                              \
  template void launch_lu_uinv<T>(const T*, T*, int, int, int, cudaStream_t);                        \
  template void launch_lu_solve_blocked<T>(const T*, const int*, const T*, const T*, const double*,  \
                                           double*, int, int, int, const int*, int, cudaStream_t,   \
                                           MassBand);                                               \
  template void launch_lu_swap_trsm<T>(T*, const int*, const T*, int, int, int, int, int, float*, float*, \
                                       cudaStream_t);                                               \
  template void launch_lu_gemm_simt<T>(T*, int, int, int, int, cudaStream_t);                       \
  template void launch_lu_solve<T>(const T*, const int*, const double*, double*, int, int, int,     \
                                   const int*, int, cudaStream_t, MassBand);
BTE_INST(double)
BTE_INST(float)
#undef BTE_INST

}  // namespace bte
