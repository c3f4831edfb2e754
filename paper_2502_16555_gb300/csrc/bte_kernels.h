// Launch wrappers of the device kernels (plain pointers; all enqueue on `st`, none synchronise).
#pragma once

#include <cuda_runtime.h>

#include "bte_internal.h"

namespace bte {

enum StatusBits : unsigned {
  kZeroPivot = 1u,     // a zero or non-finite pivot in some per-point LU
  kNonFinite = 2u,     // NaN/Inf in the result of a step
  kNoConv = 4u,        // refinement did not reach the tolerance
  kTimeout = 8u,       // a bounded device-side wait expired (tensor-core pipeline)
  kNonFiniteIn = 16u,  // NaN/Inf in an input: the state handed in, or the field array
};

// The block-diagonal Galerkin mass matrix I (x) M_v acting on one point's vector, in blocks of nr
// (one block per ordinate, or per harmonic in the reduced form). M_v is banded with half width w and
// stored as m[p * (2 w + 1) + k - p + w] = M_v[p][k]. m == nullptr stands for the identity.
struct MassBand {
  const double* m = nullptr;
  int nr = 0;
  int w = 0;
};

// tensor-core (tcgen05) trailing updates of the FP32 LU; workspace of tc_workspace_bytes(), parts
// 0-1 L21 split, 2-3 (P A12)^T split, 4-5 one panel's inv(L11) split, 6-7 U12^T split, 8-9 a
// two-panel block's inv(L11) split (layout in bte_tc.cu)
bool tc_available();
// Tensor map (128 bytes into map) of the per-point FP32 matrices as a 3-D array [nx][n][n], boxes of
// 128 rows x 32 columns, 128-byte swizzle: the K-major operand tiles the tensor cores read.
bool tc_matrix_map(void* map, float* fac, int nx, int n);
size_t tc_workspace_bytes(int nx, int n, int nbmax);
float* tc_ws_part(void* ws, int nx, int n, int part);
constexpr int kTcKs = 256;  // K capacity (row length) of the operand parts
// One 128-wide panel at k0: U12 = inv(L11) (P A12) for the first ncols trailing columns (written
// into the matrix and, transposed and split, into parts 6-7), then A22 -= L21 U12 on those columns.
// probe != 0: every CTA's bounded wait expires before any work (testing the timeout path).
void tc_lu_u12(float* fac, int nx, int n, int k0, int ncols, void* ws, unsigned* status, cudaStream_t st,
               int probe = 0);
void tc_lu_gemm(float* fac, int nx, int n, int k0, int ncols, void* ws, unsigned* status, cudaStream_t st,
                int probe = 0);
// The two panels at k0 and k0 + 128 together (K = 256) on every column right of k0 + 256.
void tc_lu_u12_pair(float* fac, int nx, int n, int k0, void* ws, unsigned* status, cudaStream_t st, int probe = 0);
// cg = 2: 256 x 256 tiles on CTA pairs (where the GPU can co-schedule them); cg = 1: 128 x 128 tiles
// on single CTAs.
void tc_lu_gemm_pair(float* fac, int nx, int n, int k0, void* ws, unsigned* status, cudaStream_t st, int probe = 0,
                     int cg = 2);

// Y2[b] = s_b M_b Y[b] for the nt * nr pairs b = a nr + i: M_b = M + b nx^2 (per_pair) or the one
// matrix M; s_b = lam[i] mu[a] when lam is given (device arrays), else 1. Y, Y2 are [nt][nr][nx].
void launch_x_matvec(const double* M, bool per_pair, const double* lam, const double* mu, const double* Y,
                     double* Y2, int nx, int nt, int nr, cudaStream_t st);
// ---- x half step (Algorithm 1): eigen-basis transform, Q_ij apply, back transform
void launch_x_to_eigen(const double* F, const double* Uinv, double* Y, int nx, int nt, int nr,
                       unsigned* status, cudaStream_t st);
void launch_x_apply_q(const double* Q, const double* Y, double* Y2, int nx, int nt, int nr,
                      cudaStream_t st);
void launch_x_from_eigen(const double* Y2, const double* U, double* F, int nx, int nt, int nr,
                         unsigned* status, cudaStream_t st);

// ---- velocity step
// kNonFiniteIn in status if any of the nx field values E[i] is NaN or infinite
void launch_check_field(const double* E, int nx, unsigned* status, cudaStream_t st);
// The per-point matrix the dense path factors, (I (x) M_v) A_i = I (x) M_v - dt (KCg + E_i KAg)
// with KCg = P_O C P_S and KAg = P_O A_v P_S (no mass scaling), in storage type T (float or
// double), row-major per point. Its solves multiply the right-hand side by I (x) M_v first.
template <typename T>
void launch_v_form(const double* KCg, const double* KAg, MassBand mass, const double* E, double E_uniform,
                   double dt, T* fac, int nx, int nv, cudaStream_t st);
// ints per point of the panel permutation record written by lu_panel
int perm_record_ints(int nbmax);
// ws_hi/ws_lo (may be NULL): K-major TF32 head/remainder copies of L21 (panel) and of U12^T
// (swap_trsm) for the tensor-core trailing update, [point][n - nbmax][nbmax] floats.
// Per-point, per-panel records ([point][panel] ...): perm (perm_record_ints each) and inv(L11)
// (nbmax x nbmax each).
// li_hi/li_lo (may be NULL): TF32 split of inv(L11) for the tensor-core U12 formation.
// uinv (may be NULL): per-panel inv(U11) ([point][panel], nbmax x nbmax), written only by the
// mark-pivoting panel kernel, i.e. when lu_panel_fuses_uinv<T>(n, nbmax) holds.
// w_pref: preferred column-block width of the mark-pivoting kernel (0: chosen by shape).
template <typename T>
// tc_ll (FP32, full 128-column panels of at most 2048 rows): the left-looking updates inside the
// panel run as TF32x3 tcgen05 MMAs instead of CUDA-core FMAs.
void launch_lu_panel(T* fac, int* piv, int* perm, T* linv, T* uinv, int nx, int n, int k0, int nb, int nbmax,
                     unsigned* status, float* ws_hi, float* ws_lo, float* li_hi, float* li_lo, int w_pref,
                     cudaStream_t st, bool tc_ll = false);
template <typename T>
bool lu_panel_fuses_uinv(int n, int nbmax, int w_pref);
// Tensor-core path: for the first ncols columns right of the panel, the displaced-row writes of the
// panel permutation and the split (P A12)^T operand (bt_hi/bt_lo); for every row below the panel,
// the split L21 operand (a_hi/a_lo). Operand rows are ks floats long.
void launch_lu_swap_pack(float* fac, const int* perm, int nx, int n, int k0, int nb, int nbmax, int ncols,
                         int ks, float* bt_hi, float* bt_lo, float* a_hi, float* a_lo, cudaStream_t st);
// The same for the two 128-wide panels at k0 and k0 + 128 taken together, on the columns and rows
// right of and below k0 + 256: both permutations applied in order, (P A12)^T over 256 rows of K, and
// the L21 operand [P_2 L21_1, L21_2] with the second panel's permutation applied to the first
// panel's columns (they stay unpermuted in the matrix, as the solve expects).
void launch_lu_swap_pack_pair(float* fac, const int* perm, int nx, int n, int k0, int ks, float* bt_hi,
                              float* bt_lo, float* a_hi, float* a_lo, cudaStream_t st);
// inv(L11) of the 256 x 256 two-panel block [L_1 0; (P_2 L21_1)_top L_2] from the two panels'
// inverses: [inv(L_1) 0; -inv(L_2) (P_2 L21_1)_top inv(L_1)  inv(L_2)], TF32-split into o_hi/o_lo
// ([point][256][256]).
void launch_lu_pair_linv(const float* fac, const int* perm, const float* linv, int nx, int n, int k0,
                         float* o_hi, float* o_lo, cudaStream_t st);
// inv(U11) of every panel of every point, once the factorisation is complete ([point][panel]).
template <typename T>
void launch_lu_uinv(const T* fac, T* uinv, int nx, int n, int nbmax, cudaStream_t st);
// x = A^-1 (I (x) M_v) b (x += when accumulate; plain A^-1 b when mass.m is NULL) through the
// per-panel block inverses; T is the arithmetic type.
template <typename T>
void launch_lu_solve_blocked(const T* fac, const int* perm, const T* linv, const T* uinv, const double* b,
                             double* x, int nx, int n, int nb, const int* conv, int accumulate, cudaStream_t st,
                             MassBand mass = {});
// ---- structure-exploiting velocity solve (block tridiagonal in l): Fout = A_i^-1 Fin per point
// (Fout += when accumulate); T is the arithmetic of the block elimination; Xscratch holds
// nx * nl * nr * nr values of T.
size_t struct_smem_bytes(int nr, int nl, size_t tsize);
template <typename T>
void launch_vsolve_struct(const double* Fin, double* Fout, const double* E, double E_uniform, double dt,
                          const double* Cs, const double* Alo, const double* Aup, const double* TO, const double* TS,
                          T* Xscratch, int nx, int nt, int nr, int nl, const int* conv, int accumulate,
                          unsigned* status, cudaStream_t st);

// The reduced dense system of the same identity when N_l < N_theta (m = N_l Nr): G_i = I - dt B_i
// (B_i = M^-1 (C + E_i A_v) in the harmonic basis) is factored in its unscaled form
// (I (x) M_v) G_i = I (x) M_v - dt (C + E_i A_v), formed densely as G[nx][m][m] from the blocks before
// the mass scaling (T the storage of the factorisation); y = P_S f and out (+)= f + P_O (z - y)
// around the solve z = G_i^-1 y (the solve multiplies y by I (x) M_v); Yr, Zr hold nx * m doubles;
// points with conv[i] != 0 are skipped (conv may be NULL).
template <typename T>
void launch_v_form_reduced(const double* Cg, const double* Aglo, const double* Agup, MassBand mass, const double* E,
                           double E_uniform, double dt, T* G, int nx, int nr, int nl, cudaStream_t st);
void launch_reduce_project(const double* F, const double* TS, double* Yr, const int* conv, int nx, int nt, int nr,
                           int nl, cudaStream_t st);
void launch_reduce_lift(const double* F, const double* Yr, const double* Zr, const double* TO, double* out,
                        const int* conv, int accumulate, int nx, int nt, int nr, int nl, cudaStream_t st);

// y = (I (x) M_v) A^-T b with the FP64 factors and pivots of the FP64 path (the adjoint of lu_solve;
// plain A^-T b when mass.m is NULL).
void launch_lu_solve_t(const double* fac, const int* piv, const double* b, double* x, int nx, int n, int nb,
                       cudaStream_t st, MassBand mass = {});
template <typename T>
void launch_lu_swap_trsm(T* fac, const int* perm, const T* linv, int nx, int n, int k0, int nb,
                         int nbmax, float* ws_hi, float* ws_lo, cudaStream_t st);
template <typename T>
void launch_lu_gemm_simt(T* fac, int nx, int n, int k0, int nb, cudaStream_t st);
// x = A^-1 (I (x) M_v) b (pivots applied lazily, panel by panel; plain A^-1 b when mass.m is NULL);
// `conv` (may be NULL) skips converged points. For T = float the arithmetic is FP32; the result is
// ADDED to x when `accumulate` is set.
template <typename T>
void launch_lu_solve(const T* fac, const int* piv, const double* b, double* x, int nx, int n, int nb,
                     const int* conv, int accumulate, cudaStream_t st, MassBand mass = {});

// The operators of the FP64 refinement residual, all before the mass scaling: C_0 dense ([nr][nr]);
// the band ([nr][2 w + 1], band[p][k - p + w]) of the loss part of C (the whole C_l for l >= 1);
// the bands of the field blocks (A_v)_{q,q-1} and (A_v)_{q,q+1} ([2][nl][nr][2 w + 1], zero where
// a block does not exist); the band of the Cholesky factor R of M_v ([nr][w + 1],
// chol[p][j] = R[p][p - w + j]) and 1 / R[p][p].
struct ResidualOps {
  const double* c0 = nullptr;
  const double* band = nullptr;
  const double* fband = nullptr;
  const double* chol = nullptr;
  const double* cinv = nullptr;
  int w = 0;
};
// FP64 residual r = b - (x - dt P_O M_v^-1 (C + E_i A_v) P_S x) (Algorithm 2's structured
// evaluation: the products with C and A_v are banded except C_0, and M_v^-1 is applied by banded
// Cholesky substitution), per-point ratio max|r|/max|b|; marks conv[i] = 1 when ratio <= tol or the
// normwise backward error is at FP64 rounding level.
void launch_residual(const double* x, const double* b, const double* E, double E_uniform, double dt,
                     const ResidualOps& ro, const double* TO, const double* TS, double* r, double* ratio, int* conv,
                     double tol, double kc_inf, double ka_inf, int nx, int nt, int nr, int nl, unsigned* status,
                     cudaStream_t st);
void launch_check_conv(const int* conv, int nx, unsigned* status, cudaStream_t st);

// ---- misc
void launch_commit(const double* src, double* dst, size_t n, const unsigned* status, cudaStream_t st);
void launch_moments(const double* F, const double* mom_n, const double* mom_e, const double* mom_r,
                    int n_proc, double* ne, double* mean, double* rates, int nx, int nv,
                    cudaStream_t st);
void launch_fill_maxwellian(double* F, const double* ne, const double* coef, int nx, int nt, int nr,
                            cudaStream_t st);

inline cudaStream_t handle_stream(const bte_handle* h) { return static_cast<cudaStream_t>(handle_stream_ptr(h)); }

}  // namespace bte
