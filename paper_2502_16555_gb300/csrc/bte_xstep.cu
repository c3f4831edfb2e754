// x half step (Algorithm 1 of arXiv 2502.16555), operator formation, FP64 refinement residual
// (Algorithm 2), moments and small helpers. All FP64 unless templated on the storage type.
#include <cuda_runtime.h>

#include <cstdint>

#include "bte_kernels.h"

namespace bte {
namespace {

constexpr int kXT = 32;  // x points per CTA in the eigen-basis transforms
constexpr int kIC = 32;  // eigen (to) or B-spline (from) indices per CTA: a third grid dimension
constexpr int kG = 4;    // output indices per thread in the transforms (one staged operand, four FMAs)

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// Y[a][i][x] = sum_k Uinv[i][k] F[x][a][k]  (the U^-1 contraction of Algorithm 1) for the kXT
// points and kIC eigen indices of this CTA: a thread takes kG consecutive i at one x, a warp shares
// them (the Uinv rows are broadcasts) and its lanes run over x. Flags non-finite inputs (blockIdx.z == 0 only), which is where a NaN handed in
// by the caller is first seen.
__global__ void x_to_eigen_kernel(const double* __restrict__ F, const double* __restrict__ Uinv,
                                  double* __restrict__ Y, int nx, int nt, int nr,
                                  unsigned* status) {
  extern __shared__ double sm[];
  const int a = blockIdx.x, x0 = blockIdx.y * kXT, i0 = blockIdx.z * kIC;
  const int nxt = min(kXT, nx - x0), nit = min(kIC, nr - i0);
  const int ld = nr + 1;  // padded row
  const bool check = status && blockIdx.z == 0;
  for (int idx = threadIdx.x; idx < nxt * nr; idx += blockDim.x) {
    const int xx = idx / nr, k = idx % nr;
    const double v = F[(static_cast<size_t>(x0 + xx) * nt + a) * nr + k];
    if (check && !finite(v)) atomicOr(status, kNonFiniteIn);
    sm[xx * ld + k] = v;
  }
  __syncthreads();
  const int ngr = (nit + kG - 1) / kG;
  for (int idx = threadIdx.x; idx < ngr * kXT; idx += blockDim.x) {
    const int ib = i0 + (idx / kXT) * kG, xx = idx % kXT;
    if (xx >= nxt) continue;
    const int nu = min(kG, i0 + nit - ib);
    const double* u = Uinv + static_cast<size_t>(ib) * nr;
    double s[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) s[g] = 0.0;
    for (int k = 0; k < nr; ++k) {
      const double f = sm[xx * ld + k];
#pragma unroll
      for (int g = 0; g < kG; ++g)
        if (g < nu) s[g] = fma(__ldg(u + static_cast<size_t>(g) * nr + k), f, s[g]);
    }
#pragma unroll
    for (int g = 0; g < kG; ++g)
      if (g < nu) Y[(static_cast<size_t>(a) * nr + ib + g) * nx + x0 + xx] = s[g];
  }
}

// Y2[b] = s_b M_b Y[b] for every (ordinate, eigen-index) pair b = a nr + i, M_b = M + b mstride
// (mstride = nx^2: the per-pair Q_ij of Algorithm 1; 0: one shared matrix), s_b = lam[i] mu[a]
// when lam is given, else 1. One CTA per pair; a warp owns 32 consecutive rows, lane l sums the
// columns c = l + 32 k of all 32 rows (each Q row chunk a coalesced 256-byte load), and a
// transpose reduction (shuffle offsets 16, 8, 4, 2, 1 exchanging half of the remaining rows) leaves
// row r0 + l's sum on lane l: 31 FP64 additions per lane for 32 rows instead of 5 per row and lane.
__global__ void x_matvec_kernel(const double* __restrict__ M, size_t mstride, const double* __restrict__ lam,
                                const double* __restrict__ mu, const double* __restrict__ Y,
                                double* __restrict__ Y2, int nx, int nr) {
  extern __shared__ double ys[];
  const size_t b = blockIdx.x;
  const double* y = Y + b * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  const double sb = lam ? lam[b % nr] * mu[b / nr] : 1.0;
  const double* Mb = M + b * mstride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r0 = 32 * warp; r0 < nx; r0 += 32 * nw) {
    const int nrow = min(32, nx - r0);
    const double* q = Mb + static_cast<size_t>(r0) * nx;
    double acc[32];
#pragma unroll
    for (int rr = 0; rr < 32; ++rr) acc[rr] = 0.0;
    for (int c = lane; c < nx; c += 32) {
      const double yc = ys[c];
#pragma unroll
      for (int rr = 0; rr < 32; ++rr)
        if (rr < nrow) acc[rr] = fma(__ldg(q + static_cast<size_t>(rr) * nx + c), yc, acc[rr]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const bool hi = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < o; ++k) {
        const double send = hi ? acc[k] : acc[k + o];
        const double keep = hi ? acc[k + o] : acc[k];
        acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    if (lane < nrow) Y2[b * nx + r0 + lane] = sb * acc[0];
  }
}

// F[x][a][k] = sum_i U[k][i] Y2[a][i][x] for the kXT points and kIC B-spline indices of this CTA:
// a thread takes kG consecutive k at one x, a warp shares them (the U rows are broadcasts) and its
// lanes run over x (consecutive shared-memory words); flags non-finite results.
__global__ void x_from_eigen_kernel(const double* __restrict__ Y2, const double* __restrict__ U,
                                    double* __restrict__ F, int nx, int nt, int nr,
                                    unsigned* status) {
  extern __shared__ double sm[];
  const int a = blockIdx.x, x0 = blockIdx.y * kXT, k0 = blockIdx.z * kIC;
  const int nxt = min(kXT, nx - x0), nkt = min(kIC, nr - k0);
  for (int idx = threadIdx.x; idx < nr * kXT; idx += blockDim.x) {
    const int i = idx / kXT, xx = idx % kXT;
    sm[i * (kXT + 1) + xx] = xx < nxt ? Y2[(static_cast<size_t>(a) * nr + i) * nx + x0 + xx] : 0.0;
  }
  __syncthreads();
  bool bad = false;
  const int ngr = (nkt + kG - 1) / kG;
  for (int idx = threadIdx.x; idx < ngr * kXT; idx += blockDim.x) {
    const int kb = k0 + (idx / kXT) * kG, xx = idx % kXT;
    if (xx >= nxt) continue;
    const int nu = min(kG, k0 + nkt - kb);
    const double* u = U + static_cast<size_t>(kb) * nr;
    double s[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) s[g] = 0.0;
    for (int i = 0; i < nr; ++i) {
      const double y = sm[i * (kXT + 1) + xx];
#pragma unroll
      for (int g = 0; g < kG; ++g)
        if (g < nu) s[g] = fma(__ldg(u + static_cast<size_t>(g) * nr + i), y, s[g]);
    }
#pragma unroll
    for (int g = 0; g < kG; ++g)
      if (g < nu) {
        bad |= !finite(s[g]);
        F[(static_cast<size_t>(x0 + xx) * nt + a) * nr + kb + g] = s[g];
      }
  }
  if (status && bad) atomicOr(status, kNonFinite);
}

template <typename T>
__global__ void v_form_kernel(const double* __restrict__ KCg, const double* __restrict__ KAg, MassBand mass,
                              const double* __restrict__ E, double E_uniform, double dt,
                              T* __restrict__ fac, int nx, int nv) {
  // Per element, base = M - dt KCg and slope = -dt KAg once in FP64; per point, one FMA in the
  // factor precision, base + E_i slope (for FP32 factors an FP32 FMA: GB300's FP64 rate would bound
  // the Nx FP64 operations per element at about eight times the store time). A per-point field is
  // staged in shared memory in that precision; the uniform field takes the same arithmetic, so
  // equal fields give equal factors on both paths.
  extern __shared__ __align__(8) unsigned char vf_smem[];
  T* Es = reinterpret_cast<T*>(vf_smem);
  if (E) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) Es[i] = static_cast<T>(E[i]);
    __syncthreads();
  }
  const T Eu = static_cast<T>(E_uniform);
  const size_t nn = static_cast<size_t>(nv) * nv;
  const int nr = mass.nr, bw = 2 * mass.w + 1;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < nn;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const double kc = KCg[e], ka = KAg[e];
    // (I (x) M_v)[(a,p),(b,k)] = M_v[p][k] when a == b and |p - k| <= w
    const int row = static_cast<int>(e / nv), col = static_cast<int>(e % nv);
    const int p = row % nr, k = col % nr, dk = k - p;
    const double d = (row - p == col - k && dk >= -mass.w && dk <= mass.w) ? __ldg(mass.m + p * bw + dk + mass.w) : 0.0;
    const T base = static_cast<T>(d - dt * kc), slope = static_cast<T>(-dt * ka);
    if (E) {
      for (int i = 0; i < nx; ++i) fac[static_cast<size_t>(i) * nn + e] = Es[i] * slope + base;
    } else {
      const T v = Eu * slope + base;
      for (int i = 0; i < nx; ++i) fac[static_cast<size_t>(i) * nn + e] = v;
    }
  }
}

// Refinement residual of one point (CTA per point), Algorithm 2 with the structured operators:
// xS = P_S x, g = M_v^-1 (C + E_i A_v) xS, r = b - x + dt P_O g. The products with C and A_v run
// over bands (the loss part of C, the field blocks; C_0 carries the gain and the heavy-temperature
// term and is dense); M_v^-1 is a forward and a backward substitution with the banded Cholesky
// factor of M_v along the B-spline index. The point has converged when
// max|r| <= tol max|b|, or when max|r| is already at the rounding level of an FP64 product A_i x,
// max|r| <= min(kBackwardFloor, tol) (|A_i| max|x| + max|b|) with |A_i| <= 1 + dt (|K_C| +
// |E_i| |K_A|) (infinity norms): a normwise backward error no refinement can improve on. The second
// test decides only for ill-conditioned A_i, where |A_i| |x| is far above |b|.
// 256 unit roundoffs of FP64: the normwise backward error at which a residual computed in FP64 is
// rounding noise.
constexpr double kBackwardFloor = 256.0 * 1.1102230246251565e-16;

__global__ void residual_kernel(const double* __restrict__ X, const double* __restrict__ B,
                                const double* __restrict__ E, double E_uniform, double dt, ResidualOps ro,
                                const double* __restrict__ TO, const double* __restrict__ TS, double* __restrict__ R,
                                double* __restrict__ ratio, int* __restrict__ conv, double tol,
                                double kc_inf, double ka_inf, int nt, int nr, int nl,
                                unsigned* __restrict__ status) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  // a point that has converged keeps its iterate (the solves skip it), so its residual is final
  if (conv[i]) return;
  const int nv = nt * nr;
  double* xs = sm;             // nv
  double* xS = xs + nv;        // nl*nr
  double* g = xS + nl * nr;    // nl*nr
  __shared__ double red_r[32], red_b[32], red_x[32];
  const double* x = X + static_cast<size_t>(i) * nv;
  const double* b = B + static_cast<size_t>(i) * nv;
  const double Ei = E ? E[i] : E_uniform;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) xs[v] = x[v];
  __syncthreads();
  for (int idx = threadIdx.x; idx < nl * nr; idx += blockDim.x) {
    const int l = idx / nr, k = idx % nr;
    double s = 0.0;
    for (int a = 0; a < nt; ++a) s = fma(__ldg(TS + l * nt + a), xs[a * nr + k], s);
    xS[idx] = s;
  }
  __syncthreads();
  const int w = ro.w, bw = 2 * w + 1;
  for (int idx = threadIdx.x; idx < nl * nr; idx += blockDim.x) {
    const int l = idx / nr, p = idx % nr;
    const int k0 = max(0, p - w), k1 = min(nr - 1, p + w);
    double c = 0.0, f = 0.0;
    if (l > 0) {   // C_0 (dense) is added in the next stage
      const double* row = ro.band + static_cast<size_t>(p) * bw + w - p;   // row[k] = loss[p][k]
      for (int k = k0; k <= k1; ++k) c = fma(__ldg(row + k), xS[l * nr + k], c);
    }
    if (l >= 1) {
      const double* row = ro.fband + (static_cast<size_t>(l) * nr + p) * bw + w - p;   // (A_v)_{l,l-1}[p][k]
      const double* y = xS + (l - 1) * nr;
      for (int k = k0; k <= k1; ++k) f = fma(__ldg(row + k), y[k], f);
    }
    if (l + 1 < nl) {
      const double* row = ro.fband + (static_cast<size_t>(nl + l) * nr + p) * bw + w - p;   // (A_v)_{l,l+1}[p][k]
      const double* y = xS + (l + 1) * nr;
      for (int k = k0; k <= k1; ++k) f = fma(__ldg(row + k), y[k], f);
    }
    g[idx] = c + Ei * f;
  }
  __syncthreads();
  // the dense C_0 rows (l = 0): eight lanes per row, each a strided part of the dot product, summed
  // over the lane group by shuffles (every thread runs the same number of rounds)
  {
    const int sub = threadIdx.x & 7, rows = blockDim.x >> 3;
    for (int pb = 0; pb < nr; pb += rows) {
      const int p = pb + (threadIdx.x >> 3);
      double c = 0.0;
      if (p < nr) {
        const double* row = ro.c0 + static_cast<size_t>(p) * nr;
        for (int k = sub; k < nr; k += 8) c = fma(__ldg(row + k), xS[k], c);
      }
      c += __shfl_down_sync(0xffffffffu, c, 4, 8);
      c += __shfl_down_sync(0xffffffffu, c, 2, 8);
      c += __shfl_down_sync(0xffffffffu, c, 1, 8);
      if (p < nr && sub == 0) g[p] += c;
    }
  }
  __syncthreads();
  // g_l <- M_v^-1 g_l, M_v = R R^T: R y = g_l (p ascending), then R^T z = y (p descending), one
  // thread per harmonic; for the cubic band (w = 3) the last three values stay in registers
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    double* gl = g + l * nr;
    if (w == 3) {
      double y1 = 0.0, y2 = 0.0, y3 = 0.0;   // y[p-1], y[p-2], y[p-3]
      for (int p = 0; p < nr; ++p) {
        const double* rrow = ro.chol + static_cast<size_t>(p) * 4;   // R[p][p-3], R[p][p-2], R[p][p-1], R[p][p]
        double s = fma(-__ldg(rrow + 2), y1, gl[p]);
        s = fma(-__ldg(rrow + 1), y2, s);
        s = fma(-__ldg(rrow), y3, s);
        const double y = s * __ldg(ro.cinv + p);
        gl[p] = y;
        y3 = y2, y2 = y1, y1 = y;
      }
      double z1 = 0.0, z2 = 0.0, z3 = 0.0;   // z[p+1], z[p+2], z[p+3]
      for (int p = nr - 1; p >= 0; --p) {
        double s = gl[p];
        if (p + 1 < nr) s = fma(-__ldg(ro.chol + static_cast<size_t>(p + 1) * 4 + 2), z1, s);
        if (p + 2 < nr) s = fma(-__ldg(ro.chol + static_cast<size_t>(p + 2) * 4 + 1), z2, s);
        if (p + 3 < nr) s = fma(-__ldg(ro.chol + static_cast<size_t>(p + 3) * 4), z3, s);
        const double z = s * __ldg(ro.cinv + p);
        gl[p] = z;
        z3 = z2, z2 = z1, z1 = z;
      }
    } else {
      for (int p = 0; p < nr; ++p) {
        const double* rrow = ro.chol + static_cast<size_t>(p) * (w + 1);   // rrow[j] = R[p][p - w + j]
        double s = gl[p];
        for (int j = max(0, w - p); j < w; ++j) s = fma(-__ldg(rrow + j), gl[p - w + j], s);
        gl[p] = s * __ldg(ro.cinv + p);
      }
      for (int p = nr - 1; p >= 0; --p) {
        double s = gl[p];
        const int kmax = min(nr - 1, p + w);
        for (int k = p + 1; k <= kmax; ++k) s = fma(-__ldg(ro.chol + static_cast<size_t>(k) * (w + 1) + p - k + w), gl[k], s);
        gl[p] = s * __ldg(ro.cinv + p);
      }
    }
  }
  __syncthreads();
  double mr = 0.0, mb = 0.0, mx = 0.0;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const int a = v / nr, p = v % nr;
    double s = 0.0;
    for (int l = 0; l < nl; ++l) s = fma(__ldg(TO + a * nl + l), g[l * nr + p], s);
    const double bv = b[v];
    const double rv = bv - xs[v] + dt * s;
    R[static_cast<size_t>(i) * nv + v] = rv;
    mr = fmax(mr, fabs(rv));
    mb = fmax(mb, fabs(bv));
    mx = fmax(mx, fabs(xs[v]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) red_r[threadIdx.x >> 5] = mr, red_b[threadIdx.x >> 5] = mb, red_x[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int wi = 1; wi < static_cast<int>(blockDim.x >> 5); ++wi)
      mr = fmax(mr, red_r[wi]), mb = fmax(mb, red_b[wi]), mx = fmax(mx, red_x[wi]);
    const double q = mb > 0.0 ? mr / mb : (mr > 0.0 ? INFINITY : 0.0);
    const double nA = 1.0 + dt * (kc_inf + fabs(Ei) * ka_inf);
    ratio[i] = q;
    conv[i] = (q <= tol || mr <= fmin(kBackwardFloor, tol) * (nA * mx + mb)) ? 1 : 0;
    atomicAdd(status + 1, 1u);  // residual evaluations (refinement accounting)
  }
}

__global__ void check_field_kernel(const double* __restrict__ E, int nx, unsigned* status) {
  bool bad = false;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) bad |= !isfinite(E[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kNonFiniteIn);
}

__global__ void check_conv_kernel(const int* conv, int nx, unsigned* status) {
  bool all = true;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) all &= conv[i] != 0;
  if (!__syncthreads_and(all) && threadIdx.x == 0) atomicOr(status, kNoConv);
}

__global__ void commit_kernel(const double* __restrict__ src, double* __restrict__ dst, size_t n,
                              const unsigned* status) {
  if (*status != 0u) return;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x)
    dst[e] = src[e];
}

// ne = mom_n . F_i, mean = (mom_e . F_i)/ne, rates_j = (mom_r_j . F_i)/ne; FP64 block reductions.
__global__ void moments_kernel(const double* __restrict__ F, const double* __restrict__ mn,
                               const double* __restrict__ me, const double* __restrict__ mr,
                               int n_proc, double* ne, double* mean, double* rates, int nx, int nv) {
  __shared__ double red[32];
  __shared__ double ne_s;
  const int i = blockIdx.x;
  const double* f = F + static_cast<size_t>(i) * nv;
  auto block_sum = [&](const double* w) {
    double s = 0.0;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) s = fma(w[v], f[v], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
      for (int w2 = 0; w2 < static_cast<int>(blockDim.x >> 5); ++w2) t += red[w2];
    return t;  // valid on thread 0
  };
  const double n = block_sum(mn);
  if (threadIdx.x == 0) {
    ne_s = n;
    if (ne) ne[i] = n;
  }
  __syncthreads();
  const double nn = ne_s;
  const double e = block_sum(me);
  if (threadIdx.x == 0 && mean) mean[i] = nn != 0.0 ? e / nn : 0.0;
  for (int j = 0; j < n_proc; ++j) {
    const double r = block_sum(mr + static_cast<size_t>(j) * nv);
    if (threadIdx.x == 0 && rates) rates[static_cast<size_t>(j) * nx + i] = nn != 0.0 ? r / nn : 0.0;
  }
}

__global__ void fill_maxwellian_kernel(double* F, const double* ne, const double* coef, int nx,
                                       int nt, int nr) {
  const size_t n = static_cast<size_t>(nx) * nt * nr;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = e / (static_cast<size_t>(nt) * nr);
    F[e] = ne[i] * coef[e % nr];
  }
}

int grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  return static_cast<int>(g < 1 ? 1 : g);
}

}  // namespace

// Both transforms stage nr x (kXT + 1) doubles: past 48 KB (nr > 186) they need the opt-in
// shared-memory size, which bte_create keeps them within (nr <= kMaxNr).
static void set_x_transform_smem() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(x_to_eigen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(x_from_eigen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  done = true;
}

void launch_x_to_eigen(const double* F, const double* Uinv, double* Y, int nx, int nt, int nr,
                       unsigned* status, cudaStream_t st) {
  set_x_transform_smem();
  dim3 grid(nt, (nx + kXT - 1) / kXT, (nr + kIC - 1) / kIC);
  const size_t smem = sizeof(double) * kXT * (nr + 1);
  x_to_eigen_kernel<<<grid, 256, smem, st>>>(F, Uinv, Y, nx, nt, nr, status);
}

void launch_x_matvec(const double* M, bool per_pair, const double* lam, const double* mu, const double* Y,
                     double* Y2, int nx, int nt, int nr, cudaStream_t st) {
  const int groups = (nx + 31) / 32;
  const int threads = 32 * (groups < 8 ? groups : 8);
  x_matvec_kernel<<<nt * nr, threads, sizeof(double) * nx, st>>>(
      M, per_pair ? static_cast<size_t>(nx) * nx : 0, lam, mu, Y, Y2, nx, nr);
}

void launch_x_apply_q(const double* Q, const double* Y, double* Y2, int nx, int nt, int nr,
                      cudaStream_t st) {
  launch_x_matvec(Q, true, nullptr, nullptr, Y, Y2, nx, nt, nr, st);
}

void launch_x_from_eigen(const double* Y2, const double* U, double* F, int nx, int nt, int nr,
                         unsigned* status, cudaStream_t st) {
  set_x_transform_smem();
  dim3 grid(nt, (nx + kXT - 1) / kXT, (nr + kIC - 1) / kIC);
  const size_t smem = sizeof(double) * nr * (kXT + 1);
  x_from_eigen_kernel<<<grid, 256, smem, st>>>(Y2, U, F, nx, nt, nr, status);
}

void launch_check_field(const double* E, int nx, unsigned* status, cudaStream_t st) {
  check_field_kernel<<<1, 256, 0, st>>>(E, nx, status);
}

template <typename T>
void launch_v_form(const double* KCg, const double* KAg, MassBand mass, const double* E, double E_uniform,
                   double dt, T* fac, int nx, int nv, cudaStream_t st) {
  const size_t nn = static_cast<size_t>(nv) * nv;
  const size_t smem = E ? sizeof(T) * static_cast<size_t>(nx) : 0;   // nx <= 4096: at most 32 KB
  v_form_kernel<T><<<grid_for(nn, 256), 256, smem, st>>>(KCg, KAg, mass, E, E_uniform, dt, fac, nx, nv);
}
template void launch_v_form<double>(const double*, const double*, MassBand, const double*, double, double,
                                    double*, int, int, cudaStream_t);
template void launch_v_form<float>(const double*, const double*, MassBand, const double*, double, double,
                                   float*, int, int, cudaStream_t);

void launch_residual(const double* x, const double* b, const double* E, double E_uniform, double dt,
                     const ResidualOps& ro, const double* TO, const double* TS, double* r, double* ratio, int* conv,
                     double tol, double kc_inf, double ka_inf, int nx, int nt, int nr, int nl, unsigned* status,
                     cudaStream_t st) {
  const size_t smem = sizeof(double) * (static_cast<size_t>(nt) * nr + 2 * nl * nr);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  residual_kernel<<<nx, 512, smem, st>>>(x, b, E, E_uniform, dt, ro, TO, TS, r, ratio, conv, tol, kc_inf, ka_inf, nt,
                                         nr, nl, status);
}

void launch_check_conv(const int* conv, int nx, unsigned* status, cudaStream_t st) {
  check_conv_kernel<<<1, 256, 0, st>>>(conv, nx, status);
}

void launch_commit(const double* src, double* dst, size_t n, const unsigned* status, cudaStream_t st) {
  commit_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, dst, n, status);
}

void launch_moments(const double* F, const double* mom_n, const double* mom_e, const double* mom_r,
                    int n_proc, double* ne, double* mean, double* rates, int nx, int nv,
                    cudaStream_t st) {
  moments_kernel<<<nx, 256, 0, st>>>(F, mom_n, mom_e, mom_r, n_proc, ne, mean, rates, nx, nv);
}

void launch_fill_maxwellian(double* F, const double* ne, const double* coef, int nx, int nt, int nr,
                            cudaStream_t st) {
  const size_t n = static_cast<size_t>(nx) * nt * nr;
  fill_maxwellian_kernel<<<grid_for(n, 256), 256, 0, st>>>(F, ne, coef, nx, nt, nr);
}

}  // namespace bte
