// Host-side (FP64) assembly of every operator of the discretisation in Section 3.4 of
// arXiv 2502.16555: Chebyshev collocation in x, clamped cubic B-splines in speed, Gauss-Legendre
// ordinates with Y_l0 projections in the polar angle, the collision and field Galerkin operators
// (eqs. "c_en_mat_1d", "c_T0_mat_1d", "adv_v_ws"), the mass-matrix scaling, the eigen-decomposition
// M_v^-1 G_v = U Lambda U^-1 and the precomputed inverses Q_ij of Algorithm 1.
//
// Readings taken where the paper is open or garbled: the collision weak form carries v^3 sigma
// (test measure v^2 times speed v); ionization releases two electrons at (eps - eps_ion)/2;
// excitation one electron at eps - eps_th; the heavy-temperature term is the dissipative
// -(n0 kB T0/m0) int v^3 sigma_el phi_p' phi_k' on the (0,0) block; the field operator follows
// from the strong form (eE/m_e)[mu d_v f + (1-mu^2)/v d_mu f] and the Legendre recurrences; T_S
// includes the azimuthal 2 pi; zero-inflow rows replace the collocation row at the inflow wall.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "bte_internal.h"

namespace bte {
namespace {

// ------------------------------------------------------------------------ small dense helpers

// In-place Cholesky A = R R^T (lower R stored in A). Returns false if A is not SPD.
bool cholesky(std::vector<double>& A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
    for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
  }
  return true;
}

// Inverse of a lower-triangular R (n x n).
std::vector<double> lower_inverse(const std::vector<double>& R, int n) {
  std::vector<double> X(n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    X[c * n + c] = 1.0 / R[c * n + c];
    for (int i = c + 1; i < n; ++i) {
      double s = 0;
      for (int k = c; k < i; ++k) s += R[i * n + k] * X[k * n + c];
      X[i * n + c] = -s / R[i * n + i];
    }
  }
  return X;
}

// Inverse of a general square matrix by LU with partial pivoting. Returns false if singular.
bool invert(std::vector<double> A, int n, double* out) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) best = std::fabs(A[i * n + k]), p = i;
    if (!(best > 0)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
    const double inv = 1.0 / A[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double l = (A[i * n + k] *= inv);
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  // solve for the identity, column by column
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    std::fill(col.begin(), col.end(), 0.0);
    col[c] = 1.0;
    for (int k = 0; k < n; ++k) std::swap(col[k], col[piv[k]]);
    for (int i = 0; i < n; ++i) {
      double s = col[i];
      for (int k = 0; k < i; ++k) s -= A[i * n + k] * col[k];
      col[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = col[i];
      for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * col[k];
      col[i] = s / A[i * n + i];
    }
    for (int i = 0; i < n; ++i) out[i * n + c] = col[i];
  }
  return true;
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations: S = Z diag(w) Z^T, w ascending.
// Each rotation zeroes a_pq exactly and moves t*a_pq between the two diagonal entries (the
// rounding-friendly form of the update), and the sweeps stop once no off-diagonal entry is larger
// than 1e-18 of the geometric mean of its two diagonal entries.
void jacobi_eigen(std::vector<double> S, int n, std::vector<double>& w, std::vector<double>& Z) {
  Z.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = S[p * n + q];
        const double app = S[p * n + p], aqq = S[q * n + q];
        if (std::fabs(apq) <= 1e-18 * std::sqrt(std::fabs(app * aqq)) || apq == 0.0) continue;
        rotated = true;
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          if (k == p || k == q) continue;
          const double skp = S[k * n + p], skq = S[k * n + q];
          const double np_ = c * skp - s * skq, nq = s * skp + c * skq;
          S[k * n + p] = S[p * n + k] = np_;
          S[k * n + q] = S[q * n + k] = nq;
        }
        S[p * n + p] = app - t * apq;
        S[q * n + q] = aqq + t * apq;
        S[p * n + q] = S[q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {
          const double zkp = Z[k * n + p], zkq = Z[k * n + q];
          Z[k * n + p] = c * zkp - s * zkq;
          Z[k * n + q] = s * zkp + c * zkq;
        }
      }
    if (!rotated) break;
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return S[a * n + a] < S[b * n + b]; });
  w.resize(n);
  std::vector<double> Zs(n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = S[order[j] * n + order[j]];
    for (int i = 0; i < n; ++i) Zs[i * n + j] = Z[i * n + order[j]];
  }
  Z.swap(Zs);
}

// ------------------------------------------------------------------------ quadrature

// Gauss-Legendre nodes (ascending) and weights on [-1, 1], Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 2; l <= n; ++l) {
        const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p1 = z, p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // one more evaluation of the derivative at the converged node
        p0 = 1.0, p1 = z;
        for (int l = 2; l <= n; ++l) {
          const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) p1 = z, p0 = 1.0;
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Rule {
  std::vector<double> x, w;
  explicit Rule(int n) { gauss_legendre(n, x, w); }
};

// Visit every node of a composite Gauss rule over the sorted, de-duplicated breakpoints.
void composite(std::vector<double> br, const Rule& r, const std::function<void(double, double)>& f) {
  std::sort(br.begin(), br.end());
  for (size_t s = 0; s + 1 < br.size(); ++s) {
    const double a = br[s], b = br[s + 1];
    if (!(b > a)) continue;
    const double h = 0.5 * (b - a), m = 0.5 * (a + b);
    for (size_t q = 0; q < r.x.size(); ++q) f(m + h * r.x[q], h * r.w[q]);
  }
}

// ------------------------------------------------------------------------ B-splines

struct Spline {
  int nr;
  double vmax, h;
  std::vector<double> t;
  Spline(int nr_, double vmax_) : nr(nr_), vmax(vmax_), h(vmax_ / (nr_ - 3)), t(nr_ + 4) {
    for (int i = 0; i < 3; ++i) t[i] = 0.0, t[nr + 1 + i] = vmax;
    for (int j = 0; j <= nr - 3; ++j) t[3 + j] = (j == nr - 3) ? vmax : j * h;
  }
  // Span s (3 <= s <= nr-1) with t[s] <= v < t[s+1]; v == vmax goes to the last span.
  int span(double v) const {
    int s = 3 + static_cast<int>(std::floor(v / h));
    s = std::min(std::max(s, 3), nr - 1);
    while (s > 3 && v < t[s]) --s;
    while (s < nr - 1 && v >= t[s + 1]) ++s;
    return s;
  }
  // Nonzero cubic functions phi_{s-3..s}(v) and their derivatives (triangular Cox-de Boor scheme).
  // Returns false when v is outside [0, vmax].
  bool eval(double v, int& s, double N[4], double dN[4]) const {
    if (v < 0.0 || v > vmax) return false;
    s = span(v);
    double left[4], right[4], B[4] = {1.0, 0, 0, 0}, B2[3] = {0, 0, 0};
    for (int j = 1; j <= 3; ++j) {
      left[j] = v - t[s + 1 - j];
      right[j] = t[s + j] - v;
      double saved = 0.0;
      for (int r = 0; r < j; ++r) {
        const double tmp = B[r] / (right[r + 1] + left[j - r]);
        B[r] = saved + right[r + 1] * tmp;
        saved = left[j - r] * tmp;
      }
      B[j] = saved;
      if (j == 2) B2[0] = B[0], B2[1] = B[1], B2[2] = B[2];
    }
    for (int m = 0; m < 4; ++m) {
      N[m] = B[m];
      const int i = s - 3 + m;  // global index of this function
      double d = 0.0;
      if (m >= 1) d += B2[m - 1] / (t[i + 3] - t[i]);
      if (m <= 2) d -= B2[m] / (t[i + 4] - t[i + 1]);
      dN[m] = 3.0 * d;
    }
    return true;
  }
};

// ------------------------------------------------------------------------ cross sections

double energy_eV(double v) { return 0.5 * kMe * v * v / kE; }
double speed(double eps_eV) { return std::sqrt(2.0 * kE * eps_eV / kMe); }

double sigma(const Process& p, double v) {
  const double eps = energy_eV(v);
  double s = 0.0;
  switch (p.form) {
    case BTE_SIGMA_CONST: s = p.sigma0; break;
    case BTE_SIGMA_LINEAR: s = eps > p.th_eV ? p.sigma0 * (1.0 - p.th_eV / eps) : 0.0; break;
    case BTE_SIGMA_LOG: {
      if (eps > p.th_eV) {
        const double r = eps / p.th_eV;
        s = p.sigma0 * std::log(r) / r;
      }
      break;
    }
    case BTE_SIGMA_NU: s = v > 0 ? p.sigma0 / v : 0.0; break;
    case BTE_SIGMA_TABLE: {
      const auto& e = p.tab_eps;
      const auto& g = p.tab_sigma;
      if (e.empty() || eps < e.front() || eps > e.back()) break;
      if (p.th_eV > 0 && eps <= p.th_eV) break;
      size_t j = std::upper_bound(e.begin(), e.end(), eps) - e.begin();
      if (j == 0) j = 1;
      if (j >= e.size()) j = e.size() - 1;
      const double a = (eps - e[j - 1]) / (e[j] - e[j - 1]);
      s = g[j - 1] + a * (g[j] - g[j - 1]);
      break;
    }
    default: break;
  }
  return p.scale * s;
}

std::vector<double> sigma_breaks(const Process& p) {
  std::vector<double> b;
  if (p.kind != BTE_ELASTIC && p.th_eV > 0) b.push_back(speed(p.th_eV));
  if (p.form == BTE_SIGMA_TABLE)
    for (double e : p.tab_eps)
      if (e > 0) b.push_back(speed(e));
  return b;
}

// Post-collision speed u(v) and its inverse v(u) with dv/du.
struct Collision {
  int kind;
  double c = 0, alpha = 1, g = 1;
  Collision(const Process& p, double m0) : kind(p.kind) {
    if (kind == BTE_ELASTIC) {
      alpha = std::sqrt(1.0 - 2.0 * kMe / m0);
    } else {
      c = 2.0 * kE * p.th_eV / kMe;
      g = (kind == BTE_IONIZATION) ? 2.0 : 1.0;
    }
  }
  double u_of_v(double v) const {
    if (kind == BTE_ELASTIC) return alpha * v;
    const double d = v * v - c;
    if (d <= 0) return 0.0;
    return kind == BTE_EXCITATION ? std::sqrt(d) : std::sqrt(0.5 * d);
  }
  double v_of_u(double u, double& dvdu) const {
    if (kind == BTE_ELASTIC) {
      dvdu = 1.0 / alpha;
      return u / alpha;
    }
    const double v = kind == BTE_EXCITATION ? std::sqrt(u * u + c) : std::sqrt(2.0 * u * u + c);
    dvdu = (kind == BTE_EXCITATION ? u : 2.0 * u) / v;
    return v;
  }
  bool maps(double v) const { return kind == BTE_ELASTIC || v * v > c; }
};

std::vector<double> clip(std::vector<double> b, double lo, double hi) {
  std::vector<double> out;
  for (double x : b)
    if (x >= lo && x <= hi) out.push_back(x);
  out.push_back(lo);
  out.push_back(hi);
  return out;
}

}  // namespace

// ------------------------------------------------------------------------ x-side assembly

std::string assemble_x(const bte_config& cfg, HostOps& o) {
  o.nx = cfg.nx;
  o.nr = cfg.nr;
  o.nt = cfg.ntheta;
  o.nl = cfg.nl > 0 ? cfg.nl : cfg.ntheta;
  o.nv = o.nr * o.nt;
  o.L = cfg.L_m;
  o.vmax = speed(cfg.vmax_eV);
  o.T0 = cfg.T0_K;
  o.n0 = cfg.p_Torr * kTorr / (kKB * cfg.T0_K);
  o.m0 = cfg.m0_amu * kAmu;
  o.dt = cfg.dt_s;
  const int nx = o.nx, nr = o.nr, nt = o.nt, nl = o.nl;

  // Chebyshev-Gauss-Lobatto points x_i = (L/2)(1 - s_i), s_i = cos(pi i/(nx-1)), and the
  // collocation derivative: D_s[i][j] = (c_i/c_j)(-1)^{i+j}/(s_i - s_j), c_0 = c_N = 2, else 1,
  // the differences written with sines for accuracy, diagonal by the negative row sum; d/dx = -(2/L) d/ds.
  const int N = nx - 1;
  o.x.resize(nx);
  for (int i = 0; i < nx; ++i) o.x[i] = 0.5 * o.L * (1.0 - std::cos(kPi * i / N));
  o.x[0] = 0.0;
  o.x[N] = o.L;
  // Clenshaw-Curtis weights for these points on [0, L]: w_i = (L/2) c_i/N (1 - sum_k b_k
  // cos(2 k theta_i)/(4k^2 - 1)), theta_i = pi i/N, b_k = 1 for k = N/2 and 2 below, c = 1/2 at the
  // ends and 1 inside (the cosine series of the interpolant integrated term by term)
  o.ccw.assign(nx, 0.0);
  for (int i = 0; i <= N; ++i) {
    const double th = kPi * i / N;
    double sum = 0.0;
    for (int k = 1; 2 * k <= N; ++k) {
      const double bk = (2 * k == N) ? 1.0 : 2.0;
      sum += bk * std::cos(2.0 * k * th) / (4.0 * k * k - 1.0);
    }
    const double ci = (i == 0 || i == N) ? 0.5 : 1.0;
    o.ccw[i] = 0.5 * o.L * 2.0 * ci / N * (1.0 - sum);
  }
  o.Dx.assign(nx * nx, 0.0);
  for (int i = 0; i < nx; ++i) {
    const double ci = (i == 0 || i == N) ? 2.0 : 1.0;
    double rs = 0.0;
    for (int j = 0; j < nx; ++j) {
      if (i == j) continue;
      const double cj = (j == 0 || j == N) ? 2.0 : 1.0;
      const double ti = kPi * i / N, tj = kPi * j / N;
      const double ds = -2.0 * std::sin(0.5 * (ti + tj)) * std::sin(0.5 * (ti - tj));
      const double sgn = ((i + j) % 2 == 0) ? 1.0 : -1.0;
      const double d = (ci / cj) * sgn / ds;
      o.Dx[i * nx + j] = -(2.0 / o.L) * d;
      rs += o.Dx[i * nx + j];
    }
    o.Dx[i * nx + i] = -rs;
  }

  // ordinates and Y_l0 projections: T_O[a][l] = Y_l(mu_a), T_S[l][a] = 2 pi w_a Y_l(mu_a)
  gauss_legendre(nt, o.mu, o.wmu);
  o.TO.assign(nt * nl, 0.0);
  o.TS.assign(nl * nt, 0.0);
  for (int a = 0; a < nt; ++a) {
    double p0 = 1.0, p1 = o.mu[a];
    for (int l = 0; l < nl; ++l) {
      double pl;
      if (l == 0) pl = 1.0;
      else if (l == 1) pl = o.mu[a];
      else {
        const double p2 = ((2.0 * l - 1.0) * o.mu[a] * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
        pl = p2;
      }
      const double Y = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi)) * pl;
      o.TO[a * nl + l] = Y;
      o.TS[l * nt + a] = 2.0 * kPi * o.wmu[a] * Y;
    }
  }

  // radial Galerkin matrices (polynomial integrands: 8 Gauss points per knot interval are exact).
  // f(vmax) = 0: the radial functions are the first nr of the nr + 1 clamped cubic B-splines; the
  // last one, the only one nonzero at vmax, is left out of trial and test spaces, so every matrix
  // and vector below accumulates only indices < nr.
  Spline sp(nr + 1, o.vmax);
  o.knots = sp.t;
  o.M.assign(nr * nr, 0.0);
  o.G = o.M;
  o.Dv = o.M;
  o.M1 = o.M;
  Rule r8(8);
  composite(sp.t, r8, [&](double v, double w) {
    int s;
    double Nv[4], dN[4];
    if (!sp.eval(v, s, Nv, dN)) return;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const int p = s - 3 + a, k = s - 3 + b;
        if (p >= nr || k >= nr) continue;
        o.M[p * nr + k] += w * v * v * Nv[a] * Nv[b];
        o.G[p * nr + k] += w * v * v * v * Nv[a] * Nv[b];
        o.Dv[p * nr + k] += w * v * v * Nv[a] * dN[b];
        o.M1[p * nr + k] += w * v * Nv[a] * Nv[b];
      }
  });

  // band of M (B-splines of degree 3 overlap only within 3 indices; entries outside stay 0)
  o.mw = 0;
  for (int p = 0; p < nr; ++p)
    for (int k = 0; k < nr; ++k)
      if (o.M[p * nr + k] != 0.0) o.mw = std::max(o.mw, std::abs(p - k));
  {
    const int bw = 2 * o.mw + 1;
    o.Mband.assign(static_cast<size_t>(nr) * bw, 0.0);
    for (int p = 0; p < nr; ++p)
      for (int k = std::max(0, p - o.mw); k <= std::min(nr - 1, p + o.mw); ++k)
        o.Mband[static_cast<size_t>(p) * bw + k - p + o.mw] = o.M[p * nr + k];
  }

  // generalized symmetric eigenproblem G u = lambda M u via M = R R^T:
  // R^-1 G R^-T = Z diag(lam) Z^T, U = R^-T Z, U^-1 = Z^T R^T.
  std::vector<double> R = o.M;
  if (!cholesky(R, nr)) return "mass matrix is not positive definite";
  std::vector<double> Ri = lower_inverse(R, nr);
  std::vector<double> S(nr * nr, 0.0), T(nr * nr, 0.0);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nr; ++j) {
      double s = 0;
      for (int k = 0; k < nr; ++k) s += Ri[i * nr + k] * o.G[k * nr + j];
      T[i * nr + j] = s;
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nr; ++j) {
      double s = 0;
      for (int k = 0; k < nr; ++k) s += T[i * nr + k] * Ri[j * nr + k];
      S[i * nr + j] = s;
    }
  for (int i = 0; i < nr; ++i)  // symmetrise rounding
    for (int j = i + 1; j < nr; ++j) S[i * nr + j] = S[j * nr + i] = 0.5 * (S[i * nr + j] + S[j * nr + i]);
  std::vector<double> Z;
  jacobi_eigen(S, nr, o.lam, Z);
  o.U.assign(nr * nr, 0.0);
  o.Uinv.assign(nr * nr, 0.0);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nr; ++j) {
      double u = 0, ui = 0;
      for (int k = 0; k < nr; ++k) {
        u += Ri[k * nr + i] * Z[k * nr + j];   // (R^-T Z)_{ij}
        ui += Z[k * nr + i] * R[j * nr + k];   // (Z^T R^T)_{ij}
      }
      o.U[i * nr + j] = u;
      o.Uinv[i * nr + j] = ui;
    }

  // Q_ij = (I + dt/2 lam_i mu_a D_x)^-1 with the inflow row replaced by the identity row; the
  // inflow column of Q is zeroed, which applies the zero right-hand side of that row.
  if (!assemble_q(o, 0.5 * o.dt, o.Q)) return "an x half-step operator is singular";
  return "";
}

bool assemble_q(const HostOps& o, double tau, std::vector<double>& Q) {
  const int nx = o.nx, nr = o.nr, nt = o.nt;
  Q.assign(static_cast<size_t>(nt) * nr * nx * nx, 0.0);
  bool ok = true;
#pragma omp parallel for schedule(dynamic) reduction(&& : ok)
  for (int ai = 0; ai < nt * nr; ++ai) {
    const int a = ai / nr, i = ai % nr;
    const int row = o.mu[a] >= 0.0 ? 0 : nx - 1;
    const double c = tau * o.lam[i] * o.mu[a];
    std::vector<double> B(nx * nx);
    for (int p = 0; p < nx; ++p)
      for (int q = 0; q < nx; ++q) B[p * nx + q] = (p == q ? 1.0 : 0.0) + c * o.Dx[p * nx + q];
    for (int q = 0; q < nx; ++q) B[row * nx + q] = (q == row) ? 1.0 : 0.0;
    double* Qa = Q.data() + static_cast<size_t>(ai) * nx * nx;
    ok = invert(B, nx, Qa) && ok;
    for (int p = 0; p < nx; ++p) Qa[p * nx + row] = 0.0;
  }
  return ok;
}

// ------------------------------------------------------------------------ velocity-side assembly

std::string assemble_v(HostOps& o, const std::vector<Process>& procs) {
  const int nr = o.nr, nt = o.nt, nl = o.nl, nv = o.nv;
  Spline sp(nr + 1, o.vmax);  // the last function is left out (f(vmax) = 0)
  const double vmax = o.vmax;
  Rule rq(24);

  std::vector<double> loss(nr * nr, 0.0), gain(nr * nr, 0.0), cT(nr * nr, 0.0);
  for (const Process& p : procs) {
    std::vector<double> br = clip(sp.t, 0.0, vmax);
    for (double b : sigma_breaks(p)) br.push_back(b);
    br = clip(br, 0.0, vmax);
    // loss, every l: -n0 int v^3 sigma phi_p phi_k
    composite(br, rq, [&](double v, double w) {
      const double sg = sigma(p, v);
      if (sg == 0.0) return;
      int s;
      double Nv[4], dN[4];
      if (!sp.eval(v, s, Nv, dN)) return;
      const double f = -o.n0 * w * v * v * v * sg;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          if (s - 3 + a < nr && s - 3 + b < nr) loss[(s - 3 + a) * nr + (s - 3 + b)] += f * Nv[a] * Nv[b];
    });
    // heavy-temperature correction from the elastic (momentum transfer) cross sections
    if (p.kind == BTE_ELASTIC && o.T0 > 0) {
      const double cf = -o.n0 * kKB * o.T0 / o.m0;
      composite(br, rq, [&](double v, double w) {
        const double sg = sigma(p, v);
        int s;
        double Nv[4], dN[4];
        if (!sp.eval(v, s, Nv, dN)) return;
        const double f = cf * w * v * v * v * sg;
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            if (s - 3 + a < nr && s - 3 + b < nr) cT[(s - 3 + a) * nr + (s - 3 + b)] += f * dN[a] * dN[b];
      });
    }
    // gain, (0,0) block: g n0 int v^3 sigma(v) phi_k(v) phi_p(u(v)) dv, integrated in u
    Collision col(p, o.m0);
    const double umax = col.u_of_v(vmax);
    if (umax > 0.0) {
      std::vector<double> bu;
      for (double b : sp.t)
        if (b <= umax) bu.push_back(b);
      for (double b : br)
        if (b <= vmax && col.maps(b)) bu.push_back(col.u_of_v(b));
      bu = clip(bu, 0.0, umax);
      composite(bu, rq, [&](double u, double w) {
        double dvdu;
        double v = col.v_of_u(u, dvdu);
        if (v > vmax) v = vmax;
        const double sg = sigma(p, v);
        if (sg == 0.0) return;
        int su, sv;
        double Nu[4], Nvv[4], d1[4], d2[4];
        if (!sp.eval(u, su, Nu, d1) || !sp.eval(v, sv, Nvv, d2)) return;
        const double f = col.g * o.n0 * w * dvdu * v * v * v * sg;
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            if (su - 3 + a < nr && sv - 3 + b < nr) gain[(su - 3 + a) * nr + (sv - 3 + b)] += f * Nu[a] * Nvv[b];
      });
    }
  }

  // M^-1 via Cholesky
  std::vector<double> R = o.M;
  if (!cholesky(R, nr)) return "mass matrix is not positive definite";
  std::vector<double> Ri = lower_inverse(R, nr), Minv(nr * nr, 0.0);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nr; ++j) {
      double s = 0;
      for (int k = std::max(i, j); k < nr; ++k) s += Ri[k * nr + i] * Ri[k * nr + j];
      Minv[i * nr + j] = s;
    }
  // the refinement residual's banded operators (bands of the loss part of C, of Dv and of M1, and
  // of the Cholesky factor of M); B-spline products of degree 3 couple only indices within mw
  {
    const int w = o.mw, bw = 2 * w + 1;
    o.rband.assign(static_cast<size_t>(nr) * bw, 0.0);
    o.rchol.assign(static_cast<size_t>(nr) * (w + 1), 0.0);
    o.rcinv.assign(nr, 0.0);
    // loss, Dv and M1 must lie within the band (the field blocks are combinations of Dv and M1)
    const std::vector<double>* src[3] = {&loss, &o.Dv, &o.M1};
    for (int m = 0; m < 3; ++m)
      for (int p = 0; p < nr; ++p)
        for (int k = 0; k < nr; ++k) {
          const double v = (*src[m])[p * nr + k];
          if (v == 0.0) continue;
          if (std::abs(p - k) > w) return "a radial operator is wider than the band of M_v";
          if (m == 0) o.rband[static_cast<size_t>(p) * bw + k - p + w] = v;
        }
    for (int p = 0; p < nr; ++p) {
      for (int j = 0; j <= w; ++j) {
        const int k = p - w + j;
        if (k >= 0) o.rchol[static_cast<size_t>(p) * (w + 1) + j] = R[p * nr + k];
      }
      o.rcinv[p] = 1.0 / R[p * nr + p];
    }
  }
  auto mscale = [&](const double* A, double* out) {
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nr; ++j) {
        double s = 0;
        for (int k = 0; k < nr; ++k) s += Minv[i * nr + k] * A[k * nr + j];
        out[i * nr + j] = s;
      }
  };

  // collision blocks C_l = loss (+ gain + C_T for l = 0), as assembled (Cg) and scaled (Cs)
  o.Cs.assign(static_cast<size_t>(nl) * nr * nr, 0.0);
  o.Cg.assign(static_cast<size_t>(nl) * nr * nr, 0.0);
  {
    std::vector<double> C0(nr * nr);
    for (int i = 0; i < nr * nr; ++i) C0[i] = loss[i] + gain[i] + cT[i];
    std::copy(C0.begin(), C0.end(), o.Cg.begin());
    mscale(C0.data(), o.Cs.data());
    for (int l = 1; l < nl; ++l) {
      std::copy(loss.begin(), loss.end(), o.Cg.begin() + static_cast<size_t>(l) * nr * nr);
      mscale(loss.data(), o.Cs.data() + static_cast<size_t>(l) * nr * nr);
    }
  }
  // field blocks: (q, q-1): (e/m_e) a_q (Dv - (q-1) M1); (q, q+1): (e/m_e) a_{q+1} (Dv + (q+2) M1),
  // a_l = l / sqrt(4 l^2 - 1)
  o.As_lo.assign(static_cast<size_t>(nl) * nr * nr, 0.0);
  o.As_up.assign(static_cast<size_t>(nl) * nr * nr, 0.0);
  o.Ag_lo.assign(static_cast<size_t>(nl) * nr * nr, 0.0);
  o.Ag_up.assign(static_cast<size_t>(nl) * nr * nr, 0.0);
  {
    const double em = kE / kMe;
    for (int q = 0; q < nl; ++q) {
      if (q >= 1) {
        const double aq = q / std::sqrt(4.0 * q * q - 1.0);
        const double cd = em * aq, cm = -em * aq * (q - 1);
        double* blk = o.Ag_lo.data() + static_cast<size_t>(q) * nr * nr;
        for (int i = 0; i < nr * nr; ++i) blk[i] = cd * o.Dv[i] + cm * o.M1[i];
        mscale(blk, o.As_lo.data() + static_cast<size_t>(q) * nr * nr);
      }
      if (q + 1 < nl) {
        const double aq = (q + 1) / std::sqrt(4.0 * (q + 1) * (q + 1) - 1.0);
        const double cd = em * aq, cm = em * aq * (q + 2);
        double* blk = o.Ag_up.data() + static_cast<size_t>(q) * nr * nr;
        for (int i = 0; i < nr * nr; ++i) blk[i] = cd * o.Dv[i] + cm * o.M1[i];
        mscale(blk, o.As_up.data() + static_cast<size_t>(q) * nr * nr);
      }
    }
  }
  // bands of the field blocks for the refinement residual (zero where a block does not exist)
  {
    const int w = o.mw, bw = 2 * w + 1;
    o.rfband.assign(static_cast<size_t>(2) * nl * nr * bw, 0.0);
    for (int side = 0; side < 2; ++side)
      for (int q = 0; q < nl; ++q) {
        const double* blk = (side == 0 ? o.Ag_lo : o.Ag_up).data() + static_cast<size_t>(q) * nr * nr;
        double* out = o.rfband.data() + (static_cast<size_t>(side) * nl + q) * nr * bw;
        for (int p = 0; p < nr; ++p)
          for (int k = std::max(0, p - w); k <= std::min(nr - 1, p + w); ++k) out[p * bw + k - p + w] = blk[p * nr + k];
      }
  }

  // K_C[(a,p),(b,k)] = sum_l T_O[a][l] Cs_l[p][k] T_S[l][b];  K_A likewise over (q, l = q -+ 1).
  // With want_kg the same sums over the blocks before the mass scaling give KCg, KAg.
  auto project = [&](const std::vector<double>& C, const std::vector<double>& Alo, const std::vector<double>& Aup,
                     std::vector<double>& KC, std::vector<double>& KA) {
    KC.assign(static_cast<size_t>(nv) * nv, 0.0);
    KA.assign(static_cast<size_t>(nv) * nv, 0.0);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) {
        for (int l = 0; l < nl; ++l) {
          const double cab = o.TO[a * nl + l] * o.TS[l * nt + b];
          const double* Cl = C.data() + static_cast<size_t>(l) * nr * nr;
          for (int p = 0; p < nr; ++p)
            for (int k = 0; k < nr; ++k) KC[static_cast<size_t>(a * nr + p) * nv + b * nr + k] += cab * Cl[p * nr + k];
        }
        for (int q = 0; q < nl; ++q) {
          if (q >= 1) {
            const double cab = o.TO[a * nl + q] * o.TS[(q - 1) * nt + b];
            const double* A = Alo.data() + static_cast<size_t>(q) * nr * nr;
            for (int p = 0; p < nr; ++p)
              for (int k = 0; k < nr; ++k) KA[static_cast<size_t>(a * nr + p) * nv + b * nr + k] += cab * A[p * nr + k];
          }
          if (q + 1 < nl) {
            const double cab = o.TO[a * nl + q] * o.TS[(q + 1) * nt + b];
            const double* A = Aup.data() + static_cast<size_t>(q) * nr * nr;
            for (int p = 0; p < nr; ++p)
              for (int k = 0; k < nr; ++k) KA[static_cast<size_t>(a * nr + p) * nv + b * nr + k] += cab * A[p * nr + k];
          }
        }
      }
  };
  project(o.Cs, o.As_lo, o.As_up, o.KC, o.KA);
  if (o.want_kg) {
    project(o.Cg, o.Ag_lo, o.Ag_up, o.KCg, o.KAg);
  } else {
    o.KCg.clear();
    o.KAg.clear();
  }

  // infinity norms of K_C and K_A (the refinement's backward-error test bounds |A_i| by them)
  o.kc_inf = 0.0;
  o.ka_inf = 0.0;
  for (int r = 0; r < nv; ++r) {
    double sc = 0.0, sa = 0.0;
    for (int c = 0; c < nv; ++c) {
      sc += std::fabs(o.KC[static_cast<size_t>(r) * nv + c]);
      sa += std::fabs(o.KA[static_cast<size_t>(r) * nv + c]);
    }
    o.kc_inf = std::max(o.kc_inf, sc);
    o.ka_inf = std::max(o.ka_inf, sa);
  }

  // moment vectors: 2 pi w_a int v^2 phi_k {1, m_e v^2/(2e), v sigma_j}
  o.n_proc = static_cast<int>(procs.size());
  std::vector<double> mn(nr, 0.0), me(nr, 0.0);
  {
    Rule r16(16);
    composite(sp.t, r16, [&](double v, double w) {
      int s;
      double Nv[4], dN[4];
      if (!sp.eval(v, s, Nv, dN)) return;
      for (int a = 0; a < 4; ++a) {
        if (s - 3 + a >= nr) continue;
        mn[s - 3 + a] += w * v * v * Nv[a];
        me[s - 3 + a] += w * v * v * energy_eV(v) * Nv[a];
      }
    });
  }
  o.mom_n.assign(nv, 0.0);
  o.mom_e.assign(nv, 0.0);
  o.mom_r.assign(static_cast<size_t>(o.n_proc) * nv, 0.0);
  for (int a = 0; a < nt; ++a)
    for (int k = 0; k < nr; ++k) {
      o.mom_n[a * nr + k] = 2.0 * kPi * o.wmu[a] * mn[k];
      o.mom_e[a * nr + k] = 2.0 * kPi * o.wmu[a] * me[k];
    }
  for (int j = 0; j < o.n_proc; ++j) {
    std::vector<double> br = clip(sp.t, 0.0, vmax);
    for (double b : sigma_breaks(procs[j])) br.push_back(b);
    br = clip(br, 0.0, vmax);
    std::vector<double> mr(nr, 0.0);
    composite(br, rq, [&](double v, double w) {
      int s;
      double Nv[4], dN[4];
      if (!sp.eval(v, s, Nv, dN)) return;
      const double f = w * v * v * v * sigma(procs[j], v);
      for (int a = 0; a < 4; ++a)
        if (s - 3 + a < nr) mr[s - 3 + a] += f * Nv[a];
    });
    for (int a = 0; a < nt; ++a)
      for (int k = 0; k < nr; ++k) o.mom_r[static_cast<size_t>(j) * nv + a * nr + k] = 2.0 * kPi * o.wmu[a] * mr[k];
  }
  o.have_v = true;
  return "";
}

std::string assemble_kc_only(const HostOps& o, const std::vector<Process>& procs, std::vector<double>& KC) {
  HostOps t;
  t.nx = o.nx, t.nr = o.nr, t.nt = o.nt, t.nl = o.nl, t.nv = o.nv;
  t.L = o.L, t.vmax = o.vmax, t.n0 = o.n0, t.T0 = o.T0, t.m0 = o.m0, t.dt = o.dt;
  t.mu = o.mu, t.wmu = o.wmu, t.knots = o.knots, t.M = o.M, t.G = o.G, t.Dv = o.Dv, t.M1 = o.M1;
  t.mw = o.mw, t.Mband = o.Mband;
  t.TO = o.TO, t.TS = o.TS;
  std::string e = assemble_v(t, procs);
  if (e.empty()) KC.swap(t.KC);
  return e;
}

std::string assemble_field(const HostOps& o, std::vector<double>& Lop, std::vector<double>& E1) {
  const int nx = o.nx;
  // Dirichlet Laplacian: D_x D_x with the wall rows replaced by V itself
  std::vector<double> A(static_cast<size_t>(nx) * nx, 0.0), Ainv(static_cast<size_t>(nx) * nx);
  for (int i = 1; i + 1 < nx; ++i)
    for (int j = 0; j < nx; ++j) {
      double s = 0.0;
      for (int k = 0; k < nx; ++k) s += o.Dx[i * nx + k] * o.Dx[k * nx + j];
      A[i * nx + j] = s;
    }
  A[0] = 1.0;
  A[static_cast<size_t>(nx) * nx - 1] = 1.0;
  if (!invert(A, nx, Ainv.data())) return "the Dirichlet Laplacian is singular";
  // V = Ainv b with b = -(e/eps0) rho inside and the wall voltages on rows 0, nx-1: Lop takes the
  // interior columns of Ainv scaled by -e/eps0, E1 its column 0; then E = -D_x V
  const double c = -kE / kEps0;
  Lop.assign(static_cast<size_t>(nx) * nx, 0.0);
  E1.assign(nx, 0.0);
  for (int i = 0; i < nx; ++i) {
    for (int j = 0; j < nx; ++j) {
      double s = 0.0;
      for (int k = 0; k < nx; ++k) s += o.Dx[i * nx + k] * Ainv[k * nx + j];
      if (j == 0) E1[i] = -s;
      else if (j + 1 < nx) Lop[i * nx + j] = -c * s;
    }
  }
  return "";
}

std::vector<double> maxwellian_coeffs(const HostOps& o, double Te_eV) {
  const int nr = o.nr;
  Spline sp(nr + 1, o.vmax);  // the last function is left out (f(vmax) = 0)
  const double vth = std::sqrt(2.0 * kE * Te_eV / kMe);
  std::vector<double> b(nr, 0.0);
  Rule r(24);
  composite(sp.t, r, [&](double v, double w) {
    int s;
    double Nv[4], dN[4];
    if (!sp.eval(v, s, Nv, dN)) return;
    const double f = std::exp(-(v / vth) * (v / vth)) / (std::pow(kPi, 1.5) * vth * vth * vth);
    for (int a = 0; a < 4; ++a)
      if (s - 3 + a < nr) b[s - 3 + a] += w * v * v * f * Nv[a];
  });
  std::vector<double> R = o.M;
  cholesky(R, nr);
  // forward R y = b, back R^T c = y
  for (int i = 0; i < nr; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= R[i * nr + k] * b[k];
    b[i] = s / R[i * nr + i];
  }
  for (int i = nr - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < nr; ++k) s -= R[k * nr + i] * b[k];
    b[i] = s / R[i * nr + i];
  }
  return b;
}

}  // namespace bte
