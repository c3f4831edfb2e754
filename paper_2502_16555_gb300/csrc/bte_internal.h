// Internal declarations shared by the host assembly (assembly.cpp) and the CUDA side (*.cu).
#pragma once

#include <string>
#include <vector>

#include "../../include/bte.h"

namespace bte {

// Physical constants: CODATA 2018 values (e, kB exact since SI 2019).
constexpr double kE = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kKB = 1.380649e-23;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kTorr = 101325.0 / 760.0;
constexpr double kEps0 = 8.8541878128e-12;  // vacuum permittivity, CODATA 2018
constexpr int kMaxNr = 880;    // B-splines: the eigen-basis transforms stage nr x 33 doubles
constexpr int kMaxNv = 7936;   // nr * ntheta: the FP64 panel of a tall first panel
constexpr double kPi = 3.14159265358979323846;

struct Process {
  int kind = 0, form = 0;
  double th_eV = 0, scale = 1, sigma0 = 0;
  std::vector<double> tab_eps, tab_sigma;
};

// Everything assembled on the host, in FP64, row-major.
struct HostOps {
  int nx = 0, nr = 0, nt = 0, nl = 0, nv = 0;
  double L = 0, vmax = 0, n0 = 0, T0 = 0, m0 = 0, dt = 0;

  std::vector<double> x, Dx;            // nx, nx*nx
  std::vector<double> ccw;              // nx Clenshaw-Curtis weights on [0, L]
  std::vector<double> mu, wmu;          // nt Gauss-Legendre nodes (ascending) and weights
  std::vector<double> knots;            // nr + 4
  std::vector<double> M, G, Dv, M1;     // nr*nr radial Galerkin matrices
  int mw = 0;                           // half bandwidth of M (M[p][k] = 0 for |p - k| > mw)
  std::vector<double> Mband;            // nr x (2 mw + 1): Mband[p][k - p + mw] = M[p][k]
  std::vector<double> lam, U, Uinv;     // M^-1 G = U diag(lam) U^-1
  std::vector<double> Q;                // [nt][nr][nx][nx] inverse x half-step operators
  std::vector<double> TO, TS;           // T_O [nt][nl], T_S [nl][nt]

  bool have_v = false;
  int n_proc = 0;
  std::vector<double> Cs;               // [nl][nr][nr]  M^-1 C (l-block diagonal)
  std::vector<double> As_lo, As_up;     // [nl][nr][nr]  M^-1 A_v blocks (q, q-1) and (q, q+1)
  std::vector<double> Cg;               // [nl][nr][nr]  C before the mass scaling
  std::vector<double> Ag_lo, Ag_up;     // [nl][nr][nr]  A_v blocks before the mass scaling
  std::vector<double> KC, KA;           // [nv][nv]  P_O M^-1 C P_S, P_O M^-1 A_v P_S
  double kc_inf = 0.0, ka_inf = 0.0;    // their infinity norms (largest absolute row sums)
  // the refinement residual's operators: C_0 dense ([nr][nr], C before the mass scaling, l = 0);
  // bands ([nr][2 mw + 1]) of the loss part of C (the whole of C for l >= 1); bands of the field
  // blocks ([2][nl][nr][2 mw + 1]: (q, q - 1) = lo_d Dv + lo_m M1, then (q, q + 1) = up_d Dv +
  // up_m M1, zero where the block does not exist); the band of the Cholesky factor R of M
  // ([nr][mw + 1], R[p][p - mw + j]) and 1 / R[p][p].
  std::vector<double> rband, rfband, rchol, rcinv;
  bool want_kg = false;                 // also form KCg, KAg (handles that factor the Nv x Nv form)
  std::vector<double> KCg, KAg;         // [nv][nv]  P_O C P_S, P_O A_v P_S (no mass scaling)
  std::vector<double> mom_n, mom_e;     // [nv]
  std::vector<double> mom_r;            // [n_proc][nv]
};

// Grids, radial matrices, eigen-decomposition and Q_ij. Returns "" on success, else a message.
std::string assemble_x(const bte_config& cfg, HostOps& ops);
// Q_ij = (I + tau lam_i mu_a D_x)^-1 with the inflow rows of Algorithm 1 (tau = dt/2 for the half
// steps). False if one of them is singular.
bool assemble_q(const HostOps& ops, double tau, std::vector<double>& Q);
// Collision and field operators, their projections and the moment vectors.
std::string assemble_v(HostOps& ops, const std::vector<Process>& procs);
// K_C of a process list on the grids of o, o untouched (for the parameter derivatives).
std::string assemble_kc_only(const HostOps& o, const std::vector<Process>& procs, std::vector<double>& KC);
// Electrostatics of Section 2.3 (eq. "hybrid_cnt_c" with the electrode voltages of eq.
// "voltage_bc") on the collocation points: d^2V/dx^2 = -(e/eps0) rho inside, V(0) = V_left,
// V(L) = 0, E = -D_x V. Linear in (rho, V_left): E = Lop rho + V_left E1 (Lop nx*nx, E1 nx).
std::string assemble_field(const HostOps& ops, std::vector<double>& Lop, std::vector<double>& E1);
// Galerkin coefficients of a unit-density Maxwellian at temperature Te (eV).
std::vector<double> maxwellian_coeffs(const HostOps& ops, double Te_eV);

// Handle accessors for entry points defined outside bte_api.cu.
const HostOps* handle_ops(const bte_handle* h);
void* handle_stream_ptr(const bte_handle* h);
bte_status handle_fail(const bte_handle* h, bte_status s, const std::string& msg);
bte_status handle_device_status(bte_handle* h);  // BTE_OK, or why the handle cannot run device work
bool handle_profiling(const bte_handle* h);
unsigned long long handle_launches(const bte_handle* h);
void handle_add_launches(bte_handle* h, unsigned long long n);
// The step sequence of bte_step (F in place, status word NOT reset) enqueued on stream st (a
// cudaStream_t) instead of the handle's own stream: used to capture several handles' steps as
// branches of one CUDA graph.
bte_status handle_enqueue_step(bte_handle* h, double* F_dev, const double* E_dev, double t, double V0, double freq,
                               struct CUstream_st* st);
bte_status handle_reset_status(bte_handle* h, struct CUstream_st* st);
// The step of bte_step with the field recomputed after the first x half step from the ion density
// ni_dev and the electrons (eq. "bte_semi_implicit_efield"), on the handle's stream.
bte_status handle_enqueue_sc_step(bte_handle* h, double* F_dev, const double* ni_dev, double t, double V0,
                                  double freq);
// One x half step (Algorithm 1) of in into out, and the per-point velocity solve of in into out with
// the field E_dev (factor: form and factor first; else reuse the last factors, no refinement).
bte_status handle_enqueue_xhalf(bte_handle* h, const double* in, double* out);
bte_status handle_enqueue_vsolve(bte_handle* h, const double* in, double* out, const double* E_dev, bool factor);
// The field of eq. "hybrid_discrete_c" (bte_hybrid.cu): E = L (ni - u^T F) + V0 sin(2 pi f t) E_1
// into E_dev on the handle's stream (ni_dev NULL: no ions; V0 = 0: no electrode voltage).
bte_status enqueue_field(bte_handle* h, const double* F_dev, const double* ni_dev, double t, double V0,
                         double freq, double* E_dev);
// Reads the status word back on the handle's stream (synchronising it) and maps it to a status.
bte_status handle_read_status(bte_handle* h);
// Algorithm variants the batch autotuner chooses between: the tensor-core trailing update (only
// if the handle holds its workspace) or the CUDA-core one; on the tensor cores, panels applied in
// pairs (K = 256) or one at a time (K = 128), and the pair update on 256 x 256 tiles of CTA pairs
// (cg 2) or on 128 x 128 tiles of single CTAs (cg 1); the panel kernel's column-block width
// (0: by shape).
struct Variant {
  bool tc = false;
  int panel_w = 0;
  bool pair = true;
  int cg = 2;
};
bool handle_has_tc(const bte_handle* h);
void handle_set_variant(bte_handle* h, const Variant& v);
Variant handle_get_variant(const bte_handle* h);

}  // namespace bte
