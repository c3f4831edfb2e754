/*
 * bte.h -- C ABI of libbte: the semi-implicit time step of the 1D3V electron Boltzmann transport
 * equation of arXiv 2502.16555 ("Boltzsim"), on one GB300 (sm_103a).
 *
 * The discrete system (Section 3.4, eq. "bte_1d_discrete") is
 *     dF/dt + A_x F D_x^T = P_O C P_S F + P_O A_v P_S (E . F),
 * F holding, at every Chebyshev collocation point x_i, the B-spline coefficients f_k(x_i, theta_a)
 * at every discrete ordinate theta_a. One call of bte_step advances F by dt with the split scheme
 * of eqs. "bte_semi_implicit": an x half step (backward Euler, dt/2, Algorithm 1), a velocity step
 * (backward Euler, dt, one dense linear solve per collocation point, eq. "vspace_batched_system"),
 * and a second x half step.
 *
 * Conventions shared by every entry point:
 *  - F layout: double F[nx][ntheta][nr], C order (x slowest, B-spline index fastest), device memory
 *    owned by the caller. nv = nr*ntheta; the velocity index inside a point is a*nr + k.
 *  - Units: SI, energies in eV. The field E is in V/m; the electron force is -eE.
 *  - Errors are returned as bte_status, never thrown or trapped. bte_last_error() gives a message.
 *    A failed bte_step leaves F unchanged (BTE_ESINGULAR / BTE_ENOCONV / BTE_ENONFINITE) and the
 *    handle usable. Arguments are validated before anything is launched. Where a step meets
 *    several failures the first of these is reported: an expired device wait (BTE_ECUDA), a
 *    non-finite state or field handed in (BTE_ENONFINITE), a failed factorisation (BTE_ESINGULAR),
 *    a non-finite result (BTE_ENONFINITE), refinement short of its tolerance (BTE_ENOCONV).
 *  - Streams: all device work is enqueued on bte_config.stream (a cudaStream_t, NULL = legacy
 *    default stream). Entry points do not synchronise the device except where stated.
 *  - Threading: a handle is used by one host thread at a time.
 */
#ifndef BTE_H
#define BTE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bte_handle bte_handle;

typedef enum {
  BTE_OK = 0,
  BTE_EINVAL = 1,      /* bad argument (NULL, size, nl > ntheta, unknown enum ...) */
  BTE_ENOMEM = 2,      /* device or host allocation failed */
  BTE_ECUDA = 3,       /* a CUDA runtime call or launch failed, or a CUDA error was already pending when
                          the call began (message in bte_last_error; a pending error is cleared) */
  BTE_ESINGULAR = 4,   /* a zero or non-finite pivot in some per-point factorisation */
  BTE_ENOCONV = 5,     /* iterative refinement did not reach refine_tol within its sweeps */
  BTE_ENONFINITE = 6,  /* the input (state or field) or the result of a step holds NaN/Inf */
  BTE_ESTATE = 7       /* call out of order (e.g. bte_step before bte_set_cross_sections) */
} bte_status;

typedef enum {
  BTE_FP64 = 0,        /* every operation in FP64; direct LU solve of each point's system */
  BTE_MIXED = 1        /* FP32 factorisation (TF32x3 tensor-core trailing updates), FP64
                          refinement residuals, FP64 x step and moments */
} bte_precision;

/* flags for bte_config.flags */
#define BTE_FLAG_HOST_ONLY 1u   /* assemble the operators on the host only: no CUDA call is made;
                                   bte_get_operator works, device entry points return BTE_ESTATE */
#define BTE_FLAG_SIMT_GEMM 2u   /* BTE_MIXED: do the trailing updates of the factorisation on the CUDA
                                   cores (FP32) instead of the tcgen05 tensor cores (TF32x3) */
#define BTE_FLAG_STRUCTURED 4u  /* solve the velocity step through its block-tridiagonal structure in l
                                   (A^-1 f = f + P_O((I - dt B)^-1 - I) P_S f, B = C + E A_v, Section 3.3)
                                   instead of the dense per-point LU: the same solution with about
                                   Nv^3 / (5 N_l Nr^3) fewer flops and no dense factors in memory. The
                                   block elimination runs in FP64 (BTE_FP64) or FP32 with the FP64
                                   refinement (BTE_MIXED). Requires nr <= 64. */
#define BTE_FLAG_TC_SINGLE 8u   /* BTE_MIXED on the tensor cores: apply each 128-column panel to the
                                   trailing matrix on its own (K = 128) instead of two panels at a time
                                   (K = 256, half the trailing-matrix traffic); same factors up to
                                   rounding order */
#define BTE_FLAG_FULL_V 16u     /* with nl < ntheta, factor the full Nv x Nv matrix A_i per point. By
                                   default such a handle factors the reduced matrix I - dt B_i of order
                                   nl * nr (B = C + E A_v in the harmonic basis, Section 3.3; both
                                   multiplied by I (x) M_v, see bte_step) and solves
                                   through A^-1 f = f + P_O((I - dt B)^-1 - I) P_S f: the same solution,
                                   (nv / (nl nr))^3 fewer factorisation flops and (nv / (nl nr))^2 less
                                   factor memory. bte_step_adjoint needs the full factors. */
#define BTE_FLAG_TC_ONE_CTA 64u  /* BTE_MIXED on the tensor cores, panels in pairs: run the K = 256 update
                                   on 128 x 128 tiles of single CTAs instead of 256 x 256 tiles of CTA
                                   pairs (same products, twice the operand bytes staged per flop) */
#define BTE_FLAG_PANEL_TC 128u  /* BTE_MIXED on the tensor cores: run the left-looking updates inside each
                                   128-column panel factorisation as TF32x3 tcgen05 MMAs (L tiles by
                                   TMA, products accumulated in tensor memory) instead of CUDA-core
                                   FMAs; same pivots up to rounding */
#define BTE_FLAG_DIAG_TC_TIMEOUT 32u  /* diagnostic, for testing the timeout path: every tensor-core
                                   launch first waits (about 1 ms, before it issues any copy or MMA)
                                   on a barrier that nothing signals, so the bounded wait expires,
                                   the launch does no work and the step returns BTE_ECUDA with F
                                   unchanged. Never set it for real work. */

typedef struct {
  int nx;            /* Chebyshev-Gauss-Lobatto points, >= 3 */
  int nr;            /* cubic B-splines in speed, >= 4: the first nr of the nr + 1 clamped cubic
                        B-splines on a uniform grid over [0, vmax], so f(vmax) = 0 (the last one,
                        the only one nonzero at vmax, is left out: without it the field term has no
                        inflow through vmax and conserves int f^2 d^3v) */
  int ntheta;        /* Gauss-Legendre ordinates in mu = cos(theta), >= 2 */
  int nl;            /* spherical harmonics Y_l0 kept, 1 <= nl <= ntheta (0 means ntheta) */
  double L_m;        /* electrode gap [m] */
  double vmax_eV;    /* largest speed of the B-spline grid, as an energy [eV] */
  double p_Torr;     /* neutral pressure [Torr]; n0 = p / (kB T0) */
  double T0_K;       /* neutral temperature [K] */
  double m0_amu;     /* neutral mass [u] */
  double dt_s;       /* time step [s] */
  int precision;     /* bte_precision */
  double refine_tol; /* stop refining a point when max|r| <= refine_tol * max|b|, or when its normwise
                        backward error is at FP64 rounding level: max|r| <= min(256 eps, refine_tol)
                        (|A_i| max|x| + max|b|), |A_i| bounded by the infinity norms of dt K_C, dt K_A
                        (<= 0: default 1e-13 FP64, 1e-12 mixed) */
  int refine_max;    /* maximum refinement sweeps per step (< 0: default: 2 FP64, 4 mixed). The dense
                        paths factor (I (x) M_v) A_i, not A_i itself; their first FP64 solve is
                        accurate to about cond(M_v) eps, one FP64 sweep restores the backward error
                        of a direct FP64 solve. BTE_MIXED
                        with nr <= 64: points still short of the test after refine_max sweeps through
                        the FP32 factors (cond(A_i) eps_32 near 1 or above: strong fields) are solved
                        again by the FP64 block-tridiagonal solve and refined through it, two more
                        sweeps, before BTE_ENOCONV is reported */
  void* stream;      /* cudaStream_t for all device work */
  unsigned flags;    /* BTE_FLAG_* */
} bte_config;

typedef enum { BTE_ELASTIC = 0, BTE_EXCITATION = 1, BTE_IONIZATION = 2 } bte_kind;

typedef enum {
  BTE_SIGMA_CONST = 0,   /* sigma = sigma0 */
  BTE_SIGMA_LINEAR = 1,  /* sigma = sigma0 (1 - th/eps) above the threshold th, else 0 */
  BTE_SIGMA_LOG = 2,     /* sigma = sigma0 ln(eps/th)/(eps/th) above th, else 0 */
  BTE_SIGMA_TABLE = 3,   /* piecewise linear in eps through (eps_eV[i], sigma_m2[i]), 0 outside
                            the table and at or below th */
  BTE_SIGMA_NU = 4       /* sigma = sigma0 / v (sigma0 in m^3/s): constant collision frequency */
} bte_form;

typedef struct {
  int kind;              /* bte_kind; elastic: u = v sqrt(1 - 2 m_e/m0); excitation: one electron
                            at eps - th; ionization: two electrons at (eps - th)/2 each */
  int form;              /* bte_form */
  double threshold_eV;   /* th (ignored for elastic) */
  double scale;          /* multiplies sigma */
  double sigma0;         /* m^2 (m^3/s for BTE_SIGMA_NU) */
  int n_tab;             /* table length (BTE_SIGMA_TABLE), host arrays below, ascending eps */
  const double* eps_eV;
  const double* sigma_m2;
} bte_process;

typedef struct {
  int nx, nr, ntheta, nl, nv, n_proc;
  int precision;
  double n0_m3;           /* neutral density */
  double vmax_ms;         /* largest speed [m/s] */
  size_t device_bytes;    /* device memory held by the handle */
  int last_refine_sweeps; /* correction sweeps per point and step of the last bte_step / bte_run, averaged
                             over points and steps and rounded up (counted on the device) */
  double last_residual;   /* max over points of max|r|/max|b| after the last step */
  unsigned last_flags;    /* device status bits of the last step (1 zero pivot, 2 non-finite result,
                             4 not converged, 8 expired device wait, 16 non-finite input) */
  unsigned long long launches; /* kernels launched by this handle so far */
  int tensor_cores;       /* 1 if the trailing updates run on tcgen05 (TF32x3) */
  int solve_n;            /* order of the per-point factorisation: nv, or nl * nr for the reduced
                             system (nl < ntheta without BTE_FLAG_FULL_V); 0 with BTE_FLAG_STRUCTURED */
  double last_refine_evals; /* refinement residuals evaluated per point and step of the last bte_step /
                             bte_run, averaged over points and steps (not rounded); each evaluation
                             but a point's last is followed by one correction solve of that point */
} bte_info;

/* Kernel classes reported by bte_profile (index into its output arrays). */
enum {
  BTE_K_X_TO_EIGEN = 0, BTE_K_X_APPLY_Q = 1, BTE_K_X_FROM_EIGEN = 2, BTE_K_V_FORM = 3,
  BTE_K_LU_PANEL = 4, BTE_K_LU_SWAP_TRSM = 5, BTE_K_LU_GEMM = 6, BTE_K_LU_SOLVE = 7,
  BTE_K_RESIDUAL = 8, BTE_K_OTHER = 9, BTE_NPROF = 10
};

/* Create a handle: validates cfg, assembles the grids and the x-step operators on the host (the
 * velocity operators need bte_set_cross_sections), and allocates its device buffers with cudaMalloc.
 * Ownership: the handle owns every buffer it allocates; free with bte_destroy.
 * Limits (BTE_EINVAL beyond them, set by the kernels' shared-memory plans): nx in [3, 4096],
 * nr in [4, 880], ntheta >= 2, 1 <= nl <= ntheta, nr * ntheta <= 7936.
 * Section 3.4 (discretisation) and Algorithm 1 (precomputed Q_ij). */
bte_status bte_create(const bte_config* cfg, bte_handle** out);

/* (Re)assemble the collision operator C (eqs. "c_en_mat_1d", "c_T0_mat_1d"), the field operator
 * A_v (eq. "adv_v_ws"), their projections K_C = P_O C P_S and K_A = P_O A_v P_S (eq. "proj_ops"),
 * and the moment vectors, for n_proc processes (host arrays, copied). Blocks until the device
 * copies are done. */
bte_status bte_set_cross_sections(bte_handle* h, int n_proc, const bte_process* procs);

/* F = n_e(x) f_M(v; Te) at every ordinate: the v^2-weighted Galerkin projection of a unit
 * Maxwellian (Section 4.1, eq. "ic_liu"), scaled by ne_dev[nx] (device). F_dev[nx][ntheta][nr]. */
bte_status bte_init_maxwellian(bte_handle* h, double* F_dev, const double* ne_dev, double Te_eV);

/* One semi-implicit step t -> t + dt of F_dev (device, in/out), eqs. "bte_semi_implicit".
 * The field of the velocity step is E_dev[nx] (device, V/m) if non-NULL, else the uniform
 * E = (V0/L) sin(2 pi freq (t + dt/2)). The velocity step solves A_i x = b at every point
 * (eq. "vspace_batched_system"); the dense paths factor (I (x) M_v) A_i = I (x) M_v -
 * dt (P_O C P_S + E_i P_O A_v P_S), the same system before the mass scaling of Section 3.4 (LU with
 * partial pivoting on the scaled A_i meets element growth of order 1e15 on speed grids of a few
 * hundred B-splines), and refine against A_i itself in FP64 (Algorithm 2).
 * On BTE_ESINGULAR/ENOCONV/ENONFINITE F is left unchanged.
 * Enqueues on the handle's stream; the status check reads back 4 bytes and synchronises it. */
bte_status bte_step(bte_handle* h, double* F_dev, const double* E_dev, double t_s, double V0,
                    double freq_Hz);

/* Same as bte_step, but n_steps steps from t_s without any host synchronisation between them
 * (the status word is read once at the end). E is the uniform sinusoidal field.
 * Launching: bte_run, bte_step with E_dev == NULL and bte_step_host replay a CUDA graph of one step,
 * captured for the state pointer (again when it, the cross sections or the solver variant change;
 * bte_step_host steps the handle's own device copy). Each step's field is formed on the host as for
 * a step launched kernel by kernel and passed through the per-point field array, which gives the
 * same factors: the results are identical. Kernel by kernel instead while bte_profile records, when
 * the caller is capturing the handle's stream, and for bte_step with a field array. */
bte_status bte_run(bte_handle* h, double* F_dev, int n_steps, double t_s, double V0, double freq_Hz);

/* bte_step on HOST buffers: copies F_host (nx*nv doubles) to the device, steps, copies the result
 * back and synchronises. F_host may be pageable or pinned. */
bte_status bte_step_host(bte_handle* h, double* F_host, double t_s, double V0, double freq_Hz);

/* Moments at every collocation point (eq. "glow_hybrid", n_e = u^T F): ne_dev[nx] [m^-3],
 * mean_eV_dev[nx] [eV], rates_dev[n_proc][nx] [m^3/s] (rate coefficient int |v| sigma_j f / n_e).
 * Where n_e == 0 the ratios are 0. Any output pointer may be NULL. FP64 accumulation. */
bte_status bte_moments(bte_handle* h, const double* F_dev, double* ne_dev, double* mean_eV_dev,
                       double* rates_dev);

/* Copy one host-assembled operator into a host array of `count` doubles (for inspection/tests):
 * which = 0 x[nx], 1 D_x[nx][nx], 2 mu[ntheta], 3 K_C[nv][nv], 4 K_A[nv][nv], 5 lambda[nr],
 * 6 U[nr][nr], 7 U^-1[nr][nr], 8 Q[ntheta][nr][nx][nx] (inflow column zeroed), 9 M_v[nr][nr],
 * 10 density moment vector [nv], 11 energy moment vector [nv], 12 rate vectors [n_proc][nv],
 * 13 Clenshaw-Curtis weights of the collocation points on [0, L] [nx], 14 P_O C P_S[nv][nv] and
 * 15 P_O A_v P_S[nv][nv] (before the mass scaling: (I (x) M_v) K_C and (I (x) M_v) K_A, the operators
 * of the matrices the dense Nv x Nv path factors; formed only for handles on that path).
 * Returns BTE_EINVAL if count does not match, BTE_ESTATE if the operator is not assembled yet
 * (or, for 14 and 15, not formed for this handle). */
bte_status bte_get_operator(const bte_handle* h, int which, double* host_out, size_t count);

bte_status bte_get_info(const bte_handle* h, bte_info* info);

/* Per-kernel timing with CUDA events recorded on the handle's stream around every launch.
 * enable = 1: clear and start recording (cheap: two event records per launch). enable = 0: stop,
 * synchronise the stream, and write the summed device time [ms] and launch count of every kernel
 * class into ms_out[BTE_NPROF] and count_out[BTE_NPROF] (either may be NULL). */
bte_status bte_profile(bte_handle* h, int enable, double* ms_out, unsigned long long* count_out);

/* The same fill as bte_init_maxwellian, for callers that cannot allocate device memory (code whose
 * device memory all comes from another runtime's pool, or a host program that passes in buffers it
 * got elsewhere): it makes no device allocation and also accepts a handle created with
 * BTE_FLAG_HOST_ONLY, which holds no device memory. The paper has no counterpart; this is an
 * interface convenience. F_dev[nx][ntheta][nr] and ne_dev[nx] are device buffers of the caller.
 * Scratch: the nr Maxwellian coefficients are staged in a file-scope __device__ array of 4096 doubles
 * (32 KB) that every GPU loading libbte holds until the process exits; nr > 4096 gives BTE_EINVAL
 * (bte_create limits nr to 880 today, so no handle reaches it). The first call on a device looks up
 * that array's device address with the device current. The call copies the coefficients from a
 * host buffer that is freed when it returns, so it must not be recorded into a CUDA graph: while
 * the handle's stream is capturing it returns BTE_ESTATE and enqueues nothing. All calls share the
 * array and it keeps the last call's coefficients (nothing in it needs to start at zero: each call
 * writes the entries it reads); calls whose work overlaps on the GPU (other streams, or other
 * threads) race on it. Work is enqueued on the handle's stream without synchronising it. */
bte_status bte_init_maxwellian_static(const bte_handle* h, double* F_dev, const double* ne_dev, double Te_eV);

/* ---- Adjoint of the step ----------------------------------------------------------------------
 * With a specified field the step of eqs. "bte_semi_implicit" (Section 3.4) is linear in F:
 * F^{n+1} = S_n F^n, S_n = X V_n X (X: x half step, Algorithm 1; V_n: the per-point solves with
 * A_i = I - dt (K_C + E_i K_A), eq. "vspace_batched_system"). These entry points give the
 * transposed map and the parameter sensitivities needed for gradients of functionals of the
 * trajectory (a discrete adjoint; the paper has no counterpart). FP64 handles only (BTE_ESTATE
 * otherwise). */

/* lambda <- S_n^T lambda + g_weight * g for the step that starts from F^n = F_dev at time t_s with
 * the uniform field (V0/L) sin(2 pi freq (t + dt/2)). F_dev, lambda_dev, g_dev: device
 * [nx][ntheta][nr] FP64 (lambda in/out; g may be NULL). If SC_dev / SA_dev (device nv x nv FP64,
 * row-major, may be NULL) are given, the step's sensitivity products are added to them:
 *     SC += sum_i mu_i F*_i^T,    SA += (sin(2 pi freq (t + dt/2)) / L) sum_i mu_i F*_i^T,
 * mu_i = A_i^-T (X^T lambda)_i the adjoint after the velocity step and F*_i = A_i^-1 (X F^n)_i the
 * state after it (both at point i, nv entries). The transposed x step uses U^T, the transposed
 * Q_ij blocks and U^-T (copied to the device on the first call); A_i^T is solved with the same LU
 * factors (recomputed from F^n). Synchronises the handle's stream. */
bte_status bte_step_adjoint(bte_handle* h, const double* F_dev, double* lambda_dev, double t_s, double V0,
                            double freq_Hz, const double* g_dev, double g_weight, double* SC_dev,
                            double* SA_dev);

/* Gradient of a functional J from the accumulated sensitivities (SC, SA from bte_step_adjoint over
 * a trajectory, device): grad_out[2 n_proc + 1] =
 *   [ dJ/dscale_j  (j < n_proc) | dJ/dthreshold_j [per eV] (j < n_proc; 0 without a threshold) |
 *     dJ/dV0 [per V] ],
 * dJ/dtheta = dt <dK/dtheta, S> (Frobenius product). dK_C/dscale_j is process j's own K_C at unit
 * scale; dK_C/dthreshold_j is the central difference of the FP64 assembly with step h_eV; the V0
 * term uses K_A and SA. Synchronises the handle's stream. */
bte_status bte_adjoint_gradient(const bte_handle* h, const double* SC_dev, const double* SA_dev, double h_eV,
                                double* grad_out);

/* ---- Self-consistent field, ions, fully-implicit electrons (Section 2.3, Section 3.4) ----------
 * n_i is the ion number density [m^-3] at the nx collocation points (device, FP64); F the electron
 * state as for bte_step. None of these entry points changes bte_step; they allocate their device
 * operators (the nx x nx field and ion matrices) on first use and bte_step_implicit its work
 * vectors ((2 restart + 10) x nx x Nv doubles) on first use or when the restart grows. */

/* Ion transport coefficients as n0 times the mobility [1/(V m s)] and n0 times the diffusion
 * coefficient [1/(m s)] (the parameter table of Section 4; defaults 4.65e21 and 2.07e20). mu >= 0,
 * D > 0, else BTE_EINVAL. */
bte_status bte_set_ion_transport(bte_handle* h, double n0_mu_i, double n0_D_i);

/* E_dev[nx] = L (n_i - u^T F) + V0 sin(2 pi f t) E_1 (eqs. "hybrid_discrete_c", "voltage_bc"): the
 * field of Gauss's law d^2V/dx^2 = -(e/eps0)(n_i - n_e) on the collocation points with
 * V(0, t) = V0 sin(2 pi f t), V(L) = 0, E = -D_x V. ni_dev may be NULL (no ions). Enqueued on the
 * handle's stream (no synchronisation). */
bte_status bte_field(bte_handle* h, const double* F_dev, const double* ni_dev, double t_s, double V0,
                     double freq_Hz, double* E_dev);

/* The ion step of eq. "fluid_step": n_i <- n_i^{n+1} solving
 * (n^{n+1} - n^n)/dt + D_x J(n^{n+1}) = n0 k_i n_e (F^n), J = mu_i E^n n - D_i D_x n, with E^n the
 * field of (n_i^n, F^n) at t_s and the wall fluxes of eq. "fl_ion_bc" (outflow only) as the first
 * and last rows. ni_dev is updated in place only on success (BTE_ESINGULAR leaves it). Synchronises
 * the handle's stream. */
bte_status bte_ion_step(bte_handle* h, double* ni_dev, const double* F_dev, double t_s, double V0,
                        double freq_Hz);

/* One semi-implicit electron step with the self-consistent field (eqs. "bte_semi_implicit" with
 * "bte_semi_implicit_efield"): after the first x half step E^{1/2} = L (n_i - u^T F^{n+1/2}) plus
 * the electrode field at t_s + dt/2; then the per-point solves with that field, refinement and the
 * second x half step as in bte_step. ni_dev is required (zeros for no ions); E_out_dev (may be NULL)
 * receives E^{1/2}. Same error contract as bte_step. Synchronises the handle's stream. */
bte_status bte_step_sc(bte_handle* h, double* F_dev, const double* ni_dev, double t_s, double V0, double freq_Hz,
                       double* E_out_dev);

/* Options and report of bte_step_implicit (zero fields take the defaults). */
typedef struct {
  double newton_rtol;  /* stop when |R(F)| <= newton_rtol |F^n| (default 1e-10) */
  int newton_max;      /* Newton iterations (default 8) */
  int gmres_restart;   /* GMRES basis size, <= 200 (default 100) */
  double gmres_rtol;   /* inner tolerance relative to |R| (default 1e-2) */
  int gmres_max;       /* GMRES iterations per Newton iteration, restarts included (default 400) */
  int precond;         /* 0: the per-point solves at the iterate's field, then one full x step
                          (default); 1: the semi-implicit step's map (x half step, solves, x half step) */
  int newton_iters;    /* out: Newton iterations taken */
  int gmres_iters;     /* out: GMRES iterations, all Newton iterations together */
  double residual;     /* out: final |R| / |F^n| */
} bte_implicit_opts;

/* One fully-implicit electron step (eqs. "bte_fully_implicit"): F <- the root of
 * R(F) = F - F^n + dt [A_x F D_x^T - P_O C P_S F - P_O A_v P_S (E(F) . F)], E(F) the field of
 * (n_i, u^T F) at t_s + dt, with the zero-inflow rows R = F. Newton with backtracking from the
 * semi-implicit self-consistent step's result; each Newton system by restarted flexible GMRES
 * (the preconditioned basis is stored, so its FP32 solves need not act linearly) on the
 * Jacobian action of eq. "1dbte_jac_action", right-preconditioned by the split operator at the
 * iterate's field (opts->precond; the per-point factors formed once per Newton iteration; the
 * full-step x operators are assembled on the first call with precond 0). A line search that
 * finds no sufficient decrease retries its Newton iteration with a 100x smaller GMRES tolerance,
 * at most twice. ni_dev is required; opts may be NULL.
 * BTE_ENOCONV if Newton stops above newton_rtol; F is written only on success. Synchronises the
 * handle's stream. */
bte_status bte_step_implicit(bte_handle* h, double* F_dev, const double* ni_dev, double t_s, double V0,
                             double freq_Hz, bte_implicit_opts* opts);

/* ---- Batched stepping of independent discharges ------------------------------------------------
 * Many discharges with uneven grids (nx, nr, ntheta), pressures and cross sections, stepped
 * together: every instance is an ordinary handle (its own operators, buffers and precision, all on
 * the current device); the batch records one CUDA graph whose concurrent branches are the
 * instances' step sequences of eqs. "bte_semi_implicit" (Section 3.4), framed by a kernel that
 * writes every instance's uniform field E_i = (V0_i/L_i) sin(2 pi f_i (t_i + dt_i/2)) from a
 * device-side clock t_i and one that advances the clocks by dt_i. n steps are n launches of that
 * graph, with no host work between them. The paper steps one discharge; batching is an
 * interface for running many. */
typedef struct bte_batch bte_batch;

/* flags for bte_batch_create */
#define BTE_BATCH_AUTOTUNE 1u  /* per distinct instance shape (nx, nr, ntheta, nl, precision), time
                                  one short run of every algorithm variant (tensor-core or CUDA-core
                                  trailing update; on the tensor cores panels in pairs on CTA-pair or
                                  single-CTA tiles, or one panel at a time; panel column-block
                                  width) on a scratch Maxwellian state and keep the fastest for the
                                  instances of that shape */

/* Group `count` (1..4096) distinct handles, created with device buffers and with cross sections
 * set. Handles stay owned by the caller and must outlive the batch; the autotuner (if asked) sets
 * their algorithm variants. `stream` is the caller's cudaStream_t: every batched run starts after
 * the work already enqueued on it. The batch owns its own stream, one branch stream and event per
 * instance, the field arrays and the graph. */
bte_status bte_batch_create(int count, bte_handle* const* handles, void* stream, unsigned flags,
                            bte_batch** out);

/* n_steps steps of every instance i on F_dev[i] (device, [nx_i][ntheta_i][nr_i] FP64, in/out)
 * from time t0_s[i], with the uniform field of amplitude V0[i] [V] and frequency freq_Hz[i]
 * (host arrays of count). The graph is recorded on the first call and again whenever the state
 * pointers differ from the recorded ones. Synchronises the batch's stream at the end, writes every
 * instance's status into status_out[count] (may be NULL) and returns the first non-OK one. As with
 * bte_run, an instance whose step fails keeps the last state that stepped cleanly. */
bte_status bte_batch_run(bte_batch* b, double* const* F_dev, int n_steps, const double* t0_s,
                         const double* V0, const double* freq_Hz, bte_status* status_out);

/* Variant used by instance i: tensor_cores 1 = tensor-core trailing update; panel_w the panel
 * column-block width (0 = by shape); tc_pair 1 = panels applied in pairs (K = 256), 0 = one at a
 * time (K = 128); tc_cg 2 = the pair update on 256 x 256 tiles of CTA pairs, 1 = on 128 x 128 tiles
 * of single CTAs; and the kernels launched per batched step (all instances, after the first run).
 * Any output pointer may be NULL. */
bte_status bte_batch_get_info(const bte_batch* b, int i, int* tensor_cores, int* panel_w, int* tc_pair,
                              int* tc_cg, unsigned long long* launches_per_step);

/* Release the batch (synchronises its stream; the handles are not touched). NULL is accepted. */
bte_status bte_batch_destroy(bte_batch* b);

/* Message of the last failing batch call ("" if none); NULL: last bte_batch_create error. */
const char* bte_batch_last_error(const bte_batch* b);

/* Release every buffer of the handle (synchronises its stream first). NULL is accepted. */
bte_status bte_destroy(bte_handle* h);

/* Message of the last failing call on this handle ("" if none); NULL handle: last create error. */
const char* bte_last_error(const bte_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* BTE_H */
