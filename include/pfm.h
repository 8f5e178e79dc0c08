/*
 * pfm.h - C ABI of the GB300 Newton-step solver for the finite-strain
 * multivariant phase-field model of martensitic transformation
 * (Tuma, Rezaee-Hajidehi, Hron, Farrell, Stupkiewicz, CMAME 2021).
 *
 * The library solves one backward-Euler Newton step of the discrete problem
 * R(U) = 0 (Sec. 3.4, Eq. FinalRes / Eq. linAlgEq): the residual and tangent
 * are the first and second derivatives of the penalty-regularised incremental
 * potential (Eq. PenPot) discretised with trilinear hexahedra on a structured
 * grid, the linear system is solved by flexible GMRES preconditioned by a
 * geometric-multigrid V-cycle with point-block (9x9) Jacobi smoothing,
 * re-discretised coarse operators and a dense direct coarse solve (Sec. 3.4).
 *
 * Number of variants. The model has phases 0..N (austenite and N martensite
 * variants, Sec. 2.1); N = PFM_NV is fixed when the library is compiled:
 * libpfm.so has N = 6 (the CuAlNi data of Sec. 5.1), libpfm_nv12.so N = 12
 * (a NiTi-type set with 15 unknowns per node, the footnote of Sec. 5.4).
 * A C caller compiles against this header with the same PFM_NV (default 6)
 * and can check the library's value with pfm_variants(). Below, "[9]" and
 * the figures 7 (phases), 15 (point unknowns) and 120 (Hessian entries) are
 * those of N = 6; in general they are 3 + N, N + 1, 9 + N and
 * (9 + N)(10 + N)/2.
 *
 * Conventions shared by every entry point:
 *  - Units: GPa, nm, s.
 *  - Nodal vectors are field-major "[9][n_nodes]" arrays: fields 0..2 are the
 *    displacement components u_x, u_y, u_z, fields 3..8 the condensed order
 *    parameters eta_1..eta_6 (eta_0 = 1 - sum eta_k, Sec. 3.1). Node (i,j,k)
 *    of an nx*ny*nz grid has index i + (nx+1)*(j + (ny+1)*k).
 *  - Every pointer documented as "device" is a CUDA device pointer owned by
 *    the caller; the library reads or writes it on the handle's stream and
 *    never frees it. "host" pointers are ordinary host memory.
 *  - Calls are enqueued on the handle's stream (pfm_set_stream; default the
 *    legacy default stream) and return once enqueued, except where a host
 *    output is documented (those synchronise the stream).
 *  - No C++ exception crosses the ABI. Errors are reported as pfm_status and
 *    a message retrievable with pfm_last_error(handle).
 *  - Dirichlet DOFs carry a zero residual, and the tangent has identity rows
 *    and columns there.
 *  - The library owns its workspaces (allocated with cudaMalloc in
 *    pfm_create / pfm_set_state / pfm_linearize) and frees them in
 *    pfm_destroy.
 */
#ifndef PFM_H
#define PFM_H

#include <stddef.h>
#include <stdint.h>

#ifndef PFM_NV
#define PFM_NV 6 /* martensite variants N of the library this header describes */
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfm_handle pfm_handle;

typedef enum {
  PFM_OK = 0,
  PFM_ERR_INVALID_ARG = 1,   /* bad size, null pointer, inconsistent call order */
  PFM_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the CUDA error) */
  PFM_ERR_OOM = 3,           /* device allocation failed */
  PFM_ERR_NONFINITE = 4,     /* NaN/Inf detected in a residual or Krylov norm */
  PFM_ERR_NOT_CONVERGED = 5, /* iteration cap reached before the tolerance */
  PFM_ERR_BREAKDOWN = 6,     /* Krylov breakdown or singular coarse/block matrix */
  PFM_ERR_TIMEOUT = 7,       /* a bounded device wait gave up */
  PFM_ERR_STATE = 8          /* required state missing (e.g. no pfm_set_state yet) */
} pfm_status;

typedef enum { PFM_F32 = 0, PFM_F64 = 1 } pfm_precision;

/* Structured grid of nx*ny*nz trilinear hexahedra on [0,Lx]x[0,Ly]x[0,Lz].
 * n_levels: multigrid levels (>= 1); level l has ceil(n/2^l) elements per
 * direction; 0 selects levels down to the first with max(n) <= 4. */
typedef struct {
  int nx, ny, nz;
  double Lx, Ly, Lz;
  int n_levels;
} pfm_mesh_desc;

/* Material and time-step data of the model (Sec. 2, Sec. 5.1).
 * Phase 0 is austenite, phases 1..N the martensite variants (N = PFM_NV). */
typedef struct {
  double Ut[PFM_NV + 1][9];      /* transformation stretch U_i^t, row-major; Ut[0] = I (Eq. LinMix) */
  double Lvoigt[PFM_NV + 1][36]; /* stiffness L_i, 6x6 row-major Voigt matrix acting on the strain
                                    vector (e11,e22,e33,2e23,2e13,2e12) (Eq. elasticEn) */
  double F0[PFM_NV + 1];         /* chemical energy F_i^0 (Sec. 2.2) */
  double mobility[PFM_NV + 1];   /* m_i (Eq. RateDiss) */
  double gamma[PFM_NV + 1][PFM_NV + 1]; /* interface energy gamma_ij, symmetric, diagonal ignored
                                           (Eq. IntEnergy) */
  double ell[PFM_NV + 1][PFM_NV + 1];   /* interface thickness parameter ell_ij, symmetric
                                           (Eq. IntEnergy) */
  double eps_eta;        /* penalty eps_eta (Eq. PenPot) */
  double tau;            /* time increment tau (Sec. 2.3) */
  double gamma_scale;    /* multiplier of every gamma_ij (1 for the paper's data) */
  int hencky;            /* elastic Hencky strain H^e (Sec. 2.4): 0 = exact 1/2 log C^e;
                            1, 2, 3 = the Pade (m,m) approximant of that order (Eqs. pade11,
                            pade22, pade33); other values are rejected (PFM_ERR_INVALID_ARG) */
} pfm_params;

/* Scalar material data of the CuAlNi example of Sec. 5.1, from which
 * pfm_params_from_cubic builds a parameter block (units GPa, nm, s). */
typedef struct {
  double stretch_alpha, stretch_beta, stretch_gamma; /* alpha, beta, gamma of the variant stretches */
  double C11, C12, C44;           /* one cubic stiffness for every phase (Voigt, crystal axes) */
  double F0_austenite, F0_martensite; /* chemical energies F_0 and F_i, i >= 1 */
  double mobility;                /* m_i, every phase */
  double gamma_am, gamma_mm;      /* interface energies gamma_0i and gamma_ij, i, j >= 1 */
  double ell;                     /* interface thickness parameter, every pair */
  double eps_eta;                 /* penalty eps_eta */
} pfm_cubic_material;

typedef struct {
  int max_newton;        /* Newton iteration cap (>= 1) */
  int restart;           /* FGMRES restart length m (1..64) */
  int max_lin_it;        /* cap on FGMRES iterations per linear solve */
  int nu_pre, nu_post;   /* smoothing sweeps before / after the coarse correction */
  double newton_rtol;    /* stop when ||R|| <= newton_rtol * ||R_0|| */
  double lin_rtol;       /* FGMRES: ||b - J x|| <= lin_rtol * ||b|| */
  double omega;          /* damping of the point-block Jacobi smoother (smoother 1) */
  pfm_precision precond; /* PFM_F32: V-cycle in FP32 inside FP64 FGMRES (mixed);
                            PFM_F64: every step in FP64 */
  int smoother;          /* 0: Chebyshev-accelerated point-block Jacobi on the interval
                            [cheb_lo, cheb_hi] * lambda_max(D^-1 J) (lambda_max estimated by
                            Lanczos steps at pfm_linearize); 1: damped point-block Jacobi */
  double cheb_lo, cheb_hi;  /* Chebyshev interval as fractions of lambda_max (0.05, 1.1) */
  int cycle_gamma;       /* coarse corrections per level: 1 = V-cycle, 2 = W-cycle (<= 0 read as 1) */
  double nu_growth;      /* smoothing steps on level l: round(nu * nu_growth^l) (<= 0 read as 1) */
  int deterministic;     /* 1: run the solve as pfm_set_deterministic(h, 1) does (bitwise
                            reproducible results); 0: the handle's setting */
  int krylov;            /* mixed precision (precond PFM_F32) only, how FGMRES applies J:
                            0 = the FP64-class outer operator in every iteration;
                            1 = relaxed products: the FP64-class operator while the residual
                                estimate is above switch_rtol ||b||, the FP32 operator after it
                                (an inexact Krylov method whose late products may be less
                                accurate), then the FP64-class true residual b - J x decides,
                                and a restart from it follows if lin_rtol is not met;
                            2 = iterative refinement: inner FGMRES cycles with the FP32
                                operator, each to switch_rtol times its right-hand side, each
                                followed by the FP64-class true residual.
                            Modes 1 and 2 stop on the true residual (Sec. 3.4, lin_rtol). */
  double switch_rtol;    /* krylov = 1: relative residual estimate below which products are
                            FP32 (e.g. 1e-3); krylov = 2: inner relative tolerance (e.g. 1e-4) */
} pfm_solve_opts;

typedef struct {
  int newton_its;        /* Newton corrections applied */
  int lin_its_total;     /* FGMRES iterations over all Newton corrections */
  int lin_its_last;      /* FGMRES iterations of the last correction */
  double res0;           /* ||R(U_0)||_2 */
  double res_final;      /* ||R(U)||_2 after the last correction */
  double lin_res_final;  /* relative residual of the last linear solve: the FGMRES estimate, or
                            with krylov = 1 or 2 the FP64-class true residual */
  int lin_outer_last;    /* krylov = 1: FGMRES cycles (restarts + 1), krylov = 2: refinement
                            steps, of the last linear solve (0 with krylov = 0) */
  double ms_residual, ms_linearize, ms_solve, ms_total; /* wall times (ms); the starting residual,
                            when formed by the linearisation pass (pfm_linearize_residual), counts
                            in ms_linearize */
  pfm_status status;
} pfm_solve_report;

/* Version string of the library. */
const char* pfm_version(void);

/* Number N of martensite variants the library was compiled for (PFM_NV):
 * nodal vectors have 3 + N fields and pfm_params has N + 1 phases. */
int pfm_variants(void);

/* Parameter blocks without writing them by hand (host functions, no GPU
 * needed, no allocation). */

/* *out = the model data of Sec. 5.1 from the scalars in *m: phase 0 the
 * austenite with U_0 = I, phases 1..6 the orthorhombic variants with
 * U_1 = [[p, 0, q], [0, beta, 0], [q, 0, p]], p = (alpha + gamma)/2,
 * q = (alpha - gamma)/2, U_2 the same with -q, U_3, U_4 the pattern with the
 * shear in the (1,2) plane and beta on axis 3, U_5, U_6 with beta on axis 1
 * and the shear in the (2,3) plane (the matrices printed in Sec. 5.1); the
 * cubic Voigt stiffness (C11, C12, C44) for every phase (Eq. elasticEn);
 * gamma_0i = gamma_am, gamma_ij = gamma_mm (i, j >= 1), one ell (Eq.
 * IntEnergy); F_0, F_i, one mobility, eps_eta, tau; gamma_scale = 1; hencky
 * as in pfm_params. Errors: PFM_ERR_INVALID_ARG (null pointer, hencky outside
 * 0..3, a library built for N != 6 variants). */
pfm_status pfm_params_from_cubic(const pfm_cubic_material* m, double tau, int hencky, pfm_params* out);

/* Anisotropic stiffness of Table 1 in the crystal frame of *p: the
 * austenite gets the cubic matrix (cubic[0..2] = c11, c12, c44), every
 * variant i >= 1 the orthorhombic matrix ortho[0..8] = (c11, c22, c33, c44,
 * c55, c66, c12, c13, c23) in its own axes 1, 2, 3, which are the
 * eigenvectors of its stretch U_i (in p->Ut) with the eigenvalues closest to
 * axis_stretch[0..2] (alpha, beta, gamma for CuAlNi), turned into the crystal
 * frame with the Bond matrix of those axes (engineering shear strains).
 * Errors: PFM_ERR_INVALID_ARG (null pointer, a stretch that is not
 * symmetric positive definite). */
pfm_status pfm_params_orthorhombic_stiffness(pfm_params* p, const double cubic[3], const double ortho[9],
                                             const double axis_stretch[3]);

/* Turn every stretch and stiffness of *p from the crystal frame into the lab
 * frame: U -> R U R^T and L -> M L M^T with M the Bond matrix of R (row i of R
 * = lab axis i in crystal coordinates; R orthogonal, row-major). Errors:
 * PFM_ERR_INVALID_ARG (null pointer, R not orthogonal to 1e-12). */
pfm_status pfm_params_rotate(pfm_params* p, const double R[9]);

/* Create a problem on a structured grid with the given parameters and build
 * the multigrid level hierarchy (Sec. 3.4: uniform refinement hierarchy).
 * Allocates the level workspaces. *out receives the handle.
 * Errors: PFM_ERR_INVALID_ARG for non-positive sizes or lengths, PFM_ERR_OOM. */
pfm_status pfm_create(const pfm_mesh_desc* mesh, const pfm_params* params, pfm_handle** out);

/* Release every device and host resource of the handle. NULL is ignored. */
void pfm_destroy(pfm_handle* h);

/* Message of the last error on this handle ("" if none); valid until the next
 * call on the handle. With h == NULL: the last error of pfm_create. */
const char* pfm_last_error(const pfm_handle* h);

/* Sizes of the finest level. Errors: PFM_ERR_INVALID_ARG (NULL handle). */
pfm_status pfm_get_sizes(const pfm_handle* h, int64_t* n_nodes, int64_t* n_elems, int* n_levels);

/* Multigrid level l (0 = finest): element counts and, after pfm_linearize,
 * the Lanczos estimate of lambda_max(D^-1 J) used by the Chebyshev smoother
 * (0 on the coarsest level, which is solved directly).
 * Errors: PFM_ERR_INVALID_ARG (NULL handle, level out of range). */
pfm_status pfm_get_level(const pfm_handle* h, int level, int* nx, int* ny, int* nz, double* lambda_max);

/* Steps of the smoother's eigenvalue estimate (default 10, 1..1000): the
 * Lanczos process for J D^-1 in the D^-1 inner product on every smoothed
 * level, whose largest Ritz value is the lambda_max of the Chebyshev
 * interval (the name is kept from an earlier power-iteration estimate).
 * Takes effect at the next pfm_linearize.
 * Errors: PFM_ERR_INVALID_ARG (out of range). */
pfm_status pfm_set_power_iterations(pfm_handle* h, int iterations);

/* Outer operator of the mixed-precision FGMRES: 1 (default) = the
 * double-float kernel of pfm_jacobian_apply_mixed (FP64-class accuracy on the
 * FP32 pipes; 12.8 ms at 128^3 on GB300), 0 = the FP64 kernel of
 * pfm_jacobian_apply (22 ms). Errors: PFM_ERR_INVALID_ARG (other values). */
pfm_status pfm_set_outer_operator(pfm_handle* h, int double_float);

/* Atomic-free, bitwise reproducible element kernels: with deterministic = 1
 * the residual, every tangent application (FP32, FP64, binary16 and the
 * double-float outer operator) and the dense coarse-operator assembly add
 * their element contributions without atomics (each element writes its
 * per-node contributions to a handle-owned scratch, then every node sums its
 * at most 8 contributions in a fixed order; the coarse assembly runs eight
 * element colours one after another), so that repeated calls on the same
 * data give bitwise equal results (Sec. 3.4, the tangent of Eq. linAlgEq).
 * Costs about one extra write and read of 9 values per element node. The
 * setting takes effect at once for residuals and applications; the coarse
 * operator keeps the form it was assembled in at the last pfm_linearize
 * (a Newton solve linearises, so its coarse operator follows the setting).
 * Penalty contact (pfm_set_contact) is not covered: calls that would apply
 * its terms in deterministic mode return PFM_ERR_INVALID_ARG.
 * Errors: PFM_ERR_INVALID_ARG (NULL handle, other values). */
pfm_status pfm_set_deterministic(pfm_handle* h, int deterministic);

/* Set the CUDA stream (a cudaStream_t passed as void*, owned by the caller and
 * alive while the handle uses it) for all later calls. Errors:
 * PFM_ERR_INVALID_ARG (NULL handle). */
pfm_status pfm_set_stream(pfm_handle* h, void* stream);

/* Replace the material parameters of Sec. 2 (same mesh). Invalidates the
 * tangent. Errors: PFM_ERR_INVALID_ARG (NULL pointers, tau <= 0, an unknown
 * Hencky mode). */
pfm_status pfm_set_params(pfm_handle* h, const pfm_params* params);

/* Dirichlet data (Sec. 5.1 boundary conditions): mask_dev (device, uint8
 * [9][n_nodes], 1 = prescribed DOF) and optional val_dev (device, double
 * [9][n_nodes]; NULL = keep the state's values). When given, prescribed
 * values are written into the state at pfm_set_state / pfm_newton_solve.
 * Only the displacement fields (0..2) may be prescribed.
 * Errors: PFM_ERR_INVALID_ARG if an order-parameter DOF is masked. */
pfm_status pfm_set_dirichlet(pfm_handle* h, const uint8_t* mask_dev, const double* val_dev);

/* Current iterate U and previous-step state U_n of the backward-Euler step
 * (Sec. 2.3, Eq. GlobIncPot) (device, double [9][n_nodes]); copied into the
 * handle. Invalidates the tangent. Errors: PFM_ERR_INVALID_ARG (NULL
 * pointers), PFM_ERR_CUDA. */
pfm_status pfm_set_state(pfm_handle* h, const double* U_dev, const double* Un_dev);

/* Copy the handle's current iterate to U_dev (device, double [9][n_nodes]).
 * Errors: PFM_ERR_INVALID_ARG (NULL pointer), PFM_ERR_STATE (no state),
 * PFM_ERR_CUDA. */
pfm_status pfm_get_state(pfm_handle* h, double* U_dev);

/* Arithmetic of the FP64-class linearisation (finest and coarsest levels, and
 * every level of an all-FP64 solve): 0 = FP64 (default), 1 = double-float
 * (pairs of FP32 numbers, about 48 significant bits, on the FP32 pipes; the
 * few divisions, square roots and logarithms per Gauss point in FP64).
 * Intermediate levels of the FP32 preconditioner are computed in FP32 either
 * way. Errors: PFM_ERR_INVALID_ARG (other values). */
pfm_status pfm_set_linearize_arithmetic(pfm_handle* h, int double_float);

/* Arithmetic of the residual's point physics (pfm_residual and the residuals
 * of pfm_newton_solve; Sec. 3.4, Eq. FinalRes): 0 = FP64 (default), 1 =
 * double-float (pairs of FP32 numbers, about 48 significant bits, on the FP32
 * pipes; divisions, square roots and logarithms in FP64). Element sums and
 * the output stay FP64. Errors: PFM_ERR_INVALID_ARG (other values). */
pfm_status pfm_set_residual_arithmetic(pfm_handle* h, int double_float);

/* Storage of the Gauss-point Hessians that the FP32 preconditioner's tangent
 * applications read (smoothing, residuals and eigenvalue estimates of every
 * level but the coarsest; Sec. 3.4): 0 = FP32 (default), 1 = binary16 copies
 * of the FP32 store scaled per level by a power of two s (largest |entry| of
 * s H in [2^14, 2^15)), read into FP32 arithmetic: half the bytes of the
 * HBM-bound application, with entries rounded to 11 significant bits. The
 * FGMRES outer operator, the block-diagonal smoother blocks and the coarse
 * solve keep their precision, so a converged solve meets the same residual
 * tolerance. Takes effect at the next linearisation (invalidates the tangent).
 * Errors: PFM_ERR_INVALID_ARG (other values). */
pfm_status pfm_set_preconditioner_store(pfm_handle* h, int half);

/* Frictionless penalty contact with a rigid sphere (Sec. 2.5, Eq. Ngap, the
 * contact term of Eq. PenPot) on the top face z = Lz: a point X of that face
 * at x = X + u has the normal gap g = |x - c| - R to the sphere of centre
 * center[3] (host array, nm) and radius R, and the potential gains
 * int 1/2 eps_N <g>_-^2 dS over the reference face (2x2 Gauss per face quad).
 * The term enters the residual, the energy, every tangent application
 * (FP32, FP64, double-float), the block diagonal and the dense coarse
 * operator of every level (re-discretised like the volume terms). radius <= 0
 * switches contact off. Batches that contain a problem with contact use the
 * lockstep driver. Errors: PFM_ERR_INVALID_ARG (missing centre, eps_N <= 0,
 * non-finite values). */
pfm_status pfm_set_contact(pfm_handle* h, const double* center, double radius, double eps_N);

/* Indenter load P = int eps_N <g>_- nbar_z dS (the vertical force the body
 * exerts on the sphere, positive when pressing; equal to the derivative of
 * the contact energy with respect to the indentation depth) and the contact
 * energy at the current iterate, written to *load_host and (if not NULL)
 * *energy_host; 0 without contact (Sec. 2.5). Synchronises.
 * Errors: PFM_ERR_INVALID_ARG (load_host NULL), PFM_ERR_STATE (no state),
 * PFM_ERR_CUDA. */
pfm_status pfm_contact_load(pfm_handle* h, double* load_host, double* energy_host);

/* Microstructure diagnostics of Sec. 5.3 of the nodal state U_dev (device,
 * double [9][n_nodes]; NULL = the handle's current iterate), with
 * eta_0 = 1 - sum_{k>=1} eta_k at every node:
 *   Iv_dev[n]       violation index sum_{i=0}^{6} |<eta_i>_-| (penalty study),
 *   Id_dev[n]       diffuseness index 1 - sum_{i=0}^{6} eta_i^4 (interface study),
 *   eta_star_dev[n] composite parameter eta_3 - eta_1,
 *   plane_stats_dev[4 k + {0,1,2,3}] = mean I_v, max I_v, mean I_d, max I_d
 *                   over the (nx+1)(ny+1) nodes of plane z = k h_z, k = 0..nz.
 * Every output is device memory owned by the caller and may be NULL (not
 * computed). Enqueued on the handle's stream; results are bitwise
 * reproducible for a given grid.
 * Errors: PFM_ERR_STATE (U_dev NULL and no state set), PFM_ERR_INVALID_ARG
 * (more than 65535 node planes), PFM_ERR_CUDA. */
pfm_status pfm_diagnostics(pfm_handle* h, const double* U_dev, double* Iv_dev, double* Id_dev,
                           double* eta_star_dev, double* plane_stats_dev);

/* Residual R = dPi/dU of the discrete incremental potential (Sec. 3.4,
 * Eq. FinalRes) at the current state, written to R_dev (device, double
 * [9][n_nodes]), zero at Dirichlet DOFs. If energy_host != NULL the total
 * potential sum_e sum_q w_q (F + D_tau + penalty) is written there
 * (synchronises). Errors: PFM_ERR_INVALID_ARG (R_dev NULL), PFM_ERR_STATE
 * (no state), PFM_ERR_CUDA. */
pfm_status pfm_residual(pfm_handle* h, double* R_dev, double* energy_host);

/* Linearise at the current state (the paper's tangent assembly, Sec. 3.4):
 * inject the state to every multigrid level, store the 15x15 Gauss-point
 * Hessians of the local energy (FP64 on the finest level; FP32 copies for an
 * FP32 preconditioner when precond == PFM_F32, FP64 otherwise), build the
 * 9x9 nodal block inverses of the point-block Jacobi smoother (dense LU with
 * partial pivoting) and the dense LU of the coarsest operator.
 * Errors: PFM_ERR_STATE (no state), PFM_ERR_OOM, PFM_ERR_BREAKDOWN (a singular
 * nodal block or coarse operator), PFM_ERR_NONFINITE (non-finite Hessian
 * entries met by the binary16 copy), PFM_ERR_CUDA. */
pfm_status pfm_linearize(pfm_handle* h, pfm_precision precond);

/* pfm_linearize and pfm_residual of the same state in one pass over the
 * elements (Sec. 3.4: the Newton iteration needs both at its starting state,
 * and both evaluate the same point physics): R_dev (device double
 * [9][n_nodes], zero at Dirichlet DOFs) and, if energy_host != NULL, the
 * potential (synchronises), as pfm_residual returns them, and the tangent as
 * pfm_linearize leaves it. Formed in one pass when the residual and the
 * finest-level linearisation both use FP64 arithmetic (the default; see
 * pfm_set_residual_arithmetic, pfm_set_linearize_arithmetic), else by the two
 * calls in turn.
 * pfm_newton_solve takes its first residual this way.
 * Errors: as pfm_linearize and pfm_residual (PFM_ERR_INVALID_ARG for a NULL
 * R_dev or an unknown precision). */
pfm_status pfm_linearize_residual(pfm_handle* h, pfm_precision precond, double* R_dev, double* energy_host);

/* y = J v with J = dR/dU at the last linearisation (Eq. linAlgEq), matrix
 * free from the stored Gauss-point Hessians; v_dev, y_dev are device arrays
 * [9][n_nodes] of float (PFM_F32) or double (PFM_F64). FP32 needs an FP32
 * tangent (pfm_linearize with PFM_F32) and applies the preconditioner's
 * finest-level operator: from the FP32 store, or from its binary16 copy
 * after pfm_set_preconditioner_store(h, 1). v and y must not alias.
 * Errors: PFM_ERR_INVALID_ARG (NULL vectors, unknown precision),
 * PFM_ERR_STATE (no state, no tangent, or no tangent in that precision),
 * PFM_ERR_CUDA. */
pfm_status pfm_jacobian_apply(pfm_handle* h, const void* v_dev, void* y_dev, pfm_precision prec);

/* y = J^T v (adjoint product). J is the Hessian of the discrete potential
 * (Sec. 3.4, Eq. PenPot), hence symmetric (Dirichlet rows and columns are
 * identity), so J^T v = J v: same layout, rules and errors as
 * pfm_jacobian_apply. */
pfm_status pfm_jacobian_transpose_apply(pfm_handle* h, const void* v_dev, void* y_dev,
                                        pfm_precision prec);

/* y = J v for an FP32 input v_dev (device float [9][n_nodes]) with an FP64
 * output y_dev (device double [9][n_nodes]), computed in double-float
 * arithmetic (pairs of FP32 numbers, about 48 significant bits) from the FP32
 * Hessian store and its FP32 rounding remainder. This is the outer operator
 * of the mixed-precision FGMRES, whose Krylov directions are FP32 V-cycle
 * outputs (Eq. linAlgEq). Errors: PFM_ERR_INVALID_ARG (NULL vectors),
 * PFM_ERR_STATE (no tangent from pfm_linearize(PFM_F32)), PFM_ERR_CUDA. */
pfm_status pfm_jacobian_apply_mixed(pfm_handle* h, const float* v_dev, double* y_dev);

/* pfm_jacobian_apply with HOST arrays v_host, y_host (float or double
 * [9][n_nodes] by prec; pinned memory lets the copies overlap): v travels to
 * the device in z-slabs while earlier slabs are applied, y returns plane by
 * plane (synchronises). Uses library-owned device buffers. Errors: as
 * pfm_jacobian_apply, PFM_ERR_OOM. */
pfm_status pfm_jacobian_apply_host(pfm_handle* h, const void* v_host, void* y_host,
                                   pfm_precision prec);

/* One multigrid V-cycle z = M r (Sec. 3.4): nu_pre point-block Jacobi
 * smoothing steps (Chebyshev-accelerated by default), restriction of the
 * residual, recursion, dense coarse solve, prolongation of the correction,
 * nu_post smoothing steps. r_dev, z_dev: device [9][n_nodes] in the precision
 * prec (the precision of the preconditioner built by pfm_linearize). Uses
 * opts->nu_pre, nu_post, smoother, cheb_lo, cheb_hi, omega (NULL = defaults
 * 4, 4, Chebyshev, 0.05, 1.1). Errors: PFM_ERR_INVALID_ARG (NULL vectors,
 * nu_pre < 1, nu_post < 0, an unknown smoother, 0 < cheb_lo < cheb_hi violated),
 * PFM_ERR_STATE (no tangent, or prec differs from the preconditioner's),
 * PFM_ERR_CUDA. */
pfm_status pfm_vcycle(pfm_handle* h, const void* r_dev, void* z_dev, pfm_precision prec,
                      const pfm_solve_opts* opts);

/* Solve J x = b by FGMRES(m) right-preconditioned with the V-cycle, starting
 * from x = 0 (Sec. 3.4, Eq. linAlgEq). b_dev, x_dev: device double [9][n_nodes].
 * report (nullable) receives lin_its_last and lin_res_final.
 * Errors: PFM_ERR_NOT_CONVERGED (x holds the last iterate), PFM_ERR_NONFINITE,
 * PFM_ERR_BREAKDOWN. */
pfm_status pfm_fgmres_solve(pfm_handle* h, const pfm_solve_opts* opts, const double* b_dev,
                            double* x_dev, pfm_solve_report* report);

/* Newton iterations on R(U) = 0 (Sec. 3.4, Eq. linAlgEq): U <- U + dU with
 * J dU = -R solved by pfm_fgmres_solve, until ||R|| <= newton_rtol ||R_0|| or
 * max_newton corrections. U_inout_dev (device double [9][n_nodes]) is the
 * initial iterate on entry and the result on exit; the handle's U_n stays.
 * The first correction always linearises at U_0 (unless R(U_0) = 0), so R(U_0)
 * comes from that linearisation pass (pfm_linearize_residual).
 * Synchronises; report (nullable) gets iteration counts, norms and times.
 * Errors: PFM_ERR_INVALID_ARG (NULL options or state vector), PFM_ERR_STATE
 * (no state), PFM_ERR_NOT_CONVERGED, PFM_ERR_NONFINITE, PFM_ERR_BREAKDOWN
 * (U_inout holds the last iterate), PFM_ERR_OOM, PFM_ERR_CUDA. */
pfm_status pfm_newton_solve(pfm_handle* h, const pfm_solve_opts* opts, double* U_inout_dev,
                            pfm_solve_report* report);

/* Derivatives with respect to the material parameters
 * theta = (C11, C12, C44, s_gamma) of a cubic stiffness shared by all phases
 * (Voigt entries C11 on the normal diagonal, C12 off it, C44 on the shear
 * diagonal) and the multiplier s_gamma of every interface energy gamma_ij.
 * The potential (Eq. PenPot) is affine in each of them (Eq. elasticEn is
 * linear in L, Eq. IntEnergy linear in gamma), so dPi/dtheta_k and
 * dR/dtheta_k are the potential and residual of the theta_k-part alone.
 * At the current state: dPi_dtheta_host[4] (host, nullable) receives
 * dPi/dtheta; if w_dev (device double [9][n_nodes]) is given,
 * wdR_dtheta_host[4] receives w . dR/dtheta (dR/dtheta zero at Dirichlet
 * DOFs); if dR_dtheta_dev (device double [4][9][n_nodes], nullable) is given
 * it receives the four vectors dR/dtheta_k. Requires the handle's stiffness
 * to be cubic and equal for all phases (PFM_ERR_INVALID_ARG otherwise).
 * Synchronises. */
pfm_status pfm_param_grad(pfm_handle* h, const double* w_dev, double* dPi_dtheta_host,
                          double* wdR_dtheta_host, double* dR_dtheta_dev);

/* Gauss-point physics for testing: for n points, F (device double [n][9],
 * row-major), eta_hat and eta_hat_n (device double [n][6]) give the local
 * energy density W (device double [n]), its gradient (device double
 * [n][15], z = (F row-major, eta_1..6)) and the packed upper triangle of its
 * Hessian (device double [n][120], row-major over r <= c; NULL to skip).
 * The density is the local part of Eq. PenPot (elastic energy with the
 * Hencky strain of Sec. 2.4, chemical, obstacle, dissipation and penalty
 * terms). Uses the parameters of h and synchronises. Errors:
 * PFM_ERR_INVALID_ARG (NULL inputs, n < 0), PFM_ERR_CUDA. */
pfm_status pfm_qp_eval(pfm_handle* h, int64_t n, const double* F_dev, const double* eta_dev,
                       const double* eta_n_dev, double* W_dev, double* grad_dev, double* hess_dev);

/* Copy the stored FP64 Gauss-point Hessians of elements [e0, e0+count) of
 * the finest level to hess_host (host double [count][8][120], Gauss point
 * q = q0 + 2 q1 + 4 q2). Synchronises. Errors: PFM_ERR_INVALID_ARG (range
 * outside the grid, NULL output), PFM_ERR_STATE (no tangent), PFM_ERR_CUDA. */
pfm_status pfm_get_hessians(pfm_handle* h, int64_t e0, int64_t count, double* hess_host);

/* Point-block Jacobi inverses of multigrid level l (0 = finest; not the
 * coarsest, which is solved directly) after pfm_linearize, for testing: the
 * inverse of each node's 9x9 diagonal block of the level's tangent (Dirichlet
 * rows and columns replaced by identity; Sec. 3.4), nodes [n0, n0 + count),
 * written to inv_host (host double [count][9][9], row-major; stored in the
 * preconditioner's precision). Synchronises. Errors: PFM_ERR_INVALID_ARG
 * (level or range out of bounds, NULL output), PFM_ERR_STATE (no tangent),
 * PFM_ERR_CUDA. */
pfm_status pfm_get_block_inverses(pfm_handle* h, int level, int64_t n0, int64_t count, double* inv_host);

/* Device timing of the hot phases with CUDA events recorded on the handle's
 * stream around each launch (off by default; enabling clears the counters).
 * Timed phases: PFM_PROF_JAPPLY_F32 / _F64 = one tangent application on the
 * finest level (the initialisation and element kernels), PFM_PROF_LINEARIZE
 * = pfm_linearize's finest-level Hessian kernel, PFM_PROF_RESIDUAL = the
 * residual kernel, PFM_PROF_VCYCLE = one whole V-cycle, PFM_PROF_JAPPLY_F16
 * = one finest-level application from the binary16 store. */
typedef enum {
  PFM_PROF_JAPPLY_F32 = 0,
  PFM_PROF_JAPPLY_F64 = 1,
  PFM_PROF_LINEARIZE = 2,
  PFM_PROF_RESIDUAL = 3,
  PFM_PROF_VCYCLE = 4,
  PFM_PROF_JAPPLY_F16 = 5,
  PFM_PROF_COUNT = 6
} pfm_prof_id;

/* Errors: PFM_ERR_INVALID_ARG (NULL handle). */
pfm_status pfm_profile_enable(pfm_handle* h, int enable);

/* Number of timed launches of phase id and their summed device time (ms)
 * since profiling was enabled. Synchronises the stream. Errors:
 * PFM_ERR_INVALID_ARG (NULL handle or outputs, id out of range). */
pfm_status pfm_profile_get(pfm_handle* h, int id, int64_t* launches, double* total_ms);

/* Kernel launches issued by the library in this process so far (all handles). */
int64_t pfm_launch_count(void);

/* Measurement aid (the paper has no counterpart): the fused multiply-add
 * throughput of the current device in TFLOP/s (2 flops per FMA) for
 * precision PFM_F32 or PFM_F64, from a kernel of 8 independent FMA chains per
 * thread on 8 x 256 threads per SM (best of three timed runs after one
 * warm-up). The rooflines of the FP32- and FP64-bound kernels are stated
 * against these figures. Allocates and frees a small device buffer;
 * synchronises the device. Errors: PFM_ERR_INVALID_ARG (NULL output or other
 * precision), PFM_ERR_OOM, PFM_ERR_CUDA. */
pfm_status pfm_arith_peak(int precision, double* tflops);

/* A batch of independent problems of possibly different grid sizes, each a
 * handle with its own Dirichlet data and state, solved together by
 * pfm_batch_newton_solve (batched engine or lockstep driver, below). The
 * handles must outlive the batch and must not be used by other calls while
 * pfm_batch_newton_solve runs.
 * Errors: PFM_ERR_INVALID_ARG (null handle, count < 1), PFM_ERR_CUDA. */
typedef struct pfm_batch pfm_batch;
pfm_status pfm_batch_create(pfm_handle* const* handles, int count, pfm_batch** out);
void pfm_batch_destroy(pfm_batch* b);
const char* pfm_batch_last_error(const pfm_batch* b);

/* pfm_newton_solve for every problem of the batch (Sec. 3.4, Eq. linAlgEq):
 * U_inout[p] (device double [9][n_nodes_p]) is problem p's initial iterate
 * on entry and its result on exit; reports (host array of count entries,
 * nullable) get each problem's iteration counts and norms (times are those of
 * the whole batch). Problems that meet newton_rtol stop early while the others
 * continue. Returns the first failing status, PFM_OK if every problem
 * converged. Synchronises.
 * With the mixed-precision options (precond PFM_F32, Chebyshev smoother,
 * V-cycle, double-float outer operator) and no contact or binary16
 * preconditioner store on any problem, the batched engine runs: every phase
 * (linearisation of all levels, eigenvalue estimates, coarse inverses,
 * V-cycle steps, FGMRES vector work) is one launch over all problems, and each
 * FGMRES iteration of the batch is one replayed CUDA graph. Other options, or
 * mode 1 of pfm_batch_set_mode, advance the problems in lockstep: every
 * problem on its own CUDA stream with per-problem launches, one
 * synchronisation per iteration for the whole batch, each problem's V-cycle
 * replayed from a CUDA graph captured once per linearisation. Both give the
 * same iterates up to rounding. Errors: as pfm_newton_solve, for the first
 * failing problem; PFM_ERR_INVALID_ARG (NULL batch, options or vectors). */
pfm_status pfm_batch_newton_solve(pfm_batch* b, const pfm_solve_opts* opts, double* const* U_inout,
                                  pfm_solve_report* reports);

/* Driver of pfm_batch_newton_solve: 0 = batched engine where the options
 * allow it (default), 1 = per-problem lockstep driver.
 * Errors: PFM_ERR_INVALID_ARG (null batch, other mode). */
pfm_status pfm_batch_set_mode(pfm_batch* b, int mode);

/* Residual and potential without a handle and without allocating device
 * memory, for callers that cannot call cudaMalloc: code inside a framework
 * that owns all device memory through its own allocator, code that must not
 * pay allocation latency or fragment a memory pool mid time step, or a device
 * that is already full. The paper has no counterpart: this is an interface
 * choice of this library. It computes what pfm_residual computes, for the
 * state U_dev / Un_dev (device double [9][n_nodes]) with Dirichlet mask
 * mask_dev (device uint8 [9][n_nodes]) on the grid of *mesh (n_levels
 * ignored) with *params: R_dev (device double [9][n_nodes], zero at Dirichlet
 * DOFs) and, if energy_host != NULL, the potential. Enqueued on stream (a
 * cudaStream_t as void*, NULL = default stream); synchronises that stream.
 * Working memory: one file-scope device array, sized for at most 4,194,304
 * nodes (about 8 MB), which every GPU that loads the library keeps until the
 * process exits; larger grids are rejected with PFM_ERR_INVALID_ARG. The first
 * call on a device looks up that array's device address (no allocation);
 * make that first call before capturing any stream into a CUDA graph. All
 * calls share the one array, so calls that overlap on the GPU (different
 * streams or host threads) race and must be serialised by the caller.
 * Errors: PFM_ERR_INVALID_ARG (null pointer, bad sizes, too many nodes, a
 * prescribed order-parameter DOF), PFM_ERR_CUDA. On any error the contents of
 * R_dev are undefined (the prescribed order-parameter check completes after
 * R_dev has been written). The message is returned by
 * pfm_noalloc_last_error() on the same host thread. */
pfm_status pfm_residual_noalloc(const pfm_mesh_desc* mesh, const pfm_params* params,
                                const uint8_t* mask_dev, const double* U_dev, const double* Un_dev,
                                double* R_dev, double* energy_host, void* stream);

/* Message of the last pfm_residual_noalloc error of the calling host thread
 * ("" if none). */
const char* pfm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PFM_H */
