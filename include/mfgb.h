/*
 * mfgb: matrix-free Q_k hexahedral finite element operators on one GB300 (sm_103a).
 *
 * C ABI of the library libmfgb.so.  The operators are the discrete forms of the
 * anisothermal two-phase flow model of arXiv 2501.18781:
 *   - Section 2.1, eq. (momentum_balance), (continuity): the linearised (Oseen)
 *     Navier-Stokes operator with Q2 velocity and Q1 pressure (Appendix B: k_u = 2,
 *     k_p = 1), density by eq. (rhoEff) and viscosity by eq. (muEff);
 *   - eq. (heat_transfer): one implicit heat step (mass + convection + diffusion);
 *   - Section 2.2: a variable-coefficient Helmholtz operator with a level-set
 *     coefficient, and the diffusive part of conservative reinitialisation;
 *   - eq. (laser_gauss): the Gaussian laser flux as a top-face load.
 * Appendix B fixes the discretisation: continuous Lagrange Q_k elements on
 * hexahedra, Gauss quadrature with (k+1)^3 points, adaptive refinement (hanging
 * nodes), CG for symmetric and GMRES for nonsymmetric systems, matrix-free
 * operator evaluation.
 *
 * Conventions shared by every call:
 *   - Vectors are caller-owned DEVICE pointers unless a parameter says "host".
 *     A vector of an operator is the concatenation of its fields' DoF blocks
 *     (Oseen: u_x, u_y, u_z on the Q2 map, then p on the Q1 map).  For nrhs > 1
 *     the right-hand sides are stored ld elements apart.
 *   - DoFs are the free nodes of the lattice of spacing h_finest / k, numbered in
 *     lexicographic (z, y, x) order of their integer lattice coordinates.
 *   - Handles are library-owned; each *_destroy frees its handle (NULL is allowed).
 *     A handle must outlive the handles created from it.
 *   - Every call returns MF_OK or a negative status and never aborts, throws
 *     across the ABI or traps the device; mf_last_error() describes the last
 *     failure of the calling thread.  Work is enqueued on the context's stream;
 *     calls documented as "synchronising" wait for it before returning.
 */
#ifndef MFGB_H
#define MFGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mf_status;
#define MF_OK 0
#define MF_EINVAL (-1)        /* bad argument, size or handle combination */
#define MF_ENOMEM (-2)        /* a device or host allocation failed */
#define MF_ECUDA (-3)         /* a CUDA runtime call failed */
#define MF_ENOTCONV (-4)      /* a solver stopped at maxit above its tolerance */
#define MF_ETIMEOUT (-5)      /* a device-side bounded wait ran out */
#define MF_EUNSUPPORTED (-6)  /* valid request that the library does not implement */

/* MF_DF64: fp64 vectors, cell arithmetic in double-float (pairs of fp32 with error-free
 * products and sums, 47-48-bit significand) on the fp32 pipes, which GB300 runs at 64x its fp64
 * rate; accurate to a few 1e-14 relative to |A||u| componentwise.  On uniform meshes (Helmholtz,
 * heat without convection or Gauss-point rho_cp, Oseen without the melt-pool terms) the inputs are
 * scaled by a power of two per warp of 32 cells (Oseen: velocity and pressure separately), so any
 * fp64 magnitude keeps 47 bits relative to the largest input of those cells and inputs more than
 * 2^126 below it count as zero; the other operators keep the fp32 exponent range (magnitudes
 * between about 1e-38 and 3e38). */
typedef enum { MF_F64 = 0, MF_F32 = 1, MF_F16 = 2, MF_BF16 = 3, MF_DF64 = 4 } mf_dtype;
/* mf_solver_params.inner_arith value beside the dtypes: fp32 inner applies on the tensor cores */
enum { MF_INNER_TENSOR_CORES = 16 };

typedef struct mf_ctx mf_ctx;
typedef struct mf_mesh mf_mesh;
typedef struct mf_dofmap mf_dofmap;
typedef struct mf_op mf_op;

/* Thread-local text of the last failure (owned by the library, valid until the next call). */
const char* mf_last_error(void);

/* Context on CUDA device `device`; `cuda_stream` is any cudaStream_t, including the special
 * handles cudaStreamLegacy and cudaStreamPerThread; NULL asks for a non-blocking stream that
 * the library creates and owns (its work is then unordered with the legacy default stream).
 * A borrowed stream must outlive the context.  CUDA graphs are captured on a private stream
 * and launched on this one.
 * One device per process: the first call with a device index that is valid (or made while no
 * device is visible) binds the process to that device, because the operator tables and error
 * flags are set up once per process; a later call naming another device returns
 * MF_EUNSUPPORTED without touching the GPU.  Calls on a context must be made with its device
 * current (cudaSetDevice / torch.cuda.set_device). */
mf_status mf_context_create(int device, void* cuda_stream, mf_ctx** out);
void mf_context_destroy(mf_ctx* ctx);
/* Replace the context's stream (borrowed). */
mf_status mf_context_set_stream(mf_ctx* ctx, void* cuda_stream);

/* Uniform mesh of n[0] x n[1] x n[2] cube cells filling the box [lo, hi] (host arrays).
 * The cells must be cubes: (hi-lo)[d] / n[d] equal for d = 0, 1, 2 (else MF_EINVAL).
 * ctx may be NULL: the mesh and the DoF maps built on it then live on the host only
 * (for inspection through mf_dofmap_export; no operator can be built on them). */
mf_status mf_mesh_uniform(mf_ctx* ctx, const int n[3], const double lo[3], const double hi[3],
                          mf_mesh** out);

/* Adaptively refined mesh (Appendix B: adaptive refinement near the interface) given
 * by its leaves: host int32 rows (level, i, j, k), 0 <= level <= levels, 0 <= i,j,k <
 * base * 2^level, on a base^3 root mesh of the cube [lo, hi].  The leaves must tile the
 * box exactly once and be 2:1 balanced across faces, edges and corners (else MF_EINVAL).
 * Leaves are ordered internally by the Morton code of their finest-level anchor
 * (bit b of x, y, z in bits 3b, 3b+1, 3b+2). */
mf_status mf_mesh_octree(mf_ctx* ctx, int base, int levels, const double lo[3], const double hi[3],
                         const int32_t* leaves, int64_t nleaves, mf_mesh** out);
void mf_mesh_destroy(mf_mesh* mesh);

/* Continuous Q_degree DoF map (degree 1 or 2) with hanging-node constraints: a node on
 * the closure of a leaf that is not a node of that leaf takes the value of the leaf's
 * Q_k interpolant there; chains are resolved to free DoFs, equal masters summed and
 * exact zeros dropped.  `dirichlet_faces` bits 0..5 = x-, x+, y-, y+, z-, z+ mark faces
 * whose DoFs get identity rows and columns in every operator built on this map. */
mf_status mf_dofmap_create(mf_mesh* mesh, int degree, uint32_t dirichlet_faces, mf_dofmap** out);
void mf_dofmap_destroy(mf_dofmap* map);
mf_status mf_dofmap_query(const mf_dofmap* map, int64_t* n_dofs, int64_t* n_cells,
                          int64_t* n_constraints, int64_t* n_constraint_entries);
/* Host copies (caller-allocated; any pointer may be NULL to skip that array):
 *   cell_map[n_cells*(k+1)^3]  per cell (in the map's cell order) and local node
 *                              (x fastest): the free DoF index, or -(1 + r) for the
 *                              hanging node of rank r (hanging nodes in lattice order);
 *   con_rowptr[n_constraints+1], con_cols[n_entries], con_w[n_entries]: CSR rows of the
 *                              hanging nodes, masters ascending;
 *   dof_coords[3*n_dofs]       physical coordinates, xyz per DoF;
 *   dirichlet[n_dofs]          1 for Dirichlet DoFs. */
mf_status mf_dofmap_export(const mf_dofmap* map, int32_t* cell_map, int64_t* con_rowptr,
                           int32_t* con_cols, double* con_w, double* dof_coords, uint8_t* dirichlet);

typedef enum {
  MF_OP_HELMHOLTZ = 0, /* int c u v + a(phi) grad u . grad v,  a = eq. (muEff) with a_l, a_g */
  MF_OP_HEAT = 1,      /* int rho_cp/dt u v + k grad u . grad v [+ rho_cp v beta . grad u];
                          k = k0 (1 + 0.5 T/T_b) at T_h^n, or per Gauss point (MF_FIELD_K_QPOINT) */
  MF_OP_OSEEN = 2,     /* [[sigma M_rho + C_rho(beta) + 2 mu eps:eps, B^T], [B, 0]], B = -div */
  MF_OP_REINIT = 3     /* int u v / dtau + eps (n . grad u)(n . grad v), n = grad phi_h/|grad phi_h| */
} mf_op_kind;

typedef enum {
  MF_HEAVISIDE_TANH = 0, /* H = clamp((1 + phi_h)/2, 0, 1): the Heaviside of phi = tanh(d / 2eps) */
  MF_HEAVISIDE_SINE = 1  /* eq. (heaviside) with d = 2 eps atanh(phi_h) */
} mf_heaviside;

typedef enum {
  MF_COEF_INKERNEL = 0,  /* coefficients re-evaluated from the nodal fields in every apply */
  MF_COEF_QPOINT = 1     /* coefficients tabulated per Gauss point when fields are set */
} mf_coef_mode;           /* reinit: fp32 applies always use the table (normals evaluated in fp64) */

typedef struct {
  int kind;        /* mf_op_kind */
  int heaviside;   /* mf_heaviside */
  int coef_mode;   /* mf_coef_mode (Oseen always tabulates) */
  int reserved;
  double eps;      /* interface thickness parameter (sine Heaviside, reinit) */
  double mass_coef, a_liquid, a_gas;            /* Helmholtz */
  double rhocp, dt, k0, t_boil;                 /* heat */
  double sigma, rho_l, rho_g, mu_l, mu_g;       /* Oseen */
  double dtau;                                  /* reinit */
  /* Oseen melt-pool extensions, switched on by oseen_flags (they need MF_FIELD_T_PREV, the nodal
   * absolute temperature on the velocity map, for the solid fraction f_s(T) of eq. solid_fraction):
   * MF_OSEEN_THREE_PHASE: rho and mu by eqs. (solid_liquid_gas_density), (solid_liquid_gas_property)
   *   with H_s = 3 f_s^2 - 2 f_s^3 (eq. heaviside_sl) and the solid rho_s, mu_s;
   * MF_OSEEN_DARCY: the damping force of eq. (darcy_damping_force) moved to the left-hand side,
   *   + int H_phi C f_s^2 / ((1 - f_s)^3 + b) u . v (dense phase only);
   * MF_OSEEN_TRACE_CORRECTION: viscous stress 2 mu (eps(u) - tr(eps(u)) n n) of Section 2.1,
   *   n = grad phi_h / |grad phi_h| (0 where |grad phi_h| < 1e-12/h); the operator is then
   *   nonsymmetric and its block-Jacobi blocks leave the correction out.
   * Any flag selects the Gauss-point-outer kernel; double-float applies reject the flags. */
  double rho_s, mu_s, t_solidus, t_liquidus;
  double darcy_c, darcy_b;
  int oseen_flags;
  int reserved2;
} mf_op_params;

enum { MF_OSEEN_THREE_PHASE = 1, MF_OSEEN_DARCY = 2, MF_OSEEN_TRACE_CORRECTION = 4 };

typedef enum {
  MF_FIELD_PHI = 0,      /* nodal level set on map 0 (n_dofs values) */
  MF_FIELD_T_PREV = 1,   /* nodal absolute temperature T^n on map 0 */
  MF_FIELD_BETA = 2,     /* nodal convection field, 3 blocks of n_dofs (x, y, z) */
  MF_FIELD_K_QPOINT = 3, /* conductivity per Gauss point, n_cells*27, cell-major, x fastest */
  /* heat operators only, for the two-phase energy equation (eq. heat_transfer with eq. muEff):
   * the volumetric heat capacity per Gauss point (n_cells*27, layout of K_QPOINT) replaces
   * rho_cp in both the value term (rho_cp,q / dt) and the convection term (rho_cp,q beta), and a
   * convection velocity per Gauss point (n_cells*27*3, cell-major, point, then x/y/z) replaces the
   * interpolated nodal MF_FIELD_BETA (the level-set transport velocity lives at Gauss points).
   * Either one makes the operator tabulated; 16-bit applies and the heat-step gradient reject it. */
  MF_FIELD_RHOCP_QPOINT = 4,
  MF_FIELD_BETA_QPOINT = 5
} mf_field;

/* Operator on `maps` (one map; Oseen: the Q2 velocity map then the Q1 pressure map on the
 * same uniform mesh).  Parameters are copied. */
mf_status mf_operator_create(mf_ctx* ctx, const mf_op_params* params, const mf_dofmap* const* maps,
                             int nmaps, mf_op** out);
void mf_operator_destroy(mf_op* op);
/* Vector length of the operator (sum of its fields' DoFs). */
mf_status mf_operator_size(const mf_op* op, int64_t* n);
/* Borrow a device field (fp64, `n` values as documented per field); the pointer must stay
 * valid while the operator is used.  With MF_COEF_QPOINT the Gauss-point table is rebuilt. */
mf_status mf_operator_set_field(mf_op* op, int field, const void* dev_ptr, int dtype, int64_t n);

/* dst = A src for nrhs vectors stored ld apart (dtype MF_F64 or MF_F32: the arithmetic
 * precision of the apply).  Dirichlet rows return src.  Asynchronous. */
mf_status mf_apply(mf_op* op, const void* src, void* dst, int nrhs, int64_t ld, int dtype);
/* dst = A src with fp32 vectors and packed 16-bit arithmetic (format MF_F16 or MF_BF16): two
 * right-hand sides share every instruction (lanes of an fp16x2 / bf16x2 register), so an odd nrhs
 * leaves one lane idle.  Helmholtz, heat without convection and reinit, coefficients from the
 * fp32 Gauss-point tables; values are scaled by a power of two near sqrt(n) and the coefficients
 * by one at or above their maximum before packing (fp16's range), and the result is unscaled in
 * fp32.  About 3 (fp16) or 2 (bf16) significant digits per operation: meant for smoothers inside a
 * higher-precision iteration.  The first call after a field change measures the coefficient
 * maximum (synchronising).  MF_EUNSUPPORTED for the Oseen operator or convection. */
mf_status mf_apply_packed16(mf_op* op, const float* src, float* dst, int nrhs, int64_t ld, int format);
/* dst = A^T src (Helmholtz, heat with convection, reinit).  Asynchronous. */
mf_status mf_apply_transpose(mf_op* op, const void* src, void* dst, int nrhs, int64_t ld, int dtype);

/* Q3 Helmholtz operators (degree-3 uniform maps) only: dst = A src for fp32 vectors on the fifth-
 * generation tensor cores.  The cell operator is applied in its dense form: U (128 cells x 64 nodal
 * values) times the 64 x 256 matrix of the shape functions and their reference derivatives at the
 * 64 Gauss points, the Gauss-point weights and a(phi) applied per row, then the transposed matrix
 * (tcgen05.mma kind::f16 with fp32 accumulation in tensor memory, operands split into bf16 hi + lo
 * parts and three products per contraction: fp32-class accuracy, about 29 times the flops of the
 * sum-factorised kernel).  nrhs vectors ld apart.  MF_EUNSUPPORTED for other operators.
 * A launch whose one-second wait limit runs out frees its tensor memory and returns (the device
 * stays usable) and sets a flag: the next mf_apply_tc call returns MF_ETIMEOUT (the call is
 * asynchronous, so it cannot see its own launch), and so does an mf_solve whose inner applies
 * timed out; each timeout is reported once and the flag is cleared.  Asynchronous. */
mf_status mf_apply_tc(mf_op* op, const float* src, float* dst, int nrhs, int64_t ld);
/* The coupling blocks of the Oseen operator on their own: the pressure-gradient term of the
 * momentum balance and the continuity constraint (Section 2, eq. momentum_balance with
 * div u = 0), in the weak form and quadrature of Appendix B, (B u, q) = -int q div u:
 *   which = MF_COUPLING_GRAD (0): dst = B^T src; src = a pressure vector (n_p values), dst =
 *           the three velocity blocks (3 n_u values), 0 in Dirichlet rows;
 *   which = MF_COUPLING_DIV (1): dst = B src; src = the three velocity blocks (Dirichlet values
 *           read as 0), dst = a pressure vector;
 *   which = MF_COUPLING_SCHUR (2): dst = B D^-1 B^T src, pressure to pressure, with D the 3 x 3
 *           nodal blocks of A_uu (the Schur complement approximation that MF_PREC_BLOCK_TRIANGULAR
 *           inverts; its fp32 form is the preconditioner's own: D and its inverses built in
 *           fp32 from the fp32 Gauss-point tables, S~ assembled as a 125-point stencil on the
 *           pressure grid from the 1D couplings of B and applied as such).  Needs the
 *           operator's fields; allocates work vectors and returns after the result is written.
 * These are the blocks of A [0; p] and A [u; 0] that mf_apply computes together with A_uu.
 * Device vectors of dtype MF_F64 or MF_F32; dst is overwritten.  MF_EINVAL for other
 * operator kinds or an unknown `which`.  Asynchronous for which 0 and 1. */
enum { MF_COUPLING_GRAD = 0, MF_COUPLING_DIV = 1, MF_COUPLING_SCHUR = 2 };
mf_status mf_oseen_coupling(mf_op* op, int which, const void* src, void* dst, int dtype);

/* dst = diag(A) (Dirichlet rows 1).  Asynchronous. */
mf_status mf_diagonal(mf_op* op, void* dst, int dtype);

typedef enum { MF_SOLVER_CG = 0, MF_SOLVER_GMRES = 1, MF_SOLVER_DEFECT_CORRECTION = 2 } mf_solver_kind;
/* MF_PREC_BLOCK_TRIANGULAR (Oseen, GMRES only): right preconditioner built on the saddle-point
 * block structure [[A_uu, B^T], [B, 0]] of Section 2 (eq. momentum_balance linearised, with the
 * continuity constraint).  Per call: the pressure part solves S~ x_p = r_p with S~ = B D^-1 B^T
 * (D = the 3x3 nodal blocks of A_uu, as in block Jacobi) by Jacobi-preconditioned CG to
 * schur_tol or schur_maxit steps, z_p = -x_p; the velocity part runs velocity_steps GMRES steps
 * on A_uu z_u = r_u - B^T z_p, right-preconditioned by D^-1.  All operator applications inside
 * it are fp32; vectors and inner products fp64.  Its inner Krylov solves make it change from
 * call to call, so the outer solver becomes flexible GMRES (Saad's FGMRES). */
typedef enum {
  MF_PREC_NONE = 0,
  MF_PREC_JACOBI = 1,
  MF_PREC_CHEBYSHEV = 2,
  MF_PREC_BLOCK_JACOBI = 3,
  MF_PREC_BLOCK_TRIANGULAR = 4
} mf_prec_kind;

typedef struct {
  int solver;          /* mf_solver_kind */
  int precond;         /* mf_prec_kind (defect correction: preconditioner of the inner solve) */
  int inner_dtype;     /* defect correction: precision of the inner solve (MF_F32): CG on the
                          symmetric operators, GMRES(restart, default 30) with MF_PREC_JACOBI or
                          MF_PREC_NONE on the convective heat operator and its transpose; the
                          outer residuals b - A x in the fp64 arithmetic fp64_arith selects */
  int restart;         /* GMRES restart length (<= 63) */
  int cheby_degree;    /* operator applications per Chebyshev preconditioner call */
  int maxit;           /* iteration cap (outer steps for defect correction) */
  int inner_maxit;     /* defect correction: inner iteration cap per step (<= 0: 100) */
  int use_graph;       /* replay recorded CUDA graphs: CG steps with the stopping test on the
                          device, eight per replay when n * nrhs <= 2^20 and one otherwise (a
                          system that has stopped is left untouched by the remaining steps; the
                          reported iterations are the steps it took), and each call of
                          MF_PREC_BLOCK_TRIANGULAR (recorded at its second call) */
  double tol;          /* stop when ||b - A x||_2 <= tol ||b||_2 (x0 = 0) */
  double inner_tol;    /* defect correction: inner relative tolerance */
  double cheby_ratio;  /* Chebyshev interval [lambda_max/ratio, 1.1 lambda_max] */
  int lanczos_steps;   /* steps of the lambda_max estimate of D^-1 A (kept on the operator and
                          reused by later solves with the same step count until a field is set) */
  int fp64_arith;      /* arithmetic of the fp64 operator applies: 0 fp64 pipes, 1 double-float,
                          2 whichever mf_autotune measured faster */
  int schur_maxit;     /* MF_PREC_BLOCK_TRIANGULAR: cap of the inner Schur CG (<= 0: 30) */
  int velocity_steps;  /* MF_PREC_BLOCK_TRIANGULAR: GMRES steps on the velocity block, 1..60 (<= 0: 10) */
  double schur_tol;    /* MF_PREC_BLOCK_TRIANGULAR: relative tolerance of the inner Schur CG (<= 0: 0.1) */
  int inner_arith;     /* defect correction: arithmetic of the inner fp32 operator applies (CG and
                          Chebyshev): MF_F32 (default, also 0), MF_F16 or MF_BF16 (packed pairs of
                          right-hand sides, see mf_apply_packed16), or MF_INNER_TENSOR_CORES (Q3
                          Helmholtz operators: the applies of mf_apply_tc) */
  int reserved3;
} mf_solver_params;

typedef struct {
  int iterations;          /* Krylov iterations (defect correction: inner iterations, summed) */
  int outer_iterations;    /* defect correction steps */
  double rel_residual;     /* final ||b - A x|| / ||b|| in fp64 */
  double lambda_max;       /* Chebyshev estimate used (0 if none) */
  double seconds;          /* wall time of the call */
  int inner_steps;         /* MF_PREC_BLOCK_TRIANGULAR: Schur CG steps taken before its stopping
                              test held, summed over the preconditioner calls (the steps after
                              it leave the iterate unchanged) */
  int reserved;
} mf_solve_info;

/* Inner products of the Krylov solvers (Appendix B: CG / GMRES): out[k] = sum_i x[k ld + i]
 * y[k ld + i] for k < nvec (1 <= nvec <= 64), device vectors of dtype MF_F64 or MF_F32, out a
 * device array of nvec doubles.  MF_F64: fp64 accumulation.  MF_F32: each thread carries its
 * products and sums as unevaluated pairs of floats (the compensated dot product of Ogita, Rump
 * and Oishi, as accurate as evaluation in twice the fp32 precision; fp64 conversions would
 * bound the kernel by the fp64 rate instead of HBM), partials are combined in fp64.  Partial sums go to the context's
 * reduction workspace (allocated once with the context) over a fixed grid and are summed in a
 * fixed order, so the result is bit-reproducible.  Asynchronous. */
mf_status mf_dot(mf_ctx* ctx, const void* x, const void* y, int64_t n, int64_t ld, int nvec, int dtype,
                 double* out);

/* The paper has no counterpart to this entry point.  The same inner products as mf_dot, for
 * callers that cannot let the library allocate device memory (an application that owns all
 * device memory through its own pool, a latency-critical loop where an allocation could
 * synchronise the device, code without an mf_ctx): it needs no context and allocates nothing.
 * Its block partial sums live in a static device array of 2 * 608 * 16 doubles (152 KB) that
 * every GPU loading the library holds until exit; hence 1 <= nvec <= 16 (larger nvec:
 * MF_EINVAL).  The first call on a device looks up that array's device address (with the
 * device current) and should come before any stream capture; the address is kept for the life
 * of the process and does not survive cudaDeviceReset (make no call on a device after resetting
 * it).  All calls share the array, so calls that overlap on the GPU race; nothing in it needs
 * clearing between calls.
 * x, y: device vectors (MF_F64 or MF_F32) ld apart; out: device array of nvec doubles;
 * cuda_stream: the cudaStream_t to launch on (NULL = the legacy default stream).
 * Asynchronous; results equal mf_dot's bit for bit (same fixed grid, same summation order). */
mf_status mf_dot_noalloc(const void* x, const void* y, int64_t n, int64_t ld, int nvec, int dtype, double* out,
                         void* cuda_stream);

/* Solve A x = b for each of nrhs right-hand sides (stored n apart), x0 = 0, in fp64 (b, x
 * fp64 device vectors).  Synchronising.  Returns MF_ENOTCONV with info filled when the
 * tolerance is not reached within maxit. */
mf_status mf_solve(mf_op* op, const mf_solver_params* params, const double* b, double* x, int nrhs,
                   mf_solve_info* info);

typedef struct {
  double power, radius, x0, y0, absorptivity;
} mf_laser;

/* Evaporation model of the interface source terms (Section 2.4; Section 5.2 for the mass flux
 * and the recoil pressure). */
typedef enum { MF_MASS_FLUX_KNIGHT = 0, MF_MASS_FLUX_TANASAWA = 1 } mf_mass_flux;
typedef struct {
  int mass_flux;          /* MF_MASS_FLUX_KNIGHT: mdot = 0.82 c_s p_sat(T) sqrt(M / (2 pi R T)) (eq. mDotPSat),
                             p_sat = p_amb exp(h_v M / (R T_v) (1 - T_v / T)) (Clausius-Clapeyron);
                             MF_MASS_FLUX_TANASAWA: mdot = tanasawa_coef (T - T_v) (eq. mDotTanasawa) */
  double p_ambient;       /* p_amb [Pa] */
  double latent_heat;     /* h_v [J/kg] */
  double molar_mass;      /* M [kg/mol] */
  double t_boil;          /* T_v [K] */
  double sticking;        /* c_s */
  double tanasawa_coef;   /* h_e [kg/(m^2 s K)] */
  double gas_constant;    /* R [J/(mol K)]; <= 0: 8.314 */
  double rhocp_liquid;    /* (rho c_p)_l, (rho c_p)_g of the arithmetic (rho c_p)(phi) */
  double rhocp_gas;
} mf_evaporation;

/* Interface source terms of Section 2.4 as load vectors on an Oseen operator's two maps, from the
 * operator's level set (MF_FIELD_PHI, its Heaviside and eps, rho_l, rho_g) and a nodal
 * temperature T (fp64 device, n_u values on the velocity map), all terms at the 27 Gauss points
 * of every cell, with delta = ||grad H(phi_h)|| (eq. delta), delta_rho = delta rho(phi) c_rho,
 * delta_rhocp = delta (rho c_p)(phi)^2 c_rhocp (the squared weight is the one c_rhocp of eq.
 * deltaRhoCp normalises to unit integral), n_Gamma = grad phi_h / ||grad phi_h||:
 *   f_p[n_p]   = int mdot (1/rho_l - 1/rho_g) delta psi_i          (eq. evaporDil, continuity)
 *   f_T[n_u]   = int -mdot h_v delta_rhocp N_i                     (eq. vapor_heat_loss, energy)
 *   f_u[3 n_u] = int (p_An(T) delta_rho - mdot^2 (1/rho_g - 1/rho_l) delta) n_Gamma N_i
 *                with p_An = 0.54 p_amb exp(-h_v M / R (1/T - 1/T_v))  (eqs. anisimov,
 *                recoilPressureEvaporDil, hybrid_recoil_pressure; momentum); Dirichlet rows 0.
 * Outputs are fp64 device vectors, overwritten; any may be NULL (skipped).  f_p and f_T have no
 * Dirichlet rows (natural loads).  Uniform maps only; MF_EINVAL for other operator kinds or a
 * missing level set.  Asynchronous. */
mf_status mf_interface_sources(mf_op* op, const mf_evaporation* evaporation, const double* T, double* f_u,
                               double* f_p, double* f_T);

/* Top-face load f_i = int_{z = hi_z} q(x, y) N_i dA of eq. (laser_gauss) (beam along -z,
 * so <-n . e_L> = 1), (k+1)^2 Gauss points per face, into fp64 device dst[n_dofs]
 * (overwritten; Dirichlet rows 0).  If d_params is not NULL it receives the four load
 * vectors of dq/dP, dq/dr, dq/dx0, dq/dy0 (4 blocks of n_dofs).  Asynchronous. */
mf_status mf_laser_load(mf_op* op, const mf_laser* laser, double* dst, double* d_params);

/* One implicit heat step and its adjoint gradient (HEAT operators).  With theta = T - T_ref:
 *   A theta = rho_cp/dt M theta_prev + f_laser,  J = 1/2 int_box (theta_h - theta*_h)^2
 * over the cells whose centre has |x|, |y| <= box_half and z >= hi_z - box_depth.
 * Outputs: *J (host), dJ_dlaser[4] (host: P, r, x0, y0), dJ_dkq (device, n_cells*27, may be
 * NULL; needs MF_FIELD_K_QPOINT), theta and lambda (device, n_dofs each, may be NULL).
 * Forward and adjoint systems are solved with `solver` (GMRES when convection is present).
 * Synchronising. */
mf_status mf_heat_step_gradient(mf_op* op, const mf_laser* laser, const mf_solver_params* solver,
                                const double* theta_prev, const double* theta_target,
                                double box_half, double box_depth, double* J, double* dJ_dlaser,
                                double* dJ_dkq, double* theta, double* lambda);

/* Time the apply variants of this operator (cells per block and persistent grids, timed on eight
 * right-hand sides for octree maps and on one for uniform ones; coefficient mode; one or nine threads
 * per cell for uniform Q2 Helmholtz and heat; fp64 pipes or double-float; Oseen: the fp64 loop order;
 * Q3 Helmholtz: the CUDA-core or the tensor-core kernel for fp32 applies, which then also serves the
 * fp32 applies inside solvers) and keep the fastest.  cache_path (may be NULL) is a
 * text file of one JSON record per line, keyed by the operator's configuration (kind, degree, mesh
 * type and sizes, optional fields, melt-pool flags, the device's SM count): if it holds a record with
 * this operator's key, the last such record's choice is applied and nothing is timed; otherwise the
 * variants are timed and the record (key, choice, timings) is appended.  Synchronising when it times. */
mf_status mf_autotune(mf_op* op, const char* cache_path);

/* Describe the variant the next apply will launch (host string, owned by the library). */
const char* mf_operator_variant(const mf_op* op);

/* Select an apply variant by name, in place of mf_autotune's choice (until the next mf_autotune):
 *   "q2_line"  1: fp64 and fp32 applies of Q2 Helmholtz and heat operators (uniform mesh, forward,
 *              no convection, no per-point heat capacity) by the line-per-thread kernel, nine threads
 *              per cell with the coefficients from the Gauss-point tables; 0: one thread per cell.
 *              Other applies (double-float, octree, convection, transpose) are unaffected.
 * MF_EINVAL for a NULL argument, an unknown name or a value other than 0 or 1.  Host only. */
mf_status mf_operator_set_variant(mf_op* op, const char* name, int value);

/* Number of kernel launches the library has issued on this context so far. */
int64_t mf_context_launch_count(const mf_ctx* ctx);

/* ---------------------------------------------------------------------------------------------
 * One time step of the overall solution algorithm (Algorithm algo:meltpooldg) on one uniform
 * mesh: velocity on a Q2 map (its Dirichlet faces are the walls, u = 0 there), pressure on a Q1
 * map, level set phi on a Q2 map without Dirichlet faces, temperature on a Q2 map whose Dirichlet
 * faces keep T^n.  With x* = 2 x^n - x^(n-1) (step 1):
 *  2. u_G = u*_h + mdot(T*_h) / rho(phi*_h) n_G(phi*_h) at the Gauss points (variant 1, eq.
 *     transport_vel_local_continuous); (M/dt + C(u_G)) phi_a = M phi^n / dt (eq. transport, backward
 *     Euler, defect correction: fp32 inner GMRES); reinit_steps pseudo-time steps (M/dtau + eps N_n) psi' = M psi / dtau + F(psi),
 *     F_i = int (1 - psi_h^2)/2 n . grad N_i, n the unit normal of phi_a (Olsson's conservative
 *     reinitialisation for phi in [-1, 1], CG), phi^(n+1) = the last psi;
 *  3. heat (eq. heat_transfer, defect correction: fp32 inner GMRES): (M_{rho_cp/dt} + K_k + C_{rho_cp}(u*)) T^(n+1) =
 *     M_{rho_cp/dt} T^n + s with rho_cp, k of phi^(n+1) (eq. muEff) and s = evaporative cooling
 *     (mdot of T*, eq. vapor_heat_loss) + laser (eq. laser_gauss with <n_G . e_L>, n_G pointing into
 *     the dense phase, e_L the beam direction); solved for T^(n+1) - T^n;
 *  4. flow (FGMRES(50) with the block-triangular preconditioner, fp32 inner solves): the melt-pool
 *     Oseen operator about u* with sigma = 1/dt, phi^(n+1), T^(n+1), velocity load sigma M_rho u^n
 *     + rho g + surface tension (eq. surface_tension, kappa = -div n_G from the Hessian of phi_h) +
 *     hybrid recoil force, pressure rows -int q sdot (eq. evaporDil).
 * The tanh Heaviside throughout (mf_op_params heaviside 0).  Every value in fp64; the residuals
 * that decide each solve's tolerance are evaluated fp64-accurately (double-float applies). */
typedef struct mf_meltpool_step mf_meltpool_step;

typedef struct {
  double dt;                                /* time step */
  double eps;                               /* interface thickness parameter */
  double rho_l, rho_g, mu_l, mu_g;          /* eqs. (rhoEff), (muEff) */
  double rhocp_l, rhocp_g, k_l, k_g;        /* eq. (muEff) for rho c_p and k */
  int oseen_flags;                          /* MF_OSEEN_* terms of the flow operator */
  int laser_on;                             /* 0: no laser flux */
  double rho_s, mu_s, t_solidus, t_liquidus, darcy_c, darcy_b;  /* as in mf_op_params */
  mf_evaporation evaporation;               /* mass flux and recoil (its rhocp_* are ignored) */
  double alpha0, alpha1, t_alpha, alpha_res;  /* eq. (surface_tension) */
  double gravity[3];
  double laser_power, laser_radius, laser_absorptivity;
  double laser_focus[3], laser_direction[3];  /* a point of the beam axis and its direction */
  int reinit_steps;                         /* >= 0 */
  int maxit;                                /* iteration limit of every solve (<= 0: 5000) */
  double dtau;                              /* pseudo-time step (reinit_steps > 0) */
  double tol;                               /* relative tolerance of the level-set and heat solves */
  double flow_tol;                          /* relative tolerance of the flow solve */
  int flow_velocity_steps;                  /* block-triangular preconditioner of the flow solve: GMRES */
  int flow_schur_maxit;                     /*   steps on the velocity block, Schur CG cap, Schur CG */
  double flow_schur_tol;                    /*   tolerance (<= 0: the defaults of mf_solver_params) */
  int reinit_mixed;                         /* 1: reinitialisation by fp32-inner defect correction
                                               (Chebyshev), 0: fp64 Jacobi-CG */
  int reserved;
} mf_meltpool_params;

typedef struct {
  int advection_iterations, reinit_iterations, heat_iterations, flow_iterations;
  double advection_residual, reinit_residual, heat_residual, flow_residual;  /* relative, last solve */
  double seconds[5];  /* level-set advection (incl. predictors), reinitialisation, heat, flow, total */
} mf_meltpool_info;

/* Optional device copies of intermediate quantities (any pointer may be NULL). */
typedef struct {
  double* u_star;        /* 3 n_u */
  double* T_star;        /* n_u */
  double* phi_star;      /* n_u */
  double* u_gamma;       /* n_cells * 27 * 3 */
  double* b_advection;   /* n_u: M phi^n / dt */
  double* phi_advected;  /* n_u */
  double* r_heat;        /* n_u: s + M_{rho_cp/dt} T^n - A T^n, Dirichlet rows 0 */
  double* b_flow;        /* 3 n_u + n_p */
  double* T_update;      /* n_u: the solved T^(n+1) - T^n */
} mf_meltpool_trace;

/* maps: velocity (Q2), pressure (Q1), level set (Q2, no Dirichlet faces), temperature (Q2), one
 * uniform mesh.  The step owns its operators and work vectors (about 40 n_u doubles plus
 * 7 n_cells * 27 for the Gauss-point tables).  MF_EINVAL on inconsistent maps or parameters. */
mf_status mf_meltpool_create(mf_ctx* ctx, const mf_meltpool_params* params, const mf_dofmap* u_map,
                             const mf_dofmap* p_map, const mf_dofmap* phi_map, const mf_dofmap* T_map,
                             mf_meltpool_step** out);
void mf_meltpool_destroy(mf_meltpool_step* step);
/* Advance one step.  Inputs (device, fp64): u^(n-1), u^n (3 n_u each), T^(n-1), T^n, phi^(n-1),
 * phi^n (n_u each); pass the same pointer twice for a first step (x* = x^n).  Outputs (device,
 * may not alias the inputs): up = [u^(n+1); p^(n+1)] (3 n_u + n_p), T^(n+1), phi^(n+1).
 * Synchronising; MF_ENOTCONV (outputs and info filled) if a solve stops at maxit. */
mf_status mf_meltpool_advance(mf_meltpool_step* step, const double* u_prev, const double* u, const double* T_prev,
                              const double* T, const double* phi_prev, const double* phi, double* up, double* T_out,
                              double* phi_out, mf_meltpool_trace* trace, mf_meltpool_info* info);

#ifdef __cplusplus
}
#endif
#endif /* MFGB_H */
