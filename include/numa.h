/*
 * numa.h -- C ABI of the GB300 HEVI 1D-IMEX library.
 *
 * The library advances the compressible Euler equations in the Set2NC perturbation form
 * (rho', u, v, w, theta') over a hydrostatic reference state, discretised with
 * continuous-Galerkin spectral elements on Legendre-Gauss-Lobatto (LGL) nodes on a
 * uniform box with walls on all six faces (Abdi, Giraldo et al., "Acceleration of the
 * IMplicit-EXplicit non-hydrostatic unified model of the atmosphere on manycore
 * processors", arXiv:1702.04316).  The time step is the horizontally-explicit,
 * vertically-implicit (HEVI) "1D-IMEX" ARK2 step of Sec. "IMEX time integration"
 * (Eq. sieqn1d, Table 1): explicit right-hand side plus per-column Schur-complement
 * solves with banded LU factors formed once per time-step size (Sec. "1D-IMEX kernels",
 * Algorithms 7 and 9).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh: nex x ney x nez elements of polynomial order N (1 <= N <= 8).  Global nodes:
 *   nxg = nex*N+1, nyg = ney*N+1, M = nez*N+1 (nodes per column), ncol = nxg*nyg,
 *   nnode = ncol*M.  Column id col = iy*nxg + ix; global node id g = col*M + iz
 *   (the nodes of one column are consecutive: Sec. "1D-IMEX kernels").
 * State layout ("SoA"): a contiguous float64 device array of 5*nnode values, field f at
 *   offset f*nnode, fields in the order rho', u, v, w, theta' (SI units: kg/m^3, m/s,
 *   m/s, m/s, K).  All device pointers must be 8-byte aligned; the library reads and
 *   writes exactly the documented extents.
 * Ownership: the caller owns every state/rhs/vector buffer it passes.  The context owns
 *   its tables, the stored LU factors and its workspace, all allocated by numa_init and
 *   released by numa_destroy.
 * Streams: every device call is enqueued on the context's stream (numa_init /
 *   numa_set_stream) and is asynchronous unless stated otherwise; a return of NUMA_OK
 *   means "validated and enqueued".  Errors detected on the device (zero pivot,
 *   non-finite values) are latched into a device status word that numa_status() reads.
 * Errors: every int-returning call returns one of the NUMA_* codes below and never
 *   aborts; numa_last_error() gives a one-line message for the last failing call.
 */
#ifndef NUMA_H
#define NUMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  NUMA_OK = 0,
  NUMA_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad mesh) */
  NUMA_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  NUMA_ERR_OOM = 3,          /* device allocation failed */
  NUMA_ERR_NOT_FACTORED = 4, /* a solve was requested before numa_factor_columns */
  NUMA_ERR_PIVOT = 5,        /* zero or non-finite pivot in the column LU */
  NUMA_ERR_NONFINITE = 6,    /* non-finite value detected in a state */
  NUMA_ERR_TIMEOUT = 7,      /* a bounded device wait gave up */
  NUMA_ERR_SCRATCH = 8       /* the problem needs more than the static scratch array holds */
};

/* Uniform box mesh and reference state (Sec. "Equation Set2NC").
 * theta_s: surface potential temperature of the reference state in K (<= 0 selects 300);
 * n_bv: Brunt-Vaisala frequency in 1/s of the reference state (0: isentropic,
 *       theta0 = theta_s; > 0: theta0 = theta_s exp(n_bv^2 z / g)). */
typedef struct numa_mesh_desc {
  int nex, ney, nez;
  double Lx, Ly, Lz;
  double theta_s;
  double n_bv;
} numa_mesh_desc;

typedef struct numa_ctx numa_ctx;

/* numa_query keys */
enum {
  NUMA_Q_NCOL = 0,          /* number of columns */
  NUMA_Q_M = 1,             /* nodes per column */
  NUMA_Q_NNODE = 2,         /* global nodes */
  NUMA_Q_NELEM = 3,         /* elements */
  NUMA_Q_HALF_BAND = 4,     /* half-bandwidth of the stored column matrix: 2N (Schur form) or
                               3N + 1 (standard form) */
  NUMA_Q_FACTOR_BYTES = 5,  /* bytes of stored LU factors */
  NUMA_Q_WORKSPACE_BYTES = 6, /* bytes of step workspace */
  NUMA_Q_FACTORED = 7,      /* 1 once numa_factor_columns succeeded */
  NUMA_Q_N = 8,             /* polynomial order */
  NUMA_Q_PRECISION = 9,     /* NUMA_PREC_FP64, NUMA_PREC_MIXED, NUMA_PREC_RHS32 or NUMA_PREC_DF */
  NUMA_Q_COLUMN_FORM = 10,  /* NUMA_COLUMN_SCHUR or NUMA_COLUMN_STANDARD */
  NUMA_Q_SCHEME = 11,       /* NUMA_SCHEME_ARK2 .. NUMA_SCHEME_ARK5 */
  NUMA_Q_IMEX = 12          /* NUMA_IMEX_1D or NUMA_IMEX_3D */
};

/* Options of numa_init_ex.
 * precision: NUMA_PREC_FP64 (default) -- the method in FP64 throughout;
 *            NUMA_PREC_MIXED -- the mixed-precision form: the explicit right-hand side in
 *            FP32 on FP32 copies of the perturbation fields (P' from the equation of state
 *            and the reference state stay FP64), the column Schur matrices factored and
 *            solved in FP32 with refine_iters sweeps of FP64 iterative refinement (FP64
 *            residual with the matrix-free Schur operator), FP64 state accumulation.
 *            NUMA_PREC_RHS32 -- the FP32 right-hand side of the mixed form with the FP64
 *            column factors and direct solve (no refinement).  On GB300 the fused FP64 stage
 *            is faster than FP32 substitutions plus an FP64 refinement residual (the
 *            substitutions are latency bound and the residual costs about what the FP64
 *            solve costs), so this keeps the FP32 part where it pays.
 *            NUMA_PREC_DF -- the right-hand side's DSS'd derivative sums in double-float
 *            arithmetic (each value an unevaluated sum of two FP32 numbers, about 48
 *            significant bits; products by Dekker's method, sums by Knuth's TwoSum), its
 *            pointwise terms, the equation of state, the column solves and the state in
 *            FP64.  Accurate to the FP64 method's parity bars; it moves the bulk of the
 *            right-hand side off GB300's narrow FP64 pipe onto the FP32 pipe.
 * refine_iters: FP64 refinement sweeps per solve in the mixed form (0..8; numa_init_ex with
 *               opt = NULL uses 1).
 * column_form: NUMA_COLUMN_SCHUR (default) -- the paper's Schur-complement column system in
 *              the pressure, M x M with half-bandwidth 2N per column;
 *              NUMA_COLUMN_STANDARD -- the standard (non-Schur) column system the paper
 *              contrasts it with (Sec. "Performance of IMEX on manycore processors"): the
 *              3M x 3M matrix I - lam L_V on (rho', w, theta') itself, unknowns ordered level
 *              by level (half-bandwidth 3N + 1), factored by the same banded LU without
 *              pivoting; M*3*(6N+3) doubles per column instead of M*(4N+1).  FP64 only;
 *              numa_solve_columns and the differentiation form need the Schur form.
 * scheme: NUMA_SCHEME_ARK2 (default) -- the second-order ARK of Table 1 (b = b~);
 *         NUMA_SCHEME_ARK3 -- a third-order ARK for the paper's higher-order runs, whose
 *         tableau the paper does not print: ARK3(2)4L[2]SA of Kennedy and Carpenter (2003),
 *         four stages, one implicit diagonal gamma = 0.4358665215084590 (the factors are
 *         formed at lam = gamma dt), b = b~ (numa_ark3_tableau);
 *         NUMA_SCHEME_ARK4, NUMA_SCHEME_ARK5 -- fourth- and fifth-order ARKs for the same
 *         runs: ARK4(3)6L[2]SA (six stages, gamma = 1/4) and ARK5(4)8L[2]SA (eight stages,
 *         gamma = 41/200) of Kennedy and Carpenter (2003), b = b~; ARK5's explicit a_86,
 *         a_87 are the solution of its fifth-order conditions given the other published
 *         entries (numa_ark_tableau).  ARK3 - ARK5: FP64 Schur form; ARK4 and ARK5 with
 *         1D-IMEX only.  The differentiation form and ensembles use ARK2.
 * imex: NUMA_IMEX_1D (default) -- the paper's 1D-IMEX (HEVI) method with stored column
 *       factors; NUMA_IMEX_3D -- 3D-IMEX in the Schur form (Eqs. utteqn, helm2nc with the
 *       full gradient): the whole linear operator implicit, one pressure unknown per node,
 *       BiCGstab left-preconditioned by a polynomial of degree pbno_order (Algorithm
 *       "BiCGstabPBNO"), no stored factors; stepped by numa_step_imex3d.  The paper's PBNO
 *       coefficients come from a least-squares fit it does not reproduce; these are the
 *       Chebyshev minimax polynomial on [1, l_max], l_max estimated by power iteration when
 *       the time step is set.  FP64 Schur form only.
 * pbno_order: polynomial degree P of the 3D preconditioner (0..NUMA_MAX_PBNO_ORDER; 0 in
 *             the struct means the default 2).
 * krylov_max_iters, krylov_tol: BiCGstab stops when the preconditioned residual's 2-norm
 *             has dropped by krylov_tol (default 1e-12; 0 means the default), or fails with
 *             NUMA_ERR_TIMEOUT after krylov_max_iters (default 500; 0 means the default).
 * precond: left preconditioner of the 3D solve: NUMA_PRECOND_PBNO (default; the paper's
 *          polynomial, Chebyshev reading) or NUMA_PRECOND_COLUMN -- the 1D-IMEX column Schur
 *          matrix of the same lam, factored and stored per column as for 1D-IMEX, solved
 *          exactly as a vertical-line preconditioner (a choice beyond the paper: the stiffest
 *          part of S is vertical when C_V > C_H; the converged solution is the same). */
enum { NUMA_PREC_FP64 = 0, NUMA_PREC_MIXED = 1, NUMA_PREC_RHS32 = 2, NUMA_PREC_DF = 3 };
enum { NUMA_COLUMN_SCHUR = 0, NUMA_COLUMN_STANDARD = 1 };
enum { NUMA_SCHEME_ARK2 = 0, NUMA_SCHEME_ARK3 = 1, NUMA_SCHEME_ARK4 = 2, NUMA_SCHEME_ARK5 = 3 };
#define NUMA_MAX_STAGES 8   /* stages of the longest scheme (ARK5) */
enum { NUMA_IMEX_1D = 0, NUMA_IMEX_3D = 1 };
enum { NUMA_PRECOND_PBNO = 0, NUMA_PRECOND_COLUMN = 1 };
#define NUMA_MAX_PBNO_ORDER 8
typedef struct numa_options {
  int precision;
  int refine_iters;
  int column_form;
  int scheme;
  int imex;
  int pbno_order;
  int krylov_max_iters;
  double krylov_tol;
  int precond;
} numa_options;

/* Create a context: validates the mesh, builds the LGL nodes/weights/derivative matrix
 * (Sec. "Volume kernels": sD), the reference state and its discrete vertical gradients
 * (Sec. "Volume kernels": reference gradients computed once at startup), uploads the
 * tables, allocates workspace and, if dt > 0, calls numa_factor_columns(ctx, dt).
 * stream: a cudaStream_t (NULL = the legacy default stream) used by every later call.
 * Synchronous.  On failure *out is NULL and the code says why (no message is kept). */
int numa_init(const numa_mesh_desc* mesh, int N, double dt, void* stream, numa_ctx** out);

/* numa_init with options (NULL = the defaults of numa_init).  Every entry point below
 * follows the context's precision; buffers passed by the caller are FP64 in both. */
int numa_init_ex(const numa_mesh_desc* mesh, int N, double dt, const numa_options* opt,
                 void* stream, numa_ctx** out);

/* Release everything the context owns (synchronises its stream).  NULL is a no-op. */
void numa_destroy(numa_ctx* ctx);

/* Change the stream later calls are enqueued on. */
int numa_set_stream(numa_ctx* ctx, void* stream);

/* Explicit right-hand side R(q) of the Set2NC perturbation equations (Sec. "Equation
 * Set2NC"), cG with LGL derivatives (Algorithm 2) and direct stiffness summation
 * (Sec. "Direct stiffness summation"), wall-normal velocity tendencies zeroed on the
 * six walls.  q, rhs: device SoA arrays of 5*nnode doubles; must not overlap. */
int numa_rhs_explicit(numa_ctx* ctx, const double* q, double* rhs);

/* Form, for every column, the Schur-complement matrix S(lam), lam = (1 - 1/sqrt2) dt
 * (the SDIRK diagonal of Table 1 times dt), by probing the left-hand side with unit
 * vectors (Algorithm 7), factor it by banded LU without pivoting (Algorithm 9) and store
 * the factors (Sec. "1D-IMEX kernels").  Also sets the context's IMEX time step to dt.
 * Per-column factor storage: M*(4N+1) doubles.  A zero or non-finite pivot latches
 * NUMA_ERR_PIVOT in the device status. */
int numa_factor_columns(numa_ctx* ctx, double dt);

/* Solve S x = b for every column with the stored factors (forward then back
 * substitution).  b, x: device arrays of ncol*M doubles in column order (g = col*M+iz);
 * x == b (in place) is allowed.  NUMA_ERR_NOT_FACTORED before numa_factor_columns.
 * FP64 contexts stream the factors into shared memory with bulk (TMA) copies; the right-hand
 * side and the solution move by bulk copies too when b and x are 16-byte aligned (plain
 * loads and stores otherwise; the result bits are the same).  A bounded device wait that
 * gives up (it never should) latches NUMA_ERR_TIMEOUT in the device status and leaves the
 * affected columns of x unwritten.  The environment variable NUMA_SOLVE=regs, read once per
 * process, selects the register-pipelined kernel instead (same arithmetic, same bits).
 * NUMA_TEST_SOLVE_TIMEOUT=1, read at every call and meant for tests only, arms the first
 * factor row's barrier of every warp for 16 bytes more than its copy delivers, so that
 * the wait gives up after its bound and the call latches NUMA_ERR_TIMEOUT. */
int numa_solve_columns(numa_ctx* ctx, const double* b, double* x);

/* nsteps >= 0 HEVI 1D-IMEX ARK2 steps of size dt (the dt of the last
 * numa_factor_columns) from q_in to q_out (Sec. "Linear multi-stage methods", Eq.
 * sieqn1d, Table 1 with b = b~).  q_in == q_out (in place) is allowed; otherwise q_in is
 * not modified.  nsteps == 0 copies q_in to q_out. */
int numa_step_imex1d(numa_ctx* ctx, const double* q_in, double* q_out, int nsteps);

/* Stage i in {2, ..., s} of the context's scheme (s = 3, 4, 6 or 8; numa_ark_tableau) in
 * the stage form of Sec. "Linear multi-stage methods": predictor q(i)_e = q^n +
 * dt sum_{j<i} a_ij R(q(j)), shift by sum_{j<i} c_ij q(j) with c_ij = (a~_ij - a_ij)/a~_ii
 * and q(1) = q^n, column solve at lam = a~_ii dt, extraction, un-shift.  R: host array of
 * i-1 device pointers R(q(1)) .. R(q(i-1)); Q: host array of i-2 device pointers q(2) ..
 * q(i-1) (may be NULL for i = 2).  Device arrays 5*nnode doubles, SoA.  q_out must not
 * overlap an input (NUMA_ERR_ARG).  FP64 Schur-form 1D-IMEX contexts only (NUMA_ERR_ARG otherwise);
 * NUMA_ERR_NOT_FACTORED before numa_factor_columns.  The general form of numa_imex_stage
 * (the same kernel phases; it reads only the terms with nonzero coefficients), exposed so
 * that each stage of ARK3 - ARK5 can be checked on its own. */
int numa_imex_stage_s(numa_ctx* ctx, int stage, const double* qn, const double* const* R,
                      const double* const* Q, double* q_out);

/* One fused 1D-IMEX stage i in {2, 3} (rows 2 and 3 of Table 1): explicit predictor,
 * Schur right-hand side (Algorithm 4), column solve, extraction of (rho', w, theta')
 * and the q~ recombination, producing the stage value q(i).  qn = q^n, R1 = R(q(1)),
 * R2 = R(q(2)) (stage 3 only), q2 = q(2) (stage 3 only; pass NULL for stage 2).  q_out
 * must not overlap an input (NUMA_ERR_ARG): the kernel parks intermediate values in it.
 * Exposed so that each row of the step can be checked on its own. */
int numa_imex_stage(numa_ctx* ctx, int stage, const double* qn, const double* R1,
                    const double* R2, const double* q2, double* q_out);

/* nsteps explicit five-stage third-order SSP Runge-Kutta steps of size dt (the RK35
 * comparator of Sec. "Performance of IMEX on manycore processors"; two-register
 * Shu-Osher form, coefficients in numa_rk35_coefficients).  q_in == q_out allowed. */
int numa_step_explicit_rk(numa_ctx* ctx, const double* q_in, double* q_out, double dt,
                          int nsteps);

/* Host-buffer driver: copies q_in_host (5*nnode doubles, pinned memory recommended) to
 * the device, runs nsteps of method 0 (1D-IMEX, dt of the factors) or 1 (RK35 with the
 * given dt), copies the result into q_out_host (may equal q_in_host) and synchronises.
 * Uses a device state buffer owned by the context (allocated on first use).  For the FP64
 * ARK2 Schur-form 1D-IMEX the copies are overlapped with the kernels: the upload runs
 * slab by slab (runs of whole tile rows of the right-hand side's thread order, at most 8
 * slabs; NUMA_HOST_SLABS overrides) on its own stream while the first right-hand side
 * consumes the slabs that have arrived, and each slab of the last step's result is
 * downloaded on a third stream as soon as its final update is done.  The result is bit
 * for bit that of numa_step_imex1d. */
int numa_run_host(numa_ctx* ctx, int method, const double* q_in_host, double* q_out_host,
                  int nsteps, double dt);

/* Per-kernel timing with CUDA events on the context's stream (off by default).
 * numa_profile(ctx, 1) clears the records and starts recording a start/stop event pair
 * around every kernel the context launches; numa_profile(ctx, 0) stops.
 * numa_profile_read synchronises and returns, for one kernel kind, the summed device
 * time in ms and the number of launches recorded. */
enum {
  NUMA_K_PRESSURE = 0,  /* equation-of-state pre-pass P'(q) of the right-hand side */
  NUMA_K_RHS = 1,       /* explicit right-hand side (with its fused update epilogue) */
  NUMA_K_STAGE = 2,     /* fused implicit stage: predictor, Schur RHS, solve, extraction */
  NUMA_K_SOLVE = 3,     /* stand-alone column solve */
  NUMA_K_FACTOR = 4,    /* probing + banded LU */
  NUMA_K_RHS_TLM = 5,   /* tangent-linear right-hand side (with its dP' pre-pass) */
  NUMA_K_RHS_ADJ = 6,   /* adjoint right-hand side (weights pass + transposed gather) */
  NUMA_K_STAGE_ADJ = 7, /* adjoint of the fused implicit stage (transposed column solve) */
  NUMA_K_SCHUR3D = 8,   /* one application of the 3D Schur operator (gradient + divergence) */
  NUMA_K_NKINDS = 9
};
int numa_profile(numa_ctx* ctx, int enable);
int numa_profile_read(numa_ctx* ctx, int kind, double* total_ms, long long* launches);

/* Element-to-global map and its inverse, produced on the device by the same index
 * functions the kernels use.  l2g: device int32 [nelem][(N+1)^3], element
 * e = ex + nex*(ey + ney*ez), local node l = i + (N+1)*(j + (N+1)*k).  g2l: device int32
 * [nnode][8]: the element-local ids e*(N+1)^3 + l that DSS sums into node g, ascending,
 * padded with -1.  Either pointer may be NULL. */
int numa_connectivity(numa_ctx* ctx, int32_t* l2g, int32_t* g2l);

/* Copy the stored factors of one column to host memory: M*(4N+1) doubles, row-major
 * [row][band], band index b = j - i + 2N for entry (i, j); the unit diagonal of L is not
 * stored (entries b < 2N hold L, b >= 2N hold U).  The mixed form's FP32 factors are
 * widened to double.  Synchronous. */
int numa_column_factors(numa_ctx* ctx, long long col, double* host_out);
/* (standard form: 3M rows of 2(3N+1)+1 = 6N+3 band entries, the level-interleaved unknowns
 * 3 l + v, v = 0 rho', 1 w, 2 theta') */

/* Host copy of the per-level reference tables, 8*M doubles in the order
 * z, rho0, theta0, P0, G0, H0, d(rho0)/dz, d(theta0)/dz.  Synchronous. */
int numa_reference_levels(const numa_ctx* ctx, double* host_out);

/* Count the non-finite entries of a device array of n doubles; synchronous. */
int numa_count_nonfinite(numa_ctx* ctx, const double* x, long long n, long long* count);

/* Synchronise the stream and return the latched device status (NUMA_OK or the first
 * NUMA_ERR_* a kernel recorded), then clear it.  NUMA_ERR_PIVOT: a zero or non-finite pivot
 * in numa_factor_columns.  NUMA_ERR_NONFINITE: a step met a non-finite state -- the
 * equation-of-state passes (the P' pre-pass of a step's or RK stage's input, the fused P'
 * of each implicit stage value) and the ARK4/ARK5 final combination test their results; a
 * non-finite u, v or w reaches them within one step through the coupled tendencies.
 * NUMA_ERR_TIMEOUT: a bounded wait of the FP64 stand-alone column solve on its bulk copies
 * gave up. */
int numa_status(numa_ctx* ctx, int* status);

int numa_query(const numa_ctx* ctx, int what, long long* out);

/* One-line message of the last failing call on this context ("" if none). */
const char* numa_last_error(const numa_ctx* ctx);

/* ---- differentiation form -------------------------------------------------------------
 * Tangent-linear (TLM) and adjoint models of the HEVI 1D-IMEX step.  The paper integrates
 * forward only; these calls apply the chain rule to its steps: R of Sec. "Equation Set2NC"
 * (Algorithm 2, Sec. "Direct stiffness summation"), the column solve of Eqs. utteqn and
 * helm2nc with the stored factors of Algorithm 9, and the ARK2 step of Table 1 in the stage
 * form of Sec. "Linear multi-stage methods".  The adjoint of a linear map A is its
 * transpose with respect to the plain Euclidean dot product of the SoA arrays:
 * <lam, A dq> = <A^T lam, dq>.  All calls need an FP64 context (NUMA_ERR_ARG otherwise),
 * work in the context's stream, and allocate, on first use, a workspace of 59*nnode
 * doubles owned by the context (NUMA_ERR_OOM if that fails).  The adjoint right-hand side
 * gathers rather than scatters (no atomics): results are bitwise reproducible.  The
 * implicit stage is linear in its inputs, so its TLM is numa_imex_stage applied to the
 * perturbations. */

/* dR = R'(q) dq.  q, dq, dR: device SoA arrays of 5*nnode doubles; dR must not overlap q
 * or dq.  Uses the context's R workspace. */
int numa_rhs_tlm(numa_ctx* ctx, const double* q, const double* dq, double* dR);

/* q_adj = R'(q)^T lam (overwritten).  q, lam, q_adj: device arrays of 5*nnode doubles;
 * q_adj must not overlap q or lam. */
int numa_rhs_adjoint(numa_ctx* ctx, const double* q, const double* lam, double* q_adj);

/* Solve S^T x = b for every column with the stored factors S = L U (U^T forward, then L^T
 * backward substitution).  Layout as numa_solve_columns; x == b (in place) allowed.
 * NUMA_ERR_NOT_FACTORED before numa_factor_columns. */
int numa_solve_columns_transposed(numa_ctx* ctx, const double* b, double* x);

/* Adjoint of numa_imex_stage: given lam, the adjoint of the stage output q(i), ADD the
 * adjoints of its inputs: qn_adj += (dq(i)/dq^n)^T lam, R1_adj += (dq(i)/dR1)^T lam, and for
 * stage 3 R2_adj and q2_adj likewise (stage 2: R2_adj and q2_adj are ignored and may be
 * NULL).  All arrays 5*nnode doubles on the device; the outputs must not overlap lam or
 * each other. */
int numa_imex_stage_adjoint(numa_ctx* ctx, int stage, const double* lam, double* qn_adj,
                            double* R1_adj, double* R2_adj, double* q2_adj);

/* nsteps >= 1 HEVI steps of the state and of its tangent: q_out = q^{n+nsteps} and
 * dq_out = (dq^{n+nsteps}/dq^n) dq.  In place (q_out == q, dq_out == dq) allowed. */
int numa_step_imex1d_tlm(numa_ctx* ctx, const double* q, const double* dq, double* q_out,
                         double* dq_out, int nsteps);

/* Adjoint of one HEVI step taken from state q: lam = (dq^{n+1}/dq^n)^T lam_next.  The
 * step is retaken from q (numa_step_imex1d) for its stage states.  lam == lam_next (in
 * place) allowed. */
int numa_step_imex1d_adjoint(numa_ctx* ctx, const double* q, const double* lam_next,
                             double* lam);

/* Checkpointed forward run: nsteps HEVI steps from q0 to qT, storing the state before step
 * s in ckpt[s/every] for every s that is a multiple of every.  ckpt: device array of
 * ceil(nsteps/every) * 5*nnode doubles.  q0 is not modified; qT must not overlap q0. */
int numa_imex1d_forward_checkpointed(numa_ctx* ctx, const double* q0, double* qT, int nsteps,
                                     int every, double* ckpt);

/* Adjoint of that run: lam0 = (dq^T/dq^0)^T lamT.  Segments are processed last to first;
 * each is retaken from its checkpoint, keeping every step's state q^n and stage states q(2),
 * q(3) in work (device, 3 * every * 5*nnode doubles, caller-owned scratch), and its steps are
 * then run backwards from those states (numa_step_imex1d_adjoint without the retaken step).
 * lam0 == lamT allowed. */
int numa_imex1d_adjoint_checkpointed(numa_ctx* ctx, const double* ckpt, int nsteps, int every,
                                     const double* lamT, double* lam0, double* work);

/* ---- 3D-IMEX (Schur form, BiCGstab + polynomial preconditioner) -------------------------
 * Calls for a context made with options.imex = NUMA_IMEX_3D (NUMA_ERR_ARG otherwise; the 1D
 * entry points numa_step_imex1d, numa_imex_stage, numa_solve_columns and the
 * differentiation form reject a 3D context).  numa_factor_columns(ctx, dt) sets the step,
 * forms the per-level tables and the preconditioner (power iteration on S, about 60
 * operator applications).  The workspace (20 x nnode doubles) is allocated on first use. */

/* SP = S(P) = P - lam F0 . u_p(P) - lam rho0 G0 div u_p(P), the 3D Schur operator (Eq.
 * helm2nc, left side).  P, SP: device arrays of nnode doubles, not overlapping. */
int numa_schur3d_apply(numa_ctx* ctx, const double* P, double* SP);

/* Solve S(x) = b by preconditioned BiCGstab from x = 0; *iters (may be NULL) receives the
 * iteration count.  b, x: nnode doubles, not overlapping.  NUMA_ERR_TIMEOUT when the
 * tolerance is not reached within krylov_max_iters. */
int numa_solve_schur3d(numa_ctx* ctx, const double* b, double* x, int* iters);

/* One 3D-IMEX stage i in {2, 3} (as numa_imex_stage, with the 3D implicit solve); *iters
 * (may be NULL) receives the BiCGstab iterations. */
int numa_imex3d_stage(numa_ctx* ctx, int stage, const double* qn, const double* R1,
                      const double* R2, const double* q2, double* q_out, int* iters);

/* nsteps 3D-IMEX steps (the context's scheme, ARK2 or ARK3) from q_in to q_out (in place
 * allowed). */
int numa_step_imex3d(numa_ctx* ctx, const double* q_in, double* q_out, int nsteps);

/* The preconditioner of a 3D context: l_max (spectrum bound used), lam_bar = 2/(1 + l_max),
 * coeffs[0..pbno_order] (c_i of the PBNO recursion), and the total BiCGstab iterations of
 * the last numa_step_imex3d call.  Any output pointer may be NULL. */
int numa_imex3d_info(const numa_ctx* ctx, double* l_max, double* lam_bar, double* coeffs,
                     long long* iters_last_step);

/* ---- ensembles ("batching form") -------------------------------------------------------
 * An ensemble of independent members, each with its own uniform box mesh, polynomial order
 * (4 <= N <= 6), reference state and HEVI time step dt (its column factors are formed at
 * its own dt).  Every phase of a step is one persistent launch per polynomial order present
 * for the whole ensemble (a work list of (member, block) items), so the launches per step
 * do not grow with the number of members; each step is captured as a CUDA graph on first
 * use for a given (q_in, q_out) pair and replayed.  numa_batch_init autotunes, per order,
 * the right-hand side's threads per CTA and the stage's columns per CTA on the ensemble.
 * States are packed: member m occupies doubles [off[m], off[m+1]) of one device array
 * (numa_batch_layout), in the single-mesh SoA layout of that member.  All calls use the
 * stream given to numa_batch_init and follow the error conventions above. */
typedef struct numa_batch numa_batch;

/* Synchronous set-up of nmembers members: meshes[m], N[m], dt[m].  On failure *out is NULL. */
int numa_batch_init(const numa_mesh_desc* meshes, const int* N, const double* dt, int nmembers,
                    void* stream, numa_batch** out);
void numa_batch_destroy(numa_batch* b);

/* Packed-state offsets: nmembers+1 values (the last is the total length in doubles). */
int numa_batch_layout(const numa_batch* b, long long* offsets);

/* nsteps HEVI 1D-IMEX steps of every member (each at its own dt) from q_in to q_out
 * (packed device arrays; in place allowed). */
int numa_batch_step_imex1d(numa_batch* b, const double* q_in, double* q_out, int nsteps);

/* 1 (default): replay each step as a CUDA graph; 0: launch the kernels directly. */
int numa_batch_set_graph(numa_batch* b, int enable);

/* The autotuned threads per CTA of the right-hand side, and columns and threads per CTA of
 * the stage, for the members of order N (all 0 if the ensemble has none); any output pointer
 * may be NULL. */
int numa_batch_tuning(const numa_batch* b, int N, int* rhs_threads, int* col_tile,
                      int* stage_threads);

/* numa_query / numa_reference_levels of one member. */
int numa_batch_member_query(const numa_batch* b, int member, int what, long long* out);
int numa_batch_reference_levels(const numa_batch* b, int member, double* host_out);
const char* numa_batch_last_error(const numa_batch* b);

/* ---- several GPUs: horizontal partition with a halo exchange ------------------------------
 * In HEVI the implicit column solves cross no partition boundary (Sec. "IMEX time
 * integration"), so a horizontal partition of the columns needs one exchange per evaluation
 * of the explicit right-hand side: the halo node columns its stencil reads (the direct
 * stiffness summation across the cut; Sec. "Scalability").  Rank r of a px x py process grid
 * owns a rectangle of elements and computes on a window: the rectangle plus one element
 * toward each neighbour, run as an ordinary context of the window's size (numa_init with
 * info.window).  Node-column ownership: a rank owns the node columns [ex0 N, ex1 N) x
 * [ey0 N, ey1 N), plus the last node column where its rectangle touches the east or north
 * wall; every other node column of its window is halo, owned by one neighbour.  With the
 * halo holding the owners' values before every right-hand side, each owned node of the
 * window evolves exactly as on the whole mesh (the same kernels and arithmetic, so bit for
 * bit). */
#define NUMA_PART_MAX_NEIGH 8

typedef struct numa_part_desc {
  int px, py;   /* process grid: px ranks along x, py along y (each rectangle >= 2 elements wide) */
  int rank;     /* this rank, 0 <= rank < px*py; its grid position (rank % px, rank / px) */
} numa_part_desc;

typedef struct numa_part_info {
  int ex0, ex1, ey0, ey1;      /* owned elements [ex0, ex1) x [ey0, ey1) of the global mesh */
  int wx0, wx1, wy0, wy1;      /* the window's elements (owned + one toward each neighbour) */
  numa_mesh_desc window;       /* the window as a box of its own (same element size, bit for bit) */
  int own_x0, own_x1, own_y0, own_y1;   /* owned node columns, window-local, [x0, x1) x [y0, y1) */
  int nneigh;                            /* neighbours, at most NUMA_PART_MAX_NEIGH */
  int neigh[NUMA_PART_MAX_NEIGH];        /* their ranks, ascending */
  int nsend[NUMA_PART_MAX_NEIGH];        /* node columns sent to each */
  int nrecv[NUMA_PART_MAX_NEIGH];        /* node columns received from each */
} numa_part_info;

/* Host only (no device work, usable without a GPU): the partition of a global mesh for one
 * rank.  NUMA_ERR_ARG for a bad mesh or grid, or a rectangle narrower than two elements. */
int numa_part_plan(const numa_mesh_desc* global, int N, const numa_part_desc* part,
                   numa_part_info* info);

/* Host only: the exchange lists with neighbour k (0 <= k < info.nneigh), as window-local
 * column ids (col = iy*nxw + ix of the window), sorted by global column id.  send_cols:
 * info.nsend[k] ints (owned columns inside the neighbour's window); recv_cols:
 * info.nrecv[k] ints (halo columns the neighbour owns).  The send list of rank a to b and
 * the receive list of b from a name the same global columns in the same order. */
int numa_part_columns(const numa_mesh_desc* global, int N, const numa_part_desc* part, int k,
                      int* send_cols, int* recv_cols);

/* Halo messages: copy the listed node columns of nf <= 8 fields into (gather) or out of
 * (scatter) one contiguous device buffer, buf[(f*ncols + c)*M + lev] = fields[f][cols[c]*M +
 * lev].  fields: host array of nf device pointers, each a field of ncol*M doubles of the
 * context's mesh (a state's field f is state + f*nnode); cols: device int32 array of ncols
 * column ids; buf: device, nf*ncols*M doubles.  Enqueued on the context's stream.  A listed
 * column outside the context is skipped and numa_status then reports NUMA_ERR_ARG. */
int numa_gather_columns(numa_ctx* ctx, const double* const* fields, int nf, const int* cols,
                        long long ncols, double* buf);
int numa_scatter_columns(numa_ctx* ctx, double* const* fields, int nf, const int* cols,
                         long long ncols, const double* buf);

/* One ARK2 step of numa_step_imex1d in three phases, for a caller that refreshes a
 * partition's halo between them (ARK2 1D-IMEX contexts; NUMA_ERR_ARG otherwise):
 *   phase 0: R1 = R(q_n), stage 2 -> q(2);
 *   phase 1: R2 = R(q(2)), stage 3 -> q(3);
 *   phase 2: q_out = q_n + dt sum_i b_i R(q(i)) (R(q(3)) in the update's epilogue).
 * q_n: the step's input (all phases; not modified), q_out: phase 2's output (may equal q_n).
 * Run in order, with nothing in between, the phases are numa_step_imex1d's kernels in its
 * order.  Before phases 1 and 2 the halo of q(2), resp. q(3), must hold the owners' values,
 * and so must P' of it when numa_step_buffers reports it fused (the stage writes P' of its
 * output for the next right-hand side); before phase 0 the halo of q_n. */
int numa_step_phase(numa_ctx* ctx, int phase, const double* q_n, double* q_out);

/* The context's stage values q(2), q(3) (5*nnode doubles each) and P' (nnode doubles, or NULL
 * where the context has none), and whether the stages write P' of their output (1) or the
 * next right-hand side recomputes it (0).  Device pointers owned by the context. */
int numa_step_buffers(numa_ctx* ctx, double** q2, double** q3, double** pp, int* pp_fused);

/* Size of the device scratch array used by numa_rhs_explicit_static.  Every GPU that loads
 * the library's device code holds an array of this size until the process exits.  With
 * CUDA's default lazy module loading the array is reserved when the module is first used on
 * a device, which can be the first call of numa_rhs_explicit_static: a process whose other
 * allocator is about to reserve most of the device memory should make one call (a warm-up)
 * first, or that first call can fail with NUMA_ERR_CUDA for lack of memory. */
#define NUMA_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* numa_rhs_explicit without any allocation.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory at the point of the call, for
 * example a latency-bound loop in which cudaMalloc/cudaFree would synchronise the device,
 * or a process whose device memory is already reserved by another allocator (a caching
 * allocator holding most of the GPU).  It takes no context: the mesh, the polynomial order
 * and the stream are passed directly.  The host builds the LGL and reference tables with
 * the same code as numa_init, so the result equals numa_rhs_explicit's bit for bit; the
 * tables reach the device inside kernel launch parameters, and the device side keeps the
 * equation-of-state pre-pass (nnode doubles) and the per-level tables in one file-scope
 * scratch array of NUMA_STATIC_SCRATCH_BYTES (64 MiB: meshes up to
 * 8,388,608 - 15 M - (2N+1) M nodes and M <= 1024 levels; larger problems return
 * NUMA_ERR_SCRATCH before any device work).
 * q, rhs: device SoA arrays of 5*nnode doubles, as for numa_rhs_explicit.  The first call
 * on each device looks up the scratch array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that first call before
 * any stream capture.  A device reset (cudaDeviceReset) can move the array, so this entry
 * point must not be called on a device after a reset in the same process.  Every call
 * overwrites the parts of the scratch it reads, so nothing has to start at zero, but all
 * calls share the one array: calls that overlap on the GPU (different streams, or different
 * host threads without ordering) race on it.  Calls no cudaMalloc, cudaFree or other
 * allocating routine. */
int numa_rhs_explicit_static(const numa_mesh_desc* mesh, int N, const double* q, double* rhs,
                             void* stream);

/* The RK35 two-register coefficients (alpha[5], beta[5]) and the ARK2 tableau
 * (a[9], at[9], b[3], row-major 3x3) the library uses.  Host only; any pointer may be
 * NULL. */
void numa_rk35_coefficients(double* alpha, double* beta);
void numa_ark2_tableau(double* a, double* at, double* b);
/* The ARK3 tableau (a[16], at[16], b[4], row-major 4x4) of NUMA_SCHEME_ARK3.  Host only; any
 * pointer may be NULL. */
void numa_ark3_tableau(double* a, double* at, double* b);
/* The tableau of any scheme: s stages (3, 4, 6 or 8), a and at row-major s x s into arrays
 * of NUMA_MAX_STAGES^2 doubles, b into NUMA_MAX_STAGES doubles.  Each published rational
 * p/q is the correctly rounded double of p/q.  Host only; returns NUMA_ERR_ARG for an
 * unknown scheme; any pointer may be NULL. */
int numa_ark_tableau(int scheme, double* a, double* at, double* b, int* s);

/* The FP64 <-> FP32 conversions that the FP32 forms' pre-pass and column stages do with
 * integer instructions (the conversion instructions compete with FP64 arithmetic on GB300),
 * exposed so that they can be checked against IEEE-754 conversion.  numa_convert_f64_f32:
 * y[i] = x[i] rounded to the nearest float, ties to even (FP32 subnormals, overflow to
 * infinity); numa_convert_f32_f64: y[i] = x[i] exactly.  A NaN gives a NaN.  x, y: device
 * arrays of n elements, n >= 0, naturally aligned; enqueued on `stream` (NULL: the default
 * stream).  Returns NUMA_ERR_ARG for a bad pointer or size, NUMA_ERR_CUDA if the launch
 * fails. */
int numa_convert_f64_f32(const double* x, float* y, long long n, void* stream);
int numa_convert_f32_f64(const float* x, double* y, long long n, void* stream);

/* y[i] = 1 / x[i] as the FP64 right-hand side computes 1 / rho: Newton's method for the
 * reciprocal from an FP32 seed with one third-order step, within one unit in the last place
 * of the correctly rounded quotient; where x or 1 / x lies outside the normal FP32 range
 * (zeros, infinities and NaN included) it is the IEEE quotient.  Exposed so that it can be
 * checked against division.  x, y: device arrays of n doubles (8-byte aligned); enqueued on
 * `stream` (NULL: the default stream).  Returns NUMA_ERR_ARG for a bad pointer or size,
 * NUMA_ERR_CUDA if the launch fails. */
int numa_reciprocal(const double* x, double* y, long long n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NUMA_H */
