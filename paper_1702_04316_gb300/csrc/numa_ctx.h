// Host-side definition of the context (include/numa.h declares it opaque).  Shared by
// numa_api.cu and batch.cu.
#pragma once
#include <string>
#include <vector>

#include "numa.h"
#include "numa_internal.cuh"

struct numa_ctx {
  Geom G;
  Coef3 C;
  cudaStream_t stream = nullptr;
  std::string err;
  double dt = 0.0, lam = 0.0;
  bool factored = false;
  double theta_s = 300.0, n_bv = 0.0;
  // host copies of the per-level tables
  std::vector<double> z, rho0, theta0, P0, G0, H0, drho0, dtheta0, F0z, dzband;
  // device memory
  double* d_lev = nullptr;      // reference tables + dz band + dz taps
  int* d_levi = nullptr;        // dz tap offsets and counts
  int col_tile = 32;            // columns per CTA of the column kernels
  RefLev R{};
  StageTab T{};
  double* d_stage_tab = nullptr;
  Factors F{};
  double* d_work = nullptr;     // Pp, R1, R2, q2, q3 (+ R3, q4 for ARK3; + R3..Rs, q4..qs
                                // for s-stage schemes), each 5*nnode but Pp
  double *Pp = nullptr, *R1 = nullptr, *R2 = nullptr, *q2 = nullptr, *q3 = nullptr;
  double *R3 = nullptr, *q4 = nullptr;     // ARK3 only
  // s-stage schemes (ARK4, ARK5): Rk[j] = R(q(j+1)), Qk[j] = q(j+1) (Qk[0] unused: q(1) = q^n)
  double* Rk[NUMA_MAX_STAGES] = {};
  double* Qk[NUMA_MAX_STAGES] = {};
  int scheme = NUMA_SCHEME_ARK2;
  // 3D-IMEX (Schur form, BiCGstab + polynomial preconditioner)
  bool imex3d = false;
  int pbno_order = 2, krylov_max_iters = 500, precond = NUMA_PRECOND_PBNO;
  double krylov_tol = 1e-12, l_max = 0.0, lam_bar = 0.0;
  double pbno_c[NUMA_MAX_PBNO_ORDER + 1] = {};
  long long krylov_last = 0;            // BiCGstab iterations of the last 3D-IMEX step
  double* d_w3 = nullptr;               // 3D-IMEX workspace (20 x nnode + reduction)
  // mixed-precision form: FP32 stencil fields (6 x nnode) and FP32 R1, R2 (5 x nnode each)
  float *F32 = nullptr, *R1f = nullptr, *R2f = nullptr;
  // double-float form: (hi, lo) FP32 pairs of the six stencil fields (6 x nnode)
  float2* F2 = nullptr;
  int precision = NUMA_PREC_FP64;
  int* d_perm = nullptr;        // class-sorted thread order of the right-hand side
  long long nperm = 0;
  unsigned* d_status = nullptr;
  unsigned long long* d_count = nullptr;
  double* d_hoststate = nullptr;
  // pipelined host runs (numa_run_host): tile-row offsets of the RHS thread order, the
  // upload and download streams and their per-slab events
  std::vector<long long> perm_row_off;
  std::vector<int> perm_row_y;
  cudaStream_t cs_in = nullptr, cs_out = nullptr, cs_p = nullptr;
  std::vector<cudaEvent_t> host_ev;
  // differentiation form (allocated on first use): 59 x nnode doubles of workspace and the
  // transposed derivative tap tables of the three axes
  double* d_adj = nullptr;
  void* d_adjtab = nullptr;
  size_t factor_bytes = 0, work_bytes = 0;
  // per-kernel event timing
  struct ProfRec { int kind; cudaEvent_t a, b; };
  std::vector<ProfRec> prof;
  size_t prof_n = 0;
  bool prof_on = false;
};


// Event pair around one launch of kernel kind `kind` when profiling is on (returns the
// record index, or -1); prof_end records the closing event.
long prof_begin(numa_ctx* c, int kind);
void prof_end(numa_ctx* c, long idx);

// 3D-IMEX start-up (imex3d.cu): spectrum estimate and preconditioner coefficients.
int numa_imex3d_setup(numa_ctx* c);
// q_out = qn + dt sum_i b_i R(q(i)) with the stored R1, R2 (and R3 for four-stage schemes)
// and R of q_last evaluated in the epilogue of the explicit right-hand side (numa_api.cu).
int numa_rhs_final(numa_ctx* c, const double* q_last, const double* qn, double* q_out,
                   const double* b);

// Coefficients of IMEX stage 2 or 3 for the context's dt (Table 1 with b = b~).
StageCoef numa_stage_coef(const numa_ctx* c, int stage);
