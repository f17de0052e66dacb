// Internal declarations shared by the CUDA translation units of libnuma.
// Nothing here is part of the C ABI (include/numa.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "numa.h"

#define NUMA_MAXN 8
#define NUMA_MAXNQ (NUMA_MAXN + 1)

// Physical constants of the model.  R and c_p reproduce the sound speed of 347.32 m/s at
// theta0 = 300 K (Sec. "Acoustic wave problem"); the paper does not give g.
#define NUMA_GRAV 9.80616
#define NUMA_P00 1.0e5
#define NUMA_RGAS 287.17
#define NUMA_CP 1004.67
#define NUMA_CV (NUMA_CP - NUMA_RGAS)
#define NUMA_GAMMA (NUMA_CP / NUMA_CV)

// Device status bits latched by kernels (read back by numa_status).
#define NUMA_ST_PIVOT 1u
#define NUMA_ST_NONFINITE 2u
#define NUMA_ST_TIMEOUT 4u
#define NUMA_ST_RANGE 8u      // an index list named a column outside the context

// Mesh sizes (see the conventions in include/numa.h).
struct Geom {
  int N, Nq;
  int nex, ney, nez;
  int nxg, nyg, M;
  long long ncol, nnode;
};

// LGL derivative rows of one axis, already scaled by the metric 2/h of that axis.
//   D[i*Nq + n]  : derivative at local node i from local node n (interior / wall rows);
//   Dl[n], Dr[n] : the two halves of the DSS-weighted derivative at an element interface
//                  node, from the element on the left (its row N) and on the right (its
//                  row 0), each multiplied by its local-weight share w/(w_N + w_0).
struct AxisCoef {
  double D[NUMA_MAXNQ * NUMA_MAXNQ];
  double Dl[NUMA_MAXNQ];
  double Dr[NUMA_MAXNQ];
};

struct Coef3 {
  AxisCoef x, y, z;
};

// Per-level reference tables on the device (length M each).  The box reference state
// depends on z only.
struct RefLev {
  const double* rho0;
  const double* inv_rho0;
  const double* theta0;
  const double* inv_theta0;
  const double* P0;
  const double* G0;
  const double* H0;
  const double* drho0;    // D_z rho0 (DSS'd discrete vertical derivative)
  const double* dtheta0;  // D_z theta0
  const double* F0z;      // G0 drho0 + H0 dtheta0
  const double* dz_band;  // DSS'd vertical derivative on a column, [M][2N+1], column j = m-N+b
  // the same rows without their exact zeros (LGL interior diagonal, the cancelling shared
  // node at an element interface): dz_n[m] taps dz_c[m*(2N+1)+t] at level m + dz_o[m*(2N+1)+t]
  const double* dz_c;
  const int* dz_o;
  const int* dz_n;
  // P0 C(gamma, k), k = 1..5, per level ([M][5]): the equation of state's five-term series
  // with P0 folded into its coefficients
  const double* P0c;
};

// Stored column factors, by matrix column j, transposed so that consecutive columns of the
// mesh are contiguous:
//   L[(j*hb + k-1)*ncol + col] = L(j+k, j),  k = 1..hb   (unit diagonal not stored)
//   U[(j*(hb+1) + 0)*ncol + col] = 1 / U(j, j)
//   U[(j*(hb+1) + k)*ncol + col] = U(j-k, j), k = 1..hb
// hb = 2N.  Entries outside the matrix are stored as zero.
// The mixed-precision form stores the same layout in float (L32, U32) and refines each
// solve refine_iters times with the FP64 operator.
// The standard column form (standard = 1) stores the 3M x 3M level-interleaved system
// I - lam L_V in the same layout with n = 3M unknowns per column and hb = 3N + 1.
// Layout of the stored column factors.  Mesh columns are grouped in blocks of kFacBlk = 32
// consecutive columns; a block stores, for every band row i and slot k in order, the entry
// of each of its 32 columns side by side.  A warp whose lanes take consecutive columns
// then reads each (i, k) as one contiguous line and walks its block's factors front to back.
// n rows (M, or 3M in the standard form), W slots per row (hb for L, hb + 1 for U); the
// allocation holds fac_cols(ncol) columns.  Entry (i, k) of column col is at
// fac_col_base(col, n, W) + (i * W + k) * kFacBlk.
constexpr int kFacBlk = 32;
__host__ __device__ inline long long fac_cols(long long ncol) {
  return (ncol + kFacBlk - 1) / kFacBlk * kFacBlk;
}
__host__ __device__ inline long long fac_col_base(long long col, int n, int W) {
  return (col / kFacBlk) * (long long)n * W * kFacBlk + (col % kFacBlk);
}

struct Factors {
  double* L;
  double* U;
  float* L32;
  float* U32;
  int hb;
  int mixed;
  int refine_iters;
  int standard;
};

// Coefficients of one IMEX stage i (a row of Table 1 with b = b~, or of the ARK3 tableau):
// the stage reads the i-1 previous stages.
struct StageCoef {
  double dt;
  double lam;       // a~_ii dt
  double a[3];      // a_i1 .. a_i3 (explicit; zero beyond i-1)
  double c[3];      // c_ij = (a~_ij - a_ij) / a~_ii
};

// Per-level coefficient tables of one lam for the fused stage (length M each):
//   wa_th = lam g / theta0;  wa_s = 1/A (0 at the two walls: w_a = 0 there)
//   kF = lam F0z;  kD = lam rho0 G0
//   kp1 = lam / (A rho0), kp2 = lam g / (A G0 rho0)  (0 at the two walls: w_p = 0 there)
//   kth = lam d(theta0)/dz;  invG0 = 1/G0;  H0G0 = H0/G0;  G0, H0
// with A = 1 + lam^2 (g/theta0) d(theta0)/dz; and, in the layout of RefLev::dz_c (M x (2N+1)),
// the column derivative's taps scaled per level: dzD = kD dz_c, dzP = kp1 dz_c, so that
// kD D_z f and kp1 D_z f cost one multiply-add per tap.
struct StageTab {
  const double *wa_th, *wa_s, *kF, *kD, *kp1, *kp2, *kth, *invG0, *H0G0, *G0, *H0;
  unsigned* status;   // the fused stage latches NUMA_ST_NONFINITE here when P' of its output
                      // is not finite (NULL: no check)
  const double *dzD, *dzP;
};

// True when x is an infinity or a NaN, from the exponent bits of its high word: integer
// instructions only, so the check takes no FP64 issue slots.
__device__ __forceinline__ unsigned not_finite(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) == 0x7ff00000u;
}

// ---- launchers (return the launch error) ----------------------------------------------
// rhs.cu
// RefLev::P0c on the host: P0c[m * 5 + k] = P0[m] C(gamma, k + 1), k < 5.
void eos_level_coefs(const double* P0, int M, double* P0c);
cudaError_t launch_pressure(const double* q, double* Pp, const Geom& G, const RefLev& R,
                            cudaStream_t s, unsigned* status = nullptr);
// P' for the nodes g0 <= g < g1 only.  Both pre-passes latch NUMA_ST_NONFINITE into status
// (NULL: no check) when a P' is not finite: a non-finite rho' or theta' of the input state.
cudaError_t launch_pressure_range(const double* q, double* Pp, const Geom& G, const RefLev& R,
                                  long long g0, long long g1, cudaStream_t s,
                                  unsigned* status = nullptr);
// MODE 0: out = R(q);  MODE 1 (RK stage): out = alpha*u0 + (1-alpha)*q + beta*dt*R(q);
// MODE 2 (ARK2 final): out = qn + dt*(b1*R1 + b2*R2 + b3*R(q));
// MODE 3 (four-stage ARK final, FP64 only): out = qn + dt*(b1*R1 + b2*R2 + b3*R3 + b4*R(q)).
struct RhsEpilogue {
  int mode;
  int use_u0;                     // mode 1: alpha != 0
  double alpha, one_minus_alpha, beta_dt;   // mode 1
  double b1dt, b2dt, b3dt, b4dt;  // modes 2, 3
  const double* u0;               // mode 1: u0; modes 2, 3: qn
  const void* R1;                 // modes 2, 3: double (FP64 method) or float (mixed form)
  const void* R2;
  const void* R3;                 // mode 3 (double)
};
// perm: class-sorted thread order from build_rhs_perm (nthreads entries), or NULL for the
// natural node order (nthreads = nnode; correct, but warps then mix node classes).
cudaError_t launch_rhs(const double* q, const double* Pp, double* out, const int* perm,
                       long long nthreads, const Geom& G, const Coef3& C, const RefLev& R,
                       const RhsEpilogue& ep, cudaStream_t s);
// Mixed-precision form: FP64 P', FP32 copies of the six stencil fields (6 x nnode floats),
// and the FP32 right-hand side (mode 0 writes out32; modes 1 and 2 as launch_rhs, with R1
// and R2 given as float arrays).
cudaError_t launch_prep32(const double* q, float* F32, const Geom& G, const RefLev& R,
                          cudaStream_t s);
// rhs_df.cu: the double-float variant -- P' and the (hi, lo) FP32 pairs of the six stencil
// fields (6 x nnode float2), then the right-hand side with double-float derivative sums and
// FP64 pointwise terms (epilogue modes as launch_rhs, FP64 arrays).
cudaError_t launch_prep_df(const double* q, float2* F2, const Geom& G, const RefLev& R,
                           cudaStream_t s);
cudaError_t launch_rhs_df(const double* q, const float2* F2, double* out, const int* perm,
                          long long nthreads, const Geom& G, const Coef3& C, const RefLev& R,
                          const RhsEpilogue& ep, cudaStream_t s);
cudaError_t launch_rhs32(const double* q, const float* F32, float* out32, double* out,
                         const int* perm, long long nthreads, const Geom& G, const Coef3& C,
                         const RefLev& R, const RhsEpilogue& ep, cudaStream_t s);
// FP32 right-hand side written as FP64 (mode 0, natural order) for numa_rhs_explicit.
cudaError_t launch_rhs32d(const double* q, const float* F32, double* out0, const Geom& G,
                          const Coef3& C, const RefLev& R, cudaStream_t s);
long long rhs_perm_size(const Geom& G);
void build_rhs_perm(const Geom& G, int* out);
// The thread order is built one row of tiles at a time (tiles of 4N x 4N node columns, the
// last row taking the end node): off[r] is the first entry of tile row r, whose node rows
// start at y0[r]; off and y0 end with the total and nyg.  A run of whole tile rows is one
// contiguous range of the order.
void rhs_perm_rows(const Geom& G, std::vector<long long>& off, std::vector<int>& y0);

// column.cu
cudaError_t launch_factor(const Geom& G, const RefLev& R, double lam, Factors F,
                          unsigned* status, cudaStream_t s);
// T: columns per CTA (one thread each; a multiple of 32).  R1, R2: float arrays when
// r_float (the mixed form's internal tendencies), else double arrays.
// status: device status word; the FP64 solve stages its factor stream with bulk copies
// only when it is given (a bounded wait that gives up latches NUMA_ST_TIMEOUT there).
cudaError_t launch_solve(const double* b, double* x, const Geom& G, Factors F, const RefLev& R,
                         const StageTab& tb, int T, cudaStream_t s, unsigned* status = nullptr);
// stage i in {2, 3, 4} reads R1..R(i-1) and q2..q(i-1); stage 4 (four-stage schemes) is
// FP64 Schur form only and takes R3, q3.  Pp_out (FP64 Schur form only; NULL to skip)
// receives P'(q(i)), the equation-of-state pre-pass of the next right-hand side.
cudaError_t launch_stage(int stage, const double* qn, const void* R1, const void* R2,
                         const double* q2, double* out, const Geom& G, const RefLev& R,
                         Factors F, const StageCoef& sc, const StageTab& tb, int T,
                         bool r_float, cudaStream_t s, const double* R3 = nullptr,
                         const double* q3 = nullptr, double* Pp_out = nullptr);
size_t stage_smem_bytes(int M, int T, bool mixed, int iters);
// The previous stages of stage i of an s-stage scheme (s <= NUMA_MAX_STAGES), read by the
// general form of the fused stage: q(i)_e = qn + sum_k adt[k] R[k] and the shift
// sum_k c[k] q[k], over the terms with nonzero coefficients only (q(1) = qn may appear in
// q[]).  Passed by value as a kernel parameter.
constexpr int kMaxPrev = NUMA_MAX_STAGES - 1;
struct StagePrev {
  const double* qn;
  int nr, nq;
  const double* R[kMaxPrev];
  double adt[kMaxPrev];          // a_ij dt
  const double* q[kMaxPrev];
  double c[kMaxPrev];            // c_ij = (a~_ij - a_ij) / a~_ii
};
// Fused stage of the FP64 Schur form for any number of previous stages.  Pp_out as for
// launch_stage.
cudaError_t launch_stage_general(const StagePrev& P, double* out, const Geom& G, const RefLev& R,
                                 const Factors& F, const StageTab& tb, int T, cudaStream_t s,
                                 double* Pp_out);
// Per-order entry points of launch_stage and launch_stage_general (column_stage_nN.cu).
#define NUMA_STAGE_ORDER_SIG(n)                                                                  \
  cudaError_t launch_stage_order##n(int stage, const double* qn, const void* R1, const void* R2, \
                                    const double* q2, double* out, const Geom& G,                \
                                    const RefLev& R, const Factors& F, const StageCoef& sc,      \
                                    const StageTab& tb, int T, bool r_float, cudaStream_t s,     \
                                    const double* R3, const double* q3, double* Pp_out)
#define NUMA_STAGE_GENERAL_ORDER_SIG(n)                                                          \
  cudaError_t launch_stage_general_order##n(const StagePrev& P, double* out, const Geom& G,      \
                                            const RefLev& R, const Factors& F,                   \
                                            const StageTab& tb, int T, cudaStream_t s,           \
                                            double* Pp_out)

NUMA_STAGE_ORDER_SIG(1); NUMA_STAGE_ORDER_SIG(2); NUMA_STAGE_ORDER_SIG(3); NUMA_STAGE_ORDER_SIG(4);
NUMA_STAGE_ORDER_SIG(5); NUMA_STAGE_ORDER_SIG(6); NUMA_STAGE_ORDER_SIG(7); NUMA_STAGE_ORDER_SIG(8);
NUMA_STAGE_GENERAL_ORDER_SIG(1); NUMA_STAGE_GENERAL_ORDER_SIG(2); NUMA_STAGE_GENERAL_ORDER_SIG(3);
NUMA_STAGE_GENERAL_ORDER_SIG(4); NUMA_STAGE_GENERAL_ORDER_SIG(5); NUMA_STAGE_GENERAL_ORDER_SIG(6);
NUMA_STAGE_GENERAL_ORDER_SIG(7); NUMA_STAGE_GENERAL_ORDER_SIG(8);
// out = qn + sum_k bdt[k] R[k] (k < n; in place on qn allowed); a value that is not finite
// latches NUMA_ST_NONFINITE into status (NULL: no check).
struct StageSum {
  int n;
  const double* R[NUMA_MAX_STAGES];
  double bdt[NUMA_MAX_STAGES];
};
cudaError_t launch_ark_combine(const double* qn, const StageSum& S, double* out, long long n,
                               unsigned* status, cudaStream_t s);

// misc.cu
cudaError_t launch_connectivity(const Geom& G, int32_t* l2g, int32_t* g2l, cudaStream_t s);
cudaError_t launch_count_nonfinite(const double* x, long long n, unsigned long long* count,
                                   cudaStream_t s);
cudaError_t launch_ark_final(const double* qn, const double* R1, const double* R2,
                             const double* R3, double* out, long long n, double b1dt,
                             double b2dt, double b3dt, cudaStream_t s);

// ---- index helpers shared by every kernel (the DSS indexing) ---------------------------
// Along one axis with nel elements of order N, global node index idx in [0, nel*N]:
// element e and local index i with idx = e*N + i, i in [0, N) except the last node
// (e = nel-1, i = N).  An interface node (i == 0 and e > 0) is also local node N of
// element e-1.
__host__ __device__ __forceinline__ void axis_owner(int idx, int N, int nel, int& e, int& i) {
  e = idx / N;
  i = idx - e * N;
  if (e == nel) {
    e = nel - 1;
    i = N;
  }
}

__host__ __device__ __forceinline__ long long global_id(const Geom& G, int ix, int iy, int iz) {
  return ((long long)iy * G.nxg + ix) * G.M + iz;
}
