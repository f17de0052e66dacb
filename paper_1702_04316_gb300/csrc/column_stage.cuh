// The fused implicit stage of the 1D-IMEX method (Algorithms 4 and 5 with the column solve
// of Algorithm 9 between them; stage_body in column_device.cuh holds the per-column work):
// the kernels and their launchers, templated on the polynomial order N.  Each order is
// compiled in its own translation unit (column_stage_nN.cu), which defines
// launch_stage_orderN and launch_stage_general_orderN; column.cu dispatches on G.N.
#pragma once
#include <algorithm>
#include <cstdlib>

#include "column_device.cuh"
#include "numa_internal.cuh"

namespace {
using namespace numa_dev;

// NP previous stages (see stage_body); R3 and q3 are read only when NP = 3.
template <int N, int NP, bool MIXED, typename RT>
__device__ __forceinline__ void stage_kernel(const double* __restrict__ qn, const RT* __restrict__ R1,
                                             const RT* __restrict__ R2, const double* __restrict__ q2,
                                             double* __restrict__ out, const Geom& G, const RefLev& R,
                                             const Factors& F, const StageCoef& sc, const StageTab& tb,
                                             int iters, int T, const RT* __restrict__ R3,
                                             const double* __restrict__ q3, double* __restrict__ Pp_out,
                                             const EosSeries& eos) {
  extern __shared__ double sm[];
  stage_body<N, NP, MIXED, RT>(blockIdx.x * (long long)T, T, sm, qn, R1, R2, q2, out, G, R, F, sc,
                               tb, iters, R3, q3, Pp_out, &eos);
}

#define NUMA_STAGE_PARAMS                                                                       \
  const double *__restrict__ qn, const RT *__restrict__ R1, const RT *__restrict__ R2,           \
      const double *__restrict__ q2, double *__restrict__ out, Geom G, RefLev R, Factors F,      \
      StageCoef sc, StageTab tb, int iters, int T, const RT *__restrict__ R3,                    \
      const double *__restrict__ q3, double *__restrict__ Pp_out, EosSeries eos
#define NUMA_STAGE_ARGS qn, R1, R2, q2, out, G, R, F, sc, tb, iters, T, R3, q3, Pp_out, eos

// Register bounds of the fused stage.  N = 4: at most 64 registers a thread (written as a
// bound of 1024 threads a CTA, so any thread count stays launchable), so 32 warps fit on an
// SM (eight 128-thread CTAs of 32 columns), as their shared memory also allows.  Other orders:
// three 256-thread CTAs per SM (at most 85 registers; a few hundred bytes of spill at
// N = 7, 8).  On the 64 x 64 x 10, N = 7 workload this beat both the compiler's own choice
// (94-100 registers, two CTAs) and a 64-register cap: 18.1 against 19.3 and 18.7 ms per FP64
// step, 8.9 against 10.1 and 9.4 ms with the FP32 right-hand side.
template <int N, int NP, bool MIXED, typename RT>
__global__ void __launch_bounds__(1024) k_stage4(NUMA_STAGE_PARAMS) {
  stage_kernel<N, NP, MIXED, RT>(NUMA_STAGE_ARGS);
}
template <int N, int NP, bool MIXED, typename RT>
__global__ void __launch_bounds__(256, 3) k_stage(NUMA_STAGE_PARAMS) {
  stage_kernel<N, NP, MIXED, RT>(NUMA_STAGE_ARGS);
}

// Any stage of an s-stage scheme: the previous stages listed in P (FP64 Schur form); the
// N = 4 variant has the 64-register bound of k_stage4.
template <int N>
__device__ __forceinline__ void stage_general_kernel(const StagePrev& P, double* __restrict__ out,
                                                     const Geom& G, const RefLev& R,
                                                     const Factors& F, const StageTab& tb, int T,
                                                     double* __restrict__ Pp_out,
                                                     const EosSeries& eos) {
  extern __shared__ double sm[];
  StageCoef sc{};
  stage_body<N, 0, false, double>(blockIdx.x * (long long)T, T, sm, P.qn, nullptr, nullptr,
                                  nullptr, out, G, R, F, sc, tb, 0, nullptr, nullptr, Pp_out,
                                  &eos, &P);
}
template <int N>
__global__ void __launch_bounds__(1024) k_stage_general4(const __grid_constant__ StagePrev P,
                                                         double* __restrict__ out, Geom G, RefLev R,
                                                         Factors F, StageTab tb, int T,
                                                         double* __restrict__ Pp_out, EosSeries eos) {
  stage_general_kernel<N>(P, out, G, R, F, tb, T, Pp_out, eos);
}
template <int N>
__global__ void k_stage_general(const __grid_constant__ StagePrev P, double* __restrict__ out,
                                Geom G, RefLev R, Factors F, StageTab tb, int T,
                                double* __restrict__ Pp_out, EosSeries eos) {
  stage_general_kernel<N>(P, out, G, R, F, tb, T, Pp_out, eos);
}

// Fused stage with the standard column system (rows 2 or 3 of Table 1).  Phase 1: the
// predictor and the shift q~_e (u, v final), with (rho~_e, w~_e, theta~_e) stored level by
// level in shared memory (3M values per column; w~_e = 0 at the walls, the wall condition).
// Phase 2 (one thread per column): the banded solve with half-bandwidth 3N + 1.  Phase 3:
// q(i) = q~ - sum_j c_ij q(j).  T columns per CTA, blockDim.x >= T threads.
template <int N, bool S3>
__global__ void k_stage_standard(const double* __restrict__ qn, const double* __restrict__ R1,
                                 const double* __restrict__ R2, const double* __restrict__ q2,
                                 double* __restrict__ out, Geom G, Factors F, StageCoef sc, int T) {
  extern __shared__ double sm[];
  const int NT = blockDim.x, M = G.M;
  const long long nn = G.nnode;
  const long long col0 = blockIdx.x * (long long)T;
  const int ncols = (int)min((long long)T, G.ncol - col0);
  const long long base = col0 * M;
  const int cnt = ncols * M;
  const double a1dt = sc.a[0] * sc.dt, a2dt = sc.a[1] * sc.dt;
  const double c1 = sc.c[0], c2 = sc.c[1];
  auto pred = [&](int f, long long o) -> double {
    const double qv = qn[o];
    double v = fma(a1dt, R1[o], qv);
    if (S3) v = fma(a2dt, R2[o], v);
    if (f == 1 || f == 2) return v;
    v = fma(c1, qv, v);
    if (S3) v = fma(c2, q2[o], v);
    return v;
  };
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
    out[nn + g] = pred(1, nn + g);
    out[2 * nn + g] = pred(2, 2 * nn + g);
    sm[(3 * lev) * T + c] = pred(0, g);
    sm[(3 * lev + 1) * T + c] = (lev == 0 || lev == M - 1) ? 0.0 : pred(3, 3 * nn + g);
    sm[(3 * lev + 2) * T + c] = pred(4, 4 * nn + g);
  }
  __syncthreads();
  if ((int)threadIdx.x < ncols)
    col_solve<3 * N + 1, double, double>(sm + threadIdx.x, T, 3 * M, F.L, F.U,
                                         col0 + threadIdx.x);
  __syncthreads();
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
    const int fl[3] = {0, 3, 4};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long o = fl[k] * nn + g;
      double v = fma(-c1, qn[o], sm[(3 * lev + k) * T + c]);
      if (S3) v = fma(-c2, q2[o], v);
      out[o] = v;
    }
  }
}

size_t stage_smem(int M, int T, bool mixed, int iters) {
  return col_smem_per_level(mixed, iters) * M * T;
}

// Threads per CTA of the fused stage for T columns.  The coalesced phases and the
// level-parallel steps of the column phase share them; only the substitutions run one thread
// per column.  Per column: four for the FP64 stage, six for the mixed form's (its refinement
// adds level-parallel FP64 residual steps), eight when the grid has fewer than two CTAs per
// SM (small meshes); at least T, at most `limit` (the kernel's bound).  On the 96 x 96 x 12,
// N = 4 workload, T = 32 columns with 128 threads took the FP64 stage from 0.908 ms (64
// columns, 256 threads) to 0.892 ms and the rhs32 stage from 0.808 to 0.788 ms; the mixed
// stage went from 1.43 to 1.27 ms with 192 threads (1.37 with 128).  Fewer, larger CTAs
// (64 or 128 columns) and fewer threads per column (2 or 3) were slower.
// NUMA_STAGE_THREADS (a multiple of 32, at least T; clamped to `limit`) overrides, for tuning.
int stage_threads(int T, long long ncol, bool mixed, int limit = 1024) {
  static int env = -1;
  static int nsm = 0;
  if (env < 0) {
    env = 0;
    if (const char* t = std::getenv("NUMA_STAGE_THREADS")) {
      const int v = std::atoi(t);
      if (v >= 32 && v <= 1024 && v % 32 == 0) env = v;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  if (env >= T) return std::max(T, std::min(limit, env));
  const long long nblocks = (ncol + T - 1) / T;
  const int per_col = nblocks < 2LL * nsm ? 8 : (mixed ? 6 : 4);
  return std::max(T, std::min(limit, per_col * T));
}

template <int N, int NP, bool MIXED, typename RT>
cudaError_t launch_stage_k(const double* qn, const RT* R1, const RT* R2, const double* q2,
                           double* out, const Geom& G, const RefLev& R, const Factors& F,
                           const StageCoef& sc, const StageTab& tb, int T, int iters,
                           cudaStream_t s, const RT* R3 = nullptr, const double* q3 = nullptr,
                           double* Pp_out = nullptr) {
  const size_t smem = stage_smem(G.M, T, MIXED, iters);
  const auto launch = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((G.ncol + T - 1) / T), stage_threads(T, G.ncol, MIXED, N == 4 ? 1024 : 256),
           smem, s>>>(qn, R1, R2, q2, out, G, R, F, sc, tb, iters, T, R3, q3, Pp_out, eos_series());
    return cudaGetLastError();
  };
  if constexpr (N == 4) return launch(k_stage4<N, NP, MIXED, RT>);
  else return launch(k_stage<N, NP, MIXED, RT>);
}

template <int N>
cudaError_t launch_stage_n(int stage, const double* qn, const void* R1, const void* R2,
                           const double* q2, double* out, const Geom& G, const RefLev& R,
                           const Factors& F, const StageCoef& sc, const StageTab& tb, int T,
                           bool r_float, cudaStream_t s, const double* R3, const double* q3,
                           double* Pp_out) {
  const int it = F.refine_iters;
  if (stage == 4) {     // four-stage schemes: FP64 Schur form only
    if (F.standard || F.mixed || !R3 || !q3) return cudaErrorInvalidValue;
    return launch_stage_k<N, 3, false>(qn, (const double*)R1, (const double*)R2, q2, out, G, R, F,
                                       sc, tb, T, it, s, R3, q3, Pp_out);
  }
  if (Pp_out && (F.standard || F.mixed)) return cudaErrorInvalidValue;
  if (F.standard) {
    const size_t smem = (size_t)3 * G.M * T * sizeof(double);
    const unsigned nb = (unsigned)((G.ncol + T - 1) / T);
    const double* a = (const double*)R1;
    const double* b = (const double*)R2;
    cudaError_t e;
    if (stage == 3) {
      e = cudaFuncSetAttribute(k_stage_standard<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_stage_standard<N, true><<<nb, stage_threads(T, G.ncol, false, 512), smem, s>>>(qn, a, b, q2, out, G, F, sc, T);
    } else {
      e = cudaFuncSetAttribute(k_stage_standard<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_stage_standard<N, false><<<nb, stage_threads(T, G.ncol, false, 512), smem, s>>>(qn, a, b, q2, out, G, F, sc, T);
    }
    return cudaGetLastError();
  }
  if (F.mixed && !r_float) {
    const double* a = (const double*)R1;
    const double* b = (const double*)R2;
    return stage == 3 ? launch_stage_k<N, 2, true>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s)
                      : launch_stage_k<N, 1, true>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s);
  }
  if (F.mixed) {
    const float* a = (const float*)R1;
    const float* b = (const float*)R2;
    return stage == 3 ? launch_stage_k<N, 2, true>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s)
                      : launch_stage_k<N, 1, true>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s);
  }
  if (r_float) {         // FP32 tendencies with FP64 factors (NUMA_PREC_RHS32)
    const float* a = (const float*)R1;
    const float* b = (const float*)R2;
    return stage == 3 ? launch_stage_k<N, 2, false>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s)
                      : launch_stage_k<N, 1, false>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s);
  }
  const double* a = (const double*)R1;
  const double* b = (const double*)R2;
  return stage == 3 ? launch_stage_k<N, 2, false, double>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s,
                                                  nullptr, nullptr, Pp_out)
                    : launch_stage_k<N, 1, false, double>(qn, a, b, q2, out, G, R, F, sc, tb, T, it, s,
                                                  nullptr, nullptr, Pp_out);
}


// Any stage of an s-stage scheme at order N (launch_stage_general checks its arguments).
template <int N>
cudaError_t launch_stage_general_n(const StagePrev& P, double* out, const Geom& G,
                                   const RefLev& R, const Factors& F, const StageTab& tb, int T,
                                   cudaStream_t s, double* Pp_out) {
  const size_t smem = stage_smem(G.M, T, false, 0);
  const unsigned nb = (unsigned)((G.ncol + T - 1) / T);
  const auto launch = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<nb, stage_threads(T, G.ncol, false, N == 4 ? 1024 : 256), smem, s>>>(P, out, G, R, F, tb, T,
                                                                            Pp_out, eos_series());
    return cudaGetLastError();
  };
  if constexpr (N == 4) return launch(k_stage_general4<N>);
  else return launch(k_stage_general<N>);
}

}  // namespace

// The definitions of one order's two entry points (used once per order, in its own file).
#define NUMA_STAGE_ORDER_DEFINE(n)                                                             \
  NUMA_STAGE_ORDER_SIG(n) {                                                                    \
    return launch_stage_n<n>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, r_float, s, R3, q3, \
                             Pp_out);                                                          \
  }                                                                                            \
  NUMA_STAGE_GENERAL_ORDER_SIG(n) {                                                            \
    return launch_stage_general_n<n>(P, out, G, R, F, tb, T, s, Pp_out);                       \
  }
