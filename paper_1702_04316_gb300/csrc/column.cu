// Column kernels of the 1D-IMEX method: factorisation of the Schur-complement matrix and
// the column solve, for the FP64 method and for the mixed-precision form (FP32 factors with
// FP64 iterative refinement); the dispatch of the fused implicit stage, whose kernels
// (column_stage.cuh) are compiled one polynomial order per translation unit
// (column_stage_n1.cu .. column_stage_n8.cu).
//
// One thread owns one column (lane-per-column).  On GB300 the FP64 pipe is the scarce
// resource (2 FP64 FMA per clock per SM, 1/64 of FP32), so every lane of a warp does
// useful FP64 work instead of cooperating on one column with shuffles.  The stored
// factors are transposed (column index fastest) so that the 32 lanes of a warp read
// contiguous factor entries, and the state columns are staged through shared memory so
// that their global loads and stores stay coalesced.
//
// The substitutions are right-looking: once y_i (x_i) is known, the next 2N rows are
// updated with 2N independent FMAs held in a register window, so the dependent path per
// row is one FMA and the factors are read by column (the layout numa_internal.cuh gives).
#include "numa_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <string>

#include "bulk_copy.cuh"
#include "column_device.cuh"

namespace {
using namespace numa_dev;

// Algorithm 7 (BuildJacobian) for the Schur form, one column per thread: column m of
// S(lam) is the left-hand side applied to the unit vector e_m,
//   w_p = A^-1 lam (D_z e_m / rho0 + g e_m / (G0 rho0))   (zero at the two walls)
//   S e_m = e_m - lam F0z w_p - lam rho0 G0 D_z w_p,
// assembled in FP64 and stored as FT, then Algorithm 9 (LUdecompose): banded LU without
// pivoting, in place, in FT arithmetic.
// Zero the band storage of one column (n unknowns, half-bandwidth hb).
template <typename FT>
__device__ void band_zero(FT* Lf, FT* Uf, int n, int hb, long long col) {
  FT* Lb = Lf + fac_col_base(col, n, hb);
  FT* Ub = Uf + fac_col_base(col, n, hb + 1);
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < hb; ++k) Lb[((long long)i * hb + k) * kFacBlk] = (FT)0;
    for (int k = 0; k <= hb; ++k) Ub[((long long)i * (hb + 1) + k) * kFacBlk] = (FT)0;
  }
}

// Algorithm 9 (LUdecompose): banded LU without pivoting of one column's n x n matrix, in
// place in FT arithmetic; the diagonal of U is stored inverted (the solves multiply).  A
// zero or non-finite pivot latches NUMA_ST_PIVOT (and is replaced by 1 so the column stays
// finite).
template <typename FT>
__device__ void band_lu(const Band<FT>& A, int n, int hb, unsigned* status) {
  for (int k = 0; k < n; ++k) {
    FT piv = A.at(k, k);
    if (!(fabs((double)piv) > 0.0) || !isfinite((double)piv)) {
      atomicOr(status, NUMA_ST_PIVOT);
      piv = (FT)1;
    }
    const FT ip = (FT)1 / piv;
    const int E = min(k + hb, n - 1);
    for (int i = k + 1; i <= E; ++i) {
      const FT l = A.at(i, k) * ip;
      A.at(i, k) = l;
      for (int j = k + 1; j <= E; ++j) A.at(i, j) = fma(-l, A.at(k, j), A.at(i, j));
    }
    A.at(k, k) = ip;
  }
}

// Algorithm 7 (BuildJacobian) for the Schur form, one column per thread: column m of
// S(lam) is the left-hand side applied to the unit vector e_m,
//   w_p = A^-1 lam (D_z e_m / rho0 + g e_m / (G0 rho0))   (zero at the two walls)
//   S e_m = e_m - lam F0z w_p - lam rho0 G0 D_z w_p,
// assembled in FP64 and stored as FT, then Algorithm 9 (band_lu) in FT arithmetic.
template <typename FT>
__global__ void k_factor(Geom G, RefLev R, double lam, FT* Lf, FT* Uf, int hb, unsigned* status) {
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (col >= G.ncol) return;
  const int M = G.M, N = G.N, W = 2 * N + 1;
  Band<FT> A(Lf, Uf, hb, M, col);
  band_zero(Lf, Uf, M, hb, col);
  auto dz = [&](int l, int j) -> double {   // D_z(l, j), |l - j| <= N
    return __ldg(R.dz_band + (long long)l * W + (j - l + N));
  };
  double wp[2 * NUMA_MAXN + 1];
  for (int m = 0; m < M; ++m) {
    const int l0 = max(0, m - N), l1 = min(M - 1, m + N);
    for (int l = l0; l <= l1; ++l) {
      double val = dz(l, m) * R.inv_rho0[l];
      if (l == m) val += NUMA_GRAV / (R.G0[l] * R.rho0[l]);
      const double Ainv = 1.0 / (1.0 + lam * lam * NUMA_GRAV * R.dtheta0[l] * R.inv_theta0[l]);
      wp[l - m + N] = (l == 0 || l == M - 1) ? 0.0 : lam * Ainv * val;
    }
    const int i0 = max(0, m - 2 * N), i1 = min(M - 1, m + 2 * N);
    for (int i = i0; i <= i1; ++i) {
      double s = (i == m) ? 1.0 : 0.0;
      if (i >= l0 && i <= l1) s -= lam * R.F0z[i] * wp[i - m + N];
      double acc = 0.0;
      const int la = max(max(0, i - N), l0), lb = min(min(M - 1, i + N), l1);
      for (int l = la; l <= lb; ++l) acc = fma(dz(i, l), wp[l - m + N], acc);
      s -= lam * R.rho0[i] * R.G0[i] * acc;
      A.at(i, m) = (FT)s;
    }
  }
  band_lu(A, M, hb, status);
}

// Entry (i, m) of the standard column system I - lam L_V (the non-Schur form), unknowns
// ordered level by level: unknown 3 l + v is variable v (0 rho', 1 w, 2 theta') at level l.
//   rho' rows:   rho' + lam (d(rho0)/dz w + rho0 D_z w)
//   w rows:      w + lam (D_z (G0 rho' + H0 theta') + g rho') / rho0   (w = 0 at the walls)
//   theta' rows: theta' + lam d(theta0)/dz w
__device__ double standard_entry(int i, int m, const Geom& G, const RefLev& R, double lam) {
  const int N = G.N, M = G.M, W = 2 * N + 1;
  const int li = i / 3, a = i - 3 * li, lj = m / 3, b = m - 3 * lj;
  if (abs(li - lj) > N) return 0.0;
  const bool same = li == lj;
  const double dz = __ldg(R.dz_band + (long long)li * W + (lj - li + N));
  if (a == 0) {
    if (b == 0) return same ? 1.0 : 0.0;
    if (b == 1) return lam * ((same ? R.drho0[li] : 0.0) + R.rho0[li] * dz);
    return 0.0;
  }
  if (a == 1) {
    if (li == 0 || li == M - 1) return (b == 1 && same) ? 1.0 : 0.0;
    if (b == 0) return lam * (dz * R.G0[lj] + (same ? NUMA_GRAV : 0.0)) * R.inv_rho0[li];
    if (b == 1) return same ? 1.0 : 0.0;
    return lam * dz * R.H0[lj] * R.inv_rho0[li];
  }
  if (b == 1) return same ? lam * R.dtheta0[li] : 0.0;
  return (b == 2 && same) ? 1.0 : 0.0;
}

// Standard form: assemble the 3M x 3M band (half-bandwidth hb = 3N + 1) of one column per
// thread and factor it with band_lu.
__global__ void k_factor_standard(Geom G, RefLev R, double lam, double* Lf, double* Uf, int hb,
                                  unsigned* status) {
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (col >= G.ncol) return;
  const int n = 3 * G.M;
  Band<double> A(Lf, Uf, hb, n, col);
  band_zero(Lf, Uf, n, hb, col);
  for (int m = 0; m < n; ++m)
    for (int i = max(0, m - hb); i <= min(n - 1, m + hb); ++i)
      A.at(i, m) = standard_entry(i, m, G, R, lam);
  band_lu(A, n, hb, status);
}

template <int N, bool MIXED>
__global__ void k_solve(const double* b, double* x, Geom G, Factors F, RefLev R, StageTab tb,
                        int iters) {
  extern __shared__ double sm[];
  const int T = blockDim.x, M = G.M;
  const long long col0 = blockIdx.x * (long long)T;
  const int ncols = (int)min((long long)T, G.ncol - col0);
  const long long base = col0 * M;
  const int cnt = ncols * M;
  double* Sb = sm;
  for (int j = threadIdx.x; j < cnt; j += T) {
    const int c = j / M, lev = j - c * M;
    Sb[lev * T + c] = b[base + j];
  }
  __syncthreads();
  if ((int)threadIdx.x < ncols) {
    const int t = threadIdx.x;
    if constexpr (MIXED) {
      // scratch columns of the refinement (the FP64 solve allocates only Sb)
      double* St = sm + M * T;
      double* Sx = sm + 2 * M * T;                              // only when iters >= 2
      float* Tf = (float*)(sm + (iters >= 2 ? 3 : 2) * M * T);
      float* Td = Tf + M * T;
      col_solve_refined<N, MIXED>(Sb + t, St + t, Tf + t, Td + t, Sx + t, T, M, F, col0 + t, R,
                                  tb, iters);
    } else {
      // the factor stream is this kernel's time: prefetch two factor columns ahead
      col_solve<2 * N, double, double, 3>(Sb + t, T, M, F.L, F.U, col0 + t);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < cnt; j += T) {
    const int c = j / M, lev = j - c * M;
    x[base + j] = Sb[lev * T + c];
  }
}

// The stand-alone FP64 column solve with its memory traffic on the TMA engine.
// One warp owns one block of kFacBlk = 32 consecutive mesh columns, one lane per column.
// * The block's right-hand side, 32 M contiguous doubles, arrives by one bulk copy and
//   stays in shared memory in its global layout (lane c reads level i at c M + i: an odd M
//   gives no bank conflicts); the solution leaves by one bulk store, in place.
// * The block's factors are one contiguous stream: M rows of L (hb slots x 32 columns, read
//   front to back), then M rows of U (hb + 1 slots, back to front).  Each stored row is one
//   chunk, copied into a ring of kSolveStages shared-memory slots of the warp, each
//   completed on its own mbarrier; a slot is refilled with the chunk kSolveStages rows ahead
//   as soon as the warp has read it into registers.
// A short ring leaves room for more warps per SM, which is what the FP64 pipe, the other
// bound of this kernel, needs.  The arithmetic is col_solve's, in the same order.
// A bounded wait that gives up latches NUMA_ST_TIMEOUT, drains the warp's copies in flight
// and leaves the block unwritten.  Where b or x is not 16-byte aligned, or the block's byte
// count is not a multiple of 16 (an odd M times an odd column count in the last block),
// plain loads and stores move the block.
// Compile-time tuning: slots per warp ring and warps (blocks) per CTA.  With the envelope's
// shorter copies, three slots and one warp per CTA are fastest on GB300 on the 96 x 96 x 12
// workload: 0.203 ms against 0.219 (two and two), 0.216 (one warp, two slots), 0.241 (two
// warps, three slots) and 0.240 (one warp, four slots).
#ifndef NUMA_SOLVE_STAGES
#define NUMA_SOLVE_STAGES 3
#endif
#ifndef NUMA_SOLVE_MAXW
#define NUMA_SOLVE_MAXW 1
#endif
constexpr int kSolveStages = NUMA_SOLVE_STAGES;   // slots in a warp's ring
constexpr size_t kSmemPerCta = 227 * 1024;           // opt-in shared memory per CTA

// NUMA_SOLVE=regs selects the register-pipelined k_solve for the FP64 stand-alone solve
// (read once per process).
inline bool solve_regs_forced() {
  static const bool f = [] {
    const char* e = std::getenv("NUMA_SOLVE");
    return e && std::string(e) == "regs";
  }();
  return f;
}

__host__ __device__ inline size_t solve_bulk_warp_bytes(int hb, int M) {
  const size_t slots = (size_t)kSolveStages * (hb + 1) * kFacBlk * sizeof(double);
  const size_t xs = (size_t)M * kFacBlk * sizeof(double);
  const size_t bars = (kSolveStages + 1) * sizeof(unsigned long long);
  return (slots + xs + bars + 127) / 128 * 128;
}

template <int N>
__global__ void __launch_bounds__(32 * NUMA_SOLVE_MAXW) k_solve_bulk(
    const double* b, double* x, long long ncol, int M, const double* __restrict__ L,
    const double* __restrict__ U, unsigned* status, int plant_timeout) {
  constexpr int HB = 2 * N;
  constexpr unsigned UROW = (HB + 1) * kFacBlk * sizeof(double);   // a slot holds the longer U row
  constexpr int S = kSolveStages;
  extern __shared__ __align__(128) unsigned char smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long blk = (long long)blockIdx.x * (blockDim.x >> 5) + wid;
  const long long col0 = blk * kFacBlk;
  if (col0 >= ncol) return;                         // whole warp; no CTA-wide sync follows
  unsigned char* base = smem + (size_t)wid * solve_bulk_warp_bytes(HB, M);
  double* xs = (double*)(base + (size_t)S * UROW);  // the block's columns, global layout
  const unsigned slot0 = smem_u32(base);
  const unsigned bar0 = smem_u32(xs + (size_t)M * kFacBlk);  // S ring barriers, then b's
  const unsigned barb = bar0 + 8 * S;
  const double* Lb = L + blk * (long long)M * HB * kFacBlk;
  const double* Ub = U + blk * (long long)M * (HB + 1) * kFacBlk;
  const int nch = 2 * M;
  const int nc = (int)min((long long)kFacBlk, ncol - col0);
  const unsigned bbytes = (unsigned)(nc * M) * sizeof(double);
  const bool bulk_io = (bbytes % 16) == 0 && ((unsigned long long)b % 16) == 0 &&
                       ((unsigned long long)x % 16) == 0;
  const double* bb = b + col0 * M;
  double* xb = x + col0 * M;

  // chunk q < M: row q of L; chunk q >= M: row 2M - 1 - q of U.  Only the slots inside the
  // factors' envelope are copied (a prefix of the stored row: env_l(r) slots of L, the
  // inverted pivot and env_u(r) slots of U, r = level mod N); the rest are exact zeros.
  auto issue = [&](int q) {
    const int s = q % S;
    const bool isL = q < M;
    const int lev = isL ? q : nch - 1 - q;
    const double* src = isL ? Lb + (long long)q * HB * kFacBlk
                            : Ub + (long long)lev * (HB + 1) * kFacBlk;
    const unsigned bytes = (unsigned)(isL ? env_l(N, lev % N) : env_u(N, lev % N) + 1) *
                           kFacBlk * sizeof(double);
    // plant_timeout (tests only): the first row's barrier expects 16 bytes more than arrive
    mbar_arrive_expect_tx(bar0 + 8 * s, bytes + ((plant_timeout && q == 0) ? 16u : 0u));
    bulk_g2s(slot0 + s * UROW, src, bytes, bar0 + 8 * s);
  };
  if (lane == 0) {
    for (int s = 0; s <= S; ++s) mbar_init(bar0 + 8 * s, 1);
    fence_proxy_async_smem();
    if (bulk_io) {
      mbar_arrive_expect_tx(barb, bbytes);
      bulk_g2s(smem_u32(xs), bb, bbytes, barb);
    }
    for (int q = 0; q < S && q < nch; ++q) issue(q);
  }
  // on a timeout: latch the status and drain this warp's copies in flight (chunks q0 ..
  // q0 + S - 1, and b's when it was still pending)
  auto give_up = [&](int q0, bool b_pending) {
    if (lane == 0) {
      atomicOr(status, NUMA_ST_TIMEOUT);
      if (b_pending) mbar_wait_bounded(barb, 0);
      for (int r = q0; r < q0 + S && r < nch; ++r) mbar_wait_bounded(bar0 + 8 * (r % S), (r / S) & 1);
    }
    __syncwarp();
  };
  if (bulk_io) {
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(barb, 0))) {
      give_up(0, true);
      return;
    }
  } else {
    for (int j = lane; j < nc * M; j += 32) xs[j] = bb[j];
    __syncwarp();
  }
  double* xc = xs + lane * M;                       // this lane's column

  int q = 0;
  auto acquire = [&]() -> const double* {
    const int s = q % S;
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar0 + 8 * s, (q / S) & 1))) {
      give_up(q, false);
      return nullptr;
    }
    return (const double*)(base + (size_t)s * UROW) + lane;
  };
  // the slot just read is refilled: every lane orders its reads of it before the bulk copy
  // (async proxy) that overwrites it, the warp synchronises, lane 0 issues the copy
  auto release = [&]() {
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0 && q + S < nch) issue(q + S);
    ++q;
  };

  // forward: y_i = w_0; w_k <- w_{k+1} - L(i+1+k, i) y_i for the env_l(r) slots of the
  // envelope, a shift beyond (levels in blocks of N: r is a compile-time constant)
  double w[HB];
#pragma unroll
  for (int k = 0; k < HB; ++k) w[k] = (k < M) ? xc[k] : 0.0;
  bool ok = true;
  for (int i0 = 0; i0 < M && ok; i0 += N) {
    static_for<N>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      constexpr int nl = env_l(N, r);
      const int i = i0 + r;
      if (!ok || i >= M) return;
      const double* sl = acquire();
      if (!sl) {
        ok = false;
        return;
      }
      double l[HB];
#pragma unroll
      for (int k = 0; k < nl; ++k) l[k] = sl[k * kFacBlk];
      release();
      const double y = w[0];
      const double nxt = (i + HB < M) ? xc[i + HB] : 0.0;
      xc[i] = y;
#pragma unroll
      for (int k = 0; k < HB - 1; ++k) w[k] = (k < nl) ? fma(-l[k], y, w[k + 1]) : w[k + 1];
      w[HB - 1] = (HB - 1 < nl) ? fma(-l[HB - 1], y, nxt) : nxt;
    });
  }
  if (!ok) return;
  // backward: x_i = v_0 / U(i,i); v_k <- v_{k+1} - U(i-1-k, i) x_i for the env_u(r) slots;
  // level i = M - 1 - (t0 + s) with t0 a multiple of N and M - 1 = nez N, so r = (N - s) mod N
  double v[HB];
#pragma unroll
  for (int k = 0; k < HB; ++k) v[k] = (M - 1 - k >= 0) ? xc[M - 1 - k] : 0.0;
  for (int t0 = 0; t0 < M && ok; t0 += N) {
    static_for<N>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr int nu = env_u(N, (N - s) % N);
      const int i = M - 1 - (t0 + s);
      if (!ok || i < 0) return;
      const double* su = acquire();
      if (!su) {
        ok = false;
        return;
      }
      double u[HB + 1];
#pragma unroll
      for (int k = 0; k <= nu; ++k) u[k] = su[k * kFacBlk];
      release();
      const double xi = v[0] * u[0];
      xc[i] = xi;
      const double nxt = (i - HB >= 0) ? xc[i - HB] : 0.0;
#pragma unroll
      for (int k = 0; k < HB - 1; ++k) v[k] = (k < nu) ? fma(-u[k + 1], xi, v[k + 1]) : v[k + 1];
      v[HB - 1] = (HB - 1 < nu) ? fma(-u[HB], xi, nxt) : nxt;
    });
  }
  if (!ok) return;
  __syncwarp();
  if (bulk_io) {
    if (lane == 0) {
      fence_proxy_async_smem();                     // the lanes' writes, before the store reads
      bulk_s2g(xb, smem_u32(xs), bbytes);
      bulk_commit();
      bulk_wait_read_all();
    }
  } else {
    for (int j = lane; j < nc * M; j += 32) xb[j] = xs[j];
  }
}

// Warps (32-column blocks) per CTA of k_solve_bulk for M levels at order N; 0 when one
// warp's slots and column do not fit in shared memory (the register-pipelined k_solve runs).
inline int solve_bulk_warps(int N, int M) {
  const size_t wb = solve_bulk_warp_bytes(2 * N, M);
  if (wb > kSmemPerCta) return 0;
  return (int)std::min<size_t>(NUMA_SOLVE_MAXW, kSmemPerCta / wb);
}

template <int N, bool MIXED>
cudaError_t launch_solve_n(const double* b, double* x, const Geom& G, const Factors& F,
                           const RefLev& R, const StageTab& tb, int T, int iters,
                           unsigned* status, cudaStream_t s) {
  if constexpr (!MIXED) {
    const int nw = solve_bulk_warps(N, G.M);
    if (nw > 0 && status && !solve_regs_forced()) {
      const size_t smem = solve_bulk_warp_bytes(2 * N, G.M) * nw;
      cudaError_t e = cudaFuncSetAttribute(k_solve_bulk<N>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const long long nblk = (G.ncol + kFacBlk - 1) / kFacBlk;
      // NUMA_TEST_SOLVE_TIMEOUT=1 (read at every call; tests only) makes the first wait of
      // every warp run out, to exercise the timeout path without a fault
      const char* pt = std::getenv("NUMA_TEST_SOLVE_TIMEOUT");
      const int plant = (pt && std::string(pt) == "1") ? 1 : 0;
      k_solve_bulk<N><<<(unsigned)((nblk + nw - 1) / nw), 32 * nw, smem, s>>>(
          b, x, G.ncol, G.M, F.L, F.U, status, plant);
      return cudaGetLastError();
    }
  }
  // the FP64 solve uses only the right-hand-side column (more resident columns per SM)
  const size_t smem = (MIXED ? col_smem_per_level(MIXED, iters) : sizeof(double)) * G.M * T;
  cudaError_t e = cudaFuncSetAttribute(k_solve<N, MIXED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_solve<N, MIXED><<<(unsigned)((G.ncol + T - 1) / T), T, smem, s>>>(b, x, G, F, R, tb, iters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_factor(const Geom& G, const RefLev& R, double lam, Factors F,
                          unsigned* status, cudaStream_t s) {
  const int bs = 128;
  const unsigned nb = (unsigned)((G.ncol + bs - 1) / bs);
  if (F.standard) k_factor_standard<<<nb, bs, 0, s>>>(G, R, lam, F.L, F.U, F.hb, status);
  else if (F.mixed) k_factor<float><<<nb, bs, 0, s>>>(G, R, lam, F.L32, F.U32, F.hb, status);
  else k_factor<double><<<nb, bs, 0, s>>>(G, R, lam, F.L, F.U, F.hb, status);
  return cudaGetLastError();
}

cudaError_t launch_solve(const double* b, double* x, const Geom& G, Factors F, const RefLev& R,
                         const StageTab& tb, int T, cudaStream_t s, unsigned* status) {
  const int it = F.refine_iters;
#define NUMA_SOLVE_CASE(n)                                                             \
  case n:                                                                              \
    return F.mixed ? launch_solve_n<n, true>(b, x, G, F, R, tb, T, it, status, s)      \
                   : launch_solve_n<n, false>(b, x, G, F, R, tb, T, it, status, s);
  switch (G.N) {
    NUMA_SOLVE_CASE(1) NUMA_SOLVE_CASE(2) NUMA_SOLVE_CASE(3) NUMA_SOLVE_CASE(4)
    NUMA_SOLVE_CASE(5) NUMA_SOLVE_CASE(6) NUMA_SOLVE_CASE(7) NUMA_SOLVE_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef NUMA_SOLVE_CASE
}


size_t stage_smem_bytes(int M, int T, bool mixed, int iters) {
  return col_smem_per_level(mixed, iters) * M * T;
}

cudaError_t launch_stage(int stage, const double* qn, const void* R1, const void* R2,
                         const double* q2, double* out, const Geom& G, const RefLev& R,
                         Factors F, const StageCoef& sc, const StageTab& tb, int T,
                         bool r_float, cudaStream_t s, const double* R3, const double* q3,
                         double* Pp_out) {
#define NUMA_STAGE_CASE(n)                                                                   \
  case n:                                                                                    \
    return launch_stage_order##n(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, r_float, s, \
                                 R3, q3, Pp_out);
  switch (G.N) {
    NUMA_STAGE_CASE(1) NUMA_STAGE_CASE(2) NUMA_STAGE_CASE(3) NUMA_STAGE_CASE(4)
    NUMA_STAGE_CASE(5) NUMA_STAGE_CASE(6) NUMA_STAGE_CASE(7) NUMA_STAGE_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef NUMA_STAGE_CASE
}

cudaError_t launch_stage_general(const StagePrev& P, double* out, const Geom& G, const RefLev& R,
                                 const Factors& F, const StageTab& tb, int T, cudaStream_t s,
                                 double* Pp_out) {
  if (F.standard || F.mixed || !P.qn || P.nr < 0 || P.nr > kMaxPrev || P.nq < 0 ||
      P.nq > kMaxPrev)
    return cudaErrorInvalidValue;
#define NUMA_STAGE_CASE(n) \
  case n: return launch_stage_general_order##n(P, out, G, R, F, tb, T, s, Pp_out);
  switch (G.N) {
    NUMA_STAGE_CASE(1) NUMA_STAGE_CASE(2) NUMA_STAGE_CASE(3) NUMA_STAGE_CASE(4)
    NUMA_STAGE_CASE(5) NUMA_STAGE_CASE(6) NUMA_STAGE_CASE(7) NUMA_STAGE_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef NUMA_STAGE_CASE
}
