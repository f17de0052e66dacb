// Device code of the column kernels (factor, solve, fused stage), shared by the
// single-mesh kernels (column.cu, column_stage.cuh) and the persistent ensemble kernels (batch.cu).
// See column.cu for the method.
#pragma once
#include "numa_internal.cuh"
#include "rhs_device.cuh"

#include <type_traits>
#include <utility>

namespace numa_dev {


// ---- band accessor of the stored factors (column-oriented layout) ----------------------
// Entry (i, j) of one column's n x n band matrix: L(i, j), j < i, in slot i - j - 1 of stored
// row j of L; U(i, j), j >= i, in slot j - i of stored row j of U (rows by matrix column).
template <typename FT>
struct Band {
  FT* L;        // L + fac_col_base(col, n, hb)
  FT* U;        // U + fac_col_base(col, n, hb + 1)
  int hb;
  __device__ Band(FT* Lf, FT* Uf, int hb_, int n, long long col)
      : L(Lf + fac_col_base(col, n, hb_)), U(Uf + fac_col_base(col, n, hb_ + 1)), hb(hb_) {}
  __device__ __forceinline__ FT& at(int i, int j) const {
    return (j < i) ? L[((long long)j * hb + (i - j) - 1) * kFacBlk]
                   : U[((long long)j * (hb + 1) + (j - i)) * kFacBlk];
  }
};

// ---- nonzero envelope of the Schur-form factors -------------------------------------------
// S(lam) has the sparsity of D_z^2.  A level inside an element (i = e N + r, 0 < r < N)
// couples to the levels (e-1) N .. (e+2) N, an element interface (r = 0) to (e-2) N ..
// (e+2) N.  The pattern is symmetric and a no-pivot LU keeps its fill inside this envelope,
// so column i of L has env_l(r) entries below the diagonal and column i of U env_u(r) above
// it; every stored band entry beyond them is an exact zero, and skipping it leaves the
// substitutions' results unchanged.
__host__ __device__ constexpr int env_l(int N, int r) { return r == 0 ? 2 * N : 2 * N - r; }
__host__ __device__ constexpr int env_u(int N, int r) { return r == 0 ? 2 * N : N + r; }

// f(integral_constant<int, 0>) .. f(integral_constant<int, K - 1>), in order.
template <typename F, int... Rs>
__device__ __forceinline__ void static_for_seq(F&& f, std::integer_sequence<int, Rs...>) {
  (f(std::integral_constant<int, Rs>{}), ...);
}
template <int K, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_seq(f, std::make_integer_sequence<int, K>{});
}

// acc + s (k D_z f)[lev] for a column held in shared memory with stride T between levels,
// with the scaled taps kc = k dz_c of a StageTab (dzD or dzP) and s = +1 or -1 (NEG): one
// multiply-add per tap, the scale and the sign riding on the taps, into one accumulator
// (FP64 issue, not latency, bounds the column kernels: a warp-wide FP64 multiply-add
// occupies the pipe 16 cycles).  lev is uniform across a warp, so the tap table reads are
// broadcasts and the branch on the tap count (N interior, 2N interface, N+1 wall) does not
// diverge.
template <int N, bool NEG, typename XT>
__device__ __forceinline__ double col_kdz(const XT* f, int T, int lev, const RefLev& R,
                                          const double* kc, double acc) {
  constexpr int W = 2 * N + 1;
  const double* c = kc + (long long)lev * W;
  const int* o = R.dz_o + (long long)lev * W;
  const int n = __ldg(R.dz_n + lev);
  const XT* p = f + lev * T;
  auto tap = [&](int t) { return NEG ? -__ldg(c + t) : __ldg(c + t); };
  if (n == N) {
#pragma unroll
    for (int t = 0; t < N; ++t) acc = fma(tap(t), to_f64(p[__ldg(o + t) * T]), acc);
    return acc;
  }
  if (n == 2 * N) {
#pragma unroll
    for (int t = 0; t < 2 * N; ++t) acc = fma(tap(t), to_f64(p[__ldg(o + t) * T]), acc);
    return acc;
  }
  for (int t = 0; t < n; ++t) acc = fma(tap(t), to_f64(p[__ldg(o + t) * T]), acc);
  return acc;
}

// w_p(x)[lev] = lam A^-1 (D_z x / rho0 + g x / (G0 rho0)), zero at the two walls (the
// tables kp1, kp2 carry the zeros).
template <int N, typename XT>
__device__ __forceinline__ double col_wp(const XT* x, int T, int lev, const RefLev& R,
                                         const StageTab& tb) {
  return col_kdz<N, false, XT>(x, T, lev, R, tb.dzP, __ldg(tb.kp2 + lev) * to_f64(x[lev * T]));
}

// Solve L U x = b in place for one column held in shared memory (stride T), VT the value
// type, FT the factor type.  Forward: y_i = w_0; x_{i+1+k} -= L(i+1+k, i) y_i for k < HB
// (window w in registers).  Backward: x_i = v_0 / U(i,i); y_{i-1-k} -= U(i-1-k, i) x_i.
// NB = 0 (the column kernels that are bound by FP64 issue): the next factor column is
// loaded before the current one is used, one column of work ahead, in two register
// buffers.  NB >= 2 (the standalone solve, whose time is the factor stream): the factor
// columns stream through NB buffers; the level loop is unrolled by NB and each buffer is
// refilled, NB levels ahead, right after its last use, so no pending load is copied from
// buffer to buffer (a copy would wait for it) and each load has NB - 1 levels of work to
// arrive.
// NE = N (Schur-form factors, HB = 2N, NB = 0): the substitutions skip the exact zeros
// outside the factors' envelope (env_l, env_u); the level loop runs in blocks of N levels so
// that each level's entry count is a compile-time constant.  NE = 0: the full band.
template <int HB, typename VT, typename FT, int NB = 0, int NE = 0>
__device__ __forceinline__ void col_solve(VT* x, int T, int M, const FT* __restrict__ L,
                                          const FT* __restrict__ U, long long col) {
  const FT* Lb = L + fac_col_base(col, M, HB);
  const FT* Ub = U + fac_col_base(col, M, HB + 1);
  static_assert(NB == 0 || (NB >= 2 && NB <= 4), "NB = 0 or 2 to 4 factor buffers");
  static_assert(NE == 0 || (NB == 0 && HB == 2 * NE), "the envelope is the Schur form's");
  if constexpr (NE > 0) {
    // forward: y_i = w_0; w_k <- w_{k+1} - L(i+1+k, i) y_i for k < env_l(r), shift beyond
    VT w[HB], ln[HB];
#pragma unroll
    for (int k = 0; k < HB; ++k) w[k] = (k < M) ? x[k * T] : (VT)0;
#pragma unroll
    for (int k = 0; k < env_l(NE, 0); ++k) ln[k] = (VT)__ldg(Lb + (long long)k * kFacBlk);
#pragma unroll 1
    for (int i0 = 0; i0 < M; i0 += NE) {
      static_for<NE>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        constexpr int nl = env_l(NE, r);
        constexpr int nn = env_l(NE, (r + 1) % NE);
        const int i = i0 + r;
        if (i < M) {
          VT l[HB];
#pragma unroll
          for (int k = 0; k < nl; ++k) l[k] = ln[k];
          if (i + 1 < M) {
            const FT* Lc = Lb + (long long)(i + 1) * HB * kFacBlk;
#pragma unroll
            for (int k = 0; k < nn; ++k) ln[k] = (VT)__ldg(Lc + (long long)k * kFacBlk);
          }
          const VT y = w[0];
          x[i * T] = y;
          const VT nxt = (i + HB < M) ? x[(i + HB) * T] : (VT)0;
#pragma unroll
          for (int k = 0; k < HB - 1; ++k) w[k] = (k < nl) ? fma(-l[k], y, w[k + 1]) : w[k + 1];
          w[HB - 1] = (HB - 1 < nl) ? fma(-l[HB - 1], y, nxt) : nxt;
        }
      });
    }
    // backward: x_i = v_0 / U(i,i); v_k <- v_{k+1} - U(i-1-k, i) x_i for k < env_u(r).
    // Level i = M - 1 - t with t = t0 + s, t0 a multiple of N, and M - 1 = nez N, so
    // r = i mod N = (N - s) mod N is a compile-time constant of s.
    VT v[HB], un[HB + 1];
#pragma unroll
    for (int k = 0; k < HB; ++k) v[k] = (M - 1 - k >= 0) ? x[(M - 1 - k) * T] : (VT)0;
    {
      const FT* Uc = Ub + (long long)(M - 1) * (HB + 1) * kFacBlk;
#pragma unroll
      for (int k = 0; k <= env_u(NE, 0); ++k) un[k] = (VT)__ldg(Uc + (long long)k * kFacBlk);
    }
#pragma unroll 1
    for (int t0 = 0; t0 < M; t0 += NE) {
      static_for<NE>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        constexpr int nu = env_u(NE, (NE - s) % NE);
        constexpr int nn = env_u(NE, (NE - (s + 1) % NE) % NE);
        const int i = M - 1 - (t0 + s);
        if (i >= 0) {
          VT u[HB + 1];
#pragma unroll
          for (int k = 0; k <= nu; ++k) u[k] = un[k];
          if (i > 0) {
            const FT* Uc = Ub + (long long)(i - 1) * (HB + 1) * kFacBlk;
#pragma unroll
            for (int k = 0; k <= nn; ++k) un[k] = (VT)__ldg(Uc + (long long)k * kFacBlk);
          }
          const VT xi = v[0] * u[0];
          x[i * T] = xi;
          const VT nxt = (i - HB >= 0) ? x[(i - HB) * T] : (VT)0;
#pragma unroll
          for (int k = 0; k < HB - 1; ++k) v[k] = (k < nu) ? fma(-u[k + 1], xi, v[k + 1]) : v[k + 1];
          v[HB - 1] = (HB - 1 < nu) ? fma(-u[HB], xi, nxt) : nxt;
        }
      });
    }
  } else if constexpr (NB == 0) {
    VT w[HB], l[HB], ln[HB];
#pragma unroll
    for (int k = 0; k < HB; ++k) w[k] = (k < M) ? x[k * T] : (VT)0;
#pragma unroll
    for (int k = 0; k < HB; ++k) ln[k] = (VT)__ldg(Lb + (long long)k * kFacBlk);
#pragma unroll 1
    for (int i = 0; i < M; ++i) {
#pragma unroll
      for (int k = 0; k < HB; ++k) l[k] = ln[k];
      if (i + 1 < M) {
        const FT* Lc = Lb + (long long)(i + 1) * HB * kFacBlk;
#pragma unroll
        for (int k = 0; k < HB; ++k) ln[k] = (VT)__ldg(Lc + (long long)k * kFacBlk);
      }
      const VT y = w[0];
      x[i * T] = y;
      const VT nxt = (i + HB < M) ? x[(i + HB) * T] : (VT)0;
#pragma unroll
      for (int k = 0; k < HB - 1; ++k) w[k] = fma(-l[k], y, w[k + 1]);
      w[HB - 1] = fma(-l[HB - 1], y, nxt);
    }
    VT v[HB], u[HB + 1], un[HB + 1];
#pragma unroll
    for (int k = 0; k < HB; ++k) v[k] = (M - 1 - k >= 0) ? x[(M - 1 - k) * T] : (VT)0;
    {
      const FT* Uc = Ub + (long long)(M - 1) * (HB + 1) * kFacBlk;
#pragma unroll
      for (int k = 0; k <= HB; ++k) un[k] = (VT)__ldg(Uc + (long long)k * kFacBlk);
    }
#pragma unroll 1
    for (int i = M - 1; i >= 0; --i) {
#pragma unroll
      for (int k = 0; k <= HB; ++k) u[k] = un[k];
      if (i > 0) {
        const FT* Uc = Ub + (long long)(i - 1) * (HB + 1) * kFacBlk;
#pragma unroll
        for (int k = 0; k <= HB; ++k) un[k] = (VT)__ldg(Uc + (long long)k * kFacBlk);
      }
      const VT xi = v[0] * u[0];
      x[i * T] = xi;
      const VT nxt = (i - HB >= 0) ? x[(i - HB) * T] : (VT)0;
#pragma unroll
      for (int k = 0; k < HB - 1; ++k) v[k] = fma(-u[k + 1], xi, v[k + 1]);
      v[HB - 1] = fma(-u[HB], xi, nxt);
    }
  } else {
    VT w[HB], rl[NB][HB];
  #pragma unroll
    for (int k = 0; k < HB; ++k) w[k] = (k < M) ? x[k * T] : (VT)0;
  #pragma unroll
    for (int p = 0; p < NB; ++p)
      if (p < M) {
        const FT* Lc = Lb + (long long)p * HB * kFacBlk;
  #pragma unroll
        for (int k = 0; k < HB; ++k) rl[p][k] = (VT)__ldg(Lc + (long long)k * kFacBlk);
      }
    for (int i0 = 0; i0 < M; i0 += NB) {
  #pragma unroll
      for (int p = 0; p < NB; ++p) {
        const int i = i0 + p;
        if (i < M) {
          const VT y = w[0];
          x[i * T] = y;
          const VT nxt = (i + HB < M) ? x[(i + HB) * T] : (VT)0;
  #pragma unroll
          for (int k = 0; k < HB - 1; ++k) w[k] = fma(-rl[p][k], y, w[k + 1]);
          w[HB - 1] = fma(-rl[p][HB - 1], y, nxt);
          if (i + NB < M) {
            const FT* Lc = Lb + (long long)(i + NB) * HB * kFacBlk;
  #pragma unroll
            for (int k = 0; k < HB; ++k) rl[p][k] = (VT)__ldg(Lc + (long long)k * kFacBlk);
          }
        }
      }
    }
    VT v[HB], ru[NB][HB + 1];
  #pragma unroll
    for (int k = 0; k < HB; ++k) v[k] = (M - 1 - k >= 0) ? x[(M - 1 - k) * T] : (VT)0;
  #pragma unroll
    for (int p = 0; p < NB; ++p)
      if (M - 1 - p >= 0) {
        const FT* Uc = Ub + (long long)(M - 1 - p) * (HB + 1) * kFacBlk;
  #pragma unroll
        for (int k = 0; k <= HB; ++k) ru[p][k] = (VT)__ldg(Uc + (long long)k * kFacBlk);
      }
    for (int i0 = 0; i0 < M; i0 += NB) {
  #pragma unroll
      for (int p = 0; p < NB; ++p) {
        const int i = M - 1 - (i0 + p);
        if (i >= 0) {
          const VT xi = v[0] * ru[p][0];
          x[i * T] = xi;
          const VT nxt = (i - HB >= 0) ? x[(i - HB) * T] : (VT)0;
  #pragma unroll
          for (int k = 0; k < HB - 1; ++k) v[k] = fma(-ru[p][k + 1], xi, v[k + 1]);
          v[HB - 1] = fma(-ru[p][HB], xi, nxt);
          if (i - NB >= 0) {
            const FT* Uc = Ub + (long long)(i - NB) * (HB + 1) * kFacBlk;
  #pragma unroll
            for (int k = 0; k <= HB; ++k) ru[p][k] = (VT)__ldg(Uc + (long long)k * kFacBlk);
          }
        }
      }
    }
  }
}

// S x = b for one column: FP64 factors, or FP32 factors with FP64 iterative refinement
// (r = b - S X with the FP64 matrix-free operator, correction solved in FP32).
//   B: FP64 right-hand side; on return it holds x.
//   tmp: FP64 scratch column (w_p of the current iterate);
//   Tf, Td: FP32 scratch columns; Xd: FP64 iterate, needed only when iters >= 2.
// The first FP32 solution x0 (Tf) is exact as a double, so the first residual reads it
// from float; later iterates are FP64 (Xd).
// r = b - S X at one level, with tmp = w_p(X) and xl = X[lev].
template <int N>
__device__ __forceinline__ double col_residual(const double* B, const double* tmp, int T, int lev,
                                               const RefLev& R, const StageTab& tb, double xl) {
  // b - (x - kF w_p - kD D_z w_p)
  return col_kdz<N, false, double>(tmp, T, lev, R, tb.dzD,
                                   fma(__ldg(tb.kF + lev), tmp[lev * T], B[lev * T] - xl));
}

template <int N, bool MIXED>
__device__ __forceinline__ void col_solve_refined(double* B, double* tmp, float* Tf, float* Td,
                                                  double* Xd, int T, int M, const Factors& F,
                                                  long long col, const RefLev& R,
                                                  const StageTab& tb, int iters) {
  if (!MIXED) {
    col_solve<2 * N, double, double, 0, N>(B, T, M, F.L, F.U, col);
    return;
  }
  for (int lev = 0; lev < M; ++lev) Tf[lev * T] = f32_of(B[lev * T]);
  col_solve<2 * N, float, float, 0, N>(Tf, T, M, F.L32, F.U32, col);
  for (int it = 0; it < iters; ++it) {
    const bool first = (it == 0), last = (it == iters - 1);
    for (int lev = 0; lev < M; ++lev)
      tmp[lev * T] = first ? col_wp<N, float>(Tf, T, lev, R, tb) : col_wp<N, double>(Xd, T, lev, R, tb);
    for (int lev = 0; lev < M; ++lev) {
      const double xl = first ? f64_of(Tf[lev * T]) : Xd[lev * T];
      Td[lev * T] = f32_of(col_residual<N>(B, tmp, T, lev, R, tb, xl));
    }
    col_solve<2 * N, float, float, 0, N>(Td, T, M, F.L32, F.U32, col);
    for (int lev = 0; lev < M; ++lev) {
      const double x = (first ? f64_of(Tf[lev * T]) : Xd[lev * T]) + f64_of(Td[lev * T]);
      if (last) B[lev * T] = x;
      else Xd[lev * T] = x;
    }
  }
  if (iters == 0)
    for (int lev = 0; lev < M; ++lev) B[lev * T] = f64_of(Tf[lev * T]);
}

// Shared memory of the column kernels, per column and level: the FP64 method keeps two
// FP64 columns; the mixed form adds two FP32 columns and, for two or more refinement
// sweeps, a third FP64 column.
__host__ __device__ inline size_t col_smem_per_level(bool mixed, int iters) {
  return mixed ? 2 * 8 + 2 * 4 + (iters >= 2 ? 8 : 0) : 2 * 8;
}

// Fused 1D-IMEX stage (rows 2 or 3 of Table 1).
// Phase 1 (all threads, coalesced): the explicit predictor q(i)_e = q^n + dt sum_j a_ij R_j
//   and the shift q~_e = q(i)_e + sum_j c_ij q(j); u, v are final here.  Shared memory keeps
//   P_e = G0 rho~_e + H0 theta~_e and w_a = A^-1 (w~_e + lam g theta~_e / theta0).
// Phase 2 (one thread per column): Schur right-hand side b (Algorithm 4), the column solve,
//   and w_p(P) (Eq. utteqn).
// Phase 3 (coalesced): w~ = w_a - w_p(P) (formed at the end of phase 2 in the FP64 form),
//   theta~ = theta~_e - lam w~ d(theta0)/dz, rho~ = (P - H0 theta~) / G0, then
//   q(i) = q~ - sum_j c_ij q(j).  theta~_e, and in the mixed form w_a, come back from the
//   output slots where phase 1 parked them (shared memory for them would cut the resident
//   columns; recomputing them would repeat the predictor's FP64 work).  So out must not
//   overlap an input.
// RT: type of R1, R2 (double, or float in the mixed form).
// col0: first column of this block, T columns (T <= blockDim.x: all threads share phases 1
// and 3, the first T run phase 2); sm: dynamic shared memory of
// col_smem_per_level(MIXED, iters) * M * T bytes.
// NP: previous stages read (1: stage 2; 2: stage 3; 3: stage 4 of a four-stage scheme,
// with R3 and q3; 0: any stage of an s-stage scheme, the terms listed in *P, with qn =
// P->qn).  Pp_out (optional): receives P'(q(i)) (the pre-pass of the next right-hand side
// fused into phase 3; eos: the series coefficients).
template <int N, int NP, bool MIXED, typename RT>
__device__ __forceinline__ void stage_body(long long col0, int T, double* sm,
                                           const double* __restrict__ qn,
                                           const RT* __restrict__ R1, const RT* __restrict__ R2,
                                           const double* __restrict__ q2, double* __restrict__ out,
                                           const Geom& G, const RefLev& R, const Factors& F,
                                           const StageCoef& sc, const StageTab& tb, int iters,
                                           const RT* __restrict__ R3 = nullptr,
                                           const double* __restrict__ q3 = nullptr,
                                           double* __restrict__ Pp_out = nullptr,
                                           const EosSeries* eos = nullptr,
                                           const StagePrev* P = nullptr) {
  const int NT = blockDim.x, M = G.M;
  const long long nn = G.nnode;
  const int ncols = (int)min((long long)T, G.ncol - col0);
  const long long base = col0 * M;
  const int cnt = ncols * M;
  double* S0 = sm;              // P_e -> b -> P
  double* S1 = sm + M * T;      // w_a -> (scratch) -> w_p(P)
  double* SXd = sm + 2 * M * T; // mixed form with >= 2 sweeps: FP64 iterate
  float* Tf = (float*)(sm + (iters >= 2 ? 3 : 2) * M * T);
  float* Td = Tf + M * T;
  const double a1dt = sc.a[0] * sc.dt, a2dt = sc.a[1] * sc.dt, a3dt = sc.a[2] * sc.dt;
  const double c1 = sc.c[0], c2 = sc.c[1], c3 = sc.c[2];

  // predictor of field f at global offset o (q(i)_e, shifted to q~_e unless u, v)
  auto pred = [&](int f, long long o) -> double {
    const double qv = qn[o];
    if (NP == 0) {
      double v = qv;
      for (int k = 0; k < P->nr; ++k) v = fma(P->adt[k], __ldg(P->R[k] + o), v);
      if (f == 1 || f == 2) return v;
      for (int k = 0; k < P->nq; ++k) v = fma(P->c[k], __ldg(P->q[k] + o), v);
      return v;
    }
    double v = fma(a1dt, to_f64(R1[o]), qv);
    if (NP >= 2) v = fma(a2dt, to_f64(R2[o]), v);
    if (NP >= 3) v = fma(a3dt, to_f64(R3[o]), v);
    if (f == 1 || f == 2) return v;
    v = fma(c1, qv, v);
    if (NP >= 2) v = fma(c2, q2[o], v);
    if (NP >= 3) v = fma(c3, q3[o], v);
    return v;
  };

  // phase 1
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
    out[nn + g] = pred(1, nn + g);
    out[2 * nn + g] = pred(2, 2 * nn + g);
    const double re = pred(0, g), we = pred(3, 3 * nn + g), te = pred(4, 4 * nn + g);
    const double wa = fma(__ldg(tb.wa_th + lev), te, we) * __ldg(tb.wa_s + lev);
    S1[lev * T + c] = wa;
    S0[lev * T + c] = fma(__ldg(tb.G0 + lev), re, __ldg(tb.H0 + lev) * te);
    // theta~_e (and, in the mixed form, w_a) wait in the output slots for phase 3, which
    // the same thread runs on the same node: no FP64 work is repeated there
    out[4 * nn + g] = te;
    if (MIXED) out[3 * nn + g] = wa;
  }
  __syncthreads();

  // phase 2: the level-parallel steps on all NT threads (level lev of column c, consecutive
  // threads on consecutive columns), the triangular substitutions one thread per column.
  // Every (level, column) value is computed by the same arithmetic as in a thread-per-column
  // sweep, so the results do not depend on NT.
  const int tid = threadIdx.x;
  auto level_loop = [&](auto&& body) {
    for (int j = tid; j < cnt; j += NT) {
      const int lev = j / ncols;
      body(lev, j - lev * ncols);
    }
  };
  level_loop([&](int lev, int c) {     // b = P_e - lam F0z w_a - lam rho0 G0 D_z w_a
    const double b = col_kdz<N, true, double>(
        S1 + c, T, lev, R, tb.dzD, fma(-__ldg(tb.kF + lev), S1[lev * T + c], S0[lev * T + c]));
    S0[lev * T + c] = b;
    if (MIXED) Tf[lev * T + c] = f32_of(b);
  });
  __syncthreads();
  if (!MIXED) {
    if (tid < ncols) col_solve<2 * N, double, double, 0, N>(S0 + tid, T, M, F.L, F.U, col0 + tid);
    __syncthreads();
  } else {
    // FP32 solve, then `iters` sweeps of FP64 refinement (r = b - S X with the FP64
    // matrix-free operator, correction solved in FP32); S1 is the scratch for w_p(X)
    if (tid < ncols) col_solve<2 * N, float, float, 0, N>(Tf + tid, T, M, F.L32, F.U32, col0 + tid);
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
      const bool first = (it == 0), last = (it == iters - 1);
      level_loop([&](int lev, int c) {
        S1[lev * T + c] = first ? col_wp<N, float>(Tf + c, T, lev, R, tb)
                                : col_wp<N, double>(SXd + c, T, lev, R, tb);
      });
      __syncthreads();
      level_loop([&](int lev, int c) {
        const double xl = first ? f64_of(Tf[lev * T + c]) : SXd[lev * T + c];
        Td[lev * T + c] = f32_of(col_residual<N>(S0 + c, S1 + c, T, lev, R, tb, xl));
      });
      __syncthreads();
      if (tid < ncols) col_solve<2 * N, float, float, 0, N>(Td + tid, T, M, F.L32, F.U32, col0 + tid);
      __syncthreads();
      level_loop([&](int lev, int c) {
        const double x = (first ? f64_of(Tf[lev * T + c]) : SXd[lev * T + c]) + f64_of(Td[lev * T + c]);
        if (last) S0[lev * T + c] = x;
        else SXd[lev * T + c] = x;
      });
      __syncthreads();
    }
    if (iters == 0) {
      level_loop([&](int lev, int c) { S0[lev * T + c] = f64_of(Tf[lev * T + c]); });
      __syncthreads();
    }
  }
  // FP64: S1 still holds w_a, so it becomes w = w_a - w_p(P) here; the mixed form used S1 as
  // scratch and keeps w_p(P) (phase 3 recomputes w_a)
  level_loop([&](int lev, int c) {
    if (MIXED) {
      S1[lev * T + c] = col_wp<N, double>(S0 + c, T, lev, R, tb);
    } else {   // w_a - (kp1 D_z P + kp2 P), the subtraction folded into the multiply-adds
      S1[lev * T + c] = col_kdz<N, true, double>(
          S0 + c, T, lev, R, tb.dzP, fma(-__ldg(tb.kp2 + lev), S0[lev * T + c], S1[lev * T + c]));
    }
  });
  __syncthreads();

  // phase 3
  unsigned bad = 0;
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
    const long long orr = g, ow = 3 * nn + g, oth = 4 * nn + g;
    const double te = out[oth];
    double wv;
    if (MIXED) {
      wv = out[ow] - S1[lev * T + c];
    } else {
      wv = S1[lev * T + c];
    }
    const double thv = fma(-__ldg(tb.kth + lev), wv, te);
    const double rv = fma(-__ldg(tb.H0G0 + lev), thv, __ldg(tb.invG0 + lev) * S0[lev * T + c]);
    double o_r, o_w, o_t;
    if (NP == 0) {
      o_r = rv;
      o_w = wv;
      o_t = thv;
      for (int k = 0; k < P->nq; ++k) {
        const double* qk = P->q[k];
        o_r = fma(-P->c[k], __ldg(qk + orr), o_r);
        o_w = fma(-P->c[k], __ldg(qk + ow), o_w);
        o_t = fma(-P->c[k], __ldg(qk + oth), o_t);
      }
    } else {
      o_r = fma(-c1, qn[orr], rv);
      o_w = fma(-c1, qn[ow], wv);
      o_t = fma(-c1, qn[oth], thv);
    }
    if (NP >= 2) {
      o_r = fma(-c2, q2[orr], o_r);
      o_w = fma(-c2, q2[ow], o_w);
      o_t = fma(-c2, q2[oth], o_t);
    }
    if (NP >= 3) {
      o_r = fma(-c3, q3[orr], o_r);
      o_w = fma(-c3, q3[ow], o_w);
      o_t = fma(-c3, q3[oth], o_t);
    }
    out[orr] = o_r;
    out[ow] = o_w;
    out[oth] = o_t;
    // P'(q(i)) for the next right-hand side, by the arithmetic of its pre-pass (eos_node)
    if (Pp_out) {
      const double pv = eos_pp(o_r, o_t, lev, R, *eos);
      Pp_out[g] = pv;
      bad |= not_finite(pv);
    }
  }
  if (bad && tb.status) atomicOr(tb.status, NUMA_ST_NONFINITE);
}

}  // namespace numa_dev
