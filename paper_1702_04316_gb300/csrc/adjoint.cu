// Differentiation form: tangent-linear (TLM) and adjoint kernels of the explicit
// right-hand side, the transposed stored-LU column solve, the adjoint of the fused
// implicit stage, and step / multi-step drivers with checkpointing and recomputation.
//
// The paper integrates forward only; these are the chain rule applied to its steps
// (Sec. "Equation Set2NC" for R, Eqs. utteqn / helm2nc and Algorithm 9 for the column
// solve, Table 1 and the stage form of Sec. "Linear multi-stage methods" for the step).
//
// * TLM of R at a state q: every term of the Set2NC tendencies differentiated by the
//   product rule; the equation of state P = p00 (rho R theta / p00)^gamma linearises to
//   dP' = gamma P (drho'/rho + dtheta'/theta).
// * Adjoint of R, owner-computes (no atomics, bitwise reproducible): a pointwise pass
//   forms, at every node h, the 18 weights W_{a,f}(h) with which the derivative of field f
//   along axis a enters lam . R'(q) dq; then each node g gathers
//     sum_a sum_h Dhat_a(h, g) W_{a,f}(h)      (the transposed DSS'd derivative)
//   from the nodes h whose stencil reads g (the transposed tap tables, built on the host
//   from the same rows as the forward stencil), adds its own pointwise terms and
//   transposes the equation of state.
// * The implicit stage is linear in (q^n, R1, R2, q(2)), so its TLM is the stage itself
//   applied to perturbations; its adjoint runs extraction, solve (S^T = U^T L^T on the
//   stored factors), Schur right-hand side and predictor backwards in one column kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "column_device.cuh"
#include "numa.h"
#include "numa_ctx.h"
#include "rhs_device.cuh"

namespace {
using namespace numa_dev;

// Transposed tap tables of the three axes: row idx of axis a lists the nodes h = idx + o
// (o in units of the axis stride) whose derivative row reads idx, with coefficient
// Dhat_a(h, idx).  Exact zeros are left out, so n is N (LGL interior node), 2N (element
// interface) or N+1 (wall), as in the forward rows.
struct AxisT {
  const double* c;   // [rows][2N+1]
  const int* o;      // [rows][2N+1]
  const int* n;      // [rows]
};
struct AdjTab {
  AxisT x, y, z;
};

// ---- kernels ----------------------------------------------------------------------------
// dP' = gamma P (drho'/rho + dtheta'/theta), P = P0 + P'.
__global__ void k_dpressure(const double* __restrict__ q, const double* __restrict__ Pp,
                            const double* __restrict__ dq, double* __restrict__ dPp, Geom G,
                            RefLev R) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long nn = G.nnode;
  const int iz = (int)(g % G.M);
  const double P = R.P0[iz] + Pp[g];
  const double rho = R.rho0[iz] + q[g], th = R.theta0[iz] + q[4 * nn + g];
  dPp[g] = NUMA_GAMMA * P * fma(dq[g], recip(rho), dq[4 * nn + g] * recip(th));
}

// dR = R'(q) dq at every node (natural node order).
template <int N>
__global__ void k_rhs_tlm(const double* __restrict__ q, const double* __restrict__ Pp,
                          const double* __restrict__ dq, const double* __restrict__ dPp,
                          double* __restrict__ dR, Geom G, Coef3 C, RefLev R) {
  constexpr int Nq = N + 1;
  __shared__ double sD[3 * Nq * Nq], sDl[3 * Nq], sDr[3 * Nq];
  load_rows<N, double>(C, sD, sDl, sDr);
  __syncthreads();
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long nn = G.nnode;
  const long long col = g / G.M;
  const int iz = (int)(g - col * G.M);
  const int iy = (int)(col / G.nxg);
  const int ix = (int)(col - (long long)iy * G.nxg);
  const long long sx = G.M, sy = (long long)G.nxg * G.M;
  const double* F[6] = {q, q + nn, q + 2 * nn, q + 3 * nn, q + 4 * nn, Pp};
  const double* dF[6] = {dq, dq + nn, dq + 2 * nn, dq + 3 * nn, dq + 4 * nn, dPp};
  double dx[6], dy[6], dz[6], ex[6], ey[6], ez[6];
  {
    Taps<N, double> T;
    int cls = axis_taps<N, double>(ix, G.nex, sD, sDl, sDr, T);
    axis_derivs<N, double>(F, g, sx, cls, T, dx);
    axis_derivs<N, double>(dF, g, sx, cls, T, ex);
    cls = axis_taps<N, double>(iy, G.ney, sD + Nq * Nq, sDl + Nq, sDr + Nq, T);
    axis_derivs<N, double>(F, g, sy, cls, T, dy);
    axis_derivs<N, double>(dF, g, sy, cls, T, ey);
    cls = axis_taps<N, double>(iz, G.nez, sD + 2 * Nq * Nq, sDl + 2 * Nq, sDr + 2 * Nq, T);
    axis_derivs<N, double>(F, g, 1, cls, T, dz);
    axis_derivs<N, double>(dF, g, 1, cls, T, ez);
  }
  const double r = q[g], u = q[nn + g], v = q[2 * nn + g], w = q[3 * nn + g];
  const double dr = dq[g], du = dq[nn + g], dv = dq[2 * nn + g], dw = dq[3 * nn + g];
  const double rho = R.rho0[iz] + r, ir = recip(rho), ir2 = ir * ir;
  // minus d(u.grad f) = -(du f_x + u df_x + ...), the minus signs on the operands so that no
  // instruction negates a result (as in the forward right-hand side)
  const double ndu = -du, nu = -u, ndv = -dv, nv = -v, ndw = -dw, nw = -w;
  auto ndadv = [&](int f) {
    return ndu * dx[f] + nu * ex[f] + ndv * dy[f] + nv * ey[f] + ndw * dz[f] + nw * ez[f];
  };
  double t[5];
  t[0] = ndadv(0) + ndw * R.drho0[iz] - dr * (dx[1] + dy[2] + dz[3]) - rho * (ex[1] + ey[2] + ez[3]);
  t[1] = ndadv(1) - ex[5] * ir + dx[5] * dr * ir2;
  t[2] = ndadv(2) - ey[5] * ir + dy[5] * dr * ir2;
  t[3] = ndadv(3) - (ez[5] + NUMA_GRAV * dr) * ir + (dz[5] + NUMA_GRAV * r) * dr * ir2;
  t[4] = ndadv(4) + ndw * R.dtheta0[iz];
  if (ix == 0 || ix == G.nxg - 1) t[1] = 0.0;
  if (iy == 0 || iy == G.nyg - 1) t[2] = 0.0;
  if (iz == 0 || iz == G.M - 1) t[3] = 0.0;
#pragma unroll
  for (int f = 0; f < 5; ++f) dR[f * nn + g] = t[f];
}

// The adjoint at node h, wall-masked as the forward tendency is.
__device__ __forceinline__ void masked_lam(const double* __restrict__ lam, long long h, long long nn,
                                           int ix, int iy, int iz, const Geom& G, double* l) {
#pragma unroll
  for (int f = 0; f < 5; ++f) l[f] = lam[f * nn + h];
  if (ix == 0 || ix == G.nxg - 1) l[1] = 0.0;
  if (iy == 0 || iy == G.nyg - 1) l[2] = 0.0;
  if (iz == 0 || iz == G.M - 1) l[3] = 0.0;
}

// Weights W[(a*6 + f)*nnode + h]: coefficient of d_a(field f)(h) in lam . R'(q) dq, fields
// rho', u, v, w, theta', P'.  With lam masked and rho = rho0 + rho':
//   a = x: (-u l_r, -(rho l_r + u l_u), -u l_v, -u l_w, -u l_t, -l_u / rho), y and z alike.
__global__ void k_adj_weights(const double* __restrict__ q, const double* __restrict__ lam,
                              double* __restrict__ W, Geom G, RefLev R) {
  const long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (h >= G.nnode) return;
  const long long nn = G.nnode;
  const long long col = h / G.M;
  const int iz = (int)(h - col * G.M);
  const int iy = (int)(col / G.nxg);
  const int ix = (int)(col - (long long)iy * G.nxg);
  double l[5];
  masked_lam(lam, h, nn, ix, iy, iz, G, l);
  const double rho = R.rho0[iz] + q[h], ir = recip(rho);
  const double vel[3] = {q[nn + h], q[2 * nn + h], q[3 * nn + h]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double* Wa = W + (long long)a * 6 * nn + h;
    const double c = vel[a];
    Wa[0] = -c * l[0];
#pragma unroll
    for (int f = 1; f <= 4; ++f) Wa[f * nn] = -c * l[f] - (f == a + 1 ? rho * l[0] : 0.0);
    Wa[5 * nn] = -l[a + 1] * ir;
  }
}

// acc[f] += sum_t c_t W_f(g + o_t stride), f = 0..5
template <int N>
__device__ __forceinline__ void gather_axis(const double* __restrict__ W, long long nn, long long g,
                                            long long stride, const AxisT& A, int idx, double* acc) {
  constexpr int Wd = 2 * N + 1;
  const int n = __ldg(A.n + idx);
  const double* c = A.c + (long long)idx * Wd;
  const int* o = A.o + (long long)idx * Wd;
#pragma unroll
  for (int t = 0; t < Wd; ++t) {
    if (t < n) {
      const double ct = __ldg(c + t);
      const double* p = W + g + (long long)__ldg(o + t) * stride;
#pragma unroll
      for (int f = 0; f < 6; ++f) acc[f] = fma(ct, __ldg(p + f * nn), acc[f]);
    }
  }
}

// out (+)= R'(q)^T lam at every node, from the weights W of k_adj_weights.
template <int N>
__global__ void k_rhs_adj(const double* __restrict__ q, const double* __restrict__ Pp,
                          const double* __restrict__ lam, const double* __restrict__ W,
                          double* __restrict__ out, int accumulate, Geom G, Coef3 C, RefLev R,
                          AdjTab A) {
  constexpr int Nq = N + 1;
  __shared__ double sD[3 * Nq * Nq], sDl[3 * Nq], sDr[3 * Nq];
  load_rows<N, double>(C, sD, sDl, sDr);
  __syncthreads();
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long nn = G.nnode;
  const long long col = g / G.M;
  const int iz = (int)(g - col * G.M);
  const int iy = (int)(col / G.nxg);
  const int ix = (int)(col - (long long)iy * G.nxg);
  const long long sx = G.M, sy = (long long)G.nxg * G.M;

  // transposed derivative terms
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  gather_axis<N>(W, nn, g, sx, A.x, ix, acc);
  gather_axis<N>(W + 6 * nn, nn, g, sy, A.y, iy, acc);
  gather_axis<N>(W + 12 * nn, nn, g, 1, A.z, iz, acc);

  // pointwise terms: the forward derivatives at g times the adjoint at g
  const double* F[6] = {q, q + nn, q + 2 * nn, q + 3 * nn, q + 4 * nn, Pp};
  double dx[6], dy[6], dz[6];
  {
    Taps<N, double> T;
    int cls = axis_taps<N, double>(ix, G.nex, sD, sDl, sDr, T);
    axis_derivs<N, double>(F, g, sx, cls, T, dx);
    cls = axis_taps<N, double>(iy, G.ney, sD + Nq * Nq, sDl + Nq, sDr + Nq, T);
    axis_derivs<N, double>(F, g, sy, cls, T, dy);
    cls = axis_taps<N, double>(iz, G.nez, sD + 2 * Nq * Nq, sDl + 2 * Nq, sDr + 2 * Nq, T);
    axis_derivs<N, double>(F, g, 1, cls, T, dz);
  }
  double l[5];
  masked_lam(lam, g, nn, ix, iy, iz, G, l);
  const double r = q[g];
  const double rho = R.rho0[iz] + r, ir = recip(rho), ir2 = ir * ir;
  acc[0] += -(dx[1] + dy[2] + dz[3]) * l[0] + dx[5] * ir2 * l[1] + dy[5] * ir2 * l[2] +
            ((dz[5] + NUMA_GRAV * r) * ir2 - NUMA_GRAV * ir) * l[3];
  acc[1] -= dx[0] * l[0] + dx[1] * l[1] + dx[2] * l[2] + dx[3] * l[3] + dx[4] * l[4];
  acc[2] -= dy[0] * l[0] + dy[1] * l[1] + dy[2] * l[2] + dy[3] * l[3] + dy[4] * l[4];
  acc[3] -= (dz[0] + R.drho0[iz]) * l[0] + dz[1] * l[1] + dz[2] * l[2] + dz[3] * l[3] +
            (dz[4] + R.dtheta0[iz]) * l[4];
  // equation of state transposed: P' = P(rho0 + rho', theta0 + theta') - P0
  const double P = R.P0[iz] + Pp[g];
  acc[0] += NUMA_GAMMA * P * ir * acc[5];
  acc[4] += NUMA_GAMMA * P / (R.theta0[iz] + q[4 * nn + g]) * acc[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const long long o = f * nn + g;
    out[o] = accumulate ? out[o] + acc[f] : acc[f];
  }
}

// (D_z^T v)[j] = sum_i D_z(i, j) v[i] for a column in shared memory (stride T).
template <int N>
__device__ __forceinline__ double col_dzT(const double* v, int T, int j, int M, const RefLev& R) {
  constexpr int W = 2 * N + 1;
  double acc = 0.0;
  const int i0 = max(0, j - N), i1 = min(M - 1, j + N);
  for (int i = i0; i <= i1; ++i)
    acc = fma(__ldg(R.dz_band + (long long)i * W + (j - i + N)), v[i * T], acc);
  return acc;
}

// Solve S^T x = b in place for one column (stride T), S = L U in the stored layout:
// U^T y = b by forward substitution (row i of U^T is stored column i of U: the entries
// U(i-k, i), k = 1..2N, and 1/U(i,i)), then L^T x = y by back substitution (row i of L^T is
// stored column i of L).  The last 2N values of the recurrence stay in registers, and the
// factor row of the next step is loaded while the current one is used.  Only the entries
// inside the factors' envelope are read and used (env_u, env_l: the stored entries beyond
// are exact zeros); the level loops run in blocks of N so that each level's count is a
// compile-time constant (r = i mod N, and M - 1 = nez N).
template <int N>
__device__ __forceinline__ void col_solve_T(double* x, int T, int M, const double* __restrict__ L,
                                            const double* __restrict__ U, long long col) {
  constexpr int HB = 2 * N;
  const double* Lb = L + fac_col_base(col, M, HB);
  const double* Ub = U + fac_col_base(col, M, HB + 1);
  double z[HB], fn[HB + 1];
#pragma unroll
  for (int k = 0; k < HB; ++k) z[k] = 0.0;          // z[k] = y_{i-1-k}
#pragma unroll
  for (int k = 0; k <= env_u(N, 0); ++k) fn[k] = __ldg(Ub + (long long)k * kFacBlk);
#pragma unroll 1
  for (int i0 = 0; i0 < M; i0 += N) {
    static_for<N>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      constexpr int nu = env_u(N, r), nn = env_u(N, (r + 1) % N);
      const int i = i0 + r;
      if (i >= M) return;
      double f[HB + 1];
#pragma unroll
      for (int k = 0; k <= nu; ++k) f[k] = fn[k];
      if (i + 1 < M) {
        const double* Uc = Ub + (long long)(i + 1) * (HB + 1) * kFacBlk;
#pragma unroll
        for (int k = 0; k <= nn; ++k) fn[k] = __ldg(Uc + (long long)k * kFacBlk);
      }
      double acc = x[i * T];
#pragma unroll
      for (int k = 1; k <= nu; ++k) acc = fma(-f[k], z[k - 1], acc);
      const double y = acc * f[0];
      x[i * T] = y;
#pragma unroll
      for (int k = HB - 1; k > 0; --k) z[k] = z[k - 1];
      z[0] = y;
    });
  }
#pragma unroll
  for (int k = 0; k < HB; ++k) z[k] = 0.0;          // z[k] = x_{i+1+k}
  {
    const double* Lc = Lb + (long long)(M - 1) * HB * kFacBlk;
#pragma unroll
    for (int k = 0; k < env_l(N, 0); ++k) fn[k] = __ldg(Lc + (long long)k * kFacBlk);
  }
#pragma unroll 1
  for (int t0 = 0; t0 < M; t0 += N) {
    static_for<N>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr int nl = env_l(N, (N - s) % N), nn = env_l(N, (N - (s + 1) % N) % N);
      const int i = M - 1 - (t0 + s);
      if (i < 0) return;
      double f[HB];
#pragma unroll
      for (int k = 0; k < nl; ++k) f[k] = fn[k];
      if (i > 0) {
        const double* Lc = Lb + (long long)(i - 1) * HB * kFacBlk;
#pragma unroll
        for (int k = 0; k < nn; ++k) fn[k] = __ldg(Lc + (long long)k * kFacBlk);
      }
      double acc = x[i * T];
#pragma unroll
      for (int k = 1; k <= nl; ++k) acc = fma(-f[k - 1], z[k - 1], acc);
      x[i * T] = acc;
#pragma unroll
      for (int k = HB - 1; k > 0; --k) z[k] = z[k - 1];
      z[0] = acc;
    });
  }
}

// S^T x = b for T columns per CTA (blockDim.x >= T threads; the first T solve).
template <int N>
__global__ void k_solve_T(const double* __restrict__ b, double* __restrict__ x, Geom G, Factors F,
                          int T) {
  extern __shared__ double sm[];
  const int NT = blockDim.x, M = G.M;
  const long long col0 = blockIdx.x * (long long)T;
  const int ncols = (int)min((long long)T, G.ncol - col0);
  const long long base = col0 * M;
  const int cnt = ncols * M;
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const int c = j / M, lev = j - c * M;
    sm[lev * T + c] = b[base + j];
  }
  __syncthreads();
  if ((int)threadIdx.x < ncols)
    col_solve_T<N>(sm + threadIdx.x, T, M, F.L, F.U, col0 + threadIdx.x);
  __syncthreads();
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const int c = j / M, lev = j - c * M;
    x[base + j] = sm[lev * T + c];
  }
}

// Adjoint of the fused stage (rows 2 or 3 of Table 1), the forward's phases run backwards.
// lam: adjoint of the stage output q(i).  Accumulates into qa (q^n), R1a, and for stage 3
// R2a and q2a.  Forward, per column (u, v: q(i) = q^n + dt sum_j a_ij R_j):
//   q~_e = (1 + c1) q^n + a1 dt R1 (+ a2 dt R2 + c2 q(2))       for rho', w, theta'
//   w_a = wa_s (w~_e + wa_th theta~_e),  P_e = G0 rho~_e + H0 theta~_e
//   b = P_e - kF w_a - kD D_z w_a,  P = S^-1 b,  w_p = kp1 D_z P + kp2 P
//   w = w_a - w_p,  theta = theta~_e - kth w,  rho = invG0 P - H0G0 theta
//   q(i) = (rho, w, theta) - c1 q^n (- c2 q(2))
// Shared memory: four columns of M levels for each of the CTA's T columns; blockDim.x >= T
// threads share the coalesced phases, the first T run the column phase.
template <int N, bool S3>
__global__ void k_stage_adj(const double* __restrict__ lam, double* __restrict__ qa,
                            double* __restrict__ R1a, double* __restrict__ R2a,
                            double* __restrict__ q2a, Geom G, RefLev R, Factors F, StageCoef sc,
                            StageTab tb, int T) {
  extern __shared__ double sm[];
  const int NT = blockDim.x, M = G.M;
  const long long nn = G.nnode;
  const long long col0 = blockIdx.x * (long long)T;
  const int ncols = (int)min((long long)T, G.ncol - col0);
  const long long base = col0 * M;
  const int cnt = ncols * M;
  double* Th = sm;             // theta*
  double* Wt = sm + M * T;     // w* -> w_a*
  double* A = sm + 2 * M * T;  // operands of D_z^T
  double* P = sm + 3 * M * T;  // P* -> b*
  const double a1dt = sc.a[0] * sc.dt, a2dt = sc.a[1] * sc.dt;
  const double c1 = sc.c[0], c2 = sc.c[1];

  // phase 3 backwards (coalesced): u, v directly; theta*, w*, P* and kp1 w_p* per level
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
#pragma unroll
    for (int f = 1; f <= 2; ++f) {
      const long long o = f * nn + g;
      const double l = lam[o];
      qa[o] += l;
      R1a[o] += a1dt * l;
      if (S3) R2a[o] += a2dt * l;
    }
    const double lr = lam[g], lw = lam[3 * nn + g], lt = lam[4 * nn + g];
    const double th = lt - __ldg(tb.H0G0 + lev) * lr;
    const double wt = lw - __ldg(tb.kth + lev) * th;
    Th[lev * T + c] = th;
    Wt[lev * T + c] = wt;
    P[lev * T + c] = __ldg(tb.invG0 + lev) * lr;
    A[lev * T + c] = -__ldg(tb.kp1 + lev) * wt;      // kp1 w_p*, with w_p* = -w*
  }
  __syncthreads();

  // phase 2 backwards.  The level-parallel steps run on all threads (level lev of column c,
  // consecutive threads on consecutive columns), the transposed substitutions one thread per
  // column; every (level, column) value is the same arithmetic as in a thread-per-column
  // sweep.
  const int tid = threadIdx.x;
  auto level_loop = [&](auto&& body) {
    for (int j = tid; j < cnt; j += NT) {
      const int lev = j / ncols;
      body(lev, j - lev * ncols);
    }
  };
  level_loop([&](int lev, int c) {      // P* += kp2 w_p* + D_z^T (kp1 w_p*)
    P[lev * T + c] += fma(-__ldg(tb.kp2 + lev), Wt[lev * T + c], col_dzT<N>(A + c, T, lev, M, R));
  });
  __syncthreads();
  if (tid < ncols) col_solve_T<N>(P + tid, T, M, F.L, F.U, col0 + tid);   // b* = S^-T P*
  __syncthreads();
  level_loop([&](int lev, int c) { A[lev * T + c] = __ldg(tb.kD + lev) * P[lev * T + c]; });
  __syncthreads();
  level_loop([&](int lev, int c) {      // w_a* = w* - kF b* - D_z^T (kD b*)
    Wt[lev * T + c] -= fma(__ldg(tb.kF + lev), P[lev * T + c], col_dzT<N>(A + c, T, lev, M, R));
  });
  __syncthreads();

  // phase 1 backwards (coalesced)
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += NT) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
    const double bs = P[lev * T + c];
    const double we = __ldg(tb.wa_s + lev) * Wt[lev * T + c];                 // w~_e*
    const double te = Th[lev * T + c] + __ldg(tb.wa_th + lev) * we + __ldg(tb.H0 + lev) * bs;
    const double re = __ldg(tb.G0 + lev) * bs;                                 // rho~_e*
    const double es[3] = {re, we, te};
    const int fl[3] = {0, 3, 4};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long o = fl[k] * nn + g;
      const double l = lam[o];
      qa[o] += fma(1.0 + c1, es[k], -c1 * l);
      R1a[o] += a1dt * es[k];
      if (S3) {
        R2a[o] += a2dt * es[k];
        q2a[o] += c2 * (es[k] - l);
      }
    }
  }
}

// y = a x + b y over n entries (grid-stride).
__global__ void k_axpby(const double* __restrict__ x, double* y, long long n, double a, double b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

// ---- launchers --------------------------------------------------------------------------
template <int N>
cudaError_t rhs_tlm_n(const double* q, const double* Pp, const double* dq, const double* dPp,
                      double* dR, const Geom& G, const Coef3& C, const RefLev& R, cudaStream_t s) {
  k_rhs_tlm<N><<<(unsigned)((G.nnode + 127) / 128), 128, 0, s>>>(q, Pp, dq, dPp, dR, G, C, R);
  return cudaGetLastError();
}

template <int N>
cudaError_t rhs_adj_n(const double* q, const double* Pp, const double* lam, const double* W,
                      double* out, int accumulate, const Geom& G, const Coef3& C, const RefLev& R,
                      const AdjTab& A, cudaStream_t s) {
  k_rhs_adj<N><<<(unsigned)((G.nnode + 127) / 128), 128, 0, s>>>(q, Pp, lam, W, out, accumulate,
                                                                  G, C, R, A);
  return cudaGetLastError();
}

// Columns per CTA of the adjoint column kernels: 32, or 16 when that leaves fewer CTAs than
// SMs, and fewer when four columns of M levels each would not fit in shared memory.  The
// CTAs have kAdjThreads threads for the coalesced phases.
const int kAdjThreads = 128;

int adj_cols(const Geom& G) {
  int T = 32;
  if ((G.ncol + T - 1) / T < 152) T = 16;
  while (T > 1 && (size_t)4 * G.M * T * sizeof(double) > 200 * 1024) T /= 2;
  return T;
}

template <int N>
cudaError_t solve_T_n(const double* b, double* x, const Geom& G, const Factors& F, cudaStream_t s) {
  const int T = adj_cols(G);
  const size_t smem = (size_t)G.M * T * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_solve_T<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_solve_T<N><<<(unsigned)((G.ncol + T - 1) / T), kAdjThreads, smem, s>>>(b, x, G, F, T);
  return cudaGetLastError();
}

template <int N, bool S3>
cudaError_t stage_adj_nt(const double* lam, double* qa, double* R1a, double* R2a, double* q2a,
                         const Geom& G, const RefLev& R, const Factors& F, const StageCoef& sc,
                         const StageTab& tb, cudaStream_t s) {
  const int T = adj_cols(G);
  const size_t smem = (size_t)4 * G.M * T * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_stage_adj<N, S3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_stage_adj<N, S3><<<(unsigned)((G.ncol + T - 1) / T), kAdjThreads, smem, s>>>(
      lam, qa, R1a, R2a, q2a, G, R, F, sc, tb, T);
  return cudaGetLastError();
}

template <int N>
cudaError_t stage_adj_n(int stage, const double* lam, double* qa, double* R1a, double* R2a,
                        double* q2a, const Geom& G, const RefLev& R, const Factors& F,
                        const StageCoef& sc, const StageTab& tb, cudaStream_t s) {
  return stage == 3 ? stage_adj_nt<N, true>(lam, qa, R1a, R2a, q2a, G, R, F, sc, tb, s)
                    : stage_adj_nt<N, false>(lam, qa, R1a, R2a, q2a, G, R, F, sc, tb, s);
}

#define NUMA_ADJ_DISPATCH(fn, ...)     \
  switch (G.N) {                       \
    case 1: return fn<1>(__VA_ARGS__); \
    case 2: return fn<2>(__VA_ARGS__); \
    case 3: return fn<3>(__VA_ARGS__); \
    case 4: return fn<4>(__VA_ARGS__); \
    case 5: return fn<5>(__VA_ARGS__); \
    case 6: return fn<6>(__VA_ARGS__); \
    case 7: return fn<7>(__VA_ARGS__); \
    case 8: return fn<8>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_rhs_tlm(const double* q, const double* Pp, const double* dq, const double* dPp,
                           double* dR, const Geom& G, const Coef3& C, const RefLev& R,
                           cudaStream_t s) {
  NUMA_ADJ_DISPATCH(rhs_tlm_n, q, Pp, dq, dPp, dR, G, C, R, s)
}
cudaError_t launch_rhs_adj(const double* q, const double* Pp, const double* lam, const double* W,
                           double* out, int accumulate, const Geom& G, const Coef3& C,
                           const RefLev& R, const AdjTab& A, cudaStream_t s) {
  NUMA_ADJ_DISPATCH(rhs_adj_n, q, Pp, lam, W, out, accumulate, G, C, R, A, s)
}
cudaError_t launch_solve_T(const double* b, double* x, const Geom& G, const Factors& F,
                           cudaStream_t s) {
  NUMA_ADJ_DISPATCH(solve_T_n, b, x, G, F, s)
}
cudaError_t launch_stage_adj(int stage, const double* lam, double* qa, double* R1a, double* R2a,
                             double* q2a, const Geom& G, const RefLev& R, const Factors& F,
                             const StageCoef& sc, const StageTab& tb, cudaStream_t s) {
  NUMA_ADJ_DISPATCH(stage_adj_n, stage, lam, qa, R1a, R2a, q2a, G, R, F, sc, tb, s)
}
#undef NUMA_ADJ_DISPATCH

// ---- host side --------------------------------------------------------------------------
int afail(numa_ctx* c, int code, const char* m) {
  c->err = m;
  return code;
}

#define NUMA_ACK(c, call)                                                  \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
      return NUMA_ERR_CUDA;                                                \
    }                                                                      \
  } while (0)

// Rows of the DSS'd derivative along one axis as a band (row idx, column idx + b - N),
// the same rows as the forward stencil (axis_taps): interface rows from the two weighted
// halves without the shared node, wall rows from the full element row, interior rows
// without the zero diagonal.
void axis_band(const AxisCoef& a, int N, int nel, std::vector<double>& band) {
  const int n = nel * N + 1, W = 2 * N + 1, Nq = N + 1;
  band.assign((size_t)n * W, 0.0);
  for (int idx = 0; idx < n; ++idx) {
    int e, i;
    axis_owner(idx, N, nel, e, i);
    double* row = &band[(size_t)idx * W];
    if (i == 0 && e > 0) {
      for (int t = 0; t < N; ++t) row[t] = a.Dl[t];            // offset t - N
      for (int t = 1; t <= N; ++t) row[t + N] = a.Dr[t];       // offset t
    } else if (i == 0 || i == N) {
      for (int t = 0; t <= N; ++t) row[t - i + N] = a.D[i * Nq + t];
    } else {
      for (int t = 0; t <= N; ++t)
        if (t != i) row[t - i + N] = a.D[i * Nq + t];
    }
  }
}

// Transposed tap table of one axis appended to (hc, ho, hn): for column idx, the rows h
// with a non-zero Dhat(h, idx), as offsets h - idx.
void axis_transposed(const AxisCoef& a, int N, int nel, std::vector<double>& hc,
                     std::vector<int>& ho, std::vector<int>& hn) {
  std::vector<double> band;
  axis_band(a, N, nel, band);
  const int n = nel * N + 1, W = 2 * N + 1;
  for (int idx = 0; idx < n; ++idx) {
    int cnt = 0;
    std::vector<double> c(W, 0.0);
    std::vector<int> o(W, 0);
    for (int h = std::max(0, idx - N); h <= std::min(n - 1, idx + N); ++h) {
      const double v = band[(size_t)h * W + (idx - h + N)];
      if (v == 0.0) continue;
      c[cnt] = v;
      o[cnt] = h - idx;
      ++cnt;
    }
    hc.insert(hc.end(), c.begin(), c.end());
    ho.insert(ho.end(), o.begin(), o.end());
    hn.push_back(cnt);
  }
}

// Workspace of the differentiation form (59 x nnode doubles) and the transposed tables.
struct AdjWork {
  double* W;      // 18 x nnode: weights of the adjoint right-hand side
  double* dP;     // nnode: dP' of the tangent-linear right-hand side
  double* B[8];   // 5 x nnode each
  AdjTab tab;
};

int adj_work(numa_ctx* c, AdjWork& w) {
  const long long nn = c->G.nnode;
  const int N = c->G.N, Wd = 2 * N + 1;
  const int rows[3] = {c->G.nxg, c->G.nyg, c->G.M};
  if (!c->d_adj) {
    if (cudaMalloc(&c->d_adj, (size_t)59 * nn * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->d_adj = nullptr;
      return afail(c, NUMA_ERR_OOM, "differentiation workspace");
    }
  }
  if (!c->d_adjtab) {
    std::vector<double> hc;
    std::vector<int> ho, hn;
    axis_transposed(c->C.x, N, c->G.nex, hc, ho, hn);
    axis_transposed(c->C.y, N, c->G.ney, hc, ho, hn);
    axis_transposed(c->C.z, N, c->G.nez, hc, ho, hn);
    const size_t bc = hc.size() * sizeof(double), bo = ho.size() * sizeof(int),
                 bn = hn.size() * sizeof(int);
    if (cudaMalloc(&c->d_adjtab, bc + bo + bn) != cudaSuccess) {
      cudaGetLastError();
      c->d_adjtab = nullptr;
      return afail(c, NUMA_ERR_OOM, "differentiation tables");
    }
    char* p = (char*)c->d_adjtab;
    NUMA_ACK(c, cudaMemcpy(p, hc.data(), bc, cudaMemcpyHostToDevice));
    NUMA_ACK(c, cudaMemcpy(p + bc, ho.data(), bo, cudaMemcpyHostToDevice));
    NUMA_ACK(c, cudaMemcpy(p + bc + bo, hn.data(), bn, cudaMemcpyHostToDevice));
  }
  const size_t ntot = (size_t)rows[0] + rows[1] + rows[2];
  const double* tc = (const double*)c->d_adjtab;
  const int* to = (const int*)(tc + ntot * Wd);
  const int* tn = to + ntot * Wd;
  AxisT* ax[3] = {&w.tab.x, &w.tab.y, &w.tab.z};
  size_t r0 = 0;
  for (int a = 0; a < 3; ++a) {
    ax[a]->c = tc + r0 * Wd;
    ax[a]->o = to + r0 * Wd;
    ax[a]->n = tn + r0;
    r0 += rows[a];
  }
  w.W = c->d_adj;
  w.dP = c->d_adj + 18 * nn;
  for (int k = 0; k < 8; ++k) w.B[k] = c->d_adj + 19 * nn + (size_t)k * 5 * nn;
  return NUMA_OK;
}

int check_diff(numa_ctx* c, bool need_factors) {
  if (c->precision != NUMA_PREC_FP64 || c->F.standard || c->scheme != NUMA_SCHEME_ARK2 || c->imex3d)
    return afail(c, NUMA_ERR_ARG, "the differentiation form needs an FP64 Schur-form ARK2 context");
  if (need_factors && !c->factored)
    return afail(c, NUMA_ERR_NOT_FACTORED, "numa_factor_columns not called");
  return NUMA_OK;
}

// dR = R'(q) dq
int enqueue_rhs_tlm(numa_ctx* c, const AdjWork& w, const double* q, const double* dq, double* dR) {
  const unsigned nb = (unsigned)((c->G.nnode + 255) / 256);
  long p = prof_begin(c, NUMA_K_RHS_TLM);
  NUMA_ACK(c, launch_pressure(q, c->Pp, c->G, c->R, c->stream));
  k_dpressure<<<nb, 256, 0, c->stream>>>(q, c->Pp, dq, w.dP, c->G, c->R);
  NUMA_ACK(c, cudaGetLastError());
  NUMA_ACK(c, launch_rhs_tlm(q, c->Pp, dq, w.dP, dR, c->G, c->C, c->R, c->stream));
  prof_end(c, p);
  return NUMA_OK;
}

// out = R'(q)^T lam (accumulate = 0) or out += R'(q)^T lam (accumulate = 1)
int enqueue_rhs_adj(numa_ctx* c, const AdjWork& w, const double* q, const double* lam, double* out,
                    int accumulate) {
  const unsigned nb = (unsigned)((c->G.nnode + 255) / 256);
  long p = prof_begin(c, NUMA_K_RHS_ADJ);
  NUMA_ACK(c, launch_pressure(q, c->Pp, c->G, c->R, c->stream));
  k_adj_weights<<<nb, 256, 0, c->stream>>>(q, lam, w.W, c->G, c->R);
  NUMA_ACK(c, cudaGetLastError());
  NUMA_ACK(c, launch_rhs_adj(q, c->Pp, lam, w.W, out, accumulate, c->G, c->C, c->R, w.tab,
                             c->stream));
  prof_end(c, p);
  return NUMA_OK;
}

int enqueue_stage_adj(numa_ctx* c, int stage, const double* lam, double* qa, double* R1a,
                      double* R2a, double* q2a) {
  long p = prof_begin(c, NUMA_K_STAGE_ADJ);
  NUMA_ACK(c, launch_stage_adj(stage, lam, qa, R1a, R2a, q2a, c->G, c->R, c->F,
                               numa_stage_coef(c, stage), c->T, c->stream));
  prof_end(c, p);
  return NUMA_OK;
}

int scale_into(numa_ctx* c, const double* x, double* y, double a) {
  k_axpby<<<152 * 4, 256, 0, c->stream>>>(x, y, 5 * c->G.nnode, a, 0.0);
  NUMA_ACK(c, cudaGetLastError());
  return NUMA_OK;
}

// The adjoint of one ARK2 step from its states qn = q^n, q2 = q(2), q3 = q(3):
// lam = (dq^{n+1}/dq^n)^T lam_next (lam may equal lam_next).  Uses w.B[0..4] and w.B[6].
int step_adjoint_core(numa_ctx* ctx, const AdjWork& w, const double* qn, const double* q2,
                      const double* q3, const double* lam_next, double* lam) {
  int rc;
  double *R1a = w.B[0], *R2a = w.B[1], *R3a = w.B[2], *q2a = w.B[3], *q3a = w.B[4],
         *qa = w.B[6];
  const size_t bytes = 5 * ctx->G.nnode * sizeof(double);
  double b[3];
  numa_ark2_tableau(nullptr, nullptr, b);
  // q^{n+1} = q^n + dt (b1 R1 + b2 R2 + b3 R3)
  NUMA_ACK(ctx, cudaMemcpyAsync(qa, lam_next, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  if ((rc = scale_into(ctx, lam_next, R1a, b[0] * ctx->dt))) return rc;
  if ((rc = scale_into(ctx, lam_next, R2a, b[1] * ctx->dt))) return rc;
  if ((rc = scale_into(ctx, lam_next, R3a, b[2] * ctx->dt))) return rc;
  NUMA_ACK(ctx, cudaMemsetAsync(q2a, 0, bytes, ctx->stream));
  // R3 = R(q(3));  q(3) = stage 3 (q^n, R1, R2, q(2))
  if ((rc = enqueue_rhs_adj(ctx, w, q3, R3a, q3a, 0))) return rc;
  if ((rc = enqueue_stage_adj(ctx, 3, q3a, qa, R1a, R2a, q2a))) return rc;
  // R2 = R(q(2));  q(2) = stage 2 (q^n, R1)
  if ((rc = enqueue_rhs_adj(ctx, w, q2, R2a, q2a, 1))) return rc;
  if ((rc = enqueue_stage_adj(ctx, 2, q2a, qa, R1a, nullptr, nullptr))) return rc;
  // R1 = R(q^n)
  if ((rc = enqueue_rhs_adj(ctx, w, qn, R1a, qa, 1))) return rc;
  NUMA_ACK(ctx, cudaMemcpyAsync(lam, qa, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return NUMA_OK;
}

}  // namespace

extern "C" {

int numa_rhs_tlm(numa_ctx* ctx, const double* q, const double* dq, double* dR) {
  if (!ctx || !q || !dq || !dR) return NUMA_ERR_ARG;
  int rc;
  AdjWork w;
  if ((rc = check_diff(ctx, false)) || (rc = adj_work(ctx, w))) return rc;
  return enqueue_rhs_tlm(ctx, w, q, dq, dR);
}

int numa_rhs_adjoint(numa_ctx* ctx, const double* q, const double* lam, double* q_adj) {
  if (!ctx || !q || !lam || !q_adj) return NUMA_ERR_ARG;
  int rc;
  AdjWork w;
  if ((rc = check_diff(ctx, false)) || (rc = adj_work(ctx, w))) return rc;
  return enqueue_rhs_adj(ctx, w, q, lam, q_adj, 0);
}

int numa_solve_columns_transposed(numa_ctx* ctx, const double* b, double* x) {
  if (!ctx || !b || !x) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_diff(ctx, true))) return rc;
  long p = prof_begin(ctx, NUMA_K_SOLVE);
  NUMA_ACK(ctx, launch_solve_T(b, x, ctx->G, ctx->F, ctx->stream));
  prof_end(ctx, p);
  return NUMA_OK;
}

int numa_imex_stage_adjoint(numa_ctx* ctx, int stage, const double* lam, double* qn_adj,
                            double* R1_adj, double* R2_adj, double* q2_adj) {
  if (!ctx || !lam || !qn_adj || !R1_adj || (stage != 2 && stage != 3)) return NUMA_ERR_ARG;
  if (stage == 3 && (!R2_adj || !q2_adj)) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_diff(ctx, true))) return rc;
  return enqueue_stage_adj(ctx, stage, lam, qn_adj, R1_adj, R2_adj, q2_adj);
}

int numa_step_imex1d_tlm(numa_ctx* ctx, const double* q, const double* dq, double* q_out,
                         double* dq_out, int nsteps) {
  if (!ctx || !q || !dq || !q_out || !dq_out || nsteps < 1) return NUMA_ERR_ARG;
  int rc;
  AdjWork w;
  if ((rc = check_diff(ctx, true)) || (rc = adj_work(ctx, w))) return rc;
  double *dR1 = w.B[0], *dR2 = w.B[1], *dR3 = w.B[2], *dq2 = w.B[3], *dq3 = w.B[4],
         *R3 = w.B[5], *qn = w.B[6], *dqn = w.B[7];
  const long long n5 = 5 * ctx->G.nnode;
  const size_t bytes = n5 * sizeof(double);
  double b[3];
  numa_ark2_tableau(nullptr, nullptr, b);
  const double b1dt = b[0] * ctx->dt, b2dt = b[1] * ctx->dt, b3dt = b[2] * ctx->dt;
  for (int s = 0; s < nsteps; ++s) {
    NUMA_ACK(ctx, cudaMemcpyAsync(qn, s ? q_out : q, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    NUMA_ACK(ctx, cudaMemcpyAsync(dqn, s ? dq_out : dq, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    // the trajectory's tendencies and stage states go to the context workspace
    if ((rc = numa_rhs_explicit(ctx, qn, ctx->R1))) return rc;
    if ((rc = enqueue_rhs_tlm(ctx, w, qn, dqn, dR1))) return rc;
    if ((rc = numa_imex_stage(ctx, 2, qn, ctx->R1, nullptr, nullptr, ctx->q2))) return rc;
    if ((rc = numa_imex_stage(ctx, 2, dqn, dR1, nullptr, nullptr, dq2))) return rc;
    if ((rc = numa_rhs_explicit(ctx, ctx->q2, ctx->R2))) return rc;
    if ((rc = enqueue_rhs_tlm(ctx, w, ctx->q2, dq2, dR2))) return rc;
    if ((rc = numa_imex_stage(ctx, 3, qn, ctx->R1, ctx->R2, ctx->q2, ctx->q3))) return rc;
    if ((rc = numa_imex_stage(ctx, 3, dqn, dR1, dR2, dq2, dq3))) return rc;
    if ((rc = numa_rhs_explicit(ctx, ctx->q3, R3))) return rc;
    if ((rc = enqueue_rhs_tlm(ctx, w, ctx->q3, dq3, dR3))) return rc;
    NUMA_ACK(ctx, launch_ark_final(qn, ctx->R1, ctx->R2, R3, q_out, n5, b1dt, b2dt, b3dt, ctx->stream));
    NUMA_ACK(ctx, launch_ark_final(dqn, dR1, dR2, dR3, dq_out, n5, b1dt, b2dt, b3dt, ctx->stream));
  }
  return NUMA_OK;
}

int numa_step_imex1d_adjoint(numa_ctx* ctx, const double* q, const double* lam_next,
                             double* lam) {
  if (!ctx || !q || !lam_next || !lam) return NUMA_ERR_ARG;
  int rc;
  AdjWork w;
  if ((rc = check_diff(ctx, true)) || (rc = adj_work(ctx, w))) return rc;
  double* qn = w.B[5];
  const size_t bytes = 5 * ctx->G.nnode * sizeof(double);
  // retake the step from q: it leaves its stage states q(2), q(3) in ctx->q2, ctx->q3
  NUMA_ACK(ctx, cudaMemcpyAsync(qn, q, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  if ((rc = numa_step_imex1d(ctx, qn, w.B[7], 1))) return rc;
  return step_adjoint_core(ctx, w, qn, ctx->q2, ctx->q3, lam_next, lam);
}

int numa_imex1d_forward_checkpointed(numa_ctx* ctx, const double* q0, double* qT, int nsteps,
                                     int every, double* ckpt) {
  if (!ctx || !q0 || !qT || !ckpt || nsteps < 1 || every < 1) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_diff(ctx, true))) return rc;
  const long long n5 = 5 * ctx->G.nnode;
  const size_t bytes = n5 * sizeof(double);
  for (int s = 0; s < nsteps; ++s) {
    const double* cur = s ? qT : q0;
    if (s % every == 0)
      NUMA_ACK(ctx, cudaMemcpyAsync(ckpt + (size_t)(s / every) * n5, cur, bytes,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
    if ((rc = numa_step_imex1d(ctx, cur, qT, 1))) return rc;
  }
  return NUMA_OK;
}

int numa_imex1d_adjoint_checkpointed(numa_ctx* ctx, const double* ckpt, int nsteps, int every,
                                     const double* lamT, double* lam0, double* work) {
  if (!ctx || !ckpt || !lamT || !lam0 || !work || nsteps < 1 || every < 1) return NUMA_ERR_ARG;
  int rc;
  AdjWork w;
  if ((rc = check_diff(ctx, true)) || (rc = adj_work(ctx, w))) return rc;
  const long long n5 = 5 * ctx->G.nnode;
  const size_t bytes = n5 * sizeof(double);
  if (lam0 != lamT)
    NUMA_ACK(ctx, cudaMemcpyAsync(lam0, lamT, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  // work holds, for step i of the current segment, q at that step and its stage states
  auto Q = [&](int i, int f) { return work + ((size_t)3 * i + f) * n5; };
  const int nseg = (nsteps + every - 1) / every;
  for (int k = nseg - 1; k >= 0; --k) {
    const int s0 = k * every, len = std::min(nsteps, s0 + every) - s0;
    // retake the segment's steps from its checkpoint
    NUMA_ACK(ctx, cudaMemcpyAsync(Q(0, 0), ckpt + (size_t)k * n5, bytes, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    for (int i = 0; i < len; ++i) {
      if ((rc = numa_step_imex1d(ctx, Q(i, 0), i + 1 < len ? Q(i + 1, 0) : w.B[7], 1))) return rc;
      NUMA_ACK(ctx, cudaMemcpyAsync(Q(i, 1), ctx->q2, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      NUMA_ACK(ctx, cudaMemcpyAsync(Q(i, 2), ctx->q3, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    for (int i = len - 1; i >= 0; --i)
      if ((rc = step_adjoint_core(ctx, w, Q(i, 0), Q(i, 1), Q(i, 2), lam0, lam0))) return rc;
  }
  return NUMA_OK;
}

}  // extern "C"
