// Column kernels of the 1D-IMEX method: factorisation of the Schur-complement matrix,
// the column solve, and the fused implicit stage.
//
// One thread owns one column (lane-per-column).  On GB300 the FP64 pipe is the scarce
// resource (2 FP64 FMA per clock per SM, 1/64 of FP32), so every lane of a warp does
// useful FP64 work instead of cooperating on one column with shuffles.  The stored
// factors are transposed (column index fastest) so that the 32 lanes of a warp read 256
// contiguous bytes per factor entry, and the state columns are staged through shared
// memory so that their global loads and stores stay coalesced.
//
// The substitutions are right-looking: once y_i (x_i) is known, the next 2N rows are
// updated with 2N independent FMAs held in a register window, so the dependent path per
// row is one FMA and the factors are read by column (the layout numa_internal.cuh gives).
#include "numa_internal.cuh"

namespace {

// ---- band accessor of the stored factors (column-oriented layout) ----------------------
struct Band {
  double* L;
  double* U;
  int hb;
  long long nc;
  long long col;
  __device__ __forceinline__ double& at(int i, int j) const {
    return (j < i) ? L[((long long)j * hb + (i - j) - 1) * nc + col]
                   : U[((long long)j * (hb + 1) + (j - i)) * nc + col];
  }
};

// (D_z f)[lev] for a column held in shared memory with stride T between levels.  lev is
// uniform across a warp, so the tap table reads are broadcasts and the branch on the tap
// count (N interior, 2N interface, N+1 wall) does not diverge.
template <int N>
__device__ __forceinline__ double col_dz(const double* f, int T, int lev, const RefLev& R) {
  constexpr int W = 2 * N + 1;
  const double* c = R.dz_c + (long long)lev * W;
  const int* o = R.dz_o + (long long)lev * W;
  const int n = __ldg(R.dz_n + lev);
  const double* p = f + lev * T;
  if (n == N) {
    double a0 = __ldg(c) * p[__ldg(o) * T], a1 = 0.0;
#pragma unroll
    for (int t = 1; t < N; ++t) {
      if (t & 1) a1 = fma(__ldg(c + t), p[__ldg(o + t) * T], a1);
      else a0 = fma(__ldg(c + t), p[__ldg(o + t) * T], a0);
    }
    return a0 + a1;
  }
  if (n == 2 * N) {
    double a0 = __ldg(c) * p[__ldg(o) * T], a1 = __ldg(c + 1) * p[__ldg(o + 1) * T];
#pragma unroll
    for (int t = 2; t < 2 * N; ++t) {
      if (t & 1) a1 = fma(__ldg(c + t), p[__ldg(o + t) * T], a1);
      else a0 = fma(__ldg(c + t), p[__ldg(o + t) * T], a0);
    }
    return a0 + a1;
  }
  double acc = 0.0;
  for (int t = 0; t < n; ++t) acc = fma(__ldg(c + t), p[__ldg(o + t) * T], acc);
  return acc;
}

// Solve L U x = b in place for one column held in shared memory (stride T).
// Forward: y_i = w_0; then x_{i+1+k} -= L(i+1+k, i) y_i for k < HB (window w in registers).
// Backward: x_i = v_0 / U(i,i); then y_{i-1-k} -= U(i-1-k, i) x_i for k < HB.
// Factor columns are prefetched one column ahead.
template <int HB>
__device__ __forceinline__ void col_solve(double* x, int T, int M, const double* __restrict__ L,
                                          const double* __restrict__ U, long long nc,
                                          long long col) {
  double w[HB], l[HB], ln[HB];
#pragma unroll
  for (int k = 0; k < HB; ++k) w[k] = (k < M) ? x[k * T] : 0.0;
#pragma unroll
  for (int k = 0; k < HB; ++k) ln[k] = __ldg(L + (long long)k * nc + col);
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int k = 0; k < HB; ++k) l[k] = ln[k];
    if (i + 1 < M) {
      const double* Lc = L + (long long)(i + 1) * HB * nc + col;
#pragma unroll
      for (int k = 0; k < HB; ++k) ln[k] = __ldg(Lc + (long long)k * nc);
    }
    const double y = w[0];
    x[i * T] = y;
    const double nxt = (i + HB < M) ? x[(i + HB) * T] : 0.0;
#pragma unroll
    for (int k = 0; k < HB - 1; ++k) w[k] = fma(-l[k], y, w[k + 1]);
    w[HB - 1] = fma(-l[HB - 1], y, nxt);
  }
  double v[HB], u[HB + 1], un[HB + 1];
#pragma unroll
  for (int k = 0; k < HB; ++k) v[k] = (M - 1 - k >= 0) ? x[(M - 1 - k) * T] : 0.0;
  {
    const double* Uc = U + (long long)(M - 1) * (HB + 1) * nc + col;
#pragma unroll
    for (int k = 0; k <= HB; ++k) un[k] = __ldg(Uc + (long long)k * nc);
  }
  for (int i = M - 1; i >= 0; --i) {
#pragma unroll
    for (int k = 0; k <= HB; ++k) u[k] = un[k];
    if (i > 0) {
      const double* Uc = U + (long long)(i - 1) * (HB + 1) * nc + col;
#pragma unroll
      for (int k = 0; k <= HB; ++k) un[k] = __ldg(Uc + (long long)k * nc);
    }
    const double xi = v[0] * u[0];
    x[i * T] = xi;
    const double nxt = (i - HB >= 0) ? x[(i - HB) * T] : 0.0;
#pragma unroll
    for (int k = 0; k < HB - 1; ++k) v[k] = fma(-u[k + 1], xi, v[k + 1]);
    v[HB - 1] = fma(-u[HB], xi, nxt);
  }
}

// Algorithm 7 (BuildJacobian) for the Schur form, one column per thread: column m of
// S(lam) is the left-hand side applied to the unit vector e_m,
//   w_p = A^-1 lam (D_z e_m / rho0 + g e_m / (G0 rho0))   (zero at the two walls)
//   S e_m = e_m - lam F0z w_p - lam rho0 G0 D_z w_p,
// then Algorithm 9 (LUdecompose): banded LU without pivoting, in place.
__global__ void k_factor(Geom G, RefLev R, double lam, Factors F, unsigned* status) {
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (col >= G.ncol) return;
  const int M = G.M, N = G.N, hb = F.hb, W = 2 * N + 1;
  const long long nc = G.ncol;
  Band A{F.L, F.U, hb, nc, col};
  for (int i = 0; i < M; ++i) {
    for (int k = 0; k < hb; ++k) F.L[((long long)i * hb + k) * nc + col] = 0.0;
    for (int k = 0; k <= hb; ++k) F.U[((long long)i * (hb + 1) + k) * nc + col] = 0.0;
  }
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
      A.at(i, m) = s;
    }
  }
  for (int k = 0; k < M; ++k) {
    double piv = A.at(k, k);
    if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
      atomicOr(status, NUMA_ST_PIVOT);
      piv = 1.0;
    }
    const double ip = 1.0 / piv;
    const int E = min(k + hb, M - 1);
    for (int i = k + 1; i <= E; ++i) {
      const double l = A.at(i, k) * ip;
      A.at(i, k) = l;
      for (int j = k + 1; j <= E; ++j) A.at(i, j) = fma(-l, A.at(k, j), A.at(i, j));
    }
    A.at(k, k) = ip;   // the solve multiplies by 1/U(k,k)
  }
}

template <int N>
__global__ void k_solve(const double* b, double* x, Geom G, Factors F) {
  extern __shared__ double sm[];
  const int T = blockDim.x, M = G.M;
  const long long col0 = blockIdx.x * (long long)T;
  const int ncols = (int)min((long long)T, G.ncol - col0);
  const long long base = col0 * M;
  const int cnt = ncols * M;
  for (int j = threadIdx.x; j < cnt; j += T) {
    const int c = j / M, lev = j - c * M;
    sm[lev * T + c] = b[base + j];
  }
  __syncthreads();
  if ((int)threadIdx.x < ncols)
    col_solve<2 * N>(sm + threadIdx.x, T, M, F.L, F.U, G.ncol, col0 + threadIdx.x);
  __syncthreads();
  for (int j = threadIdx.x; j < cnt; j += T) {
    const int c = j / M, lev = j - c * M;
    x[base + j] = sm[lev * T + c];
  }
}

// Fused 1D-IMEX stage (rows 2 or 3 of Table 1).  Phase 1 (all threads, coalesced): the
// explicit predictor q(i)_e = q^n + dt sum_j a_ij R_j, the q~ shift q~_e = q(i)_e +
// sum_j c_ij q(j), and the final u, v.  Phase 2 (one thread per column): Schur right-hand
// side (Algorithm 4), column solve, extraction of (rho', w, theta') (Eq. utteqn).
// Phase 3 (coalesced): q(i) = q~ - sum_j c_ij q(j).
template <int N, bool S3>
__global__ void k_stage(const double* __restrict__ qn, const double* __restrict__ R1,
                        const double* __restrict__ R2, const double* __restrict__ q2,
                        double* __restrict__ out, Geom G, RefLev R, Factors F, StageCoef sc,
                        StageTab tb) {
  extern __shared__ double sm[];
  const int T = blockDim.x, M = G.M;
  const long long nn = G.nnode;
  const long long col0 = blockIdx.x * (long long)T;
  const int ncols = (int)min((long long)T, G.ncol - col0);
  const long long base = col0 * M;
  const int cnt = ncols * M;
  double* S0 = sm;              // rho~_e -> b -> P -> rho~
  double* S1 = sm + M * T;      // w~_e -> w_a -> w~
  double* S2 = sm + 2 * M * T;  // theta~_e -> theta~
  const double a1dt = sc.a[0] * sc.dt, a2dt = sc.a[1] * sc.dt;

  // phase 1
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += T) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
#pragma unroll
    for (int f = 1; f <= 2; ++f) {   // u, v: explicit only
      const long long o = f * nn + g;
      double e = fma(a1dt, R1[o], qn[o]);
      if (S3) e = fma(a2dt, R2[o], e);
      out[o] = e;
    }
    const int fl[3] = {0, 3, 4};
    double* Sd[3] = {S0, S1, S2};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const long long o = fl[t] * nn + g;
      const double qv = qn[o];
      double e = fma(a1dt, R1[o], qv);
      if (S3) e = fma(a2dt, R2[o], e);
      e = fma(sc.c[0], qv, e);
      if (S3) e = fma(sc.c[1], q2[o], e);
      Sd[t][lev * T + c] = e;
    }
  }
  __syncthreads();

  // phase 2
  if ((int)threadIdx.x < ncols) {
    const int t = threadIdx.x;
    double* P = S0 + t;
    double* Wc = S1 + t;
    double* Th = S2 + t;
    for (int lev = 0; lev < M; ++lev) {     // w_a, then P_e
      const double th = Th[lev * T];
      Wc[lev * T] = fma(__ldg(tb.wa_th + lev), th, Wc[lev * T]) * __ldg(tb.wa_s + lev);
      P[lev * T] = fma(__ldg(tb.G0 + lev), P[lev * T], __ldg(tb.H0 + lev) * th);
    }
    for (int lev = 0; lev < M; ++lev) {     // b = P_e - lam F0z w_a - lam rho0 G0 D_z w_a
      const double dzw = col_dz<N>(Wc, T, lev, R);
      P[lev * T] = fma(-__ldg(tb.kF + lev), Wc[lev * T], fma(-__ldg(tb.kD + lev), dzw, P[lev * T]));
    }
    col_solve<2 * N>(P, T, M, F.L, F.U, G.ncol, col0 + t);
    for (int lev = 0; lev < M; ++lev) {     // w = w_a - w_p(P); theta = theta_e - lam w dtheta0
      const double dzp = col_dz<N>(P, T, lev, R);
      const double wp = fma(__ldg(tb.kp1 + lev), dzp, __ldg(tb.kp2 + lev) * P[lev * T]);
      const double wv = Wc[lev * T] - wp;
      Wc[lev * T] = wv;
      Th[lev * T] = fma(-__ldg(tb.kth + lev), wv, Th[lev * T]);
    }
    for (int lev = 0; lev < M; ++lev)       // rho = (P - H0 theta) / G0
      P[lev * T] = fma(-__ldg(tb.H0G0 + lev), Th[lev * T], __ldg(tb.invG0 + lev) * P[lev * T]);
  }
  __syncthreads();

  // phase 3
#pragma unroll 2
  for (int j = threadIdx.x; j < cnt; j += T) {
    const long long g = base + j;
    const int c = j / M, lev = j - c * M;
    const int fl[3] = {0, 3, 4};
    const double* Sd[3] = {S0, S1, S2};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const long long o = fl[t] * nn + g;
      double v = fma(-sc.c[0], qn[o], Sd[t][lev * T + c]);
      if (S3) v = fma(-sc.c[1], q2[o], v);
      out[o] = v;
    }
  }
}

template <int N>
cudaError_t launch_solve_n(const double* b, double* x, const Geom& G, Factors F, int T,
                           cudaStream_t s) {
  const size_t smem = (size_t)G.M * T * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_solve<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_solve<N><<<(unsigned)((G.ncol + T - 1) / T), T, smem, s>>>(b, x, G, F);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_stage_n(int stage, const double* qn, const double* R1, const double* R2,
                           const double* q2, double* out, const Geom& G, const RefLev& R,
                           Factors F, const StageCoef& sc, const StageTab& tb, int T,
                           cudaStream_t s) {
  const size_t smem = (size_t)3 * G.M * T * sizeof(double);
  const unsigned nb = (unsigned)((G.ncol + T - 1) / T);
  cudaError_t e;
  if (stage == 3) {
    e = cudaFuncSetAttribute(k_stage<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_stage<N, true><<<nb, T, smem, s>>>(qn, R1, R2, q2, out, G, R, F, sc, tb);
  } else {
    e = cudaFuncSetAttribute(k_stage<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_stage<N, false><<<nb, T, smem, s>>>(qn, R1, R2, q2, out, G, R, F, sc, tb);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_factor(const Geom& G, const RefLev& R, double lam, Factors F,
                          unsigned* status, cudaStream_t s) {
  const int bs = 128;
  k_factor<<<(unsigned)((G.ncol + bs - 1) / bs), bs, 0, s>>>(G, R, lam, F, status);
  return cudaGetLastError();
}

cudaError_t launch_solve(const double* b, double* x, const Geom& G, Factors F, int T,
                         cudaStream_t s) {
  switch (G.N) {
    case 1: return launch_solve_n<1>(b, x, G, F, T, s);
    case 2: return launch_solve_n<2>(b, x, G, F, T, s);
    case 3: return launch_solve_n<3>(b, x, G, F, T, s);
    case 4: return launch_solve_n<4>(b, x, G, F, T, s);
    case 5: return launch_solve_n<5>(b, x, G, F, T, s);
    case 6: return launch_solve_n<6>(b, x, G, F, T, s);
    case 7: return launch_solve_n<7>(b, x, G, F, T, s);
    case 8: return launch_solve_n<8>(b, x, G, F, T, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stage(int stage, const double* qn, const double* R1, const double* R2,
                         const double* q2, double* out, const Geom& G, const RefLev& R,
                         Factors F, const StageCoef& sc, const StageTab& tb, int T,
                         cudaStream_t s) {
  switch (G.N) {
    case 1: return launch_stage_n<1>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    case 2: return launch_stage_n<2>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    case 3: return launch_stage_n<3>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    case 4: return launch_stage_n<4>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    case 5: return launch_stage_n<5>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    case 6: return launch_stage_n<6>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    case 7: return launch_stage_n<7>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    case 8: return launch_stage_n<8>(stage, qn, R1, R2, q2, out, G, R, F, sc, tb, T, s);
    default: return cudaErrorInvalidValue;
  }
}
