// Explicit right-hand side R(q) of the Set2NC perturbation equations (Sec. "Equation
// Set2NC"), continuous Galerkin on LGL nodes with direct stiffness summation.
//
// Owner-computes formulation.  On the uniform box every coefficient of the tendencies
// (u, v, w, rho, 1/rho, the reference fields) is a continuous nodal field, so DSS of the
// element-local tendency equals the pointwise tendency evaluated with DSS'd derivatives.
// The DSS'd x-derivative of a continuous field at a global node only involves the
// elements adjacent along x: elements that share the node across a y- or z-face see the
// same polynomial along the x-line through it, so they contribute identical values that
// the mass weighting averages back to themselves.  Hence, per axis,
//   d_x f (node) = D_x-row of its element                       (interior / wall nodes)
//                = (w_N d_left + w_0 d_right) / (w_N + w_0)      (element interfaces),
// which is what the element-by-element gather/scatter of Algorithm 2 + DSS produces.
//
// GB300 is FP64-issue bound here (2 FP64 FMA per clock per SM), so the kernel minimises
// FP64 instructions:
//  * LGL rows of interior nodes have a zero diagonal: N taps instead of N+1;
//  * at an interface the two elements' weights are equal (w_0 = w_N) and D_00 = -D_NN, so
//    the shared node cancels: 2N taps instead of 2N+2;
//  * threads run in a permuted node order in which every warp holds nodes of one class
//    (interior / interface / wall) per axis, so no warp executes both tap counts.
#include <vector>

#include "numa_internal.cuh"

namespace {

// ---- equation of state ---------------------------------------------------------------------
// P' = P(rho0 + rho', theta0 + theta') - P0 without cancellation:
//   (rho theta)/(rho0 theta0) = (1 + a)(1 + b),  a = rho'/rho0,  b = theta'/theta0,
//   P' = P0 ((1 + x)^gamma - 1),  x = a + b + a b.
// For |x| <= 1/64 the binomial series sum_{k=1..9} C(gamma, k) x^k is used (truncation
// below 1e-19 relative); otherwise P0 expm1(gamma log1p(x)).
struct EosSeries {
  double c[9];   // C(gamma, k), k = 1..9
};

__global__ void k_pressure(const double* __restrict__ q, double* __restrict__ Pp, Geom G,
                           RefLev R, double gamma, EosSeries S) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const int iz = (int)(g % G.M);
  const double a = q[g] * R.inv_rho0[iz];
  const double b = q[4 * G.nnode + g] * R.inv_theta0[iz];
  const double x = fma(a, b, a + b);
  double r;
  if (fabs(x) <= 0.015625) {
    double p = S.c[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) p = fma(p, x, S.c[k]);
    r = p * x;
  } else {
    r = expm1(gamma * log1p(x));
  }
  Pp[g] = R.P0[iz] * r;
}

// Mixed-precision form: P' in FP64 (as above), then FP32 copies of the six stencil fields
// (rho', u, v, w, theta', P') for the FP32 right-hand side.
__global__ void k_prep32(const double* __restrict__ q, float* __restrict__ F32, Geom G, RefLev R,
                         double gamma, EosSeries S) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long nn = G.nnode;
  const int iz = (int)(g % G.M);
  const double rp = q[g], tp = q[4 * nn + g];
  const double a = rp * R.inv_rho0[iz];
  const double b = tp * R.inv_theta0[iz];
  const double x = fma(a, b, a + b);
  double r;
  if (fabs(x) <= 0.015625) {
    double p = S.c[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) p = fma(p, x, S.c[k]);
    r = p * x;
  } else {
    r = expm1(gamma * log1p(x));
  }
  F32[g] = (float)rp;
  F32[nn + g] = (float)q[nn + g];
  F32[2 * nn + g] = (float)q[2 * nn + g];
  F32[3 * nn + g] = (float)q[3 * nn + g];
  F32[4 * nn + g] = (float)tp;
  F32[5 * nn + g] = (float)(R.P0[iz] * r);
}

// ---- right-hand side ---------------------------------------------------------------------
enum { CLS_INTERIOR = 0, CLS_IFACE = 1, CLS_WALL = 2 };

template <int N, typename RT>
struct Taps {
  RT c[2 * N + 1];
  int o[2 * N + 1];
};

// Row of the DSS'd derivative at axis index idx: coefficients and node offsets relative to
// the node itself (in units of the axis stride).  The class is uniform across a warp.
template <int N, typename RT>
__device__ __forceinline__ int axis_taps(int idx, int nel, const RT* sD, const RT* sDl,
                                         const RT* sDr, Taps<N, RT>& T) {
  constexpr int Nq = N + 1;
  int e, i;
  axis_owner(idx, N, nel, e, i);
  if (i == 0 && e > 0) {
#pragma unroll
    for (int t = 0; t < N; ++t) {          // left element, its nodes 0..N-1
      T.c[t] = sDl[t];
      T.o[t] = t - N;
    }
#pragma unroll
    for (int t = 1; t <= N; ++t) {         // right element, its nodes 1..N
      T.c[N - 1 + t] = sDr[t];
      T.o[N - 1 + t] = t;
    }
    return CLS_IFACE;
  }
  if (i == 0 || i == N) {                  // wall: the full row of the one element
#pragma unroll
    for (int t = 0; t <= N; ++t) {
      T.c[t] = sD[i * Nq + t];
      T.o[t] = t - i;
    }
    return CLS_WALL;
  }
#pragma unroll
  for (int t = 0; t < N; ++t) {            // interior: the zero diagonal dropped
    const int n = t + (t >= i ? 1 : 0);
    T.c[t] = sD[i * Nq + n];
    T.o[t] = n - i;
  }
  return CLS_INTERIOR;
}

// d/d(axis) of the six fields at node g.
template <int N, typename RT>
__device__ __forceinline__ void axis_derivs(const RT* const* F, long long g, long long stride,
                                            int cls, const Taps<N, RT>& T, RT* d) {
  if (cls == CLS_IFACE) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const RT* p = F[f] + g;
      RT acc = T.c[0] * __ldg(p + T.o[0] * stride);
#pragma unroll
      for (int t = 1; t < 2 * N; ++t) acc = fma(T.c[t], __ldg(p + T.o[t] * stride), acc);
      d[f] = acc;
    }
  } else if (cls == CLS_WALL) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const RT* p = F[f] + g;
      RT acc = T.c[0] * __ldg(p + T.o[0] * stride);
#pragma unroll
      for (int t = 1; t <= N; ++t) acc = fma(T.c[t], __ldg(p + T.o[t] * stride), acc);
      d[f] = acc;
    }
  } else {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const RT* p = F[f] + g;
      RT acc = T.c[0] * __ldg(p + T.o[0] * stride);
#pragma unroll
      for (int t = 1; t < N; ++t) acc = fma(T.c[t], __ldg(p + T.o[t] * stride), acc);
      d[f] = acc;
    }
  }
}

// RT: type of the stencil fields and of the arithmetic (double: the FP64 method, fields =
// the state and P'; float: the mixed-precision form, fields = the FP32 copies from
// k_prep32).  fld holds rho', u, v, w, theta' (stride nnode), fp holds P'.  OT: type
// written in mode 0.  Modes 1 and 2 read and write the FP64 state; R1, R2 are OT arrays.
template <int N, typename RT, typename OT>
__global__ void __launch_bounds__(256) k_rhs(const double* __restrict__ q,
                                             const RT* __restrict__ fld,
                                             const RT* __restrict__ fp, OT* out0, double* out,
                                             const int* __restrict__ perm, long long nthreads,
                                             Geom G, Coef3 C, RefLev R, RhsEpilogue ep) {
  constexpr int Nq = N + 1;
  __shared__ RT sD[3][Nq * Nq], sDl[3][Nq], sDr[3][Nq];
  for (int t = threadIdx.x; t < Nq * Nq; t += blockDim.x) {
    sD[0][t] = (RT)C.x.D[t];
    sD[1][t] = (RT)C.y.D[t];
    sD[2][t] = (RT)C.z.D[t];
  }
  for (int t = threadIdx.x; t < Nq; t += blockDim.x) {
    sDl[0][t] = (RT)C.x.Dl[t]; sDr[0][t] = (RT)C.x.Dr[t];
    sDl[1][t] = (RT)C.y.Dl[t]; sDr[1][t] = (RT)C.y.Dr[t];
    sDl[2][t] = (RT)C.z.Dl[t]; sDr[2][t] = (RT)C.z.Dr[t];
  }
  __syncthreads();
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= nthreads) return;
  const int gi = perm ? perm[tid] : (int)tid;
  if (gi < 0) return;                       // padding of a class group
  const long long g = gi;
  const long long nn = G.nnode;
  const long long col = g / G.M;
  const int iz = (int)(g - col * G.M);
  const int iy = (int)(col / G.nxg);
  const int ix = (int)(col - (long long)iy * G.nxg);
  const long long sxs = G.M, sys = (long long)G.nxg * G.M;

  // fields: 0 rho', 1 u, 2 v, 3 w, 4 theta', 5 P'
  const RT* Fld[6] = {fld, fld + nn, fld + 2 * nn, fld + 3 * nn, fld + 4 * nn, fp};
  RT dx[6], dy[6], dz[6];
  {
    Taps<N, RT> T;
    int cls = axis_taps<N, RT>(ix, G.nex, sD[0], sDl[0], sDr[0], T);
    axis_derivs<N, RT>(Fld, g, sxs, cls, T, dx);
    cls = axis_taps<N, RT>(iy, G.ney, sD[1], sDl[1], sDr[1], T);
    axis_derivs<N, RT>(Fld, g, sys, cls, T, dy);
    cls = axis_taps<N, RT>(iz, G.nez, sD[2], sDl[2], sDr[2], T);
    axis_derivs<N, RT>(Fld, g, 1, cls, T, dz);
  }
  const RT r_ = fld[g], u_ = fld[nn + g], v_ = fld[2 * nn + g], w_ = fld[3 * nn + g];
  const RT rho = (RT)R.rho0[iz] + r_;
  const RT irho = (RT)1 / rho;
  const RT grav = (RT)NUMA_GRAV;
  RT t_r = -fma(u_, dx[0], fma(v_, dy[0], fma(w_, dz[0] + (RT)R.drho0[iz], rho * (dx[1] + dy[2] + dz[3]))));
  RT t_u = -fma(u_, dx[1], fma(v_, dy[1], fma(w_, dz[1], dx[5] * irho)));
  RT t_v = -fma(u_, dx[2], fma(v_, dy[2], fma(w_, dz[2], dy[5] * irho)));
  RT t_w = -fma(u_, dx[3], fma(v_, dy[3], fma(w_, dz[3], fma(grav, r_, dz[5]) * irho)));
  RT t_t = -fma(u_, dx[4], fma(v_, dy[4], w_ * (dz[4] + (RT)R.dtheta0[iz])));
  // walls: no normal flow
  if (ix == 0 || ix == G.nxg - 1) t_u = (RT)0;
  if (iy == 0 || iy == G.nyg - 1) t_v = (RT)0;
  if (iz == 0 || iz == G.M - 1) t_w = (RT)0;

  const RT t[5] = {t_r, t_u, t_v, t_w, t_t};
  if (ep.mode == 0) {
#pragma unroll
    for (int f = 0; f < 5; ++f) out0[f * nn + g] = (OT)t[f];
  } else if (ep.mode == 1) {
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      double val = fma(ep.beta_dt, (double)t[f], ep.one_minus_alpha * q[f * nn + g]);
      if (ep.use_u0) val = fma(ep.alpha, ep.u0[f * nn + g], val);
      out[f * nn + g] = val;
    }
  } else {
    const OT* R1 = (const OT*)ep.R1;
    const OT* R2 = (const OT*)ep.R2;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const long long o = f * nn + g;
      out[o] = fma(ep.b3dt, (double)t[f], fma(ep.b2dt, (double)R2[o], fma(ep.b1dt, (double)R1[o], ep.u0[o])));
    }
  }
}

template <int N, typename RT, typename OT>
cudaError_t launch_rhs_n(const double* q, const RT* fld, const RT* fp, OT* out0, double* out,
                         const int* perm, long long nthreads, const Geom& G, const Coef3& C,
                         const RefLev& R, const RhsEpilogue& ep, cudaStream_t s) {
  const int bs = 256;
  k_rhs<N, RT, OT><<<(unsigned)((nthreads + bs - 1) / bs), bs, 0, s>>>(q, fld, fp, out0, out,
                                                                        perm, nthreads, G, C, R, ep);
  return cudaGetLastError();
}

template <typename RT, typename OT>
cudaError_t launch_rhs_t(const double* q, const RT* fld, const RT* fp, OT* out0, double* out,
                         const int* perm, long long nthreads, const Geom& G, const Coef3& C,
                         const RefLev& R, const RhsEpilogue& ep, cudaStream_t s) {
  switch (G.N) {
    case 1: return launch_rhs_n<1, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    case 2: return launch_rhs_n<2, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    case 3: return launch_rhs_n<3, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    case 4: return launch_rhs_n<4, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    case 5: return launch_rhs_n<5, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    case 6: return launch_rhs_n<6, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    case 7: return launch_rhs_n<7, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    case 8: return launch_rhs_n<8, RT, OT>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep, s);
    default: return cudaErrorInvalidValue;
  }
}

EosSeries eos_series() {
  EosSeries S;
  double c = 1.0;
  for (int k = 1; k <= 9; ++k) {
    c *= (NUMA_GAMMA - k + 1) / k;
    S.c[k - 1] = c;
  }
  return S;
}

int node_class(int idx, int N, int nel) {
  int e, i;
  axis_owner(idx, N, nel, e, i);
  if (i == 0 && e > 0) return CLS_IFACE;
  if (i == 0 || i == N) return CLS_WALL;
  return CLS_INTERIOR;
}

}  // namespace

cudaError_t launch_pressure(const double* q, double* Pp, const Geom& G, const RefLev& R,
                            cudaStream_t s) {
  const int bs = 256;
  const long long nb = (G.nnode + bs - 1) / bs;
  k_pressure<<<(unsigned)nb, bs, 0, s>>>(q, Pp, G, R, NUMA_GAMMA, eos_series());
  return cudaGetLastError();
}

cudaError_t launch_prep32(const double* q, float* F32, const Geom& G, const RefLev& R,
                          cudaStream_t s) {
  const int bs = 256;
  const long long nb = (G.nnode + bs - 1) / bs;
  k_prep32<<<(unsigned)nb, bs, 0, s>>>(q, F32, G, R, NUMA_GAMMA, eos_series());
  return cudaGetLastError();
}

cudaError_t launch_rhs(const double* q, const double* Pp, double* out, const int* perm,
                       long long nthreads, const Geom& G, const Coef3& C, const RefLev& R,
                       const RhsEpilogue& ep, cudaStream_t s) {
  return launch_rhs_t<double, double>(q, q, Pp, out, out, perm, nthreads, G, C, R, ep, s);
}

cudaError_t launch_rhs32d(const double* q, const float* F32, double* out0, const Geom& G,
                          const Coef3& C, const RefLev& R, cudaStream_t s) {
  RhsEpilogue ep{};
  ep.mode = 0;
  return launch_rhs_t<float, double>(q, F32, F32 + 5 * G.nnode, out0, out0, nullptr, G.nnode, G,
                                     C, R, ep, s);
}

cudaError_t launch_rhs32(const double* q, const float* F32, float* out32, double* out,
                         const int* perm, long long nthreads, const Geom& G, const Coef3& C,
                         const RefLev& R, const RhsEpilogue& ep, cudaStream_t s) {
  return launch_rhs_t<float, float>(q, F32, F32 + 5 * G.nnode, out32, out, perm, nthreads, G,
                                    C, R, ep, s);
}

// Class-sorted thread order: the (x, y) node plane is cut into tiles of kTile x kTile
// elements (all levels); inside a tile, nodes are grouped by (x-class, y-class, z-class),
// ascending node id inside a group, and each group is padded with -1 to a multiple of 32,
// so that no warp mixes classes while consecutive blocks stay within one tile (its
// stencil neighbours are still in L2).
static const int kTile = 4;

template <typename Emit>
static void walk_rhs_perm(const Geom& G, Emit emit) {
  const int tn = kTile * G.N;
  std::vector<int> cz(G.M);
  for (int iz = 0; iz < G.M; ++iz) cz[iz] = node_class(iz, G.N, G.nez);
  std::vector<long long> bucket[27];
  for (int y0 = 0; y0 < G.nyg; y0 += tn) {
    const int y1 = (G.nyg - y0 <= tn + 1) ? G.nyg : y0 + tn;   // the last tile takes the end node
    for (int x0 = 0; x0 < G.nxg; x0 += tn) {
      const int x1 = (G.nxg - x0 <= tn + 1) ? G.nxg : x0 + tn;
      for (auto& b : bucket) b.clear();
      for (int iy = y0; iy < y1; ++iy) {
        const int cy = node_class(iy, G.N, G.ney);
        for (int ix = x0; ix < x1; ++ix) {
          const int cx = node_class(ix, G.N, G.nex);
          const long long base = ((long long)iy * G.nxg + ix) * G.M;
          for (int iz = 0; iz < G.M; ++iz) bucket[cx * 9 + cy * 3 + cz[iz]].push_back(base + iz);
        }
      }
      for (auto& b : bucket) {
        if (b.empty()) continue;
        for (long long g : b) emit(g);
        for (size_t p = b.size(); p % 32; ++p) emit(-1);
      }
      if (x1 == G.nxg) break;
    }
    if (y1 == G.nyg) break;
  }
}

long long rhs_perm_size(const Geom& G) {
  long long n = 0;
  walk_rhs_perm(G, [&](long long) { ++n; });
  return n;
}

void build_rhs_perm(const Geom& G, int* out) {
  long long n = 0;
  walk_rhs_perm(G, [&](long long g) { out[n++] = (int)g; });
}
