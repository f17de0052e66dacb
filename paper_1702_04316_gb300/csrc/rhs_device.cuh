// Device code of the explicit right-hand side, shared by the single-mesh kernels (rhs.cu)
// and the persistent ensemble kernels (batch.cu).  See rhs.cu for the method.
#pragma once
#include "numa_internal.cuh"

namespace numa_dev {

// ---- FP64 <-> FP32 conversions on the integer pipe ---------------------------------------------
// On GB300 the conversion instructions between FP64 and FP32 issue at about the FP64 pipe's
// rate (two a clock per SM, like a multiply-add) and compete with the FP64 arithmetic of the
// kernels around them.  These two do the same conversions on the IEEE-754 bit patterns with
// integer instructions and return the same bits (NaN payloads aside: a NaN stays a NaN).
// They pay where the FP64 pipe is the bound (the FP32 forms' pre-pass and column stages:
// 0.232 -> 0.158 ms and 0.852 -> 0.809 ms per launch on 96 x 96 x 12 elements, N = 4), not
// in the FP32 right-hand side, whose FP64 pipe is mostly idle and whose issue slots are
// not (0.36 -> 0.43 ms there with them).
//
// f32_of: round to nearest, ties to even.  The 52-bit fraction keeps its top 23 bits; the
// 29 bits below decide the rounding, whose carry may run into the exponent (up to infinity).
// Results below 2^-126 are FP32 subnormals: the 53-bit significand is shifted right with the
// same rounding.
__device__ __forceinline__ float f32_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned s = hi & 0x80000000u;
  const int ed = (int)((hi >> 20) & 0x7ffu);
  const int e = ed - 896;                         // FP32 biased exponent (1023 - 127 = 896)
  if (e >= 1) {
    if (e >= 255)                                 // beyond FP32's range, infinity or NaN
      return __uint_as_float(s | ((ed == 0x7ff && (b << 12)) ? 0x7fffffffu : 0x7f800000u));
    unsigned r = ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    r += (rem > 0x10000000u) | ((rem == 0x10000000u) & (r & 1u));
    return __uint_as_float(s | r);
  }
  const int sh = 30 - e;                          // value = significand * 2^-149 >> sh
  if (sh >= 54) return __uint_as_float(s);
  const unsigned long long m = (1ull << 52) | (b & 0xfffffffffffffull);
  unsigned long long k = m >> sh;
  const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  k += (rem > half) | ((rem == half) & (k & 1ull));
  return __uint_as_float(s | (unsigned)k);
}

// f64_of: exact.  A subnormal float is normalised with its leading one.
__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u, ef = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi, lo;
  if (ef - 1u < 254u) {                           // normal
    hi = s | ((ef + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (ef == 255u) {                        // infinity, NaN
    hi = s | 0x7ff00000u | (m ? 0x80000u : 0u);
    lo = 0u;
  } else if (m == 0u) {                           // zero
    hi = s;
    lo = 0u;
  } else {                                        // subnormal: m 2^-149
    const int p = 31 - __clz(m);
    const unsigned long long fr = (unsigned long long)(m ^ (1u << p)) << (52 - p);
    hi = s | ((unsigned)(p + 874) << 20) | (unsigned)(fr >> 32);
    lo = (unsigned)fr;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// x as a double (exact); the identity for a double.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f64_of(x); }

// 1 / x in FP64 by Newton's method for the reciprocal from an FP32 seed, with the
// third-order step: y0 = rcp.approx of x narrowed by truncation (relative error below
// 2^-21), e = 1 - x y0, y = y0 (1 + e + e^2), whose error is about e^3 < 2^-63.  The result
// lies within one unit in the last place of the correctly rounded 1 / x, for three FP64
// multiply-adds (the seed runs on the integer pipe and the special-function unit).  Where x
// or 1 / x leaves the normal FP32 range (zeros, infinities and NaN included) it divides.
__device__ __forceinline__ double recip(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ed = (hi >> 20) & 0x7ffu;
  if (ed - 897u >= 252u) return 1.0 / x;            // x outside [2^-126, 2^126): x or 1 / x
                                                    // not a normal float
  const float xf = __uint_as_float((hi & 0x80000000u) | ((ed - 896u) << 23) |
                                   ((hi & 0xfffffu) << 3) | (lo >> 29));
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
  const double y0 = f64_of(yf);
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }


// ---- equation of state ---------------------------------------------------------------------
// P' = P(rho0 + rho', theta0 + theta') - P0 without cancellation:
//   (rho theta)/(rho0 theta0) = (1 + a)(1 + b),  a = rho'/rho0,  b = theta'/theta0,
//   P' = P0 ((1 + x)^gamma - 1),  x = a + b + a b.
// The binomial series sum_k C(gamma, k) x^k is used: five terms for |x| <= 2^-10 (truncation
// below 5e-18 relative; x is about P'/(gamma P0), of order 1e-3 or less in atmospheric
// flows), nine for |x| <= 1/64 (below 1e-19); otherwise P0 expm1(gamma log1p(x)).  The
// choice is made per node, so a node's P' does not depend on which nodes share its warp.
struct EosSeries {
  double c[9];   // C(gamma, k), k = 1..9
};

// P' at level lev from rho' and theta' (x = a + b + a b as above).  Where |x| <= 2^-10 the
// five-term series runs with P0 folded into its coefficients (R.P0c: one multiplication
// fewer); otherwise P0 times the nine-term series or expm1(gamma log1p(x)).  |x| is compared
// on the bit pattern without its sign, which orders like |x| for every x that is not a NaN:
// integer instructions instead of FP64 comparisons.
__device__ __forceinline__ double eos_pp(double rp, double tp, int lev, const RefLev& R,
                                         const EosSeries& S) {
  const double a = rp * R.inv_rho0[lev];
  const double b = tp * R.inv_theta0[lev];
  const double x = fma(a, b, a + b);
  const unsigned long long ax = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  if (ax <= 0x3F50000000000000ull) {            // 2^-10
    const double* k = R.P0c + (long long)lev * 5;
    double p = __ldg(k + 4);
#pragma unroll
    for (int j = 3; j >= 0; --j) p = fma(p, x, __ldg(k + j));
    return p * x;
  }
  double r;
  if (ax <= 0x3F90000000000000ull) {            // 2^-6
    double p = S.c[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) p = fma(p, x, S.c[k]);
    r = p * x;
  } else {
    r = expm1(NUMA_GAMMA * log1p(x));
  }
  return R.P0[lev] * r;
}

// P' of node g of state q (FP64).
__device__ __forceinline__ double eos_node(const double* __restrict__ q, long long g, const Geom& G,
                                           const RefLev& R, const EosSeries& S) {
  return eos_pp(q[g], q[4 * G.nnode + g], (int)(g % G.M), R, S);
}

// The series coefficients C(gamma, k), k = 1..9.
inline EosSeries eos_series() {
  EosSeries S;
  double c = 1.0;
  for (int k = 1; k <= 9; ++k) {
    c *= (NUMA_GAMMA - k + 1) / k;
    S.c[k - 1] = c;
  }
  return S;
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

// d/d(axis) of the six fields at node g.  ZINIT: d[0] and d[4] start from i0 and i4, the
// addition taken by the first multiply-add (along z the tendencies add the reference
// gradients d(rho0)/dz and d(theta0)/dz to them).
template <int N, typename RT, bool ZINIT = false>
__device__ __forceinline__ void axis_derivs(const RT* const* F, long long g, long long stride,
                                            int cls, const Taps<N, RT>& T, RT* d,
                                            const double* i0 = nullptr, const double* i4 = nullptr) {
  auto first = [&](int f, const RT* p) {
    const RT a = __ldg(p + T.o[0] * stride);
    if (ZINIT && (f == 0 || f == 4)) return fma(T.c[0], a, (RT)__ldg(f == 0 ? i0 : i4));
    return T.c[0] * a;
  };
  if (cls == CLS_IFACE) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const RT* p = F[f] + g;
      RT acc = first(f, p);
#pragma unroll
      for (int t = 1; t < 2 * N; ++t) acc = fma(T.c[t], __ldg(p + T.o[t] * stride), acc);
      d[f] = acc;
    }
  } else if (cls == CLS_WALL) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const RT* p = F[f] + g;
      RT acc = first(f, p);
#pragma unroll
      for (int t = 1; t <= N; ++t) acc = fma(T.c[t], __ldg(p + T.o[t] * stride), acc);
      d[f] = acc;
    }
  } else {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const RT* p = F[f] + g;
      RT acc = first(f, p);
#pragma unroll
      for (int t = 1; t < N; ++t) acc = fma(T.c[t], __ldg(p + T.o[t] * stride), acc);
      d[f] = acc;
    }
  }
}

// The Set2NC tendencies at node g from the DSS'd derivatives of the six fields (dx, dy, dz:
// rho', u, v, w, theta', P'; dz[0] and dz[4] with d(rho0)/dz and d(theta0)/dz added), and
// the epilogue.  RT: arithmetic type; fld: the fields read at
// g (rho', u, v, w; stride nnode); OT: type written in mode 0.  Modes 1 and 2 read and
// write the FP64 state; R1, R2 are OT arrays.
template <typename RT, typename OT, typename FT>
__device__ __forceinline__ void rhs_point(long long g, int ix, int iy, int iz, const double* __restrict__ q,
                                          const FT* __restrict__ fld, const RT* dx, const RT* dy,
                                          const RT* dz, OT* out0, double* out, const Geom& G,
                                          const RefLev& R, const RhsEpilogue& ep);

template <typename RT, typename OT>
__device__ __forceinline__ void rhs_store(long long g, const RT* t, const double* __restrict__ q,
                                          OT* out0, double* out, const Geom& G,
                                          const RhsEpilogue& ep);

// The same with rho', u, v, w at g given as values.
template <typename RT, typename OT>
__device__ __forceinline__ void rhs_point_v(long long g, int ix, int iy, int iz,
                                            const double* __restrict__ q, RT r_, RT u_, RT v_,
                                            RT w_, const RT* dx, const RT* dy, const RT* dz,
                                            OT* out0, double* out, const Geom& G, const RefLev& R,
                                            const RhsEpilogue& ep) {
  const RT rho = (RT)R.rho0[iz] + r_;
  const RT irho = recip(rho);
  const RT grav = (RT)NUMA_GRAV;
  // the tendencies are minus sums of products; the minus sign sits on the operands (-x y =
  // (-x) y and -fma(a, b, c) = fma(-a, b, -c) exactly, rounding being symmetric), so no
  // instruction negates a result
  const RT nu = -u_, nv = -v_, nw = -w_;
  // dz[0] and dz[4] arrive with d(rho0)/dz and d(theta0)/dz added (rhs_node)
  RT t_r = fma(nu, dx[0], fma(nv, dy[0], fma(nw, dz[0], -rho * (dx[1] + dy[2] + dz[3]))));
  RT t_u = fma(nu, dx[1], fma(nv, dy[1], fma(nw, dz[1], -dx[5] * irho)));
  RT t_v = fma(nu, dx[2], fma(nv, dy[2], fma(nw, dz[2], -dy[5] * irho)));
  RT t_w = fma(nu, dx[3], fma(nv, dy[3], fma(nw, dz[3], fma(-grav, r_, -dz[5]) * irho)));
  RT t_t = fma(nu, dx[4], fma(nv, dy[4], nw * dz[4]));
  // walls: no normal flow
  if (ix == 0 || ix == G.nxg - 1) t_u = (RT)0;
  if (iy == 0 || iy == G.nyg - 1) t_v = (RT)0;
  if (iz == 0 || iz == G.M - 1) t_w = (RT)0;

  const RT t[5] = {t_r, t_u, t_v, t_w, t_t};
  rhs_store<RT, OT>(g, t, q, out0, out, G, ep);
}

// The epilogue of a right-hand side at node g: mode 0 writes the tendencies t (to out0);
// modes 1-3 combine them with states and earlier tendencies into out (RhsEpilogue).
template <typename RT, typename OT>
__device__ __forceinline__ void rhs_store(long long g, const RT* t, const double* __restrict__ q,
                                          OT* out0, double* out, const Geom& G,
                                          const RhsEpilogue& ep) {
  const long long nn = G.nnode;
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
  } else if (ep.mode == 2) {
    const OT* R1 = (const OT*)ep.R1;
    const OT* R2 = (const OT*)ep.R2;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const long long o = f * nn + g;
      out[o] = fma(ep.b3dt, (double)t[f], fma(ep.b2dt, (double)R2[o], fma(ep.b1dt, (double)R1[o], ep.u0[o])));
    }
  } else {
    const double* R1 = (const double*)ep.R1;
    const double* R2 = (const double*)ep.R2;
    const double* R3 = (const double*)ep.R3;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const long long o = f * nn + g;
      out[o] = fma(ep.b4dt, (double)t[f],
                   fma(ep.b3dt, R3[o], fma(ep.b2dt, R2[o], fma(ep.b1dt, R1[o], ep.u0[o]))));
    }
  }
}

template <typename RT, typename OT, typename FT>
__device__ __forceinline__ void rhs_point(long long g, int ix, int iy, int iz, const double* __restrict__ q,
                                          const FT* __restrict__ fld, const RT* dx, const RT* dy,
                                          const RT* dz, OT* out0, double* out, const Geom& G,
                                          const RefLev& R, const RhsEpilogue& ep) {
  const long long nn = G.nnode;
  rhs_point_v<RT, OT>(g, ix, iy, iz, q, (RT)fld[g], (RT)fld[nn + g], (RT)fld[2 * nn + g],
                      (RT)fld[3 * nn + g], dx, dy, dz, out0, out, G, R, ep);
}

// One node of the right-hand side (thread index tid of the class-sorted order, or of the
// natural order when perm is NULL).  sD, sDl, sDr: the three axes' derivative rows
// (axis a at sD + a*(N+1)^2, sDl + a*(N+1), sDr + a*(N+1)), normally in shared memory.
// RT: type of the stencil fields and of the arithmetic (double: the FP64 method, fields =
// the state and P'; float: the mixed-precision form, fields = the FP32 copies from
// k_prep32).  fld holds rho', u, v, w, theta' (stride nnode), fp holds P'.  OT: type
// written in mode 0.  Modes 1 and 2 read and write the FP64 state; R1, R2 are OT arrays.
template <int N, typename RT, typename OT>
__device__ __forceinline__ void rhs_node(long long tid, const double* __restrict__ q,
                                         const RT* __restrict__ fld, const RT* __restrict__ fp,
                                         OT* out0, double* out, const int* __restrict__ perm,
                                         long long nthreads, const Geom& G, const RefLev& R,
                                         const RhsEpilogue& ep, const RT* sD, const RT* sDl,
                                         const RT* sDr) {
  constexpr int Nq = N + 1;
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
    int cls = axis_taps<N, RT>(ix, G.nex, sD, sDl, sDr, T);
    axis_derivs<N, RT>(Fld, g, sxs, cls, T, dx);
    cls = axis_taps<N, RT>(iy, G.ney, sD + Nq * Nq, sDl + Nq, sDr + Nq, T);
    axis_derivs<N, RT>(Fld, g, sys, cls, T, dy);
    cls = axis_taps<N, RT>(iz, G.nez, sD + 2 * Nq * Nq, sDl + 2 * Nq, sDr + 2 * Nq, T);
    // the z derivatives of rho' and theta' start from d(rho0)/dz and d(theta0)/dz, the
    // reference gradients the tendencies add to them (one multiply-add instead of an add)
    axis_derivs<N, RT, true>(Fld, g, 1, cls, T, dz, R.drho0 + iz, R.dtheta0 + iz);
  }
  rhs_point<RT, OT, RT>(g, ix, iy, iz, q, fld, dx, dy, dz, out0, out, G, R, ep);
}

// The three axes' derivative rows of C into shared memory (cast to RT).
template <int N, typename RT>
__device__ __forceinline__ void load_rows(const Coef3& C, RT* sD, RT* sDl, RT* sDr) {
  constexpr int Nq = N + 1;
  for (int t = threadIdx.x; t < Nq * Nq; t += blockDim.x) {
    sD[t] = (RT)C.x.D[t];
    sD[Nq * Nq + t] = (RT)C.y.D[t];
    sD[2 * Nq * Nq + t] = (RT)C.z.D[t];
  }
  for (int t = threadIdx.x; t < Nq; t += blockDim.x) {
    sDl[t] = (RT)C.x.Dl[t]; sDr[t] = (RT)C.x.Dr[t];
    sDl[Nq + t] = (RT)C.y.Dl[t]; sDr[Nq + t] = (RT)C.y.Dr[t];
    sDl[2 * Nq + t] = (RT)C.z.Dl[t]; sDr[2 * Nq + t] = (RT)C.z.Dr[t];
  }
}

}  // namespace numa_dev
