// Double-float ("DF") variant of the explicit right-hand side (precision NUMA_PREC_DF).
//
// GB300 issues FP64 at 2 FMA per clock per SM and FP32 at 128, and the FP64 right-hand side
// is bound by the FP64 pipe (93 % busy).  Here the derivative sums (about 90 multiply-adds
// per node at N = 4) and the pointwise products of the Set2NC tendencies (u.grad f,
// rho div u, grad P' / rho) run in double-float arithmetic: every value is an unevaluated
// sum hi + lo of two FP32 numbers (about 48 significant bits), products by Dekker's method
// (the exact residual of a product from one fused multiply-add), sums by Knuth's TwoSum,
// the low-order parts accumulated without renormalisation.  FP64 is left with rho, 1 / rho,
// g rho', the five tendencies formed from their pairs, and the epilogue; the equation of
// state, the column solves and the state stay FP64.
//
// A pre-pass writes every stencil field -- rho', u, v, w, theta' and P' from the FP64
// equation of state -- as a (hi, lo) pair of FP32 numbers (see split): 8 bytes per value, as
// a double, so the stencil reads the same bytes as the FP64 kernel.  The derivative rows are
// split the same way, once per CTA, into shared memory.
#include <algorithm>

#include "numa_internal.cuh"
#include "rhs_device.cuh"

namespace {
using namespace numa_dev;

// TwoSum (Knuth): s + e = a + b exactly.  The round-to-nearest intrinsics keep the compiler
// from fusing or reassociating the steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (ah, al) += (ch + cl) (fh + fl): the product's high part ph = fl32(ch fh) with its exact
// residual ch fh - ph from one fused multiply-add (Dekker), the cross terms ch fl + cl fh
// added to it (cl fl, below 2^-48 relative, is dropped), ph added to ah by TwoSum and all
// low-order parts to al.
__device__ __forceinline__ void df_mac(float ch, float cl, float fh, float fl, float& ah,
                                       float& al) {
  const float ph = __fmul_rn(ch, fh);
  const float pe = __fmaf_rn(ch, fh, -ph);
  const float pl = __fmaf_rn(ch, fl, __fmaf_rn(cl, fh, pe));
  float s, e;
  two_sum(ah, ph, s, e);
  ah = s;
  al = __fadd_rn(al, __fadd_rn(e, pl));
}

// On GB300 the FP64 <-> FP32 conversion instructions run at about the FP64 pipe's rate, so
// the splits and recombinations below work on the IEEE-754 bit patterns with integer
// instructions instead.
//
// split: hi = x with its significand truncated to 24 bits, lo = the remaining 29 bits,
// truncated to a 24-bit float: x - hi - lo is below 2^-47 |x|.  Magnitudes below 2^-100 are
// taken as 0; magnitudes from 2^128 up and non-finite values become NaN, so that a state
// gone bad stays visible (the model's fields lie far inside both bounds).
__device__ __forceinline__ float2 split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned s = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023;                 // unbiased exponent
  if (e < -100) return make_float2(0.0f, 0.0f);
  if (e > 127) return make_float2(__uint_as_float(0x7fc00000u), 0.0f);   // beyond FP32, or not finite: NaN
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;           // 52-bit fraction
  const float hi = __uint_as_float(s | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
  const unsigned low = (unsigned)(m & 0x1FFFFFFFull);            // 29 bits below hi
  if (low == 0) return make_float2(hi, 0.0f);
  const int p = 31 - __clz(low);                                 // leading one of low
  const int el = e - 52 + p;                                     // its exponent
  if (el < -126) return make_float2(hi, 0.0f);
  const unsigned frac = low ^ (1u << p);
  const unsigned f23 = (p >= 23) ? (frac >> (p - 23)) : (frac << (23 - p));
  return make_float2(hi, __uint_as_float(s | ((unsigned)(el + 127) << 23) | f23));
}

// The double equal to a normal float (exact), or 0 for a zero or subnormal float.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0) return 0.0;
  if (ef == 255) return __longlong_as_double(0x7ff8000000000000ll);     // not finite: NaN
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ef - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// (ah, al) += (bh + bl) for a pair whose parts need not be normalised: TwoSum of the high
// parts, the low parts added to the low accumulator.
__device__ __forceinline__ void df_add(float bh, float bl, float& ah, float& al) {
  float s, e;
  two_sum(ah, bh, s, e);
  ah = s;
  al = __fadd_rn(al, __fadd_rn(e, bl));
}

// The six fields' derivatives along one axis with K taps (the class's exact count), as
// unnormalised (hi, lo) pairs.
template <int K, int N>
__device__ __forceinline__ void derivs_df(const float2* const* F, long long g, long long stride,
                                          const Taps<N, float2>& T, float2* d) {
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const float2* p = F[f] + g;
    float ah = 0.0f, al = 0.0f;
#pragma unroll
    for (int t = 0; t < K; ++t) {
      const float2 v = __ldg(p + T.o[t] * stride);
      df_mac(T.c[t].x, T.c[t].y, v.x, v.y, ah, al);
    }
    d[f] = make_float2(ah, al);
  }
}

template <int N>
__device__ __forceinline__ void axis_derivs_df(const float2* const* F, long long g, long long stride,
                                               int cls, const Taps<N, float2>& T, float2* d) {
  if (cls == CLS_IFACE) derivs_df<2 * N, N>(F, g, stride, T, d);
  else if (cls == CLS_WALL) derivs_df<N + 1, N>(F, g, stride, T, d);
  else derivs_df<N, N>(F, g, stride, T, d);
}

// P' from the FP64 equation of state, and the (hi, lo) pairs of the six stencil fields.
__global__ void k_prep_df(const double* __restrict__ q, float2* __restrict__ F2, Geom G, RefLev R,
                          EosSeries S) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long nn = G.nnode;
#pragma unroll
  for (int f = 0; f < 5; ++f) F2[f * nn + g] = split(q[f * nn + g]);
  F2[5 * nn + g] = split(eos_node(q, g, G, R, S));
}

// One node of the right-hand side (g, at ix, iy, iz).  The three axes run through one copy of
// the derivative code (a loop that is not unrolled): three unrolled copies, each with its three
// tap-count variants, overflowed the instruction cache (ncu: "no instruction" stalls).
template <int N>
__device__ __forceinline__ void rhs_df_node(long long g, const double* __restrict__ q,
                                            const float2* __restrict__ F2, double* out0,
                                            double* out, const Geom& G, const RefLev& R,
                                            const RhsEpilogue& ep, const float2* sD,
                                            const float2* sDl, const float2* sDr) {
  constexpr int Nq = N + 1;
  const long long nn = G.nnode;
  const long long col = g / G.M;
  const int iz = (int)(g - col * G.M);
  const int iy = (int)(col / G.nxg);
  const int ix = (int)(col - (long long)iy * G.nxg);
  const float2* Fld[6] = {F2, F2 + nn, F2 + 2 * nn, F2 + 3 * nn, F2 + 4 * nn, F2 + 5 * nn};
  // FP64: rho = rho0 + rho', 1 / rho and g rho'; everything else in pairs
  const double r_ = q[g];
  const double rho = R.rho0[iz] + r_;
  const double irho = 1.0 / rho;
  const float2 U = split(q[nn + g]), V = split(q[2 * nn + g]), W = split(q[3 * nn + g]);
  const float2 IR = split(irho);
  float2 A[5], DV = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int f = 0; f < 5; ++f) A[f] = make_float2(0.0f, 0.0f);
  // axis a: the six derivatives d, then  A_f += X d_f (X = u, v, w),  DV += d_{1+a},
  // A_{1+a} += (1 / rho) d_5
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    const int ia = a == 0 ? ix : (a == 1 ? iy : iz);
    const int nel = a == 0 ? G.nex : (a == 1 ? G.ney : G.nez);
    const long long stride = a == 0 ? (long long)G.M : (a == 1 ? (long long)G.nxg * G.M : 1LL);
    Taps<N, float2> T;
    const int cls = axis_taps<N, float2>(ia, nel, sD + a * Nq * Nq, sDl + a * Nq, sDr + a * Nq, T);
    float2 d[6];
    axis_derivs_df<N>(Fld, g, stride, cls, T, d);
    if (a == 2) {   // the reference gradients and the buoyancy join the vertical derivatives
      const float2 dr0 = split(R.drho0[iz]), dt0 = split(R.dtheta0[iz]);
      const float2 gr = split(NUMA_GRAV * r_);
      df_add(dr0.x, dr0.y, d[0].x, d[0].y);
      df_add(dt0.x, dt0.y, d[4].x, d[4].y);
      df_add(gr.x, gr.y, d[5].x, d[5].y);
    }
    const float2 X = a == 0 ? U : (a == 1 ? V : W);
#pragma unroll
    for (int f = 0; f < 5; ++f) df_mac(X.x, X.y, d[f].x, d[f].y, A[f].x, A[f].y);
    const float2 dv = a == 0 ? d[1] : (a == 1 ? d[2] : d[3]);
    df_add(dv.x, dv.y, DV.x, DV.y);
#pragma unroll
    for (int f = 1; f <= 3; ++f)
      if (f == 1 + a) df_mac(IR.x, IR.y, d[5].x, d[5].y, A[f].x, A[f].y);
  }
  const float2 RH = split(rho);
  df_mac(RH.x, RH.y, DV.x, DV.y, A[0].x, A[0].y);
  double t[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) t[f] = -(widen(A[f].x) + widen(A[f].y));
  // walls: no normal flow
  if (ix == 0 || ix == G.nxg - 1) t[1] = 0.0;
  if (iy == 0 || iy == G.nyg - 1) t[2] = 0.0;
  if (iz == 0 || iz == G.M - 1) t[3] = 0.0;
  rhs_store<double, double>(g, t, q, out0, out, G, ep);
}

// Five 128-thread CTAs per SM (at most 102 registers): measured fastest against three, four,
// six and eight.  Each CTA splits the derivative rows into shared memory once and then walks
// 128-node chunks of the thread order with a grid stride (a grid of five CTAs per SM), so the
// split and its barrier are not repeated for every 128 nodes.
template <int N>
__global__ void __launch_bounds__(128, 5) k_rhs_df(const double* __restrict__ q,
                                                   const float2* __restrict__ F2, double* out0,
                                                   double* out, const int* __restrict__ perm,
                                                   long long nthreads, Geom G, Coef3 C, RefLev R,
                                                   RhsEpilogue ep) {
  constexpr int Nq = N + 1;
  __shared__ float2 sD[3 * Nq * Nq], sDl[3 * Nq], sDr[3 * Nq];
  for (int t = threadIdx.x; t < Nq * Nq; t += blockDim.x) {
    sD[t] = split(C.x.D[t]);
    sD[Nq * Nq + t] = split(C.y.D[t]);
    sD[2 * Nq * Nq + t] = split(C.z.D[t]);
  }
  for (int t = threadIdx.x; t < Nq; t += blockDim.x) {
    sDl[t] = split(C.x.Dl[t]); sDr[t] = split(C.x.Dr[t]);
    sDl[Nq + t] = split(C.y.Dl[t]); sDr[Nq + t] = split(C.y.Dr[t]);
    sDl[2 * Nq + t] = split(C.z.Dl[t]); sDr[2 * Nq + t] = split(C.z.Dr[t]);
  }
  __syncthreads();
  const long long nchunk = (nthreads + blockDim.x - 1) / blockDim.x;
  for (long long c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const long long tid = c * blockDim.x + threadIdx.x;
    if (tid >= nthreads) continue;
    const int gi = perm[tid];
    if (gi < 0) continue;                 // padding of a class group
    rhs_df_node<N>(gi, q, F2, out0, out, G, R, ep, sD, sDl, sDr);
  }
}

}  // namespace

cudaError_t launch_prep_df(const double* q, float2* F2, const Geom& G, const RefLev& R,
                           cudaStream_t s) {
  k_prep_df<<<(unsigned)((G.nnode + 255) / 256), 256, 0, s>>>(q, F2, G, R, eos_series());
  return cudaGetLastError();
}

cudaError_t launch_rhs_df(const double* q, const float2* F2, double* out, const int* perm,
                          long long nthreads, const Geom& G, const Coef3& C, const RefLev& R,
                          const RhsEpilogue& ep, cudaStream_t s) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  const unsigned nb = (unsigned)std::min<long long>((nthreads + 127) / 128, 5LL * nsm);
#define NUMA_DF_CASE(n) \
  case n: k_rhs_df<n><<<nb, 128, 0, s>>>(q, F2, out, out, perm, nthreads, G, C, R, ep); break;
  switch (G.N) {
    NUMA_DF_CASE(1) NUMA_DF_CASE(2) NUMA_DF_CASE(3) NUMA_DF_CASE(4)
    NUMA_DF_CASE(5) NUMA_DF_CASE(6) NUMA_DF_CASE(7) NUMA_DF_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef NUMA_DF_CASE
  return cudaGetLastError();
}
