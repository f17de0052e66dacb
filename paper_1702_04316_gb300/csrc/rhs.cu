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
// Each thread computes one global node: no atomics, no element-local scratch, and the
// column-major layout (z fastest) makes every stencil load of a warp contiguous.
#include "numa_internal.cuh"

namespace {

__device__ __forceinline__ double dss_deriv(const double* __restrict__ f, long long g,
                                            long long stride, int idx, int nel, int N,
                                            const AxisCoef& c) {
  int e, i;
  axis_owner(idx, N, nel, e, i);
  const int Nq = N + 1;
  const double* p0 = f + g - (long long)i * stride;   // local node 0 of element e
  double acc = 0.0;
  if (i == 0 && e > 0) {
    const double* pl = p0 - (long long)N * stride;    // local node 0 of element e-1
#pragma unroll 4
    for (int n = 0; n < Nq; ++n) acc = fma(c.Dl[n], __ldg(pl + n * stride), acc);
#pragma unroll 4
    for (int n = 0; n < Nq; ++n) acc = fma(c.Dr[n], __ldg(p0 + n * stride), acc);
  } else {
    const double* Drow = c.D + i * Nq;
#pragma unroll 4
    for (int n = 0; n < Nq; ++n) acc = fma(Drow[n], __ldg(p0 + n * stride), acc);
  }
  return acc;
}

// P' = P(rho0 + rho', theta0 + theta') - P0 without cancellation:
//   (rho theta)/(rho0 theta0) = (1 + a)(1 + b),  a = rho'/rho0,  b = theta'/theta0,
//   P' = P0 ((1 + x)^gamma - 1) = P0 expm1(gamma log1p(x)),  x = a + b + a b.
__global__ void k_pressure(const double* __restrict__ q, double* __restrict__ Pp, Geom G,
                           RefLev R, double gamma) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  int iz = (int)(g % G.M);
  double a = q[g] * R.inv_rho0[iz];
  double b = q[4 * G.nnode + g] * R.inv_theta0[iz];
  double x = fma(a, b, a + b);
  Pp[g] = R.P0[iz] * expm1(gamma * log1p(x));
}

__global__ void k_rhs(const double* __restrict__ q, const double* __restrict__ Pp,
                      double* out, Geom G, Coef3 C, RefLev R, RhsEpilogue ep) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long nn = G.nnode;
  const long long col = g / G.M;
  const int iz = (int)(g - col * G.M);
  const int iy = (int)(col / G.nxg);
  const int ix = (int)(col - (long long)iy * G.nxg);
  const long long sx = G.M, sy = (long long)G.nxg * G.M;
  const int N = G.N;

  const double* rp = q;
  const double* u = q + nn;
  const double* v = q + 2 * nn;
  const double* w = q + 3 * nn;
  const double* tp = q + 4 * nn;

  const double r_ = rp[g], u_ = u[g], v_ = v[g], w_ = w[g];

  // gradients of rho', u, v, w, theta', P'
  const double rx = dss_deriv(rp, g, sx, ix, G.nex, N, C.x);
  const double ry = dss_deriv(rp, g, sy, iy, G.ney, N, C.y);
  const double rz = dss_deriv(rp, g, 1, iz, G.nez, N, C.z);
  const double ux = dss_deriv(u, g, sx, ix, G.nex, N, C.x);
  const double uy = dss_deriv(u, g, sy, iy, G.ney, N, C.y);
  const double uz = dss_deriv(u, g, 1, iz, G.nez, N, C.z);
  const double vx = dss_deriv(v, g, sx, ix, G.nex, N, C.x);
  const double vy = dss_deriv(v, g, sy, iy, G.ney, N, C.y);
  const double vz = dss_deriv(v, g, 1, iz, G.nez, N, C.z);
  const double wx = dss_deriv(w, g, sx, ix, G.nex, N, C.x);
  const double wy = dss_deriv(w, g, sy, iy, G.ney, N, C.y);
  const double wz = dss_deriv(w, g, 1, iz, G.nez, N, C.z);
  const double tx = dss_deriv(tp, g, sx, ix, G.nex, N, C.x);
  const double ty = dss_deriv(tp, g, sy, iy, G.ney, N, C.y);
  const double tz = dss_deriv(tp, g, 1, iz, G.nez, N, C.z);
  const double px = dss_deriv(Pp, g, sx, ix, G.nex, N, C.x);
  const double py = dss_deriv(Pp, g, sy, iy, G.ney, N, C.y);
  const double pz = dss_deriv(Pp, g, 1, iz, G.nez, N, C.z);

  const double rho = R.rho0[iz] + r_;
  const double irho = 1.0 / rho;
  double t_r = -(u_ * rx + v_ * ry + w_ * (rz + R.drho0[iz]) + rho * (ux + vy + wz));
  double t_u = -(u_ * ux + v_ * uy + w_ * uz + px * irho);
  double t_v = -(u_ * vx + v_ * vy + w_ * vz + py * irho);
  double t_w = -(u_ * wx + v_ * wy + w_ * wz + (pz + NUMA_GRAV * r_) * irho);
  double t_t = -(u_ * tx + v_ * ty + w_ * (tz + R.dtheta0[iz]));
  // walls: no normal flow
  if (ix == 0 || ix == G.nxg - 1) t_u = 0.0;
  if (iy == 0 || iy == G.nyg - 1) t_v = 0.0;
  if (iz == 0 || iz == G.M - 1) t_w = 0.0;

  const double t[5] = {t_r, t_u, t_v, t_w, t_t};
  if (ep.mode == 0) {
#pragma unroll
    for (int f = 0; f < 5; ++f) out[f * nn + g] = t[f];
  } else if (ep.mode == 1) {
    const double om = 1.0 - ep.alpha;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const double cur = q[f * nn + g];
      double val = fma(ep.beta_dt, t[f], om * cur);
      if (ep.alpha != 0.0) val = fma(ep.alpha, ep.u0[f * nn + g], val);
      out[f * nn + g] = val;
    }
  } else {
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const long long o = f * nn + g;
      out[o] = fma(ep.b3dt, t[f], fma(ep.b2dt, ep.R2[o], fma(ep.b1dt, ep.R1[o], ep.u0[o])));
    }
  }
}

}  // namespace

cudaError_t launch_pressure(const double* q, double* Pp, const Geom& G, const RefLev& R,
                            cudaStream_t s) {
  const double gamma = NUMA_GAMMA;
  const int bs = 256;
  const long long nb = (G.nnode + bs - 1) / bs;
  k_pressure<<<(unsigned)nb, bs, 0, s>>>(q, Pp, G, R, gamma);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const double* q, const double* Pp, double* out, const Geom& G,
                       const Coef3& C, const RefLev& R, const RhsEpilogue& ep,
                       cudaStream_t s) {
  const int bs = 256;
  const long long nb = (G.nnode + bs - 1) / bs;
  k_rhs<<<(unsigned)nb, bs, 0, s>>>(q, Pp, out, G, C, R, ep);
  return cudaGetLastError();
}
