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
//    (interior / interface / wall) per axis, so no warp executes both tap counts;
//  * no instruction that the method does not need: 1 / rho by a Newton reciprocal (three
//    multiply-adds), the tendencies' minus signs on the operands, the reference gradients
//    d(rho0)/dz and d(theta0)/dz as the start of two z derivatives (rhs_device.cuh).
#include <algorithm>
#include <type_traits>
#include <vector>

#include "numa_internal.cuh"

#include "rhs_device.cuh"

namespace {
using namespace numa_dev;

__global__ void k_pressure(const double* __restrict__ q, double* __restrict__ Pp, Geom G,
                           RefLev R, EosSeries S, long long g0, long long g1, unsigned* status) {
  const long long g = g0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= g1) return;
  const double p = eos_node(q, g, G, R, S);
  Pp[g] = p;
  if (status && not_finite(p)) atomicOr(status, NUMA_ST_NONFINITE);
}

// Mixed-precision form: P' in FP64, then FP32 copies of the six stencil fields
// (rho', u, v, w, theta', P') for the FP32 right-hand side.
__global__ void k_prep32(const double* __restrict__ q, float* __restrict__ F32, Geom G, RefLev R,
                         EosSeries S) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long nn = G.nnode;
  const double Pp = eos_node(q, g, G, R, S);
  F32[g] = f32_of(q[g]);
  F32[nn + g] = f32_of(q[nn + g]);
  F32[2 * nn + g] = f32_of(q[2 * nn + g]);
  F32[3 * nn + g] = f32_of(q[3 * nn + g]);
  F32[4 * nn + g] = f32_of(q[4 * nn + g]);
  F32[5 * nn + g] = f32_of(Pp);
}

// Three 256-thread CTAs per SM (at most 85 registers a thread; a few dozen bytes of spill at
// N = 4): with the reference gradients folded into the z derivatives the compiler's own
// choice rose to 104 registers and two CTAs per SM.  1.537 -> 1.505 ms per launch on the
// 96 x 96 x 12 workload, 4.28 -> 4.19 ms at N = 7 (64 x 64 x 10).
template <int N, typename RT, typename OT>
__global__ void __launch_bounds__(256, 3) k_rhs(const double* __restrict__ q,
                                                const RT* __restrict__ fld,
                                                const RT* __restrict__ fp, OT* out0, double* out,
                                                const int* __restrict__ perm, long long nthreads,
                                                Geom G, Coef3 C, RefLev R, RhsEpilogue ep) {
  constexpr int Nq = N + 1;
  __shared__ RT sD[3 * Nq * Nq], sDl[3 * Nq], sDr[3 * Nq];
  load_rows<N, RT>(C, sD, sDl, sDr);
  __syncthreads();
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  rhs_node<N, RT, OT>(tid, q, fld, fp, out0, out, perm, nthreads, G, R, ep, sD, sDl, sDr);
}

// The FP32 right-hand side of the precision forms (RT = float).  Its FP32 work is light, so
// the per-CTA row load and barrier of k_rhs showed up in its time (ncu: barrier stalls 2.0 per
// issue): here a grid of as many CTAs as fit on the GPU loads the rows once per CTA and walks
// the thread order in CTA-sized chunks (grid stride).  The per-node arithmetic is k_rhs's.
// Three 256-thread CTAs per SM (at most 85 registers) measured fastest: 0.36 ms per launch on
// the 96 x 96 x 12 workload and 0.89 ms on the 64 x 64 x 10, N = 7 one, against 0.46 and
// 1.10 ms for k_rhs, 0.37 and 1.00 ms for the compiler's own register choice, 0.37 and 0.99 ms
// for four CTAs per SM.
template <int N, typename RT, typename OT>
__global__ void __launch_bounds__(256, 3) k_rhs_gs(const double* __restrict__ q,
                                                const RT* __restrict__ fld,
                                                const RT* __restrict__ fp, OT* out0, double* out,
                                                const int* __restrict__ perm, long long nthreads,
                                                Geom G, Coef3 C, RefLev R, RhsEpilogue ep) {
  constexpr int Nq = N + 1;
  __shared__ RT sD[3 * Nq * Nq], sDl[3 * Nq], sDr[3 * Nq];
  load_rows<N, RT>(C, sD, sDl, sDr);
  __syncthreads();
  const long long nchunk = (nthreads + blockDim.x - 1) / blockDim.x;
  for (long long c = blockIdx.x; c < nchunk; c += gridDim.x)
    rhs_node<N, RT, OT>(c * blockDim.x + threadIdx.x, q, fld, fp, out0, out, perm, nthreads, G, R,
                        ep, sD, sDl, sDr);
}

template <int N, typename RT, typename OT>
cudaError_t launch_rhs_n(const double* q, const RT* fld, const RT* fp, OT* out0, double* out,
                         const int* perm, long long nthreads, const Geom& G, const Coef3& C,
                         const RefLev& R, const RhsEpilogue& ep, cudaStream_t s) {
  const int bs = 256;
  const long long nb = (nthreads + bs - 1) / bs;
  if constexpr (std::is_same<RT, float>::value) {
    static int resident = 0;     // CTAs of this instantiation that fit on the GPU at once
    if (resident == 0) {
      int dev = 0, nsm = 0, per_sm = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rhs_gs<N, RT, OT>, bs, 0) !=
              cudaSuccess ||
          nsm < 1 || per_sm < 1)
        return cudaErrorUnknown;
      resident = nsm * per_sm;
    }
    if (nb < 1) return cudaSuccess;
    k_rhs_gs<N, RT, OT><<<(unsigned)std::min<long long>(nb, resident), bs, 0, s>>>(
        q, fld, fp, out0, out, perm, nthreads, G, C, R, ep);
  } else {
    k_rhs<N, RT, OT><<<(unsigned)nb, bs, 0, s>>>(q, fld, fp, out0, out, perm, nthreads, G, C, R, ep);
  }
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

int node_class(int idx, int N, int nel) {
  int e, i;
  axis_owner(idx, N, nel, e, i);
  if (i == 0 && e > 0) return CLS_IFACE;
  if (i == 0 || i == N) return CLS_WALL;
  return CLS_INTERIOR;
}

}  // namespace

cudaError_t launch_pressure(const double* q, double* Pp, const Geom& G, const RefLev& R,
                            cudaStream_t s, unsigned* status) {
  const int bs = 256;
  const long long nb = (G.nnode + bs - 1) / bs;
  k_pressure<<<(unsigned)nb, bs, 0, s>>>(q, Pp, G, R, eos_series(), 0, G.nnode, status);
  return cudaGetLastError();
}

cudaError_t launch_pressure_range(const double* q, double* Pp, const Geom& G, const RefLev& R,
                                  long long g0, long long g1, cudaStream_t s, unsigned* status) {
  if (g0 < 0 || g1 > G.nnode || g0 > g1) return cudaErrorInvalidValue;
  if (g0 == g1) return cudaSuccess;
  const int bs = 256;
  k_pressure<<<(unsigned)((g1 - g0 + bs - 1) / bs), bs, 0, s>>>(q, Pp, G, R, eos_series(), g0, g1,
                                                                 status);
  return cudaGetLastError();
}

void eos_level_coefs(const double* P0, int M, double* P0c) {
  const EosSeries S = eos_series();
  for (int m = 0; m < M; ++m)
    for (int k = 0; k < 5; ++k) P0c[(size_t)m * 5 + k] = P0[m] * S.c[k];
}

cudaError_t launch_prep32(const double* q, float* F32, const Geom& G, const RefLev& R,
                          cudaStream_t s) {
  const int bs = 256;
  const long long nb = (G.nnode + bs - 1) / bs;
  k_prep32<<<(unsigned)nb, bs, 0, s>>>(q, F32, G, R, eos_series());
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

template <typename Emit, typename Row>
static void walk_rhs_perm(const Geom& G, Emit emit, Row row) {
  const int tn = kTile * G.N;
  std::vector<int> cz(G.M);
  for (int iz = 0; iz < G.M; ++iz) cz[iz] = node_class(iz, G.N, G.nez);
  std::vector<long long> bucket[27];
  for (int y0 = 0; y0 < G.nyg; y0 += tn) {
    const int y1 = (G.nyg - y0 <= tn + 1) ? G.nyg : y0 + tn;   // the last tile takes the end node
    row(y0);
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
  walk_rhs_perm(G, [&](long long) { ++n; }, [](int) {});
  return n;
}

void build_rhs_perm(const Geom& G, int* out) {
  long long n = 0;
  walk_rhs_perm(G, [&](long long g) { out[n++] = (int)g; }, [](int) {});
}

void rhs_perm_rows(const Geom& G, std::vector<long long>& off, std::vector<int>& y0) {
  off.clear();
  y0.clear();
  long long n = 0;
  walk_rhs_perm(G, [&](long long) { ++n; }, [&](int y) {
    off.push_back(n);
    y0.push_back(y);
  });
  off.push_back(n);
  y0.push_back(G.nyg);
}

// ---- the integer-pipe conversions and the reciprocal, exposed for testing ---------------------
namespace {
__global__ void k_convert_f64_f32(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = numa_dev::f32_of(x[i]);
}
__global__ void k_convert_f32_f64(const float* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = numa_dev::f64_of(x[i]);
}
__global__ void k_reciprocal(const double* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = numa_dev::recip(x[i]);
}
unsigned convert_grid(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 8));
}
}  // namespace

extern "C" int numa_convert_f64_f32(const double* x, float* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y)) || ((uintptr_t)x % 8) || ((uintptr_t)y % 4)) return NUMA_ERR_ARG;
  if (n == 0) return NUMA_OK;
  k_convert_f64_f32<<<convert_grid(n), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? NUMA_OK : NUMA_ERR_CUDA;
}

extern "C" int numa_convert_f32_f64(const float* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y)) || ((uintptr_t)x % 4) || ((uintptr_t)y % 8)) return NUMA_ERR_ARG;
  if (n == 0) return NUMA_OK;
  k_convert_f32_f64<<<convert_grid(n), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? NUMA_OK : NUMA_ERR_CUDA;
}

extern "C" int numa_reciprocal(const double* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y)) || ((uintptr_t)x % 8) || ((uintptr_t)y % 8)) return NUMA_ERR_ARG;
  if (n == 0) return NUMA_OK;
  k_reciprocal<<<convert_grid(n), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? NUMA_OK : NUMA_ERR_CUDA;
}
