// Small kernels: connectivity tables, non-finite counting and the ARK2 final update.
#include "numa_internal.cuh"

namespace {

// Element-to-global map, written through the same axis_owner/global_id helpers that the
// right-hand side uses for its DSS'd derivatives.
__global__ void k_l2g(Geom G, int32_t* l2g) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nq3 = (long long)G.Nq * G.Nq * G.Nq;
  const long long total = (long long)G.nex * G.ney * G.nez * nq3;
  if (t >= total) return;
  const long long e = t / nq3;
  const int l = (int)(t - e * nq3);
  const int i = l % G.Nq, j = (l / G.Nq) % G.Nq, k = l / (G.Nq * G.Nq);
  const int ex = (int)(e % G.nex), ey = (int)((e / G.nex) % G.ney), ez = (int)(e / ((long long)G.nex * G.ney));
  l2g[t] = (int32_t)global_id(G, ex * G.N + i, ey * G.N + j, ez * G.N + k);
}

// Inverse map: for each global node the element-local ids (e*(N+1)^3 + l) that DSS sums
// into it, ascending, padded with -1.  Per axis the contributing (element, local index)
// pairs are (e, i) from axis_owner and, at an interface, (e-1, N).
__global__ void k_g2l(Geom G, int32_t* g2l) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= G.nnode) return;
  const long long col = g / G.M;
  const int iz = (int)(g - col * G.M), iy = (int)(col / G.nxg), ix = (int)(col - (long long)iy * G.nxg);
  int ce[3][2], ci[3][2], cn[3];
  const int idx[3] = {ix, iy, iz}, nel[3] = {G.nex, G.ney, G.nez};
  for (int a = 0; a < 3; ++a) {
    int e, i;
    axis_owner(idx[a], G.N, nel[a], e, i);
    cn[a] = 0;
    if (i == 0 && e > 0) { ce[a][cn[a]] = e - 1; ci[a][cn[a]] = G.N; cn[a]++; }
    ce[a][cn[a]] = e; ci[a][cn[a]] = i; cn[a]++;
  }
  int32_t ids[8];
  int n = 0;
  const int Nq = G.Nq;
  for (int c = 0; c < cn[2]; ++c)
    for (int b = 0; b < cn[1]; ++b)
      for (int a = 0; a < cn[0]; ++a) {
        const long long e = ce[0][a] + (long long)G.nex * (ce[1][b] + (long long)G.ney * ce[2][c]);
        const int l = ci[0][a] + Nq * (ci[1][b] + Nq * ci[2][c]);
        ids[n++] = (int32_t)(e * Nq * Nq * Nq + l);
      }
  for (int p = 1; p < n; ++p) {   // insertion sort, n <= 8
    int32_t v = ids[p];
    int q = p - 1;
    while (q >= 0 && ids[q] > v) { ids[q + 1] = ids[q]; --q; }
    ids[q + 1] = v;
  }
  for (int p = 0; p < 8; ++p) g2l[g * 8 + p] = (p < n) ? ids[p] : -1;
}

// Non-finite test on the exponent bits (integer pipe only).
__global__ void k_nonfinite(const double* __restrict__ x, long long n, unsigned long long* count) {
  unsigned long long local = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x[t]);
    local += ((bits >> 52) & 0x7ffull) == 0x7ffull;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

__global__ void k_ark_final(const double* __restrict__ qn, const double* __restrict__ R1,
                            const double* __restrict__ R2, const double* __restrict__ R3,
                            double* out, long long n, double b1dt, double b2dt, double b3dt) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = fma(b3dt, R3[t], fma(b2dt, R2[t], fma(b1dt, R1[t], qn[t])));
}

__global__ void k_ark_combine(const double* __restrict__ qn, const __grid_constant__ StageSum S,
                              double* out, long long n, unsigned* status) {
  unsigned bad = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    double v = qn[t];
    for (int k = 0; k < S.n; ++k) v = fma(S.bdt[k], __ldg(S.R[k] + t), v);
    out[t] = v;
    bad |= not_finite(v);
  }
  if (bad && status) atomicOr(status, NUMA_ST_NONFINITE);
}

}  // namespace

cudaError_t launch_ark_combine(const double* qn, const StageSum& S, double* out, long long n,
                               unsigned* status, cudaStream_t s) {
  k_ark_combine<<<152 * 8, 256, 0, s>>>(qn, S, out, n, status);
  return cudaGetLastError();
}

cudaError_t launch_connectivity(const Geom& G, int32_t* l2g, int32_t* g2l, cudaStream_t s) {
  const int bs = 256;
  if (l2g) {
    const long long total = (long long)G.nex * G.ney * G.nez * G.Nq * G.Nq * G.Nq;
    k_l2g<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(G, l2g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (g2l) {
    k_g2l<<<(unsigned)((G.nnode + bs - 1) / bs), bs, 0, s>>>(G, g2l);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_count_nonfinite(const double* x, long long n, unsigned long long* count,
                                   cudaStream_t s) {
  k_nonfinite<<<152 * 8, 256, 0, s>>>(x, n, count);
  return cudaGetLastError();
}

cudaError_t launch_ark_final(const double* qn, const double* R1, const double* R2,
                             const double* R3, double* out, long long n, double b1dt,
                             double b2dt, double b3dt, cudaStream_t s) {
  k_ark_final<<<152 * 8, 256, 0, s>>>(qn, R1, R2, R3, out, n, b1dt, b2dt, b3dt);
  return cudaGetLastError();
}
