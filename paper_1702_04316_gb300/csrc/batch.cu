// Ensembles of independent forecasts ("batching form"): members with their own mesh,
// polynomial order, reference state and time step are advanced together.
//
// Each member is set up exactly like a single-mesh context (tables, per-column factors at
// its own dt, workspace).  Every phase of a HEVI step (EOS pre-pass, right-hand side,
// implicit stage) is then one persistent launch per polynomial order present (at most
// three, N = 4..6) for the whole ensemble: a grid sized to the GPU walks a work list of
// (member, block) items, so the number of launches per step does not grow with the number
// of members; each step is captured once as a CUDA graph and replayed.  Each order group
// has its own kernels (registers and shared memory sized for that order and its tallest
// column) and its own work lists, built for the right-hand side's threads per CTA and the
// stage's columns per CTA that an autotuner picks by timing candidates on the ensemble.
// Blocks never wait on one another: items are assigned by a static stride.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "column_device.cuh"
#include "numa.h"
#include "numa_ctx.h"
#include "rhs_device.cuh"

namespace {
using namespace numa_dev;

// Device descriptor of one member.
struct MemberDev {
  Geom G;
  Coef3 C;
  RefLev R;
  StageTab tb;
  Factors F;
  StageCoef s2, s3;
  double b1dt, b2dt, b3dt;
  const int* perm;
  long long nperm;
  long long soff;        // offset of the member's state in the packed arrays
  double *Pp, *R1, *R2, *q2, *q3;
};

// Work list of one kernel: items [start[k], start[k+1]) belong to member order[k].
struct WorkList {
  const long long* start;
  const int* order;
  int nmem;
  long long nitems;
};

__device__ __forceinline__ int find_slot(const WorkList& W, long long item) {
  int lo = 0, hi = W.nmem;     // start[lo] <= item < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (W.start[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// src: 0 = the packed input state, 1 = the member's q(2), 2 = the member's q(3).
__device__ __forceinline__ const double* src_state(const MemberDev& d, int src, const double* qin) {
  return src == 0 ? qin + d.soff : (src == 1 ? d.q2 : d.q3);
}

__global__ void k_batch_pressure(const MemberDev* __restrict__ md, WorkList W, int src,
                                 const double* qin, EosSeries S) {
  for (long long item = blockIdx.x; item < W.nitems; item += gridDim.x) {
    const int k = find_slot(W, item);
    const MemberDev& d = md[W.order[k]];
    const long long g = (item - W.start[k]) * blockDim.x + threadIdx.x;
    if (g < d.G.nnode) d.Pp[g] = eos_node(src_state(d, src, qin), g, d.G, d.R, S);
  }
}

template <int N>
__device__ __forceinline__ void batch_rhs_item(const MemberDev& d, long long tid, int src, int mode,
                                               const double* qin, double* qout, double* sD,
                                               double* sDl, double* sDr) {
  load_rows<N, double>(d.C, sD, sDl, sDr);
  __syncthreads();
  const double* q = src_state(d, src, qin);
  RhsEpilogue ep{};
  ep.mode = mode;
  double* out0 = (src == 0) ? d.R1 : d.R2;
  double* out = nullptr;
  if (mode == 2) {
    ep.b1dt = d.b1dt;
    ep.b2dt = d.b2dt;
    ep.b3dt = d.b3dt;
    ep.u0 = qin + d.soff;
    ep.R1 = d.R1;
    ep.R2 = d.R2;
    out = qout + d.soff;
  }
  rhs_node<N, double, double>(tid, q, q, d.Pp, out0, out, d.perm, d.nperm, d.G, d.R, ep, sD, sDl,
                              sDr);
}

// At most 85 registers a thread (three 256-thread or six 128-thread CTAs per SM), as k_rhs.
template <int N>
__global__ void __launch_bounds__(256, 3) k_batch_rhs(const MemberDev* __restrict__ md, WorkList W,
                                                      int src, int mode, const double* qin,
                                                      double* qout) {
  constexpr int Nq = N + 1;
  __shared__ double sD[3 * Nq * Nq], sDl[3 * Nq], sDr[3 * Nq];
  for (long long item = blockIdx.x; item < W.nitems; item += gridDim.x) {
    const int k = find_slot(W, item);
    const MemberDev& d = md[W.order[k]];
    const long long tid = (item - W.start[k]) * blockDim.x + threadIdx.x;
    batch_rhs_item<N>(d, tid, src, mode, qin, qout, sD, sDl, sDr);
    __syncthreads();
  }
}

// T columns per work item; blockDim.x >= T threads share the stage's coalesced phases.
// The stage writes P' of its output for the next right-hand side (as the single-mesh step
// does), so the ensemble's step needs the equation-of-state pass only at its start.
template <int N, bool S3>
__global__ void k_batch_stage(const MemberDev* __restrict__ md, WorkList W, const double* qin,
                              int T, EosSeries eos) {
  extern __shared__ double sm[];
  for (long long item = blockIdx.x; item < W.nitems; item += gridDim.x) {
    const int k = find_slot(W, item);
    const MemberDev& d = md[W.order[k]];
    const long long col0 = (item - W.start[k]) * T;
    stage_body<N, S3 ? 2 : 1, false, double>(col0, T, sm, qin + d.soff, d.R1, d.R2, d.q2,
                                              S3 ? d.q3 : d.q2, d.G, d.R, d.F, S3 ? d.s3 : d.s2,
                                              d.tb, 0, nullptr, nullptr, d.Pp, &eos);
    __syncthreads();
  }
}

// Host copy of a work list and its device arrays.
struct HostList {
  std::vector<long long> start;
  std::vector<int> order;
  long long* d_start = nullptr;
  int* d_order = nullptr;
  WorkList dev() const { return WorkList{d_start, d_order, (int)order.size(), start.back()}; }
};

}  // namespace

// The members of one polynomial order: their work lists, tiles and launch shapes.
struct OrderGroup {
  int N = 0;
  std::vector<int> members;
  HostList rhs_list, col_list;
  int rhs_threads = 256, col_tile = 64, col_threads = 4;
  int grid_rhs = 0, grid_col = 0;
  size_t stage_smem = 0;
  // threads per CTA of the stage: col_threads per column of the tile (the coalesced phases
  // and the level-parallel steps; the substitutions run one thread per column)
  int stage_threads() const { return std::min(1024, col_threads * col_tile); }
};

struct numa_batch {
  std::vector<numa_ctx*> mem;
  cudaStream_t stream = nullptr;
  std::string err;
  MemberDev* d_md = nullptr;
  std::vector<long long> soff;
  long long total = 0;                 // doubles of one packed state
  HostList node_list;
  int grid_node = 0;
  OrderGroup groups[3];                // N = 4, 5, 6
  double* d_state = nullptr;           // packed scratch state for tuning
  bool use_graph = true;
  // graphs are captured and launched on a private stream (capture is not allowed on the
  // legacy default stream), ordered against the caller's stream with two events
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  struct G { const double* in; double* out; cudaGraphExec_t exec; } graphs[2] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int ngraph = 0;
  std::vector<float> tune_ms;          // timings of the candidates, for the record
};

namespace {

int bfail(numa_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  return code;
}

#define NUMA_BCK(b, call)                                                           \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return bfail(b, NUMA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void free_list(HostList& L) {
  cudaFree(L.d_start);
  cudaFree(L.d_order);
  L.d_start = nullptr;
  L.d_order = nullptr;
}

int upload_list(numa_batch* b, HostList& L) {
  free_list(L);
  NUMA_BCK(b, cudaMalloc(&L.d_start, L.start.size() * sizeof(long long)));
  NUMA_BCK(b, cudaMalloc(&L.d_order, std::max<size_t>(1, L.order.size()) * sizeof(int)));
  NUMA_BCK(b, cudaMemcpy(L.d_start, L.start.data(), L.start.size() * sizeof(long long), cudaMemcpyHostToDevice));
  if (!L.order.empty())
    NUMA_BCK(b, cudaMemcpy(L.d_order, L.order.data(), L.order.size() * sizeof(int), cudaMemcpyHostToDevice));
  return NUMA_OK;
}

// items per member -> list (members in the given order)
void make_list(HostList& L, const std::vector<int>& order, const std::vector<long long>& items) {
  L.order = order;
  L.start.assign(1, 0);
  for (int m : order) L.start.push_back(L.start.back() + items[m]);
}

template <int N>
int group_shapes(numa_batch* b, OrderGroup& g, int nsm) {
  int per = 0;
  NUMA_BCK(b, cudaFuncSetAttribute(k_batch_stage<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.stage_smem));
  NUMA_BCK(b, cudaFuncSetAttribute(k_batch_stage<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.stage_smem));
  NUMA_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_rhs<N>, g.rhs_threads, 0));
  g.grid_rhs = nsm * std::max(per, 1);
  NUMA_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_stage<N, true>, g.stage_threads(), g.stage_smem));
  if (per < 1) return bfail(b, NUMA_ERR_ARG, "stage tile does not fit in shared memory");
  g.grid_col = nsm * per;
  return NUMA_OK;
}

// Work lists and launch shapes of one order group (its members' RHS blocks, and their
// stage blocks with the tallest columns dealt first so that static striding balances).
int build_group(numa_batch* b, OrderGroup& g) {
  const int n = (int)b->mem.size();
  std::vector<long long> it_rhs(n, 0), it_col(n, 0);
  int maxM = 0;
  for (int m : g.members) {
    const numa_ctx* c = b->mem[m];
    it_rhs[m] = (c->nperm + g.rhs_threads - 1) / g.rhs_threads;
    it_col[m] = (c->G.ncol + g.col_tile - 1) / g.col_tile;
    maxM = std::max(maxM, c->G.M);
  }
  std::vector<int> by_m = g.members;
  std::stable_sort(by_m.begin(), by_m.end(),
                   [&](int a, int c) { return b->mem[a]->G.M > b->mem[c]->G.M; });
  make_list(g.rhs_list, g.members, it_rhs);
  make_list(g.col_list, by_m, it_col);
  int rc;
  if ((rc = upload_list(b, g.rhs_list)) || (rc = upload_list(b, g.col_list))) return rc;
  g.stage_smem = col_smem_per_level(false, 0) * (size_t)maxM * g.col_tile;
  int dev = 0, nsm = 0;
  NUMA_BCK(b, cudaGetDevice(&dev));
  NUMA_BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  switch (g.N) {
    case 4: return group_shapes<4>(b, g, nsm);
    case 5: return group_shapes<5>(b, g, nsm);
    case 6: return group_shapes<6>(b, g, nsm);
    default: return NUMA_ERR_ARG;
  }
}

int build_lists(numa_batch* b) {
  const int n = (int)b->mem.size();
  std::vector<int> natural(n);
  for (int m = 0; m < n; ++m) natural[m] = m;
  std::vector<long long> it_node(n);
  for (int m = 0; m < n; ++m) it_node[m] = (b->mem[m]->G.nnode + 255) / 256;
  make_list(b->node_list, natural, it_node);
  int rc = upload_list(b, b->node_list);
  if (rc) return rc;
  int dev = 0, nsm = 0, per = 0;
  NUMA_BCK(b, cudaGetDevice(&dev));
  NUMA_BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  NUMA_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_pressure, 256, 0));
  b->grid_node = nsm * std::max(per, 1);
  for (auto& g : b->groups)
    if (!g.members.empty() && (rc = build_group(b, g))) return rc;
  return NUMA_OK;
}

template <int N>
void launch_group_rhs(numa_batch* b, const OrderGroup& g, int src, int mode, const double* qin,
                      double* qout, cudaStream_t s) {
  k_batch_rhs<N><<<g.grid_rhs, g.rhs_threads, 0, s>>>(b->d_md, g.rhs_list.dev(), src, mode, qin, qout);
}

template <int N>
void launch_group_stage(numa_batch* b, const OrderGroup& g, bool s3, const double* qin,
                        cudaStream_t s) {
  const EosSeries S = eos_series();
  if (s3) k_batch_stage<N, true><<<g.grid_col, g.stage_threads(), g.stage_smem, s>>>(b->d_md, g.col_list.dev(), qin, g.col_tile, S);
  else k_batch_stage<N, false><<<g.grid_col, g.stage_threads(), g.stage_smem, s>>>(b->d_md, g.col_list.dev(), qin, g.col_tile, S);
}

void enqueue_rhs_all(numa_batch* b, int src, int mode, const double* qin, double* qout, cudaStream_t s) {
  for (auto& g : b->groups) {
    if (g.members.empty()) continue;
    if (g.N == 4) launch_group_rhs<4>(b, g, src, mode, qin, qout, s);
    else if (g.N == 5) launch_group_rhs<5>(b, g, src, mode, qin, qout, s);
    else launch_group_rhs<6>(b, g, src, mode, qin, qout, s);
  }
}

void enqueue_stage_all(numa_batch* b, bool s3, const double* qin, cudaStream_t s) {
  for (auto& g : b->groups) {
    if (g.members.empty()) continue;
    if (g.N == 4) launch_group_stage<4>(b, g, s3, qin, s);
    else if (g.N == 5) launch_group_stage<5>(b, g, s3, qin, s);
    else launch_group_stage<6>(b, g, s3, qin, s);
  }
}

int enqueue_step(numa_batch* b, const double* qin, double* qout, cudaStream_t s) {
  const EosSeries S = eos_series();
  const WorkList Wn = b->node_list.dev();
  k_batch_pressure<<<b->grid_node, 256, 0, s>>>(b->d_md, Wn, 0, qin, S);
  enqueue_rhs_all(b, 0, 0, qin, qout, s);
  enqueue_stage_all(b, false, qin, s);          // also P' of q(2)
  enqueue_rhs_all(b, 1, 0, qin, qout, s);
  enqueue_stage_all(b, true, qin, s);           // also P' of q(3)
  enqueue_rhs_all(b, 2, 2, qin, qout, s);
  NUMA_BCK(b, cudaGetLastError());
  return NUMA_OK;
}

void drop_graphs(numa_batch* b) {
  for (auto& g : b->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = {nullptr, nullptr, nullptr};
  }
  b->ngraph = 0;
}

// The graph of one step for (qin, qout), captured on first use.
int step_graph(numa_batch* b, const double* qin, double* qout, cudaGraphExec_t* exec) {
  for (auto& g : b->graphs)
    if (g.exec && g.in == qin && g.out == qout) {
      *exec = g.exec;
      return NUMA_OK;
    }
  cudaGraph_t graph = nullptr;
  NUMA_BCK(b, cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_step(b, qin, qout, b->gstream);
  cudaError_t e = cudaStreamEndCapture(b->gstream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, NUMA_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, NUMA_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  auto& slot = b->graphs[b->ngraph % 2];
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot = {qin, qout, ex};
  b->ngraph++;
  *exec = ex;
  return NUMA_OK;
}

// Autotuner: for every order group, time its right-hand side for each threads-per-CTA
// candidate and its stage for each columns-per-CTA candidate on the ensemble (rest
// state), and keep the fastest.
int autotune(numa_batch* b) {
  cudaEvent_t e0, e1;
  NUMA_BCK(b, cudaEventCreate(&e0));
  NUMA_BCK(b, cudaEventCreate(&e1));
  NUMA_BCK(b, cudaMemsetAsync(b->d_state, 0, b->total * sizeof(double), b->stream));
  const EosSeries S = eos_series();
  k_batch_pressure<<<b->grid_node, 256, 0, b->stream>>>(b->d_md, b->node_list.dev(), 0, b->d_state, S);
  auto time_it = [&](auto launch, float* ms) -> int {
    for (int r = 0; r < 2; ++r) launch();
    NUMA_BCK(b, cudaEventRecord(e0, b->stream));
    for (int r = 0; r < 3; ++r) launch();
    NUMA_BCK(b, cudaEventRecord(e1, b->stream));
    NUMA_BCK(b, cudaEventSynchronize(e1));
    NUMA_BCK(b, cudaGetLastError());
    NUMA_BCK(b, cudaEventElapsedTime(ms, e0, e1));
    return NUMA_OK;
  };
  int rc = NUMA_OK;
  for (auto& g : b->groups) {
    if (g.members.empty()) continue;
    float best = 1e30f;
    int best_rt = 256;
    for (int rt : {128, 256}) {
      g.rhs_threads = rt;
      if ((rc = build_group(b, g))) break;
      float ms = 0;
      rc = time_it([&] { enqueue_rhs_all(b, 0, 0, b->d_state, b->d_state, b->stream); }, &ms);
      if (rc) break;
      b->tune_ms.push_back(ms);
      if (ms < best) { best = ms; best_rt = rt; }
    }
    if (rc) break;
    g.rhs_threads = best_rt;
    best = 1e30f;
    int best_ct = 32, best_tc = 8;
    for (int ct : {32, 64, 96})
      for (int tc : {4, 8}) {
        g.col_tile = ct;
        g.col_threads = tc;
        if (build_group(b, g)) { b->err.clear(); continue; }     // does not fit: skip
        float ms = 0;
        rc = time_it([&] { enqueue_stage_all(b, false, b->d_state, b->stream); }, &ms);
        if (rc) break;
        b->tune_ms.push_back(ms);
        if (ms < best) { best = ms; best_ct = ct; best_tc = tc; }
      }
    if (rc) break;
    g.col_tile = best_ct;
    g.col_threads = best_tc;
    if ((rc = build_group(b, g))) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" {

int numa_batch_init(const numa_mesh_desc* meshes, const int* N, const double* dt, int nmembers,
                    void* stream, numa_batch** out) {
  if (!out) return NUMA_ERR_ARG;
  *out = nullptr;
  if (!meshes || !N || !dt || nmembers < 1 || nmembers > 4096) return NUMA_ERR_ARG;
  for (int m = 0; m < nmembers; ++m)
    if (N[m] < 4 || N[m] > 6 || !(dt[m] > 0)) return NUMA_ERR_ARG;
  numa_batch* b = new numa_batch();
  b->stream = (cudaStream_t)stream;
  int rc = NUMA_OK;
  std::vector<MemberDev> h(nmembers);
  double at[9], bb[3];
  numa_ark2_tableau(nullptr, at, bb);
  for (int m = 0; m < nmembers && rc == NUMA_OK; ++m) {
    numa_ctx* c = nullptr;
    rc = numa_init(&meshes[m], N[m], dt[m], stream, &c);
    if (rc) break;
    b->mem.push_back(c);
    b->soff.push_back(b->total);
    MemberDev& d = h[m];
    std::memset(&d, 0, sizeof(d));
    d.G = c->G;
    d.C = c->C;
    d.R = c->R;
    d.tb = c->T;
    d.F = c->F;
    d.s2 = numa_stage_coef(c, 2);
    d.s3 = numa_stage_coef(c, 3);
    d.b1dt = bb[0] * dt[m];
    d.b2dt = bb[1] * dt[m];
    d.b3dt = bb[2] * dt[m];
    d.perm = c->d_perm;
    d.nperm = c->nperm;
    d.soff = b->total;
    d.Pp = c->Pp;
    d.R1 = c->R1;
    d.R2 = c->R2;
    d.q2 = c->q2;
    d.q3 = c->q3;
    b->total += 5 * c->G.nnode;
  }
  b->soff.push_back(b->total);
  for (int g = 0; g < 3; ++g) b->groups[g].N = 4 + g;
  if (rc == NUMA_OK)
    for (int m = 0; m < nmembers; ++m) b->groups[N[m] - 4].members.push_back(m);
  if (rc == NUMA_OK && (cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess))
    rc = NUMA_ERR_CUDA;
  if (rc == NUMA_OK) {
    if (cudaMalloc(&b->d_md, h.size() * sizeof(MemberDev)) != cudaSuccess ||
        cudaMalloc(&b->d_state, b->total * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      rc = NUMA_ERR_OOM;
    } else if (cudaMemcpy(b->d_md, h.data(), h.size() * sizeof(MemberDev), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = NUMA_ERR_CUDA;
    }
  }
  if (rc == NUMA_OK) rc = build_lists(b);
  if (rc == NUMA_OK) rc = autotune(b);
  if (rc == NUMA_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = NUMA_ERR_CUDA;
  if (rc != NUMA_OK) {
    numa_batch_destroy(b);
    return rc;
  }
  *out = b;
  return NUMA_OK;
}

void numa_batch_destroy(numa_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  free_list(b->node_list);
  for (auto& g : b->groups) {
    free_list(g.rhs_list);
    free_list(g.col_list);
  }
  cudaFree(b->d_md);
  cudaFree(b->d_state);
  if (b->gstream) {
    cudaStreamSynchronize(b->gstream);
    cudaStreamDestroy(b->gstream);
  }
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (auto* c : b->mem) numa_destroy(c);
  delete b;
}

int numa_batch_layout(const numa_batch* b, long long* offsets) {
  if (!b || !offsets) return NUMA_ERR_ARG;
  for (size_t m = 0; m < b->soff.size(); ++m) offsets[m] = b->soff[m];
  return NUMA_OK;
}

int numa_batch_set_graph(numa_batch* b, int enable) {
  if (!b) return NUMA_ERR_ARG;
  b->use_graph = enable != 0;
  return NUMA_OK;
}

int numa_batch_step_imex1d(numa_batch* b, const double* q_in, double* q_out, int nsteps) {
  if (!b || !q_in || !q_out || nsteps < 0) return bfail(b, NUMA_ERR_ARG, "bad arguments");
  if (nsteps == 0) {
    if (q_in != q_out)
      NUMA_BCK(b, cudaMemcpyAsync(q_out, q_in, b->total * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    return NUMA_OK;
  }
  const double* cur = q_in;
  if (b->use_graph) {
    NUMA_BCK(b, cudaEventRecord(b->ev_in, b->stream));
    NUMA_BCK(b, cudaStreamWaitEvent(b->gstream, b->ev_in, 0));
  }
  for (int s = 0; s < nsteps; ++s) {
    int rc;
    if (b->use_graph) {
      cudaGraphExec_t ex = nullptr;
      if ((rc = step_graph(b, cur, q_out, &ex))) return rc;
      NUMA_BCK(b, cudaGraphLaunch(ex, b->gstream));
    } else if ((rc = enqueue_step(b, cur, q_out, b->stream))) {
      return rc;
    }
    cur = q_out;
  }
  if (b->use_graph) {
    NUMA_BCK(b, cudaEventRecord(b->ev_out, b->gstream));
    NUMA_BCK(b, cudaStreamWaitEvent(b->stream, b->ev_out, 0));
  }
  return NUMA_OK;
}

int numa_batch_tuning(const numa_batch* b, int N, int* rhs_threads, int* col_tile,
                      int* stage_threads) {
  if (!b || N < 4 || N > 6) return NUMA_ERR_ARG;
  const OrderGroup& g = b->groups[N - 4];
  if (rhs_threads) *rhs_threads = g.members.empty() ? 0 : g.rhs_threads;
  if (col_tile) *col_tile = g.members.empty() ? 0 : g.col_tile;
  if (stage_threads) *stage_threads = g.members.empty() ? 0 : g.stage_threads();
  return NUMA_OK;
}

int numa_batch_member_query(const numa_batch* b, int member, int what, long long* out) {
  if (!b || member < 0 || member >= (int)b->mem.size()) return NUMA_ERR_ARG;
  return numa_query(b->mem[member], what, out);
}

int numa_batch_reference_levels(const numa_batch* b, int member, double* host_out) {
  if (!b || member < 0 || member >= (int)b->mem.size()) return NUMA_ERR_ARG;
  return numa_reference_levels(b->mem[member], host_out);
}

const char* numa_batch_last_error(const numa_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
