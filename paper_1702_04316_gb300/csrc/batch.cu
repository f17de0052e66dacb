// Ensembles of independent forecasts ("batching form"): members with their own mesh,
// polynomial order, reference state and time step are advanced together.
//
// Each member is set up exactly like a single-mesh context (tables, per-column factors at
// its own dt, workspace).  Every phase of a HEVI step (EOS pre-pass, right-hand side,
// implicit stage) is then ONE persistent launch for the whole ensemble: a grid sized to
// the GPU walks a work list of (member, block) items, so a step is eight launches for any
// number of members; each step is captured once as a CUDA graph and replayed.  The
// members' work lists are built for the right-hand side's threads per CTA and the stage's
// columns per CTA that an autotuner picks by timing the candidates on the ensemble itself.
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

__global__ void k_batch_rhs(const MemberDev* __restrict__ md, WorkList W, int src, int mode,
                            const double* qin, double* qout) {
  __shared__ double sD[3 * NUMA_MAXNQ * NUMA_MAXNQ], sDl[3 * NUMA_MAXNQ], sDr[3 * NUMA_MAXNQ];
  for (long long item = blockIdx.x; item < W.nitems; item += gridDim.x) {
    const int k = find_slot(W, item);
    const MemberDev& d = md[W.order[k]];
    const long long tid = (item - W.start[k]) * blockDim.x + threadIdx.x;
    switch (d.G.N) {
      case 4: batch_rhs_item<4>(d, tid, src, mode, qin, qout, sD, sDl, sDr); break;
      case 5: batch_rhs_item<5>(d, tid, src, mode, qin, qout, sD, sDl, sDr); break;
      case 6: batch_rhs_item<6>(d, tid, src, mode, qin, qout, sD, sDl, sDr); break;
      default: break;
    }
    __syncthreads();
  }
}

template <bool S3>
__global__ void k_batch_stage(const MemberDev* __restrict__ md, WorkList W, const double* qin) {
  extern __shared__ double sm[];
  for (long long item = blockIdx.x; item < W.nitems; item += gridDim.x) {
    const int k = find_slot(W, item);
    const MemberDev& d = md[W.order[k]];
    const long long col0 = (item - W.start[k]) * blockDim.x;
    const double* qn = qin + d.soff;
    double* out = S3 ? d.q3 : d.q2;
    const StageCoef& sc = S3 ? d.s3 : d.s2;
    switch (d.G.N) {
      case 4: stage_body<4, S3, false, double>(col0, sm, qn, d.R1, d.R2, d.q2, out, d.G, d.R, d.F, sc, d.tb, 0); break;
      case 5: stage_body<5, S3, false, double>(col0, sm, qn, d.R1, d.R2, d.q2, out, d.G, d.R, d.F, sc, d.tb, 0); break;
      case 6: stage_body<6, S3, false, double>(col0, sm, qn, d.R1, d.R2, d.q2, out, d.G, d.R, d.F, sc, d.tb, 0); break;
      default: break;
    }
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

struct numa_batch {
  std::vector<numa_ctx*> mem;
  cudaStream_t stream = nullptr;
  std::string err;
  MemberDev* d_md = nullptr;
  std::vector<long long> soff;
  long long total = 0;                 // doubles of one packed state
  HostList node_list, rhs_list, col_list;
  int rhs_threads = 256, col_tile = 64;
  int grid_node = 0, grid_rhs = 0, grid_col = 0;
  size_t stage_smem = 0;
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

int build_lists(numa_batch* b) {
  const int n = (int)b->mem.size();
  std::vector<int> natural(n);
  for (int m = 0; m < n; ++m) natural[m] = m;
  std::vector<long long> it_node(n), it_rhs(n), it_col(n);
  for (int m = 0; m < n; ++m) {
    const numa_ctx* c = b->mem[m];
    it_node[m] = (c->G.nnode + 255) / 256;
    it_rhs[m] = (c->nperm + b->rhs_threads - 1) / b->rhs_threads;
    it_col[m] = (c->G.ncol + b->col_tile - 1) / b->col_tile;
  }
  // stage items cost ~ M: deal the tallest columns first so static striding balances
  std::vector<int> by_m = natural;
  std::stable_sort(by_m.begin(), by_m.end(),
                   [&](int a, int c) { return b->mem[a]->G.M > b->mem[c]->G.M; });
  make_list(b->node_list, natural, it_node);
  make_list(b->rhs_list, natural, it_rhs);
  make_list(b->col_list, by_m, it_col);
  int rc;
  if ((rc = upload_list(b, b->node_list)) || (rc = upload_list(b, b->rhs_list)) ||
      (rc = upload_list(b, b->col_list)))
    return rc;
  int maxM = 0;
  for (auto* c : b->mem) maxM = std::max(maxM, c->G.M);
  b->stage_smem = col_smem_per_level(false, 0) * (size_t)maxM * b->col_tile;
  int dev = 0, nsm = 0, per = 0;
  NUMA_BCK(b, cudaGetDevice(&dev));
  NUMA_BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  NUMA_BCK(b, cudaFuncSetAttribute(k_batch_stage<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->stage_smem));
  NUMA_BCK(b, cudaFuncSetAttribute(k_batch_stage<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->stage_smem));
  NUMA_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_pressure, 256, 0));
  b->grid_node = nsm * std::max(per, 1);
  NUMA_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_rhs, b->rhs_threads, 0));
  b->grid_rhs = nsm * std::max(per, 1);
  NUMA_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_stage<true>, b->col_tile, b->stage_smem));
  if (per < 1) return bfail(b, NUMA_ERR_ARG, "stage tile does not fit in shared memory");
  b->grid_col = nsm * per;
  return NUMA_OK;
}

int enqueue_step(numa_batch* b, const double* qin, double* qout, cudaStream_t s) {
  const EosSeries S = eos_series();
  const WorkList Wn = b->node_list.dev(), Wr = b->rhs_list.dev(), Wc = b->col_list.dev();
  const int rt = b->rhs_threads, ct = b->col_tile;
  const size_t sm = b->stage_smem;
  k_batch_pressure<<<b->grid_node, 256, 0, s>>>(b->d_md, Wn, 0, qin, S);
  k_batch_rhs<<<b->grid_rhs, rt, 0, s>>>(b->d_md, Wr, 0, 0, qin, qout);
  k_batch_stage<false><<<b->grid_col, ct, sm, s>>>(b->d_md, Wc, qin);
  k_batch_pressure<<<b->grid_node, 256, 0, s>>>(b->d_md, Wn, 1, qin, S);
  k_batch_rhs<<<b->grid_rhs, rt, 0, s>>>(b->d_md, Wr, 1, 0, qin, qout);
  k_batch_stage<true><<<b->grid_col, ct, sm, s>>>(b->d_md, Wc, qin);
  k_batch_pressure<<<b->grid_node, 256, 0, s>>>(b->d_md, Wn, 2, qin, S);
  k_batch_rhs<<<b->grid_rhs, rt, 0, s>>>(b->d_md, Wr, 2, 2, qin, qout);
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

// Autotuner: time the right-hand side for each threads-per-CTA candidate and the stage
// for each columns-per-CTA candidate on the ensemble (rest state), keep the fastest.
int autotune(numa_batch* b) {
  cudaEvent_t e0, e1;
  NUMA_BCK(b, cudaEventCreate(&e0));
  NUMA_BCK(b, cudaEventCreate(&e1));
  NUMA_BCK(b, cudaMemsetAsync(b->d_state, 0, b->total * sizeof(double), b->stream));
  const EosSeries S = eos_series();
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
  k_batch_pressure<<<b->grid_node, 256, 0, b->stream>>>(b->d_md, b->node_list.dev(), 0, b->d_state, S);
  const int rhs_c[2] = {128, 256};
  float best = 1e30f;
  int best_rt = 256;
  for (int rt : rhs_c) {
    b->rhs_threads = rt;
    if ((rc = build_lists(b))) break;
    float ms = 0;
    rc = time_it([&] { k_batch_rhs<<<b->grid_rhs, rt, 0, b->stream>>>(b->d_md, b->rhs_list.dev(), 0, 0, b->d_state, b->d_state); }, &ms);
    if (rc) break;
    b->tune_ms.push_back(ms);
    if (ms < best) { best = ms; best_rt = rt; }
  }
  b->rhs_threads = best_rt;
  const int col_c[3] = {32, 64, 96};
  best = 1e30f;
  int best_ct = 64;
  for (int ct : col_c) {
    if (rc) break;
    b->col_tile = ct;
    if ((rc = build_lists(b))) { rc = NUMA_OK; b->err.clear(); continue; }   // does not fit: skip
    float ms = 0;
    rc = time_it([&] { k_batch_stage<false><<<b->grid_col, ct, b->stage_smem, b->stream>>>(b->d_md, b->col_list.dev(), b->d_state); }, &ms);
    if (rc) break;
    b->tune_ms.push_back(ms);
    if (ms < best) { best = ms; best_ct = ct; }
  }
  b->col_tile = best_ct;
  if (!rc) rc = build_lists(b);
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
  free_list(b->rhs_list);
  free_list(b->col_list);
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

int numa_batch_tuning(const numa_batch* b, int* rhs_threads, int* col_tile) {
  if (!b) return NUMA_ERR_ARG;
  if (rhs_threads) *rhs_threads = b->rhs_threads;
  if (col_tile) *col_tile = b->col_tile;
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
