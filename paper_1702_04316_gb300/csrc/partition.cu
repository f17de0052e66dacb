// Horizontal partition of the box for several GPUs (Sec. "IMEX time integration": in HEVI
// the implicit column solves cross no partition boundary, so the only exchange is the
// horizontal halo that the explicit right-hand side reads; Sec. "Scalability").
//
// Rank r of a px x py process grid owns a rectangle of elements.  It computes on a window:
// its rectangle plus one element toward every neighbour, set up as a box of its own (a
// context of the window's size).  Node-column ownership: a rank owns the node columns
// [ex0 N, ex1 N) x [ey0 N, ey1 N) of the global grid, plus the last node column where its
// rectangle touches the east or north wall.  Every other node column of the window is
// halo, owned by exactly one other rank.  Once the halo holds the owners' values, the
// right-hand side at every owned node is exact: its stencil stays within the elements
// around it, all inside the window, with the same interface / interior / wall rows as on
// the whole mesh (the window's artificial walls lie one element beyond the owned nodes).
//
// The exchange lists pair up: the columns rank a sends to rank b are the columns b receives
// from a, both sorted by global column id.
//
// Also here: the gather / scatter kernels that move listed node columns of several fields
// into and out of one contiguous buffer (the halo messages).
#include <algorithm>
#include <cmath>
#include <vector>

#include "numa.h"
#include "numa_internal.cuh"
#include "numa_ctx.h"

namespace {

struct Rect {           // node columns [x0, x1) x [y0, y1) of the global grid
  int x0, x1, y0, y1;
  bool has(int ix, int iy) const { return ix >= x0 && ix < x1 && iy >= y0 && iy < y1; }
};

struct Block {
  int ex0, ex1, ey0, ey1, wx0, wx1, wy0, wy1;
  Rect own, win;
};

Block block_of(const numa_mesh_desc& g, int N, int px, int py, int r) {
  const int bx = r % px, by = r / px;
  Block b;
  b.ex0 = (int)((long long)g.nex * bx / px);
  b.ex1 = (int)((long long)g.nex * (bx + 1) / px);
  b.ey0 = (int)((long long)g.ney * by / py);
  b.ey1 = (int)((long long)g.ney * (by + 1) / py);
  b.wx0 = std::max(0, b.ex0 - 1);
  b.wx1 = std::min(g.nex, b.ex1 + 1);
  b.wy0 = std::max(0, b.ey0 - 1);
  b.wy1 = std::min(g.ney, b.ey1 + 1);
  b.own = Rect{b.ex0 * N, b.ex1 * N + (b.ex1 == g.nex ? 1 : 0), b.ey0 * N,
               b.ey1 * N + (b.ey1 == g.ney ? 1 : 0)};
  b.win = Rect{b.wx0 * N, b.wx1 * N + 1, b.wy0 * N, b.wy1 * N + 1};
  return b;
}

int check_part(const numa_mesh_desc* g, int N, const numa_part_desc* p) {
  if (!g || !p || N < 1 || N > NUMA_MAXN || g->nex < 1 || g->ney < 1 || g->nez < 1 ||
      !(g->Lx > 0) || !(g->Ly > 0) || !(g->Lz > 0) || p->px < 1 || p->py < 1 || p->rank < 0 ||
      p->rank >= p->px * p->py)
    return NUMA_ERR_ARG;
  // every rectangle at least two elements wide: the window then meets its eight neighbours
  // at most
  if (g->nex < 2 * p->px && p->px > 1) return NUMA_ERR_ARG;
  if (g->ney < 2 * p->py && p->py > 1) return NUMA_ERR_ARG;
  return NUMA_OK;
}

// The node columns of a's window that lie in both regions, sorted by global column id, as
// window-local ids of a's window (out may be NULL: count only).  (region_own, region_win) =
// (b.own, a.win): what a receives from b; (a.own, b.win): what a sends to b.
void list_columns(const Block& a, const Rect& region_own, const Rect& region_win, int* out,
                  int* count) {
  const int nxw = a.win.x1 - a.win.x0;
  int n = 0;
  for (int iy = a.win.y0; iy < a.win.y1; ++iy)
    for (int ix = a.win.x0; ix < a.win.x1; ++ix)
      if (region_own.has(ix, iy) && region_win.has(ix, iy)) {
        if (out) out[n] = (iy - a.win.y0) * nxw + (ix - a.win.x0);
        ++n;
      }
  *count = n;
}

// The neighbours of rank me (every other rank whose owned columns meet my window, or whose
// window meets my owned columns), in rank order.
std::vector<int> neighbours(const numa_mesh_desc& g, int N, const numa_part_desc& p) {
  const Block me = block_of(g, N, p.px, p.py, p.rank);
  std::vector<int> out;
  for (int r = 0; r < p.px * p.py; ++r) {
    if (r == p.rank) continue;
    const Block o = block_of(g, N, p.px, p.py, r);
    int nr = 0, ns = 0;
    list_columns(me, o.own, me.win, nullptr, &nr);
    list_columns(me, me.own, o.win, nullptr, &ns);
    if (nr || ns) out.push_back(r);
  }
  return out;
}

// ---- gather / scatter of listed node columns -------------------------------------------------
constexpr int kMaxFields = 8;
struct FieldPtrs {
  double* f[kMaxFields];
};

// buf[(f ncols + c) M + lev] <- fields[f][cols[c] M + lev]: one thread per value, the M levels
// of a column consecutive on both sides.  A listed column outside [0, ncol_ctx) is skipped and
// latches NUMA_ST_RANGE.
__global__ void k_gather_columns(FieldPtrs F, int nf, const int* __restrict__ cols, long long ncols,
                                 int M, long long ncol_ctx, double* __restrict__ buf,
                                 unsigned* status) {
  const long long n = (long long)nf * ncols * M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long fc = t / M;
    const int lev = (int)(t - fc * M);
    const int f = (int)(fc / ncols);
    const long long c = fc - (long long)f * ncols;
    const int col = cols[c];
    if (col < 0 || col >= ncol_ctx) {
      atomicOr(status, NUMA_ST_RANGE);
      continue;
    }
    buf[t] = F.f[f][(long long)col * M + lev];
  }
}

__global__ void k_scatter_columns(FieldPtrs F, int nf, const int* __restrict__ cols, long long ncols,
                                  int M, long long ncol_ctx, const double* __restrict__ buf,
                                  unsigned* status) {
  const long long n = (long long)nf * ncols * M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long fc = t / M;
    const int lev = (int)(t - fc * M);
    const int f = (int)(fc / ncols);
    const long long c = fc - (long long)f * ncols;
    const int col = cols[c];
    if (col < 0 || col >= ncol_ctx) {
      atomicOr(status, NUMA_ST_RANGE);
      continue;
    }
    F.f[f][(long long)col * M + lev] = buf[t];
  }
}

int columns_args(const numa_ctx* ctx, const void* const* fields, int nf, const int* cols,
                 long long ncols, const void* buf, FieldPtrs& F) {
  if (!ctx || !fields || nf < 1 || nf > kMaxFields || ncols < 0 || (ncols > 0 && (!cols || !buf)))
    return NUMA_ERR_ARG;
  if (((uintptr_t)cols % 4) || ((uintptr_t)buf % 8)) return NUMA_ERR_ARG;
  for (int f = 0; f < nf; ++f) {
    if (!fields[f] || ((uintptr_t)fields[f] % 8)) return NUMA_ERR_ARG;
    F.f[f] = (double*)fields[f];
  }
  return NUMA_OK;
}

// A box length L with L / n == h exactly, so that the window's element size (and with it
// every metric term of its context) equals the whole mesh's bit for bit.
double span_for(double h, int n) {
  double L = h * n;
  for (int it = 0; it < 64 && L / n != h; ++it)
    L = std::nextafter(L, (L / n < h) ? HUGE_VAL : -HUGE_VAL);
  return L;
}

unsigned columns_grid(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16));
}

}  // namespace

extern "C" {

int numa_part_plan(const numa_mesh_desc* global, int N, const numa_part_desc* part,
                   numa_part_info* info) {
  int rc = check_part(global, N, part);
  if (rc) return rc;
  if (!info) return NUMA_ERR_ARG;
  const Block b = block_of(*global, N, part->px, part->py, part->rank);
  numa_part_info o{};
  o.ex0 = b.ex0; o.ex1 = b.ex1; o.ey0 = b.ey0; o.ey1 = b.ey1;
  o.wx0 = b.wx0; o.wx1 = b.wx1; o.wy0 = b.wy0; o.wy1 = b.wy1;
  o.window = *global;
  o.window.nex = b.wx1 - b.wx0;
  o.window.ney = b.wy1 - b.wy0;
  o.window.Lx = span_for(global->Lx / global->nex, o.window.nex);
  o.window.Ly = span_for(global->Ly / global->ney, o.window.ney);
  o.own_x0 = b.own.x0 - b.win.x0; o.own_x1 = b.own.x1 - b.win.x0;
  o.own_y0 = b.own.y0 - b.win.y0; o.own_y1 = b.own.y1 - b.win.y0;
  const std::vector<int> nb = neighbours(*global, N, *part);
  if (nb.size() > NUMA_PART_MAX_NEIGH) return NUMA_ERR_ARG;
  o.nneigh = (int)nb.size();
  for (int k = 0; k < o.nneigh; ++k) {
    const Block n = block_of(*global, N, part->px, part->py, nb[k]);
    o.neigh[k] = nb[k];
    list_columns(b, n.own, b.win, nullptr, &o.nrecv[k]);
    list_columns(b, b.own, n.win, nullptr, &o.nsend[k]);
  }
  *info = o;
  return NUMA_OK;
}

int numa_part_columns(const numa_mesh_desc* global, int N, const numa_part_desc* part, int k,
                      int* send_cols, int* recv_cols) {
  int rc = check_part(global, N, part);
  if (rc) return rc;
  const std::vector<int> nb = neighbours(*global, N, *part);
  if (k < 0 || k >= (int)nb.size() || !send_cols || !recv_cols) return NUMA_ERR_ARG;
  const Block b = block_of(*global, N, part->px, part->py, part->rank);
  const Block n = block_of(*global, N, part->px, part->py, nb[k]);
  int c;
  list_columns(b, b.own, n.win, send_cols, &c);
  list_columns(b, n.own, b.win, recv_cols, &c);
  return NUMA_OK;
}

int numa_gather_columns(numa_ctx* ctx, const double* const* fields, int nf, const int* cols,
                        long long ncols, double* buf) {
  FieldPtrs F{};
  int rc = columns_args(ctx, (const void* const*)fields, nf, cols, ncols, buf, F);
  if (rc) return rc;
  const long long n = (long long)nf * ncols * ctx->G.M;
  if (n == 0) return NUMA_OK;
  k_gather_columns<<<columns_grid(n), 256, 0, ctx->stream>>>(F, nf, cols, ncols, ctx->G.M,
                                                              ctx->G.ncol, buf, ctx->d_status);
  return cudaGetLastError() == cudaSuccess ? NUMA_OK : NUMA_ERR_CUDA;
}

int numa_scatter_columns(numa_ctx* ctx, double* const* fields, int nf, const int* cols,
                         long long ncols, const double* buf) {
  FieldPtrs F{};
  int rc = columns_args(ctx, (const void* const*)fields, nf, cols, ncols, buf, F);
  if (rc) return rc;
  const long long n = (long long)nf * ncols * ctx->G.M;
  if (n == 0) return NUMA_OK;
  k_scatter_columns<<<columns_grid(n), 256, 0, ctx->stream>>>(F, nf, cols, ncols, ctx->G.M,
                                                               ctx->G.ncol, buf, ctx->d_status);
  return cudaGetLastError() == cudaSuccess ? NUMA_OK : NUMA_ERR_CUDA;
}

}  // extern "C"
