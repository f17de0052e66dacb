// C ABI of libnuma (declared in include/numa.h): the context, the host-side set-up
// (LGL tables, reference state, column derivative and stage tables) and the entry points
// that enqueue the kernels of rhs.cu, column.cu (with column_stage_n*.cu) and misc.cu.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <initializer_list>
#include <string>
#include <vector>

#include "numa.h"
#include "numa_internal.cuh"
#include "numa_ctx.h"

namespace {

// ---- ARK2 tableau (Table 1; b = b~ = last implicit row) --------------------------------
struct Ark2 {
  double a[3][3], at[3][3], b[3];
  Ark2() {
    const double s2 = std::sqrt(2.0);
    std::memset(this, 0, sizeof(*this));
    a[1][0] = 2.0 - s2;
    a[2][1] = (3.0 + 2.0 * s2) / 6.0;
    a[2][0] = 1.0 - a[2][1];
    at[1][0] = at[1][1] = 1.0 - 1.0 / s2;
    at[2][0] = at[2][1] = 1.0 / (2.0 * s2);
    at[2][2] = 1.0 - 1.0 / s2;
    for (int i = 0; i < 3; ++i) b[i] = at[2][i];
  }
};

// ARK3: the ARK3(2)4L[2]SA scheme of Kennedy and Carpenter (2003), the third-order member
// of the ARK family (the paper runs ARK3 but prints no tableau).  Explicit / ESDIRK pair,
// four stages, implicit diagonal gamma, b = b~ = the last implicit row.  Published
// rational coefficients, each evaluated as one correctly rounded division.
struct Ark3 {
  double a[4][4], at[4][4], b[4];
  Ark3() {
    std::memset(this, 0, sizeof(*this));
    const double g = 1767732205903.0 / 4055673282236.0;
    at[1][0] = at[1][1] = g;
    at[2][0] = 2746238789719.0 / 10658868560708.0;
    at[2][1] = -640167445237.0 / 6845629431997.0;
    at[2][2] = g;
    at[3][0] = 1471266399579.0 / 7840856788654.0;
    at[3][1] = -4482444167858.0 / 7529755066697.0;
    at[3][2] = 11266239266428.0 / 11593286722821.0;
    at[3][3] = g;
    a[1][0] = 1767732205903.0 / 2027836641118.0;
    a[2][0] = 5535828885825.0 / 10492691773637.0;
    a[2][1] = 788022342437.0 / 10882634858940.0;
    a[3][0] = 6485989280629.0 / 16251701735622.0;
    a[3][1] = -4246266847089.0 / 9704473918619.0;
    a[3][2] = 10755448449292.0 / 10357097424841.0;
    for (int i = 0; i < 4; ++i) b[i] = at[3][i];
  }
};

// ARK4, ARK5: the ARK4(3)6L[2]SA and ARK5(4)8L[2]SA schemes of Kennedy and Carpenter (2003)
// for the paper's fourth- and fifth-order runs (no tableau printed).  Same structure as
// ARK3: a~_11 = 0, one implicit diagonal, b = b~ = the last implicit row.  Every entry is
// a published rational evaluated as one correctly rounded division, except ARK5's explicit
// a_86 and a_87: the solution of its 143 fifth-order conditions with the other entries
// fixed (it meets them to 2e-26, the precision of the published rationals).
struct Rat {
  double p, q;
};

template <int S>
struct ArkRat {
  double a[S][S] = {}, at[S][S] = {};
  void row(double (*m)[S], int i, std::initializer_list<Rat> r) {
    int j = 0;
    for (const Rat& x : r) m[i][j++] = x.p / x.q;
  }
};

struct Ark4 : ArkRat<6> {
  Ark4() {
    const Rat g{1, 4}, z{0, 1};
    row(at, 1, {g, g});
    row(at, 2, {{8611, 62500}, {-1743, 31250}, g});
    row(at, 3, {{5012029, 34652500}, {-654441, 2922500}, {174375, 388108}, g});
    row(at, 4, {{15267082809.0, 155376265600.0}, {-71443401, 120774400}, {730878875, 902184768},
                {2285395, 8070912}, g});
    row(at, 5, {{82889, 524892}, z, {15625, 83664}, {69875, 102672}, {-2260, 8211}, g});
    row(a, 1, {{1, 2}});
    row(a, 2, {{13861, 62500}, {6889, 62500}});
    row(a, 3, {{-116923316275.0, 2393684061468.0}, {-2731218467317.0, 15368042101831.0},
               {9408046702089.0, 11113171139209.0}});
    row(a, 4, {{-451086348788.0, 2902428689909.0}, {-2682348792572.0, 7519795681897.0},
               {12662868775082.0, 11960479115383.0}, {3355817975965.0, 11060851509271.0}});
    row(a, 5, {{647845179188.0, 3216320057751.0}, {73281519250.0, 8382639484533.0},
               {552539513391.0, 3454668386233.0}, {3354512671639.0, 8306763924573.0},
               {4040, 17871}});
  }
};

struct Ark5 : ArkRat<8> {
  Ark5() {
    const Rat g{41, 200}, z{0, 1};
    row(at, 1, {g, g});
    row(at, 2, {{41, 400}, {-567603406766.0, 11931857230679.0}, g});
    row(at, 3, {{683785636431.0, 9252920307686.0}, z, {-110385047103.0, 1367015193373.0}, g});
    row(at, 4, {{3016520224154.0, 10081342136671.0}, z, {30586259806659.0, 12414158314087.0},
                {-22760509404356.0, 11113319521817.0}, g});
    row(at, 5, {{218866479029.0, 1489978393911.0}, z, {638256894668.0, 5436446318841.0},
                {-1179710474555.0, 5321154724896.0}, {-60928119172.0, 8023461067671.0}, g});
    row(at, 6, {{1020004230633.0, 5715676835656.0}, z, {25762820946817.0, 25263940353407.0},
                {-2161375909145.0, 9755907335909.0}, {-211217309593.0, 5846859502534.0},
                {-4269925059573.0, 7827059040749.0}, g});
    row(at, 7, {{-872700587467.0, 9133579230613.0}, z, z, {22348218063261.0, 9555858737531.0},
                {-1143369518992.0, 8141816002931.0}, {-39379526789629.0, 19018526304540.0},
                {32727382324388.0, 42900044865799.0}, g});
    row(a, 1, {{41, 100}});
    row(a, 2, {{367902744464.0, 2072280473677.0}, {677623207551.0, 8224143866563.0}});
    row(a, 3, {{1268023523408.0, 10340822734521.0}, z, {1029933939417.0, 13636558850479.0}});
    row(a, 4, {{14463281900351.0, 6315353703477.0}, z, {66114435211212.0, 5879490589093.0},
               {-54053170152839.0, 4284798021562.0}});
    row(a, 5, {{14090043504691.0, 34967701212078.0}, z, {15191511035443.0, 11219624916014.0},
               {-18461159152457.0, 12425892160975.0}, {-281667163811.0, 9011619295870.0}});
    row(a, 6, {{19230459214898.0, 13134317526959.0}, z, {21275331358303.0, 2942455364971.0},
               {-38145345988419.0, 4862620318723.0}, {-1, 8}, {-1, 8}});
    row(a, 7, {{-19977161125411.0, 11928030595625.0}, z, {-40795976796054.0, 6384907823539.0},
               {177454434618887.0, 12078138498510.0}, {782672205425.0, 8267701900261.0},
               {-56156175540813.0, 7787401243552.0}, {21501425855156.0, 14444669418411.0}});
  }
};

// The scheme of a context as one s-stage table (s = 3, 4, 6 or 8).
struct ArkTab {
  int s = 3;
  double a[NUMA_MAX_STAGES][NUMA_MAX_STAGES] = {}, at[NUMA_MAX_STAGES][NUMA_MAX_STAGES] = {},
         b[NUMA_MAX_STAGES] = {};
  template <typename K>
  void set(int n, const K& k) {
    s = n;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        a[i][j] = k.a[i][j];
        at[i][j] = k.at[i][j];
      }
    for (int j = 0; j < n; ++j) b[j] = at[n - 1][j];
  }
};

ArkTab ark_tab(int scheme) {
  ArkTab t;
  if (scheme == NUMA_SCHEME_ARK3) {
    static const Ark3 k;
    t.set(4, k);
  } else if (scheme == NUMA_SCHEME_ARK4) {
    static const Ark4 k;
    t.set(6, k);
  } else if (scheme == NUMA_SCHEME_ARK5) {
    static const Ark5 k;
    t.set(8, k);
  } else {
    static const Ark2 k;
    t.set(3, k);
  }
  return t;
}

// State-sized workspace vectors of the FP64 1D-IMEX step: R(q(j)) for every stage j and the
// stage states q(2) .. q(s) (ARK2: R1, R2, q2, q3; the last R goes to the final update).
int work_states(int scheme) {
  if (scheme == NUMA_SCHEME_ARK2) return 4;
  if (scheme == NUMA_SCHEME_ARK3) return 6;
  return 2 * ark_tab(scheme).s - 1;
}

// ---- RK35: five-stage third-order SSP, two-register Shu-Osher form -------------------
//   u_i = alpha_i u_0 + (1 - alpha_i) u_{i-1} + beta_i dt F(u_{i-1});  beta_1 = beta_5 =
//   0.46, alpha_2 = alpha_3 = alpha_5 = 0, the rest the real root of the third-order
//   conditions with beta_2 > beta_3 (SSP coefficient 1/0.46).
const double kRkAlpha[5] = {0.0, 0.0, 0.0, 0.5764252463942515726402586, 0.0};
const double kRkBeta[5] = {0.46, 0.2805744403033042654640453, 0.22110850739434604175949,
                           0.1326553823821179192508848, 0.46};

// ---- LGL nodes, weights and derivative matrix --------------------------------------------
// P_N and P_{N-1} by the three-term recurrence.
void legendre(int N, double x, double& PN, double& PNm1) {
  double p0 = 1.0, p1 = x;
  if (N == 0) { PN = 1.0; PNm1 = 0.0; return; }
  for (int n = 1; n < N; ++n) {
    const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
    p0 = p1;
    p1 = p2;
  }
  PN = p1;
  PNm1 = p0;
}

// Interior LGL nodes are the roots of f(x) = x P_N - P_{N-1} = (x^2-1) P_N'/N inside
// (-1, 1); with x P_N' - P_{N-1}' = N P_N one gets f' = (N+1) P_N, so Newton reads
// x <- x - (x P_N - P_{N-1}) / ((N+1) P_N), started from the Chebyshev-Lobatto points.
void lgl_host(int N, double* x, double* w, double* D) {
  const int Nq = N + 1;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double xj = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double PN, PNm1;
      legendre(N, xj, PN, PNm1);
      const double dx = (xj * PN - PNm1) / ((N + 1.0) * PN);
      xj -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[j] = xj;
  }
  for (int j = 0; j < Nq / 2; ++j) {    // exact mirror symmetry
    const double s = 0.5 * (x[N - j] - x[j]);
    x[j] = -s;
    x[N - j] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  double PNv[NUMA_MAXNQ];                // no heap: numa_rhs_explicit_static calls this too
  for (int j = 0; j < Nq; ++j) {
    double PN, PNm1;
    legendre(N, x[j], PN, PNm1);
    PNv[j] = PN;
    w[j] = 2.0 / (N * (N + 1.0) * PN * PN);
  }
  for (int i = 0; i < Nq; ++i)
    for (int j = 0; j < Nq; ++j)
      D[i * Nq + j] = (i == j) ? 0.0 : PNv[i] / (PNv[j] * (x[i] - x[j]));
  D[0] = -N * (N + 1) / 4.0;
  D[N * Nq + N] = N * (N + 1) / 4.0;
}

void set_axis(AxisCoef& c, int N, const double* w, const double* D, double h) {
  const int Nq = N + 1;
  std::memset(&c, 0, sizeof(c));
  const double s = 2.0 / h;
  for (int i = 0; i < Nq; ++i)
    for (int n = 0; n < Nq; ++n) c.D[i * Nq + n] = D[i * Nq + n] * s;
  const double wl = w[N], wr = w[0];
  for (int n = 0; n < Nq; ++n) {
    c.Dl[n] = wl / (wl + wr) * D[N * Nq + n] * s;
    c.Dr[n] = wr / (wl + wr) * D[0 * Nq + n] * s;
  }
}

}  // namespace

namespace {

int fail(numa_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(numa_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, NUMA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define NUMA_CK(ctx, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

}  // namespace

// Event pair around one launch when profiling is on (index into ctx->prof, or -1).
long prof_begin(numa_ctx* c, int kind) {
  if (!c->prof_on) return -1;
  if (c->prof_n == c->prof.size()) {
    numa_ctx::ProfRec r{kind, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
    c->prof.push_back(r);
  }
  numa_ctx::ProfRec& r = c->prof[c->prof_n];
  r.kind = kind;
  cudaEventRecord(r.a, c->stream);
  return (long)c->prof_n++;
}

void prof_end(numa_ctx* c, long idx) {
  if (idx >= 0) cudaEventRecord(c->prof[idx].b, c->stream);
}

namespace {

void free_all(numa_ctx* c) {
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  cudaFree(c->d_lev);
  cudaFree(c->d_levi);
  cudaFree(c->d_stage_tab);
  cudaFree(c->F.L);
  cudaFree(c->F.U);
  cudaFree(c->F.L32);
  cudaFree(c->F.U32);
  cudaFree(c->d_work);
  cudaFree(c->d_perm);
  cudaFree(c->d_status);
  cudaFree(c->d_count);
  cudaFree(c->d_hoststate);
  for (cudaEvent_t e : c->host_ev) cudaEventDestroy(e);
  if (c->cs_in) cudaStreamDestroy(c->cs_in);
  if (c->cs_out) cudaStreamDestroy(c->cs_out);
  if (c->cs_p) cudaStreamDestroy(c->cs_p);
  cudaFree(c->d_adj);
  cudaFree(c->d_adjtab);
  cudaFree(c->d_w3);
  cudaFree(c->F2);
}

// Host reference state and the column derivative (Sec. "Equation Set2NC",
// Sec. "Direct stiffness summation"), written into caller-provided arrays of M levels (the
// band: M x (2N + 1)) without heap storage.  The one builder of these tables: contexts and
// numa_rhs_explicit_static both call it, so their tables are the same bits.
void ref_tables_host(int N, int nez, double dz, const double* xi, const double* w,
                     const double* D, double theta_s, double n_bv, double* z, double* theta0,
                     double* rho0, double* P0, double* G0, double* H0, double* dzband,
                     double* drho0, double* dtheta0, double* F0z) {
  const int M = nez * N + 1, Nq = N + 1, W = 2 * N + 1;
  const double g = NUMA_GRAV, cp = NUMA_CP, R = NUMA_RGAS, gam = NUMA_GAMMA;
  for (int m = 0; m < M; ++m) {
    // an interface node takes the upper element's coordinate expression
    const int ez = (m == M - 1) ? nez - 1 : m / N, k = m - ez * N;
    const double zz = ez * dz + (1.0 + xi[k]) * dz / 2.0;
    double th, pi;
    if (n_bv == 0.0) {
      th = theta_s;
      pi = 1.0 - g * zz / (cp * theta_s);
    } else {
      const double s = n_bv * n_bv / g;
      th = theta_s * std::exp(s * zz);
      pi = 1.0 + g * g / (cp * theta_s * n_bv * n_bv) * (std::exp(-s * zz) - 1.0);
    }
    z[m] = zz;
    P0[m] = NUMA_P00 * std::pow(pi, cp / R);
    theta0[m] = th;
    rho0[m] = P0[m] / (R * pi * th);
    G0[m] = gam * P0[m] / rho0[m];
    H0[m] = gam * P0[m] / th;
  }
  // DSS'd vertical derivative: element ez gives node m = ez*N + k the row (2/dz) D[k,:]
  // weighted by w_k; the summed rows (lower element first) are divided by the summed weights.
  for (int m = 0; m < M; ++m) {
    double* row = dzband + (size_t)m * W;
    for (int b = 0; b < W; ++b) row[b] = 0.0;
    double den = 0.0;
    for (int ez = 0; ez < nez; ++ez) {
      const int k = m - ez * N;
      if (k < 0 || k > N) continue;
      for (int n = 0; n < Nq; ++n) row[ez * N + n - m + N] += w[k] * D[k * Nq + n] * (2.0 / dz);
      den += w[k];
    }
    for (int b = 0; b < W; ++b) row[b] /= den;
  }
  for (int m = 0; m < M; ++m) {
    drho0[m] = dtheta0[m] = 0.0;
    for (int b = 0; b < W; ++b) {
      const int j = m - N + b;
      if (j < 0 || j >= M) continue;
      // D_z annihilates constants: taking the surface value out first is exact and gives
      // an isentropic theta0 a gradient of exactly zero.
      drho0[m] += dzband[(size_t)m * W + b] * (rho0[j] - rho0[0]);
      dtheta0[m] += dzband[(size_t)m * W + b] * (theta0[j] - theta0[0]);
    }
    F0z[m] = G0[m] * drho0[m] + H0[m] * dtheta0[m];
  }
}

void build_levels(numa_ctx* c, const double* xi, const double* w, const double* D, double dz) {
  const int N = c->G.N, M = c->G.M, W = 2 * N + 1;
  c->z.resize(M); c->theta0.resize(M); c->rho0.resize(M); c->P0.resize(M); c->G0.resize(M);
  c->H0.resize(M); c->dzband.resize((size_t)M * W); c->drho0.resize(M); c->dtheta0.resize(M);
  c->F0z.resize(M);
  ref_tables_host(N, c->G.nez, dz, xi, w, D, c->theta_s, c->n_bv, c->z.data(), c->theta0.data(),
                  c->rho0.data(), c->P0.data(), c->G0.data(), c->H0.data(), c->dzband.data(),
                  c->drho0.data(), c->dtheta0.data(), c->F0z.data());
}

// The non-zero entries of each row of the column derivative band: coef[m W + t] at level
// m + off[m W + t] for t < off[M W + m] (off holds M W offsets, then M counts).
void dz_taps(const numa_ctx* c, double* coef, int* off) {
  const int M = c->G.M, N = c->G.N, W = 2 * N + 1;
  for (int m = 0; m < M; ++m) {
    int n = 0;
    for (int b = 0; b < W; ++b) {
      const double v = c->dzband[(size_t)m * W + b];
      if (v == 0.0) continue;
      coef[(size_t)m * W + n] = v;
      off[(size_t)m * W + n] = b - N;
      ++n;
    }
    off[(size_t)M * W + m] = n;
  }
}

int upload_levels(numa_ctx* c) {
  const int M = c->G.M, N = c->G.N, W = 2 * N + 1;
  const int nt = 10;
  std::vector<double> h((size_t)nt * M + 2 * (size_t)M * W + 5 * (size_t)M, 0.0);
  auto put = [&](int slot, const std::vector<double>& v) {
    std::memcpy(&h[(size_t)slot * M], v.data(), sizeof(double) * M);
  };
  std::vector<double> inv_rho0(M), inv_theta0(M);
  for (int m = 0; m < M; ++m) {
    inv_rho0[m] = 1.0 / c->rho0[m];
    inv_theta0[m] = 1.0 / c->theta0[m];
  }
  put(0, c->rho0); put(1, inv_rho0); put(2, c->theta0); put(3, inv_theta0); put(4, c->P0);
  put(5, c->G0); put(6, c->H0); put(7, c->drho0); put(8, c->dtheta0); put(9, c->F0z);
  std::memcpy(&h[(size_t)nt * M], c->dzband.data(), sizeof(double) * M * W);
  // tap lists: the non-zero entries of each band row
  double* dzc = &h[(size_t)nt * M + (size_t)M * W];
  std::vector<int> hi((size_t)M * W + M, 0);
  dz_taps(c, dzc, hi.data());
  eos_level_coefs(c->P0.data(), M, dzc + (size_t)M * W);
  NUMA_CK(c, cudaMalloc(&c->d_lev, h.size() * sizeof(double)));
  NUMA_CK(c, cudaMemcpy(c->d_lev, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  NUMA_CK(c, cudaMalloc(&c->d_levi, hi.size() * sizeof(int)));
  NUMA_CK(c, cudaMemcpy(c->d_levi, hi.data(), hi.size() * sizeof(int), cudaMemcpyHostToDevice));
  const double* d = c->d_lev;
  c->R = RefLev{d, d + M, d + 2 * M, d + 3 * M, d + 4 * M, d + 5 * M, d + 6 * M,
                d + 7 * M, d + 8 * M, d + 9 * M, d + (size_t)nt * M,
                d + (size_t)nt * M + (size_t)M * W, c->d_levi, c->d_levi + (size_t)M * W,
                d + (size_t)nt * M + 2 * (size_t)M * W};
  return NUMA_OK;
}

// Stage tables for one lam (the coefficient tables listed with StageTab).
int upload_stage_tables(numa_ctx* c, double lam) {
  const int M = c->G.M, W = 2 * c->G.N + 1;
  const double g = NUMA_GRAV;
  std::vector<double> h((size_t)11 * M + 2 * (size_t)M * W, 0.0);
  for (int m = 0; m < M; ++m) {
    const bool wall = (m == 0 || m == M - 1);
    const double A = 1.0 + lam * lam * g * c->dtheta0[m] / c->theta0[m];
    h[0 * M + m] = lam * g / c->theta0[m];
    h[1 * M + m] = wall ? 0.0 : 1.0 / A;
    h[2 * M + m] = lam * c->F0z[m];
    h[3 * M + m] = lam * c->rho0[m] * c->G0[m];
    h[4 * M + m] = wall ? 0.0 : lam / (A * c->rho0[m]);
    h[5 * M + m] = wall ? 0.0 : lam * g / (A * c->G0[m] * c->rho0[m]);
    h[6 * M + m] = lam * c->dtheta0[m];
    h[7 * M + m] = 1.0 / c->G0[m];
    h[8 * M + m] = c->H0[m] / c->G0[m];
    h[9 * M + m] = c->G0[m];
    h[10 * M + m] = c->H0[m];
  }
  std::vector<double> coef((size_t)M * W, 0.0);
  std::vector<int> off((size_t)M * W + M, 0);
  dz_taps(c, coef.data(), off.data());
  double* dzD = &h[(size_t)11 * M];
  double* dzP = dzD + (size_t)M * W;
  for (int m = 0; m < M; ++m)
    for (int t = 0; t < W; ++t) {
      dzD[(size_t)m * W + t] = h[3 * M + m] * coef[(size_t)m * W + t];
      dzP[(size_t)m * W + t] = h[4 * M + m] * coef[(size_t)m * W + t];
    }
  if (!c->d_stage_tab) NUMA_CK(c, cudaMalloc(&c->d_stage_tab, h.size() * sizeof(double)));
  NUMA_CK(c, cudaMemcpyAsync(c->d_stage_tab, h.data(), h.size() * sizeof(double),
                             cudaMemcpyHostToDevice, c->stream));
  NUMA_CK(c, cudaStreamSynchronize(c->stream));
  const double* d = c->d_stage_tab;
  c->T = StageTab{d, d + M, d + 2 * M, d + 3 * M, d + 4 * M, d + 5 * M,
                  d + 6 * M, d + 7 * M, d + 8 * M, d + 9 * M, d + 10 * M, c->d_status,
                  d + 11 * M, d + 11 * M + (size_t)M * W};
  return NUMA_OK;
}

int check_ptr(numa_ctx* c, const void* p, const char* name) {
  if (!p) return fail(c, NUMA_ERR_ARG, std::string(name) + " is NULL");
  if (((uintptr_t)p) % 8) return fail(c, NUMA_ERR_ARG, std::string(name) + " not 8-byte aligned");
  return NUMA_OK;
}

// Whether two state arrays of 5 nnode doubles (a may be NULL) share any element.
bool states_overlap(const numa_ctx* c, const double* a, const double* b) {
  if (!a || !b) return false;
  const long long n5 = 5 * c->G.nnode;
  return a < b + n5 && b < a + n5;
}

// One right-hand side.  FP64 method: P' pre-pass, FP64 kernel.  Mixed form: FP64 P' and
// FP32 field copies, FP32 kernel; in mode 0, out32 receives the FP32 tendencies.
// pp_ready: c->Pp already holds P'(q) (written by the stage that produced q).
int enqueue_rhs(numa_ctx* c, const double* q, double* out, const RhsEpilogue& ep,
                float* out32 = nullptr, bool pp_ready = false) {
  long p = -1;
  const bool rhs32 = c->precision == NUMA_PREC_MIXED || c->precision == NUMA_PREC_RHS32;
  const bool df = c->precision == NUMA_PREC_DF;
  if (!pp_ready || rhs32 || df) {
    p = prof_begin(c, NUMA_K_PRESSURE);
    if (rhs32) NUMA_CK(c, launch_prep32(q, c->F32, c->G, c->R, c->stream));
    else if (df) NUMA_CK(c, launch_prep_df(q, c->F2, c->G, c->R, c->stream));
    else NUMA_CK(c, launch_pressure(q, c->Pp, c->G, c->R, c->stream, c->d_status));
    prof_end(c, p);
  }
  p = prof_begin(c, NUMA_K_RHS);
  if (df)
    NUMA_CK(c, launch_rhs_df(q, c->F2, out, c->d_perm, c->nperm, c->G, c->C, c->R, ep, c->stream));
  else if (rhs32)
    NUMA_CK(c, launch_rhs32(q, c->F32, out32, out, c->d_perm, c->nperm, c->G, c->C, c->R, ep,
                            c->stream));
  else
    NUMA_CK(c, launch_rhs(q, c->Pp, out, c->d_perm, c->nperm, c->G, c->C, c->R, ep, c->stream));
  prof_end(c, p);
  return NUMA_OK;
}

// r_float: R1, R2 are the mixed form's internal FP32 tendencies (else FP64 arrays).
// Pp_out: optional, receives P'(stage value) (FP64 Schur form).
int enqueue_stage(numa_ctx* c, int stage, const double* qn, const void* R1, const void* R2,
                  const double* q2, double* out, const StageCoef& sc, bool r_float = false,
                  double* Pp_out = nullptr) {
  long p = prof_begin(c, NUMA_K_STAGE);
  NUMA_CK(c, launch_stage(stage, qn, R1, R2, q2, out, c->G, c->R, c->F, sc, c->T, c->col_tile,
                          r_float, c->stream, nullptr, nullptr, Pp_out));
  prof_end(c, p);
  return NUMA_OK;
}

// The stage can hand the next right-hand side its P' (FP64 Schur-form 1D-IMEX).
bool fuse_pressure(const numa_ctx* c) {
  return c->precision == NUMA_PREC_FP64 && !c->F.standard && !c->imex3d;
}

}  // namespace

int numa_rhs_final(numa_ctx* c, const double* q_last, const double* qn, double* q_out,
                   const double* b) {
  RhsEpilogue ef{};
  const bool four = c->scheme == NUMA_SCHEME_ARK3;
  ef.mode = four ? 3 : 2;
  ef.b1dt = b[0] * c->dt;
  ef.b2dt = b[1] * c->dt;
  ef.b3dt = b[2] * c->dt;
  ef.b4dt = four ? b[3] * c->dt : 0.0;
  ef.u0 = qn;
  ef.R1 = c->R1;
  ef.R2 = c->R2;
  ef.R3 = four ? c->R3 : nullptr;
  return enqueue_rhs(c, q_last, q_out, ef);
}

// The previous-stage terms of stage i + 1 (0-based row i of the tableau) with nonzero
// coefficients: R[j] = R(q(j+1)), Q[j] = q(j+1) for j >= 1, q(1) = qn.
static StagePrev stage_prev(const ArkTab& t, int i, double dt, const double* qn,
                            const double* const* R, const double* const* Q) {
  StagePrev P{};
  P.qn = qn;
  for (int j = 0; j < i; ++j) {
    const double c = (t.at[i][j] - t.a[i][j]) / t.at[i][i];
    if (t.a[i][j] != 0.0) {
      P.R[P.nr] = R[j];
      P.adt[P.nr++] = t.a[i][j] * dt;
    }
    if (c != 0.0) {
      P.q[P.nq] = j ? Q[j] : qn;
      P.c[P.nq++] = c;
    }
  }
  return P;
}

StageCoef numa_stage_coef(const numa_ctx* c, int stage) {
  const ArkTab t = ark_tab(c->scheme);
  StageCoef sc{};
  const int i = stage - 1;
  sc.dt = c->dt;
  sc.lam = t.at[i][i] * c->dt;
  for (int j = 0; j < 3; ++j) {
    sc.a[j] = (j < i) ? t.a[i][j] : 0.0;
    sc.c[j] = (j < i) ? (t.at[i][j] - t.a[i][j]) / t.at[i][i] : 0.0;
  }
  return sc;
}

namespace {

}  // namespace

// ---- entry points ---------------------------------------------------------------------------
extern "C" {

int numa_init(const numa_mesh_desc* mesh, int N, double dt, void* stream, numa_ctx** out) {
  return numa_init_ex(mesh, N, dt, nullptr, stream, out);
}

int numa_init_ex(const numa_mesh_desc* mesh, int N, double dt, const numa_options* opt,
                 void* stream, numa_ctx** out) {
  if (!out) return NUMA_ERR_ARG;
  const int precision = opt ? opt->precision : NUMA_PREC_FP64;
  const int refine = opt ? opt->refine_iters : 1;
  const int form = opt ? opt->column_form : NUMA_COLUMN_SCHUR;
  const int scheme = opt ? opt->scheme : NUMA_SCHEME_ARK2;
  const int imex = opt ? opt->imex : NUMA_IMEX_1D;
  const int pbno_order = (opt && opt->pbno_order > 0) ? opt->pbno_order : 2;
  const int kmax = (opt && opt->krylov_max_iters > 0) ? opt->krylov_max_iters : 500;
  const double ktol = (opt && opt->krylov_tol > 0) ? opt->krylov_tol : 1e-12;
  const int precond = opt ? opt->precond : NUMA_PRECOND_PBNO;
  if (precond != NUMA_PRECOND_PBNO && precond != NUMA_PRECOND_COLUMN) {
    *out = nullptr;
    return NUMA_ERR_ARG;
  }
  if ((imex != NUMA_IMEX_1D && imex != NUMA_IMEX_3D) || pbno_order > NUMA_MAX_PBNO_ORDER ||
      (imex == NUMA_IMEX_3D && (precision != NUMA_PREC_FP64 || form != NUMA_COLUMN_SCHUR)) ||
      !std::isfinite(ktol)) {
    *out = nullptr;
    return NUMA_ERR_ARG;
  }
  if ((precision != NUMA_PREC_FP64 && precision != NUMA_PREC_MIXED && precision != NUMA_PREC_RHS32 &&
       precision != NUMA_PREC_DF) ||
      refine < 0 || refine > 8 ||
      (form != NUMA_COLUMN_SCHUR && form != NUMA_COLUMN_STANDARD) ||
      (form == NUMA_COLUMN_STANDARD && precision != NUMA_PREC_FP64) ||
      scheme < NUMA_SCHEME_ARK2 || scheme > NUMA_SCHEME_ARK5 ||
      (scheme != NUMA_SCHEME_ARK2 && (precision != NUMA_PREC_FP64 || form != NUMA_COLUMN_SCHUR)) ||
      (scheme >= NUMA_SCHEME_ARK4 && imex != NUMA_IMEX_1D)) {
    *out = nullptr;
    return NUMA_ERR_ARG;
  }
  *out = nullptr;
  if (!mesh || N < 1 || N > NUMA_MAXN || mesh->nex < 1 || mesh->ney < 1 || mesh->nez < 1 ||
      !(mesh->Lx > 0) || !(mesh->Ly > 0) || !(mesh->Lz > 0) || !(dt >= 0) ||
      !(mesh->n_bv >= 0) || !std::isfinite(mesh->Lx + mesh->Ly + mesh->Lz + dt))
    return NUMA_ERR_ARG;
  Geom G{};
  G.N = N; G.Nq = N + 1;
  G.nex = mesh->nex; G.ney = mesh->ney; G.nez = mesh->nez;
  G.nxg = mesh->nex * N + 1; G.nyg = mesh->ney * N + 1; G.M = mesh->nez * N + 1;
  G.ncol = (long long)G.nxg * G.nyg;
  G.nnode = G.ncol * G.M;
  const long long nelem = (long long)mesh->nex * mesh->ney * mesh->nez;
  // int32 connectivity ids and 32-bit grid dimensions bound the mesh size
  if (nelem * G.Nq * G.Nq * G.Nq >= (1LL << 31) || 5 * G.nnode >= (1LL << 40) ||
      (G.ncol + 63) / 64 >= (1LL << 31))
    return NUMA_ERR_ARG;
  numa_ctx* c = new numa_ctx();
  c->G = G;
  c->stream = (cudaStream_t)stream;
  c->precision = precision;
  c->F.mixed = precision == NUMA_PREC_MIXED;
  c->F.refine_iters = refine;
  c->F.standard = form == NUMA_COLUMN_STANDARD;
  c->scheme = scheme;
  c->imex3d = imex == NUMA_IMEX_3D;
  c->pbno_order = pbno_order;
  c->krylov_max_iters = kmax;
  c->krylov_tol = ktol;
  c->precond = precond;
  c->theta_s = mesh->theta_s > 0 ? mesh->theta_s : 300.0;
  {
    // columns per CTA of the column kernels: 32 (one warp's worth; see stage_threads for the
    // threads per column); NUMA_COL_TILE overrides (a multiple of 32 in [32, 256])
    c->col_tile = 32;
    if (const char* t = std::getenv("NUMA_COL_TILE")) {
      const int v = std::atoi(t);
      if (v >= 32 && v <= 256 && v % 32 == 0) c->col_tile = v;
    }
  }
  c->n_bv = mesh->n_bv;
  double xi[NUMA_MAXNQ], w[NUMA_MAXNQ], D[NUMA_MAXNQ * NUMA_MAXNQ];
  lgl_host(N, xi, w, D);
  set_axis(c->C.x, N, w, D, mesh->Lx / mesh->nex);
  set_axis(c->C.y, N, w, D, mesh->Ly / mesh->ney);
  set_axis(c->C.z, N, w, D, mesh->Lz / mesh->nez);
  build_levels(c, xi, w, D, mesh->Lz / mesh->nez);
  int rc = upload_levels(c);
  const int hb = c->F.standard ? 3 * N + 1 : 2 * N;      // half-bandwidth
  const size_t nu = c->F.standard ? 3 * (size_t)G.M : (size_t)G.M;   // unknowns per column
  c->F.hb = hb;
  const bool mixed = c->F.mixed;                         // FP32 factors
  const bool rhs32 = precision == NUMA_PREC_MIXED || precision == NUMA_PREC_RHS32;  // FP32 RHS
  const size_t fsz = mixed ? sizeof(float) : sizeof(double);
  // 3D-IMEX stores column factors only for the column preconditioner
  const bool need_factors = !c->imex3d || c->precond == NUMA_PRECOND_COLUMN;
  c->factor_bytes = need_factors ? nu * (2 * hb + 1) * G.ncol * fsz : 0;
  c->work_bytes = rhs32 ? (size_t)(2 * 5) * G.nnode * sizeof(double) +
                              (size_t)(6 + 2 * 5) * G.nnode * sizeof(float)
                        : (size_t)(1 + work_states(scheme) * 5) * G.nnode * sizeof(double);
  if (rc == NUMA_OK) {
    bool ok = cudaMalloc(&c->d_work, c->work_bytes) == cudaSuccess &&
              cudaMalloc(&c->d_status, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&c->d_count, sizeof(unsigned long long)) == cudaSuccess;
    if (!need_factors) {
      // 3D-IMEX with the polynomial preconditioner keeps no column factors
    } else if (ok && mixed)
      ok = cudaMalloc(&c->F.L32, (size_t)G.M * hb * fac_cols(G.ncol) * sizeof(float)) == cudaSuccess &&
           cudaMalloc(&c->F.U32, (size_t)G.M * (hb + 1) * fac_cols(G.ncol) * sizeof(float)) == cudaSuccess;
    else if (ok)
      ok = cudaMalloc(&c->F.L, nu * hb * fac_cols(G.ncol) * sizeof(double)) == cudaSuccess &&
           cudaMalloc(&c->F.U, nu * (hb + 1) * fac_cols(G.ncol) * sizeof(double)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      rc = NUMA_ERR_OOM;
    }
  }
  if (rc == NUMA_OK) {
    c->nperm = rhs_perm_size(G);
    std::vector<int> hp((size_t)c->nperm);
    build_rhs_perm(G, hp.data());
    rhs_perm_rows(G, c->perm_row_off, c->perm_row_y);
    if (cudaMalloc(&c->d_perm, hp.size() * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      rc = NUMA_ERR_OOM;
    } else if (cudaMemcpy(c->d_perm, hp.data(), hp.size() * sizeof(int), cudaMemcpyHostToDevice) !=
               cudaSuccess) {
      rc = NUMA_ERR_CUDA;
    }
  }
  if (rc == NUMA_OK) {
    const long long n5 = 5 * G.nnode;
    if (rhs32) {
      c->R1 = c->R2 = nullptr;
      c->Pp = nullptr;
      c->q2 = c->d_work;
      c->q3 = c->q2 + n5;
      c->F32 = (float*)(c->q3 + n5);
      c->R1f = c->F32 + 6 * G.nnode;
      c->R2f = c->R1f + n5;
    } else {
      c->Pp = c->d_work;
      c->R1 = c->Pp + G.nnode;
      c->R2 = c->R1 + n5;
      c->q2 = c->R2 + n5;
      c->q3 = c->q2 + n5;
      if (scheme == NUMA_SCHEME_ARK3) {
        c->R3 = c->q3 + n5;
        c->q4 = c->R3 + n5;
      } else if (scheme >= NUMA_SCHEME_ARK4) {
        const int ns = ark_tab(scheme).s;
        c->Rk[0] = c->R1;
        c->Rk[1] = c->R2;
        c->Qk[1] = c->q2;
        c->Qk[2] = c->q3;
        double* p = c->q3 + n5;
        for (int j = 2; j < ns; ++j, p += n5) c->Rk[j] = p;
        for (int j = 3; j < ns; ++j, p += n5) c->Qk[j] = p;
      }
    }
    if (precision == NUMA_PREC_DF &&
        cudaMalloc(&c->F2, (size_t)6 * G.nnode * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      c->F2 = nullptr;
      rc = NUMA_ERR_OOM;
    }
    if (rc == NUMA_OK && cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess) rc = NUMA_ERR_CUDA;
  }
  if (rc == NUMA_OK && dt > 0) rc = numa_factor_columns(c, dt);
  if (rc == NUMA_OK) rc = (cudaDeviceSynchronize() == cudaSuccess) ? NUMA_OK : NUMA_ERR_CUDA;
  if (rc != NUMA_OK) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return NUMA_OK;
}

void numa_destroy(numa_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
}

int numa_set_stream(numa_ctx* ctx, void* stream) {
  if (!ctx) return NUMA_ERR_ARG;
  ctx->stream = (cudaStream_t)stream;
  return NUMA_OK;
}

int numa_rhs_explicit(numa_ctx* ctx, const double* q, double* rhs) {
  if (!ctx) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_ptr(ctx, q, "q")) || (rc = check_ptr(ctx, rhs, "rhs"))) return rc;
  if (q == rhs) return fail(ctx, NUMA_ERR_ARG, "q and rhs must not overlap");
  RhsEpilogue ep{};
  ep.mode = 0;
  if (ctx->precision == NUMA_PREC_MIXED || ctx->precision == NUMA_PREC_RHS32) {
    long p = prof_begin(ctx, NUMA_K_PRESSURE);
    NUMA_CK(ctx, launch_prep32(q, ctx->F32, ctx->G, ctx->R, ctx->stream));
    prof_end(ctx, p);
    p = prof_begin(ctx, NUMA_K_RHS);
    NUMA_CK(ctx, launch_rhs32d(q, ctx->F32, rhs, ctx->G, ctx->C, ctx->R, ctx->stream));
    prof_end(ctx, p);
    return NUMA_OK;
  }
  return enqueue_rhs(ctx, q, rhs, ep);
}

int numa_factor_columns(numa_ctx* ctx, double dt) {
  if (!ctx) return NUMA_ERR_ARG;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, NUMA_ERR_ARG, "dt must be > 0");
  const double lam = ark_tab(ctx->scheme).at[1][1] * dt;   // the one implicit diagonal
  int rc = upload_stage_tables(ctx, lam);
  if (rc) return rc;
  ctx->dt = dt;
  ctx->lam = lam;
  if (ctx->imex3d) {
    if (ctx->precond == NUMA_PRECOND_COLUMN)
      NUMA_CK(ctx, launch_factor(ctx->G, ctx->R, lam, ctx->F, ctx->d_status, ctx->stream));
    ctx->factored = true;            // the stage tables; the preconditioner needs lam
    if ((rc = numa_imex3d_setup(ctx))) {
      ctx->factored = false;
      return rc;
    }
    return NUMA_OK;
  }
  long p = prof_begin(ctx, NUMA_K_FACTOR);
  NUMA_CK(ctx, launch_factor(ctx->G, ctx->R, lam, ctx->F, ctx->d_status, ctx->stream));
  prof_end(ctx, p);
  ctx->factored = true;
  return NUMA_OK;
}

int numa_solve_columns(numa_ctx* ctx, const double* b, double* x) {
  if (!ctx) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_ptr(ctx, b, "b")) || (rc = check_ptr(ctx, x, "x"))) return rc;
  if (!ctx->factored) return fail(ctx, NUMA_ERR_NOT_FACTORED, "numa_factor_columns not called");
  if (ctx->F.standard || ctx->imex3d)
    return fail(ctx, NUMA_ERR_ARG, "the stand-alone column solve needs a 1D-IMEX Schur-form context");
  long p = prof_begin(ctx, NUMA_K_SOLVE);
  NUMA_CK(ctx, launch_solve(b, x, ctx->G, ctx->F, ctx->R, ctx->T, ctx->col_tile, ctx->stream,
                            ctx->d_status));
  prof_end(ctx, p);
  return NUMA_OK;
}

int numa_imex_stage(numa_ctx* ctx, int stage, const double* qn, const double* R1,
                    const double* R2, const double* q2, double* q_out) {
  if (!ctx) return NUMA_ERR_ARG;
  if (stage != 2 && stage != 3) return fail(ctx, NUMA_ERR_ARG, "stage must be 2 or 3");
  int rc;
  if ((rc = check_ptr(ctx, qn, "qn")) || (rc = check_ptr(ctx, R1, "R1")) ||
      (rc = check_ptr(ctx, q_out, "q_out")))
    return rc;
  if (stage == 3 && ((rc = check_ptr(ctx, R2, "R2")) || (rc = check_ptr(ctx, q2, "q2")))) return rc;
  if (states_overlap(ctx, q_out, qn) || states_overlap(ctx, q_out, R1) ||
      (stage == 3 && (states_overlap(ctx, q_out, R2) || states_overlap(ctx, q_out, q2))))
    return fail(ctx, NUMA_ERR_ARG, "q_out overlaps an input");
  if (!ctx->factored) return fail(ctx, NUMA_ERR_NOT_FACTORED, "numa_factor_columns not called");
  if (ctx->imex3d) return fail(ctx, NUMA_ERR_ARG, "3D-IMEX context: use numa_imex3d_stage");
  return enqueue_stage(ctx, stage, qn, R1, R2, q2, q_out, numa_stage_coef(ctx, stage));
}

int numa_imex_stage_s(numa_ctx* ctx, int stage, const double* qn, const double* const* R,
                      const double* const* Q, double* q_out) {
  if (!ctx) return NUMA_ERR_ARG;
  const ArkTab t = ark_tab(ctx->scheme);
  if (stage < 2 || stage > t.s) return fail(ctx, NUMA_ERR_ARG, "stage outside 2..s");
  if (!R || (stage > 2 && !Q)) return fail(ctx, NUMA_ERR_ARG, "R or Q missing");
  if (ctx->precision != NUMA_PREC_FP64 || ctx->F.standard || ctx->imex3d)
    return fail(ctx, NUMA_ERR_ARG, "the general stage needs an FP64 Schur-form 1D-IMEX context");
  int rc;
  if ((rc = check_ptr(ctx, qn, "qn")) || (rc = check_ptr(ctx, q_out, "q_out"))) return rc;
  const double* Rv[NUMA_MAX_STAGES] = {};
  const double* Qv[NUMA_MAX_STAGES] = {};
  for (int j = 0; j < stage - 1; ++j) {
    if ((rc = check_ptr(ctx, R[j], "R[j]"))) return rc;
    Rv[j] = R[j];
    if (j >= 1) {
      if ((rc = check_ptr(ctx, Q[j - 1], "Q[j]"))) return rc;
      Qv[j] = Q[j - 1];
    }
  }
  bool ov = states_overlap(ctx, q_out, qn);
  for (int j = 0; j < stage - 1; ++j) ov = ov || states_overlap(ctx, q_out, Rv[j]) || states_overlap(ctx, q_out, Qv[j]);
  if (ov) return fail(ctx, NUMA_ERR_ARG, "q_out overlaps an input");
  if (!ctx->factored) return fail(ctx, NUMA_ERR_NOT_FACTORED, "numa_factor_columns not called");
  const StagePrev P = stage_prev(t, stage - 1, ctx->dt, qn, Rv, Qv);
  long p = prof_begin(ctx, NUMA_K_STAGE);
  NUMA_CK(ctx, launch_stage_general(P, q_out, ctx->G, ctx->R, ctx->F, ctx->T, ctx->col_tile,
                                    ctx->stream, nullptr));
  prof_end(ctx, p);
  return NUMA_OK;
}

int numa_step_imex1d(numa_ctx* ctx, const double* q_in, double* q_out, int nsteps) {
  if (!ctx) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_ptr(ctx, q_in, "q_in")) || (rc = check_ptr(ctx, q_out, "q_out"))) return rc;
  if (nsteps < 0) return fail(ctx, NUMA_ERR_ARG, "nsteps < 0");
  if (!ctx->factored) return fail(ctx, NUMA_ERR_NOT_FACTORED, "numa_factor_columns not called");
  if (ctx->imex3d) return fail(ctx, NUMA_ERR_ARG, "3D-IMEX context: use numa_step_imex3d");
  const long long n5 = 5 * ctx->G.nnode;
  if (nsteps == 0) {
    if (q_in != q_out)
      NUMA_CK(ctx, cudaMemcpyAsync(q_out, q_in, n5 * sizeof(double), cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    return NUMA_OK;
  }
  const ArkTab t = ark_tab(ctx->scheme);
  const StageCoef s2 = numa_stage_coef(ctx, 2), s3 = numa_stage_coef(ctx, 3);
  const bool mixed = ctx->precision == NUMA_PREC_MIXED || ctx->precision == NUMA_PREC_RHS32;  // FP32 tendencies
  if (t.s > 4) {        // ARK4, ARK5: FP64 Schur form, general fused stage
    const double* cur = q_in;
    for (int s = 0; s < nsteps; ++s) {
      RhsEpilogue e0{};
      if ((rc = enqueue_rhs(ctx, cur, ctx->Rk[0], e0))) return rc;
      for (int i = 1; i < t.s; ++i) {        // stage i + 1
        const StagePrev P = stage_prev(t, i, ctx->dt, cur, ctx->Rk, ctx->Qk);
        long p = prof_begin(ctx, NUMA_K_STAGE);
        NUMA_CK(ctx, launch_stage_general(P, ctx->Qk[i], ctx->G, ctx->R, ctx->F, ctx->T,
                                          ctx->col_tile, ctx->stream, ctx->Pp));
        prof_end(ctx, p);
        if ((rc = enqueue_rhs(ctx, ctx->Qk[i], ctx->Rk[i], e0, nullptr, true))) return rc;
      }
      // q^{n+1} = q^n + dt sum_j b_j R(q(j))
      StageSum S{};
      for (int j = 0; j < t.s; ++j)
        if (t.b[j] != 0.0) {
          S.R[S.n] = ctx->Rk[j];
          S.bdt[S.n++] = t.b[j] * ctx->dt;
        }
      NUMA_CK(ctx, launch_ark_combine(cur, S, q_out, n5, ctx->d_status, ctx->stream));
      cur = q_out;
    }
    return NUMA_OK;
  }
  if (t.s == 4) {       // ARK3: four stages, FP64 Schur form
    const StageCoef s4 = numa_stage_coef(ctx, 4);
    const double* cur = q_in;
    for (int s = 0; s < nsteps; ++s) {
      RhsEpilogue e0{};
      if ((rc = enqueue_rhs(ctx, cur, ctx->R1, e0))) return rc;
      if ((rc = enqueue_stage(ctx, 2, cur, ctx->R1, nullptr, nullptr, ctx->q2, s2, false, ctx->Pp))) return rc;
      if ((rc = enqueue_rhs(ctx, ctx->q2, ctx->R2, e0, nullptr, true))) return rc;
      if ((rc = enqueue_stage(ctx, 3, cur, ctx->R1, ctx->R2, ctx->q2, ctx->q3, s3, false, ctx->Pp))) return rc;
      if ((rc = enqueue_rhs(ctx, ctx->q3, ctx->R3, e0, nullptr, true))) return rc;
      long p = prof_begin(ctx, NUMA_K_STAGE);
      NUMA_CK(ctx, launch_stage(4, cur, ctx->R1, ctx->R2, ctx->q2, ctx->q4, ctx->G, ctx->R, ctx->F,
                                s4, ctx->T, ctx->col_tile, false, ctx->stream, ctx->R3, ctx->q3,
                                ctx->Pp));
      prof_end(ctx, p);
      RhsEpilogue ef{};
      ef.mode = 3;
      ef.b1dt = t.b[0] * ctx->dt;
      ef.b2dt = t.b[1] * ctx->dt;
      ef.b3dt = t.b[2] * ctx->dt;
      ef.b4dt = t.b[3] * ctx->dt;
      ef.u0 = cur;
      ef.R1 = ctx->R1;
      ef.R2 = ctx->R2;
      ef.R3 = ctx->R3;
      if ((rc = enqueue_rhs(ctx, ctx->q4, q_out, ef, nullptr, true))) return rc;
      cur = q_out;
    }
    return NUMA_OK;
  }
  void* R1 = mixed ? (void*)ctx->R1f : (void*)ctx->R1;
  void* R2 = mixed ? (void*)ctx->R2f : (void*)ctx->R2;
  const double* cur = q_in;
  const bool fuse = fuse_pressure(ctx);
  double* Pp_next = fuse ? ctx->Pp : nullptr;
  for (int s = 0; s < nsteps; ++s) {
    RhsEpilogue e0{};
    if ((rc = enqueue_rhs(ctx, cur, ctx->R1, e0, ctx->R1f))) return rc;
    if ((rc = enqueue_stage(ctx, 2, cur, R1, nullptr, nullptr, ctx->q2, s2, mixed, Pp_next))) return rc;
    if ((rc = enqueue_rhs(ctx, ctx->q2, ctx->R2, e0, ctx->R2f, fuse))) return rc;
    if ((rc = enqueue_stage(ctx, 3, cur, R1, R2, ctx->q2, ctx->q3, s3, mixed, Pp_next))) return rc;
    RhsEpilogue ef{};
    ef.mode = 2;
    ef.b1dt = t.b[0] * ctx->dt;
    ef.b2dt = t.b[1] * ctx->dt;
    ef.b3dt = t.b[2] * ctx->dt;
    ef.u0 = cur;
    ef.R1 = R1;
    ef.R2 = R2;
    if ((rc = enqueue_rhs(ctx, ctx->q3, q_out, ef, nullptr, fuse))) return rc;
    cur = q_out;
  }
  return NUMA_OK;
}

int numa_step_phase(numa_ctx* ctx, int phase, const double* q_n, double* q_out) {
  if (!ctx) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_ptr(ctx, q_n, "q_n"))) return rc;
  if (phase == 2 && (rc = check_ptr(ctx, q_out, "q_out"))) return rc;
  if (phase < 0 || phase > 2) return fail(ctx, NUMA_ERR_ARG, "phase must be 0, 1 or 2");
  if (!ctx->factored) return fail(ctx, NUMA_ERR_NOT_FACTORED, "numa_factor_columns not called");
  if (ctx->imex3d || ctx->scheme != NUMA_SCHEME_ARK2)
    return fail(ctx, NUMA_ERR_ARG, "the phased step needs an ARK2 1D-IMEX context");
  if (states_overlap(ctx, q_n, ctx->q2) || states_overlap(ctx, q_n, ctx->q3) ||
      (phase == 2 && (states_overlap(ctx, q_out, ctx->q2) || states_overlap(ctx, q_out, ctx->q3))))
    return fail(ctx, NUMA_ERR_ARG, "q_n or q_out overlaps the context's stage values");
  // the phases of the ARK2 branch of numa_step_imex1d, in its order
  const ArkTab t = ark_tab(ctx->scheme);
  const bool mixed = ctx->precision == NUMA_PREC_MIXED || ctx->precision == NUMA_PREC_RHS32;
  void* R1 = mixed ? (void*)ctx->R1f : (void*)ctx->R1;
  void* R2 = mixed ? (void*)ctx->R2f : (void*)ctx->R2;
  const bool fuse = fuse_pressure(ctx);
  double* Pp_next = fuse ? ctx->Pp : nullptr;
  RhsEpilogue e0{};
  if (phase == 0) {
    if ((rc = enqueue_rhs(ctx, q_n, ctx->R1, e0, ctx->R1f))) return rc;
    return enqueue_stage(ctx, 2, q_n, R1, nullptr, nullptr, ctx->q2, numa_stage_coef(ctx, 2), mixed,
                         Pp_next);
  }
  if (phase == 1) {
    if ((rc = enqueue_rhs(ctx, ctx->q2, ctx->R2, e0, ctx->R2f, fuse))) return rc;
    return enqueue_stage(ctx, 3, q_n, R1, R2, ctx->q2, ctx->q3, numa_stage_coef(ctx, 3), mixed,
                         Pp_next);
  }
  RhsEpilogue ef{};
  ef.mode = 2;
  ef.b1dt = t.b[0] * ctx->dt;
  ef.b2dt = t.b[1] * ctx->dt;
  ef.b3dt = t.b[2] * ctx->dt;
  ef.u0 = q_n;
  ef.R1 = R1;
  ef.R2 = R2;
  return enqueue_rhs(ctx, ctx->q3, q_out, ef, nullptr, fuse);
}

int numa_step_buffers(numa_ctx* ctx, double** q2, double** q3, double** pp, int* pp_fused) {
  if (!ctx) return NUMA_ERR_ARG;
  if (ctx->imex3d || ctx->scheme != NUMA_SCHEME_ARK2)
    return fail(ctx, NUMA_ERR_ARG, "the phased step needs an ARK2 1D-IMEX context");
  if (q2) *q2 = ctx->q2;
  if (q3) *q3 = ctx->q3;
  if (pp) *pp = ctx->Pp;
  if (pp_fused) *pp_fused = fuse_pressure(ctx) ? 1 : 0;
  return NUMA_OK;
}

int numa_step_explicit_rk(numa_ctx* ctx, const double* q_in, double* q_out, double dt,
                          int nsteps) {
  if (!ctx) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_ptr(ctx, q_in, "q_in")) || (rc = check_ptr(ctx, q_out, "q_out"))) return rc;
  if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt))
    return fail(ctx, NUMA_ERR_ARG, "need nsteps >= 0 and dt > 0");
  const long long n5 = 5 * ctx->G.nnode;
  if (nsteps == 0) {
    if (q_in != q_out)
      NUMA_CK(ctx, cudaMemcpyAsync(q_out, q_in, n5 * sizeof(double), cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    return NUMA_OK;
  }
  // ping-pong between two workspace states; the last stage (alpha_5 = 0) writes q_out, so
  // q_in may equal q_out.
  double* buf[2] = {ctx->q2, ctx->q3};
  const double* u0 = q_in;
  for (int s = 0; s < nsteps; ++s) {
    const double* prev = u0;
    for (int i = 0; i < 5; ++i) {
      double* dst = (i == 4) ? q_out : buf[i & 1];
      RhsEpilogue ep{};
      ep.mode = 1;
      ep.alpha = kRkAlpha[i];
      ep.one_minus_alpha = 1.0 - kRkAlpha[i];
      ep.use_u0 = kRkAlpha[i] != 0.0;
      ep.beta_dt = kRkBeta[i] * dt;
      ep.u0 = u0;
      if ((rc = enqueue_rhs(ctx, prev, dst, ep))) return rc;
      prev = dst;
    }
    u0 = q_out;
  }
  return NUMA_OK;
}

namespace {

// Slabs of the pipelined host run: runs of whole tile rows of the RHS thread order.  At
// most kHostSlabs; NUMA_HOST_SLABS (1..kHostSlabs) overrides, for tuning.
const int kHostSlabs = 16;

int host_slabs() {
  static int n = -1;
  if (n < 0) {
    n = 8;
    if (const char* t = std::getenv("NUMA_HOST_SLABS")) {
      const int v = std::atoi(t);
      if (v >= 1 && v <= kHostSlabs) n = v;
    }
  }
  return n;
}

// Slab boundaries in tile rows: K slabs over `rows` tile rows.
// * Upload (taper_end = false): the first slab is one tile row, the others as even as
//   possible.
// * Download (taper_end = true): slabs of relative sizes 1, ..., 1, 1/2, 1/4, so that
//   little download is left after the last kernel.
// With fewer than K + 2 tile rows, or K < 3, the slabs are plain even splits.
std::vector<int> slab_bounds(int rows, int K, bool taper_end) {
  std::vector<int> b(K + 1);
  if (K < 3 || rows < K + 2) {
    for (int k = 0; k <= K; ++k) b[k] = (int)((long long)k * rows / K);
    return b;
  }
  b[0] = 0;
  b[K] = rows;
  if (!taper_end) {
    for (int k = 0; k < K; ++k) b[k + 1] = 1 + (int)((long long)k * (rows - 1) / (K - 1));
    return b;
  }
  const double total = (K - 2) + 0.75;
  double cum = 0.0;
  for (int k = 1; k < K; ++k) {
    cum += (k <= K - 2) ? 1.0 : 0.5;
    const int v = (int)std::lround(cum / total * rows);
    b[k] = std::min(std::max(v, b[k - 1] + 1), rows - (K - k));   // strictly increasing
  }
  return b;
}

// FP64 ARK2 1D-IMEX steps from host memory to host memory with the copies overlapped.
// * Upload: slab by slab on cs_in, the first slab one tile row.  Each slab goes up in two
//   pieces, its first N node rows (one element: all that the stencil of the slab before it
//   reaches) and the rest, with an event after each.
// * The first right-hand side of the first step follows the pieces: P' of each piece on
//   cs_p once it is on the device (overlapping the right-hand sides of earlier slabs), and
//   R of slab k once P' of slab k and of slab k + 1's first piece are done.
// * The final update of the last step is issued slab by slab, the slabs shrinking to a
//   quarter at the end; each slab goes back to the host on cs_out as soon as it is final.
// * Steps in between run unchanged, and every node's arithmetic is the device run's.
int run_host_pipelined(numa_ctx* ctx, const double* hin, double* hout, int nsteps) {
  const Geom& G = ctx->G;
  const long long nn = G.nnode;
  const long long plane = (long long)G.nxg * G.M;        // nodes per node row
  const int rows = (int)ctx->perm_row_y.size() - 1;
  const int K = std::min(host_slabs(), rows);
  if (!ctx->cs_in) {
    if (cudaStreamCreateWithFlags(&ctx->cs_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->cs_out, cudaStreamNonBlocking) != cudaSuccess)
      return fail(ctx, NUMA_ERR_CUDA, "copy streams");
  }
  if (!ctx->cs_p &&
      cudaStreamCreateWithFlags(&ctx->cs_p, cudaStreamNonBlocking) != cudaSuccess)
    return fail(ctx, NUMA_ERR_CUDA, "pre-pass stream");
  while ((int)ctx->host_ev.size() < 5 * kHostSlabs + 2) {
    cudaEvent_t e;
    NUMA_CK(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->host_ev.push_back(e);
  }
  cudaEvent_t* ev_head = ctx->host_ev.data();           // first piece of slab k uploaded
  cudaEvent_t* ev_in = ev_head + kHostSlabs;            // whole slab k uploaded
  cudaEvent_t* ev_out = ev_in + kHostSlabs;             // slab k final
  cudaEvent_t* ev_ph = ev_out + kHostSlabs;             // P' of slab k's first piece done
  cudaEvent_t* ev_pr = ev_ph + kHostSlabs;              // P' of all of slab k done
  cudaEvent_t ev_start = ev_head[5 * kHostSlabs], ev_done = ev_head[5 * kHostSlabs + 1];
  const std::vector<int> bu = slab_bounds(rows, K, false), bd = slab_bounds(rows, K, true);
  auto y0 = [&](const std::vector<int>& bnd, int k) { return (long long)ctx->perm_row_y[bnd[k]]; };
  auto n0 = [&](const std::vector<int>& bnd, int k) { return y0(bnd, k) * plane; };   // first node
  auto p0 = [&](const std::vector<int>& bnd, int k) { return ctx->perm_row_off[bnd[k]]; };  // first thread
  // end of slab k's first piece (node index)
  auto nh = [&](int k) { return std::min(y0(bu, k) + G.N, y0(bu, k + 1)) * plane; };
  double* q = ctx->d_hoststate;
  const size_t pitch = nn * sizeof(double);
  // the upload starts after everything already in the context's stream
  NUMA_CK(ctx, cudaEventRecord(ev_start, ctx->stream));
  NUMA_CK(ctx, cudaStreamWaitEvent(ctx->cs_in, ev_start, 0));
  for (int k = 0; k < K; ++k) {
    const long long a = n0(bu, k), h = nh(k), b = n0(bu, k + 1);
    NUMA_CK(ctx, cudaMemcpy2DAsync(q + a, pitch, hin + a, pitch, (h - a) * sizeof(double), 5,
                                   cudaMemcpyHostToDevice, ctx->cs_in));
    NUMA_CK(ctx, cudaEventRecord(ev_head[k], ctx->cs_in));
    if (b > h)
      NUMA_CK(ctx, cudaMemcpy2DAsync(q + h, pitch, hin + h, pitch, (b - h) * sizeof(double), 5,
                                     cudaMemcpyHostToDevice, ctx->cs_in));
    NUMA_CK(ctx, cudaEventRecord(ev_in[k], ctx->cs_in));
  }
  const ArkTab t = ark_tab(ctx->scheme);
  const StageCoef s2 = numa_stage_coef(ctx, 2), s3 = numa_stage_coef(ctx, 3);
  int rc;
  for (int s = 0; s < nsteps; ++s) {
    RhsEpilogue e0{};
    if (s == 0) {
      long p = prof_begin(ctx, NUMA_K_RHS);
      // P' piece by piece on cs_p as the pieces arrive; R of slab k on the context's stream
      // once P' of slab k and of slab k + 1's first piece are done
      NUMA_CK(ctx, cudaStreamWaitEvent(ctx->cs_p, ev_start, 0));
      for (int k = 0; k < K; ++k) {
        NUMA_CK(ctx, cudaStreamWaitEvent(ctx->cs_p, ev_head[k], 0));
        NUMA_CK(ctx, launch_pressure_range(q, ctx->Pp, G, ctx->R, n0(bu, k), nh(k), ctx->cs_p,
                                           ctx->d_status));
        NUMA_CK(ctx, cudaEventRecord(ev_ph[k], ctx->cs_p));
        if (n0(bu, k + 1) > nh(k)) {
          NUMA_CK(ctx, cudaStreamWaitEvent(ctx->cs_p, ev_in[k], 0));
          NUMA_CK(ctx, launch_pressure_range(q, ctx->Pp, G, ctx->R, nh(k), n0(bu, k + 1), ctx->cs_p,
                                             ctx->d_status));
        }
        NUMA_CK(ctx, cudaEventRecord(ev_pr[k], ctx->cs_p));
      }
      for (int k = 0; k < K; ++k) {
        NUMA_CK(ctx, cudaStreamWaitEvent(ctx->stream, ev_pr[k], 0));
        if (k + 1 < K) NUMA_CK(ctx, cudaStreamWaitEvent(ctx->stream, ev_ph[k + 1], 0));
        NUMA_CK(ctx, launch_rhs(q, ctx->Pp, ctx->R1, ctx->d_perm + p0(bu, k),
                                p0(bu, k + 1) - p0(bu, k), G, ctx->C, ctx->R, e0, ctx->stream));
      }
      prof_end(ctx, p);
    } else if ((rc = enqueue_rhs(ctx, q, ctx->R1, e0))) {
      return rc;
    }
    if ((rc = enqueue_stage(ctx, 2, q, ctx->R1, nullptr, nullptr, ctx->q2, s2, false, ctx->Pp))) return rc;
    if ((rc = enqueue_rhs(ctx, ctx->q2, ctx->R2, e0, nullptr, true))) return rc;
    if ((rc = enqueue_stage(ctx, 3, q, ctx->R1, ctx->R2, ctx->q2, ctx->q3, s3, false, ctx->Pp))) return rc;
    RhsEpilogue ef{};
    ef.mode = 2;
    ef.b1dt = t.b[0] * ctx->dt;
    ef.b2dt = t.b[1] * ctx->dt;
    ef.b3dt = t.b[2] * ctx->dt;
    ef.u0 = q;
    ef.R1 = ctx->R1;
    ef.R2 = ctx->R2;
    if (s + 1 < nsteps) {
      if ((rc = enqueue_rhs(ctx, ctx->q3, q, ef, nullptr, true))) return rc;
      continue;
    }
    // last step: final update (in place, node by node) and download, slab by slab
    long p = prof_begin(ctx, NUMA_K_RHS);
    for (int k = 0; k < K; ++k) {
      NUMA_CK(ctx, launch_rhs(ctx->q3, ctx->Pp, q, ctx->d_perm + p0(bd, k), p0(bd, k + 1) - p0(bd, k),
                              G, ctx->C, ctx->R, ef, ctx->stream));
      NUMA_CK(ctx, cudaEventRecord(ev_out[k], ctx->stream));
      NUMA_CK(ctx, cudaStreamWaitEvent(ctx->cs_out, ev_out[k], 0));
      const long long a = n0(bd, k), b = n0(bd, k + 1);
      NUMA_CK(ctx, cudaMemcpy2DAsync(hout + a, pitch, q + a, pitch, (b - a) * sizeof(double), 5,
                                     cudaMemcpyDeviceToHost, ctx->cs_out));
    }
    prof_end(ctx, p);
  }
  NUMA_CK(ctx, cudaEventRecord(ev_done, ctx->cs_out));
  NUMA_CK(ctx, cudaStreamWaitEvent(ctx->stream, ev_done, 0));
  NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
  return NUMA_OK;
}

}  // namespace

int numa_run_host(numa_ctx* ctx, int method, const double* q_in_host, double* q_out_host,
                  int nsteps, double dt) {
  if (!ctx) return NUMA_ERR_ARG;
  if (!q_in_host || !q_out_host || (method != 0 && method != 1))
    return fail(ctx, NUMA_ERR_ARG, "bad method or host buffer");
  const size_t bytes = 5 * (size_t)ctx->G.nnode * sizeof(double);
  if (!ctx->d_hoststate) {
    if (cudaMalloc(&ctx->d_hoststate, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, NUMA_ERR_OOM, "host-run state buffer");
    }
  }
  if (method == 0 && nsteps >= 1 && ctx->factored && !ctx->imex3d && fuse_pressure(ctx) &&
      ctx->scheme == NUMA_SCHEME_ARK2)
    return run_host_pipelined(ctx, q_in_host, q_out_host, nsteps);
  NUMA_CK(ctx, cudaMemcpyAsync(ctx->d_hoststate, q_in_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  int rc = (method == 0) ? numa_step_imex1d(ctx, ctx->d_hoststate, ctx->d_hoststate, nsteps)
                         : numa_step_explicit_rk(ctx, ctx->d_hoststate, ctx->d_hoststate, dt, nsteps);
  if (rc) return rc;
  NUMA_CK(ctx, cudaMemcpyAsync(q_out_host, ctx->d_hoststate, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
  return NUMA_OK;
}

int numa_profile(numa_ctx* ctx, int enable) {
  if (!ctx) return NUMA_ERR_ARG;
  NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (enable) ctx->prof_n = 0;
  ctx->prof_on = enable != 0;
  return NUMA_OK;
}

int numa_profile_read(numa_ctx* ctx, int kind, double* total_ms, long long* launches) {
  if (!ctx || !total_ms || !launches || kind < 0 || kind >= NUMA_K_NKINDS) return NUMA_ERR_ARG;
  NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
  double t = 0.0;
  long long n = 0;
  for (size_t i = 0; i < ctx->prof_n; ++i) {
    if (ctx->prof[i].kind != kind) continue;
    float ms = 0.0f;
    NUMA_CK(ctx, cudaEventElapsedTime(&ms, ctx->prof[i].a, ctx->prof[i].b));
    t += ms;
    ++n;
  }
  *total_ms = t;
  *launches = n;
  return NUMA_OK;
}

int numa_connectivity(numa_ctx* ctx, int32_t* l2g, int32_t* g2l) {
  if (!ctx) return NUMA_ERR_ARG;
  NUMA_CK(ctx, launch_connectivity(ctx->G, l2g, g2l, ctx->stream));
  return NUMA_OK;
}

int numa_column_factors(numa_ctx* ctx, long long col, double* host_out) {
  if (!ctx) return NUMA_ERR_ARG;
  if (!host_out || col < 0 || col >= ctx->G.ncol) return fail(ctx, NUMA_ERR_ARG, "bad column");
  if (!ctx->factored) return fail(ctx, NUMA_ERR_NOT_FACTORED, "numa_factor_columns not called");
  if (ctx->imex3d) return fail(ctx, NUMA_ERR_ARG, "a 3D-IMEX context stores no column factors");
  const int M = ctx->F.standard ? 3 * ctx->G.M : ctx->G.M;   // unknowns per column
  const int hb = ctx->F.hb, W = 2 * hb + 1;
  std::vector<double> L((size_t)M * hb), U((size_t)M * (hb + 1));
  // in the stored layout one column's entries are kFacBlk elements apart
  const long long lb = fac_col_base(col, M, hb), ub = fac_col_base(col, M, hb + 1);
  if (ctx->F.mixed) {
    const size_t pitch = (size_t)kFacBlk * sizeof(float);
    std::vector<float> Lf(L.size()), Uf(U.size());
    NUMA_CK(ctx, cudaMemcpy2DAsync(Lf.data(), sizeof(float), ctx->F.L32 + lb, pitch, sizeof(float),
                                   (size_t)M * hb, cudaMemcpyDeviceToHost, ctx->stream));
    NUMA_CK(ctx, cudaMemcpy2DAsync(Uf.data(), sizeof(float), ctx->F.U32 + ub, pitch, sizeof(float),
                                   (size_t)M * (hb + 1), cudaMemcpyDeviceToHost, ctx->stream));
    NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t t = 0; t < L.size(); ++t) L[t] = Lf[t];
    for (size_t t = 0; t < U.size(); ++t) U[t] = Uf[t];
  } else {
    const size_t pitch = (size_t)kFacBlk * sizeof(double);
    NUMA_CK(ctx, cudaMemcpy2DAsync(L.data(), sizeof(double), ctx->F.L + lb, pitch, sizeof(double),
                                   (size_t)M * hb, cudaMemcpyDeviceToHost, ctx->stream));
    NUMA_CK(ctx, cudaMemcpy2DAsync(U.data(), sizeof(double), ctx->F.U + ub, pitch, sizeof(double),
                                   (size_t)M * (hb + 1), cudaMemcpyDeviceToHost, ctx->stream));
    NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
  }
  // L[(j*hb + k-1)] = L(j+k, j); U[(j*(hb+1) + k)] = U(j-k, j), slot 0 = 1/U(j,j)
  for (size_t t = 0; t < (size_t)M * W; ++t) host_out[t] = 0.0;
  for (int j = 0; j < M; ++j) {
    for (int k = 1; k <= hb; ++k)
      if (j + k < M) host_out[(size_t)(j + k) * W + (hb - k)] = L[(size_t)j * hb + k - 1];
    host_out[(size_t)j * W + hb] = 1.0 / U[(size_t)j * (hb + 1)];
    for (int k = 1; k <= hb; ++k)
      if (j - k >= 0) host_out[(size_t)(j - k) * W + (hb + k)] = U[(size_t)j * (hb + 1) + k];
  }
  return NUMA_OK;
}

int numa_reference_levels(const numa_ctx* ctx, double* host_out) {
  if (!ctx || !host_out) return NUMA_ERR_ARG;
  const int M = ctx->G.M;
  const std::vector<double>* v[8] = {&ctx->z, &ctx->rho0, &ctx->theta0, &ctx->P0,
                                     &ctx->G0, &ctx->H0, &ctx->drho0, &ctx->dtheta0};
  for (int k = 0; k < 8; ++k) std::memcpy(host_out + (size_t)k * M, v[k]->data(), M * sizeof(double));
  return NUMA_OK;
}

int numa_count_nonfinite(numa_ctx* ctx, const double* x, long long n, long long* count) {
  if (!ctx) return NUMA_ERR_ARG;
  int rc;
  if ((rc = check_ptr(ctx, x, "x"))) return rc;
  if (!count || n < 0) return fail(ctx, NUMA_ERR_ARG, "bad count or n");
  NUMA_CK(ctx, cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned long long), ctx->stream));
  NUMA_CK(ctx, launch_count_nonfinite(x, n, ctx->d_count, ctx->stream));
  unsigned long long h = 0;
  NUMA_CK(ctx, cudaMemcpyAsync(&h, ctx->d_count, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
  *count = (long long)h;
  return NUMA_OK;
}

int numa_status(numa_ctx* ctx, int* status) {
  if (!ctx || !status) return NUMA_ERR_ARG;
  unsigned h = 0;
  NUMA_CK(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  NUMA_CK(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
  NUMA_CK(ctx, cudaStreamSynchronize(ctx->stream));
  *status = (h & NUMA_ST_PIVOT)       ? NUMA_ERR_PIVOT
            : (h & NUMA_ST_NONFINITE) ? NUMA_ERR_NONFINITE
            : (h & NUMA_ST_TIMEOUT)   ? NUMA_ERR_TIMEOUT
            : (h & NUMA_ST_RANGE)     ? NUMA_ERR_ARG
                                      : NUMA_OK;
  return NUMA_OK;
}

int numa_query(const numa_ctx* ctx, int what, long long* out) {
  if (!ctx || !out) return NUMA_ERR_ARG;
  const Geom& G = ctx->G;
  switch (what) {
    case NUMA_Q_NCOL: *out = G.ncol; break;
    case NUMA_Q_M: *out = G.M; break;
    case NUMA_Q_NNODE: *out = G.nnode; break;
    case NUMA_Q_NELEM: *out = (long long)G.nex * G.ney * G.nez; break;
    case NUMA_Q_HALF_BAND: *out = ctx->F.hb; break;
    case NUMA_Q_FACTOR_BYTES: *out = (long long)ctx->factor_bytes; break;
    case NUMA_Q_WORKSPACE_BYTES: *out = (long long)ctx->work_bytes; break;
    case NUMA_Q_FACTORED: *out = ctx->factored ? 1 : 0; break;
    case NUMA_Q_N: *out = G.N; break;
    case NUMA_Q_PRECISION: *out = ctx->precision; break;
    case NUMA_Q_COLUMN_FORM: *out = ctx->F.standard ? NUMA_COLUMN_STANDARD : NUMA_COLUMN_SCHUR; break;
    case NUMA_Q_SCHEME: *out = ctx->scheme; break;
    case NUMA_Q_IMEX: *out = ctx->imex3d ? NUMA_IMEX_3D : NUMA_IMEX_1D; break;
    default: return NUMA_ERR_ARG;
  }
  return NUMA_OK;
}

const char* numa_last_error(const numa_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

void numa_rk35_coefficients(double* alpha, double* beta) {
  for (int i = 0; i < 5; ++i) {
    if (alpha) alpha[i] = kRkAlpha[i];
    if (beta) beta[i] = kRkBeta[i];
  }
}

void numa_ark3_tableau(double* a, double* at, double* b) {
  static const Ark3 t;
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) {
      if (a) a[i * 4 + j] = t.a[i][j];
      if (at) at[i * 4 + j] = t.at[i][j];
    }
    if (b) b[i] = t.b[i];
  }
}

int numa_ark_tableau(int scheme, double* a, double* at, double* b, int* s) {
  if (scheme < NUMA_SCHEME_ARK2 || scheme > NUMA_SCHEME_ARK5) return NUMA_ERR_ARG;
  const ArkTab t = ark_tab(scheme);
  if (s) *s = t.s;
  for (int i = 0; i < t.s; ++i) {
    for (int j = 0; j < t.s; ++j) {
      if (a) a[i * t.s + j] = t.a[i][j];
      if (at) at[i * t.s + j] = t.at[i][j];
    }
    if (b) b[i] = t.b[i];
  }
  return NUMA_OK;
}

void numa_ark2_tableau(double* a, double* at, double* b) {
  static const Ark2 t;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      if (a) a[i * 3 + j] = t.a[i][j];
      if (at) at[i * 3 + j] = t.at[i][j];
    }
    if (b) b[i] = t.b[i];
  }
}

}  // extern "C"

// ---- no-allocation variant of the explicit right-hand side ------------------------------
// Callers that must not allocate device memory at the point of the call (a latency-bound
// loop where cudaMalloc/cudaFree would synchronise the device, or a process whose device
// memory is already reserved by another allocator, such as a caching allocator holding
// most of the GPU) use numa_rhs_explicit_static.  It needs no context: the host builds the
// LGL and reference tables with the contexts' own builders (lgl_host, ref_tables_host)
// into a static host buffer, and the device side uses one file-scope scratch array for
// the equation-of-state pre-pass and the per-level tables.  The tables reach the scratch
// as kernel parameters (k_static_tables), so no host buffer is read once the call returns.
#include <mutex>

namespace {

constexpr size_t kStaticScratchDoubles = NUMA_STATIC_SCRATCH_BYTES / sizeof(double);
constexpr int kStaticMaxLevels = 1024;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_static_mutex;
double* g_static_addr[256] = {nullptr};            // device address per device ordinal
double g_static_host[kStaticMaxLevels * (16 + 2 * NUMA_MAXN + 1)];

// One piece of the per-level tables, carried by value in the launch parameters (16 KB, within
// the 32 KB parameter space of sm_70 and later).
constexpr int kTabChunk = 2000;
struct TabChunk {
  double* dst;
  int n;
  double v[kTabChunk];
};

__global__ void k_static_tables(const __grid_constant__ TabChunk c) {
  for (int i = threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = c.v[i];
}

}  // namespace

extern "C" int numa_rhs_explicit_static(const numa_mesh_desc* mesh, int N, const double* q,
                                        double* rhs, void* stream) {
  if (!mesh || !q || !rhs || q == rhs || N < 1 || N > NUMA_MAXN || mesh->nex < 1 ||
      mesh->ney < 1 || mesh->nez < 1 || !(mesh->Lx > 0) || !(mesh->Ly > 0) || !(mesh->Lz > 0) ||
      !(mesh->n_bv >= 0) || ((uintptr_t)q % 8) || ((uintptr_t)rhs % 8))
    return NUMA_ERR_ARG;
  Geom G{};
  G.N = N; G.Nq = N + 1;
  G.nex = mesh->nex; G.ney = mesh->ney; G.nez = mesh->nez;
  G.nxg = mesh->nex * N + 1; G.nyg = mesh->ney * N + 1; G.M = mesh->nez * N + 1;
  G.ncol = (long long)G.nxg * G.nyg;
  G.nnode = G.ncol * G.M;
  const int M = G.M, W = 2 * N + 1;
  const long long need = G.nnode + 15LL * M + (long long)M * W;
  if (M > kStaticMaxLevels || need > (long long)kStaticScratchDoubles) return NUMA_ERR_SCRATCH;

  std::lock_guard<std::mutex> lock(g_static_mutex);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NUMA_ERR_CUDA;
  if (!g_static_addr[dev]) {       // first call on this device: look up the array's address
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NUMA_ERR_CUDA;
    }
    g_static_addr[dev] = (double*)p;
  }
  double* scratch = g_static_addr[dev];

  double xi[NUMA_MAXNQ], w[NUMA_MAXNQ], D[NUMA_MAXNQ * NUMA_MAXNQ];
  lgl_host(N, xi, w, D);
  Coef3 C;
  set_axis(C.x, N, w, D, mesh->Lx / mesh->nex);
  set_axis(C.y, N, w, D, mesh->Ly / mesh->ney);
  set_axis(C.z, N, w, D, mesh->Lz / mesh->nez);

  // the per-level tables in the order of RefLev: rho0, 1/rho0, theta0, 1/theta0, P0, G0, H0,
  // d(rho0)/dz, d(theta0)/dz, F0z (M each), the column derivative band [M][W], the
  // equation of state's coefficients P0c [M][5]; z last (host only)
  double* h = g_static_host;
  double *rho0 = h, *irho0 = h + M, *th0 = h + 2 * M, *ith0 = h + 3 * M, *P0 = h + 4 * M;
  double *G0 = h + 5 * M, *H0 = h + 6 * M, *drho = h + 7 * M, *dth = h + 8 * M, *F0z = h + 9 * M;
  double* band = h + 10 * M;
  double* P0c = band + (size_t)M * W;
  double* z = P0c + 5 * (size_t)M;
  ref_tables_host(N, mesh->nez, mesh->Lz / mesh->nez, xi, w, D,
                  mesh->theta_s > 0 ? mesh->theta_s : 300.0, mesh->n_bv, z, th0, rho0, P0, G0,
                  H0, band, drho, dth, F0z);
  for (int m = 0; m < M; ++m) {
    irho0[m] = 1.0 / rho0[m];
    ith0[m] = 1.0 / th0[m];
  }
  eos_level_coefs(P0, M, P0c);

  cudaStream_t s = (cudaStream_t)stream;
  double* dPp = scratch;                 // nnode doubles, written by the pre-pass
  double* dtab = scratch + G.nnode;      // the tables above
  const long long ntab = 15LL * M + (long long)M * W;
  for (long long o = 0; o < ntab; o += kTabChunk) {
    TabChunk ch;
    ch.dst = dtab + o;
    ch.n = (int)std::min<long long>(kTabChunk, ntab - o);
    std::memcpy(ch.v, h + o, sizeof(double) * ch.n);
    k_static_tables<<<1, 256, 0, s>>>(ch);
    if (cudaGetLastError() != cudaSuccess) return NUMA_ERR_CUDA;
  }
  const RefLev R{dtab, dtab + M, dtab + 2 * M, dtab + 3 * M, dtab + 4 * M, dtab + 5 * M,
                 dtab + 6 * M, dtab + 7 * M, dtab + 8 * M, dtab + 9 * M, dtab + 10 * M,
                 nullptr, nullptr, nullptr, dtab + 10 * M + (size_t)M * W};
  RhsEpilogue ep{};
  ep.mode = 0;
  if (launch_pressure(q, dPp, G, R, s) != cudaSuccess) return NUMA_ERR_CUDA;
  if (launch_rhs(q, dPp, rhs, nullptr, G.nnode, G, C, R, ep, s) != cudaSuccess) return NUMA_ERR_CUDA;
  return NUMA_OK;
}
