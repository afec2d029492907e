// Host side of the solver: descriptor validation, the level hierarchy and
// its coefficient tables, FAS V-cycles and the FP32/FP64 defect-correction
// loop, the xCFC solve order and divergence cleaning, behind the C ABI of
// include/mg.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "mg.h"
#include "mg_internal.h"

using namespace gmg;

namespace {

constexpr int MAX_LEVELS = 16;
constexpr int NPARTS = 1024;           // blocks of the deterministic sums
constexpr int COARSE_SWEEPS = 16;      // coarsest-grid sweep cap (Sec. 2.7.2)
// Sweep cap of the coarsest scalar correction equation inside the FP32
// correction cycle (mixed precision only; vector equations are solved
// exactly there).  A few sweeps leave the outer FP64 iteration count
// unchanged and cost a quarter of the time on the 3D spherical grids.
constexpr int COARSE_SWEEPS_MIXED = 4;
constexpr double PI = 3.14159265358979323846;

thread_local char g_last_error[256] = "";

struct Level {
  int n[3];
  double h[3], lo[3];
  long sx, sy, off, ng;
  LevelView<double> v64;
  LevelView<float> v32;
  double* ti64 = nullptr;
  double* tj64 = nullptr;
  double* vc64 = nullptr;  // spherical, four-point mixed derivatives: VC_N x n0 x n1
  float* vc32 = nullptr;   // the same in FP32 (FP32 vector smoother and residual)
  float* ti32 = nullptr;
  float* tj32 = nullptr;
  double *u[3] = {}, *uh[3] = {}, *f[3] = {}, *r[3] = {}, *s0 = nullptr, *s1 = nullptr;
  float *e[3] = {}, *f32[3] = {}, *k32 = nullptr;
  GhostPush push[3][2];  // per component and colour (Dirichlet-0 ghosts), or empty
  // tensor maps of the FP32 one-launch sweep (inputs e[leg], f32[0], k32)
  // per sweep leg, when the level stages its planes with them
  SweepMaps sweep_maps[2];
  bool maps_on = false;
  long cells() const { return (long)n[0] * n[1] * n[2]; }
};

}  // namespace

struct GraphEntry {
  int key;
  cudaGraphExec_t exec;
  int64_t updates;    // smoother updates one replay performs
  uint64_t launches;  // kernels one replay launches
};

struct mg_hierarchy {
  mg_grid_desc d;
  cudaStream_t st = nullptr;   // work stream (the caller's, or an owned one)
  bool own_stream = false;
  cudaStream_t user_st = nullptr;   // the caller's stream when st is owned
  cudaEvent_t ev_in = nullptr;      // orders st after the caller's stream
  std::vector<GraphEntry> graphs;
  int nlev = 0;
  Level L[MAX_LEVELS];
  // level-0 arrays of the xCFC sequence (ghosted)
  double *Xg[3] = {}, *dpsi = nullptr, *dap = nullptr, *sg = nullptr, *Ug = nullptr, *Sg = nullptr,
         *Sig[3] = {};
  unsigned long long* d_red = nullptr;   // 8 reduction slots
  unsigned long long* h_red = nullptr;   // pinned mirror
  double* d_part = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // staging buffers for MG_HOST_POINTERS (allocated on first use)
  std::vector<double*> stage;
  int64_t updates = 0;
  // optional event timing of finest-level kernels (mg_profile_enable)
  // Anderson mixing storage (allocated on first use): x, fprev, gprev, then
  // m columns of dF and m of dG, each ncomp arrays of L0.ng doubles
  double* aa = nullptr;
  size_t aa_bytes = 0;
  // mixed precision, vector equations: inverse of the coarsest operator per
  // boundary rule (transposed), state 0 not built, 1 built, -1 unavailable
  double* cinv[3] = {};
  int cinv_state[3] = {0, 0, 0};
  double* cmat[3] = {};  // scalar equations: the coarsest operator per boundary rule (same states)
  int cmat_state[3] = {0, 0, 0};
  double* d_aa_part = nullptr;  // AA_SCRATCH_DOUBLES of device scratch
  // ghost-push tables of the vector colour passes: state 0 not built, 1
  // built, -1 unavailable; one device buffer holds every level's tables
  int push_state = 0;
  int* push_buf = nullptr;
  // MG_DIVB_EXACT: the hierarchy of the parity-class problems (n / 2 cells
  // per dimension), on this hierarchy's stream
  mg_hierarchy* sub = nullptr;
  // device-side cycle loops: one executable graph per equation signature
  // (a while node around the cycle), their state, and whether the device
  // refused graphs with conditional nodes (then the host loop runs)
  struct LoopGraph {
    int key;
    cudaGraphExec_t exec;
    int64_t updates;                 // smoother updates of one cycle
    uint64_t launches_pre, launches; // kernels before the loop and per cycle
  };
  std::vector<LoopGraph> loops;
  LoopState* d_loop = nullptr;
  LoopState* h_loop = nullptr;
  bool loop_off = false;
  // composite grid (mg_solve_scalar_amr): the refined patch of the last box
  // used, allocated on first use
  struct Amr {
    AmrBox box{};
    bool valid = false;
    int n[3] = {1, 1, 1};
    long sx = 0, sy = 0, off = 0, ng = 0;
    LevelView<double> v{};
    double *ti = nullptr, *tj = nullptr;
    double *u = nullptr, *f = nullptr, *r = nullptr, *s0 = nullptr, *s1 = nullptr;
    int* bmap = nullptr;     // ghosted offsets of the uncovered base cells
    long nbase = 0, nvec = 0;
    LevelView<double> flat{};  // the composite unknowns as one row (Anderson mixing)
    double* aa = nullptr;    // g, x, fprev, gprev, then 2 m history columns of flat.n0 doubles
    int aa_m = 0;
    char* mem = nullptr;
    // the composite cycle replayed from a CUDA graph, per equation signature
    int graph_key = -1;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_updates = 0;
    uint64_t graph_launches = 0;
  } amr;
  // persistent batched solves led by this hierarchy (mg_solve_cfc_batch):
  // one device allocation for the descriptors, outcomes, histories, order
  // and queue counter of up to batch_cap problems; events around the launch
  char* batch_mem = nullptr;
  int batch_cap = 0;
  int batch_cycles = 0;  // cycles (psi + alpha psi) of this problem's last batched solve, 0 before one
  BatchItem* b_items = nullptr;
  BatchOut* b_outs = nullptr;
  double* b_hist = nullptr;
  int* b_order = nullptr;
  unsigned int* b_next = nullptr;
  cudaEvent_t b_ev[3] = {};
  bool prof_on = false;
  bool maps_on = false;  // some level's one-launch sweeps stage with tensor maps (d_red[7]: their timeout flag)
  bool fold_k32 = false;  // while capturing a V-cycle of eq. psi: K is restricted on the way down
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_cls;
  std::vector<int64_t> ev_cells;
  size_t ev_used = 0;
};

namespace {

// Event pair around a finest-level launch when profiling is on (any level
// for the classes that are not finest-level ones); returns the pair's slot
// or -1.
long prof_begin(mg_hierarchy* H, int l, int cls, int64_t cells) {
  if (!H->prof_on || (l != 0 && cls < MG_PROF_SMOOTH32_COARSE)) return -1;
  const size_t pair = H->ev_used / 2;
  if (H->ev_used + 2 > H->ev.size()) {
    for (int q = 0; q < 512; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      H->ev.push_back(e);
    }
  }
  if (H->ev_cls.size() <= pair) {
    H->ev_cls.resize(pair + 256);
    H->ev_cells.resize(pair + 256);
  }
  H->ev_cls[pair] = cls;
  H->ev_cells[pair] = cells;
  cudaEventRecord(H->ev[H->ev_used], H->st);
  H->ev_used += 1;
  return (long)pair;
}
void prof_end(mg_hierarchy* H, long tok) {
  if (tok < 0) return;
  cudaEventRecord(H->ev[H->ev_used], H->st);
  H->ev_used += 1;
}

struct Eq {
  int kind, bc, zero_mean, ncomp;
  bool has_c;    // EQ_LIN with a coefficient array
  bool amr = false;  // composite-grid solve: the finest base level carries an FAS right-hand side
};

int fail(int status, const char* what) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", what);
  return status;
}

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", #call, cudaGetErrorString(e_)); \
      return MG_ERR_CUDA;                                                           \
    }                                                                               \
  } while (0)

bool pow2(int v) { return v >= 2 && (v & (v - 1)) == 0; }

int validate(const mg_grid_desc* d) {
  if (!d) return fail(MG_ERR_INVALID, "null descriptor");
  if (d->ndim != 2 && d->ndim != 3) return fail(MG_ERR_INVALID, "ndim must be 2 or 3");
  if (d->geom < MG_CART || d->geom > MG_SPH) return fail(MG_ERR_INVALID, "bad geometry");
  for (int k = 0; k < d->ndim; ++k) {
    if (!pow2(d->n[k])) return fail(MG_ERR_INVALID, "each n must be a power of two >= 2");
    if (!(d->hi[k] > d->lo[k])) return fail(MG_ERR_INVALID, "need lo < hi");
  }
  long cells = 1;
  for (int k = 0; k < d->ndim; ++k) cells *= d->n[k];
  if (cells > (1L << 31)) return fail(MG_ERR_INVALID, "grid too large");
  const double tol_ang = 1e-12;
  if (d->geom == MG_SPH) {
    if (d->lo[0] != 0.0 || d->lo[1] != 0.0 || std::fabs(d->hi[1] - PI) > tol_ang)
      return fail(MG_ERR_INVALID, "spherical grids need r in [0, r_max], theta in [0, pi]");
    if (d->ndim == 3 && (d->lo[2] != 0.0 || std::fabs(d->hi[2] - 2 * PI) > tol_ang))
      return fail(MG_ERR_INVALID, "spherical 3D grids need phi in [0, 2 pi)");
  }
  if (d->geom == MG_CYL) {
    if (d->lo[0] != 0.0) return fail(MG_ERR_INVALID, "cylindrical grids need R in [0, R_max]");
    if (d->ndim == 3 && (d->lo[2] != 0.0 || std::fabs(d->hi[2] - 2 * PI) > tol_ang))
      return fail(MG_ERR_INVALID, "cylindrical 3D grids need phi in [0, 2 pi)");
  }
  if (d->precision != MG_FP64 && d->precision != MG_MIXED) return fail(MG_ERR_INVALID, "bad precision");
  if (d->nu1 < 0 || d->nu2 < 0 || d->nu1 > 64 || d->nu2 > 64 || d->nu1 + d->nu2 == 0)
    return fail(MG_ERR_INVALID, "bad nu1/nu2");
  if (d->max_cycles < 0 || d->max_cycles >= MG_HIST) return fail(MG_ERR_INVALID, "max_cycles out of range");
  if (!(d->tol >= 0.0)) return fail(MG_ERR_INVALID, "bad tol");
  if (d->mixed_deriv != MG_MIXED_4PT && d->mixed_deriv != MG_MIXED_CORNER)
    return fail(MG_ERR_INVALID, "bad mixed_deriv");
  if (d->stall_window < 0) return fail(MG_ERR_INVALID, "bad stall_window");
  if (d->accel_depth < 0 || d->accel_depth > AA_MAX) return fail(MG_ERR_INVALID, "accel_depth must be in 0..16");
  if (d->cycle != MG_CYCLE_V && d->cycle != MG_CYCLE_FMG) return fail(MG_ERR_INVALID, "cycle must be V or FMG");
  if (d->divb_variant != MG_DIVB_COMPACT && d->divb_variant != MG_DIVB_EXACT)
    return fail(MG_ERR_INVALID, "divb_variant must be MG_DIVB_COMPACT or MG_DIVB_EXACT");
  if (d->divb_variant == MG_DIVB_EXACT) {
    if (d->geom != MG_CART) return fail(MG_ERR_INVALID, "MG_DIVB_EXACT needs a Cartesian grid");
    for (int k = 0; k < d->ndim; ++k)
      if (d->n[k] < 4) return fail(MG_ERR_INVALID, "MG_DIVB_EXACT needs every n >= 4");
  }
  return MG_OK;
}

// Descriptor of the parity-class problems of the exact-projection cleaning:
// n / 2 cells per dimension over the same domain (spacing 2 h), the same
// solver settings.
mg_grid_desc class_desc(const mg_grid_desc* d) {
  mg_grid_desc c = *d;
  for (int k = 0; k < d->ndim; ++k) c.n[k] = d->n[k] / 2;
  c.divb_variant = MG_DIVB_COMPACT;
  return c;
}

// Level sizes: halve every dimension while all are even and >= 4.
int level_sizes(const mg_grid_desc* d, int n[][3], double h[][3]) {
  int m[3] = {d->n[0], d->n[1], d->ndim == 3 ? d->n[2] : 1};
  double hh[3];
  for (int k = 0; k < 3; ++k) hh[k] = (k < d->ndim) ? (d->hi[k] - d->lo[k]) / m[k] : 1.0;
  int nl = 0;
  for (;;) {
    for (int k = 0; k < 3; ++k) {
      n[nl][k] = m[k];
      h[nl][k] = hh[k];
    }
    ++nl;
    bool ok = nl < MAX_LEVELS;
    for (int k = 0; k < d->ndim; ++k)
      if (m[k] < 4 || (m[k] & 1)) ok = false;
    if (!ok) break;
    for (int k = 0; k < d->ndim; ++k) {
      m[k] /= 2;
      hh[k] *= 2;
    }
  }
  return nl;
}

// Walk the arena layout; with base == nullptr only sizes are summed.
size_t layout(mg_hierarchy* H, const mg_grid_desc* d, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 255) & ~size_t(255);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  int n[MAX_LEVELS][3];
  double h[MAX_LEVELS][3];
  const int nl = level_sizes(d, n, h);
  const bool mixed = d->precision == MG_MIXED;
  const int three = d->ndim == 3;
  for (int l = 0; l < nl; ++l) {
    const long sx = row_stride(n[l][0]), sy = sx * (n[l][1] + 2);
    const long ng = sy * (n[l][2] + 2 * three);
    const size_t b64 = sizeof(double) * ng, b32 = sizeof(float) * ng;
    Level* L = H ? &H->L[l] : nullptr;
    auto t64 = [&](double** slot, size_t bytes) {
      char* p = take(bytes);
      if (L) *slot = (double*)p;
    };
    auto t32 = [&](float** slot, size_t bytes) {
      char* p = take(bytes);
      if (L) *slot = (float*)p;
    };
    double* dummy64 = nullptr;
    float* dummy32 = nullptr;
    t64(L ? &L->ti64 : &dummy64, sizeof(double) * NTI * (n[l][0] + 2));
    t64(L ? &L->tj64 : &dummy64, sizeof(double) * NTJ * (n[l][1] + 2));
    t32(L ? &L->ti32 : &dummy32, sizeof(float) * NTI * (n[l][0] + 2));
    if (d->geom == MG_SPH && d->mixed_deriv == MG_MIXED_4PT) {
      t64(L ? &L->vc64 : &dummy64, sizeof(double) * VC_N * n[l][0] * n[l][1]);
      if (mixed) t32(L ? &L->vc32 : &dummy32, sizeof(float) * VC_N * n[l][0] * n[l][1]);
    }
    t32(L ? &L->tj32 : &dummy32, sizeof(float) * NTJ * (n[l][1] + 2));
    for (int c = 0; c < 3; ++c) {
      t64(L ? &L->u[c] : &dummy64, b64);
      if (l > 0) t64(L ? &L->uh[c] : &dummy64, b64);
      t64(L ? &L->f[c] : &dummy64, b64);
      t64(L ? &L->r[c] : &dummy64, b64);
    }
    t64(L ? &L->s0 : &dummy64, b64);
    t64(L ? &L->s1 : &dummy64, b64);
    if (mixed) {
      for (int c = 0; c < 3; ++c) {
        t32(L ? &L->e[c] : &dummy32, b32);
        t32(L ? &L->f32[c] : &dummy32, b32);
      }
      t32(L ? &L->k32 : &dummy32, b32);
    }
    if (l == 0) {
      double* dm = nullptr;
      for (int c = 0; c < 3; ++c) {
        char* p = take(b64);
        if (H) H->Xg[c] = (double*)p;
        p = take(b64);
        if (H) H->Sig[c] = (double*)p;
      }
      double** singles[] = {H ? &H->dpsi : &dm, H ? &H->dap : &dm, H ? &H->sg : &dm, H ? &H->Ug : &dm,
                            H ? &H->Sg : &dm};
      for (double** s : singles) {
        char* p = take(b64);
        if (H) *s = (double*)p;
      }
    }
  }
  char* p = take(sizeof(unsigned long long) * 8);
  if (H) H->d_red = (unsigned long long*)p;
  p = take(sizeof(double) * NPARTS);
  if (H) H->d_part = (double*)p;
  return (off + 255) & ~size_t(255);
}

// 1D coefficient tables of one level (Sec. 2.7.1 flux-form operators,
// Appendix A cell volumes for the restriction weights).
void make_tables(const mg_grid_desc* d, const Level& L, std::vector<double>& ti, std::vector<double>& tj) {
  const int n0 = L.n[0], n1 = L.n[1];
  ti.assign((size_t)NTI * (n0 + 2), 0.0);
  tj.assign((size_t)NTJ * (n1 + 2), 0.0);
  const double h0 = L.h[0], h1 = L.h[1], h2 = L.h[2];
  for (int i = -1; i <= n0; ++i) {
    const double x = L.lo[0] + (i + 0.5) * h0, xm = L.lo[0] + i * h0, xp = L.lo[0] + (i + 1) * h0;
    double* T = ti.data() + (i + 1);
    auto S = [&](int slot) -> double& { return T[(size_t)slot * (n0 + 2)]; };
    S(TI_X) = x;
    S(TI_IX) = 1.0 / x;
    S(TI_IX2) = 1.0 / (x * x);
    if (d->geom == MG_CART) {
      S(TI_CE) = S(TI_CW) = 1.0 / (h0 * h0);
      S(TI_VW) = 1.0;
    } else if (d->geom == MG_CYL) {
      S(TI_CE) = xp / (x * h0 * h0);
      S(TI_CW) = xm / (x * h0 * h0);
      S(TI_PHI) = (d->ndim == 3) ? 1.0 / (x * x * h2 * h2) : 0.0;
      S(TI_VW) = x;
    } else {
      S(TI_CE) = xp * xp / (x * x * h0 * h0);
      S(TI_CW) = xm * xm / (x * x * h0 * h0);
      S(TI_VW) = x * x + h0 * h0 / 12.0;
    }
  }
  for (int j = -1; j <= n1; ++j) {
    double* T = tj.data() + (j + 1);
    auto S = [&](int slot) -> double& { return T[(size_t)slot * (n1 + 2)]; };
    if (d->geom == MG_SPH) {
      const double th = L.lo[1] + (j + 0.5) * h1;
      const double s = std::sin(th), c = std::cos(th);
      auto sface = [&](int jf) { return (jf == 0 || jf == n1) ? 0.0 : std::sin(L.lo[1] + jf * h1); };
      S(TJ_S) = s;
      S(TJ_C) = c;
      S(TJ_IS) = 1.0 / s;
      S(TJ_IS2) = 1.0 / (s * s);
      S(TJ_COT) = c / s;
      S(TJ_TN) = sface(j + 1) / (s * h1 * h1);
      S(TJ_TS) = sface(j) / (s * h1 * h1);
      S(TJ_PF) = (d->ndim == 3) ? 1.0 / (s * s * h2 * h2) : 0.0;
      S(TJ_VW) = s;
    } else {
      S(TJ_S) = 1.0;
      S(TJ_VW) = 1.0;
    }
  }
}

// The vector operator lap V + 1/3 grad div V on a spherical level as a
// stencil per component: the coefficients of vec_op (metric factors, the
// 1/3 of the grad-div part and the difference scales) multiplied out per
// (i, j), so that the FP64 residual spends one FMA per stencil term.  Same
// operator, different rounding order.
void make_vec_coeffs(const mg_grid_desc* d, const Level& L, const std::vector<double>& ti,
                     const std::vector<double>& tj, std::vector<double>& vc) {
  const int n0 = L.n[0], n1 = L.n[1];
  const bool three = d->ndim == 3;
  vc.assign((size_t)VC_N * n0 * n1, 0.0);
  const double ih0s = 1.0 / (L.h[0] * L.h[0]), ih1s = 1.0 / (L.h[1] * L.h[1]), ih2s = 1.0 / (L.h[2] * L.h[2]);
  const double hc0 = 0.5 / L.h[0], hc1 = 0.5 / L.h[1], hc2 = 0.5 / L.h[2];
  const double m01 = 1.0 / (4.0 * L.h[0] * L.h[1]), m02 = 1.0 / (4.0 * L.h[0] * L.h[2]);
  const double m12 = 1.0 / (4.0 * L.h[1] * L.h[2]);
  const double t3 = 1.0 / 3.0;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      auto I = [&](int s) { return ti[(size_t)s * (n0 + 2) + i + 1]; };
      auto J = [&](int s) { return tj[(size_t)s * (n1 + 2) + j + 1]; };
      const double x = I(TI_X), ir = I(TI_IX), ir2 = I(TI_IX2), cE = I(TI_CE), cW = I(TI_CW);
      const double s = J(TJ_S), ct = J(TJ_C), ist = J(TJ_IS), ist2 = J(TJ_IS2), cot = J(TJ_COT);
      const double tN = J(TJ_TN), tS = J(TJ_TS), pf = three ? J(TJ_PF) : 0.0;
      const double lapc = cE + cW + ir2 * (tN + tS) + 2.0 * ir2 * pf;
      double c[VC_N] = {0.0};
      // r: lap V_r + 1/3 d_rr V_r + 2/3 r^-1 d_r V_r - 8/3 r^-2 V_r
      //    - 7/3 r^-2 d_th V_th - 7/3 cot r^-2 V_th + 1/3 cot r^-1 d_r V_th + 1/3 r^-1 d_r d_th V_th
      //    - 7/3 r^-2 sin^-1 d_ph V_ph + 1/3 r^-1 sin^-1 d_r d_ph V_ph
      c[0] = cE + t3 * ih0s + 2.0 * t3 * ir * hc0;
      c[1] = cW + t3 * ih0s - 2.0 * t3 * ir * hc0;
      c[2] = ir2 * tN;
      c[3] = ir2 * tS;
      c[4] = ir2 * pf;
      c[5] = -lapc - 2.0 * t3 * ih0s - 8.0 * t3 * ir2;
      c[6] = -7.0 * t3 * ir2 * hc1;
      c[7] = -7.0 * t3 * cot * ir2;
      c[8] = t3 * cot * ir * hc0;
      c[9] = t3 * ir * m01;
      c[10] = three ? -7.0 * t3 * ir2 * ist * hc2 : 0.0;
      c[11] = three ? t3 * ir * ist * m02 : 0.0;
      // theta: lap V_th + 1/3 r^-2 d_thth V_th + 1/3 cot r^-2 d_th V_th - 4/3 r^-2 sin^-2 V_th
      //    + 8/3 r^-2 d_th V_r + 1/3 r^-1 d_r d_th V_r
      //    - 7/3 cos r^-2 sin^-2 d_ph V_ph + 1/3 r^-2 sin^-1 d_th d_ph V_ph
      c[12] = cE;
      c[13] = cW;
      c[14] = ir2 * tN + t3 * ir2 * ih1s + t3 * cot * ir2 * hc1;
      c[15] = ir2 * tS + t3 * ir2 * ih1s - t3 * cot * ir2 * hc1;
      c[16] = ir2 * pf;
      c[17] = -lapc - 2.0 * t3 * ir2 * ih1s - 4.0 * t3 * ir2 * ist2;
      c[18] = 8.0 * t3 * ir2 * hc1;
      c[19] = t3 * ir * m01;
      c[20] = three ? -7.0 * t3 * ct * ir2 * ist2 * hc2 : 0.0;
      c[21] = three ? t3 * ir2 * ist * m12 : 0.0;
      // phi: lap V_ph + 1/3 r^-2 sin^-2 d_phph V_ph - r^-2 sin^-2 V_ph
      //    + 8/3 r^-2 sin^-1 d_ph V_r + 1/3 r^-1 sin^-1 d_r d_ph V_r
      //    + 7/3 cos r^-2 sin^-2 d_ph V_th + 1/3 r^-2 sin^-1 d_th d_ph V_th
      c[22] = cE;
      c[23] = cW;
      c[24] = ir2 * tN;
      c[25] = ir2 * tS;
      c[26] = ir2 * pf + (three ? t3 * ir2 * ist2 * ih2s : 0.0);
      c[27] = -lapc - (three ? 2.0 * t3 * ir2 * ist2 * ih2s : 0.0) - ir2 * ist2;
      c[28] = three ? 8.0 * t3 * ir2 * ist * hc2 : 0.0;
      c[29] = three ? t3 * ir * ist * m02 : 0.0;
      c[30] = three ? 7.0 * t3 * ct * ir2 * ist2 * hc2 : 0.0;
      c[31] = three ? t3 * ir2 * ist * m12 : 0.0;
      c[32] = x * x * s;  // norm weight r^2 sin(theta)
      for (int q = 0; q < VC_N; ++q) vc[((size_t)q * n1 + j) * n0 + i] = c[q];
    }
}

template <typename T>
LevelView<T> make_view(const mg_grid_desc* d, const Level& L, const T* ti, const T* tj) {
  LevelView<T> v;
  v.n0 = L.n[0];
  v.n1 = L.n[1];
  v.n2 = L.n[2];
  v.three = d->ndim == 3;
  v.geom = d->geom;
  v.bc = MG_BC_ROBIN;
  v.mixed = d->mixed_deriv;
  v.sx = L.sx;
  v.sy = L.sy;
  v.off = L.off;
  v.h0 = (T)L.h[0];
  v.h1 = (T)L.h[1];
  v.h2 = (T)L.h[2];
  v.lo0 = (T)L.lo[0];
  v.lo1 = (T)L.lo[1];
  v.lo2 = (T)L.lo[2];
  v.ih0s = (T)(1.0 / (L.h[0] * L.h[0]));
  v.ih1s = (T)(1.0 / (L.h[1] * L.h[1]));
  v.ih2s = (T)(1.0 / (L.h[2] * L.h[2]));
  v.hc0 = (T)(0.5 / L.h[0]);
  v.hc1 = (T)(0.5 / L.h[1]);
  v.hc2 = (T)(0.5 / L.h[2]);
  const double mf = d->mixed_deriv == MG_MIXED_4PT ? 4.0 : 2.0;
  v.m01 = (T)(1.0 / (mf * L.h[0] * L.h[1]));
  v.m02 = (T)(1.0 / (mf * L.h[0] * L.h[2]));
  v.m12 = (T)(1.0 / (mf * L.h[1] * L.h[2]));
  const double rN = L.lo[0] + (L.n[0] - 0.5) * L.h[0], rG = L.lo[0] + (L.n[0] + 0.5) * L.h[0];
  v.robin0 = (T)(rN / rG);
  v.ln0 = 0;
  while ((1 << v.ln0) < L.n[0]) ++v.ln0;
  v.ln1 = 0;
  while ((1 << v.ln1) < L.n[1]) ++v.ln1;
  v.ti = ti;
  v.tj = tj;
  v.vc = nullptr;
  return v;
}

template <typename T>
LevelView<T> with_bc(LevelView<T> v, int bc) {
  v.bc = bc;
  return v;
}

// Ghost-push table of a vector colour pass, when built and the pass's ghost
// rule is the one it was built for.
GhostPush ghost_push(const mg_hierarchy* H, int l, int c, int colour, int bc) {
  if (H->push_state != 1 || bc != MG_BC_DIRICHLET) return GhostPush{};
  return H->L[l].push[c][colour];
}

// ------------------------------------------------------------- FP64 FAS

const double* fptr(const mg_hierarchy* H, const Eq& e, int l, int c) {
  if (l == 0 && e.kind == EQ_PSI && !e.amr) return nullptr;  // finest right-hand side is zero
  return H->L[l].f[c];
}
const double* s0ptr(const mg_hierarchy* H, const Eq& e, int l) {
  return e.kind == EQ_PSI ? H->L[l].s0 : nullptr;
}
const double* s1ptr(const mg_hierarchy* H, const Eq& e, int l) {
  return (e.kind == EQ_PSI || e.has_c) ? H->L[l].s1 : nullptr;
}

void fill_all64(mg_hierarchy* H, const Eq& e, int l) {
  Level& L = H->L[l];
  launch_fill_ghosts3(with_bc(L.v64, e.bc), L.u, 3, 1, H->st);
}

void smooth64(mg_hierarchy* H, const Eq& e, int l, int nsweeps) {
  Level& L = H->L[l];
  auto v = with_bc(L.v64, e.bc);
  int s0 = 0;
  if (e.kind == EQ_LIN && fused_sweep_applies(v)) {
    // sweeps in pairs, out of place through the free component-1 array:
    // u[0] -> u[1] -> u[0]; an odd last sweep runs as two colour passes
    for (; s0 + 2 <= nsweeps; s0 += 2) {
      for (int leg = 0; leg < 2; ++leg) {
        long tok = prof_begin(H, l, MG_PROF_SWEEP64_FUSED, L.cells());
        launch_sweep_fused<double>(v, L.u[leg], L.u[1 - leg], fptr(H, e, l, 0), s1ptr(H, e, l), H->st);
        prof_end(H, tok);
      }
    }
  }
  for (int s = s0; s < nsweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour) {
      if (e.kind != EQ_VEC) {
        long tok = prof_begin(H, l, MG_PROF_SMOOTH64_SCALAR, L.cells() / 2);
        launch_smooth_scalar(v, e.kind, L.u[0], fptr(H, e, l, 0), s0ptr(H, e, l), s1ptr(H, e, l), colour, H->st);
        prof_end(H, tok);
      } else {
        for (int c = 0; c < 3; ++c) {
          long tok = prof_begin(H, l, MG_PROF_SMOOTH64_VEC, L.cells() / 2);
          const GhostPush gp = ghost_push(H, l, c, colour, e.bc);
          launch_smooth_vec(v, L.u, fptr(H, e, l, c), c, colour, H->st, gp);
          prof_end(H, tok);
          if (!gp.off) launch_fill_ghosts(v, L.u[c], c, H->st);
        }
      }
    }
  }
  H->updates += (int64_t)nsweeps * L.cells() * e.ncomp;
}

void coarse64(mg_hierarchy* H, const Eq& e, int l) {
  Level& L = H->L[l];
  auto v = with_bc(L.v64, e.bc);
  if (e.kind != EQ_VEC) {
    launch_coarse_scalar(v, e.kind, L.u[0], fptr(H, e, l, 0), s0ptr(H, e, l), s1ptr(H, e, l), COARSE_SWEEPS, H->st);
  } else {
    const double* f[3] = {fptr(H, e, l, 0), fptr(H, e, l, 1), fptr(H, e, l, 2)};
    launch_coarse_vec(v, L.u, f, COARSE_SWEEPS, H->st);
  }
}

// FAS V(nu1, nu2): pre-smooth; r = f - L(u); u_H = R u (kept as uh_H);
// f_H = L_H(u_H) + R r; recurse; u += P(u_H - uh_H); post-smooth.
// FAS restriction from level l to l + 1 at the current u_l:
// r = f - L(u); u_H = R u (kept as uh_H); f_H = L_H(u_H) + R r.
void fas_down64(mg_hierarchy* H, const Eq& e, int l) {
  Level& L = H->L[l];
  Level& C = H->L[l + 1];
  auto v = with_bc(L.v64, e.bc);
  auto vc = with_bc(C.v64, e.bc);
  if (e.kind != EQ_VEC) {
    launch_residual_scalar(v, e.kind, L.u[0], fptr(H, e, l, 0), s0ptr(H, e, l), s1ptr(H, e, l), L.r[0],
                           (unsigned long long*)nullptr, 0, H->st);
  } else {
    const double* f[3] = {fptr(H, e, l, 0), fptr(H, e, l, 1), fptr(H, e, l, 2)};
    launch_residual_vec(v, L.u, f, L.r, (unsigned long long*)nullptr, 0, H->st);
  }
  for (int c = 0; c < e.ncomp; ++c) {
    const double* a[4] = {L.u[c], L.r[c], nullptr, nullptr};
    double* b[4] = {C.u[c], C.f[c], nullptr, nullptr};
    double* cp[3] = {C.uh[c], nullptr, nullptr};
    launch_restrict(v, vc, 2, a, b, cp, H->st);
  }
  if (e.kind != EQ_VEC) {
    launch_apply_scalar(vc, e.kind, C.u[0], s0ptr(H, e, l + 1), s1ptr(H, e, l + 1), C.f[0], 1, H->st);
  } else {
    fill_all64(H, e, l + 1);
    launch_apply_vec(vc, C.u, C.f, 1, H->st);
  }
}

// FAS correction of level l from level l + 1: u += P(u_H - uh_H).
void fas_up64(mg_hierarchy* H, const Eq& e, int l) {
  Level& L = H->L[l];
  Level& C = H->L[l + 1];
  auto v = with_bc(L.v64, e.bc);
  auto vc = with_bc(C.v64, e.bc);
  const double* uH[3] = {C.u[0], C.u[1], C.u[2]};
  const double* uhH[3] = {C.uh[0], C.uh[1], C.uh[2]};
  launch_prolong3(v, vc, L.u, uH, uhH, e.ncomp, e.kind == EQ_VEC, H->st);
  if (e.kind == EQ_VEC) fill_all64(H, e, l);
}

void vcycle64(mg_hierarchy* H, const Eq& e, int l) {
  if (l == H->nlev - 1) {
    coarse64(H, e, l);
    return;
  }
  smooth64(H, e, l, H->d.nu1);
  fas_down64(H, e, l);
  vcycle64(H, e, l + 1);
  fas_up64(H, e, l);
  smooth64(H, e, l, H->d.nu2);
}

// FAS full-multigrid cycle (Sec. 4.2 times FMG cycles): restrict the
// current solution and FAS sources to every level, solve the coarsest, then
// per level upward: FAS correction from below and one V-cycle from there.
void fmg64(mg_hierarchy* H, const Eq& e) {
  for (int l = 0; l + 1 < H->nlev; ++l) fas_down64(H, e, l);
  coarse64(H, e, H->nlev - 1);
  for (int l = H->nlev - 2; l >= 0; --l) {
    fas_up64(H, e, l);
    vcycle64(H, e, l);
  }
}

double bits_to_double(unsigned long long b) {
  double x;
  std::memcpy(&x, &b, sizeof(x));
  return x;
}

// Finest-level residual with the norms of the stopping rule into the
// reduction slots 0..2 (enqueued only); in mixed precision the residual is
// also stored, rounded, as the FP32 right-hand side f32.
int finest_residual(mg_hierarchy* H, const Eq& e) {
  Level& L = H->L[0];
  auto v = with_bc(L.v64, e.bc);
  CK(cudaMemsetAsync(H->d_red, 0, sizeof(unsigned long long) * 3, H->st));
  long tok = prof_begin(H, 0,
                        e.kind == EQ_VEC ? MG_PROF_RESID64_VEC
                                         : (e.kind == EQ_PSI ? MG_PROF_RESID64_PSI : MG_PROF_RESID64_SCALAR),
                        L.cells());
  // the residual itself is needed only as the FP32 right-hand side of the
  // next correction cycle (mixed); the FP64 V-cycle recomputes its own
  const bool mixed = H->d.precision == MG_MIXED;
  if (e.kind != EQ_VEC) {
    launch_residual_scalar(v, e.kind, L.u[0], fptr(H, e, 0, 0), s0ptr(H, e, 0), s1ptr(H, e, 0),
                           (double*)nullptr, H->d_red, 1, H->st, mixed ? L.f32[0] : nullptr,
                           (mixed && e.kind == EQ_PSI) ? L.k32 : nullptr);
  } else {
    const double* f[3] = {L.f[0], L.f[1], L.f[2]};
    double* const none[3] = {nullptr, nullptr, nullptr};
    launch_residual_vec(v, L.u, f, none, H->d_red, 1, H->st, mixed ? L.f32 : nullptr);
  }
  prof_end(H, tok);
  CK(cudaGetLastError());
  return MG_OK;
}

// Finest-level residual and its weighted relative norm, read on the host.
int finest_norm(mg_hierarchy* H, const Eq& e, double* rel) {
  if (int st = finest_residual(H, e)) return st;
  // slot 3: status of this cycle's mixing solve (read by run_solve)
  CK(cudaMemcpyAsync(H->h_red, H->d_red, sizeof(unsigned long long) * 4, cudaMemcpyDeviceToHost, H->st));
  CK(cudaStreamSynchronize(H->st));
  const double num = bits_to_double(H->h_red[1]), den = bits_to_double(H->h_red[2]);
  if (std::isinf(num) || std::isinf(den) || std::isnan(num) || std::isnan(den)) {
    *rel = NAN;
  } else {
    *rel = num / (den > 1e-300 ? den : 1e-300);
  }
  return MG_OK;
}

void restrict_sources(mg_hierarchy* H, const Eq& e) {
  if (e.kind == EQ_VEC) return;
  const int nf = e.kind == EQ_PSI ? 2 : (e.has_c ? 1 : 0);
  if (!nf) return;
  for (int l = 1; l < H->nlev; ++l) {
    Level& F = H->L[l - 1];
    Level& C = H->L[l];
    const double* a[4] = {e.kind == EQ_PSI ? F.s0 : F.s1, F.s1, nullptr, nullptr};
    double* b[4] = {e.kind == EQ_PSI ? C.s0 : C.s1, C.s1, nullptr, nullptr};
    double* cp[3] = {nullptr, nullptr, nullptr};
    launch_restrict(F.v64, C.v64, nf, a, b, cp, H->st);
  }
}

// ------------------------------------------------ FP32 correction cycle

void smooth32(mg_hierarchy* H, const Eq& e, int l, int nsweeps) {
  Level& L = H->L[l];
  auto v = with_bc(L.v32, e.bc);
  const float* K = (e.kind == EQ_PSI || e.has_c) ? L.k32 : nullptr;
  int s0 = 0;
  if (e.kind != EQ_VEC && fused_sweep_applies(v)) {
    // as in smooth64: pairs of out-of-place sweeps e[0] -> e[1] -> e[0]
    for (; s0 + 2 <= nsweeps; s0 += 2) {
      for (int leg = 0; leg < 2; ++leg) {
        long tok = prof_begin(H, l, MG_PROF_SWEEP32_FUSED, L.cells());
        launch_sweep_fused<float>(v, L.e[leg], L.e[1 - leg], L.f32[0], K, H->st,
                                  L.maps_on ? &L.sweep_maps[leg] : nullptr);
        prof_end(H, tok);
      }
    }
  }
  for (int s = s0; s < nsweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour) {
      if (e.kind != EQ_VEC) {
        long tok = prof_begin(H, l, l ? MG_PROF_SMOOTH32_COARSE : MG_PROF_SMOOTH32_SCALAR, L.cells() / 2);
        launch_smooth_scalar<float>(v, EQ_LIN, L.e[0], L.f32[0], nullptr, K, colour, H->st);
        prof_end(H, tok);
      } else {
        for (int c = 0; c < 3; ++c) {
          long tok = prof_begin(H, l, l ? MG_PROF_SMOOTH32_COARSE : MG_PROF_SMOOTH32_VEC, L.cells() / 2);
          const GhostPush gp = ghost_push(H, l, c, colour, e.bc);
          launch_smooth_vec<float>(v, L.e, L.f32[c], c, colour, H->st, gp);
          prof_end(H, tok);
          if (!gp.off) launch_fill_ghosts<float>(v, L.e[c], c, H->st);
        }
      }
    }
  }
  H->updates += (int64_t)nsweeps * L.cells() * e.ncomp;
}

// Coarsest correction equation solved in FP64 on the level's FP64 scratch.
void coarse32(mg_hierarchy* H, const Eq& e, int l) {
  Level& L = H->L[l];
  auto v = with_bc(L.v64, e.bc);
  const size_t b64 = sizeof(double) * L.ng;
  for (int c = 0; c < e.ncomp; ++c) {
    launch_convert<float, double>(L.v32, L.f32[c], L.f[c], H->st);
    cudaMemsetAsync(L.u[c], 0, b64, H->st);
  }
  if (e.kind != EQ_VEC) {
    const bool hasK = e.kind == EQ_PSI || e.has_c;
    if (hasK) launch_convert<float, double>(L.v32, L.k32, L.r[0], H->st);
    launch_coarse_scalar<double>(v, EQ_LIN, L.u[0], L.f[0], nullptr, hasK ? L.r[0] : nullptr, COARSE_SWEEPS,
                                 H->st);
  } else {
    const double* f[3] = {L.f[0], L.f[1], L.f[2]};
    launch_coarse_vec<double>(v, L.u, f, COARSE_SWEEPS, H->st);
  }
  for (int c = 0; c < e.ncomp; ++c) launch_convert<double, float>(L.v64, L.u[c], L.e[c], H->st);
  if (e.kind == EQ_VEC) launch_fill_ghosts3<float>(with_bc(L.v32, e.bc), L.e, 3, 1, H->st);
}

// Parameters of the one-block coarse cycle from level l0 (mg_block.cu):
// shared-memory offsets of every level's arrays; P.smem = 0 when they do
// not fit.
BlockCycle32 block_cycle_params(mg_hierarchy* H, const Eq& e, int l0) {
  BlockCycle32 P{};
  const bool hasK = e.kind == EQ_PSI || e.has_c;
  const int nc = e.kind == EQ_VEC ? 3 : 1;
  P.nl = H->nlev - l0;
  if (P.nl > BC_MAX) return P;
  P.vec = e.kind == EQ_VEC;
  P.nu1 = H->d.nu1;
  P.nu2 = H->d.nu2;
  P.coarse_sweeps = COARSE_SWEEPS_MIXED;
  long fl = 0;  // floats
  auto take = [&](long n) {
    const long at = fl;
    fl += (n + 3) & ~3L;
    return (int)at;
  };
  for (int q = 0; q < P.nl; ++q) {
    Level& L = H->L[l0 + q];
    BlockLevel32& B = P.lv[q];
    B.v = with_bc(L.v32, e.bc);
    for (int c = 0; c < 3; ++c) {
      if (c < nc) {
        B.e[c] = take(L.ng);
        B.f32[c] = take(L.ng);
        B.r32[c] = take(L.ng);
      } else {
        B.e[c] = B.e[0];
        B.f32[c] = B.f32[0];
        B.r32[c] = B.r32[0];
      }
    }
    B.k32 = hasK ? L.k32 : nullptr;
    B.ti_at = take((long)NTI * (L.n[0] + 2));
    B.tj_at = take((long)NTJ * (L.n[1] + 2));
    B.k_at = hasK ? take(L.ng) : -1;
  }
  Level& Lc = H->L[H->nlev - 1];
  P.c64 = with_bc(Lc.v64, e.bc);
  P.fp64_at = (long)sizeof(float) * fl;
  long dl = 0;  // doubles
  auto taked = [&](long n) {
    const long at = dl;
    dl += (n + 1) & ~1L;
    return (int)at;
  };
  for (int c = 0; c < 3; ++c) {
    P.cu[c] = c < nc ? taked(Lc.ng) : P.cu[0];
    P.cf[c] = c < nc ? taked(Lc.ng) : P.cf[0];
  }
  P.ck = (hasK && !P.vec) ? taked(Lc.ng) : -1;
  if (P.vec && H->cinv_state[e.bc] == 1) {
    P.cinv = H->cinv[e.bc];
    P.cn = (int)(3 * Lc.cells());
  }
  if (!P.vec && H->cmat_state[e.bc] == 1) {
    P.cA = H->cmat[e.bc];
    P.cn = (int)Lc.cells();
  }
  Level& L0 = H->L[l0];
  P.ng0 = L0.ng;
  for (int c = 0; c < 3; ++c) {
    P.f_in[c] = L0.f32[c];
    P.e_out[c] = L0.e[c];
  }
  const size_t bytes = (size_t)P.fp64_at + sizeof(double) * (size_t)dl;
  P.smem = bytes <= BC_SMEM_MAX ? bytes : 0;
  return P;
}

// First level of the one-block coarse cycle: the first level of at most
// BLOCK_CYCLE_CELLS cells whose levels down to the coarsest fit the block's
// shared memory.
int block_cycle_level(mg_hierarchy* H, const Eq& e) {
  for (int l = 0; l < H->nlev; ++l)
    if (H->L[l].cells() <= BLOCK_CYCLE_CELLS && block_cycle_params(H, e, l).smem > 0) return l;
  return H->nlev;
}

void restrict_k32(mg_hierarchy* H, int from);

// vcycle32 from level l0 down, in one block.
void block_vcycle32(mg_hierarchy* H, const Eq& e, int l0) {
  // K of eq. psi reached level l0 with the down leg; on to the block's levels
  if (H->fold_k32) restrict_k32(H, l0 + 1);
  const BlockCycle32 P = block_cycle_params(H, e, l0);
  for (int l = l0; l + 1 < H->nlev; ++l) H->updates += (int64_t)(H->d.nu1 + H->d.nu2) * H->L[l].cells() * e.ncomp;
  long tok = prof_begin(H, l0, MG_PROF_BLOCK_CYCLE32, H->L[l0].cells());
  launch_block_vcycle32(P, H->d.geom, H->st);
  prof_end(H, tok);
}

// Linear correction-scheme V-cycle on (L - K) e = f32, e = 0 initially.
void vcycle32(mg_hierarchy* H, const Eq& e, int l) {
  if (l >= block_cycle_level(H, e)) {
    block_vcycle32(H, e, l);
    return;
  }
  if (l == H->nlev - 1) {
    coarse32(H, e, l);
    return;
  }
  Level& L = H->L[l];
  Level& C = H->L[l + 1];
  auto v = with_bc(L.v32, e.bc);
  auto vc = with_bc(C.v32, e.bc);
  const float* K = (e.kind == EQ_PSI || e.has_c) ? L.k32 : nullptr;
  smooth32(H, e, l, H->d.nu1);
  // residual restricted into the coarse right-hand side, coarse e zeroed
  // (and K of eq. psi restricted) in one launch
  launch_resid_restrict32(v, vc, e.kind == EQ_VEC, L.e, L.f32, K, C.f32, C.e, H->fold_k32 ? C.k32 : nullptr,
                          H->st);
  vcycle32(H, e, l + 1);
  const float* eH[3] = {C.e[0], C.e[1], C.e[2]};
  launch_prolong3<float>(v, vc, L.e, eH, nullptr, e.ncomp, e.kind == EQ_VEC, H->st);
  if (e.kind == EQ_VEC) launch_fill_ghosts3<float>(v, L.e, 3, 1, H->st);
  smooth32(H, e, l, H->d.nu2);
}

// K of the correction equation restricted into levels from .. nlev - 1.
void restrict_k32(mg_hierarchy* H, int from) {
  for (int l = from; l < H->nlev; ++l) {
    Level& F = H->L[l - 1];
    Level& C = H->L[l];
    const float* a[4] = {F.k32, nullptr, nullptr, nullptr};
    float* b[4] = {C.k32, nullptr, nullptr, nullptr};
    float* cp[3] = {nullptr, nullptr, nullptr};
    launch_restrict<float>(F.v32, C.v32, 1, a, b, cp, H->st);
  }
}

// FMG for the correction equation (L - K) e = f32 from e = 0: the
// right-hand side restricted down (the residual of e = 0 is f32 itself) to
// the first level of the one-block cycle (or the coarsest), one correction
// cycle there, then per level upward: e_l = P e_{l+1} and one correction
// V-cycle from that level.
void fmg32(mg_hierarchy* H, const Eq& e) {
  const int lb = std::min(block_cycle_level(H, e), H->nlev - 1);
  for (int l = 0; l < lb; ++l) {
    Level& L = H->L[l];
    Level& C = H->L[l + 1];
    auto v = with_bc(L.v32, e.bc);
    auto vc = with_bc(C.v32, e.bc);
    for (int c = 0; c < e.ncomp; ++c) {
      const float* a[4] = {L.f32[c], nullptr, nullptr, nullptr};
      float* b[4] = {C.f32[c], nullptr, nullptr, nullptr};
      float* cp[3] = {nullptr, nullptr, nullptr};
      launch_restrict<float>(v, vc, 1, a, b, cp, H->st);
    }
  }
  for (int c = 0; c < e.ncomp; ++c) cudaMemsetAsync(H->L[lb].e[c], 0, sizeof(float) * H->L[lb].ng, H->st);
  vcycle32(H, e, lb);
  for (int l = lb - 1; l >= 0; --l) {
    Level& L = H->L[l];
    Level& C = H->L[l + 1];
    auto v = with_bc(L.v32, e.bc);
    auto vc = with_bc(C.v32, e.bc);
    for (int c = 0; c < e.ncomp; ++c) cudaMemsetAsync(L.e[c], 0, sizeof(float) * L.ng, H->st);
    const float* eH[3] = {C.e[0], C.e[1], C.e[2]};
    launch_prolong3<float>(v, vc, L.e, eH, nullptr, e.ncomp, e.kind == EQ_VEC, H->st);
    if (e.kind == EQ_VEC) launch_fill_ghosts3<float>(v, L.e, 3, 1, H->st);
    vcycle32(H, e, l);
  }
}

// ---------------------------------------------------------- cycle control

// One application of the iteration map: a V-cycle (FP64 FAS, or the FP32
// correction cycle of the defect-correction loop) and the Neumann gauge.
int cycle_map(mg_hierarchy* H, const Eq& e) {
  Level& L0 = H->L[0];
  const bool fmg = H->d.cycle == MG_CYCLE_FMG;
  if (H->d.precision != MG_MIXED) {
    if (fmg)
      fmg64(H, e);
    else
      vcycle64(H, e, 0);
  } else {
    auto v = with_bc(L0.v64, e.bc);
    // f32 holds the FP32 residual written by the preceding finest_norm
    for (int c = 0; c < e.ncomp; ++c) CK(cudaMemsetAsync(L0.e[c], 0, sizeof(float) * L0.ng, H->st));
    // eq. psi: K = dS/du at this u was written by finest_norm with f32; the
    // V-cycle restricts it level by level on its way down (fold_k32)
    if (e.kind == EQ_PSI && fmg) restrict_k32(H, 1);
    H->fold_k32 = e.kind == EQ_PSI && !fmg;
    if (fmg)
      fmg32(H, e);
    else
      vcycle32(H, e, 0);
    H->fold_k32 = false;
    const float* ee[3] = {L0.e[0], L0.e[1], L0.e[2]};
    launch_add_correction<float>(v, e.ncomp, L0.u, ee, H->st, e.zero_mean ? H->d_part : nullptr, NPARTS);
  }
  if (e.zero_mean) launch_sub_mean(L0.v64, L0.u[0], H->d_part, NPARTS, H->st, H->d.precision == MG_MIXED);
  if (e.kind == EQ_VEC) fill_all64(H, e, 0);
  return MG_OK;
}

// The cycle map replayed from a CUDA graph captured on first use (one per
// equation signature): the launch sequence and every pointer it touches are
// fixed for a hierarchy.  Direct launches while profiling.
int run_cycle_map(mg_hierarchy* H, const Eq& e) {
  if (H->prof_on) return cycle_map(H, e);
  const int key = e.kind | (e.bc << 2) | (e.zero_mean << 4) | ((int)e.has_c << 5) | (H->d.precision << 6);
  for (const GraphEntry& g : H->graphs)
    if (g.key == key) {
      CK(cudaGraphLaunch(g.exec, H->st));
      H->updates += g.updates;
      count_launch((int)g.launches);
      return MG_OK;
    }
  const int64_t u0 = H->updates;
  const unsigned long long l0 = launch_count();
  CK(cudaStreamBeginCapture(H->st, cudaStreamCaptureModeThreadLocal));
  int st = cycle_map(H, e);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(H->st, &graph);
  if (st) return st;
  if (ce != cudaSuccess || !graph) {
    std::snprintf(g_last_error, sizeof(g_last_error), "graph capture: %s", cudaGetErrorString(ce));
    return MG_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    std::snprintf(g_last_error, sizeof(g_last_error), "graph instantiate: %s", cudaGetErrorString(ce));
    return MG_ERR_CUDA;
  }
  GraphEntry g{key, exec, H->updates - u0, launch_count() - l0};
  H->graphs.push_back(g);
  H->updates = u0;
  CK(cudaGraphLaunch(exec, H->st));
  H->updates += g.updates;
  return MG_OK;
}

// Mixing storage: x, fprev, gprev (FP64) and 2 m history columns of
// col_bytes per value, each ncomp arrays of L0.ng values.
int ensure_aa(mg_hierarchy* H, int ncomp, int m, size_t col_bytes) {
  const size_t vals = (size_t)H->L[0].ng * ncomp;
  const size_t need = vals * (3 * sizeof(double) + 2 * (size_t)m * col_bytes);
  if (H->aa_bytes < need) {
    if (H->aa) cudaFree(H->aa);
    H->aa = nullptr;
    H->aa_bytes = 0;
    if (cudaMalloc(&H->aa, need) != cudaSuccess) return fail(MG_ERR_OOM, "mixing storage allocation failed");
    H->aa_bytes = need;
  }
  if (!H->d_aa_part) {
    if (cudaMalloc(&H->d_aa_part, sizeof(double) * AA_SCRATCH_DOUBLES) != cudaSuccess) {
      H->d_aa_part = nullptr;
      return fail(MG_ERR_OOM, "mixing scratch failed");
    }
    // the finished-block counter starts at zero
    CK(cudaMemsetAsync(H->d_aa_part, 0, sizeof(double) * AA_SCRATCH_DOUBLES, H->st));
  }
  return MG_OK;
}

// Inverse of a dense n x n matrix (column-major, A[col * n + r]) by
// Gauss-Jordan elimination with partial pivoting, returned transposed
// (T[col * n + r] = inv[r][col]); false when A is numerically singular.
bool invert_dense(int n, const std::vector<double>& A, std::vector<double>& T) {
  std::vector<double> M((size_t)n * 2 * n, 0.0);  // row-major [A | I]
  double amax = 0.0;
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < n; ++c) {
      M[(size_t)r * 2 * n + c] = A[(size_t)c * n + r];
      amax = std::max(amax, std::fabs(A[(size_t)c * n + r]));
    }
    M[(size_t)r * 2 * n + n + r] = 1.0;
  }
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(M[(size_t)r * 2 * n + k]) > std::fabs(M[(size_t)piv * 2 * n + k])) piv = r;
    const double pv = M[(size_t)piv * 2 * n + k];
    if (!(std::fabs(pv) > 1e-13 * amax)) return false;
    if (piv != k)
      for (int c = 0; c < 2 * n; ++c) std::swap(M[(size_t)k * 2 * n + c], M[(size_t)piv * 2 * n + c]);
    for (int c = 0; c < 2 * n; ++c) M[(size_t)k * 2 * n + c] /= pv;
    for (int r = 0; r < n; ++r) {
      if (r == k) continue;
      const double f = M[(size_t)r * 2 * n + k];
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * n; ++c) M[(size_t)r * 2 * n + c] -= f * M[(size_t)k * 2 * n + c];
    }
  }
  T.assign((size_t)n * n, 0.0);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) T[(size_t)c * n + r] = M[(size_t)r * 2 * n + n + c];
  return true;
}

// Mixed precision, vector equations: the coarsest correction equation is
// solved exactly (FP64) with the inverse of the coarsest operator, built
// once per boundary rule before the first cycle (outside graph capture).
// Coarsest levels too large, or singular operators, keep the NGS solve.
int ensure_coarse_inverse(mg_hierarchy* H, int bc) {
  if (H->cinv_state[bc] != 0) return MG_OK;
  H->cinv_state[bc] = -1;
  Level& Lc = H->L[H->nlev - 1];
  const int n = (int)(3 * Lc.cells());
  if (n > BC_CINV_MAX) return MG_OK;
  double *scratch = nullptr, *dA = nullptr;
  if (cudaMalloc(&scratch, sizeof(double) * 3 * (size_t)n * Lc.ng) != cudaSuccess ||
      cudaMalloc(&dA, sizeof(double) * (size_t)n * n) != cudaSuccess) {
    cudaFree(scratch);
    cudaFree(dA);
    cudaGetLastError();
    return MG_OK;
  }
  launch_coarse_assemble_vec(with_bc(Lc.v64, bc), scratch, dA, n, H->st);
  std::vector<double> A((size_t)n * n), T;
  cudaError_t ce = cudaMemcpyAsync(A.data(), dA, sizeof(double) * A.size(), cudaMemcpyDeviceToHost, H->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(H->st);
  cudaFree(scratch);
  cudaFree(dA);
  if (ce != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(ce));
  if (!invert_dense(n, A, T)) return MG_OK;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * T.size()) != cudaSuccess) {
    cudaGetLastError();
    return MG_OK;
  }
  ce = cudaMemcpyAsync(d, T.data(), sizeof(double) * T.size(), cudaMemcpyHostToDevice, H->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(H->st);
  if (ce != cudaSuccess) {
    cudaFree(d);
    return fail(MG_ERR_CUDA, cudaGetErrorString(ce));
  }
  H->cinv[bc] = d;
  H->cinv_state[bc] = 1;
  return MG_OK;
}

// Mixed precision, scalar equations: the coarsest operator as dense rows
// (its boundary rule folded in), assembled once per boundary rule before the
// first cycle (outside graph capture), for the one-block cycle's coarsest
// sweeps.  Coarsest levels of more than BC_CMAT_MAX cells keep the stencil
// sweeps.
int ensure_coarse_matrix(mg_hierarchy* H, int bc) {
  if (H->cmat_state[bc] != 0) return MG_OK;
  H->cmat_state[bc] = -1;
  Level& Lc = H->L[H->nlev - 1];
  const int n = (int)Lc.cells();
  if (n > BC_CMAT_MAX) return MG_OK;
  double *scratch = nullptr, *dA = nullptr;
  if (cudaMalloc(&scratch, sizeof(double) * (size_t)n * Lc.ng) != cudaSuccess ||
      cudaMalloc(&dA, sizeof(double) * (size_t)n * n) != cudaSuccess) {
    cudaFree(scratch);
    cudaFree(dA);
    cudaGetLastError();
    return MG_OK;
  }
  launch_coarse_assemble_scalar(with_bc(Lc.v64, bc), scratch, dA, n, H->st);
  const cudaError_t ce = cudaStreamSynchronize(H->st);
  cudaFree(scratch);
  if (ce != cudaSuccess) {
    cudaFree(dA);
    return fail(MG_ERR_CUDA, cudaGetErrorString(ce));
  }
  H->cmat[bc] = dA;
  H->cmat_state[bc] = 1;
  return MG_OK;
}

// Ghost-push tables (GhostPush) of the vector colour passes with Dirichlet-0
// ghosts, for every level below the coarsest, built once per hierarchy
// before its first vector solve (outside graph capture).  The sources come
// from the device's own ghost rules.  A level and component keep the
// ghost-fill launch when a ghost is not plus or minus one interior cell, or
// when a cell of the pass that updates a ghost's source reads that ghost
// (as a face neighbour; a component's own stencil reaches no further) from
// another block.
int ensure_ghost_push(mg_hierarchy* H) {
  if (H->push_state != 0) return MG_OK;
  H->push_state = -1;
  const int nl = H->nlev - 1;
  if (nl <= 0) return MG_OK;
  long gmax = 0;
  for (int l = 0; l < nl; ++l) gmax = std::max(gmax, ghost_count_host(H->L[l].v64));
  int* dgc = nullptr;
  double* dfac = nullptr;
  if (cudaMalloc(&dgc, sizeof(int) * 8 * 3 * (size_t)gmax) != cudaSuccess ||
      cudaMalloc(&dfac, sizeof(double) * 3 * (size_t)gmax) != cudaSuccess) {
    cudaFree(dgc);
    cudaFree(dfac);
    cudaGetLastError();
    return MG_OK;
  }
  std::vector<int> gc(8 * 3 * (size_t)gmax);
  std::vector<double> fac(3 * (size_t)gmax);
  std::vector<int> buf;  // per (level, component, colour): off[nb + 1], then 2 ints per entry
  struct Where {
    long off, ent;
  };
  std::vector<Where> at((size_t)nl * 6, Where{-1, -1});
  cudaError_t ce = cudaSuccess;
  for (int l = 0; l < nl && ce == cudaSuccess; ++l) {
    const LevelView<double> v = with_bc(H->L[l].v64, MG_BC_DIRICHLET);
    const long ng = ghost_count_host(v);
    for (int c = 0; c < 3; ++c) launch_ghost_sources(v, c, dgc + 8 * c * ng, dfac + c * ng, H->st);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(gc.data(), dgc, sizeof(int) * 8 * 3 * ng, cudaMemcpyDeviceToHost, H->st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(fac.data(), dfac, sizeof(double) * 3 * ng, cudaMemcpyDeviceToHost, H->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(H->st);
    if (ce != cudaSuccess) break;
    const int n0 = v.n0, n1 = v.n1, n2 = v.three ? v.n2 : 1;
    const long ncell = H->L[l].ng;  // cells of the level array, ghosts and padding included
    const int nb = push_blocks(v);
    auto interior = [&](int i, int j, int k) { return i >= 0 && i < n0 && j >= 0 && j < n1 && k >= 0 && k < n2; };
    for (int c = 0; c < 3; ++c) {
      const int* G = gc.data() + 8 * c * ng;
      const double* F = fac.data() + c * ng;
      std::vector<int> blk(ng), slot(ng), col(ng);
      bool ok = true;
      for (long g = 0; g < ng && ok; ++g) {
        const int* o = G + 8 * g;
        if (interior(o[0], o[1], o[2]) || !interior(o[3], o[4], o[5]) || (F[g] != 1.0 && F[g] != -1.0) ||
            o[6] < 0 || o[6] >= ncell || o[7] < 0 || o[7] >= ncell) {
          ok = false;
          break;
        }
        push_slot(v, o[3], o[4], o[5], &blk[g], &slot[g]);
        col[g] = (o[3] + o[4] + o[5]) & 1;
        if (blk[g] < 0 || blk[g] >= nb || slot[g] < 0 || slot[g] >= 256 * vec_cells_per_thread(v)) ok = false;
        // face neighbours of the ghost updated in the same pass as its source
        for (int d = 0; d < (v.three ? 3 : 2) && ok; ++d)
          for (int s = -1; s <= 1 && ok; s += 2) {
            const int r[3] = {o[0] + (d == 0) * s, o[1] + (d == 1) * s, o[2] + (d == 2) * s};
            if (!interior(r[0], r[1], r[2]) || ((r[0] + r[1] + r[2]) & 1) != col[g]) continue;
            if (r[0] == o[3] && r[1] == o[4] && r[2] == o[5]) continue;
            int rb, rt;
            push_slot(v, r[0], r[1], r[2], &rb, &rt);
            if (rb != blk[g]) ok = false;
          }
      }
      if (!ok) continue;
      for (int colour = 0; colour < 2; ++colour) {
        Where w;
        w.off = (long)buf.size();
        buf.resize(buf.size() + nb + 1, 0);
        if (buf.size() & 1) buf.push_back(0);  // entries 8-byte aligned
        w.ent = (long)buf.size();
        long cnt = 0;
        for (long g = 0; g < ng; ++g) cnt += col[g] == colour;
        buf.resize(buf.size() + 2 * cnt);
        int* offp = buf.data() + w.off;  // after the last resize
        for (long g = 0; g < ng; ++g)
          if (col[g] == colour) offp[blk[g] + 1] += 1;
        for (int b = 0; b < nb; ++b) offp[b + 1] += offp[b];
        std::vector<int> fillp(offp, offp + nb);
        for (long g = 0; g < ng; ++g) {
          if (col[g] != colour) continue;
          int* q = buf.data() + w.ent + 2 * (long)(fillp[blk[g]]++);
          q[0] = G[8 * g + 6];
          q[1] = 2 * slot[g] + (F[g] < 0.0 ? 1 : 0);
        }
        at[(size_t)(l * 3 + c) * 2 + colour] = w;
      }
    }
  }
  cudaFree(dgc);
  cudaFree(dfac);
  if (ce != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(ce));
  if (buf.empty()) return MG_OK;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int) * buf.size()) != cudaSuccess) {
    cudaGetLastError();
    return MG_OK;
  }
  ce = cudaMemcpyAsync(d, buf.data(), sizeof(int) * buf.size(), cudaMemcpyHostToDevice, H->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(H->st);
  if (ce != cudaSuccess) {
    cudaFree(d);
    return fail(MG_ERR_CUDA, cudaGetErrorString(ce));
  }
  H->push_buf = d;
  for (int l = 0; l < nl; ++l)
    for (int c = 0; c < 3; ++c)
      for (int colour = 0; colour < 2; ++colour) {
        const Where w = at[(size_t)(l * 3 + c) * 2 + colour];
        if (w.off < 0) continue;
        H->L[l].push[c][colour].off = d + w.off;
        H->L[l].push[c][colour].ent = reinterpret_cast<const int2*>(d + w.ent);
      }
  H->push_state = 1;
  return MG_OK;
}

// The whole cycle loop of one equation as one graph launch: the initial
// residual, then a while node whose body is one cycle (the cycle map, the
// mixing step, the residual and k_loop_decide, which applies the stopping
// rule on the device and sets the node's condition).  No host round trip
// per cycle; the host reads the loop state once at the end.  Returns
// LOOP_UNSUPPORTED (nothing enqueued) when the graph cannot be built.
constexpr int LOOP_UNSUPPORTED = -1;

int build_loop_graph(mg_hierarchy* H, const Eq& e, int key, double* ax, double* afp, double* agp, double* adF,
                     double* adG, float* adF32, float* adG32) {
  const mg_grid_desc& d = H->d;
  const bool mixed = d.precision == MG_MIXED;
  Level& L0 = H->L[0];
  const int m = d.accel_depth;
  const long stride = L0.ng;
  cudaGraph_t top = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle hc;
  if (cudaGraphCreate(&top, 0) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&hc, top, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGetLastError();
    if (top) cudaGraphDestroy(top);
    return LOOP_UNSUPPORTED;
  }
  const LoopParams P{d.tol, d.max_cycles, d.stall_window, m};
  const int64_t u0 = H->updates;
  // The kernels are captured straight into the graph and into the while
  // node's body (no child-graph nodes), so the programmatic edges between
  // consecutive kernels stay.
  auto abort_capture = [&]() {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(H->st, &g);
    cudaGetLastError();
    cudaGraphDestroy(top);
  };
  // before the loop: the mixing's starting iterate, the initial residual,
  // the first decision; then the while node after them
  const unsigned long long l0 = launch_count();
  if (cudaStreamBeginCaptureToGraph(H->st, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(top);
    return LOOP_UNSUPPORTED;
  }
  if (m > 0)
    for (int c = 0; c < e.ncomp; ++c)
      cudaMemcpyAsync(ax + (long)c * stride, L0.u[c], sizeof(double) * L0.ng, cudaMemcpyDeviceToDevice, H->st);
  int st = finest_residual(H, e);
  launch_loop_decide(H->d_loop, H->d_red, P, hc, 1, H->st);
  const unsigned long long lpre = launch_count() - l0;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphNode_t ncond;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (st || cudaStreamGetCaptureInfo(H->st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps) != cudaSuccess ||
      cudaGraphAddNode(&ncond, top, deps, nullptr, ndeps, &cp) != cudaSuccess ||
      cudaStreamUpdateCaptureDependencies(H->st, &ncond, nullptr, 1, cudaStreamSetCaptureDependencies) !=
          cudaSuccess) {
    abort_capture();
    count_launch(-(int)lpre);
    return st ? st : LOOP_UNSUPPORTED;
  }
  cudaGraph_t done = nullptr;
  if (cudaStreamEndCapture(H->st, &done) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(top);
    count_launch(-(int)lpre);
    return LOOP_UNSUPPORTED;
  }
  // one cycle, captured into the body of the while node
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const unsigned long long l1 = launch_count();
  const int64_t u1 = H->updates;
  if (cudaStreamBeginCaptureToGraph(H->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(top);
    count_launch(-(int)lpre);
    return LOOP_UNSUPPORTED;
  }
  st = cycle_map(H, e);
  if (m > 0) {
    const AACols none{};
    const AACols* dc = &H->d_loop->cols;
    double* scr = H->d_aa_part;
    if (mixed) {
      launch_aa_update_dots<float>(L0.v64, e.ncomp, stride, L0.u, ax, afp, agp, adF32, adG32, none, scr,
                                   H->d_red + 3, H->st, dc);
      launch_aa_combine<float>(L0.v64, e.ncomp, stride, L0.u, ax, adG32, none, scr, H->d_red + 3, H->st, dc);
    } else {
      launch_aa_update_dots<double>(L0.v64, e.ncomp, stride, L0.u, ax, afp, agp, adF, adG, none, scr, H->d_red + 3,
                                    H->st, dc);
      launch_aa_combine<double>(L0.v64, e.ncomp, stride, L0.u, ax, adG, none, scr, H->d_red + 3, H->st, dc);
    }
    if (e.kind == EQ_VEC) fill_all64(H, e, 0);
  }
  if (!st) st = finest_residual(H, e);
  launch_loop_decide(H->d_loop, H->d_red, P, hc, 0, H->st);
  cudaGraph_t body_out = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(H->st, &body_out);
  const unsigned long long lbody = launch_count() - l1;
  const int64_t ubody = H->updates - u1;
  H->updates = u0;
  count_launch(-(int)(lpre + lbody));  // counted per run below
  if (st || ce != cudaSuccess || cudaGraphInstantiate(&exec, top, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(top);
    return st ? st : LOOP_UNSUPPORTED;
  }
  cudaGraphDestroy(top);
  H->loops.push_back(mg_hierarchy::LoopGraph{key, exec, ubody, lpre, lbody});
  return MG_OK;
}

int run_loop_graph(mg_hierarchy* H, const Eq& e, double* ax, double* afp, double* agp, double* adF, double* adG,
                   float* adF32, float* adG32, mg_solve_report* rep, std::chrono::steady_clock::time_point t0) {
  if (!H->d_loop) {
    if (cudaMalloc(&H->d_loop, sizeof(LoopState)) != cudaSuccess) {
      H->d_loop = nullptr;
      return fail(MG_ERR_OOM, "loop state allocation failed");
    }
    if (cudaMallocHost(&H->h_loop, sizeof(LoopState)) != cudaSuccess) {
      H->h_loop = nullptr;
      return fail(MG_ERR_OOM, "pinned loop state allocation failed");
    }
  }
  const int key = e.kind | (e.bc << 2) | (e.zero_mean << 4) | ((int)e.has_c << 5) | (H->d.precision << 6);
  const mg_hierarchy::LoopGraph* g = nullptr;
  for (const auto& q : H->loops)
    if (q.key == key) g = &q;
  if (!g) {
    const int st = build_loop_graph(H, e, key, ax, afp, agp, adF, adG, adF32, adG32);
    if (st) return st;
    g = &H->loops.back();
  }
  CK(cudaGraphLaunch(g->exec, H->st));
  CK(cudaMemcpyAsync(H->h_loop, H->d_loop, sizeof(LoopState), cudaMemcpyDeviceToHost, H->st));
  CK(cudaStreamSynchronize(H->st));
  const LoopState& S = *H->h_loop;
  const int cyc = S.cyc;
  H->updates += (int64_t)cyc * g->updates;
  count_launch((int)(g->launches_pre + (uint64_t)cyc * g->launches));
  auto t1 = std::chrono::steady_clock::now();
  if (rep) {
    rep->status = S.status;
    rep->cycles = cyc;
    rep->rel = S.rel;
    rep->nhist = std::min(cyc + 1, (int)MG_HIST);
    for (int q = 0; q < rep->nhist; ++q) rep->hist[q] = S.hist[q];
    rep->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    rep->cell_updates = H->updates;
  }
  return S.status;
}

int run_solve_body(mg_hierarchy* H, const Eq& e, mg_solve_report* rep);

// A solve, then the timeout flag of the tensor-map staged sweeps (set when a
// block gave up waiting for a staged plane and stopped early).
int run_solve(mg_hierarchy* H, const Eq& e, mg_solve_report* rep) {
  const int st = run_solve_body(H, e, rep);
  if (H->maps_on) {
    unsigned long long flag = 0;
    CK(cudaMemcpyAsync(&flag, H->d_red + 7, sizeof(flag), cudaMemcpyDeviceToHost, H->st));
    CK(cudaStreamSynchronize(H->st));
    if (flag) {
      CK(cudaMemsetAsync(H->d_red + 7, 0, sizeof(flag), H->st));
      return fail(MG_ERR_CUDA, "one-launch sweep: a staged plane did not arrive");
    }
  }
  return st;
}

int run_solve_body(mg_hierarchy* H, const Eq& e, mg_solve_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  H->updates = 0;
  const mg_grid_desc& d = H->d;
  const bool mixed = d.precision == MG_MIXED;
  Level& L0 = H->L[0];
  const int m = d.accel_depth;
  if (mixed && e.kind == EQ_VEC)
    if (int est = ensure_coarse_inverse(H, e.bc)) return est;
  if (mixed && e.kind != EQ_VEC)
    if (int est = ensure_coarse_matrix(H, e.bc)) return est;
  if (e.kind == EQ_VEC && e.bc == MG_BC_DIRICHLET)
    if (int est = ensure_ghost_push(H)) return est;
  if (e.kind == EQ_VEC) fill_all64(H, e, 0);
  restrict_sources(H, e);
  if (mixed && e.kind == EQ_LIN && e.has_c) {
    launch_convert<double, float>(L0.v64, L0.s1, L0.k32, H->st);
    restrict_k32(H, 1);
  }
  int st = MG_OK;
  // mixing state
  const long stride = L0.ng, vlen = (long)e.ncomp * L0.ng;
  // history columns in FP32 in mixed precision (mg_accel.cu)
  double *ax = nullptr, *afp = nullptr, *agp = nullptr, *adF = nullptr, *adG = nullptr;
  float *adF32 = nullptr, *adG32 = nullptr;
  int ncol = 0, head = 0;
  if (m > 0) {
    if ((st = ensure_aa(H, e.ncomp, m, mixed ? sizeof(float) : sizeof(double)))) return st;
    ax = H->aa;
    afp = ax + vlen;
    agp = afp + vlen;
    if (mixed) {
      adF32 = reinterpret_cast<float*>(agp + vlen);
      adG32 = adF32 + (long)m * vlen;
    } else {
      adF = agp + vlen;
      adG = adF + (long)m * vlen;
    }
  }
  if (!H->prof_on && !H->loop_off) {
    st = run_loop_graph(H, e, ax, afp, agp, adF, adG, adF32, adG32, rep, t0);
    if (st != LOOP_UNSUPPORTED) return st;
    H->loop_off = true;  // no graphs with while nodes here: the host loop from now on
  }
  std::vector<double> hist;
  double rel;
  st = finest_norm(H, e, &rel);
  if (st) return st;
  hist.push_back(rel);
  int cyc = 0, status = MG_OK;
  for (;;) {
    if (std::isnan(rel)) {
      status = MG_ERR_NAN;
      break;
    }
    if (rel <= d.tol) break;
    if (cyc >= d.max_cycles) {
      status = MG_ERR_NOCONV;
      break;
    }
    if (d.stall_window > 0 && cyc >= d.stall_window && rel > 0.95 * hist[cyc - d.stall_window]) {
      status = MG_ERR_STALLED;
      break;
    }
    // x holds the iterate the cycle starts from: copied once, then kept by
    // the mixing kernels
    if (m > 0 && cyc == 0)
      for (int c = 0; c < e.ncomp; ++c)
        CK(cudaMemcpyAsync(ax + (long)c * stride, L0.u[c], sizeof(double) * L0.ng, cudaMemcpyDeviceToDevice,
                           H->st));
    if ((st = run_cycle_map(H, e))) return st;
    bool mixed_step = false;
    if (m > 0) {
      // dF, dG of this cycle go to ring slot head (none on the first cycle)
      AACols cols{};
      if (cyc > 0) {
        const int slot = head;
        head = (head + 1) % m;
        if (ncol < m) ++ncol;
        cols.n = ncol;
        for (int a = 0; a < ncol; ++a) cols.slot[a] = (slot - ncol + 1 + a + m) % m;  // oldest first
      }
      double* scr = H->d_aa_part;
      const int64_t nval = L0.cells() * e.ncomp;
      long tok = prof_begin(H, 0, MG_PROF_AA_UPDATE, nval);
      if (mixed)
        launch_aa_update_dots<float>(L0.v64, e.ncomp, stride, L0.u, ax, afp, agp, adF32, adG32, cols, scr,
                                     H->d_red + 3, H->st);
      else
        launch_aa_update_dots<double>(L0.v64, e.ncomp, stride, L0.u, ax, afp, agp, adF, adG, cols, scr,
                                      H->d_red + 3, H->st);
      prof_end(H, tok);
      if (cols.n > 0) {
        tok = prof_begin(H, 0, MG_PROF_AA_COMBINE, nval);
        if (mixed)
          launch_aa_combine<float>(L0.v64, e.ncomp, stride, L0.u, ax, adG32, cols, scr, H->d_red + 3, H->st);
        else
          launch_aa_combine<double>(L0.v64, e.ncomp, stride, L0.u, ax, adG, cols, scr, H->d_red + 3, H->st);
        prof_end(H, tok);
        if (e.kind == EQ_VEC) fill_all64(H, e, 0);
        mixed_step = true;
      }
    }
    ++cyc;
    st = finest_norm(H, e, &rel);
    if (st) return st;
    if (mixed_step && H->h_red[3] != 0) ncol = 0;  // degenerate history: restart the mixing
    hist.push_back(rel);
  }
  CK(cudaGetLastError());
  auto t1 = std::chrono::steady_clock::now();
  if (rep) {
    rep->status = status;
    rep->cycles = cyc;
    rep->rel = rel;
    rep->nhist = (int)std::min<size_t>(hist.size(), MG_HIST);
    for (int q = 0; q < rep->nhist; ++q) rep->hist[q] = hist[q];
    rep->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    rep->cell_updates = H->updates;
  }
  return status;
}

// ------------------------------------------------- composite grid (AMR)

// The box of a refined patch over base cells a <= I < b, with its
// coarse-fine faces; MG_ERR_INVALID unless it lies inside the grid, every
// patch size 2 (b - a) is a power of two, and it spans the whole angular
// range where a rule across the origin or axis needs it (spherical: theta
// and phi; cylindrical 3D: phi).
int amr_box(const mg_hierarchy* H, const int a[3], const int b[3], AmrBox* out) {
  const mg_grid_desc& d = H->d;
  AmrBox box{};
  box.cf = 0;
  for (int t = 0; t < 3; ++t) {
    if (t >= d.ndim) {
      box.a[t] = 0;
      box.b[t] = 1;
      continue;
    }
    if (!(0 <= a[t] && a[t] < b[t] && b[t] <= d.n[t])) return fail(MG_ERR_INVALID, "patch box outside the grid");
    if (!pow2(2 * (b[t] - a[t]))) return fail(MG_ERR_INVALID, "patch sizes 2 (b - a) must be powers of two");
    box.a[t] = a[t];
    box.b[t] = b[t];
    if (a[t] > 0) box.cf |= 1 << (2 * t);
    if (b[t] < d.n[t]) box.cf |= 1 << (2 * t + 1);
  }
  if (d.geom == MG_SPH && (box.a[1] != 0 || box.b[1] != d.n[1]))
    return fail(MG_ERR_INVALID, "a spherical patch must span theta");
  if (d.geom != MG_CART && d.ndim == 3 && (box.a[2] != 0 || box.b[2] != d.n[2]))
    return fail(MG_ERR_INVALID, "a curvilinear 3D patch must span phi");
  *out = box;
  return MG_OK;
}

// Patch level of a box (tables, arrays, the map of the uncovered base
// cells), allocated on first use and kept while the box is the same.
int ensure_amr(mg_hierarchy* H, const AmrBox& box) {
  auto& A = H->amr;
  if (A.valid && std::memcmp(A.box.a, box.a, sizeof(box.a)) == 0 && std::memcmp(A.box.b, box.b, sizeof(box.b)) == 0)
    return MG_OK;
  CK(cudaStreamSynchronize(H->st));
  if (A.mem) cudaFree(A.mem);
  if (A.aa) cudaFree(A.aa);
  if (A.graph) cudaGraphExecDestroy(A.graph);
  A = mg_hierarchy::Amr{};
  const Level& B = H->L[0];
  const int three = H->d.ndim == 3;
  mg_grid_desc dp = H->d;
  Level Lp;
  for (int t = 0; t < 3; ++t) {
    const bool act = t < H->d.ndim;
    Lp.n[t] = act ? 2 * (box.b[t] - box.a[t]) : 1;
    Lp.h[t] = act ? 0.5 * B.h[t] : B.h[t];
    Lp.lo[t] = act ? B.lo[t] + box.a[t] * B.h[t] : B.lo[t];
    dp.n[t] = Lp.n[t];
    dp.lo[t] = Lp.lo[t];
    dp.hi[t] = act ? B.lo[t] + box.b[t] * B.h[t] : H->d.hi[t];
  }
  Lp.sx = row_stride(Lp.n[0]);
  Lp.sy = Lp.sx * (Lp.n[1] + 2);
  Lp.off = ROW_PAD + Lp.sx + three * Lp.sy;
  Lp.ng = Lp.sy * (Lp.n[2] + 2 * three);
  std::vector<double> ti, tj;
  make_tables(&dp, Lp, ti, tj);
  // uncovered base cells, interior order
  std::vector<int> bmap;
  for (int k = 0; k < B.n[2]; ++k)
    for (int j = 0; j < B.n[1]; ++j)
      for (int i = 0; i < B.n[0]; ++i) {
        const bool cov = i >= box.a[0] && i < box.b[0] && j >= box.a[1] && j < box.b[1] &&
                         (!three || (k >= box.a[2] && k < box.b[2]));
        if (!cov) bmap.push_back((int)(B.off + i + j * B.sx + (long)k * B.sy));
      }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += bytes;
    return at;
  };
  const size_t o_ti = take(sizeof(double) * ti.size()), o_tj = take(sizeof(double) * tj.size());
  size_t o_arr[5];
  for (int q = 0; q < 5; ++q) o_arr[q] = take(sizeof(double) * Lp.ng);
  const size_t o_map = take(sizeof(int) * std::max<size_t>(bmap.size(), 1));
  if (cudaMalloc(&A.mem, off) != cudaSuccess) {
    A.mem = nullptr;
    return fail(MG_ERR_OOM, "patch allocation failed");
  }
  CK(cudaMemsetAsync(A.mem, 0, off, H->st));
  A.ti = (double*)(A.mem + o_ti);
  A.tj = (double*)(A.mem + o_tj);
  double** arr[5] = {&A.u, &A.f, &A.r, &A.s0, &A.s1};
  for (int q = 0; q < 5; ++q) *arr[q] = (double*)(A.mem + o_arr[q]);
  A.bmap = (int*)(A.mem + o_map);
  CK(cudaMemcpyAsync(A.ti, ti.data(), sizeof(double) * ti.size(), cudaMemcpyHostToDevice, H->st));
  CK(cudaMemcpyAsync(A.tj, tj.data(), sizeof(double) * tj.size(), cudaMemcpyHostToDevice, H->st));
  if (!bmap.empty())
    CK(cudaMemcpyAsync(A.bmap, bmap.data(), sizeof(int) * bmap.size(), cudaMemcpyHostToDevice, H->st));
  CK(cudaStreamSynchronize(H->st));  // host tables go out of scope
  for (int t = 0; t < 3; ++t) A.n[t] = Lp.n[t];
  A.sx = Lp.sx;
  A.sy = Lp.sy;
  A.off = Lp.off;
  A.ng = Lp.ng;
  A.v = make_view<double>(&dp, Lp, A.ti, A.tj);
  A.box = box;
  A.nbase = (long)bmap.size();
  A.nvec = Lp.cells() + A.nbase;
  long nf = 4;
  int lg = 2;
  while (nf < A.nvec) nf <<= 1, ++lg;
  A.flat = LevelView<double>{};
  A.flat.n0 = (int)nf;
  A.flat.n1 = A.flat.n2 = 1;
  A.flat.three = 0;
  A.flat.sx = A.flat.sy = nf;
  A.flat.off = 0;
  A.flat.ln0 = lg;
  A.flat.ln1 = 0;
  A.valid = true;
  return MG_OK;
}

// Anderson storage of the composite iteration: g, x, fprev, gprev and 2 m
// history columns of flat.n0 doubles (zero beyond the composite unknowns).
int ensure_amr_aa(mg_hierarchy* H, int m) {
  auto& A = H->amr;
  if (A.aa && A.aa_m >= m) return MG_OK;
  if (A.aa) cudaFree(A.aa);
  A.aa = nullptr;
  const size_t bytes = sizeof(double) * (size_t)A.flat.n0 * (4 + 2 * (size_t)m);
  if (cudaMalloc(&A.aa, bytes) != cudaSuccess) {
    A.aa = nullptr;
    return fail(MG_ERR_OOM, "composite mixing storage allocation failed");
  }
  CK(cudaMemsetAsync(A.aa, 0, bytes, H->st));
  A.aa_m = m;
  if (!H->d_aa_part) {
    if (cudaMalloc(&H->d_aa_part, sizeof(double) * AA_SCRATCH_DOUBLES) != cudaSuccess) {
      H->d_aa_part = nullptr;
      return fail(MG_ERR_OOM, "mixing scratch failed");
    }
    CK(cudaMemsetAsync(H->d_aa_part, 0, sizeof(double) * AA_SCRATCH_DOUBLES, H->st));
  }
  return MG_OK;
}

// Arrays of the composite iteration on the finest base level (scalar
// equations leave components 1 and 2 free): the original right-hand side,
// the flux correction, the restricted patch residual, the base state before
// the base V-cycle and its change.
struct AmrArrays {
  double *f0, *corr, *rr, *uh, *eb;
};
AmrArrays amr_arrays(mg_hierarchy* H, const Eq& e) {
  Level& L0 = H->L[0];
  return AmrArrays{e.kind == EQ_LIN ? L0.f[1] : nullptr, L0.f[2], L0.r[1], L0.u[2], L0.r[2]};
}

// Base ghosts, patch ghosts (boundary rules, then the coarse-fine values)
// and the flux correction of the uncovered interface cells.
void amr_refresh(mg_hierarchy* H, const Eq& e, bool corr) {
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const auto vb = with_bc(L0.v64, e.bc);
  const auto vp = with_bc(A.v, e.bc);
  launch_fill_ghosts(vb, L0.u[0], -1, H->st);
  launch_fill_ghosts(vp, A.u, -1, H->st);
  launch_amr_cf_ghosts(vp, vb, A.box, A.u, L0.u[0], H->st);
  if (corr) {
    const AmrArrays W = amr_arrays(H, e);
    cudaMemsetAsync(W.corr, 0, sizeof(double) * L0.ng, H->st);
    launch_amr_flux_corr(vp, vb, A.box, A.u, L0.u[0], W.corr, H->st);
  }
}

// Relative weighted residual over the composite cells (stopping rule).
int amr_norm(mg_hierarchy* H, const Eq& e, double* rel) {
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const AmrArrays W = amr_arrays(H, e);
  amr_refresh(H, e, true);
  CK(cudaMemsetAsync(H->d_red, 0, sizeof(unsigned long long) * 3, H->st));
  const double* s0p = e.kind == EQ_PSI ? A.s0 : nullptr;
  const double* s1p = (e.kind == EQ_PSI || e.has_c) ? A.s1 : nullptr;
  launch_amr_patch_resid(with_bc(A.v, e.bc), e.kind, A.u, A.f, s0p, s1p, nullptr, H->d_red, 0, H->st);
  launch_amr_base(with_bc(L0.v64, e.bc), A.box, e.kind, L0.u[0], s0ptr(H, e, 0), s1ptr(H, e, 0), W.f0, nullptr,
                  W.corr, nullptr, H->d_red, 1, H->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(H->h_red, H->d_red, sizeof(unsigned long long) * 4, cudaMemcpyDeviceToHost, H->st));
  CK(cudaStreamSynchronize(H->st));
  const double num = bits_to_double(H->h_red[1]), den = bits_to_double(H->h_red[2]);
  if (std::isinf(num) || std::isinf(den) || std::isnan(num) || std::isnan(den))
    *rel = NAN;
  else
    *rel = num / (den > 1e-300 ? den : 1e-300);
  return MG_OK;
}

// Red-black Newton-Gauss-Seidel sweeps of the patch, its ghosts refilled
// before each colour (the base ghosts are current).
void amr_patch_sweeps(mg_hierarchy* H, const Eq& e, int nsweeps) {
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const auto vb = with_bc(L0.v64, e.bc);
  const auto vp = with_bc(A.v, e.bc);
  const double* s0p = e.kind == EQ_PSI ? A.s0 : nullptr;
  const double* s1p = (e.kind == EQ_PSI || e.has_c) ? A.s1 : nullptr;
  for (int sw = 0; sw < nsweeps; ++sw)
    for (int colour = 0; colour < 2; ++colour) {
      launch_fill_ghosts(vp, A.u, -1, H->st);
      launch_amr_cf_ghosts(vp, vb, A.box, A.u, L0.u[0], H->st);
      launch_amr_smooth(vp, e.kind, A.u, A.f, s0p, s1p, colour, H->st);
    }
  H->updates += (int64_t)nsweeps * (int64_t)A.n[0] * A.n[1] * A.n[2];
}

// One composite FAS V(nu1, nu2) cycle.
void amr_cycle(mg_hierarchy* H, const Eq& e) {
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const auto vb = with_bc(L0.v64, e.bc);
  const auto vp = with_bc(A.v, e.bc);
  const AmrArrays W = amr_arrays(H, e);
  const double* s0p = e.kind == EQ_PSI ? A.s0 : nullptr;
  const double* s1p = (e.kind == EQ_PSI || e.has_c) ? A.s1 : nullptr;
  launch_fill_ghosts(vb, L0.u[0], -1, H->st);
  amr_patch_sweeps(H, e, H->d.nu1);
  launch_fill_ghosts(vp, A.u, -1, H->st);
  launch_amr_cf_ghosts(vp, vb, A.box, A.u, L0.u[0], H->st);
  launch_amr_patch_resid(vp, e.kind, A.u, A.f, s0p, s1p, A.r, nullptr, 0, H->st);
  launch_amr_restrict(vp, vb, A.box, A.u, A.r, L0.u[0], W.rr, H->st);
  cudaMemcpyAsync(W.uh, L0.u[0], sizeof(double) * L0.ng, cudaMemcpyDeviceToDevice, H->st);
  amr_refresh(H, e, true);
  launch_amr_base(vb, A.box, e.kind, L0.u[0], s0ptr(H, e, 0), s1ptr(H, e, 0), W.f0, W.rr, W.corr, L0.f[0], nullptr,
                  0, H->st);
  vcycle64(H, e, 0);
  launch_amr_diff(vb, L0.u[0], W.uh, W.eb, H->st);
  launch_fill_ghosts(vb, W.eb, -1, H->st);  // the rules are linear: homogeneous for a change
  launch_amr_prolong(vp, vb, A.box, W.eb, A.u, H->st);
  launch_fill_ghosts(vb, L0.u[0], -1, H->st);
  amr_patch_sweeps(H, e, H->d.nu2);
}

// The composite cycle replayed from a CUDA graph captured on first use for
// the patch and the equation signature (direct launches while profiling).
int run_amr_cycle(mg_hierarchy* H, const Eq& e) {
  auto& A = H->amr;
  if (H->prof_on) {
    amr_cycle(H, e);
    return MG_OK;
  }
  const int key = e.kind | (e.bc << 2) | ((int)e.has_c << 5);
  if (A.graph && A.graph_key == key) {
    CK(cudaGraphLaunch(A.graph, H->st));
    H->updates += A.graph_updates;
    count_launch((int)A.graph_launches);
    return MG_OK;
  }
  if (A.graph) {
    cudaGraphExecDestroy(A.graph);
    A.graph = nullptr;
  }
  const int64_t u0 = H->updates;
  const unsigned long long l0 = launch_count();
  CK(cudaStreamBeginCapture(H->st, cudaStreamCaptureModeThreadLocal));
  amr_cycle(H, e);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(H->st, &graph);
  if (ce != cudaSuccess || !graph) return fail(MG_ERR_CUDA, "composite cycle capture failed");
  ce = cudaGraphInstantiate(&A.graph, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    A.graph = nullptr;
    return fail(MG_ERR_CUDA, "composite cycle instantiation failed");
  }
  A.graph_key = key;
  A.graph_updates = H->updates - u0;
  A.graph_launches = launch_count() - l0;
  CK(cudaGraphLaunch(A.graph, H->st));
  return MG_OK;
}

// Cycle control of the composite iteration, as run_solve: tol, max_cycles,
// stall window, non-finite values, Anderson mixing of depth accel_depth
// over the composite unknowns (FP64 columns).
int run_solve_amr(mg_hierarchy* H, const Eq& e, mg_solve_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const mg_grid_desc& d = H->d;
  const int m = d.accel_depth;
  H->updates = 0;
  restrict_sources(H, e);
  const long nfl = A.flat.n0;
  double *ag = nullptr, *ax = nullptr, *afp = nullptr, *agp = nullptr, *adF = nullptr, *adG = nullptr;
  if (m > 0) {
    if (int st = ensure_amr_aa(H, m)) return st;
    ag = A.aa;
    ax = ag + nfl;
    afp = ax + nfl;
    agp = afp + nfl;
    adF = agp + nfl;
    adG = adF + (long)m * nfl;
  }
  auto flat = [&](double* x, int to_flat) {
    launch_amr_flat(A.v, L0.v64, A.box, A.u, L0.u[0], A.bmap, A.nbase, x, to_flat, H->st);
  };
  std::vector<double> hist;
  double rel;
  int st = amr_norm(H, e, &rel);
  if (st) return st;
  hist.push_back(rel);
  int cyc = 0, status = MG_OK, ncol = 0, head = 0;
  for (;;) {
    if (std::isnan(rel)) {
      status = MG_ERR_NAN;
      break;
    }
    if (rel <= d.tol) break;
    if (cyc >= d.max_cycles) {
      status = MG_ERR_NOCONV;
      break;
    }
    if (d.stall_window > 0 && cyc >= d.stall_window && rel > 0.95 * hist[cyc - d.stall_window]) {
      status = MG_ERR_STALLED;
      break;
    }
    if (m > 0 && cyc == 0) flat(ax, 1);
    if ((st = run_amr_cycle(H, e))) return st;
    bool mixed_step = false;
    if (m > 0) {
      flat(ag, 1);
      AACols cols{};
      if (cyc > 0) {
        const int slot = head;
        head = (head + 1) % m;
        if (ncol < m) ++ncol;
        cols.n = ncol;
        for (int a = 0; a < ncol; ++a) cols.slot[a] = (slot - ncol + 1 + a + m) % m;
      }
      double* const g3[3] = {ag, ag, ag};
      launch_aa_update_dots<double>(A.flat, 1, nfl, g3, ax, afp, agp, adF, adG, cols, H->d_aa_part, H->d_red + 3,
                                    H->st);
      if (cols.n > 0) {
        launch_aa_combine<double>(A.flat, 1, nfl, g3, ax, adG, cols, H->d_aa_part, H->d_red + 3, H->st);
        flat(ag, 0);
        mixed_step = true;
      }
    }
    ++cyc;
    if ((st = amr_norm(H, e, &rel))) return st;
    if (mixed_step && H->h_red[3] != 0) ncol = 0;
    hist.push_back(rel);
  }
  CK(cudaGetLastError());
  auto t1 = std::chrono::steady_clock::now();
  if (rep) {
    rep->status = status;
    rep->cycles = cyc;
    rep->rel = rel;
    rep->nhist = (int)std::min<size_t>(hist.size(), MG_HIST);
    for (int q = 0; q < rep->nhist; ++q) rep->hist[q] = hist[q];
    rep->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    rep->cell_updates = H->updates;
  }
  return status;
}

// ------------------------------------------------------------ staging

long interior_cells(const mg_hierarchy* H) { return H->L[0].cells(); }

int stage_get(mg_hierarchy* H, int slot, double** out) {
  while ((int)H->stage.size() <= slot) H->stage.push_back(nullptr);
  if (!H->stage[slot]) {
    double* p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * interior_cells(H)) != cudaSuccess)
      return fail(MG_ERR_OOM, "staging allocation failed");
    H->stage[slot] = p;
  }
  *out = H->stage[slot];
  return MG_OK;
}

// Host -> staged device copy (src may be null: the slot is left alone).
int stage_in(mg_hierarchy* H, int slot, const double* host, double** dev) {
  if (!host) {
    *dev = nullptr;
    return MG_OK;
  }
  int st = stage_get(H, slot, dev);
  if (st) return st;
  CK(cudaMemcpyAsync(*dev, host, sizeof(double) * interior_cells(H), cudaMemcpyHostToDevice, H->st));
  return MG_OK;
}
int stage_out(mg_hierarchy* H, const double* dev, double* host) {
  if (!host) return MG_OK;
  CK(cudaMemcpyAsync(host, dev, sizeof(double) * interior_cells(H), cudaMemcpyDeviceToHost, H->st));
  return MG_OK;
}

// Order the hierarchy's own stream after the work the caller queued on its
// stream (every entry point that enqueues work calls this first).
int enter(mg_hierarchy* H) {
  if (!H->own_stream) return MG_OK;
  CK(cudaEventRecord(H->ev_in, H->user_st));
  CK(cudaStreamWaitEvent(H->st, H->ev_in, 0));
  return MG_OK;
}

void copy_in(mg_hierarchy* H, const double* src, double* dst, double shift = 0.0) {
  launch_copy_in<double, double>(H->L[0].v64, src, dst, shift, H->st);
}
void copy_out(mg_hierarchy* H, const double* src, double* dst, double shift = 0.0) {
  launch_copy_out<double, double>(H->L[0].v64, src, dst, shift, H->st);
}

}  // namespace

int gmg::set_last_error(int status, const char* msg) { return fail(status, msg); }

void gmg::hier_set_host_loop(mg_hierarchy* H, bool on) {
  H->loop_off = on;
  if (H->sub) H->sub->loop_off = on;
}

void gmg::hier_set_stream(mg_hierarchy* H, cudaStream_t st) {
  if (H->own_stream || st == nullptr) return;
  H->st = st;
  if (H->sub) H->sub->st = st;
}

// ================================================================== C ABI

extern "C" {

const char* mg_strerror(int s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID: return "invalid argument";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_NOCONV: return "not converged";
    case MG_ERR_STALLED: return "stalled";
    case MG_ERR_NAN: return "non-finite value";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_BUSY: return "busy";
    case MG_ERR_NOTFOUND: return "not found";
    default: return "unknown status";
  }
}

const char* mg_last_error(void) { return g_last_error; }

int mg_hierarchy_bytes(const mg_grid_desc* desc, size_t* bytes) {
  int st = validate(desc);
  if (st) return st;
  if (!bytes) return fail(MG_ERR_INVALID, "null output");
  *bytes = layout(nullptr, desc, nullptr);
  if (desc->divb_variant == MG_DIVB_EXACT) {
    const mg_grid_desc c = class_desc(desc);
    *bytes += layout(nullptr, &c, nullptr);
  }
  return MG_OK;
}

int mg_create_hierarchy(const mg_grid_desc* desc, void* cuda_stream, mg_hierarchy** out) {
  int st = validate(desc);
  if (st) return st;
  if (!out) return fail(MG_ERR_INVALID, "null output");
  mg_hierarchy* H = new (std::nothrow) mg_hierarchy();
  if (!H) return fail(MG_ERR_OOM, "host allocation failed");
  H->d = *desc;
  if (H->d.ndim == 2) {
    H->d.n[2] = 1;
    H->d.lo[2] = 0.0;
    H->d.hi[2] = 1.0;
  }
  H->st = (cudaStream_t)cuda_stream;
  if (H->st == nullptr || H->st == cudaStreamLegacy || H->st == cudaStreamPerThread) {
    // the default streams cannot be captured into CUDA graphs: work runs on
    // an owned non-blocking stream that each call orders after the caller's
    // stream with an event (a blocking stream would tie the legacy stream to
    // our captures)
    H->user_st = H->st;
    if (cudaStreamCreateWithFlags(&H->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&H->ev_in, cudaEventDisableTiming) != cudaSuccess) {
      delete H;
      return fail(MG_ERR_CUDA, "stream creation failed");
    }
    H->own_stream = true;
  }
  int n[MAX_LEVELS][3];
  double h[MAX_LEVELS][3];
  H->nlev = level_sizes(&H->d, n, h);
  const size_t bytes = layout(nullptr, &H->d, nullptr);
  if (cudaMalloc(&H->arena, bytes) != cudaSuccess) {
    H->arena = nullptr;
    mg_destroy_hierarchy(H);
    return fail(MG_ERR_OOM, "arena allocation failed");
  }
  H->arena_bytes = bytes;
  layout(H, &H->d, H->arena);
  if (cudaMallocHost(&H->h_red, sizeof(unsigned long long) * 8) != cudaSuccess) {
    H->h_red = nullptr;
    mg_destroy_hierarchy(H);
    return fail(MG_ERR_OOM, "pinned allocation failed");
  }
  cudaMemsetAsync(H->arena, 0, bytes, H->st);
  init_fused_sweep_attributes<double>();
  init_fused_sweep_attributes<float>();
  init_block_cycle_attributes();
  const int three = H->d.ndim == 3;
  for (int l = 0; l < H->nlev; ++l) {
    Level& L = H->L[l];
    for (int k = 0; k < 3; ++k) {
      L.n[k] = n[l][k];
      L.h[k] = h[l][k];
      L.lo[k] = H->d.lo[k];
    }
    L.sx = row_stride(L.n[0]);
    L.sy = L.sx * (L.n[1] + 2);
    L.off = ROW_PAD + L.sx + three * L.sy;
    L.ng = L.sy * (L.n[2] + 2 * three);
    std::vector<double> ti, tj;
    make_tables(&H->d, L, ti, tj);
    std::vector<float> ti32(ti.begin(), ti.end()), tj32(tj.begin(), tj.end());
    cudaError_t ce = cudaMemcpyAsync(L.ti64, ti.data(), sizeof(double) * ti.size(), cudaMemcpyHostToDevice, H->st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(L.tj64, tj.data(), sizeof(double) * tj.size(), cudaMemcpyHostToDevice, H->st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(L.ti32, ti32.data(), sizeof(float) * ti32.size(), cudaMemcpyHostToDevice, H->st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(L.tj32, tj32.data(), sizeof(float) * tj32.size(), cudaMemcpyHostToDevice, H->st);
    std::vector<double> vc;
    std::vector<float> vc32;
    if (L.vc64) {
      make_vec_coeffs(&H->d, L, ti, tj, vc);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(L.vc64, vc.data(), sizeof(double) * vc.size(), cudaMemcpyHostToDevice, H->st);
      if (L.vc32) {
        vc32.assign(vc.begin(), vc.end());
        if (ce == cudaSuccess)
          ce = cudaMemcpyAsync(L.vc32, vc32.data(), sizeof(float) * vc32.size(), cudaMemcpyHostToDevice, H->st);
      }
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(H->st);  // host tables go out of scope
    if (ce != cudaSuccess) {
      mg_destroy_hierarchy(H);
      std::snprintf(g_last_error, sizeof(g_last_error), "table upload: %s", cudaGetErrorString(ce));
      return MG_ERR_CUDA;
    }
    L.v64 = make_view<double>(&H->d, L, L.ti64, L.tj64);
    L.v64.vc = L.vc64;
    L.v32 = make_view<float>(&H->d, L, L.ti32, L.tj32);
    L.v32.vc = L.vc32;
    if (H->d.precision == MG_MIXED && sweep_uses_maps(L.v32)) {
      bool ok = true;
      for (int leg = 0; leg < 2; ++leg) {
        SweepMaps& m = L.sweep_maps[leg];
        std::memset(&m, 0, sizeof(m));
        ok = ok && sweep_plane_map(&m.u, L.e[leg], L.v32) && sweep_plane_map(&m.f, L.f32[0], L.v32) &&
             (!L.k32 || sweep_plane_map(&m.c, L.k32, L.v32));
        m.err = H->d_red + 7;
        m.on = 1;
      }
      L.maps_on = ok;
      H->maps_on = H->maps_on || ok;
    }
  }
  if (H->d.divb_variant == MG_DIVB_EXACT) {
    const mg_grid_desc c = class_desc(&H->d);
    const int sst = mg_create_hierarchy(&c, (void*)H->st, &H->sub);
    if (sst != MG_OK) {
      H->sub = nullptr;
      mg_destroy_hierarchy(H);
      return sst;
    }
  }
  *out = H;
  return MG_OK;
}

uint64_t mg_kernel_launches(void) { return (uint64_t)launch_count(); }

int mg_profile_enable(mg_hierarchy* H, int enable) {
  if (!H) return fail(MG_ERR_INVALID, "null hierarchy");
  CK(cudaStreamSynchronize(H->st));
  H->prof_on = enable != 0;
  H->ev_used = 0;
  return MG_OK;
}

int mg_profile_read(mg_hierarchy* H, int klass, int64_t* launches, double* ms, int64_t* cells) {
  if (!H || !launches || !ms || !cells || klass < 0 || klass >= MG_PROF_NCLASS)
    return fail(MG_ERR_INVALID, "bad argument");
  CK(cudaStreamSynchronize(H->st));
  int64_t n = 0, c = 0;
  double t = 0.0;
  for (size_t pr = 0; pr < H->ev_used / 2; ++pr) {
    if (H->ev_cls[pr] != klass) continue;
    float m = 0.f;
    CK(cudaEventElapsedTime(&m, H->ev[2 * pr], H->ev[2 * pr + 1]));
    ++n;
    c += H->ev_cells[pr];
    t += m;
  }
  *launches = n;
  *ms = t;
  *cells = c;
  return MG_OK;
}

int mg_destroy_hierarchy(mg_hierarchy* H) {
  if (!H) return MG_OK;
  if (H->st) cudaStreamSynchronize(H->st);
  if (H->sub) mg_destroy_hierarchy(H->sub);
  if (H->amr.mem) cudaFree(H->amr.mem);
  if (H->amr.aa) cudaFree(H->amr.aa);
  if (H->amr.graph) cudaGraphExecDestroy(H->amr.graph);
  for (cudaEvent_t e : H->ev) cudaEventDestroy(e);
  for (double* p : H->stage) cudaFree(p);
  if (H->aa) cudaFree(H->aa);
  for (double* p : H->cinv)
    if (p) cudaFree(p);
  for (double* p : H->cmat)
    if (p) cudaFree(p);
  if (H->d_aa_part) cudaFree(H->d_aa_part);
  if (H->batch_mem) cudaFree(H->batch_mem);
  for (cudaEvent_t e : H->b_ev)
    if (e) cudaEventDestroy(e);
  if (H->push_buf) cudaFree(H->push_buf);
  for (GraphEntry& g : H->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : H->loops) cudaGraphExecDestroy(g.exec);
  if (H->d_loop) cudaFree(H->d_loop);
  if (H->h_loop) cudaFreeHost(H->h_loop);
  if (H->own_stream) cudaStreamDestroy(H->st);
  if (H->ev_in) cudaEventDestroy(H->ev_in);
  cudaFree(H->arena);
  cudaFreeHost(H->h_red);
  delete H;
  return MG_OK;
}

int mg_num_levels(const mg_hierarchy* H, int* nlev) {
  if (!H || !nlev) return fail(MG_ERR_INVALID, "null argument");
  *nlev = H->nlev;
  return MG_OK;
}

int mg_solve_scalar(mg_hierarchy* H, int kind, int bc, int zero_mean, const double* U, const double* A2,
                    const double* c, const double* f, double* u, mg_solve_report* rep) {
  if (!H || !u) return fail(MG_ERR_INVALID, "null argument");
  if (kind != MG_EQ_PSI && kind != MG_EQ_LIN) return fail(MG_ERR_INVALID, "bad equation kind");
  if (bc < MG_BC_ROBIN || bc > MG_BC_NEUMANN) return fail(MG_ERR_INVALID, "bad boundary condition");
  if (kind == MG_EQ_PSI && (!U || !A2)) return fail(MG_ERR_INVALID, "psi equation needs U and A2");
  if (kind == MG_EQ_LIN && !f) return fail(MG_ERR_INVALID, "linear equation needs f");
  if (int est = enter(H)) return est;
  Level& L0 = H->L[0];
  Eq e{kind, bc, zero_mean ? 1 : 0, 1, kind == MG_EQ_LIN && c != nullptr};
  copy_in(H, u, L0.u[0]);
  if (kind == MG_EQ_PSI) {
    copy_in(H, U, L0.s0);
    copy_in(H, A2, L0.s1);
  } else {
    if (c) copy_in(H, c, L0.s1);
    copy_in(H, f, L0.f[0]);
  }
  int st = run_solve(H, e, rep);
  copy_out(H, L0.u[0], u);
  CK(cudaStreamSynchronize(H->st));
  return st;
}

int mg_solve_vector(mg_hierarchy* H, int bc, const double* f[3], double* V[3], mg_solve_report* rep) {
  if (!H || !f || !V) return fail(MG_ERR_INVALID, "null argument");
  for (int c = 0; c < 3; ++c)
    if (!f[c] || !V[c]) return fail(MG_ERR_INVALID, "null component");
  if (int est = enter(H)) return est;
  Level& L0 = H->L[0];
  Eq e{MG_EQ_VEC, bc, 0, 3, false};
  for (int c = 0; c < 3; ++c) {
    copy_in(H, V[c], L0.u[c]);
    copy_in(H, f[c], L0.f[c]);
  }
  int st = run_solve(H, e, rep);
  for (int c = 0; c < 3; ++c) copy_out(H, L0.u[c], V[c]);
  CK(cudaStreamSynchronize(H->st));
  return st;
}

int mg_solve_cfc(mg_hierarchy* H, const mg_cfc_sources* src, mg_cfc_fields* io, int flags, mg_cfc_report* rep) {
  if (!H || !src || !io) return fail(MG_ERR_INVALID, "null argument");
  if (int est = enter(H)) return est;
  auto t0 = std::chrono::steady_clock::now();
  const bool psi_only = flags & MG_CFC_PSI_ONLY;
  const bool host = flags & MG_HOST_POINTERS;
  if (!src->U || !io->psi) return fail(MG_ERR_INVALID, "missing U or psi");
  if (!psi_only) {
    if (!src->S || !io->alpha) return fail(MG_ERR_INVALID, "missing S or alpha");
    for (int c = 0; c < 3; ++c)
      if (!src->Si[c] || !io->beta[c] || !io->X[c]) return fail(MG_ERR_INVALID, "missing vector component");
  }
  // device views of the caller's arrays
  const double *U = src->U, *S = src->S, *Si[3] = {src->Si[0], src->Si[1], src->Si[2]};
  double *psi = io->psi, *alpha = io->alpha, *beta[3] = {io->beta[0], io->beta[1], io->beta[2]},
         *X[3] = {io->X[0], io->X[1], io->X[2]};
  int st = MG_OK;
  if (host) {
    double* dv;
    if ((st = stage_in(H, 0, src->U, &dv))) return st;
    U = dv;
    if ((st = stage_in(H, 1, io->psi, &psi))) return st;
    if (!psi_only) {
      if ((st = stage_in(H, 2, src->S, &dv))) return st;
      S = dv;
      if ((st = stage_in(H, 3, io->alpha, &alpha))) return st;
      for (int c = 0; c < 3; ++c) {
        if ((st = stage_in(H, 4 + c, src->Si[c], &dv))) return st;
        Si[c] = dv;
        if ((st = stage_in(H, 7 + c, io->beta[c], &beta[c]))) return st;
        if ((st = stage_in(H, 10 + c, io->X[c], &X[c]))) return st;
      }
    }
  }
  Level& L0 = H->L[0];
  const LevelView<double>& v = L0.v64;
  mg_solve_report* reps = rep ? rep->eq : nullptr;
  if (rep) std::memset(rep, 0, sizeof(*rep));
  const size_t b64 = sizeof(double) * L0.ng;
  copy_in(H, U, H->Ug);
  if (!psi_only) {
    copy_in(H, S, H->Sg);
    for (int c = 0; c < 3; ++c) copy_in(H, Si[c], H->Sig[c]);
    // Step 1: lap X + 1/3 grad div X = 8 pi S_i
    Eq ex{MG_EQ_VEC, MG_BC_DIRICHLET, 0, 3, false};
    for (int c = 0; c < 3; ++c) {
      copy_in(H, X[c], L0.u[c]);
      launch_scale_into(v, H->Sig[c], 8.0 * PI, L0.f[c], H->st);
    }
    st = run_solve(H, ex, reps ? &reps[0] : nullptr);
    for (int c = 0; c < 3; ++c) {
      copy_out(H, L0.u[c], X[c]);
      CK(cudaMemcpyAsync(H->Xg[c], L0.u[c], b64, cudaMemcpyDeviceToDevice, H->st));
      launch_fill_ghosts(with_bc(v, MG_BC_DIRICHLET), H->Xg[c], c, H->st);
    }
    if (st) goto out;
    // Step 2: A2 = A~_ij A~^ij (into the psi equation's s1)
    launch_xcfc_a2(v, H->Xg, L0.s1, H->st);
  } else {
    CK(cudaMemsetAsync(L0.s1, 0, b64, H->st));
  }
  {
    // Step 3: psi equation for delta = psi - 1
    Eq ep{MG_EQ_PSI, MG_BC_ROBIN, 0, 1, false};
    copy_in(H, psi, L0.u[0], -1.0);
    CK(cudaMemcpyAsync(L0.s0, H->Ug, b64, cudaMemcpyDeviceToDevice, H->st));
    st = run_solve(H, ep, reps ? &reps[1] : nullptr);
    copy_out(H, L0.u[0], psi, 1.0);
    CK(cudaMemcpyAsync(H->dpsi, L0.u[0], b64, cudaMemcpyDeviceToDevice, H->st));
    if (st || psi_only) goto out;
    // Step 5: alpha psi equation, coefficient c = 2 pi (U + 2 S) psi^-2 + 7/8 A2 psi^-8
    launch_xcfc_alpha_coef(v, H->Ug, H->Sg, L0.s1, H->dpsi, L0.f[0], H->st);
    CK(cudaMemcpyAsync(L0.s1, L0.f[0], b64, cudaMemcpyDeviceToDevice, H->st));
    launch_xcfc_ap_init(v, alpha, H->dpsi, L0.u[0], H->st);
    Eq ea{MG_EQ_LIN, MG_BC_ROBIN, 0, 1, true};
    st = run_solve(H, ea, reps ? &reps[2] : nullptr);
    CK(cudaMemcpyAsync(H->dap, L0.u[0], b64, cudaMemcpyDeviceToDevice, H->st));
    launch_xcfc_alpha_out(v, H->dap, H->dpsi, alpha, H->st);
    if (st) goto out;
    // Step 6: shift, source 16 pi alpha psi^-6 S_i + 2 A~_ij grad_j(alpha psi^-6)
    launch_fill_ghosts(with_bc(v, MG_BC_ROBIN), H->dpsi, -1, H->st);
    launch_fill_ghosts(with_bc(v, MG_BC_ROBIN), H->dap, -1, H->st);
    launch_xcfc_beta_rhs(v, H->Xg, H->dpsi, H->dap, H->sg, H->Sig, L0.f, H->st);
    Eq eb{MG_EQ_VEC, MG_BC_DIRICHLET, 0, 3, false};
    for (int c = 0; c < 3; ++c) copy_in(H, beta[c], L0.u[c]);
    st = run_solve(H, eb, reps ? &reps[3] : nullptr);
    for (int c = 0; c < 3; ++c) copy_out(H, L0.u[c], beta[c]);
  }
out:
  if (host) {
    int s2 = stage_out(H, psi, io->psi);
    if (!s2 && !psi_only) {
      s2 = stage_out(H, alpha, io->alpha);
      for (int c = 0; c < 3 && !s2; ++c) {
        s2 = stage_out(H, beta[c], io->beta[c]);
        if (!s2) s2 = stage_out(H, X[c], io->X[c]);
      }
    }
    if (s2 && !st) st = s2;
  }
  CK(cudaStreamSynchronize(H->st));
  CK(cudaGetLastError());
  if (rep) rep->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

static_assert(BATCH_HIST == MG_HIST, "batched reports keep MG_HIST residuals per equation");
constexpr int BATCH_GENERAL_THREADS = 16;

namespace {

// Device workspace of a batch of count problems, led by hierarchy H.
int ensure_batch_ws(mg_hierarchy* H, int count) {
  if (H->batch_cap >= count) return MG_OK;
  CK(cudaStreamSynchronize(H->st));
  if (H->batch_mem) cudaFree(H->batch_mem);
  H->batch_mem = nullptr;
  H->batch_cap = 0;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += bytes;
    return at;
  };
  const size_t o_items = take(sizeof(BatchItem) * count), o_outs = take(sizeof(BatchOut) * count),
               o_hist = take(sizeof(double) * 4 * BATCH_HIST * count), o_order = take(sizeof(int) * count),
               o_next = take(sizeof(unsigned int));
  if (cudaMalloc(&H->batch_mem, off) != cudaSuccess) {
    H->batch_mem = nullptr;
    return fail(MG_ERR_OOM, "batch workspace allocation failed");
  }
  H->b_items = (BatchItem*)(H->batch_mem + o_items);
  H->b_outs = (BatchOut*)(H->batch_mem + o_outs);
  H->b_hist = (double*)(H->batch_mem + o_hist);
  H->b_order = (int*)(H->batch_mem + o_order);
  H->b_next = (unsigned int*)(H->batch_mem + o_next);
  for (cudaEvent_t& e : H->b_ev)
    if (!e) CK(cudaEventCreate(&e));
  H->batch_cap = count;
  return MG_OK;
}

// Descriptor of problem (h, src, io) for the persistent launch.
int batch_item(mg_hierarchy* h, const mg_cfc_sources& src, const mg_cfc_fields& io, bool psi_only, BatchItem* B) {
  const mg_grid_desc& d = h->d;
  if (d.precision != MG_MIXED) return fail(MG_ERR_INVALID, "batched solves run in mixed precision");
  if (d.cycle != MG_CYCLE_V) return fail(MG_ERR_INVALID, "batched solves run V-cycles");
  if (d.accel_depth < 0 || d.accel_depth > AA_MAX) return fail(MG_ERR_INVALID, "accel_depth out of range");
  if (d.max_cycles >= BATCH_HIST) return fail(MG_ERR_INVALID, "batched solves take max_cycles < MG_HIST");
  if (!src.U || !io.psi) return fail(MG_ERR_INVALID, "missing U or psi");
  if (!psi_only) {
    if (!src.S || !io.alpha) return fail(MG_ERR_INVALID, "missing S or alpha");
    for (int c = 0; c < 3; ++c)
      if (!src.Si[c] || !io.beta[c] || !io.X[c]) return fail(MG_ERR_INVALID, "missing vector component");
  }
  // the first level (of at most BLOCK_CYCLE_CELLS cells) whose one-block
  // cycle fits the batch kernel's shared memory beside its static arrays
  const size_t limit = batch_smem_limit();
  auto first_fit = [&](const Eq& e, BlockCycle32* out) {
    for (int l = block_cycle_level(h, e); l < h->nlev && l <= BATCH_MAX_LEVELS; ++l) {
      const BlockCycle32 Q = block_cycle_params(h, e, l);
      if (Q.smem && Q.smem <= limit) {
        *out = Q;
        return l;
      }
    }
    return -1;
  };
  const Eq ep{MG_EQ_PSI, MG_BC_ROBIN, 0, 1, false};
  if (int est = ensure_coarse_matrix(h, MG_BC_ROBIN)) return est;
  BlockCycle32 P{};
  const int lb = first_fit(ep, &P);
  if (lb < 0) return fail(MG_ERR_INVALID, "batched solves need coarse levels that fit the one-block cycle");
  if (!P.cA) return fail(MG_ERR_INVALID, "batched solves need the dense coarsest operator (at most 64 cells)");
  // the vector equations (X, beta) in the kernel when their levels fit
  int vec_ok = 0, nlv = 0;
  BlockCycle32 Pv{};
  if (!psi_only) {
    const Eq ex{MG_EQ_VEC, MG_BC_DIRICHLET, 0, 3, false};
    if (int est = ensure_coarse_inverse(h, MG_BC_DIRICHLET)) return est;
    nlv = first_fit(ex, &Pv);
    vec_ok = nlv >= 0 && Pv.cinv;
    if (!vec_ok) nlv = 0;
  }
  const int m = d.accel_depth;
  if (m > 0)
    if (int est = ensure_aa(h, vec_ok ? 3 : 1, m, sizeof(float))) return est;
  std::memset(B, 0, sizeof(*B));
  Level& L0 = h->L[0];
  B->geom = d.geom;
  B->nl = lb;
  B->nlev = h->nlev;
  B->nu1 = d.nu1;
  B->nu2 = d.nu2;
  B->m = m;
  B->max_cycles = d.max_cycles;
  B->stall_window = d.stall_window;
  B->psi_only = psi_only ? 1 : 0;
  B->tol = d.tol;
  B->vec_ok = vec_ok;
  B->nlv = nlv;
  B->v64 = with_bc(L0.v64, MG_BC_ROBIN);
  for (int l = 0; l <= std::max(lb, vec_ok ? nlv : 0); ++l) {
    Level& L = h->L[l];
    BatchLevel& b = B->lv[l];
    b.v = with_bc(L.v32, MG_BC_ROBIN);
    b.e = L.e[0];
    b.f32 = L.f32[0];
    b.r32 = L.f32[1];
    b.k32 = L.k32;
    for (int c = 0; c < 3; ++c) {
      b.e3[c] = L.e[c];
      b.f3[c] = L.f32[c];
    }
  }
  B->bc = P;
  B->bcv = Pv;
  B->u = L0.u[0];
  B->f = L0.f[0];
  B->s0 = L0.s0;
  B->s1 = L0.s1;
  B->dpsi = h->dpsi;
  B->dap = h->dap;
  B->sg = h->sg;
  for (int c = 0; c < 3; ++c) {
    B->u3[c] = L0.u[c];
    B->f3[c] = L0.f[c];
    B->Xg[c] = h->Xg[c];
  }
  B->aa = h->aa;
  B->U = src.U;
  B->S = src.S;
  B->psi = io.psi;
  B->alpha = io.alpha;
  for (int c = 0; c < 3; ++c) {
    B->Si[c] = src.Si[c];
    B->beta[c] = io.beta[c];
    B->X[c] = io.X[c];
  }
  return MG_OK;
}

// Smoother cell updates of one cycle (as the launched path counts them).
int64_t cycle_updates(const mg_hierarchy* h) {
  int64_t u = 0;
  for (int l = 0; l + 1 < h->nlev; ++l) u += (int64_t)(h->d.nu1 + h->d.nu2) * h->L[l].cells();
  return u;
}

}  // namespace

int mg_solve_cfc_batch(mg_hierarchy* const* hs, int count, const mg_cfc_sources* src, mg_cfc_fields* io, int flags,
                       const mg_batch_opts* opts, mg_cfc_report* rep, mg_batch_report* brep) {
  if (!hs || !src || !io || count <= 0) return fail(MG_ERR_INVALID, "null argument or empty batch");
  int team_opt = opts && opts->team ? opts->team : BATCH_TEAM_DEFAULT;
  const long team_cells = opts && opts->team_cells > 0 ? (long)opts->team_cells : BATCH_TEAM_CELLS;
  if (team_opt != 1 && team_opt != 2 && team_opt != 4 && team_opt != 8)
    return fail(MG_ERR_INVALID, "team must be 1, 2, 4 or 8");
  if (flags & MG_HOST_POINTERS) return fail(MG_ERR_INVALID, "batched solves take device pointers");
  const bool psi_only = flags & MG_CFC_PSI_ONLY;
  {
    std::vector<mg_hierarchy*> seen(hs, hs + count);
    std::sort(seen.begin(), seen.end());
    if (!seen[0]) return fail(MG_ERR_INVALID, "null hierarchy");
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(MG_ERR_INVALID, "each problem of a batch needs its own hierarchy");
  }
  mg_hierarchy* H0 = hs[0];
  const cudaStream_t st = H0->st;
  std::vector<BatchItem> items(count);
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    if (int est = enter(hs[i])) return est;
    if (int est = batch_item(hs[i], src[i], io[i], psi_only, &items[i])) return est;
    smem = std::max(smem, std::max(items[i].bc.smem, items[i].bcv.smem));
  }
  if (int est = ensure_batch_ws(H0, count)) return est;
  // the launch runs on the first hierarchy's stream, after the work queued
  // on every other one
  for (int i = 1; i < count; ++i)
    if (hs[i]->st != st) {
      CK(cudaEventRecord(H0->b_ev[2], hs[i]->st));
      CK(cudaStreamWaitEvent(st, H0->b_ev[2], 0));
    }
  // longest problems first, so that the last ones to start are the
  // shortest: the estimated cost is cells x cycles, the cycles those of the
  // problem's previous batched solve (100 before one); the problems a whole
  // cluster runs come before the others
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto team_of = [&](int a) { return team_opt > 1 && hs[a]->L[0].cells() >= team_cells; };
  auto cost = [&](int a) { return (double)hs[a]->L[0].cells() * (hs[a]->batch_cycles > 0 ? hs[a]->batch_cycles : 100); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (team_of(a) != team_of(b)) return team_of(a);
    return cost(a) > cost(b);
  });
  // clusters of team_opt blocks when some grid has team_cells cells or more
  // (those problems run on a whole cluster), else single blocks
  bool big = false;
  for (int i = 0; i < count; ++i) big = big || team_of(i);
  int team = big ? team_opt : 1;
  int clusters = batch_clusters(smem, team);
  if (clusters < 1 && team > 1) {
    team = 1;
    clusters = batch_clusters(smem, 1);
  }
  if (clusters < 1) return fail(MG_ERR_INVALID, "batch kernel does not fit an SM");
  clusters = std::min(clusters, count);
  const int blocks = clusters * team;
  CK(cudaMemcpyAsync(H0->b_items, items.data(), sizeof(BatchItem) * count, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(H0->b_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(H0->b_next, 0, sizeof(unsigned int), st));
  CK(cudaEventRecord(H0->b_ev[0], st));
  if (launch_batch_cfc(H0->b_items, H0->b_outs, H0->b_hist, H0->b_order, count, H0->b_next, clusters, team,
                       team_cells, smem, st)) {
    CK(cudaGetLastError());
    return fail(MG_ERR_CUDA, "batch launch refused");
  }
  CK(cudaEventRecord(H0->b_ev[1], st));
  std::vector<BatchOut> outs(count);
  CK(cudaMemcpyAsync(outs.data(), H0->b_outs, sizeof(BatchOut) * count, cudaMemcpyDeviceToHost, st));
  std::vector<double> hist;
  if (rep) {
    hist.resize((size_t)4 * BATCH_HIST * count);
    CK(cudaMemcpyAsync(hist.data(), H0->b_hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  float kms = 0.0f;
  CK(cudaEventElapsedTime(&kms, H0->b_ev[0], H0->b_ev[1]));
  unsigned long long t0 = ~0ULL;
  for (const BatchOut& o : outs) t0 = std::min(t0, o.t_start);
  int status = MG_OK, general = 0;
  // problems with momentum: mg_solve_cfc on up to BATCH_GENERAL_THREADS host
  // threads, each hierarchy on its own stream so that their kernels overlap
  // (host cycle loops, as in the request server's slots)
  std::vector<int> gen;
  for (int i = 0; i < count; ++i)
    if (outs[i].status[0] == BATCH_GENERAL) gen.push_back(i);
  general = (int)gen.size();
  if (!gen.empty()) {
    std::vector<int> gst(gen.size(), MG_OK);
    std::atomic<int> take{0};
    auto work = [&]() {
      for (;;) {
        const int q = take.fetch_add(1);
        if (q >= (int)gen.size()) return;
        mg_hierarchy* h = hs[gen[q]];
        const bool host_loop = h->loop_off;
        hier_set_host_loop(h, true);
        gst[q] = mg_solve_cfc(h, &src[gen[q]], &io[gen[q]], flags, rep ? &rep[gen[q]] : nullptr);
        hier_set_host_loop(h, host_loop);
      }
    };
    const int nt = std::min<int>((int)gen.size(), BATCH_GENERAL_THREADS);
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (std::thread& t : pool) t.join();
    for (int s : gst)
      if (s && !status) status = s;
  }
  for (int i = 0; i < count; ++i) {
    const BatchOut& o = outs[i];
    if (o.status[0] == BATCH_GENERAL) continue;
    for (int e = 0; e < 4; ++e)
      if ((o.ran & (1 << e)) && o.status[e] && !status) status = o.status[e];
    hs[i]->batch_cycles = o.cycles[1] + o.cycles[2];
    if (!rep) continue;
    mg_cfc_report& r = rep[i];
    std::memset(&r, 0, sizeof(r));
    const int64_t cu = cycle_updates(hs[i]);
    for (int e = 0; e < 4; ++e) {
      if (!(o.ran & (1 << e))) continue;
      mg_solve_report& q = r.eq[e];
      q.status = o.status[e];
      q.cycles = o.cycles[e];
      q.rel = o.rel[e];
      q.cell_updates = (int64_t)o.cycles[e] * cu * (e == 0 || e == 3 ? 3 : 1);
      q.nhist = std::min(o.cycles[e] + 1, MG_HIST);
      const double* hh = hist.data() + ((size_t)i * 4 + e) * BATCH_HIST;
      for (int c = 0; c < q.nhist; ++c) q.hist[c] = hh[c];
    }
    r.ms = (double)(o.t_end - t0) * 1e-6;
  }
  if (brep) {
    brep->kernel_ms = kms;
    brep->blocks = blocks;
    brep->team = team;
    brep->persistent = count - general;
    brep->general = general;
  }
  return status;
}

int mg_clean_divB(mg_hierarchy* H, double* B[3], double* phi_out, int flags, mg_divb_report* rep) {
  if (!H || !B) return fail(MG_ERR_INVALID, "null argument");
  const int nd = H->d.ndim;
  const bool curv = H->d.geom != MG_CART;
  for (int c = 0; c < nd; ++c)
    if (!B[c]) return fail(MG_ERR_INVALID, "null B component");
  if (int est = enter(H)) return est;
  const bool host = flags & MG_HOST_POINTERS;
  double* Bd[3] = {B[0], B[1], nd == 3 ? B[2] : B[0]};
  int st = MG_OK;
  if (host)
    for (int c = 0; c < nd; ++c)
      if ((st = stage_in(H, c, B[c], &Bd[c]))) return st;
  if (nd == 2) Bd[2] = Bd[0];
  Level& L0 = H->L[0];
  const LevelView<double>& v = L0.v64;
  const double N = (double)L0.cells();
  auto norms = [&](double* mx, double* l2) -> int {
    CK(cudaMemsetAsync(H->d_red, 0, sizeof(unsigned long long), H->st));
    launch_div_norms(v, L0.r[0], H->d_part, NPARTS, H->d_red, H->st);
    std::vector<double> part(NPARTS);
    CK(cudaMemcpyAsync(H->h_red, H->d_red, sizeof(unsigned long long), cudaMemcpyDeviceToHost, H->st));
    CK(cudaMemcpyAsync(part.data(), H->d_part, sizeof(double) * NPARTS, cudaMemcpyDeviceToHost, H->st));
    CK(cudaStreamSynchronize(H->st));
    double s = 0.0;
    for (double x : part) s += x;
    *mx = bits_to_double(H->h_red[0]);
    *l2 = std::sqrt(s / N);
    return MG_OK;
  };
  // curvilinear grids: B into ghosted copies with the vector rules (outer
  // copies, origin / axis parities), then the divergence of Sec. 2.2
  auto vn = with_bc(v, MG_BC_NEUMANN);
  auto div_into_r = [&]() {
    if (!curv) {
      launch_div_central(v, Bd, L0.r[0], H->d_part, NPARTS, H->st);
      return;
    }
    for (int c = 0; c < nd; ++c) {
      copy_in(H, Bd[c], H->Xg[c]);
      launch_fill_ghosts(vn, H->Xg[c], c, H->st);
    }
    double* Xg[3] = {H->Xg[0], H->Xg[1], nd == 3 ? H->Xg[2] : H->Xg[0]};
    launch_div_curv(v, Xg, L0.r[0], H->d_part, NPARTS, H->st);
  };
  // sum of the weights w (1, R, r^2 sin theta) of the compatible mean
  double wsum = N;
  if (curv) {
    double si = 0.0, sj = 0.0;
    for (int i = 0; i < L0.n[0]; ++i) {
      const double x = L0.lo[0] + (i + 0.5) * L0.h[0];
      si += H->d.geom == MG_SPH ? x * x : x;
    }
    for (int j = 0; j < L0.n[1]; ++j) sj += H->d.geom == MG_SPH ? std::sin(L0.lo[1] + (j + 0.5) * L0.h[1]) : 1.0;
    wsum = si * sj * L0.n[2];
  }
  double mb, lb, ma, la;
  if (H->d.divb_variant == MG_DIVB_EXACT) {
    // the parity classes of div minus their means (class-major in r[1]),
    // one compact Neumann solve per class on the half-size hierarchy (Phi
    // class-major in r[2]), B -= grad Phi with mirrored Phi ghosts
    const int ncl = nd == 3 ? 8 : 4;
    const long M = (long)L0.cells() / ncl;
    div_into_r();
    launch_class_gather(v, L0.r[0], H->d_part, NPARTS / 8, L0.r[1], H->st);
    if ((st = norms(&mb, &lb))) return st;
    CK(cudaMemsetAsync(L0.r[2], 0, sizeof(double) * L0.cells(), H->st));
    mg_solve_report agg{};
    for (int q = 0; q < ncl; ++q) {
      mg_solve_report r{};
      const int sq = mg_solve_scalar(H->sub, MG_EQ_LIN, MG_BC_NEUMANN, 1, nullptr, nullptr, nullptr,
                                     L0.r[1] + q * M, L0.r[2] + q * M, &r);
      if (sq == MG_ERR_CUDA || sq == MG_ERR_INVALID || sq == MG_ERR_OOM) return sq;
      if (q == 0 || r.cycles > agg.cycles) {
        agg.cycles = r.cycles;
        agg.nhist = r.nhist;
        std::memcpy(agg.hist, r.hist, sizeof(double) * (size_t)r.nhist);
      }
      agg.rel = q == 0 ? r.rel : std::max(agg.rel, r.rel);
      agg.ms += r.ms;
      agg.cell_updates += r.cell_updates;
      if (st == MG_OK && sq != MG_OK) st = sq;
    }
    agg.status = st;
    if (rep) rep->solve = agg;
    double* pd = nullptr;
    int s2 = MG_OK;
    if (phi_out) {
      pd = phi_out;
      if (host && (s2 = stage_get(H, 3, &pd))) return s2;
    }
    launch_grad_update_exact(v, L0.r[2], Bd, pd, H->st);
    div_into_r();
    if ((s2 = norms(&ma, &la))) return s2;
    if (phi_out && host && (s2 = stage_out(H, pd, phi_out))) return s2;
    if (host)
      for (int c = 0; c < nd; ++c)
        if ((s2 = stage_out(H, Bd[c], B[c]))) return s2;
    CK(cudaStreamSynchronize(H->st));
    if (rep) {
      rep->max_div_before = mb;
      rep->l2_div_before = lb;
      rep->max_div_after = ma;
      rep->l2_div_after = la;
    }
    return st;
  }
  div_into_r();
  if (curv)
    launch_sub_wmean_into(v, L0.r[0], H->d_part, NPARTS, wsum, L0.f[0], H->st);
  else
    launch_sub_mean_into(v, L0.r[0], H->d_part, NPARTS, L0.f[0], H->st);
  if ((st = norms(&mb, &lb))) return st;
  CK(cudaMemsetAsync(L0.u[0], 0, sizeof(double) * L0.ng, H->st));
  Eq e{MG_EQ_LIN, MG_BC_NEUMANN, 1, 1, false};
  st = run_solve(H, e, rep ? &rep->solve : nullptr);
  if (curv) {
    launch_fill_ghosts(vn, L0.u[0], -1, H->st);
    launch_grad_update_curv(v, L0.u[0], Bd, H->st);
  } else {
    launch_grad_update(v, L0.u[0], Bd, H->st);
  }
  div_into_r();
  int s2 = norms(&ma, &la);
  if (s2) return s2;
  if (phi_out) {
    double* pd = phi_out;
    if (host && (s2 = stage_get(H, 3, &pd))) return s2;
    copy_out(H, L0.u[0], pd);
    if (host && (s2 = stage_out(H, pd, phi_out))) return s2;
  }
  if (host)
    for (int c = 0; c < nd; ++c)
      if ((s2 = stage_out(H, Bd[c], B[c]))) return s2;
  CK(cudaStreamSynchronize(H->st));
  if (rep) {
    rep->max_div_before = mb;
    rep->l2_div_before = lb;
    rep->max_div_after = ma;
    rep->l2_div_after = la;
  }
  return st;
}

int mg_apply_operator(mg_hierarchy* H, int kind, int bc, const double* u[3], const double* U, const double* A2,
                      const double* c, double* out[3]) {
  if (!H || !u || !out) return fail(MG_ERR_INVALID, "null argument");
  if (int est = enter(H)) return est;
  Level& L0 = H->L[0];
  auto v = with_bc(L0.v64, bc);
  if (kind == MG_EQ_VEC) {
    for (int q = 0; q < 3; ++q) {
      copy_in(H, u[q], L0.u[q]);
      launch_fill_ghosts(v, L0.u[q], q, H->st);
    }
    launch_apply_vec(v, L0.u, L0.r, 0, H->st);
    for (int q = 0; q < 3; ++q) copy_out(H, L0.r[q], out[q]);
  } else if (kind == MG_EQ_PSI || kind == MG_EQ_LIN) {
    copy_in(H, u[0], L0.u[0]);
    if (kind == MG_EQ_PSI) {
      if (!U || !A2) return fail(MG_ERR_INVALID, "psi operator needs U and A2");
      copy_in(H, U, L0.s0);
      copy_in(H, A2, L0.s1);
    } else if (c) {
      copy_in(H, c, L0.s1);
    }
    launch_apply_scalar(v, kind, L0.u[0], L0.s0, (kind == MG_EQ_PSI || c) ? L0.s1 : nullptr, L0.r[0], 0, H->st);
    copy_out(H, L0.r[0], out[0]);
  } else {
    return fail(MG_ERR_INVALID, "bad equation kind");
  }
  CK(cudaStreamSynchronize(H->st));
  CK(cudaGetLastError());
  return MG_OK;
}

int mg_smooth(mg_hierarchy* H, int kind, int bc, int nsweeps, double* u[3], const double* f[3], const double* U,
              const double* A2, const double* c) {
  if (!H || !u || nsweeps < 0) return fail(MG_ERR_INVALID, "bad argument");
  if (int est = enter(H)) return est;
  Level& L0 = H->L[0];
  const int nc = kind == MG_EQ_VEC ? 3 : 1;
  Eq e{kind, bc, 0, nc, kind == MG_EQ_LIN && c != nullptr};
  for (int q = 0; q < nc; ++q) {
    copy_in(H, u[q], L0.u[q]);
    if (f && f[q]) copy_in(H, f[q], L0.f[q]);
    else cudaMemsetAsync(L0.f[q], 0, sizeof(double) * L0.ng, H->st);
  }
  if (kind == MG_EQ_PSI) {
    copy_in(H, U, L0.s0);
    copy_in(H, A2, L0.s1);
  } else if (c) {
    copy_in(H, c, L0.s1);
  }
  if (kind == MG_EQ_VEC && bc == MG_BC_DIRICHLET)
    if (int est = ensure_ghost_push(H)) return est;
  if (kind == MG_EQ_VEC) fill_all64(H, e, 0);
  smooth64(H, e, 0, nsweeps);
  for (int q = 0; q < nc; ++q) copy_out(H, L0.u[q], u[q]);
  CK(cudaStreamSynchronize(H->st));
  CK(cudaGetLastError());
  return MG_OK;
}

int mg_compute_a2(mg_hierarchy* H, const double* X[3], double* A2) {
  if (!H || !X || !A2) return fail(MG_ERR_INVALID, "null argument");
  if (int est = enter(H)) return est;
  Level& L0 = H->L[0];
  auto v = with_bc(L0.v64, MG_BC_DIRICHLET);
  for (int c = 0; c < 3; ++c) {
    copy_in(H, X[c], H->Xg[c]);
    launch_fill_ghosts(v, H->Xg[c], c, H->st);
  }
  launch_xcfc_a2(v, H->Xg, L0.r[0], H->st);
  copy_out(H, L0.r[0], A2);
  CK(cudaStreamSynchronize(H->st));
  CK(cudaGetLastError());
  return MG_OK;
}

int mg_divergence(mg_hierarchy* H, const double* B[3], double* div) {
  if (!H || !B || !div) return fail(MG_ERR_INVALID, "null argument");
  if (H->d.geom != MG_CART) return fail(MG_ERR_INVALID, "Cartesian only");
  if (int est = enter(H)) return est;
  Level& L0 = H->L[0];
  double* Bd[3] = {(double*)B[0], (double*)B[1], (double*)(H->d.ndim == 3 ? B[2] : B[0])};
  launch_div_central(L0.v64, Bd, L0.r[0], H->d_part, NPARTS, H->st);
  copy_out(H, L0.r[0], div);
  CK(cudaStreamSynchronize(H->st));
  CK(cudaGetLastError());
  return MG_OK;
}

int mg_restrict(mg_hierarchy* H, const double* fine, double* coarse) {
  if (!H || !fine || !coarse) return fail(MG_ERR_INVALID, "null argument");
  if (H->nlev < 2) return fail(MG_ERR_INVALID, "hierarchy has one level");
  if (int est = enter(H)) return est;
  Level& F = H->L[0];
  Level& C = H->L[1];
  copy_in(H, fine, F.r[0]);
  const double* a[4] = {F.r[0], nullptr, nullptr, nullptr};
  double* b[4] = {C.r[0], nullptr, nullptr, nullptr};
  double* cp[3] = {nullptr, nullptr, nullptr};
  launch_restrict(F.v64, C.v64, 1, a, b, cp, H->st);
  launch_copy_out<double, double>(C.v64, C.r[0], coarse, 0.0, H->st);
  CK(cudaStreamSynchronize(H->st));
  CK(cudaGetLastError());
  return MG_OK;
}

int mg_prolong_add(mg_hierarchy* H, int bc, const double* coarse_e, double* fine) {
  if (!H || !coarse_e || !fine) return fail(MG_ERR_INVALID, "null argument");
  if (H->nlev < 2) return fail(MG_ERR_INVALID, "hierarchy has one level");
  if (int est = enter(H)) return est;
  Level& F = H->L[0];
  Level& C = H->L[1];
  launch_copy_in<double, double>(C.v64, coarse_e, C.r[0], 0.0, H->st);
  copy_in(H, fine, F.u[0]);
  launch_prolong(with_bc(F.v64, bc), with_bc(C.v64, bc), F.u[0], C.r[0], (const double*)nullptr, -1, H->st);
  copy_out(H, F.u[0], fine);
  CK(cudaStreamSynchronize(H->st));
  CK(cudaGetLastError());
  return MG_OK;
}

}  // extern "C"

// ------------------------------------------------------ composite grid (AMR)

namespace {

// Argument checks and the copies of a composite call into the level arrays
// (interior layout in, ghosted arrays of the base's finest level and the
// patch out); the box's patch level is set up first.
int amr_enter(mg_hierarchy* H, const int box_lo[3], const int box_hi[3], int kind, int bc, const double* U,
              const double* A2, const double* c, const double* f, const double* Up, const double* A2p,
              const double* cp, const double* fp, const double* u, const double* up, bool need_f, Eq* eq) {
  if (!H || !box_lo || !box_hi || !u || !up) return fail(MG_ERR_INVALID, "null argument");
  if (kind != MG_EQ_PSI && kind != MG_EQ_LIN) return fail(MG_ERR_INVALID, "bad equation kind");
  if (bc < MG_BC_ROBIN || bc > MG_BC_NEUMANN) return fail(MG_ERR_INVALID, "bad boundary condition");
  if (kind == MG_EQ_PSI && (!U || !A2 || !Up || !A2p))
    return fail(MG_ERR_INVALID, "psi equation needs U and A2 on both levels");
  if (kind == MG_EQ_LIN && need_f && (!f || !fp)) return fail(MG_ERR_INVALID, "linear equation needs f on both levels");
  if (kind == MG_EQ_LIN && (!c) != (!cp)) return fail(MG_ERR_INVALID, "give c on both levels or on neither");
  AmrBox box;
  if (int st = amr_box(H, box_lo, box_hi, &box)) return st;
  if (int st = enter(H)) return st;
  if (int st = ensure_amr(H, box)) return st;
  Eq e{kind, bc, 0, 1, kind == MG_EQ_LIN && c != nullptr};
  e.amr = true;
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const AmrArrays W = amr_arrays(H, e);
  copy_in(H, u, L0.u[0]);
  launch_copy_in<double, double>(A.v, up, A.u, 0.0, H->st);
  if (kind == MG_EQ_PSI) {
    copy_in(H, U, L0.s0);
    copy_in(H, A2, L0.s1);
    launch_copy_in<double, double>(A.v, Up, A.s0, 0.0, H->st);
    launch_copy_in<double, double>(A.v, A2p, A.s1, 0.0, H->st);
    CK(cudaMemsetAsync(A.f, 0, sizeof(double) * A.ng, H->st));
  } else {
    if (c) {
      copy_in(H, c, L0.s1);
      launch_copy_in<double, double>(A.v, cp, A.s1, 0.0, H->st);
    }
    if (f) copy_in(H, f, W.f0);
    if (fp) launch_copy_in<double, double>(A.v, fp, A.f, 0.0, H->st);
  }
  *eq = e;
  return MG_OK;
}

}  // namespace

int mg_solve_scalar_amr(mg_hierarchy* H, const int box_lo[3], const int box_hi[3], int kind, int bc,
                        const double* U, const double* A2, const double* c, const double* f, const double* Up,
                        const double* A2p, const double* cp, const double* fp, double* u, double* up,
                        mg_solve_report* rep) {
  Eq e{};
  if (int st = amr_enter(H, box_lo, box_hi, kind, bc, U, A2, c, f, Up, A2p, cp, fp, u, up, true, &e)) return st;
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const int st = run_solve_amr(H, e, rep);
  // covered base cells: the restriction of the patch
  const AmrArrays W = amr_arrays(H, e);
  launch_amr_restrict(with_bc(A.v, e.bc), with_bc(L0.v64, e.bc), A.box, A.u, A.r, L0.u[0], W.rr, H->st);
  copy_out(H, L0.u[0], u);
  launch_copy_out<double, double>(A.v, A.u, up, 0.0, H->st);
  CK(cudaStreamSynchronize(H->st));
  return st;
}

int mg_apply_amr(mg_hierarchy* H, const int box_lo[3], const int box_hi[3], int kind, int bc, const double* U,
                 const double* A2, const double* c, const double* Up, const double* A2p, const double* cp,
                 const double* u, const double* up, double* out, double* outp) {
  if (!out || !outp) return fail(MG_ERR_INVALID, "null output");
  Eq e{};
  if (int st = amr_enter(H, box_lo, box_hi, kind, bc, U, A2, c, nullptr, Up, A2p, cp, nullptr, u, up, false, &e))
    return st;
  auto& A = H->amr;
  Level& L0 = H->L[0];
  const AmrArrays W = amr_arrays(H, e);
  restrict_sources(H, e);
  amr_refresh(H, e, true);
  const double* s0p = e.kind == EQ_PSI ? A.s0 : nullptr;
  const double* s1p = (e.kind == EQ_PSI || e.has_c) ? A.s1 : nullptr;
  launch_amr_patch_resid(with_bc(A.v, e.bc), e.kind, A.u, nullptr, s0p, s1p, A.r, nullptr, 1, H->st);
  launch_amr_base(with_bc(L0.v64, e.bc), A.box, e.kind, L0.u[0], s0ptr(H, e, 0), s1ptr(H, e, 0), nullptr, nullptr,
                  W.corr, L0.r[0], nullptr, 2, H->st);
  copy_out(H, L0.r[0], out);
  launch_copy_out<double, double>(A.v, A.r, outp, 0.0, H->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(H->st));
  return MG_OK;
}
