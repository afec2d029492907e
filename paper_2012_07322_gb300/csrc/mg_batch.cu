// Batched xCFC solves in one persistent launch.  Each thread block (a
// cluster of blocks for the largest grids) takes a problem from a shared
// queue (longest first) and runs its whole xCFC solve in the order of
// Sec. 2.6 (Steps 1-6: eq. X, A~^2, eq. psi, the alpha-psi coefficient,
// eq. alpha, the shift source and eq. beta), each equation by the
// mixed-precision defect correction of the launched path: the FP64 residual
// and stopping norm (Sec. 2.7.2), a V-cycle of the FP32 correction equation
// (red-black NGS, volume-weighted restriction, Kwak prolongation; Secs.
// 2.7.2-2.7.3) whose levels of at most BLOCK_CYCLE_CELLS cells run the
// one-block cycle in shared memory, the FP64 update and the Anderson mixing
// step.  The phases are those of the launched kernels, with the same
// per-cell functions, separated by block (or cluster) barriers: a 2D problem of a few
// thousand to a hundred thousand cells leaves a launched V-cycle
// latency-bound, and one block per problem lets many problems of different
// sizes fill the GPU together without a launch per phase.
//
// Without momentum (S_i and the X and beta guesses all zero) X = beta = 0
// is exact: both right-hand sides vanish and the solves stop at cycle 0, so
// those steps are skipped.  Problems with momentum on a hierarchy whose
// vector levels do not fit the kernel are marked BATCH_GENERAL and the host
// solves them through mg_solve_cfc after the launch.
#include <cooperative_groups.h>

#include "mg_internal.h"
#include "mg_kernels.cuh"
#include "mg_block.cuh"
#include "mg_accel.cuh"
#include "mg_xcfc.cuh"

namespace cg = cooperative_groups;

namespace gmg {

static_assert(BATCH_THREADS == BC_THREADS, "the batch kernel runs the one-block cycle");

// The blocks that run one problem: a whole thread-block cluster (a team of
// up to BATCH_TEAM blocks) for the largest grids, else one block alone.  Passes
// stride over the team's threads; its barrier is the cluster barrier with
// release / acquire semantics at cluster scope (which orders the team's
// global and shared memory accesses) and a compiler memory barrier;
// reductions meet in rank 0's shared memory, each block writing its own row
// there (no shared slot that a block resets while another updates it).
struct Team {
  int rank, size;
  __device__ __forceinline__ long start() const { return (long)rank * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ long stride() const { return (long)size * blockDim.x; }
  __device__ __forceinline__ void sync() const {
    if (size > 1)
      asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
    else
      __syncthreads();
  }
  // p (a shared-memory address of this block) in rank 0's shared memory
  template <typename T>
  __device__ __forceinline__ T* at0(T* p) const {
    return size > 1 ? cg::this_cluster().map_shared_rank(p, 0) : p;
  }
};

struct BtShared {
  unsigned long long red[3];
  unsigned long long cred[BATCH_TEAM][3];  // rank 0: the team's per-block maxima
  float part[BATCH_THREADS / 32][2 * AA_MAX];
  float cpart[BATCH_TEAM][2 * AA_MAX];  // rank 0: the team's per-block dot products
  float s[2 * AA_MAX];
  float M[AA_MAX * AA_MAX];  // Gram matrix over ring slots (lives for one equation)
  float gamma[AA_MAX];
  AACols cols;
  long coff[AA_MAX];  // offsets of the live history columns (cols.slot x the column length)
  int status;
  int flags[BATCH_TEAM];  // rank 0: the team's per-block flags
  int item;
  double hist[BATCH_HIST];  // this block's copy of the residual history (stall window)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ long bt_cells(const LevelView<double>& L) { return (long)L.n0 * L.n1 * L.n2; }
template <typename T>
__device__ __forceinline__ long bt_ghosted(const LevelView<T>& L) {
  return L.sy * (L.n2 + 2 * L.three);
}

// The team's maxima of three non-negative values given as abs_bits: each
// block reduces its own, writes them into its row of rank 0's cred, and
// every block takes the maximum over the rows.
__device__ void bt_team_max3(const Team& T, unsigned long long (&m)[3], BtShared& S) {
  if (threadIdx.x < 3) S.red[threadIdx.x] = 0ULL;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) m[c] = warp_max_bits(m[c]);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicMax(&S.red[c], m[c]);
  __syncthreads();
  if (threadIdx.x < 3) T.at0(S.cred[T.rank])[threadIdx.x] = S.red[threadIdx.x];
  T.sync();
  if (threadIdx.x < 3) {
    const unsigned long long* rows = T.at0(&S.cred[0][0]);
    unsigned long long v = 0ULL;
    for (int r = 0; r < T.size; ++r) v = umax64(v, rows[3 * r + threadIdx.x]);
    S.red[threadIdx.x] = v;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) m[c] = S.red[c];
  T.sync();  // rank 0's rows are rewritten only after every block has read them
}

// The FP32 passes and the mixing below copy the level views they stream
// over out of shared memory: held by reference, every field would be read
// back after each global store (the compiler cannot tell the two apart).

// FP64 residual of the finest level with the stopping norms (as
// k_residual_scalar, weighted): the FP32 right-hand side of the correction
// cycle into lv[0].f32 and, for eq. psi, its linearisation K into lv[0].k32;
// returns rel = max |w r| / max |w S| (NaN when a norm is not finite).
template <int G, int KIND>
__device__ double bt_norm(const Team& T, const BatchItem& I, const double* f, const double* s0, const double* s1,
                          BtShared& S) {
  const LevelView<double>& L = I.v64;  // passed on to the out-of-line FP64 edge rules: stays in shared memory
  float* __restrict__ r32 = I.lv[0].f32;
  float* __restrict__ k32 = I.lv[0].k32;
  const double* __restrict__ u = I.u;
  unsigned long long m0 = 0ULL, m1 = 0ULL, m2 = 0ULL;
  const long n = bt_cells(L);
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    const double w = (double)norm_weight(L, i, j);
    double Sv, kp;
    const double rv =
        scalar_residual_cell<double, G, KIND>(L, u, f, s0, s1, i, j, k, p, Sv, KIND == EQ_PSI ? &kp : nullptr);
    r32[p] = (float)rv;
    if (KIND == EQ_PSI) k32[p] = (float)kp;
    m0 = umax64(m0, abs_bits(rv));
    if (G != CART) m1 = umax64(m1, abs_bits(w * rv));
    m2 = umax64(m2, abs_bits(G == CART ? Sv : w * Sv));
  }
  if (G == CART) m1 = m0;
  unsigned long long mm[3] = {m0, m1, m2};
  bt_team_max3(T, mm, S);
  const double num = __longlong_as_double((long long)mm[1]), den = __longlong_as_double((long long)mm[2]);
  if (isinf(num) || isinf(den) || isnan(num) || isnan(den)) return __longlong_as_double(0x7ff8000000000000LL);
  return num / (den > 1e-300 ? den : 1e-300);
}

// nsweeps red-black sweeps of the correction equation (L - K) e = f at one
// level (the cells of a colour are independent).
template <int G>
__device__ void bt_smooth(const Team& T, const BatchLevel& B, int nsweeps) {
  const LevelView<float> L = B.v;
  float* __restrict__ e = B.e;
  const float* __restrict__ f = B.f32;
  const float* __restrict__ K = B.k32;
  const long nh = (long)L.n0 * L.n1 * L.n2 / 2;
  for (int s = 0; s < nsweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      for (long q = T.start(); q < nh; q += T.stride()) {
        int i, j, k;
        L.colour_cell(q, colour, i, j, k);
        scalar_update<float, G, EQ_LIN>(L, e, f, nullptr, K, i, j, k);
      }
      T.sync();
    }
}

// Residual of level F restricted into the coarse right-hand side, coarse
// correction zeroed; with fold K is restricted alongside (eq. psi: K is
// evaluated at the current iterate and restricted on the way down).
template <int G>
__device__ void bt_resid_restrict(const Team& T, const BatchLevel& F, const BatchLevel& C, bool fold) {
  const LevelView<float> L = F.v;
  const long n = (long)L.n0 * L.n1 * L.n2;
  float* __restrict__ r32 = F.r32;
  const float* __restrict__ e = F.e;
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    float Sv;
    r32[p] = scalar_residual_cell<float, G, EQ_LIN>(L, e, F.f32, nullptr, F.k32, i, j, k, p, Sv);
  }
  T.sync();
  const LevelView<float> Cv = C.v;
  const long nC = (long)Cv.n0 * Cv.n1 * Cv.n2, ngC = bt_ghosted(Cv);
  const float* const as[4] = {F.r32, F.k32, nullptr, nullptr};
  float* const bs[4] = {C.f32, C.k32, nullptr, nullptr};
  float* const cs[3] = {nullptr, nullptr, nullptr};
  for (long q = T.start(); q < nC; q += T.stride()) {
    int I, J, K;
    Cv.cell(q, I, J, K);
    restrict_cell(L, Cv, fold ? 2 : 1, as, bs, cs, I, J, K);
  }
  for (long q = T.start(); q < ngC; q += T.stride()) C.e[q] = 0.0f;
  T.sync();
}

// K of a level restricted into the next coarser one.
__device__ void bt_restrict_k(const Team& T, const LevelView<float>& F, const float* kF, const LevelView<float>& Cv,
                              float* kC) {
  const long nC = (long)Cv.n0 * Cv.n1 * Cv.n2;
  const float* const as[4] = {kF, nullptr, nullptr, nullptr};
  float* const bs[4] = {kC, nullptr, nullptr, nullptr};
  float* const cs[3] = {nullptr, nullptr, nullptr};
  for (long q = T.start(); q < nC; q += T.stride()) {
    int I, J, K;
    Cv.cell(q, I, J, K);
    restrict_cell(F, Cv, 1, as, bs, cs, I, J, K);
  }
  T.sync();
}

// K from level 0 down to the coarsest (linear equation: c is fixed).
__device__ void bt_restrict_k_all(const Team& T, const BatchItem& I) {
  for (int l = 1; l <= I.nl; ++l) bt_restrict_k(T, I.lv[l - 1].v, I.lv[l - 1].k32, I.lv[l].v, I.lv[l].k32);
  for (int q = 1; q < I.bc.nl; ++q)
    bt_restrict_k(T, I.bc.lv[q - 1].v, I.bc.lv[q - 1].k32, I.bc.lv[q].v, const_cast<float*>(I.bc.lv[q].k32));
}

// One V-cycle of the FP32 correction equation from e = 0 at level 0 (lv[0].e
// zeroed by the caller): pre-smoothing and residual restriction down to
// level nl, the one-block cycle from there (rank 0 of a team runs it alone),
// prolongation and post-smoothing back up.
template <int G>
__device__ void bt_vcycle(const Team& T, const BatchItem& I, bool fold, float* sm, double* smd) {
  for (int l = 0; l < I.nl; ++l) {
    bt_smooth<G>(T, I.lv[l], I.nu1);
    bt_resid_restrict<G>(T, I.lv[l], I.lv[l + 1], fold);
  }
  if (fold)
    for (int q = 1; q < I.bc.nl; ++q)
      bt_restrict_k(T, I.bc.lv[q - 1].v, I.bc.lv[q - 1].k32, I.bc.lv[q].v, const_cast<float*>(I.bc.lv[q].k32));
  if (T.rank == 0) bc_run<G, false, true>(I.bc, sm, smd);
  T.sync();
  for (int l = I.nl - 1; l >= 0; --l) {
    const BatchLevel& F = I.lv[l];
    const BatchLevel& C = I.lv[l + 1];
    const LevelView<float> Fv = F.v;
    const long nF = (long)Fv.n0 * Fv.n1 * Fv.n2;
    float* __restrict__ e = F.e;
    const float* __restrict__ eC = C.e;
    for (long q = T.start(); q < nF; q += T.stride()) {
      int i, j, k;
      Fv.cell(q, i, j, k);
      prolong_cell(Fv, C.v, e, eC, (const float*)nullptr, -1, i, j, k);
    }
    T.sync();
    bt_smooth<G>(T, F, I.nu2);
  }
}

// The mixing step after a cycle (as k_aa_update_dots + k_aa_combine with
// FP32 history): g = u, f = g - x, the newest difference columns, their dot
// products with the live columns, the Gram solve by warp 0, and
// u = g - sum gamma_a dG_a, x = u.  Values stream in groups of G4
// consecutive cells of a row; a vector of ncomp components is ncomp ghosted
// arrays back to back (the storage at I.aa holds x, f', g' and the m
// columns of dF and dG in that layout).  Returns the solve's status (0
// solved, 1 degenerate history; 0 when no column is live).
template <int G4>
__device__ int bt_mix_g(const Team& T, const BatchItem& I, int ncomp, const AACols& cols, BtShared& S) {
  const LevelView<double> L = I.v64;
  const long nq = bt_cells(L) / G4, ng = bt_ghosted(L), vs = ncomp * ng;
  const int nc = cols.n;
  const long onew = nc > 0 ? (long)cols.slot[nc - 1] * vs : 0;
  // the live columns' offsets in shared memory: read there in the streaming
  // loops (broadcast), they leave the registers to the streams
  if (threadIdx.x == 0) S.cols = cols;
  if (threadIdx.x < AA_MAX) S.coff[threadIdx.x] = (long)cols.slot[threadIdx.x] * vs;
  __syncthreads();
  double* __restrict__ x = I.aa;
  double* __restrict__ fpr = x + vs;
  double* __restrict__ gpr = fpr + vs;
  float* const dF = reinterpret_cast<float*>(gpr + vs);
  float* const dG = dF + (long)I.m * vs;
  const float* __restrict__ dFr = dF;
  float* __restrict__ dFw = dF + onew;
  float* __restrict__ dGw = dG + onew;
  float v[32];
#pragma unroll
  for (int a = 0; a < 32; ++a) v[a] = 0.0f;
  for (int c = 0; c < ncomp; ++c)
  for (long q = T.start(); q < nq; q += T.stride()) {
    double* __restrict__ u = I.u3[c];
    const long pu = aa_pos<G4>(L, q), p = (long)c * ng + pu;
    double g[G4], xv[G4], fp[G4], gp[G4], f[G4];
    aa_ld_u<G4>(u + pu, g);
    aa_ld<G4>(x + p, xv);
    aa_ld<G4>(fpr + p, fp);
    aa_ld<G4>(gpr + p, gp);
#pragma unroll
    for (int t = 0; t < G4; ++t) f[t] = g[t] - xv[t];
    aa_st<G4>(x + p, g);
    aa_st<G4>(fpr + p, f);
    aa_st<G4>(gpr + p, g);
    if (nc == 0) continue;
    float dn[G4], dg[G4], ft[G4];
#pragma unroll
    for (int t = 0; t < G4; ++t) {
      dn[t] = (float)(f[t] - fp[t]);
      dg[t] = (float)(g[t] - gp[t]);
      ft[t] = (float)f[t];
    }
    aa_st<G4>(dFw + p, dn);
    aa_st<G4>(dGw + p, dg);
#pragma unroll
    for (int a = 0; a < AA_MAX; ++a) {
      float da[G4];
      if (a < nc - 1)
        aa_ld<G4>(dFr + S.coff[a] + p, da);
      else if (a == nc - 1)
#pragma unroll
        for (int t = 0; t < G4; ++t) da[t] = dn[t];
      else
        continue;
#pragma unroll
      for (int t = 0; t < G4; ++t) {
        v[a] += da[t] * ft[t];
        v[AA_MAX + a] += da[t] * dn[t];
      }
    }
  }
  if (nc == 0) {
    T.sync();
    return 0;
  }
  // the block's sums (fixed order) into row rank of rank 0's cpart, then
  // rank 0 adds the rows in rank order and solves
  const float w = warp_sum32(v);
  S.part[threadIdx.x >> 5][threadIdx.x & 31] = w;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s = 0.0f;
#pragma unroll
    for (int b = 0; b < BATCH_THREADS / 32; ++b) s += S.part[b][threadIdx.x];
    T.at0(S.cpart[T.rank])[threadIdx.x] = s;
  }
  T.sync();
  if (T.rank == 0 && threadIdx.x < 32) {
    const int t = threadIdx.x;
    float s = 0.0f;
    for (int r = 0; r < T.size; ++r) s += S.cpart[r][t];
    S.s[t] = s;
    __syncwarp();
    // the newest column's row of the Gram matrix, then the scaled,
    // shifted system solved by Cholesky (as aa_solve_block in FP32)
    const int newest = S.cols.slot[nc - 1];
    if (t < nc) {
      const int c = S.cols.slot[t];
      const float gv = S.s[AA_MAX + t];
      S.M[newest * AA_MAX + c] = gv;
      S.M[c * AA_MAX + newest] = gv;
    }
    __syncwarp();
    float dmax = 0.0f;
    for (int a = 0; a < nc; ++a) dmax = fmaxf(dmax, S.M[S.cols.slot[a] * AA_MAX + S.cols.slot[a]]);
    bool ok = dmax > 0.0f && dmax <= 3.4e38f;
    const float sc = ok ? 1.0f / dmax : 0.0f;
    float row[AA_MAX];
    const int ra = t < nc ? S.cols.slot[t] : 0;
#pragma unroll
    for (int k = 0; k < AA_MAX; ++k)
      row[k] = (t < nc && k < nc) ? S.M[ra * AA_MAX + S.cols.slot[k]] * sc + (k == t ? AA_SHIFT<float> : 0.0f)
                                  : (k == t ? 1.0f : 0.0f);
    float z = t < nc ? S.s[t] * sc : 0.0f;
    ok = __all_sync(0xffffffffu, ok);
    if (ok) ok = chol_warp_f32(row, z, t);
    if (ok) ok = __all_sync(0xffffffffu, z - z == 0.0f);
    if (ok && t < nc) S.gamma[t] = z;
    if (t == 0) S.status = ok ? 0 : 1;
  }
  T.sync();
  if (T.rank != 0) {
    // the weights and status from rank 0 (rewritten there only after the
    // barriers of the next cycle)
    if (threadIdx.x < AA_MAX) S.gamma[threadIdx.x] = T.at0(S.gamma)[threadIdx.x];
    if (threadIdx.x == 0) S.status = *T.at0(&S.status);
    __syncthreads();
  }
  const int st = S.status;
  if (st == 0) {
    float gm[AA_MAX];
#pragma unroll
    for (int a = 0; a < AA_MAX; ++a) gm[a] = a < nc ? S.gamma[a] : 0.0f;
    const float* __restrict__ dGr = dG;
    for (int c = 0; c < ncomp; ++c)
    for (long q = T.start(); q < nq; q += T.stride()) {
      double* __restrict__ u = I.u3[c];
      const long pu = aa_pos<G4>(L, q), p = (long)c * ng + pu;
      float sacc[G4];
#pragma unroll
      for (int t = 0; t < G4; ++t) sacc[t] = 0.0f;
#pragma unroll
      for (int a = 0; a < AA_MAX; ++a) {
        if (a >= nc) break;
        float d[G4];
        aa_ld<G4>(dGr + S.coff[a] + p, d);
#pragma unroll
        for (int t = 0; t < G4; ++t) sacc[t] += gm[a] * d[t];
      }
      double uv[G4];
      aa_ld_u<G4>(u + pu, uv);
#pragma unroll
      for (int t = 0; t < G4; ++t) uv[t] -= (double)sacc[t];
      aa_st_u<G4>(u + pu, uv);
      aa_st<G4>(x + p, uv);
    }
  }
  T.sync();
  return st;
}

__device__ int bt_mix(const Team& T, const BatchItem& I, int ncomp, const AACols& cols, BtShared& S) {
  return I.v64.n0 >= 4 ? bt_mix_g<4>(T, I, ncomp, cols, S) : bt_mix_g<1>(T, I, ncomp, cols, S);
}

// u += e on the interior of level 0 (the FP64 update of the defect
// correction), in groups of four cells of a row where n0 allows.
__device__ void bt_add_correction(const Team& T, const BatchItem& I) {
  const LevelView<double> L = I.v64;
  const long n = bt_cells(L);
  double* __restrict__ u = I.u;
  const float* __restrict__ e = I.lv[0].e;
  if (L.n0 >= 4) {
    for (long q = T.start(); q < n / 4; q += T.stride()) {
      const long p = group4(L, q);
      double a[4], b[4];
      ld4(u + p, a);
      ld4(e + p, b);
#pragma unroll
      for (int t = 0; t < 4; ++t) a[t] += b[t];
      st4(u + p, a);
    }
  } else {
    for (long q = T.start(); q < n; q += T.stride()) {
      const long p = interior_p(L, q);
      u[p] += (double)e[p];
    }
  }
  T.sync();
}

// ------------------------------------------------- vector equations (X, beta)
// The vector equation lap V + 1/3 grad div V = f with the Dirichlet outer
// rule (eqs. X, beta): ghosts are stored, refreshed after every pass that
// changes a component, as in the launched path.  The FP32 passes use the
// flux form of the operator (as the one-block cycle does).

// The ghosts of one component of a level (each ghost reads only interior
// cells, so one pass suffices); the caller's barrier follows.
template <typename TT>
__device__ void bt_fill(const Team& T, const LevelView<TT>& L, TT* u, int comp) {
  const long ng = ghost_count(L);
  for (long g = T.start(); g < ng; g += T.stride()) fill_one_ghost(L, u, comp, g);
}

// FP64 residual of the finest level (ghosts current) with the stopping
// norms (as k_residual_vec, weighted), the FP32 right-hand sides of the
// correction cycle into lv[0].f3.
template <int G>
__device__ __noinline__ double bt_norm_vec(const Team& T, const BatchItem& I, BtShared& S) {
  const LevelView<double>& L = I.v64;
  unsigned long long m0 = 0ULL, m1 = 0ULL, m2 = 0ULL;
  const long n = bt_cells(L);
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    const double w = (double)norm_weight(L, i, j);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double fv = I.f3[c][p];
      const double rv = vec_residual_cell<double, G>(L, I.u3[0], I.u3[1], I.u3[2], I.f3[c], c, i, j, p);
      I.lv[0].f3[c][p] = (float)rv;
      m0 = umax64(m0, abs_bits(rv));
      m1 = umax64(m1, abs_bits(w * rv));
      m2 = umax64(m2, abs_bits(w * fv));
    }
  }
  unsigned long long mm[3] = {m0, m1, m2};
  bt_team_max3(T, mm, S);
  const double num = __longlong_as_double((long long)mm[1]), den = __longlong_as_double((long long)mm[2]);
  if (isinf(num) || isinf(den) || isnan(num) || isnan(den)) return __longlong_as_double(0x7ff8000000000000LL);
  return num / (den > 1e-300 ? den : 1e-300);
}

// nsweeps red-black sweeps, component by component, each component's
// ghosts refreshed after its pass.
template <int G>
__device__ void bt_smooth_vec(const Team& T, const BatchLevel& B, int nsweeps) {
  LevelView<float> L = B.v;
  L.bc = BC_DIRICHLET;
  float* const e0 = B.e3[0];
  float* const e1 = B.e3[1];
  float* const e2 = B.e3[2];
  const long nh = (long)L.n0 * L.n1 * L.n2 / 2;
  for (int s = 0; s < nsweeps; ++s)
    for (int colour = 0; colour < 2; ++colour)
#pragma unroll 1
      for (int c = 0; c < 3; ++c) {
        for (long q = T.start(); q < nh; q += T.stride()) {
          int i, j, k;
          L.colour_cell(q, colour, i, j, k);
          vec_update<float, G, false>(L, e0, e1, e2, B.f3[c], c, i, j, k);
        }
        T.sync();
        bt_fill(T, L, B.e3[c], c);
        T.sync();
      }
}

// Residual of every component restricted into the coarse right-hand sides
// (each coarse cell evaluates the residuals of its own children, with the
// weights and summation order of restrict_cell); coarse corrections zeroed.
template <int G>
__device__ void bt_resid_restrict_vec(const Team& T, const BatchLevel& F, const BatchLevel& C) {
  const LevelView<float> L = F.v;
  const LevelView<float> Cv = C.v;
  const long nC = (long)Cv.n0 * Cv.n1 * Cv.n2, ngC = bt_ghosted(Cv);
  const int nk = L.three ? 2 : 1;
  for (long q = T.start(); q < nC; q += T.stride()) {
    int I, J, K;
    Cv.cell(q, I, J, K);
    float wi[2], wj[2];
    wi[0] = L.TI(TI_VW, 2 * I);
    wi[1] = L.TI(TI_VW, 2 * I + 1);
    wj[0] = L.TJ(TJ_VW, 2 * J);
    wj[1] = L.TJ(TJ_VW, 2 * J + 1);
    float wsum = 0.0f;
    for (int dk = 0; dk < nk; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) wsum += wi[di] * wj[dj];
    const float inv = 1.0f / wsum;
    const long qc = Cv.idx(I, J, K);
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      float sr = 0.0f;
      for (int dk = 0; dk < nk; ++dk)
        for (int dj = 0; dj < 2; ++dj)
          for (int di = 0; di < 2; ++di) {
            const int i = 2 * I + di, j = 2 * J + dj, k = L.three ? 2 * K + dk : 0;
            const float r = vec_residual_cell<float, G, false>(L, F.e3[0], F.e3[1], F.e3[2], F.f3[c], c, i, j,
                                                               L.idx(i, j, k));
            sr += wi[di] * wj[dj] * r;
          }
      C.f3[c][qc] = sr * inv;
    }
  }
  for (long q = T.start(); q < ngC; q += T.stride())
#pragma unroll
    for (int c = 0; c < 3; ++c) C.e3[c][q] = 0.0f;
  T.sync();
}

// One FP32 correction V-cycle of the vector equation from e = 0 at level 0.
template <int G>
__device__ __noinline__ void bt_vcycle_vec(const Team& T, const BatchItem& I, unsigned char* smem_raw) {
  for (int l = 0; l < I.nlv; ++l) {
    bt_smooth_vec<G>(T, I.lv[l], I.nu1);
    bt_resid_restrict_vec<G>(T, I.lv[l], I.lv[l + 1]);
  }
  if (T.rank == 0)
    bc_run<G, true, true>(I.bcv, reinterpret_cast<float*>(smem_raw),
                    reinterpret_cast<double*>(smem_raw + I.bcv.fp64_at));
  T.sync();
  for (int l = I.nlv - 1; l >= 0; --l) {
    const BatchLevel& F = I.lv[l];
    const BatchLevel& C = I.lv[l + 1];
    LevelView<float> Fv = F.v;
    Fv.bc = BC_DIRICHLET;
    const long nF = (long)Fv.n0 * Fv.n1 * Fv.n2;
    for (long q = T.start(); q < nF; q += T.stride()) {
      int i, j, k;
      Fv.cell(q, i, j, k);
#pragma unroll 1
      for (int c = 0; c < 3; ++c) prolong_cell(Fv, C.v, F.e3[c], C.e3[c], (const float*)nullptr, c, i, j, k);
    }
    T.sync();
#pragma unroll 1
    for (int c = 0; c < 3; ++c) bt_fill(T, Fv, F.e3[c], c);
    T.sync();
    bt_smooth_vec<G>(T, F, I.nu2);
  }
}

// The finest FP64 components' ghosts (Dirichlet rule).
__device__ void bt_fill_u3(const Team& T, const BatchItem& I) {
  LevelView<double> L = I.v64;
  L.bc = BC_DIRICHLET;
#pragma unroll 1
  for (int c = 0; c < 3; ++c) bt_fill(T, L, I.u3[c], c);
  T.sync();
}

// One scalar equation by the defect-correction loop of the launched path
// (the stopping rule in its order: non-finite, tol, max_cycles, stall
// window); u, f, s0, s1 as the equation's operator takes them.  Every block
// of a team takes the same decisions: they depend only on values read from
// rank 0's shared memory after a barrier.  Returns the status.
template <int G, int KIND>
__device__ __noinline__ int bt_solve(const Team& T, const BatchItem& I, const double* f, const double* s0, const double* s1,
                        BatchOut& O, int eq, double* hist, float* sm, double* smd, BtShared& S) {
  const LevelView<double>& L = I.v64;
  const long n = bt_cells(L), ng = bt_ghosted(L);
  if (KIND == EQ_LIN) {
    // c of the correction equation: the FP64 coefficient rounded, restricted
    // to every level once
    for (long q = T.start(); q < n; q += T.stride()) {
      int i, j, k;
      L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      I.lv[0].k32[p] = (float)s1[p];
    }
    T.sync();
    bt_restrict_k_all(T, I);
  }
  const int m = I.m;
  int cyc = 0, ncol = 0, head = 0, status = 0;
  double rel = bt_norm<G, KIND>(T, I, f, s0, s1, S);
  if (threadIdx.x == 0) {
    S.hist[0] = rel;
    if (T.rank == 0) hist[0] = rel;
  }
  __syncthreads();
  for (;;) {
    if (rel != rel) {
      status = 5;  // MG_ERR_NAN
      break;
    }
    if (rel <= I.tol) break;
    if (cyc >= I.max_cycles) {
      status = 3;  // MG_ERR_NOCONV
      break;
    }
    if (I.stall_window > 0 && cyc >= I.stall_window && rel > 0.95 * S.hist[cyc - I.stall_window]) {
      status = 4;  // MG_ERR_STALLED
      break;
    }
    if (m > 0 && cyc == 0)
      for (long q = T.start(); q < ng; q += T.stride()) I.aa[q] = I.u[q];
    for (long q = T.start(); q < ng; q += T.stride()) I.lv[0].e[q] = 0.0f;
    T.sync();
    bt_vcycle<G>(T, I, KIND == EQ_PSI, sm, smd);
    bt_add_correction(T, I);
    bool mixstep = false;
    int mst = 0;
    if (m > 0) {
      AACols cols;
      cols.n = 0;
#pragma unroll
      for (int a = 0; a < AA_MAX; ++a) cols.slot[a] = 0;
      if (cyc > 0) {
        const int slot = head;
        head = (head + 1) % m;
        if (ncol < m) ++ncol;
        cols.n = ncol;
#pragma unroll
        for (int a = 0; a < AA_MAX; ++a)
          if (a < ncol) cols.slot[a] = (slot - ncol + 1 + a + m) % m;  // oldest first
      }
      mst = bt_mix(T, I, 1, cols, S);
      mixstep = cols.n > 0;
    }
    ++cyc;
    rel = bt_norm<G, KIND>(T, I, f, s0, s1, S);
    if (mixstep && mst != 0) ncol = 0;  // degenerate history: restart the mixing
    if (threadIdx.x == 0 && cyc < BATCH_HIST) {
      S.hist[cyc] = rel;
      if (T.rank == 0) hist[cyc] = rel;
    }
    __syncthreads();
  }
  if (T.rank == 0 && threadIdx.x == 0) {
    O.status[eq] = status;
    O.cycles[eq] = cyc;
    O.rel[eq] = rel;
  }
  return status;
}

// X, beta and the vector guesses all zero (the static-star case)?
__device__ bool bt_momentum_free(const Team& T, const BatchItem& I, BtShared& S) {
  const long n = bt_cells(I.v64);
  int nz = 0;
  for (long q = T.start(); q < n; q += T.stride())
#pragma unroll
    for (int c = 0; c < 3; ++c) nz |= (I.Si[c][q] != 0.0) | (I.X[c][q] != 0.0) | (I.beta[c][q] != 0.0);
  nz = __syncthreads_or(nz);
  if (threadIdx.x == 0) T.at0(S.flags)[T.rank] = nz;
  T.sync();
  const int* flags = T.at0(S.flags);
  int any = 0;
  for (int r = 0; r < T.size; ++r) any |= flags[r];
  T.sync();
  return !any;
}

// One vector equation (X or beta) by the defect-correction loop, as
// bt_solve (the mixing over the three components); u3 and f3 set by the
// caller.  Returns the status.
template <int G>
__device__ __noinline__ int bt_solve_vec(const Team& T, const BatchItem& I, BatchOut& O, int eq, double* hist,
                            unsigned char* smem_raw, BtShared& S) {
  const LevelView<double>& L = I.v64;
  const long n = bt_cells(L), ng = bt_ghosted(L);
  bt_fill_u3(T, I);
  const int m = I.m;
  int cyc = 0, ncol = 0, head = 0, status = 0;
  double rel = bt_norm_vec<G>(T, I, S);
  if (threadIdx.x == 0) {
    S.hist[0] = rel;
    if (T.rank == 0) hist[0] = rel;
  }
  __syncthreads();
  for (;;) {
    if (rel != rel) {
      status = 5;  // MG_ERR_NAN
      break;
    }
    if (rel <= I.tol) break;
    if (cyc >= I.max_cycles) {
      status = 3;  // MG_ERR_NOCONV
      break;
    }
    if (I.stall_window > 0 && cyc >= I.stall_window && rel > 0.95 * S.hist[cyc - I.stall_window]) {
      status = 4;  // MG_ERR_STALLED
      break;
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      if (m > 0 && cyc == 0)
        for (long q = T.start(); q < ng; q += T.stride()) I.aa[c * ng + q] = I.u3[c][q];
      for (long q = T.start(); q < ng; q += T.stride()) I.lv[0].e3[c][q] = 0.0f;
    }
    T.sync();
    bt_vcycle_vec<G>(T, I, smem_raw);
    // u += e, then the FP64 ghosts
    for (long q = T.start(); q < n; q += T.stride()) {
      int i, j, k;
      L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) I.u3[c][p] += (double)I.lv[0].e3[c][p];
    }
    T.sync();
    bt_fill_u3(T, I);
    bool mixstep = false;
    int mst = 0;
    if (m > 0) {
      AACols cols;
      cols.n = 0;
#pragma unroll
      for (int a = 0; a < AA_MAX; ++a) cols.slot[a] = 0;
      if (cyc > 0) {
        const int slot = head;
        head = (head + 1) % m;
        if (ncol < m) ++ncol;
        cols.n = ncol;
#pragma unroll
        for (int a = 0; a < AA_MAX; ++a)
          if (a < ncol) cols.slot[a] = (slot - ncol + 1 + a + m) % m;  // oldest first
      }
      mst = bt_mix(T, I, 3, cols, S);
      mixstep = cols.n > 0;
      if (mixstep) bt_fill_u3(T, I);
    }
    ++cyc;
    rel = bt_norm_vec<G>(T, I, S);
    if (mixstep && mst != 0) ncol = 0;  // degenerate history: restart the mixing
    if (threadIdx.x == 0 && cyc < BATCH_HIST) {
      S.hist[cyc] = rel;
      if (T.rank == 0) hist[cyc] = rel;
    }
    __syncthreads();
  }
  if (T.rank == 0 && threadIdx.x == 0) {
    O.status[eq] = status;
    O.cycles[eq] = cyc;
    O.rel[eq] = rel;
    O.ran |= 1 << eq;
  }
  return status;
}

// The report of an equation that stops at cycle 0 with rel = 0 (zero
// right-hand side and guess).
__device__ void bt_trivial(const Team& T, BatchOut& O, int eq, double* hist) {
  if (T.rank == 0 && threadIdx.x == 0) {
    O.status[eq] = 0;
    O.cycles[eq] = 0;
    O.rel[eq] = 0.0;
    O.ran |= 1 << eq;
    hist[0] = 0.0;
  }
}

// The xCFC sequence of mg_solve_cfc (Steps 1-6) for one problem; hist holds
// the four equations' histories.  Problems with momentum on a hierarchy
// whose vector levels do not fit are marked BATCH_GENERAL.
template <int G>
__device__ void bt_problem(const Team& T, const BatchItem& I, BatchOut& O, double* hist, unsigned char* smem_raw,
                           BtShared& S) {
  float* sm = reinterpret_cast<float*>(smem_raw);
  double* smd = reinterpret_cast<double*>(smem_raw + I.bc.fp64_at);
  const LevelView<double>& L = I.v64;
  const long n = bt_cells(L), ng = bt_ghosted(L);
  bool mf = true;  // momentum-free: X = beta = 0 exactly
  if (!I.psi_only) {
    mf = bt_momentum_free(T, I, S);
    if (!mf && !I.vec_ok) {
      if (T.rank == 0 && threadIdx.x == 0) O.status[0] = BATCH_GENERAL;
      return;
    }
    if (mf) {
      bt_trivial(T, O, 0, hist);
    } else {
      // Step 1: lap X + 1/3 grad div X = 8 pi S_i
      for (long q = T.start(); q < n; q += T.stride()) {
        int i, j, k;
        L.cell(q, i, j, k);
        const long p = L.idx(i, j, k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          I.u3[c][p] = I.X[c][q];
          I.f3[c][p] = 8.0 * PI_D * I.Si[c][q];
        }
      }
      T.sync();
      const int sx = bt_solve_vec<G>(T, I, O, 0, hist, smem_raw, S);
      for (long q = T.start(); q < ng; q += T.stride())
#pragma unroll
        for (int c = 0; c < 3; ++c) I.Xg[c][q] = I.u3[c][q];
      for (long q = T.start(); q < n; q += T.stride()) {
        int i, j, k;
        L.cell(q, i, j, k);
        const long p = L.idx(i, j, k);
#pragma unroll
        for (int c = 0; c < 3; ++c) I.X[c][q] = I.u3[c][p];
      }
      T.sync();
      {
        LevelView<double> Ld = I.v64;
        Ld.bc = BC_DIRICHLET;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) bt_fill(T, Ld, I.Xg[c], c);
      }
      T.sync();
      if (sx != 0) return;
    }
  }
  // Step 2: A~^2 from X (0 without momentum).  Step 3: eq. psi for psi - 1
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    I.u[p] = I.psi[q] + -1.0;
    I.s0[p] = I.U[q];
    double a2 = 0.0;
    if (!mf) {
      double A[6];
      aij_cell<G>(L, I.Xg[0], I.Xg[1], I.Xg[2], i, j, p, A);
      a2 = A[0] * A[0] + A[1] * A[1] + A[2] * A[2] + 2.0 * (A[3] * A[3] + A[4] * A[4] + A[5] * A[5]);
    }
    I.s1[p] = a2;
  }
  T.sync();
  const int st = bt_solve<G, EQ_PSI>(T, I, nullptr, I.s0, I.s1, O, 1, hist + BATCH_HIST, sm, smd, S);
  if (T.rank == 0 && threadIdx.x == 0) O.ran |= 1 << 1;
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    I.psi[q] = I.u[p] + 1.0;
    I.dpsi[p] = I.u[p];
  }
  T.sync();
  if (I.psi_only || st != 0) return;
  // Step 5: c = 2 pi (U + 2 S) psi^-2 + 7/8 A~^2 psi^-8, the equation
  // lap d - c d = c for d = alpha psi - 1
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    const double ip = 1.0 / (1.0 + I.dpsi[p]);
    const double ip2 = ip * ip;
    const double ip8 = (ip2 * ip2) * (ip2 * ip2);
    const double a2 = I.s1[p];
    const double c = 2.0 * PI_D * (I.U[q] + 2.0 * I.S[q]) * ip2 + 0.875 * a2 * ip8;
    I.f[p] = c;
    I.s1[p] = c;
    I.u[p] = I.alpha[q] * (1.0 + I.dpsi[p]) - 1.0;
  }
  T.sync();
  const int sa = bt_solve<G, EQ_LIN>(T, I, I.f, nullptr, I.s1, O, 2, hist + 2 * BATCH_HIST, sm, smd, S);
  if (T.rank == 0 && threadIdx.x == 0) O.ran |= 1 << 2;
  for (long q = T.start(); q < ng; q += T.stride()) I.dap[q] = I.u[q];
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    I.alpha[q] = (1.0 + I.u[p]) / (1.0 + I.dpsi[p]);
  }
  T.sync();
  if (sa != 0) return;
  if (mf) {
    // Step 6: the shift's right-hand side and guess are zero
    bt_trivial(T, O, 3, hist + 3 * BATCH_HIST);
    return;
  }
  // Step 6: s = alpha psi^-6 on every cell (the deviations' Robin ghosts
  // first), the source 16 pi s S_i + 2 A~_ij grad_j s, eq. beta
  bt_fill(T, L, I.dpsi, -1);
  bt_fill(T, L, I.dap, -1);
  T.sync();
  for (long q = T.start(); q < ng; q += T.stride()) {
    const double ip = 1.0 / (1.0 + I.dpsi[q]);
    const double ip2 = ip * ip;
    I.sg[q] = (1.0 + I.dap[q]) * (ip2 * ip2 * ip2 * ip);
  }
  T.sync();
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    const double Sv[3] = {I.Si[0][q], I.Si[1][q], I.Si[2][q]};
    double f[3];
    beta_rhs_cell<G>(L, I.Xg[0], I.Xg[1], I.Xg[2], I.sg, i, j, p, Sv, f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      I.f3[c][p] = f[c];
      I.u3[c][p] = I.beta[c][q];
    }
  }
  T.sync();
  bt_solve_vec<G>(T, I, O, 3, hist + 3 * BATCH_HIST, smem_raw, S);
  for (long q = T.start(); q < n; q += T.stride()) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) I.beta[c][q] = I.u3[c][p];
  }
  T.sync();
}

// Problem idx by team T (each block holds its own copy of the descriptor).
__device__ void bt_run(const Team& T, const BatchItem* items, BatchOut* outs, double* hist, int idx,
                       unsigned char* smem_raw, BatchItem& I, BtShared& S) {
  {
    const int* src = reinterpret_cast<const int*>(items + idx);
    int* dst = reinterpret_cast<int*>(&I);
    for (int w = threadIdx.x; w < (int)(sizeof(BatchItem) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  }
  BatchOut& O = outs[idx];
  if (T.rank == 0 && threadIdx.x == 0) {
    O.t_start = global_ns();
    O.ran = 0;
    for (int e = 0; e < 4; ++e) {
      O.status[e] = 0;
      O.cycles[e] = 0;
      O.rel[e] = 0.0;
    }
  }
  __syncthreads();
  double* h = hist + (long)idx * 4 * BATCH_HIST;
  if (I.geom == CART)
    bt_problem<CART>(T, I, O, h, smem_raw, S);
  else if (I.geom == CYL)
    bt_problem<CYL>(T, I, O, h, smem_raw, S);
  else
    bt_problem<SPH>(T, I, O, h, smem_raw, S);
  T.sync();
  if (T.rank == 0 && threadIdx.x == 0) O.t_end = global_ns();
}

// Problems are taken in the order order[0 ..] (the team's first).  Launched
// in clusters (of at most BATCH_TEAM blocks), a cluster takes the problems of at least
// team_cells cells together; at the first smaller one it splits, its rank 0
// keeping that problem, and from then on every block takes problems alone.
// A launch without clusters is all single blocks.
__global__ void __launch_bounds__(BATCH_THREADS, 1)
    k_batch_cfc(const BatchItem* __restrict__ items, BatchOut* __restrict__ outs, double* __restrict__ hist,
                const int* __restrict__ order, int count, unsigned int* __restrict__ next, long team_cells) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) BatchItem I;
  __shared__ BtShared S;
  int first = -1;
  const int csize = (int)cg::this_cluster().num_blocks();
  if (csize > 1) {
    const Team T{(int)cg::this_cluster().block_rank(), csize};
    for (;;) {
      if (T.rank == 0 && threadIdx.x == 0) S.item = (int)atomicAdd(next, 1u);
      T.sync();
      const int it = *T.at0(&S.item);
      T.sync();
      if (it >= count) return;
      const int idx = order[it];
      const LevelView<double>& v = items[idx].v64;
      if ((long)v.n0 * v.n1 * v.n2 < team_cells) {
        if (T.rank == 0) first = it;
        break;
      }
      bt_run(T, items, outs, hist, idx, smem_raw, I, S);
    }
  }
  const Team T{0, 1};
  for (;;) {
    int it = first;
    first = -1;
    if (it < 0) {
      if (threadIdx.x == 0) S.item = (int)atomicAdd(next, 1u);
      __syncthreads();
      it = S.item;
      __syncthreads();
    }
    if (it >= count) return;
    bt_run(T, items, outs, hist, order[it], smem_raw, I, S);
  }
}

size_t batch_smem_limit() {
  cudaFuncAttributes a{};
  int dev = 0, optin = 0;
  if (cudaFuncGetAttributes(&a, k_batch_cfc) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return optin > (int)a.sharedSizeBytes ? (size_t)optin - a.sharedSizeBytes : 0;
}

int batch_clusters(size_t smem, int team) {
  if (cudaFuncSetAttribute(k_batch_cfc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (team == 1) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_cfc, BATCH_THREADS, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n * sms;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(team);
  cfg.blockDim = dim3(BATCH_THREADS);
  cfg.dynamicSmemBytes = smem;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = team;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaOccupancyMaxActiveClusters(&n, k_batch_cfc, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int launch_batch_cfc(const BatchItem* items, BatchOut* outs, double* hist, const int* order, int count,
                     unsigned int* next, int clusters, int team, long team_cells, size_t smem, cudaStream_t st) {
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(clusters * team);
  cfg.blockDim = dim3(BATCH_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = team;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = team > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_batch_cfc, items, outs, hist, order, count, next, team_cells) == cudaSuccess
             ? 0
             : 1;
}

}  // namespace gmg
