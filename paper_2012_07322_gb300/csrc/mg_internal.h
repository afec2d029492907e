// Host-side declarations shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <utility>

#include "mg_dev.cuh"

struct mg_hierarchy;

namespace gmg {

// Kernel launch with programmatic stream serialisation: the kernel may be
// scheduled before its predecessor in the stream has finished and waits for
// it in pdl_entry().  Inside a captured graph the dependency becomes a
// programmatic edge.
template <typename... K, typename... A>
inline void launch_k(void (*k)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Record a message for mg_last_error on the calling thread; returns status.
int set_last_error(int status, const char* msg);

// Move a hierarchy's work to another stream (serving workers share cached
// hierarchies; captured graphs are stream-independent).
void hier_set_stream(mg_hierarchy* h, cudaStream_t st);
// Run the hierarchy's cycle loops on the host (one stream synchronisation
// per cycle) instead of as device-side loops.  Device-side loops save the
// per-cycle round trip of one solve, but several of them on concurrent
// streams ran slower than host loops: 64 small 2D solves on 16 streams took
// 304 ms against 181 ms.  The request server's slots therefore use host loops.
void hier_set_host_loop(mg_hierarchy* h, bool on);

// Count of kernel launches issued by the library (all hierarchies).
// Up to three field pointers passed by value to a kernel (entries past
// the field count repeat the first).
template <typename T>
struct Ptr3 {
  T* p[3];
  // selected, not indexed: a run-time index into a kernel parameter array
  // would copy the array to local memory in every thread
  __host__ __device__ __forceinline__ T* at(int c) const { return c == 0 ? p[0] : (c == 1 ? p[1] : p[2]); }
  template <typename P>
  static Ptr3 of(const P* a, int n) {
    Ptr3 o{};
    for (int c = 0; c < 3; ++c) o.p[c] = a[c < n ? c : 0];
    return o;
  }
};
template <typename T>
struct CPtr3 {
  const T* p[3];
  __host__ __device__ __forceinline__ const T* at(int c) const { return c == 0 ? p[0] : (c == 1 ? p[1] : p[2]); }
  template <typename P>
  static CPtr3 of(const P* a, int n) {
    CPtr3 o{};
    for (int c = 0; c < 3; ++c) o.p[c] = a[c < n ? c : 0];
    return o;
  }
};
template <typename T>
inline long ghost_count_host(const LevelView<T>& L) {
  const long nk = L.n2 + 2 * L.three;
  return 2L * (L.n1 + 2) * nk + 2L * L.n0 * nk + (L.three ? 2L * L.n0 * L.n1 : 0L);
}

void count_launch(int n = 1);
unsigned long long launch_count();

template <typename T>
void launch_smooth_scalar(const LevelView<T>& L, int kind, T* u, const T* f, const T* s0, const T* s1,
                          int colour, cudaStream_t st);
template <typename T>
void launch_fill_ghosts(const LevelView<T>& L, T* u, int comp, cudaStream_t st);
// The ghosts of ncomp fields in one launch (vector components when vec).
template <typename T>
void launch_fill_ghosts3(const LevelView<T>& L, T* const u[3], int ncomp, int vec, cudaStream_t st);
// Row layout of every level array: ROW_PAD - 1 padding cells, the low
// ghost, the n0 interior cells, the high ghost, then padding to a multiple
// of ROW_PAD cells.  Interior rows (i = 0) and row strides are then 16-byte
// aligned for FP32 and FP64 arrays alike, and a row can be read in 16-byte
// pieces from i = -ROW_PAD to i = n0 + ROW_PAD - 1 without leaving it.
constexpr long ROW_PAD = 4;
inline long row_stride(int n0) { return (n0 + 2 * ROW_PAD + ROW_PAD - 1) / ROW_PAD * ROW_PAD; }

// One red-black sweep in one launch (3D linear scalar equations on levels
// tiled by 64 x 8 columns: n0 a multiple of 64, n1 of 8; Cartesian,
// cylindrical and spherical), out of place: uin -> uout, which must not
// alias; only the interior of uout is written.  Returns false when it does
// not apply.  On cylindrical and spherical levels it is used from
// FUSED_CURV_CELLS cells on.  Below that the colour passes win: measured on
// the 128 x 64 x 64 xCFC solve, a block marching a short chunk of phi planes
// behind its staging pipeline took as long as the two colour passes of a
// sweep, and a block staging all planes of its chunk at once (one copy
// latency per sweep) made the solve slower by 9-11 ms, since programmatic
// dependent launch hides most of each colour pass's launch latency while
// the one-launch sweep's staging is a serial prologue.
// Tensor maps of the one-launch sweep's inputs, for staging its planes with
// the tensor memory accelerator (cp.async.bulk.tensor, one thread per block,
// mbarrier completion): FP32 Cartesian levels of 128-cell columns.  Each map
// views a level array as (padded row, row, plane) with a box of one staged
// plane (136 x 20 values); err (device) is set when a wait for a staged
// plane exceeds its iteration limit (the launch then stops early).
struct SweepMaps {
  CUtensorMap u, f, c;
  unsigned long long* err;
  int on;
};
// Encodes the map of one FP32 level array for the sweep's plane box; false
// when the driver entry point is missing or rejects the layout.
bool sweep_plane_map(CUtensorMap* m, const float* base, const LevelView<float>& L);
// Whether the level's sweeps stage with tensor maps (FP32, Cartesian,
// 128-cell columns).
bool sweep_uses_maps(const LevelView<float>& L);
template <typename T>
bool launch_sweep_fused(const LevelView<T>& L, const T* uin, T* uout, const T* f, const T* c, cudaStream_t st,
                        const SweepMaps* maps = nullptr);
template <typename T>
void init_fused_sweep_attributes();
constexpr long FUSED_CURV_CELLS = 1L << 22;
template <typename T>
inline bool fused_sweep_applies(const LevelView<T>& L) {
  if (!(L.three && L.n0 % 64 == 0 && L.n1 % 8 == 0 && L.n2 >= 4)) return false;
  return L.geom == CART || (long)L.n0 * L.n1 * L.n2 >= FUSED_CURV_CELLS;
}
// Ghost push of the vector smoother's colour passes.  With a table, the
// pass of component c also rewrites, at its end, every ghost of c whose
// source cell it has just updated, in place of a ghost-fill launch after
// it.  The entries of block b (blocks numbered x fastest) are ent[off[b]]
// .. ent[off[b + 1] - 1]: x = the ghost's index in the level array, y = 2 *
// (the source cell's thread in the block) + 1 when the ghost is the negated
// source.  A 3D pass with a table puts planes k and k + n2 / 2 in one block
// (thread z), so that a pole ghost and the same-colour cell that reads it
// in the same pass belong to one block, which reads before it writes.
struct GhostPush {
  const int* off = nullptr;
  const int2* ent = nullptr;
};
template <typename T>
void launch_smooth_vec(const LevelView<T>& L, T* V[3], const T* f, int comp, int colour, cudaStream_t st,
                       GhostPush gp = GhostPush{});
// Block count of a pass with a ghost-push table, and the block of that pass
// which updates cell (i, j, k) with the cell's slot in its new values.
template <typename T>
int push_blocks(const LevelView<T>& L);
// Cells a thread of the vector colour pass updates when it pushes ghosts
// (2 on 3D levels of 2^19 cells and more, whose pass then fits one wave).
template <typename T>
int vec_cells_per_thread(const LevelView<T>& L);
template <typename T>
void push_slot(const LevelView<T>& L, int i, int j, int k, int* block, int* slot);
// Source of every ghost of vector component comp, in the enumeration of
// the ghost fill: gc[8 g ..] = ghost i, j, k, source i, j, k, ghost index,
// source index; fac[g] = the product of the boundary factors.
template <typename T>
void launch_ghost_sources(const LevelView<T>& L, int comp, int* gc, T* fac, cudaStream_t st);
// r = f - L(u) into r (nullable) and, rounded to FP32, into r32 (nullable);
// red (nullable) receives the norms of the finest-level stopping rule; for
// eq. psi, k32 (nullable) receives the linearisation 2 pi U (1+u)^-2 +
// 7/8 A2 (1+u)^-8 at the same u, rounded to FP32.
template <typename T>
void launch_residual_scalar(const LevelView<T>& L, int kind, const T* u, const T* f, const T* s0,
                            const T* s1, T* r, unsigned long long* red, int weighted, cudaStream_t st,
                            float* r32 = nullptr, float* k32 = nullptr);
template <typename T>
void launch_residual_vec(const LevelView<T>& L, T* const V[3], const T* const f[3], T* const r[3],
                         unsigned long long* red, int weighted, cudaStream_t st, float* const r32[3] = nullptr);
template <typename T>
void launch_apply_scalar(const LevelView<T>& L, int kind, const T* u, const T* s0, const T* s1, T* out,
                         int add, cudaStream_t st);
template <typename T>
void launch_apply_vec(const LevelView<T>& L, T* const V[3], T* const out[3], int add, cudaStream_t st);
template <typename T>
void launch_restrict(const LevelView<T>& F, const LevelView<T>& C, int nf, const T* const a[4],
                     T* const b[4], T* const copy[3], cudaStream_t st);
template <typename T>
void launch_prolong(const LevelView<T>& F, const LevelView<T>& C, T* u, const T* uH, const T* uhH, int comp,
                    cudaStream_t st);
// Kwak prolongation of ncomp fields in one launch (uhH may be null).
template <typename T>
void launch_prolong3(const LevelView<T>& F, const LevelView<T>& C, T* const u[3], const T* const uH[3],
                     const T* const uhH[3], int ncomp, int vec, cudaStream_t st);
// Down leg of the FP32 correction cycle: residual of (L - K) e = f (or the
// vector operator) restricted into fc, K into Kc (if non-null), ec zeroed.
void launch_resid_restrict32(const LevelView<float>& F, const LevelView<float>& C, int vec, float* const e[3],
                             float* const f[3], const float* K, float* const fc[3], float* const ec[3], float* Kc,
                             cudaStream_t st);
template <typename T>
void launch_coarse_scalar(const LevelView<T>& L, int kind, T* u, const T* f, const T* s0, const T* s1,
                          int max_sweeps, cudaStream_t st);
template <typename T>
void launch_coarse_vec(const LevelView<T>& L, T* V[3], const T* const f[3], int max_sweeps, cudaStream_t st);
// u -= mean(u) over the interior (the Neumann gauge); the nparts block sums
// are computed first unless have_part (left by launch_add_correction).
template <typename T>
void launch_sub_mean(const LevelView<T>& L, T* u, double* part, int nparts, cudaStream_t st,
                     bool have_part = false);
template <typename A, typename B>
void launch_copy_in(const LevelView<B>& L, const A* src, B* dst, A shift, cudaStream_t st);
template <typename A, typename B>
void launch_copy_out(const LevelView<A>& L, const A* src, B* dst, A shift, cudaStream_t st);
template <typename A, typename B>
void launch_convert(const LevelView<A>& L, const A* src, B* dst, cudaStream_t st);
// u += e over the interior of ncomp fields; with part non-null also the
// nparts block sums of the updated field 0 for launch_sub_mean.
template <typename T>
void launch_add_correction(const LevelView<double>& L, int ncomp, double* const u[3], const T* const e[3],
                           cudaStream_t st, double* part = nullptr, int nparts = 0);

// xCFC and divergence-cleaning pointwise kernels (mg_xcfc.cu).
void launch_xcfc_a2(const LevelView<double>& L, double* const X[3], double* A2, cudaStream_t st);
void launch_xcfc_alpha_coef(const LevelView<double>& L, const double* U, const double* S, const double* A2,
                            const double* dpsi, double* c, cudaStream_t st);
void launch_xcfc_beta_rhs(const LevelView<double>& L, double* const X[3], const double* dpsi,
                          const double* dap, double* sg, double* const Si[3], double* const f[3],
                          cudaStream_t st);
void launch_scale_into(const LevelView<double>& L, const double* src, double a, double* dst, cudaStream_t st);
void launch_div_central(const LevelView<double>& L, double* const B[3], double* div, double* part, int nparts,
                        cudaStream_t st);
void launch_div_norms(const LevelView<double>& L, const double* div, double* part, int nparts,
                      unsigned long long* red, cudaStream_t st);
// Curvilinear divergence cleaning: divergence from ghosted B with weighted
// block sums, weighted-mean removal, gradient update of ghost-free B.
void launch_div_curv(const LevelView<double>& L, double* const Bg[3], double* div, double* part, int nparts,
                     cudaStream_t st);
void launch_sub_wmean_into(const LevelView<double>& L, const double* div, const double* part, int nparts,
                           double wsum, double* b, cudaStream_t st);
void launch_grad_update_curv(const LevelView<double>& L, const double* phi, double* const B[3], cudaStream_t st);
void launch_sub_mean_into(const LevelView<double>& L, const double* div, const double* part, int nparts,
                          double* b, cudaStream_t st);
void launch_grad_update(const LevelView<double>& L, const double* phi, double* const B[3], cudaStream_t st);
// Exact-projection cleaning (Cartesian, n >= 4): the parity classes of div
// minus their class means into a class-major buffer (nparts blocks per
// class; part holds nparts x 2^d doubles), and B -= grad Phi with mirrored
// Phi ghosts from the class-major Phi (phi_out nullable, ghost-free).
void launch_class_gather(const LevelView<double>& L, const double* div, double* part, int nparts, double* dst,
                         cudaStream_t st);
void launch_grad_update_exact(const LevelView<double>& L, const double* phis, double* const B[3], double* phi_out,
                              cudaStream_t st);
void launch_xcfc_ap_init(const LevelView<double>& L, const double* alpha, const double* dpsi, double* dap,
                         cudaStream_t st);
void launch_xcfc_alpha_out(const LevelView<double>& L, const double* dap, const double* dpsi, double* alpha,
                           cudaStream_t st);

// Two-level composite grid (mg_amr.cu): the refined patch covers base cells
// a <= I < b (b[2] = 1 in 2D); bit 2 d + (side > 0) of cf marks the patch
// faces that are coarse-fine interfaces (the others lie on the domain
// boundary and take its rules).
struct AmrBox {
  int a[3], b[3];
  int cf;
};
void launch_amr_cf_ghosts(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, double* up,
                          const double* ub, cudaStream_t st);
void launch_amr_smooth(const LevelView<double>& L, int kind, double* u, const double* f, const double* s0,
                       const double* s1, int colour, cudaStream_t st);
// r = f - L(u) on the patch (f nullable; apply: r = L(u)), norms into red.
void launch_amr_patch_resid(const LevelView<double>& L, int kind, const double* u, const double* f, const double* s0,
                            const double* s1, double* r, unsigned long long* red, int apply, cudaStream_t st);
void launch_amr_restrict(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, const double* up,
                         const double* rp, double* ub, double* rr, cudaStream_t st);
void launch_amr_flux_corr(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box,
                          const double* up, const double* ub, double* corr, cudaStream_t st);
// Base level of the composite grid: mode 0 the FAS right-hand side f, 1 the
// composite residual norms of the uncovered cells into red, 2 the composite
// operator into f (0 on covered cells).
void launch_amr_base(const LevelView<double>& B, const AmrBox& box, int kind, const double* u, const double* s0,
                     const double* s1, const double* f0, const double* rr, const double* corr, double* f,
                     unsigned long long* red, int mode, cudaStream_t st);
void launch_amr_prolong(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, const double* e,
                        double* up, cudaStream_t st);
// Composite unknowns <-> flat vector x (patch cells, then the uncovered
// base cells at the ghosted offsets bmap[0 .. nbase - 1]).
void launch_amr_flat(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, double* up,
                     double* ub, const int* bmap, long nbase, double* x, int to_flat, cudaStream_t st);
// out = a - b over the interior (ghosted arrays of L).
void launch_amr_diff(const LevelView<double>& L, const double* a, const double* b, double* out, cudaStream_t st);

// Anderson mixing (mg_accel.cu): live ring slots of the difference columns
// in age order (the newest last).
constexpr int AA_MAX = 16;
constexpr int AA_BLOCKS = 304;  // 2 x 152 SMs: partial sums of the dot products
struct AACols {
  int n;
  int slot[AA_MAX];
};
// Device scratch of the mixing step (doubles): AA_BLOCKS x 2 AA_MAX partial
// sums, the Gram matrix (AA_MAX x AA_MAX), the weights (AA_MAX) and a
// finished-block counter (zero between launches).
constexpr size_t AA_SCRATCH_DOUBLES = (size_t)AA_BLOCKS * 2 * AA_MAX + AA_MAX * AA_MAX + AA_MAX + 1;
struct AAScratch {
  double* part;
  double* M;
  double* gamma;
  unsigned int* done;
};
inline AAScratch aa_scratch(double* s) {
  AAScratch o;
  o.part = s;
  o.M = s + (size_t)AA_BLOCKS * 2 * AA_MAX;
  o.gamma = o.M + AA_MAX * AA_MAX;
  o.done = reinterpret_cast<unsigned int*>(o.gamma + AA_MAX);
  return o;
}
// History columns TC: double, or float in mixed precision.  status gets the
// least-squares outcome (0 solved, 1 degenerate) when cols.n > 0.  With
// dcols non-null the live columns are read from device memory instead of
// cols (the device-side cycle loop), and the combination does nothing when
// they are none.
template <typename TC>
void launch_aa_update_dots(const LevelView<double>& L, int ncomp, long stride, double* const g[3], double* x,
                           double* fprev, double* gprev, TC* dF, TC* dG, const AACols& cols, double* scratch,
                           unsigned long long* status, cudaStream_t st, const AACols* dcols = nullptr);
template <typename TC>
void launch_aa_combine(const LevelView<double>& L, int ncomp, long stride, double* const u[3], double* x,
                       const TC* dG, const AACols& cols, const double* scratch, const unsigned long long* status,
                       cudaStream_t st, const AACols* dcols = nullptr);

// Device-side cycle loop: the state one solve's loop keeps on the device
// (cycle count, status, the mixing ring and the live columns of the next
// mixing step, the residual history) and the step that ends every cycle:
// it reads the stopping norms, records them, applies the stopping rule of
// the host loop (non-finite, tol, max_cycles, stall window), advances the
// mixing ring and sets the condition of the enclosing while node.
struct LoopState {
  int cyc, status, stop, ncol, head, mixstep, pad0, pad1;
  AACols cols;
  double rel;
  double hist[1024];
};
struct LoopParams {
  double tol;
  int max_cycles, stall_window, m;
};
void launch_loop_decide(LoopState* S, const unsigned long long* red, const LoopParams& P,
                        cudaGraphConditionalHandle h, int first, cudaStream_t st);

// One-block FP32 correction V-cycle over the coarse levels (mg_block.cu):
// the levels l0 .. l0 + nl - 1 of a hierarchy, the last the coarsest, all
// held in the block's shared memory (same ghosted layout as in HBM).
constexpr int BC_MAX = 8;                     // levels one block cycle may span
constexpr long BLOCK_CYCLE_CELLS = 4096;       // levels this small run in the block cycle
constexpr size_t BC_SMEM_MAX = 200 * 1024;     // dynamic shared memory of the block cycle
struct BlockLevel32 {
  LevelView<float> v;        // boundary rule applied
  int e[3], f32[3], r32[3];  // offsets (floats) of correction, right-hand side, residual in shared memory
  const float* k32;          // c of (L - c) e = f in HBM, null without
  int ti_at, tj_at, k_at;    // offsets (floats) of the level's coefficient tables and of c in shared memory
};
struct BlockCycle32 {
  int nl, vec, nu1, nu2, coarse_sweeps;
  BlockLevel32 lv[BC_MAX];
  LevelView<double> c64;  // the coarsest level, boundary rule applied
  int cu[3], cf[3], ck;   // offsets (doubles, from fp64_at) of the FP64 coarsest solve; ck < 0: no c
  long fp64_at;           // byte offset of the FP64 area in shared memory
  const double* cinv;     // vector equations: inverse of the coarsest operator (transposed), or null
  int cn;                 // its order (3 x coarsest cells); scalar equations: the cells
  const double* cA;       // scalar equations: the coarsest operator, A[col * cn + r], or null
  long ng0;               // ghosted size of level l0
  const float* f_in[3];   // level l0 right-hand side in HBM
  float* e_out[3];        // level l0 correction in HBM (written at the end)
  size_t smem;            // dynamic shared memory bytes
};
void launch_block_vcycle32(const BlockCycle32& P, int geom, cudaStream_t st);
void init_block_cycle_attributes();
// The largest coarsest vector system solved exactly (3 x cells).
constexpr int BC_CINV_MAX = 768;
// The largest coarsest scalar level swept with dense operator rows (cells).
constexpr int BC_CMAT_MAX = 64;
// Columns of the coarsest scalar operator (the flux-form Laplacian with its
// boundary rule folded in) into A[col * n + r], n = coarsest cells; scratch
// holds n ghosted fields.
void launch_coarse_assemble_scalar(const LevelView<double>& L, double* scratch, double* A, int n, cudaStream_t st);
// Columns of the coarsest vector operator (L with its boundary rule) into
// A[col * n + r], n = 3 x coarsest cells; scratch holds 3 n ghosted fields.
void launch_coarse_assemble_vec(const LevelView<double>& L, double* scratch, double* A, int n, cudaStream_t st);

// Persistent batched xCFC solves (mg_batch.cu): one thread block (or a
// cluster) takes one problem at a time from a shared queue and runs its
// whole solve (Steps 1-6 of the xCFC order, mixed precision, with mixing),
// every phase separated by barriers instead of kernel boundaries.
constexpr int BATCH_THREADS = 512;
constexpr int BATCH_MAX_LEVELS = 16;
constexpr int BATCH_HIST = 1024;  // residual history entries per equation (the reports' length)
// Status of a problem whose X and beta equations need vector solves (its
// momentum sources or vector guesses are not all zero) on a hierarchy whose
// vector levels do not fit the kernel: the host runs it through
// mg_solve_cfc after the launch.
constexpr int BATCH_GENERAL = -1;
struct BatchLevel {
  LevelView<float> v;  // Robin rule applied
  float *e, *f32, *r32, *k32;
  float *e3[3], *f3[3];  // vector equations: the components' correction and right-hand side
};
struct BatchItem {
  int geom, nl;  // nl levels run phase by phase; level nl is the first of the one-block cycle
  int nlev, nu1, nu2, m, max_cycles, stall_window, psi_only;
  int vec_ok, nlv;  // vector equations solvable in the kernel; their first one-block-cycle level
  double tol;
  LevelView<double> v64;                  // level 0, Robin rule applied
  BatchLevel lv[BATCH_MAX_LEVELS + 1];    // levels 0 .. max(nl, nlv) (HBM arrays)
  BlockCycle32 bc;                        // levels nl .. nlev - 1 (Robin rule, c present)
  BlockCycle32 bcv;                       // vector equations: levels nlv .. nlev - 1 (Dirichlet rule)
  double *u, *f, *s0, *s1, *dpsi, *dap;   // level 0, ghosted
  double *u3[3], *f3[3];                  // level 0 components (u3[0] = u, f3[0] = f)
  double *Xg[3], *sg;                     // X with its ghosts; alpha psi^-6 (ghosted)
  double* aa;  // mixing: iterate, previous f and g, then m columns each of dF and dG (FP32), per component
  const double *U, *S, *Si[3];            // the caller's arrays (interior order)
  double *psi, *alpha, *beta[3], *X[3];
};
struct BatchOut {
  int status[4], cycles[4];
  int ran;  // bit e: equation e (X, psi, alpha psi, beta) was solved and its report is set
  double rel[4];
  unsigned long long t_start, t_end;  // %globaltimer (ns) when the problem was taken and finished
};
// Blocks a cluster of the batch kernel (team = blocks per cluster, 1 for
// none) holds; the clusters of that shape co-resident on the device (0 when
// it does not fit).
constexpr int BATCH_TEAM = 8;                     // the largest cluster a launch may use
constexpr int BATCH_TEAM_DEFAULT = 2;
constexpr long BATCH_TEAM_CELLS = 16384;  // default: grids this large run on a whole cluster
int batch_clusters(size_t smem, int team);
// Dynamic shared memory a block of the batch kernel may take beside its
// static arrays (0 when unknown).
size_t batch_smem_limit();
// One launch over count problems (items in device memory, taken in the
// order order[0 ..]) on clusters x team blocks; problems of at least
// team_cells cells are run by a whole cluster.  hist receives 4 x
// BATCH_HIST residual histories per problem (X, psi, alpha psi, beta);
// next is a zeroed counter.  Returns 0, or 1 when the launch was refused.
int launch_batch_cfc(const BatchItem* items, BatchOut* outs, double* hist, const int* order, int count,
                     unsigned int* next, int clusters, int team, long team_cells, size_t smem, cudaStream_t st);

}  // namespace gmg
