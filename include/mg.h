/*
 * mg.h -- C ABI of the GB300 multigrid solver for the xCFC metric equations
 * and elliptic divergence cleaning of Gmunu (arXiv:2012.07322).
 *
 * What is solved (section / equation of the paper):
 *   - the xCFC system, Sec. 2.6, eqs. (X), (psi), (alpha), (beta), (Aij), in
 *     the solve order Steps 1-6 of Sec. 2.6, with the outer conditions of
 *     eq. (bc) and the Robin condition of eq. (robin) on the deviations
 *     psi - 1 and alpha psi - 1;
 *   - elliptic divergence cleaning, Sec. 2.2, eqs. (poisson) and
 *     (update_bfield), on Cartesian grids;
 * each by the non-linear cell-centred multigrid of Sec. 2.7: the flux-form
 * discretisation of Sec. 2.7.1, red-black Newton-Gauss-Seidel smoothing
 * (eq. ngs_iteration), piecewise-constant restriction and Kwak prolongation
 * (Sec. 2.7.3), in FAS V(nu1, nu2) cycles.
 *
 * Conventions shared by every entry point:
 *   - Arrays are contiguous FP64, cell-centred, WITHOUT ghost cells,
 *     dimension 0 fastest: element (i, j, k) is at i + n0 * (j + n1 * k).
 *     2D grids have no dimension 2 (axisymmetric cylindrical (R, z) and
 *     spherical (r, theta), or planar Cartesian (x, y)).
 *   - Vector fields are given by their orthonormal (physical) components:
 *     (x, y, z), (R, z, phi) or (r, theta, phi).
 *   - Pointers are DEVICE pointers on the hierarchy's device unless a
 *     function says otherwise (MG_HOST_POINTERS).  The caller owns them and
 *     keeps them valid until the call returns; the library never frees them.
 *   - Every function returns an mg_status.  No exception crosses the ABI.
 *     On an error a solve leaves its output arrays holding the last iterate.
 *   - Calls on one hierarchy are serialised on its stream and block until
 *     their result is known; different hierarchies are independent.
 */
#ifndef GMUNU_MG_H
#define GMUNU_MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status */
typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,   /* bad descriptor or argument */
  MG_ERR_OOM = 2,       /* device allocation failed */
  MG_ERR_NOCONV = 3,    /* max_cycles reached before tol */
  MG_ERR_STALLED = 4,   /* no 5 % residual gain over stall_window cycles */
  MG_ERR_NAN = 5,       /* a non-finite residual or source was met */
  MG_ERR_CUDA = 6,      /* a CUDA runtime call failed */
  MG_ERR_BUSY = 7,      /* admission refused (request queue) */
  MG_ERR_NOTFOUND = 8   /* unknown ticket */
} mg_status;

/* Human-readable name of a status code (static string). */
const char* mg_strerror(int status);

/* Detail of the last error raised on the calling thread (static buffer;
 * empty if none). */
const char* mg_last_error(void);

/* -------------------------------------------------------- descriptor */
enum { MG_CART = 0, MG_CYL = 1, MG_SPH = 2 };             /* geometry */
enum { MG_FP64 = 0, MG_MIXED = 1 };                        /* precision */
enum { MG_MIXED_4PT = 0, MG_MIXED_CORNER = 1 };            /* mixed derivative */
enum { MG_BC_ROBIN = 0, MG_BC_DIRICHLET = 1, MG_BC_NEUMANN = 2 };
enum { MG_EQ_PSI = 0, MG_EQ_LIN = 1, MG_EQ_VEC = 2 };      /* equation kinds */
enum { MG_CYCLE_V = 0, MG_CYCLE_FMG = 1 };                 /* iteration */
enum { MG_DIVB_COMPACT = 0, MG_DIVB_EXACT = 1 };           /* div-B cleaning */

/*
 * Grid and solver settings.
 *   ndim      2 or 3.
 *   geom      MG_CART, MG_CYL (R, z[, phi]) or MG_SPH (r, theta[, phi]).
 *   n[d]      cells per dimension, each a power of two >= 2 (n[2] ignored
 *             in 2D).  The hierarchy halves every dimension while all are
 *             even and >= 4 (so the coarsest has >= 2 cells per dimension).
 *   lo, hi    domain.  Spherical: lo = (0, 0[, 0]), hi = (r_max, pi[, 2 pi]).
 *             Cylindrical: lo[0] = 0, and in 3D lo[2] = 0, hi[2] = 2 pi.
 *   precision MG_FP64, or MG_MIXED: FP32 smoothing / restriction /
 *             prolongation inside an FP64 defect-correction loop (the FP64
 *             residual, non-linear sources, coarsest solve and norm).
 *   nu1, nu2  pre / post smoothing sweeps (the paper uses 2 and 2).
 *   max_cycles, tol   stop when rel <= tol (see mg_solve_report) or after
 *             max_cycles V-cycles (MG_ERR_NOCONV).
 *   mixed_deriv   MG_MIXED_4PT (four-corner stencil) or MG_MIXED_CORNER
 *             (the block-corner stencil of Sec. 2.7.1, used on every cell).
 *   stall_window  cycles over which a 5 % gain is required (0: off).
 *   accel_depth   0: plain V-cycles (the paper's iteration).  m in 1..16:
 *             Anderson mixing of depth m over the V-cycle map (not in the
 *             paper): with f = G(u) - u the change one cycle G makes,
 *             u <- G(u) - dG gamma, gamma = argmin |f - dF gamma| over the
 *             last m differences dF, dG of f and G(u).  Point smoothing
 *             converges slowly on spherical grids (Sec. 2.7.2 notes it);
 *             the mixing restores a rate of tens of cycles.  Each mixed
 *             iteration is one V-cycle and counts as one cycle.
 *   cycle     MG_CYCLE_V: FAS V(nu1, nu2) cycles.  MG_CYCLE_FMG: full
 *             multigrid cycles (the cycle Sec. 4.2 times; the paper does not
 *             spell it out, the FAS form is used): the current solution and
 *             FAS sources restricted to every level, the coarsest solved,
 *             then per level upward the FAS correction from below and one
 *             V-cycle from that level.  In MG_MIXED the FP32 correction
 *             equation gets the same structure from a zero correction.
 *             One FMG cycle counts as one cycle.
 *   divb_variant  MG_DIVB_COMPACT: mg_clean_divB solves the paper's compact
 *             Poisson equation (Sec. 2.2, eq. poisson).  MG_DIVB_EXACT
 *             (Cartesian grids with every n >= 4; not the paper's method):
 *             it solves div_c grad_c Phi = b, the operator the update of
 *             eq. (update_bfield) applies, so that the cleaned field's
 *             central divergence is exactly removed up to one constant per
 *             parity class of cells (see mg_clean_divB).
 */
typedef struct {
  int ndim;
  int geom;
  int n[3];
  double lo[3];
  double hi[3];
  int precision;
  int nu1, nu2;
  int max_cycles;
  double tol;
  int mixed_deriv;
  int stall_window;
  int accel_depth;
  int cycle;
  int divb_variant;
} mg_grid_desc;

#define MG_HIST 1024

/*
 * Per-solve report.  rel = max_i |w_i r_i| / max_i |w_i S_i(u)| over the
 * finest cells (and components), r = f - L(u) the residual, S the source
 * of the equation as the paper writes it, w = r^2 sin(theta) (spherical),
 * R (cylindrical), 1 (Cartesian).  hist[0] is rel of the initial guess,
 * hist[c] after c cycles (outer iterations in MG_MIXED).
 */
typedef struct {
  int status;
  int cycles;
  double rel;
  int nhist;
  double hist[MG_HIST];
  double ms;             /* wall time of the solve */
  int64_t cell_updates;  /* smoother cell updates (all levels) */
} mg_solve_report;

typedef struct mg_hierarchy mg_hierarchy;

/* Device bytes mg_create_hierarchy would allocate for desc (for admission). */
int mg_hierarchy_bytes(const mg_grid_desc* desc, size_t* bytes);

/*
 * Validate desc and allocate every level, coefficient table and work array
 * on the current CUDA device.  cuda_stream is a cudaStream_t (NULL: the
 * legacy default stream); all work of the hierarchy is enqueued on it.
 * The hierarchy owns its allocations; mg_destroy_hierarchy frees them.
 * With a default stream (NULL, legacy or per-thread) the work runs on a
 * stream the hierarchy owns, ordered after the work already queued on the
 * default stream at each call (default streams cannot be captured into
 * the CUDA graphs the cycle replays).
 */
int mg_create_hierarchy(const mg_grid_desc* desc, void* cuda_stream, mg_hierarchy** out);
int mg_destroy_hierarchy(mg_hierarchy* h);

/* Number of levels of the hierarchy (finest = 0). */
int mg_num_levels(const mg_hierarchy* h, int* nlev);

/* ------------------------------------------------------------- xCFC */

/* Sources of the xCFC equations (Sec. 2.6), held fixed during the solve
 * (Step 4, the primitive recovery, is the caller's): U = U~ = psi^6 U,
 * S = S~ = psi^6 gamma_ij S^ij, Si = S~_i (orthonormal components). */
typedef struct {
  const double* U;
  const double* S;
  const double* Si[3];
} mg_cfc_sources;

/* Metric fields: initial guess in (flat: psi = alpha = 1, beta = X = 0, or
 * a warm start), solution out. */
typedef struct {
  double* psi;
  double* alpha;
  double* beta[3];
  double* X[3];
} mg_cfc_fields;

enum {
  MG_CFC_PSI_ONLY = 1,        /* solve eq. psi only with A~_ij = 0 */
  MG_HOST_POINTERS = 2        /* sources / fields are host memory */
};

typedef struct {
  mg_solve_report eq[4];      /* X, psi, alpha psi, beta */
  double ms;                  /* total wall time */
} mg_cfc_report;

/*
 * The xCFC solve order (Steps 1-6, Sec. 2.6): solve eq. (X) for X, form
 * A~_ij (eq. Aij), solve eq. (psi), form the alpha-psi coefficient
 * 2 pi (U + 2 S) psi^-2 + 7/8 A~^2 psi^-8, solve eq. (alpha) for alpha psi,
 * form the shift source 16 pi alpha psi^-6 S_i + 2 A~_ij grad_j(alpha psi^-6),
 * solve eq. (beta), and return alpha = (alpha psi) / psi.
 * flags: MG_CFC_PSI_ONLY, MG_HOST_POINTERS.  rep may be NULL.
 */
int mg_solve_cfc(mg_hierarchy* h, const mg_cfc_sources* src, mg_cfc_fields* io, int flags,
                 mg_cfc_report* rep);

/* Launch shape of mg_solve_cfc_batch (NULL, or 0 in a field: the default). */
typedef struct {
  int team;            /* blocks of a cluster that run one large problem: 1, 2 (default), 4 or 8 */
  int64_t team_cells;  /* grids of at least this many cells run on a cluster (default 16384) */
} mg_batch_opts;

typedef struct {
  double kernel_ms;   /* the persistent launch (CUDA events) */
  int blocks;         /* thread blocks it ran */
  int team;           /* blocks of a cluster that run one large problem together (1: none) */
  int persistent;     /* problems solved inside the launch */
  int general;        /* problems passed on to mg_solve_cfc afterwards */
} mg_batch_report;

/*
 * count independent xCFC solves (the same Steps as mg_solve_cfc) in ONE
 * persistent launch: thread blocks take problems from a queue, longest
 * first (cells x the cycles of the problem's previous batched solve), and
 * run a problem's whole solve (eq. X, A~^2, eq. psi, the alpha-psi
 * coefficient, eq. alpha, the shift source, eq. beta, alpha = (alpha psi) /
 * psi), every phase of its V-cycles, residuals and mixing steps separated
 * by barriers.  Grids of opts->team_cells cells and more are run by a
 * cluster of opts->team blocks together (cluster barriers), smaller ones by
 * one block each.  Problem i is hs[i] (one hierarchy per problem, all
 * distinct, on the current device; MG_MIXED, MG_CYCLE_V, accel_depth <= 16,
 * max_cycles < MG_HIST, a coarsest level of at most 64 cells) with src[i],
 * io[i] as in mg_solve_cfc (device pointers only: MG_HOST_POINTERS is
 * refused).  Without momentum (S_i and the X and beta guesses all zero) X
 * = beta = 0 exactly and those equations stop at cycle 0.  A problem with
 * momentum whose vector levels do not fit the kernel's shared memory is
 * solved by mg_solve_cfc after the launch (up to 16 at once, from host
 * threads, each on its hierarchy's stream).  flags: MG_CFC_PSI_ONLY.  opts
 * may be NULL.  The launch runs on hs[0]'s stream after the work queued on
 * every hierarchy's stream; the call returns when all problems are done.
 * rep (NULL or count entries): per-equation reports as mg_solve_cfc's, and
 * rep[i].ms = the time from the launch's first problem start to problem i's
 * end (its latency in the batch; eq[].ms are 0).  brep may be NULL.
 * Returns MG_OK or the first failing status; MG_ERR_INVALID before any work
 * for a bad argument or a hierarchy outside the limits above.
 */
int mg_solve_cfc_batch(mg_hierarchy* const* hs, int count, const mg_cfc_sources* src, mg_cfc_fields* io,
                       int flags, const mg_batch_opts* opts, mg_cfc_report* rep, mg_batch_report* brep);

/* --------------------------------------------------- divergence cleaning */

typedef struct {
  mg_solve_report solve;
  double max_div_before, l2_div_before;   /* of the central divergence */
  double max_div_after, l2_div_after;     /* l2 = sqrt(mean(div^2)), Sec. 3.2.4 */
} mg_divb_report;

/*
 * Elliptic divergence cleaning (Sec. 2.2, eqs. poisson, update_bfield):
 * b = div B - <div B>, solve lap Phi = b with Neumann outer ghosts
 * (zero-mean Phi), then B <- B - grad Phi.  B[0..ndim-1] hold physical
 * (orthonormal) components, ghost-free, dimension 0 fastest, and are
 * modified in place; phi_out (may be NULL) receives Phi.  Flags:
 * MG_HOST_POINTERS.
 *   Cartesian: div B = sum_d central differences, B ghosts copied from the
 *     boundary cells, <.> the plain mean.
 *   Cylindrical / spherical: div B = (1/sqrt(g)) d_i (sqrt(g) q^i) by
 *     central differences of sqrt(g) q^i, every metric factor at the centre
 *     of the cell it multiplies; B ghosts copied on the outer faces, the
 *     vector parities across the origin / axis; <.> weighted by R or
 *     r^2 sin(theta), the weights under which the flux-form Laplacian with
 *     Neumann ghosts sums to zero (so the Neumann problem is compatible);
 *     grad Phi in physical components.
 * The report's divergence norms are unweighted over the cells.
 * With desc.divb_variant = MG_DIVB_EXACT (Cartesian) the Poisson operator is
 * div_c grad_c, grad_c taking Phi ghosts mirrored about the boundary cell's
 * centre (Phi_{-1} = Phi_1, Phi_n = Phi_{n-2}) and div_c copied ghosts of
 * its argument.  It splits into 2^ndim compact Neumann problems, one per
 * parity class of cells (i mod 2, j mod 2[, k mod 2]), of n / 2 cells per
 * dimension and spacing 2 h; each is solved by the multigrid of the same
 * settings for b = div B minus its mean over the class.  After the update
 * div_c B equals that class mean on every cell of the class.  The report's
 * solve entry holds the largest cycle count and residual over the classes,
 * the summed time and cell updates, and the first failing status.
 */
int mg_clean_divB(mg_hierarchy* h, double* B[3], double* phi_out, int flags, mg_divb_report* rep);

/* ------------------------------------------- single equations (expert) */

/*
 * Solve one scalar equation L(u) = f on the hierarchy (Sec. 2.7):
 *   MG_EQ_PSI: L(u) = lap u + 2 pi U (1+u)^-1 + 1/8 A2 (1+u)^-7, f = 0
 *              (eq. psi for u = psi - 1; f is ignored and may be NULL);
 *   MG_EQ_LIN: L(u) = lap u - c u (c may be NULL: Poisson), f given.
 * bc: outer boundary condition; zero_mean: remove the mean of u after
 * every cycle (Neumann gauge).  u: initial guess in, solution out.
 */
int mg_solve_scalar(mg_hierarchy* h, int kind, int bc, int zero_mean, const double* U,
                    const double* A2, const double* c, const double* f, double* u,
                    mg_solve_report* rep);

/* Solve lap V + 1/3 grad div V = f (eqs. X, beta) with outer condition bc
 * (MG_BC_DIRICHLET for X and beta). */
int mg_solve_vector(mg_hierarchy* h, int bc, const double* f[3], double* V[3], mg_solve_report* rep);

/* ------------------------------------- two-level composite grid (AMR) */

/*
 * Solve one scalar equation (kind MG_EQ_PSI or MG_EQ_LIN, as in
 * mg_solve_scalar) on a two-level composite grid: the hierarchy's grid (the
 * base) and one refined patch of ratio 2 over the base cells box_lo[d] <=
 * I_d < box_hi[d] (the block tree of Sec. 2.8 on one device: a box of whole
 * blocks).  The patch has 2 (box_hi - box_lo) cells per dimension, each a
 * power of two; a spherical patch spans theta (and phi in 3D), a
 * cylindrical 3D patch spans phi.  The paper's multigrid on AMR grids lives
 * in the library it cites; this one takes the following readings:
 *   - the composite cells are the patch cells and the base cells the patch
 *     does not cover;
 *   - patch faces on the domain boundary take its rules; the others take
 *     coarse-fine ghosts, quadratic in both directions (the base solution
 *     interpolated to the ghost's tangential position from the uncovered
 *     base cells around its parent, then g = 8/15 u~ + 2/3 u_1 - 1/5 u_2
 *     with the two patch cells inward);
 *   - an uncovered base cell next to the patch takes, for its face to the
 *     patch, the sum of the fine fluxes through that face: the composite
 *     operator is conservative;
 *   - FAS across the two levels: patch smoothing (red-black NGS, ghosts
 *     refilled per colour), the patch residual and solution restricted
 *     (volume-weighted) to the covered cells, one FAS V-cycle of the base
 *     hierarchy, the Kwak prolongation of the base change onto the patch,
 *     patch smoothing; FP64 throughout whatever desc.precision says;
 *   - stopping rule: rel over the composite cells (see mg_solve_report),
 *     Anderson mixing (accel_depth) over the composite unknowns; V-cycles
 *     only (desc.cycle ignored).
 * Base-grid arrays (U, A2 or c, f, u) have the hierarchy's size; patch
 * arrays (Up, A2p or cp, fp, up) the patch's, both ghost-free, dimension 0
 * fastest, device pointers.  Sources are given on both levels (sampled at
 * each level's cell centres).  u, up: initial guess in, solution out; on
 * return the covered base cells hold the restriction of the patch.  The
 * patch arrays of the hierarchy are allocated at the first call with a box
 * and kept while the box is the same.
 */
int mg_solve_scalar_amr(mg_hierarchy* h, const int box_lo[3], const int box_hi[3], int kind, int bc,
                        const double* U, const double* A2, const double* c, const double* f, const double* Up,
                        const double* A2p, const double* cp, const double* fp, double* u, double* up,
                        mg_solve_report* rep);

/* The composite operator of mg_solve_scalar_amr applied to (u, up): out on
 * the uncovered base cells (0 on covered ones), outp on the patch. */
int mg_apply_amr(mg_hierarchy* h, const int box_lo[3], const int box_hi[3], int kind, int bc, const double* U,
                 const double* A2, const double* c, const double* Up, const double* A2p, const double* cp,
                 const double* u, const double* up, double* out, double* outp);

/* ----------------------------------------------- unit-level (testing) */

/*
 * Apply L of an equation kind to u on the finest level (ghosts from the
 * boundary rules): out = L(u).  For MG_EQ_VEC u, out have 3 components;
 * otherwise component 0 only and U, A2, c as in mg_solve_scalar.
 */
int mg_apply_operator(mg_hierarchy* h, int kind, int bc, const double* u[3], const double* U,
                      const double* A2, const double* c, double* out[3]);

/* nsweeps red-black NGS sweeps of L(u) = f on the finest level, in place. */
int mg_smooth(mg_hierarchy* h, int kind, int bc, int nsweeps, double* u[3], const double* f[3],
              const double* U, const double* A2, const double* c);

/* A2 = A~_ij A~^ij (eq. Aij) of X (Dirichlet-0 outer, parity inner ghosts). */
int mg_compute_a2(mg_hierarchy* h, const double* X[3], double* A2);

/* Central divergence of B (Cartesian; ghosts copied from boundary cells). */
int mg_divergence(mg_hierarchy* h, const double* B[3], double* div);

/* Restrict a finest-level field to level 1 (out has level-1 size), or
 * add the Kwak prolongation of a level-1 correction e (Robin/Dirichlet/
 * Neumann ghosts by bc, scalar parity) into a finest-level field. */
int mg_restrict(mg_hierarchy* h, const double* fine, double* coarse);
int mg_prolong_add(mg_hierarchy* h, int bc, const double* coarse_e, double* fine);

/* --------------------------------------------------------------- serving */

/*
 * A request server: a FIFO queue feeding max_slots worker slots, each a
 * host thread with its own CUDA stream, so requests admitted while others
 * run overlap on the device.  Hierarchies are cached per grid descriptor
 * and reused; with a stream_id the solution of a CFC request stays resident
 * and warm-starts the next request of that stream (the previous time
 * step's metric as initial guess, Sec. 4.2.1), and the requests of one
 * stream run in submission order.  Cached hierarchies and resident
 * solutions stay within hbm_budget bytes (idle hierarchies are evicted,
 * least recently used first; a request that does not fit waits).
 */
typedef struct mg_server mg_server;

enum { MG_REQ_CFC = 0, MG_REQ_DIVB = 1, MG_REQ_AMR = 2 };

/* Arrays of an MG_REQ_AMR request: eq. psi on a two-level composite grid
 * (mg_solve_scalar_amr with MG_EQ_PSI and the Robin outer condition), the
 * base grid the request's descriptor, the patch over base cells box_lo <= I
 * < box_hi.  Deviations u = psi - 1: initial guess in, solution out. */
typedef struct {
  int box_lo[3], box_hi[3];
  const double* A2;        /* base grid A~^2 (U~ is src.U) */
  const double* Up;        /* patch U~ */
  const double* A2p;       /* patch A~^2 */
  double* u;               /* base grid psi - 1 */
  double* up;              /* patch psi - 1 */
} mg_amr_arrays;

typedef struct {
  mg_grid_desc desc;       /* grid and solver settings of the request */
  int kind;                /* MG_REQ_CFC or MG_REQ_DIVB */
  int flags;               /* MG_CFC_PSI_ONLY (CFC) */
  uint64_t stream_id;      /* 0: no warm start; else the request stream */
  mg_cfc_sources src;      /* CFC: device pointers, caller-owned until done */
  mg_cfc_fields io;        /* CFC: initial guess in (ignored when warm-started), solution out */
  double* B[3];            /* DIVB: field cleaned in place */
  double* phi;             /* DIVB: optional potential out */
  void* wait_stream;       /* cudaStream_t whose work queued before mg_submit
                              produced the inputs (NULL: the legacy stream) */
  mg_amr_arrays amr;       /* AMR: eq. psi on the composite grid (its report
                              in the result's cfc.eq[1]); no warm start */
} mg_request;

typedef struct {
  int status;
  mg_cfc_report cfc;       /* CFC reports */
  mg_divb_report divb;     /* DIVB report */
  double latency_ms;       /* submission to completion */
  double queue_ms;         /* submission to start */
  int warm_started;        /* 1 if the stream's resident solution was the guess */
} mg_result;

/* Start a server on the current device. */
int mg_server_create(size_t hbm_budget, int max_slots, int max_queue, mg_server** out);
/* Stop it: running requests finish, queued ones complete with MG_ERR_BUSY;
 * frees every hierarchy and resident solution. */
int mg_server_destroy(mg_server* s);
/* Queue a request (never blocks).  MG_ERR_BUSY when max_queue requests
 * wait already, MG_ERR_OOM when the request alone exceeds the budget. */
int mg_submit(mg_server* s, const mg_request* req, uint64_t* ticket);
/* Non-blocking: *done = 1 once finished; then out (may be NULL) receives
 * the result, the ticket is released and the request's status returned. */
int mg_poll(mg_server* s, uint64_t ticket, int* done, mg_result* out);

/* ------------------------------------------------------ instrumentation */

/* Kernel launches issued by the library since it was loaded (all
 * hierarchies, all threads). */
uint64_t mg_kernel_launches(void);

/* Kernel classes timed by mg_profile_*: red-black colour passes (one
 * launch updates half of the finest cells, one component), fused
 * red-black sweeps (both colours of a Cartesian scalar level in one launch)
 * and the finest residual with its norms (every cell, every component),
 * all on the finest level; and, for a breakdown of the cycle, the FP32
 * colour passes of the coarser launched levels (cells: those updated), the
 * two Anderson mixing kernels (cells: the finest unknowns, components
 * counted) and the one-block FP32 cycle (cells: those of its top level). */
enum {
  MG_PROF_SMOOTH64_SCALAR = 0,
  MG_PROF_SMOOTH64_VEC = 1,
  MG_PROF_SMOOTH32_SCALAR = 2,
  MG_PROF_SMOOTH32_VEC = 3,
  MG_PROF_RESID64_SCALAR = 4,
  MG_PROF_RESID64_VEC = 5,
  MG_PROF_SWEEP64_FUSED = 6,  /* fused red-black sweep: all finest cells */
  MG_PROF_SWEEP32_FUSED = 7,
  MG_PROF_SMOOTH32_COARSE = 8,
  MG_PROF_AA_UPDATE = 9,
  MG_PROF_AA_COMBINE = 10,
  MG_PROF_BLOCK_CYCLE32 = 11,
  MG_PROF_RESID64_PSI = 12,   /* the finest residual of eq. psi (RESID64_SCALAR: linear equations) */
  MG_PROF_NCLASS = 13
};

/* Enable (1) or disable (0) CUDA-event timing, on the hierarchy's stream,
 * of every finest-level launch of the classes above; clears the records. */
int mg_profile_enable(mg_hierarchy* h, int enable);

/* Launch count, summed device milliseconds and summed cells processed of
 * one class since the last mg_profile_enable (synchronises the stream). */
int mg_profile_read(mg_hierarchy* h, int klass, int64_t* launches, double* ms, int64_t* cells);

/* ------------------------------------------ allocation-free diagnostics */

/* Largest grid (cells) mg_divb_norms_noalloc accepts: the size of its
 * static device scratch (16 MiB on every GPU that loads the library). */
#define MG_NOALLOC_MAX_CELLS 2097152

/*
 * Max |div B| and |div B|_2 = sqrt(mean(div^2)) of the central divergence
 * of a Cartesian field (the same numbers mg_clean_divB reports as
 * max_div_before / l2_div_before), for callers that cannot allocate device
 * memory and so cannot create a hierarchy: a host framework that owns all
 * device memory and forbids allocation inside its time loop, or code whose
 * cudaMalloc would synchronise the device.  The paper has no counterpart:
 * this entry point exists only for such callers.
 *   ndim, n, lo, hi   the grid (n[d] >= 1, lo < hi; n[2], lo[2], hi[2]
 *                     ignored in 2D); at most MG_NOALLOC_MAX_CELLS cells,
 *                     larger grids get MG_ERR_INVALID (see mg_last_error).
 *   B                 ndim device arrays, ghost-free, dimension 0 fastest;
 *                     ghosts are copies of the boundary cells.
 *   cuda_stream       cudaStream_t to run on (NULL: the legacy stream); the
 *                     call synchronises it before returning.
 *   max_div, l2_div   host outputs.
 * It allocates nothing: its scratch (the divergence values, per-block sums
 * and the max word) is a file-scope __device__ array.  The first call on a
 * device looks up that array's device address with the device current
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array and it keeps the last call's contents (the
 * max word is cleared by each call): calls whose work overlaps on the GPU
 * (different streams or threads at once) race, so serialise them.
 */
int mg_divb_norms_noalloc(int ndim, const int n[3], const double lo[3], const double hi[3],
                          const double* B[3], void* cuda_stream, double* max_div, double* l2_div);

#ifdef __cplusplus
}
#endif
#endif /* GMUNU_MG_H */
