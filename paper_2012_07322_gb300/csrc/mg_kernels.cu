// Grid-wide multigrid kernels (red-black Newton-Gauss-Seidel, residual with
// fused norms, FAS coarse right-hand side, ghost fill, volume-weighted
// restriction, Kwak prolongation) and the single-block coarsest solver, with
// their host-side launchers.  Sec. 2.7 of the paper.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <type_traits>

#include "mg_internal.h"
#include "mg_kernels.cuh"

namespace gmg {

static std::atomic<unsigned long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

static inline dim3 block_for(int three) { return three ? dim3(32, 4, 2) : dim3(32, 8, 1); }
static inline unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------ smoothers

// One colour of the red-black sweep: cells with (i + j + k) % 2 == colour.
// Thread t of a row handles i = 2 t + ((j + k + colour) & 1).
template <typename T, int G, int KIND>
__global__ void k_smooth_scalar(LevelView<T> L, T* __restrict__ u, const T* __restrict__ f,
                                const T* __restrict__ s0, const T* __restrict__ s1, int colour) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (2 * t >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const int i = 2 * t + ((j + k + colour) & 1);
  scalar_update<T, G, KIND>(L, u, f, s0, s1, i, j, k);
}

// One colour of component comp of the vector sweep.  With a ghost-push
// table the block then rewrites the ghosts sourced by the cells it updated
// (their new values kept in shared memory), and in 3D thread z takes plane
// blockIdx.z + z n2 / 2; with NK = 2 (levels of 2^19 cells and more) each
// thread also takes the plane n2 / 4 above, so the pass runs in one wave of
// blocks.  A colour's cells of one component are independent of each other.
template <typename T, int G, int NK>
__global__ void k_smooth_vec(LevelView<T> L, T* __restrict__ A, T* __restrict__ B, T* __restrict__ C,
                             const T* __restrict__ f, int comp, int colour, GhostPush gp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (!gp.off) {
    pdl_entry();
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (2 * t >= L.n0 || j >= L.n1 || k >= L.n2) return;
    const int i = 2 * t + ((j + k + colour) & 1);
    vec_update<T, G>(L, A, B, C, f, comp, i, j, k);
    return;
  }
  __shared__ T nv[NK * 256];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  // the table is written once, when the hierarchy builds it: its first
  // entries are read before waiting for the preceding launch
  const int e0 = gp.off[b], e1 = gp.off[b + 1];
  int2 q0 = make_int2(0, 0);
  if (e0 + tid < e1) q0 = gp.ent[e0 + tid];
  pdl_entry();
  const int k0 = L.three ? (int)blockIdx.z + (int)threadIdx.z * (L.n2 >> 1) : 0;
  T* V = comp == 0 ? A : (comp == 1 ? B : C);
  if (2 * t < L.n0 && j < L.n1 && k0 < L.n2) {
    // nv slot of the w-th cell: tid + 256 w
#pragma unroll
    for (int w = 0; w < NK; ++w) {
      const int k = k0 + w * (L.n2 >> 2);
      const int i = 2 * t + ((j + k + colour) & 1);
      const long p = L.idx(i, j, k);
      const T v = vec_new_value<T, G>(L, A, B, C, f, comp, i, j, p);
      V[p] = v;
      nv[tid + 256 * w] = v;
    }
  }
  if (e0 == e1) return;  // the same for the whole block
  __syncthreads();
  for (int e = e0 + tid; e < e1; e += nthr) {
    const int2 q = e == e0 + tid ? q0 : gp.ent[e];
    const T v = nv[q.y >> 1];
    V[q.x] = (q.y & 1) ? -v : v;
  }
}

// One full red-black sweep of a 3D linear scalar equation in one launch,
// out of place (uin -> uout): Cartesian levels, and cylindrical / spherical
// levels, whose dimension 2 (phi) is periodic: the march along k then wraps
// (plane -1 is plane n2 - 1), and the coefficients come per (i, j) from the
// level's tables.  A block owns a column of TX x TY
// cells over a chunk of planes [z0, z1) and marches along k.  Plane by
// plane it stages a (TX + 8) x (TY + 4) box of u, f and c (the column
// with a 4-cell halo in i, 2 cells in j; rows are 16-byte aligned, so the
// box moves in 16-byte asynchronous copies issued two planes ahead),
// relaxes the red cells of plane s over its column and a one-cell ring
// around it (the ring cells are relaxed with the same arithmetic by the
// neighbouring columns), then the black cells of plane s - 1, and stores
// plane s - 1.  The red cells of planes z0 - 1 and z1 are likewise relaxed
// by two chunks.  Every value read comes from uin, which no block writes, so
// the result is the red-black sweep of k_smooth_scalar whatever order the
// blocks run in, and u, f and c cross DRAM once per sweep instead of once
// per colour.  Warp w owns row w; each lane owns TX / 64 pairs of cells.
constexpr int RB_HX = 4, RB_HY = 2;  // staged halo
constexpr int RB_RING_FIRST = 64;     // first thread of the ring cells
// plane buffers: u planes s-1..s+2 and f, c planes s-1..s+1 are in use or
// in flight at step s (the f ring is indexed by plane & 3); groups are
// staged RB_AHEAD planes beyond the plane the step waits for (2 measured
// slower at 256^3: 57.8 against 55.3 us per sweep)
constexpr int RB_NU = 6, RB_NF = 4, RB_AHEAD = 1;
static_assert(RB_HX == ROW_PAD, "the staged box starts on a 16-byte boundary");

// Column shape: TX cells by TY rows, one warp per row (128-cell columns
// take 16 rows: the ring and the staged halo rows cost half as much per
// cell as with 8).
template <int TX>
struct RbShape {
  static constexpr int TY = TX == 128 ? 16 : 8, THREADS = 32 * TY;
  static constexpr int BY = TY + 2 * RB_HY;
  static constexpr int BX = TX + 2 * RB_HX, BP = BX * BY;
  static constexpr int RING = TX + 2 + TY;  // red ring cells: two rows of (TX+2)/2, two columns of TY/2
  static_assert(RB_RING_FIRST + RING <= THREADS - 32, "ring threads clear of the last warp");
};

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tensor-memory-accelerator staging: one thread per block issues a plane's
// copy, which signals the plane slot's mbarrier with its byte count.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_plane(void* dst, const CUtensorMap* map, int x, int y, int z,
                                          unsigned long long* m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(m))
      : "memory");
}
// Iterations of mbarrier.try_wait (each suspends for a bounded time) before
// a wait for a staged plane gives up.
constexpr long RB_WAIT_LIMIT = 1L << 22;

// The 16-byte pieces of the staged box this thread copies, fixed for the
// whole march: global offset within a plane, offset in the plane buffer.
template <typename T, int TX>
struct RbPieces {
  static constexpr int BX = RbShape<TX>::BX, THREADS = RbShape<TX>::THREADS;
  static constexpr int PER_ROW = BX * (int)sizeof(T) / 16, N = RbShape<TX>::BY * PER_ROW;
  static constexpr int ITEMS = (N + THREADS - 1) / THREADS;
  long g[ITEMS];
  int s[ITEMS];
  bool ok[ITEMS];
  __device__ __forceinline__ RbPieces(const LevelView<T>& L, int i0, int j0) {
#pragma unroll
    for (int m = 0; m < ITEMS; ++m) {
      const int q = threadIdx.x + m * THREADS;
      const int ly = q / PER_ROW, cx = q - ly * PER_ROW;
      const int j = j0 - RB_HY + ly, x = cx * (16 / (int)sizeof(T));
      ok[m] = q < N && j >= -1 && j <= L.n1;  // rows of the ghosted array
      g[m] = L.off + (i0 - RB_HX + x) + (long)j * L.sx;
      s[m] = ly * BX + x;
    }
  }
  __device__ __forceinline__ void copy(T* buf, const T* __restrict__ src, long plane) const {
#pragma unroll
    for (int m = 0; m < ITEMS; ++m)
      if (ok[m]) cp_async16(buf + s[m], src + g[m] + plane);
  }
};

// The staged planes of one relaxation step.
template <typename T>
struct RbPlanes {
  const T* Pd;  // plane s - 1
  T* P;         // plane s (updated in place)
  const T* Pu;  // plane s + 1
  const T* F;   // f of plane s
  const T* Cc;  // c of plane s
};

// Stencil coefficients of one cell of the flux-form Laplacian (Sec. 2.7.1,
// the terms of lap_scalar): east / west fluxes, the dimension-1 pair (north
// and south on spherical levels, where they carry sin(theta) at the faces;
// one value on the others), the dimension-2 coefficient, and the diagonal.
template <typename T>
struct RbCoef {
  T cE, cW, cN, cS, cZ, D;
};
template <typename T, int G>
__device__ __forceinline__ RbCoef<T> rb_coef(const LevelView<T>& L, int i, int j) {
  RbCoef<T> c;
  c.cE = L.TI(TI_CE, i);
  c.cW = L.TI(TI_CW, i);
  c.D = -(c.cE + c.cW);
  if (G == SPH) {
    const T ir2 = L.TI(TI_IX2, i);
    c.cN = ir2 * L.TJ(TJ_TN, j);
    c.cS = ir2 * L.TJ(TJ_TS, j);
    c.D -= c.cN + c.cS;
    c.cZ = ir2 * L.TJ(TJ_PF, j);
  } else {
    c.cN = c.cS = L.ih1s;
    c.D -= T(2) * L.ih1s;
    c.cZ = G == CART ? L.ih2s : L.TI(TI_PHI, i);
  }
  c.D -= T(2) * c.cZ;
  return c;
}

// Newton-Gauss-Seidel update of cell (i0 + x, j0 + y, s): the arithmetic of
// lap_scalar and scalar_update<EQ_LIN>.  The outer ghosts a boundary cell
// needs sit in the staged planes already (rb_fix_ghosts; across the origin
// or the axis, and at the poles, the flux coefficient is zero), so every
// cell takes the same path; RING cells outside the domain are skipped.
template <typename T, int G, int TX, bool HAS_C, bool RING>
__device__ __forceinline__ void rb_relax(const LevelView<T>& L, const RbPlanes<T>& R, int i0, int j0, int x, int y,
                                         const RbCoef<T>& k, T iD0) {
  constexpr int BX = RbShape<TX>::BX;
  if (RING) {
    const int i = i0 + x, j = j0 + y;
    if (i < 0 || i >= L.n0 || j < 0 || j >= L.n1) return;
  }
  const int q = (x + RB_HX) + (y + RB_HY) * BX;
  const T uc = R.P[q];
  T Lu = k.cE * (R.P[q + 1] - uc) - k.cW * (uc - R.P[q - 1]);
  if (G == SPH)
    Lu += k.cN * (R.P[q + BX] - uc) - k.cS * (uc - R.P[q - BX]);
  else
    Lu += k.cN * (R.P[q + BX] - T(2) * uc + R.P[q - BX]);
  Lu += k.cZ * (R.Pu[q] - T(2) * uc + R.Pd[q]);
  if (HAS_C) {
    const T cv = R.Cc[q];
    Lu -= cv * uc;
    R.P[q] = uc - (Lu - R.F[q]) / (k.D - cv);
  } else if (G == CART) {
    R.P[q] = uc - (Lu - R.F[q]) * iD0;
  } else {
    R.P[q] = uc - (Lu - R.F[q]) / k.D;
  }
}

// Coefficients of cell q (0 or 1) of a lane's pair, member by member (a
// select of the whole struct would put it in local memory).
template <typename T>
__device__ __forceinline__ RbCoef<T> rb_pick(int q, const RbCoef<T>& a, const RbCoef<T>& b) {
  RbCoef<T> c;
  c.cE = q ? b.cE : a.cE;
  c.cW = q ? b.cW : a.cW;
  c.cN = q ? b.cN : a.cN;
  c.cS = q ? b.cS : a.cS;
  c.cZ = q ? b.cZ : a.cZ;
  c.D = q ? b.D : a.D;
  return c;
}

// The same update from operand values: centre uc, neighbours e, w, n, s (in
// i and j), up and down (in k), right-hand side fv and coefficient cv.
template <typename T, int G, bool HAS_C>
__device__ __forceinline__ T rb_new_value(const RbCoef<T>& k, T iD0, T uc, T ue, T uw, T un, T us, T uu, T ud, T fv,
                                          T cv) {
  T Lu = k.cE * (ue - uc) - k.cW * (uc - uw);
  if (G == SPH)
    Lu += k.cN * (un - uc) - k.cS * (uc - us);
  else
    Lu += k.cN * (un - T(2) * uc + us);
  Lu += k.cZ * (uu - T(2) * uc + ud);
  if (HAS_C) {
    Lu -= cv * uc;
    return uc - (Lu - fv) / (k.D - cv);
  } else if (G == CART) {
    return uc - (Lu - fv) * iD0;
  } else {
    return uc - (Lu - fv) / k.D;
  }
}

// Outer ghosts of staged plane p (just landed, still the sweep's input) in
// the i and j directions: g = factor * u of the boundary cell, the values
// lap_scalar folds in.  A ghost is read only by its own boundary cell, whose
// value is unchanged until that cell's own update, so a ghost written from
// the input stays exact.
template <typename T, int TX>
__device__ __forceinline__ void rb_fix_ghosts(const LevelView<T>& L, T* P, int i0, int j0, int p) {
  constexpr int BX = RbShape<TX>::BX, TY = RbShape<TX>::TY, NY = TY + 2, NX = TX + 2;
  const bool xl = i0 == 0, xh = i0 + TX == L.n0, yl = j0 == 0, yh = j0 + TY == L.n1;
  const int t = threadIdx.x;
  // i ghosts of rows y = -1 .. TY on the low / high faces (threads 0 .. 2 NY)
  if (t < 2 * NY) {
    const bool hi = t >= NY;
    const int y = (hi ? t - NY : t) - 1, j = j0 + y;
    if ((hi ? xh : xl) && j >= 0 && j < L.n1) {
      const int xs = hi ? TX - 1 : 0, xg = hi ? TX : -1;
      const T fac = hi ? outer_factor(L, L.n0, j, p, L.n0 - 1, j, p) : outer_factor(L, -1, j, p, 0, j, p);
      P[(xg + RB_HX) + (y + RB_HY) * BX] = fac * P[(xs + RB_HX) + (y + RB_HY) * BX];
    }
  }
  // j ghosts of columns x = -1 .. TX, only on blocks at a j face
  if (yl || yh)
    for (int u = t; u < 2 * NX; u += RbShape<TX>::THREADS) {
      const bool hi = u >= NX;
      const int x = (hi ? u - NX : u) - 1, i = i0 + x;
      if (!(hi ? yh : yl) || i < 0 || i >= L.n0) continue;
      const int ys = hi ? TY - 1 : 0, yg = hi ? TY : -1;
      const T fac = hi ? outer_factor(L, i, L.n1, p, i, L.n1 - 1, p) : outer_factor(L, i, -1, p, i, 0, p);
      P[(x + RB_HX) + (yg + RB_HY) * BX] = fac * P[(x + RB_HX) + (ys + RB_HY) * BX];
    }
}

// Ghost plane pg (-1 or n2) from the staged plane ps next to it.
template <typename T, int TX>
__device__ __forceinline__ void rb_ghost_plane(const LevelView<T>& L, T* G, const T* S, int i0, int j0, int pg,
                                               int ps) {
  constexpr int BX = RbShape<TX>::BX, NY = RbShape<TX>::TY + 2, NX = TX + 2;
  for (int t = threadIdx.x; t < NX * NY; t += RbShape<TX>::THREADS) {
    const int y = t / NX - 1, x = t % NX - 1, i = i0 + x, j = j0 + y;
    if (i < 0 || i >= L.n0 || j < 0 || j >= L.n1) continue;
    const int q = (x + RB_HX) + (y + RB_HY) * BX;
    G[q] = outer_factor(L, i, j, pg, i, j, ps) * S[q];
  }
}

// The coefficients of the cells a lane relaxes in its row: for pair h, the
// even (q = 0) and odd (q = 1) cell, whichever the colour of the plane
// selects.
template <typename T, int TX>
struct RbLaneCoef {
  RbCoef<T> k[TX / 64][2];
};

// Red cells of plane s on the ring around the column (the lane cells are
// relaxed from registers in k_sweep_rb).  On a Cartesian level every cell
// has the lane cells' coefficients.
template <typename T, int G, int TX, bool HAS_C>
__device__ __forceinline__ void rb_red_ring(const LevelView<T>& L, const RbPlanes<T>& R, int i0, int j0, int s,
                                            const RbLaneCoef<T, TX>& lc, T iD0) {
  // threads 64 .. 64 + RING - 1 (from warp 2 on: warps 0 and 1 fix the
  // outer ghosts of blocks on an i face, and the last warp issues the copies)
  const int t = (int)threadIdx.x - RB_RING_FIRST;
  const int par = (i0 + j0 + s) & 1;  // red: (i + j + s) even
  if (t >= 0 && t < RbShape<TX>::RING) {
    constexpr int TY = RbShape<TX>::TY, HR = (TX + 2) / 2, HC = TY / 2;
    int x, y;
    if (t < HR) {
      y = -1;
      x = -1 + 2 * t + par;
    } else if (t < 2 * HR) {
      y = TY;
      x = -1 + 2 * (t - HR) + (par ^ 1);
    } else if (t < 2 * HR + HC) {
      x = -1;
      y = 2 * (t - 2 * HR) + (par ^ 1);
    } else {
      x = TX;
      y = 2 * (t - 2 * HR - HC) + par;
    }
    if (G == CART) {
      rb_relax<T, G, TX, HAS_C, true>(L, R, i0, j0, x, y, lc.k[0][0], iD0);
    } else {
      const int ic = min(max(i0 + x, 0), L.n0 - 1), jc = min(max(j0 + y, 0), L.n1 - 1);
      rb_relax<T, G, TX, HAS_C, true>(L, R, i0, j0, x, y, rb_coef<T, G>(L, ic, jc), iD0);
    }
  }
}

// FP32 Cartesian sweeps of 128-cell columns stage their planes with the
// tensor memory accelerator when the launch carries tensor maps: one thread
// issues a plane group's copies (u plane p, f and c plane p - 1) into the
// group's slot and arms the slot's mbarrier with their bytes; the block
// waits on the slot instead of on its own 16-byte copies.
template <typename T, int G, int TX>
__host__ __device__ constexpr bool rb_tma() {
  return sizeof(T) == 4 && G == CART && TX == 128;
}

template <typename T, int G, int TX, bool HAS_C>
__global__ void __launch_bounds__(RbShape<TX>::THREADS, TX == 128 ? (G == CART ? 2 : 1) : (sizeof(T) == 4 ? 4 : 2))
    k_sweep_rb(LevelView<T> L, const T* __restrict__ uin, T* __restrict__ uout, const T* __restrict__ f,
               const T* __restrict__ c, int zc, const __grid_constant__ SweepMaps M) {
  pdl_entry();
  constexpr int BX = RbShape<TX>::BX, BP = RbShape<TX>::BP;
  constexpr bool PER = G != CART;  // periodic dimension 2
  constexpr bool TMA = rb_tma<T, G, TX>();
  static_assert(!TMA || (BP * sizeof(T)) % 128 == 0, "plane buffers 128-byte aligned");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long mbar[RB_NU];
  // (copies land on 128-byte boundaries: a misaligned dynamic shared
  // memory base would take the 16-byte copies instead)
  const bool tma = TMA && M.on && (smem_u32(smem_raw) & 127u) == 0;
  // the copies are issued by lane 0 of the last warp (the ring cells fall
  // on the first warps)
  constexpr int ISSUER = RbShape<TX>::THREADS - 32;
  if (tma) {
    if (threadIdx.x == ISSUER) {
      for (int q = 0; q < RB_NU; ++q) mbar_init(&mbar[q]);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  unsigned ph = 0, pending = 0;  // per slot: parity of its next phase, copies not yet waited for
  bool timed_out = false;
  T* su = reinterpret_cast<T*>(smem_raw);
  T* sf = su + RB_NU * BP;
  T* sc = sf + RB_NF * BP;
  constexpr int TY = RbShape<TX>::TY;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, L.n2);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // coefficients of the lane's cells (uniform on a Cartesian grid)
  RbLaneCoef<T, TX> lc;
#pragma unroll
  for (int h = 0; h < TX / 64; ++h)
#pragma unroll
    for (int q = 0; q < 2; ++q) lc.k[h][q] = rb_coef<T, G>(L, i0 + 64 * h + 2 * lane + q, min(j0 + w, L.n1 - 1));
  const T iD0 = T(1) / lc.k[0][0].D;
  const bool edge_xy = i0 == 0 || j0 == 0 || i0 + TX >= L.n0 || j0 + TY >= L.n1;
  const RbPieces<T, TX> pc(L, i0, j0);
  auto wrap = [&](int p) { return PER ? (p + L.n2) % L.n2 : p; };
  // group p: u plane p (into u buffer bu) and f, c plane p - 1, for the
  // planes the chunk needs (periodic levels: the wrapped planes)
  auto stage = [&](int p, int bu) {
    const bool uok = (PER || (p >= 0 && p < L.n2)) && p >= z0 - 2 && p <= z1 + 1;
    const int pf = p - 1;
    const bool fok = (PER || (pf >= 0 && pf < L.n2)) && pf >= z0 - 1 && pf <= z1;
    const int bf = (pf & (RB_NF - 1)) * BP;
    if constexpr (TMA) {
      if (tma) {
        // box origin: column i0 - 4 (padded-row index i0), row j0 - 2 (row
        // index j0 - 1: the row above the ghost row reads as zeros), plane
        if (threadIdx.x == ISSUER) {
          constexpr unsigned PB = (unsigned)(BP * sizeof(T));
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect(&mbar[bu], (uok ? PB : 0u) + (fok ? PB * (HAS_C ? 2u : 1u) : 0u));
          if (uok) tma_plane(su + bu * BP, &M.u, i0, j0 - 1, wrap(p) + 1, &mbar[bu]);
          if (fok) {
            tma_plane(sf + bf, &M.f, i0, j0 - 1, wrap(pf) + 1, &mbar[bu]);
            if (HAS_C) tma_plane(sc + bf, &M.c, i0, j0 - 1, wrap(pf) + 1, &mbar[bu]);
          }
        }
        pending |= 1u << bu;
        return;
      }
    }
    if (uok) pc.copy(su + bu * BP, uin, (long)wrap(p) * L.sy);
    if (fok) {
      pc.copy(sf + bf, f, (long)wrap(pf) * L.sy);
      if (HAS_C) pc.copy(sc + bf, c, (long)wrap(pf) * L.sy);
    }
    cp_async_commit();
  };
  // wait for the group in slot q (tensor-map staging); false after the
  // iteration limit
  auto wait_slot = [&](int q) {
    const unsigned par = (ph >> q) & 1u;
    for (long it = 0; it < RB_WAIT_LIMIT; ++it)
      if (mbar_try(&mbar[q], par)) {
        ph ^= 1u << q;
        pending &= ~(1u << q);
        return true;
      }
    return false;
  };
  // u plane p lives in buffer p mod RB_NU.  Groups are staged RB_AHEAD
  // planes ahead of the plane a step waits for (at step s: plane s + 1;
  // staged: s + 1 + RB_AHEAD at the latest).  Since a step's barrier comes
  // after its black cells, the buffers a copy overwrites (u plane s - 3, f
  // plane s - 2) were last read before the previous step's barrier.
  auto sl = [](int p) { return (p + 2 * RB_NU) % RB_NU; };
  for (int p = z0 - 2; p <= z0 - 1 + RB_AHEAD; ++p) stage(p, sl(p));
  // The lane's pairs (i, i + 1), i = i0 + 64 h + 2 lane, of row w in
  // registers for planes s - 2 .. s + 1.  A pair's red cell of plane s and
  // its black cell of plane s - 1 are the same column q: in k a cell's
  // neighbours are the lane's own values, in i one of them is; the other
  // neighbours (other lanes and rows, the ring, the outer ghosts) are read
  // from the staged planes.  Red values are written back to the plane for
  // the other threads; black values are read by nobody before the store.
  constexpr int NH = TX / 64;
  using V2 = typename Vec2<T>::type;  // pairs (i, i + 1): n0 a multiple of TX, rows 16-byte aligned
  V2 rm2[NH], rm1[NH], r0[NH], rp1[NH];
  const int po = (2 * lane + RB_HX) + (w + RB_HY) * BX;  // the lane's first pair in a staged plane
  T* const orow = uout + L.idx(i0 + 2 * lane, j0 + w, 0);  // ... and in plane 0 of uout
  for (int s = z0 - 1; s <= z1; ++s) {
    // u buffers of planes s - 1, s, s + 1, s + 2
    const int bd = sl(s - 1), bs = sl(s), bu = sl(s + 1), bn2 = sl(s + 2);
    stage(s + RB_AHEAD + 1, sl(s + RB_AHEAD + 1));
    if (tma) {
      // u plane s + 1 and f, c plane s (the first step: the prologue's
      // three).  Each thread waits for the copies itself, so no barrier
      // follows: the ghosts fixed below (plane s + 1) are read in the next
      // step, after this step's second barrier, and the first step has a
      // barrier of its own.
      bool ok = true;
      if (s == z0 - 1) ok = wait_slot(bd) && wait_slot(bs);
      ok = ok && wait_slot(bu);
      timed_out = timed_out || !ok;
    } else {
      cp_async_wait<RB_AHEAD>();  // u plane s + 1 and f, c plane s have landed
      __syncthreads();
    }
    // outer ghosts of the planes about to be relaxed
    if (edge_xy) {
      if (s == z0 - 1 && (PER || s >= 0)) rb_fix_ghosts<T, TX>(L, su + bs * BP, i0, j0, wrap(s));
      if (PER || (s + 1 >= 0 && s + 1 < L.n2)) rb_fix_ghosts<T, TX>(L, su + bu * BP, i0, j0, wrap(s + 1));
    }
    if (!PER) {
      if (s + 1 == 0) rb_ghost_plane<T, TX>(L, su + bs * BP, su + bu * BP, i0, j0, -1, 0);
      if (s + 1 == L.n2 - 1) rb_ghost_plane<T, TX>(L, su + bn2 * BP, su + bu * BP, i0, j0, L.n2, L.n2 - 1);
    }
    if (s == z0 - 1) {
      __syncthreads();
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        // plane z0 - 2 (not staged below a non-periodic edge: unused there) and z0 - 1
        rm1[h] = *reinterpret_cast<const V2*>(su + bd * BP + po + 64 * h);
        r0[h] = *reinterpret_cast<const V2*>(su + bs * BP + po + 64 * h);
      }
    }
#pragma unroll
    for (int h = 0; h < NH; ++h) rp1[h] = *reinterpret_cast<const V2*>(su + bu * BP + po + 64 * h);  // plane s + 1
    // the pair's red cell of plane s and black cell of plane s - 1: the same
    // for the whole warp, so each update below is compiled for both values
    const int q = (i0 + j0 + s + w) & 1;
    if (PER || (s >= 0 && s < L.n2)) {
      const int bf = (s & (RB_NF - 1)) * BP;
      T* P = su + bs * BP;
      const T* F = sf + bf;
      const T* Cc = sc + bf;
      auto red = [&](auto QC) {
        constexpr int Q = decltype(QC)::value;
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          const int o = po + 64 * h + Q;
          const T uc = Q ? r0[h].y : r0[h].x, other = Q ? r0[h].x : r0[h].y;
          const T ue = Q ? P[o + 1] : other, uw = Q ? other : P[o - 1];
          const T v = rb_new_value<T, G, HAS_C>(G == CART ? lc.k[0][0] : lc.k[h][Q], iD0, uc, ue, uw, P[o + BX],
                                                P[o - BX], Q ? rp1[h].y : rp1[h].x, Q ? rm1[h].y : rm1[h].x, F[o],
                                                HAS_C ? Cc[o] : T(0));
          P[o] = v;
          if (Q)
            r0[h].y = v;
          else
            r0[h].x = v;
        }
      };
      if (q)
        red(std::integral_constant<int, 1>{});
      else
        red(std::integral_constant<int, 0>{});
      const RbPlanes<T> R{su + bd * BP, P, su + bu * BP, F, Cc};
      rb_red_ring<T, G, TX, HAS_C>(L, R, i0, j0, s, lc, iD0);
    }
    const int sb = s - 1;
    if (sb >= z0) {
      // black cells of plane sb = s - 1 (its red neighbours: planes s - 2,
      // s - 1, s; those of plane s - 1 relaxed before the last barrier, the
      // others in this lane's registers), then store the pairs
      const int bf = (sb & (RB_NF - 1)) * BP;
      const T* P = su + bd * BP;
      const T* F = sf + bf;
      const T* Cc = sc + bf;
      T* out = orow + (long)sb * L.sy;
      auto black = [&](auto QC) {
        constexpr int Q = decltype(QC)::value;
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          const int o = po + 64 * h + Q;
          const T uc = Q ? rm1[h].y : rm1[h].x, other = Q ? rm1[h].x : rm1[h].y;
          const T ue = Q ? P[o + 1] : other, uw = Q ? other : P[o - 1];
          const T v = rb_new_value<T, G, HAS_C>(G == CART ? lc.k[0][0] : lc.k[h][Q], iD0, uc, ue, uw, P[o + BX],
                                                P[o - BX], Q ? r0[h].y : r0[h].x, Q ? rm2[h].y : rm2[h].x, F[o],
                                                HAS_C ? Cc[o] : T(0));
          if (Q)
            rm1[h].y = v;
          else
            rm1[h].x = v;
          *reinterpret_cast<V2*>(out + 64 * h) = rm1[h];
        }
      };
      if (q)
        black(std::integral_constant<int, 1>{});
      else
        black(std::integral_constant<int, 0>{});
    }
    // One barrier per plane step.  Black cells read only red values of
    // other threads from the previous step's plane (and their own registers),
    // and red cells only black values, which no thread writes to the staged
    // planes: the barrier orders this step's red values before the next
    // step's black cells, and the staged planes' reuse.
    if (tma) {
      if (__syncthreads_or(timed_out)) {
        // a staged plane never arrived: report it, let the copies still in
        // flight land (again within the limit) and stop
        if (threadIdx.x == ISSUER) atomicExch(M.err, 1ULL);
        for (int q = 0; q < RB_NU; ++q)
          if (pending & (1u << q)) wait_slot(q);
        return;
      }
    } else {
      __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      rm2[h] = rm1[h];
      rm1[h] = r0[h];
      r0[h] = rp1[h];
    }
  }
  if (!tma) cp_async_wait<0>();
}

template <typename T>
__global__ void k_fill_ghosts(LevelView<T> L, T* __restrict__ u, int comp) {
  pdl_entry();
  const long n = ghost_count(L);
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n; g += (long)gridDim.x * blockDim.x)
    fill_one_ghost(L, u, comp, g);
}

// The ghosts of ncomp fields in one launch: field c is vector component c
// (vec != 0) or a scalar.
template <typename T>
__global__ void k_fill_ghosts3(LevelView<T> L, T* __restrict__ u0, T* __restrict__ u1, T* __restrict__ u2,
                               int ncomp, int vec) {
  pdl_entry();
  const long n = ghost_count(L);
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < ncomp * n; g += (long)gridDim.x * blockDim.x) {
    const int c = (int)(g / n);
    fill_one_ghost(L, c == 0 ? u0 : (c == 1 ? u1 : u2), vec ? c : -1, g - (long)c * n);
  }
}

// ------------------------------------------------------------ residuals

// r = f - L(u) on every interior cell.  red (if non-null) receives
// max |r| (slot 0) and, when weighted, max |w r| (slot 1), max |w S| (slot 2).
// A thread walks RES_KZ planes (k strided by blockDim.z) so that the block
// reduction of the norms is paid once per RES_KZ cells.
constexpr int RES_KZ = 4;
// The vector residual carries three components' worth of FP64 work per
// cell: one plane per thread and at most 128 registers (two blocks per SM)
// spread it over more blocks.
constexpr int RES_KZ_VEC = 1;

template <typename T, int G, int KIND>
__global__ void k_residual_scalar(LevelView<T> L, const T* __restrict__ u, const T* __restrict__ f,
                                  const T* __restrict__ s0, const T* __restrict__ s1, T* __restrict__ r,
                                  float* __restrict__ r32, float* __restrict__ k32, unsigned long long* red,
                                  int weighted) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long m[3] = {0ULL, 0ULL, 0ULL};
  if (i < L.n0 && j < L.n1) {
    const double w = weighted ? (double)norm_weight(L, i, j) : 1.0;
#pragma unroll
    for (int it = 0; it < RES_KZ; ++it) {
      const int k = (blockIdx.z * RES_KZ + it) * blockDim.z + threadIdx.z;
      if (k >= L.n2) continue;
      const long p = L.idx(i, j, k);
      T Sv, kp;
      const T rv = scalar_residual_cell<T, G, KIND>(L, u, f, s0, s1, i, j, k, p, Sv, k32 ? &kp : nullptr);
      if (r) r[p] = rv;
      if (r32) r32[p] = (float)rv;
      if (KIND == EQ_PSI && k32) k32[p] = (float)kp;
      if (red) {
        m[0] = umax64(m[0], abs_bits((double)rv));
        if (weighted) {
          if (G != CART) m[1] = umax64(m[1], abs_bits(w * (double)rv));
          m[2] = umax64(m[2], abs_bits(G == CART ? (double)Sv : w * (double)Sv));
        }
      }
    }
    if (G == CART && weighted) m[1] = m[0];  // unit weight
  }
  if (red) block_max_bits<3>(m, red);
}

template <typename T, int G>
__global__ void __launch_bounds__(256, 2) k_residual_vec(LevelView<T> L, const T* __restrict__ A, const T* __restrict__ B,
                               const T* __restrict__ C, const T* __restrict__ f0, const T* __restrict__ f1,
                               const T* __restrict__ f2, T* __restrict__ r0, T* __restrict__ r1,
                               T* __restrict__ r2, float* __restrict__ q0, float* __restrict__ q1,
                               float* __restrict__ q2, unsigned long long* red, int weighted) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long m[3] = {0ULL, 0ULL, 0ULL};
  if (i < L.n0 && j < L.n1) {
    const double w = weighted ? (double)norm_weight(L, i, j) : 1.0;
    const T* fs[3] = {f0, f1, f2};
    T* rs[3] = {r0, r1, r2};
    float* qs[3] = {q0, q1, q2};
#pragma unroll 1
    for (int it = 0; it < RES_KZ_VEC; ++it) {
      const int k = (blockIdx.z * RES_KZ_VEC + it) * blockDim.z + threadIdx.z;
      if (k >= L.n2) continue;
      const long p = L.idx(i, j, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T fv = fs[c] ? fs[c][p] : T(0);
        const T rv = vec_residual_cell<T, G>(L, A, B, C, fs[c], c, i, j, p);
        if (rs[c]) rs[c][p] = rv;
        if (qs[c]) qs[c][p] = (float)rv;
        if (red) {
          m[0] = umax64(m[0], abs_bits((double)rv));
          if (weighted) {
            m[1] = umax64(m[1], abs_bits(w * (double)rv));
            m[2] = umax64(m[2], abs_bits(w * (double)fv));
          }
        }
      }
    }
  }
  if (red) block_max_bits<3>(m, red);
}

// The FP64 vector residual on a spherical level with four-point mixed
// derivatives from the per-(i, j) stencil coefficients L.vc (make_vec_coeffs):
// the operator of vec_op with its metric factors multiplied out, one FMA per
// stencil term, about a third of vec_op's FP64 operations (the FP64 pipe
// bounds this kernel).  Outputs and norms as k_residual_vec.  A 3D block is
// 32 x 2 x 4 cells, so four k-planes share each (i, j) coefficient load.
__global__ void __launch_bounds__(256, 2)
    k_residual_vec_sph(LevelView<double> L, const double* __restrict__ A, const double* __restrict__ B,
                       const double* __restrict__ C, const double* __restrict__ f0, const double* __restrict__ f1,
                       const double* __restrict__ f2, double* __restrict__ r0, double* __restrict__ r1,
                       double* __restrict__ r2, float* __restrict__ q0, float* __restrict__ q1,
                       float* __restrict__ q2, unsigned long long* red, int weighted) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  unsigned long long m[3] = {0ULL, 0ULL, 0ULL};
  if (i < L.n0 && j < L.n1 && k < L.n2) {
    const long p = L.idx(i, j, k), sx = L.sx, sy = L.sy;
    const long qs = (long)L.n0 * L.n1;
    const double* __restrict__ V = L.vc + (long)j * L.n0 + i;
    auto cf = [&](int q) { return V[q * qs]; };
    // mix4(F; a, b) = F(+a+b) - F(+a-b) - F(-a+b) + F(-a-b)
    auto mix4 = [&](const double* F, long a, long b) {
      return ((F[p + a + b] - F[p + a - b]) - F[p - a + b]) + F[p - a - b];
    };
    const double Ac = A[p], Bc = B[p], Cc = C[p];
    double Lu0 = cf(0) * A[p + 1] + cf(1) * A[p - 1] + cf(2) * A[p + sx] + cf(3) * A[p - sx] + cf(5) * Ac +
                 cf(6) * (B[p + sx] - B[p - sx]) + cf(7) * Bc + cf(8) * (B[p + 1] - B[p - 1]) +
                 cf(9) * mix4(B, 1, sx);
    double Lu1 = cf(12) * B[p + 1] + cf(13) * B[p - 1] + cf(14) * B[p + sx] + cf(15) * B[p - sx] + cf(17) * Bc +
                 cf(18) * (A[p + sx] - A[p - sx]) + cf(19) * mix4(A, 1, sx);
    double Lu2 = cf(22) * C[p + 1] + cf(23) * C[p - 1] + cf(24) * C[p + sx] + cf(25) * C[p - sx] + cf(27) * Cc;
    if (L.three) {
      Lu0 += cf(4) * (A[p + sy] + A[p - sy]) + cf(10) * (C[p + sy] - C[p - sy]) + cf(11) * mix4(C, 1, sy);
      Lu1 += cf(16) * (B[p + sy] + B[p - sy]) + cf(20) * (C[p + sy] - C[p - sy]) + cf(21) * mix4(C, sx, sy);
      Lu2 += cf(26) * (C[p + sy] + C[p - sy]) + cf(28) * (A[p + sy] - A[p - sy]) + cf(29) * mix4(A, 1, sy) +
             cf(30) * (B[p + sy] - B[p - sy]) + cf(31) * mix4(B, sx, sy);
    }
    const double w = weighted ? cf(32) : 1.0;
    const double* fs[3] = {f0, f1, f2};
    double* rs[3] = {r0, r1, r2};
    float* qo[3] = {q0, q1, q2};
    const double Lu[3] = {Lu0, Lu1, Lu2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double fv = fs[c] ? fs[c][p] : 0.0;
      const double rv = fv - Lu[c];
      if (rs[c]) rs[c][p] = rv;
      if (qo[c]) qo[c][p] = (float)rv;
      if (red) {
        m[0] = umax64(m[0], abs_bits(rv));
        if (weighted) {
          m[1] = umax64(m[1], abs_bits(w * rv));
          m[2] = umax64(m[2], abs_bits(w * fv));
        }
      }
    }
  }
  if (red) block_max_bits<3>(m, red);
}

// f <- L(u) + f (the FAS coarse right-hand side after restriction placed
// R r into f), or out = L(u) when add == 0.
template <typename T, int G, int KIND>
__global__ void k_apply_scalar(LevelView<T> L, const T* __restrict__ u, const T* __restrict__ s0,
                               const T* __restrict__ s1, T* __restrict__ out, int add) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const long p = L.idx(i, j, k);
  T D;
  const T Lu = scalar_op<T, G, KIND>(L, u, s0, s1, i, j, k, p, D);
  out[p] = add ? out[p] + Lu : Lu;
}

template <typename T, int G>
__global__ void k_apply_vec(LevelView<T> L, const T* __restrict__ A, const T* __restrict__ B,
                            const T* __restrict__ C, T* __restrict__ o0, T* __restrict__ o1,
                            T* __restrict__ o2, int add) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const long p = L.idx(i, j, k);
  T* os[3] = {o0, o1, o2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T D;
    const T Lu = vec_op<T, G>(L, A, B, C, c, i, j, p, D);
    os[c][p] = add ? os[c][p] + Lu : Lu;
  }
}

// --------------------------------------------------------- grid transfer

// Piecewise-constant restriction (Sec. 2.7.3): coarse = volume-weighted mean
// of the 2^d children (Cartesian: the equal-weight 1/4, 1/8 stencil).
// Restricts up to 4 fields; copy (if non-null) receives a second copy of
// field 0 (the FAS u_H kept for the correction).
template <typename T>
__global__ void k_restrict(LevelView<T> F, LevelView<T> Cv, int nf, const T* __restrict__ a0,
                           const T* __restrict__ a1, const T* __restrict__ a2, const T* __restrict__ a3,
                           T* __restrict__ b0, T* __restrict__ b1, T* __restrict__ b2, T* __restrict__ b3,
                           T* __restrict__ copy0, T* __restrict__ copy1, T* __restrict__ copy2) {
  pdl_entry();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  if (I >= Cv.n0 || J >= Cv.n1 || K >= Cv.n2) return;
  const T* as[4] = {a0, a1, a2, a3};
  T* bs[4] = {b0, b1, b2, b3};
  T* cs[3] = {copy0, copy1, copy2};
  restrict_cell(F, Cv, nf, as, bs, cs, I, J, K);
}

// Kwak prolongation (Sec. 2.7.3, Fig. kwak) of e = uH - uhH, added into u.
template <typename T>
__global__ void k_prolong(LevelView<T> F, LevelView<T> Cv, T* __restrict__ u, const T* __restrict__ uH,
                          const T* __restrict__ uhH, int comp) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= F.n0 || j >= F.n1 || k >= F.n2) return;
  prolong_cell(F, Cv, u, uH, uhH, comp, i, j, k);
}

// A block of fine cells whose coarse reads (the parent and its face
// neighbours) all lie inside the coarse level: i in [i0, i1) reads coarse
// columns i0 / 2 - 1 .. (i1 - 1) / 2 + 1, likewise in j and k.  Such blocks
// run the prolongation and the residual without the boundary rules, which
// FP32 code otherwise evaluates for every cell.
__device__ __forceinline__ bool block_coarse_interior(int n0, int n1, int n2, bool three) {
  const int i0 = blockIdx.x * blockDim.x, i1 = i0 + blockDim.x;
  const int j0 = blockIdx.y * blockDim.y, j1 = j0 + blockDim.y;
  const int k0 = blockIdx.z * blockDim.z, k1 = k0 + blockDim.z;
  return i0 >= 2 && i1 + 2 <= n0 && j0 >= 2 && j1 + 2 <= n1 && (!three || (k0 >= 2 && k1 + 2 <= n2));
}

template <typename T, int NC>
__global__ void k_prolong3(LevelView<T> F, LevelView<T> Cv, Ptr3<T> u, CPtr3<T> uH, CPtr3<T> uhH, int vec) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= F.n0 || j >= F.n1 || k >= F.n2) return;
  if (block_coarse_interior(F.n0, F.n1, F.n2, F.three)) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
      prolong_cell<T, true>(F, Cv, u.at(c), uH.at(c), uhH.at(c), vec ? c : -1, i, j, k);
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) prolong_cell(F, Cv, u.at(c), uH.at(c), uhH.at(c), vec ? c : -1, i, j, k);
  }
}

// Down leg of the FP32 correction cycle at one level in one launch: the
// residual f - (L - K) e (scalar) or f - (lap + 1/3 grad div) e (vector) of
// every fine cell, with the per-cell functions of the residual kernels,
// restricted with the weights and summation order of restrict_cell into the
// coarse right-hand side fc; K restricted into Kc alongside when Kc is
// non-null; the coarse corrections ec zeroed (ghosts included).  A block
// covers a tile of fine cells whose 2 x 2 (x 2) groups are whole, keeps its
// residuals in shared memory, and one thread per coarse cell and component
// sums them: the result equals the residual kernel followed by the
// restriction, without the residual's round trip through memory.
template <int G, bool VEC>
__global__ void __launch_bounds__(256) k_resid_restrict32(LevelView<float> F, LevelView<float> Cv,
                                                          CPtr3<float> e, CPtr3<float> f,
                                                          const float* __restrict__ K, Ptr3<float> fc,
                                                          Ptr3<float> ec, float* __restrict__ Kc) {
  pdl_entry();
  constexpr int NC = VEC ? 3 : 1;
  __shared__ float rt[NC][256];
  const int bx = blockDim.x, by = blockDim.y, bz = blockDim.z;
  const int t = threadIdx.x + bx * (threadIdx.y + by * threadIdx.z);
  const int i = blockIdx.x * bx + threadIdx.x;
  const int j = blockIdx.y * by + threadIdx.y;
  const int k = blockIdx.z * bz + threadIdx.z;
  if (i < F.n0 && j < F.n1 && k < F.n2) {
    const long p = F.idx(i, j, k);
    if (VEC) {
#pragma unroll
      for (int c = 0; c < NC; ++c) rt[c][t] = vec_residual_cell<float, G>(F, e.p[0], e.p[1], e.p[2], f.at(c), c, i, j, p);
    } else if (block_coarse_interior(F.n0, F.n1, F.n2, F.three)) {
      float Sv;
      rt[0][t] = scalar_residual_cell<float, G, EQ_LIN, true>(F, e.p[0], f.p[0], nullptr, K, i, j, k, p, Sv);
    } else {
      float Sv;
      rt[0][t] = scalar_residual_cell<float, G, EQ_LIN>(F, e.p[0], f.p[0], nullptr, K, i, j, k, p, Sv);
    }
  }
  __syncthreads();
  const int cx = bx >> 1, cy = by >> 1, cz = F.three ? (bz >> 1) : 1;
  const int ncell = cx * cy * cz, nk = F.three ? 2 : 1;
  for (int w = t; w < NC * ncell; w += bx * by * bz) {
    const int c = w / ncell, q = w - c * ncell;
    const int ci = q % cx, cj = (q / cx) % cy, ck = q / (cx * cy);
    const int I = blockIdx.x * cx + ci, J = blockIdx.y * cy + cj, KK = F.three ? blockIdx.z * cz + ck : 0;
    if (I >= Cv.n0 || J >= Cv.n1 || KK >= Cv.n2) continue;
    float wi[2], wj[2];
    wi[0] = F.TI(TI_VW, 2 * I);
    wi[1] = F.TI(TI_VW, 2 * I + 1);
    wj[0] = F.TJ(TJ_VW, 2 * J);
    wj[1] = F.TJ(TJ_VW, 2 * J + 1);
    float wsum = 0.0f;
    for (int dk = 0; dk < nk; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) wsum += wi[di] * wj[dj];
    const float inv = 1.0f / wsum;
    float sr = 0.0f;
    for (int dk = 0; dk < nk; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di)
          sr += wi[di] * wj[dj] * rt[c][(2 * ci + di) + bx * ((2 * cj + dj) + by * (2 * ck + dk))];
    const long qc = Cv.idx(I, J, KK);
    fc.at(c)[qc] = sr * inv;
    if (c == 0 && Kc) {
      float sk = 0.0f;
      for (int dk = 0; dk < nk; ++dk)
        for (int dj = 0; dj < 2; ++dj)
          for (int di = 0; di < 2; ++di)
            sk += wi[di] * wj[dj] * K[F.idx(2 * I + di, 2 * J + dj, F.three ? 2 * KK + dk : 0)];
      Kc[qc] = sk * inv;
    }
  }
  const long nz = Cv.sy * (Cv.n2 + 2 * Cv.three);
  const long gt = (long)t + (long)bx * by * bz * (blockIdx.x + gridDim.x * (blockIdx.y + (long)gridDim.y * blockIdx.z));
  const long gs = (long)bx * by * bz * gridDim.x * gridDim.y * gridDim.z;
  for (long q = gt; q < nz; q += gs)
#pragma unroll
    for (int c = 0; c < NC; ++c) ec.at(c)[q] = 0.0f;
}

// --------------------------------------------------------- coarsest grid

// Block copies between global and shared memory (all ghosted cells).
template <typename T>
__device__ __forceinline__ void block_copy(T* dst, const T* src, long n) {
  for (long q = threadIdx.x; q < n; q += blockDim.x) dst[q] = src[q];
}

template <typename T, int G, int KIND>
__global__ void k_coarse_scalar(LevelView<T> L, T* __restrict__ u, const T* __restrict__ f,
                                const T* __restrict__ s0, const T* __restrict__ s1, int max_sweeps, int use_smem) {
  pdl_entry();
  if (!use_smem) {
    coarse_scalar_body<T, G, KIND>(L, u, f, s0, s1, max_sweeps);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const long ng = L.sy * (L.n2 + 2 * L.three);
  T* su = sm;
  T* sf = f ? sm + ng : nullptr;
  T* s0s = s0 ? sm + 2 * ng : nullptr;
  T* s1s = s1 ? sm + 3 * ng : nullptr;
  block_copy(su, u, ng);
  if (f) block_copy(sf, f, ng);
  if (s0) block_copy(s0s, s0, ng);
  if (s1) block_copy(s1s, s1, ng);
  __syncthreads();
  coarse_scalar_body<T, G, KIND>(L, su, sf, s0s, s1s, max_sweeps);
  __syncthreads();
  block_copy(u, su, ng);
}

template <typename T, int G>
__global__ void k_coarse_vec(LevelView<T> L, T* __restrict__ A, T* __restrict__ B, T* __restrict__ C,
                             const T* __restrict__ f0, const T* __restrict__ f1, const T* __restrict__ f2,
                             int max_sweeps, int use_smem) {
  pdl_entry();
  if (!use_smem) {
    coarse_vec_body<T, G>(L, A, B, C, f0, f1, f2, max_sweeps);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const long ng = L.sy * (L.n2 + 2 * L.three);
  T* V[3] = {sm, sm + ng, sm + 2 * ng};
  const T* fg[3] = {f0, f1, f2};
  T* fsm[3];
  for (int c = 0; c < 3; ++c) {
    fsm[c] = fg[c] ? sm + (3 + c) * ng : nullptr;
    if (fg[c]) block_copy(fsm[c], fg[c], ng);
  }
  block_copy(V[0], A, ng);
  block_copy(V[1], B, ng);
  block_copy(V[2], C, ng);
  __syncthreads();
  coarse_vec_body<T, G>(L, V[0], V[1], V[2], fsm[0], fsm[1], fsm[2], max_sweeps);
  __syncthreads();
  block_copy(A, V[0], ng);
  block_copy(B, V[1], ng);
  block_copy(C, V[2], ng);
}

// ------------------------------------------------------------- helpers

// u -= mean(u interior); sums in a fixed order (deterministic).
// Mean of the interior from nparts partial sums (warp 0 of every block).
__device__ __forceinline__ double mean_of(const double* __restrict__ part, int nparts, double ncells) {
  __shared__ double mean;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += 32) s += part[b];
    s = warp_sum(s);
    if (threadIdx.x == 0) mean = s / ncells;
  }
  __syncthreads();
  return mean;
}

template <typename T>
__global__ void k_partial_sum(LevelView<T> L, const T* __restrict__ u, double* __restrict__ part) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long stride = (long)gridDim.x * blockDim.x;
  double s = 0.0;
  if (L.n0 >= 4) {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n / 4; q += stride) {
      double v[4];
      ld4(u + group4(L, q), v);
      s += (v[0] + v[1]) + (v[2] + v[3]);
    }
  } else {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += stride) s += (double)u[interior_p(L, q)];
  }
  block_sum_to(s, part);
}

template <typename T>
__global__ void k_sub_mean(LevelView<T> L, T* __restrict__ u, const double* __restrict__ part, int nparts) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  const double mean = mean_of(part, nparts, (double)n);
  const long stride = (long)gridDim.x * blockDim.x;
  if (L.n0 >= 4) {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n / 4; q += stride) {
      const long p = group4(L, q);
      double v[4];
      ld4(u + p, v);
      for (int t = 0; t < 4; ++t) v[t] -= mean;
      st4(u + p, v);
    }
  } else {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += stride) {
      const long p = interior_p(L, q);
      u[p] = (T)((double)u[p] - mean);
    }
  }
}

// Interior <-> ghosted copies, FP64 <-> storage type conversions.
template <typename A, typename B>
__global__ void k_copy_in(LevelView<B> L, const A* __restrict__ src, B* __restrict__ dst, A shift) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    dst[L.idx(i, j, k)] = (B)(src[q] + shift);
  }
}
template <typename A, typename B>
__global__ void k_copy_out(LevelView<A> L, const A* __restrict__ src, B* __restrict__ dst, A shift) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    dst[q] = (B)(src[L.idx(i, j, k)] + shift);
  }
}
// Ghosted-to-ghosted interior conversion (e.g. FP64 residual -> FP32 rhs).
template <typename A, typename B>
__global__ void k_convert(LevelView<A> L, const A* __restrict__ src, B* __restrict__ dst) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long stride = (long)gridDim.x * blockDim.x;
  if (L.n0 >= 4) {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n / 4; q += stride) {
      const long p = group4(L, q);
      double v[4];
      ld4(src + p, v);
      st4(dst + p, v);
    }
  } else {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += stride) {
      const long p = interior_p(L, q);
      dst[p] = (B)src[p];
    }
  }
}
// u64 += e32 (interior) for ncomp fields, the defect-correction update;
// with part non-null also the block sums of the updated field 0 (for the
// Neumann gauge).
template <typename T>
__global__ void k_add_correction(LevelView<double> L, Ptr3<double> u, CPtr3<T> e, int ncomp,
                                 double* __restrict__ part) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long stride = (long)gridDim.x * blockDim.x;
  double s = 0.0;
  for (int c = 0; c < ncomp; ++c) {
    double* __restrict__ uc = u.at(c);
    const T* __restrict__ ecp = e.at(c);
    if (L.n0 >= 4) {
      for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n / 4; q += stride) {
        const long p = group4(L, q);
        double a[4], b[4];
        ld4(uc + p, a);
        ld4(ecp + p, b);
        for (int t = 0; t < 4; ++t) a[t] += b[t];
        st4(uc + p, a);
        if (c == 0) s += (a[0] + a[1]) + (a[2] + a[3]);
      }
    } else {
      for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += stride) {
        const long p = interior_p(L, q);
        uc[p] += (double)ecp[p];
        if (c == 0) s += uc[p];
      }
    }
  }
  if (part) block_sum_to(s, part);
}

// ======================================================== host launchers

template <typename T>
static dim3 grid_colour(const LevelView<T>& L, dim3 b) {
  return dim3(cdiv(L.n0 / 2, b.x), cdiv(L.n1, b.y), cdiv(L.n2, b.z));
}
template <typename T>
static dim3 grid_cells(const LevelView<T>& L, dim3 b) {
  return dim3(cdiv(L.n0, b.x), cdiv(L.n1, b.y), cdiv(L.n2, b.z));
}
static unsigned grid_flat(long n, int threads) {
  long g = (n + threads - 1) / threads;
  if (g > 4096) g = 4096;
  return (unsigned)(g < 1 ? 1 : g);
}

#define GMG_GEOM_DISPATCH(G_, ...)              \
  switch (G_) {                                  \
    case CART: { constexpr int GG = CART; __VA_ARGS__; } break; \
    case CYL:  { constexpr int GG = CYL;  __VA_ARGS__; } break; \
    default:   { constexpr int GG = SPH;  __VA_ARGS__; } break; \
  }

template <typename T>
void launch_smooth_scalar(const LevelView<T>& L, int kind, T* u, const T* f, const T* s0, const T* s1,
                          int colour, cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_colour(L, b);
  GMG_GEOM_DISPATCH(L.geom, if (kind == EQ_PSI) launch_k(k_smooth_scalar<T, GG, EQ_PSI>, g, b, 0, st, L, u, f, s0, s1, colour);
                    else launch_k(k_smooth_scalar<T, GG, EQ_LIN>, g, b, 0, st, L, u, f, s0, s1, colour));
}

template <typename T, int TX>
size_t fused_sweep_smem(bool with_c) {
  return sizeof(T) * (size_t)RbShape<TX>::BP * (RB_NU + RB_NF * (with_c ? 2 : 1));
}

// Column width of the one-launch sweep: 128 cells for FP32 levels at least
// that wide (fewer instructions per cell), else 64.
template <typename T>
int fused_sweep_tx(const LevelView<T>& L) {
  return (sizeof(T) == 4 && L.n0 % 128 == 0 && L.n1 % RbShape<128>::TY == 0) ? 128 : 64;
}

// Blocks of k_sweep_rb resident on the whole device, [geometry][TX == 128]
// [with c], set when a hierarchy is created (outside any stream capture).
static int g_fused_sms = 0;

template <typename T>
struct FusedCapacity {
  static int blocks[3][2][2];
};
template <typename T>
int FusedCapacity<T>::blocks[3][2][2] = {{{1, 1}, {1, 1}}, {{1, 1}, {1, 1}}, {{1, 1}, {1, 1}}};

template <typename T, int G, int TX, bool HAS_C>
static void set_fused_capacity(int sms) {
  const size_t smem = fused_sweep_smem<T, TX>(HAS_C);
  cudaFuncSetAttribute(k_sweep_rb<T, G, TX, HAS_C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_rb<T, G, TX, HAS_C>, RbShape<TX>::THREADS, smem) !=
          cudaSuccess ||
      nb < 1)
    nb = 1;
  FusedCapacity<T>::blocks[G][TX == 128][HAS_C] = nb * sms;
}

template <typename T, int G>
static void set_fused_capacity_g(int sms) {
  set_fused_capacity<T, G, 64, false>(sms);
  set_fused_capacity<T, G, 64, true>(sms);
  if constexpr (sizeof(T) == 4) {
    set_fused_capacity<T, G, 128, false>(sms);
    set_fused_capacity<T, G, 128, true>(sms);
  }
}

template <typename T>
void init_fused_sweep_attributes() {
  int d = 0, sms = 0;
  cudaGetDevice(&d);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || sms < 1) sms = 1;
  g_fused_sms = sms;
  set_fused_capacity_g<T, CART>(sms);
  set_fused_capacity_g<T, CYL>(sms);
  set_fused_capacity_g<T, SPH>(sms);
}

// Planes per block: each block re-relaxes two red planes beyond its chunk
// and marches two steps more than it stores.  The busiest SM decides the
// time, so take the chunk length (any, 4 to 64 planes) with the fewest
// plane steps on the SM that gets the most blocks: with the blocks resident
// at once, a 256^3 level of 32 columns takes 9 chunks of 29 planes (288
// blocks, two on almost every SM) rather than 8 of 32 (256 blocks: one SM
// in three runs a single block, the others two blocks of 34 steps).
template <typename T>
int fused_sweep_chunk(const LevelView<T>& L, int tx, bool with_c) {
  const long cols = (long)cdiv(L.n0, tx) * cdiv(L.n1, tx == 128 ? RbShape<128>::TY : RbShape<64>::TY);
  const long cap = FusedCapacity<T>::blocks[L.geom][tx == 128][with_c];
  const long sms = g_fused_sms > 0 ? g_fused_sms : 1;
  int best = 8;
  long best_cost = -1;
  for (int zc = 4; zc <= 64; ++zc) {
    const long chunks = cdiv(L.n2, zc), blocks = cols * chunks;
    const long len = cdiv(L.n2, chunks);  // the longest chunk
    const long per_sm = ((blocks + cap - 1) / cap) * ((std::min(blocks, cap) + sms - 1) / sms);
    const long cost = per_sm * (2L * len + 5);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}

template <typename T, int G, int TX>
static void launch_rb(const LevelView<T>& L, const T* uin, T* uout, const T* f, const T* c, cudaStream_t st,
                      const SweepMaps* maps) {
  const int zc = fused_sweep_chunk(L, TX, c != nullptr);
  constexpr int NT = RbShape<TX>::THREADS;
  dim3 g(cdiv(L.n0, TX), cdiv(L.n1, RbShape<TX>::TY), cdiv(L.n2, zc));
  SweepMaps none;
  std::memset(&none, 0, sizeof(none));
  const SweepMaps& M = (rb_tma<T, G, TX>() && maps) ? *maps : none;
  if (c)
    launch_k(k_sweep_rb<T, G, TX, true>, g, NT, fused_sweep_smem<T, TX>(true), st, L, uin, uout, f, c, zc, M);
  else
    launch_k(k_sweep_rb<T, G, TX, false>, g, NT, fused_sweep_smem<T, TX>(false), st, L, uin, uout, f,
             nullptr, zc, M);
}

template <typename T, int G>
static void launch_rb_g(const LevelView<T>& L, const T* uin, T* uout, const T* f, const T* c, cudaStream_t st,
                        const SweepMaps* maps) {
  if constexpr (sizeof(T) == 4) {
    if (fused_sweep_tx(L) == 128) {
      launch_rb<T, G, 128>(L, uin, uout, f, c, st, maps);
      return;
    }
  }
  launch_rb<T, G, 64>(L, uin, uout, f, c, st, maps);
}

template <typename T>
bool launch_sweep_fused(const LevelView<T>& L, const T* uin, T* uout, const T* f, const T* c, cudaStream_t st,
                        const SweepMaps* maps) {
  if (!fused_sweep_applies(L)) return false;
  count_launch();
  if (L.geom == CART)
    launch_rb_g<T, CART>(L, uin, uout, f, c, st, maps);
  else if (L.geom == CYL)
    launch_rb_g<T, CYL>(L, uin, uout, f, c, st, maps);
  else
    launch_rb_g<T, SPH>(L, uin, uout, f, c, st, maps);
  return true;
}

bool sweep_uses_maps(const LevelView<float>& L) {
  return fused_sweep_applies(L) && L.geom == CART && fused_sweep_tx(L) == 128;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
bool sweep_plane_map(CUtensorMap* m, const float* base, const LevelView<float>& L) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode enc = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<Encode>(fn);
    cudaGetLastError();
  }
  if (!enc || !base) return false;
  // (padded row index, row index, plane index) of the ghosted array; cell
  // (i, j, k) sits at (i + ROW_PAD, j + 1, k + 1)
  const cuuint64_t dims[3] = {(cuuint64_t)L.sx, (cuuint64_t)(L.n1 + 2), (cuuint64_t)(L.n2 + 2)};
  const cuuint64_t strides[2] = {(cuuint64_t)L.sx * sizeof(float), (cuuint64_t)L.sy * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)RbShape<128>::BX, (cuuint32_t)RbShape<128>::BY, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
void launch_fill_ghosts(const LevelView<T>& L, T* u, int comp, cudaStream_t st) {
  count_launch();
  const long nk = L.n2 + 2 * L.three;
  const long n = 2L * (L.n1 + 2) * nk + 2L * L.n0 * nk + (L.three ? 2L * L.n0 * L.n1 : 0L);
  launch_k(k_fill_ghosts<T>, grid_flat(n, 256), 256, 0, st, L, u, comp);
}

template <typename T>
void launch_smooth_vec(const LevelView<T>& L, T* V[3], const T* f, int comp, int colour, cudaStream_t st,
                       GhostPush gp) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_colour(L, b);
  const int nk = gp.off ? vec_cells_per_thread(L) : 1;
  if (gp.off && L.three) g.z = (unsigned)(L.n2 / (2 * nk));  // b.z = 2: planes k and k + n2 / 2 (and n2 / 4 up)
  if (nk == 2) {
    GMG_GEOM_DISPATCH(L.geom,
                      launch_k(k_smooth_vec<T, GG, 2>, g, b, 0, st, L, V[0], V[1], V[2], f, comp, colour, gp));
  } else {
    GMG_GEOM_DISPATCH(L.geom,
                      launch_k(k_smooth_vec<T, GG, 1>, g, b, 0, st, L, V[0], V[1], V[2], f, comp, colour, gp));
  }
}

template <typename T>
int vec_cells_per_thread(const LevelView<T>& L) {
  return (L.three && L.n2 % 4 == 0 && (long)L.n0 * L.n1 * L.n2 >= (1L << 19)) ? 2 : 1;
}

template <typename T>
int push_blocks(const LevelView<T>& L) {
  const dim3 b = block_for(L.three), g = grid_colour(L, b);
  return (int)(g.x * g.y * (L.three ? L.n2 / (2 * vec_cells_per_thread(L)) : 1));
}

// The block of a pass with a ghost-push table that updates cell (i, j, k),
// and the cell's slot in the block's shared new values: with NK cells per
// thread, plane k = bz + (2 tz + w) q (q = n2 / (2 NK)) is thread z = tz's
// w-th cell, slot = thread + 256 w.
template <typename T>
void push_slot(const LevelView<T>& L, int i, int j, int k, int* block, int* slot) {
  const dim3 b = block_for(L.three), g = grid_colour(L, b);
  const int t = i >> 1, nk = vec_cells_per_thread(L);
  const int q = L.three ? L.n2 / (2 * nk) : 1;
  const int bz = L.three ? k % q : 0, r = L.three ? k / q : 0;  // r = nk tz + w
  const int tz = r / nk, w = r % nk;
  *block = (int)(t / b.x + g.x * (j / b.y + g.y * bz));
  *slot = (int)(t % b.x + b.x * (j % b.y + b.y * tz)) + 256 * w;
}

template <typename T>
__global__ void k_ghost_sources(LevelView<T> L, int comp, int* __restrict__ gc, T* __restrict__ fac) {
  const long n = ghost_count(L);
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n; g += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    ghost_coords(L, g, i, j, k);
    int* o = gc + 8 * g;
    o[0] = i;
    o[1] = j;
    o[2] = k;
    o[6] = (int)L.idx(i, j, k);
    T f0, f1, f2;
    ghost_source(L, comp, i, j, k, f0, f1, f2);
    o[3] = i;
    o[4] = j;
    o[5] = k;
    o[7] = (int)L.idx(i, j, k);
    fac[g] = (f0 * f1) * f2;
  }
}

template <typename T>
void launch_ghost_sources(const LevelView<T>& L, int comp, int* gc, T* fac, cudaStream_t st) {
  count_launch();
  k_ghost_sources<T><<<grid_flat(ghost_count_host(L), 256), 256, 0, st>>>(L, comp, gc, fac);
}

template <typename T>
void launch_residual_scalar(const LevelView<T>& L, int kind, const T* u, const T* f, const T* s0,
                            const T* s1, T* r, unsigned long long* red, int weighted, cudaStream_t st, float* r32,
                            float* k32) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  g.z = cdiv(L.n2, (long)b.z * RES_KZ);
  GMG_GEOM_DISPATCH(L.geom, if (kind == EQ_PSI) launch_k(k_residual_scalar<T, GG, EQ_PSI>, g, b, 0, st, L, u, f, s0, s1, r, r32, k32, red, weighted);
                    else launch_k(k_residual_scalar<T, GG, EQ_LIN>, g, b, 0, st, L, u, f, s0, s1, r, r32, nullptr, red, weighted));
}

template <typename T>
void launch_residual_vec(const LevelView<T>& L, T* const V[3], const T* const f[3], T* const r[3],
                         unsigned long long* red, int weighted, cudaStream_t st, float* const r32[3]) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  g.z = cdiv(L.n2, (long)b.z * RES_KZ_VEC);
  float* q[3] = {nullptr, nullptr, nullptr};
  if (r32)
    for (int c = 0; c < 3; ++c) q[c] = r32[c];
  if constexpr (sizeof(T) == 8) {
    if (L.geom == SPH && L.vc && L.mixed == 0) {
      const dim3 bs(32, L.three ? 2 : 8, L.three ? 4 : 1);
      const dim3 gs(cdiv(L.n0, 32), cdiv(L.n1, bs.y), cdiv(L.n2, bs.z));
      launch_k(k_residual_vec_sph, gs, bs, 0, st, L, V[0], V[1], V[2], f[0], f[1], f[2], r[0], r[1], r[2], q[0],
               q[1], q[2], red, weighted);
      return;
    }
  }
  GMG_GEOM_DISPATCH(L.geom, launch_k(k_residual_vec<T, GG>, g, b, 0, st, L, V[0], V[1], V[2], f[0], f[1], f[2], r[0], r[1], r[2], q[0], q[1], q[2], red, weighted));
}

template <typename T>
void launch_apply_scalar(const LevelView<T>& L, int kind, const T* u, const T* s0, const T* s1, T* out, int add,
                         cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  GMG_GEOM_DISPATCH(L.geom, if (kind == EQ_PSI) launch_k(k_apply_scalar<T, GG, EQ_PSI>, g, b, 0, st, L, u, s0, s1, out, add);
                    else launch_k(k_apply_scalar<T, GG, EQ_LIN>, g, b, 0, st, L, u, s0, s1, out, add));
}

template <typename T>
void launch_apply_vec(const LevelView<T>& L, T* const V[3], T* const out[3], int add, cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  GMG_GEOM_DISPATCH(L.geom, launch_k(k_apply_vec<T, GG>, g, b, 0, st, L, V[0], V[1], V[2], out[0], out[1], out[2], add));
}

template <typename T>
void launch_restrict(const LevelView<T>& F, const LevelView<T>& C, int nf, const T* const a[4], T* const b[4],
                     T* const copy[3], cudaStream_t st) {
  count_launch();
  dim3 bl = block_for(C.three), g = grid_cells(C, bl);
  launch_k(k_restrict<T>, g, bl, 0, st, F, C, nf, a[0], a[1], a[2], a[3], b[0], b[1], b[2], b[3], copy[0], copy[1],
                                   copy[2]);
}

template <typename T>
void launch_fill_ghosts3(const LevelView<T>& L, T* const u[3], int ncomp, int vec, cudaStream_t st) {
  count_launch();
  const long n = ghost_count_host(L) * ncomp;
  launch_k(k_fill_ghosts3<T>, grid_flat(n, 256), 256, 0, st, L, u[0], ncomp > 1 ? u[1] : u[0],
           ncomp > 2 ? u[2] : u[0], ncomp, vec);
}

template <typename T>
void launch_prolong3(const LevelView<T>& F, const LevelView<T>& C, T* const u[3], const T* const uH[3],
                     const T* const uhH[3], int ncomp, int vec, cudaStream_t st) {
  count_launch();
  dim3 b = block_for(F.three), g = grid_cells(F, b);
  CPtr3<T> hh{};
  if (uhH) hh = CPtr3<T>::of(uhH, ncomp);
  if (ncomp == 1)
    launch_k(k_prolong3<T, 1>, g, b, 0, st, F, C, Ptr3<T>::of(u, 1), CPtr3<T>::of(uH, 1), hh, vec);
  else
    launch_k(k_prolong3<T, 3>, g, b, 0, st, F, C, Ptr3<T>::of(u, 3), CPtr3<T>::of(uH, 3), hh, vec);
}

void launch_resid_restrict32(const LevelView<float>& F, const LevelView<float>& C, int vec, float* const e[3],
                             float* const f[3], const float* K, float* const fc[3], float* const ec[3], float* Kc,
                             cudaStream_t st) {
  count_launch();
  const int nc = vec ? 3 : 1;
  dim3 b = block_for(F.three), g = grid_cells(F, b);
  const CPtr3<float> ce = CPtr3<float>::of(e, nc), cf = CPtr3<float>::of(f, nc);
  const Ptr3<float> pfc = Ptr3<float>::of(fc, nc), pec = Ptr3<float>::of(ec, nc);
  if (vec) {
    GMG_GEOM_DISPATCH(F.geom, launch_k(k_resid_restrict32<GG, true>, g, b, 0, st, F, C, ce, cf, K, pfc, pec, Kc));
  } else {
    GMG_GEOM_DISPATCH(F.geom, launch_k(k_resid_restrict32<GG, false>, g, b, 0, st, F, C, ce, cf, K, pfc, pec, Kc));
  }
}

template <typename T>
void launch_prolong(const LevelView<T>& F, const LevelView<T>& C, T* u, const T* uH, const T* uhH, int comp,
                    cudaStream_t st) {
  count_launch();
  dim3 b = block_for(F.three), g = grid_cells(F, b);
  launch_k(k_prolong<T>, g, b, 0, st, F, C, u, uH, uhH, comp);
}

// The coarsest level runs from shared memory when its ghosted arrays fit.
constexpr size_t COARSE_SMEM_MAX = 160 * 1024;

template <typename T>
static size_t coarse_smem_bytes(const LevelView<T>& L, int narrays) {
  const long ng = L.sy * (L.n2 + 2 * L.three);
  return sizeof(T) * (size_t)ng * narrays;
}

template <typename T>
void launch_coarse_scalar(const LevelView<T>& L, int kind, T* u, const T* f, const T* s0, const T* s1,
                          int max_sweeps, cudaStream_t st) {
  count_launch();
  const size_t sb = coarse_smem_bytes(L, 4);
  const int use = sb <= COARSE_SMEM_MAX;
  const size_t dyn = use ? sb : 0;
  GMG_GEOM_DISPATCH(L.geom, if (kind == EQ_PSI) {
    if (dyn + 16 * 1024 > 48 * 1024) cudaFuncSetAttribute(k_coarse_scalar<T, GG, EQ_PSI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    launch_k(k_coarse_scalar<T, GG, EQ_PSI>, 1, 256, dyn, st, L, u, f, s0, s1, max_sweeps, use);
  } else {
    if (dyn + 16 * 1024 > 48 * 1024) cudaFuncSetAttribute(k_coarse_scalar<T, GG, EQ_LIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    launch_k(k_coarse_scalar<T, GG, EQ_LIN>, 1, 256, dyn, st, L, u, f, s0, s1, max_sweeps, use);
  });
}

template <typename T>
void launch_coarse_vec(const LevelView<T>& L, T* V[3], const T* const f[3], int max_sweeps, cudaStream_t st) {
  count_launch();
  const size_t sb = coarse_smem_bytes(L, 6);
  const int use = sb <= COARSE_SMEM_MAX;
  const size_t dyn = use ? sb : 0;
  GMG_GEOM_DISPATCH(L.geom, {
    if (dyn + 16 * 1024 > 48 * 1024) cudaFuncSetAttribute(k_coarse_vec<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    launch_k(k_coarse_vec<T, GG>, 1, 256, dyn, st, L, V[0], V[1], V[2], f[0], f[1], f[2], max_sweeps, use);
  });
}

template <typename T>
void launch_sub_mean(const LevelView<T>& L, T* u, double* part, int nparts, cudaStream_t st, bool have_part) {
  count_launch(have_part ? 1 : 2);
  if (!have_part) launch_k(k_partial_sum<T>, nparts, 256, 0, st, L, u, part);
  launch_k(k_sub_mean<T>, nparts, 256, 0, st, L, u, part, nparts);
}

template <typename A, typename B>
void launch_copy_in(const LevelView<B>& L, const A* src, B* dst, A shift, cudaStream_t st) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  launch_k(k_copy_in<A, B>, grid_flat(n, 256), 256, 0, st, L, src, dst, shift);
}
template <typename A, typename B>
void launch_copy_out(const LevelView<A>& L, const A* src, B* dst, A shift, cudaStream_t st) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  launch_k(k_copy_out<A, B>, grid_flat(n, 256), 256, 0, st, L, src, dst, shift);
}
template <typename A, typename B>
void launch_convert(const LevelView<A>& L, const A* src, B* dst, cudaStream_t st) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  launch_k(k_convert<A, B>, grid_flat(L.n0 >= 4 ? n / 4 : n, 256), 256, 0, st, L, src, dst);
}
template <typename T>
void launch_add_correction(const LevelView<double>& L, int ncomp, double* const u[3], const T* const e[3],
                           cudaStream_t st, double* part, int nparts) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  const unsigned g = part ? (unsigned)nparts : grid_flat((L.n0 >= 4 ? n / 4 : n) * ncomp, 256);
  launch_k(k_add_correction<T>, g, 256, 0, st, L, Ptr3<double>::of(u, ncomp), CPtr3<T>::of(e, ncomp), ncomp,
           part);
}

// explicit instantiations
#define GMG_INST(T)                                                                                            \
  template bool launch_sweep_fused<T>(const LevelView<T>&, const T*, T*, const T*, const T*, cudaStream_t,      \
                                      const SweepMaps*);                                                          \
  template void init_fused_sweep_attributes<T>();                                                              \
  template void launch_smooth_scalar<T>(const LevelView<T>&, int, T*, const T*, const T*, const T*, int,       \
                                        cudaStream_t);                                                          \
  template void launch_fill_ghosts<T>(const LevelView<T>&, T*, int, cudaStream_t);                             \
  template void launch_fill_ghosts3<T>(const LevelView<T>&, T* const[3], int, int, cudaStream_t);             \
  template void launch_prolong3<T>(const LevelView<T>&, const LevelView<T>&, T* const[3], const T* const[3],  \
                                   const T* const[3], int, int, cudaStream_t);                                 \
  template void launch_smooth_vec<T>(const LevelView<T>&, T* [3], const T*, int, int, cudaStream_t, GhostPush); \
  template int push_blocks<T>(const LevelView<T>&);                                                            \
  template int vec_cells_per_thread<T>(const LevelView<T>&);                                                   \
  template void push_slot<T>(const LevelView<T>&, int, int, int, int*, int*);                                  \
  template void launch_residual_scalar<T>(const LevelView<T>&, int, const T*, const T*, const T*, const T*, T*, \
                                          unsigned long long*, int, cudaStream_t, float*, float*);              \
  template void launch_residual_vec<T>(const LevelView<T>&, T* const[3], const T* const[3], T* const[3],       \
                                       unsigned long long*, int, cudaStream_t, float* const[3]);                \
  template void launch_apply_scalar<T>(const LevelView<T>&, int, const T*, const T*, const T*, T*, int,        \
                                       cudaStream_t);                                                           \
  template void launch_apply_vec<T>(const LevelView<T>&, T* const[3], T* const[3], int, cudaStream_t);         \
  template void launch_restrict<T>(const LevelView<T>&, const LevelView<T>&, int, const T* const[4],           \
                                   T* const[4], T* const[3], cudaStream_t);                                     \
  template void launch_prolong<T>(const LevelView<T>&, const LevelView<T>&, T*, const T*, const T*, int,       \
                                  cudaStream_t);                                                                \
  template void launch_coarse_scalar<T>(const LevelView<T>&, int, T*, const T*, const T*, const T*, int,       \
                                        cudaStream_t);                                                          \
  template void launch_coarse_vec<T>(const LevelView<T>&, T* [3], const T* const[3], int, cudaStream_t);       \
  template void launch_sub_mean<T>(const LevelView<T>&, T*, double*, int, cudaStream_t, bool);
GMG_INST(double)
GMG_INST(float)
template void launch_ghost_sources<double>(const LevelView<double>&, int, int*, double*, cudaStream_t);
template void launch_copy_in<double, double>(const LevelView<double>&, const double*, double*, double, cudaStream_t);
template void launch_copy_out<double, double>(const LevelView<double>&, const double*, double*, double, cudaStream_t);
template void launch_convert<double, float>(const LevelView<double>&, const double*, float*, cudaStream_t);
template void launch_convert<float, double>(const LevelView<float>&, const float*, double*, cudaStream_t);
template void launch_add_correction<float>(const LevelView<double>&, int, double* const[3], const float* const[3],
                                           cudaStream_t, double*,
                                           int);

}  // namespace gmg
