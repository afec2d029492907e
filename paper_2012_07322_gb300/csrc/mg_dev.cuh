// Device-side building blocks of the multigrid solver: the per-level view
// passed to kernels, ghost / boundary rules, the discrete operators of
// Sec. 2.7.1 (scalar flux-form Laplacian, vector operator lap V + 1/3 grad
// div V of eqs. X and beta) and block reductions.
//
// Storage: every level array is "ghosted": one ghost layer per active
// dimension, dimension 0 fastest, element (i, j, k) at
// off + i + j * sx + k * sy with i in [-1, n0], j in [-1, n1], k in
// [-three, n2 - 1 + three].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gmg {

// Programmatic dependent launch (every kernel is launched with it, see
// launch_k): wait until the preceding kernel in the stream has completed and
// its writes are visible (a no-op for a kernel launched without it), then
// allow the next kernel to be scheduled while this one runs.  Called first
// in every kernel, so no kernel touches memory before its predecessor is
// done; what it saves is the launch latency between dependent kernels.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

enum Geom { CART = 0, CYL = 1, SPH = 2 };
enum Bc { BC_ROBIN = 0, BC_DIRICHLET = 1, BC_NEUMANN = 2 };
enum Kind { EQ_PSI = 0, EQ_LIN = 1, EQ_VEC = 2 };

// Per-i table slots (length n0 + 2, entry i + 1).
enum { TI_X = 0, TI_IX, TI_IX2, TI_CE, TI_CW, TI_PHI, TI_VW, NTI };
// Per-j table slots (length n1 + 2, entry j + 1).
enum { TJ_S = 0, TJ_C, TJ_IS, TJ_IS2, TJ_COT, TJ_TN, TJ_TS, TJ_PF, TJ_VW, NTJ };
// Per-(i, j) stencil coefficients of the vector operator on spherical
// levels with four-point mixed derivatives (FP64 residual), stored
// coefficient-major: vc[(q * n1 + j) * n0 + i].  Slots 0-11 component r,
// 12-21 theta, 22-31 phi (k_residual_vec_sph), 32 the norm weight.
constexpr int VC_N = 34;

template <typename T>
struct LevelView {
  int n0, n1, n2, three;
  int geom, bc, mixed;
  long sx, sy, off;
  T h0, h1, h2;        // spacings
  T lo0, lo1, lo2;     // domain origin
  T ih0s, ih1s, ih2s;  // 1 / h^2
  T hc0, hc1, hc2;     // 1 / (2 h): central first differences
  T m01, m02, m12;     // mixed-derivative factors: 1/(4 ha hb), or 1/(2 ha hb) (block-corner)
  T robin0;            // spherical Robin ghost factor r_{n-1} / r_n
  int ln0, ln1;        // log2 of n0, n1 (all sizes are powers of two)
  const T* ti;         // NTI tables of n0 + 2
  const T* tj;         // NTJ tables of n1 + 2
  const T* vc;         // VC_N per-(i, j) coefficients of the vector operator, or null
  __device__ __forceinline__ long idx(int i, int j, int k) const { return off + i + j * sx + (long)k * sy; }
  __device__ __forceinline__ T TI(int s, int i) const { return ti[s * (n0 + 2) + i + 1]; }
  __device__ __forceinline__ T TJ(int s, int j) const { return tj[s * (n1 + 2) + j + 1]; }
  // Interior cell (i, j, k) of the flat index r = i + n0 (j + n1 k).
  __device__ __forceinline__ void cell(long r, int& i, int& j, int& k) const {
    i = (int)(r & (n0 - 1));
    const long jk = r >> ln0;
    j = (int)(jk & (n1 - 1));
    k = (int)(jk >> ln1);
  }
  // Cell (i, j, k) of colour (i + j + k) % 2 from its rank r among the
  // cells of that colour (n0 even): i = 2 t + parity, t the rank in the row.
  __device__ __forceinline__ void colour_cell(long r, int colour, int& i, int& j, int& k) const {
    const int t = (int)(r & ((n0 >> 1) - 1));
    const long jk = r >> (ln0 - 1);
    j = (int)(jk & (n1 - 1));
    k = (int)(jk >> ln1);
    i = 2 * t + ((j + k + colour) & 1);
  }
  __device__ __forceinline__ T xc0(int i) const { return lo0 + (T(i) + T(0.5)) * h0; }
  __device__ __forceinline__ T xc1(int j) const { return lo1 + (T(j) + T(0.5)) * h1; }
  __device__ __forceinline__ T xc2(int k) const { return lo2 + (T(k) + T(0.5)) * h2; }
};

// ----------------------------------------------------------- boundaries

// Parity of a component across the spherical origin or the cylinder axis
// (physical components of a regular vector field; comp < 0: scalar).
__host__ __device__ __forceinline__ int parity_origin(int comp) {
  return comp < 0 ? 1 : (comp == 1 ? 1 : -1);
}
// Parity across the spherical polar axis (theta = 0, pi).
__host__ __device__ __forceinline__ int parity_axis(int comp) {
  return comp < 0 ? 1 : (comp == 0 ? 1 : -1);
}

// Distance from the origin (Cartesian / cylindrical Robin rule).
template <typename T>
__device__ __forceinline__ T rho_at(const LevelView<T>& L, int i, int j, int k) {
  T x = L.xc0(i), y = L.xc1(j);
  T s = x * x + y * y;
  if (L.geom == CART && L.three) {
    T z = L.xc2(k);
    s += z * z;
  }
  return sqrt(s);
}

// rho(source cell) / rho(ghost) for the Cartesian / cylindrical Robin
// rule (z = 0 when the distance has no third term).  Out of line: inlined,
// the compiler may evaluate its square roots and division speculatively on
// every stencil that only might touch the boundary, which costs FP64 kernels
// far more than the rare call.
template <typename T>
__device__ __noinline__ T robin_rho_ratio(T xs, T ys, T zs, T xg, T yg, T zg) {
  T s = xs * xs + ys * ys;
  s += zs * zs;
  T g = xg * xg + yg * yg;
  g += zg * zg;
  return sqrt(s) / sqrt(g);
}

// Factor g / u_src of an outer-boundary ghost (eq. bc / eq. robin):
// Dirichlet-0 -> -1, Neumann -> +1, Robin -> u ~ 1/distance.
template <typename T>
__device__ __forceinline__ T outer_factor(const LevelView<T>& L, int gi, int gj, int gk, int si, int sj,
                                          int sk) {
  if (L.bc == BC_DIRICHLET) return T(-1);
  if (L.bc == BC_NEUMANN) return T(1);
  if (L.geom == SPH) return L.robin0;
  const bool z3 = L.geom == CART && L.three;
  return robin_rho_ratio(L.xc0(si), L.xc1(sj), z3 ? L.xc2(sk) : T(0), L.xc0(gi), L.xc1(gj),
                         z3 ? L.xc2(gk) : T(0));
}

// Source of a face ghost: the ghost at (i,j,k) lies outside exactly one
// dimension d (the others may be interior or ghosts already resolved).
// Returns the index triple of the cell it copies from and its factor.
// Mirrors the fill order of dimension 0, then 1, then 2.
template <typename T>
__device__ __forceinline__ T ghost_rule(const LevelView<T>& L, int comp, int d, int& i, int& j, int& k) {
  const int n0 = L.n0, n1 = L.n1, n2 = L.n2;
  if (d == 0) {
    if (i < 0) {
      if (L.geom == CART) {
        T f = outer_factor(L, -1, j, k, 0, j, k);
        i = 0;
        return f;
      }
      int ks = L.three ? (k + n2 / 2) % n2 : k;
      if (L.geom == CYL) {
        i = 0;
        k = ks;
        return T(parity_origin(comp));
      }
      i = 0;
      j = n1 - 1 - j;
      k = ks;
      return T(parity_origin(comp));
    }
    T f = outer_factor(L, n0, j, k, n0 - 1, j, k);
    i = n0 - 1;
    return f;
  }
  if (d == 1) {
    if (L.geom == SPH) {
      int ks = L.three ? (k + n2 / 2) % n2 : k;
      j = (j < 0) ? 0 : n1 - 1;
      k = ks;
      return T(parity_axis(comp));
    }
    if (j < 0) {
      T f = outer_factor(L, i, -1, k, i, 0, k);
      j = 0;
      return f;
    }
    T f = outer_factor(L, i, n1, k, i, n1 - 1, k);
    j = n1 - 1;
    return f;
  }
  // d == 2 (3D only)
  if (L.geom != CART) {
    k = (k < 0) ? n2 - 1 : 0;
    return T(1);
  }
  if (k < 0) {
    T f = outer_factor(L, i, j, -1, i, j, 0);
    k = 0;
    return f;
  }
  T f = outer_factor(L, i, j, n2, i, j, n2 - 1);
  k = n2 - 1;
  return f;
}

// Interior source of any ghost (face, edge or corner): (i, j, k) becomes
// the cell the ghost derives from, f0, f1, f2 the factors of the
// per-dimension rules, composed in the fill order 0, 1, 2.
template <typename T>
__device__ __forceinline__ void ghost_source(const LevelView<T>& L, int comp, int& i, int& j, int& k, T& f0,
                                             T& f1, T& f2) {
  f2 = f1 = f0 = T(1);
  if (L.three && (k < 0 || k >= L.n2)) f2 = ghost_rule(L, comp, 2, i, j, k);
  if (j < 0 || j >= L.n1) f1 = ghost_rule(L, comp, 1, i, j, k);
  if (i < 0 || i >= L.n0) f0 = ghost_rule(L, comp, 0, i, j, k);
}

// Value of any ghost of field u from its interior.
template <typename T>
__device__ __forceinline__ T ghost_value(const LevelView<T>& L, const T* __restrict__ u, int comp, int i,
                                         int j, int k) {
  T f0, f1, f2;
  ghost_source(L, comp, i, j, k, f0, f1, f2);
  return ((u[L.idx(i, j, k)] * f0) * f1) * f2;
}

// ------------------------------------------------------ scalar operator

// The six neighbour values a cell's scalar Laplacian uses.
template <typename T>
struct Nb6 {
  T e, w, n, s, up, dn;
};

// Neighbours of a cell on the edge of the level: outer ghosts from the
// boundary rule on the fly, the origin / axis neighbours replaced by the
// cell itself (their face areas vanish, so they drop out of the flux),
// periodic phi neighbours wrapped.  FP64 kernels call it out of line
// (lap_edge_neighbours): interior cells, the vast majority, never evaluate
// the boundary rules there.
template <typename T, int G>
__device__ __forceinline__ Nb6<T> lap_edge_neighbours_body(const LevelView<T>& L, const T* __restrict__ u, int i,
                                                           int j, int k, long p) {
  const T uc = u[p];
  Nb6<T> nb;
  nb.e = (i < L.n0 - 1) ? u[p + 1] : outer_factor(L, L.n0, j, k, L.n0 - 1, j, k) * uc;
  if (G == CART)
    nb.w = (i > 0) ? u[p - 1] : outer_factor(L, -1, j, k, 0, j, k) * uc;
  else
    nb.w = (i > 0) ? u[p - 1] : uc;  // R_{-1/2} = 0 / r_{-1/2} = 0
  if (G == SPH) {
    nb.n = (j < L.n1 - 1) ? u[p + L.sx] : uc;  // sin(theta) = 0 on the poles
    nb.s = (j > 0) ? u[p - L.sx] : uc;
  } else {
    nb.n = (j < L.n1 - 1) ? u[p + L.sx] : outer_factor(L, i, L.n1, k, i, L.n1 - 1, k) * uc;
    nb.s = (j > 0) ? u[p - L.sx] : outer_factor(L, i, -1, k, i, 0, k) * uc;
  }
  nb.up = nb.dn = uc;
  if (L.three) {
    if (G == CART) {
      nb.up = (k < L.n2 - 1) ? u[p + L.sy] : outer_factor(L, i, j, L.n2, i, j, L.n2 - 1) * uc;
      nb.dn = (k > 0) ? u[p - L.sy] : outer_factor(L, i, j, -1, i, j, 0) * uc;
    } else {
      nb.up = (k < L.n2 - 1) ? u[p + L.sy] : u[p - (long)(L.n2 - 1) * L.sy];
      nb.dn = (k > 0) ? u[p - L.sy] : u[p + (long)(L.n2 - 1) * L.sy];
    }
  }
  return nb;
}
template <typename T, int G>
__device__ __noinline__ Nb6<T> lap_edge_neighbours(const LevelView<T>& L, const T* __restrict__ u, int i, int j,
                                                   int k, long p) {
  return lap_edge_neighbours_body<T, G>(L, u, i, j, k, p);
}

// Flux-form Laplacian (Sec. 2.7.1) at an interior cell, with outer ghosts
// taken from the boundary rule on the fly and the origin / axis fluxes
// (whose face areas vanish) dropped; periodic phi neighbours wrap.  D gets
// the derivative with respect to the cell's own value (ghosts held fixed).
// INNER: the caller knows the cell is interior (a block whose cells all
// are), and no edge code is compiled in.
template <typename T, int G, bool INNER = false>
__device__ __forceinline__ T lap_scalar(const LevelView<T>& L, const T* __restrict__ u, int i, int j, int k,
                                        long p, T& D) {
  const T uc = u[p];
  Nb6<T> nb;
  const bool inner =
      INNER || (i > 0 && i < L.n0 - 1 && j > 0 && j < L.n1 - 1 && (!L.three || (k > 0 && k < L.n2 - 1)));
  if (inner) {
    nb.e = u[p + 1];
    nb.w = u[p - 1];
    nb.n = u[p + L.sx];
    nb.s = u[p - L.sx];
    nb.up = L.three ? u[p + L.sy] : uc;
    nb.dn = L.three ? u[p - L.sy] : uc;
  } else if constexpr (INNER) {
  } else if constexpr (sizeof(T) == 4) {
    // FP32: the edge rules inline (speculating them costs the FP32 units
    // little; a call passes the neighbours through local memory)
    nb = lap_edge_neighbours_body<T, G>(L, u, i, j, k, p);
  } else {
    nb = lap_edge_neighbours<T, G>(L, u, i, j, k, p);
  }
  const T cE = L.TI(TI_CE, i), cW = L.TI(TI_CW, i);
  T Lu = cE * (nb.e - uc) - cW * (uc - nb.w);
  D = -(cE + cW);
  if (G == SPH) {
    const T ir2 = L.TI(TI_IX2, i);
    const T tN = L.TJ(TJ_TN, j), tS = L.TJ(TJ_TS, j);
    Lu += ir2 * (tN * (nb.n - uc) - tS * (uc - nb.s));
    D -= ir2 * (tN + tS);
  } else {
    Lu += L.ih1s * (nb.n - T(2) * uc + nb.s);
    D -= T(2) * L.ih1s;
  }
  if (L.three) {
    T c;
    if (G == CART)
      c = L.ih2s;
    else if (G == CYL)
      c = L.TI(TI_PHI, i);
    else
      c = L.TI(TI_IX2, i) * L.TJ(TJ_PF, j);
    Lu += c * (nb.up - T(2) * uc + nb.dn);
    D -= T(2) * c;
  }
  return Lu;
}

// ------------------------------------------------------ vector operator
// Fields with materialised ghosts (edges included).  Components are the
// orthonormal ones: (x, y, z), (R, z, phi), (r, theta, phi).

template <typename T>
struct Stencil {
  const LevelView<T>& L;
  long p;
  __device__ __forceinline__ T d1(const T* F, int d) const {
    if (d == 0) return (F[p + 1] - F[p - 1]) * L.hc0;
    if (d == 1) return (F[p + L.sx] - F[p - L.sx]) * L.hc1;
    if (!L.three) return T(0);
    return (F[p + L.sy] - F[p - L.sy]) * L.hc2;
  }
  __device__ __forceinline__ long step(int d) const { return d == 0 ? 1 : (d == 1 ? L.sx : L.sy); }
  __device__ __forceinline__ T hs(int d) const { return d == 0 ? L.ih0s : (d == 1 ? L.ih1s : L.ih2s); }
  __device__ __forceinline__ T d2(const T* F, int d) const {
    if (d == 2 && !L.three) return T(0);
    long s = step(d);
    return (F[p + s] - T(2) * F[p] + F[p - s]) * hs(d);
  }
  __device__ __forceinline__ T mix(const T* F, int a, int b) const {
    if (b == 2 && !L.three) return T(0);
    long sa = step(a), sb = step(b);
    const T w = (a == 0 && b == 1) ? L.m01 : (a == 0 ? L.m02 : L.m12);
    if (L.mixed == 0) return (F[p + sa + sb] - F[p + sa - sb] - F[p - sa + sb] + F[p - sa - sb]) * w;
    return (-F[p + sa - sb] - F[p - sa + sb] + F[p + sa] + F[p - sa] + F[p + sb] + F[p - sb] - T(2) * F[p]) * w;
  }
};

// Flux-form Laplacian of a component with materialised ghosts.
template <typename T, int G>
__device__ __forceinline__ T lap_ghosted(const LevelView<T>& L, const T* __restrict__ F, int i, int j, long p,
                                         T& D) {
  const T c = F[p];
  const T cE = L.TI(TI_CE, i), cW = L.TI(TI_CW, i);
  T Lu = cE * (F[p + 1] - c) - cW * (c - F[p - 1]);
  D = -(cE + cW);
  if (G == SPH) {
    const T ir2 = L.TI(TI_IX2, i);
    const T tN = L.TJ(TJ_TN, j), tS = L.TJ(TJ_TS, j);
    Lu += ir2 * (tN * (F[p + L.sx] - c) - tS * (c - F[p - L.sx]));
    D -= ir2 * (tN + tS);
  } else {
    Lu += L.ih1s * (F[p + L.sx] - T(2) * c + F[p - L.sx]);
    D -= T(2) * L.ih1s;
  }
  if (L.three) {
    T cc = (G == CART) ? L.ih2s : (G == CYL ? L.TI(TI_PHI, i) : L.TI(TI_IX2, i) * L.TJ(TJ_PF, j));
    Lu += cc * (F[p + L.sy] - T(2) * c + F[p - L.sy]);
    D -= T(2) * cc;
  }
  return Lu;
}

// Component c of lap V + 1/3 grad div V on a spherical level from the
// per-(i, j) stencil coefficients L.vc (four-point mixed derivatives; slot
// layout of VC_N), and its own-value derivative (the centre coefficient).
// The operator of the flux form below with the metric factors multiplied
// out: about a third of the arithmetic and a third of the table loads.
template <typename T>
__device__ __forceinline__ T vec_op_vc(const LevelView<T>& L, const T* __restrict__ A, const T* __restrict__ B,
                                       const T* __restrict__ C, int c, int i, int j, long p, T& diag) {
  const long sx = L.sx, sy = L.sy, qs = (long)L.n0 * L.n1;
  const T* __restrict__ V = L.vc + (long)j * L.n0 + i;
  auto cf = [&](int q) { return V[q * qs]; };
  auto mix4 = [&](const T* F, long a, long b) {
    return ((F[p + a + b] - F[p + a - b]) - F[p - a + b]) + F[p - a - b];
  };
  T Lu;
  if (c == 0) {
    diag = cf(5);
    Lu = cf(0) * A[p + 1] + cf(1) * A[p - 1] + cf(2) * A[p + sx] + cf(3) * A[p - sx] + diag * A[p] +
         cf(6) * (B[p + sx] - B[p - sx]) + cf(7) * B[p] + cf(8) * (B[p + 1] - B[p - 1]) + cf(9) * mix4(B, 1, sx);
    if (L.three)
      Lu += cf(4) * (A[p + sy] + A[p - sy]) + cf(10) * (C[p + sy] - C[p - sy]) + cf(11) * mix4(C, 1, sy);
  } else if (c == 1) {
    diag = cf(17);
    Lu = cf(12) * B[p + 1] + cf(13) * B[p - 1] + cf(14) * B[p + sx] + cf(15) * B[p - sx] + diag * B[p] +
         cf(18) * (A[p + sx] - A[p - sx]) + cf(19) * mix4(A, 1, sx);
    if (L.three)
      Lu += cf(16) * (B[p + sy] + B[p - sy]) + cf(20) * (C[p + sy] - C[p - sy]) + cf(21) * mix4(C, sx, sy);
  } else {
    diag = cf(27);
    Lu = cf(22) * C[p + 1] + cf(23) * C[p - 1] + cf(24) * C[p + sx] + cf(25) * C[p - sx] + diag * C[p];
    if (L.three)
      Lu += cf(26) * (C[p + sy] + C[p - sy]) + cf(28) * (A[p + sy] - A[p - sy]) + cf(29) * mix4(A, 1, sy) +
            cf(30) * (B[p + sy] - B[p - sy]) + cf(31) * mix4(B, sx, sy);
  }
  return Lu;
}

// Component c of lap V + 1/3 grad div V and its own-value derivative.  VC
// false compiles the flux form only (the one-block cycle: its register
// budget of 128 would spill with both forms).
template <typename T, int G, bool VC = true>
__device__ __forceinline__ T vec_op(const LevelView<T>& L, const T* __restrict__ A, const T* __restrict__ B,
                                    const T* __restrict__ C, int c, int i, int j, long p, T& diag) {
  if constexpr (VC && G == SPH && sizeof(T) == 4) {
    // FP32 (smoother and correction residual of mixed precision): the
    // coefficient form when the level carries the table
    if (L.vc && L.mixed == 0) return vec_op_vc<T>(L, A, B, C, c, i, j, p, diag);
  }
  const T third = T(1) / T(3);
  Stencil<T> s{L, p};
  T LD;
  if (G == CART) {
    const T* V = (c == 0) ? A : (c == 1 ? B : C);
    T v = lap_ghosted<T, G>(L, V, i, j, p, LD);
    T gd;
    if (c == 0)
      gd = s.d2(A, 0) + s.mix(B, 0, 1) + s.mix(C, 0, 2);
    else if (c == 1)
      gd = s.mix(A, 0, 1) + s.d2(B, 1) + s.mix(C, 1, 2);
    else
      gd = s.mix(A, 0, 2) + s.mix(B, 1, 2) + s.d2(C, 2);
    const bool has = (c < 2) || L.three;
    diag = LD + (has ? third * (T(-2) * s.hs(c)) : T(0));
    return v + third * gd;
  }
  if (G == CYL) {
    const T iR = L.TI(TI_IX, i), iR2 = L.TI(TI_IX2, i);
    if (c == 0) {
      T v = lap_ghosted<T, G>(L, A, i, j, p, LD) - iR2 * A[p] - T(2) * iR2 * s.d1(C, 2);
      T gd = s.d2(A, 0) + iR * s.d1(A, 0) - iR2 * A[p] + s.mix(B, 0, 1) + iR * s.mix(C, 0, 2) -
             iR2 * s.d1(C, 2);
      diag = LD - iR2 + third * (T(-2) * L.ih0s - iR2);
      return v + third * gd;
    } else if (c == 1) {
      T v = lap_ghosted<T, G>(L, B, i, j, p, LD);
      T gd = s.mix(A, 0, 1) + iR * s.d1(A, 1) + s.d2(B, 1) + iR * s.mix(C, 1, 2);
      diag = LD + third * (T(-2) * L.ih1s);
      return v + third * gd;
    } else {
      T v = lap_ghosted<T, G>(L, C, i, j, p, LD) - iR2 * C[p] + T(2) * iR2 * s.d1(A, 2);
      T gd = iR * s.mix(A, 0, 2) + iR2 * s.d1(A, 2) + iR * s.mix(B, 1, 2) + iR2 * s.d2(C, 2);
      diag = LD - iR2 + (L.three ? third * (T(-2) * iR2 * L.ih2s) : T(0));
      return v + third * gd;
    }
  }
  // spherical
  const T ir = L.TI(TI_IX, i), ir2 = L.TI(TI_IX2, i);
  const T ist = L.TJ(TJ_IS, j), ist2 = L.TJ(TJ_IS2, j), ct = L.TJ(TJ_C, j), cot = L.TJ(TJ_COT, j);
  if (c == 0) {
    T v = lap_ghosted<T, G>(L, A, i, j, p, LD) - T(2) * ir2 * A[p] - T(2) * ir2 * s.d1(B, 1) -
          T(2) * cot * ir2 * B[p] - T(2) * ir2 * ist * s.d1(C, 2);
    T gd = s.d2(A, 0) + T(2) * ir * s.d1(A, 0) - T(2) * ir2 * A[p] + ir * s.mix(B, 0, 1) - ir2 * s.d1(B, 1) +
           cot * ir * s.d1(B, 0) - cot * ir2 * B[p] + ir * ist * s.mix(C, 0, 2) - ir2 * ist * s.d1(C, 2);
    diag = LD - T(2) * ir2 + third * (T(-2) * L.ih0s - T(2) * ir2);
    return v + third * gd;
  } else if (c == 1) {
    T v = lap_ghosted<T, G>(L, B, i, j, p, LD) - ir2 * ist2 * B[p] + T(2) * ir2 * s.d1(A, 1) -
          T(2) * ct * ir2 * ist2 * s.d1(C, 2);
    T gd = ir * s.mix(A, 0, 1) + T(2) * ir2 * s.d1(A, 1) + ir2 * s.d2(B, 1) + cot * ir2 * s.d1(B, 1) -
           ir2 * ist2 * B[p] - ct * ir2 * ist2 * s.d1(C, 2) + ir2 * ist * s.mix(C, 1, 2);
    diag = LD - ir2 * ist2 + third * (T(-2) * ir2 * L.ih1s - ir2 * ist2);
    return v + third * gd;
  } else {
    T v = lap_ghosted<T, G>(L, C, i, j, p, LD) - ir2 * ist2 * C[p] + T(2) * ir2 * ist * s.d1(A, 2) +
          T(2) * ct * ir2 * ist2 * s.d1(B, 2);
    T gd = ir * ist * s.mix(A, 0, 2) + T(2) * ir2 * ist * s.d1(A, 2) + ir2 * ist * s.mix(B, 1, 2) +
           cot * ir2 * ist * s.d1(B, 2) + ir2 * ist2 * s.d2(C, 2);
    diag = LD - ir2 * ist2 + (L.three ? third * (T(-2) * ir2 * ist2 * L.ih2s) : T(0));
    return v + third * gd;
  }
}

// Weight of the stopping norm: r^2 sin(theta) / R / 1.
template <typename T>
__device__ __forceinline__ T norm_weight(const LevelView<T>& L, int i, int j) {
  if (L.geom == SPH) {
    T r = L.TI(TI_X, i);
    return r * r * L.TJ(TJ_S, j);
  }
  if (L.geom == CYL) return L.TI(TI_X, i);
  return T(1);
}

// ------------------------------------------------------------ reductions

// Non-negative doubles order like their bit patterns; non-finite values
// are recorded as +inf.
__device__ __forceinline__ unsigned long long ord_bits(double v) {
  if (!(v <= 1.7976931348623157e308)) v = __longlong_as_double(0x7ff0000000000000LL);
  return (unsigned long long)__double_as_longlong(v);
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// |v| as ordered bits (non-negative doubles order like their bit
// patterns); NaN -> +inf.  Integer work only: on GPUs with few FP64 units
// the norms of a residual must not compete with its stencil for them.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
  return b > 0x7ff0000000000000ULL ? 0x7ff0000000000000ULL : b;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long warp_max_bits(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide max of NV values given as abs_bits, one atomicMax per value
// per block.  Every thread of the block must call it.
template <int NV>
__device__ __forceinline__ void block_max_bits(unsigned long long (&v)[NV], unsigned long long* out) {
  __shared__ unsigned long long sm[NV][32];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const unsigned long long x = warp_max_bits(v[q]);
    if (lane == 0) sm[q][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (nthr + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const unsigned long long x = warp_max_bits((lane < nw) ? sm[q][lane] : 0ULL);
      if (lane == 0 && x > 0ULL) atomicMax(out + q, x);
    }
  }
}

// Block-wide max of NV non-negative doubles (NaN -> +inf).
template <int NV>
__device__ __forceinline__ void block_max_atomic(double (&v)[NV], unsigned long long* out) {
  unsigned long long b[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) b[q] = abs_bits(v[q]);
  block_max_bits<NV>(b, out);
}

}  // namespace gmg
