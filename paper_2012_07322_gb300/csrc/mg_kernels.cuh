// Per-cell work of the multigrid kernels, shared by the grid-wide kernels
// and the single-block coarsest-grid solver.
#pragma once
#include "mg_dev.cuh"

namespace gmg {

constexpr double PI_D = 3.14159265358979323846;

// Operator L(u) of a scalar equation at a cell (Sec. 2.7.1 / eqs. psi,
// alpha) and dL/du_ijk:
//   EQ_PSI: lap u + 2 pi U (1+u)^-1 + 1/8 A2 (1+u)^-7   (s0 = U, s1 = A2)
//   EQ_LIN: lap u - c u                                  (s1 = c, nullable)
template <typename T, int G, int KIND>
__device__ __forceinline__ T scalar_op(const LevelView<T>& L, const T* __restrict__ u,
                                       const T* __restrict__ s0, const T* __restrict__ s1, int i, int j,
                                       int k, long p, T& D) {
  T Lu = lap_scalar<T, G>(L, u, i, j, k, p, D);
  if (KIND == EQ_PSI) {
    const T ip = T(1) / (T(1) + u[p]);
    const T ip2 = ip * ip;
    const T ip4 = ip2 * ip2;
    const T ip7 = ip4 * ip2 * ip;
    const T a = T(2 * PI_D) * s0[p];
    const T b = s1[p];
    Lu += a * ip + T(0.125) * b * ip7;
    D -= a * ip2 + T(0.875) * b * ip7 * ip;
  } else {
    if (s1) {
      const T c = s1[p];
      Lu -= c * u[p];
      D -= c;
    }
  }
  return Lu;
}

// Source S(u) as the paper writes the right-hand side (stopping norm).
template <typename T, int KIND>
__device__ __forceinline__ T scalar_source(const T* __restrict__ u, const T* __restrict__ s0,
                                           const T* __restrict__ s1, const T* __restrict__ f, long p) {
  if (KIND == EQ_PSI) {
    const T ip = T(1) / (T(1) + u[p]);
    const T ip2 = ip * ip;
    const T ip7 = ip2 * ip2 * ip2 * ip;
    return -T(2 * PI_D) * s0[p] * ip - T(0.125) * s1[p] * ip7;
  }
  T s = f ? f[p] : T(0);
  if (s1) s += s1[p] * u[p];
  return s;
}

// One Newton-Gauss-Seidel update (eq. ngs_iteration) of a scalar cell.
// For eq. psi the step N / dN is evaluated with one division: numerator and
// denominator are both multiplied by p^8, p = 1 + u (p ~ 1, no overflow).
template <typename T, int G, int KIND>
__device__ __forceinline__ void scalar_update(const LevelView<T>& L, T* __restrict__ u,
                                              const T* __restrict__ f, const T* __restrict__ s0,
                                              const T* __restrict__ s1, int i, int j, int k) {
  const long p = L.idx(i, j, k);
  T D;
  const T lap = lap_scalar<T, G>(L, u, i, j, k, p, D);
  const T fv = f ? f[p] : T(0);
  if (KIND == EQ_PSI) {
    const T q = T(1) + u[p];
    const T q2 = q * q;
    const T q4 = q2 * q2;
    const T q6 = q4 * q2;
    const T q8 = q4 * q4;
    const T a = T(2 * PI_D) * s0[p];
    const T b = s1[p];
    const T num = (lap - fv) * q8 + a * q6 * q + T(0.125) * b * q;
    const T den = D * q8 - a * q6 - T(0.875) * b;
    u[p] = u[p] - num / den;
  } else {
    T Lu = lap;
    if (s1) {
      const T c = s1[p];
      Lu -= c * u[p];
      D -= c;
    }
    u[p] = u[p] - (Lu - fv) / D;
  }
}

// Linear update with a precomputed inverse diagonal (coarsest solver).
template <typename T, int G>
__device__ __forceinline__ void scalar_update_lin_inv(const LevelView<T>& L, T* __restrict__ u,
                                                      const T* __restrict__ f, const T* __restrict__ c,
                                                      T invD, int i, int j, int k) {
  const long p = L.idx(i, j, k);
  T D;
  T Lu = lap_scalar<T, G>(L, u, i, j, k, p, D);
  if (c) Lu -= c[p] * u[p];
  const T fv = f ? f[p] : T(0);
  u[p] = u[p] - (Lu - fv) * invD;
}

// New value of vector component c at a cell after one Newton-Gauss-Seidel
// update (ghosts current).
template <typename T, int G, bool VC = true>
__device__ __forceinline__ T vec_new_value(const LevelView<T>& L, T* __restrict__ A, T* __restrict__ B,
                                           T* __restrict__ C, const T* __restrict__ f, int c, int i, int j,
                                           long p) {
  T D;
  T Lu = vec_op<T, G, VC>(L, A, B, C, c, i, j, p, D);
  const T* V = (c == 0) ? A : (c == 1 ? B : C);
  const T fv = f ? f[p] : T(0);
  return V[p] - (Lu - fv) / D;
}

// One Newton-Gauss-Seidel update of vector component c (ghosts current).
template <typename T, int G, bool VC = true>
__device__ __forceinline__ void vec_update(const LevelView<T>& L, T* __restrict__ A, T* __restrict__ B,
                                           T* __restrict__ C, const T* __restrict__ f, int c, int i, int j,
                                           int k) {
  const long p = L.idx(i, j, k);
  T* V = (c == 0) ? A : (c == 1 ? B : C);
  V[p] = vec_new_value<T, G, VC>(L, A, B, C, f, c, i, j, p);
}

// Ghost cells of one field, enumerated as three disjoint layers:
//   A: i in {-1, n0}, all j and k (ghosted ranges);
//   B: i interior, j in {-1, n1}, all k;
//   C: i, j interior, k in {-1, n2} (3D).
template <typename T>
__device__ __forceinline__ long ghost_count(const LevelView<T>& L) {
  const long nk = L.n2 + 2 * L.three;
  return 2L * (L.n1 + 2) * nk + 2L * L.n0 * nk + (L.three ? 2L * L.n0 * L.n1 : 0L);
}
template <typename T>
__device__ __forceinline__ void ghost_coords(const LevelView<T>& L, long gl, int& i, int& j, int& k) {
  // 32-bit arithmetic: a level's ghost count is far below 2^31
  int g = (int)gl;
  const int nk = L.n2 + 2 * L.three;
  const int a = 2 * (L.n1 + 2) * nk;
  if (g < a) {
    const int side = g & 1, q = g >> 1;
    j = q % (L.n1 + 2) - 1;
    k = q / (L.n1 + 2) - L.three;
    i = side ? L.n0 : -1;
    return;
  }
  g -= a;
  const int b = 2 * L.n0 * nk;
  if (g < b) {
    const int side = g & 1, q = g >> 1;
    i = q & (L.n0 - 1);
    k = (q >> L.ln0) - L.three;
    j = side ? L.n1 : -1;
    return;
  }
  g -= b;
  const int side = g & 1, q = g >> 1;
  i = q & (L.n0 - 1);
  j = q >> L.ln0;
  k = side ? L.n2 : -1;
}

template <typename T>
__device__ __forceinline__ void fill_one_ghost(const LevelView<T>& L, T* __restrict__ u, int comp, long g) {
  int i, j, k;
  ghost_coords(L, g, i, j, k);
  u[L.idx(i, j, k)] = ghost_value(L, u, comp, i, j, k);
}

// Coarse correction e = uH - uhH at coarse cell (I, J, K), which may be a
// face ghost: then the boundary rule of that face applies (homogeneous in
// every case, Sec. 2.6 eq. robin / eq. bc).
template <typename T, bool INNER = false>
__device__ __forceinline__ T coarse_corr(const LevelView<T>& C, const T* __restrict__ uH,
                                         const T* __restrict__ uhH, int comp, int I, int J, int K) {
  T f = T(1);
  if (INNER) {
  } else if (I < 0 || I >= C.n0)
    f = ghost_rule(C, comp, 0, I, J, K);
  else if (J < 0 || J >= C.n1)
    f = ghost_rule(C, comp, 1, I, J, K);
  else if (C.three && (K < 0 || K >= C.n2))
    f = ghost_rule(C, comp, 2, I, J, K);
  const long q = C.idx(I, J, K);
  const T e = uhH ? (uH[q] - uhH[q]) : uH[q];
  return f * e;
}

// Residual f - L(u) of a scalar equation at an interior cell; Sv gets the
// source S(u) as the paper writes the right-hand side (L(u) = lap u - S(u)
// for eq. psi; lap u - c u with S = f + c u for linear equations).
// For eq. psi, kpsi (if non-null) also receives its linearisation
// dS/du = 2 pi U (1+u)^-2 + 7/8 A2 (1+u)^-8 at the same u, the c of the
// mixed-precision correction equation (L - c) e = r.
template <typename T, int G, int KIND, bool INNER = false>
__device__ __forceinline__ T scalar_residual_cell(const LevelView<T>& L, const T* __restrict__ u,
                                                  const T* __restrict__ f, const T* __restrict__ s0,
                                                  const T* __restrict__ s1, int i, int j, int k, long p, T& Sv,
                                                  T* kpsi = nullptr) {
  T D;
  const T lap = lap_scalar<T, G, INNER>(L, u, i, j, k, p, D);
  const T fv = f ? f[p] : T(0);
  T Lu;
  if (KIND == EQ_PSI) {
    const T ip = T(1) / (T(1) + u[p]);
    const T ip2 = ip * ip;
    const T ip7 = ip2 * ip2 * ip2 * ip;
    Sv = -T(2 * PI_D) * s0[p] * ip - T(0.125) * s1[p] * ip7;
    Lu = lap - Sv;
    if (kpsi) *kpsi = T(2 * PI_D) * s0[p] * ip2 + T(0.875) * s1[p] * ((ip2 * ip2) * (ip2 * ip2));
  } else if (s1) {
    const T cu = s1[p] * u[p];
    Lu = lap - cu;
    Sv = fv + cu;
  } else {
    Lu = lap;
    Sv = fv;
  }
  return fv - Lu;
}

// Residual f_c - (lap V + 1/3 grad div V)_c of a vector equation (ghosts
// current).
template <typename T, int G, bool VC = true>
__device__ __forceinline__ T vec_residual_cell(const LevelView<T>& L, const T* __restrict__ A,
                                               const T* __restrict__ B, const T* __restrict__ C,
                                               const T* __restrict__ f, int c, int i, int j, long p) {
  T D;
  const T Lu = vec_op<T, G, VC>(L, A, B, C, c, i, j, p, D);
  const T fv = f ? f[p] : T(0);
  return fv - Lu;
}

// Volume-weighted piecewise-constant restriction (Sec. 2.7.3, weights
// Delta V of the fine cells) of nf fields a[m] into b[m] at coarse cell
// (I, J, K); copies into cs[m] too when non-null.
template <typename T>
__device__ __forceinline__ void restrict_cell(const LevelView<T>& F, const LevelView<T>& Cv, int nf,
                                              const T* const (&as)[4], T* const (&bs)[4], T* const (&cs)[3],
                                              int I, int J, int K) {
  T wi[2], wj[2];
  wi[0] = F.TI(TI_VW, 2 * I);
  wi[1] = F.TI(TI_VW, 2 * I + 1);
  wj[0] = F.TJ(TJ_VW, 2 * J);
  wj[1] = F.TJ(TJ_VW, 2 * J + 1);
  T wsum = T(0);
  const int nk = F.three ? 2 : 1;
  for (int dk = 0; dk < nk; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) wsum += wi[di] * wj[dj];
  const T inv = T(1) / wsum;
  const long q = Cv.idx(I, J, K);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (m >= nf) break;
    T s = T(0);
    for (int dk = 0; dk < nk; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di)
          s += wi[di] * wj[dj] * as[m][F.idx(2 * I + di, 2 * J + dj, F.three ? 2 * K + dk : 0)];
    const T v = s * inv;
    bs[m][q] = v;
    if (m < 3 && cs[m]) cs[m][q] = v;
  }
}

// Kwak prolongation (Sec. 2.7.3, Fig. kwak) of e = uH - uhH (uhH may be
// null: e = uH) into fine cell (i, j, k): the parent and, per dimension,
// the parent's face neighbour on the cell's side;
// 2D 1/4 (2 e_c + e_x + e_y), 3D 1/4 (e_c + e_x + e_y + e_z).
// INNER: every coarse cell read is interior (no ghost rule compiled in).
template <typename T, bool INNER = false>
__device__ __forceinline__ void prolong_cell(const LevelView<T>& F, const LevelView<T>& Cv, T* __restrict__ u,
                                             const T* __restrict__ uH, const T* __restrict__ uhH, int comp, int i,
                                             int j, int k) {
  const int I = i >> 1, J = j >> 1, K = F.three ? (k >> 1) : 0;
  const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
  const T ec = coarse_corr<T, INNER>(Cv, uH, uhH, comp, I, J, K);
  const T ex = coarse_corr<T, INNER>(Cv, uH, uhH, comp, I + si, J, K);
  const T ey = coarse_corr<T, INNER>(Cv, uH, uhH, comp, I, J + sj, K);
  T add;
  if (F.three) {
    const T ez = coarse_corr<T, INNER>(Cv, uH, uhH, comp, I, J, K + sk);
    add = T(0.25) * (ec + ex + ey + ez);
  } else {
    add = T(0.25) * (T(2) * ec + ex + ey);
  }
  u[F.idx(i, j, k)] += add;
}

// ----------------------------------------------------------- coarsest grid

constexpr int COARSE_INV_MAX = 1024;      // scalar cells with a cached inverse diagonal
constexpr int COARSE_VEC_INV_MAX = 256;   // vector cells with cached inverse diagonals

// Newton-Gauss-Seidel as the coarsest-grid solver (Sec. 2.7.2): one block
// sweeps until the max residual falls below 1e-12 of its initial value or
// max_sweeps sweeps.  The bodies work on any address space: the kernels
// below run them on shared-memory copies of the level when it fits.
// Block-wide max of non-negative values given as abs_bits, returned to
// every thread (1D blocks).  Integer work only: the single block of a coarse
// solve must not queue its reductions on the few FP64 units.
__device__ __forceinline__ double block_max_abs(unsigned long long m) {
  __shared__ unsigned long long red[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  m = warp_max_bits(m);
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const unsigned long long b = warp_max_bits(lane < nw ? red[lane] : 0ULL);
    if (lane == 0) red[32] = b;
  }
  __syncthreads();
  const unsigned long long b = red[32];
  __syncthreads();
  return __longlong_as_double((long long)b);
}

// NGS sweeps of the coarsest level in one block.  CHECK: until the residual
// has dropped 1e-12 x or max_sweeps (the FP64 cycle's coarsest solve);
// without it exactly max_sweeps sweeps from the given start (the FP32
// correction cycle's: its residual maxima, a block reduction after every
// sweep, cost more than the sweeps on a few cells).
template <typename T, int G, int KIND, bool CHECK = true>
__device__ void coarse_scalar_body(const LevelView<T>& L, T* __restrict__ u, const T* __restrict__ f,
                                   const T* __restrict__ s0, const T* __restrict__ s1, int max_sweeps) {
  __shared__ double r0s;
  const long n = (long)L.n0 * L.n1 * L.n2;
  const int tid = threadIdx.x;
  auto resmax = [&]() -> double {
    unsigned long long m = 0ULL;
    for (long q = tid; q < n; q += blockDim.x) {
      int i, j, k;
      L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      T D;
      const T Lu = scalar_op<T, G, KIND>(L, u, s0, s1, i, j, k, p, D);
      m = umax64(m, abs_bits((double)((f ? f[p] : T(0)) - Lu)));
    }
    return block_max_abs(m);
  };
  if (CHECK) {
    const double r0 = resmax();
    if (tid == 0) r0s = r0;
    __syncthreads();
    if (!(r0s > 0.0)) return;
  }
  // linear equations: the Newton diagonal is fixed, invert it once
  __shared__ T invd[COARSE_INV_MAX];
  const bool use_inv = KIND == EQ_LIN && n <= COARSE_INV_MAX;
  if (use_inv) {
    for (long q = tid; q < n; q += blockDim.x) {
      int i, j, k;
      L.cell(q, i, j, k);
      T D;
      lap_scalar<T, G>(L, u, i, j, k, L.idx(i, j, k), D);
      if (s1) D -= s1[L.idx(i, j, k)];
      invd[q] = T(1) / D;
    }
    __syncthreads();
  }
  for (int it = 0; it < max_sweeps; ++it) {
    for (int colour = 0; colour < 2; ++colour) {
      const long nh = n / 2;
      for (long q = tid; q < nh; q += blockDim.x) {
        int i, j, k;
        L.colour_cell(q, colour, i, j, k);
        if (use_inv)
          scalar_update_lin_inv<T, G>(L, u, f, s1, invd[i + (long)L.n0 * (j + (long)L.n1 * k)], i, j, k);
        else
          scalar_update<T, G, KIND>(L, u, f, s0, s1, i, j, k);
      }
      __syncthreads();
    }
    if (CHECK) {
      const double r = resmax();
      if (!(r > 1e-12 * r0s)) break;
    }
  }
}

template <typename T, int G>
__device__ void coarse_vec_body(const LevelView<T>& L, T* __restrict__ A, T* __restrict__ B, T* __restrict__ C,
                                const T* __restrict__ f0, const T* __restrict__ f1, const T* __restrict__ f2,
                                int max_sweeps) {
  __shared__ double r0s;
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long ng = ghost_count(L);
  const int tid = threadIdx.x;
  T* V[3] = {A, B, C};
  const T* fs[3] = {f0, f1, f2};
  auto fill = [&](int c) {
    for (long g = tid; g < ng; g += blockDim.x) fill_one_ghost(L, V[c], c, g);
    __syncthreads();
  };
  auto resmax = [&]() -> double {
    unsigned long long m = 0ULL;
    for (long q = tid; q < n; q += blockDim.x) {
      int i, j, k;
      L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      for (int c = 0; c < 3; ++c) {
        T D;
        const T Lu = vec_op<T, G>(L, A, B, C, c, i, j, p, D);
        m = umax64(m, abs_bits((double)((fs[c] ? fs[c][p] : T(0)) - Lu)));
      }
    }
    return block_max_abs(m);
  };
  for (int c = 0; c < 3; ++c) fill(c);
  const double r0 = resmax();
  if (tid == 0) r0s = r0;
  __syncthreads();
  if (!(r0s > 0.0)) return;
  // the Newton diagonal of each component is fixed: invert it once
  __shared__ T invd[3 * COARSE_VEC_INV_MAX];
  const bool use_inv = n <= COARSE_VEC_INV_MAX;
  if (use_inv) {
    for (long q = tid; q < n; q += blockDim.x) {
      int i, j, k;
      L.cell(q, i, j, k);
      for (int c = 0; c < 3; ++c) {
        T D;
        vec_op<T, G>(L, A, B, C, c, i, j, L.idx(i, j, k), D);
        invd[c * COARSE_VEC_INV_MAX + q] = T(1) / D;
      }
    }
    __syncthreads();
  }
  for (int it = 0; it < max_sweeps; ++it) {
    for (int colour = 0; colour < 2; ++colour)
      for (int c = 0; c < 3; ++c) {
        const long nh = n / 2;
        for (long q = tid; q < nh; q += blockDim.x) {
          int i, j, k;
          L.colour_cell(q, colour, i, j, k);
          if (use_inv) {
            const long p = L.idx(i, j, k);
            T D;
            const T Lu = vec_op<T, G>(L, A, B, C, c, i, j, p, D);
            T* Vc = V[c];
            const T fv = fs[c] ? fs[c][p] : T(0);
            Vc[p] = Vc[p] - (Lu - fv) * invd[c * COARSE_VEC_INV_MAX + i + (long)L.n0 * (j + (long)L.n1 * k)];
          } else {
            vec_update<T, G>(L, A, B, C, fs[c], c, i, j, k);
          }
        }
        __syncthreads();
        fill(c);
      }
    const double r = resmax();
    if (!(r > 1e-12 * r0s)) break;
  }
}

// ------------------------------------------------- elementwise helpers

// Elementwise passes over the interior in groups of four consecutive cells
// of a row: rows start 16-byte aligned and n0 (a power of two) is a
// multiple of 4 on every level but the smallest, which take one cell at a
// time.  Values travel as doubles (exact for both storage types).
template <typename T>
__device__ __forceinline__ long group4(const LevelView<T>& L, long q) {
  const int i = (int)(q & ((L.n0 >> 2) - 1)) << 2;
  const long jk = q >> (L.ln0 - 2);
  return L.idx(i, (int)(jk & (L.n1 - 1)), (int)(jk >> L.ln1));
}
__device__ __forceinline__ void ld4(const float* p, double (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const double (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
template <typename T>
__device__ __forceinline__ long interior_p(const LevelView<T>& L, long q) {
  int i, j, k;
  L.cell(q, i, j, k);
  return L.idx(i, j, k);
}

// Sum of a block's doubles into part[blockIdx.x] (fixed order).
__device__ __forceinline__ void block_sum_to(double s, double* part) {
  __shared__ double sm[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double b = threadIdx.x < (blockDim.x + 31) / 32 ? sm[threadIdx.x] : 0.0;
    b = warp_sum(b);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
  }
}

}  // namespace gmg
