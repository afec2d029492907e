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

// One Newton-Gauss-Seidel update of vector component c (ghosts current).
template <typename T, int G>
__device__ __forceinline__ void vec_update(const LevelView<T>& L, T* __restrict__ A, T* __restrict__ B,
                                           T* __restrict__ C, const T* __restrict__ f, int c, int i, int j,
                                           int k) {
  const long p = L.idx(i, j, k);
  T D;
  T Lu = vec_op<T, G>(L, A, B, C, c, i, j, p, D);
  T* V = (c == 0) ? A : (c == 1 ? B : C);
  const T fv = f ? f[p] : T(0);
  V[p] = V[p] - (Lu - fv) / D;
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
__device__ __forceinline__ void ghost_coords(const LevelView<T>& L, long g, int& i, int& j, int& k) {
  const long nk = L.n2 + 2 * L.three;
  const long a = 2L * (L.n1 + 2) * nk;
  if (g < a) {
    int side = (int)(g % 2);
    long q = g / 2;
    j = (int)(q % (L.n1 + 2)) - 1;
    k = (int)(q / (L.n1 + 2)) - L.three;
    i = side ? L.n0 : -1;
    return;
  }
  g -= a;
  const long b = 2L * L.n0 * nk;
  if (g < b) {
    int side = (int)(g % 2);
    long q = g / 2;
    i = (int)(q % L.n0);
    k = (int)(q / L.n0) - L.three;
    j = side ? L.n1 : -1;
    return;
  }
  g -= b;
  int side = (int)(g % 2);
  long q = g / 2;
  i = (int)(q % L.n0);
  j = (int)(q / L.n0);
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
template <typename T>
__device__ __forceinline__ T coarse_corr(const LevelView<T>& C, const T* __restrict__ uH,
                                         const T* __restrict__ uhH, int comp, int I, int J, int K) {
  T f = T(1);
  if (I < 0 || I >= C.n0)
    f = ghost_rule(C, comp, 0, I, J, K);
  else if (J < 0 || J >= C.n1)
    f = ghost_rule(C, comp, 1, I, J, K);
  else if (C.three && (K < 0 || K >= C.n2))
    f = ghost_rule(C, comp, 2, I, J, K);
  const long q = C.idx(I, J, K);
  const T e = uhH ? (uH[q] - uhH[q]) : uH[q];
  return f * e;
}

}  // namespace gmg
