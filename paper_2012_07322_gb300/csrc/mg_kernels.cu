// Grid-wide multigrid kernels (red-black Newton-Gauss-Seidel, residual with
// fused norms, FAS coarse right-hand side, ghost fill, volume-weighted
// restriction, Kwak prolongation) and the single-block coarsest solver, with
// their host-side launchers.  Sec. 2.7 of the paper.
#include <atomic>

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
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (2 * t >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const int i = 2 * t + ((j + k + colour) & 1);
  scalar_update<T, G, KIND>(L, u, f, s0, s1, i, j, k);
}

template <typename T, int G>
__global__ void k_smooth_vec(LevelView<T> L, T* __restrict__ A, T* __restrict__ B, T* __restrict__ C,
                             const T* __restrict__ f, int comp, int colour) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (2 * t >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const int i = 2 * t + ((j + k + colour) & 1);
  vec_update<T, G>(L, A, B, C, f, comp, i, j, k);
}

// One full red-black sweep of a Cartesian linear scalar equation in one
// launch.  A block stages a TX x TY x TZ tile of u, f (and c) with a
// two-cell halo in shared memory, relaxes the red cells of the tile and of
// a one-cell ring around it (the ring is recomputed by the neighbouring
// tiles with the same arithmetic), then the black cells of the tile, and
// writes the tile back: u and f cross DRAM once per sweep instead of once
// per colour.  The cell updates are the ones of k_smooth_scalar.
constexpr int FT_X = 32, FT_Y = 8, FT_Z = 8, FH = 2;
constexpr int FS_X = FT_X + 2 * FH, FS_Y = FT_Y + 2 * FH, FS_Z = FT_Z + 2 * FH;
constexpr int FS_N = FS_X * FS_Y * FS_Z;

template <typename T>
__global__ void __launch_bounds__(256) k_sweep_fused_cart(LevelView<T> L, T* __restrict__ u,
                                                          const T* __restrict__ f, const T* __restrict__ c) {
  extern __shared__ unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* sf = su + FS_N;
  T* sc = sf + FS_N;
  const int i0 = blockIdx.x * FT_X - FH, j0 = blockIdx.y * FT_Y - FH, k0 = blockIdx.z * FT_Z - FH;
  const int tid = threadIdx.x;
  const bool inner = i0 >= 0 && j0 >= 0 && k0 >= 0 && i0 + FS_X <= L.n0 && j0 + FS_Y <= L.n1 &&
                     k0 + FS_Z <= L.n2;
  // stage the tile with its halo, one smem row (FS_X cells) per step
  for (int q = tid; q < FS_N; q += blockDim.x) {
    const int row = q / FS_X, a = q - row * FS_X;
    const int b = row % FS_Y, cz = row / FS_Y;
    const int i = i0 + a, j = j0 + b, k = k0 + cz;
    const bool in = inner || (i >= 0 && i < L.n0 && j >= 0 && j < L.n1 && k >= 0 && k < L.n2);
    const long p = in ? L.idx(i, j, k) : 0;
    su[q] = in ? u[p] : T(0);
    sf[q] = (in && f) ? f[p] : T(0);
    if (c) sc[q] = in ? c[p] : T(0);
  }
  __syncthreads();
  LevelView<T> S = L;  // shared-memory view: same geometry, tile strides
  S.sx = FS_X;
  S.sy = (long)FS_X * FS_Y;
  // red over the tile and a one-cell ring (recomputed identically by the
  // neighbouring tiles), then black over the tile; work items enumerate
  // only the cells of the colour: (row, t) -> x = lo + 2 t + parity
  for (int colour = 0; colour < 2; ++colour) {
    const int ring = colour == 0 ? 1 : 0;
    const int ex = FT_X + 2 * ring, ey = FT_Y + 2 * ring, ez = FT_Z + 2 * ring;
    const int half = ex / 2;
    const int nwork = half * ey * ez;
    const int xlo = FH - ring, ylo = FH - ring, zlo = FH - ring;  // smem coordinates
    for (int q = tid; q < nwork; q += blockDim.x) {
      const int row = q / half, t = q - row * half;
      const int b = ylo + row % ey, cz = zlo + row / ey;
      const int j = j0 + b, k = k0 + cz;
      // i0 + a with a = xlo + 2 t + shift has parity colour
      const int shift = (colour - (i0 + xlo + j + k)) & 1;
      const int a = xlo + 2 * t + shift;
      const int i = i0 + a;
      if (a >= xlo + ex) continue;
      if (!inner && (i < 0 || i >= L.n0 || j < 0 || j >= L.n1 || k < 0 || k >= L.n2)) continue;
      const long ps = a + (long)b * FS_X + (long)cz * FS_X * FS_Y;
      T D;
      T Lu = lap_scalar<T, CART>(S, su, i, j, k, ps, D);
      if (c) {
        const T cv = sc[ps];
        Lu -= cv * su[ps];
        D -= cv;
      }
      su[ps] = su[ps] - (Lu - sf[ps]) / D;
    }
    __syncthreads();
  }
  // write the tile back
  for (int q = tid; q < FT_X * FT_Y * FT_Z; q += blockDim.x) {
    const int row = q / FT_X, a = q - row * FT_X;
    const int b = row % FT_Y, cz = row / FT_Y;
    const int i = i0 + FH + a, j = j0 + FH + b, k = k0 + FH + cz;
    if (!inner && (i >= L.n0 || j >= L.n1 || k >= L.n2)) continue;
    u[L.idx(i, j, k)] = su[(a + FH) + (long)(b + FH) * FS_X + (long)(cz + FH) * FS_X * FS_Y];
  }
}

template <typename T>
__global__ void k_fill_ghosts(LevelView<T> L, T* __restrict__ u, int comp) {
  const long n = ghost_count(L);
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n; g += (long)gridDim.x * blockDim.x)
    fill_one_ghost(L, u, comp, g);
}

// ------------------------------------------------------------ residuals

// r = f - L(u) on every interior cell.  red (if non-null) receives
// max |r| (slot 0) and, when weighted, max |w r| (slot 1), max |w S| (slot 2).
template <typename T, int G, int KIND>
__global__ void k_residual_scalar(LevelView<T> L, const T* __restrict__ u, const T* __restrict__ f,
                                  const T* __restrict__ s0, const T* __restrict__ s1, T* __restrict__ r,
                                  unsigned long long* red, int weighted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  double m[3] = {0.0, 0.0, 0.0};
  if (i < L.n0 && j < L.n1 && k < L.n2) {
    const long p = L.idx(i, j, k);
    T D;
    const T lap = lap_scalar<T, G>(L, u, i, j, k, p, D);
    const T fv = f ? f[p] : T(0);
    // S(u) as the paper writes the right-hand side; L(u) = lap u - S(u)
    // (eq. psi) or lap u - c u (linear, S = f + c u)
    T Sv, Lu;
    if (KIND == EQ_PSI) {
      const T ip = T(1) / (T(1) + u[p]);
      const T ip2 = ip * ip;
      const T ip7 = ip2 * ip2 * ip2 * ip;
      Sv = -T(2 * PI_D) * s0[p] * ip - T(0.125) * s1[p] * ip7;
      Lu = lap - Sv;
    } else {
      const T cu = s1 ? s1[p] * u[p] : T(0);
      Lu = lap - cu;
      Sv = fv + cu;
    }
    const T rv = fv - Lu;
    if (r) r[p] = rv;
    m[0] = fabs((double)rv);
    if (weighted) {
      const double w = (double)norm_weight(L, i, j);
      m[1] = fabs(w * (double)rv);
      m[2] = fabs(w * (double)Sv);
    }
  }
  if (red) block_max_atomic<3>(m, red);
}

template <typename T, int G>
__global__ void k_residual_vec(LevelView<T> L, const T* __restrict__ A, const T* __restrict__ B,
                               const T* __restrict__ C, const T* __restrict__ f0, const T* __restrict__ f1,
                               const T* __restrict__ f2, T* __restrict__ r0, T* __restrict__ r1,
                               T* __restrict__ r2, unsigned long long* red, int weighted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  double m[3] = {0.0, 0.0, 0.0};
  if (i < L.n0 && j < L.n1 && k < L.n2) {
    const long p = L.idx(i, j, k);
    const double w = weighted ? (double)norm_weight(L, i, j) : 1.0;
    const T* fs[3] = {f0, f1, f2};
    T* rs[3] = {r0, r1, r2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T D;
      const T Lu = vec_op<T, G>(L, A, B, C, c, i, j, p, D);
      const T fv = fs[c] ? fs[c][p] : T(0);
      const T rv = fv - Lu;
      if (rs[c]) rs[c][p] = rv;
      m[0] = fmax(m[0], fabs((double)rv));
      if (weighted) {
        m[1] = fmax(m[1], fabs(w * (double)rv));
        m[2] = fmax(m[2], fabs(w * (double)fv));
      }
      if (rv != rv) m[0] = m[1] = INFINITY;
    }
  }
  if (red) block_max_atomic<3>(m, red);
}

// f <- L(u) + f (the FAS coarse right-hand side after restriction placed
// R r into f), or out = L(u) when add == 0.
template <typename T, int G, int KIND>
__global__ void k_apply_scalar(LevelView<T> L, const T* __restrict__ u, const T* __restrict__ s0,
                               const T* __restrict__ s1, T* __restrict__ out, int add) {
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
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  if (I >= Cv.n0 || J >= Cv.n1 || K >= Cv.n2) return;
  const T* as[4] = {a0, a1, a2, a3};
  T* bs[4] = {b0, b1, b2, b3};
  T* cs[3] = {copy0, copy1, copy2};
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
  for (int m = 0; m < nf; ++m) {
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
// null: e = uH), added into the fine field u.  Each fine cell takes its
// parent and, per dimension, the parent's face neighbour on its side:
// 2D 1/4 (2 e_c + e_x + e_y), 3D 1/4 (e_c + e_x + e_y + e_z).
template <typename T>
__global__ void k_prolong(LevelView<T> F, LevelView<T> Cv, T* __restrict__ u, const T* __restrict__ uH,
                          const T* __restrict__ uhH, int comp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= F.n0 || j >= F.n1 || k >= F.n2) return;
  const int I = i >> 1, J = j >> 1, K = F.three ? (k >> 1) : 0;
  const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
  const T ec = coarse_corr(Cv, uH, uhH, comp, I, J, K);
  const T ex = coarse_corr(Cv, uH, uhH, comp, I + si, J, K);
  const T ey = coarse_corr(Cv, uH, uhH, comp, I, J + sj, K);
  T add;
  if (F.three) {
    const T ez = coarse_corr(Cv, uH, uhH, comp, I, J, K + sk);
    add = T(0.25) * (ec + ex + ey + ez);
  } else {
    add = T(0.25) * (T(2) * ec + ex + ey);
  }
  u[F.idx(i, j, k)] += add;
}

// --------------------------------------------------------- coarsest grid

constexpr int COARSE_INV_MAX = 1024;      // scalar cells with a cached inverse diagonal
constexpr int COARSE_VEC_INV_MAX = 256;   // vector cells with cached inverse diagonals

// Newton-Gauss-Seidel as the coarsest-grid solver (Sec. 2.7.2): one block
// sweeps until the max residual falls below 1e-12 of its initial value or
// max_sweeps sweeps.  The bodies work on any address space: the kernels
// below run them on shared-memory copies of the level when it fits.
template <typename T, int G, int KIND>
__device__ void coarse_scalar_body(const LevelView<T>& L, T* __restrict__ u, const T* __restrict__ f,
                                   const T* __restrict__ s0, const T* __restrict__ s1, int max_sweeps) {
  __shared__ double red[32];
  __shared__ double r0s;
  const long n = (long)L.n0 * L.n1 * L.n2;
  const int tid = threadIdx.x;
  auto resmax = [&]() -> double {
    double m = 0.0;
    for (long q = tid; q < n; q += blockDim.x) {
      int i, j, k;
    L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      T D;
      const T Lu = scalar_op<T, G, KIND>(L, u, s0, s1, i, j, k, p, D);
      const double rv = fabs((double)((f ? f[p] : T(0)) - Lu));
      m = (rv > m || rv != rv) ? rv : m;
    }
    m = warp_max(m);
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) b = fmax(b, red[w]);
    __syncthreads();
    return b;
  };
  const double r0 = resmax();
  if (tid == 0) r0s = r0;
  __syncthreads();
  if (!(r0s > 0.0)) return;
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
        const int t = (int)(q % (L.n0 / 2)), j = (int)((q / (L.n0 / 2)) % L.n1),
                  k = (int)(q / ((long)(L.n0 / 2) * L.n1));
        const int i = 2 * t + ((j + k + colour) & 1);
        if (use_inv)
          scalar_update_lin_inv<T, G>(L, u, f, s1, invd[i + (long)L.n0 * (j + (long)L.n1 * k)], i, j, k);
        else
          scalar_update<T, G, KIND>(L, u, f, s0, s1, i, j, k);
      }
      __syncthreads();
    }
    const double r = resmax();
    if (!(r > 1e-12 * r0s)) break;
  }
}

template <typename T, int G>
__device__ void coarse_vec_body(const LevelView<T>& L, T* __restrict__ A, T* __restrict__ B, T* __restrict__ C,
                                const T* __restrict__ f0, const T* __restrict__ f1, const T* __restrict__ f2,
                                int max_sweeps) {
  __shared__ double red[32];
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
    double m = 0.0;
    for (long q = tid; q < n; q += blockDim.x) {
      int i, j, k;
    L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      for (int c = 0; c < 3; ++c) {
        T D;
        const T Lu = vec_op<T, G>(L, A, B, C, c, i, j, p, D);
        const double rv = fabs((double)((fs[c] ? fs[c][p] : T(0)) - Lu));
        m = (rv > m || rv != rv) ? rv : m;
      }
    }
    m = warp_max(m);
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) b = fmax(b, red[w]);
    __syncthreads();
    return b;
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
          const int t = (int)(q % (L.n0 / 2)), j = (int)((q / (L.n0 / 2)) % L.n1),
                    k = (int)(q / ((long)(L.n0 / 2) * L.n1));
          const int i = 2 * t + ((j + k + colour) & 1);
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

// Block copies between global and shared memory (all ghosted cells).
template <typename T>
__device__ __forceinline__ void block_copy(T* dst, const T* src, long n) {
  for (long q = threadIdx.x; q < n; q += blockDim.x) dst[q] = src[q];
}

template <typename T, int G, int KIND>
__global__ void k_coarse_scalar(LevelView<T> L, T* __restrict__ u, const T* __restrict__ f,
                                const T* __restrict__ s0, const T* __restrict__ s1, int max_sweeps, int use_smem) {
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
template <typename T>
__global__ void k_partial_sum(LevelView<T> L, const T* __restrict__ u, double* __restrict__ part) {
  __shared__ double sm[32];
  const long n = (long)L.n0 * L.n1 * L.n2;
  double s = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    s += (double)u[L.idx(i, j, k)];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) b += sm[w];
    part[blockIdx.x] = b;
  }
}

template <typename T>
__global__ void k_sub_mean(LevelView<T> L, T* __restrict__ u, const double* __restrict__ part, int nparts) {
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[b];
    mean = s / ((double)L.n0 * L.n1 * L.n2);
  }
  __syncthreads();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    u[p] = (T)((double)u[p] - mean);
  }
}

// Interior <-> ghosted copies, FP64 <-> storage type conversions.
template <typename A, typename B>
__global__ void k_copy_in(LevelView<B> L, const A* __restrict__ src, B* __restrict__ dst, A shift) {
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    dst[L.idx(i, j, k)] = (B)(src[q] + shift);
  }
}
template <typename A, typename B>
__global__ void k_copy_out(LevelView<A> L, const A* __restrict__ src, B* __restrict__ dst, A shift) {
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
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    dst[p] = (B)src[p];
  }
}
// u64 += e32 (interior), the defect-correction update.
template <typename T>
__global__ void k_add_correction(LevelView<double> L, double* __restrict__ u, const T* __restrict__ e) {
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    u[p] += (double)e[p];
  }
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
  GMG_GEOM_DISPATCH(L.geom, if (kind == EQ_PSI) k_smooth_scalar<T, GG, EQ_PSI><<<g, b, 0, st>>>(L, u, f, s0, s1, colour);
                    else k_smooth_scalar<T, GG, EQ_LIN><<<g, b, 0, st>>>(L, u, f, s0, s1, colour));
}

template <typename T>
size_t fused_sweep_smem(bool with_c) {
  return sizeof(T) * (size_t)FS_N * (with_c ? 3 : 2);
}

template <typename T>
void init_fused_sweep_attributes() {
  cudaFuncSetAttribute(k_sweep_fused_cart<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused_sweep_smem<T>(true));
}

template <typename T>
bool launch_sweep_fused(const LevelView<T>& L, T* u, const T* f, const T* c, cudaStream_t st) {
  if (L.geom != CART || !L.three || L.n0 < FT_X || L.n1 < FT_Y || L.n2 < FT_Z) return false;
  count_launch();
  dim3 g(cdiv(L.n0, FT_X), cdiv(L.n1, FT_Y), cdiv(L.n2, FT_Z));
  k_sweep_fused_cart<T><<<g, 256, fused_sweep_smem<T>(c != nullptr), st>>>(L, u, f, c);
  return true;
}

template <typename T>
void launch_fill_ghosts(const LevelView<T>& L, T* u, int comp, cudaStream_t st) {
  count_launch();
  const long nk = L.n2 + 2 * L.three;
  const long n = 2L * (L.n1 + 2) * nk + 2L * L.n0 * nk + (L.three ? 2L * L.n0 * L.n1 : 0L);
  k_fill_ghosts<T><<<grid_flat(n, 256), 256, 0, st>>>(L, u, comp);
}

template <typename T>
void launch_smooth_vec(const LevelView<T>& L, T* V[3], const T* f, int comp, int colour, cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_colour(L, b);
  GMG_GEOM_DISPATCH(L.geom, k_smooth_vec<T, GG><<<g, b, 0, st>>>(L, V[0], V[1], V[2], f, comp, colour));
}

template <typename T>
void launch_residual_scalar(const LevelView<T>& L, int kind, const T* u, const T* f, const T* s0,
                            const T* s1, T* r, unsigned long long* red, int weighted, cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  GMG_GEOM_DISPATCH(L.geom, if (kind == EQ_PSI) k_residual_scalar<T, GG, EQ_PSI><<<g, b, 0, st>>>(L, u, f, s0, s1, r, red, weighted);
                    else k_residual_scalar<T, GG, EQ_LIN><<<g, b, 0, st>>>(L, u, f, s0, s1, r, red, weighted));
}

template <typename T>
void launch_residual_vec(const LevelView<T>& L, T* const V[3], const T* const f[3], T* const r[3],
                         unsigned long long* red, int weighted, cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  GMG_GEOM_DISPATCH(L.geom, k_residual_vec<T, GG><<<g, b, 0, st>>>(L, V[0], V[1], V[2], f[0], f[1], f[2], r[0], r[1], r[2], red, weighted));
}

template <typename T>
void launch_apply_scalar(const LevelView<T>& L, int kind, const T* u, const T* s0, const T* s1, T* out, int add,
                         cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  GMG_GEOM_DISPATCH(L.geom, if (kind == EQ_PSI) k_apply_scalar<T, GG, EQ_PSI><<<g, b, 0, st>>>(L, u, s0, s1, out, add);
                    else k_apply_scalar<T, GG, EQ_LIN><<<g, b, 0, st>>>(L, u, s0, s1, out, add));
}

template <typename T>
void launch_apply_vec(const LevelView<T>& L, T* const V[3], T* const out[3], int add, cudaStream_t st) {
  count_launch();
  dim3 b = block_for(L.three), g = grid_cells(L, b);
  GMG_GEOM_DISPATCH(L.geom, k_apply_vec<T, GG><<<g, b, 0, st>>>(L, V[0], V[1], V[2], out[0], out[1], out[2], add));
}

template <typename T>
void launch_restrict(const LevelView<T>& F, const LevelView<T>& C, int nf, const T* const a[4], T* const b[4],
                     T* const copy[3], cudaStream_t st) {
  count_launch();
  dim3 bl = block_for(C.three), g = grid_cells(C, bl);
  k_restrict<T><<<g, bl, 0, st>>>(F, C, nf, a[0], a[1], a[2], a[3], b[0], b[1], b[2], b[3], copy[0], copy[1],
                                   copy[2]);
}

template <typename T>
void launch_prolong(const LevelView<T>& F, const LevelView<T>& C, T* u, const T* uH, const T* uhH, int comp,
                    cudaStream_t st) {
  count_launch();
  dim3 b = block_for(F.three), g = grid_cells(F, b);
  k_prolong<T><<<g, b, 0, st>>>(F, C, u, uH, uhH, comp);
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
    k_coarse_scalar<T, GG, EQ_PSI><<<1, 256, dyn, st>>>(L, u, f, s0, s1, max_sweeps, use);
  } else {
    if (dyn + 16 * 1024 > 48 * 1024) cudaFuncSetAttribute(k_coarse_scalar<T, GG, EQ_LIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    k_coarse_scalar<T, GG, EQ_LIN><<<1, 256, dyn, st>>>(L, u, f, s0, s1, max_sweeps, use);
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
    k_coarse_vec<T, GG><<<1, 256, dyn, st>>>(L, V[0], V[1], V[2], f[0], f[1], f[2], max_sweeps, use);
  });
}

template <typename T>
void launch_sub_mean(const LevelView<T>& L, T* u, double* part, int nparts, cudaStream_t st) {
  count_launch(2);
  k_partial_sum<T><<<nparts, 256, 0, st>>>(L, u, part);
  k_sub_mean<T><<<nparts, 256, 0, st>>>(L, u, part, nparts);
}

template <typename A, typename B>
void launch_copy_in(const LevelView<B>& L, const A* src, B* dst, A shift, cudaStream_t st) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  k_copy_in<A, B><<<grid_flat(n, 256), 256, 0, st>>>(L, src, dst, shift);
}
template <typename A, typename B>
void launch_copy_out(const LevelView<A>& L, const A* src, B* dst, A shift, cudaStream_t st) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  k_copy_out<A, B><<<grid_flat(n, 256), 256, 0, st>>>(L, src, dst, shift);
}
template <typename A, typename B>
void launch_convert(const LevelView<A>& L, const A* src, B* dst, cudaStream_t st) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  k_convert<A, B><<<grid_flat(n, 256), 256, 0, st>>>(L, src, dst);
}
template <typename T>
void launch_add_correction(const LevelView<double>& L, double* u, const T* e, cudaStream_t st) {
  count_launch();
  long n = (long)L.n0 * L.n1 * L.n2;
  k_add_correction<T><<<grid_flat(n, 256), 256, 0, st>>>(L, u, e);
}

// explicit instantiations
#define GMG_INST(T)                                                                                            \
  template bool launch_sweep_fused<T>(const LevelView<T>&, T*, const T*, const T*, cudaStream_t);              \
  template void init_fused_sweep_attributes<T>();                                                              \
  template void launch_smooth_scalar<T>(const LevelView<T>&, int, T*, const T*, const T*, const T*, int,       \
                                        cudaStream_t);                                                          \
  template void launch_fill_ghosts<T>(const LevelView<T>&, T*, int, cudaStream_t);                             \
  template void launch_smooth_vec<T>(const LevelView<T>&, T* [3], const T*, int, int, cudaStream_t);           \
  template void launch_residual_scalar<T>(const LevelView<T>&, int, const T*, const T*, const T*, const T*, T*, \
                                          unsigned long long*, int, cudaStream_t);                              \
  template void launch_residual_vec<T>(const LevelView<T>&, T* const[3], const T* const[3], T* const[3],       \
                                       unsigned long long*, int, cudaStream_t);                                 \
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
  template void launch_sub_mean<T>(const LevelView<T>&, T*, double*, int, cudaStream_t);
GMG_INST(double)
GMG_INST(float)
template void launch_copy_in<double, double>(const LevelView<double>&, const double*, double*, double, cudaStream_t);
template void launch_copy_out<double, double>(const LevelView<double>&, const double*, double*, double, cudaStream_t);
template void launch_convert<double, float>(const LevelView<double>&, const double*, float*, cudaStream_t);
template void launch_convert<float, double>(const LevelView<float>&, const float*, double*, cudaStream_t);
template void launch_add_correction<float>(const LevelView<double>&, double*, const float*, cudaStream_t);

}  // namespace gmg
