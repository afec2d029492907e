// Anderson mixing of successive multigrid iterates (outer acceleration of
// the V-cycle fixed-point map; not part of the paper's method, which runs
// plain cycles).  Vectors are the finest-level unknowns of all components
// (interior cells of ghosted arrays); storage of a vector is ncomp arrays
// of L.ng values laid out back to back.  The iterate x and the previous f
// and g stay FP64; the history columns dF, dG are TC: FP64, or FP32 in
// mixed precision, where the mixing coefficients only steer the iteration
// (the FP64 residual decides convergence) and the columns' products and
// sums run on the FP32 units.
//
// One mixing step is two launches and no host round trip: the update of
// the differences fused with the dot products of the least-squares problem
// and its solve (the Gram matrix lives on the device), then the
// combination.
#include "mg_internal.h"
#include "mg_kernels.cuh"

namespace gmg {

// G consecutive interior cells of a row (G = 4 when n0 >= 4, else 1).
template <int G>
__device__ __forceinline__ long aa_pos(const LevelView<double>& L, long q) {
  if (G == 4) return group4(L, q);
  return interior_p(L, q);
}
template <int G, typename T>
__device__ __forceinline__ void aa_ld(const T* p, T (&v)[G]) {
  if constexpr (G == 1) {
    v[0] = *p;
  } else if constexpr (sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
}
template <int G, typename T>
__device__ __forceinline__ void aa_st(T* p, const T (&v)[G]) {
  if constexpr (G == 1) {
    *p = v[0];
  } else if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// Sum over the warp of 32 values per lane; afterwards lane l holds the sum
// of value l (31 exchanges instead of 32 x 5).
__device__ __forceinline__ double warp_sum32(double (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = lane & s;
#pragma unroll
    for (int q = 0; q < s; ++q) {
      const double send = upper ? v[q] : v[q + s];
      const double keep = upper ? v[q + s] : v[q];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// The least-squares step (run by the last block of k_aa_update_dots to
// finish): reduce the blocks' partial dot products in a fixed order, enter
// the newest column's row into the Gram matrix M (AA_MAX x AA_MAX over ring
// slots), and solve (M_live + lambda I) gamma = b with lambda = 1e-12
// max diag(M_live) by Cholesky.  status = 0 with gamma written, or 1 when
// the history is degenerate (non-positive pivot, non-finite values): the
// host then restarts the mixing and the combination is skipped.
__device__ void aa_solve_block(const AACols& cols, const double* part, int nblocks, double* __restrict__ M,
                               double* __restrict__ gamma, unsigned long long* __restrict__ status) {
  __shared__ double red[8][2 * AA_MAX];
  __shared__ double s[2 * AA_MAX];
  __shared__ double A[AA_MAX][AA_MAX + 1];
  __shared__ double z[AA_MAX];
  const int t = threadIdx.x, q = t & 31, w = t >> 5;
  double acc = 0.0;
#pragma unroll 8
  for (int b = w; b < nblocks; b += 8) acc += __ldcg(part + (long)b * 2 * AA_MAX + q);
  red[w][q] = acc;
  __syncthreads();
  if (t >= 32) return;
  double sum = 0.0;
  for (int k = 0; k < 8; ++k) sum += red[k][t];
  s[t] = sum;
  const int n = cols.n, slot = cols.slot[n - 1];
  __syncwarp();
  if (t < n) {
    M[slot * AA_MAX + cols.slot[t]] = s[AA_MAX + t];
    M[cols.slot[t] * AA_MAX + slot] = s[AA_MAX + t];
  }
  __syncwarp();
  for (int e = t; e < n * n; e += 32) {
    const int a = e / n, b = e - a * n;
    A[a][b] = M[cols.slot[a] * AA_MAX + cols.slot[b]];
  }
  __syncwarp();
  double dmax = 0.0;
  for (int a = 0; a < n; ++a) dmax = fmax(dmax, A[a][a]);
  bool ok = dmax > 0.0;
  __syncwarp();
  if (ok && t < n) A[t][t] += 1e-12 * dmax;
  __syncwarp();
  // right-looking Cholesky, lane t owns row t; L overwrites the lower triangle
  for (int j = 0; ok && j < n; ++j) {
    const double piv = A[j][j];
    if (!(piv > 0.0)) {
      ok = false;
      break;
    }
    const double d = sqrt(piv), id = 1.0 / d;
    __syncwarp();
    if (t == j) A[j][j] = d;
    if (t > j && t < n) A[t][j] *= id;
    __syncwarp();
    if (t > j && t < n) {
      const double lt = A[t][j];
      for (int k = j + 1; k <= t; ++k) A[t][k] -= lt * A[k][j];
    }
    __syncwarp();
  }
  if (t == 0) {
    if (ok) {
      for (int i = 0; i < n; ++i) {
        double a = s[i];
        for (int k = 0; k < i; ++k) a -= A[i][k] * z[k];
        z[i] = a / A[i][i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double a = z[i];
        for (int k = i + 1; k < n; ++k) a -= A[k][i] * z[k];
        z[i] = a / A[i][i];
      }
      for (int i = 0; i < n; ++i) ok = ok && (z[i] - z[i] == 0.0);
      for (int i = 0; i < n; ++i) gamma[i] = z[i];
    }
    *status = ok ? 0ULL : 1ULL;
  }
}

// With the live columns cols (oldest first; the newest, slot cols.n - 1, is
// this cycle's, cols.n = 0 on the first cycle):
//   f = g - x;  dF_new = f - fprev, dG_new = g - gprev (unless first);
//   fprev = f, gprev = g, x = g (the next cycle's start unless mixed);
//   part[block] = { sum dF_a . f ; sum dF_a . dF_new } over a < cols.n;
// the last block to finish then runs the least-squares step (aa_solve_block;
// done counts finished blocks and is reset by that block).
template <typename TC, int G>
__global__ void __launch_bounds__(256, 2)
    k_aa_update_dots(LevelView<double> L, int ncomp, long stride, const double* __restrict__ g0,
                     const double* __restrict__ g1, const double* __restrict__ g2, double* __restrict__ x,
                     double* __restrict__ fprev, double* __restrict__ gprev, TC* __restrict__ dF,
                     TC* __restrict__ dG, const __grid_constant__ AACols cols, double* __restrict__ part,
                     unsigned int* __restrict__ done, double* __restrict__ M, double* __restrict__ gamma,
                     unsigned long long* __restrict__ status) {
  pdl_entry();
  const long nq = (long)L.n0 * L.n1 * L.n2 / G;
  const long vstride = (long)ncomp * stride;
  const int nc = cols.n;
  const long onew = nc > 0 ? (long)cols.slot[nc - 1] * vstride : 0;
  TC sb[AA_MAX], sn[AA_MAX];
#pragma unroll
  for (int a = 0; a < AA_MAX; ++a) sb[a] = sn[a] = TC(0);
  for (int c = 0; c < ncomp; ++c) {
    const double* gc = c == 0 ? g0 : (c == 1 ? g1 : g2);
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < nq; q += (long)gridDim.x * blockDim.x) {
      const long p = aa_pos<G>(L, q);
      const long o = (long)c * stride + p;
      double g[G], xv[G], fp[G], gp[G], f[G];
      aa_ld<G>(gc + p, g);
      aa_ld<G>(x + o, xv);
      aa_ld<G>(fprev + o, fp);
      aa_ld<G>(gprev + o, gp);
#pragma unroll
      for (int t = 0; t < G; ++t) f[t] = g[t] - xv[t];
      aa_st<G>(x + o, g);
      aa_st<G>(fprev + o, f);
      aa_st<G>(gprev + o, g);
      if (nc == 0) continue;
      TC dn[G], dg[G], ft[G];
#pragma unroll
      for (int t = 0; t < G; ++t) {
        dn[t] = (TC)(f[t] - fp[t]);
        dg[t] = (TC)(g[t] - gp[t]);
        ft[t] = (TC)f[t];
      }
      aa_st<G>(dF + onew + o, dn);
      aa_st<G>(dG + onew + o, dg);
#pragma unroll
      for (int a = 0; a < AA_MAX; ++a) {
        TC da[G];
        if (a < nc - 1)
          aa_ld<G>(dF + (long)cols.slot[a] * vstride + o, da);
        else if (a == nc - 1)
#pragma unroll
          for (int t = 0; t < G; ++t) da[t] = dn[t];
        else
          continue;
#pragma unroll
        for (int t = 0; t < G; ++t) {
          sb[a] += da[t] * ft[t];
          sn[a] += da[t] * dn[t];
        }
      }
    }
  }
  __shared__ double sm[8][2 * AA_MAX];
  double v[32];
#pragma unroll
  for (int a = 0; a < AA_MAX; ++a) {
    v[a] = (double)sb[a];
    v[AA_MAX + a] = (double)sn[a];
  }
  const double w = warp_sum32(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  sm[warp][lane] = w;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sm[k][threadIdx.x];
    part[(long)blockIdx.x * 2 * AA_MAX + threadIdx.x] = s;
  }
  if (nc == 0) return;
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(done, 1u) == gridDim.x - 1;
    if (last) *done = 0u;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    aa_solve_block(cols, part, gridDim.x, M, gamma, status);
  }
}

// u -= sum_a gamma_a dG_a over the live columns, and x = u (the next
// cycle's start); nothing when the solve reported a degenerate history.
template <typename TC, int G>
__global__ void __launch_bounds__(256)
    k_aa_combine(LevelView<double> L, int ncomp, long stride, double* __restrict__ u0, double* __restrict__ u1,
                 double* __restrict__ u2, double* __restrict__ x, const TC* __restrict__ dG,
                 const __grid_constant__ AACols cols, const double* __restrict__ gamma,
                 const unsigned long long* __restrict__ status) {
  pdl_entry();
  if (*status) return;
  const long nq = (long)L.n0 * L.n1 * L.n2 / G;
  const long vstride = (long)ncomp * stride;
  const int nc = cols.n;
  TC gm[AA_MAX];
#pragma unroll
  for (int a = 0; a < AA_MAX; ++a) gm[a] = a < nc ? (TC)gamma[a] : TC(0);
  for (int c = 0; c < ncomp; ++c) {
    double* uc = c == 0 ? u0 : (c == 1 ? u1 : u2);
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < nq; q += (long)gridDim.x * blockDim.x) {
      const long p = aa_pos<G>(L, q);
      const long o = (long)c * stride + p;
      TC sacc[G];
#pragma unroll
      for (int t = 0; t < G; ++t) sacc[t] = TC(0);
#pragma unroll
      for (int a = 0; a < AA_MAX; ++a) {
        if (a >= nc) break;
        TC d[G];
        aa_ld<G>(dG + (long)cols.slot[a] * vstride + o, d);
#pragma unroll
        for (int t = 0; t < G; ++t) sacc[t] += gm[a] * d[t];
      }
      double uv[G];
      aa_ld<G>(uc + p, uv);
#pragma unroll
      for (int t = 0; t < G; ++t) uv[t] -= (double)sacc[t];
      aa_st<G>(uc + p, uv);
      aa_st<G>(x + o, uv);
    }
  }
}

// Blocks for a hierarchy's values: enough to stream them, at most cap (a
// small hierarchy must not fill the GPU with idle blocks that other
// streams' solves could use).
static unsigned aa_grid(const LevelView<double>& L, int ncomp, int per_block, int cap) {
  const long nq = (long)L.n0 * L.n1 * L.n2 / (L.n0 >= 4 ? 4 : 1) * ncomp;
  long g = (nq + per_block - 1) / per_block;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

template <typename TC>
void launch_aa_update_dots(const LevelView<double>& L, int ncomp, long stride, double* const g[3], double* x,
                           double* fprev, double* gprev, TC* dF, TC* dG, const AACols& cols, double* scratch,
                           unsigned long long* status, cudaStream_t st) {
  count_launch();
  AAScratch S = aa_scratch(scratch);
  if (L.n0 >= 4)
    launch_k(k_aa_update_dots<TC, 4>, aa_grid(L, ncomp, 4 * 256, AA_BLOCKS), 256, 0, st, L, ncomp, stride, g[0], g[1], g[2], x, fprev, gprev, dF, dG,
                                                       cols, S.part, S.done, S.M, S.gamma, status);
  else
    launch_k(k_aa_update_dots<TC, 1>, aa_grid(L, ncomp, 4 * 256, AA_BLOCKS), 256, 0, st, L, ncomp, stride, g[0], g[1], g[2], x, fprev, gprev, dF, dG,
                                                       cols, S.part, S.done, S.M, S.gamma, status);
}
template <typename TC>
void launch_aa_combine(const LevelView<double>& L, int ncomp, long stride, double* const u[3], double* x,
                       const TC* dG, const AACols& cols, const double* scratch, const unsigned long long* status,
                       cudaStream_t st) {
  count_launch();
  const double* gamma = aa_scratch(const_cast<double*>(scratch)).gamma;
  if (L.n0 >= 4)
    launch_k(k_aa_combine<TC, 4>, aa_grid(L, ncomp, 256, AA_BLOCKS * 2), 256, 0, st, L, ncomp, stride, u[0], u[1], u[2], x, dG, cols, gamma,
                                                       status);
  else
    launch_k(k_aa_combine<TC, 1>, aa_grid(L, ncomp, 256, AA_BLOCKS * 2), 256, 0, st, L, ncomp, stride, u[0], u[1], u[2], x, dG, cols, gamma,
                                                       status);
}

#define GMG_AA_INST(TC)                                                                                         \
  template void launch_aa_update_dots<TC>(const LevelView<double>&, int, long, double* const[3], double*,        \
                                          double*, double*, TC*, TC*, const AACols&, double*,                    \
                                          unsigned long long*, cudaStream_t);                                    \
  template void launch_aa_combine<TC>(const LevelView<double>&, int, long, double* const[3], double*, const TC*, \
                                      const AACols&, const double*, const unsigned long long*, cudaStream_t);
GMG_AA_INST(double)
GMG_AA_INST(float)

}  // namespace gmg
