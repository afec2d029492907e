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
#include "mg_accel.cuh"

namespace gmg {

// An L2 prefetch of the 16-byte (or 8-byte) group at p.  The mixing kernels
// issue them before waiting for the kernel they depend on, for data that
// kernel does not write, so the DRAM reads overlap its tail; a prefetch
// changes no value.
__device__ __forceinline__ void l2_prefetch(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}


// The least-squares step (run by the last block of k_aa_update_dots to
// finish): reduce the blocks' partial dot products in a fixed order, enter
// the newest column's row into the Gram matrix M (AA_MAX x AA_MAX over ring
// slots, stored in TC), and solve (M_live / dmax + shift I) gamma = b / dmax
// by Cholesky, dmax the largest live diagonal entry.  status = 0 with gamma
// written, or 1 when the history is degenerate (non-positive pivot,
// non-finite values): the host then restarts the mixing and the
// combination is skipped.
template <typename TC>
__device__ void aa_solve_block(const AACols& cols, const double* part_d, int nblocks, double* __restrict__ M_d,
                               double* __restrict__ gamma, unsigned long long* __restrict__ status) {
  const TC* part = reinterpret_cast<const TC*>(part_d);
  TC* M = reinterpret_cast<TC*>(M_d);
  __shared__ TC red[8][2 * AA_MAX];
  __shared__ TC s[2 * AA_MAX];
  __shared__ TC Ms[AA_MAX * AA_MAX];
  const int t = threadIdx.x, q = t & 31, w = t >> 5;
  // every load issued at once: the stored Gram matrix and the partial sums
  // (at most AA_BLOCKS / 8 per thread), summed pairwise
  if (t < AA_MAX * AA_MAX) Ms[t] = __ldcg(M + t);
  TC pv[AA_BLOCKS / 8];
#pragma unroll
  for (int r = 0; r < AA_BLOCKS / 8; ++r) {
    const int b = w + 8 * r;
    pv[r] = b < nblocks ? __ldcg(part + (long)b * 2 * AA_MAX + q) : TC(0);
  }
#pragma unroll
  for (int h = 1; h < AA_BLOCKS / 8; h *= 2)
#pragma unroll
    for (int r = 0; r + h < AA_BLOCKS / 8; r += 2 * h) pv[r] += pv[r + h];
  red[w][q] = pv[0];
  __syncthreads();
  if (t >= 32) return;
  s[t] = ((red[0][t] + red[1][t]) + (red[2][t] + red[3][t])) + ((red[4][t] + red[5][t]) + (red[6][t] + red[7][t]));
  const int n = cols.n, slot = cols.slot[n - 1];
  __syncwarp();
  if (t < n) {
    const int c = cols.slot[t];
    const TC v = s[AA_MAX + t];
    Ms[slot * AA_MAX + c] = v;
    Ms[c * AA_MAX + slot] = v;
    M[slot * AA_MAX + c] = v;
    M[c * AA_MAX + slot] = v;
  }
  __syncwarp();
  TC dmax = TC(0);
  for (int a = 0; a < n; ++a) dmax = fmax(dmax, Ms[cols.slot[a] * AA_MAX + cols.slot[a]]);
  bool ok = dmax > TC(0) && dmax <= (sizeof(TC) == 4 ? TC(3.4e38f) : TC(1.7976931348623157e308));
  const TC sc = ok ? TC(1) / dmax : TC(0);
  if constexpr (sizeof(TC) == 4) {
    float row[AA_MAX];
    const int ra = t < n ? cols.slot[t] : 0;
#pragma unroll
    for (int k = 0; k < AA_MAX; ++k)
      row[k] = (t < n && k < n) ? Ms[ra * AA_MAX + cols.slot[k]] * sc + (k == t ? AA_SHIFT<float> : 0.0f)
                                : (k == t ? 1.0f : 0.0f);
    float z = t < n ? s[t] * sc : 0.0f;
    ok = __all_sync(0xffffffffu, ok);
    if (ok) ok = chol_warp_f32(row, z, t);
    if (ok) ok = __all_sync(0xffffffffu, z - z == 0.0f);
    if (ok && t < n) gamma[t] = (double)z;
  } else {
    // FP64: the augmented matrix in shared memory, lane t owning row t;
    // L overwrites the lower triangle and L^-1 b column n
    __shared__ double A[AA_MAX][AA_MAX + 2];
    __shared__ double inv[AA_MAX];
    if (t < n) {
      const int ra = cols.slot[t];
      for (int b = 0; b < n; ++b) A[t][b] = Ms[ra * AA_MAX + cols.slot[b]] * sc;
      A[t][n] = s[t] * sc;
      A[t][t] += AA_SHIFT<double>;
    }
    __syncwarp();
    for (int j = 0; ok && j < n; ++j) {
      const double piv = A[j][j];
      if (!(piv > 0.0)) {
        ok = false;
        break;
      }
      const double id = rsqrt(piv);
      __syncwarp();
      if (t == j) {
        A[j][j] = piv * id;
        A[j][n] *= id;
        inv[j] = id;
      }
      if (t > j && t < n) A[t][j] *= id;
      __syncwarp();
      if (t > j && t < n) {
        // all operands first: the updates are independent, but stores and
        // loads to the same array would otherwise serialise them
        const double lt = A[t][j], zj = A[j][n];
        double rw[AA_MAX], cl[AA_MAX];
#pragma unroll
        for (int k = 1; k < AA_MAX; ++k) {
          const bool in = j + k <= t;
          rw[k] = in ? A[t][j + k] : 0.0;
          cl[k] = in ? A[j + k][j] : 0.0;
        }
        const double rn = A[t][n];
#pragma unroll
        for (int k = 1; k < AA_MAX; ++k)
          if (j + k <= t) A[t][j + k] = rw[k] - lt * cl[k];
        A[t][n] = rn - lt * zj;
      }
      __syncwarp();
    }
    // back substitution L^T y = z, lane r holding z_r
    double z = (ok && t < n) ? A[t][n] : 0.0;
    for (int i = n - 1; ok && i >= 0; --i) {
      const double yi = __shfl_sync(0xffffffffu, z * inv[t < n ? t : 0], i);
      if (t == i) z = yi;
      if (t < i) z -= A[i][t] * yi;
    }
    if (ok) ok = __all_sync(0xffffffffu, t >= n || z - z == 0.0);
    if (ok && t < n) gamma[t] = z;
  }
  if (t == 0) *status = ok ? 0ULL : 1ULL;
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
                     TC* __restrict__ dG, const __grid_constant__ AACols hcols, const AACols* __restrict__ dcols,
                     double* __restrict__ part, unsigned int* __restrict__ done, double* __restrict__ M,
                     double* __restrict__ gamma, unsigned long long* __restrict__ status) {
  // Before waiting for the cycle's last kernel: L2 prefetches of this
  // thread's first group of x, f', g' and the older dF columns (written by
  // earlier cycles, not by that kernel).  The live columns come from the
  // launch, or (device-side cycle loop) from the loop step of the previous
  // cycle, several kernels back.
  {
    const long q0 = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (q0 < (long)L.n0 * L.n1 * L.n2 / G) {
      const long o = aa_pos<G>(L, q0), vs = (long)ncomp * stride;
      l2_prefetch(x + o);
      l2_prefetch(fprev + o);
      l2_prefetch(gprev + o);
      const int n = dcols ? __ldcg(&dcols->n) : hcols.n;
      for (int a = 0; a + 1 < n && a < AA_MAX; ++a)
        l2_prefetch(dF + (long)(dcols ? __ldcg(&dcols->slot[a]) : hcols.slot[a]) * vs + o);
    }
  }
  pdl_entry();
  // the live columns: from the launch, or (device-side cycle loop) from
  // device memory written by the preceding loop step
  __shared__ AACols scols;
  if (dcols) {
    if (threadIdx.x == 0) scols = *dcols;
    __syncthreads();
  }
  const AACols& cols = dcols ? scols : hcols;
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
      aa_ld_u<G>(gc + p, g);
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
  // block sums in the history's precision (FP32 in mixed precision: FP64
  // additions are long-latency on this GPU, and the products are FP32)
  __shared__ TC sm[8][2 * AA_MAX];
  TC v[32];
#pragma unroll
  for (int a = 0; a < AA_MAX; ++a) {
    v[a] = sb[a];
    v[AA_MAX + a] = sn[a];
  }
  const TC w = warp_sum32(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  sm[warp][lane] = w;
  __syncthreads();
  if (threadIdx.x < 32) {
    TC s = TC(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += sm[k][threadIdx.x];
    reinterpret_cast<TC*>(part)[(long)blockIdx.x * 2 * AA_MAX + threadIdx.x] = s;
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
    aa_solve_block<TC>(cols, part, gridDim.x, M, gamma, status);
  }
}

// u -= sum_a gamma_a dG_a over the live columns, and x = u (the next
// cycle's start); nothing when the solve reported a degenerate history.
template <typename TC, int G>
__global__ void __launch_bounds__(256)
    k_aa_combine(LevelView<double> L, int ncomp, long stride, double* __restrict__ u0, double* __restrict__ u1,
                 double* __restrict__ u2, double* __restrict__ x, const TC* __restrict__ dG,
                 const __grid_constant__ AACols hcols, const AACols* __restrict__ dcols,
                 const double* __restrict__ gamma, const unsigned long long* __restrict__ status) {
  // Before waiting for the update kernel (whose last block solves the
  // least-squares problem while the other SMs idle): L2 prefetches of this
  // thread's first group of u and of the older dG columns, which that
  // kernel does not write (it writes the newest column, gamma and status).
  {
    const long q0 = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (q0 < (long)L.n0 * L.n1 * L.n2 / G) {
      const long p = aa_pos<G>(L, q0), vs = (long)ncomp * stride;
      l2_prefetch(u0 + p);
      const int n = dcols ? __ldcg(&dcols->n) : hcols.n;
      for (int a = 0; a + 1 < n && a < AA_MAX; ++a)
        l2_prefetch(dG + (long)(dcols ? __ldcg(&dcols->slot[a]) : hcols.slot[a]) * vs + p);
    }
  }
  pdl_entry();
  __shared__ AACols scols;
  if (dcols) {
    if (threadIdx.x == 0) scols = *dcols;
    __syncthreads();
  }
  const AACols& cols = dcols ? scols : hcols;
  if (*status || cols.n == 0) return;
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
      aa_ld_u<G>(uc + p, uv);
#pragma unroll
      for (int t = 0; t < G; ++t) uv[t] -= (double)sacc[t];
      aa_st_u<G>(uc + p, uv);
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
                           unsigned long long* status, cudaStream_t st, const AACols* dcols) {
  count_launch();
  AAScratch S = aa_scratch(scratch);
  const unsigned gb = aa_grid(L, ncomp, 256, AA_BLOCKS);
  if (L.n0 >= 4)
    launch_k(k_aa_update_dots<TC, 4>, gb, 256, 0, st, L, ncomp, stride, g[0], g[1], g[2], x, fprev, gprev, dF, dG,
             cols, dcols, S.part, S.done, S.M, S.gamma, status);
  else
    launch_k(k_aa_update_dots<TC, 1>, gb, 256, 0, st, L, ncomp, stride, g[0], g[1], g[2], x, fprev, gprev, dF, dG,
             cols, dcols, S.part, S.done, S.M, S.gamma, status);
}
template <typename TC>
void launch_aa_combine(const LevelView<double>& L, int ncomp, long stride, double* const u[3], double* x,
                       const TC* dG, const AACols& cols, const double* scratch, const unsigned long long* status,
                       cudaStream_t st, const AACols* dcols) {
  count_launch();
  const double* gamma = aa_scratch(const_cast<double*>(scratch)).gamma;
  const unsigned gb = aa_grid(L, ncomp, 256, AA_BLOCKS * 2);
  if (L.n0 >= 4)
    launch_k(k_aa_combine<TC, 4>, gb, 256, 0, st, L, ncomp, stride, u[0], u[1], u[2], x, dG, cols, dcols, gamma,
             status);
  else
    launch_k(k_aa_combine<TC, 1>, gb, 256, 0, st, L, ncomp, stride, u[0], u[1], u[2], x, dG, cols, dcols, gamma,
             status);
}

// One step of the device-side cycle loop (one thread): the weighted
// relative residual rel = red[1] / max(red[2], 1e-300) of the residual just
// evaluated (non-finite norms give NaN), the cycle count, the mixing ring
// (restarted when the last mixing step found a degenerate history, red[3]),
// the stopping rule in the order of the host loop, the live columns of the
// next cycle's mixing step, and the while node's condition.
__global__ void k_loop_decide(LoopState* __restrict__ S, const unsigned long long* __restrict__ red, LoopParams P,
                              cudaGraphConditionalHandle h, int first) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double num = __longlong_as_double((long long)red[1]), den = __longlong_as_double((long long)red[2]);
  double rel;
  if (isinf(num) || isinf(den) || isnan(num) || isnan(den))
    rel = __longlong_as_double(0x7ff8000000000000LL);
  else
    rel = num / (den > 1e-300 ? den : 1e-300);
  if (first) {
    S->cyc = 0;
    S->ncol = 0;
    S->head = 0;
    S->mixstep = 0;
  } else {
    S->cyc += 1;
    if (S->mixstep && red[3] != 0ULL) S->ncol = 0;
  }
  const int cyc = S->cyc;
  if (cyc < 1024) S->hist[cyc] = rel;
  S->rel = rel;
  int stop = 1, status = 0;
  if (rel != rel)
    status = 5;  // MG_ERR_NAN
  else if (rel <= P.tol)
    status = 0;
  else if (cyc >= P.max_cycles)
    status = 3;  // MG_ERR_NOCONV
  else if (P.stall_window > 0 && cyc >= P.stall_window && rel > 0.95 * S->hist[cyc - P.stall_window])
    status = 4;  // MG_ERR_STALLED
  else
    stop = 0;
  AACols c;
  c.n = 0;
  if (!stop && P.m > 0 && cyc > 0) {
    const int m = P.m, slot = S->head;
    S->head = (S->head + 1) % m;
    if (S->ncol < m) S->ncol += 1;
    c.n = S->ncol;
    for (int a = 0; a < c.n; ++a) c.slot[a] = (slot - c.n + 1 + a + m) % m;
  }
  S->cols = c;
  S->mixstep = c.n > 0;
  S->status = status;
  S->stop = stop;
  cudaGraphSetConditional(h, stop ? 0u : 1u);
}

void launch_loop_decide(LoopState* S, const unsigned long long* red, const LoopParams& P,
                        cudaGraphConditionalHandle h, int first, cudaStream_t st) {
  count_launch();
  launch_k(k_loop_decide, 1, 32, 0, st, S, red, P, h, first);
}

#define GMG_AA_INST(TC)                                                                                         \
  template void launch_aa_update_dots<TC>(const LevelView<double>&, int, long, double* const[3], double*,        \
                                          double*, double*, TC*, TC*, const AACols&, double*,                    \
                                          unsigned long long*, cudaStream_t, const AACols*);                     \
  template void launch_aa_combine<TC>(const LevelView<double>&, int, long, double* const[3], double*, const TC*, \
                                      const AACols&, const double*, const unsigned long long*, cudaStream_t,     \
                                      const AACols*);
GMG_AA_INST(double)
GMG_AA_INST(float)

}  // namespace gmg
