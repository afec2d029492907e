// Anderson mixing of successive multigrid iterates (outer acceleration of
// the V-cycle fixed-point map; not part of the paper's method, which runs
// plain cycles).  Vectors are the finest-level unknowns of all components
// (interior cells of ghosted arrays); storage of a vector is ncomp arrays
// of L.ng values laid out back to back.  The iterate x and the previous f
// and g stay FP64; the history columns dF, dG are TC: FP64, or FP32 in
// mixed precision, where the mixing coefficients only steer the iteration
// (the FP64 residual decides convergence) and the columns' products and
// sums run on the FP32 units.
#include "mg_internal.h"
#include "mg_kernels.cuh"

namespace gmg {

// f = g - x;  dF_s = f - fprev, dG_s = g - gprev (unless first);  fprev = f,
// gprev = g.  g is the iterate after the cycle (u itself).
template <typename TC>
__global__ void k_aa_update(LevelView<double> L, int ncomp, long stride, const double* __restrict__ g0,
                            const double* __restrict__ g1, const double* __restrict__ g2,
                            const double* __restrict__ x, double* __restrict__ fprev, double* __restrict__ gprev,
                            TC* __restrict__ dF, TC* __restrict__ dG, int first) {
  const long n = (long)L.n0 * L.n1 * L.n2;
  const double* gs[3] = {g0, g1, g2};
  for (int c = 0; c < ncomp; ++c) {
    const double* gc = gs[c];
    for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x) {
      int i, j, k;
      L.cell(r, i, j, k);
      const long p = L.idx(i, j, k);
      const long o = (long)c * stride + p;
      const double g = gc[p];
      const double f = g - x[o];
      if (!first) {
        dF[o] = (TC)(f - fprev[o]);
        dG[o] = (TC)(g - gprev[o]);
      }
      fprev[o] = f;
      gprev[o] = g;
    }
  }
}

// Block partial sums of dF_a . f and, when newcol >= 0, dF_a . dF_newcol for
// the live columns.  Thread row y of the block handles column y.
template <typename TC>
__global__ void k_aa_dots(LevelView<double> L, int ncomp, long stride, const double* __restrict__ f,
                          const TC* __restrict__ dF, AACols cols, int newcol, double* __restrict__ part) {
  __shared__ double sm[2][AA_MAX][AA_DOT_X / 32];
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long vstride = (long)ncomp * stride;
  const int a = threadIdx.y;
  TC sb = TC(0), sn = TC(0);
  if (a < cols.n) {
    const TC* col = dF + (long)cols.slot[a] * vstride;
    const TC* nw = newcol >= 0 ? dF + (long)newcol * vstride : nullptr;
    for (int c = 0; c < ncomp; ++c)
      for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x) {
        int i, j, k;
        L.cell(r, i, j, k);
        const long o = (long)c * stride + L.idx(i, j, k);
        const TC da = col[o];
        sb += da * (TC)f[o];
        if (nw) sn += da * nw[o];
      }
  }
  const double sbd = warp_sum((double)sb);
  const double snd = warp_sum((double)sn);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sm[0][a][warp] = sbd;
    sm[1][a][warp] = snd;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < AA_DOT_X / 32; ++w) t += sm[threadIdx.x][a][w];
    part[(long)blockIdx.x * 2 * AA_MAX + threadIdx.x * AA_MAX + a] = t;
  }
}

// u -= sum_a gamma_a dG_a over the live columns.
template <typename TC>
__global__ void k_aa_combine(LevelView<double> L, int ncomp, long stride, double* __restrict__ u0,
                             double* __restrict__ u1, double* __restrict__ u2, const TC* __restrict__ dG,
                             AACols cols) {
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long vstride = (long)ncomp * stride;
  double* us[3] = {u0, u1, u2};
  for (int c = 0; c < ncomp; ++c) {
    double* uc = us[c];
    for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x) {
      int i, j, k;
      L.cell(r, i, j, k);
      const long p = L.idx(i, j, k);
      const long o = (long)c * stride + p;
      TC s = TC(0);
      for (int a = 0; a < cols.n; ++a) s += (TC)cols.gamma[a] * dG[(long)cols.slot[a] * vstride + o];
      uc[p] -= (double)s;
    }
  }
}

template <typename TC>
void launch_aa_update(const LevelView<double>& L, int ncomp, long stride, double* const g[3], const double* x,
                      double* fprev, double* gprev, TC* dF, TC* dG, int first, cudaStream_t st) {
  count_launch();
  k_aa_update<TC><<<AA_BLOCKS, 256, 0, st>>>(L, ncomp, stride, g[0], g[1], g[2], x, fprev, gprev, dF, dG, first);
}
template <typename TC>
void launch_aa_dots(const LevelView<double>& L, int ncomp, long stride, const double* f, const TC* dF,
                    const AACols& cols, int newcol, double* part, cudaStream_t st) {
  count_launch();
  k_aa_dots<TC><<<AA_BLOCKS, dim3(AA_DOT_X, AA_MAX), 0, st>>>(L, ncomp, stride, f, dF, cols, newcol, part);
}
template <typename TC>
void launch_aa_combine(const LevelView<double>& L, int ncomp, long stride, double* const u[3], const TC* dG,
                       const AACols& cols, cudaStream_t st) {
  count_launch();
  k_aa_combine<TC><<<AA_BLOCKS, 256, 0, st>>>(L, ncomp, stride, u[0], u[1], u[2], dG, cols);
}

#define GMG_AA_INST(TC)                                                                                        \
  template void launch_aa_update<TC>(const LevelView<double>&, int, long, double* const[3], const double*,      \
                                     double*, double*, TC*, TC*, int, cudaStream_t);                            \
  template void launch_aa_dots<TC>(const LevelView<double>&, int, long, const double*, const TC*,               \
                                   const AACols&, int, double*, cudaStream_t);                                  \
  template void launch_aa_combine<TC>(const LevelView<double>&, int, long, double* const[3], const TC*,         \
                                      const AACols&, cudaStream_t);
GMG_AA_INST(double)
GMG_AA_INST(float)

}  // namespace gmg
