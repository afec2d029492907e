// Pointwise kernels of the xCFC solve order (Sec. 2.6) and of elliptic
// divergence cleaning (Sec. 2.2).
#include "mg_internal.h"
#include "mg_kernels.cuh"
#include "mg_xcfc.cuh"

namespace gmg {

static inline unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }
static inline dim3 blk(int three) { return three ? dim3(32, 4, 2) : dim3(32, 8, 1); }
static inline dim3 grd(const LevelView<double>& L, dim3 b) {
  return dim3(cdiv(L.n0, b.x), cdiv(L.n1, b.y), cdiv(L.n2, b.z));
}

// A~^2 = A~_ij A~^ij with A~_ij = 2 E_ij - 2/3 div X delta_ij, E the
// symmetric gradient of X in orthonormal components (eq. Aij); order rr,
// tt, pp, rt, rp, tp.
template <int G>
__global__ void k_a2(LevelView<double> L, const double* __restrict__ a, const double* __restrict__ b,
                     const double* __restrict__ c, double* __restrict__ A2) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const long p = L.idx(i, j, k);
  double A[6];
  aij_cell<G>(L, a, b, c, i, j, p, A);
  A2[p] = A[0] * A[0] + A[1] * A[1] + A[2] * A[2] + 2.0 * (A[3] * A[3] + A[4] * A[4] + A[5] * A[5]);
}

// alpha-psi coefficient c = 2 pi (U + 2 S) psi^-2 + 7/8 A2 psi^-8 (eq. alpha).
__global__ void k_alpha_coef(LevelView<double> L, const double* __restrict__ U, const double* __restrict__ S,
                             const double* __restrict__ A2, const double* __restrict__ dpsi,
                             double* __restrict__ c) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const long p = L.idx(i, j, k);
  const double ip = 1.0 / (1.0 + dpsi[p]);
  const double ip2 = ip * ip;
  const double ip8 = (ip2 * ip2) * (ip2 * ip2);
  c[p] = 2.0 * PI_D * (U[p] + 2.0 * S[p]) * ip2 + 0.875 * A2[p] * ip8;
}

// s = alpha psi^-6 = (alpha psi) psi^-7 on every cell, ghosts included
// (the ghosts of both deviations carry their boundary values).
__global__ void k_lapse_factor(long n, const double* __restrict__ dpsi, const double* __restrict__ dap,
                               double* __restrict__ s) {
  pdl_entry();
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const double ip = 1.0 / (1.0 + dpsi[p]);
    const double ip2 = ip * ip;
    s[p] = (1.0 + dap[p]) * (ip2 * ip2 * ip2 * ip);
  }
}

// Shift source 16 pi s S_i + 2 A~_ij (grad s)_j (eq. beta), s = alpha psi^-6.
template <int G>
__global__ void k_beta_rhs(LevelView<double> L, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ c, const double* __restrict__ sg,
                           const double* __restrict__ S0, const double* __restrict__ S1,
                           const double* __restrict__ S2, double* __restrict__ f0, double* __restrict__ f1,
                           double* __restrict__ f2) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const long p = L.idx(i, j, k);
  double A[6];
  aij_cell<G>(L, a, b, c, i, j, p, A);
  Stencil<double> st{L, p};
  double g0 = st.d1(sg, 0), g1 = st.d1(sg, 1), g2 = st.d1(sg, 2);
  if (G == CYL) {
    g2 *= L.TI(TI_IX, i);
  } else if (G == SPH) {
    const double ir = L.TI(TI_IX, i);
    g1 *= ir;
    g2 *= ir * L.TJ(TJ_IS, j);
  }
  const double sv = sg[p];
  const double k16 = 16.0 * PI_D * sv;
  f0[p] = k16 * S0[p] + 2.0 * (A[0] * g0 + A[3] * g1 + A[4] * g2);
  f1[p] = k16 * S1[p] + 2.0 * (A[3] * g0 + A[1] * g1 + A[5] * g2);
  f2[p] = k16 * S2[p] + 2.0 * (A[4] * g0 + A[5] * g1 + A[2] * g2);
}

__global__ void k_scale_into(LevelView<double> L, const double* __restrict__ src, double a,
                             double* __restrict__ dst) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const long p = L.idx(i, j, k);
  dst[p] = a * src[p];
}

// --------------------------------------------------- divergence cleaning
// B is in the caller's ghost-free layout; its ghosts are copies of the
// boundary cells (zero normal gradient).

__global__ void k_div_central(LevelView<double> L, const double* __restrict__ B0,
                              const double* __restrict__ B1, const double* __restrict__ B2,
                              double* __restrict__ div, double* __restrict__ part) {
  pdl_entry();
  __shared__ double sm[32];
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long s1 = L.n0, s2 = (long)L.n0 * L.n1;
  const double c0 = 0.5 / L.h0, c1 = 0.5 / L.h1, c2 = 0.5 / L.h2;
  double acc = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    double d = (B0[i < L.n0 - 1 ? q + 1 : q] - B0[i > 0 ? q - 1 : q]) * c0 +
               (B1[j < L.n1 - 1 ? q + s1 : q] - B1[j > 0 ? q - s1 : q]) * c1;
    if (L.three) d += (B2[k < L.n2 - 1 ? q + s2 : q] - B2[k > 0 ? q - s2 : q]) * c2;
    div[L.idx(i, j, k)] = d;
    acc += d;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
}

// max |div| -> red[0] (atomic), sum div^2 -> part (per block).
__global__ void k_div_norms(LevelView<double> L, const double* __restrict__ div, double* __restrict__ part,
                            unsigned long long* red) {
  pdl_entry();
  __shared__ double sm[32];
  const long n = (long)L.n0 * L.n1 * L.n2;
  double s = 0.0;
  double m[1] = {0.0};
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const double d = div[L.idx(i, j, k)];
    s += d * d;
    m[0] = fmax(m[0], fabs(d));
    if (d != d) m[0] = INFINITY;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
  __syncthreads();
  block_max_atomic<1>(m, red);
}

__global__ void k_sub_mean_into(LevelView<double> L, const double* __restrict__ div,
                                const double* __restrict__ part, int nparts, double* __restrict__ b) {
  pdl_entry();
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += part[q];
    mean = s / ((double)L.n0 * L.n1 * L.n2);
  }
  __syncthreads();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    b[p] = div[p] - mean;
  }
}

// B <- B - grad Phi (central differences, Neumann ghosts of Phi).
__global__ void k_grad_update(LevelView<double> L, const double* __restrict__ phi, double* __restrict__ B0,
                              double* __restrict__ B1, double* __restrict__ B2) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  const double c0 = 0.5 / L.h0, c1 = 0.5 / L.h1, c2 = 0.5 / L.h2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    const double pc = phi[p];
    B0[q] -= ((i < L.n0 - 1 ? phi[p + 1] : pc) - (i > 0 ? phi[p - 1] : pc)) * c0;
    B1[q] -= ((j < L.n1 - 1 ? phi[p + L.sx] : pc) - (j > 0 ? phi[p - L.sx] : pc)) * c1;
    if (L.three) B2[q] -= ((k < L.n2 - 1 ? phi[p + L.sy] : pc) - (k > 0 ? phi[p - L.sy] : pc)) * c2;
  }
}

// Central divergence on cylindrical / spherical grids (Sec. 2.2,
// (1/sqrt(g)) d_i (sqrt(g) q^i) in physical components, every metric factor
// at the centre of the cell it multiplies) from ghosted B (outer ghosts
// copied, origin / axis parities); part gets the block sums of w div, w the
// weight under which the flux-form Laplacian sums to zero (R, r^2 sin).
template <int G>
__global__ void k_div_curv(LevelView<double> L, const double* __restrict__ B0, const double* __restrict__ B1,
                           const double* __restrict__ B2, double* __restrict__ div, double* __restrict__ part) {
  pdl_entry();
  __shared__ double sm[32];
  const long n = (long)L.n0 * L.n1 * L.n2;
  double acc = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    const double x = L.TI(TI_X, i), xp = L.TI(TI_X, i + 1), xm = L.TI(TI_X, i - 1);
    double d;
    if (G == CYL) {
      d = (xp * B0[p + 1] - xm * B0[p - 1]) / (2.0 * L.h0 * x) + (B1[p + L.sx] - B1[p - L.sx]) / (2.0 * L.h1);
      if (L.three) d += (B2[p + L.sy] - B2[p - L.sy]) / (2.0 * L.h2 * x);
    } else {
      const double st = L.TJ(TJ_S, j), sp = L.TJ(TJ_S, j + 1), sn = L.TJ(TJ_S, j - 1);
      d = (xp * xp * B0[p + 1] - xm * xm * B0[p - 1]) / (2.0 * L.h0 * x * x) +
          (sp * B1[p + L.sx] - sn * B1[p - L.sx]) / (2.0 * L.h1 * x * st);
      if (L.three) d += (B2[p + L.sy] - B2[p - L.sy]) / (2.0 * L.h2 * x * st);
    }
    div[p] = d;
    acc += norm_weight(L, i, j) * d;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
}

// b = div - (sum of part) / wsum (the weighted mean).
__global__ void k_sub_wmean_into(LevelView<double> L, const double* __restrict__ div,
                                 const double* __restrict__ part, int nparts, double wsum,
                                 double* __restrict__ b) {
  pdl_entry();
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += part[q];
    mean = s / wsum;
  }
  __syncthreads();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    b[p] = div[p] - mean;
  }
}

// B <- B - grad Phi in physical components (central differences, Phi's
// ghosts filled): (d_0, d_1, d_2 / R) cylindrical, (d_0, d_1 / r,
// d_2 / (r sin)) spherical.  B ghost-free (the caller's layout).
template <int G>
__global__ void k_grad_update_curv(LevelView<double> L, const double* __restrict__ phi, double* __restrict__ B0,
                                   double* __restrict__ B1, double* __restrict__ B2) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    const double x = L.TI(TI_X, i);
    const double g0 = (phi[p + 1] - phi[p - 1]) / (2.0 * L.h0);
    double g1 = (phi[p + L.sx] - phi[p - L.sx]) / (2.0 * L.h1);
    double g2 = L.three ? (phi[p + L.sy] - phi[p - L.sy]) / (2.0 * L.h2) : 0.0;
    if (G == CYL) {
      g2 /= x;
    } else {
      g1 /= x;
      g2 /= (x * L.TJ(TJ_S, j));
    }
    B0[q] -= g0;
    B1[q] -= g1;
    if (L.three) B2[q] -= g2;
  }
}

// Initial alpha psi deviation from the caller's alpha (ghost-free) and the
// solved psi deviation; and alpha = (alpha psi) / psi back to the caller.
__global__ void k_ap_init(LevelView<double> L, const double* __restrict__ alpha, const double* __restrict__ dpsi,
                          double* __restrict__ dap) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    dap[p] = alpha[q] * (1.0 + dpsi[p]) - 1.0;
  }
}
__global__ void k_alpha_out(LevelView<double> L, const double* __restrict__ dap, const double* __restrict__ dpsi,
                            double* __restrict__ alpha) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    alpha[q] = (1.0 + dap[p]) / (1.0 + dpsi[p]);
  }
}

// ------------------------------------------------------------ launchers
#define GEOMS(G_, ...)                                              \
  switch (G_) {                                                      \
    case CART: { constexpr int GG = CART; __VA_ARGS__; } break;     \
    case CYL:  { constexpr int GG = CYL;  __VA_ARGS__; } break;     \
    default:   { constexpr int GG = SPH;  __VA_ARGS__; } break;     \
  }

void launch_xcfc_a2(const LevelView<double>& L, double* const X[3], double* A2, cudaStream_t st) {
  count_launch();
  dim3 b = blk(L.three), g = grd(L, b);
  GEOMS(L.geom, launch_k(k_a2<GG>, g, b, 0, st, L, X[0], X[1], X[2], A2));
}

void launch_xcfc_alpha_coef(const LevelView<double>& L, const double* U, const double* S, const double* A2,
                            const double* dpsi, double* c, cudaStream_t st) {
  count_launch();
  dim3 b = blk(L.three), g = grd(L, b);
  launch_k(k_alpha_coef, g, b, 0, st, L, U, S, A2, dpsi, c);
}

void launch_xcfc_beta_rhs(const LevelView<double>& L, double* const X[3], const double* dpsi, const double* dap,
                          double* sg, double* const Si[3], double* const f[3], cudaStream_t st) {
  count_launch(2);
  const long ng = L.sy * (L.n2 + 2 * L.three);
  launch_k(k_lapse_factor, (unsigned)((ng + 255) / 256 > 4096 ? 4096 : (ng + 255) / 256), 256, 0, st, ng, dpsi, dap,
                                                                                                  sg);
  dim3 b = blk(L.three), g = grd(L, b);
  GEOMS(L.geom, launch_k(k_beta_rhs<GG>, g, b, 0, st, L, X[0], X[1], X[2], sg, Si[0], Si[1], Si[2], f[0], f[1], f[2]));
}

void launch_scale_into(const LevelView<double>& L, const double* src, double a, double* dst, cudaStream_t st) {
  count_launch();
  dim3 b = blk(L.three), g = grd(L, b);
  launch_k(k_scale_into, g, b, 0, st, L, src, a, dst);
}

void launch_div_central(const LevelView<double>& L, double* const B[3], double* div, double* part, int nparts,
                        cudaStream_t st) {
  count_launch();
  launch_k(k_div_central, nparts, 256, 0, st, L, B[0], B[1], B[2], div, part);
}

void launch_div_norms(const LevelView<double>& L, const double* div, double* part, int nparts,
                      unsigned long long* red, cudaStream_t st) {
  count_launch();
  launch_k(k_div_norms, nparts, 256, 0, st, L, div, part, red);
}

void launch_sub_mean_into(const LevelView<double>& L, const double* div, const double* part, int nparts,
                          double* b, cudaStream_t st) {
  count_launch();
  launch_k(k_sub_mean_into, nparts, 256, 0, st, L, div, part, nparts, b);
}

void launch_grad_update(const LevelView<double>& L, const double* phi, double* const B[3], cudaStream_t st) {
  count_launch();
  const long n = (long)L.n0 * L.n1 * L.n2;
  long g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  launch_k(k_grad_update, (unsigned)g, 256, 0, st, L, phi, B[0], B[1], B[2]);
}

// ------------------------------------------ exact-projection div-B cleaning
// Cartesian grids, every n >= 4.  The parity classes of the cells, s = (i &
// 1) | (j & 1) << 1 | (k & 1) << 2, are solved as separate compact Neumann
// problems of n / 2 cells per dimension (div_c grad_c with mirrored Phi
// ghosts and copied ghosts of its argument splits that way).  Class-major
// buffers: class s holds [s M, (s + 1) M), M = N / 2^d, its cell (i, j, k)
// at (i >> 1) + m0 ((j >> 1) + m1 (k >> 1)), m = n / 2.

struct ClassGrid {
  int lm0, lm1;  // log2 of n0 / 2, n1 / 2
  long M;        // cells per class
  __device__ __forceinline__ void fine(int s, long r, int three, int& i, int& j, int& k) const {
    const int a = (int)(r & ((1L << lm0) - 1));
    const long t = r >> lm0;
    const int b = (int)(t & ((1L << lm1) - 1));
    const int c = (int)(t >> lm1);
    i = 2 * a + (s & 1);
    j = 2 * b + ((s >> 1) & 1);
    k = three ? 2 * c + ((s >> 2) & 1) : 0;
  }
  __device__ __forceinline__ long at(int i, int j, int k) const {
    const int s = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    return (long)s * M + (i >> 1) + ((long)(j >> 1) << lm0) + ((long)(k >> 1) << (lm0 + lm1));
  }
};

__host__ __device__ inline ClassGrid class_grid(const LevelView<double>& L) {
  ClassGrid g;
  g.lm0 = L.ln0 - 1;
  g.lm1 = L.ln1 - 1;
  g.M = ((long)L.n0 * L.n1 * L.n2) >> (L.three ? 3 : 2);
  return g;
}

// Block sums of div over each class: block (p, s) strides over class s.
__global__ void k_class_sums(LevelView<double> L, ClassGrid G, const double* __restrict__ div,
                             double* __restrict__ part) {
  pdl_entry();
  __shared__ double sm[32];
  const int s = blockIdx.y;
  double acc = 0.0;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < G.M; r += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    G.fine(s, r, L.three, i, j, k);
    acc += div[L.idx(i, j, k)];
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += sm[w];
    part[s * gridDim.x + blockIdx.x] = t;
  }
}

// Class s of div minus its mean into the class-major buffer dst.
__global__ void k_class_gather(LevelView<double> L, ClassGrid G, const double* __restrict__ div,
                               const double* __restrict__ part, int nparts, double* __restrict__ dst) {
  pdl_entry();
  __shared__ double mean;
  const int s = blockIdx.y;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nparts; ++q) t += part[s * nparts + q];
    mean = t / (double)G.M;
  }
  __syncthreads();
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < G.M; r += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    G.fine(s, r, L.three, i, j, k);
    dst[s * G.M + r] = div[L.idx(i, j, k)] - mean;
  }
}

// B <- B - grad Phi, central differences with Phi ghosts mirrored about the
// boundary cell's centre (Phi_{-1} = Phi_1, Phi_n = Phi_{n-2}), Phi read
// from the class-major buffer; phi_out (nullable, ghost-free) receives Phi.
__global__ void k_grad_update_exact(LevelView<double> L, ClassGrid G, const double* __restrict__ phis,
                                    double* __restrict__ B0, double* __restrict__ B1, double* __restrict__ B2,
                                    double* __restrict__ phi_out) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  const double c0 = 0.5 / L.h0, c1 = 0.5 / L.h1, c2 = 0.5 / L.h2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const int ip = i < L.n0 - 1 ? i + 1 : L.n0 - 2, im = i > 0 ? i - 1 : 1;
    const int jp = j < L.n1 - 1 ? j + 1 : L.n1 - 2, jm = j > 0 ? j - 1 : 1;
    B0[q] -= (phis[G.at(ip, j, k)] - phis[G.at(im, j, k)]) * c0;
    B1[q] -= (phis[G.at(i, jp, k)] - phis[G.at(i, jm, k)]) * c1;
    if (L.three) {
      const int kp = k < L.n2 - 1 ? k + 1 : L.n2 - 2, km = k > 0 ? k - 1 : 1;
      B2[q] -= (phis[G.at(i, j, kp)] - phis[G.at(i, j, km)]) * c2;
    }
    if (phi_out) phi_out[q] = phis[G.at(i, j, k)];
  }
}

void launch_class_gather(const LevelView<double>& L, const double* div, double* part, int nparts, double* dst,
                         cudaStream_t st) {
  count_launch(2);
  const ClassGrid G = class_grid(L);
  const dim3 grid(nparts, L.three ? 8 : 4);
  launch_k(k_class_sums, grid, 256, 0, st, L, G, div, part);
  launch_k(k_class_gather, grid, 256, 0, st, L, G, div, (const double*)part, nparts, dst);
}

void launch_grad_update_exact(const LevelView<double>& L, const double* phis, double* const B[3], double* phi_out,
                              cudaStream_t st) {
  count_launch();
  const long n = (long)L.n0 * L.n1 * L.n2;
  long g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  launch_k(k_grad_update_exact, (unsigned)g, 256, 0, st, L, class_grid(L), phis, B[0], B[1], B[2], phi_out);
}

void launch_div_curv(const LevelView<double>& L, double* const Bg[3], double* div, double* part, int nparts,
                     cudaStream_t st) {
  count_launch();
  if (L.geom == CYL)
    launch_k(k_div_curv<CYL>, nparts, 256, 0, st, L, Bg[0], Bg[1], Bg[2], div, part);
  else
    launch_k(k_div_curv<SPH>, nparts, 256, 0, st, L, Bg[0], Bg[1], Bg[2], div, part);
}

void launch_sub_wmean_into(const LevelView<double>& L, const double* div, const double* part, int nparts,
                           double wsum, double* b, cudaStream_t st) {
  count_launch();
  launch_k(k_sub_wmean_into, nparts, 256, 0, st, L, div, part, nparts, wsum, b);
}

void launch_grad_update_curv(const LevelView<double>& L, const double* phi, double* const B[3], cudaStream_t st) {
  count_launch();
  const long n = (long)L.n0 * L.n1 * L.n2;
  long g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  if (L.geom == CYL)
    launch_k(k_grad_update_curv<CYL>, (unsigned)g, 256, 0, st, L, phi, B[0], B[1], B[2]);
  else
    launch_k(k_grad_update_curv<SPH>, (unsigned)g, 256, 0, st, L, phi, B[0], B[1], B[2]);
}

static unsigned flat_grid(const LevelView<double>& L) {
  long n = (long)L.n0 * L.n1 * L.n2;
  long g = (n + 255) / 256;
  return (unsigned)(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

void launch_xcfc_ap_init(const LevelView<double>& L, const double* alpha, const double* dpsi, double* dap,
                         cudaStream_t st) {
  count_launch();
  launch_k(k_ap_init, flat_grid(L), 256, 0, st, L, alpha, dpsi, dap);
}

void launch_xcfc_alpha_out(const LevelView<double>& L, const double* dap, const double* dpsi, double* alpha,
                           cudaStream_t st) {
  count_launch();
  launch_k(k_alpha_out, flat_grid(L), 256, 0, st, L, dap, dpsi, alpha);
}

}  // namespace gmg
