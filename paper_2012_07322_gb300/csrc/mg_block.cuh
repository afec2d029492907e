// The one-block FP32 correction V-cycle as device code: the phases of
// k_block_vcycle32 (mg_block.cu), callable from any kernel whose block has
// BC_THREADS threads and P.smem bytes of dynamic shared memory.
#pragma once
#include "mg_internal.h"
#include "mg_kernels.cuh"

namespace gmg {

constexpr int BC_THREADS = 512;

// One level with its arrays resolved to shared memory.  The view is copied
// out of the kernel parameters: indexed by a run-time level, the parameter
// would be read through memory on every access of the stencil loops.
struct BcLevel {
  LevelView<float> v;
  float* e[3];
  float* f[3];
  float* r[3];
  const float* k;
};

__device__ __forceinline__ BcLevel bc_level(const BlockCycle32& P, float* sm, int l) {
  const BlockLevel32& B = P.lv[l];
  BcLevel o;
  o.v = B.v;
  // the coefficient tables and c were copied into shared memory when the
  // kernel started: every phase reads them, and from HBM (through an L1
  // mostly given to shared memory) each read is an L2 round trip
  o.v.ti = sm + B.ti_at;
  o.v.tj = sm + B.tj_at;
  for (int c = 0; c < 3; ++c) {
    o.e[c] = sm + B.e[c];
    o.f[c] = sm + B.f32[c];
    o.r[c] = sm + B.r32[c];
  }
  o.k = B.k32 ? sm + B.k_at : nullptr;
  return o;
}

// Copies of every level's coefficient tables and c into shared memory.
inline __device__ void bc_stage_tables(const BlockCycle32& P, float* sm) {
  for (int l = 0; l < P.nl; ++l) {
    const BlockLevel32& B = P.lv[l];
    const int nti = NTI * (B.v.n0 + 2), ntj = NTJ * (B.v.n1 + 2);
    for (int q = threadIdx.x; q < nti; q += blockDim.x) sm[B.ti_at + q] = B.v.ti[q];
    for (int q = threadIdx.x; q < ntj; q += blockDim.x) sm[B.tj_at + q] = B.v.tj[q];
    if (B.k32) {
      const long ng = B.v.sy * (B.v.n2 + 2 * B.v.three);
      for (long q = threadIdx.x; q < ng; q += blockDim.x) sm[B.k_at + q] = B.k32[q];
    }
  }
}

template <typename T>
__device__ __forceinline__ void bc_fill(const LevelView<T>& L, T* u, int comp) {
  const long ng = ghost_count(L);
  for (long g = threadIdx.x; g < ng; g += blockDim.x) fill_one_ghost(L, u, comp, g);
  __syncthreads();
}

// smooth32: nsweeps red-black sweeps (vector: component by component, the
// ghosts of a component refreshed after its pass).
template <int G, bool VEC>
__device__ void bc_smooth(const BcLevel& B, int nsweeps) {
  const LevelView<float> L = B.v;
  const long nh = (long)L.n0 * L.n1 * L.n2 / 2;
  for (int s = 0; s < nsweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      if (!VEC) {
        for (long q = threadIdx.x; q < nh; q += blockDim.x) {
          int i, j, k;
          L.colour_cell(q, colour, i, j, k);
          scalar_update<float, G, EQ_LIN>(L, B.e[0], B.f[0], nullptr, B.k, i, j, k);
        }
        __syncthreads();
      } else {
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
          for (long q = threadIdx.x; q < nh; q += blockDim.x) {
            int i, j, k;
            L.colour_cell(q, colour, i, j, k);
            vec_update<float, G, false>(L, B.e[0], B.e[1], B.e[2], B.f[c], c, i, j, k);
          }
          __syncthreads();
          bc_fill(L, B.e[c], c);
        }
      }
    }
}

template <int G, bool VEC>
__device__ void bc_residual(const BcLevel& B) {
  const LevelView<float> L = B.v;
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    if (!VEC) {
      float Sv;
      B.r[0][p] = scalar_residual_cell<float, G, EQ_LIN>(L, B.e[0], B.f[0], nullptr, B.k, i, j, k, p, Sv);
    } else {
      #pragma unroll
      for (int c = 0; c < 3; ++c) B.r[c][p] = vec_residual_cell<float, G, false>(L, B.e[0], B.e[1], B.e[2], B.f[c], c, i, j, p);
    }
  }
  __syncthreads();
}

// coarse32: the coarsest correction equation in FP64 (right-hand side and
// c converted up, zero start), the solution rounded back into e.
// Shared-memory scratch of the coarsest solves with a dense operator: one
// per translation unit, so that the instantiations of bc_coarse in one
// kernel share it.
union BcCoarseShared {
  struct {
    double uq[BC_CMAT_MAX], fq[BC_CMAT_MAX], kq[BC_CMAT_MAX], dq[BC_CMAT_MAX];
    long pq[BC_CMAT_MAX];
    unsigned char colq[BC_CMAT_MAX];
  } rows;
  double fp[BC_CINV_MAX];
};
static __shared__ BcCoarseShared bc_coarse_sh;

// DENSE_ONLY: the hierarchy is known to carry the dense coarsest operator
// (scalar) or its inverse (vector); the sweeping fallbacks are not compiled.
template <int G, bool VEC, bool DENSE_ONLY = false>
__device__ void bc_coarse(const BlockCycle32& P, const BcLevel& B, double* smd) {
  const LevelView<double>& L = P.c64;
  constexpr int nc = VEC ? 3 : 1;
  const long n = (long)L.n0 * L.n1 * L.n2;
  const long ng = L.sy * (L.n2 + 2 * L.three);
  double* cu[3] = {smd + P.cu[0], smd + P.cu[1], smd + P.cu[2]};
  double* cf[3] = {smd + P.cf[0], smd + P.cf[1], smd + P.cf[2]};
  double* ck = P.ck >= 0 ? smd + P.ck : nullptr;
  #pragma unroll
  for (int c = 0; c < nc; ++c) {
    for (long q = threadIdx.x; q < n; q += blockDim.x) {
      int i, j, k;
      L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      cf[c][p] = (double)B.f[c][p];
      if (!VEC && ck) ck[p] = (double)B.k[p];
    }
    for (long q = threadIdx.x; q < ng; q += blockDim.x) cu[c][q] = 0.0;
  }
  __syncthreads();
  if (!VEC && P.cA) {
    // red-black NGS sweeps with dense rows of the coarsest operator (its
    // boundary rules folded in), K subtracted on the diagonal: row r of a
    // colour is summed by the BC_SPLIT lanes of one group and folded by
    // shuffles; the cells of one colour couple only to the other colour
    constexpr int BC_SPLIT = 8;
    double* const uq = bc_coarse_sh.rows.uq;
    double* const fq = bc_coarse_sh.rows.fq;
    double* const kq = bc_coarse_sh.rows.kq;
    double* const dq = bc_coarse_sh.rows.dq;
    long* const pq = bc_coarse_sh.rows.pq;
    unsigned char* const colq = bc_coarse_sh.rows.colq;
    const int n = P.cn;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int i, j, k;
      L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      const double kv = ck ? ck[p] : 0.0;
      pq[q] = p;
      colq[q] = (unsigned char)((i + j + k) & 1);
      fq[q] = cf[0][p];
      kq[q] = kv;
      uq[q] = 0.0;
      dq[q] = 1.0 / (P.cA[(long)q * n + q] - kv);
    }
    __syncthreads();
    const int sub = threadIdx.x % BC_SPLIT, rows = blockDim.x / BC_SPLIT;
    for (int it = 0; it < P.coarse_sweeps; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        for (int base = 0; base < n; base += rows) {  // the same trip count in every thread
          const int r = base + (int)threadIdx.x / BC_SPLIT;
          const bool on = r < n && colq[r] == colour;
          double x = 0.0;
          if (on)
            for (int col = sub; col < n; col += BC_SPLIT) x += P.cA[(long)col * n + r] * uq[col];
#pragma unroll
          for (int o = BC_SPLIT / 2; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, BC_SPLIT);
          if (on && sub == 0) uq[r] -= (x - kq[r] * uq[r] - fq[r]) * dq[r];
        }
        __syncthreads();
      }
    for (int q = threadIdx.x; q < n; q += blockDim.x) cu[0][pq[q]] = uq[q];
  } else if (!VEC) {
    if constexpr (!DENSE_ONLY) coarse_scalar_body<double, G, EQ_LIN, false>(L, cu[0], cf[0], nullptr, ck,
                                                                            P.coarse_sweeps);
  } else if (P.cinv) {
    // exact solve with the precomputed inverse of the coarsest operator:
    // unknown r = c * cells + q (q the interior flat index)
    double* const fp = bc_coarse_sh.fp;
    const int n = P.cn, cells = n / 3;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      int i, j, k;
      L.cell(r % cells, i, j, k);
      const int c = r / cells;
      fp[r] = (c == 0 ? cf[0] : (c == 1 ? cf[1] : cf[2]))[L.idx(i, j, k)];
    }
    __syncthreads();
    // row r is summed by the BC_SPLIT lanes of one group, each over every
    // BC_SPLIT-th column, and the partial sums folded by shuffles: the
    // dependent FP64 chain of a row is n / BC_SPLIT long instead of n
    constexpr int BC_SPLIT = 8;
    const int sub = threadIdx.x % BC_SPLIT, rows = blockDim.x / BC_SPLIT;
    for (int base = 0; base < n; base += rows) {  // the same trip count in every thread
      const int r = base + (int)threadIdx.x / BC_SPLIT;
      double x = 0.0;
      if (r < n)
        for (int col = sub; col < n; col += BC_SPLIT) x += P.cinv[(long)col * n + r] * fp[col];
#pragma unroll
      for (int o = BC_SPLIT / 2; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, BC_SPLIT);
      if (r < n && sub == 0) {
        int i, j, k;
        L.cell(r % cells, i, j, k);
        const int c = r / cells;
        (c == 0 ? cu[0] : (c == 1 ? cu[1] : cu[2]))[L.idx(i, j, k)] = x;
      }
    }
  } else {
    if constexpr (!DENSE_ONLY) coarse_vec_body<double, G>(L, cu[0], cu[1], cu[2], cf[0], cf[1], cf[2], P.coarse_sweeps);
  }
  __syncthreads();
  #pragma unroll
  for (int c = 0; c < nc; ++c)
    for (long q = threadIdx.x; q < n; q += blockDim.x) {
      int i, j, k;
      L.cell(q, i, j, k);
      const long p = L.idx(i, j, k);
      B.e[c][p] = (float)cu[c][p];
    }
  __syncthreads();
  if (VEC)
    #pragma unroll
    for (int c = 0; c < 3; ++c) bc_fill(B.v, B.e[c], c);
}

// The whole cycle from level l0 of P: its right-hand side in from P.f_in,
// the correction out to P.e_out (ghosts included); sm is the dynamic shared
// memory, smd its FP64 area (sm + P.fp64_at bytes).  No barrier after the
// final stores.  DENSE_ONLY: P carries the dense coarsest operator (cA) or
// its inverse (cinv).
template <int G, bool VEC, bool DENSE_ONLY = false>
__device__ void bc_run(const BlockCycle32& P, float* sm, double* smd) {
  constexpr int nc = VEC ? 3 : 1;
  bc_stage_tables(P, sm);
  {
    // level l0: right-hand side in, zero correction
    const BcLevel B = bc_level(P, sm, 0);
    #pragma unroll
    for (int c = 0; c < nc; ++c)
      for (long q = threadIdx.x; q < P.ng0; q += blockDim.x) {
        B.f[c][q] = P.f_in[c][q];
        B.e[c][q] = 0.0f;
      }
    __syncthreads();
  }
  // down: pre-smooth, residual, restriction into the next level's
  // right-hand side, zero correction there
  for (int l = 0; l + 1 < P.nl; ++l) {
    const BcLevel F = bc_level(P, sm, l), C = bc_level(P, sm, l + 1);
    bc_smooth<G, VEC>(F, P.nu1);
    bc_residual<G, VEC>(F);
    const LevelView<float> Cv = C.v;
    const long nC = (long)Cv.n0 * Cv.n1 * Cv.n2;
    const long ngC = Cv.sy * (Cv.n2 + 2 * Cv.three);
    #pragma unroll
    for (int c = 0; c < nc; ++c) {
      const float* const as[4] = {F.r[c], nullptr, nullptr, nullptr};
      float* const bs[4] = {C.f[c], nullptr, nullptr, nullptr};
      float* const cs[3] = {nullptr, nullptr, nullptr};
      for (long q = threadIdx.x; q < nC; q += blockDim.x) {
        int I, J, K;
        Cv.cell(q, I, J, K);
        restrict_cell(F.v, Cv, 1, as, bs, cs, I, J, K);
      }
      for (long q = threadIdx.x; q < ngC; q += blockDim.x) C.e[c][q] = 0.0f;
    }
    __syncthreads();
  }
  bc_coarse<G, VEC, DENSE_ONLY>(P, bc_level(P, sm, P.nl - 1), smd);
  // up: Kwak prolongation of the correction, post-smooth
  for (int l = P.nl - 2; l >= 0; --l) {
    const BcLevel F = bc_level(P, sm, l), C = bc_level(P, sm, l + 1);
    const LevelView<float> Fv = F.v;
    const long nF = (long)Fv.n0 * Fv.n1 * Fv.n2;
    #pragma unroll
    for (int c = 0; c < nc; ++c)
      for (long q = threadIdx.x; q < nF; q += blockDim.x) {
        int i, j, k;
        Fv.cell(q, i, j, k);
        prolong_cell(Fv, C.v, F.e[c], C.e[c], (const float*)nullptr, VEC ? c : -1, i, j, k);
      }
    __syncthreads();
    if (VEC)
      #pragma unroll
      for (int c = 0; c < 3; ++c) bc_fill(Fv, F.e[c], c);
    bc_smooth<G, VEC>(F, P.nu2);
  }
  // level l0 correction out (ghosts included)
  const BcLevel B = bc_level(P, sm, 0);
  #pragma unroll
  for (int c = 0; c < nc; ++c)
    for (long q = threadIdx.x; q < P.ng0; q += blockDim.x) P.e_out[c][q] = B.e[c][q];
}

}  // namespace gmg
