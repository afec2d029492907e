// Pieces of the Anderson mixing step (mg_accel.cu) shared with the
// persistent batched solve (mg_batch.cu): the grouped loads and stores of
// its streams, the warp sums and the warp Cholesky solve.
#pragma once
#include "mg_internal.h"
#include "mg_kernels.cuh"

namespace gmg {

// G consecutive interior cells of a row (G = 4 when n0 >= 4, else 1).
template <int G>
__device__ __forceinline__ long aa_pos(const LevelView<double>& L, long q) {
  if (G == 4) return group4(L, q);
  return interior_p(L, q);
}
// Loads and stores of the mixing streams are marked evict-first: every
// array is touched once per cycle, and the multigrid cycle's working set
// (which fits the L2 at the bench sizes) should stay cached across them.
template <int G, typename T>
__device__ __forceinline__ void aa_ld(const T* p, T (&v)[G]) {
  if constexpr (G == 1) {
    v[0] = __ldcs(p);
  } else if constexpr (sizeof(T) == 4) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  } else {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p)), b = __ldcs(reinterpret_cast<const double2*>(p + 2));
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
}
template <int G, typename T>
__device__ __forceinline__ void aa_st(T* p, const T (&v)[G]) {
  if constexpr (G == 1) {
    __stcs(p, v[0]);
  } else if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2*>(p + 2), make_double2(v[2], v[3]));
  }
}

// u itself stays cached (the residual reads it next).
template <int G>
__device__ __forceinline__ void aa_ld_u(const double* p, double (&v)[G]) {
  if constexpr (G == 1) {
    v[0] = *p;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
}
template <int G>
__device__ __forceinline__ void aa_st_u(double* p, const double (&v)[G]) {
  if constexpr (G == 1) {
    *p = v[0];
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// Sum over the warp of 32 values per lane; afterwards lane l holds the sum
// of value l (31 exchanges instead of 32 x 5).
template <typename T>
__device__ __forceinline__ T warp_sum32(T (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = lane & s;
#pragma unroll
    for (int q = 0; q < s; ++q) {
      const T send = upper ? v[q] : v[q + s];
      const T keep = upper ? v[q + s] : v[q];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// Relative shift of the Gram system scaled to unit maximum diagonal:
// 1e-12 in FP64; in mixed precision the system is solved in FP32 (its dot
// products are FP32 sums already) and the shift is about one FP32 ulp of
// the unit diagonal (1e-6 and 1e-5 cost 3-5 % more cycles on the
// 128 x 64 x 64 xCFC solve).
// FP64 is long-latency on this GPU (a dependent FMA takes ~64 cycles, a
// reciprocal square root ~430): the 16-step factorisation costs tens of
// microseconds in FP64 and a few in FP32 registers.
template <typename T>
constexpr T AA_SHIFT = T(1e-12);
template <>
constexpr float AA_SHIFT<float> = 1e-7f;

// Cholesky solve of the n x n system held by one warp, lane t owning row t
// (entries k < n) and right-hand side z; rows and columns n .. AA_MAX - 1
// are the identity, so every loop runs its full static length.  On return
// lane t holds y_t (0 beyond n); false for a non-positive pivot.
__device__ __forceinline__ bool chol_warp_f32(float (&row)[AA_MAX], float& z, int t) {
  __shared__ float Ls[AA_MAX][AA_MAX + 1];
  bool ok = true;
  float idt = 1.0f;
#pragma unroll
  for (int j = 0; j < AA_MAX; ++j) {
    const float piv = __shfl_sync(0xffffffffu, row[j], j);
    ok = ok && piv > 0.0f;
    const float id = rsqrtf(piv);
    if (t == j) {
      row[j] = piv * id;
      z *= id;
      idt = id;
    } else if (t > j) {
      row[j] *= id;  // L[t][j]
    }
    const float zj = __shfl_sync(0xffffffffu, z, j);
#pragma unroll
    for (int k = j + 1; k < AA_MAX; ++k) {
      const float lkj = __shfl_sync(0xffffffffu, row[j], k);  // L[k][j]
      if (t >= k) row[k] -= row[j] * lkj;
    }
    if (t > j) z -= row[j] * zj;
  }
  // back substitution L^T y = z with L transposed through shared memory:
  // lane r needs L[i][r], held by lane i
  if (t < AA_MAX)
#pragma unroll
    for (int k = 0; k < AA_MAX; ++k) Ls[t][k] = row[k];
  __syncwarp();
#pragma unroll
  for (int i = AA_MAX - 1; i >= 0; --i) {
    const float yi = __shfl_sync(0xffffffffu, z * idt, i);
    if (t == i) z = yi;
    if (t < i) z -= Ls[i][t] * yi;
  }
  return ok;
}

}  // namespace gmg
