// Warp-level pieces of the Anderson mixing step (mg_accel.cu), shared with
// the persistent batched solve (mg_batch.cu).
#pragma once
#include "mg_internal.h"

namespace gmg {

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
