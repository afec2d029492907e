// The FP32 correction V-cycle (Sec. 2.7.2 / 2.7.3 in correction form, the
// inner cycle of the mixed-precision defect correction) over the coarse
// levels of a hierarchy in ONE thread block.  Below a few thousand cells a
// level's kernels are too small to fill the GPU and each launch costs more
// than its work; inside one block the same phases are separated by block
// barriers instead of kernel boundaries, and every level lives in shared
// memory (the same ghosted layout as in HBM).  Every phase applies the
// per-cell functions the grid-wide kernels apply, in the same order, so the
// result is identical to the launched cycle.
#include "mg_internal.h"
#include "mg_kernels.cuh"
#include "mg_block.cuh"

namespace gmg {

template <int G, bool VEC>
__global__ void __launch_bounds__(BC_THREADS) k_block_vcycle32(const __grid_constant__ BlockCycle32 P) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  double* smd = reinterpret_cast<double*>(smem_raw + P.fp64_at);
  bc_run<G, VEC>(P, sm, smd);
}

// Column col of the coarsest vector operator (lap V + 1/3 grad div V with
// the level's ghost rules): the operator applied to unit field col, stored
// in A[col * n + r], unknown r = c * cells + q.  One block per column;
// scratch holds n fields of 3 ghosted components.
template <int G>
__global__ void k_coarse_assemble_vec(LevelView<double> L, double* __restrict__ scratch, double* __restrict__ A,
                                      int n) {
  pdl_entry();
  const int col = blockIdx.x, cells = n / 3;
  const long ng = L.sy * (L.n2 + 2 * L.three);
  double* U[3];
  for (int c = 0; c < 3; ++c) U[c] = scratch + ((long)col * 3 + c) * ng;
  for (long q = threadIdx.x; q < 3 * ng; q += blockDim.x) U[0][q] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int i, j, k;
    L.cell(col % cells, i, j, k);
    U[col / cells][L.idx(i, j, k)] = 1.0;
  }
  __syncthreads();
  const long ngh = ghost_count(L);
  for (int c = 0; c < 3; ++c)
    for (long g = threadIdx.x; g < ngh; g += blockDim.x) fill_one_ghost(L, U[c], c, g);
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    int i, j, k;
    L.cell(r % cells, i, j, k);
    double D;
    A[(long)col * n + r] = vec_op<double, G>(L, U[0], U[1], U[2], r / cells, i, j, L.idx(i, j, k), D);
  }
}

// Column col of the coarsest scalar operator: lap_scalar (its boundary rule
// folded in) applied to unit field col, into A[col * n + r].  One block per
// column; scratch holds n ghosted fields.
template <int G>
__global__ void k_coarse_assemble_scalar(LevelView<double> L, double* __restrict__ scratch, double* __restrict__ A,
                                         int n) {
  pdl_entry();
  const int col = blockIdx.x;
  const long ng = L.sy * (L.n2 + 2 * L.three);
  double* U = scratch + (long)col * ng;
  for (long q = threadIdx.x; q < ng; q += blockDim.x) U[q] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int i, j, k;
    L.cell(col, i, j, k);
    U[L.idx(i, j, k)] = 1.0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    int i, j, k;
    L.cell(r, i, j, k);
    double D;
    A[(long)col * n + r] = lap_scalar<double, G>(L, U, i, j, k, L.idx(i, j, k), D);
  }
}

void launch_coarse_assemble_scalar(const LevelView<double>& L, double* scratch, double* A, int n, cudaStream_t st) {
  count_launch();
  if (L.geom == CART)
    launch_k(k_coarse_assemble_scalar<CART>, n, 256, 0, st, L, scratch, A, n);
  else if (L.geom == CYL)
    launch_k(k_coarse_assemble_scalar<CYL>, n, 256, 0, st, L, scratch, A, n);
  else
    launch_k(k_coarse_assemble_scalar<SPH>, n, 256, 0, st, L, scratch, A, n);
}

void launch_coarse_assemble_vec(const LevelView<double>& L, double* scratch, double* A, int n, cudaStream_t st) {
  count_launch();
  if (L.geom == CART)
    launch_k(k_coarse_assemble_vec<CART>, n, 256, 0, st, L, scratch, A, n);
  else if (L.geom == CYL)
    launch_k(k_coarse_assemble_vec<CYL>, n, 256, 0, st, L, scratch, A, n);
  else
    launch_k(k_coarse_assemble_vec<SPH>, n, 256, 0, st, L, scratch, A, n);
}

template <int G>
static void launch_g(const BlockCycle32& P, cudaStream_t st) {
  if (P.vec)
    launch_k(k_block_vcycle32<G, true>, 1, BC_THREADS, P.smem, st, P);
  else
    launch_k(k_block_vcycle32<G, false>, 1, BC_THREADS, P.smem, st, P);
}

void launch_block_vcycle32(const BlockCycle32& P, int geom, cudaStream_t st) {
  count_launch();
  if (geom == CART)
    launch_g<CART>(P, st);
  else if (geom == CYL)
    launch_g<CYL>(P, st);
  else
    launch_g<SPH>(P, st);
}

template <int G>
static void set_attrs() {
  cudaFuncSetAttribute(k_block_vcycle32<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BC_SMEM_MAX);
  cudaFuncSetAttribute(k_block_vcycle32<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BC_SMEM_MAX);
}

void init_block_cycle_attributes() {
  set_attrs<CART>();
  set_attrs<CYL>();
  set_attrs<SPH>();
}

}  // namespace gmg
