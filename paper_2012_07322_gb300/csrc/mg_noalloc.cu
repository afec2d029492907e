// Divergence diagnostics of a Cartesian field without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs between the steps of
// a host framework which owns all device memory and forbids allocations in
// its time loop, or code whose allocations would synchronise the device
// and break the overlap of its streams.  They cannot create a hierarchy
// (mg_create_hierarchy allocates), yet still want the divergence monitor.
// This file gives them mg_divb_norms_noalloc: the same two kernels as the
// divergence pipeline of mg_clean_divB (central divergence into scratch,
// then its max and the per-block sums of div^2), with the scratch in a
// file-scope __device__ array instead of the hierarchy's arena.
//
// The array holds MG_NOALLOC_MAX_CELLS divergence values plus the block
// partial sums and the max word (about 16 MiB); every GPU that loads the
// library keeps it until the process exits.  All calls share it: calls
// whose work overlaps on the GPU race with each other.
#include <cmath>
#include <cstring>
#include <mutex>

#include "mg.h"
#include "mg_internal.h"
#include "mg_kernels.cuh"

namespace {

constexpr int NOALLOC_BLOCKS = 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;
// [0, MAX_CELLS): divergence; then NOALLOC_BLOCKS partial sums; then the max
// word (bit pattern of a non-negative double).
constexpr long SCRATCH_WORDS = (long)MG_NOALLOC_MAX_CELLS + NOALLOC_BLOCKS + 32;

}  // namespace

static __device__ __align__(256) double g_divb_scratch[SCRATCH_WORDS];

namespace {

std::mutex g_setup_mutex;
double* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};

// Central divergence with zero-gradient (copied) ghosts into scratch.
__global__ void k_noalloc_div(int n0, int n1, int n2, int three, double c0, double c1, double c2,
                              const double* __restrict__ B0, const double* __restrict__ B1,
                              const double* __restrict__ B2, double* __restrict__ div) {
  gmg::pdl_entry();
  const long n = (long)n0 * n1 * n2;
  const long s1 = n0, s2 = (long)n0 * n1;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int i = (int)(q % n0), j = (int)((q / n0) % n1), k = (int)(q / s2);
    double d = (B0[i < n0 - 1 ? q + 1 : q] - B0[i > 0 ? q - 1 : q]) * c0 +
               (B1[j < n1 - 1 ? q + s1 : q] - B1[j > 0 ? q - s1 : q]) * c1;
    if (three) d += (B2[k < n2 - 1 ? q + s2 : q] - B2[k > 0 ? q - s2 : q]) * c2;
    div[q] = d;
  }
}

// Per-block sums of div^2 into part[], max |div| into *maxw (atomic).
__global__ void k_noalloc_norms(long n, const double* __restrict__ div, double* __restrict__ part,
                                unsigned long long* maxw) {
  gmg::pdl_entry();
  __shared__ double sm[32];
  double s = 0.0;
  double m[1] = {0.0};
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const double d = div[q];
    s += d * d;
    m[0] = fmax(m[0], fabs(d));
    if (d != d) m[0] = INFINITY;
  }
  s = gmg::warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
  __syncthreads();
  gmg::block_max_atomic<1>(m, maxw);
}

// Device address of the scratch array on the current device, looked up
// once per device (cudaGetSymbolAddress with that device current).
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return MG_ERR_CUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MG_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_divb_scratch);
    if (e != cudaSuccess || !p) return MG_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MG_OK;
}

}  // namespace

extern "C" int mg_divb_norms_noalloc(int ndim, const int n[3], const double lo[3], const double hi[3],
                                     const double* B[3], void* cuda_stream, double* max_div, double* l2_div) {
  using gmg::set_last_error;
  if (ndim != 2 && ndim != 3) return set_last_error(MG_ERR_INVALID, "ndim must be 2 or 3");
  if (!n || !lo || !hi || !B || !max_div || !l2_div) return set_last_error(MG_ERR_INVALID, "null argument");
  long cells = 1;
  for (int d = 0; d < ndim; ++d) {
    if (n[d] < 1 || !(hi[d] > lo[d])) return set_last_error(MG_ERR_INVALID, "need n >= 1 and lo < hi");
    if (!B[d]) return set_last_error(MG_ERR_INVALID, "null B component");
    cells *= n[d];
    if (cells > (long)MG_NOALLOC_MAX_CELLS)
      return set_last_error(MG_ERR_INVALID,
                            "grid larger than MG_NOALLOC_MAX_CELLS (2097152 cells), the size of the static "
                            "scratch of the allocation-free entry point");
  }
  // an error left by earlier, unrelated work of the caller must not be
  // reported as this call's: drop it (launch errors are checked below)
  (void)cudaGetLastError();
  double* scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st) return set_last_error(st, "looking up the device address of the static scratch failed");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n0 = n[0], n1 = n[1], n2 = ndim == 3 ? n[2] : 1;
  double* div = scratch;
  double* part = scratch + MG_NOALLOC_MAX_CELLS;
  unsigned long long* maxw = reinterpret_cast<unsigned long long*>(part + NOALLOC_BLOCKS);
  // the max word keeps the previous call's value: clear it
  if (cudaMemsetAsync(maxw, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return set_last_error(MG_ERR_CUDA, "clearing the max word failed");
  const double c0 = 0.5 / ((hi[0] - lo[0]) / n0), c1 = 0.5 / ((hi[1] - lo[1]) / n1);
  const double c2 = ndim == 3 ? 0.5 / ((hi[2] - lo[2]) / n2) : 0.0;
  long g = (cells + 255) / 256;
  if (g > NOALLOC_BLOCKS) g = NOALLOC_BLOCKS;
  gmg::count_launch(2);
  gmg::launch_k(k_noalloc_div, (unsigned)g, 256, 0, s, n0, n1, n2, ndim == 3, c0, c1, c2, B[0], B[1],
                                             ndim == 3 ? B[2] : B[0], div);
  gmg::launch_k(k_noalloc_norms, NOALLOC_BLOCKS, 256, 0, s, cells, div, part, maxw);
  if (cudaGetLastError() != cudaSuccess) return set_last_error(MG_ERR_CUDA, "launching the divergence kernels failed");
  double hpart[NOALLOC_BLOCKS];
  unsigned long long hmax = 0;
  if (cudaMemcpyAsync(hpart, part, sizeof(hpart), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&hmax, maxw, sizeof(hmax), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return set_last_error(MG_ERR_CUDA, "divergence kernels or read-back failed");
  double sum = 0.0;
  for (int b = 0; b < NOALLOC_BLOCKS; ++b) sum += hpart[b];
  double mx;
  static_assert(sizeof(mx) == sizeof(hmax), "word size");
  memcpy(&mx, &hmax, sizeof(mx));
  *max_div = mx;
  *l2_div = sqrt(sum / (double)cells);
  return MG_OK;
}
