// Host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include "mg_dev.cuh"

struct mg_hierarchy;

namespace gmg {

// Record a message for mg_last_error on the calling thread; returns status.
int set_last_error(int status, const char* msg);

// Move a hierarchy's work to another stream (serving workers share cached
// hierarchies; captured graphs are stream-independent).
void hier_set_stream(mg_hierarchy* h, cudaStream_t st);

// Count of kernel launches issued by the library (all hierarchies).
void count_launch(int n = 1);
unsigned long long launch_count();

template <typename T>
void launch_smooth_scalar(const LevelView<T>& L, int kind, T* u, const T* f, const T* s0, const T* s1,
                          int colour, cudaStream_t st);
template <typename T>
void launch_fill_ghosts(const LevelView<T>& L, T* u, int comp, cudaStream_t st);
// One fused red-black sweep (Cartesian 3D linear scalar equations, levels of
// at least one tile); returns false when it does not apply.
template <typename T>
bool launch_sweep_fused(const LevelView<T>& L, T* u, const T* f, const T* c, cudaStream_t st);
template <typename T>
void init_fused_sweep_attributes();
template <typename T>
inline bool fused_sweep_applies(const LevelView<T>& L) {
  return L.geom == CART && L.three && L.n0 >= 32 && L.n1 >= 8 && L.n2 >= 8;
}
template <typename T>
void launch_smooth_vec(const LevelView<T>& L, T* V[3], const T* f, int comp, int colour, cudaStream_t st);
template <typename T>
void launch_residual_scalar(const LevelView<T>& L, int kind, const T* u, const T* f, const T* s0,
                            const T* s1, T* r, unsigned long long* red, int weighted, cudaStream_t st);
template <typename T>
void launch_residual_vec(const LevelView<T>& L, T* const V[3], const T* const f[3], T* const r[3],
                         unsigned long long* red, int weighted, cudaStream_t st);
template <typename T>
void launch_apply_scalar(const LevelView<T>& L, int kind, const T* u, const T* s0, const T* s1, T* out,
                         int add, cudaStream_t st);
template <typename T>
void launch_apply_vec(const LevelView<T>& L, T* const V[3], T* const out[3], int add, cudaStream_t st);
template <typename T>
void launch_restrict(const LevelView<T>& F, const LevelView<T>& C, int nf, const T* const a[4],
                     T* const b[4], T* const copy[3], cudaStream_t st);
template <typename T>
void launch_prolong(const LevelView<T>& F, const LevelView<T>& C, T* u, const T* uH, const T* uhH, int comp,
                    cudaStream_t st);
template <typename T>
void launch_coarse_scalar(const LevelView<T>& L, int kind, T* u, const T* f, const T* s0, const T* s1,
                          int max_sweeps, cudaStream_t st);
template <typename T>
void launch_coarse_vec(const LevelView<T>& L, T* V[3], const T* const f[3], int max_sweeps, cudaStream_t st);
template <typename T>
void launch_sub_mean(const LevelView<T>& L, T* u, double* part, int nparts, cudaStream_t st);
template <typename A, typename B>
void launch_copy_in(const LevelView<B>& L, const A* src, B* dst, A shift, cudaStream_t st);
template <typename A, typename B>
void launch_copy_out(const LevelView<A>& L, const A* src, B* dst, A shift, cudaStream_t st);
template <typename A, typename B>
void launch_convert(const LevelView<A>& L, const A* src, B* dst, cudaStream_t st);
template <typename T>
void launch_add_correction(const LevelView<double>& L, double* u, const T* e, cudaStream_t st);

// xCFC and divergence-cleaning pointwise kernels (mg_xcfc.cu).
void launch_xcfc_a2(const LevelView<double>& L, double* const X[3], double* A2, cudaStream_t st);
void launch_xcfc_alpha_coef(const LevelView<double>& L, const double* U, const double* S, const double* A2,
                            const double* dpsi, double* c, cudaStream_t st);
void launch_xcfc_beta_rhs(const LevelView<double>& L, double* const X[3], const double* dpsi,
                          const double* dap, double* sg, double* const Si[3], double* const f[3],
                          cudaStream_t st);
void launch_scale_into(const LevelView<double>& L, const double* src, double a, double* dst, cudaStream_t st);
void launch_div_central(const LevelView<double>& L, double* const B[3], double* div, double* part, int nparts,
                        cudaStream_t st);
void launch_div_norms(const LevelView<double>& L, const double* div, double* part, int nparts,
                      unsigned long long* red, cudaStream_t st);
void launch_sub_mean_into(const LevelView<double>& L, const double* div, const double* part, int nparts,
                          double* b, cudaStream_t st);
void launch_grad_update(const LevelView<double>& L, const double* phi, double* const B[3], cudaStream_t st);
void launch_psi_linearisation(const LevelView<double>& L, const double* u, const double* U, const double* A2,
                              float* K, cudaStream_t st);
void launch_xcfc_ap_init(const LevelView<double>& L, const double* alpha, const double* dpsi, double* dap,
                         cudaStream_t st);
void launch_xcfc_alpha_out(const LevelView<double>& L, const double* dap, const double* dpsi, double* alpha,
                           cudaStream_t st);

// Anderson mixing (mg_accel.cu): live ring slots of the difference columns
// in age order, with their mixing weights.
constexpr int AA_MAX = 16;
constexpr int AA_BLOCKS = 304;     // 2 x 152 SMs
constexpr int AA_DOT_X = 64;       // threads per column in the dot-product kernel
struct AACols {
  int n;
  int slot[AA_MAX];
  double gamma[AA_MAX];
};
void launch_aa_update(const LevelView<double>& L, int ncomp, long stride, double* const g[3], const double* x,
                      double* fprev, double* gprev, double* dF, double* dG, int first, cudaStream_t st);
void launch_aa_dots(const LevelView<double>& L, int ncomp, long stride, const double* f, const double* dF,
                    const AACols& cols, int newcol, double* part, cudaStream_t st);
void launch_aa_combine(const LevelView<double>& L, int ncomp, long stride, double* const u[3], const double* dG,
                       const AACols& cols, cudaStream_t st);

}  // namespace gmg
