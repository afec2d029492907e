// Per-cell work of the xCFC sources (Sec. 2.6), shared by the launched
// kernels (mg_xcfc.cu) and the persistent batch kernel (mg_batch.cu).
#pragma once
#include "mg_kernels.cuh"

namespace gmg {

// A~_ij of eq. (Aij) at an interior cell from the ghosted components a, b,
// c of X (physical components; ghosts current): A[0..2] the diagonal,
// A[3] = (0,1), A[4] = (0,2), A[5] = (1,2).
template <int G>
__device__ __forceinline__ void aij_cell(const LevelView<double>& L, const double* __restrict__ a,
                                         const double* __restrict__ b, const double* __restrict__ c, int i,
                                         int j, long p, double A[6]) {
  Stencil<double> s{L, p};
  double E00, E11, E22, E01, E02, E12;
  if (G == CART) {
    E00 = s.d1(a, 0);
    E11 = s.d1(b, 1);
    E22 = s.d1(c, 2);
    E01 = 0.5 * (s.d1(a, 1) + s.d1(b, 0));
    E02 = 0.5 * (s.d1(a, 2) + s.d1(c, 0));
    E12 = 0.5 * (s.d1(b, 2) + s.d1(c, 1));
  } else if (G == CYL) {
    const double iR = L.TI(TI_IX, i);
    E00 = s.d1(a, 0);
    E11 = s.d1(b, 1);
    E22 = iR * (s.d1(c, 2) + a[p]);
    E01 = 0.5 * (s.d1(a, 1) + s.d1(b, 0));
    E02 = 0.5 * (iR * s.d1(a, 2) + s.d1(c, 0) - iR * c[p]);
    E12 = 0.5 * (s.d1(c, 1) + iR * s.d1(b, 2));
  } else {
    const double ir = L.TI(TI_IX, i), ist = L.TJ(TJ_IS, j), cot = L.TJ(TJ_COT, j);
    E00 = s.d1(a, 0);
    E11 = ir * (s.d1(b, 1) + a[p]);
    E22 = ir * (ist * s.d1(c, 2) + a[p] + cot * b[p]);
    E01 = 0.5 * (s.d1(b, 0) - ir * b[p] + ir * s.d1(a, 1));
    E02 = 0.5 * (ir * ist * s.d1(a, 2) + s.d1(c, 0) - ir * c[p]);
    E12 = 0.5 * (ir * s.d1(c, 1) - ir * cot * c[p] + ir * ist * s.d1(b, 2));
  }
  const double div = E00 + E11 + E22;
  A[0] = 2.0 * E00 - (2.0 / 3.0) * div;
  A[1] = 2.0 * E11 - (2.0 / 3.0) * div;
  A[2] = 2.0 * E22 - (2.0 / 3.0) * div;
  A[3] = 2.0 * E01;
  A[4] = 2.0 * E02;
  A[5] = 2.0 * E12;
}

// Shift right-hand side of eq. (beta) at an interior cell:
// 16 pi s S_i + 2 A~_ij (grad s)_j with s = alpha psi^-6 (ghosted, ghosts
// current), S the cell's momentum components.
template <int G>
__device__ __forceinline__ void beta_rhs_cell(const LevelView<double>& L, const double* __restrict__ a,
                                              const double* __restrict__ b, const double* __restrict__ c,
                                              const double* __restrict__ sg, int i, int j, long p,
                                              const double (&S)[3], double (&f)[3]) {
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
  f[0] = k16 * S[0] + 2.0 * (A[0] * g0 + A[3] * g1 + A[4] * g2);
  f[1] = k16 * S[1] + 2.0 * (A[3] * g0 + A[1] * g1 + A[5] * g2);
  f[2] = k16 * S[2] + 2.0 * (A[4] * g0 + A[5] * g1 + A[2] * g2);
}

}  // namespace gmg
