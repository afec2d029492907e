// Two-level composite grid (block AMR of ratio 2) for the scalar equations:
// a refined patch over a box of base cells, solved by FAS across the patch
// and the base hierarchy (the paper's block tree, Sec. 2.8, held on one
// device as one box of whole blocks).  Readings of the interface (the
// paper's multigrid on AMR grids lives in the library it cites):
//   - coarse-fine ghosts of the patch: the base solution interpolated to the
//     ghost's tangential position (second-order centred differences of the
//     uncovered base cells around the parent, offsets +-1/4 base spacing,
//     the cross term in 3D), then quadratic in the normal direction through
//     the two patch cells inward: g = 8/15 u~ + 2/3 u_1 - 1/5 u_2;
//   - the uncovered base cell next to the patch takes, for its face to the
//     patch, the sum of the fine fluxes through that face (area x
//     difference, in the pseudo-volume form of the printed operators);
//   - FAS: the patch residual and solution restricted (volume-weighted) to
//     the cells the patch covers, f = L_H(R u) + R r there and f0 minus the
//     flux correction on uncovered cells, one base V-cycle, the Kwak
//     prolongation of the base change onto the patch.
#include "mg_internal.h"
#include "mg_kernels.cuh"

namespace gmg {

static inline unsigned cdiv_u(long a, long b) { return (unsigned)((a + b - 1) / b); }

// Pseudo volume of a cell and area of its face on side sd along d (the
// flux form of the printed operators multiplied by the cell measure).
__device__ __forceinline__ double amr_volume(const LevelView<double>& L, int i, int j) {
  double v = L.h0 * L.h1 * (L.three ? L.h2 : 1.0);
  if (L.geom == CYL) v *= L.xc0(i);
  if (L.geom == SPH) {
    const double r = L.xc0(i);
    v *= r * r * sin(L.xc1(j));
  }
  return v;
}
__device__ __forceinline__ double amr_area(const LevelView<double>& L, int d, int sd, int i, int j) {
  const double h2 = L.three ? L.h2 : 1.0;
  const double hd = d == 0 ? L.h0 : (d == 1 ? L.h1 : L.h2);
  if (L.geom == CART) return L.h0 * L.h1 * h2 / hd;
  if (L.geom == CYL) {
    if (d == 0) return (L.lo0 + (sd > 0 ? i + 1 : i) * L.h0) * L.h1 * h2;
    if (d == 1) return L.xc0(i) * L.h0 * h2;
    return L.h0 * L.h1 / L.xc0(i);
  }
  if (d == 0) {
    const double rf = L.lo0 + (sd > 0 ? i + 1 : i) * L.h0;
    return rf * rf * sin(L.xc1(j)) * L.h1 * h2;
  }
  if (d == 1) {
    // sin at the face, exactly zero on the poles
    const int jf = sd > 0 ? j + 1 : j;
    const double s = (jf == 0 || jf == L.n1) && L.lo1 == 0.0 ? 0.0 : sin(L.lo1 + jf * L.h1);
    return s * L.h0 * h2;
  }
  return L.h0 * L.h1 / sin(L.xc1(j));
}

// ------------------------------------------------------ coarse-fine ghosts

// Face (d, side) of the patch is a coarse-fine interface when bit
// (2 d + (side > 0)) of cf is set.
__device__ __forceinline__ bool amr_cf(int cf, int d, int side) { return (cf >> (2 * d + (side > 0))) & 1; }

// The per-dimension quantities of these kernels are kept in scalars chosen
// by dimension, never in arrays indexed at run time: indexing the box's
// arrays or small local arrays with a run-time dimension gave wrong values
// (a coordinate that stayed 0) in an earlier form of these kernels.
// Base solution ub (ghosts filled) at the tangential position of a patch
// ghost whose parent is base cell (I, J, K), normal dimension d, offsets
// t0, t1, t2 (+-1/4 base spacing along the tangential dimensions, 0 along
// d): second-order centred differences per tangential dimension and, in 3D,
// the cross term.
__device__ double amr_tangential(const LevelView<double>& B, const double* __restrict__ ub, int d, int I, int J,
                                 int K, double t0, double t1, double t2) {
  const double uc = ub[B.idx(I, J, K)];
  double v = uc;
  // dimension 0
  if (d != 0) {
    const double up = ub[B.idx(I + 1, J, K)], um = ub[B.idx(I - 1, J, K)];
    v += t0 * 0.5 * (up - um) + 0.5 * t0 * t0 * (up - 2.0 * uc + um);
  }
  if (d != 1) {
    const double up = ub[B.idx(I, J + 1, K)], um = ub[B.idx(I, J - 1, K)];
    v += t1 * 0.5 * (up - um) + 0.5 * t1 * t1 * (up - 2.0 * uc + um);
  }
  if (B.three && d != 2) {
    const double up = ub[B.idx(I, J, K + 1)], um = ub[B.idx(I, J, K - 1)];
    v += t2 * 0.5 * (up - um) + 0.5 * t2 * t2 * (up - 2.0 * uc + um);
  }
  if (B.three) {
    // cross term of the two tangential dimensions
    double mix, ta, tb;
    if (d == 0) {
      mix = ub[B.idx(I, J + 1, K + 1)] - ub[B.idx(I, J + 1, K - 1)] - ub[B.idx(I, J - 1, K + 1)] +
            ub[B.idx(I, J - 1, K - 1)];
      ta = t1, tb = t2;
    } else if (d == 1) {
      mix = ub[B.idx(I + 1, J, K + 1)] - ub[B.idx(I + 1, J, K - 1)] - ub[B.idx(I - 1, J, K + 1)] +
            ub[B.idx(I - 1, J, K - 1)];
      ta = t0, tb = t2;
    } else {
      mix = ub[B.idx(I + 1, J + 1, K)] - ub[B.idx(I + 1, J - 1, K)] - ub[B.idx(I - 1, J + 1, K)] +
            ub[B.idx(I - 1, J - 1, K)];
      ta = t0, tb = t1;
    }
    v += ta * tb * 0.25 * mix;
  }
  return v;
}

// Face (d, side) of a thread g of the interface kernels: faces enumerated
// d = 0, 1, 2, low then high side; fsz(d) cells per face; on return g is
// the thread's index within its face.  False past the last face.
__device__ __forceinline__ bool amr_face(long& g, int nd, long f0, long f1, long f2, int& d, int& side) {
  for (d = 0; d < nd; ++d) {
    const long fsz = d == 0 ? f0 : (d == 1 ? f1 : f2);
    for (side = -1; side <= 1; side += 2) {
      if (g < fsz) return true;
      g -= fsz;
    }
  }
  return false;
}

// One thread per coarse-fine ghost of the patch, faces enumerated as in
// amr_face, the cells of a face dimension-0 fastest over the patch's
// tangential extent.
__global__ void k_amr_cf_ghosts(LevelView<double> Pv, LevelView<double> B, AmrBox box, double* __restrict__ up,
                                const double* __restrict__ ub) {
  pdl_entry();
  const int nd = Pv.three ? 3 : 2;
  const long n0 = Pv.n0, n1 = Pv.n1, n2 = Pv.three ? Pv.n2 : 1;
  long g = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int d, side;
  if (!amr_face(g, nd, n1 * n2, n0 * n2, n0 * n1, d, side)) return;
  if (!amr_cf(box.cf, d, side)) return;
  // fine indices (i, j, k) of the patch cell next to the ghost
  int i, j, k;
  if (d == 0) {
    j = (int)(g % n1), k = (int)(g / n1);
    i = side < 0 ? 0 : (int)n0 - 1;
  } else if (d == 1) {
    i = (int)(g % n0), k = (int)(g / n0);
    j = side < 0 ? 0 : (int)n1 - 1;
  } else {
    i = (int)(g % n0), j = (int)(g / n0);
    k = side < 0 ? 0 : (int)n2 - 1;
  }
  const int a0 = box.a[0], a1 = box.a[1], a2 = box.a[2], b0 = box.b[0], b1 = box.b[1], b2 = box.b[2];
  // parent base cell and tangential offsets
  int I = a0 + (i >> 1), J = a1 + (j >> 1), K = Pv.three ? a2 + (k >> 1) : 0;
  double t0 = (i & 1) ? 0.25 : -0.25, t1 = (j & 1) ? 0.25 : -0.25, t2 = (k & 1) ? 0.25 : -0.25;
  const int s = side < 0 ? -1 : 1;
  if (d == 0) {
    I = side < 0 ? a0 - 1 : b0;
    t0 = 0.0;
  } else if (d == 1) {
    J = side < 0 ? a1 - 1 : b1;
    t1 = 0.0;
  } else {
    K = side < 0 ? a2 - 1 : b2;
    t2 = 0.0;
  }
  if (!Pv.three) t2 = 0.0;
  const double ut = amr_tangential(B, ub, d, I, J, K, t0, t1, t2);
  // the ghost, the first and the second patch cell inward along d
  const long pg = Pv.idx(i + (d == 0) * s, j + (d == 1) * s, k + (d == 2) * s);
  const long p1 = Pv.idx(i, j, k);
  const long p2 = Pv.idx(i - (d == 0) * s, j - (d == 1) * s, k - (d == 2) * s);
  up[pg] = (8.0 / 15.0) * ut + (2.0 / 3.0) * up[p1] - (1.0 / 5.0) * up[p2];
}

// ------------------------------------------------------------ patch level

// Scalar operator of the patch with every neighbour read from memory (the
// ghosts are materialised: boundary rules or coarse-fine values); D gets
// dL/du at the cell, ghosts held fixed.
template <int G, int KIND>
__device__ __forceinline__ double amr_op(const LevelView<double>& L, const double* __restrict__ u,
                                         const double* __restrict__ s0, const double* __restrict__ s1, int i, int j,
                                         long p, double& D) {
  double Lu = lap_ghosted<double, G>(L, u, i, j, p, D);
  if (KIND == EQ_PSI) {
    const double ip = 1.0 / (1.0 + u[p]);
    const double ip2 = ip * ip;
    const double ip7 = ip2 * ip2 * ip2 * ip;
    const double a = 2.0 * PI_D * s0[p], b = s1[p];
    Lu += a * ip + 0.125 * b * ip7;
    D -= a * ip2 + 0.875 * b * ip7 * ip;
  } else if (s1) {
    Lu -= s1[p] * u[p];
    D -= s1[p];
  }
  return Lu;
}

template <int G, int KIND>
__global__ void k_amr_smooth(LevelView<double> L, double* __restrict__ u, const double* __restrict__ f,
                             const double* __restrict__ s0, const double* __restrict__ s1, int colour) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (2 * t >= L.n0 || j >= L.n1 || k >= L.n2) return;
  const int i = 2 * t + ((j + k + colour) & 1);
  const long p = L.idx(i, j, k);
  double D;
  const double Lu = amr_op<G, KIND>(L, u, s0, s1, i, j, p, D);
  u[p] = u[p] - (Lu - f[p]) / D;
}

// r = f - L(u) on the patch (apply: r = L(u)); red (nullable) gets max |r|
// (slot 0), max |w r| (slot 1) and max |w S| (slot 2), w = r^2 sin(theta) /
// R / 1, S the source as the paper writes the right-hand side.
template <int G, int KIND>
__global__ void k_amr_patch_resid(LevelView<double> L, const double* __restrict__ u, const double* __restrict__ f,
                                  const double* __restrict__ s0, const double* __restrict__ s1,
                                  double* __restrict__ r, unsigned long long* red, int apply) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  unsigned long long m[3] = {0ULL, 0ULL, 0ULL};
  if (i < L.n0 && j < L.n1 && k < L.n2) {
    const long p = L.idx(i, j, k);
    double D;
    const double Lu = amr_op<G, KIND>(L, u, s0, s1, i, j, p, D);
    const double fv = f ? f[p] : 0.0;
    const double rv = fv - Lu;
    if (r) r[p] = apply ? Lu : rv;
    double S;
    if (KIND == EQ_PSI) {
      const double ip = 1.0 / (1.0 + u[p]);
      const double ip2 = ip * ip;
      S = -2.0 * PI_D * s0[p] * ip - 0.125 * s1[p] * (ip2 * ip2 * ip2 * ip);
    } else {
      S = fv + (s1 ? s1[p] * u[p] : 0.0);
    }
    const double w = norm_weight(L, i, j);
    m[0] = abs_bits(rv);
    m[1] = abs_bits(w * rv);
    m[2] = abs_bits(w * S);
  }
  if (red) block_max_bits<3>(m, red);
}

// Covered base cells: the volume-weighted restriction of the patch's u and
// r (Sec. 2.7.3) into ub and rr.
__global__ void k_amr_restrict(LevelView<double> Pv, LevelView<double> B, AmrBox box, const double* __restrict__ up,
                               const double* __restrict__ rp, double* __restrict__ ub, double* __restrict__ rr) {
  pdl_entry();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  const int m0 = box.b[0] - box.a[0], m1 = box.b[1] - box.a[1], m2 = box.b[2] - box.a[2];
  if (I >= m0 || J >= m1 || K >= m2) return;
  const LevelView<double> C = B;
  // the patch-local coarse cell (I, J, K) is base cell a + (I, J, K)
  const double* as[4] = {up, rp, nullptr, nullptr};
  double su = 0.0, sr = 0.0, ws = 0.0;
  const int nk = Pv.three ? 2 : 1;
  for (int dk = 0; dk < nk; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const double w = Pv.TI(TI_VW, 2 * I + di) * Pv.TJ(TJ_VW, 2 * J + dj);
        const long q = Pv.idx(2 * I + di, 2 * J + dj, Pv.three ? 2 * K + dk : 0);
        su += w * as[0][q];
        sr += w * as[1][q];
        ws += w;
      }
  const long pb = C.idx(box.a[0] + I, box.a[1] + J, Pv.three ? box.a[2] + K : 0);
  ub[pb] = su / ws;
  rr[pb] = sr / ws;
}

// The composite operator minus the base operator at the uncovered base cells
// next to the patch (corr zero elsewhere; zeroed before): one thread per
// coarse cell of a coarse-fine face, faces enumerated as in amr_face over
// the box's tangential extent.
__global__ void k_amr_flux_corr(LevelView<double> Pv, LevelView<double> B, AmrBox box, const double* __restrict__ up,
                                const double* __restrict__ ub, double* __restrict__ corr) {
  pdl_entry();
  const int nd = B.three ? 3 : 2;
  const int a0 = box.a[0], a1 = box.a[1], a2 = box.a[2], b0 = box.b[0], b1 = box.b[1], b2 = box.b[2];
  const long m0 = b0 - a0, m1 = b1 - a1, m2 = nd == 3 ? b2 - a2 : 1;
  long g = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int d, side;
  if (!amr_face(g, nd, m1 * m2, m0 * m2, m0 * m1, d, side)) return;
  if (!amr_cf(box.cf, d, side)) return;
  // the uncovered coarse cell Q and its covered neighbour across the face
  int QI, QJ, QK;
  if (d == 0) {
    QJ = a1 + (int)(g % m1), QK = nd == 3 ? a2 + (int)(g / m1) : 0;
    QI = side < 0 ? a0 - 1 : b0;
  } else if (d == 1) {
    QI = a0 + (int)(g % m0), QK = nd == 3 ? a2 + (int)(g / m0) : 0;
    QJ = side < 0 ? a1 - 1 : b1;
  } else {
    QI = a0 + (int)(g % m0), QJ = a1 + (int)(g / m0);
    QK = side < 0 ? a2 - 1 : b2;
  }
  const int s = side < 0 ? -1 : 1;  // from the patch out to Q
  const int INi = QI - (d == 0) * s, INj = QJ - (d == 1) * s, INk = QK - (d == 2) * s;
  const double hb = d == 0 ? B.h0 : (d == 1 ? B.h1 : B.h2), hp = d == 0 ? Pv.h0 : (d == 1 ? Pv.h1 : Pv.h2);
  const double Ac = amr_area(B, d, -s, QI, QJ);
  const double Dc = (ub[B.idx(INi, INj, INk)] - ub[B.idx(QI, QJ, QK)]) / hb;
  // the fine faces: the patch cells next to the face under Q (2 in 2D, 4
  // in 3D) and their ghosts on Q's side
  const int fi0 = 2 * (QI - a0), fj0 = 2 * (QJ - a1), fk0 = nd == 3 ? 2 * (QK - a2) : 0;
  const int ni = (int)Pv.n0, nj = (int)Pv.n1, nk = Pv.three ? (int)Pv.n2 : 1;
  double fsum = 0.0;
  const int nq2 = nd == 3 ? 2 : 1;
  for (int q2 = 0; q2 < nq2; ++q2)
    for (int q1 = 0; q1 < 2; ++q1) {
      int fi, fj, fk;
      if (d == 0) {
        fi = side < 0 ? 0 : ni - 1, fj = fj0 + q1, fk = fk0 + q2;
      } else if (d == 1) {
        fj = side < 0 ? 0 : nj - 1, fi = fi0 + q1, fk = fk0 + q2;
      } else {
        fk = side < 0 ? 0 : nk - 1, fi = fi0 + q1, fj = fj0 + q2;
      }
      if (!Pv.three) fk = 0;
      const long pf = Pv.idx(fi, fj, fk);
      const long pg = Pv.idx(fi + (d == 0) * s, fj + (d == 1) * s, fk + (d == 2) * s);
      const double Af = amr_area(Pv, d, s, fi, fj);
      fsum += Af * (up[pf] - up[pg]) / hp;
    }
  corr[B.idx(QI, QJ, QK)] = (fsum - Ac * Dc) / amr_volume(B, QI, QJ);
}

__device__ __forceinline__ bool amr_covered(const AmrBox& box, int three, int I, int J, int K) {
  return I >= box.a[0] && I < box.b[0] && J >= box.a[1] && J < box.b[1] &&
         (!three || (K >= box.a[2] && K < box.b[2]));
}

// Base level of the composite grid, by mode:
//   0: FAS right-hand side f: covered cells L_H(u) + R r, uncovered cells
//      f0 - corr;
//   1: the composite residual norms of the uncovered cells into red (r =
//      f0 - L_H(u) - corr, slots as in k_amr_patch_resid), nothing written;
//   2: the composite operator L_H(u) + corr into f on uncovered cells, 0 on
//      covered ones.
template <int G, int KIND>
__global__ void k_amr_base(LevelView<double> B, AmrBox box, const double* __restrict__ u,
                           const double* __restrict__ s0, const double* __restrict__ s1, const double* __restrict__ f0,
                           const double* __restrict__ rr, const double* __restrict__ corr, double* __restrict__ f,
                           unsigned long long* red, int mode) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  unsigned long long m[3] = {0ULL, 0ULL, 0ULL};
  if (i < B.n0 && j < B.n1 && k < B.n2) {
    const long p = B.idx(i, j, k);
    const bool cov = amr_covered(box, B.three, i, j, k);
    if (mode == 0) {
      if (cov) {
        double D;
        f[p] = scalar_op<double, G, KIND>(B, u, s0, s1, i, j, k, p, D) + rr[p];
      } else {
        f[p] = (f0 ? f0[p] : 0.0) - corr[p];
      }
    } else if (mode == 2) {
      double D;
      f[p] = cov ? 0.0 : scalar_op<double, G, KIND>(B, u, s0, s1, i, j, k, p, D) + corr[p];
    } else if (!cov) {
      double D;
      const double Lu = scalar_op<double, G, KIND>(B, u, s0, s1, i, j, k, p, D) + corr[p];
      const double fv = f0 ? f0[p] : 0.0;
      const double rv = fv - Lu;
      double S;
      if (KIND == EQ_PSI) {
        const double ip = 1.0 / (1.0 + u[p]);
        const double ip2 = ip * ip;
        S = -2.0 * PI_D * s0[p] * ip - 0.125 * s1[p] * (ip2 * ip2 * ip2 * ip);
      } else {
        S = fv + (s1 ? s1[p] * u[p] : 0.0);
      }
      const double w = norm_weight(B, i, j);
      m[0] = abs_bits(rv);
      m[1] = abs_bits(w * rv);
      m[2] = abs_bits(w * S);
    }
  }
  if (mode == 1) block_max_bits<3>(m, red);
}

// Kwak prolongation (Sec. 2.7.3) of the base change e (ghosts filled with
// the homogeneous rules) onto the patch: parent a + (i, j, k) / 2 and, per
// dimension, the parent's neighbour on the fine cell's side.
__global__ void k_amr_prolong(LevelView<double> Pv, LevelView<double> B, AmrBox box, const double* __restrict__ e,
                              double* __restrict__ up) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= Pv.n0 || j >= Pv.n1 || k >= Pv.n2) return;
  const int I = box.a[0] + (i >> 1), J = box.a[1] + (j >> 1), K = Pv.three ? box.a[2] + (k >> 1) : 0;
  const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
  const double ec = e[B.idx(I, J, K)];
  const double ex = e[B.idx(I + si, J, K)], ey = e[B.idx(I, J + sj, K)];
  double add;
  if (Pv.three)
    add = 0.25 * (ec + ex + ey + e[B.idx(I, J, K + sk)]);
  else
    add = 0.25 * (2.0 * ec + ex + ey);
  up[Pv.idx(i, j, k)] += add;
}

// Composite unknowns (patch cells, then uncovered base cells, each in
// interior order) <-> a flat vector; patch cells first.
__global__ void k_amr_flat(LevelView<double> Pv, LevelView<double> B, AmrBox box, double* __restrict__ up,
                           double* __restrict__ ub, const int* __restrict__ bmap, long nbase, double* __restrict__ x,
                           int to_flat) {
  pdl_entry();
  const long np = (long)Pv.n0 * Pv.n1 * Pv.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < np + nbase; q += (long)gridDim.x * blockDim.x) {
    double* src;
    if (q < np) {
      int i, j, k;
      Pv.cell(q, i, j, k);
      src = up + Pv.idx(i, j, k);
    } else {
      src = ub + bmap[q - np];
    }
    if (to_flat)
      x[q] = *src;
    else
      *src = x[q];
  }
}

__global__ void k_amr_diff(LevelView<double> L, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  pdl_entry();
  const long n = (long)L.n0 * L.n1 * L.n2;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    int i, j, k;
    L.cell(q, i, j, k);
    const long p = L.idx(i, j, k);
    out[p] = a[p] - b[p];
  }
}

// ---------------------------------------------------------------- launchers

void launch_amr_diff(const LevelView<double>& L, const double* a, const double* b, double* out, cudaStream_t st) {
  count_launch();
  const long n = (long)L.n0 * L.n1 * L.n2;
  long g = cdiv_u(n, 256);
  if (g > 4096) g = 4096;
  launch_k(k_amr_diff, (unsigned)g, 256, 0, st, L, a, b, out);
}

static dim3 amr_block(int three) { return three ? dim3(32, 4, 2) : dim3(32, 8, 1); }

void launch_amr_cf_ghosts(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, double* up,
                          const double* ub, cudaStream_t st) {
  count_launch();
  const long n = 2L * ((long)Pv.n1 * Pv.n2 + (long)Pv.n0 * Pv.n2 + (Pv.three ? (long)Pv.n0 * Pv.n1 : 0L));
  launch_k(k_amr_cf_ghosts, cdiv_u(n, 256), 256, 0, st, Pv, B, box, up, ub);
}

template <int G>
static void amr_smooth_g(const LevelView<double>& L, int kind, double* u, const double* f, const double* s0,
                         const double* s1, int colour, cudaStream_t st) {
  const dim3 b = amr_block(L.three), g(cdiv_u(L.n0 / 2, b.x), cdiv_u(L.n1, b.y), cdiv_u(L.n2, b.z));
  if (kind == EQ_PSI)
    launch_k(k_amr_smooth<G, EQ_PSI>, g, b, 0, st, L, u, f, s0, s1, colour);
  else
    launch_k(k_amr_smooth<G, EQ_LIN>, g, b, 0, st, L, u, f, s0, s1, colour);
}
void launch_amr_smooth(const LevelView<double>& L, int kind, double* u, const double* f, const double* s0,
                       const double* s1, int colour, cudaStream_t st) {
  count_launch();
  if (L.geom == CART)
    amr_smooth_g<CART>(L, kind, u, f, s0, s1, colour, st);
  else if (L.geom == CYL)
    amr_smooth_g<CYL>(L, kind, u, f, s0, s1, colour, st);
  else
    amr_smooth_g<SPH>(L, kind, u, f, s0, s1, colour, st);
}

template <int G>
static void amr_resid_g(const LevelView<double>& L, int kind, const double* u, const double* f, const double* s0,
                        const double* s1, double* r, unsigned long long* red, int apply, cudaStream_t st) {
  const dim3 b = amr_block(L.three), g(cdiv_u(L.n0, b.x), cdiv_u(L.n1, b.y), cdiv_u(L.n2, b.z));
  if (kind == EQ_PSI)
    launch_k(k_amr_patch_resid<G, EQ_PSI>, g, b, 0, st, L, u, f, s0, s1, r, red, apply);
  else
    launch_k(k_amr_patch_resid<G, EQ_LIN>, g, b, 0, st, L, u, f, s0, s1, r, red, apply);
}
void launch_amr_patch_resid(const LevelView<double>& L, int kind, const double* u, const double* f, const double* s0,
                            const double* s1, double* r, unsigned long long* red, int apply, cudaStream_t st) {
  count_launch();
  if (L.geom == CART)
    amr_resid_g<CART>(L, kind, u, f, s0, s1, r, red, apply, st);
  else if (L.geom == CYL)
    amr_resid_g<CYL>(L, kind, u, f, s0, s1, r, red, apply, st);
  else
    amr_resid_g<SPH>(L, kind, u, f, s0, s1, r, red, apply, st);
}

void launch_amr_restrict(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, const double* up,
                         const double* rp, double* ub, double* rr, cudaStream_t st) {
  count_launch();
  const int m0 = box.b[0] - box.a[0], m1 = box.b[1] - box.a[1], m2 = box.b[2] - box.a[2];
  const dim3 b = amr_block(Pv.three), g(cdiv_u(m0, b.x), cdiv_u(m1, b.y), cdiv_u(m2, b.z));
  launch_k(k_amr_restrict, g, b, 0, st, Pv, B, box, up, rp, ub, rr);
}

void launch_amr_flux_corr(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box,
                          const double* up, const double* ub, double* corr, cudaStream_t st) {
  count_launch();
  const long m0 = box.b[0] - box.a[0], m1 = box.b[1] - box.a[1], m2 = B.three ? box.b[2] - box.a[2] : 1;
  const long n = 2L * (m1 * m2 + m0 * m2 + (B.three ? m0 * m1 : 0L));
  launch_k(k_amr_flux_corr, cdiv_u(n, 256), 256, 0, st, Pv, B, box, up, ub, corr);
}

template <int G>
static void amr_base_g(const LevelView<double>& B, const AmrBox& box, int kind, const double* u, const double* s0,
                       const double* s1, const double* f0, const double* rr, const double* corr, double* f,
                       unsigned long long* red, int mode, cudaStream_t st) {
  const dim3 b = amr_block(B.three), g(cdiv_u(B.n0, b.x), cdiv_u(B.n1, b.y), cdiv_u(B.n2, b.z));
  if (kind == EQ_PSI)
    launch_k(k_amr_base<G, EQ_PSI>, g, b, 0, st, B, box, u, s0, s1, f0, rr, corr, f, red, mode);
  else
    launch_k(k_amr_base<G, EQ_LIN>, g, b, 0, st, B, box, u, s0, s1, f0, rr, corr, f, red, mode);
}
void launch_amr_base(const LevelView<double>& B, const AmrBox& box, int kind, const double* u, const double* s0,
                     const double* s1, const double* f0, const double* rr, const double* corr, double* f,
                     unsigned long long* red, int mode, cudaStream_t st) {
  count_launch();
  if (B.geom == CART)
    amr_base_g<CART>(B, box, kind, u, s0, s1, f0, rr, corr, f, red, mode, st);
  else if (B.geom == CYL)
    amr_base_g<CYL>(B, box, kind, u, s0, s1, f0, rr, corr, f, red, mode, st);
  else
    amr_base_g<SPH>(B, box, kind, u, s0, s1, f0, rr, corr, f, red, mode, st);
}

void launch_amr_prolong(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, const double* e,
                        double* up, cudaStream_t st) {
  count_launch();
  const dim3 b = amr_block(Pv.three), g(cdiv_u(Pv.n0, b.x), cdiv_u(Pv.n1, b.y), cdiv_u(Pv.n2, b.z));
  launch_k(k_amr_prolong, g, b, 0, st, Pv, B, box, e, up);
}

void launch_amr_flat(const LevelView<double>& Pv, const LevelView<double>& B, const AmrBox& box, double* up,
                     double* ub, const int* bmap, long nbase, double* x, int to_flat, cudaStream_t st) {
  count_launch();
  const long n = (long)Pv.n0 * Pv.n1 * Pv.n2 + nbase;
  long g = cdiv_u(n, 256);
  if (g > 4096) g = 4096;
  launch_k(k_amr_flat, (unsigned)g, 256, 0, st, Pv, B, box, up, ub, bmap, nbase, x, to_flat);
}

}  // namespace gmg
