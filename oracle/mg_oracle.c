/*
 * Plain FP64 CPU oracle for the non-linear cell-centred multigrid solver of
 * Gmunu (Cheong et al.): FAS V-cycles with red-black Newton-Gauss-Seidel
 * smoothing, piecewise-constant restriction and Kwak prolongation, applied to
 * the xCFC metric equations and to elliptic divergence cleaning.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is slow and literal on purpose: every
 * cell update is written as a loop over cells in the order the paper states.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA library; both sides receive the same input arrays and nothing else.
 *
 * Paper passages followed (section / equation of arXiv:2012.07322):
 *   Sec. 2.6, eqs. (X), (psi), (alpha), (beta), (Aij)  -- xCFC equations
 *   Sec. 2.6, eqs. (bc), (robin)                       -- outer boundary
 *   Sec. 2.7.1, eq. (elliptic_op) and the Laplacians    -- discretisation
 *   Sec. 2.7.1, first / second / mixed derivatives      -- incl. block-corner
 *   Sec. 2.7.2, eq. (ngs_iteration), red-black ordering -- smoother
 *   Sec. 2.7.3, Kwak prolongation, piecewise-constant restriction
 *   Sec. 2.2, eqs. (poisson), (update_bfield)           -- div-B cleaning
 *   Sec. 4.2 (metric-solver performance): 2 + 2 red-black smoothing steps,
 *     full multigrid (FMG) cycles.
 *
 * Readings where the paper is silent or garbled (each listed in the design
 * notes of the repository):
 *   - the cylindrical and spherical Laplacians print "u_{j+1} - 2u - u_{j-1}";
 *     the consistent second difference "+ u_{j-1}" is used;
 *   - cells are coloured by (i+j+k) mod 2 with 0-based indices, even first;
 *   - vector equations are smoothed component by component inside a colour
 *     (all cells of the colour for component 0, then 1, then 2);
 *   - ghosts of a field are recomputed from its interior before every colour
 *     (or component) pass; the Newton diagonal treats them as fixed;
 *   - Cartesian / cylindrical Robin ghosts: g = u_N * rho(x_N) / rho(x_G),
 *     rho the distance from the origin, which satisfies delta + x.grad delta
 *     = 0 exactly for delta ~ 1/rho;
 *   - restriction averages the children weighted by their cell volumes
 *     (Appendix A); on Cartesian grids that is the printed equal-weight
 *     stencil;
 *   - FAS coarse-grid sources are restrictions of the fine sources; coarse
 *     operators are rediscretised;
 *   - coarsest grid: Newton-Gauss-Seidel sweeps until its residual falls by
 *     1e-12 or 16 sweeps (more sweeps leave the V-cycle counts unchanged);
 *   - stopping rule: rel = max|w r| / max|w S(u)|, w = r^2 sin(theta)
 *     (spherical), R (cylindrical), 1 (Cartesian);
 *   - FMG cycle (the paper times FMG cycles but does not spell one out): the
 *     textbook FAS form -- restrict the current solution and FAS sources to
 *     every level, solve the coarsest, then per level up: FAS correction from
 *     below and one V-cycle from that level;
 *   - optional Anderson mixing of successive V-cycle iterates (not in the
 *     paper; off when accel_depth = 0), in the difference form of Walker &
 *     Ni (SIAM J. Numer. Anal. 49, 2011): point smoothing converges slowly
 *     on spherical grids (the paper notes it), mixing restores the rate.
 *
 * Layout of every ghosted array: one ghost layer in each active dimension,
 * index (i, j, k) with i in [-1, n0], j in [-1, n1], k in [-1, n2] (3D) or
 * k = 0 (2D), dimension 0 fastest.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

enum { GEOM_CART = 0, GEOM_CYL = 1, GEOM_SPH = 2 };
enum { BC_ROBIN = 0, BC_DIRICHLET = 1, BC_NEUMANN = 2 };
enum { EQ_PSI = 0, EQ_LIN = 1, EQ_VEC = 2 };
enum { MIX_4PT = 0, MIX_CORNER = 1 };
#define OR_MAX_LEVELS 16
#define OR_HIST 1024

/* ------------------------------------------------------------------ grid */

typedef struct {
  int ndim, geom;
  int n[3];
  int gz;             /* ghost width in dimension 2: 1 in 3D, 0 in 2D */
  long s1, s2;        /* strides of dimensions 1 and 2 */
  long size;          /* ghosted cell count */
  double lo[3], h[3];
} OGrid;

static long IX(const OGrid* g, int i, int j, int k) {
  return (long)(i + 1) + (long)(j + 1) * g->s1 + (long)(k + g->gz) * g->s2;
}

/* Cell-centre coordinate of index i (ghosts included) in dimension d. */
static double xc(const OGrid* g, int d, int i) { return g->lo[d] + (i + 0.5) * g->h[d]; }
/* Face coordinate x_{i-1/2} in dimension d. */
static double xf(const OGrid* g, int d, int i) { return g->lo[d] + i * g->h[d]; }

static void grid_init(OGrid* g, int ndim, int geom, const int n[3], const double lo[3],
                      const double h[3]) {
  memset(g, 0, sizeof(*g));
  g->ndim = ndim;
  g->geom = geom;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = (d < ndim) ? n[d] : 1;
    g->lo[d] = (d < ndim) ? lo[d] : 0.0;
    g->h[d] = (d < ndim) ? h[d] : 1.0;
  }
  g->gz = (ndim == 3) ? 1 : 0;
  g->s1 = g->n[0] + 2;
  g->s2 = g->s1 * (g->n[1] + 2);
  g->size = g->s2 * (g->n[2] + 2 * g->gz);
}

/* sin(theta) at a theta face; exactly zero on the two poles (Sec. 2.7.1:
 * the flux through a pole vanishes). */
static double sin_face(const OGrid* g, int j) {
  if (j == 0 || j == g->n[1]) return 0.0;
  return sin(xf(g, 1, j));
}

/* --------------------------------------------------------- ghost filling */

/* Parity of a component under the reflections through the origin / axis
 * (regularity of physical vector components; comp = -1 is a scalar). */
static double parity_origin(int geom, int comp) {
  if (comp < 0) return 1.0;
  if (geom == GEOM_SPH) return (comp == 1) ? 1.0 : -1.0;   /* V_r -, V_th +, V_ph - */
  if (geom == GEOM_CYL) return (comp == 1) ? 1.0 : -1.0;   /* V_R -, V_z +, V_ph - */
  return 1.0;
}
static double parity_axis(int comp) {                        /* spherical theta = 0, pi */
  if (comp < 0) return 1.0;
  return (comp == 0) ? 1.0 : -1.0;                           /* V_r +, V_th -, V_ph - */
}

/* Distance from the origin of a cell centre (Cartesian / cylindrical Robin). */
static double rho_of(const OGrid* g, int i, int j, int k) {
  double x = xc(g, 0, i), y = xc(g, 1, j);
  if (g->geom == GEOM_CART) {
    double z = (g->ndim == 3) ? xc(g, 2, k) : 0.0;
    return sqrt(x * x + y * y + z * z);
  }
  return sqrt(x * x + y * y);                                /* (R, z) */
}

/* Outer-boundary ghost: 'gi,gj,gk' is the ghost, 'si,sj,sk' the interior
 * (or previously filled) cell across the face. */
static double outer_ghost(const OGrid* g, const double* u, int bc, int d, int gi, int gj, int gk,
                          int si, int sj, int sk) {
  double us = u[IX(g, si, sj, sk)];
  if (bc == BC_DIRICHLET) return -us;                        /* face value zero */
  if (bc == BC_NEUMANN) return us;                           /* zero normal gradient */
  /* Robin d(r delta)/dr = 0, eq. (robin) */
  if (g->geom == GEOM_SPH) {
    (void)d;
    return us * xc(g, 0, si) / xc(g, 0, gi);
  }
  return us * rho_of(g, si, sj, sk) / rho_of(g, gi, gj, gk);
}

/* Fill every ghost of one field.  Dimensions are filled in the order 0, 1,
 * 2, each over the index range already extended by the earlier ones, so
 * edge and corner ghosts are defined. */
static void fill_ghosts(const OGrid* g, double* u, int bc, int comp) {
  const int n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
  const int three = (g->ndim == 3);
  /* dimension 0 */
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j) {
      /* low side */
      if (g->geom == GEOM_CART) {
        u[IX(g, -1, j, k)] = outer_ghost(g, u, bc, 0, -1, j, k, 0, j, k);
      } else if (g->geom == GEOM_CYL) {
        int ks = three ? (k + n2 / 2) % n2 : k;
        u[IX(g, -1, j, k)] = parity_origin(GEOM_CYL, comp) * u[IX(g, 0, j, ks)];
      } else {
        int ks = three ? (k + n2 / 2) % n2 : k;
        u[IX(g, -1, j, k)] = parity_origin(GEOM_SPH, comp) * u[IX(g, 0, n1 - 1 - j, ks)];
      }
      /* high side: always the outer boundary */
      u[IX(g, n0, j, k)] = outer_ghost(g, u, bc, 0, n0, j, k, n0 - 1, j, k);
    }
  /* dimension 1 */
  for (int k = 0; k < n2; ++k)
    for (int i = -1; i <= n0; ++i) {
      if (g->geom == GEOM_SPH) {
        int ks = three ? (k + n2 / 2) % n2 : k;
        u[IX(g, i, -1, k)] = parity_axis(comp) * u[IX(g, i, 0, ks)];
        u[IX(g, i, n1, k)] = parity_axis(comp) * u[IX(g, i, n1 - 1, ks)];
      } else {
        u[IX(g, i, -1, k)] = outer_ghost(g, u, bc, 1, i, -1, k, i, 0, k);
        u[IX(g, i, n1, k)] = outer_ghost(g, u, bc, 1, i, n1, k, i, n1 - 1, k);
      }
    }
  /* dimension 2 */
  if (three)
    for (int j = -1; j <= n1; ++j)
      for (int i = -1; i <= n0; ++i) {
        if (g->geom == GEOM_CART) {
          u[IX(g, i, j, -1)] = outer_ghost(g, u, bc, 2, i, j, -1, i, j, 0);
          u[IX(g, i, j, n2)] = outer_ghost(g, u, bc, 2, i, j, n2, i, j, n2 - 1);
        } else {                                             /* periodic phi */
          u[IX(g, i, j, -1)] = u[IX(g, i, j, n2 - 1)];
          u[IX(g, i, j, n2)] = u[IX(g, i, j, 0)];
        }
      }
}

/* ----------------------------------------------------- discrete operators */

/* Scalar Laplacian in flux form (Sec. 2.7.1). */
static double lap(const OGrid* g, const double* u, int i, int j, int k) {
  const double uc = u[IX(g, i, j, k)];
  const double ue = u[IX(g, i + 1, j, k)], uw = u[IX(g, i - 1, j, k)];
  const double un = u[IX(g, i, j + 1, k)], us = u[IX(g, i, j - 1, k)];
  const double h0 = g->h[0], h1 = g->h[1], h2 = g->h[2];
  double L;
  if (g->geom == GEOM_CART) {
    L = (ue - 2.0 * uc + uw) / (h0 * h0) + (un - 2.0 * uc + us) / (h1 * h1);
    if (g->ndim == 3) L += (u[IX(g, i, j, k + 1)] - 2.0 * uc + u[IX(g, i, j, k - 1)]) / (h2 * h2);
  } else if (g->geom == GEOM_CYL) {
    const double R = xc(g, 0, i), Rp = xf(g, 0, i + 1), Rm = xf(g, 0, i);
    L = (Rp * (ue - uc) / h0 - Rm * (uc - uw) / h0) / (R * h0) + (un - 2.0 * uc + us) / (h1 * h1);
    if (g->ndim == 3)
      L += (u[IX(g, i, j, k + 1)] - 2.0 * uc + u[IX(g, i, j, k - 1)]) / (R * R * h2 * h2);
  } else {
    const double r = xc(g, 0, i), rp = xf(g, 0, i + 1), rm = xf(g, 0, i);
    const double st = sin(xc(g, 1, j)), sp = sin_face(g, j + 1), sm = sin_face(g, j);
    L = (rp * rp * (ue - uc) / h0 - rm * rm * (uc - uw) / h0) / (r * r * h0) +
        (sp * (un - uc) / h1 - sm * (uc - us) / h1) / (r * r * st * h1);
    if (g->ndim == 3)
      L += (u[IX(g, i, j, k + 1)] - 2.0 * uc + u[IX(g, i, j, k - 1)]) / (r * r * st * st * h2 * h2);
  }
  return L;
}

/* d(lap u)/d(u_ijk) with the neighbours (ghosts included) held fixed. */
static double lap_diag(const OGrid* g, int i, int j, int k) {
  (void)k;
  const double h0 = g->h[0], h1 = g->h[1], h2 = g->h[2];
  double D;
  if (g->geom == GEOM_CART) {
    D = -2.0 / (h0 * h0) - 2.0 / (h1 * h1);
    if (g->ndim == 3) D += -2.0 / (h2 * h2);
  } else if (g->geom == GEOM_CYL) {
    const double R = xc(g, 0, i), Rp = xf(g, 0, i + 1), Rm = xf(g, 0, i);
    D = -(Rp + Rm) / (R * h0 * h0) - 2.0 / (h1 * h1);
    if (g->ndim == 3) D += -2.0 / (R * R * h2 * h2);
  } else {
    const double r = xc(g, 0, i), rp = xf(g, 0, i + 1), rm = xf(g, 0, i);
    const double st = sin(xc(g, 1, j)), sp = sin_face(g, j + 1), sm = sin_face(g, j);
    D = -(rp * rp + rm * rm) / (r * r * h0 * h0) - (sp + sm) / (r * r * st * h1 * h1);
    if (g->ndim == 3) D += -2.0 / (r * r * st * st * h2 * h2);
  }
  return D;
}

/* Central first derivative along dimension d (Sec. 2.7.1); zero along a
 * dimension the grid does not have (axisymmetry / translation invariance). */
static double d1(const OGrid* g, const double* u, int d, int i, int j, int k) {
  if (d >= g->ndim) return 0.0;
  int di = (d == 0), dj = (d == 1), dk = (d == 2);
  return (u[IX(g, i + di, j + dj, k + dk)] - u[IX(g, i - di, j - dj, k - dk)]) / (2.0 * g->h[d]);
}
/* Compact second derivative along d. */
static double d2(const OGrid* g, const double* u, int d, int i, int j, int k) {
  if (d >= g->ndim) return 0.0;
  int di = (d == 0), dj = (d == 1), dk = (d == 2);
  return (u[IX(g, i + di, j + dj, k + dk)] - 2.0 * u[IX(g, i, j, k)] +
          u[IX(g, i - di, j - dj, k - dk)]) / (g->h[d] * g->h[d]);
}
/* Mixed second derivative along dimensions a < b: the four-corner stencil,
 * or the block-corner stencil of Sec. 2.7.1 which avoids one diagonal pair. */
static double dmix(const OGrid* g, const double* u, int a, int b, int mixed, int i, int j, int k) {
  if (a >= g->ndim || b >= g->ndim) return 0.0;
  int ai = (a == 0), aj = (a == 1), ak = (a == 2);
  int bi = (b == 0), bj = (b == 1), bk = (b == 2);
#define U_(p, q) u[IX(g, i + (p) * ai + (q) * bi, j + (p) * aj + (q) * bj, k + (p) * ak + (q) * bk)]
  if (mixed == MIX_4PT)
    return (U_(1, 1) - U_(1, -1) - U_(-1, 1) + U_(-1, -1)) / (4.0 * g->h[a] * g->h[b]);
  return (-U_(1, -1) - U_(-1, 1) + U_(1, 0) + U_(-1, 0) + U_(0, 1) + U_(0, -1) - 2.0 * U_(0, 0)) /
         (2.0 * g->h[a] * g->h[b]);
#undef U_
}

/* Vector operator lap V + (1/3) grad div V, physical component c, at a cell;
 * eqs. (X) and (beta) written out in orthonormal components of the flat
 * reference metric (Appendix A gives its Christoffel symbols). */
static double vec_op(const OGrid* g, double* const V[3], int c, int mixed, int i, int j, int k) {
  const double *A = V[0], *B = V[1], *C = V[2];
  const double third = 1.0 / 3.0;
  if (g->geom == GEOM_CART) {
    double gd;   /* d_c (div V) */
    if (c == 0)
      gd = d2(g, A, 0, i, j, k) + dmix(g, B, 0, 1, mixed, i, j, k) + dmix(g, C, 0, 2, mixed, i, j, k);
    else if (c == 1)
      gd = dmix(g, A, 0, 1, mixed, i, j, k) + d2(g, B, 1, i, j, k) + dmix(g, C, 1, 2, mixed, i, j, k);
    else
      gd = dmix(g, A, 0, 2, mixed, i, j, k) + dmix(g, B, 1, 2, mixed, i, j, k) + d2(g, C, 2, i, j, k);
    return lap(g, V[c], i, j, k) + third * gd;
  }
  if (g->geom == GEOM_CYL) {   /* components (R, z, phi) */
    const double R = xc(g, 0, i);
    if (c == 0) {
      double vl = lap(g, A, i, j, k) - A[IX(g, i, j, k)] / (R * R) - 2.0 / (R * R) * d1(g, C, 2, i, j, k);
      double gd = d2(g, A, 0, i, j, k) + d1(g, A, 0, i, j, k) / R - A[IX(g, i, j, k)] / (R * R) +
                  dmix(g, B, 0, 1, mixed, i, j, k) + dmix(g, C, 0, 2, mixed, i, j, k) / R -
                  d1(g, C, 2, i, j, k) / (R * R);
      return vl + third * gd;
    } else if (c == 1) {
      double vl = lap(g, B, i, j, k);
      double gd = dmix(g, A, 0, 1, mixed, i, j, k) + d1(g, A, 1, i, j, k) / R + d2(g, B, 1, i, j, k) +
                  dmix(g, C, 1, 2, mixed, i, j, k) / R;
      return vl + third * gd;
    } else {
      double vl = lap(g, C, i, j, k) - C[IX(g, i, j, k)] / (R * R) + 2.0 / (R * R) * d1(g, A, 2, i, j, k);
      double gd = dmix(g, A, 0, 2, mixed, i, j, k) / R + d1(g, A, 2, i, j, k) / (R * R) +
                  dmix(g, B, 1, 2, mixed, i, j, k) / R + d2(g, C, 2, i, j, k) / (R * R);
      return vl + third * gd;
    }
  }
  /* spherical, components (r, theta, phi) */
  const double r = xc(g, 0, i), th = xc(g, 1, j);
  const double st = sin(th), ct = cos(th), cot = ct / st;
  const double r2 = r * r, st2 = st * st;
  if (c == 0) {
    double vl = lap(g, A, i, j, k) - 2.0 * A[IX(g, i, j, k)] / r2 - 2.0 / r2 * d1(g, B, 1, i, j, k) -
                2.0 * cot / r2 * B[IX(g, i, j, k)] - 2.0 / (r2 * st) * d1(g, C, 2, i, j, k);
    double gd = d2(g, A, 0, i, j, k) + 2.0 / r * d1(g, A, 0, i, j, k) - 2.0 * A[IX(g, i, j, k)] / r2 +
                dmix(g, B, 0, 1, mixed, i, j, k) / r - d1(g, B, 1, i, j, k) / r2 +
                cot / r * d1(g, B, 0, i, j, k) - cot / r2 * B[IX(g, i, j, k)] +
                dmix(g, C, 0, 2, mixed, i, j, k) / (r * st) - d1(g, C, 2, i, j, k) / (r2 * st);
    return vl + third * gd;
  } else if (c == 1) {
    double vl = lap(g, B, i, j, k) - B[IX(g, i, j, k)] / (r2 * st2) + 2.0 / r2 * d1(g, A, 1, i, j, k) -
                2.0 * ct / (r2 * st2) * d1(g, C, 2, i, j, k);
    double gd = dmix(g, A, 0, 1, mixed, i, j, k) / r + 2.0 / r2 * d1(g, A, 1, i, j, k) +
                d2(g, B, 1, i, j, k) / r2 + cot / r2 * d1(g, B, 1, i, j, k) -
                B[IX(g, i, j, k)] / (r2 * st2) - ct / (r2 * st2) * d1(g, C, 2, i, j, k) +
                dmix(g, C, 1, 2, mixed, i, j, k) / (r2 * st);
    return vl + third * gd;
  } else {
    double vl = lap(g, C, i, j, k) - C[IX(g, i, j, k)] / (r2 * st2) +
                2.0 / (r2 * st) * d1(g, A, 2, i, j, k) + 2.0 * ct / (r2 * st2) * d1(g, B, 2, i, j, k);
    double gd = dmix(g, A, 0, 2, mixed, i, j, k) / (r * st) + 2.0 / (r2 * st) * d1(g, A, 2, i, j, k) +
                dmix(g, B, 1, 2, mixed, i, j, k) / (r2 * st) + cot / (r2 * st) * d1(g, B, 2, i, j, k) +
                d2(g, C, 2, i, j, k) / (r2 * st2);
    return vl + third * gd;
  }
}

/* d(vec_op_c)/d(V_c at the cell), neighbours held fixed. */
static double vec_diag(const OGrid* g, int c, int i, int j, int k) {
  const double third = 1.0 / 3.0;
  const double D = lap_diag(g, i, j, k);
  const double h0 = g->h[0], h1 = g->h[1], h2 = g->h[2];
  const int three = (g->ndim == 3);
  if (g->geom == GEOM_CART) {
    if (c < g->ndim) return D + third * (-2.0 / (g->h[c] * g->h[c]));
    return D;
  }
  if (g->geom == GEOM_CYL) {
    const double R = xc(g, 0, i);
    if (c == 0) return D - 1.0 / (R * R) + third * (-2.0 / (h0 * h0) - 1.0 / (R * R));
    if (c == 1) return D + third * (-2.0 / (h1 * h1));
    return D - 1.0 / (R * R) + (three ? third * (-2.0 / (R * R * h2 * h2)) : 0.0);
  }
  const double r = xc(g, 0, i), st = sin(xc(g, 1, j));
  const double r2 = r * r, st2 = st * st;
  if (c == 0) return D - 2.0 / r2 + third * (-2.0 / (h0 * h0) - 2.0 / r2);
  if (c == 1) return D - 1.0 / (r2 * st2) + third * (-2.0 / (r2 * h1 * h1) - 1.0 / (r2 * st2));
  return D - 1.0 / (r2 * st2) + (three ? third * (-2.0 / (r2 * st2 * h2 * h2)) : 0.0);
}

/* Weight of the stopping norm: the flux-form (volume) weight of a cell. */
static double norm_weight(const OGrid* g, int i, int j) {
  if (g->geom == GEOM_SPH) {
    double r = xc(g, 0, i);
    return r * r * sin(xc(g, 1, j));
  }
  if (g->geom == GEOM_CYL) return xc(g, 0, i);
  return 1.0;
}

/* ------------------------------------------------------------ equations */

/* One level of the hierarchy with the arrays an equation needs. */
typedef struct {
  OGrid g;
  double* u[3];    /* unknown (deviation form for psi / alpha*psi) */
  double* uh[3];   /* restricted fine solution, kept for the FAS correction */
  double* f[3];    /* right-hand side f of L(u) = f */
  double* r[3];    /* residual / scratch */
  double* U;       /* psi equation: conformal energy density U~ */
  double* A2;      /* psi equation: A~_ij A~^ij */
  double* c;       /* linear equations: coefficient of u in L(u) = lap u - c u */
} OLevel;

typedef struct {
  int kind, bc, ncomp, mixed, zero_mean;
  int nu1, nu2, max_cycles, stall_window, accel, fmg;
  double tol;
  int nlev;
  OLevel lev[OR_MAX_LEVELS];
} OSolver;

/* The operator L(u) at a cell for component c (eq. elliptic_op), and its
 * derivative with respect to the cell's own value for the Newton step.
 *   EQ_PSI : L(u) = lap u + 2 pi U (1+u)^-1 + (1/8) A2 (1+u)^-7      (eq. psi)
 *   EQ_LIN : L(u) = lap u - c u                 (eq. alpha; Poisson if c = 0)
 *   EQ_VEC : L(V) = lap V + (1/3) grad div V                (eqs. X, beta) */
static double op_at(const OSolver* s, const OLevel* L, int c, int i, int j, int k, double* diag) {
  const OGrid* g = &L->g;
  long p = IX(g, i, j, k);
  if (s->kind == EQ_VEC) {
    if (diag) *diag = vec_diag(g, c, i, j, k);
    return vec_op(g, (double* const*)L->u, c, s->mixed, i, j, k);
  }
  double lu = lap(g, L->u[0], i, j, k);
  double D = lap_diag(g, i, j, k);
  if (s->kind == EQ_PSI) {
    double psi = 1.0 + L->u[0][p];
    double val = lu + 2.0 * OR_PI * L->U[p] / psi + 0.125 * L->A2[p] / pow(psi, 7);
    if (diag) *diag = D - 2.0 * OR_PI * L->U[p] / (psi * psi) - 0.875 * L->A2[p] / pow(psi, 8);
    return val;
  }
  double cc = L->c ? L->c[p] : 0.0;
  if (diag) *diag = D - cc;
  return lu - cc * L->u[0][p];
}

/* The source S(u) of the equation as the paper writes it (right-hand side of
 * eqs. psi / alpha / X / beta / poisson), used to normalise the residual. */
static double source_at(const OSolver* s, const OLevel* L, int c, long p) {
  if (s->kind == EQ_PSI) {
    double psi = 1.0 + L->u[0][p];
    return -2.0 * OR_PI * L->U[p] / psi - 0.125 * L->A2[p] / pow(psi, 7);
  }
  if (s->kind == EQ_LIN) return (L->c ? L->c[p] * L->u[0][p] : 0.0) + L->f[0][p];
  return L->f[c][p];
}

static int comp_of(const OSolver* s, int c) { return s->kind == EQ_VEC ? c : -1; }

static void fill_all(const OSolver* s, OLevel* L) {
  for (int c = 0; c < s->ncomp; ++c) fill_ghosts(&L->g, L->u[c], s->bc, comp_of(s, c));
}

/* One red-black Newton-Gauss-Seidel sweep, eq. (ngs_iteration): cells with
 * (i+j+k) even first, then odd.  Vector equations take the components one
 * after another inside each colour. */
static void smooth_sweep(const OSolver* s, OLevel* L) {
  const OGrid* g = &L->g;
  for (int colour = 0; colour < 2; ++colour)
    for (int c = 0; c < s->ncomp; ++c) {
      fill_all(s, L);
#pragma omp parallel for collapse(2) schedule(static)
      for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
          for (int i = 0; i < g->n[0]; ++i) {
            if (((i + j + k) & 1) != colour) continue;
            double diag;
            double Lu = op_at(s, L, c, i, j, k, &diag);
            long p = IX(g, i, j, k);
            L->u[c][p] = L->u[c][p] - (Lu - L->f[c][p]) / diag;
          }
    }
}

/* r = f - L(u) on the interior; returns max |r| (unweighted). */
static double residual(const OSolver* s, OLevel* L) {
  const OGrid* g = &L->g;
  double m = 0.0;
  fill_all(s, L);
  for (int c = 0; c < s->ncomp; ++c)
#pragma omp parallel for collapse(2) reduction(max : m) schedule(static)
    for (int k = 0; k < g->n[2]; ++k)
      for (int j = 0; j < g->n[1]; ++j)
        for (int i = 0; i < g->n[0]; ++i) {
          long p = IX(g, i, j, k);
          L->r[c][p] = L->f[c][p] - op_at(s, L, c, i, j, k, NULL);
          double a = fabs(L->r[c][p]);
          if (a > m || a != a) m = (a != a) ? INFINITY : a;
        }
  return m;
}

/* Relative weighted residual of the finest level: the stopping rule. */
static double rel_residual(const OSolver* s, OLevel* L) {
  const OGrid* g = &L->g;
  residual(s, L);
  double num = 0.0, den = 0.0;
  int bad = 0;
  for (int c = 0; c < s->ncomp; ++c)
    for (int k = 0; k < g->n[2]; ++k)
      for (int j = 0; j < g->n[1]; ++j)
        for (int i = 0; i < g->n[0]; ++i) {
          long p = IX(g, i, j, k);
          double w = norm_weight(g, i, j);
          double a = fabs(w * L->r[c][p]), b = fabs(w * source_at(s, L, c, p));
          if (!(a == a) || !(b == b) || isinf(a) || isinf(b)) bad = 1;
          if (a > num) num = a;
          if (b > den) den = b;
        }
  if (bad) return NAN;
  return num / (den > 1e-300 ? den : 1e-300);
}

/* Cell volume Delta V of Appendix A (cylindrical and spherical; Cartesian
 * cells all have the same volume).  Only ratios between the children of one
 * coarse cell are used, so the factors the children share are dropped. */
static double cell_volume(const OGrid* g, int i, int j) {
  if (g->geom == GEOM_SPH) {
    double r = xc(g, 0, i), dr = g->h[0];
    return (r * r + dr * dr / 12.0) * dr * 2.0 * sin(xc(g, 1, j)) * sin(0.5 * g->h[1]);
  }
  if (g->geom == GEOM_CYL) return xc(g, 0, i) * g->h[0];
  return 1.0;
}

/* Piecewise-constant restriction (Sec. 2.7.3, Fig. pc): the coarse value is
 * the average of its 2^d children.  On Cartesian grids this is the printed
 * 1/4 (2D) or 1/8 (3D) stencil; on curvilinear grids the children are
 * weighted by their volumes, which keeps the restriction conservative (with
 * equal weights the V-cycle diverges next to the spherical origin). */
static void restrict_field(const OGrid* gf, const double* uf, const OGrid* gc, double* uc) {
  const int three = (gc->ndim == 3);
  for (int K = 0; K < gc->n[2]; ++K)
    for (int J = 0; J < gc->n[1]; ++J)
      for (int I = 0; I < gc->n[0]; ++I) {
        double sum = 0.0, vol = 0.0;
        for (int dk = 0; dk <= three; ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
              double v = cell_volume(gf, 2 * I + di, 2 * J + dj);
              sum += v * uf[IX(gf, 2 * I + di, 2 * J + dj, three ? 2 * K + dk : 0)];
              vol += v;
            }
        uc[IX(gc, I, J, K)] = sum / vol;
      }
}

/* Kwak prolongation (Sec. 2.7.3, Fig. kwak) of a coarse correction e (with
 * ghosts filled), added into the fine field.  Each fine cell takes its parent
 * and, per dimension, the parent's neighbour on the fine cell's side:
 * 2D 1/4 (2 e_c + e_x + e_y), 3D 1/4 (e_c + e_x + e_y + e_z). */
static void prolong_add(const OGrid* gf, double* uf, const OGrid* gc, const double* e) {
  const int three = (gf->ndim == 3);
  for (int k = 0; k < gf->n[2]; ++k)
    for (int j = 0; j < gf->n[1]; ++j)
      for (int i = 0; i < gf->n[0]; ++i) {
        int I = i / 2, J = j / 2, K = three ? k / 2 : 0;
        int si = (i % 2 == 0) ? -1 : 1, sj = (j % 2 == 0) ? -1 : 1, sk = (k % 2 == 0) ? -1 : 1;
        double ec = e[IX(gc, I, J, K)];
        double ex = e[IX(gc, I + si, J, K)], ey = e[IX(gc, I, J + sj, K)];
        double add;
        if (three)
          add = 0.25 * (ec + ex + ey + e[IX(gc, I, J, K + sk)]);
        else
          add = 0.25 * (2.0 * ec + ex + ey);
        uf[IX(gf, i, j, k)] += add;
      }
}

static double interior_mean(const OGrid* g, const double* u) {
  double sum = 0.0;
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) sum += u[IX(g, i, j, k)];
  return sum / ((double)g->n[0] * g->n[1] * g->n[2]);
}

/* Newton-Gauss-Seidel on the coarsest grid used as the direct solver
 * (Sec. 2.7.2): sweeps until the residual drops by 1e-12 or 16 sweeps. */
#define OR_COARSE_SWEEPS 16
static void coarse_solve(const OSolver* s, OLevel* L) {
  double r0 = residual(s, L);
  if (r0 == 0.0) return;
  for (int it = 0; it < OR_COARSE_SWEEPS; ++it) {
    smooth_sweep(s, L);
    double r = residual(s, L);
    if (r <= 1e-12 * r0) break;
  }
}

/* FAS restriction from level l to l + 1 at the current u_l:
 *   r = f - L(u); u_H = R u, uh_H = u_H; f_H = L_H(u_H) + R r. */
static void fas_down(const OSolver* s, OSolver* sm, int l) {
  OLevel* L = &sm->lev[l];
  OLevel* C = &sm->lev[l + 1];
  residual(s, L);
  for (int c = 0; c < s->ncomp; ++c) {
    restrict_field(&L->g, L->u[c], &C->g, C->u[c]);
    memcpy(C->uh[c], C->u[c], sizeof(double) * C->g.size);
    restrict_field(&L->g, L->r[c], &C->g, C->r[c]);
  }
  fill_all(s, C);
  for (int c = 0; c < s->ncomp; ++c)
    for (int k = 0; k < C->g.n[2]; ++k)
      for (int j = 0; j < C->g.n[1]; ++j)
        for (int i = 0; i < C->g.n[0]; ++i) {
          long p = IX(&C->g, i, j, k);
          C->f[c][p] = op_at(s, C, c, i, j, k, NULL) + C->r[c][p];
        }
}

/* FAS correction of level l from level l + 1: u += P(u_H - uh_H), the
 * coarse change taking the homogeneous boundary ghosts. */
static void fas_up(const OSolver* s, OSolver* sm, int l) {
  OLevel* L = &sm->lev[l];
  OLevel* C = &sm->lev[l + 1];
  for (int c = 0; c < s->ncomp; ++c) {
    double* e = C->r[c];
    for (long p = 0; p < C->g.size; ++p) e[p] = C->u[c][p] - C->uh[c][p];
    fill_ghosts(&C->g, e, s->bc, comp_of(s, c));
    prolong_add(&L->g, L->u[c], &C->g, e);
  }
}

/* FAS V(nu1, nu2) cycle (the paper cites the FAS scheme of Cheong et al.):
 *   pre-smooth; restrict (fas_down); recurse; correct (fas_up); post-smooth. */
static void vcycle(const OSolver* s, OSolver* sm, int l) {
  OLevel* L = &sm->lev[l];
  if (l == s->nlev - 1) {
    coarse_solve(s, L);
    return;
  }
  for (int it = 0; it < s->nu1; ++it) smooth_sweep(s, L);
  fas_down(s, sm, l);
  vcycle(s, sm, l + 1);
  fas_up(s, sm, l);
  for (int it = 0; it < s->nu2; ++it) smooth_sweep(s, L);
}

/* Full multigrid (FMG) cycle in FAS form, the cycle the paper times in its
 * solver-performance tests (Sec. 4.2): the current solution and its FAS
 * right-hand sides are restricted to every level without smoothing, the
 * coarsest level is solved, then each finer level is corrected from the
 * level below and improved by one V-cycle starting at that level. */
static void fmg_cycle(const OSolver* s, OSolver* sm) {
  for (int l = 0; l + 1 < s->nlev; ++l) fas_down(s, sm, l);
  coarse_solve(s, &sm->lev[s->nlev - 1]);
  for (int l = s->nlev - 2; l >= 0; --l) {
    fas_up(s, sm, l);
    vcycle(s, sm, l);
  }
}

/* ------------------------------------------------------------- hierarchy */

static int build_levels(OSolver* s, int ndim, int geom, const int n[3], const double lo[3],
                        const double hi[3]) {
  int m[3] = {n[0], ndim > 1 ? n[1] : 1, ndim > 2 ? n[2] : 1};
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (d < ndim) ? (hi[d] - lo[d]) / m[d] : 1.0;
  int nl = 0;
  for (;;) {
    OLevel* L = &s->lev[nl];
    memset(L, 0, sizeof(*L));
    grid_init(&L->g, ndim, geom, m, lo, h);
    long sz = L->g.size;
    for (int c = 0; c < 3; ++c) {
      L->u[c] = calloc(sz, sizeof(double));
      L->uh[c] = calloc(sz, sizeof(double));
      L->f[c] = calloc(sz, sizeof(double));
      L->r[c] = calloc(sz, sizeof(double));
    }
    L->U = calloc(sz, sizeof(double));
    L->A2 = calloc(sz, sizeof(double));
    L->c = calloc(sz, sizeof(double));
    ++nl;
    /* halve while every dimension is even and at least 4 */
    int ok = (nl < OR_MAX_LEVELS);
    for (int d = 0; d < ndim; ++d)
      if (m[d] < 4 || m[d] % 2) ok = 0;
    if (!ok) break;
    for (int d = 0; d < ndim; ++d) {
      m[d] /= 2;
      h[d] *= 2.0;
    }
  }
  s->nlev = nl;
  return nl;
}

static void free_levels(OSolver* s) {
  for (int l = 0; l < s->nlev; ++l) {
    OLevel* L = &s->lev[l];
    for (int c = 0; c < 3; ++c) {
      free(L->u[c]);
      free(L->uh[c]);
      free(L->f[c]);
      free(L->r[c]);
    }
    free(L->U);
    free(L->A2);
    free(L->c);
  }
  s->nlev = 0;
}

/* Interior (ghost-free, dimension 0 fastest) <-> ghosted copies. */
static void load_interior(const OGrid* g, double* dst, const double* src) {
  long q = 0;
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) dst[IX(g, i, j, k)] = src[q++];
}
static void store_interior(const OGrid* g, double* dst, const double* src) {
  long q = 0;
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) dst[q++] = src[IX(g, i, j, k)];
}

/* ------------------------------------------------------------ public API */

typedef struct {
  int ndim, geom;
  int n[3];
  double lo[3], hi[3];
  int nu1, nu2, max_cycles;
  double tol;
  int mixed;
  int stall_window;   /* cycles over which a 5 % gain is required; 0: off */
  int accel_depth;    /* Anderson mixing depth m over the V-cycle map; 0: off */
  int cycle;          /* 0: V-cycles, 1: FMG cycles */
} or_desc;

typedef struct {
  int status;      /* 0 ok, 3 not converged, 4 stalled, 5 non-finite */
  int cycles;
  double rel;      /* final relative weighted residual */
  int nhist;
  double hist[OR_HIST];
} or_report;

/* Restrict the equation's sources down the hierarchy. */
static void restrict_sources(OSolver* s) {
  for (int l = 1; l < s->nlev; ++l) {
    OLevel *F = &s->lev[l - 1], *C = &s->lev[l];
    restrict_field(&F->g, F->U, &C->g, C->U);
    restrict_field(&F->g, F->A2, &C->g, C->A2);
    restrict_field(&F->g, F->c, &C->g, C->c);
  }
}

/* The fixed-point map of the iteration: one FAS V-cycle from the current
 * finest u, then (Neumann gauge) removal of the mean. */
static void cycle_map(OSolver* s) {
  OLevel* F = &s->lev[0];
  if (s->fmg)
    fmg_cycle(s, s);
  else
    vcycle(s, s, 0);
  if (s->zero_mean) {
    double m = interior_mean(&F->g, F->u[0]);
    for (int k = 0; k < F->g.n[2]; ++k)
      for (int j = 0; j < F->g.n[1]; ++j)
        for (int i = 0; i < F->g.n[0]; ++i) F->u[0][IX(&F->g, i, j, k)] -= m;
  }
}

/* Finest unknowns (all components) <-> one flat vector. */
static void gather_u(const OSolver* s, double* x) {
  const OLevel* F = &s->lev[0];
  long q = 0;
  for (int c = 0; c < s->ncomp; ++c)
    for (int k = 0; k < F->g.n[2]; ++k)
      for (int j = 0; j < F->g.n[1]; ++j)
        for (int i = 0; i < F->g.n[0]; ++i) x[q++] = F->u[c][IX(&F->g, i, j, k)];
}
static void scatter_u(OSolver* s, const double* x) {
  OLevel* F = &s->lev[0];
  long q = 0;
  for (int c = 0; c < s->ncomp; ++c)
    for (int k = 0; k < F->g.n[2]; ++k)
      for (int j = 0; j < F->g.n[1]; ++j)
        for (int i = 0; i < F->g.n[0]; ++i) F->u[c][IX(&F->g, i, j, k)] = x[q++];
}

/* Solve (M + lambda I) y = b for the small symmetric Gram matrix M (order
 * m, row-major) by Cholesky, lambda = 1e-12 max diag(M).  Returns 0 on
 * success, -1 if M is degenerate. */
static int small_spd_solve(int m, const double* M, const double* b, double* y) {
  double A[64 * 64], L[64 * 64];
  double dmax = 0.0;
  for (int i = 0; i < m; ++i) dmax = M[i * m + i] > dmax ? M[i * m + i] : dmax;
  if (!(dmax > 0.0)) return -1;
  for (int i = 0; i < m * m; ++i) A[i] = M[i];
  for (int i = 0; i < m; ++i) A[i * m + i] += 1e-12 * dmax;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) {
      double sum = A[i * m + j];
      for (int k = 0; k < j; ++k) sum -= L[i * m + k] * L[j * m + k];
      if (i == j) {
        if (!(sum > 0.0)) return -1;
        L[i * m + i] = sqrt(sum);
      } else {
        L[i * m + j] = sum / L[j * m + j];
      }
    }
  double z[64];
  for (int i = 0; i < m; ++i) {
    double sum = b[i];
    for (int k = 0; k < i; ++k) sum -= L[i * m + k] * z[k];
    z[i] = sum / L[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double sum = z[i];
    for (int k = i + 1; k < m; ++k) sum -= L[k * m + i] * y[k];
    y[i] = sum / L[i * m + i];
  }
  return 0;
}

/* Cycle control: V-cycles until rel <= tol, max_cycles (not converged),
 * no 5 % gain over stall_window cycles (stalled) or a non-finite value.
 * With accel > 0 the iterates are Anderson-mixed (depth m = accel):
 * f = G(x) - x, x_next = G(x) - dG gamma, gamma = argmin |f - dF gamma|
 * over the last m differences dF, dG of f and G (one V-cycle each). */
static int run_cycles(OSolver* s, or_report* rep) {
  OLevel* F = &s->lev[0];
  double rel = rel_residual(s, F);
  int cyc = 0, status = 0;
  double hist[OR_HIST];
  int nh = 0;
  hist[nh++] = rel;
  const int m = s->accel < 0 ? 0 : (s->accel > 32 ? 32 : s->accel);
  const long nv = (long)s->ncomp * F->g.n[0] * F->g.n[1] * F->g.n[2];
  double *x = NULL, *g = NULL, *fcur = NULL, *fprev = NULL, *gprev = NULL, *dF = NULL, *dG = NULL;
  int ncol = 0, head = 0;   /* columns kept; ring position of the next column */
  if (m > 0) {
    x = malloc(sizeof(double) * nv);
    g = malloc(sizeof(double) * nv);
    fcur = malloc(sizeof(double) * nv);
    fprev = malloc(sizeof(double) * nv);
    gprev = malloc(sizeof(double) * nv);
    dF = malloc(sizeof(double) * nv * m);
    dG = malloc(sizeof(double) * nv * m);
  }
  while (1) {
    if (rel != rel) { status = 5; break; }
    if (rel <= s->tol) break;
    if (cyc >= s->max_cycles) { status = 3; break; }
    if (s->stall_window > 0 && cyc >= s->stall_window && rel > 0.95 * hist[cyc - s->stall_window]) {
      status = 4;
      break;
    }
    if (m == 0) {
      cycle_map(s);
    } else {
      gather_u(s, x);
      cycle_map(s);
      gather_u(s, g);
      for (long q = 0; q < nv; ++q) fcur[q] = g[q] - x[q];
      if (cyc > 0) {
        double* cf = dF + (long)head * nv;
        double* cg = dG + (long)head * nv;
        for (long q = 0; q < nv; ++q) {
          cf[q] = fcur[q] - fprev[q];
          cg[q] = g[q] - gprev[q];
        }
        head = (head + 1) % m;
        if (ncol < m) ++ncol;
      }
      memcpy(fprev, fcur, sizeof(double) * nv);
      memcpy(gprev, g, sizeof(double) * nv);
      if (ncol > 0) {
        /* columns in age order: oldest first */
        double M[32 * 32], b[32], gam[32];
        int col[32];
        for (int a = 0; a < ncol; ++a) col[a] = (head - ncol + a + m) % m;
        for (int a = 0; a < ncol; ++a) {
          const double* fa = dF + (long)col[a] * nv;
          double sb = 0.0;
          for (long q = 0; q < nv; ++q) sb += fa[q] * fcur[q];
          b[a] = sb;
          for (int c2 = 0; c2 <= a; ++c2) {
            const double* fc = dF + (long)col[c2] * nv;
            double sm = 0.0;
            for (long q = 0; q < nv; ++q) sm += fa[q] * fc[q];
            M[a * ncol + c2] = sm;
            M[c2 * ncol + a] = sm;
          }
        }
        if (small_spd_solve(ncol, M, b, gam) == 0) {
          for (int a = 0; a < ncol; ++a) {
            const double* ga = dG + (long)col[a] * nv;
            for (long q = 0; q < nv; ++q) g[q] -= gam[a] * ga[q];
          }
        } else {
          ncol = 0;   /* degenerate history: restart the mixing */
        }
      }
      scatter_u(s, g);
    }
    ++cyc;
    rel = rel_residual(s, F);
    if (nh < OR_HIST) hist[nh++] = rel;
  }
  free(x);
  free(g);
  free(fcur);
  free(fprev);
  free(gprev);
  free(dF);
  free(dG);
  if (rep) {
    rep->status = status;
    rep->cycles = cyc;
    rep->rel = rel;
    rep->nhist = nh;
    memcpy(rep->hist, hist, sizeof(double) * nh);
  }
  return status;
}

static void setup(OSolver* s, const or_desc* d, int kind, int bc, int ncomp) {
  memset(s, 0, sizeof(*s));
  s->kind = kind;
  s->bc = bc;
  s->ncomp = ncomp;
  s->mixed = d->mixed;
  s->nu1 = d->nu1;
  s->nu2 = d->nu2;
  s->max_cycles = d->max_cycles;
  s->tol = d->tol;
  s->stall_window = d->stall_window;
  s->accel = d->accel_depth;
  s->fmg = d->cycle == 1;
  build_levels(s, d->ndim, d->geom, d->n, d->lo, d->hi);
}

static long ncells(const or_desc* d) {
  long m = 1;
  for (int k = 0; k < d->ndim; ++k) m *= d->n[k];
  return m;
}

/* Number of levels the hierarchy rule gives. */
int or_num_levels(const or_desc* d) {
  OSolver s;
  setup(&s, d, EQ_LIN, BC_NEUMANN, 1);
  int n = s.nlev;
  free_levels(&s);
  return n;
}

/* Scalar solve: kind EQ_PSI (U, A2 used) or EQ_LIN (c may be NULL, f used).
 * All arrays are interior layout; u is the initial guess in, solution out. */
int or_solve_scalar(const or_desc* d, int kind, int bc, int zero_mean, const double* U,
                    const double* A2, const double* c, const double* f, double* u, or_report* rep) {
  OSolver s;
  setup(&s, d, kind, bc, 1);
  s.zero_mean = zero_mean;
  OLevel* F = &s.lev[0];
  if (U) load_interior(&F->g, F->U, U);
  if (A2) load_interior(&F->g, F->A2, A2);
  if (c) load_interior(&F->g, F->c, c);
  if (f) load_interior(&F->g, F->f[0], f);
  load_interior(&F->g, F->u[0], u);
  restrict_sources(&s);
  int st = run_cycles(&s, rep);
  store_interior(&F->g, u, F->u[0]);
  free_levels(&s);
  return st;
}

/* Vector solve of lap V + 1/3 grad div V = f (three components). */
int or_solve_vector(const or_desc* d, int bc, double* const f[3], double* const V[3], or_report* rep) {
  OSolver s;
  setup(&s, d, EQ_VEC, bc, 3);
  OLevel* F = &s.lev[0];
  for (int c = 0; c < 3; ++c) {
    load_interior(&F->g, F->f[c], f[c]);
    load_interior(&F->g, F->u[c], V[c]);
  }
  int st = run_cycles(&s, rep);
  for (int c = 0; c < 3; ++c) store_interior(&F->g, V[c], F->u[c]);
  free_levels(&s);
  return st;
}

/* ---- unit-level entry points on ghosted arrays (finest level only) ---- */

/* Ghosted size of the finest grid. */
long or_ghosted_size(const or_desc* d) {
  OGrid g;
  int m[3] = {d->n[0], d->n[1], d->ndim > 2 ? d->n[2] : 1};
  double h[3];
  for (int k = 0; k < 3; ++k) h[k] = (k < d->ndim) ? (d->hi[k] - d->lo[k]) / m[k] : 1.0;
  grid_init(&g, d->ndim, d->geom, m, d->lo, h);
  return g.size;
}

static void finest_grid(const or_desc* d, OGrid* g) {
  int m[3] = {d->n[0], d->n[1], d->ndim > 2 ? d->n[2] : 1};
  double h[3];
  for (int k = 0; k < 3; ++k) h[k] = (k < d->ndim) ? (d->hi[k] - d->lo[k]) / m[k] : 1.0;
  grid_init(g, d->ndim, d->geom, m, d->lo, h);
}

/* Fill the ghosts of one ghosted field (comp -1 scalar, 0..2 vector). */
void or_fill_ghosts(const or_desc* d, int bc, int comp, double* u) {
  OGrid g;
  finest_grid(d, &g);
  fill_ghosts(&g, u, bc, comp);
}

/* Apply L to ghosted fields WITHOUT touching their ghosts; out is ghosted
 * (interior written).  kind EQ_VEC uses V[0..2] and writes out[0..2]. */
void or_apply_raw(const or_desc* d, int kind, double* const V[3], const double* U,
                  const double* A2, const double* c, double* const out[3]) {
  OSolver s;
  memset(&s, 0, sizeof(s));
  s.kind = kind;
  s.ncomp = (kind == EQ_VEC) ? 3 : 1;
  s.mixed = d->mixed;
  OLevel L;
  memset(&L, 0, sizeof(L));
  finest_grid(d, &L.g);
  for (int k = 0; k < 3; ++k) L.u[k] = V[k];
  L.U = (double*)U;
  L.A2 = (double*)A2;
  L.c = (double*)c;
  for (int cc = 0; cc < s.ncomp; ++cc)
    for (int k = 0; k < L.g.n[2]; ++k)
      for (int j = 0; j < L.g.n[1]; ++j)
        for (int i = 0; i < L.g.n[0]; ++i)
          out[cc][IX(&L.g, i, j, k)] = op_at(&s, &L, cc, i, j, k, NULL);
}

/* nsweeps red-black NGS sweeps on the finest level (ghosted arrays; ghosts
 * are refilled as in the solver).  For EQ_VEC, f and u have 3 components. */
void or_smooth(const or_desc* d, int kind, int bc, int nsweeps, double* const u[3],
               double* const f[3], const double* U, const double* A2, const double* c) {
  OSolver s;
  memset(&s, 0, sizeof(s));
  s.kind = kind;
  s.bc = bc;
  s.ncomp = (kind == EQ_VEC) ? 3 : 1;
  s.mixed = d->mixed;
  OLevel L;
  memset(&L, 0, sizeof(L));
  finest_grid(d, &L.g);
  for (int k = 0; k < 3; ++k) {
    L.u[k] = u[k];
    L.f[k] = f[k];
  }
  L.U = (double*)U;
  L.A2 = (double*)A2;
  L.c = (double*)c;
  for (int it = 0; it < nsweeps; ++it) smooth_sweep(&s, &L);
}

/* Restriction / Kwak prolongation between the finest grid of d and the next
 * coarser grid (ghosted arrays).  'e' must already carry its ghosts. */
void or_restrict(const or_desc* d, const double* uf, double* uc) {
  OGrid gf, gc;
  finest_grid(d, &gf);
  int m[3];
  double h[3];
  for (int k = 0; k < 3; ++k) {
    m[k] = (k < d->ndim) ? gf.n[k] / 2 : 1;
    h[k] = gf.h[k] * ((k < d->ndim) ? 2.0 : 1.0);
  }
  grid_init(&gc, d->ndim, d->geom, m, gf.lo, h);
  restrict_field(&gf, uf, &gc, uc);
}
void or_prolong_add(const or_desc* d, double* uf, const double* e) {
  OGrid gf, gc;
  finest_grid(d, &gf);
  int m[3];
  double h[3];
  for (int k = 0; k < 3; ++k) {
    m[k] = (k < d->ndim) ? gf.n[k] / 2 : 1;
    h[k] = gf.h[k] * ((k < d->ndim) ? 2.0 : 1.0);
  }
  grid_init(&gc, d->ndim, d->geom, m, gf.lo, h);
  prolong_add(&gf, uf, &gc, e);
}

/* ---------------------------------------------------------- xCFC pieces */

/* A~_ij (orthonormal components, eq. Aij) from X with its ghosts filled:
 * A~ = 2 E - (2/3) div X delta, E the symmetric gradient of X.  Writes the
 * six independent components (rr, tt, pp, rt, rp, tp) and A2 = sum A~_ij^2. */
static void aij_at(const OGrid* g, double* const X[3], int i, int j, int k, double A[6]) {
  const double* a = X[0];
  const double* b = X[1];
  const double* cc = X[2];
  long p = IX(g, i, j, k);
  double E00, E11, E22, E01, E02, E12, div;
  if (g->geom == GEOM_CART) {
    E00 = d1(g, a, 0, i, j, k);
    E11 = d1(g, b, 1, i, j, k);
    E22 = d1(g, cc, 2, i, j, k);
    E01 = 0.5 * (d1(g, a, 1, i, j, k) + d1(g, b, 0, i, j, k));
    E02 = 0.5 * (d1(g, a, 2, i, j, k) + d1(g, cc, 0, i, j, k));
    E12 = 0.5 * (d1(g, b, 2, i, j, k) + d1(g, cc, 1, i, j, k));
  } else if (g->geom == GEOM_CYL) {   /* (R, z, phi) */
    const double R = xc(g, 0, i);
    E00 = d1(g, a, 0, i, j, k);
    E11 = d1(g, b, 1, i, j, k);
    E22 = d1(g, cc, 2, i, j, k) / R + a[p] / R;
    E01 = 0.5 * (d1(g, a, 1, i, j, k) + d1(g, b, 0, i, j, k));
    E02 = 0.5 * (d1(g, a, 2, i, j, k) / R + d1(g, cc, 0, i, j, k) - cc[p] / R);
    E12 = 0.5 * (d1(g, cc, 1, i, j, k) + d1(g, b, 2, i, j, k) / R);
  } else {                            /* (r, theta, phi) */
    const double r = xc(g, 0, i), th = xc(g, 1, j);
    const double st = sin(th), cot = cos(th) / st;
    E00 = d1(g, a, 0, i, j, k);
    E11 = d1(g, b, 1, i, j, k) / r + a[p] / r;
    E22 = d1(g, cc, 2, i, j, k) / (r * st) + a[p] / r + cot * b[p] / r;
    E01 = 0.5 * (d1(g, b, 0, i, j, k) - b[p] / r + d1(g, a, 1, i, j, k) / r);
    E02 = 0.5 * (d1(g, a, 2, i, j, k) / (r * st) + d1(g, cc, 0, i, j, k) - cc[p] / r);
    E12 = 0.5 * (d1(g, cc, 1, i, j, k) / r - cot * cc[p] / r + d1(g, b, 2, i, j, k) / (r * st));
  }
  div = E00 + E11 + E22;
  A[0] = 2.0 * E00 - 2.0 / 3.0 * div;
  A[1] = 2.0 * E11 - 2.0 / 3.0 * div;
  A[2] = 2.0 * E22 - 2.0 / 3.0 * div;
  A[3] = 2.0 * E01;
  A[4] = 2.0 * E02;
  A[5] = 2.0 * E12;
}

static double a2_of(const double A[6]) {
  return A[0] * A[0] + A[1] * A[1] + A[2] * A[2] + 2.0 * (A[3] * A[3] + A[4] * A[4] + A[5] * A[5]);
}

/* Physical gradient of a scalar with ghosts. */
static void grad_phys(const OGrid* g, const double* s, int i, int j, int k, double G[3]) {
  G[0] = d1(g, s, 0, i, j, k);
  G[1] = d1(g, s, 1, i, j, k);
  G[2] = d1(g, s, 2, i, j, k);
  if (g->geom == GEOM_CYL) {
    G[2] /= xc(g, 0, i);
  } else if (g->geom == GEOM_SPH) {
    double r = xc(g, 0, i), st = sin(xc(g, 1, j));
    G[1] /= r;
    G[2] /= (r * st);
  }
}

/* A~_ij and A2 from X given on the interior (Dirichlet-0 outer ghosts,
 * parity inner ghosts).  Outputs interior arrays: A6[6] (may be NULL) and A2. */
void or_aij(const or_desc* d, double* const X[3], double* const A6[6], double* A2) {
  OGrid g;
  finest_grid(d, &g);
  double* Xg[3];
  for (int c = 0; c < 3; ++c) {
    Xg[c] = calloc(g.size, sizeof(double));
    load_interior(&g, Xg[c], X[c]);
    fill_ghosts(&g, Xg[c], BC_DIRICHLET, c);
  }
  long q = 0;
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i, ++q) {
        double A[6];
        aij_at(&g, Xg, i, j, k, A);
        if (A6)
          for (int m = 0; m < 6; ++m) A6[m][q] = A[m];
        A2[q] = a2_of(A);
      }
  for (int c = 0; c < 3; ++c) free(Xg[c]);
}

typedef struct {
  int psi_only;     /* 1: solve the psi equation only with A2 = 0 */
  or_report rep[4]; /* X, psi, alpha*psi, beta */
  double seconds;
} or_cfc_report;

/* The xCFC solve order, Steps 1-6 of Sec. 2.6 (Step 4, the primitive
 * recovery, is replaced by the fixed sources the caller gives):
 *   1 X:   lap X + 1/3 grad div X = 8 pi S_i                          (eq. X)
 *   2 A~_ij from X                                                   (eq. Aij)
 *   3 psi: lap psi = -2 pi U psi^-1 - 1/8 A2 psi^-7                   (eq. psi)
 *   5 alpha psi: lap(a psi) = (a psi) [2 pi (U + 2 S) psi^-2 + 7/8 A2 psi^-8]
 *   6 beta: lap b + 1/3 grad div b = 16 pi a psi^-6 S_i
 *                                    + 2 A~_ij grad_j(a psi^-6)      (eq. beta)
 * Deviations delta = psi - 1 and alpha psi - 1 are the scalar unknowns, with
 * the Robin outer condition of eq. (robin); X and beta vanish at the outer
 * boundary (eq. bc).  Fields are interior arrays; psi, alpha, beta, X carry
 * the initial guess in and the solution out. */
/* Step 6 of Sec. 2.6: the right-hand side of eq. (beta),
 * 16 pi alpha psi^-6 S_i + 2 A~_ij grad_j(alpha psi^-6), from the interior
 * fields X[3], dpsi = psi - 1 and dap = alpha psi - 1.  s = alpha psi^-6 =
 * (alpha psi) psi^-7 is formed on the ghosted grid (Robin ghosts of the two
 * deviations), X with its Dirichlet ghosts. */
static void beta_rhs(const or_desc* d, double* const X[3], const double* dpsi, const double* dap,
                     double* const Si[3], double* const f[3]) {
  OGrid g;
  finest_grid(d, &g);
  double* gp = calloc(g.size, sizeof(double));
  double* ga = calloc(g.size, sizeof(double));
  double* sg = calloc(g.size, sizeof(double));
  load_interior(&g, gp, dpsi);
  load_interior(&g, ga, dap);
  fill_ghosts(&g, gp, BC_ROBIN, -1);
  fill_ghosts(&g, ga, BC_ROBIN, -1);
  for (long p = 0; p < g.size; ++p) sg[p] = (1.0 + ga[p]) / pow(1.0 + gp[p], 7);
  double* Xg[3];
  for (int c = 0; c < 3; ++c) {
    Xg[c] = calloc(g.size, sizeof(double));
    load_interior(&g, Xg[c], X[c]);
    fill_ghosts(&g, Xg[c], BC_DIRICHLET, c);
  }
  long q = 0;
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i, ++q) {
        double A[6], G[3];
        aij_at(&g, Xg, i, j, k, A);
        grad_phys(&g, sg, i, j, k, G);
        double sv = sg[IX(&g, i, j, k)];
        /* (A~ . grad s)_i with A~ symmetric: rows (0: A0 A3 A4), (1: A3 A1 A5), (2: A4 A5 A2) */
        double AG0 = A[0] * G[0] + A[3] * G[1] + A[4] * G[2];
        double AG1 = A[3] * G[0] + A[1] * G[1] + A[5] * G[2];
        double AG2 = A[4] * G[0] + A[5] * G[1] + A[2] * G[2];
        f[0][q] = 16.0 * OR_PI * sv * Si[0][q] + 2.0 * AG0;
        f[1][q] = 16.0 * OR_PI * sv * Si[1][q] + 2.0 * AG1;
        f[2][q] = 16.0 * OR_PI * sv * Si[2][q] + 2.0 * AG2;
      }
  for (int c = 0; c < 3; ++c) free(Xg[c]);
  free(gp);
  free(ga);
  free(sg);
}

/* Exported Step 6 (interior psi and alpha in): used by the tests to check
 * full-size GPU solutions against the discrete equations. */
void or_beta_rhs(const or_desc* d, double* const X[3], const double* psi, const double* alpha,
                 double* const Si[3], double* const f[3]) {
  long N = ncells(d);
  double* dpsi = calloc(N, sizeof(double));
  double* dap = calloc(N, sizeof(double));
  for (long q = 0; q < N; ++q) {
    dpsi[q] = psi[q] - 1.0;
    dap[q] = alpha[q] * psi[q] - 1.0;
  }
  beta_rhs(d, X, dpsi, dap, Si, f);
  free(dpsi);
  free(dap);
}

int or_solve_cfc(const or_desc* d, const double* U, const double* S, double* const Si[3],
                 double* psi, double* alpha, double* const beta[3], double* const X[3],
                 or_cfc_report* rep) {
  long N = ncells(d);
  OGrid g;
  finest_grid(d, &g);
  int status = 0;
  double* A2 = calloc(N, sizeof(double));
  double* f[3];
  for (int c = 0; c < 3; ++c) f[c] = calloc(N, sizeof(double));
  if (!rep->psi_only) {
    /* Step 1 */
    for (int c = 0; c < 3; ++c)
      for (long q = 0; q < N; ++q) f[c][q] = 8.0 * OR_PI * Si[c][q];
    status = or_solve_vector(d, BC_DIRICHLET, f, X, &rep->rep[0]);
    if (status) goto done;
    /* Step 2 */
    or_aij(d, X, NULL, A2);
  }
  /* Step 3 */
  double* dpsi = calloc(N, sizeof(double));
  for (long q = 0; q < N; ++q) dpsi[q] = psi[q] - 1.0;
  status = or_solve_scalar(d, EQ_PSI, BC_ROBIN, 0, U, A2, NULL, NULL, dpsi, &rep->rep[1]);
  for (long q = 0; q < N; ++q) psi[q] = 1.0 + dpsi[q];
  if (status || rep->psi_only) {
    free(dpsi);
    goto done;
  }
  /* Step 5 */
  {
    double* cf = calloc(N, sizeof(double));
    double* dap = calloc(N, sizeof(double));
    for (long q = 0; q < N; ++q) {
      double p = psi[q];
      cf[q] = 2.0 * OR_PI * (U[q] + 2.0 * S[q]) / (p * p) + 0.875 * A2[q] / pow(p, 8);
      dap[q] = alpha[q] * psi[q] - 1.0;
    }
    status = or_solve_scalar(d, EQ_LIN, BC_ROBIN, 0, NULL, NULL, cf, cf, dap, &rep->rep[2]);
    if (status) {
      for (long q = 0; q < N; ++q) alpha[q] = (1.0 + dap[q]) / psi[q];
      free(cf);
      free(dap);
      free(dpsi);
      goto done;
    }
    /* Step 6 */
    beta_rhs(d, X, dpsi, dap, Si, f);
    status = or_solve_vector(d, BC_DIRICHLET, f, beta, &rep->rep[3]);
    for (long q2 = 0; q2 < N; ++q2) alpha[q2] = (1.0 + dap[q2]) / psi[q2];
    free(cf);
    free(dap);
  }
  free(dpsi);
done:
  free(A2);
  for (int c = 0; c < 3; ++c) free(f[c]);
  return status;
}

/* -------------------------------------------------- divergence cleaning */

typedef struct {
  or_report solve;
  double max_div_before, l2_div_before, max_div_after, l2_div_after;
} or_divb_report;

/* Central divergence of B (physical components), (1/sqrt(g)) d_i (sqrt(g)
 * q^i) of Sec. 2.2 with sqrt(g) = 1, R, r^2 sin(theta), every factor taken
 * at the centre of the cell it multiplies:
 *   Cartesian   sum_d (B_d,+ - B_d,-) / (2 h_d)
 *   cylindrical (R+ B_R,+ - R- B_R,-) / (2 h_R R) + (B_z,+ - B_z,-) / (2 h_z)
 *               + (B_phi,+ - B_phi,-) / (2 h_phi R)
 *   spherical   (r+^2 B_r,+ - r-^2 B_r,-) / (2 h_r r^2)
 *               + (s+ B_th,+ - s- B_th,-) / (2 h_th r s)
 *               + (B_phi,+ - B_phi,-) / (2 h_phi r s),   s = sin(theta).
 * B ghosts: copies of the boundary cell on the outer faces (zero normal
 * gradient), the component parities across the origin / axis. */
static void div_c(const OGrid* g, double* const Bg[3], double* div) {
  for (int c = 0; c < g->ndim; ++c) fill_ghosts(g, Bg[c], BC_NEUMANN, g->geom == GEOM_CART ? -1 : c);
  long q = 0;
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i, ++q) {
        double s = 0.0;
        if (g->geom == GEOM_CART) {
          for (int c = 0; c < g->ndim; ++c) s += d1(g, Bg[c], c, i, j, k);
        } else {
          const double x = xc(g, 0, i), xp = xc(g, 0, i + 1), xm = xc(g, 0, i - 1);
          const double* B0 = Bg[0];
          const double* B1 = Bg[1];
          if (g->geom == GEOM_CYL) {
            s = (xp * B0[IX(g, i + 1, j, k)] - xm * B0[IX(g, i - 1, j, k)]) / (2.0 * g->h[0] * x) +
                (B1[IX(g, i, j + 1, k)] - B1[IX(g, i, j - 1, k)]) / (2.0 * g->h[1]);
            if (g->ndim == 3)
              s += (Bg[2][IX(g, i, j, k + 1)] - Bg[2][IX(g, i, j, k - 1)]) / (2.0 * g->h[2] * x);
          } else {
            const double st = sin(xc(g, 1, j)), sp = sin(xc(g, 1, j + 1)), sm = sin(xc(g, 1, j - 1));
            s = (xp * xp * B0[IX(g, i + 1, j, k)] - xm * xm * B0[IX(g, i - 1, j, k)]) / (2.0 * g->h[0] * x * x) +
                (sp * B1[IX(g, i, j + 1, k)] - sm * B1[IX(g, i, j - 1, k)]) / (2.0 * g->h[1] * x * st);
            if (g->ndim == 3)
              s += (Bg[2][IX(g, i, j, k + 1)] - Bg[2][IX(g, i, j, k - 1)]) / (2.0 * g->h[2] * x * st);
          }
        }
        div[q] = s;
      }
}

static void div_norms(const double* div, long N, double* mx, double* l2) {
  double m = 0.0, s = 0.0;
  for (long q = 0; q < N; ++q) {
    double a = fabs(div[q]);
    if (a > m) m = a;
    s += div[q] * div[q];
  }
  *mx = m;
  *l2 = sqrt(s / (double)N);
}

/* Elliptic divergence cleaning, eqs. (poisson) and (update_bfield):
 * b = div B - <div B>, the mean weighted by w = 1, R, r^2 sin(theta) (the
 * weights under which the flux-form Laplacian with Neumann ghosts sums to
 * zero, so that the Neumann problem is compatible); lap Phi = b with
 * Neumann outer ghosts, Phi's mean removed after every cycle; B <- B -
 * grad Phi (central, physical components).  B holds ndim (interior)
 * components, modified in place; phi (interior) out. */
int or_clean_divb(const or_desc* d, double* const B[3], double* phi, or_divb_report* rep) {
  OGrid g;
  finest_grid(d, &g);
  long N = ncells(d);
  double* Bg[3] = {NULL, NULL, NULL};
  for (int c = 0; c < d->ndim; ++c) {
    Bg[c] = calloc(g.size, sizeof(double));
    load_interior(&g, Bg[c], B[c]);
  }
  double* div = calloc(N, sizeof(double));
  div_c(&g, Bg, div);
  div_norms(div, N, &rep->max_div_before, &rep->l2_div_before);
  double sw = 0.0, swd = 0.0;
  {
    long q = 0;
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i, ++q) {
          const double w = norm_weight(&g, i, j);
          sw += w;
          swd += w * div[q];
        }
  }
  const double mean = swd / sw;
  for (long q = 0; q < N; ++q) div[q] -= mean;
  for (long q = 0; q < N; ++q) phi[q] = 0.0;
  int st = or_solve_scalar(d, EQ_LIN, BC_NEUMANN, 1, NULL, NULL, NULL, div, phi, &rep->solve);
  double* pg = calloc(g.size, sizeof(double));
  load_interior(&g, pg, phi);
  fill_ghosts(&g, pg, BC_NEUMANN, -1);
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        double G[3];
        grad_phys(&g, pg, i, j, k, G);
        for (int c = 0; c < d->ndim; ++c) Bg[c][IX(&g, i, j, k)] -= G[c];
      }
  div_c(&g, Bg, div);
  div_norms(div, N, &rep->max_div_after, &rep->l2_div_after);
  for (int c = 0; c < d->ndim; ++c) {
    store_interior(&g, B[c], Bg[c]);
    free(Bg[c]);
  }
  free(pg);
  free(div);
  return st;
}

/* Central divergence only (for tests / diagnostics). */
void or_div_c(const or_desc* d, double* const B[3], double* div) {
  OGrid g;
  finest_grid(d, &g);
  double* Bg[3] = {NULL, NULL, NULL};
  for (int c = 0; c < d->ndim; ++c) {
    Bg[c] = calloc(g.size, sizeof(double));
    load_interior(&g, Bg[c], B[c]);
  }
  div_c(&g, Bg, div);
  for (int c = 0; c < d->ndim; ++c) free(Bg[c]);
}

/* ------------------------------------ divergence cleaning, exact projection */

/* Exact-projection variant of the divergence cleaning on Cartesian grids
 * (not the paper's method: Sec. 2.2 eqs. (poisson) and (update_bfield) with
 * the compact Laplacian replaced by div_c grad_c, the operator the update
 * actually applies).
 *   grad_c Phi: central differences, the Phi ghost mirrored about the
 *     boundary cell's centre (Phi_{-1} = Phi_1, Phi_n = Phi_{n-2}), so the
 *     normal gradient vanishes in the boundary cells;
 *   div_c: central differences, ghosts of its argument copied from the
 *     boundary cell (the rule of B).
 * With these rules div_c grad_c restricted to one parity class of cells
 * (i mod 2, j mod 2, k mod 2) is the compact Laplacian of spacing 2 h with
 * copied (Neumann) ghosts, and classes do not couple: the solve splits into
 * 2^d compact Neumann problems of n/2 cells per dimension.  Each needs a
 * mean-free right-hand side: b = div_c B minus its mean over the class.
 * After B <- B - grad_c Phi, div_c B equals that class mean on every cell
 * of the class.  Each class is solved by the same multigrid (d's solver
 * settings, n/2 cells, spacing 2 h); rep->solve gets the largest cycle
 * count and residual over the classes and the worst status. */
int or_clean_divb_exact(const or_desc* d, double* const B[3], double* phi, or_divb_report* rep) {
  if (d->geom != GEOM_CART) return 1;
  OGrid g;
  finest_grid(d, &g);
  const long N = ncells(d);
  const int three = d->ndim == 3;
  const int nclass = three ? 8 : 4;
  double* Bg[3] = {NULL, NULL, NULL};
  for (int c = 0; c < d->ndim; ++c) {
    Bg[c] = calloc(g.size, sizeof(double));
    load_interior(&g, Bg[c], B[c]);
  }
  double* div = calloc(N, sizeof(double));
  div_c(&g, Bg, div);
  div_norms(div, N, &rep->max_div_before, &rep->l2_div_before);
  or_desc ds = *d;
  for (int a = 0; a < d->ndim; ++a) ds.n[a] = d->n[a] / 2;
  const int m0 = ds.n[0], m1 = ds.n[1], m2 = three ? ds.n[2] : 1;
  const long M = (long)m0 * m1 * m2;
  double* bs = calloc(M, sizeof(double));
  double* ps = calloc(M, sizeof(double));
  int status = 0;
  memset(&rep->solve, 0, sizeof(rep->solve));
  for (int s = 0; s < nclass; ++s) {
    const int pi = s & 1, pj = (s >> 1) & 1, pk = (s >> 2) & 1;
    /* gather the class (dimension 0 fastest) and remove its mean */
    double sum = 0.0;
    for (int k = 0; k < m2; ++k)
      for (int j = 0; j < m1; ++j)
        for (int i = 0; i < m0; ++i) {
          const int fi = 2 * i + pi, fj = 2 * j + pj, fk = three ? 2 * k + pk : 0;
          const double v = div[fi + (long)d->n[0] * (fj + (long)d->n[1] * fk)];
          bs[i + (long)m0 * (j + (long)m1 * k)] = v;
          sum += v;
        }
    const double mean = sum / (double)M;
    for (long q = 0; q < M; ++q) {
      bs[q] -= mean;
      ps[q] = 0.0;
    }
    or_report r;
    const int st = or_solve_scalar(&ds, EQ_LIN, BC_NEUMANN, 1, NULL, NULL, NULL, bs, ps, &r);
    if (st != 0 && status == 0) status = st;
    if (r.cycles > rep->solve.cycles) rep->solve.cycles = r.cycles;
    if (r.rel > rep->solve.rel || s == 0) rep->solve.rel = r.rel;
    for (int k = 0; k < m2; ++k)
      for (int j = 0; j < m1; ++j)
        for (int i = 0; i < m0; ++i) {
          const int fi = 2 * i + pi, fj = 2 * j + pj, fk = three ? 2 * k + pk : 0;
          phi[fi + (long)d->n[0] * (fj + (long)d->n[1] * fk)] = ps[i + (long)m0 * (j + (long)m1 * k)];
        }
  }
  rep->solve.status = status;
  /* Phi with mirrored ghosts, dimensions filled in the order 0, 1, 2 over
   * the ranges already extended */
  double* pg = calloc(g.size, sizeof(double));
  load_interior(&g, pg, phi);
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j) {
      pg[IX(&g, -1, j, k)] = pg[IX(&g, 1, j, k)];
      pg[IX(&g, n0, j, k)] = pg[IX(&g, n0 - 2, j, k)];
    }
  for (int k = 0; k < n2; ++k)
    for (int i = -1; i <= n0; ++i) {
      pg[IX(&g, i, -1, k)] = pg[IX(&g, i, 1, k)];
      pg[IX(&g, i, n1, k)] = pg[IX(&g, i, n1 - 2, k)];
    }
  if (three)
    for (int j = -1; j <= n1; ++j)
      for (int i = -1; i <= n0; ++i) {
        pg[IX(&g, i, j, -1)] = pg[IX(&g, i, j, 1)];
        pg[IX(&g, i, j, n2)] = pg[IX(&g, i, j, n2 - 2)];
      }
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        double G[3];
        grad_phys(&g, pg, i, j, k, G);
        for (int c = 0; c < d->ndim; ++c) Bg[c][IX(&g, i, j, k)] -= G[c];
      }
  div_c(&g, Bg, div);
  div_norms(div, N, &rep->max_div_after, &rep->l2_div_after);
  for (int c = 0; c < d->ndim; ++c) {
    store_interior(&g, B[c], Bg[c]);
    free(Bg[c]);
  }
  free(pg);
  free(bs);
  free(ps);
  free(div);
  return status;
}

/* ------------------------------------------ two-level composite grid (AMR) */

/* A two-level composite grid: the base grid (the hierarchy of d) and one
 * refined patch of ratio 2 over the box a <= I < b of base cells (the block
 * tree of Sec. 2.8 on one device: a box of whole blocks).  The paper's
 * multigrid on its block-AMR grids lives in the library it cites and is not
 * printed; the readings used here (each listed in the design notes):
 *   - composite cells: the patch's fine cells and the base cells it does not
 *     cover ("uncovered");
 *   - fine operator: the operator of Sec. 2.7.1 on the patch grid.  Patch
 *     faces on the domain boundary take the boundary rules; faces inside
 *     the domain take coarse-fine ghosts, quadratic in both directions:
 *     the base solution interpolated to the ghost's tangential position
 *     (second-order centred differences of the uncovered base cells around
 *     the parent, offsets +-h/4 per tangential dimension, with the cross
 *     term in 3D), then g = 8/15 u~ + 2/3 u_1 - 1/5 u_2 from it and the two
 *     patch cells inward (the quadratic through the points at -3/2, -1/2
 *     and +1 fine spacings from the interface, evaluated at +1/2);
 *   - coarse operator on an uncovered cell next to the patch: the flux of
 *     its face to the patch replaced by the sum of the fine fluxes through
 *     that face (area x difference, in the pseudo-volume form of the printed
 *     operators: V = 1 / r_i^2 sin(theta_j) / R_i x dx dy dz, areas from the
 *     face radii and sines), so the composite operator is conservative;
 *   - FAS across the two levels: restrict u and the residual of the patch
 *     to the cells it covers (volume-weighted, Sec. 2.7.3), right-hand side
 *     L_H(R u) + R r there and f + L_H(u) - L_comp(u) on uncovered cells,
 *     one FAS V-cycle of the base hierarchy, the Kwak prolongation of the
 *     base change onto the patch, smoothing of the patch before and after;
 *   - stopping rule: the weighted relative residual over the composite
 *     cells (w = r^2 sin(theta), R, 1 at each cell's own centre).
 * Scalar equations (eq. psi, linear equations) only. */

typedef struct {
  OSolver s;       /* base hierarchy */
  OGrid gp;        /* patch grid */
  int a[3], b[3];  /* patch box in base cells */
  OLevel P;        /* patch arrays (u, f, r, U, A2, c) */
  double* f0;      /* original right-hand side of the base grid */
  double* e;       /* scratch, base level 0 */
} OComp;

static int comp_covered(const OComp* C, int I, int J, int K) {
  const OGrid* g = &C->s.lev[0].g;
  if (I < C->a[0] || I >= C->b[0] || J < C->a[1] || J >= C->b[1]) return 0;
  if (g->ndim == 3 && (K < C->a[2] || K >= C->b[2])) return 0;
  return 1;
}

/* Pseudo volume of a cell and area of its face on side sd (+-1) along dim
 * d, in the form the printed operators take when multiplied by the volume
 * (dims absent in 2D drop out). */
static double comp_volume(const OGrid* g, int i, int j) {
  double v = g->h[0] * g->h[1] * (g->ndim == 3 ? g->h[2] : 1.0);
  if (g->geom == GEOM_CYL) v *= xc(g, 0, i);
  if (g->geom == GEOM_SPH) v *= xc(g, 0, i) * xc(g, 0, i) * sin(xc(g, 1, j));
  return v;
}
static double comp_area(const OGrid* g, int d, int sd, int i, int j) {
  const double h2 = g->ndim == 3 ? g->h[2] : 1.0;
  if (g->geom == GEOM_CART) return g->h[0] * g->h[1] * h2 / g->h[d];
  if (g->geom == GEOM_CYL) {
    if (d == 0) return xf(g, 0, sd > 0 ? i + 1 : i) * g->h[1] * h2;
    if (d == 1) return xc(g, 0, i) * g->h[0] * h2;
    return g->h[0] * g->h[1] / xc(g, 0, i);
  }
  if (d == 0) {
    const double rf = xf(g, 0, sd > 0 ? i + 1 : i);
    return rf * rf * sin(xc(g, 1, j)) * g->h[1] * h2;
  }
  if (d == 1) return sin_face(g, sd > 0 ? j + 1 : j) * g->h[0] * h2;
  return g->h[0] * g->h[1] / sin(xc(g, 1, j));
}

/* Base solution interpolated to the tangential position of a patch ghost:
 * parent base cell P (its index along d is outside the patch), offsets
 * dt = +-1/4 base spacing per tangential dimension (0 along d). */
static double comp_tangential(const OComp* C, const double* uc, int d, const int P[3], const double dt[3]) {
  const OGrid* g = &C->s.lev[0].g;
  const int nd = g->ndim;
  double v = uc[IX(g, P[0], P[1], P[2])];
  int tt[2], nt = 0;
  for (int t = 0; t < nd; ++t)
    if (t != d) tt[nt++] = t;
  for (int q = 0; q < nt; ++q) {
    const int t = tt[q];
    int Pp[3] = {P[0], P[1], P[2]}, Pm[3] = {P[0], P[1], P[2]};
    Pp[t] += 1;
    Pm[t] -= 1;
    const double up = uc[IX(g, Pp[0], Pp[1], Pp[2])], um = uc[IX(g, Pm[0], Pm[1], Pm[2])];
    v += dt[t] * 0.5 * (up - um) + 0.5 * dt[t] * dt[t] * (up - 2.0 * uc[IX(g, P[0], P[1], P[2])] + um);
  }
  if (nt == 2) {
    const int t1 = tt[0], t2 = tt[1];
    int q1[3], q2[3], q3[3], q4[3];
    for (int x = 0; x < 3; ++x) q1[x] = q2[x] = q3[x] = q4[x] = P[x];
    q1[t1] += 1; q1[t2] += 1;
    q2[t1] += 1; q2[t2] -= 1;
    q3[t1] -= 1; q3[t2] += 1;
    q4[t1] -= 1; q4[t2] -= 1;
    const double mix = 0.25 * (uc[IX(g, q1[0], q1[1], q1[2])] - uc[IX(g, q2[0], q2[1], q2[2])] -
                               uc[IX(g, q3[0], q3[1], q3[2])] + uc[IX(g, q4[0], q4[1], q4[2])]);
    v += dt[t1] * dt[t2] * mix;
  }
  return v;
}

/* Is face (d, side) of the patch a coarse-fine interface (else it lies on
 * the domain boundary)? */
static int comp_cf_face(const OComp* C, int d, int side) {
  const OGrid* g = &C->s.lev[0].g;
  return side < 0 ? C->a[d] > 0 : C->b[d] < g->n[d];
}

/* Fill the patch ghosts of up: boundary rules on faces on the domain
 * boundary, coarse-fine ghosts from the base solution uc (ghosts filled)
 * on the others. */
static void comp_fill_patch(const OComp* C, double* up, const double* uc) {
  const OGrid* gp = &C->gp;
  const int nd = gp->ndim;
  fill_ghosts(gp, up, C->s.bc, -1);
  for (int d = 0; d < nd; ++d)
    for (int side = -1; side <= 1; side += 2) {
      if (!comp_cf_face(C, d, side)) continue;
      const int n0 = gp->n[0], n1 = gp->n[1], n2 = gp->n[2];
      for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
          for (int i = 0; i < n0; ++i) {
            const int idx[3] = {i, j, k};
            const int edge = side < 0 ? 0 : gp->n[d] - 1;
            if (idx[d] != edge) continue;
            int g3[3] = {i, j, k}, u1[3] = {i, j, k}, u2[3] = {i, j, k}, P[3];
            g3[d] = side < 0 ? -1 : gp->n[d];
            u2[d] = side < 0 ? 1 : gp->n[d] - 2;
            double dt[3] = {0.0, 0.0, 0.0};
            for (int t = 0; t < 3; ++t) {
              if (t >= nd) {
                P[t] = 0;
                continue;
              }
              if (t == d) {
                P[t] = side < 0 ? C->a[d] - 1 : C->b[d];
              } else {
                P[t] = C->a[t] + idx[t] / 2;
                dt[t] = (idx[t] % 2 == 0) ? -0.25 : 0.25;
              }
            }
            const double ut = comp_tangential(C, uc, d, P, dt);
            up[IX(gp, g3[0], g3[1], g3[2])] = (8.0 / 15.0) * ut + (2.0 / 3.0) * up[IX(gp, u1[0], u1[1], u1[2])] -
                                             (1.0 / 5.0) * up[IX(gp, u2[0], u2[1], u2[2])];
          }
    }
}

/* The composite operator minus the base operator on the uncovered base
 * cells next to the patch (the fine fluxes through their face to the patch
 * in place of the coarse one), added into corr (base ghosted layout); the
 * patch ghosts of up must be current. */
static void comp_flux_correction(const OComp* C, const double* up, const double* uc, double* corr) {
  const OGrid* g = &C->s.lev[0].g;
  const OGrid* gp = &C->gp;
  const int nd = g->ndim;
  memset(corr, 0, sizeof(double) * g->size);
  for (int d = 0; d < nd; ++d)
    for (int side = -1; side <= 1; side += 2) {
      if (!comp_cf_face(C, d, side)) continue;
      /* coarse cells just outside this face of the patch: the box's range
       * in the tangential dimensions, one index along d */
      int rlo[3], rhi[3];
      for (int t = 0; t < 3; ++t) {
        rlo[t] = (t < nd && t != d) ? C->a[t] : 0;
        rhi[t] = (t < nd && t != d) ? C->b[t] : 1;
      }
      for (int K = rlo[2]; K < rhi[2]; ++K)
        for (int J = rlo[1]; J < rhi[1]; ++J)
          for (int I = rlo[0]; I < rhi[0]; ++I) {
            int Q[3] = {I, J, K};
            Q[d] = side < 0 ? C->a[d] - 1 : C->b[d];   /* the uncovered cell */
            int Qin[3] = {Q[0], Q[1], Q[2]};
            Qin[d] = side < 0 ? C->a[d] : C->b[d] - 1;   /* its covered neighbour */
            /* the coarse flux out of Q through this face (toward the patch) */
            const int sd = side < 0 ? 1 : -1;             /* the face is on Q's side sd */
            const double Ac = comp_area(g, d, sd, Q[0], Q[1]);
            const double Dc = (uc[IX(g, Qin[0], Qin[1], Qin[2])] - uc[IX(g, Q[0], Q[1], Q[2])]) / g->h[d];
            /* the fine fluxes through the same face */
            double fsum = 0.0;
            const int nf1 = nd == 3 ? 2 : 1;
            for (int q2 = 0; q2 < nf1; ++q2)
              for (int q1 = 0; q1 < 2; ++q1) {
                int f[3];
                int tq = 0;
                for (int t = 0; t < 3; ++t) {
                  if (t >= nd) {
                    f[t] = 0;
                  } else if (t == d) {
                    f[t] = side < 0 ? 0 : gp->n[d] - 1;
                  } else {
                    f[t] = 2 * (Q[t] - C->a[t]) + (tq == 0 ? q1 : q2);
                    ++tq;
                  }
                }
                int gg[3] = {f[0], f[1], f[2]};
                gg[d] = side < 0 ? -1 : gp->n[d];
                const double Af = comp_area(gp, d, side, f[0], f[1]);
                const double Df = (up[IX(gp, f[0], f[1], f[2])] - up[IX(gp, gg[0], gg[1], gg[2])]) / gp->h[d];
                fsum += Af * Df;
              }
            corr[IX(g, Q[0], Q[1], Q[2])] += (fsum - Ac * Dc) / comp_volume(g, Q[0], Q[1]);
          }
    }
}

/* One red-black Newton-Gauss-Seidel sweep of the patch (eq. ngs_iteration),
 * the patch ghosts refilled from the current patch and base values before
 * each colour (the Newton diagonal holds them fixed). */
static void comp_patch_sweep(OComp* C) {
  const OGrid* gp = &C->gp;
  const double* uc = C->s.lev[0].u[0];
  for (int colour = 0; colour < 2; ++colour) {
    comp_fill_patch(C, C->P.u[0], uc);
    for (int k = 0; k < gp->n[2]; ++k)
      for (int j = 0; j < gp->n[1]; ++j)
        for (int i = 0; i < gp->n[0]; ++i) {
          if (((i + j + k) & 1) != colour) continue;
          double diag;
          const double Lu = op_at(&C->s, &C->P, 0, i, j, k, &diag);
          const long p = IX(gp, i, j, k);
          C->P.u[0][p] = C->P.u[0][p] - (Lu - C->P.f[0][p]) / diag;
        }
  }
}

/* Source S(u) of the equation at a cell (the right-hand side as the paper
 * writes it), with the original right-hand side f. */
static double comp_source(const OComp* C, const OLevel* L, long p, double f) {
  if (C->s.kind == EQ_PSI) {
    const double psi = 1.0 + L->u[0][p];
    return -2.0 * OR_PI * L->U[p] / psi - 0.125 * L->A2[p] / pow(psi, 7);
  }
  return (L->c ? L->c[p] * L->u[0][p] : 0.0) + f;
}

/* Base ghosts, patch ghosts and the flux correction at the current state
 * (into C->e). */
static void comp_refresh(OComp* C) {
  OLevel* B = &C->s.lev[0];
  fill_ghosts(&B->g, B->u[0], C->s.bc, -1);
  comp_fill_patch(C, C->P.u[0], B->u[0]);
  comp_flux_correction(C, C->P.u[0], B->u[0], C->e);
}

/* Relative weighted residual over the composite cells (stopping rule). */
static double comp_rel(OComp* C) {
  OLevel* B = &C->s.lev[0];
  const OGrid* g = &B->g;
  const OGrid* gp = &C->gp;
  comp_refresh(C);
  double num = 0.0, den = 0.0;
  for (int k = 0; k < gp->n[2]; ++k)
    for (int j = 0; j < gp->n[1]; ++j)
      for (int i = 0; i < gp->n[0]; ++i) {
        const long p = IX(gp, i, j, k);
        const double w = norm_weight(gp, i, j);
        const double r = C->P.f[0][p] - op_at(&C->s, &C->P, 0, i, j, k, NULL);
        const double S = comp_source(C, &C->P, p, C->P.f[0][p]);
        if (r != r || S != S) return NAN;
        if (fabs(w * r) > num) num = fabs(w * r);
        if (fabs(w * S) > den) den = fabs(w * S);
      }
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) {
        if (comp_covered(C, i, j, k)) continue;
        const long p = IX(g, i, j, k);
        const double w = norm_weight(g, i, j);
        const double r = C->f0[p] - op_at(&C->s, B, 0, i, j, k, NULL) - C->e[p];
        const double S = comp_source(C, B, p, C->f0[p]);
        if (r != r || S != S) return NAN;
        if (fabs(w * r) > num) num = fabs(w * r);
        if (fabs(w * S) > den) den = fabs(w * S);
      }
  return num / (den > 1e-300 ? den : 1e-300);
}

/* One composite FAS V(nu1, nu2) cycle (the readings above). */
static void comp_cycle(OComp* C) {
  OSolver* s = &C->s;
  OLevel* B = &s->lev[0];
  const OGrid* g = &B->g;
  const OGrid* gp = &C->gp;
  const int three = g->ndim == 3;
  for (int it = 0; it < s->nu1; ++it) comp_patch_sweep(C);
  /* patch residual */
  comp_fill_patch(C, C->P.u[0], B->u[0]);
  for (int k = 0; k < gp->n[2]; ++k)
    for (int j = 0; j < gp->n[1]; ++j)
      for (int i = 0; i < gp->n[0]; ++i) {
        const long p = IX(gp, i, j, k);
        C->P.r[0][p] = C->P.f[0][p] - op_at(s, &C->P, 0, i, j, k, NULL);
      }
  /* restriction to the covered cells (volume-weighted children); R r kept
   * in the base residual array */
  for (int K = 0; K < g->n[2]; ++K)
    for (int J = 0; J < g->n[1]; ++J)
      for (int I = 0; I < g->n[0]; ++I) {
        if (!comp_covered(C, I, J, K)) continue;
        double su = 0.0, sr = 0.0, vol = 0.0;
        for (int dk = 0; dk <= three; ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
              const int fi = 2 * (I - C->a[0]) + di, fj = 2 * (J - C->a[1]) + dj;
              const int fk = three ? 2 * (K - C->a[2]) + dk : 0;
              const double v = cell_volume(gp, fi, fj);
              su += v * C->P.u[0][IX(gp, fi, fj, fk)];
              sr += v * C->P.r[0][IX(gp, fi, fj, fk)];
              vol += v;
            }
        B->u[0][IX(g, I, J, K)] = su / vol;
        B->r[0][IX(g, I, J, K)] = sr / vol;
      }
  memcpy(B->uh[0], B->u[0], sizeof(double) * g->size);
  /* FAS right-hand side of the base level */
  comp_refresh(C);
  for (int K = 0; K < g->n[2]; ++K)
    for (int J = 0; J < g->n[1]; ++J)
      for (int I = 0; I < g->n[0]; ++I) {
        const long p = IX(g, I, J, K);
        if (comp_covered(C, I, J, K))
          B->f[0][p] = op_at(s, B, 0, I, J, K, NULL) + B->r[0][p];
        else
          B->f[0][p] = C->f0[p] - C->e[p];
      }
  /* one FAS V-cycle of the base hierarchy */
  vcycle(s, s, 0);
  /* the base change onto the patch (Kwak), homogeneous ghosts */
  for (long p = 0; p < g->size; ++p) C->e[p] = B->u[0][p] - B->uh[0][p];
  fill_ghosts(g, C->e, s->bc, -1);
  for (int k = 0; k < gp->n[2]; ++k)
    for (int j = 0; j < gp->n[1]; ++j)
      for (int i = 0; i < gp->n[0]; ++i) {
        const int I = C->a[0] + i / 2, J = C->a[1] + j / 2, K = three ? C->a[2] + k / 2 : 0;
        const int si = (i % 2 == 0) ? -1 : 1, sj = (j % 2 == 0) ? -1 : 1, sk = (k % 2 == 0) ? -1 : 1;
        const double ec = C->e[IX(g, I, J, K)];
        const double ex = C->e[IX(g, I + si, J, K)], ey = C->e[IX(g, I, J + sj, K)];
        double add;
        if (three)
          add = 0.25 * (ec + ex + ey + C->e[IX(g, I, J, K + sk)]);
        else
          add = 0.25 * (2.0 * ec + ex + ey);
        C->P.u[0][IX(gp, i, j, k)] += add;
      }
  for (int it = 0; it < s->nu2; ++it) comp_patch_sweep(C);
}

/* Composite unknowns (patch cells, then uncovered base cells) <-> a flat
 * vector. */
static long comp_nv(const OComp* C) {
  const OGrid* g = &C->s.lev[0].g;
  long n = (long)C->gp.n[0] * C->gp.n[1] * C->gp.n[2];
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) n += !comp_covered(C, i, j, k);
  return n;
}
static void comp_gather(const OComp* C, double* x) {
  const OGrid* g = &C->s.lev[0].g;
  const OGrid* gp = &C->gp;
  long q = 0;
  for (int k = 0; k < gp->n[2]; ++k)
    for (int j = 0; j < gp->n[1]; ++j)
      for (int i = 0; i < gp->n[0]; ++i) x[q++] = C->P.u[0][IX(gp, i, j, k)];
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i)
        if (!comp_covered(C, i, j, k)) x[q++] = C->s.lev[0].u[0][IX(g, i, j, k)];
}
static void comp_scatter(OComp* C, const double* x) {
  const OGrid* g = &C->s.lev[0].g;
  const OGrid* gp = &C->gp;
  long q = 0;
  for (int k = 0; k < gp->n[2]; ++k)
    for (int j = 0; j < gp->n[1]; ++j)
      for (int i = 0; i < gp->n[0]; ++i) C->P.u[0][IX(gp, i, j, k)] = x[q++];
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i)
        if (!comp_covered(C, i, j, k)) C->s.lev[0].u[0][IX(g, i, j, k)] = x[q++];
}

/* Cycle control of the composite iteration: the rule of run_cycles (tol,
 * max_cycles, stall window, non-finite values, optional Anderson mixing of
 * depth accel over the composite unknowns). */
static int comp_run_cycles(OComp* C, or_report* rep) {
  OSolver* s = &C->s;
  double rel = comp_rel(C);
  int cyc = 0, status = 0;
  double hist[OR_HIST];
  int nh = 0;
  hist[nh++] = rel;
  const int m = s->accel < 0 ? 0 : (s->accel > 32 ? 32 : s->accel);
  const long nv = comp_nv(C);
  double *x = NULL, *g = NULL, *fcur = NULL, *fprev = NULL, *gprev = NULL, *dF = NULL, *dG = NULL;
  int ncol = 0, head = 0;
  if (m > 0) {
    x = malloc(sizeof(double) * nv);
    g = malloc(sizeof(double) * nv);
    fcur = malloc(sizeof(double) * nv);
    fprev = malloc(sizeof(double) * nv);
    gprev = malloc(sizeof(double) * nv);
    dF = malloc(sizeof(double) * nv * m);
    dG = malloc(sizeof(double) * nv * m);
  }
  while (1) {
    if (rel != rel) { status = 5; break; }
    if (rel <= s->tol) break;
    if (cyc >= s->max_cycles) { status = 3; break; }
    if (s->stall_window > 0 && cyc >= s->stall_window && rel > 0.95 * hist[cyc - s->stall_window]) {
      status = 4;
      break;
    }
    if (m == 0) {
      comp_cycle(C);
    } else {
      comp_gather(C, x);
      comp_cycle(C);
      comp_gather(C, g);
      for (long q = 0; q < nv; ++q) fcur[q] = g[q] - x[q];
      if (cyc > 0) {
        double* cf = dF + (long)head * nv;
        double* cg = dG + (long)head * nv;
        for (long q = 0; q < nv; ++q) {
          cf[q] = fcur[q] - fprev[q];
          cg[q] = g[q] - gprev[q];
        }
        head = (head + 1) % m;
        if (ncol < m) ++ncol;
      }
      memcpy(fprev, fcur, sizeof(double) * nv);
      memcpy(gprev, g, sizeof(double) * nv);
      if (ncol > 0) {
        double M[32 * 32], b[32], gam[32];
        int col[32];
        for (int a = 0; a < ncol; ++a) col[a] = (head - ncol + a + m) % m;
        for (int a = 0; a < ncol; ++a) {
          const double* fa = dF + (long)col[a] * nv;
          double sb = 0.0;
          for (long q = 0; q < nv; ++q) sb += fa[q] * fcur[q];
          b[a] = sb;
          for (int c2 = 0; c2 <= a; ++c2) {
            const double* fc = dF + (long)col[c2] * nv;
            double sm = 0.0;
            for (long q = 0; q < nv; ++q) sm += fa[q] * fc[q];
            M[a * ncol + c2] = sm;
            M[c2 * ncol + a] = sm;
          }
        }
        if (small_spd_solve(ncol, M, b, gam) == 0) {
          for (int a = 0; a < ncol; ++a) {
            const double* ga = dG + (long)col[a] * nv;
            for (long q = 0; q < nv; ++q) g[q] -= gam[a] * ga[q];
          }
        } else {
          ncol = 0;
        }
      }
      comp_scatter(C, g);
    }
    ++cyc;
    rel = comp_rel(C);
    if (nh < OR_HIST) hist[nh++] = rel;
  }
  free(x);
  free(g);
  free(fcur);
  free(fprev);
  free(gprev);
  free(dF);
  free(dG);
  if (rep) {
    rep->status = status;
    rep->cycles = cyc;
    rep->rel = rel;
    rep->nhist = nh;
    memcpy(rep->hist, hist, sizeof(double) * nh);
  }
  return status;
}

/* Set up a composite grid: the base hierarchy of d, the patch over base
 * cells a <= I < b.  Returns 0, or 1 if the box is not inside the grid, is
 * empty, or does not span the whole angular range where a rule across the
 * origin or axis needs it (spherical: theta and phi; cylindrical: phi). */
static int comp_setup(OComp* C, const or_desc* d, const int a[3], const int b[3], int kind, int bc) {
  memset(C, 0, sizeof(*C));
  const int nd = d->ndim;
  for (int t = 0; t < 3; ++t) {
    C->a[t] = t < nd ? a[t] : 0;
    C->b[t] = t < nd ? b[t] : 1;
    if (t < nd && !(0 <= a[t] && a[t] < b[t] && b[t] <= d->n[t])) return 1;
  }
  if (d->geom == GEOM_SPH && (C->a[1] != 0 || C->b[1] != d->n[1])) return 1;
  if (d->geom != GEOM_CART && nd == 3 && (C->a[2] != 0 || C->b[2] != d->n[2])) return 1;
  setup(&C->s, d, kind, bc, 1);
  const OGrid* g = &C->s.lev[0].g;
  int np[3];
  double lop[3], hp[3];
  for (int t = 0; t < 3; ++t) {
    np[t] = t < nd ? 2 * (C->b[t] - C->a[t]) : 1;
    lop[t] = t < nd ? g->lo[t] + C->a[t] * g->h[t] : g->lo[t];
    hp[t] = t < nd ? 0.5 * g->h[t] : g->h[t];
  }
  grid_init(&C->gp, nd, d->geom, np, lop, hp);
  const long sz = C->gp.size;
  C->P.g = C->gp;
  C->P.u[0] = calloc(sz, sizeof(double));
  C->P.f[0] = calloc(sz, sizeof(double));
  C->P.r[0] = calloc(sz, sizeof(double));
  C->P.U = calloc(sz, sizeof(double));
  C->P.A2 = calloc(sz, sizeof(double));
  C->P.c = calloc(sz, sizeof(double));
  C->f0 = calloc(g->size, sizeof(double));
  C->e = calloc(g->size, sizeof(double));
  return 0;
}

static void comp_free(OComp* C) {
  free(C->P.u[0]);
  free(C->P.f[0]);
  free(C->P.r[0]);
  free(C->P.U);
  free(C->P.A2);
  free(C->P.c);
  free(C->f0);
  free(C->e);
  free_levels(&C->s);
}

static void comp_load(OComp* C, const double* U, const double* A2, const double* c, const double* f,
                      const double* Up, const double* A2p, const double* cp, const double* fp, const double* u,
                      const double* up) {
  OLevel* B = &C->s.lev[0];
  if (U) load_interior(&B->g, B->U, U);
  if (A2) load_interior(&B->g, B->A2, A2);
  if (c) load_interior(&B->g, B->c, c);
  if (f) load_interior(&B->g, C->f0, f);
  load_interior(&B->g, B->u[0], u);
  if (Up) load_interior(&C->gp, C->P.U, Up);
  if (A2p) load_interior(&C->gp, C->P.A2, A2p);
  if (cp) load_interior(&C->gp, C->P.c, cp);
  if (fp) load_interior(&C->gp, C->P.f[0], fp);
  load_interior(&C->gp, C->P.u[0], up);
  restrict_sources(&C->s);
}

/* Composite solve of a scalar equation (kind EQ_PSI with U, A2; EQ_LIN with
 * c (nullable) and f) on the base grid of d and the patch a <= I < b.
 * Base-grid and patch arrays are interior layout (the patch has 2 (b - a)
 * cells per dimension); u and up: initial guess in, solution out (covered
 * base cells receive the restriction of the patch). */
int or_solve_scalar_amr(const or_desc* d, const int a[3], const int b[3], int kind, int bc, const double* U,
                        const double* A2, const double* c, const double* f, const double* Up, const double* A2p,
                        const double* cp, const double* fp, double* u, double* up, or_report* rep) {
  OComp C;
  if (comp_setup(&C, d, a, b, kind, bc)) return 1;
  comp_load(&C, U, A2, c, f, Up, A2p, cp, fp, u, up);
  const int st = comp_run_cycles(&C, rep);
  OLevel* B = &C.s.lev[0];
  const OGrid* g = &B->g;
  const int three = g->ndim == 3;
  /* covered base cells: the volume-weighted restriction of the patch */
  for (int K = 0; K < g->n[2]; ++K)
    for (int J = 0; J < g->n[1]; ++J)
      for (int I = 0; I < g->n[0]; ++I) {
        if (!comp_covered(&C, I, J, K)) continue;
        double su = 0.0, vol = 0.0;
        for (int dk = 0; dk <= three; ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
              const int fi = 2 * (I - C.a[0]) + di, fj = 2 * (J - C.a[1]) + dj;
              const int fk = three ? 2 * (K - C.a[2]) + dk : 0;
              const double v = cell_volume(&C.gp, fi, fj);
              su += v * C.P.u[0][IX(&C.gp, fi, fj, fk)];
              vol += v;
            }
        B->u[0][IX(g, I, J, K)] = su / vol;
      }
  store_interior(g, u, B->u[0]);
  store_interior(&C.gp, up, C.P.u[0]);
  comp_free(&C);
  return st;
}

/* The composite operator applied to (u, up) (interior layout, sources as in
 * or_solve_scalar_amr): out on the uncovered base cells (0 on covered ones),
 * outp on the patch cells. */
int or_apply_amr(const or_desc* d, const int a[3], const int b[3], int kind, int bc, const double* U,
                 const double* A2, const double* c, const double* Up, const double* A2p, const double* cp,
                 const double* u, const double* up, double* out, double* outp) {
  OComp C;
  if (comp_setup(&C, d, a, b, kind, bc)) return 1;
  comp_load(&C, U, A2, c, NULL, Up, A2p, cp, NULL, u, up);
  comp_refresh(&C);
  OLevel* B = &C.s.lev[0];
  const OGrid* g = &B->g;
  long q = 0;
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i, ++q)
        out[q] = comp_covered(&C, i, j, k) ? 0.0 : op_at(&C.s, B, 0, i, j, k, NULL) + C.e[IX(g, i, j, k)];
  q = 0;
  for (int k = 0; k < C.gp.n[2]; ++k)
    for (int j = 0; j < C.gp.n[1]; ++j)
      for (int i = 0; i < C.gp.n[0]; ++i, ++q) outp[q] = op_at(&C.s, &C.P, 0, i, j, k, NULL);
  comp_free(&C);
  return 0;
}
