/*
 * smg_oracle.c -- plain, slow, single-threaded FP64 reference of the StructMG
 * hot path (arXiv 2506.21932): stencil Galerkin coarsening with the vertex,
 * cell-centred and x-y semi-coarsening transfer pairs, dependence-preserving
 * Gauss-Seidel, ILU(0) and line (z) Gauss-Seidel smoothers, V-cycle, PCG /
 * flexible PCG / FGMRES.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no source with the CUDA library; every routine below is a
 * direct transcription of a definition or of the paper's algorithm steps, with no
 * blocking, fusion or reordering beyond what the definition states.
 *
 * Conventions (paper Sec. 4.1, SG-DIA format; Sec. 4.3, Eq. 5-10 for offsets):
 *   grid point (i,j,k), 0 <= i < nx (slowest), 0 <= k < nz (fastest),
 *   linear index p = (i*ny + j)*nz + k;
 *   a structured matrix stores, for every point, one coefficient (or one BxB
 *   block) per stencil offset o in {-1,0,1}^3: A[((p*ns + e)*B + r)*B + c];
 *   coefficients whose neighbour falls off the grid are zero (padding).
 * Floating point: compiled with -O2 -ffp-contract=off, so every a*b+c rounds twice.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EBREAKDOWN 4
#define ORC_ENOTCONV 5
#define ORC_ENAN 6

/* ------------------------------------------------------------------------- */
/* grid helpers                                                              */
/* ------------------------------------------------------------------------- */

static long npts(const int d[3]) { return (long)d[0] * d[1] * d[2]; }

static int inside(const int d[3], int i, int j, int k) {
  return i >= 0 && i < d[0] && j >= 0 && j < d[1] && k >= 0 && k < d[2];
}

static long pidx(const int d[3], int i, int j, int k) { return ((long)i * d[1] + j) * d[2] + k; }

/* index of offset (dx,dy,dz) in the stencil list, or -1 */
static int find_off(int ns, const int* off, int dx, int dy, int dz) {
  for (int e = 0; e < ns; ++e)
    if (off[3 * e] == dx && off[3 * e + 1] == dy && off[3 * e + 2] == dz) return e;
  return -1;
}

/* Mask rules of Sec. 4.2: offsets in {-1,0,1}^3,
 * no duplicates, the centre present; we additionally require structural symmetry
 * (o in mask <=> -o in mask), which every pattern the paper lists satisfies. */
int orc_mask_validate(int ns, const int* off) {
  if (ns < 1 || ns > 27) return ORC_EINVAL;
  for (int e = 0; e < ns; ++e) {
    for (int t = 0; t < 3; ++t)
      if (off[3 * e + t] < -1 || off[3 * e + t] > 1) return ORC_EINVAL;
    for (int f = 0; f < e; ++f)
      if (off[3 * e] == off[3 * f] && off[3 * e + 1] == off[3 * f + 1] && off[3 * e + 2] == off[3 * f + 2])
        return ORC_EINVAL;
    if (find_off(ns, off, -off[3 * e], -off[3 * e + 1], -off[3 * e + 2]) < 0) return ORC_EINVAL;
  }
  if (find_off(ns, off, 0, 0, 0) < 0) return ORC_EINVAL;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* SpMV and residual (Sec. 6.1.1: r = b - A u over the stencil)              */
/* ------------------------------------------------------------------------- */

/* y = A x, summed over stencil entries in list order; block entries act as BxB
 * matrices on the B unknowns of the neighbour. */
void orc_spmv(const int d[3], int ns, const int* off, int B, const double* A, const double* x, double* y) {
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j)
      for (int k = 0; k < d[2]; ++k) {
        long p = pidx(d, i, j, k);
        for (int r = 0; r < B; ++r) {
          double s = 0.0;
          for (int e = 0; e < ns; ++e) {
            int a = i + off[3 * e], b = j + off[3 * e + 1], c = k + off[3 * e + 2];
            if (!inside(d, a, b, c)) continue;
            long q = pidx(d, a, b, c);
            for (int cc = 0; cc < B; ++cc) s += A[((p * ns + e) * B + r) * B + cc] * x[q * B + cc];
          }
          y[p * B + r] = s;
        }
      }
}

void orc_residual(const int d[3], int ns, const int* off, int B, const double* A, const double* b, const double* x,
                  double* r) {
  long n = npts(d) * B;
  double* ax = (double*)malloc(sizeof(double) * (n ? n : 1));
  orc_spmv(d, ns, off, B, A, x, ax);
  for (long t = 0; t < n; ++t) r[t] = b[t] - ax[t];
  free(ax);
}

/* ------------------------------------------------------------------------- */
/* Diagonal (block) inverses used by Gauss-Seidel                            */
/* ------------------------------------------------------------------------- */

/* Gauss-Jordan inverse of a small dense n x n matrix with partial pivoting.
 * Returns nonzero if a pivot is exactly zero. */
static int dense_inverse(int n, const double* M, double* Minv) {
  double* W = (double*)malloc(sizeof(double) * n * 2 * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) W[r * 2 * n + c] = c < n ? M[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(W[r * 2 * n + col]) > fabs(W[piv * 2 * n + col])) piv = r;
    if (W[piv * 2 * n + col] == 0.0) { free(W); return 1; }
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) {
        double t = W[col * 2 * n + c]; W[col * 2 * n + c] = W[piv * 2 * n + c]; W[piv * 2 * n + c] = t;
      }
    double inv = 1.0 / W[col * 2 * n + col];
    for (int c = 0; c < 2 * n; ++c) W[col * 2 * n + c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = W[r * 2 * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * n; ++c) W[r * 2 * n + c] -= f * W[col * 2 * n + c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Minv[r * n + c] = W[r * 2 * n + n + c];
  free(W);
  return 0;
}

/* Dinv[p] = inverse of the diagonal entry (scalar: 1/a_pp; block: BxB inverse). */
int orc_diag_inverse(const int d[3], int ns, const int* off, int B, const double* A, double* Dinv) {
  int ec = find_off(ns, off, 0, 0, 0);
  long n = npts(d);
  for (long p = 0; p < n; ++p) {
    const double* D = A + (p * ns + ec) * B * B;
    if (B == 1) {
      if (D[0] == 0.0) return ORC_EBREAKDOWN;
      Dinv[p] = 1.0 / D[0];
    } else if (dense_inverse(B, D, Dinv + p * B * B)) {
      return ORC_EBREAKDOWN;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Gauss-Seidel (Sec. 4.4, GS-Forward / GS-Backward formulas, weight w)      */
/* ------------------------------------------------------------------------- */

/* One point update of u <- u + w (D + wL)^{-1}(b - A u) written row by row:
 * the new value is (1-w) u_p + w D_p^{-1}(b_p - sum_{o != 0} a_{p,o} u_{p+o}),
 * with neighbours earlier in the sweep already holding new values.  For w == 1
 * the blend is skipped, so the update is exactly D_p^{-1}(b_p - sum ...). */
static void gs_point(const int d[3], int ns, const int* off, int B, const double* A, const double* Dinv,
                     const double* b, double* u, double w, int i, int j, int k) {
  long p = pidx(d, i, j, k);
  double s[3];
  for (int r = 0; r < B; ++r) {
    s[r] = b[p * B + r];
    for (int e = 0; e < ns; ++e) {
      if (off[3 * e] == 0 && off[3 * e + 1] == 0 && off[3 * e + 2] == 0) continue;
      int a = i + off[3 * e], bb = j + off[3 * e + 1], c = k + off[3 * e + 2];
      if (!inside(d, a, bb, c)) continue;
      long q = pidx(d, a, bb, c);
      for (int cc = 0; cc < B; ++cc) s[r] -= A[((p * ns + e) * B + r) * B + cc] * u[q * B + cc];
    }
  }
  for (int r = 0; r < B; ++r) {
    double v = 0.0;
    for (int cc = 0; cc < B; ++cc) v += Dinv[(p * B + r) * B + cc] * s[cc];
    if (w == 1.0)
      u[p * B + r] = v;
    else
      u[p * B + r] = (1.0 - w) * u[p * B + r] + w * v;
  }
}

/* Forward sweep in lexicographic order (x slowest, z fastest). */
void orc_gs_forward(const int d[3], int ns, const int* off, int B, const double* A, const double* Dinv,
                    const double* b, double* u, double w) {
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j)
      for (int k = 0; k < d[2]; ++k) gs_point(d, ns, off, B, A, Dinv, b, u, w, i, j, k);
}

/* Backward sweep: the same update in exactly the reverse order. */
void orc_gs_backward(const int d[3], int ns, const int* off, int B, const double* A, const double* Dinv,
                     const double* b, double* u, double w) {
  for (int i = d[0] - 1; i >= 0; --i)
    for (int j = d[1] - 1; j >= 0; --j)
      for (int k = d[2] - 1; k >= 0; --k) gs_point(d, ns, off, B, A, Dinv, b, u, w, i, j, k);
}

/* ------------------------------------------------------------------------- */
/* Line Gauss-Seidel along z (Sec. 4.4, LGS): the points of a z-column       */
/* (i, j) are updated together.  The right-hand side of the column gathers   */
/* b minus every coupling to another column (columns earlier in the sweep   */
/* already hold new values), and the tridiagonal system formed by the        */
/* offsets (0,0,-1), (0,0,0), (0,0,+1) is solved by the Thomas algorithm.    */
/* Scalar problems only; the relaxation weight is 1.                         */
/* ------------------------------------------------------------------------- */

/* stencil entries of the column's tridiagonal part (-1 where absent) */
static void line_entries(int ns, const int* off, int* esub, int* ediag, int* esup) {
  *esub = find_off(ns, off, 0, 0, -1);
  *ediag = find_off(ns, off, 0, 0, 0);
  *esup = find_off(ns, off, 0, 0, 1);
}

/* Thomas elimination pivots of every column; ORC_EBREAKDOWN if one is zero,
 * or not positive when spd_check is set. */
int orc_lgs_check(const int d[3], int ns, const int* off, const double* A, int spd_check) {
  int es, ed, eu;
  line_entries(ns, off, &es, &ed, &eu);
  if (ed < 0) return ORC_EBREAKDOWN;
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j) {
      double cprev = 0.0;
      for (int k = 0; k < d[2]; ++k) {
        long p = pidx(d, i, j, k);
        double sub = (es >= 0 && k > 0) ? A[p * ns + es] : 0.0;
        double sup = (eu >= 0 && k + 1 < d[2]) ? A[p * ns + eu] : 0.0;
        double m = A[p * ns + ed] - sub * cprev;
        if (m == 0.0 || (spd_check && !(m > 0.0))) return ORC_EBREAKDOWN;
        cprev = sup / m;
      }
    }
  return ORC_OK;
}

/* Update column (i, j) in place.  rhs, cp, dp: scratch of d[2] doubles. */
static void lgs_column(const int d[3], int ns, const int* off, const double* A, const double* b, double* u, int i,
                       int j, double* rhs, double* cp, double* dp) {
  int es, ed, eu;
  line_entries(ns, off, &es, &ed, &eu);
  int nz = d[2];
  for (int k = 0; k < nz; ++k) {
    long p = pidx(d, i, j, k);
    double s = b[p];
    for (int e = 0; e < ns; ++e) {
      if (off[3 * e] == 0 && off[3 * e + 1] == 0) continue; /* in the column */
      int a = i + off[3 * e], bb = j + off[3 * e + 1], c = k + off[3 * e + 2];
      if (!inside(d, a, bb, c)) continue;
      s -= A[p * ns + e] * u[pidx(d, a, bb, c)];
    }
    rhs[k] = s;
  }
  /* Thomas: forward elimination, then back substitution */
  for (int k = 0; k < nz; ++k) {
    long p = pidx(d, i, j, k);
    double sub = (es >= 0 && k > 0) ? A[p * ns + es] : 0.0;
    double sup = (eu >= 0 && k + 1 < nz) ? A[p * ns + eu] : 0.0;
    double m = A[p * ns + ed] - (k > 0 ? sub * cp[k - 1] : 0.0);
    cp[k] = sup / m;
    dp[k] = (rhs[k] - (k > 0 ? sub * dp[k - 1] : 0.0)) / m;
  }
  u[pidx(d, i, j, nz - 1)] = dp[nz - 1];
  for (int k = nz - 2; k >= 0; --k) u[pidx(d, i, j, k)] = dp[k] - cp[k] * u[pidx(d, i, j, k + 1)];
}

/* Forward line sweep: columns in lexicographic (i, j) order. */
void orc_lgs_forward(const int d[3], int ns, const int* off, const double* A, const double* b, double* u) {
  double* t = (double*)malloc(sizeof(double) * 3 * d[2]);
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j) lgs_column(d, ns, off, A, b, u, i, j, t, t + d[2], t + 2 * d[2]);
  free(t);
}

/* Backward line sweep: the same column update in the reverse column order. */
void orc_lgs_backward(const int d[3], int ns, const int* off, const double* A, const double* b, double* u) {
  double* t = (double*)malloc(sizeof(double) * 3 * d[2]);
  for (int i = d[0] - 1; i >= 0; --i)
    for (int j = d[1] - 1; j >= 0; --j) lgs_column(d, ns, off, A, b, u, i, j, t, t + d[2], t + 2 * d[2]);
  free(t);
}

/* ------------------------------------------------------------------------- */
/* ILU(0) on the matrix mask (Sec. 4.2 "Flexibility" and Sec. 4.4 ILU formula) */
/* ------------------------------------------------------------------------- */

/* Linear offset of an on-grid neighbour: q - p.  Two different offsets can
 * share it only if at most one of them is on-grid, so ordering by it orders
 * the on-grid neighbours of a row by column index. */
static long lin(const int d[3], const int* o) { return ((long)o[0] * d[1] + o[1]) * d[2] + o[2]; }

/* Row-by-row incomplete LU restricted to the mask (IKJ form of Gaussian
 * elimination, fill outside the mask discarded).  Output LU has the layout of
 * A: entries with a lower (negative-linear-offset) neighbour hold the unit-lower
 * factor L, the centre and upper entries hold U.  Returns ORC_EBREAKDOWN on a
 * zero pivot, or on a non-positive pivot if spd_check is set. */
int orc_ilu0_factor(const int d[3], int ns, const int* off, const double* A, double* LU, int spd_check) {
  long n = npts(d);
  int ec = find_off(ns, off, 0, 0, 0);
  memcpy(LU, A, sizeof(double) * n * ns);
  /* entries ordered by linear offset, so the elimination runs in column order */
  int* ord = (int*)malloc(sizeof(int) * ns);
  for (int e = 0; e < ns; ++e) ord[e] = e;
  for (int a = 1; a < ns; ++a)
    for (int b = a; b > 0 && lin(d, off + 3 * ord[b]) < lin(d, off + 3 * ord[b - 1]); --b) {
      int t = ord[b]; ord[b] = ord[b - 1]; ord[b - 1] = t;
    }
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j)
      for (int k = 0; k < d[2]; ++k) {
        long p = pidx(d, i, j, k);
        for (int tk = 0; tk < ns; ++tk) {
          int ek = ord[tk];
          const int* ok = off + 3 * ek;
          if (lin(d, ok) >= 0) break; /* only strictly lower columns q < p */
          if (!inside(d, i + ok[0], j + ok[1], k + ok[2])) continue;
          long q = pidx(d, i + ok[0], j + ok[1], k + ok[2]);
          double piv = LU[q * ns + ec];
          double l = LU[p * ns + ek] / piv;
          LU[p * ns + ek] = l;
          /* a_{p,j} -= l * u_{q,j} for every later column j of row p kept by the mask */
          for (int tj = tk + 1; tj < ns; ++tj) {
            int ej = ord[tj];
            const int* oj = off + 3 * ej;
            if (!inside(d, i + oj[0], j + oj[1], k + oj[2])) continue;
            int eq = find_off(ns, off, oj[0] - ok[0], oj[1] - ok[1], oj[2] - ok[2]);
            if (eq < 0) continue; /* fill-in outside the mask is dropped */
            LU[p * ns + ej] -= l * LU[q * ns + eq];
          }
        }
        double piv = LU[p * ns + ec];
        if (piv == 0.0 || (spd_check && !(piv > 0.0))) { free(ord); return ORC_EBREAKDOWN; }
      }
  free(ord);
  return ORC_OK;
}

/* x = U^{-1} L^{-1} r: forward unit-lower solve in lexicographic order, then the
 * backward upper solve in reverse order.  Udinv[p] = 1/u_pp. */
void orc_ilu0_apply(const int d[3], int ns, const int* off, const double* LU, const double* Udinv, const double* r,
                    double* x) {
  long n = npts(d);
  for (long t = 0; t < n; ++t) x[t] = r[t];
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j)
      for (int k = 0; k < d[2]; ++k) {
        long p = pidx(d, i, j, k);
        double s = x[p];
        for (int e = 0; e < ns; ++e) {
          const int* o = off + 3 * e;
          if (lin(d, o) >= 0 || !inside(d, i + o[0], j + o[1], k + o[2])) continue;
          s -= LU[p * ns + e] * x[pidx(d, i + o[0], j + o[1], k + o[2])];
        }
        x[p] = s;
      }
  for (int i = d[0] - 1; i >= 0; --i)
    for (int j = d[1] - 1; j >= 0; --j)
      for (int k = d[2] - 1; k >= 0; --k) {
        long p = pidx(d, i, j, k);
        double s = x[p];
        for (int e = 0; e < ns; ++e) {
          const int* o = off + 3 * e;
          if (lin(d, o) <= 0 || !inside(d, i + o[0], j + o[1], k + o[2])) continue;
          s -= LU[p * ns + e] * x[pidx(d, i + o[0], j + o[1], k + o[2])];
        }
        x[p] = s * Udinv[p];
      }
}

/* ------------------------------------------------------------------------- */
/* Grid transfers (Sec. 2 V-cycle; Table 2 patterns 3d27v, 3d8c and 3d64c)  */
/* ------------------------------------------------------------------------- */
/* Transfer 0 = vertex full weighting: coarse point I sits on fine point 2I+1;
 *   P(v,J) = prod_d w(v_d - (2J_d+1)), w(0)=1, w(+-1)=1/2 (trilinear, 3d27v),
 *   R = P^T / 8 (full weighting).
 * Transfer 1 = cell piecewise constant 3d8c: R(I,u) = 1 for u in 2I+{0,1}^3,
 *   P = R^T.
 * Transfer 2 = cell-centred trilinear interpolation 3d64c with the 3d8c
 *   restriction of transfer 1 (Table 2 columns 3d8c / A / 3d64c; the
 *   interpolation of the Table 8 settings for rhd-3T and solid-3D).  Coarse
 *   cell J covers fine cells 2J and 2J+1 in every dimension; a fine cell
 *   centre lies a quarter of a coarse cell from the centre of its own coarse
 *   cell and three quarters from the nearest other one, so per dimension
 *   c(v - 2J) = 3/4 for v - 2J in {0, 1} and 1/4 for v - 2J in {-1, 2}, and
 *   P(v,J) = prod_d c(v_d - 2J_d): every coarse cell feeds the 4^3 = 64 fine
 *   cells 2J + {-1,0,1,2}^3 (hence "3d64c"), every fine cell takes 8 coarse
 *   cells.  Coarse cells off the grid are dropped (their weight is lost, as
 *   for the vertex transfer).  R is not a multiple of P^T, so A^C is in
 *   general nonsymmetric.
 * Transfer 3 = 2-D semi-coarsening in x and y (the weather setting of
 *   Table 8: 2-D semi-coarsening, R 2d4c, P 2d16c): the x and y dimensions
 *   are coarsened as in transfer 2 (restriction = sum over the 2 x 2 fine
 *   cells of a coarse cell, interpolation = cell-centred bilinear with the
 *   weights c above, coarse cells off the grid dropped), z is kept: coarse
 *   point (I, J, K) owns fine points (2I + {0,1}, 2J + {0,1}, K). */

/* coarse grid of a fine grid: halved in every dimension, or in x and y only
 * for the semi-coarsening transfer 3 */
void orc_coarse_dims_t(int transfer, const int f[3], int c[3]) {
  for (int t = 0; t < 3; ++t) c[t] = (transfer == 3 && t == 2) ? f[t] : f[t] / 2;
}

void orc_coarse_dims(const int f[3], int c[3]) { orc_coarse_dims_t(0, f, c); }

static double w1(int dlt) { return dlt == 0 ? 1.0 : (dlt == 1 || dlt == -1 ? 0.5 : 0.0); }

/* 1-D cell-centred linear interpolation weight of fine cell 2J + d from coarse cell J */
static double wc(int d) { return (d == 0 || d == 1) ? 0.75 : ((d == -1 || d == 2) ? 0.25 : 0.0); }

/* P(v,J) for fine point v, coarse point J */
static double pweight(int transfer, const int* v, const int* J) {
  if (transfer == 0) return w1(v[0] - (2 * J[0] + 1)) * w1(v[1] - (2 * J[1] + 1)) * w1(v[2] - (2 * J[2] + 1));
  if (transfer == 2) return wc(v[0] - 2 * J[0]) * wc(v[1] - 2 * J[1]) * wc(v[2] - 2 * J[2]);
  if (transfer == 3) return v[2] == J[2] ? wc(v[0] - 2 * J[0]) * wc(v[1] - 2 * J[1]) : 0.0;
  for (int t = 0; t < 3; ++t)
    if (v[t] - 2 * J[t] < 0 || v[t] - 2 * J[t] > 1) return 0.0;
  return 1.0;
}

/* R(I,u) */
static double rweight(int transfer, const int* I, const int* u) {
  if (transfer == 3) {
    for (int t = 0; t < 2; ++t)
      if (u[t] - 2 * I[t] < 0 || u[t] - 2 * I[t] > 1) return 0.0;
    return u[2] == I[2] ? 1.0 : 0.0;
  }
  return transfer == 0 ? pweight(0, u, I) / 8.0 : pweight(1, u, I); /* transfers 1 and 2: 3d8c */
}

/* fine points that the coarse point I touches: base[t] + [0, span[t]) */
static void support(int transfer, const int* I, int base[3], int span[3]) {
  for (int t = 0; t < 3; ++t) {
    const int keep = transfer == 3 && t == 2; /* semi-coarsening keeps z */
    base[t] = keep ? I[t] : 2 * I[t];
    span[t] = keep ? 1 : (transfer == 0 ? 3 : 2);
  }
}

/* the coarse coordinate a fine coordinate v[t] lies next to */
static int coarse_of(int transfer, int t, int v) { return (transfer == 3 && t == 2) ? v : v / 2; }

/* fc = R rf (B unknowns per point, each restricted separately). */
void orc_restrict(int transfer, const int fd[3], int B, const double* rf, double* fc) {
  int cd[3];
  orc_coarse_dims_t(transfer, fd, cd);
  for (int I0 = 0; I0 < cd[0]; ++I0)
    for (int I1 = 0; I1 < cd[1]; ++I1)
      for (int I2 = 0; I2 < cd[2]; ++I2) {
        int I[3] = {I0, I1, I2}, base[3], span[3];
        support(transfer, I, base, span);
        long P = pidx(cd, I0, I1, I2);
        for (int r = 0; r < B; ++r) {
          double s = 0.0;
          for (int a = 0; a < span[0]; ++a)
            for (int b = 0; b < span[1]; ++b)
              for (int c = 0; c < span[2]; ++c) {
                int u[3] = {base[0] + a, base[1] + b, base[2] + c};
                if (!inside(fd, u[0], u[1], u[2])) continue;
                s += rweight(transfer, I, u) * rf[pidx(fd, u[0], u[1], u[2]) * B + r];
              }
          fc[P * B + r] = s;
        }
      }
}

/* uf += P ec */
void orc_prolong_add(int transfer, const int fd[3], int B, const double* ec, double* uf) {
  int cd[3];
  orc_coarse_dims_t(transfer, fd, cd);
  for (int v0 = 0; v0 < fd[0]; ++v0)
    for (int v1 = 0; v1 < fd[1]; ++v1)
      for (int v2 = 0; v2 < fd[2]; ++v2) {
        int v[3] = {v0, v1, v2};
        long q = pidx(fd, v0, v1, v2);
        for (int r = 0; r < B; ++r) {
          double s = 0.0;
          /* every coarse J with a nonzero weight lies within 1 of v's coarse point */
          for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b)
              for (int c = -1; c <= 1; ++c) {
                int J[3] = {coarse_of(transfer, 0, v0) + a, coarse_of(transfer, 1, v1) + b,
                            coarse_of(transfer, 2, v2) + c};
                if (!inside(cd, J[0], J[1], J[2])) continue;
                double wgt = pweight(transfer, v, J);
                if (wgt == 0.0) continue;
                s += wgt * ec[pidx(cd, J[0], J[1], J[2]) * B + r];
              }
          uf[q * B + r] += s;
        }
      }
}

/* ------------------------------------------------------------------------- */
/* Galerkin coarse operator, Eq. (4) and the influence-chain sum Eq. (5):    */
/*   A^C(I,J) = sum_{u,v} R(I,u) A^F(u,v) P(v,J),                            */
/* evaluated by brute force over every coarse point I, every fine u in the   */
/* support of R(I,.), every stencil neighbour v of u and every coarse J with */
/* P(v,J) != 0.  The coarse offsets are discovered on the fly.               */
/* ------------------------------------------------------------------------- */

/* Ac27 receives, for every coarse point, all 27 offsets of {-1,0,1}^3 in
 * lexicographic order (dx slowest): Ac27[((P*27 + o)*B + r)*B + c].
 * present[o] is set when some chain reaches offset o.  Returns ORC_EINVAL if a
 * chain reaches a coarse offset outside {-1,0,1}^3. */
/* All chains of one coarse point I, accumulated into out27[27][B][B]. */
static int rap_point(int transfer, const int fd[3], const int cd[3], int ns, const int* off, int B, const double* Af,
                     const int I[3], double* out27, int* present) {
  int base[3], span[3];
  support(transfer, I, base, span);
  for (int a = 0; a < span[0]; ++a)
    for (int b = 0; b < span[1]; ++b)
      for (int c = 0; c < span[2]; ++c) {
        int u[3] = {base[0] + a, base[1] + b, base[2] + c};
        if (!inside(fd, u[0], u[1], u[2])) continue;
        double wr = rweight(transfer, I, u);
        if (wr == 0.0) continue;
        long pu = pidx(fd, u[0], u[1], u[2]);
        for (int e = 0; e < ns; ++e) {
          int v[3] = {u[0] + off[3 * e], u[1] + off[3 * e + 1], u[2] + off[3 * e + 2]};
          if (!inside(fd, v[0], v[1], v[2])) continue;
          for (int ja = -2; ja <= 2; ++ja)
            for (int jb = -2; jb <= 2; ++jb)
              for (int jc = -2; jc <= 2; ++jc) {
                int J[3] = {I[0] + ja, I[1] + jb, I[2] + jc};
                if (!inside(cd, J[0], J[1], J[2])) continue;
                double wp = pweight(transfer, v, J);
                if (wp == 0.0) continue;
                if (ja < -1 || ja > 1 || jb < -1 || jb > 1 || jc < -1 || jc > 1) return ORC_EINVAL;
                int o = (ja + 1) * 9 + (jb + 1) * 3 + (jc + 1);
                present[o] = 1;
                for (int r = 0; r < B; ++r)
                  for (int cc = 0; cc < B; ++cc)
                    out27[(o * B + r) * B + cc] += wr * Af[((pu * ns + e) * B + r) * B + cc] * wp;
              }
        }
      }
  return ORC_OK;
}

int orc_rap27(int transfer, const int fd[3], int ns, const int* off, int B, const double* Af, double* Ac27,
              int* present) {
  int cd[3];
  orc_coarse_dims_t(transfer, fd, cd);
  long nc = npts(cd);
  memset(Ac27, 0, sizeof(double) * nc * 27 * B * B);
  for (int o = 0; o < 27; ++o) present[o] = 0;
  int bad = 0;
  /* Coarse points are independent (each sums its own chains into its own
   * row), so they may run on several threads without changing any sum. */
#pragma omp parallel
  {
    int pres[27] = {0};
#pragma omp for schedule(dynamic, 64)
    for (long Pc = 0; Pc < nc; ++Pc) {
      int I[3] = {(int)(Pc / ((long)cd[1] * cd[2])), (int)((Pc / cd[2]) % cd[1]), (int)(Pc % cd[2])};
      if (rap_point(transfer, fd, cd, ns, off, B, Af, I, Ac27 + Pc * 27 * B * B, pres)) {
#pragma omp atomic write
        bad = 1;
      }
    }
#pragma omp critical
    for (int o = 0; o < 27; ++o) present[o] |= pres[o];
  }
  return bad ? ORC_EINVAL : ORC_OK;
}

/* Threads of the parallel loops above (no effect in a serial build). */
#ifdef _OPENMP
#include <omp.h>
#endif
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* The same chain sums for a list of coarse point indices only (for checking
 * single entries of a large hierarchy): out27[t][27][B][B]. */
int orc_rap27_at(int transfer, const int fd[3], int ns, const int* off, int B, const double* Af, long npoints,
                 const long* points, double* out27) {
  int cd[3], present[27];
  orc_coarse_dims_t(transfer, fd, cd);
  memset(out27, 0, sizeof(double) * npoints * 27 * B * B);
  for (long t = 0; t < npoints; ++t) {
    long P = points[t];
    int I[3] = {(int)(P / ((long)cd[1] * cd[2])), (int)((P / cd[2]) % cd[1]), (int)(P % cd[2])};
    int rc = rap_point(transfer, fd, cd, ns, off, B, Af, I, out27 + t * 27 * B * B, present);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Dense direct solve for the coarsest level (the paper does not specify it; */
/* LU with partial pivoting of the assembled coarsest matrix).               */
/* ------------------------------------------------------------------------- */

/* Assemble the stencil matrix as a dense (n*B) x (n*B) row-major matrix. */
void orc_assemble_dense(const int d[3], int ns, const int* off, int B, const double* A, double* M) {
  long n = npts(d) * B;
  memset(M, 0, sizeof(double) * n * n);
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j)
      for (int k = 0; k < d[2]; ++k) {
        long p = pidx(d, i, j, k);
        for (int e = 0; e < ns; ++e) {
          int a = i + off[3 * e], b = j + off[3 * e + 1], c = k + off[3 * e + 2];
          if (!inside(d, a, b, c)) continue;
          long q = pidx(d, a, b, c);
          for (int r = 0; r < B; ++r)
            for (int cc = 0; cc < B; ++cc) M[(p * B + r) * n + q * B + cc] = A[((p * ns + e) * B + r) * B + cc];
        }
      }
}

/* In-place LU with partial pivoting: M = P L U, piv[r] = row swapped into r. */
int orc_lu_factor(int n, double* M, int* piv) {
  for (int c = 0; c < n; ++c) {
    int pr = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[(long)r * n + c]) > fabs(M[(long)pr * n + c])) pr = r;
    piv[c] = pr;
    if (M[(long)pr * n + c] == 0.0) return ORC_EBREAKDOWN;
    if (pr != c)
      for (int t = 0; t < n; ++t) {
        double s = M[(long)c * n + t]; M[(long)c * n + t] = M[(long)pr * n + t]; M[(long)pr * n + t] = s;
      }
    for (int r = c + 1; r < n; ++r) {
      double l = M[(long)r * n + c] / M[(long)c * n + c];
      M[(long)r * n + c] = l;
      for (int t = c + 1; t < n; ++t) M[(long)r * n + t] -= l * M[(long)c * n + t];
    }
  }
  return ORC_OK;
}

void orc_lu_solve(int n, const double* LU, const int* piv, const double* b, double* x) {
  for (int t = 0; t < n; ++t) x[t] = b[t];
  for (int c = 0; c < n; ++c)
    if (piv[c] != c) { double s = x[c]; x[c] = x[piv[c]]; x[piv[c]] = s; }
  for (int r = 0; r < n; ++r) {
    double s = x[r];
    for (int t = 0; t < r; ++t) s -= LU[(long)r * n + t] * x[t];
    x[r] = s;
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = x[r];
    for (int t = r + 1; t < n; ++t) s -= LU[(long)r * n + t] * x[t];
    x[r] = s / LU[(long)r * n + r];
  }
}

/* ------------------------------------------------------------------------- */
/* Reduced precision (not in the paper): FP32 cast, and BF16 with a per-row  */
/* FP32 scale s_p = max_e |a_pe|, stored value bf16(a_pe / s_p), products    */
/* accumulated in FP32 and multiplied by s_p once per row.                   */
/* ------------------------------------------------------------------------- */

/* Round a double to the nearest bfloat16 (8 significant bits), ties to even,
 * written from the IEEE-754 binary64 layout; returns the bf16 value as float.
 * Subnormal bf16 results are not produced by the inputs here; Inf/NaN pass. */
float orc_bf16_round(double x) {
  if (x != x || x == INFINITY || x == -INFINITY) return (float)x;
  if (x == 0.0) return (float)x;
  int ex;
  double m = frexp(fabs(x), &ex);  /* |x| = m * 2^ex, m in [0.5,1) */
  double scaled = ldexp(m, 8);     /* 8 significant bits to the left of the point */
  double fl = floor(scaled);
  double rem = scaled - fl;        /* exact: scaled < 256 and has <= 53 bits */
  if (rem > 0.5 || (rem == 0.5 && fmod(fl, 2.0) == 1.0)) fl += 1.0;
  double r = ldexp(fl, ex - 8);
  return (float)(x < 0 ? -r : r);
}

/* Low-precision copy of a scalar stencil matrix.  mode 1: vals = fp32(a),
 * scale = 1.  mode 2: scale_p = fp32(max |a_pe| over the entries selected by
 * sel: 0 all, -1 strictly lower, +1 strictly upper (centre excluded for +-1)),
 * vals = bf16(a_pe / scale_p) (0 if the row is all zero, scale then 1). */
static int entry_sel(const int d[3], const int* o, int sel) {
  long l = lin(d, o);
  if (sel == 0) return 1;
  return sel < 0 ? l < 0 : l > 0;
}

void orc_lower_matrix(const int d[3], int ns, const int* off, const double* A, int mode, int sel, float* vals,
                      float* scale) {
  long n = npts(d);
  for (long p = 0; p < n; ++p) {
    double mx = 0.0;
    for (int e = 0; e < ns; ++e)
      if (entry_sel(d, off + 3 * e, sel) && fabs(A[p * ns + e]) > mx) mx = fabs(A[p * ns + e]);
    float s = (mode == 2 && mx > 0.0) ? (float)mx : 1.0f;
    scale[p] = s;
    for (int e = 0; e < ns; ++e) {
      double a = A[p * ns + e];
      vals[p * ns + e] = mode == 2 ? orc_bf16_round(a / (double)s) : (float)a;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Multigrid hierarchy and V-cycle (Sec. 2, Fig. 1 V-cycle; Eq. 1 T_tot)     */
/* ------------------------------------------------------------------------- */

enum { SM_SGS = 0, SM_ILU0 = 1, SM_LGS = 2 };

typedef struct {
  int d[3], ns, off[27 * 3];
  double* A;      /* [n][ns][B][B] */
  double* Dinv;   /* GS: [n][B][B] */
  double* LU;     /* ILU */
  double* Udinv;  /* ILU: 1/u_pp */
  /* reduced-precision copies */
  float *Av, *As, *Lv, *Ls, *Uv, *Us, *Dv32;
} orc_level;

typedef struct {
  int B, nlev, smoother, transfer, precision;
  double w;
  orc_level lev[16];
  /* coarsest dense LU */
  int nco;
  double* cLU;
  int* cpiv;
} orc_mg;

/* Coarsening schedule: halve every dimension while all of them are even and
 * the smallest is at least 8 (fixed stride-2 full coarsening, Sec. 4.1 P2). */
/* The same for a transfer: with the x-y semi-coarsening of transfer 3 only
 * x and y are halved, while both are even and the smaller is at least 8. */
int orc_plan_levels_t(int transfer, const int d[3], int max_levels, int dims_out[][3]) {
  int c[3] = {d[0], d[1], d[2]};
  const int nd = transfer == 3 ? 2 : 3;
  int L = 0;
  for (;;) {
    dims_out[L][0] = c[0]; dims_out[L][1] = c[1]; dims_out[L][2] = c[2];
    ++L;
    int mn = c[0];
    int odd = 0;
    for (int t = 0; t < nd; ++t) {
      if (c[t] < mn) mn = c[t];
      odd |= c[t] % 2;
    }
    if (L >= max_levels || mn < 8 || odd) break;
    int cn[3];
    orc_coarse_dims_t(transfer, c, cn);
    c[0] = cn[0]; c[1] = cn[1]; c[2] = cn[2];
  }
  return L;
}

int orc_plan_levels(const int d[3], int max_levels, int dims_out[][3]) {
  return orc_plan_levels_t(0, d, max_levels, dims_out);
}

static void level_free(orc_level* L) {
  free(L->A); free(L->Dinv); free(L->LU); free(L->Udinv);
  free(L->Av); free(L->As); free(L->Lv); free(L->Ls); free(L->Uv); free(L->Us); free(L->Dv32);
}

void orc_mg_free(void* h) {
  orc_mg* mg = (orc_mg*)h;
  if (!mg) return;
  for (int l = 0; l < mg->nlev; ++l) level_free(&mg->lev[l]);
  free(mg->cLU); free(mg->cpiv);
  free(mg);
}

/* Build the hierarchy: Galerkin coarse operators by orc_rap27 (kept on the
 * offsets a chain reaches, in lexicographic order), smoother set-up on every
 * non-coarsest level, dense LU of the coarsest.  precision: 0 FP64, 1 FP32
 * (scalar or 3x3 blocks), 2 BF16 with row scales (scalar only); other
 * combinations are rejected. */
int orc_mg_setup(void** out, const int d[3], int ns, const int* off, int B, const double* A, int smoother,
                 int transfer, double w, int precision, int max_levels) {
  *out = NULL;
  if (orc_mask_validate(ns, off)) return ORC_EINVAL;
  if (B != 1 && B != 3) return ORC_EINVAL;
  if (transfer < 0 || transfer > 3) return ORC_EINVAL;
  if (B == 3 && smoother != SM_SGS) return ORC_EINVAL;
  if (smoother < SM_SGS || smoother > SM_LGS) return ORC_EINVAL;
  if (smoother == SM_LGS && (precision != 0 || w != 1.0)) return ORC_EINVAL;
  if (precision == 2 && B != 1) return ORC_EINVAL; /* BF16 row scales: scalar problems only */
  for (int t = 0; t < 3; ++t)
    if (d[t] < 1) return ORC_EINVAL;
  orc_mg* mg = (orc_mg*)calloc(1, sizeof(orc_mg));
  mg->B = B; mg->smoother = smoother; mg->transfer = transfer; mg->w = w; mg->precision = precision;
  int dims[16][3];
  mg->nlev = orc_plan_levels_t(transfer, d, max_levels < 16 ? max_levels : 16, dims);
  int rc = ORC_OK;
  for (int l = 0; l < mg->nlev; ++l) {
    orc_level* L = &mg->lev[l];
    memcpy(L->d, dims[l], sizeof(int) * 3);
    long n = npts(L->d);
    if (l == 0) {
      L->ns = ns;
      memcpy(L->off, off, sizeof(int) * 3 * ns);
      L->A = (double*)malloc(sizeof(double) * n * ns * B * B);
      memcpy(L->A, A, sizeof(double) * n * ns * B * B);
    } else {
      orc_level* F = &mg->lev[l - 1];
      double* A27 = (double*)malloc(sizeof(double) * n * 27 * B * B);
      int present[27];
      rc = orc_rap27(transfer, F->d, F->ns, F->off, B, F->A, A27, present);
      if (rc) { free(A27); break; }
      int m = 0;
      for (int o = 0; o < 27; ++o)
        if (present[o]) {
          L->off[3 * m] = o / 9 - 1; L->off[3 * m + 1] = (o / 3) % 3 - 1; L->off[3 * m + 2] = o % 3 - 1;
          ++m;
        }
      L->ns = m;
      L->A = (double*)malloc(sizeof(double) * n * m * B * B);
      for (long p = 0; p < n; ++p) {
        int e = 0;
        for (int o = 0; o < 27; ++o)
          if (present[o]) {
            memcpy(L->A + (p * m + e) * B * B, A27 + (p * 27 + o) * B * B, sizeof(double) * B * B);
            ++e;
          }
      }
      free(A27);
    }
    if (l < mg->nlev - 1) {
      if (smoother == SM_SGS) {
        L->Dinv = (double*)malloc(sizeof(double) * n * B * B);
        rc = orc_diag_inverse(L->d, L->ns, L->off, B, L->A, L->Dinv);
      } else if (smoother == SM_LGS) {
        rc = orc_lgs_check(L->d, L->ns, L->off, L->A, 1);
      } else {
        L->LU = (double*)malloc(sizeof(double) * n * L->ns);
        L->Udinv = (double*)malloc(sizeof(double) * n);
        rc = orc_ilu0_factor(L->d, L->ns, L->off, L->A, L->LU, 1);
        if (!rc) {
          int ec = find_off(L->ns, L->off, 0, 0, 0);
          for (long p = 0; p < n; ++p) L->Udinv[p] = 1.0 / L->LU[p * L->ns + ec];
        }
      }
      if (rc) break;
      if (precision && B == 3) {
        /* FP32 blocks: every coefficient and the FP64 block inverse cast */
        long nb2 = n * L->ns * 9;
        L->Av = (float*)malloc(sizeof(float) * nb2);
        L->As = (float*)malloc(sizeof(float) * n);
        L->Dv32 = (float*)malloc(sizeof(float) * n * 9);
        for (long t = 0; t < nb2; ++t) L->Av[t] = (float)L->A[t];
        for (long p = 0; p < n; ++p) L->As[p] = 1.0f;
        for (long t = 0; t < n * 9; ++t) L->Dv32[t] = (float)L->Dinv[t];
      } else if (precision) {
        int mode = precision == 2 ? 2 : 1;
        L->Av = (float*)malloc(sizeof(float) * n * L->ns);
        L->As = (float*)malloc(sizeof(float) * n);
        orc_lower_matrix(L->d, L->ns, L->off, L->A, mode, 0, L->Av, L->As);
        L->Dv32 = (float*)malloc(sizeof(float) * n);
        if (smoother == SM_SGS) {
          for (long p = 0; p < n; ++p) L->Dv32[p] = (float)L->Dinv[p];
        } else {
          L->Lv = (float*)malloc(sizeof(float) * n * L->ns);
          L->Ls = (float*)malloc(sizeof(float) * n);
          L->Uv = (float*)malloc(sizeof(float) * n * L->ns);
          L->Us = (float*)malloc(sizeof(float) * n);
          orc_lower_matrix(L->d, L->ns, L->off, L->LU, mode, -1, L->Lv, L->Ls);
          orc_lower_matrix(L->d, L->ns, L->off, L->LU, mode, +1, L->Uv, L->Us);
          for (long p = 0; p < n; ++p) L->Dv32[p] = (float)L->Udinv[p];
        }
      }
    } else {
      mg->nco = (int)(n * B);
      mg->cLU = (double*)malloc(sizeof(double) * mg->nco * mg->nco);
      mg->cpiv = (int*)malloc(sizeof(int) * mg->nco);
      orc_assemble_dense(L->d, L->ns, L->off, B, L->A, mg->cLU);
      rc = orc_lu_factor(mg->nco, mg->cLU, mg->cpiv);
      if (rc) break;
    }
  }
  if (rc) { orc_mg_free(mg); return rc; }
  *out = mg;
  return ORC_OK;
}

int orc_mg_nlevels(void* h) { return ((orc_mg*)h)->nlev; }

void orc_mg_level_info(void* h, int l, int d[3], int* ns, int* off) {
  orc_level* L = &((orc_mg*)h)->lev[l];
  memcpy(d, L->d, sizeof(int) * 3);
  *ns = L->ns;
  memcpy(off, L->off, sizeof(int) * 3 * L->ns);
}

/* which: 0 = A, 1 = ILU factors LU, 2 = Dinv / Udinv, 3 = low-precision A values,
 * 4 = low-precision A row scale, 5/6 = L values/scales, 7/8 = U values/scales,
 * 9 = low-precision inverse diagonal.  Returns the element count copied. */
long orc_mg_level_array(void* h, int l, int which, void* dst) {
  orc_mg* mg = (orc_mg*)h;
  orc_level* L = &mg->lev[l];
  long n = npts(L->d), B2 = (long)mg->B * mg->B;
  const void* src = NULL;
  long cnt = 0, sz = 8;
  switch (which) {
    case 0: src = L->A; cnt = n * L->ns * B2; break;
    case 1: src = L->LU; cnt = L->LU ? n * L->ns : 0; break;
    case 2: src = L->Dinv ? (const void*)L->Dinv : (const void*)L->Udinv; cnt = L->Dinv ? n * B2 : (L->Udinv ? n : 0); break;
    case 3: src = L->Av; cnt = L->Av ? n * L->ns * B2 : 0; sz = 4; break;
    case 4: src = L->As; cnt = L->As ? n : 0; sz = 4; break;
    case 5: src = L->Lv; cnt = L->Lv ? n * L->ns : 0; sz = 4; break;
    case 6: src = L->Ls; cnt = L->Ls ? n : 0; sz = 4; break;
    case 7: src = L->Uv; cnt = L->Uv ? n * L->ns : 0; sz = 4; break;
    case 8: src = L->Us; cnt = L->Us ? n : 0; sz = 4; break;
    case 9: src = L->Dv32; cnt = L->Dv32 ? n * B2 : 0; sz = 4; break;
  }
  if (src && dst && cnt) memcpy(dst, src, cnt * sz);
  return src ? cnt : 0;
}

/* ---- FP64 smoothing on one level ---------------------------------------- */

/* pre-smoothing from a zero initial guess (ZeroGuess, Table 8): u = S f */
static void smooth_pre64(orc_mg* mg, orc_level* L, const double* f, double* u) {
  long n = npts(L->d) * mg->B;
  for (long t = 0; t < n; ++t) u[t] = 0.0;
  if (mg->smoother == SM_SGS) {
    orc_gs_forward(L->d, L->ns, L->off, mg->B, L->A, L->Dinv, f, u, mg->w);
    orc_gs_backward(L->d, L->ns, L->off, mg->B, L->A, L->Dinv, f, u, mg->w);
  } else if (mg->smoother == SM_LGS) {
    orc_lgs_forward(L->d, L->ns, L->off, L->A, f, u);
    orc_lgs_backward(L->d, L->ns, L->off, L->A, f, u);
  } else {
    orc_ilu0_apply(L->d, L->ns, L->off, L->LU, L->Udinv, f, u);
  }
}

/* post-smoothing on a nonzero iterate */
static void smooth_post64(orc_mg* mg, orc_level* L, const double* f, double* u) {
  if (mg->smoother == SM_SGS) {
    orc_gs_forward(L->d, L->ns, L->off, mg->B, L->A, L->Dinv, f, u, mg->w);
    orc_gs_backward(L->d, L->ns, L->off, mg->B, L->A, L->Dinv, f, u, mg->w);
  } else if (mg->smoother == SM_LGS) {
    orc_lgs_forward(L->d, L->ns, L->off, L->A, f, u);
    orc_lgs_backward(L->d, L->ns, L->off, L->A, f, u);
  } else {
    long n = npts(L->d);
    double* r = (double*)malloc(sizeof(double) * n);
    double* x = (double*)malloc(sizeof(double) * n);
    orc_residual(L->d, L->ns, L->off, 1, L->A, f, u, r);
    orc_ilu0_apply(L->d, L->ns, L->off, L->LU, L->Udinv, r, x);
    for (long t = 0; t < n; ++t) u[t] += x[t];
    free(r); free(x);
  }
}

static void coarse_solve64(orc_mg* mg, const double* f, double* u) { orc_lu_solve(mg->nco, mg->cLU, mg->cpiv, f, u); }

/* One V(1,1)-cycle: z = M^{-1} r.  Down: pre-smooth (zero guess), residual,
 * restrict.  Coarsest: direct solve.  Up: prolong and correct, post-smooth. */
static void vcycle64(orc_mg* mg, const double* r, double* z) {
  int Lc = mg->nlev;
  double *f[16], *u[16];
  for (int l = 0; l < Lc; ++l) {
    long n = npts(mg->lev[l].d) * mg->B;
    f[l] = (double*)malloc(sizeof(double) * n);
    u[l] = (double*)malloc(sizeof(double) * n);
  }
  memcpy(f[0], r, sizeof(double) * npts(mg->lev[0].d) * mg->B);
  for (int l = 0; l < Lc - 1; ++l) {
    orc_level* L = &mg->lev[l];
    long n = npts(L->d) * mg->B;
    smooth_pre64(mg, L, f[l], u[l]);
    double* res = (double*)malloc(sizeof(double) * n);
    orc_residual(L->d, L->ns, L->off, mg->B, L->A, f[l], u[l], res);
    orc_restrict(mg->transfer, L->d, mg->B, res, f[l + 1]);
    free(res);
  }
  coarse_solve64(mg, f[Lc - 1], u[Lc - 1]);
  for (int l = Lc - 2; l >= 0; --l) {
    orc_level* L = &mg->lev[l];
    orc_prolong_add(mg->transfer, L->d, mg->B, u[l + 1], u[l]);
    smooth_post64(mg, L, f[l], u[l]);
  }
  memcpy(z, u[0], sizeof(double) * npts(mg->lev[0].d) * mg->B);
  for (int l = 0; l < Lc; ++l) { free(f[l]); free(u[l]); }
}

/* ---- reduced-precision V-cycle: all level arithmetic in FP32 ------------- */
/* The paper has no reduced-precision cycle; this is the build's extension.
 * Scalar levels keep FP32 values, or BF16 values with an FP32 row scale s_p;
 * 3x3-block levels keep FP32 blocks and the FP32 cast of the FP64 block
 * inverse.  Every sum is accumulated in FP32, in the loop order below. */

/* t_r = s_p * sum_e sum_c v_{p,e,r,c} x_{p+e,c}: the stencil row sum of point
 * (i,j,k) in FP32, the row scale applied to the finished sum (scalar levels;
 * it is 1 in FP32 mode), the centre left out when skip_centre. */
static void rowsum32(const orc_level* L, int B, const float* x, int i, int j, int k, int skip_centre, float* t) {
  const int* d = L->d;
  long p = pidx(d, i, j, k);
  for (int r = 0; r < B; ++r) {
    float s = 0.0f;
    for (int e = 0; e < L->ns; ++e) {
      const int* o = L->off + 3 * e;
      if (skip_centre && (o[0] | o[1] | o[2]) == 0) continue;
      if (!inside(d, i + o[0], j + o[1], k + o[2])) continue;
      long q = pidx(d, i + o[0], j + o[1], k + o[2]);
      for (int c = 0; c < B; ++c) s += L->Av[((p * L->ns + e) * B + r) * B + c] * x[q * B + c];
    }
    t[r] = B == 1 ? L->As[p] * s : s;
  }
}

/* r = b - A x in FP32 */
static void residual32(const orc_level* L, int B, const float* b, const float* x, float* r) {
  const int* d = L->d;
  float t[3];
  for (int i = 0; i < d[0]; ++i)
    for (int j = 0; j < d[1]; ++j)
      for (int k = 0; k < d[2]; ++k) {
        long p = pidx(d, i, j, k);
        rowsum32(L, B, x, i, j, k, 0, t);
        for (int c = 0; c < B; ++c) r[p * B + c] = b[p * B + c] - t[c];
      }
}

/* One point of Gauss-Seidel in FP32: g = b_p - sum_{o != 0} A_po u_{p+o}, then
 * v = dinv_p g (scalar) or v = Dinv_p g (3x3 block, row by row), and with a
 * weight w != 1 the Sec. 4.4 update u_p = (1-w) u_p + w v, all in float. */
static void gs32_point(const orc_level* L, int B, const float* b, float* u, double w, int i, int j, int k) {
  const int* d = L->d;
  long p = pidx(d, i, j, k);
  float t[3], g[3];
  rowsum32(L, B, u, i, j, k, 1, t);
  for (int c = 0; c < B; ++c) g[c] = b[p * B + c] - t[c];
  const float wf = (float)w;
  for (int r = 0; r < B; ++r) {
    float v = 0.0f;
    if (B == 1) {
      v = g[0] * L->Dv32[p];
    } else {
      for (int c = 0; c < B; ++c) v += L->Dv32[(p * B + r) * B + c] * g[c];
    }
    u[p * B + r] = (w == 1.0) ? v : (1.0f - wf) * u[p * B + r] + wf * v;
  }
}

/* Gauss-Seidel sweep in FP32 with weight w, dir +1 lexicographic, -1 reverse. */
static void gs32(const orc_level* L, int B, const float* b, float* u, double w, int dir) {
  const int* d = L->d;
  if (dir > 0) {
    for (int i = 0; i < d[0]; ++i)
      for (int j = 0; j < d[1]; ++j)
        for (int k = 0; k < d[2]; ++k) gs32_point(L, B, b, u, w, i, j, k);
  } else {
    for (int i = d[0] - 1; i >= 0; --i)
      for (int j = d[1] - 1; j >= 0; --j)
        for (int k = d[2] - 1; k >= 0; --k) gs32_point(L, B, b, u, w, i, j, k);
  }
}

/* ILU apply in FP32: y = L^{-1} r with y_p = r_p - sL_p sum_lower lv y_q, then
 * x_p = (y_p - sU_p sum_upper uv x_q) * dinv_p in reverse order. */
static void ilu32(const orc_level* L, const float* r, float* x) {
  const int* d = L->d;
  long n = npts(d);
  for (long t = 0; t < n; ++t) x[t] = r[t];
  for (long p = 0; p < n; ++p) {
    int k = (int)(p % d[2]), j = (int)((p / d[2]) % d[1]), i = (int)(p / ((long)d[1] * d[2]));
    float s = 0.0f;
    for (int e = 0; e < L->ns; ++e) {
      const int* o = L->off + 3 * e;
      if (lin(d, o) >= 0 || !inside(d, i + o[0], j + o[1], k + o[2])) continue;
      s += L->Lv[p * L->ns + e] * x[pidx(d, i + o[0], j + o[1], k + o[2])];
    }
    x[p] = x[p] - L->Ls[p] * s;
  }
  for (long p = n - 1; p >= 0; --p) {
    int k = (int)(p % d[2]), j = (int)((p / d[2]) % d[1]), i = (int)(p / ((long)d[1] * d[2]));
    float s = 0.0f;
    for (int e = 0; e < L->ns; ++e) {
      const int* o = L->off + 3 * e;
      if (lin(d, o) <= 0 || !inside(d, i + o[0], j + o[1], k + o[2])) continue;
      s += L->Uv[p * L->ns + e] * x[pidx(d, i + o[0], j + o[1], k + o[2])];
    }
    x[p] = (x[p] - L->Us[p] * s) * L->Dv32[p];
  }
}

/* fc = R rf in FP32 (weights exact in FP32), per unknown, support order. */
static void restrict32(int transfer, const int fd[3], int B, const float* rf, float* fc) {
  int cd[3];
  orc_coarse_dims_t(transfer, fd, cd);
  for (int I0 = 0; I0 < cd[0]; ++I0)
    for (int I1 = 0; I1 < cd[1]; ++I1)
      for (int I2 = 0; I2 < cd[2]; ++I2) {
        int I[3] = {I0, I1, I2}, base[3], span[3];
        support(transfer, I, base, span);
        for (int r = 0; r < B; ++r) {
          float s = 0.0f;
          for (int a = 0; a < span[0]; ++a)
            for (int b = 0; b < span[1]; ++b)
              for (int c = 0; c < span[2]; ++c) {
                int u[3] = {base[0] + a, base[1] + b, base[2] + c};
                if (!inside(fd, u[0], u[1], u[2])) continue;
                s += (float)rweight(transfer, I, u) * rf[pidx(fd, u[0], u[1], u[2]) * B + r];
              }
          fc[pidx(cd, I0, I1, I2) * B + r] = s;
        }
      }
}

/* uf += P ec in FP32: the interpolated value is summed first, then added. */
static void prolong32(int transfer, const int fd[3], int B, const float* ec, float* uf) {
  int cd[3];
  orc_coarse_dims_t(transfer, fd, cd);
  for (int v0 = 0; v0 < fd[0]; ++v0)
    for (int v1 = 0; v1 < fd[1]; ++v1)
      for (int v2 = 0; v2 < fd[2]; ++v2) {
        int v[3] = {v0, v1, v2};
        for (int r = 0; r < B; ++r) {
          float s = 0.0f;
          for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b)
              for (int c = -1; c <= 1; ++c) {
                int J[3] = {coarse_of(transfer, 0, v0) + a, coarse_of(transfer, 1, v1) + b,
                            coarse_of(transfer, 2, v2) + c};
                if (!inside(cd, J[0], J[1], J[2])) continue;
                double wgt = pweight(transfer, v, J);
                if (wgt == 0.0) continue;
                s += (float)wgt * ec[pidx(cd, J[0], J[1], J[2]) * B + r];
              }
          uf[pidx(fd, v0, v1, v2) * B + r] += s;
        }
      }
}

static void vcycle32(orc_mg* mg, const double* r, double* z) {
  int Lc = mg->nlev, B = mg->B;
  float *f[16], *u[16];
  for (int l = 0; l < Lc; ++l) {
    long n = npts(mg->lev[l].d) * B;
    f[l] = (float*)malloc(sizeof(float) * n);
    u[l] = (float*)malloc(sizeof(float) * n);
  }
  long n0 = npts(mg->lev[0].d) * B;
  for (long t = 0; t < n0; ++t) f[0][t] = (float)r[t];
  for (int l = 0; l < Lc - 1; ++l) {
    orc_level* L = &mg->lev[l];
    long n = npts(L->d) * B;
    float* res = (float*)malloc(sizeof(float) * n);
    if (mg->smoother == SM_SGS) {
      for (long t = 0; t < n; ++t) u[l][t] = 0.0f;
      gs32(L, B, f[l], u[l], mg->w, +1);
      gs32(L, B, f[l], u[l], mg->w, -1);
    } else {
      ilu32(L, f[l], u[l]);
    }
    residual32(L, B, f[l], u[l], res);
    restrict32(mg->transfer, L->d, B, res, f[l + 1]);
    free(res);
  }
  {
    long n = npts(mg->lev[Lc - 1].d) * B;
    double *fd = (double*)malloc(sizeof(double) * n), *ud = (double*)malloc(sizeof(double) * n);
    for (long t = 0; t < n; ++t) fd[t] = (double)f[Lc - 1][t];
    coarse_solve64(mg, fd, ud);
    for (long t = 0; t < n; ++t) u[Lc - 1][t] = (float)ud[t];
    free(fd); free(ud);
  }
  for (int l = Lc - 2; l >= 0; --l) {
    orc_level* L = &mg->lev[l];
    long n = npts(L->d) * B;
    prolong32(mg->transfer, L->d, B, u[l + 1], u[l]);
    if (mg->smoother == SM_SGS) {
      gs32(L, B, f[l], u[l], mg->w, +1);
      gs32(L, B, f[l], u[l], mg->w, -1);
    } else {
      float *res = (float*)malloc(sizeof(float) * n), *x = (float*)malloc(sizeof(float) * n);
      residual32(L, B, f[l], u[l], res);
      ilu32(L, res, x);
      for (long t = 0; t < n; ++t) u[l][t] += x[t];
      free(res); free(x);
    }
  }
  for (long t = 0; t < n0; ++t) z[t] = (double)u[0][t];
  for (int l = 0; l < Lc; ++l) { free(f[l]); free(u[l]); }
}

/* One reduced-precision level operation of a hierarchy set up with precision
 * 1 or 2 (for the pins of the FP32 / BF16 arithmetic), on FP32 vectors of
 * level l: op 0 y = b - A x; 1 x <- GS forward sweep; 2 x <- GS backward
 * sweep; 3 y = U^-1 L^-1 b (ILU(0) apply); 4 y = R x (x on level l, y on
 * l+1); 5 y += P x (x on level l+1, y on level l).  Returns ORC_EINVAL when
 * the operation does not exist for this hierarchy. */
int orc_mg_level_apply32(void* h, int l, int op, float* x, const float* b, float* y) {
  orc_mg* mg = (orc_mg*)h;
  if (!mg->precision || l < 0 || l >= mg->nlev) return ORC_EINVAL;
  orc_level* L = &mg->lev[l];
  const int last = l == mg->nlev - 1;
  switch (op) {
    case 0: if (!L->Av) return ORC_EINVAL; residual32(L, mg->B, b, x, y); return ORC_OK;
    case 1: case 2:
      if (mg->smoother != SM_SGS || !L->Av) return ORC_EINVAL;
      gs32(L, mg->B, b, x, mg->w, op == 1 ? +1 : -1);
      return ORC_OK;
    case 3: if (mg->smoother != SM_ILU0 || !L->Lv) return ORC_EINVAL; ilu32(L, b, y); return ORC_OK;
    case 4: if (last) return ORC_EINVAL; restrict32(mg->transfer, L->d, mg->B, x, y); return ORC_OK;
    case 5: if (last) return ORC_EINVAL; prolong32(mg->transfer, L->d, mg->B, x, y); return ORC_OK;
  }
  return ORC_EINVAL;
}

void orc_mg_vcycle(void* h, const double* r, double* z) {
  orc_mg* mg = (orc_mg*)h;
  if (mg->precision) vcycle32(mg, r, z);
  else vcycle64(mg, r, z);
}

/* ------------------------------------------------------------------------- */
/* Krylov solvers (Sec. 5.2: CG and GMRES following hypre's algorithms)      */
/* ------------------------------------------------------------------------- */

static double dot(long n, const double* a, const double* b) {
  double s = 0.0;
  for (long t = 0; t < n; ++t) s += a[t] * b[t];
  return s;
}

/* Preconditioned CG with the V-cycle as M^{-1}; stop when ||r_k||_2/||b||_2 <
 * tol on the recursively updated residual.  flexible != 0 selects the
 * Polak-Ribiere beta = <z_{k+1}, r_{k+1} - r_k> / <z_k, r_k>.  On exit relres
 * holds the TRUE residual ||b - A x||/||b||.  hist (optional, maxit+1 long)
 * receives the recursive relative residual of every iteration. */
int orc_pcg(void* h, const double* b, double* x, double tol, int maxit, int flexible, int* iters, double* relres,
            double* hist) {
  orc_mg* mg = (orc_mg*)h;
  orc_level* L = &mg->lev[0];
  long n = npts(L->d) * mg->B;
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n),
         *q = malloc(sizeof(double) * n), *rold = malloc(sizeof(double) * n);
  int rc = ORC_ENOTCONV, it = 0;
  orc_residual(L->d, L->ns, L->off, mg->B, L->A, b, x, r);
  double bn = sqrt(dot(n, b, b));
  if (bn == 0.0) {
    for (long t = 0; t < n; ++t) x[t] = 0.0;
    *iters = 0; *relres = 0.0; rc = ORC_OK; goto done;
  }
  double rn = sqrt(dot(n, r, r));
  if (hist) hist[0] = rn / bn;
  if (rn / bn < tol) { rc = ORC_OK; goto fin; }
  orc_mg_vcycle(h, r, z);
  memcpy(p, z, sizeof(double) * n);
  double rho = dot(n, r, z);
  for (it = 1; it <= maxit; ++it) {
    orc_spmv(L->d, L->ns, L->off, mg->B, L->A, p, q);
    double pq = dot(n, p, q);
    if (!(pq > 0.0)) { rc = (pq != pq) ? ORC_ENAN : ORC_EBREAKDOWN; goto fin; }
    double alpha = rho / pq;
    if (flexible) memcpy(rold, r, sizeof(double) * n);
    for (long t = 0; t < n; ++t) { x[t] += alpha * p[t]; r[t] -= alpha * q[t]; }
    rn = sqrt(dot(n, r, r));
    if (hist) hist[it] = rn / bn;
    if (rn != rn) { rc = ORC_ENAN; goto fin; }
    if (rn / bn < tol) { rc = ORC_OK; goto fin; }
    if (it == maxit) break;
    orc_mg_vcycle(h, r, z);
    double rz = dot(n, r, z), num = rz;
    if (flexible) {
      num = 0.0;
      for (long t = 0; t < n; ++t) num += z[t] * (r[t] - rold[t]);
    }
    double beta = num / rho;
    rho = rz;
    for (long t = 0; t < n; ++t) p[t] = z[t] + beta * p[t];
  }
  it = maxit;
fin:
  *iters = it;
  orc_residual(L->d, L->ns, L->off, mg->B, L->A, b, x, r);
  *relres = sqrt(dot(n, r, r)) / bn;
done:
  free(r); free(z); free(p); free(q); free(rold);
  return rc;
}

/* Right-preconditioned flexible GMRES(m): Arnoldi on A M^{-1} with the
 * preconditioned directions Z kept, classical Gram-Schmidt applied twice,
 * Givens rotations for the least-squares problem; the true residual is
 * recomputed at every restart and at exit.  iters counts Arnoldi steps. */
int orc_fgmres(void* h, const double* b, double* x, double tol, int maxit, int m, int* iters, double* relres,
               double* hist) {
  orc_mg* mg = (orc_mg*)h;
  orc_level* L = &mg->lev[0];
  long n = npts(L->d) * mg->B;
  double* V = malloc(sizeof(double) * n * (m + 1));
  double* Z = malloc(sizeof(double) * n * m);
  double* H = calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = malloc(sizeof(double) * m), *sn = malloc(sizeof(double) * m), *g = malloc(sizeof(double) * (m + 1));
  double *w = malloc(sizeof(double) * n), *hh = malloc(sizeof(double) * (m + 1)), *y = malloc(sizeof(double) * m);
  int rc = ORC_ENOTCONV, total = 0;
  double bn = sqrt(dot(n, b, b));
  if (bn == 0.0) {
    for (long t = 0; t < n; ++t) x[t] = 0.0;
    *iters = 0; *relres = 0.0; rc = ORC_OK; goto done;
  }
  orc_residual(L->d, L->ns, L->off, mg->B, L->A, b, x, w);
  double beta = sqrt(dot(n, w, w));
  if (hist) hist[0] = beta / bn;
  while (beta / bn >= tol && total < maxit) {
    for (long t = 0; t < n; ++t) V[t] = w[t] / beta;
    for (int t = 0; t <= m; ++t) g[t] = 0.0;
    g[0] = beta;
    int j, jdone = 0;
    for (j = 0; j < m && total < maxit; ++j) {
      double* vj = V + (long)j * n;
      double* zj = Z + (long)j * n;
      orc_mg_vcycle(h, vj, zj);
      orc_spmv(L->d, L->ns, L->off, mg->B, L->A, zj, w);
      for (int i = 0; i <= j; ++i) hh[i] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        double c[64];
        for (int i = 0; i <= j; ++i) c[i] = dot(n, V + (long)i * n, w);
        for (int i = 0; i <= j; ++i) {
          for (long t = 0; t < n; ++t) w[t] -= c[i] * V[(long)i * n + t];
          hh[i] += c[i];
        }
      }
      double hn = sqrt(dot(n, w, w));
      for (int i = 0; i <= j; ++i) H[i * m + j] = hh[i];
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (long t = 0; t < n; ++t) V[(long)(j + 1) * n + t] = w[t] / hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[j * m + j], bb = H[(j + 1) * m + j];
      double den = sqrt(a * a + bb * bb);
      cs[j] = den == 0.0 ? 1.0 : a / den;
      sn[j] = den == 0.0 ? 0.0 : bb / den;
      H[j * m + j] = cs[j] * a + sn[j] * bb;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      jdone = j + 1;
      if (hist) hist[total] = fabs(g[j + 1]) / bn;
      if (fabs(g[j + 1]) / bn < tol || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < jdone; ++t) s -= H[i * m + t] * y[t];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < jdone; ++i)
      for (long t = 0; t < n; ++t) x[t] += y[i] * Z[(long)i * n + t];
    orc_residual(L->d, L->ns, L->off, mg->B, L->A, b, x, w);
    beta = sqrt(dot(n, w, w));
    if (beta != beta) { rc = ORC_ENAN; break; }
  }
  if (beta / bn < tol) rc = ORC_OK;
  *iters = total;
  *relres = beta / bn;
done:
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(w); free(hh); free(y);
  return rc;
}
