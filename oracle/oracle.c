/*
 * place3d oracle (FP64, CPU).  TEST INFRASTRUCTURE ONLY: loaded by the tests,
 * the smoke check and the bench's CPU legs, never by the product path.
 * Independent of the CUDA path: no shared code, headers or tables.
 *
 * Every function follows the paper (arXiv 2403.09070) step by step; the
 * section / equation each one restates is named beside it.  Readings taken
 * where the paper is silent or ambiguous:
 *   R1 local smoothness: the footprint is stretched to max(w, sqrt2 w_b) x
 *      max(h, sqrt2 h_b) and weighted by omega, so that omega x stretched area
 *      = w h (charge preserved).  Applied to every instance.
 *   R2 Poisson: the cosine series carries weights c_0 = 1, c_j>0 = 2 per axis
 *      so that it reproduces rho at bin centres; the DC term is dropped.
 *   R3 energy U = 1/2 vol(b) sum_b rho_b phi_b; its gradient is taken as the
 *      field gather -omega sum_b vol(D cap b) E_b (E = -grad phi).
 *   R4 the bistratal max is taken on the smoothed values, ties to the
 *      whole-net branch; an empty side has p = 0.
 *   R5 the FD depth gradient uses the exact W_Bi and switches the moved
 *      instance's pin offsets to the other die; z = d_z/2 counts as bottom.
 *   R6 g = (S_x + S_y) / (2 S_z), and 0 when S_z = 0.
 *   R7 gamma_z <= 0 means gamma_z = gamma; net weights are 1.
 *   R8 overlaps are clipped to the region; macro corners are clamped to it.
 *   R9 macro size factor t = 2 z / d_z - 1/2 is clamped to [0, 1].
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* Sec. II-A region Omega = [0,d_x]x[0,d_y]x[0,d_z]; Sec. V-A d_b, d_z. */
void orc_geometry(const orc_problem *p, double out[6]) {
  double dx = p->xh - p->xl, dy = p->yh - p->yl;
  double wb = dx / p->nx, hb = dy / p->ny;
  double db = 0.5 * (wb + hb);
  out[0] = wb;
  out[1] = hb;
  out[2] = db;
  out[3] = dx;
  out[4] = dy;
  out[5] = p->nz * db;
}

/* Sec. V-A: alpha = alpha0 (d_x eta^2 / d_z) log(90 beta eta - 1),
 * alpha0 = 3.5e-3, eta = 2 w' / (RH+ + RH-). */
double orc_alpha(double dx, double dz, double beta, double w_hbt, double rh_top,
                 double rh_bot) {
  double eta = 2.0 * w_hbt / (rh_top + rh_bot);
  return 3.5e-3 * (dx * eta * eta / dz) * log(90.0 * beta * eta - 1.0);
}

/* Partition, dynamic size and local smoothness of one instance.
 * delta: Sec. II-B, delta_i = 1 if z_i - d_z/2 > 0.
 * std cells: eq. std-size-tech (size of the die the cell sits on).
 * macros: eq. macro-size-tech, linear in z (R9).
 * omega and stretched size: Sec. IV-A local smoothness (R1). */
static int is_hbt(const orc_problem *p, int i) {
  return p->mode == 1 && p->is_hbt && p->is_hbt[i];
}

static void attr_one(const orc_problem *p, const double g[6], int i, double zi,
                     int *delta, double *w, double *h, double *sw, double *sh,
                     double *om) {
  double dz = g[5];
  int top = zi - 0.5 * dz > 0.0;
  double ww, hh;
  if (is_hbt(p, i)) { /* 2D mode: an HBT has one footprint (Sec. V-B) */
    top = 0;
    ww = p->w_bot[i];
    hh = p->h_bot[i];
  } else if (p->is_macro[i] && p->mode != 1) {
    double t = 2.0 * zi / dz - 0.5; /* weight of the top-die size */
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    ww = t * p->w_top[i] + (1.0 - t) * p->w_bot[i];
    hh = t * p->h_top[i] + (1.0 - t) * p->h_bot[i];
  } else {
    ww = top ? p->w_top[i] : p->w_bot[i];
    hh = top ? p->h_top[i] : p->h_bot[i];
  }
  double rw = sqrt(2.0) * g[0], rh = sqrt(2.0) * g[1];
  if (delta) *delta = top;
  if (w) *w = ww;
  if (h) *h = hh;
  if (sw) *sw = dmax(ww, rw);
  if (sh) *sh = dmax(hh, rh);
  if (om) *om = dmin(1.0, ww / rw) * dmin(1.0, hh / rh);
}

void orc_attributes(const orc_problem *p, const double *x, const double *y,
                    const double *z, int *delta, double *w, double *h,
                    double *sw, double *sh, double *omega) {
  double g[6];
  (void)x;
  (void)y;
  orc_geometry(p, g);
  for (int i = 0; i < p->n_inst; ++i)
    attr_one(p, g, i, z[i], delta ? delta + i : NULL, w ? w + i : NULL,
             h ? h + i : NULL, sw ? sw + i : NULL, sh ? sh + i : NULL,
             omega ? omega + i : NULL);
}

/* Length of [a0,a1] cap [b0,b1]. */
static double overlap(double a0, double a1, double b0, double b1) {
  return dmax(0.0, dmin(a1, b1) - dmax(a0, b0));
}

/* Bin index range [lo, hi] that may overlap [a0, a1] on an axis starting at
 * origin with bin size s and n bins (one bin of margin on each side). */
static void bin_range(double a0, double a1, double origin, double s, int n,
                      int *lo, int *hi) {
  int l = (int)floor((a0 - origin) / s) - 1;
  int h = (int)floor((a1 - origin) / s) + 1;
  *lo = l < 0 ? 0 : l;
  *hi = h > n - 1 ? n - 1 : h;
}

/* Cuboid D_i of Sec. IV-A with the stretched footprint (R1). */
static void box_of(const orc_problem *p, const double g[6], int i,
                   const double *x, const double *y, const double *z,
                   double b[6], double *om) {
  double sw, sh;
  attr_one(p, g, i, z[i], NULL, NULL, NULL, &sw, &sh, om);
  b[0] = x[i] - 0.5 * sw;
  b[1] = x[i] + 0.5 * sw;
  b[2] = y[i] - 0.5 * sh;
  b[3] = y[i] + 0.5 * sh;
  b[4] = z[i] - 0.25 * g[5]; /* depth d_z/2 (Sec. III-A) */
  b[5] = z[i] + 0.25 * g[5];
  if (p->mode == 1) { /* 2D mode: the instance fills its layer's one bin in z */
    int layer = is_hbt(p, i) ? 2 : (z[i] - 0.5 * g[5] > 0.0);
    b[4] = layer * g[2];
    b[5] = (layer + 1) * g[2];
  }
}

/* Eq. density-map-accum: rho_b = sum_i omega_i vol(D_i cap b) / vol(b). */
void orc_density_direct(const orc_problem *p, const double *x, const double *y,
                        const double *z, double *rho) {
  double g[6];
  orc_geometry(p, g);
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const double volb = g[0] * g[1] * g[2];
  memset(rho, 0, sizeof(double) * (size_t)nx * ny * nz);
  for (int i = 0; i < p->n_inst; ++i) {
    double b[6], om;
    box_of(p, g, i, x, y, z, b, &om);
    int i0, i1, j0, j1, k0, k1;
    bin_range(b[0], b[1], p->xl, g[0], nx, &i0, &i1);
    bin_range(b[2], b[3], p->yl, g[1], ny, &j0, &j1);
    bin_range(b[4], b[5], 0.0, g[2], nz, &k0, &k1);
    for (int k = k0; k <= k1; ++k) {
      double oz = overlap(b[4], b[5], k * g[2], (k + 1) * g[2]);
      if (oz <= 0) continue;
      for (int j = j0; j <= j1; ++j) {
        double oy = overlap(b[2], b[3], p->yl + j * g[1], p->yl + (j + 1) * g[1]);
        if (oy <= 0) continue;
        for (int ii = i0; ii <= i1; ++ii) {
          double ox = overlap(b[0], b[1], p->xl + ii * g[0], p->xl + (ii + 1) * g[0]);
          if (ox <= 0) continue;
          rho[((size_t)k * ny + j) * nx + ii] += om * ox * oy * oz / volb;
        }
      }
    }
  }
}

/* g(a) = max{1 - |a|, 0} of eq. 3d-density-accum-corner. */
static double gtri(double a) { return dmax(1.0 - fabs(a), 0.0); }

/* Theorem 1 / eq. 3d-density-accum-cuboid: A_v = sum over the 8 corners of
 * -sigma_x sigma_y sigma_z A^(corner), A^(c)_ijk = g(i - x^) g(j - y^) g(k - z^)
 * with 0-based bin indices (the reading that reproduces Fig. prefix-example)
 * and (x^, y^, z^) the corner in bin units, clamped to [0, N] (R8).  Scaled by
 * the instance's omega. */
void orc_macro_corner_map(const orc_problem *p, const double *x,
                          const double *y, const double *z, double *A) {
  double g[6];
  orc_geometry(p, g);
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  memset(A, 0, sizeof(double) * (size_t)nx * ny * nz);
  for (int i = 0; i < p->n_inst; ++i) {
    if (!p->is_macro[i]) continue;
    double b[6], om;
    box_of(p, g, i, x, y, z, b, &om);
    for (int sx = -1; sx <= 1; sx += 2)
      for (int sy = -1; sy <= 1; sy += 2)
        for (int sz = -1; sz <= 1; sz += 2) {
          double cx = ((sx < 0 ? b[0] : b[1]) - p->xl) / g[0];
          double cy = ((sy < 0 ? b[2] : b[3]) - p->yl) / g[1];
          double cz = (sz < 0 ? b[4] : b[5]) / g[2];
          cx = dmin(dmax(cx, 0.0), (double)nx);
          cy = dmin(dmax(cy, 0.0), (double)ny);
          cz = dmin(dmax(cz, 0.0), (double)nz);
          double sign = -(double)(sx * sy * sz);
          int fx = (int)floor(cx), fy = (int)floor(cy), fz = (int)floor(cz);
          for (int k = fz; k <= fz + 1; ++k) {
            if (k < 0 || k >= nz) continue;
            for (int j = fy; j <= fy + 1; ++j) {
              if (j < 0 || j >= ny) continue;
              for (int ii = fx; ii <= fx + 1; ++ii) {
                if (ii < 0 || ii >= nx) continue;
                A[((size_t)k * ny + j) * nx + ii] +=
                    sign * om * gtri(ii - cx) * gtri(j - cy) * gtri(k - cz);
              }
            }
          }
        }
  }
}

/* Eq. def-prefix-sum-3d, inclusive, as three running sums. */
void orc_prefix_sum3(double *a, int nx, int ny, int nz) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i)
        a[((size_t)k * ny + j) * nx + i] += a[((size_t)k * ny + j) * nx + i - 1];
  for (int k = 0; k < nz; ++k)
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        a[((size_t)k * ny + j) * nx + i] += a[((size_t)k * ny + j - 1) * nx + i];
  for (int k = 1; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        a[((size_t)k * ny + j) * nx + i] += a[((size_t)(k - 1) * ny + j) * nx + i];
}

void orc_prefix_sum3_i64(int64_t *a, int nx, int ny, int nz) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i)
        a[((size_t)k * ny + j) * nx + i] += a[((size_t)k * ny + j) * nx + i - 1];
  for (int k = 0; k < nz; ++k)
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        a[((size_t)k * ny + j) * nx + i] += a[((size_t)k * ny + j - 1) * nx + i];
  for (int k = 1; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        a[((size_t)k * ny + j) * nx + i] += a[((size_t)(k - 1) * ny + j) * nx + i];
}

/* Fixed-point replica in float and in double (same steps, two precisions). */
#define REAL double
#define SUF _d
#define RFLOOR floor
#define RCEIL ceil
#define RRINT llrint
#include "oracle_fixed.inc"
#undef REAL
#undef SUF
#undef RFLOOR
#undef RCEIL
#undef RRINT
#define REAL float
#define SUF _f
#define RFLOOR floorf
#define RCEIL ceilf
#define RRINT llrintf
#include "oracle_fixed.inc"
#undef REAL
#undef SUF
#undef RFLOOR
#undef RCEIL
#undef RRINT

void orc_density_fixed(const orc_problem *p, const double *x, const double *y,
                       const double *z, int use_float, int64_t *q) {
  if (use_float)
    density_fixed_f(p, x, y, z, q);
  else
    density_fixed_d(p, x, y, z, q);
}

/* out[..., o, ...] = sum_t M[o][t] in[..., t, ...] along one axis of a
 * [nz][ny][nx] array (axis 0 = x, 1 = y, 2 = z); M is n x n. */
static void apply_axis(const double *in, double *out, int nx, int ny, int nz,
                       int axis, const double *M) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        if (axis == 0)
          for (int t = 0; t < nx; ++t)
            s += M[(size_t)i * nx + t] * in[((size_t)k * ny + j) * nx + t];
        else if (axis == 1)
          for (int t = 0; t < ny; ++t)
            s += M[(size_t)j * ny + t] * in[((size_t)k * ny + t) * nx + i];
        else
          for (int t = 0; t < nz; ++t)
            s += M[(size_t)k * nz + t] * in[((size_t)t * ny + j) * nx + i];
        out[((size_t)k * ny + j) * nx + i] = s;
      }
}

/* Basis matrices of eqs. density-coef .. possion-sol-force on bin centres
 * u_i = (i + 1/2) * (d / n):  cos(omega_j u_i) = cos(pi j (i + 1/2) / n).
 * kind 0: F[j][i] = cos (forward);  1: C[i][j] = cos (inverse);
 * kind 2: S[i][j] = omega_j sin(omega_j u_i) with omega_j = j pi / d. */
static double *basis(int n, double d, int kind) {
  double *M = (double *)malloc(sizeof(double) * (size_t)n * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      int j = kind == 0 ? r : c, i = kind == 0 ? c : r;
      double arg = ORC_PI * j * (i + 0.5) / n;
      M[(size_t)r * n + c] = kind == 2 ? (j * ORC_PI / d) * sin(arg) : cos(arg);
    }
  return M;
}

/* Eqs. density-coef, poisson-sol-potential, possion-sol-force (R2, R3). */
void orc_poisson(const orc_problem *p, const double *rho, double *a_out,
                 double *psi_out, double *phi, double *ex, double *ey,
                 double *ez, double *energy) {
  double g[6];
  orc_geometry(p, g);
  if (p->mode == 1) {
    /* eq. 2d-place: each layer an independent 2D field.  A one-layer 3D
     * solve is the 2D cosine series (the only z index is 0, E_z = 0); its
     * energy 1/2 w_b h_b d_b N sum c a^2/omega^2 is d_b times the 2D energy
     * 1/2 A_b sum rho phi.  energy[l] receives layer l's. */
    orc_problem q = *p;
    q.mode = 0;
    q.nz = 1;
    const size_t pl = (size_t)p->nx * p->ny;
    for (int l = 0; l < p->nz; ++l) {
      double e = 0.0;
#define ORC_AT(ptr) ((ptr) ? (ptr) + l * pl : NULL)
      orc_poisson(&q, rho + l * pl, ORC_AT(a_out), ORC_AT(psi_out), ORC_AT(phi), ORC_AT(ex), ORC_AT(ey),
                  ORC_AT(ez), &e);
#undef ORC_AT
      if (energy) energy[l] = e / g[2];
    }
    return;
  }
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t nb = (size_t)nx * ny * nz;
  double *Fx = basis(nx, g[3], 0), *Fy = basis(ny, g[4], 0), *Fz = basis(nz, g[5], 0);
  double *Cx = basis(nx, g[3], 1), *Cy = basis(ny, g[4], 1), *Cz = basis(nz, g[5], 1);
  double *Sx = basis(nx, g[3], 2), *Sy = basis(ny, g[4], 2), *Sz = basis(nz, g[5], 2);
  double *t1 = (double *)malloc(sizeof(double) * nb);
  double *t2 = (double *)malloc(sizeof(double) * nb);
  double *a = (double *)malloc(sizeof(double) * nb);
  double *psi = (double *)malloc(sizeof(double) * nb);
  /* a_jkl = (1/N) sum rho cos cos cos */
  apply_axis(rho, t1, nx, ny, nz, 0, Fx);
  apply_axis(t1, t2, nx, ny, nz, 1, Fy);
  apply_axis(t2, a, nx, ny, nz, 2, Fz);
  const double N = (double)nb;
  double esum = 0.0;
  for (int l = 0; l < nz; ++l)
    for (int k = 0; k < ny; ++k)
      for (int j = 0; j < nx; ++j) {
        size_t id = ((size_t)l * ny + k) * nx + j;
        a[id] /= N;
        double wj = j * ORC_PI / g[3], wk = k * ORC_PI / g[4], wl = l * ORC_PI / g[5];
        double w2 = wj * wj + wk * wk + wl * wl;
        double c = (j ? 2.0 : 1.0) * (k ? 2.0 : 1.0) * (l ? 2.0 : 1.0);
        if (j == 0 && k == 0 && l == 0) {
          psi[id] = 0.0;
        } else {
          psi[id] = c * a[id] / w2;
          esum += c * a[id] * a[id] / w2;
        }
      }
  if (energy) *energy = 0.5 * (g[0] * g[1] * g[2]) * N * esum;
  if (a_out) memcpy(a_out, a, sizeof(double) * nb);
  if (psi_out) memcpy(psi_out, psi, sizeof(double) * nb);
  /* phi = C C C psi ; E_x = S_x C_y C_z psi ; ... (axis order z, y, x) */
  if (phi) {
    apply_axis(psi, t1, nx, ny, nz, 2, Cz);
    apply_axis(t1, t2, nx, ny, nz, 1, Cy);
    apply_axis(t2, phi, nx, ny, nz, 0, Cx);
  }
  if (ex) {
    apply_axis(psi, t1, nx, ny, nz, 2, Cz);
    apply_axis(t1, t2, nx, ny, nz, 1, Cy);
    apply_axis(t2, ex, nx, ny, nz, 0, Sx);
  }
  if (ey) {
    apply_axis(psi, t1, nx, ny, nz, 2, Cz);
    apply_axis(t1, t2, nx, ny, nz, 1, Sy);
    apply_axis(t2, ey, nx, ny, nz, 0, Cx);
  }
  if (ez) {
    apply_axis(psi, t1, nx, ny, nz, 2, Sz);
    apply_axis(t1, t2, nx, ny, nz, 1, Cy);
    apply_axis(t2, ez, nx, ny, nz, 0, Cx);
  }
  free(Fx); free(Fy); free(Fz); free(Cx); free(Cy); free(Cz);
  free(Sx); free(Sy); free(Sz); free(t1); free(t2); free(a); free(psi);
}

/* The series of eqs. density-coef .. possion-sol-force written out term by
 * term with physical bin-centre coordinates (tiny grids). */
void orc_poisson_series_direct(const orc_problem *p, const double *rho,
                               double *a_out, double *phi, double *ex,
                               double *ey, double *ez) {
  double g[6];
  orc_geometry(p, g);
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t nb = (size_t)nx * ny * nz;
  double *a = (double *)calloc(nb, sizeof(double));
  for (int l = 0; l < nz; ++l)
    for (int k = 0; k < ny; ++k)
      for (int j = 0; j < nx; ++j) {
        double wj = j * ORC_PI / g[3], wk = k * ORC_PI / g[4], wl = l * ORC_PI / g[5];
        double s = 0.0;
        for (int bz = 0; bz < nz; ++bz)
          for (int by = 0; by < ny; ++by)
            for (int bx = 0; bx < nx; ++bx) {
              double X = (bx + 0.5) * g[0], Y = (by + 0.5) * g[1], Z = (bz + 0.5) * g[2];
              s += rho[((size_t)bz * ny + by) * nx + bx] * cos(wj * X) * cos(wk * Y) * cos(wl * Z);
            }
        a[((size_t)l * ny + k) * nx + j] = s / (double)nb;
      }
  if (a_out) memcpy(a_out, a, sizeof(double) * nb);
  for (int bz = 0; bz < nz; ++bz)
    for (int by = 0; by < ny; ++by)
      for (int bx = 0; bx < nx; ++bx) {
        double X = (bx + 0.5) * g[0], Y = (by + 0.5) * g[1], Z = (bz + 0.5) * g[2];
        double sp = 0, sx = 0, sy = 0, sz = 0;
        for (int l = 0; l < nz; ++l)
          for (int k = 0; k < ny; ++k)
            for (int j = 0; j < nx; ++j) {
              if (!j && !k && !l) continue;
              double wj = j * ORC_PI / g[3], wk = k * ORC_PI / g[4], wl = l * ORC_PI / g[5];
              double c = (j ? 2.0 : 1.0) * (k ? 2.0 : 1.0) * (l ? 2.0 : 1.0);
              double coef = c * a[((size_t)l * ny + k) * nx + j] / (wj * wj + wk * wk + wl * wl);
              sp += coef * cos(wj * X) * cos(wk * Y) * cos(wl * Z);
              sx += coef * wj * sin(wj * X) * cos(wk * Y) * cos(wl * Z);
              sy += coef * wk * cos(wj * X) * sin(wk * Y) * cos(wl * Z);
              sz += coef * wl * cos(wj * X) * cos(wk * Y) * sin(wl * Z);
            }
        size_t id = ((size_t)bz * ny + by) * nx + bx;
        if (phi) phi[id] = sp;
        if (ex) ex[id] = sx;
        if (ey) ey[id] = sy;
        if (ez) ez[id] = sz;
      }
  free(a);
}

/* Sec. III-A "the electric force is q_i E_i", as the field gather of R3. */
void orc_density_grad_gather(const orc_problem *p, const double *x,
                             const double *y, const double *z,
                             const double *ex, const double *ey,
                             const double *ez, double *gx, double *gy,
                             double *gz) {
  double g[6];
  orc_geometry(p, g);
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  for (int i = 0; i < p->n_inst; ++i) {
    double b[6], om;
    box_of(p, g, i, x, y, z, b, &om);
    int i0, i1, j0, j1, k0, k1;
    bin_range(b[0], b[1], p->xl, g[0], nx, &i0, &i1);
    bin_range(b[2], b[3], p->yl, g[1], ny, &j0, &j1);
    bin_range(b[4], b[5], 0.0, g[2], nz, &k0, &k1);
    double sx = 0, sy = 0, sz = 0;
    for (int k = k0; k <= k1; ++k) {
      double oz = overlap(b[4], b[5], k * g[2], (k + 1) * g[2]);
      if (oz <= 0) continue;
      for (int j = j0; j <= j1; ++j) {
        double oy = overlap(b[2], b[3], p->yl + j * g[1], p->yl + (j + 1) * g[1]);
        if (oy <= 0) continue;
        for (int ii = i0; ii <= i1; ++ii) {
          double ox = overlap(b[0], b[1], p->xl + ii * g[0], p->xl + (ii + 1) * g[0]);
          if (ox <= 0) continue;
          size_t id = ((size_t)k * ny + j) * nx + ii;
          double v = ox * oy * oz;
          sx += v * ex[id];
          sy += v * ey[id];
          sz += v * ez[id];
        }
      }
    }
    gx[i] = -om * sx;
    gy[i] = -om * sy;
    gz[i] = -om * sz;
  }
}

/* Backward of Theorem 1 (Sec. IV-A, last paragraphs): the prefix sum's
 * adjoint is the suffix sum; sum_b phi(A_v)_b E_b = sum_b A_v,b S_b with
 * S_b = sum_{b' >= b} E_b'. */
void orc_macro_grad_suffix(const orc_problem *p, const double *x,
                           const double *y, const double *z, const double *ex,
                           const double *ey, const double *ez, double *gx,
                           double *gy, double *gz) {
  double g[6];
  orc_geometry(p, g);
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t nb = (size_t)nx * ny * nz;
  const double volb = g[0] * g[1] * g[2];
  const double *E[3] = {ex, ey, ez};
  double *S[3];
  for (int c = 0; c < 3; ++c) {
    S[c] = (double *)malloc(sizeof(double) * nb);
    /* suffix sum = reversed array, prefix sum, reversed back */
    for (size_t t = 0; t < nb; ++t) {
      size_t k = t / ((size_t)nx * ny), j = (t / nx) % ny, i = t % nx;
      size_t r = ((size_t)(nz - 1 - k) * ny + (ny - 1 - j)) * nx + (nx - 1 - i);
      S[c][r] = E[c][t];
    }
    orc_prefix_sum3(S[c], nx, ny, nz);
    for (size_t t = 0; t < nb / 2; ++t) {
      double tmp = S[c][t];
      S[c][t] = S[c][nb - 1 - t];
      S[c][nb - 1 - t] = tmp;
    }
  }
  for (int i = 0; i < p->n_inst; ++i) {
    if (!p->is_macro[i]) continue;
    double b[6], om;
    box_of(p, g, i, x, y, z, b, &om);
    double acc[3] = {0, 0, 0};
    for (int sx = -1; sx <= 1; sx += 2)
      for (int sy = -1; sy <= 1; sy += 2)
        for (int sz = -1; sz <= 1; sz += 2) {
          double cx = dmin(dmax(((sx < 0 ? b[0] : b[1]) - p->xl) / g[0], 0.0), (double)nx);
          double cy = dmin(dmax(((sy < 0 ? b[2] : b[3]) - p->yl) / g[1], 0.0), (double)ny);
          double cz = dmin(dmax((sz < 0 ? b[4] : b[5]) / g[2], 0.0), (double)nz);
          double sign = -(double)(sx * sy * sz);
          int fx = (int)floor(cx), fy = (int)floor(cy), fz = (int)floor(cz);
          for (int k = fz; k <= fz + 1; ++k) {
            if (k < 0 || k >= nz) continue;
            for (int j = fy; j <= fy + 1; ++j) {
              if (j < 0 || j >= ny) continue;
              for (int ii = fx; ii <= fx + 1; ++ii) {
                if (ii < 0 || ii >= nx) continue;
                double a = sign * gtri(ii - cx) * gtri(j - cy) * gtri(k - cz);
                size_t id = ((size_t)k * ny + j) * nx + ii;
                for (int c = 0; c < 3; ++c) acc[c] += a * S[c][id];
              }
            }
          }
        }
    gx[i] = -om * volb * acc[0];
    gy[i] = -om * volb * acc[1];
    gz[i] = -om * volb * acc[2];
  }
  for (int c = 0; c < 3; ++c) free(S[c]);
}

/* dU/dx_i for U = 1/2 vol(b) sum rho phi: vol(b) sum_b (d rho_b / d x_i)
 * phi_b; only the bins that hold a face of D_i change, by +-omega times the
 * overlap of the other two axes over vol(b). */
void orc_density_grad_exact(const orc_problem *p, const double *x,
                            const double *y, const double *z,
                            const double *phi, double *gx, double *gy,
                            double *gz) {
  double g[6];
  orc_geometry(p, g);
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  for (int i = 0; i < p->n_inst; ++i) {
    double b[6], om;
    box_of(p, g, i, x, y, z, b, &om);
    int i0, i1, j0, j1, k0, k1;
    bin_range(b[0], b[1], p->xl, g[0], nx, &i0, &i1);
    bin_range(b[2], b[3], p->yl, g[1], ny, &j0, &j1);
    bin_range(b[4], b[5], 0.0, g[2], nz, &k0, &k1);
    double sx = 0, sy = 0, sz = 0;
    for (int k = k0; k <= k1; ++k) {
      double z0 = k * g[2], z1 = (k + 1) * g[2];
      double oz = overlap(b[4], b[5], z0, z1);
      double dz = (b[5] > z0 && b[5] < z1 ? 1.0 : 0.0) - (b[4] > z0 && b[4] < z1 ? 1.0 : 0.0);
      for (int j = j0; j <= j1; ++j) {
        double y0 = p->yl + j * g[1], y1 = p->yl + (j + 1) * g[1];
        double oy = overlap(b[2], b[3], y0, y1);
        double dy = (b[3] > y0 && b[3] < y1 ? 1.0 : 0.0) - (b[2] > y0 && b[2] < y1 ? 1.0 : 0.0);
        for (int ii = i0; ii <= i1; ++ii) {
          double x0 = p->xl + ii * g[0], x1 = p->xl + (ii + 1) * g[0];
          double ox = overlap(b[0], b[1], x0, x1);
          double dx = (b[1] > x0 && b[1] < x1 ? 1.0 : 0.0) - (b[0] > x0 && b[0] < x1 ? 1.0 : 0.0);
          double ph = phi[((size_t)k * ny + j) * nx + ii];
          sx += dx * oy * oz * ph;
          sy += ox * dy * oz * ph;
          sz += ox * oy * dz * ph;
        }
      }
    }
    gx[i] = om * sx;
    gy[i] = om * sy;
    gz[i] = om * sz;
  }
}

/* ---------------------------- wirelength ------------------------------ */

/* Eq. wa-model-approx over the pins k with mask[k] != 0 (WA of one axis).
 * The exponent is shifted by the set's max (resp. min); the common factor
 * cancels in each ratio.  Returns 0 for an empty set.  If grad != NULL,
 * grad[k] = d p^ / d v_k for members (left untouched for others). */
static double wa_axis(const double *v, const unsigned char *mask, int d,
                      double gamma, double *grad) {
  double vmax = -DBL_MAX, vmin = DBL_MAX;
  int n = 0;
  for (int k = 0; k < d; ++k)
    if (mask[k]) {
      vmax = dmax(vmax, v[k]);
      vmin = dmin(vmin, v[k]);
      ++n;
    }
  if (n == 0) return 0.0;
  double s1 = 0, n1 = 0, s2 = 0, n2 = 0;
  for (int k = 0; k < d; ++k)
    if (mask[k]) {
      double e1 = exp((v[k] - vmax) / gamma), e2 = exp(-(v[k] - vmin) / gamma);
      s1 += e1;
      n1 += v[k] * e1;
      s2 += e2;
      n2 += v[k] * e2;
    }
  double M = n1 / s1, m = n2 / s2;
  if (grad)
    for (int k = 0; k < d; ++k)
      if (mask[k]) {
        double e1 = exp((v[k] - vmax) / gamma), e2 = exp(-(v[k] - vmin) / gamma);
        grad[k] = (e1 / s1) * (1.0 + (v[k] - M) / gamma) -
                  (e2 / s2) * (1.0 - (v[k] - m) / gamma);
      }
  return M - m;
}

/* Exact partial HPWL p(.) = max - min over a masked set; 0 if empty. */
static double hp_axis(const double *v, const unsigned char *mask, int d) {
  double vmax = -DBL_MAX, vmin = DBL_MAX;
  int n = 0;
  for (int k = 0; k < d; ++k)
    if (mask[k]) {
      vmax = dmax(vmax, v[k]);
      vmin = dmin(vmin, v[k]);
      ++n;
    }
  return n ? vmax - vmin : 0.0;
}

/* Eq. wl-obj per axis and W_Bi = W_ex + W_ey (Sec. III-A bistratal model). */
static double wbi_exact(const double *px, const double *py,
                        const unsigned char *top, int d, unsigned char *tmp) {
  unsigned char *all = tmp, *bot = tmp + d;
  for (int k = 0; k < d; ++k) {
    all[k] = 1;
    bot[k] = !top[k];
  }
  double wx = dmax(hp_axis(px, all, d), hp_axis(px, top, d) + hp_axis(px, bot, d));
  double wy = dmax(hp_axis(py, all, d), hp_axis(py, top, d) + hp_axis(py, bot, d));
  return wx + wy;
}

/* 1st and 2nd extremes of the top or bottom pins on one axis (the 1st and
 * 2nd outermost boxes of Sec. IV-B); argmax/argmin are pin slots. */
typedef struct {
  double max1, max2, min1, min2;
  int amax, amin, n;
} orc_ext;

static orc_ext extremes(const double *v, const unsigned char *top, int side,
                        int d) {
  orc_ext e = {-DBL_MAX, -DBL_MAX, DBL_MAX, DBL_MAX, -1, -1, 0};
  for (int k = 0; k < d; ++k) {
    if ((top[k] != 0) != (side != 0)) continue;
    e.n++;
    if (v[k] > e.max1) {
      e.max2 = e.max1;
      e.max1 = v[k];
      e.amax = k;
    } else if (v[k] > e.max2) {
      e.max2 = v[k];
    }
    if (v[k] < e.min1) {
      e.min2 = e.min1;
      e.min1 = v[k];
      e.amin = k;
    } else if (v[k] < e.min2) {
      e.min2 = v[k];
    }
  }
  return e;
}

/* W_e,x after pin k leaves side s (extremes es) for side 1-s (extremes eo)
 * at coordinate c: eq. wl-obj on the updated boxes, O(1). */
static double moved_axis(const orc_ext *es, const orc_ext *eo, int k, double c) {
  int ns = es->n - 1, no = eo->n + 1;
  double smax = 0, smin = 0, ps = 0;
  if (ns > 0) {
    smax = k == es->amax ? es->max2 : es->max1;
    smin = k == es->amin ? es->min2 : es->min1;
    ps = smax - smin;
  }
  double omax = eo->n ? dmax(eo->max1, c) : c;
  double omin = eo->n ? dmin(eo->min1, c) : c;
  double po = omax - omin;
  double amax = ns > 0 ? dmax(smax, omax) : omax;
  double amin = ns > 0 ? dmin(smin, omin) : omin;
  (void)no;
  return dmax(amax - amin, ps + po);
}

void orc_wirelength(const orc_problem *p, const double *x, const double *y,
                    const double *z, int fd_mode, double out[4], double *gx,
                    double *gy, double *gfd, double *gwaz) {
  double g[6];
  orc_geometry(p, g);
  const double dz = g[5];
  const double gam = p->gamma, gamz = p->gamma_z > 0 ? p->gamma_z : p->gamma;
  double wl_bi = 0, wl_z = 0, hpwl = 0, ncross = 0;
  for (int i = 0; i < p->n_inst; ++i) gx[i] = gy[i] = gfd[i] = gwaz[i] = 0.0;
  int dmax_ = 0;
  for (int e = 0; e < p->n_net; ++e) {
    int d = p->net_start[e + 1] - p->net_start[e];
    if (d > dmax_) dmax_ = d;
  }
  double *px = malloc(sizeof(double) * (dmax_ + 1)), *py = malloc(sizeof(double) * (dmax_ + 1));
  double *pz = malloc(sizeof(double) * (dmax_ + 1));
  double *qx = malloc(sizeof(double) * (dmax_ + 1)), *qy = malloc(sizeof(double) * (dmax_ + 1));
  double *ga = malloc(sizeof(double) * (dmax_ + 1)), *gs = malloc(sizeof(double) * (dmax_ + 1));
  unsigned char *top = malloc(dmax_ + 1), *bot = malloc(dmax_ + 1), *all = malloc(dmax_ + 1);
  unsigned char *top2 = malloc(dmax_ + 1), *tmp = malloc(2 * (dmax_ + 1));
  double *px2 = malloc(sizeof(double) * (dmax_ + 1)), *py2 = malloc(sizeof(double) * (dmax_ + 1));
  for (int e = 0; e < p->n_net; ++e) {
    const int s0 = p->net_start[e], d = p->net_start[e + 1] - s0;
    if (d < 2) continue; /* a one-pin net has zero length and zero gradient */
    for (int k = 0; k < d; ++k) {
      int pin = s0 + k, i = p->pin_inst[pin];
      int t = z[i] - 0.5 * dz > 0.0; /* delta_i, Sec. II-B */
      top[k] = (unsigned char)t;
      bot[k] = (unsigned char)!t;
      all[k] = 1;
      /* pin offsets follow the partition (Sec. III-A, as eq. std-size-tech) */
      px[k] = x[i] + (t ? p->off_tx[pin] : p->off_bx[pin]);
      py[k] = y[i] + (t ? p->off_ty[pin] : p->off_by[pin]);
      qx[k] = x[i] + (t ? p->off_bx[pin] : p->off_tx[pin]); /* on the other die */
      qy[k] = y[i] + (t ? p->off_by[pin] : p->off_ty[pin]);
      pz[k] = z[i];
    }
    /* smoothed bistratal wirelength, eq. wl-obj with WA on each p (R4) */
    for (int ax = 0; ax < 2; ++ax) {
      const double *v = ax ? py : px;
      double *G = ax ? gy : gx;
      double pa = wa_axis(v, all, d, gam, ga);
      double pt = wa_axis(v, top, d, gam, gs);
      double pb = wa_axis(v, bot, d, gam, gs);
      if (pa >= pt + pb) {
        wl_bi += pa;
        for (int k = 0; k < d; ++k) G[p->pin_inst[s0 + k]] += ga[k];
      } else {
        wl_bi += pt + pb;
        for (int k = 0; k < d; ++k) G[p->pin_inst[s0 + k]] += gs[k];
      }
    }
    /* HBT cost term alpha p^_e(z) (eq. wl-model) */
    wl_z += wa_axis(pz, all, d, gamz, ga);
    for (int k = 0; k < d; ++k) gwaz[p->pin_inst[s0 + k]] += ga[k];
    /* exact D2D HPWL (eq. wl-obj) and crossing indicator C_e (Sec. II-B) */
    double W = wbi_exact(px, py, top, d, tmp);
    hpwl += W;
    int nt = 0;
    for (int k = 0; k < d; ++k) nt += top[k];
    if (nt > 0 && nt < d) ncross += 1.0;
    /* FD depth gradient, eq. fda-grad: (4/d_z)(W(i on top) - W(i on bottom)) */
    if (fd_mode == 0) { /* vanilla: rebuild the boxes for every moved pin */
      for (int k = 0; k < d; ++k) {
        memcpy(px2, px, sizeof(double) * d);
        memcpy(py2, py, sizeof(double) * d);
        memcpy(top2, top, d);
        top2[k] = !top[k];
        px2[k] = qx[k];
        py2[k] = qy[k];
        double Wm = wbi_exact(px2, py2, top2, d, tmp);
        double dW = top[k] ? (W - Wm) : (Wm - W);
        gfd[p->pin_inst[s0 + k]] += (4.0 / dz) * dW;
      }
    } else { /* incremental (Sec. IV-B): 1st/2nd outermost top/bottom boxes */
      orc_ext ext[2][2];
      for (int ax = 0; ax < 2; ++ax)
        for (int s = 0; s < 2; ++s) ext[ax][s] = extremes(ax ? py : px, top, s, d);
      for (int k = 0; k < d; ++k) {
        int s = top[k];
        double Wm = moved_axis(&ext[0][s], &ext[0][1 - s], k, qx[k]) +
                    moved_axis(&ext[1][s], &ext[1][1 - s], k, qy[k]);
        double dW = s ? (W - Wm) : (Wm - W);
        gfd[p->pin_inst[s0 + k]] += (4.0 / dz) * dW;
      }
    }
  }
  out[0] = wl_bi;
  out[1] = wl_z;
  out[2] = hpwl;
  out[3] = ncross;
  free(px); free(py); free(pz); free(qx); free(qy); free(ga); free(gs);
  free(top); free(bot); free(all); free(top2); free(tmp); free(px2); free(py2);
}

/* Objective of eq. analytical-placement with W_e of eq. wl-model and the
 * gradient (grad_x, grad_y, g + alpha grad_z p^(z)) of eq. fda-normalize plus
 * lambda times the density gradient. */
void orc_eval(const orc_problem *p, const double *x, const double *y,
              const double *z, int density_mode, int fd_mode, double out[10],
              double *gx, double *gy, double *gz) {
  const int n = p->n_inst;
  const size_t nb = (size_t)p->nx * p->ny * p->nz;
  double wl[4];
  double *wgx = malloc(sizeof(double) * n), *wgy = malloc(sizeof(double) * n);
  double *wfd = malloc(sizeof(double) * n), *wgz = malloc(sizeof(double) * n);
  orc_wirelength(p, x, y, z, fd_mode, wl, wgx, wgy, wfd, wgz);
  /* eq. fda-normalize (R6) */
  double Sx = 0, Sy = 0, Sz = 0;
  for (int i = 0; i < n; ++i) {
    Sx += fabs(wgx[i]);
    Sy += fabs(wgy[i]);
    Sz += fabs(wfd[i]);
  }
  double gs = Sz > 0 ? (Sx + Sy) / (2.0 * Sz) : 0.0;
  /* density map, spectral solve, field gather */
  double *rho = malloc(sizeof(double) * nb);
  if (density_mode == 0) {
    orc_density_direct(p, x, y, z, rho);
  } else {
    int64_t *q = malloc(sizeof(int64_t) * nb);
    orc_density_fixed(p, x, y, z, density_mode == 2, q);
    for (size_t b = 0; b < nb; ++b) rho[b] = (double)q[b] * (1.0 / 68719476736.0);
    free(q);
  }
  double *ex = malloc(sizeof(double) * nb), *ey = malloc(sizeof(double) * nb);
  double *ez = malloc(sizeof(double) * nb);
  double energy = 0;
  orc_poisson(p, rho, NULL, NULL, NULL, ex, ey, ez, &energy);
  double *dgx = malloc(sizeof(double) * n), *dgy = malloc(sizeof(double) * n);
  double *dgz = malloc(sizeof(double) * n);
  orc_density_grad_gather(p, x, y, z, ex, ey, ez, dgx, dgy, dgz);
  if (gx && gy && gz)
    for (int i = 0; i < n; ++i) {
      gx[i] = wgx[i] + p->lambda * dgx[i];
      gy[i] = wgy[i] + p->lambda * dgy[i];
      gz[i] = gs * wfd[i] + p->alpha * wgz[i] + p->lambda * dgz[i];
      if (p->z_fixed && p->z_fixed[i]) gz[i] = 0.0;
    }
  out[0] = wl[0] + p->alpha * wl[1] + p->lambda * energy;
  out[1] = wl[0];
  out[2] = wl[1];
  out[3] = energy;
  out[4] = wl[2];
  out[5] = wl[3];
  out[6] = gs;
  out[7] = Sx;
  out[8] = Sy;
  out[9] = Sz;
  free(wgx); free(wgy); free(wfd); free(wgz); free(rho);
  free(ex); free(ey); free(ez); free(dgx); free(dgy); free(dgz);
}

/* Sec. III-A, eqs. filler-vol and free-filler-vol (see oracle.h). */
void orc_filler_plan(const orc_problem *p, const double *z, double u_top,
                     double u_bot, double out[11]) {
  double g[6];
  orc_geometry(p, g);
  const double depth = 0.5 * g[5];
  const double V = g[3] * g[4] * g[5];
  double vol_a = 0.0, sw_t = 0.0, sh_t = 0.0, sw_b = 0.0, sh_b = 0.0;
  long n_std = 0;
  for (int i = 0; i < p->n_inst; ++i) {
    double w, h;
    attr_one(p, g, i, z[i], NULL, &w, &h, NULL, NULL, NULL);
    vol_a += w * h * depth;
    if (!p->is_macro[i] && !(p->z_fixed && p->z_fixed[i])) {
      sw_t += p->w_top[i];
      sh_t += p->h_top[i];
      sw_b += p->w_bot[i];
      sh_b += p->h_bot[i];
      ++n_std;
    }
  }
  double vf_t = 0.5 * V * (1.0 - u_top);
  double vf_b = 0.5 * V * (1.0 - u_bot);
  double vfr = V - (vf_t + vf_b + vol_a);
  if (vfr < 0.0) vfr = 0.0;
  double wt = n_std ? sw_t / n_std : 0.0, ht = n_std ? sh_t / n_std : 0.0;
  double wb = n_std ? sw_b / n_std : 0.0, hb = n_std ? sh_b / n_std : 0.0;
  double unit_t = wt * ht * depth, unit_b = wb * hb * depth;
  double unit_fr = 0.5 * (unit_t + unit_b);
  out[0] = vol_a;
  out[1] = vf_t;
  out[2] = vf_b;
  out[3] = vfr;
  out[4] = wt;
  out[5] = ht;
  out[6] = wb;
  out[7] = hb;
  out[8] = unit_t > 0.0 ? floor(vf_t / unit_t + 0.5) : 0.0;
  out[9] = unit_b > 0.0 ? floor(vf_b / unit_b + 0.5) : 0.0;
  out[10] = unit_fr > 0.0 ? floor(vfr / unit_fr + 0.5) : 0.0;
}

/* ---------------- multi-die 2D mode (eq. 2d-place) ---------------- */

/* D2D wirelength of eq. exact-wirelength smoothed by eq. wa-model-approx,
 * partition fixed by z: per net, WA(top pins + HBT pins) + WA(bottom pins +
 * HBT pins) per axis.  out = {sum W^, exact D2D HPWL, #crossing nets}.
 * Pin position: instance centre + its die's offset (bottom offset for HBTs). */
static void wirelength2d(const orc_problem *p, const double *x, const double *y,
                         const double *z, double out[3], double *gx, double *gy) {
  double g[6];
  orc_geometry(p, g);
  const double dz = g[5];
  int dmax_ = 1;
  for (int e = 0; e < p->n_net; ++e) {
    int d = p->net_start[e + 1] - p->net_start[e];
    if (d > dmax_) dmax_ = d;
  }
  double *px = malloc(sizeof(double) * dmax_), *py = malloc(sizeof(double) * dmax_);
  double *gpx = malloc(sizeof(double) * dmax_), *gpy = malloc(sizeof(double) * dmax_);
  unsigned char *top = malloc(dmax_), *bot = malloc(dmax_);
  memset(gx, 0, sizeof(double) * p->n_inst);
  memset(gy, 0, sizeof(double) * p->n_inst);
  double wsum = 0, hsum = 0, ncross = 0;
  for (int e = 0; e < p->n_net; ++e) {
    const int s0 = p->net_start[e], d = p->net_start[e + 1] - s0;
    int nt = 0, nb = 0;
    for (int k = 0; k < d; ++k) {
      const int i = p->pin_inst[s0 + k];
      const int h = is_hbt(p, i);
      const int t = !h && z[i] - 0.5 * dz > 0.0;
      px[k] = x[i] + (t ? p->off_tx[s0 + k] : p->off_bx[s0 + k]);
      py[k] = y[i] + (t ? p->off_ty[s0 + k] : p->off_by[s0 + k]);
      top[k] = (unsigned char)(h || t);
      bot[k] = (unsigned char)(h || !t);
      nt += !h && t;
      nb += !h && !t;
    }
    if (nt > 0 && nb > 0) ncross += 1.0;
    for (int side = 0; side < 2; ++side) {
      const unsigned char *m = side ? top : bot;
      for (int k = 0; k < d; ++k) gpx[k] = gpy[k] = 0.0;
      wsum += wa_axis(px, m, d, p->gamma, gpx) + wa_axis(py, m, d, p->gamma, gpy);
      hsum += hp_axis(px, m, d) + hp_axis(py, m, d);
      for (int k = 0; k < d; ++k)
        if (m[k]) {
          gx[p->pin_inst[s0 + k]] += gpx[k];
          gy[p->pin_inst[s0 + k]] += gpy[k];
        }
    }
  }
  out[0] = wsum;
  out[1] = hsum;
  out[2] = ncross;
  free(px); free(py); free(gpx); free(gpy); free(top); free(bot);
}

void orc_eval2d(const orc_problem *p, const double *x, const double *y,
                const double *z, int density_mode, double out[7], double *gx,
                double *gy) {
  const int n = p->n_inst;
  const size_t nb = (size_t)p->nx * p->ny * p->nz;
  double g[6];
  orc_geometry(p, g);
  double wl[3];
  double *wgx = malloc(sizeof(double) * (n ? n : 1)), *wgy = malloc(sizeof(double) * (n ? n : 1));
  wirelength2d(p, x, y, z, wl, wgx, wgy);
  double *rho = malloc(sizeof(double) * nb);
  if (density_mode == 0) {
    orc_density_direct(p, x, y, z, rho);
  } else {
    int64_t *q = malloc(sizeof(int64_t) * nb);
    orc_density_fixed(p, x, y, z, density_mode == 2, q);
    for (size_t b = 0; b < nb; ++b) rho[b] = (double)q[b] * (1.0 / 68719476736.0);
    free(q);
  }
  double *ex = malloc(sizeof(double) * nb), *ey = malloc(sizeof(double) * nb);
  double *ez = malloc(sizeof(double) * nb);
  double energy[3] = {0, 0, 0};
  orc_poisson(p, rho, NULL, NULL, NULL, ex, ey, ez, energy);
  double *dgx = malloc(sizeof(double) * (n ? n : 1)), *dgy = malloc(sizeof(double) * (n ? n : 1));
  double *dgz = malloc(sizeof(double) * (n ? n : 1));
  /* the gather's vol(D cap b) spans the whole layer depth d_b: area = vol / d_b */
  orc_density_grad_gather(p, x, y, z, ex, ey, ez, dgx, dgy, dgz);
  if (gx && gy)
    for (int i = 0; i < n; ++i) {
      const int layer = is_hbt(p, i) ? 2 : (z[i] - 0.5 * g[5] > 0.0);
      const double lam = p->lam_layer[layer] / g[2];
      gx[i] = wgx[i] + lam * dgx[i];
      gy[i] = wgy[i] + lam * dgy[i];
    }
  out[0] = wl[0] + p->lam_layer[0] * energy[0] + p->lam_layer[1] * energy[1] + p->lam_layer[2] * energy[2];
  out[1] = wl[0];
  out[2] = energy[0];
  out[3] = energy[1];
  out[4] = energy[2];
  out[5] = wl[1];
  out[6] = wl[2];
  free(wgx); free(wgy); free(rho); free(ex); free(ey); free(ez); free(dgx); free(dgy); free(dgz);
}
