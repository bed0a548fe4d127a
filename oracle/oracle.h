/*
 * place3d oracle: a plain, slow, obviously correct CPU implementation of one
 * evaluation of the objective and gradient of the 3D die-to-die placer in
 * "Analytical Heterogeneous Die-to-Die 3D Placement with Macros"
 * (arXiv 2403.09070).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline / reference legs load this library.  It shares no code, header,
 * table or constant generator with the CUDA path and never calls it.
 *
 * Precision: FP64 throughout, except the fixed-point density replica, which
 * evaluates each quantised contribution in the precision the GPU kernel uses
 * (float or double) so that both sides take the same rounding decision.
 *
 * Parity status of each function is stated beside it; every function is
 * pinned by a test against a closed form, a printed example, an invariant or
 * brute force, except where "parity pinned only approximately" is written.
 */
#ifndef PLACE3D_ORACLE_H
#define PLACE3D_ORACLE_H
#include <stdint.h>

typedef struct {
  int n_inst;
  const unsigned char *is_macro; /* [n_inst] 1 = macro (Sec. III-A, V_M) */
  const unsigned char *z_fixed;  /* [n_inst] or NULL: z-gradient forced to 0 */
  const double *w_bot, *h_bot, *w_top, *h_top; /* per-die sizes */
  int n_net, n_pin;
  const int *net_start; /* [n_net+1] CSR */
  const int *pin_inst;  /* [n_pin] */
  const double *off_bx, *off_by, *off_tx, *off_ty; /* pin offsets per die */
  double xl, yl, xh, yh;
  int nx, ny, nz;
  double gamma, gamma_z, alpha, lambda;
  /* Multi-die 2D mode (Sec. V-B "multi-die 2D global placement", eq.
   * 2d-place): mode = 1, nz = 3 layers (0 bottom die, 1 top die, 2 HBT
   * layer), is_hbt marks the hybrid bonding terminals (instances of the HBT
   * layer, footprint w_bot x h_bot, pins counted in both partial nets),
   * lam_layer = (lambda-, lambda+, lambda') per layer.  mode = 0: 3D. */
  const unsigned char *is_hbt; /* [n_inst] or NULL */
  int mode;
  double lam_layer[3];
} orc_problem;

/* Region and bin geometry (Sec. II-A, Sec. V-A: d_b=(w_b+h_b)/2, d_z=N_z d_b).
 * out = {w_b, h_b, d_b, d_x, d_y, d_z} */
void orc_geometry(const orc_problem *p, double out[6]);

/* HBT penalty factor of Sec. V-A. */
double orc_alpha(double dx, double dz, double beta, double w_hbt, double rh_top,
                 double rh_bot);

/* Eq. std-size-tech / macro-size-tech and the local smoothness weight of
 * Sec. IV-A: per instance delta, w, h, stretched w and h, omega. */
void orc_attributes(const orc_problem *p, const double *x, const double *y,
                    const double *z, int *delta, double *w, double *h,
                    double *sw, double *sh, double *omega);

/* Eq. density-map-accum, definition form: direct cuboid/bin overlap in FP64
 * for every instance (cells and macros).  rho is [nz][ny][nx]. */
void orc_density_direct(const orc_problem *p, const double *x, const double *y,
                        const double *z, double *rho);

/* Theorem 1 for macros only: the summed corner map A (eq. 3d-density-accum-
 * cuboid, unquantised FP64, corners clamped to the region).  Its inclusive
 * prefix sum (orc_prefix_sum3) is the macros' density. */
void orc_macro_corner_map(const orc_problem *p, const double *x,
                          const double *y, const double *z, double *A);

/* Eq. def-prefix-sum-3d (inclusive), in place, on [nz][ny][nx]. */
void orc_prefix_sum3(double *a, int nx, int ny, int nz);
void orc_prefix_sum3_i64(int64_t *a, int nx, int ny, int nz);

/* Fixed-point density replica: every cell contribution and every macro corner
 * entry quantised to int64 at scale 2^36 (round half to even), summed in
 * integers, macro corners prefix-summed in integers.  use_float selects the
 * precision of the contribution arithmetic (1 = float, 0 = double). */
void orc_density_fixed(const orc_problem *p, const double *x, const double *y,
                       const double *z, int use_float, int64_t *q);

/* Spectral solve of eq. 3d-poisson-equation, separable per-axis form of eqs.
 * density-coef, poisson-sol-potential, possion-sol-force with the cosine
 * series weights c_0=1, c_j=2.  Any output pointer may be NULL.
 * energy = 1/2 vol(b) N sum c_j c_k c_l a^2/omega^2 (spectral form).
 * mode 1 (2D): one 2D solve per layer, E_z = 0, energy[l] = 1/2 A_b
 * sum_b rho_b phi_b of layer l (energy then points to nz values). */
void orc_poisson(const orc_problem *p, const double *rho, double *a,
                 double *psi, double *phi, double *ex, double *ey, double *ez,
                 double *energy);

/* The same series evaluated directly, one bin and one mode at a time
 * (O(|B|^2), tiny grids only): a from eq. density-coef, then phi and E. */
void orc_poisson_series_direct(const orc_problem *p, const double *rho,
                               double *a, double *phi, double *ex, double *ey,
                               double *ez);

/* Density-penalty gradient by field gather: dU/dx_i = -omega_i sum_b
 * vol(D_i cap b) E_x(b), likewise y and z, for every instance (direct
 * overlap). */
void orc_density_grad_gather(const orc_problem *p, const double *x,
                             const double *y, const double *z,
                             const double *ex, const double *ey,
                             const double *ez, double *gx, double *gy,
                             double *gz);

/* Macro gather by Theorem 1's adjoint: suffix sums of E and the 8 corners.
 * Writes gx/gy/gz for macros only (others untouched). */
void orc_macro_grad_suffix(const orc_problem *p, const double *x,
                           const double *y, const double *z, const double *ex,
                           const double *ey, const double *ez, double *gx,
                           double *gy, double *gz);

/* Exact derivative of U = 1/2 vol(b) sum rho phi with respect to x, y, z of
 * every instance, for the discrete (bin-overlap) density with the instance's
 * size held fixed: phi differences at the bins holding the box faces. */
void orc_density_grad_exact(const orc_problem *p, const double *x,
                            const double *y, const double *z,
                            const double *phi, double *gx, double *gy,
                            double *gz);

/* Bistratal WA wirelength of eq. wl-model with the FD depth gradient of eq.
 * fda-grad.  fd_mode 0 = brute force (re-traverse the net for each moved
 * pin), 1 = incremental (1st/2nd extremes of the top and bottom sets).
 * out = {sum_e W^_Bi, sum_e p^_e(z), exact D2D HPWL (eq. wl-obj), #crossing
 * nets}.  Per instance: gx, gy = gradient of sum W^_Bi; gfd = eq. fda-grad;
 * gwaz = gradient of sum p^_e(z).  Arrays are overwritten. */
void orc_wirelength(const orc_problem *p, const double *x, const double *y,
                    const double *z, int fd_mode, double out[4], double *gx,
                    double *gy, double *gfd, double *gwaz);

/* Dummy fillers of Sec. III-A: eq. filler-vol (z-fixed fillers, one set per
 * die, volume (1/2) d_x d_y d_z (1 - u)) and eq. free-filler-vol (free
 * fillers, the remaining white space).  vol_a is the total instance volume at
 * the initial depths z: each instance a cuboid of depth d_z/2 whose footprint
 * is that of its die (eq. std-size-tech; eq. macro-size-tech for macros).
 * Filler footprint on a die (reading): the mean std-cell width and height on
 * that die, std cells being the instances that are neither macros nor
 * z-fixed.  Counts: the set's volume over one filler's volume, rounded to the
 * nearest integer; a free filler counts the mean of the two dies' filler
 * volumes.
 * out = {vol_a, vol_f+, vol_f-, vol_fr, w+, h+, w-, h-, n+, n-, n_fr}. */
void orc_filler_plan(const orc_problem *p, const double *z, double u_top,
                     double u_bot, double out[11]);

/* Multi-die 2D evaluation (eq. 2d-place).  The partition is fixed: delta_i
 * = 1[z_i > d_z/2] for non-HBT instances.  Per net, the D2D wirelength
 * (eq. exact-wirelength, smoothed by eq. wa-model-approx) is the WA span of
 * the top partial net plus that of the bottom partial net, each including
 * the net's HBT pins (a net on one die is its own partial net).  Each layer
 * is an independent 2D electrostatic field: rho_l by eq. density-map-accum
 * in 2D (area overlap, local smoothness), potential of the 2D cosine series,
 * energy U_l = 1/2 A_b sum_b rho_b phi_b, force -omega sum_b area(D cap b)
 * E_b.  Instance sizes are their die's (macros too); HBTs are w_bot x h_bot.
 * density_mode as in orc_eval.  out = {obj, sum W^, U-, U+, U', exact D2D
 * HPWL, #crossing nets}.  gx, gy may be NULL. */
void orc_eval2d(const orc_problem *p, const double *x, const double *y,
                const double *z, int density_mode, double out[7], double *gx,
                double *gy);

/* Full objective and gradient (a1..a11).  density_mode: 0 = direct FP64
 * density, 1 = fixed-point replica in double, 2 = fixed-point replica in
 * float.  out = {obj, wl_bi, wl_z, energy, hpwl_d2d, n_cross, g_scale,
 * S_x, S_y, S_z}.  g* may be NULL. */
void orc_eval(const orc_problem *p, const double *x, const double *y,
              const double *z, int density_mode, int fd_mode, double out[10],
              double *gx, double *gy, double *gz);

#endif
