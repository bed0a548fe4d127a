/* Minimal use of the place3d C ABI from C: one evaluation of the 3D
 * placement objective and its gradient for a tiny problem (six standard
 * cells and one macro, three nets, a 32 x 32 region on a 16 x 16 x 2 grid),
 * FP64.  Prints the objective, its parts and the gradient of every
 * instance; exits non-zero (with place3d_last_error()) on any failure.
 *
 * Build (from the repository root, after building libplace3d.so):
 *   gcc -std=c99 -O2 -Iinclude paper_2403_09070_gb300/examples/place3d_minimal.c \
 *       -Lpaper_2403_09070_gb300 -lplace3d -Wl,-rpath,$PWD/paper_2403_09070_gb300 -o place3d_minimal
 */
#include <stdio.h>
#include <string.h>

#include "place3d.h"

#define N_INST 7
#define N_NET 3
#define N_PIN 9

int main(void) {
  /* instances 0-5: standard cells, 6: a macro (pins are on the macro too) */
  const uint8_t is_macro[N_INST] = {0, 0, 0, 0, 0, 0, 1};
  const double w_bot[N_INST] = {1, 2, 3, 1, 2, 4, 6}, h_bot[N_INST] = {1, 1, 1, 1, 1, 1, 6};
  double w_top[N_INST], h_top[N_INST];
  for (int i = 0; i < N_INST; ++i) {
    w_top[i] = 0.8 * w_bot[i];
    h_top[i] = 0.8 * h_bot[i];
  }
  /* nets {0, 1, 6}, {2, 3}, {1, 4, 5, 6} */
  const int32_t net_start[N_NET + 1] = {0, 3, 5, 9};
  const int32_t pin_inst[N_PIN] = {0, 1, 6, 2, 3, 1, 4, 5, 6};
  const double off_bx[N_PIN] = {0.2, -0.3, 1.0, 0.0, 0.1, 0.2, -0.4, 0.3, -1.5};
  const double off_by[N_PIN] = {0.1, 0.2, -1.0, 0.3, -0.2, 0.0, 0.1, -0.3, 2.0};
  double off_tx[N_PIN], off_ty[N_PIN];
  for (int k = 0; k < N_PIN; ++k) {
    off_tx[k] = 0.8 * off_bx[k];
    off_ty[k] = 0.8 * off_by[k];
  }
  /* region 32 x 32 on 16 x 16 x 2 bins: w_b = h_b = d_b = 2, d_z = 4 */
  place3d_problem p;
  memset(&p, 0, sizeof(p));
  p.n_inst = N_INST;
  p.is_macro = is_macro;
  p.w_bot = w_bot;
  p.h_bot = h_bot;
  p.w_top = w_top;
  p.h_top = h_top;
  p.n_net = N_NET;
  p.n_pin = N_PIN;
  p.net_start = net_start;
  p.pin_inst = pin_inst;
  p.pin_off_bot_x = off_bx;
  p.pin_off_bot_y = off_by;
  p.pin_off_top_x = off_tx;
  p.pin_off_top_y = off_ty;
  p.xl = 0;
  p.yl = 0;
  p.xh = 32;
  p.yh = 32;
  p.nx = 16;
  p.ny = 16;
  p.nz = 2;
  p.gamma = 8.0; /* 4 w_b */
  p.gamma_z = 0.0;
  p.alpha = place3d_alpha(32.0, 4.0, 10.0, 1.0, 0.8, 1.0);
  p.lambda = 1e-3;
  p.precision = PLACE3D_FP64;
  p.flags = PLACE3D_FLAG_CHECKS;
  p.mode = PLACE3D_MODE_3D;

  place3d_handle *h = NULL;
  if (place3d_create(&p, 0, NULL, &h) != PLACE3D_OK) {
    fprintf(stderr, "create: %s\n", place3d_last_error(NULL));
    return 1;
  }
  /* centres; z in [d_z/4, 3 d_z/4] = [1, 3]: cells 0, 2, 4 on the top die */
  const double x[N_INST] = {5, 9, 14, 18, 22, 26, 12};
  const double y[N_INST] = {6, 11, 20, 24, 8, 15, 16};
  const double z[N_INST] = {2.7, 1.2, 2.9, 1.4, 2.5, 1.1, 2.0};
  double gx[N_INST], gy[N_INST], gz[N_INST];
  place3d_result r;
  if (place3d_set_positions(h, x, y, z, PLACE3D_F64, PLACE3D_MEM_HOST) != PLACE3D_OK ||
      place3d_eval_objective_and_grad(h, &r, gx, gy, gz, PLACE3D_F64, PLACE3D_MEM_HOST) != PLACE3D_OK) {
    fprintf(stderr, "evaluation: %s\n", place3d_last_error(h));
    place3d_destroy(h);
    return 1;
  }
  printf("obj %.17g\nwl_bi %.17g\nwl_z %.17g\nenergy %.17g\nhpwl_d2d %.17g\nn_cross %.17g\n", r.obj, r.wl_bi,
         r.wl_z, r.energy, r.hpwl_d2d, r.n_cross);
  for (int i = 0; i < N_INST; ++i) printf("grad %d %.17g %.17g %.17g\n", i, gx[i], gy[i], gz[i]);
  place3d_destroy(h);
  return 0;
}
