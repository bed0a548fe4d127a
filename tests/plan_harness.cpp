// Test driver for the wirelength launch-plan logic (host code of the
// library's autotuner).  Reads from stdin:
//   nd nf span tol
//   lanes[nf]
//   t[(i * nd + j) * nf + f] for i, j < nd, f < nf   (< 0: the form does not fit)
// applies break_ties when tol >= 0, then best_split, and prints one line
// "i j f" per run (nothing when no split covers every class).
#include <cstdio>
#include <vector>

#include "../paper_2403_09070_gb300/csrc/plan.h"

int main() {
  int nd = 0, nf = 0, span = 0;
  float tol = 0;
  if (std::scanf("%d %d %d %f", &nd, &nf, &span, &tol) != 4 || nd < 0 || nf < 1) return 2;
  std::vector<int> lanes(nf);
  for (int f = 0; f < nf; ++f)
    if (std::scanf("%d", &lanes[f]) != 1) return 2;
  std::vector<float> t((size_t)nd * nd * nf);
  for (float &v : t)
    if (std::scanf("%f", &v) != 1) return 2;
  if (tol >= 0) p3d_plan::break_ties(t, nd, nf, lanes.data(), tol);
  for (const p3d_plan::Run &r : p3d_plan::best_split(t, nd, nf, span)) std::printf("%d %d %d\n", r.i, r.j, r.f);
  return 0;
}
