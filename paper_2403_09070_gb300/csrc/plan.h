// Launch plans of the wirelength stage from measured run times: host code,
// shared by the library's autotuner and its tests.
//
// The nets are held in nd degree classes (ascending degree).  A launch
// group is a run of adjacent classes i..j evaluated with one form f (lanes
// per net, pins per lane).  t[(i * nd + j) * nf + f] is the measured time
// of that launch, < 0 where the form does not fit the run.
#pragma once
#include <vector>

namespace p3d_plan {

// Of the forms within (1 + tol) of a run's fastest, keeps the one with the
// fewest lanes per net (lanes[f]; among equal lanes the faster) and marks
// the others as not fitting.  Near ties are inside the timing noise, and
// fewer lanes mean fewer shuffle rounds and more nets per warp.
inline void break_ties(std::vector<float> &t, int nd, int nf, const int *lanes, float tol) {
  for (int j = 0; j < nd; ++j)
    for (int i = 0; i <= j; ++i) {
      float *row = &t[((size_t)i * nd + j) * nf];
      float tmin = 1e30f;
      for (int f = 0; f < nf; ++f)
        if (row[f] >= 0 && row[f] < tmin) tmin = row[f];
      int keep = -1;
      for (int f = 0; f < nf; ++f)
        if (row[f] >= 0 && row[f] <= (1.0f + tol) * tmin &&
            (keep < 0 || lanes[f] < lanes[keep] || (lanes[f] == lanes[keep] && row[f] < row[keep])))
          keep = f;
      for (int f = 0; f < nf; ++f)
        if (f != keep) row[f] = -1.0f;
    }
}

struct Run {
  int i, j, f;  // classes i..j, form f
};

// The split of classes 0..nd-1 into runs of at most `span` adjacent classes
// with the least total time (dynamic programming: best[j] is the least time
// of classes 0..j-1), runs in ascending order; empty when some class cannot
// be covered.
inline std::vector<Run> best_split(const std::vector<float> &t, int nd, int nf, int span) {
  std::vector<double> best(nd + 1, 1e300);
  std::vector<int> from(nd + 1, 0), form(nd + 1, -1);
  best[0] = 0;
  for (int j = 0; j < nd; ++j)
    for (int i = j - span + 1 > 0 ? j - span + 1 : 0; i <= j; ++i)
      for (int f = 0; f < nf; ++f) {
        const float v = t[((size_t)i * nd + j) * nf + f];
        if (v >= 0 && best[i] + v < best[j + 1]) {
          best[j + 1] = best[i] + v;
          from[j + 1] = i;
          form[j + 1] = f;
        }
      }
  std::vector<Run> runs;
  if (nd < 1 || best[nd] >= 1e299) return runs;
  for (int j = nd; j > 0; j = from[j]) runs.push_back({from[j], j - 1, form[j]});
  for (size_t a = 0, b = runs.size(); a + 1 < b; ++a, --b) {
    const Run r = runs[a];
    runs[a] = runs[b - 1];
    runs[b - 1] = r;
  }
  return runs;
}

}  // namespace p3d_plan
