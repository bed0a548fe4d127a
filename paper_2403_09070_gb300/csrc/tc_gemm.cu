// Tensor-core spectral solve (placeholder until the tcgen05 kernels land).
#include "tc_gemm.h"

namespace p3d_tc {
struct TcPlan {};
TcPlan *create(int, int, int, int, double, double, double, void *, void *, void *, const p3d::ZStageC *,
               std::string *why) {
  if (why) *why = "tensor-core transforms are not built in this library";
  return nullptr;
}
void densify(TcPlan *, cudaStream_t, int, int, const long long *, const long long *) {}
int forward(TcPlan *, cudaStream_t) { return 0; }
int zstage(TcPlan *, cudaStream_t, double *) { return 0; }
int inverse(TcPlan *, cudaStream_t) { return 0; }
void destroy(TcPlan *) {}
}  // namespace p3d_tc
