// Allocation-free density map: the fixed-point density accumulation of the
// evaluation (cells by direct overlap, macros by 8 corners + integer prefix
// sums, FP64 contribution arithmetic) writing rho to a caller buffer, with
// its two int64 accumulator maps in a file-scope device array instead of
// memory the library allocates.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/place3d.h"
#include "common.cuh"
#include "density.cuh"

using namespace p3d;

namespace {

// Scratch shared by every call on a device: two int64 maps of at most
// PLACE3D_NOALLOC_MAX_BINS bins (cell counts, then macro corners).
static __device__ __align__(256) long long g_noalloc_scratch[2 * PLACE3D_NOALLOC_MAX_BINS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;

// Cached device address of the scratch array per device, tagged with the
// unique id of the context it was looked up in.  The array's address belongs
// to the module loaded into one context: after a device reset, or after the
// primary context was released and created again, the module is loaded anew
// and the array can sit elsewhere, so a cached address whose context id no
// longer matches the current one is looked up again.
struct ScratchAddr {
  unsigned long long ctx_id;
  long long *ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the
// library does not link the driver library itself).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_entry_once;

void resolve_entry_points() {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
  f = nullptr;
  q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
}

// Unique id of the calling thread's current context; false if there is none
// yet (the runtime makes the device's primary context current on its first
// call that needs one) or the entry points are unavailable.
bool current_ctx_id(unsigned long long *id) {
  std::call_once(g_entry_once, resolve_entry_points);
  if (!g_ctx_get_current || !g_ctx_get_id) return false;
  CUcontext c = nullptr;
  if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return false;
  return g_ctx_get_id(c, id) == CUDA_SUCCESS;
}

// The device address of the scratch array for `dev` (the current device):
// looked up with cudaGetSymbolAddress on the first call in a context (this
// first lookup loads the library's module on the device if it is not loaded
// yet), then reused while the current context stays the same.  Without a
// context id the address is looked up on every call.
cudaError_t scratch_for(int dev, long long **out) {
  unsigned long long id = 0;
  const bool have_id = current_ctx_id(&id);
  std::lock_guard<std::mutex> lock(g_mu);
  if (have_id && g_scratch[dev].ptr && g_scratch[dev].ctx_id == id) {
    *out = g_scratch[dev].ptr;
    return cudaSuccess;
  }
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  unsigned long long id2 = 0;
  g_scratch[dev] = current_ctx_id(&id2) ? ScratchAddr{id2, static_cast<long long *>(p)} : ScratchAddr{0, nullptr};
  *out = static_cast<long long *>(p);
  return cudaSuccess;
}

struct SoA {
  const double *x, *y, *z, *wb, *hb, *wt, *ht;
  const uint8_t *is_macro;
};

__device__ __forceinline__ V4<double> size_of(const SoA &a, int i) {
  V4<double> s;
  s.x = a.wb[i];
  s.y = a.hb[i];
  s.z = a.wt[i];
  s.w = a.ht[i];
  return s;
}

// Cell contributions, same steps and quantisation as k_scatter_cells.
__global__ void __launch_bounds__(256) k_noalloc_cells(int n, SoA a, DensC<double> c, long long *q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || a.is_macro[i]) return;
  const Box<double> b = inst_box(c, a.x[i], a.y[i], a.z[i], size_of(a, i), false);
  double cl[3], chh[3];
  int b0[3], b1[3];
  if (!clip_axis(b.lo[0], b.hi[0], c.fnx, c.nx, cl[0], chh[0], b0[0], b1[0])) return;
  if (!clip_axis(b.lo[1], b.hi[1], c.fny, c.ny, cl[1], chh[1], b0[1], b1[1])) return;
  if (!clip_axis(b.lo[2], b.hi[2], c.fnz, c.nz, cl[2], chh[2], b0[2], b1[2])) return;
  for (int k = b0[2]; k <= b1[2]; ++k) {
    const double oz = ov_axis(cl[2], chh[2], k);
    for (int j = b0[1]; j <= b1[1]; ++j) {
      const double oy = ov_axis(cl[1], chh[1], j);
      for (int ii = b0[0]; ii <= b1[0]; ++ii) {
        const double ox = ov_axis(cl[0], chh[0], ii);
        const double v = rn_mul(rn_mul(rn_mul(b.om, ox), oy), oz);
        atomic_add_i64(q + ((size_t)k * c.ny + j) * c.nx + ii, r_rint(rn_mul(v, kFixedScale)));
      }
    }
  }
}

// Macro corner entries (Theorem 1), one thread per instance, same steps and
// quantisation as k_macro_corners.
__global__ void __launch_bounds__(256) k_noalloc_corners(int n, SoA a, DensC<double> c, long long *A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !a.is_macro[i]) return;
  const Box<double> b = inst_box(c, a.x[i], a.y[i], a.z[i], size_of(a, i), true);
  const double fN[3] = {c.fnx, c.fny, c.fnz};
  for (int s = 0; s < 8; ++s) {
    int base[3];
    double wg[3][2];
    int sign = -1;
    for (int ax = 0; ax < 3; ++ax) {
      const bool up = (s >> ax) & 1;
      corner_axis(up ? b.hi[ax] : b.lo[ax], fN[ax], base[ax], wg[ax][0], wg[ax][1]);
      sign *= up ? 1 : -1;
    }
    for (int cz = 0; cz < 2; ++cz)
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
          const int ii = base[0] + cx, j = base[1] + cy, k = base[2] + cz;
          if (ii >= c.nx || j >= c.ny || k >= c.nz) continue;
          const double e = rn_mul(rn_mul(rn_mul(b.om, wg[0][cx]), wg[1][cy]), wg[2][cz]);
          const long long qe = r_rint(rn_mul(e, kFixedScale));
          if (qe) atomic_add_i64(A + ((size_t)k * c.ny + j) * c.nx + ii, sign > 0 ? qe : -qe);
        }
  }
}

int grid_of(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

extern "C" int place3d_density_map_noalloc(int n_inst, const double *x, const double *y, const double *z,
                                           const double *w_bot, const double *h_bot, const double *w_top,
                                           const double *h_top, const uint8_t *is_macro, double xl, double yl,
                                           double xh, double yh, int nx, int ny, int nz, double *rho,
                                           void *cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1 || n_inst < 0 || !rho) return PLACE3D_ERR_INVALID_ARG;
  if (!(xh > xl) || !(yh > yl)) return PLACE3D_ERR_INVALID_ARG;
  if ((long long)nx * ny * nz > PLACE3D_NOALLOC_MAX_BINS) return PLACE3D_ERR_OUT_OF_RANGE;
  if (n_inst > 0 && (!x || !y || !z || !w_bot || !h_bot || !w_top || !h_top || !is_macro))
    return PLACE3D_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PLACE3D_ERR_CUDA;
  long long *scratch = nullptr;
  if (scratch_for(dev, &scratch) != cudaSuccess) return PLACE3D_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t nb = (size_t)nx * ny * nz;
  long long *q = scratch, *A = scratch + nb;
  // geometry and constants exactly as the handle computes them (Sec. V-A)
  const double dx = xh - xl, dy = yh - yl, wb = dx / nx, hb = dy / ny, db = 0.5 * (wb + hb), dz = nz * db;
  DensC<double> c;
  c.x0 = xl;
  c.y0 = yl;
  c.iwb = 1.0 / wb;
  c.ihb = 1.0 / hb;
  c.idb = 1.0 / db;
  c.cw = std::sqrt(2.0) * wb;
  c.ch = std::sqrt(2.0) * hb;
  c.zmid = 0.5 * dz;
  c.qz = 0.25 * dz;
  c.tz = 2.0 / dz;
  c.fnx = nx;
  c.fny = ny;
  c.fnz = nz;
  c.nx = nx;
  c.ny = ny;
  c.nz = nz;
  c.mode2d = 0;
  SoA a{x, y, z, w_bot, h_bot, w_top, h_top, is_macro};
  // the scratch keeps the previous call's contents: clear both maps first
  if (cudaMemsetAsync(scratch, 0, 2 * nb * sizeof(long long), s) != cudaSuccess) return PLACE3D_ERR_CUDA;
  if (n_inst > 0) {
    k_noalloc_cells<<<grid_of(n_inst, 256), 256, 0, s>>>(n_inst, a, c, q);
    k_noalloc_corners<<<grid_of(n_inst, 256), 256, 0, s>>>(n_inst, a, c, A);
  }
  const int rows = ny * nz;
  k_scan_rows<long long, long long, false><<<grid_of(rows, 8), 256, 0, s>>>(rows, nx, A, 1, A);
  k_scan_cols<long long, false><<<dim3(grid_of(nx, 32), nz), 1024, 0, s>>>(nx, ny, A);
  k_densify<double><<<grid_of((long long)nx * ny, 256), 256, 0, s>>>(nx * ny, nz, q, A, OutPlain<double>{rho});
  return cudaGetLastError() == cudaSuccess ? PLACE3D_OK : PLACE3D_ERR_CUDA;
}
