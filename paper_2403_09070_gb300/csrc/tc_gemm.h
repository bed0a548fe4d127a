// Tensor-core (tcgen05) form of the spectral solve, FP32 accuracy from
// split-BF16 operands.  Host interface used by place3d.cu.
#pragma once
#include <cuda_runtime.h>

#include <string>

namespace p3d {
struct ZStageC;
}

namespace p3d_tc {

struct TcPlan;

// Build the plan for an nx x ny x nz grid (nx, ny multiples of 128) on the
// current device; e4 is the handle's FP32 field map [z][y][x] of (E_x, E_y,
// E_z, unused) (output of inverse()), zc the device copy of the z-stage
// constants.  Returns NULL and sets *why when the device or the grid is not
// supported.
TcPlan *create(int device, int nx, int ny, int nz, double dx, double dy, double dz, void *e4,
               const p3d::ZStageC *zc, std::string *why);
// rho (cells + macro corners, z prefix) -> split-BF16 planes of the input.
// (part: the per-warp overflow rows, see k_densify)
void densify(TcPlan *p, cudaStream_t s, int nxy, int nz, const long long *q, const long long *corner, float *part);
// Forward x and y products; z stage (scaling, energy, z transforms);
// inverse x and y products into the interleaved field map e4.  Each returns its launch count.
int forward(TcPlan *p, cudaStream_t s);
int zstage(TcPlan *p, cudaStream_t s, float *part);  // per-block energy rows (see k_zstage)
int inverse(TcPlan *p, cudaStream_t s);
// Times both tile widths (64 and 128 columns) of each of the four product
// groups on stream s and keeps the faster (0, or -1 on a CUDA error).
int autotune(TcPlan *p, cudaStream_t s, int repeats);
// Tile columns in use for group k (0 x forward, 1 y forward, 2 x inverse,
// 3 y inverse), and a way to set them (64 or 128).
int tile_columns(const TcPlan *p, int group);
void set_tile_columns(TcPlan *p, int group, int bn);
// Error code left by a bounded wait of the tensor-core kernel (0 = none);
// synchronises with the device.
int error_code(TcPlan *p);
void destroy(TcPlan *p);

}  // namespace p3d_tc
