// Shared launches for batches of independent placement problems: one launch
// per stage covers every instance of the batch.  A launch's blocks are dealt
// out to the instances by a prefix table (blk0[i] = first block of instance
// i, blk0[count] = grid size); each block finds its instance by binary
// search and runs the stage's ordinary kernel body on that instance's
// buffers, with its block index inside the instance's share of the grid.
// Covered here: zeroing of the scalars and wirelength accumulators plus
// position packing, the wirelength degree groups (FP32, 3D mode), their
// partial-sum reducer, and the L1 norms (eq. fda-normalize) with theirs.
#pragma once
#include "common.cuh"
#include "wirelength.cuh"

namespace p3d {

constexpr int kBatchGroups = 12;  // launch groups of degree classes up to 128 pins

// One instance of a batch, as the shared wirelength-stage launches see it.
struct BWl {
  int n;                          // instances of the problem
  int rows_wl;                    // partial-sum rows of the degree groups
  const float *x, *y, *z;         // caller positions (device)
  V4<float> *pos, *acc;           // packed positions, WL accumulators (gx, gy, FD, dp(z)/dz)
  const V4<float> *off;           // pin offsets
  const int *net_start, *pin_inst;
  float *part;                    // partial-sum rows (the handle's buffer)
  double *scal;                   // the handle's scalars
  WlC<float> c;
  int gfirst[kBatchGroups], gcount[kBatchGroups], gpin0[kBatchGroups], grow[kBatchGroups];
};

// Instance of block b: the largest i with blk0[i] <= b (instances with no
// blocks in this launch are passed over); local = b - blk0[i], nblk = the
// instance's block count.
__device__ __forceinline__ int batch_instance(const int *__restrict__ blk0, int count, int b, int &local,
                                              int &nblk) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(blk0 + mid) <= b)
      lo = mid;
    else
      hi = mid;
  }
  local = b - __ldg(blk0 + lo);
  nblk = __ldg(blk0 + lo + 1) - __ldg(blk0 + lo);
  return lo;
}

// Scalars and accumulators to zero, positions packed (float).
__global__ void __launch_bounds__(256) k_b_prep(const BWl *__restrict__ d, const int *__restrict__ blk0, int count) {
  int local, nb;
  const BWl &w = d[batch_instance(blk0, count, blockIdx.x, local, nb)];
  if (local == 0 && threadIdx.x < S_COUNT) w.scal[threadIdx.x] = 0.0;
  for (int k = local * blockDim.x + threadIdx.x; k < w.n; k += nb * blockDim.x) {
    w.acc[k] = V4<float>{0.f, 0.f, 0.f, 0.f};
    w.pos[k] = V4<float>{w.x[k], w.y[k], w.z[k], 0.f};
  }
}

// Degree group g of every instance: the 2-pin closed form ...
__global__ void __launch_bounds__(256) k_b_wl_pair(const BWl *__restrict__ d, const int *__restrict__ blk0, int count,
                                                   int g) {
  int local, nb;
  const BWl &w = d[batch_instance(blk0, count, blockIdx.x, local, nb)];
  wl_pair_body<float>(w.gpin0[g], w.gcount[g], w.pin_inst, w.off, w.pos, w.c, w.acc, w.part + 4 * (size_t)w.grow[g],
                      local, nb);
}

// ... or G lanes per net holding PPL pins each.
template <int G, int PPL>
__global__ void __launch_bounds__(wl_block<float>()) k_b_wl_group(const BWl *__restrict__ d,
                                                                  const int *__restrict__ blk0, int count, int g) {
  int local, nb;
  const BWl &w = d[batch_instance(blk0, count, blockIdx.x, local, nb)];
  wl_group_body<float, G, PPL, false>(w.gfirst[g], w.gcount[g], w.net_start, w.pin_inst, w.off, w.pos, w.c, w.acc,
                                      w.part + 4 * (size_t)w.grow[g], local);
}

// The wirelength rows of every instance into its scalars (W^_Bi, p^(z),
// W_Bi, crossing nets).
__global__ void __launch_bounds__(256) k_b_sum_wl(const BWl *__restrict__ d, const int *__restrict__ blk0, int count) {
  int local, nb;
  const BWl &w = d[batch_instance(blk0, count, blockIdx.x, local, nb)];
  sum_parts_body<4, float>(w.part, w.rows_wl, w.scal + S_WL_BI, local, nb);
}

// L1 norms of every instance's WL gradient: rows, then (S_x, S_y, S_z).
__global__ void __launch_bounds__(256) k_b_norms(const BWl *__restrict__ d, const int *__restrict__ blk0, int count) {
  int local, nb;
  const BWl &w = d[batch_instance(blk0, count, blockIdx.x, local, nb)];
  norms_body<float>(w.n, w.acc, w.part, local, nb);
}
__global__ void __launch_bounds__(256) k_b_sum_norms(const BWl *__restrict__ d, const int *__restrict__ blk0,
                                                     const int *__restrict__ rows, int count) {
  int local, nb;
  const int i = batch_instance(blk0, count, blockIdx.x, local, nb);
  const BWl &w = d[i];
  sum_parts_body<3, float>(w.part, rows[i], w.scal + S_SX, local, nb);
}

}  // namespace p3d
