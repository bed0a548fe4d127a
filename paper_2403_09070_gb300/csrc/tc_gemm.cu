// Tensor-core form of the spectral solve (eqs. density-coef,
// poisson-sol-potential, possion-sol-force) on sm_103a.
//
// Each axis transform is a batched product out[b][n][m] = sum_k A[b][m][k]
// W[n][k] (W = cosine or sine matrix), computed with tcgen05.mma (kind::f16,
// BF16 operands, FP32 accumulation in tensor memory).  FP32 accuracy is won
// back by splitting every operand into two BF16 planes, v = hi + lo, and
// accumulating hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding).
// Operand tiles are staged by TMA (128-byte swizzle) through a 4-deep
// mbarrier pipeline: one thread issues the TMA loads, one thread issues the
// MMAs, four warps drain the accumulator from tensor memory and store it
// transposed (the next axis becomes the contiguous one), either as FP32 or
// again as split-BF16 planes for the next product.
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the CTA
// records an error code, stops issuing work, waits (bounded) for its own TMA
// copies, frees its tensor memory and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/place3d.h"
#include "common.cuh"
#include "density.cuh"
#include "tc_gemm.h"
#include "transform.cuh"

namespace p3d_tc {
using namespace p3d;

// Tile shapes: M = 128 rows, K-blocks of 64, and N = 64 or 128 columns
// (chosen per product group by the autotuner: N = 128 reads each A tile for
// twice the outputs, N = 64 gives twice the tiles to spread over the SMs).
// Pipeline depth: 3 stages of 48 KiB (N = 64) or of 64 KiB (N = 128), one
// persistent CTA per SM.  (A fourth 48 KiB stage measured no faster alone,
// and it left too little shared memory beside the CTA for the wirelength
// blocks that run concurrently on the other stream: the evaluation was
// 2 % slower.)
constexpr int BM = 128, BK = 64;
constexpr int A_BYTES = BM * BK * 2;  // one BF16 plane of an A tile (16 KiB)
template <int BN> struct TileCfg {
  static constexpr int W_BYTES = BN * BK * 2;                    // one BF16 plane of a W tile
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * W_BYTES;  // A hi, A lo, W hi, W lo
  static constexpr int STAGES = 3;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  static constexpr int TMEM_COLS = BN;  // FP32 accumulator columns of one buffer (two are allocated)
  // instruction descriptor: D FP32, A and B BF16, both K-major, M = BM, N = BN
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};
constexpr int kMinBN = 64;  // every product's N and K are multiples of this
constexpr long long kWaitCycles = 4000000000LL;         // about 2 s at 2 GHz

enum { OUT_F32 = 0, OUT_SPLIT = 1 };
enum { ERR_FULL = 1, ERR_EMPTY = 2, ERR_ACC = 3 };

struct Prob {
  void *out;          // float* (OUT_F32) or bf16* hi plane (OUT_SPLIT)
  long long plane;    // elements from the hi plane to the lo plane
  long long o_bstride;
  int M, N, K, batches, tiles_m, tiles_n, kind;
  int ostride;        // OUT_F32: element stride of the output (4 = one component of an interleaved map)
};

struct Group {
  CUtensorMap amap[3];  // A: dims {K, M, batch, plane}
  CUtensorMap wmap[3];  // W: dims {K, N, plane}, box of bn rows
  Prob p[3];
  int count;
  int bn;               // tile columns (64 or 128)
  int tile_start[4];
  int *err;
  long long wait_cycles;  // clock budget of every mbarrier wait (kWaitCycles)
  int skip_loads;         // test hook: the producer arms and loads nothing, so the MMA's first wait runs out
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tma_load_4d(const CUtensorMap *map, uint32_t dst, uint32_t bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(const CUtensorMap *map, uint32_t dst, uint32_t bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, BF16 x BF16 -> FP32.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 B, 8-row groups 1024 B apart (stride byte offset), descriptor
// version 1, swizzle mode 2 (128 B).  The tile base is 1024-byte aligned; a
// step of 16 K-elements inside the swizzle row advances the start by 32 B.
__device__ __forceinline__ uint64_t desc_k_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                             int *err, int code, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) {
      *abort_flag = 1;
      atomicExch(err, code);
      return false;
    }
  }
  return true;
}

// ------------------------------------------------------------------ kernel
// Persistent: CTA c takes tiles c, c + gridDim.x, ... of the group.  The
// shared-memory pipeline runs continuously across a CTA's tiles (k-block
// counter `it`), and the accumulator is double-buffered in tensor memory
// (2 x BN columns): the MMA thread fills buffer j & 1 for the CTA's j-th
// tile while the epilogue warps drain the other, so one tile's epilogue
// overlaps the next tile's loads and MMAs.  acc_full[b] (MMA commit ->
// epilogue) and acc_empty[b] (four epilogue warps -> MMA) hand the buffers
// over.
__device__ __forceinline__ void tile_coords(const Group &g, int tile, int &pi, int &b, int &m0, int &n0) {
  pi = 0;
  while (pi + 1 < g.count && tile >= g.tile_start[pi + 1]) ++pi;
  const Prob &P = g.p[pi];
  tile -= g.tile_start[pi];
  const int per_b = P.tiles_m * P.tiles_n;
  b = tile / per_b;
  const int r = tile - b * per_b;
  m0 = (r % P.tiles_m) * BM;
  n0 = (r / P.tiles_m) * g.bn;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ Group g) {
  using C = TileCfg<BN>;
  constexpr int STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES, W_BYTES = C::W_BYTES, TMEM_COLS = C::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * STAGES + 5];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = g.tile_start[g.count];

  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]);
  const uint32_t accf0 = smem_u32(&bars[2 * STAGES]), acce0 = smem_u32(&bars[2 * STAGES + 2]);
  const uint32_t done = smem_u32(&bars[2 * STAGES + 4]);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(accf0 + 8 * k, 1);
      mbar_init(acce0 + 8 * k, 4);  // one arrival per epilogue warp
    }
    mbar_init(done, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_slot), 2 * TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int *abort_p = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      int it = 0;
      bool stop = false;
      for (int tile = blockIdx.x; tile < ntiles && !stop && !g.skip_loads; tile += gridDim.x) {
        int pi, b, m0, n0;
        tile_coords(g, tile, pi, b, m0, n0);
        const CUtensorMap *am = &g.amap[pi], *wm = &g.wmap[pi];
        const int nk = g.p[pi].K / BK;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES, round = it / STAGES;
          if (it >= STAGES &&
              !wait_bounded(empty0 + 8 * s, (round - 1) & 1, abort_p, g.err, ERR_EMPTY, g.wait_cycles)) {
            stop = true;
            break;
          }
          const uint32_t st = smem_u32(smem + s * STAGE_BYTES), fb = full0 + 8 * s;
          mbar_expect_tx(fb, STAGE_BYTES);
          tma_load_4d(am, st, fb, kb * BK, m0, b, 0);
          tma_load_4d(am, st + A_BYTES, fb, kb * BK, m0, b, 1);
          tma_load_3d(wm, st + 2 * A_BYTES, fb, kb * BK, n0, 0);
          tma_load_3d(wm, st + 2 * A_BYTES + W_BYTES, fb, kb * BK, n0, 1);
        }
      }
      // every armed stage's last copy must have landed before the CTA exits
      const int issued = it;
      for (int s = 0; s < STAGES && s < issued; ++s) {
        const int last = s + ((issued - 1 - s) / STAGES) * STAGES;
        const long long t0 = clock64();
        while (!mbar_try_wait(full0 + 8 * s, (last / STAGES) & 1) && clock64() - t0 < g.wait_cycles) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      int it = 0, j = 0;
      bool stop = false;
      for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x, ++j) {
        int pi, b, m0, n0;
        tile_coords(g, tile, pi, b, m0, n0);
        const int nk = g.p[pi].K / BK;
        const int buf = j & 1;
        if (j >= 2 && !wait_bounded(acce0 + 8 * buf, ((j >> 1) - 1) & 1, abort_p, g.err, ERR_ACC, g.wait_cycles))
          break;
        tc_fence_after();
        const uint32_t td = tmem + (uint32_t)(buf * TMEM_COLS);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES, round = it / STAGES;
          if (!wait_bounded(full0 + 8 * s, round & 1, abort_p, g.err, ERR_FULL, g.wait_cycles)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t a_hi = smem_u32(smem + s * STAGE_BYTES), a_lo = a_hi + A_BYTES;
          const uint32_t w_hi = a_hi + 2 * A_BYTES, w_lo = w_hi + W_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t dah = desc_k_sw128(a_hi + kk * 32), dal = desc_k_sw128(a_lo + kk * 32);
            const uint64_t dwh = desc_k_sw128(w_hi + kk * 32), dwl = desc_k_sw128(w_lo + kk * 32);
            mma_bf16(td, dah, dwh, C::IDESC, (kb | kk) != 0);
            mma_bf16(td, dah, dwl, C::IDESC, 1u);
            mma_bf16(td, dal, dwh, C::IDESC, 1u);
          }
          mma_commit(empty0 + 8 * s);  // frees the stage once these MMAs have read it
        }
        mma_commit(accf0 + 8 * buf);  // this tile's accumulator is complete (also after an abort)
      }
      mma_commit(done);  // every MMA this CTA issued has completed
    }
  } else {
    // ---- epilogue: TMEM -> registers -> global, transposed ----
    const int q = warp & 3;  // this warp's TMEM lane quarter
    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      int pi, b, m0, n0;
      tile_coords(g, tile, pi, b, m0, n0);
      const Prob &P = g.p[pi];
      const int buf = j & 1;
      if (!wait_bounded(accf0 + 8 * buf, (j >> 1) & 1, abort_p, g.err, ERR_ACC, g.wait_cycles)) break;
      tc_fence_after();
      const int m = m0 + q * 32 + lane;
      const long long base = (long long)b * P.o_bstride + m;
      const uint32_t ta = tmem + (uint32_t)(buf * TMEM_COLS) + ((uint32_t)(q * 32) << 16);
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(ta + (uint32_t)c0, v);
        if (P.kind == OUT_F32) {
          float *o = static_cast<float *>(P.out);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            o[(base + (long long)(n0 + c0 + jj) * P.M) * P.ostride] = __uint_as_float(v[jj]);
        } else {
          __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(P.out);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const float f = __uint_as_float(v[jj]);
            const __nv_bfloat16 h = __float2bfloat16_rn(f);
            const long long id = base + (long long)(n0 + c0 + jj) * P.M;
            o[id] = h;
            o[id + P.plane] = __float2bfloat16_rn(f - __bfloat162float(h));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * buf);  // this warp's quarter of the buffer is drained
    }
  }
  __syncthreads();
  if (warp == 1) {
    // no MMA may still write tensor memory when it is freed: wait (bounded,
    // whatever the abort state) for the commit that follows the last one
    if (lane == 0) {
      const long long t0 = clock64();
      while (!mbar_try_wait(done, 0) && clock64() - t0 < g.wait_cycles) {
      }
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 2 * TMEM_COLS);
  }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn(std::string *why) {
  static EncodeTiledFn fn = nullptr;
  if (fn) return fn;
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    if (why) *why = "cuTensorMapEncodeTiled is not available from the driver";
    return nullptr;
  }
  fn = reinterpret_cast<EncodeTiledFn>(p);
  return fn;
}

// A operand: BF16 planes [plane][batch][M][K] with the given strides (elements).
static bool map_a(CUtensorMap *m, const void *base, int K, int M, int batches, long long bstride,
                  long long plane, std::string *why) {
  EncodeTiledFn f = encode_fn(why);
  if (!f) return false;
  cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)M, (cuuint64_t)batches, 2};
  cuuint64_t strides[3] = {(cuuint64_t)K * 2, (cuuint64_t)bstride * 2, (cuuint64_t)plane * 2};
  cuuint32_t box[4] = {BK, BM, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (why) *why = "cuTensorMapEncodeTiled failed for an A operand (code " + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// W operand: BF16 planes [plane][N][K].
static bool map_w(CUtensorMap *m, const void *base, int K, int N, long long plane, int bn, std::string *why) {
  EncodeTiledFn f = encode_fn(why);
  if (!f) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)N, 2};
  cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)plane * 2};
  cuuint32_t box[3] = {BK, (cuuint32_t)bn, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (why) *why = "cuTensorMapEncodeTiled failed for a W operand (code " + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// One product of a group: A planes (base, batch stride, plane stride), W
// planes (base, plane stride), output.
struct ProbSpec {
  const __nv_bfloat16 *A;
  long long a_bstride, a_plane;
  const __nv_bfloat16 *W;
  long long w_plane;
  void *out;
  long long o_bstride, o_plane;
  int kind, batches, M, N, K;
  int ostride;  // 0 or 1: contiguous
};

static bool make_group(Group *g, std::initializer_list<ProbSpec> specs, int *err, std::string *why, int bn = 64) {
  std::memset(g, 0, sizeof(Group));
  g->err = err;
  g->bn = bn;
  g->wait_cycles = kWaitCycles;
  g->skip_loads = 0;
  int tiles = 0;
  for (const ProbSpec &s : specs) {
    if (s.M % BM || s.N % bn || s.K % BK) {
      if (why) *why = "product sizes must be multiples of 128 (M), the tile width (N) and 64 (K)";
      return false;
    }
    const int i = g->count;
    if (!map_a(&g->amap[i], s.A, s.K, s.M, s.batches, s.a_bstride, s.a_plane, why)) return false;
    if (!map_w(&g->wmap[i], s.W, s.K, s.N, s.w_plane, bn, why)) return false;
    Prob &p = g->p[i];
    p.out = s.out;
    p.plane = s.o_plane;
    p.o_bstride = s.o_bstride;
    p.M = s.M;
    p.N = s.N;
    p.K = s.K;
    p.batches = s.batches;
    p.tiles_m = s.M / BM;
    p.tiles_n = s.N / bn;
    p.kind = s.kind;
    p.ostride = s.ostride > 1 ? s.ostride : 1;
    g->tile_start[i] = tiles;
    tiles += s.batches * p.tiles_m * p.tiles_n;
    g->count++;
  }
  g->tile_start[g->count] = tiles;
  return true;
}

static int group_tiles(const Group &g) { return g.tile_start[g.count]; }

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      n = v;
  }
  return n > 0 ? n : 1;
}

// One persistent CTA per SM at most (4-stage pipeline, 193 KiB of shared
// memory); a CTA loops over its tiles.
static void launch(const Group &g, cudaStream_t s) {
  const int ctas = std::min(group_tiles(g), sm_count());
  if (g.bn == 128)
    k_tc_gemm<128><<<ctas, 192, TileCfg<128>::SMEM, s>>>(g);
  else
    k_tc_gemm<64><<<ctas, 192, TileCfg<64>::SMEM, s>>>(g);
}

static bool reserve_smem() {
  return cudaFuncSetAttribute(k_tc_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TileCfg<64>::SMEM) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_tc_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, TileCfg<128>::SMEM) ==
             cudaSuccess;
}

// Round-to-nearest-even FP32 -> BF16 on the host.
static uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
static float host_f32(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// Split v into hi/lo planes: dst[i] = bf16(v), dst[plane + i] = bf16(v - hi).
static void host_split(const std::vector<double> &v, std::vector<uint16_t> &dst) {
  dst.resize(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const uint16_t h = host_bf16((float)v[i]);
    dst[i] = h;
    dst[v.size() + i] = host_bf16((float)(v[i] - (double)host_f32(h)));
  }
}

struct TcPlan {
  int nx = 0, ny = 0, nz = 0;
  size_t nb = 0;
  __nv_bfloat16 *rho = nullptr, *t1 = nullptr, *cz = nullptr, *sz = nullptr, *xinv = nullptr, *x2 = nullptr;
  float *t2 = nullptr;
  __nv_bfloat16 *Wfx = nullptr, *Wfy = nullptr, *Wbx = nullptr, *Wcy = nullptr, *Wsy = nullptr;
  const ZStageC *zc = nullptr;
  int *err = nullptr;
  // the four product groups (x forward, y forward, x inverse, y inverse),
  // each built with 64- and 128-column tiles; pick[k] is the variant used
  enum { FX = 0, FY = 1, IX = 2, IY = 3 };
  Group g[4][2];
  int pick[4] = {0, 0, 0, 0};
};

static void free_plan(TcPlan *p) {
  void *bufs[] = {p->rho, p->t1, p->cz, p->sz, p->xinv, p->x2, p->t2, p->Wfx, p->Wfy, p->Wbx, p->Wcy, p->Wsy, p->err};
  for (void *b : bufs)
    if (b) cudaFree(b);
  delete p;
}

template <typename T> static bool dev_alloc(T **p, size_t elems, std::string *why) {
  if (cudaMalloc(reinterpret_cast<void **>(p), elems * sizeof(T)) != cudaSuccess) {
    if (why) *why = "device allocation failed";
    return false;
  }
  return true;
}

static bool upload_split(__nv_bfloat16 **dst, const std::vector<double> &v, std::string *why) {
  std::vector<uint16_t> h;
  host_split(v, h);
  if (!dev_alloc(dst, h.size(), why)) return false;
  return cudaMemcpy(*dst, h.data(), h.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess;
}

TcPlan *create(int device, int nx, int ny, int nz, double dx, double dy, double dz, void *e4, const ZStageC *zc,
               std::string *why) {
  (void)dz;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess || prop.major != 10 || prop.minor != 3) {
    if (why) *why = "the tensor-core path is built for sm_103 (GB300) devices";
    return nullptr;
  }
  if (nx % 128 || ny % 128) {
    if (why) *why = "N_x and N_y must be multiples of 128";
    return nullptr;
  }
  if (!reserve_smem()) {
    if (why) *why = "cannot reserve shared memory for the tensor-core kernel";
    return nullptr;
  }
  TcPlan *p = new TcPlan();
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->nb = (size_t)nx * ny * nz;
  p->zc = zc;
  const size_t nb = p->nb;
  bool ok = dev_alloc(&p->rho, 2 * nb, why) && dev_alloc(&p->t1, 2 * nb, why) && dev_alloc(&p->cz, 2 * nb, why) &&
            dev_alloc(&p->sz, 2 * nb, why) && dev_alloc(&p->xinv, 4 * nb, why) && dev_alloc(&p->x2, 2 * nb, why) &&
            dev_alloc(&p->t2, nb, why) && dev_alloc(&p->err, 1, why);
  if (ok) ok = cudaMemset(p->err, 0, sizeof(int)) == cudaSuccess;
  // trig matrices (rows = output index n, K-contiguous), split into BF16 planes
  const double pi = 3.14159265358979323846;
  auto fwd = [&](int n) {
    std::vector<double> m((size_t)n * n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) m[(size_t)j * n + i] = std::cos(pi * j * (i + 0.5) / n);
    return m;
  };
  auto inv = [&](int n, double d, bool sine) {
    std::vector<double> m((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double arg = pi * j * (i + 0.5) / n;
        m[(size_t)i * n + j] = sine ? (j * pi / d) * std::sin(arg) : std::cos(arg);
      }
    return m;
  };
  if (ok) {
    std::vector<double> bx = inv(nx, dx, true), cx = inv(nx, dx, false);
    bx.insert(bx.end(), cx.begin(), cx.end());  // [S_x; C_x], 2 nx rows
    ok = upload_split(&p->Wfx, fwd(nx), why) && upload_split(&p->Wfy, fwd(ny), why) &&
         upload_split(&p->Wbx, bx, why) && upload_split(&p->Wcy, inv(ny, dy, false), why) &&
         upload_split(&p->Wsy, inv(ny, dy, true), why);
  }
  const long long pl = (long long)nx * ny, snb = (long long)nb;
  const long long wx = (long long)nx * nx, wy = (long long)ny * ny;
  float *e = static_cast<float *>(e4);
  for (int v = 0; v < 2 && ok; ++v) {
    const int bn = v ? 128 : 64;
    // x forward: rho[z][y][x] -> t1[z][j][y] (split)
    ok = make_group(&p->g[TcPlan::FX][v], {{p->rho, pl, snb, p->Wfx, wx, p->t1, pl, snb, OUT_SPLIT, nz, ny, nx, nx}},
                    p->err, why, bn);
    // y forward: t1[z][j][y] -> t2[z][k][j] (FP32, for the z stage)
    if (ok)
      ok = make_group(&p->g[TcPlan::FY][v], {{p->t1, pl, snb, p->Wfy, wy, p->t2, pl, 0, OUT_F32, nz, nx, ny, ny}},
                      p->err, why, bn);
    // x inverse: [S_x; C_x] Czpsi -> xinv[z][2nx][ny], C_x Szpsi -> x2[z][nx][ny]
    if (ok)
      ok = make_group(&p->g[TcPlan::IX][v],
                      {{p->cz, pl, snb, p->Wbx, 2 * wx, p->xinv, 2 * pl, 2 * snb, OUT_SPLIT, nz, ny, 2 * nx, nx},
                       {p->sz, pl, snb, p->Wbx + wx, 2 * wx, p->x2, pl, snb, OUT_SPLIT, nz, ny, nx, nx}},
                      p->err, why, bn);
    // y inverse: E_x = C_y (S_x C_z psi), E_y = S_y (C_x C_z psi), E_z = C_y (C_x S_z psi), written
    // interleaved into e4[z][y][x] = (E_x, E_y, E_z, -) so the gather reads one vector per bin
    if (ok)
      ok = make_group(&p->g[TcPlan::IY][v],
                      {{p->xinv, 2 * pl, 2 * snb, p->Wcy, wy, e + 0, pl, 0, OUT_F32, nz, nx, ny, ny, 4},
                       {p->xinv + pl, 2 * pl, 2 * snb, p->Wsy, wy, e + 1, pl, 0, OUT_F32, nz, nx, ny, ny, 4},
                       {p->x2, pl, snb, p->Wcy, wy, e + 2, pl, 0, OUT_F32, nz, nx, ny, ny, 4}},
                      p->err, why, bn);
  }
  if (!ok) {
    free_plan(p);
    return nullptr;
  }
  return p;
}

void densify(TcPlan *p, cudaStream_t s, int nxy, int nz, const long long *q, const long long *corner, float *part) {
  k_densify<float><<<(nxy + 255) / 256, 256, 0, s>>>(nxy, nz, q, corner, OutSplit{p->rho, (long long)p->nb}, part);
}

int forward(TcPlan *p, cudaStream_t s) {
  launch(p->g[TcPlan::FX][p->pick[TcPlan::FX]], s);
  launch(p->g[TcPlan::FY][p->pick[TcPlan::FY]], s);
  return 2;
}

int zstage(TcPlan *p, cudaStream_t s, float *part) {
  const int pl = p->nx * p->ny;
  const int g = (pl + 255) / 256;
  const OutSplit cz{p->cz, (long long)p->nb}, sz{p->sz, (long long)p->nb};
  if (p->nz <= 2)
    k_zstage<float, 2><<<g, 256, 0, s>>>(p->zc, p->t2, cz, sz, part);
  else if (p->nz <= 4)
    k_zstage<float, 4><<<g, 256, 0, s>>>(p->zc, p->t2, cz, sz, part);
  else if (p->nz <= 8)
    k_zstage<float, 8><<<g, 256, 0, s>>>(p->zc, p->t2, cz, sz, part);
  else
    k_zstage<float, 16><<<g, 256, 0, s>>>(p->zc, p->t2, cz, sz, part);
  return 1;
}

int inverse(TcPlan *p, cudaStream_t s) {
  launch(p->g[TcPlan::IX][p->pick[TcPlan::IX]], s);
  launch(p->g[TcPlan::IY][p->pick[TcPlan::IY]], s);
  return 2;
}

int autotune(TcPlan *p, cudaStream_t s, int repeats) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1;
  }
  int rc = 0;
  for (int k = 0; k < 4 && rc == 0; ++k) {
    float best = 1e30f;
    for (int v = 0; v < 2; ++v) {
      float ms = 1e30f;  // fastest of `repeats` timed launches after one warm-up launch
      for (int r = 0; r <= repeats; ++r) {
        cudaEventRecord(e0, s);
        launch(p->g[k][v], s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = -1;
          break;
        }
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) ms = std::min(ms, t);
      }
      if (rc == 0 && ms < best) {
        best = ms;
        p->pick[k] = v;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc != 0 || cudaGetLastError() != cudaSuccess ? -1 : 0;
}

int tile_columns(const TcPlan *p, int group) { return p->g[group][p->pick[group]].bn; }
void set_tile_columns(TcPlan *p, int group, int bn) { p->pick[group] = bn == 128 ? 1 : 0; }

int error_code(TcPlan *p) {
  int e = 0;
  if (cudaMemcpy(&e, p->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return e;
}

void destroy(TcPlan *p) {
  if (p) free_plan(p);
}

}  // namespace p3d_tc

// Self-test of one product through the tensor cores: A [batches][M][K] and
// W [N][K] (host FP32, row-major) -> out [batches][N][M] (host FP32).
extern "C" int place3d_tc_selftest(int M, int N, int K, int batches, const float *A, const float *W, float *out,
                                   int *wait_error) {
  using namespace p3d_tc;
  if (M <= 0 || N <= 0 || K <= 0 || batches <= 0 || !A || !W || !out) return PLACE3D_ERR_INVALID_ARG;
  if (M % BM || N % kMinBN || K % BK) return PLACE3D_ERR_INVALID_ARG;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
      prop.major != 10 || prop.minor != 3)
    return PLACE3D_ERR_UNSUPPORTED;
  if (!reserve_smem()) return PLACE3D_ERR_CUDA;
  const size_t na = (size_t)batches * M * K, nw = (size_t)N * K, no = (size_t)batches * N * M;
  std::vector<double> av(A, A + na), wv(W, W + nw);
  std::string why;
  __nv_bfloat16 *da = nullptr, *dw = nullptr;
  float *dout = nullptr;
  int *err = nullptr;
  int rc = PLACE3D_ERR_CUDA;
  Group g;
  if (upload_split(&da, av, &why) && upload_split(&dw, wv, &why) && dev_alloc(&dout, no, &why) &&
      dev_alloc(&err, 1, &why) && cudaMemset(err, 0, sizeof(int)) == cudaSuccess &&
      cudaMemset(dout, 0, no * sizeof(float)) == cudaSuccess &&
      make_group(&g, {{da, (long long)M * K, (long long)na, dw, (long long)nw, dout, (long long)N * M, 0, OUT_F32,
                       batches, M, N, K}},
                 err, &why)) {
    launch(g, 0);
    if (cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(out, dout, no * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess) {
      int e = 0;
      cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
      if (wait_error) *wait_error = e;
      rc = e ? PLACE3D_ERR_TIMEOUT : PLACE3D_OK;
    }
  }
  if (da) cudaFree(da);
  if (dw) cudaFree(dw);
  if (dout) cudaFree(dout);
  if (err) cudaFree(err);
  return rc;
}

// Failure-path self-test: a 128x64x64 product whose producer arms and loads
// nothing, with every wait bounded by wait_cycles.  A wait runs out, the CTA
// records its code, stops, frees its tensor memory and exits; the call
// returns PLACE3D_ERR_TIMEOUT with *wait_error > 0 and the context stays
// usable.
extern "C" int place3d_tc_timeout_selftest(long long wait_cycles, int *wait_error) {
  using namespace p3d_tc;
  if (wait_cycles <= 0) return PLACE3D_ERR_INVALID_ARG;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
      prop.major != 10 || prop.minor != 3)
    return PLACE3D_ERR_UNSUPPORTED;
  if (!reserve_smem()) return PLACE3D_ERR_CUDA;
  const int M = BM, N = kMinBN, K = BK;
  std::vector<double> av((size_t)M * K, 0.0), wv((size_t)N * K, 0.0);
  std::string why;
  __nv_bfloat16 *da = nullptr, *dw = nullptr;
  float *dout = nullptr;
  int *err = nullptr;
  int rc = PLACE3D_ERR_CUDA;
  Group g;
  if (upload_split(&da, av, &why) && upload_split(&dw, wv, &why) && dev_alloc(&dout, (size_t)N * M, &why) &&
      dev_alloc(&err, 1, &why) && cudaMemset(err, 0, sizeof(int)) == cudaSuccess &&
      make_group(&g, {{da, (long long)M * K, (long long)M * K, dw, (long long)N * K, dout, (long long)N * M, 0,
                       OUT_F32, 1, M, N, K}},
                 err, &why)) {
    g.wait_cycles = wait_cycles;
    g.skip_loads = 1;
    launch(g, 0);
    if (cudaDeviceSynchronize() == cudaSuccess) {
      int e = 0;
      cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
      if (wait_error) *wait_error = e;
      rc = e ? PLACE3D_ERR_TIMEOUT : PLACE3D_OK;
    }
  }
  if (da) cudaFree(da);
  if (dw) cudaFree(dw);
  if (dout) cudaFree(dout);
  if (err) cudaFree(err);
  return rc;
}
