// Shared device helpers of the place3d kernels (sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace p3d {

template <typename T> struct V4;
template <> struct alignas(16) V4<float> { float x, y, z, w; };
template <> struct alignas(32) V4<double> { double x, y, z, w; };

// One IEEE-rounded operation each; never contracted into an FMA.  The
// fixed-point density contract (quantised contributions) is defined on these.
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float r_floor(float a) { return floorf(a); }
__device__ __forceinline__ double r_floor(double a) { return floor(a); }
__device__ __forceinline__ float r_ceil(float a) { return ceilf(a); }
__device__ __forceinline__ double r_ceil(double a) { return ceil(a); }
// Round-half-to-even of a non-negative float to int64 without the
// float -> 64-bit conversion instruction (it runs on the FP64 pipe, which is
// narrow on this GPU), and without branches (the lanes of a warp quantise
// contributions of very different sizes).  a = m * 2^s with a 24-bit
// mantissa m:
//   a >= 2^23 (s >= 0): a is an integer, m << s;
//   a < 2^23: a + 2^23 lies in [2^23, 2^24), where one ulp is 1, so the FP32
//   add itself rounds a to the nearest integer (ties to even), read off the
//   sum's mantissa.
// Exactly llrintf for 0 <= a < 2^63; 0 for a <= 0.
__device__ __forceinline__ long long r_rint(float a) {
  const unsigned u = __float_as_uint(a);
  const int s = (int)((u >> 23) & 0xffu) - 150;
  const long long big = (long long)((unsigned long long)((u & 0x7fffffu) | 0x800000u) << (s > 0 ? s : 0));
  const long long small = (long long)(__float_as_int(__fadd_rn(a, 8388608.0f)) - 0x4B000000);
  return a >= 8388608.0f ? big : (a > 0.0f ? small : 0ll);
}
__device__ __forceinline__ long long r_rint(double a) { return __double2ll_rn(a); }
// int64 -> FP32, round half to even, with 32-bit and integer operations only
// (the 64-bit integer conversion instruction runs on the FP64 pipe).  |v| =
// m 2^sh + rem with a 24-bit m: round m by rem against half of 2^sh (ties to
// even), then scale by 2^sh, exact.  Equal to __ll2float_rn for every v.
__device__ __forceinline__ float r_ll2f(long long v) {
  const bool neg = v < 0;
  const unsigned long long u = neg ? 0ull - (unsigned long long)v : (unsigned long long)v;
  float r;
  if (u < (1ull << 24)) {
    r = __uint2float_rn((unsigned)u);  // exact
  } else {
    const int sh = 63 - __clzll((long long)u) - 23;  // 1 <= sh <= 40
    unsigned m = (unsigned)(u >> sh);
    const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    m += (rem > half || (rem == half && (m & 1u))) ? 1u : 0u;  // m <= 2^24
    r = __uint2float_rn(m) * __int_as_float((127 + sh) << 23);
  }
  return neg ? -r : r;
}
__device__ __forceinline__ double r_ll2f(long long v, double) { return (double)v; }
__device__ __forceinline__ float r_ll2f(long long v, float) { return r_ll2f(v); }
// FP32 mode uses the fast exponential (a few ulp near 0, where the dominant
// WA terms are); FP64 mode the full-precision one.
__device__ __forceinline__ float r_exp(float a) { return __expf(a); }
__device__ __forceinline__ double r_exp(double a) { return exp(a); }
// 2^a: the hardware's approximate base-2 exponential in FP32 (the same unit
// __expf uses, without its scaling multiply), exp2 in FP64.
__device__ __forceinline__ float r_exp2(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double r_exp2(double a) { return exp2(a); }
// 1/a for the wirelength's WA sums (a in [1, #pins]): the fast approximate
// division in FP32 (a few ulp, far inside the FP32 path's tolerance), IEEE
// division in FP64.
__device__ __forceinline__ float r_rcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double r_rcp(double a) { return 1.0 / a; }

// Packed FP32 pair arithmetic (sm_100 and later): (d0, d1) = (a0 b0 + c0,
// a1 b1 + c1) in one instruction, each lane rounded to nearest as a single
// FMA.  Used where the x and y axes take the same steps.
__device__ __forceinline__ void fma2(float a0, float a1, float b0, float b1, float &c0, float &c1) {
  asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%0, %1};\n\t"
      "fma.rn.f32x2 rc, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rc;\n\t}"
      : "+f"(c0), "+f"(c1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void fma2(double a0, double a1, double b0, double b1, double &c0, double &c1) {
  c0 = fma(a0, b0, c0);
  c1 = fma(a1, b1, c1);
}
// (a0 - b0, a1 - b1) * (s0, s1), the subtraction and the product each rounded.
__device__ __forceinline__ void submul2(float a0, float a1, float b0, float b1, float s0, float s1, float &d0,
                                        float &d1) {
  asm("{\n\t.reg .b64 ra, rb, rs, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rs, {%6, %7};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mul.rn.f32x2 rd, rd, rs;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(s0), "f"(s1));
}
__device__ __forceinline__ void submul2(double a0, double a1, double b0, double b1, double s0, double s1, double &d0,
                                        double &d1) {
  d0 = (a0 - b0) * s0;
  d1 = (a1 - b1) * s1;
}
// WA gradient of both axes at once: g_a = (e+_a A_a)(1 + (v_a - B_a) ig) -
// (e-_a C_a)(1 - (v_a - D_a) ig), a = x, y.
__device__ __forceinline__ void wa_grad2(const float (&ep)[2], const float (&em)[2], const float (&v)[2],
                                         const float (&A)[2], const float (&B)[2], const float (&C)[2],
                                         const float (&D)[2], float ig, float (&g)[2]) {
  asm("{\n\t.reg .b64 ep, em, v, A, B, C, D, ig, nig, one, t1, t2, u1, u2, r;\n\t"
      "mov.b64 ep, {%2, %3};\n\t"
      "mov.b64 em, {%4, %5};\n\t"
      "mov.b64 v, {%6, %7};\n\t"
      "mov.b64 A, {%8, %9};\n\t"
      "mov.b64 B, {%10, %11};\n\t"
      "mov.b64 C, {%12, %13};\n\t"
      "mov.b64 D, {%14, %15};\n\t"
      "mov.b64 ig, {%16, %16};\n\t"
      "mov.b64 nig, {%18, %18};\n\t"
      "mov.b64 one, {%17, %17};\n\t"
      "mul.rn.f32x2 t1, ep, A;\n\t"
      "mul.rn.f32x2 t2, em, C;\n\t"
      "sub.rn.f32x2 u1, v, B;\n\t"
      "sub.rn.f32x2 u2, v, D;\n\t"
      "fma.rn.f32x2 u1, u1, ig, one;\n\t"
      "fma.rn.f32x2 u2, u2, nig, one;\n\t"
      "mul.rn.f32x2 r, t1, u1;\n\t"
      "mul.rn.f32x2 t2, t2, u2;\n\t"
      "sub.rn.f32x2 r, r, t2;\n\t"
      "mov.b64 {%0, %1}, r;\n\t}"
      : "=f"(g[0]), "=f"(g[1])
      : "f"(ep[0]), "f"(ep[1]), "f"(em[0]), "f"(em[1]), "f"(v[0]), "f"(v[1]), "f"(A[0]), "f"(A[1]), "f"(B[0]),
        "f"(B[1]), "f"(C[0]), "f"(C[1]), "f"(D[0]), "f"(D[1]), "f"(ig), "f"(1.0f), "f"(-ig));
}
__device__ __forceinline__ void wa_grad2(const double (&ep)[2], const double (&em)[2], const double (&v)[2],
                                         const double (&A)[2], const double (&B)[2], const double (&C)[2],
                                         const double (&D)[2], double ig, double (&g)[2]) {
  for (int a = 0; a < 2; ++a)
    g[a] = (ep[a] * A[a]) * (1.0 + (v[a] - B[a]) * ig) - (em[a] * C[a]) * (1.0 - (v[a] - D[a]) * ig);
}

template <typename T> __device__ __forceinline__ T big();
template <> __device__ __forceinline__ float big<float>() { return 3.0e38f; }
template <> __device__ __forceinline__ double big<double>() { return 1.0e300; }

__device__ __forceinline__ float shfl_xor(float v, int m, int w) {
  return __shfl_xor_sync(0xffffffffu, v, m, w);
}
__device__ __forceinline__ double shfl_xor(double v, int m, int w) {
  return __shfl_xor_sync(0xffffffffu, v, m, w);
}
__device__ __forceinline__ int shfl_xor(int v, int m, int w) {
  return __shfl_xor_sync(0xffffffffu, v, m, w);
}
__device__ __forceinline__ long long shfl_up_ll(long long v, int d) {
  return __shfl_up_sync(0xffffffffu, v, d);
}

__device__ __forceinline__ void atomic_add_i64(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// Per-instance gradient accumulators (gx, gy, fd, waz).
__device__ __forceinline__ void acc_add(V4<float> *p, float a, float b, float c, float d) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
#else
  atomicAdd(&p->x, a);
  atomicAdd(&p->y, b);
  atomicAdd(&p->z, c);
  atomicAdd(&p->w, d);
#endif
}
__device__ __forceinline__ void acc_add(V4<double> *p, double a, double b, double c, double d) {
  atomicAdd(&p->x, a);
  atomicAdd(&p->y, b);
  atomicAdd(&p->z, c);
  atomicAdd(&p->w, d);
}

// Block-wide sum of NV values into FP64 global accumulators (one atomic per
// block and value).  Lanes reduce in their own precision T (FP32 lanes stay
// off the slow FP64 pipe); each warp's partial is widened to FP64 once and
// one thread adds the block's warps in FP64.  All threads must call it.
template <int NV, typename T>
__device__ __forceinline__ void block_sum_atomic(T (&v)[NV], double *dst) {
  __shared__ double red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T s = v[k];
#pragma unroll
    for (int m = 16; m; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) red[warp][k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w][k];
      if (s != 0.0) atomicAdd(dst + k, s);
    }
  }
}

// Warp-wide sum of NV values stored (plain store, in the lanes' precision T)
// into this warp's row part[global warp][NV]; k_sum_parts adds the rows up
// later.  No block barrier and no atomics: a block-wide reduction at the end
// of a kernel makes every warp wait for the block's slowest one, and
// thousands of FP64 atomics to the same words serialise in the L2.  FP32
// rows stay FP32: widening each to FP64 here would put one conversion per
// warp and value on the FP64 pipe, which is narrow on this GPU.
// One-dimensional grids with whole warps; every lane must call it.
// bid: the block's index in its grid (a batched launch passes the block's
// index within its instance's share of the grid).
template <int NV, typename T>
__device__ __forceinline__ void warp_sum_part(T (&v)[NV], T *__restrict__ part, int bid = blockIdx.x) {
  const int lane = threadIdx.x & 31;
  const size_t row = ((size_t)bid * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T s = v[k];
#pragma unroll
    for (int m = 16; m; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) part[row * NV + k] = s;
  }
}

// (hi, lo) += v.  FP64: a plain sum (lo stays 0).  FP32: Knuth's two-sum,
// each addition rounded on its own, so hi + lo carries the sum to about
// 2^-44 relative with FP32 operations only (integer-valued sums below 2^48,
// such as crossing counts, stay exact).
__device__ __forceinline__ void ff_add(double &hi, double &, double v) { hi += v; }
__device__ __forceinline__ void ff_add(float &hi, float &lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// dst[k] += sum over rows r < rows of part[r][NV]: a grid-stride pass in
// the rows' precision (FP32 rows as hi + lo pairs), one block reduction
// widened to FP64 per warp and one FP64 atomic per block and value.
constexpr int kSumBlocks = 256;
// Body of k_sum_parts for block bid of nblk (256 threads each).
template <int NV, typename TP>
__device__ __forceinline__ void sum_parts_body(const TP *__restrict__ part, int rows, double *__restrict__ dst,
                                               int bid, int nblk);
template <int NV, typename TP>
__global__ void __launch_bounds__(256) k_sum_parts(const TP *__restrict__ part, int rows,
                                                   double *__restrict__ dst) {
  sum_parts_body<NV, TP>(part, rows, dst, blockIdx.x, gridDim.x);
}
template <int NV, typename TP>
__device__ __forceinline__ void sum_parts_body(const TP *__restrict__ part, int rows, double *__restrict__ dst,
                                               int bid, int nblk) {
  TP hi[NV], lo[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) hi[k] = lo[k] = TP(0);
  for (int r = bid * blockDim.x + threadIdx.x; r < rows; r += nblk * blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) ff_add(hi[k], lo[k], part[(size_t)r * NV + k]);
  __shared__ double red[8][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    TP h = hi[k], l = lo[k];
#pragma unroll
    for (int m = 16; m; m >>= 1) {
      const TP oh = __shfl_xor_sync(0xffffffffu, h, m), ol = __shfl_xor_sync(0xffffffffu, l, m);
      ff_add(h, l, oh);
      l += ol;
    }
    if (lane == 0) red[warp][k] = (double)h + (double)l;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w][k];
      if (s != 0.0) atomicAdd(dst + k, s);
    }
  }
}

// Map writers: plain values, or an FP32 value split into two BF16 planes
// (hi = bf16(v), lo = bf16(v - hi); lo plane `plane` elements after hi) for
// the tensor-core products.
template <typename T> struct OutPlain {
  T *p;
  __device__ __forceinline__ void put(size_t i, T v) const { p[i] = v; }
};
struct OutSplit {
  __nv_bfloat16 *hi;
  long long plane;
  __device__ __forceinline__ void put(size_t i, float v) const {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    hi[i + plane] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
};

// Indices of the device scalar accumulators.
enum Scalar {
  S_WL_BI = 0,
  S_WL_Z,
  S_HPWL,
  S_NCROSS,
  S_ESUM,  // sum c_j c_k c_l a^2 / w^2 (energy before the 1/2 vol(b) N factor)
  S_SX,
  S_SY,
  S_SZ,
  S_EL0,  // 2D mode: per-layer energy sums (bottom, top, HBT layer)
  S_EL1,
  S_EL2,
  S_OVFL,  // sum over bins of max(rho - 1, 0) (density overflow, target density 1)
  S_RHO,   // sum over bins of rho
  S_COUNT
};

}  // namespace p3d
