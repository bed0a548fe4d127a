// Spectral Poisson solve (eqs. density-coef, poisson-sol-potential,
// possion-sol-force) as per-axis dense matrix products, CUDA-core form
// (FP64 plain path and FP32 path), plus the z-axis stage that applies the
// N_z-point transforms, the spectral scaling and the energy sum.
#pragma once
#include "common.cuh"

namespace p3d {

// One batched product out[b][n][m] = sum_k A[b][m][k] * W[n][k]: rows of A
// are contracted with rows of W (both K-contiguous) and the result is
// stored transposed, so that the next axis becomes the contiguous one.
template <typename T> struct GemmProb {
  const T *A;
  const T *W;
  T *out;
  long long a_bstride, o_bstride;  // elements between batches
  int ostride;                     // element stride of the output (4: one component of an interleaved map)
  int batches, M, N, K;
  int tiles_m, tiles_n;            // filled by the launcher
};

template <typename T> struct GemmGroup {
  GemmProb<T> p[3];
  int count;
  int tile_start[4];
};

constexpr int kBM = 64, kBN = 64, kBK = 16;

// 256 threads, 64x64 tile, each thread 4 (m) x 4 (n) outputs.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_simt(GemmGroup<T> g) {
  __shared__ T As[kBK][kBM + 4];
  __shared__ T Ws[kBK][kBN + 4];
  int tile = blockIdx.x, pi = 0;
  while (pi + 1 < g.count && tile >= g.tile_start[pi + 1]) ++pi;
  const GemmProb<T> &P = g.p[pi];
  tile -= g.tile_start[pi];
  const int per_batch = P.tiles_m * P.tiles_n;
  const int b = tile / per_batch;
  const int r = tile - b * per_batch;
  const int m0 = (r % P.tiles_m) * kBM, n0 = (r / P.tiles_m) * kBN;
  const T *A = P.A + (long long)b * P.a_bstride;
  T *O = P.out + (long long)b * P.o_bstride * P.ostride;
  const int t = threadIdx.x;
  const int tm = t & 15, tn = t >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  // loader mapping: 64 rows x 16 k, 4 consecutive k per thread
  const int lr = t >> 2, lk = (t & 3) * 4;
  for (int k0 = 0; k0 < P.K; k0 += kBK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int kk = k0 + lk + u;
      const int am = m0 + lr, wn = n0 + lr;
      As[lk + u][lr] = (am < P.M && kk < P.K) ? A[(long long)am * P.K + kk] : T(0);
      Ws[lk + u][lr] = (wn < P.N && kk < P.K) ? P.W[(long long)wn * P.K + kk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      T a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = Ws[kk][tn * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * w[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = n0 + tn * 4 + j;
    if (n >= P.N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + tm * 4 + i;
      if (m < P.M) O[((long long)n * P.M + m) * P.ostride] = acc[i][j];
    }
  }
}

// z-stage constants.
constexpr int kMaxNz = 16;
struct ZStageC {
  int nx, ny, nz;
  int mode2d;                  // 1: each layer an independent 2D field (eq. 2d-place)
  double pi_dx, pi_dy, pi_dz;  // pi/d_x, pi/d_y, pi/d_z
  double inv_n;                // 1/N
  float pi_dx_f, pi_dy_f, pi_dz_f, inv_n_f;  // the same, rounded to FP32
  double cz[kMaxNz * kMaxNz];  // cos(pi l (z+1/2)/N_z), [l][z]
  double sz[kMaxNz * kMaxNz];  // w_l sin(pi l (z+1/2)/N_z), [l][z]
  // The same tables rounded to FP32: an FP64 -> FP32 conversion per use runs
  // on the FP64 pipe, a small fraction of the FP32 rate on this GPU.
  float cz_f[kMaxNz * kMaxNz];
  float sz_f[kMaxNz * kMaxNz];
};

// Input T2[z][k][j] (x and y already transformed, j fastest).  For each
// (k, j): a_l = (1/N) sum_z T2[z] cos(...), psi = c_j c_k c_l a/|w|^2 (psi_000
// = 0), energy sum += c c c a^2/|w|^2, then Czpsi[z] = sum_l psi_l cos(...)
// and Szpsi[z] = sum_l psi_l w_l sin(...).  One thread per (k, j); the z
// loops are unrolled to NZM >= N_z so the per-thread vectors stay in
// registers.
template <typename T> struct ZPar;
template <> struct ZPar<double> {
  static __device__ __forceinline__ double pdx(const ZStageC *z) { return z->pi_dx; }
  static __device__ __forceinline__ double pdy(const ZStageC *z) { return z->pi_dy; }
  static __device__ __forceinline__ double pdz(const ZStageC *z) { return z->pi_dz; }
  static __device__ __forceinline__ double invn(const ZStageC *z) { return z->inv_n; }
  static __device__ __forceinline__ double cz(const ZStageC *z, int i) { return z->cz[i]; }
  static __device__ __forceinline__ double sz(const ZStageC *z, int i) { return z->sz[i]; }
};
template <> struct ZPar<float> {
  static __device__ __forceinline__ float pdx(const ZStageC *z) { return z->pi_dx_f; }
  static __device__ __forceinline__ float pdy(const ZStageC *z) { return z->pi_dy_f; }
  static __device__ __forceinline__ float pdz(const ZStageC *z) { return z->pi_dz_f; }
  static __device__ __forceinline__ float invn(const ZStageC *z) { return z->inv_n_f; }
  static __device__ __forceinline__ float cz(const ZStageC *z, int i) { return z->cz_f[i]; }
  static __device__ __forceinline__ float sz(const ZStageC *z, int i) { return z->sz_f[i]; }
};

// All arithmetic in T (FP32 threads stay off the FP64 pipe); the energy sums
// leave one row per warp in T for k_sum_parts.  2D mode (zc->mode2d, N_z = 3 layers): no z
// transform, psi = c_j c_k a / (w_j^2 + w_k^2) per layer with a = (1/(N_x
// N_y)) T2, E_z = 0 (Szpsi = 0), one energy sum per layer.  The warp
// sums go to part[warp][1] (3D) or part[warp][3] (2D), added up by
// k_sum_parts into S_ESUM or S_EL0..S_EL2.
template <typename T, int NZM, typename Out>
__global__ void __launch_bounds__(256) k_zstage(const ZStageC *__restrict__ zc, const T *__restrict__ in,
                                                Out czpsi, Out szpsi, T *__restrict__ part) {
  const int nx = zc->nx, ny = zc->ny, nz = zc->nz;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (zc->mode2d) {
    T el[3] = {0, 0, 0};
    if (t < nx * ny) {
      const int j = t % nx, k = t / nx;
      const size_t plane = (size_t)nx * ny;
      const T wj = (T)j * ZPar<T>::pdx(zc), wk = (T)k * ZPar<T>::pdy(zc);
      const T w2 = wj * wj + wk * wk;
      const T cw = (j | k) ? (j ? T(2) : T(1)) * (k ? T(2) : T(1)) / w2 : T(0);
      const T invn = ZPar<T>::invn(zc);
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const T a = in[l * plane + t] * invn;
        const T psi = cw * a;
        el[l] = cw * a * a;
        czpsi.put(l * plane + t, psi);
        szpsi.put(l * plane + t, T(0));
      }
    }
    warp_sum_part<3>(el, part);  // per-layer energy rows
    return;
  }
  T e = 0;
  if (t < nx * ny) {
    const int j = t % nx, k = t / nx;
    const size_t plane = (size_t)nx * ny;
    T v[NZM];
#pragma unroll
    for (int z = 0; z < NZM; ++z) v[z] = z < nz ? in[z * plane + t] : T(0);
    const T wj = (T)j * ZPar<T>::pdx(zc), wk = (T)k * ZPar<T>::pdy(zc);
    const T cjk = (j ? T(2) : T(1)) * (k ? T(2) : T(1));
    const T invn = ZPar<T>::invn(zc);
    T psi[NZM];
#pragma unroll
    for (int l = 0; l < NZM; ++l) {
      T a = 0;
#pragma unroll
      for (int z = 0; z < NZM; ++z) a += v[z] * ZPar<T>::cz(zc, l * kMaxNz + z);
      a *= invn;
      const T wl = (T)l * ZPar<T>::pdz(zc);
      const T w2 = wj * wj + wk * wk + wl * wl;
      psi[l] = T(0);
      if (l < nz && (j | k | l)) {
        const T cw = cjk * (l ? T(2) : T(1)) / w2;
        psi[l] = cw * a;
        e += cw * a * a;
      }
    }
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
      if (z >= nz) break;
      T sc = 0, ss = 0;
#pragma unroll
      for (int l = 0; l < NZM; ++l) {
        sc += psi[l] * ZPar<T>::cz(zc, l * kMaxNz + z);
        ss += psi[l] * ZPar<T>::sz(zc, l * kMaxNz + z);
      }
      czpsi.put(z * plane + t, sc);
      szpsi.put(z * plane + t, ss);
    }
  }
  T v1[1] = {e};
  warp_sum_part<1>(v1, part);  // energy rows
}

}  // namespace p3d
