// Density kernels: fixed-point charge scatter (eq. density-map-accum for
// cells, Theorem 1 corners + 3D integer prefix sum for macros), conversion to
// the transform's input, suffix sums of the field for the macro gather, and
// the field gather fused with the wirelength-gradient add.
#pragma once
#include "common.cuh"

namespace p3d {

// Density constants, computed in double on the host and rounded once to T.
template <typename T> struct DensC {
  T x0, y0;          // region origin
  T iwb, ihb, idb;   // 1/w_b, 1/h_b, 1/d_b
  T cw, ch;          // sqrt(2) w_b, sqrt(2) h_b: local-smoothness thresholds
  T zmid, qz, tz;    // d_z/2, d_z/4, 2/d_z
  T fnx, fny, fnz;   // N_x, N_y, N_z as T
  int nx, ny, nz;
  int mode2d;        // 1: multi-die 2D (eq. 2d-place): layer = HBT ? 2 : top, die sizes, no z extent
};

constexpr double kFixedScale = 68719476736.0;  // 2^36 counts per unit density

template <typename T> struct Box {
  T lo[3], hi[3];  // stretched cuboid in bin units (x, y, z), unclipped
  T om;            // local-smoothness weight omega
};

// Instance cuboid D_i (Sec. IV-A) with the partition-dependent size (eq.
// std-size-tech for cells, eq. macro-size-tech for macros, clamped to the
// movable range) and local smoothness (omega, stretched footprint).  Every
// step is one IEEE-rounded operation in the order the fixed-point contract
// states, so that quantised contributions are reproducible bit for bit.
// 2D mode (c.mode2d): the partition is fixed, every instance (macros too)
// has its die's size, an HBT (hbt) its bottom-table size, and the cuboid
// fills exactly its layer's bin in z: [layer, layer + 1) in bin units.
template <typename T>
__device__ __forceinline__ Box<T> inst_box(const DensC<T> &c, T X, T Y, T Z, const V4<T> &sz,
                                           bool macro, bool hbt = false) {
  const bool top = !hbt && Z > c.zmid;
  T w, h;
  if (hbt) {
    w = sz.x;
    h = sz.y;
  } else if (macro && !c.mode2d) {
    T t = rn_sub(rn_mul(Z, c.tz), T(0.5));
    if (t < T(0)) t = T(0);
    if (t > T(1)) t = T(1);
    const T u = rn_sub(T(1), t);
    w = rn_add(rn_mul(t, sz.z), rn_mul(u, sz.x));
    h = rn_add(rn_mul(t, sz.w), rn_mul(u, sz.y));
  } else {
    w = top ? sz.z : sz.x;
    h = top ? sz.w : sz.y;
  }
  const T sw = w > c.cw ? w : c.cw;
  const T sh = h > c.ch ? h : c.ch;
  Box<T> b;
  b.om = rn_div(rn_mul(w, h), rn_mul(sw, sh));
  const T hw = rn_mul(T(0.5), sw), hh = rn_mul(T(0.5), sh);
  const T dx = rn_sub(X, c.x0), dy = rn_sub(Y, c.y0);
  b.lo[0] = rn_mul(rn_sub(dx, hw), c.iwb);
  b.hi[0] = rn_mul(rn_add(dx, hw), c.iwb);
  b.lo[1] = rn_mul(rn_sub(dy, hh), c.ihb);
  b.hi[1] = rn_mul(rn_add(dy, hh), c.ihb);
  if (c.mode2d) {
    const int layer = hbt ? 2 : (top ? 1 : 0);
    b.lo[2] = (T)layer;
    b.hi[2] = (T)(layer + 1);
  } else {
    b.lo[2] = rn_mul(rn_sub(Z, c.qz), c.idb);
    b.hi[2] = rn_mul(rn_add(Z, c.qz), c.idb);
  }
  return b;
}

// Clip [lo, hi] to [0, N] and return the bin index range; false if empty.
template <typename T>
__device__ __forceinline__ bool clip_axis(T lo, T hi, T fN, int n, T &cl, T &chh, int &b0, int &b1) {
  cl = lo > T(0) ? lo : T(0);
  chh = hi < fN ? hi : fN;
  if (!(cl < chh)) return false;
  b0 = (int)r_floor(cl);
  b1 = (int)r_ceil(chh) - 1;
  if (b1 > n - 1) b1 = n - 1;
  return true;
}

// The same with the bin's lower edge e given as T (an integer, so e + 1 is
// exact): the loops step e in T instead of converting every bin index (an
// int -> float conversion runs on the narrow conversion pipe).
template <typename T>
__device__ __forceinline__ T ov_edge(T cl, T chh, T e) {
  const T hi = e + T(1);
  return rn_sub(chh < hi ? chh : hi, cl > e ? cl : e);
}

template <typename T>
__device__ __forceinline__ T ov_axis(T cl, T chh, int b) {
  const T lo = (T)b, hi = (T)(b + 1);
  return rn_sub(chh < hi ? chh : hi, cl > lo ? cl : lo);
}

// ---- a2: std-cell scatter, two lanes per instance (macros skipped) ----
// Each (cell, bin) contribution c = ((omega*ovx)*ovy)*ovz is quantised to
// rint(c * 2^36) and added with a 64-bit integer atomic: the map is exact
// and independent of the order of the additions.  The two lanes of a cell
// take alternate bins of its x-run (a cell stretched to the bin width covers
// two): their atomics in one instruction hit adjacent words, which the L2
// serves as one sector request three times in four, about half the requests
// of one lane per cell looping over every bin.
template <typename T>
__global__ void __launch_bounds__(256) k_scatter_cells(int n, const V4<T> *__restrict__ pos,
                                                       const V4<T> *__restrict__ size,
                                                       const uint8_t *__restrict__ flags,
                                                       DensC<T> c, long long *__restrict__ q) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(t >> 1), h = (int)(t & 1);
  if (i >= n) return;
  const uint8_t f = flags[i];
  if (f & 1) return;  // macro: Theorem 1 path
  const V4<T> p = pos[i];
  const Box<T> b = inst_box(c, p.x, p.y, p.z, size[i], false, (f & 4) != 0);
  T cl[3], chh[3];
  int b0[3], b1[3];
  if (!clip_axis(b.lo[0], b.hi[0], c.fnx, c.nx, cl[0], chh[0], b0[0], b1[0])) return;
  if (!clip_axis(b.lo[1], b.hi[1], c.fny, c.ny, cl[1], chh[1], b0[1], b1[1])) return;
  if (!clip_axis(b.lo[2], b.hi[2], c.fnz, c.nz, cl[2], chh[2], b0[2], b1[2])) return;
  const T scale = (T)kFixedScale;
  const T ey0 = (T)b0[1], ex0 = (T)(b0[0] + h);
  T ez = (T)b0[2];
  for (int k = b0[2]; k <= b1[2]; ++k, ez += T(1)) {
    const T oz = ov_edge(cl[2], chh[2], ez);
    T ey = ey0;
    for (int j = b0[1]; j <= b1[1]; ++j, ey += T(1)) {
      const T oy = ov_edge(cl[1], chh[1], ey);
      long long *row = q + ((size_t)k * c.ny + j) * c.nx;
      T ex = ex0;
      for (int ii = b0[0] + h; ii <= b1[0]; ii += 2, ex += T(2)) {
        const T ox = ov_edge(cl[0], chh[0], ex);
        const T v = rn_mul(rn_mul(rn_mul(b.om, ox), oy), oz);
        atomic_add_i64(row + ii, r_rint(rn_mul(v, scale)));
      }
    }
  }
}

// Corner s (bit a set = upper face on axis a) of a macro's cuboid in bin
// units, clamped to [0, N]: base index and the two weights g(i - c).
template <typename T>
__device__ __forceinline__ void corner_axis(T c, T fN, int &base, T &w0, T &w1) {
  if (c < T(0)) c = T(0);
  if (c > fN) c = fN;
  base = (int)r_floor(c);
  const T f = rn_sub(c, (T)base);
  w0 = rn_sub(T(1), f);
  w1 = f;
}

// ---- a3: macro corner map (Theorem 1), one thread per (macro, corner) ----
// Entries e = ((omega*gx)*gy)*gz with sign -sx*sy*sz, quantised like cell
// contributions, accumulated into the corner map A (int64).
template <typename T>
__global__ void k_macro_corners(int nm, const int *__restrict__ macro_ids,
                                const V4<T> *__restrict__ pos, const V4<T> *__restrict__ size,
                                DensC<T> c, long long *__restrict__ A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nm * 8) return;
  const int i = macro_ids[t >> 3], s = t & 7;
  const V4<T> p = pos[i];
  const Box<T> b = inst_box(c, p.x, p.y, p.z, size[i], true);
  const T fN[3] = {c.fnx, c.fny, c.fnz};
  const int nn[3] = {c.nx, c.ny, c.nz};
  int base[3];
  T wg[3][2];
  int sign = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool up = (s >> a) & 1;
    corner_axis(up ? b.hi[a] : b.lo[a], fN[a], base[a], wg[a][0], wg[a][1]);
    sign *= up ? 1 : -1;
  }
  const T scale = (T)kFixedScale;
#pragma unroll
  for (int cz = 0; cz < 2; ++cz)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const int ii = base[0] + cx, j = base[1] + cy, k = base[2] + cz;
        if (ii >= nn[0] || j >= nn[1] || k >= nn[2]) continue;
        const T e = rn_mul(rn_mul(rn_mul(b.om, wg[0][cx]), wg[1][cy]), wg[2][cz]);
        const long long qe = r_rint(rn_mul(e, scale));
        if (qe) atomic_add_i64(A + ((size_t)k * c.ny + j) * c.nx + ii, sign > 0 ? qe : -qe);
      }
}

// ---- eq. def-prefix-sum-3d: inclusive scan along x (one warp per row) ----
// REV = true scans from the high end (suffix sums).  In/out may alias (with
// istride = 1); istride is the input's element stride (4 for one component
// of the interleaved field map).  The row goes in segments of 32 x kScanCh
// elements: all (coalesced) loads of a segment are issued before the first
// warp scan, so the segment waits for one load latency, not kScanCh.
constexpr int kScanCh = 16;
template <typename TI, typename TO, bool REV>
__global__ void __launch_bounds__(256) k_scan_rows(int rows, int nx, const TI *in, int istride, TO *out) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= rows) return;
  const size_t off = (size_t)row * nx;
  TO carry = 0;
  for (int base = 0; base < nx; base += 32 * kScanCh) {
    TO v[kScanCh];
#pragma unroll
    for (int c = 0; c < kScanCh; ++c) {
      const int t = base + c * 32 + lane;
      v[c] = t < nx ? (TO)in[(off + (REV ? nx - 1 - t : t)) * istride] : (TO)0;
    }
#pragma unroll
    for (int c = 0; c < kScanCh; ++c) {
      TO x = v[c];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const TO u = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += u;
      }
      x += carry;
      const int t = base + c * 32 + lane;
      if (t < nx) out[off + (REV ? nx - 1 - t : t)] = x;
      carry = __shfl_sync(0xffffffffu, x, 31);
    }
  }
}

// ---- inclusive scan along y, in place; block = 32 columns x W warps ----
// Each warp scans a chunk of rows per column (lane = column), chunk totals
// are combined through shared memory.  grid = (ceil(nx/32), nz).  Rows go in
// groups of kColCh held in registers with all their loads in flight; a chunk
// of at most kColCh rows is read once, a longer one twice (sum, then scan).
constexpr int kColCh = 16;
template <typename TA, bool REV>
__global__ void __launch_bounds__(1024) k_scan_cols(int nx, int ny, TA *a) {
  __shared__ TA tot[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int x = blockIdx.x * 32 + lane;
  const size_t slab = (size_t)blockIdx.y * ny * nx;
  const int chunk = (ny + nw - 1) / nw;
  const int r0 = warp * chunk, r1 = min(ny, r0 + chunk);
  auto at = [&](int r) { return slab + (size_t)(REV ? ny - 1 - r : r) * nx + x; };
  TA v[kColCh];
  TA s = 0;
  if (x < nx)
    for (int g = r0; g < r1; g += kColCh) {
#pragma unroll
      for (int c = 0; c < kColCh; ++c) v[c] = g + c < r1 ? a[at(g + c)] : TA(0);
#pragma unroll
      for (int c = 0; c < kColCh; ++c) s += v[c];
    }
  tot[warp][lane] = s;
  __syncthreads();
  TA run = 0;
  for (int w = 0; w < warp; ++w) run += tot[w][lane];
  if (x < nx)
    for (int g = r0; g < r1; g += kColCh) {
      if (chunk > kColCh) {  // the group is no longer in registers
#pragma unroll
        for (int c = 0; c < kColCh; ++c) v[c] = g + c < r1 ? a[at(g + c)] : TA(0);
      }
#pragma unroll
      for (int c = 0; c < kColCh; ++c)
        if (g + c < r1) {
          run += v[c];
          a[at(g + c)] = run;
        }
    }
}

// ---- density -> transform input: z prefix of the macro map + cell map ----
// rho[z][y][x] = (q[z][y][x] + sum_{z' <= z} A[z'][y][x]) * 2^-36.
// A may be NULL (no macros).  One thread per (y, x) column.
// part != NULL: also the per-warp rows (sum of max(rho - 1, 0), sum of rho)
// of the density overflow (target density 1).
template <typename T, typename Out>
__global__ void __launch_bounds__(256) k_densify(int nxy, int nz, const long long *__restrict__ q,
                                                 const long long *__restrict__ A, Out rho,
                                                 T *__restrict__ part = nullptr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  T v[2] = {0, 0};
  if (t < nxy) {
    long long acc = 0;
    for (int z0 = 0; z0 < nz; z0 += 4) {  // the loads of up to four layers issued together
      long long qv[4], av[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t id = (size_t)(z0 + u) * nxy + t;
        qv[u] = z0 + u < nz ? q[id] : 0;
        av[u] = A && z0 + u < nz ? A[id] : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (z0 + u >= nz) break;
        acc += av[u];
        const T r = r_ll2f(qv[u] + acc, T(0)) * (T)(1.0 / kFixedScale);
        rho.put((size_t)(z0 + u) * nxy + t, r);
        v[0] += r > T(1) ? r - T(1) : T(0);
        v[1] += r;
      }
    }
  }
  if (part) warp_sum_part<2>(v, part);
}

// ---- a10 (macros): Theorem 1's adjoint, one thread per (macro, corner) ----
// S holds the x- and y-suffix sums of E_x, E_y, E_z (double, 3 maps); the
// z-suffix is summed here.  out[m][3] accumulates sum_entries sign*e*S.
template <typename T>
__global__ void k_macro_gather(int nm, const int *__restrict__ macro_ids,
                               const V4<T> *__restrict__ pos, const V4<T> *__restrict__ size,
                               DensC<T> c, const double *__restrict__ S, size_t nb,
                               double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nm * 8) return;
  const int m = t >> 3, s = t & 7, i = macro_ids[m];
  const V4<T> p = pos[i];
  const Box<T> b = inst_box(c, p.x, p.y, p.z, size[i], true);
  const T fN[3] = {c.fnx, c.fny, c.fnz};
  int base[3];
  T wg[3][2];
  int sign = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool up = (s >> a) & 1;
    corner_axis(up ? b.hi[a] : b.lo[a], fN[a], base[a], wg[a][0], wg[a][1]);
    sign *= up ? 1 : -1;
  }
  double acc[3] = {0, 0, 0};
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const int ii = base[0] + cx, j = base[1] + cy, k = base[2] + cz;
        if (ii >= c.nx || j >= c.ny || k >= c.nz) continue;
        const double e = (double)(b.om * wg[0][cx] * wg[1][cy] * wg[2][cz]);
        if (e == 0.0) continue;
        for (int kk = k; kk < c.nz; ++kk) {
          const size_t id = ((size_t)kk * c.ny + j) * c.nx + ii;
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) acc[comp] += e * S[comp * nb + id];
        }
      }
#pragma unroll
  for (int comp = 0; comp < 3; ++comp)
    if (acc[comp] != 0.0) atomicAdd(out + m * 3 + comp, sign > 0 ? acc[comp] : -acc[comp]);
}

// ---- a10 (macros), bin-parallel direct form: grid (macros, slices) ----
// Block (m, s) sums omega * ovx*ovy*ovz * E over every S-th (z, y) row of
// macro m's clipped cuboid, threads striding over the rows' x bins.  Same
// result as the suffix-sum adjoint; cost proportional to the macros' bins.
template <typename T>
__global__ void __launch_bounds__(256) k_macro_gather_direct(const int *__restrict__ macro_ids,
                                                             const V4<T> *__restrict__ pos,
                                                             const V4<T> *__restrict__ size, DensC<T> c,
                                                             const V4<T> *__restrict__ e4, double *__restrict__ out) {
  const int m = blockIdx.x, i = macro_ids[m];
  const V4<T> p = pos[i];
  const Box<T> b = inst_box(c, p.x, p.y, p.z, size[i], true);
  T cl[3], chh[3];
  int b0[3], b1[3];
  T acc[3] = {0, 0, 0};
  if (clip_axis(b.lo[0], b.hi[0], c.fnx, c.nx, cl[0], chh[0], b0[0], b1[0]) &&
      clip_axis(b.lo[1], b.hi[1], c.fny, c.ny, cl[1], chh[1], b0[1], b1[1]) &&
      clip_axis(b.lo[2], b.hi[2], c.fnz, c.nz, cl[2], chh[2], b0[2], b1[2])) {
    const int nyr = b1[1] - b0[1] + 1, nzr = b1[2] - b0[2] + 1, nxr = b1[0] - b0[0] + 1;
    for (int r = blockIdx.y; r < nyr * nzr; r += gridDim.y) {
      const int j = b0[1] + r % nyr, k = b0[2] + r / nyr;
      const T oyz = ov_axis(cl[1], chh[1], j) * ov_axis(cl[2], chh[2], k);
      const size_t row = ((size_t)k * c.ny + j) * c.nx;
      for (int u = threadIdx.x; u < nxr; u += blockDim.x) {
        const int ii = b0[0] + u;
        const T v = ov_axis(cl[0], chh[0], ii) * oyz;
        const V4<T> e = e4[row + ii];
        acc[0] += v * e.x;
        acc[1] += v * e.y;
        acc[2] += v * e.z;
      }
    }
  }
  acc[0] *= b.om;
  acc[1] *= b.om;
  acc[2] *= b.om;
  block_sum_atomic<3>(acc, out + 3 * m);
}

// Final assembly constants.
// The density weights live in device memory (lam_dev), read once per block:
// a placement loop raises lambda every iteration, and a weight read at run
// time keeps captured CUDA graphs valid across the change.
template <typename T> struct FinalC {
  T alpha, volb;         // volb: bin volume (2D mode: bin area)
  const double *scal;    // device scalars (S_x, S_y, S_z for g)
  const T *lam_dev;      // device: lambda, then the 2D layer weights (lambda-, lambda+, lambda')
  T g;                   // filled per block from scal
  int mode2d;            // 2D mode: per-layer lambda, no z-gradient
};

__device__ __forceinline__ double g_scale_of(const double *scal) {
  const double sz = scal[S_SZ];
  return sz > 0.0 ? (scal[S_SX] + scal[S_SY]) / (2.0 * sz) : 0.0;
}
// g in the gather's precision: FP32 gathers narrow the three norms first
// (three conversions instead of an FP64 division on the narrow FP64 pipe).
template <typename T> __device__ __forceinline__ T g_scale_t(const double *scal);
template <> __device__ __forceinline__ double g_scale_t<double>(const double *scal) { return g_scale_of(scal); }
template <> __device__ __forceinline__ float g_scale_t<float>(const double *scal) {
  const float sz = (float)scal[S_SZ];
  return sz > 0.0f ? ((float)scal[S_SX] + (float)scal[S_SY]) / (2.0f * sz) : 0.0f;
}

// Final gradient of instance i from its WL accumulators a and its density
// force (dgx, dgy, dgz): x, y = WL + lambda force; z = g FD + alpha dp(z)/dz
// + lambda force (0 for z-fixed instances and in 2D mode).
template <typename T, typename TO>
__device__ __forceinline__ void final_out(int i, uint8_t f, T z, const V4<T> &a, T dgx, T dgy, T dgz, T g,
                                          const T *lam4, const FinalC<T> &fc, T zmid, TO *__restrict__ gx,
                                          TO *__restrict__ gy, TO *__restrict__ gz) {
  T lam = lam4[0];
  if (fc.mode2d) lam = lam4[1 + ((f & 4) ? 2 : (z > zmid ? 1 : 0))];
  T ozg = g * a.z + fc.alpha * a.w + lam * dgz;
  if ((f & 2) || fc.mode2d) ozg = T(0);
  gx[i] = (TO)(a.x + lam * dgx);
  gy[i] = (TO)(a.y + lam * dgy);
  gz[i] = (TO)ozg;
}

// Density force of macro slot m from the macro gather's FP64 sums.
template <typename T>
__device__ __forceinline__ void macro_force(const double *__restrict__ mgrad, int m, T volb, T &dgx, T &dgy,
                                            T &dgz) {
  dgx = (T)(-(double)volb * mgrad[m * 3 + 0]);
  dgy = (T)(-(double)volb * mgrad[m * 3 + 1]);
  dgz = (T)(-(double)volb * mgrad[m * 3 + 2]);
}

// ---- a10 + a9 + a11 per instance: cell field gather fused with the WL add ----
// g = acc_wl + lambda * (-omega sum_b vol(D cap b) E_b); gz uses the
// normalised FD gradient.  Macros take their density part from mgrad, or,
// with skip_macros, are left to k_final_macro_out (so that the cells need
// not wait for the macro gather).
template <typename T, typename TO>
__global__ void __launch_bounds__(256) k_final(int n, const V4<T> *__restrict__ pos,
                                               const V4<T> *__restrict__ size,
                                               const uint8_t *__restrict__ flags,
                                               const int *__restrict__ macro_slot, DensC<T> c,
                                               const V4<T> *__restrict__ e4,
                                               const double *__restrict__ mgrad,
                                               const V4<T> *__restrict__ acc, FinalC<T> fc,
                                               TO *__restrict__ gx, TO *__restrict__ gy,
                                               TO *__restrict__ gz, int skip_macros) {
  __shared__ T g_sh, lam_sh[4];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // the instance's loads issued before the block waits for g
  uint8_t f = 0;
  V4<T> p{}, sz4{};
  if (i < n) {
    f = flags[i];
    p = pos[i];
    sz4 = size[i];
  }
  if (threadIdx.x == 0) g_sh = g_scale_t<T>(fc.scal);  // once per block
  if (threadIdx.x < 4) lam_sh[threadIdx.x] = fc.lam_dev[threadIdx.x];
  __syncthreads();
  fc.g = g_sh;
  if (i >= n) return;
  T dgx = 0, dgy = 0, dgz = 0;
  if (f & 1) {
    if (skip_macros) return;
    macro_force(mgrad, macro_slot[i], fc.volb, dgx, dgy, dgz);
  } else {
    const Box<T> b = inst_box(c, p.x, p.y, p.z, sz4, false, (f & 4) != 0);
    T cl[3], chh[3];
    int b0[3], b1[3];
    if (clip_axis(b.lo[0], b.hi[0], c.fnx, c.nx, cl[0], chh[0], b0[0], b1[0]) &&
        clip_axis(b.lo[1], b.hi[1], c.fny, c.ny, cl[1], chh[1], b0[1], b1[1]) &&
        clip_axis(b.lo[2], b.hi[2], c.fnz, c.nz, cl[2], chh[2], b0[2], b1[2])) {
      T sx = 0, sy = 0, sz = 0;
      for (int k = b0[2]; k <= b1[2]; ++k) {
        const T oz = ov_axis(cl[2], chh[2], k);
        for (int j = b0[1]; j <= b1[1]; ++j) {
          const T oyz = ov_axis(cl[1], chh[1], j) * oz;
          const size_t row = ((size_t)k * c.ny + j) * c.nx;
          for (int ii = b0[0]; ii <= b1[0]; ++ii) {
            const T v = ov_axis(cl[0], chh[0], ii) * oyz;
            const V4<T> e = e4[row + ii];  // (E_x, E_y, E_z, -) of one bin: one vector load
            sx += v * e.x;
            sy += v * e.y;
            sz += v * e.z;
          }
        }
      }
      const T k = -b.om * fc.volb;
      dgx = k * sx;
      dgy = k * sy;
      dgz = k * sz;
    }
  }
  final_out(i, f, p.z, acc[i], dgx, dgy, dgz, fc.g, lam_sh, fc, c.zmid, gx, gy, gz);
}

// The macros' final gradients (the part k_final skips with skip_macros).
template <typename T, typename TO>
__global__ void k_final_macro_out(int nm, const int *__restrict__ macro_ids, const V4<T> *__restrict__ pos,
                                  const uint8_t *__restrict__ flags, const double *__restrict__ mgrad,
                                  const V4<T> *__restrict__ acc, FinalC<T> fc, T zmid, TO *__restrict__ gx,
                                  TO *__restrict__ gy, TO *__restrict__ gz) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nm) return;
  const int i = macro_ids[m];
  T lam4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) lam4[k] = fc.lam_dev[k];
  T dgx, dgy, dgz;
  macro_force(mgrad, m, fc.volb, dgx, dgy, dgz);
  final_out(i, flags[i], pos[i].z, acc[i], dgx, dgy, dgz, g_scale_t<T>(fc.scal), lam4, fc, zmid, gx, gy, gz);
}

// ======================= tile-sorted scatter and gather =======================
// Cells are sorted per evaluation by the 16x16-bin tile (all layers) that
// holds their centre: a counting sort (block histograms give each cell its
// rank in its tile, a scan gives the tile starts), then one 32-byte record
// per cell in tile order holding its stretched cuboid and omega (inst_box,
// computed once for both the scatter and the gather).  A work item is a
// chunk of at most kChunk cells of one tile; its block accumulates the
// chunk's charge in a shared-memory window (the tile plus a halo of R bins,
// all layers) and adds the window to the map with one global atomic per
// nonzero bin, and later gathers the field of the same window from a
// shared-memory copy.  A cell whose footprint leaves the window (only when
// it is wider than the halo allows) uses the global map directly.
constexpr int kTile = 16;
constexpr int kChunk = 1024;  // cells per work item: bounds the window's split sums (k_scatter_tiles)
constexpr int kTileMinInst = 100000;  // default: tiles from this many instances up
constexpr int kCountPerThread = 8;
// The tile counters lie one per 128-byte line: the count blocks' atomics on
// different tiles then never queue on the same line in the L2.
constexpr int kCountPad = 32;

struct TileC {
  int ntx, nty, R, WX, WY;  // tiles per axis, halo, window size (bins)
};

template <typename T>
__device__ __forceinline__ int tile_of(const DensC<T> &c, const TileC &tc, T X, T Y) {
  const int ix = (int)r_floor(rn_mul(rn_sub(X, c.x0), c.iwb)), iy = (int)r_floor(rn_mul(rn_sub(Y, c.y0), c.ihb));
  int tx = ix < 0 ? 0 : ix / kTile, ty = iy < 0 ? 0 : iy / kTile;
  tx = tx >= tc.ntx ? tc.ntx - 1 : tx;
  ty = ty >= tc.nty ? tc.nty - 1 : ty;
  return ty * tc.ntx + tx;
}

constexpr int kCountBlock = 512;  // threads of a tile-count block

// Exclusive scan of the tile counts into the tile starts and the work-item
// list (items of at most kChunk cells per tile), by one block of
// kCountBlock threads; the counts are read from the L2 (they were written by
// other blocks' atomics).
__device__ __forceinline__ void tile_scan_block(int ntiles, const int *__restrict__ count, int *__restrict__ start,
                                                int2 *__restrict__ items, int *__restrict__ nitems) {
  __shared__ int s_cells[kCountBlock / 32], s_items[kCountBlock / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, per = (ntiles + kCountBlock - 1) / kCountBlock;
  const int t0 = t * per, t1 = min(ntiles, t0 + per);
  int cells = 0, its = 0;
  for (int k = t0; k < t1; ++k) {
    const int ck = __ldcg(count + k * kCountPad);
    cells += ck;
    its += (ck + kChunk - 1) / kChunk;
  }
  int ic = cells, ii = its;  // inclusive warp scans
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int vc = __shfl_up_sync(0xffffffffu, ic, d), vi = __shfl_up_sync(0xffffffffu, ii, d);
    if (lane >= d) {
      ic += vc;
      ii += vi;
    }
  }
  if (lane == 31) {
    s_cells[warp] = ic;
    s_items[warp] = ii;
  }
  __syncthreads();
  if (warp == 0) {  // the warp totals, scanned by the first warp
    constexpr int NW = kCountBlock / 32;
    int wc = lane < NW ? s_cells[lane] : 0, wi = lane < NW ? s_items[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int vc = __shfl_up_sync(0xffffffffu, wc, d), vi = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) {
        wc += vc;
        wi += vi;
      }
    }
    if (lane < NW) {
      s_cells[lane] = wc;
      s_items[lane] = wi;
    }
  }
  __syncthreads();
  int cs = ic - cells + (warp ? s_cells[warp - 1] : 0), is = ii - its + (warp ? s_items[warp - 1] : 0);
  for (int k = t0; k < t1; ++k) {
    const int ck = __ldcg(count + k * kCountPad);
    start[k] = cs;
    const int nc = (ck + kChunk - 1) / kChunk;
    for (int j = 0; j < nc; ++j) items[is + j] = make_int2(k, j);
    cs += ck;
    is += nc;
  }
  if (t == kCountBlock - 1) {
    start[ntiles] = cs;
    *nitems = is;
  }
}

// Tile of every cell and its rank inside the tile (macros get -1).  Each
// block of kCountBlock threads takes kCountPerThread cells per thread (few,
// large blocks: the per-(block, tile) global atomics contend less), ranks them in a
// shared-memory histogram, then reserves its range of every tile it holds
// cells of with one global atomic per (block, tile).  The last block to
// finish (a ticket counter after a memory fence; no block waits for
// another) scans the counts into the tile starts and the work items.
// count holds the ntiles counters (one per kCountPad ints) and then the
// ticket counter; all are zero on entry.
template <typename T>
__global__ void __launch_bounds__(kCountBlock) k_tile_count(int n, const V4<T> *__restrict__ pos,
                                                     const uint8_t *__restrict__ flags, DensC<T> c, TileC tc,
                                                     int ntiles, int *__restrict__ count, int2 *__restrict__ key,
                                                     int *__restrict__ start, int2 *__restrict__ items,
                                                     int *__restrict__ nitems) {
  extern __shared__ int hist[];
  __shared__ int last;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  const int base = blockIdx.x * blockDim.x * kCountPerThread + threadIdx.x;
  int tl[kCountPerThread], rk[kCountPerThread];
#pragma unroll
  for (int u = 0; u < kCountPerThread; ++u) {
    const int i = base + u * blockDim.x;
    tl[u] = -1;
    rk[u] = 0;
    if (i < n && !(flags[i] & 1)) {
      const V4<T> p = pos[i];
      tl[u] = tile_of(c, tc, p.x, p.y);
      rk[u] = atomicAdd(hist + tl[u], 1);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const int v = hist[t];
    hist[t] = v ? atomicAdd(count + t * kCountPad, v) : 0;  // this block's first rank in tile t
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kCountPerThread; ++u) {
    const int i = base + u * blockDim.x;
    if (i < n) key[i] = tl[u] >= 0 ? make_int2(tl[u], hist[tl[u]] + rk[u]) : make_int2(-1, 0);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(count + ntiles * kCountPad, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  tile_scan_block(ntiles, count, start, items, nitems);
}

// One cell in tile order: its stretched cuboid in bin units (unclipped, as
// inst_box gives it), omega, and the instance index with its flags in the
// top byte.  32 bytes in FP32 (one sector), 64 in FP64.
template <typename T> struct TileRec;
template <> struct alignas(32) TileRec<float> {
  float lo[3], hi[3], om;
  int idx_flags;
};
template <> struct alignas(64) TileRec<double> {
  double lo[3], hi[3], om;
  int idx_flags, pad;
};

template <typename T>
__global__ void __launch_bounds__(256) k_tile_place(int n, const int2 *__restrict__ key, const int *__restrict__ start,
                                                    const V4<T> *__restrict__ pos, const V4<T> *__restrict__ size,
                                                    const uint8_t *__restrict__ flags, DensC<T> c,
                                                    TileRec<T> *__restrict__ rec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int2 k = key[i];
  if (k.x < 0) return;
  const uint8_t f = flags[i];
  const V4<T> p = pos[i];
  const Box<T> b = inst_box(c, p.x, p.y, p.z, size[i], false, (f & 4) != 0);
  TileRec<T> r;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r.lo[a] = b.lo[a];
    r.hi[a] = b.hi[a];
  }
  r.om = b.om;
  r.idx_flags = i | ((int)f << 24);
  rec[start[k.x] + k.y] = r;
}

// Window of a tile: bins [x0, x0 + WX) x [y0, y0 + WY) x all layers.
__device__ __forceinline__ void tile_window(const TileC &tc, int tile, int &x0, int &y0) {
  x0 = (tile % tc.ntx) * kTile - tc.R;
  y0 = (tile / tc.ntx) * kTile - tc.R;
}

// Per-axis overlaps of a clipped cuboid with its (at most 3) bins, for the
// separable fast paths: o[a] = overlap with bin b0 + a (0 past the last bin).
template <typename T>
__device__ __forceinline__ void axis_ov3(T cl, T chh, int b0, int nb, T (&o)[3]) {
  const T e0 = (T)b0;
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = a < nb ? ov_edge(cl, chh, e0 + T(a)) : T(0);
}

// ---- a2 through shared-memory windows ----
// Each quantised contribution v (0 <= v <= 2^36: a contribution is at most
// one bin of density) is split as v = hi * 2^22 + lo and the two parts are
// added to two 32-bit words of the bin with native shared-memory adds.  A
// chunk holds at most kChunk = 1024 cells and a cell adds to a bin at most
// once, so the low sums stay below 1024 * 2^22 = 2^32 and the high sums
// below 2^24: no 32-bit sum wraps, and hi_sum * 2^22 + lo_sum is the exact
// int64 total, added to the map once per bin.
// A cell covering at most 3 bins per axis (every std cell whose stretched
// footprint is under 2 bins wide: all of them on the usual grids) takes the
// separable path: 3 overlaps per axis, the products ((omega*ox)*oy) once per
// (x, y) pair, then *oz and the scale per bin -- the same IEEE operations in
// the same order as the per-bin form, so the same quantised values.
template <typename T>
__device__ __forceinline__ void win_add(unsigned *wlo, unsigned *whi, int w, long long v) {
  const unsigned long long u = (unsigned long long)v;
  atomicAdd(wlo + w, (unsigned)(u & 0x3fffffull));
  atomicAdd(whi + w, (unsigned)(u >> 22));
}

// rint(a) split as hi * 2^22 + lo (0 <= lo < 2^22) for 0 <= a <= 2^36, in
// 32-bit integer operations: for a >= 2^23, a = m 2^s with a 24-bit mantissa
// m and 0 <= s <= 13, so hi = m >> (22 - s) and lo = (m << s) mod 2^22; below
// 2^23 the FP32 add of 2^23 rounds a to an integer (ties to even) as in
// r_rint.  Equal to splitting r_rint(a).
__device__ __forceinline__ void rint_split(float a, unsigned &hi, unsigned &lo) {
  const unsigned u = __float_as_uint(a);
  const int s = (int)((u >> 23) & 0xffu) - 150;
  const unsigned m = (u & 0x7fffffu) | 0x800000u;
  const unsigned sm = (unsigned)(__float_as_int(__fadd_rn(a, 8388608.0f)) - 0x4B000000);
  const bool big = a >= 8388608.0f;
  const int sc = s < 0 ? 0 : (s > 22 ? 22 : s);
  hi = big ? (m >> (22 - sc)) : (a > 0.0f ? sm >> 22 : 0u);
  lo = big ? ((m << sc) & 0x3fffffu) : (a > 0.0f ? sm & 0x3fffffu : 0u);
}
__device__ __forceinline__ void rint_split(double a, unsigned &hi, unsigned &lo) {
  const unsigned long long u = (unsigned long long)r_rint(a);
  hi = (unsigned)(u >> 22);
  lo = (unsigned)(u & 0x3fffffull);
}

template <typename T>
__global__ void __launch_bounds__(256) k_scatter_tiles(const int2 *__restrict__ items, const int *__restrict__ nitems,
                                                       const int *__restrict__ start,
                                                       const TileRec<T> *__restrict__ rec, DensC<T> c, TileC tc,
                                                       long long *__restrict__ q) {
  extern __shared__ unsigned win32[];
  if ((int)blockIdx.x >= *nitems) return;
  const int2 it = items[blockIdx.x];
  int x0, y0;
  tile_window(tc, it.x, x0, y0);
  const int nwin = tc.WX * tc.WY * c.nz;
  unsigned *wlo = win32, *whi = win32 + nwin;
  for (int k = threadIdx.x; k < 2 * nwin; k += blockDim.x) win32[k] = 0u;
  __syncthreads();
  const int c0 = start[it.x] + it.y * kChunk, c1 = min(start[it.x + 1], c0 + kChunk);
  const T scale = (T)kFixedScale;
  for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x) {
    const TileRec<T> r = rec[s];
    T cl[3], chh[3];
    int b0[3], b1[3];
    if (!clip_axis(r.lo[0], r.hi[0], c.fnx, c.nx, cl[0], chh[0], b0[0], b1[0])) continue;
    if (!clip_axis(r.lo[1], r.hi[1], c.fny, c.ny, cl[1], chh[1], b0[1], b1[1])) continue;
    if (!clip_axis(r.lo[2], r.hi[2], c.fnz, c.nz, cl[2], chh[2], b0[2], b1[2])) continue;
    const bool inwin = b0[0] >= x0 && b1[0] < x0 + tc.WX && b0[1] >= y0 && b1[1] < y0 + tc.WY;
    const int nxb = b1[0] - b0[0] + 1, nyb = b1[1] - b0[1] + 1, nzb = b1[2] - b0[2] + 1;
    if (inwin && nxb <= 3 && nyb <= 3 && nzb <= 3) {
      T ox[3], oy[3], oz[3];
      axis_ov3(cl[0], chh[0], b0[0], nxb, ox);
      axis_ov3(cl[1], chh[1], b0[1], nyb, oy);
      axis_ov3(cl[2], chh[2], b0[2], nzb, oz);
      T t[3][3];  // ((omega * ox) * oy) per (y, x) pair
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T wo = rn_mul(r.om, ox[a]);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) t[bb][a] = rn_mul(wo, oy[bb]);
      }
      // the cuboid's z bins (3 in 3D mode nearly always, 1 in 2D mode: the
      // same count across a warp), each with 9 (y, x) slots without
      // branches: a slot past the cuboid's last bin has a zero overlap, so
      // its value is 0 and its (possibly out-of-window) add is skipped by
      // predicate
      const int wbase = (b0[2] * tc.WY + (b0[1] - y0)) * tc.WX + (b0[0] - x0);
      auto slots = [&](int cz) {
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          const int wrow = wbase + (cz * tc.WY + bb) * tc.WX;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            unsigned hi, lo;
            rint_split(rn_mul(rn_mul(t[bb][a], oz[cz]), scale), hi, lo);
            if (hi | lo) {
              atomicAdd(wlo + wrow + a, lo);
              atomicAdd(whi + wrow + a, hi);
            }
          }
        }
      };
      if (nzb == 3) {  // the usual 3D case, fully unrolled
#pragma unroll
        for (int cz = 0; cz < 3; ++cz) slots(cz);
      } else {
        for (int cz = 0; cz < nzb; ++cz) slots(cz);
      }
      continue;
    }
    T ez = (T)b0[2];
    for (int k = b0[2]; k <= b1[2]; ++k, ez += T(1)) {
      const T oz = ov_edge(cl[2], chh[2], ez);
      T ey = (T)b0[1];
      for (int j = b0[1]; j <= b1[1]; ++j, ey += T(1)) {
        const T oy = ov_edge(cl[1], chh[1], ey);
        const int wrow = (k * tc.WY + (j - y0)) * tc.WX - x0;
        T ex = (T)b0[0];
        for (int ii = b0[0]; ii <= b1[0]; ++ii, ex += T(1)) {
          const T ox = ov_edge(cl[0], chh[0], ex);
          const long long v = r_rint(rn_mul(rn_mul(rn_mul(rn_mul(r.om, ox), oy), oz), scale));
          if (inwin)
            win_add<T>(wlo, whi, wrow + ii, v);
          else
            atomic_add_i64(q + ((size_t)k * c.ny + j) * c.nx + ii, v);
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nwin; k += blockDim.x) {
    const long long v = (long long)(((unsigned long long)whi[k] << 22) + (unsigned long long)wlo[k]);
    if (!v) continue;
    const int xx = x0 + k % tc.WX, yy = y0 + (k / tc.WX) % tc.WY, zz = k / (tc.WX * tc.WY);
    if (xx >= 0 && xx < c.nx && yy >= 0 && yy < c.ny) atomic_add_i64(q + ((size_t)zz * c.ny + yy) * c.nx + xx, v);
  }
}

// ---- a10 (density part) for the cells of one work item, field from shared memory ----
// Writes each cell's lambda-weighted density force (lambda dgx, lambda dgy,
// lambda dgz, 0) into the interleaved buffer d4 (one 16- or 32-byte write
// per cell).  Nothing here depends on the wirelength path, so the gather
// runs while that path is still going; k_combine adds the two per instance
// once both are done.  Cells covering at most 3 bins per axis sum the window
// with 3 overlaps per axis computed once.
template <typename T>
__global__ void __launch_bounds__(256) k_final_tiles(const int2 *__restrict__ items, const int *__restrict__ nitems,
                                                     const int *__restrict__ start,
                                                     const TileRec<T> *__restrict__ rec, DensC<T> c, TileC tc,
                                                     const V4<T> *__restrict__ e4, FinalC<T> fc,
                                                     V4<T> *__restrict__ d4) {
  extern __shared__ __align__(16) unsigned char fwin_raw[];
  V4<T> *fw = reinterpret_cast<V4<T> *>(fwin_raw);
  __shared__ T lam_sh[4];
  if ((int)blockIdx.x >= *nitems) return;
  const int2 it = items[blockIdx.x];
  int x0, y0;
  tile_window(tc, it.x, x0, y0);
  const int nwin = tc.WX * tc.WY * c.nz;
  for (int k = threadIdx.x; k < nwin; k += blockDim.x) {
    const int xx = x0 + k % tc.WX, yy = y0 + (k / tc.WX) % tc.WY, zz = k / (tc.WX * tc.WY);
    V4<T> e{T(0), T(0), T(0), T(0)};
    if (xx >= 0 && xx < c.nx && yy >= 0 && yy < c.ny) e = e4[((size_t)zz * c.ny + yy) * c.nx + xx];
    fw[k] = e;
  }
  if (threadIdx.x < 4) lam_sh[threadIdx.x] = fc.lam_dev[threadIdx.x];
  __syncthreads();
  const int c0 = start[it.x] + it.y * kChunk, c1 = min(start[it.x + 1], c0 + kChunk);
  for (int s = c0 + threadIdx.x; s < c1; s += blockDim.x) {
    const TileRec<T> r = rec[s];
    const int i = r.idx_flags & 0xffffff;
    T cl[3], chh[3];
    int b0[3], b1[3];
    T sx = 0, sy = 0, sz = 0;
    if (clip_axis(r.lo[0], r.hi[0], c.fnx, c.nx, cl[0], chh[0], b0[0], b1[0]) &&
        clip_axis(r.lo[1], r.hi[1], c.fny, c.ny, cl[1], chh[1], b0[1], b1[1]) &&
        clip_axis(r.lo[2], r.hi[2], c.fnz, c.nz, cl[2], chh[2], b0[2], b1[2])) {
      const bool inwin = b0[0] >= x0 && b1[0] < x0 + tc.WX && b0[1] >= y0 && b1[1] < y0 + tc.WY;
      const int nxb = b1[0] - b0[0] + 1, nyb = b1[1] - b0[1] + 1, nzb = b1[2] - b0[2] + 1;
      if (inwin && nxb <= 3 && nyb <= 3 && nzb <= 3) {
        T ox[3], oy[3], oz[3];
        axis_ov3(cl[0], chh[0], b0[0], nxb, ox);
        axis_ov3(cl[1], chh[1], b0[1], nyb, oy);
        axis_ov3(cl[2], chh[2], b0[2], nzb, oz);
        // the cuboid's z bins (3 in 3D mode nearly always, 1 in 2D mode),
        // each with 9 (y, x) slots without branches: a slot past the
        // cuboid's last bin has weight 0 and reads the cuboid's first bin of
        // that row (always in the window)
        const int wbase = (b0[2] * tc.WY + (b0[1] - y0)) * tc.WX + (b0[0] - x0);
        auto slots = [&](int cz) {
#pragma unroll
          for (int bb = 0; bb < 3; ++bb) {
            const T oyz = oy[bb] * oz[cz];
            const int wrow = wbase + cz * tc.WY * tc.WX + (bb < nyb ? bb : 0) * tc.WX;
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
              const V4<T> e = fw[wrow + (aa < nxb ? aa : 0)];
              const T v = ox[aa] * oyz;  // 0 past the last bin
              sx += v * e.x;
              sy += v * e.y;
              sz += v * e.z;
            }
          }
        };
        if (nzb == 3) {  // the usual 3D case, fully unrolled
#pragma unroll
          for (int cz = 0; cz < 3; ++cz) slots(cz);
        } else {
          for (int cz = 0; cz < nzb; ++cz) slots(cz);
        }
      } else {
        for (int k = b0[2]; k <= b1[2]; ++k) {
          const T oz = ov_axis(cl[2], chh[2], k);
          for (int j = b0[1]; j <= b1[1]; ++j) {
            const T oyz = ov_axis(cl[1], chh[1], j) * oz;
            const int wrow = (k * tc.WY + (j - y0)) * tc.WX - x0;
            for (int ii = b0[0]; ii <= b1[0]; ++ii) {
              const T v = ov_axis(cl[0], chh[0], ii) * oyz;
              const V4<T> e = inwin ? fw[wrow + ii] : e4[((size_t)k * c.ny + j) * c.nx + ii];
              sx += v * e.x;
              sy += v * e.y;
              sz += v * e.z;
            }
          }
        }
      }
    }
    const T kk = -r.om * fc.volb;
    // 2D mode: the layer is the cuboid's z bin (0 bottom, 1 top, 2 HBT)
    const T lam = fc.mode2d ? lam_sh[1 + (int)r.lo[2]] : lam_sh[0];
    d4[i] = V4<T>{lam * (kk * sx), lam * (kk * sy), lam * (kk * sz), T(0)};
  }
}

// The macros' lambda-weighted density force into d4 (from mgrad).
template <typename T>
__global__ void k_final_macros(int nm, const int *__restrict__ macro_ids, const V4<T> *__restrict__ pos,
                               const double *__restrict__ mgrad, FinalC<T> fc, T zmid, V4<T> *__restrict__ d4) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nm) return;
  const int i = macro_ids[m];
  // 2D mode: the weight of the macro's die layer
  const T lam = fc.mode2d ? fc.lam_dev[pos[i].z > zmid ? 2 : 1] : fc.lam_dev[0];
  T dgx, dgy, dgz;
  macro_force(mgrad, m, fc.volb, dgx, dgy, dgz);
  d4[i] = V4<T>{lam * dgx, lam * dgy, lam * dgz, T(0)};
}

// a9 + a11 per instance, coalesced: x, y = WL + the density force from d4;
// z = g FD + alpha dp(z)/dz + the density force (0 for z-fixed instances and
// in 2D mode), written to the caller's three arrays.
template <typename T, typename TO>
__global__ void __launch_bounds__(256) k_combine(int n, const V4<T> *__restrict__ acc, const V4<T> *__restrict__ d4,
                                                 const uint8_t *__restrict__ flags, FinalC<T> fc,
                                                 TO *__restrict__ gx, TO *__restrict__ gy, TO *__restrict__ gz) {
  __shared__ T g_sh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // the instance's loads issued before the block waits for g
  V4<T> a{}, d{};
  uint8_t f = 0;
  if (i < n) {
    a = acc[i];
    d = d4[i];
    f = flags[i];
  }
  if (threadIdx.x == 0) g_sh = g_scale_t<T>(fc.scal);  // once per block
  __syncthreads();
  if (i >= n) return;
  const T g = g_sh;
  T ozg = g * a.z + fc.alpha * a.w + d.z;
  if ((f & 2) || fc.mode2d) ozg = T(0);
  gx[i] = (TO)(a.x + d.x);
  gy[i] = (TO)(a.y + d.y);
  gz[i] = (TO)ozg;
}

}  // namespace p3d
