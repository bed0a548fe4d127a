// Device side of the Nesterov placement loop (Sec. III-A: gradient-based 3D
// global placement with the 3D mixed-size preconditioner of eq.
// improved-precond, the movable range z in [d_z/4, 3 d_z/4], and the
// accelerated step with a Lipschitz step-length estimate).  The step
// length and the two squared norms it is estimated from stay on the device,
// so an iteration needs no host synchronisation.
#pragma once
#include "common.cuh"

namespace p3d {

// Loop state on the device: step (FP64 and FP32 copies), |v_new - v|^2,
// |g_new - g|^2 and max |g| (the bits of a non-negative double, for the
// first step).
struct NestState {
  double step, dv2, dg2;
  unsigned long long gmax_bits;
  float step_f;
};

template <typename T> struct NestBox {
  T lo[3], hi[3];  // projection box of the centres: x, y in the region, z in [d_z/4, 3 d_z/4]
};

template <typename T> __device__ __forceinline__ T nest_step(const NestState *s);
template <> __device__ __forceinline__ double nest_step<double>(const NestState *s) { return s->step; }
template <> __device__ __forceinline__ float nest_step<float>(const NestState *s) { return s->step_f; }

template <typename T> __device__ __forceinline__ T clampv(T v, T lo, T hi) { return v < lo ? lo : (v > hi ? hi : v); }

// u_new = P(v - step g); v_new = P(u_new + coef (u_new - u)); u <- u_new,
// v <- v_new, and v_new packed as the next evaluation's positions; per-warp
// rows of |v_new - v|^2.  Every load is issued before the first store (the
// arrays are distinct, so no store can alias a later load).
template <typename T>
__global__ void __launch_bounds__(256) k_nest_update(int n, T *__restrict__ ux, T *__restrict__ uy,
                                                     T *__restrict__ uz, T *__restrict__ vx, T *__restrict__ vy,
                                                     T *__restrict__ vz, const T *__restrict__ gx,
                                                     const T *__restrict__ gy, const T *__restrict__ gz,
                                                     const NestState *__restrict__ st, T coef, NestBox<T> b,
                                                     V4<T> *__restrict__ pos, T *__restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T dv[1] = {T(0)};
  if (i < n) {
    const T step = nest_step<T>(st);
    const T u[3] = {ux[i], uy[i], uz[i]}, v[3] = {vx[i], vy[i], vz[i]}, g[3] = {gx[i], gy[i], gz[i]};
    T un[3], vn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      un[a] = clampv(v[a] - step * g[a], b.lo[a], b.hi[a]);
      vn[a] = clampv(un[a] + coef * (un[a] - u[a]), b.lo[a], b.hi[a]);
      dv[0] += (vn[a] - v[a]) * (vn[a] - v[a]);
    }
    ux[i] = un[0];
    uy[i] = un[1];
    uz[i] = un[2];
    vx[i] = vn[0];
    vy[i] = vn[1];
    vz[i] = vn[2];
    pos[i] = V4<T>{vn[0], vn[1], vn[2], T(0)};
  }
  warp_sum_part<1>(dv, part);
}

// Eq. improved-precond: H_i = max(1, |E_i| + lambda q_i) for macros and
// max(1, lambda q_i) for every other instance, q_i its volume on its die
// (w h d_z/2).  g_new = G / H (z component 0 for z-fixed instances); per-warp
// rows of |g_new - g|^2 (and the maximum of |g_new| when gmax is set);
// g <- g_new.  All loads are issued up front, unconditionally.
template <typename T>
__global__ void __launch_bounds__(256) k_nest_precond(int n, const T *__restrict__ Gx, const T *__restrict__ Gy,
                                                      const T *__restrict__ Gz, T *__restrict__ gx,
                                                      T *__restrict__ gy, T *__restrict__ gz,
                                                      const V4<T> *__restrict__ pos, const V4<T> *__restrict__ size,
                                                      const uint8_t *__restrict__ flags,
                                                      const float *__restrict__ npins, const T *__restrict__ lam_dev,
                                                      T zmid, T half_dz, T *__restrict__ part,
                                                      unsigned long long *__restrict__ gmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T dg[1] = {T(0)};
  T amax = T(0);
  if (i < n) {
    const T lam = lam_dev[0];
    const V4<T> s = size[i];
    const T z = pos[i].z;
    const uint8_t f = flags[i];
    const T np = (T)npins[i];
    const T G[3] = {Gx[i], Gy[i], Gz[i]}, go[3] = {gx[i], gy[i], gz[i]};
    const T q = (z > zmid ? s.z * s.w : s.x * s.y) * half_dz;
    T H = lam * q + ((f & 1) ? np : T(0));
    H = H > T(1) ? H : T(1);
    T pre[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      pre[a] = (a == 2 && (f & 2)) ? T(0) : G[a] / H;
      const T d = pre[a] - go[a];
      dg[0] += d * d;
      const T ap = pre[a] < T(0) ? -pre[a] : pre[a];
      amax = ap > amax ? ap : amax;
    }
    gx[i] = pre[0];
    gy[i] = pre[1];
    gz[i] = pre[2];
  }
  warp_sum_part<1>(dg, part);
  if (gmax) {
#pragma unroll
    for (int m = 16; m; m >>= 1) {
      const T o = __shfl_xor_sync(0xffffffffu, amax, m);
      amax = o > amax ? o : amax;
    }
    // non-negative doubles order as their bit patterns (one widening per warp, at start-up only)
    if ((threadIdx.x & 31) == 0 && amax > T(0))
      atomicMax(gmax, (unsigned long long)__double_as_longlong((double)amax));
  }
}

// step = sqrt(dv2 / dg2) when both are positive (else unchanged); with
// init_step > 0 instead step = init_step / max |g|.  Then clears the sums
// for the next iteration's reducers.
__global__ void k_nest_step(NestState *st, double init_step) {
  if (init_step > 0.0) {
    const double gm = __longlong_as_double((long long)st->gmax_bits);
    st->step = init_step / (gm > 1e-30 ? gm : 1e-30);
  } else if (st->dv2 > 0.0 && st->dg2 > 0.0) {
    st->step = sqrt(st->dv2 / st->dg2);
  }
  st->step_f = (float)st->step;
  st->dv2 = 0.0;
  st->dg2 = 0.0;
  st->gmax_bits = 0ull;
}

}  // namespace p3d
