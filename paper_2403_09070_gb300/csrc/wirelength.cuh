// Bistratal weighted-average wirelength (eqs. wa-model-approx, wl-obj,
// wl-model), its gradient and the incremental FD depth gradient (eq.
// fda-grad, Sec. IV-B), per net with segmented reductions.
//
// Each net is reduced by a group of G lanes (G = 4, 8, 16, 32; PPL pins per
// lane held in registers), or by a whole block for high-fanout nets.  Per
// net: the 1st and 2nd extremes of the top and bottom pins in x and y, the
// WA sums of the top and bottom pins (each shifted by its own extreme, so no
// exponential can overflow and none of a sub-net's terms underflows because
// of the other die), and the depth span.  The whole-net WA sums are derived
// from the two sides' sums by one rescale per net.  The per-pin gradient is
// then pushed to the instance accumulators (gx, gy, fd, waz).
#pragma once
#include "common.cuh"

namespace p3d {

template <typename T> struct WlC {
  T zmid;      // d_z/2 (partition threshold, Sec. II-B)
  T inv_g;     // 1/gamma
  T inv_gz;    // 1/gamma_z
  T fd_scale;  // 4/d_z (eq. fda-grad)
  T inv_g2, inv_gz2;  // log2(e)/gamma, log2(e)/gamma_z: exp(v/gamma) = 2^(v inv_g2)
  int mode2d;  // multi-die 2D (eq. 2d-place): W = WA(top + HBT) + WA(bottom + HBT), no z terms
};

template <typename T> struct Pin {
  int inst;
  bool top;
  bool hbt;      // 2D mode: the net's HBT, a member of both partial nets
  T px, py, pz;  // pin on its current die
  T qx, qy;      // the same pin if its instance were on the other die
};

// HBTS: the netlist may hold HBT pins, stored as ~instance (2D mode only);
// false compiles the 3D kernels without the HBT cases.
template <typename T, bool HBTS = true>
__device__ __forceinline__ Pin<T> load_pin(int p, const int *__restrict__ pin_inst,
                                           const V4<T> *__restrict__ off,
                                           const V4<T> *__restrict__ pos, const WlC<T> &c) {
  Pin<T> q;
  const int raw = __ldg(pin_inst + p);
  q.hbt = HBTS && raw < 0;
  q.inst = q.hbt ? ~raw : raw;
  const V4<T> o = off[p];  // (bot x, bot y, top x, top y)
  const V4<T> s = pos[q.inst];
  q.top = !q.hbt && s.z > c.zmid;
  q.px = s.x + (q.top ? o.z : o.x);
  q.py = s.y + (q.top ? o.w : o.y);
  q.qx = s.x + (q.top ? o.x : o.z);
  q.qy = s.y + (q.top ? o.y : o.w);
  q.pz = s.z;
  return q;
}

// 1st/2nd extremes of one side on one axis (the 1st and 2nd outermost boxes).
template <typename T> struct Ext {
  T mx1, mx2, mn1, mn2;
  int amx, amn;
  __device__ __forceinline__ void init() {
    mx1 = mx2 = -big<T>();
    mn1 = mn2 = big<T>();
    amx = amn = -1;
  }
  __device__ __forceinline__ void add(T v, int k) {
    if (v > mx1) { mx2 = mx1; mx1 = v; amx = k; } else if (v > mx2) { mx2 = v; }
    if (v < mn1) { mn2 = mn1; mn1 = v; amn = k; } else if (v < mn2) { mn2 = v; }
  }
  __device__ __forceinline__ void merge(T bmx1, T bmx2, int bamx, T bmn1, T bmn2, int bamn) {
    if (bmx1 > mx1) { mx2 = mx1 > bmx2 ? mx1 : bmx2; mx1 = bmx1; amx = bamx; }
    else { mx2 = mx2 > bmx1 ? mx2 : bmx1; }
    if (bmn1 < mn1) { mn2 = mn1 < bmn2 ? mn1 : bmn2; mn1 = bmn1; amn = bamn; }
    else { mn2 = mn2 < bmn1 ? mn2 : bmn1; }
  }
  template <int W> __device__ __forceinline__ void shfl_reduce() {
#pragma unroll
    for (int m = W / 2; m; m >>= 1) {
      const T a = shfl_xor(mx1, m, W), b = shfl_xor(mx2, m, W);
      const T c = shfl_xor(mn1, m, W), d = shfl_xor(mn2, m, W);
      const int ia = shfl_xor(amx, m, W), ic = shfl_xor(amn, m, W);
      merge(a, b, ia, c, d, ic);
    }
  }
};

template <typename T> struct NetExt {
  Ext<T> e[2][2];  // [axis x/y][side bottom/top]
  int ntop, n;
  T zmx, zmn;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int s = 0; s < 2; ++s) e[a][s].init();
    ntop = n = 0;
    zmx = -big<T>();
    zmn = big<T>();
  }
  // slot: the pin's index within its net (identifies the extreme pins)
  __device__ __forceinline__ void add(const Pin<T> &p, int slot) {
    if (p.hbt) {  // both partial nets; not counted as a die's pin
      e[0][0].add(p.px, slot);
      e[1][0].add(p.py, slot);
      e[0][1].add(p.px, slot);
      e[1][1].add(p.py, slot);
      return;
    }
    if (p.top) {
      e[0][1].add(p.px, slot);
      e[1][1].add(p.py, slot);
    } else {
      e[0][0].add(p.px, slot);
      e[1][0].add(p.py, slot);
    }
    ntop += p.top ? 1 : 0;
    n += 1;
    zmx = p.pz > zmx ? p.pz : zmx;
    zmn = p.pz < zmn ? p.pz : zmn;
  }
  __device__ __forceinline__ void merge(const NetExt &b) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const Ext<T> &x = b.e[a][s];
        e[a][s].merge(x.mx1, x.mx2, x.amx, x.mn1, x.mn2, x.amn);
      }
    ntop += b.ntop;
    n += b.n;
    zmx = b.zmx > zmx ? b.zmx : zmx;
    zmn = b.zmn < zmn ? b.zmn : zmn;
  }
  template <int W> __device__ __forceinline__ void shfl_reduce() {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int s = 0; s < 2; ++s) e[a][s].template shfl_reduce<W>();
#pragma unroll
    for (int m = W / 2; m; m >>= 1) {
      ntop += shfl_xor(ntop, m, W);
      n += shfl_xor(n, m, W);
      const T a = shfl_xor(zmx, m, W), b = shfl_xor(zmn, m, W);
      zmx = a > zmx ? a : zmx;
      zmn = b < zmn ? b : zmn;
    }
  }
};

// WA sums per [axis][side]: sum e+, sum v e+, sum e-, sum v e-; and for z.
template <typename T> struct Sums {
  T v[2][2][4];
  T z[4];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[a][s][k] = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = 0;
  }
  __device__ __forceinline__ void merge(const Sums &b) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[a][s][k] += b.v[a][s][k];
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] += b.z[k];
  }
  template <int W> __device__ __forceinline__ void shfl_reduce() {
#pragma unroll
    for (int m = W / 2; m; m >>= 1) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int k = 0; k < 4; ++k) v[a][s][k] += shfl_xor(v[a][s][k], m, W);
#pragma unroll
      for (int k = 0; k < 4; ++k) z[k] += shfl_xor(z[k], m, W);
    }
  }
};

// Exponentials of one pin: x+, x-, y+, y-, z+, z- (shifted by its side's
// extremes in x, y and by the net's extremes in z).
template <typename T>
__device__ __forceinline__ void pin_exps(const Pin<T> &p, const NetExt<T> &X, const WlC<T> &c,
                                         T (&ex)[6], bool s) {
  const T xmx = s ? X.e[0][1].mx1 : X.e[0][0].mx1, xmn = s ? X.e[0][1].mn1 : X.e[0][0].mn1;
  const T ymx = s ? X.e[1][1].mx1 : X.e[1][0].mx1, ymn = s ? X.e[1][1].mn1 : X.e[1][0].mn1;
  ex[0] = r_exp2((p.px - xmx) * c.inv_g2);
  ex[1] = r_exp2((xmn - p.px) * c.inv_g2);
  ex[2] = r_exp2((p.py - ymx) * c.inv_g2);
  ex[3] = r_exp2((ymn - p.py) * c.inv_g2);
  ex[4] = r_exp2((p.pz - X.zmx) * c.inv_gz2);
  ex[5] = r_exp2((X.zmn - p.pz) * c.inv_gz2);
}

template <typename T>
__device__ __forceinline__ void sums_add(Sums<T> &S, const Pin<T> &p, const T (&ex)[6], bool top) {
  // masked fused multiply-adds into side `top` (no dynamic indexing, no
  // selects): the other side's weights are exactly 0
  const T mt = top ? T(1) : T(0), mb = T(1) - mt;
  const T xt = mt * p.px, xb = mb * p.px, yt = mt * p.py, yb = mb * p.py;
#pragma unroll
  for (int q = 0; q < 2; ++q) {  // q = 0: the + exponential, 1: the - one
    const T ea = ex[q], eb = ex[2 + q];
    // x and y in step: one packed FMA per (side, sum) pair
    fma2(mt, mt, ea, eb, S.v[0][1][2 * q], S.v[1][1][2 * q]);
    fma2(mb, mb, ea, eb, S.v[0][0][2 * q], S.v[1][0][2 * q]);
    fma2(xt, yt, ea, eb, S.v[0][1][2 * q + 1], S.v[1][1][2 * q + 1]);
    fma2(xb, yb, ea, eb, S.v[0][0][2 * q + 1], S.v[1][0][2 * q + 1]);
  }
  if (!p.hbt) {  // an HBT has no depth
    S.z[0] += ex[4];
    S.z[1] += p.pz * ex[4];
    S.z[2] += ex[5];
    S.z[3] += p.pz * ex[5];
  }
}

// Sums of one pin: its side's, or both partial nets' for an HBT (2D mode).
template <typename T>
__device__ __forceinline__ void pin_sums(Sums<T> &S, const Pin<T> &p, const NetExt<T> &X, const WlC<T> &c) {
  T ex[6];
  if (p.hbt) {
    pin_exps(p, X, c, ex, false);
    sums_add(S, p, ex, false);
    pin_exps(p, X, c, ex, true);
    sums_add(S, p, ex, true);
  } else {
    pin_exps(p, X, c, ex, p.top);
    sums_add(S, p, ex, p.top);
  }
}



// Per-net results of one axis.
template <typename T> struct AxisNet {
  bool all;          // active branch of max{p^_e, p^_e+ + p^_e-} (ties -> whole net)
  T f[2], h[2];      // rescale of each side's + and - sums to the whole net's shifts
  T iSP, iSM, M, m;  // reciprocals of the whole-net WA sums, the two weighted averages
  T Ms[2], ms[2];    // per side weighted averages
  T iSs[2], iSm[2];  // per side reciprocals of the + and - sums
  T what;            // W^_e on this axis
  T wexact;          // eq. wl-obj on this axis, exact extremes
};

template <typename T>
__device__ __forceinline__ AxisNet<T> axis_net(int a, const NetExt<T> &X, const Sums<T> &S,
                                               const WlC<T> &c) {
  AxisNet<T> r;
  const int nt = X.ntop, nb = X.n - X.ntop;
  const bool has[2] = {nb > 0, nt > 0};
  T mxA = -big<T>(), mnA = big<T>();
  T p[2] = {T(0), T(0)}, hp[2] = {T(0), T(0)};
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    r.Ms[s] = r.ms[s] = r.iSs[s] = r.iSm[s] = T(0);
    if (has[s]) {
      const Ext<T> &e = X.e[a][s];
      mxA = e.mx1 > mxA ? e.mx1 : mxA;
      mnA = e.mn1 < mnA ? e.mn1 : mnA;
      r.iSs[s] = r_rcp(S.v[a][s][0]);
      r.iSm[s] = r_rcp(S.v[a][s][2]);
      r.Ms[s] = S.v[a][s][1] * r.iSs[s];
      r.ms[s] = S.v[a][s][3] * r.iSm[s];
      p[s] = r.Ms[s] - r.ms[s];
      hp[s] = e.mx1 - e.mn1;
    }
  }
  T SP = 0, NP = 0, SM = 0, NM = 0;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    r.f[s] = r.h[s] = T(0);
    if (has[s]) {
      r.f[s] = r_exp2((X.e[a][s].mx1 - mxA) * c.inv_g2);
      r.h[s] = r_exp2((mnA - X.e[a][s].mn1) * c.inv_g2);
      SP += S.v[a][s][0] * r.f[s];
      NP += S.v[a][s][1] * r.f[s];
      SM += S.v[a][s][2] * r.h[s];
      NM += S.v[a][s][3] * r.h[s];
    }
  }
  r.iSP = r_rcp(SP);
  r.iSM = r_rcp(SM);
  r.M = NP * r.iSP;
  r.m = NM * r.iSM;
  const T pall = r.M - r.m;
  r.all = !c.mode2d && pall >= p[0] + p[1];  // 2D mode: always the two partial nets
  r.what = r.all ? pall : p[0] + p[1];
  const T hall = mxA - mnA;
  r.wexact = (!c.mode2d && hall > hp[0] + hp[1]) ? hall : hp[0] + hp[1];
  return r;
}

template <typename T> struct NetScal {
  AxisNet<T> ax[2];
  T zM, zm, izS1, izS2, pz;
  T wcur;  // exact W_Bi
};

template <typename T>
__device__ __forceinline__ NetScal<T> net_scalars(const NetExt<T> &X, const Sums<T> &S,
                                                  const WlC<T> &c) {
  NetScal<T> r;
  r.ax[0] = axis_net(0, X, S, c);
  r.ax[1] = axis_net(1, X, S, c);
  r.izS1 = r_rcp(S.z[0]);
  r.izS2 = r_rcp(S.z[2]);
  r.zM = S.z[1] * r.izS1;
  r.zm = S.z[3] * r.izS2;
  r.pz = r.zM - r.zm;
  r.wcur = r.ax[0].wexact + r.ax[1].wexact;
  return r;
}

// Gradient of one WA average pair at v given the exponentials (eq.
// wa-model-approx differentiated): (e+/S+)(1 + (v-M)/g) - (e-/S-)(1 - (v-m)/g),
// with the reciprocals 1/S+ and 1/S- precomputed per net.
template <typename T>
__device__ __forceinline__ T wa_grad(T v, T ep, T iSP, T M, T em, T iSM, T m, T inv_g) {
  return (ep * iSP) * (T(1) + (v - M) * inv_g) - (em * iSM) * (T(1) - (v - m) * inv_g);
}

// W_e on one axis (eq. wl-obj) after pin `slot` leaves side s (extremes in
// the s-side Ext, ns pins) for the other side (o-side Ext, no pins) at
// coordinate v; the 2nd extremes replace the 1st when the pin was extreme.
template <typename T>
__device__ __forceinline__ T moved_sel(bool s, const Ext<T> &e1, const Ext<T> &e0, int ns, int no, int slot,
                                       T v) {
  const T smx1 = s ? e1.mx1 : e0.mx1, smx2 = s ? e1.mx2 : e0.mx2;
  const T smn1 = s ? e1.mn1 : e0.mn1, smn2 = s ? e1.mn2 : e0.mn2;
  const int samx = s ? e1.amx : e0.amx, samn = s ? e1.amn : e0.amn;
  const T omx = s ? e0.mx1 : e1.mx1, omn = s ? e0.mn1 : e1.mn1;
  const bool keep = ns > 1;
  const T smax = slot == samx ? smx2 : smx1, smin = slot == samn ? smn2 : smn1;
  const T ps = keep ? smax - smin : T(0);
  const T omax = no ? (omx > v ? omx : v) : v;
  const T omin = no ? (omn < v ? omn : v) : v;
  const T po = omax - omin;
  const T amax = keep ? (smax > omax ? smax : omax) : omax;
  const T amin = keep ? (smin < omin ? smin : omin) : omin;
  const T hall = amax - amin;
  return hall > ps + po ? hall : ps + po;
}

// Per-pin outputs (gx, gy, fd, waz) -> instance accumulators.
template <typename T>
__device__ __forceinline__ void pin_outputs(const Pin<T> &p, int slot, const T (&ex)[6], const NetExt<T> &X,
                                            const Sums<T> &S, const NetScal<T> &N,
                                            const WlC<T> &c, V4<T> *__restrict__ acc) {
  const bool s = p.top;
  T g[2];
  const T v[2] = {p.px, p.py};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const AxisNet<T> &A = N.ax[a];
    if (A.all) {
      const T f = s ? A.f[1] : A.f[0], h = s ? A.h[1] : A.h[0];
      g[a] = wa_grad(v[a], ex[2 * a] * f, A.iSP, A.M, ex[2 * a + 1] * h, A.iSM, A.m, c.inv_g);
    } else {
      const T isp = s ? A.iSs[1] : A.iSs[0], ism = s ? A.iSm[1] : A.iSm[0];
      const T Ms = s ? A.Ms[1] : A.Ms[0], ms = s ? A.ms[1] : A.ms[0];
      g[a] = wa_grad(v[a], ex[2 * a], isp, Ms, ex[2 * a + 1], ism, ms, c.inv_g);
    }
  }
  const T gz = wa_grad(p.pz, ex[4], N.izS1, N.zM, ex[5], N.izS2, N.zm, c.inv_gz);
  const int ns = s ? X.ntop : X.n - X.ntop, no = X.n - ns;
  const T wm = moved_sel(s, X.e[0][1], X.e[0][0], ns, no, slot, p.qx) +
               moved_sel(s, X.e[1][1], X.e[1][0], ns, no, slot, p.qy);
  const T fd = c.fd_scale * (s ? (N.wcur - wm) : (wm - N.wcur));
  acc_add(acc + p.inst, g[0], g[1], fd, gz);
}

// 2D mode (eq. 2d-place): gradient of WA(top + HBT) + WA(bottom + HBT) at
// one pin (both partial nets for an HBT); no FD and no z terms.
template <typename T>
__device__ __forceinline__ void pin_outputs_2d(const Pin<T> &p, const NetExt<T> &X, const NetScal<T> &N,
                                               const WlC<T> &c, V4<T> *__restrict__ acc) {
  T g[2] = {T(0), T(0)};
  const T v[2] = {p.px, p.py};
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if (!(p.hbt || (side == 1) == p.top)) continue;
    T ex[6];
    pin_exps(p, X, c, ex, side == 1);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const AxisNet<T> &A = N.ax[a];
      g[a] += wa_grad(v[a], ex[2 * a], A.iSs[side], A.Ms[side], ex[2 * a + 1], A.iSm[side], A.ms[side], c.inv_g);
    }
  }
  acc_add(acc + p.inst, g[0], g[1], T(0), T(0));
}

// ---- 2-pin nets, one thread per net, closed form ----
// For two pins every branch of eq. wl-obj collapses to the two-point WA
// span L tanh(L / 2g) (same die: the sub-net is the net; different dies:
// both sub-nets are single pins), with derivative tanh(u) + u sech^2(u),
// u = L / 2g, written with e = exp(-L/g).  Moving pin a to the other die
// changes the exact W_Bi from |a - b| to |a' - b| per axis.
template <typename T>
__device__ __forceinline__ T wa_pair(T va, T vb, T inv_g, T &ga) {
  const T L = va > vb ? va - vb : vb - va;
  const T e = r_exp(-L * inv_g);
  const T i1e = r_rcp(T(1) + e);
  const T th = (T(1) - e) * i1e;
  const T der = th + T(2) * L * inv_g * e * i1e * i1e;
  ga = va >= vb ? der : -der;
  return L * th;
}

// The bucket's nets all have two pins, stored back to back from pin0: net t
// holds pins pin0 + 2t and pin0 + 2t + 1 (no net_start load on the chain).
// Each thread takes kPairNets nets, t and t + (number of threads), with
// every load of all its nets issued before the first use, so that the
// dependent chains (pin -> instance position) of its nets overlap.
constexpr int kPairNets = 2;
template <typename T>
__device__ __forceinline__ void pair_net(const Pin<T> &a, const Pin<T> &b, const WlC<T> &c, V4<T> *__restrict__ acc,
                                         T (&vals)[4]) {
  T gx, gy, gz;
  const T wx = wa_pair(a.px, b.px, c.inv_g, gx);
  const T wy = wa_pair(a.py, b.py, c.inv_g, gy);
  const T wz = wa_pair(a.pz, b.pz, c.inv_gz, gz);
  const T dx = a.px - b.px, dy = a.py - b.py;
  const T W = fabs(dx) + fabs(dy);
  const T Wa = fabs(a.qx - b.px) + fabs(a.qy - b.py);  // a on the other die
  const T Wb = fabs(a.px - b.qx) + fabs(a.py - b.qy);  // b on the other die
  const T fa = c.fd_scale * (a.top ? W - Wa : Wa - W);
  const T fb = c.fd_scale * (b.top ? W - Wb : Wb - W);
  acc_add(acc + a.inst, gx, gy, fa, gz);
  acc_add(acc + b.inst, -gx, -gy, fb, -gz);
  vals[0] += wx + wy;
  vals[1] += wz;
  vals[2] += W;
  vals[3] += a.top != b.top ? T(1) : T(0);
}

// Body for block bid of nblk (a batched launch passes the block's place in
// its instance's share of the grid).
template <typename T>
__device__ __forceinline__ void wl_pair_body(int pin0, int nnets, const int *__restrict__ pin_inst,
                                             const V4<T> *__restrict__ off, const V4<T> *__restrict__ pos, WlC<T> c,
                                             V4<T> *__restrict__ acc, T *__restrict__ part, int bid, int nblk);
template <typename T>
__global__ void __launch_bounds__(256) k_wl_pair(int pin0, int nnets,
                                                 const int *__restrict__ pin_inst, const V4<T> *__restrict__ off,
                                                 const V4<T> *__restrict__ pos, WlC<T> c, V4<T> *__restrict__ acc,
                                                 T *__restrict__ part) {
  wl_pair_body<T>(pin0, nnets, pin_inst, off, pos, c, acc, part, blockIdx.x, gridDim.x);
}
template <typename T>
__device__ __forceinline__ void wl_pair_body(int pin0, int nnets, const int *__restrict__ pin_inst,
                                             const V4<T> *__restrict__ off, const V4<T> *__restrict__ pos, WlC<T> c,
                                             V4<T> *__restrict__ acc, T *__restrict__ part, int bid, int nblk) {
  const int t0 = bid * blockDim.x + threadIdx.x, nth = nblk * blockDim.x;
  T vals[4] = {0, 0, 0, 0};
  int ia[kPairNets], ib[kPairNets];
  V4<T> oa[kPairNets], ob[kPairNets], sa[kPairNets], sb[kPairNets];
  bool ok[kPairNets];
#pragma unroll
  for (int u = 0; u < kPairNets; ++u) {
    const int t = t0 + u * nth;
    ok[u] = t < nnets;
    const int s0 = pin0 + 2 * (ok[u] ? t : 0);
    ia[u] = __ldg(pin_inst + s0);
    ib[u] = __ldg(pin_inst + s0 + 1);
    oa[u] = off[s0];
    ob[u] = off[s0 + 1];
  }
#pragma unroll
  for (int u = 0; u < kPairNets; ++u) {
    sa[u] = pos[ia[u]];
    sb[u] = pos[ib[u]];
  }
#pragma unroll
  for (int u = 0; u < kPairNets; ++u) {
    if (!ok[u]) continue;
    Pin<T> pa, pb;
    const V4<T> *o[2] = {&oa[u], &ob[u]};
    const V4<T> *q[2] = {&sa[u], &sb[u]};
    Pin<T> *pp[2] = {&pa, &pb};
    const int ii[2] = {ia[u], ib[u]};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      Pin<T> &P = *pp[k];
      const V4<T> &oo = *o[k], &ss = *q[k];
      P.hbt = false;
      P.inst = ii[k];
      P.top = ss.z > c.zmid;
      P.px = ss.x + (P.top ? oo.z : oo.x);
      P.py = ss.y + (P.top ? oo.w : oo.y);
      P.qx = ss.x + (P.top ? oo.x : oo.z);
      P.qy = ss.y + (P.top ? oo.y : oo.w);
      P.pz = ss.z;
    }
    pair_net(pa, pb, c, acc, vals);
  }
  warp_sum_part<4>(vals, part, bid);  // (W^_Bi, p^(z), W_Bi, crossing) rows
}

// ---- nets of degree <= G*PPL, one group of G lanes per net ----
// Block size of the group kernel: 128 threads (FP32), 64 (FP64).
template <typename T> __host__ __device__ constexpr int wl_block() { return sizeof(T) == 8 ? 64 : 128; }

// Per-net values staged in shared memory, one column per group (structure of
// arrays: lanes of different groups read consecutive words, lanes of one
// group read the same word).  Staging them keeps the per-pin loop's register
// footprint to the pins themselves, which doubles the resident warps.
enum : int {
  F_EXT = 0,    // [(a*2+s)*4 + {0: max1, 1: max2, 2: min1, 3: min2}], a = axis, s = side (0 bottom, 1 top)
  F_Z = 16,     // +0 max z, +1 min z (the z shifts)
  F_COEF = 18,  // [(a*2+s)*4 + {A, B, C, D}]: dW/dv = e+ A (1 + (v-B)/g) - e- C (1 - (v-D)/g)
  F_ZC = 34,    // +0 1/S+z, +1 M_z, +2 1/S-z, +3 m_z
  F_WCUR = 38,  // exact W_Bi of the net (eq. wl-obj)
  F_COUNT = 39
};
enum : int { I_ARG = 0, I_NTOP = 8, I_N = 9, I_COUNT = 10 };  // I_ARG + (a*2+s)*2 + {argmax, argmin}

template <typename T, int GR> struct WlShared {
  T f[F_COUNT][GR];
  int i[I_COUNT][GR];
};

template <typename T, int GR>
__device__ __forceinline__ void stage_ext(WlShared<T, GR> &sh, int grp, const NetExt<T> &X) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const Ext<T> &e = X.e[a][s];
      const int b = (a * 2 + s) * 4;
      sh.f[F_EXT + b + 0][grp] = e.mx1;
      sh.f[F_EXT + b + 1][grp] = e.mx2;
      sh.f[F_EXT + b + 2][grp] = e.mn1;
      sh.f[F_EXT + b + 3][grp] = e.mn2;
      sh.i[I_ARG + (a * 2 + s) * 2 + 0][grp] = e.amx;
      sh.i[I_ARG + (a * 2 + s) * 2 + 1][grp] = e.amn;
    }
  sh.f[F_Z + 0][grp] = X.zmx;
  sh.f[F_Z + 1][grp] = X.zmn;
  sh.i[I_NTOP][grp] = X.ntop;
  sh.i[I_N][grp] = X.n;
}

// Exponentials of one pin with the shifts read from the staged extremes.
template <typename T, int GR>
__device__ __forceinline__ void pin_exps_sh(const Pin<T> &p, const WlShared<T, GR> &sh, int grp, const WlC<T> &c,
                                            T (&ex)[6], bool side) {
  const int s = side ? 1 : 0;
  const T xmx = sh.f[F_EXT + (0 + s) * 4 + 0][grp], xmn = sh.f[F_EXT + (0 + s) * 4 + 2][grp];
  const T ymx = sh.f[F_EXT + (2 + s) * 4 + 0][grp], ymn = sh.f[F_EXT + (2 + s) * 4 + 2][grp];
  T ax, ay, bx, by;  // x and y arguments in step (packed pairs in FP32)
  submul2(p.px, p.py, xmx, ymx, c.inv_g2, c.inv_g2, ax, ay);
  submul2(xmn, ymn, p.px, p.py, c.inv_g2, c.inv_g2, bx, by);
  ex[0] = r_exp2(ax);
  ex[1] = r_exp2(bx);
  ex[2] = r_exp2(ay);
  ex[3] = r_exp2(by);
  ex[4] = r_exp2((p.pz - sh.f[F_Z + 0][grp]) * c.inv_gz2);
  ex[5] = r_exp2((sh.f[F_Z + 1][grp] - p.pz) * c.inv_gz2);
}

// W_e on one axis after the pin (side s, index slot) moves to the other die
// at coordinate v: moved_sel with the extremes read from shared memory.
template <typename T, int GR>
__device__ __forceinline__ T moved_sh(const WlShared<T, GR> &sh, int grp, int a, int s, int ns, int no, int slot,
                                      T v) {
  const int bs = F_EXT + (a * 2 + s) * 4, bo = F_EXT + (a * 2 + (1 - s)) * 4;
  const T smx1 = sh.f[bs + 0][grp], smx2 = sh.f[bs + 1][grp], smn1 = sh.f[bs + 2][grp], smn2 = sh.f[bs + 3][grp];
  const int samx = sh.i[I_ARG + (a * 2 + s) * 2 + 0][grp], samn = sh.i[I_ARG + (a * 2 + s) * 2 + 1][grp];
  const T omx = sh.f[bo + 0][grp], omn = sh.f[bo + 2][grp];
  const bool keep = ns > 1;
  const T smax = slot == samx ? smx2 : smx1, smin = slot == samn ? smn2 : smn1;
  const T ps = keep ? smax - smin : T(0);
  const T omax = no ? (omx > v ? omx : v) : v;
  const T omin = no ? (omn < v ? omn : v) : v;
  const T po = omax - omin;
  const T amax = keep ? (smax > omax ? smax : omax) : omax;
  const T amin = keep ? (smin < omin ? smin : omin) : omin;
  const T hall = amax - amin;
  return hall > ps + po ? hall : ps + po;
}

// ---- the three per-pin phases and the per-net step, shared by the group
// forms (pins held in registers) and the streamed forms (pins read again in
// every phase) ----

// Phase 2 of one pin: its exponentials (shifts from the staged extremes)
// into the WA sums; in 2D mode an HBT adds to both partial nets.
template <typename T, int GR, bool M2D>
__device__ __forceinline__ void pin_phase_sums(Sums<T> &S, const Pin<T> &q, const WlShared<T, GR> &sh, int grp,
                                               const WlC<T> &c) {
  T ex[6];
  if (M2D && q.hbt) {  // 2D mode: a member of both partial nets
    pin_exps_sh(q, sh, grp, c, ex, false);
    sums_add(S, q, ex, false);
    pin_exps_sh(q, sh, grp, c, ex, true);
    sums_add(S, q, ex, true);
  } else {
    pin_exps_sh(q, sh, grp, c, ex, q.top);
    sums_add(S, q, ex, q.top);
  }
}

// The net step (one lane per net, after the sums are reduced): the eq.
// wl-obj branch and the WA averages, staged as per-side gradient
// coefficients, and the net's contributions to the scalar rows.
template <typename T, int GR, bool M2D>
__device__ __forceinline__ void net_phase(WlShared<T, GR> &sh, int grp, const Sums<T> &S, const WlC<T> &c,
                                          T (&vals)[4]) {
  NetExt<T> X;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      Ext<T> &e = X.e[a][q];
      const int b = F_EXT + (a * 2 + q) * 4;
      e.mx1 = sh.f[b + 0][grp];
      e.mx2 = sh.f[b + 1][grp];
      e.mn1 = sh.f[b + 2][grp];
      e.mn2 = sh.f[b + 3][grp];
      e.amx = e.amn = 0;
    }
  X.zmx = sh.f[F_Z + 0][grp];
  X.zmn = sh.f[F_Z + 1][grp];
  X.ntop = sh.i[I_NTOP][grp];
  X.n = sh.i[I_N][grp];
  const NetScal<T> N = net_scalars(X, S, c);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const AxisNet<T> &A = N.ax[a];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int b = F_COEF + (a * 2 + q) * 4;
      sh.f[b + 0][grp] = A.all ? A.f[q] * A.iSP : A.iSs[q];
      sh.f[b + 1][grp] = A.all ? A.M : A.Ms[q];
      sh.f[b + 2][grp] = A.all ? A.h[q] * A.iSM : A.iSm[q];
      sh.f[b + 3][grp] = A.all ? A.m : A.ms[q];
    }
  }
  sh.f[F_ZC + 0][grp] = N.izS1;
  sh.f[F_ZC + 1][grp] = N.zM;
  sh.f[F_ZC + 2][grp] = N.izS2;
  sh.f[F_ZC + 3][grp] = N.zm;
  sh.f[F_WCUR][grp] = N.wcur;
  vals[0] = N.ax[0].what + N.ax[1].what;
  vals[1] = M2D ? T(0) : N.pz;
  vals[2] = N.wcur;
  vals[3] = (X.ntop > 0 && X.ntop < X.n) ? T(1) : T(0);
}

// Phase 3 of one pin, 2D mode: split-branch coefficients of each partial
// net, no FD, no z.
template <typename T, int GR>
__device__ __forceinline__ void pin_phase_out_2d(const Pin<T> &p, const WlShared<T, GR> &sh, int grp,
                                                 const WlC<T> &c, V4<T> *__restrict__ acc) {
  T g[2] = {T(0), T(0)};
  const T v[2] = {p.px, p.py};
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if (!(p.hbt || (side == 1) == p.top)) continue;
    T ex[6];
    pin_exps_sh(p, sh, grp, c, ex, side == 1);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int b = F_COEF + (a * 2 + side) * 4;
      const T A = sh.f[b + 0][grp], B = sh.f[b + 1][grp], C = sh.f[b + 2][grp], D = sh.f[b + 3][grp];
      g[a] += (ex[2 * a] * A) * (T(1) + (v[a] - B) * c.inv_g) - (ex[2 * a + 1] * C) * (T(1) - (v[a] - D) * c.inv_g);
    }
  }
  acc_add(acc + p.inst, g[0], g[1], T(0), T(0));
}

// Phase 3 of one pin, 3D mode: WA gradient on x, y and z, and the
// incremental FD step (eq. fda-grad) from the staged extremes.
template <typename T, int GR>
__device__ __forceinline__ void pin_phase_out(const Pin<T> &p, int slot, const WlShared<T, GR> &sh, int grp,
                                              const WlC<T> &c, int ntop, int n, T wcur, V4<T> *__restrict__ acc) {
  T ex[6];  // recomputed: keeping them live across the reductions costs registers
  pin_exps_sh(p, sh, grp, c, ex, p.top);
  const int s = p.top ? 1 : 0;
  T g[2];
  const T v[2] = {p.px, p.py};
  T cA[2], cB[2], cC[2], cD[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int b = F_COEF + (a * 2 + s) * 4;
    cA[a] = sh.f[b + 0][grp];
    cB[a] = sh.f[b + 1][grp];
    cC[a] = sh.f[b + 2][grp];
    cD[a] = sh.f[b + 3][grp];
  }
  const T ep[2] = {ex[0], ex[2]}, em[2] = {ex[1], ex[3]};
  wa_grad2(ep, em, v, cA, cB, cC, cD, c.inv_g, g);  // both axes in step
  const T gz = wa_grad(p.pz, ex[4], sh.f[F_ZC + 0][grp], sh.f[F_ZC + 1][grp], ex[5], sh.f[F_ZC + 2][grp],
                       sh.f[F_ZC + 3][grp], c.inv_gz);
  const int ns = s ? ntop : n - ntop, no = n - ns;
  const T wm = moved_sh(sh, grp, 0, s, ns, no, slot, p.qx) + moved_sh(sh, grp, 1, s, ns, no, slot, p.qy);
  const T fd = c.fd_scale * (s ? (wcur - wm) : (wm - wcur));
  acc_add(acc + p.inst, g[0], g[1], fd, gz);
}

// M2D: multi-die 2D mode (compile-time, so the 3D kernels carry none of the
// HBT and partial-net-only cases).
// Body for block bid (a batched launch passes the block's place in its
// instance's share of the grid).
template <typename T, int G, int PPL, bool M2D>
__device__ __forceinline__ void wl_group_body(int net0, int nnets, const int *__restrict__ net_start,
                                              const int *__restrict__ pin_inst, const V4<T> *__restrict__ off,
                                              const V4<T> *__restrict__ pos, WlC<T> c0, V4<T> *__restrict__ acc,
                                              T *__restrict__ part, int bid);
template <typename T, int G, int PPL, bool M2D>
__global__ void __launch_bounds__(wl_block<T>()) k_wl_group(int net0, int nnets, const int *__restrict__ net_start,
                                                            const int *__restrict__ pin_inst,
                                                            const V4<T> *__restrict__ off,
                                                            const V4<T> *__restrict__ pos, WlC<T> c0,
                                                            V4<T> *__restrict__ acc, T *__restrict__ part) {
  wl_group_body<T, G, PPL, M2D>(net0, nnets, net_start, pin_inst, off, pos, c0, acc, part, blockIdx.x);
}
template <typename T, int G, int PPL, bool M2D>
__device__ __forceinline__ void wl_group_body(int net0, int nnets, const int *__restrict__ net_start,
                                              const int *__restrict__ pin_inst, const V4<T> *__restrict__ off,
                                              const V4<T> *__restrict__ pos, WlC<T> c0, V4<T> *__restrict__ acc,
                                              T *__restrict__ part, int bid) {
  WlC<T> c = c0;
  c.mode2d = M2D ? 1 : 0;
  constexpr int GR = wl_block<T>() / G;  // groups (nets) per block
  __shared__ WlShared<T, GR> sh;
  const int lane = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G;
  const int gid = bid * GR + grp;
  const bool valid = gid < nnets;
  int s0 = 0, d = 0;
  if (valid) {
    s0 = __ldg(net_start + net0 + gid);
    d = __ldg(net_start + net0 + gid + 1) - s0;
  }
  Pin<T> pin[PPL];
  bool has[PPL];
  {
    NetExt<T> X;
    X.init();
#pragma unroll
    for (int r = 0; r < PPL; ++r) {
      const int k = lane + r * G;
      has[r] = k < d;
      if (has[r]) {
        pin[r] = load_pin<T, M2D>(s0 + k, pin_inst, off, pos, c);
        X.add(pin[r], k);
      }
    }
    X.template shfl_reduce<G>();
    if (lane == 0) stage_ext(sh, grp, X);
  }
  __syncwarp();
  T vals[4] = {0, 0, 0, 0};
  {
    Sums<T> S;
    S.init();
#pragma unroll
    for (int r = 0; r < PPL; ++r)
      if (has[r]) pin_phase_sums<T, GR, M2D>(S, pin[r], sh, grp, c);
    S.template shfl_reduce<G>();
    if (d >= 2 && lane == 0) net_phase<T, GR, M2D>(sh, grp, S, c, vals);
  }
  __syncwarp();
  if (M2D && d >= 2) {
#pragma unroll
    for (int r = 0; r < PPL; ++r)
      if (has[r]) pin_phase_out_2d(pin[r], sh, grp, c, acc);
  } else if (!M2D && d >= 2) {
    const int ntop = sh.i[I_NTOP][grp], n = sh.i[I_N][grp];
    const T wcur = sh.f[F_WCUR][grp];
#pragma unroll
    for (int r = 0; r < PPL; ++r)
      if (has[r]) pin_phase_out(pin[r], lane + r * G, sh, grp, c, ntop, n, wcur, acc);
  }
  warp_sum_part<4>(vals, part, bid);  // (W^_Bi, p^(z), W_Bi, crossing) rows
}

// ---- high-fanout nets, split across blocks ----
// A net above 128 pins is cut into chunks of at most kWlChunk pins, one
// 256-thread block per chunk, in three passes (three launches): the 1st/2nd
// extremes, the WA sums, the per-pin outputs.  Each block of a pass writes
// its chunk's partial result; the net's last block to finish the pass (an
// atomic counter per net after a memory fence: no block ever waits for
// another) merges the net's partials in chunk order, so the merged values do
// not depend on the blocks' timing, and resets the counter for the next pass.
constexpr int kWlChunk = 1024;

struct WlBig {
  const int4 *chunk;  // [chunks]: (net in the reordered CSR, first pin, pin count, big-net slot)
  const int2 *net;    // [big nets]: (first chunk, chunk count)
  int *done;          // [big nets]: chunks finished in the current pass (0 between passes)
};

// A POD struct read through the L2 (another block's partial result).
template <typename S> __device__ __forceinline__ S ld_l2(const S *p) {
  static_assert(sizeof(S) % 4 == 0, "word-sized struct");
  S r;
  const unsigned *src = reinterpret_cast<const unsigned *>(p);
  unsigned *dst = reinterpret_cast<unsigned *>(&r);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(S) / 4); ++k) dst[k] = __ldcg(src + k);
  return r;
}

// Counts this block's chunk as done; true in the net's last block (which
// then sees every other chunk's partial result).
__device__ __forceinline__ bool big_last_block(const WlBig &bg, int slot, int nch) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(bg.done + slot, 1) == nch - 1;
    if (last) {
      __threadfence();
      bg.done[slot] = 0;
    }
  }
  __syncthreads();
  return last != 0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_wl_big_ext(WlBig bg, const int *__restrict__ net_start,
                                                    const int *__restrict__ pin_inst, const V4<T> *__restrict__ off,
                                                    const V4<T> *__restrict__ pos, WlC<T> c,
                                                    NetExt<T> *__restrict__ ext_part, NetExt<T> *__restrict__ ext) {
  __shared__ NetExt<T> sx[8];
  const int4 ch = bg.chunk[blockIdx.x];
  const int s0 = net_start[ch.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  NetExt<T> X;
  X.init();
  for (int k = tid; k < ch.z; k += blockDim.x) X.add(load_pin(ch.y + k, pin_inst, off, pos, c), ch.y + k - s0);
  X.template shfl_reduce<32>();
  if (lane == 0) sx[warp] = X;
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) sx[0].merge(sx[w]);
    ext_part[blockIdx.x] = sx[0];
  }
  const int2 nt = bg.net[ch.w];
  if (big_last_block(bg, ch.w, nt.y) && tid == 0) {
    NetExt<T> m = ld_l2(ext_part + nt.x);
    for (int k = 1; k < nt.y; ++k) m.merge(ld_l2(ext_part + nt.x + k));
    ext[ch.w] = m;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_wl_big_sums(WlBig bg, const int *__restrict__ pin_inst,
                                                     const V4<T> *__restrict__ off, const V4<T> *__restrict__ pos,
                                                     WlC<T> c, const NetExt<T> *__restrict__ ext,
                                                     Sums<T> *__restrict__ sum_part, Sums<T> *__restrict__ sums,
                                                     double *__restrict__ scal) {
  __shared__ Sums<T> ss[8];
  const int4 ch = bg.chunk[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const NetExt<T> X = ext[ch.w];
  Sums<T> S;
  S.init();
  for (int k = tid; k < ch.z; k += blockDim.x) pin_sums(S, load_pin(ch.y + k, pin_inst, off, pos, c), X, c);
  S.template shfl_reduce<32>();
  if (lane == 0) ss[warp] = S;
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) ss[0].merge(ss[w]);
    sum_part[blockIdx.x] = ss[0];
  }
  const int2 nt = bg.net[ch.w];
  if (big_last_block(bg, ch.w, nt.y) && tid == 0) {
    Sums<T> m = ld_l2(sum_part + nt.x);
    for (int k = 1; k < nt.y; ++k) m.merge(ld_l2(sum_part + nt.x + k));
    sums[ch.w] = m;
    const NetScal<T> N = net_scalars(X, m, c);
    atomicAdd(scal + S_WL_BI, (double)N.ax[0].what + (double)N.ax[1].what);
    if (!c.mode2d) atomicAdd(scal + S_WL_Z, (double)N.pz);
    atomicAdd(scal + S_HPWL, (double)N.wcur);
    if (X.ntop > 0 && X.ntop < X.n) atomicAdd(scal + S_NCROSS, 1.0);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_wl_big_out(WlBig bg, const int *__restrict__ net_start,
                                                    const int *__restrict__ pin_inst, const V4<T> *__restrict__ off,
                                                    const V4<T> *__restrict__ pos, WlC<T> c,
                                                    const NetExt<T> *__restrict__ ext,
                                                    const Sums<T> *__restrict__ sums, V4<T> *__restrict__ acc) {
  const int4 ch = bg.chunk[blockIdx.x];
  const int s0 = net_start[ch.x];
  const NetExt<T> X = ext[ch.w];
  const Sums<T> S = sums[ch.w];
  const NetScal<T> N = net_scalars(X, S, c);
  for (int k = threadIdx.x; k < ch.z; k += blockDim.x) {
    const Pin<T> p = load_pin(ch.y + k, pin_inst, off, pos, c);
    if (c.mode2d) {
      pin_outputs_2d(p, X, N, c, acc);
    } else {
      T ex[6];
      pin_exps(p, X, c, ex, p.top);
      pin_outputs(p, ch.y + k - s0, ex, X, S, N, c, acc);
    }
  }
}

// ---- a9: L1 norms S_x, S_y, S_z of the wirelength gradient (FP64) ----
template <typename T>
__device__ __forceinline__ void norms_body(int n, const V4<T> *__restrict__ acc, T *__restrict__ part, int bid,
                                           int nblk) {
  T v[3] = {0, 0, 0};
  for (int i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
    const V4<T> a = acc[i];
    v[0] += fabs(a.x);
    v[1] += fabs(a.y);
    v[2] += fabs(a.z);
  }
  warp_sum_part<3>(v, part, bid);  // (S_x, S_y, S_z) rows
}
template <typename T>
__global__ void __launch_bounds__(256) k_norms(int n, const V4<T> *__restrict__ acc, T *__restrict__ part) {
  norms_body<T>(n, acc, part, blockIdx.x, gridDim.x);
}

}  // namespace p3d
