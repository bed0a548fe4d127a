// place3d C ABI: problem validation and upload, net-degree buckets, transform
// matrices, and the evaluation schedule (density path on a high-priority
// stream, wirelength path on two side streams, joined before the final
// per-instance combine).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/place3d.h"
#include "common.cuh"
#include "density.cuh"
#include "tc_gemm.h"
#include "transform.cuh"
#include "wirelength.cuh"
#include "nesterov.cuh"
#include "plan.h"
#include "batch.cuh"

using namespace p3d;

namespace {

thread_local std::string g_thread_err = "";

// Profiling stages.
enum Stage {
  ST_PREP = 0,
  ST_SCATTER,
  ST_PREFIX,
  ST_FWD,
  ST_ZSTAGE,
  ST_INV,
  ST_MACRO_GATHER,
  ST_WIRELENGTH,
  ST_NORMS,
  ST_FINAL,
  ST_COUNT
};
const char *kStageNames[ST_COUNT] = {"prep",         "scatter",    "prefix_densify", "transform_fwd",
                                     "zstage",       "transform_inv", "macro_gather", "wirelength",
                                     "norms",        "final"};

struct Bucket {
  int first, count;  // net range in the reordered CSR
  int dmax;          // largest degree in the bucket
  int G, PPL;        // lanes per net x pins per lane (G = 0: one block per net)
  int pin0;          // first pin of the bucket (2-pin bucket: net t's pins are pin0 + 2t, + 1)
};

// (lanes per net, pins per lane) forms of the group kernel; G = 1 is one
// thread per net with no shuffles.
// (1, 1) is the closed-form kernel of 2-pin nets.
const int kForms[][2] = {{1, 1}, {1, 2}, {1, 4}, {2, 2}, {4, 1}, {2, 4}, {8, 1}, {4, 4},
                         {16, 1}, {8, 4}, {32, 1}, {16, 4}, {32, 2}, {32, 4}};
const int kNumForms = sizeof(kForms) / sizeof(kForms[0]);

struct StageEv {
  cudaEvent_t a, b;
  int stage;
  cudaStream_t s;
};

}  // namespace

struct place3d_handle {
  int device = 0;
  bool mode2d = false;                 // multi-die 2D placement (eq. 2d-place)
  double lam_layer[3] = {0, 0, 0};     // 2D mode: density weights of the three layers
  cudaStream_t stream = nullptr, side = nullptr;
  cudaStream_t side2 = nullptr;  // second wirelength stream: the launch groups alternate between the two
  cudaEvent_t ev_w2a = nullptr, ev_w2b = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_dens = nullptr;
  // density weights on the device: double[4] then float[4] (lambda, then the
  // 2D layer weights), written on the handle's stream by set_params /
  // set_layer_weights; ev_param marks the last such write
  void *d_lam = nullptr;
  cudaEvent_t ev_param = nullptr;
  // the macros' path (corner map + scans before densify, field gather after
  // the transforms) on its own stream, overlapped with the cells' scatter and
  // gather
  cudaStream_t mac = nullptr;
  cudaEvent_t ev_mac = nullptr, ev_field = nullptr, ev_mgrad = nullptr, ev_z = nullptr;
  // Nesterov loop helpers: pins per instance (eq. improved-precond), the
  // loop state and its per-warp partial rows
  float *npins = nullptr;
  NestState *nest = nullptr;
  void *part_n = nullptr;
  // the density path (the critical chain into the final gather) runs on a
  // greatest-priority stream so that its kernels take SMs first; the
  // wirelength path fills the rest
  cudaStream_t dens = nullptr;
  int precision = 0, flags = 0;
  bool macro_direct = true;  // bin-parallel direct macro gather (else Theorem 1 suffix sums)
  // tile-bucketed scatter / gather
  bool tiles = false;
  bool host_out = false;  // the evaluation being enqueued writes host-mapped gradient arrays
  TileC tcfg{};
  int ntiles = 0, max_items = 0;
  size_t smem_scatter = 0, smem_final = 0;
  int2 *tkey = nullptr, *titems = nullptr;
  void *trec = nullptr;  // TileRec<T>[n] in tile order
  void *g4 = nullptr;    // interleaved density force V4<T>[n] (tiled final)
  int *tcount = nullptr, *tstart = nullptr, *tnitems = nullptr;
  int n = 0, nm = 0, nnet = 0, npin = 0;
  int nx = 0, ny = 0, nz = 0;
  size_t nb = 0;
  double wb = 0, hb = 0, db = 0, dx = 0, dy = 0, dz = 0;
  double xl = 0, yl = 0, xh = 0, yh = 0;  // region
  double gamma = 0, gamma_z = 0, alpha = 0, lambda = 0;
  size_t esz = 8;  // bytes per real
  // device buffers
  void *pos = nullptr, *size = nullptr, *off = nullptr, *acc = nullptr;
  uint8_t *flags_d = nullptr;
  int *macro_ids = nullptr, *macro_slot = nullptr, *net_start = nullptr, *pin_inst = nullptr;
  long long *q = nullptr, *corner = nullptr;
  void *rho = nullptr, *t1 = nullptr, *t2 = nullptr, *czpsi = nullptr, *szpsi = nullptr;
  void *xinv = nullptr, *x2 = nullptr;
  void *e4 = nullptr;  // field map [z][y][x] of (E_x, E_y, E_z, 0) in the handle's real type
  void *mats = nullptr;
  size_t mat_off[5] = {0, 0, 0, 0, 0};  // Fx, Fy, Bx(=[Sx;Cx]), Cy, Sy (elements)
  double *suffix = nullptr, *mgrad = nullptr, *scal = nullptr;
  // per-block partial sums of the scalars (rows of 4 / 3 doubles), added up
  // once per path by k_sum_parts: wirelength kernels then norms (part_w),
  // the z stage (part_d)
  double *part_w = nullptr, *part_d = nullptr;
  ZStageC *zc = nullptr;
  void *gout = nullptr;  // internal gradient output [3][n] (handle precision)
  void *stage_in = nullptr;  // staging for host positions [3][n] doubles
  int *check_flag = nullptr;
  // degree classes of the reordered netlist (contiguous, by ascending
  // degree) and the launch groups over them: each bucket is a run of
  // adjacent classes evaluated by one launch with one reduction form
  std::vector<Bucket> fine;
  std::vector<Bucket> buckets;
  // nets above 128 pins split into chunks (k_wl_big_*): chunk and net
  // tables, per-net pass counters, per-chunk partial and per-net merged
  // extremes (NetExt) and WA sums (Sums) in the handle's precision
  int4 *big_chunk = nullptr;
  int2 *big_net = nullptr;
  int *big_done = nullptr;
  void *big_ext_part = nullptr, *big_sum_part = nullptr, *big_ext = nullptr, *big_sums = nullptr;
  int big_nchunks = 0, big_nnets = 0;
  // tensor-core transform state (FP32_TC)
  p3d_tc::TcPlan *tc = nullptr;
  // CUDA graph of one evaluation (place3d_eval_graph)
  cudaGraphExec_t gexec = nullptr;
  // place3d_eval_objective_and_grad's own graph of the evaluation (positions
  // already packed), keyed by its output buffers and the parameter version
  cudaGraphExec_t egexec = nullptr;
  const void *egptr[3] = {nullptr, nullptr, nullptr};
  unsigned egversion = 0;
  // bumped by every change that a captured graph bakes in (gamma, gamma_z,
  // alpha, reduction forms; lambda and the layer weights are read from the
  // device); graphs re-capture when it moved
  unsigned version = 0, gversion = 0;
  long long captures = 0;  // graph captures (eval_graph and the internal evaluation graph)
  cudaStream_t cap_stream = nullptr;
  const void *gptr[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int gdtype = -1;
  // results
  double host_scal[S_COUNT];
  bool have_result = false;
  bool gout_fresh = false;  // the last evaluation's gradient is in gout (what the Nesterov helpers read)
  std::string err;
  int launches = 0;
  // profiling
  bool profiling = false;
  std::vector<StageEv> ev_pool, ev_live;
  double stage_ms[ST_COUNT];
  long long stage_launch[ST_COUNT];
  long long prof_evals = 0;
};

namespace {

int fail(place3d_handle *h, int code, const std::string &msg) {
  if (h)
    h->err = msg;
  else
    g_thread_err = msg;
  return code;
}

int cuda_fail(place3d_handle *h, cudaError_t e, const char *what) {
  return fail(h, e == cudaErrorMemoryAllocation ? PLACE3D_ERR_OOM : PLACE3D_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define P3D_CUDA(h, call)                                 \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

template <typename T> T *as(void *p) { return static_cast<T *>(p); }

// Stage timing helpers (events drawn from a pool, resolved on query).
struct StageScope {
  place3d_handle *h;
  int stage;
  cudaStream_t s;
  StageEv ev{};
  StageScope(place3d_handle *h_, int st, cudaStream_t s_) : h(h_), stage(st), s(s_) {
    if (!h->profiling) return;
    if (h->ev_pool.empty()) {
      cudaEventCreate(&ev.a);
      cudaEventCreate(&ev.b);
    } else {
      ev = h->ev_pool.back();
      h->ev_pool.pop_back();
    }
    ev.stage = st;
    ev.s = s;
    cudaEventRecord(ev.a, s);
    nvtxRangePushA(kStageNames[st]);  // the stage's launches, for profilers (ncu --nvtx-include)
  }
  ~StageScope() {
    if (!h->profiling) return;
    nvtxRangePop();
    cudaEventRecord(ev.b, s);
    h->ev_live.push_back(ev);
  }
};

void count_launch(place3d_handle *h, int stage) {
  h->launches++;
  if (h->profiling) h->stage_launch[stage]++;
}

int grid_for(long long n, int block) { return (int)((n + block - 1) / block); }

// The device density weights in precision T (see place3d_handle::d_lam).
template <typename T> const T *lam_dev(const place3d_handle *h) {
  return reinterpret_cast<const T *>(static_cast<const char *>(h->d_lam) + (sizeof(T) == 8 ? 0 : 4 * sizeof(double)));
}

__global__ void k_set_lam(void *dst, double l0, double l1, double l2, double l3) {
  double *d = static_cast<double *>(dst);
  float *f = reinterpret_cast<float *>(d + 4);
  const double v[4] = {l0, l1, l2, l3};
  for (int k = 0; k < 4; ++k) {
    d[k] = v[k];
    f[k] = (float)v[k];
  }
}

// Write lambda and the layer weights to the device on the handle's stream
// (ordered before every later evaluation on it; batches on other streams
// wait for ev_param).
int upload_lam(place3d_handle *h) {
  k_set_lam<<<1, 1, 0, h->stream>>>(h->d_lam, h->lambda, h->lam_layer[0], h->lam_layer[1], h->lam_layer[2]);
  P3D_CUDA(h, cudaGetLastError());
  P3D_CUDA(h, cudaEventRecord(h->ev_param, h->stream));
  return PLACE3D_OK;
}

// Test hook (place3d_debug_fail_alloc): when positive, the n-th device
// allocation of a later place3d_create on this thread reports
// cudaErrorMemoryAllocation without allocating (a fake of the failing call).
thread_local int g_fail_alloc = 0;
cudaError_t p3d_malloc(void **p, size_t bytes) {
  if (g_fail_alloc > 0 && --g_fail_alloc == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

// ---- position packing (and optional range checks) ----
template <typename TI, typename T>
__global__ void k_pack(int n, const TI *__restrict__ x, const TI *__restrict__ y, const TI *__restrict__ z,
                       V4<T> *__restrict__ pos, double zlo, double zhi, int *__restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  V4<T> p;
  p.x = (T)x[i];
  p.y = (T)y[i];
  p.z = (T)z[i];
  p.w = T(0);
  pos[i] = p;
  if (bad) {
    const double zz = (double)z[i];
    if (!isfinite((double)x[i]) || !isfinite((double)y[i]) || !(zz >= zlo && zz <= zhi)) atomicOr(bad, 1);
  }
}

template <typename T>
void host_mats(int n, double d, std::vector<T> &F, std::vector<T> &C, std::vector<T> &S) {
  // F[j][i] = cos(pi j (i+1/2)/n); C[i][j] = cos(...); S[i][j] = (j pi/d) sin(...)
  F.resize((size_t)n * n);
  C.resize((size_t)n * n);
  S.resize((size_t)n * n);
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const double arg = pi * j * (i + 0.5) / n;
      F[(size_t)j * n + i] = (T)std::cos(arg);
      C[(size_t)i * n + j] = (T)std::cos(arg);
      S[(size_t)i * n + j] = (T)((j * pi / d) * std::sin(arg));
    }
}

template <typename T> DensC<T> dens_consts(const place3d_handle *h, double xl, double yl) {
  DensC<T> c;
  c.x0 = (T)xl;
  c.y0 = (T)yl;
  c.iwb = (T)(1.0 / h->wb);
  c.ihb = (T)(1.0 / h->hb);
  c.idb = (T)(1.0 / h->db);
  c.cw = (T)(std::sqrt(2.0) * h->wb);
  c.ch = (T)(std::sqrt(2.0) * h->hb);
  c.zmid = (T)(0.5 * h->dz);
  c.qz = (T)(0.25 * h->dz);
  c.tz = (T)(2.0 / h->dz);
  c.fnx = (T)h->nx;
  c.fny = (T)h->ny;
  c.fnz = (T)h->nz;
  c.nx = h->nx;
  c.ny = h->ny;
  c.nz = h->nz;
  c.mode2d = h->mode2d ? 1 : 0;
  return c;
}

}  // namespace

namespace {

template <typename T>
GemmProb<T> gp(const void *A, const void *W, void *out, long long abs, long long obs, int batches, int M,
               int N, int K, int ostride = 1) {
  GemmProb<T> p;
  p.A = static_cast<const T *>(A);
  p.W = static_cast<const T *>(W);
  p.out = static_cast<T *>(out);
  p.a_bstride = abs;
  p.o_bstride = obs;
  p.ostride = ostride;
  p.batches = batches;
  p.M = M;
  p.N = N;
  p.K = K;
  p.tiles_m = (M + kBM - 1) / kBM;
  p.tiles_n = (N + kBN - 1) / kBN;
  return p;
}

template <typename T>
void launch_gemm(place3d_handle *h, cudaStream_t s, std::initializer_list<GemmProb<T>> probs, int stage) {
  GemmGroup<T> g;
  g.count = 0;
  int tiles = 0;
  for (const auto &p : probs) {
    g.p[g.count] = p;
    g.tile_start[g.count] = tiles;
    tiles += p.batches * p.tiles_m * p.tiles_n;
    g.count++;
  }
  g.tile_start[g.count] = tiles;
  k_gemm_simt<T><<<tiles, 256, 0, s>>>(g);
  count_launch(h, stage);
}

// Net-degree classes (largest degree of each, ascending) and the default
// launch groups over them: {2}, {3-4}, {5-8}, {9-16}, {17-32}, {33-64},
// {65-128}, {>128} with their default forms (lanes, pins per lane);
// place3d_autotune regroups the classes and picks the forms by timing.
const int kClassMax[] = {2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 128, 1 << 30};
const int kNumClasses = sizeof(kClassMax) / sizeof(kClassMax[0]);
const int kDefaultGroupMax[] = {2, 4, 8, 16, 32, 64, 128, 1 << 30};
const int kDefaultForm[][2] = {{1, 1}, {1, 4}, {8, 1}, {16, 1}, {32, 1}, {32, 2}, {32, 4}, {0, 0}};

// The launch group over classes fine[i..j] with form (G, PPL).
Bucket make_group_of(const place3d_handle *h, int i, int j, int G, int PPL) {
  Bucket b = h->fine[i];
  b.count = 0;
  for (int k = i; k <= j; ++k) b.count += h->fine[k].count;
  b.dmax = h->fine[j].dmax;
  b.G = G;
  b.PPL = PPL;
  return b;
}

// Whether form (G, PPL) can evaluate a group whose largest degree is dmax.
bool form_fits(const place3d_handle *h, int dmax, int G, int PPL) {
  if (dmax > 128) return G == 0;
  if (G == 0) return false;
  if (G == 1 && PPL == 1) return dmax == 2 && !h->mode2d;  // 2-pin closed form
  return G * PPL >= dmax && G * PPL <= 4 * std::max(dmax, 8);
}

void default_groups(place3d_handle *h) {
  h->buckets.clear();
  const int nf = (int)h->fine.size();
  for (int i = 0; i < nf;) {
    int g = 0;
    while (h->fine[i].dmax > kDefaultGroupMax[g]) ++g;
    int j = i;
    while (j + 1 < nf && h->fine[j + 1].dmax <= kDefaultGroupMax[g]) ++j;
    int G = kDefaultForm[g][0], PPL = kDefaultForm[g][1];
    if (G == 1 && PPL == 1 && h->mode2d) PPL = 2;  // 2D mode: no 2-pin closed form
    h->buckets.push_back(make_group_of(h, i, j, G, PPL));
    i = j + 1;
  }
}

// Launches one bucket's wirelength kernel; the group and pair forms write
// one row of 4 partial sums per warp at part (returns the row count), the
// block form adds its per-net sums to the scalars directly (returns 0).
template <typename T>
int launch_wl(place3d_handle *h, const Bucket &b, int G, int PPL, cudaStream_t w, const WlC<T> &c, T *part) {
  V4<T> *acc = as<V4<T>>(h->acc);
  const V4<T> *pos = as<V4<T>>(h->pos), *off = as<V4<T>>(h->off);
  if (G == 0) {  // nets above 128 pins: three passes over their chunks
    const WlBig bg{h->big_chunk, h->big_net, h->big_done};
    const int nc = h->big_nchunks;
    k_wl_big_ext<T><<<nc, 256, 0, w>>>(bg, h->net_start, h->pin_inst, off, pos, c, as<NetExt<T>>(h->big_ext_part),
                                       as<NetExt<T>>(h->big_ext));
    k_wl_big_sums<T><<<nc, 256, 0, w>>>(bg, h->pin_inst, off, pos, c, as<NetExt<T>>(h->big_ext),
                                        as<Sums<T>>(h->big_sum_part), as<Sums<T>>(h->big_sums), h->scal);
    k_wl_big_out<T><<<nc, 256, 0, w>>>(bg, h->net_start, h->pin_inst, off, pos, c, as<NetExt<T>>(h->big_ext),
                                       as<Sums<T>>(h->big_sums), acc);
    count_launch(h, ST_WIRELENGTH);
    count_launch(h, ST_WIRELENGTH);
    return 0;
  }
  if (G == 1 && PPL == 1) {  // 2-pin nets, closed form, kPairNets nets per thread
    const int gr = grid_for(b.count, 256 * kPairNets);
    k_wl_pair<T><<<gr, 256, 0, w>>>(b.pin0, b.count, h->pin_inst, off, pos, c, acc, part);
    return gr * (256 / 32);
  }
  constexpr int BS = wl_block<T>();
  const int blocks = grid_for((long long)b.count * G, BS);
#define P3D_WL(GG, PP)                                                                                  \
  if (G == GG && PPL == PP) {                                                                           \
    if (h->mode2d)                                                                                      \
      k_wl_group<T, GG, PP, true><<<blocks, BS, 0, w>>>(b.first, b.count, h->net_start, h->pin_inst, off, \
                                                        pos, c, acc, part);                             \
    else                                                                                                \
      k_wl_group<T, GG, PP, false><<<blocks, BS, 0, w>>>(b.first, b.count, h->net_start, h->pin_inst, off, \
                                                         pos, c, acc, part);                            \
    return blocks * (BS / 32);                                                                          \
  }
  P3D_WL(1, 2) P3D_WL(1, 4) P3D_WL(2, 2) P3D_WL(4, 1) P3D_WL(2, 4) P3D_WL(8, 1) P3D_WL(4, 4)
  P3D_WL(16, 1) P3D_WL(8, 4) P3D_WL(32, 1) P3D_WL(16, 4) P3D_WL(32, 2) P3D_WL(32, 4)
#undef P3D_WL
  return 0;
}

template <typename T> WlC<T> wl_consts(const place3d_handle *h) {
  WlC<T> c;
  c.zmid = (T)(0.5 * h->dz);
  c.inv_g = (T)(1.0 / h->gamma);
  c.inv_gz = (T)(1.0 / (h->gamma_z > 0 ? h->gamma_z : h->gamma));
  c.fd_scale = (T)(4.0 / h->dz);
  c.inv_g2 = (T)(1.4426950408889634 / h->gamma);
  c.inv_gz2 = (T)(1.4426950408889634 / (h->gamma_z > 0 ? h->gamma_z : h->gamma));
  c.mode2d = h->mode2d ? 1 : 0;
  return c;
}

// Add the z stage's per-block energy rows into the scalars (one per layer in 2D mode).
int sum_grid(int rows) { return std::max(1, std::min(kSumBlocks, grid_for(rows, 256))); }

// Add the z stage's per-warp energy rows (blocks of 256 threads) into the
// scalars (one per layer in 2D mode).
// rs: the stream for the reduction (it only feeds the scalars, so it can run
// beside the inverse products); rs == s keeps it in line.
template <typename T> void sum_energy(place3d_handle *h, cudaStream_t s, cudaStream_t rs, int blocks) {
  const int rows = blocks * 8;
  if (rs != s) {
    cudaEventRecord(h->ev_z, s);
    cudaStreamWaitEvent(rs, h->ev_z, 0);
    s = rs;
  }
  if (h->mode2d)
    k_sum_parts<3, T><<<sum_grid(rows), 256, 0, s>>>(as<T>(h->part_d), rows, h->scal + S_EL0);
  else
    k_sum_parts<1, T><<<sum_grid(rows), 256, 0, s>>>(as<T>(h->part_d), rows, h->scal + S_ESUM);
  count_launch(h, ST_ZSTAGE);
}

// The spectral solve: rho -> E_x, E_y, E_z (and the energy sum).
template <typename T> void run_transforms(place3d_handle *h, cudaStream_t s, cudaStream_t rs) {
  const int nx = h->nx, ny = h->ny, nz = h->nz;
  const long long pl = (long long)nx * ny;
  const T *M = as<T>(h->mats);
  const T *Fx = M + h->mat_off[0], *Fy = M + h->mat_off[1], *Bx = M + h->mat_off[2];
  const T *Cy = M + h->mat_off[3], *Sy = M + h->mat_off[4];
  {
    StageScope sc(h, ST_FWD, s);
    launch_gemm<T>(h, s, {gp<T>(h->rho, Fx, h->t1, pl, pl, nz, ny, nx, nx)}, ST_FWD);
    launch_gemm<T>(h, s, {gp<T>(h->t1, Fy, h->t2, pl, pl, nz, nx, ny, ny)}, ST_FWD);
  }
  {
    StageScope sc(h, ST_ZSTAGE, s);
    const int g = grid_for(pl, 256);
    const T *t2 = as<T>(h->t2);
    const OutPlain<T> cz{as<T>(h->czpsi)}, sz{as<T>(h->szpsi)};
    T *es = as<T>(h->part_d);
    if (nz <= 2)
      k_zstage<T, 2><<<g, 256, 0, s>>>(h->zc, t2, cz, sz, es);
    else if (nz <= 4)
      k_zstage<T, 4><<<g, 256, 0, s>>>(h->zc, t2, cz, sz, es);
    else if (nz <= 8)
      k_zstage<T, 8><<<g, 256, 0, s>>>(h->zc, t2, cz, sz, es);
    else
      k_zstage<T, 16><<<g, 256, 0, s>>>(h->zc, t2, cz, sz, es);
    count_launch(h, ST_ZSTAGE);
    sum_energy<T>(h, s, rs, g);
  }
  {
    StageScope sc(h, ST_INV, s);
    launch_gemm<T>(h, s,
                   {gp<T>(h->czpsi, Bx, h->xinv, pl, 2 * pl, nz, ny, 2 * nx, nx),
                    gp<T>(h->szpsi, Bx + (size_t)nx * nx, h->x2, pl, pl, nz, ny, nx, nx)},
                   ST_INV);
    launch_gemm<T>(h, s,
                   {gp<T>(h->xinv, Cy, as<T>(h->e4) + 0, 2 * pl, pl, nz, nx, ny, ny, 4),
                    gp<T>(as<T>(h->xinv) + pl, Sy, as<T>(h->e4) + 1, 2 * pl, pl, nz, nx, ny, ny, 4),
                    gp<T>(h->x2, Cy, as<T>(h->e4) + 2, pl, pl, nz, nx, ny, ny, 4)},
                   ST_INV);
  }
}

// The same solve on the tensor cores (split-BF16 tcgen05 products).
void run_transforms_tc(place3d_handle *h, cudaStream_t s, cudaStream_t rs) {
  {
    StageScope sc(h, ST_FWD, s);
    const int k = p3d_tc::forward(h->tc, s);
    for (int i = 0; i < k; ++i) count_launch(h, ST_FWD);
  }
  {
    StageScope sc(h, ST_ZSTAGE, s);
    const int k = p3d_tc::zstage(h->tc, s, as<float>(h->part_d));
    for (int i = 0; i < k; ++i) count_launch(h, ST_ZSTAGE);
    sum_energy<float>(h, s, rs, (int)(((long long)h->nx * h->ny + 255) / 256));
  }
  {
    StageScope sc(h, ST_INV, s);
    const int k = p3d_tc::inverse(h->tc, s);
    for (int i = 0; i < k; ++i) count_launch(h, ST_INV);
  }
}

// Tiled final assembly, density part (before the join: nothing in it waits
// for the wirelength path): the cells' windowed field gather writes their
// lambda-weighted density force into d4 (the handle's g4 buffer), and the
// macros' rows follow on the stream of their field gather.
template <typename T>
void launch_final_dens(place3d_handle *h, cudaStream_t s, cudaStream_t mgs, const DensC<T> &dc, const FinalC<T> &fc) {
  k_final_tiles<T><<<h->max_items, 256, h->smem_final, s>>>(h->titems, h->tnitems, h->tstart, as<TileRec<T>>(h->trec),
                                                            dc, h->tcfg, as<V4<T>>(h->e4), fc, as<V4<T>>(h->g4));
  count_launch(h, ST_FINAL);
  if (h->nm > 0) {
    k_final_macros<T><<<grid_for(h->nm, 128), 128, 0, mgs>>>(h->nm, h->macro_ids, as<V4<T>>(h->pos), h->mgrad, fc,
                                                             dc.zmid, as<V4<T>>(h->g4));
    count_launch(h, ST_FINAL);
  }
}

// Batch capture with a shared wirelength stage: the scalars, the WL
// accumulators and the packed positions are set by the batch's own launches
// before this instance's branch starts, the WL stage runs once for the whole
// batch, and the final assembly waits for `wl_done` instead of this handle's
// own WL path.
struct BatchHook {
  cudaEvent_t wl_done;
};

template <typename T>
int eval_impl(place3d_handle *h, void *gx, void *gy, void *gz, int dtype, int mem, const BatchHook *bh = nullptr) {
  const bool serial = (h->flags & PLACE3D_FLAG_SERIAL) != 0;
  cudaStream_t caller = h->stream, s = serial ? caller : h->dens, w = serial ? caller : h->side;
  const int n = h->n;
  const DensC<T> dc = dens_consts<T>(h, h->xl, h->yl);
  h->launches = 0;
  if (!bh) P3D_CUDA(h, cudaMemsetAsync(h->scal, 0, sizeof(double) * S_COUNT, caller));  // before the fork: both paths add
  P3D_CUDA(h, cudaEventRecord(h->ev_fork, caller));
  if (s != caller) P3D_CUDA(h, cudaStreamWaitEvent(s, h->ev_fork, 0));
  // macros on their own stream (direct field gather, untiled scatter)
  // third stream (not in serial mode): the macros' path when their field
  // gather is direct and the scatter untiled, and the scalar reductions that
  // nothing on the density chain waits for
  const bool split = !serial && h->nm > 0 && h->macro_direct;
  cudaStream_t ms = serial ? s : h->mac;
  if (ms != s) P3D_CUDA(h, cudaStreamWaitEvent(ms, h->ev_fork, 0));
  cudaStream_t mcs = split ? ms : s;  // stream of the macros' kernels
  if (!bh) {  // (in a batch with a shared WL stage, the batch runs it)
    // ---------------- wirelength path (side stream) ----------------
    P3D_CUDA(h, cudaStreamWaitEvent(w, h->ev_fork, 0));
    {
      StageScope sc(h, ST_WIRELENGTH, w);
      P3D_CUDA(h, cudaMemsetAsync(h->acc, 0, sizeof(V4<T>) * (size_t)std::max(n, 1), w));
      const WlC<T> c = wl_consts<T>(h);
      // the launch groups alternate between two streams: one group's tail
      // (its last blocks) overlaps the next group's start
      int rows = 0;
      cudaStream_t w2 = serial ? w : h->side2;
      if (w2 != w) {
        P3D_CUDA(h, cudaEventRecord(h->ev_w2a, w));
        P3D_CUDA(h, cudaStreamWaitEvent(w2, h->ev_w2a, 0));
      }
      int kb = 0;
      for (const Bucket &b : h->buckets) {
        rows += launch_wl<T>(h, b, b.G, b.PPL, (kb++ & 1) ? w2 : w, c, as<T>(h->part_w) + 4 * (size_t)rows);
        count_launch(h, ST_WIRELENGTH);
      }
      if (w2 != w) {
        P3D_CUDA(h, cudaEventRecord(h->ev_w2b, w2));
        P3D_CUDA(h, cudaStreamWaitEvent(w, h->ev_w2b, 0));
      }
      if (rows > 0) {
        k_sum_parts<4, T><<<sum_grid(rows), 256, 0, w>>>(as<T>(h->part_w), rows, h->scal + S_WL_BI);
        count_launch(h, ST_WIRELENGTH);
      }
    }
    {
      StageScope sc(h, ST_NORMS, w);
      const int gn = std::min(grid_for(std::max(n, 1), 256), 1216);
      k_norms<T><<<gn, 256, 0, w>>>(n, as<V4<T>>(h->acc), as<T>(h->part_w));
      k_sum_parts<3, T><<<sum_grid(gn * 8), 256, 0, w>>>(as<T>(h->part_w), gn * 8, h->scal + S_SX);
      count_launch(h, ST_NORMS);
      count_launch(h, ST_NORMS);
    }
    P3D_CUDA(h, cudaEventRecord(h->ev_join, w));
  }
  // ---------------- density path (caller's stream) ----------------
  {
    StageScope sc(h, ST_SCATTER, s);
    P3D_CUDA(h, cudaMemsetAsync(h->q, 0, sizeof(long long) * h->nb, s));
    if (n > 0 && h->tiles) {
      P3D_CUDA(h, cudaMemsetAsync(h->tcount, 0, sizeof(int) * kCountPad * (h->ntiles + 1), s));
      k_tile_count<T><<<grid_for(n, kCountBlock * kCountPerThread), kCountBlock, sizeof(int) * h->ntiles, s>>>(
          n, as<V4<T>>(h->pos), h->flags_d, dc, h->tcfg, h->ntiles, h->tcount, h->tkey, h->tstart, h->titems,
          h->tnitems);
      k_tile_place<T><<<grid_for(n, 256), 256, 0, s>>>(n, h->tkey, h->tstart, as<V4<T>>(h->pos), as<V4<T>>(h->size),
                                                       h->flags_d, dc, as<TileRec<T>>(h->trec));
      k_scatter_tiles<T><<<h->max_items, 256, h->smem_scatter, s>>>(h->titems, h->tnitems, h->tstart,
                                                                    as<TileRec<T>>(h->trec), dc, h->tcfg, h->q);
      for (int k = 0; k < 3; ++k) count_launch(h, ST_SCATTER);
    } else if (n > 0) {
      k_scatter_cells<T><<<grid_for(2 * (long long)n, 256), 256, 0, s>>>(n, as<V4<T>>(h->pos), as<V4<T>>(h->size), h->flags_d,
                                                          dc, h->q);
      count_launch(h, ST_SCATTER);
    }
    if (h->nm > 0) {
      P3D_CUDA(h, cudaMemsetAsync(h->corner, 0, sizeof(long long) * h->nb, mcs));
      k_macro_corners<T><<<grid_for(h->nm * 8, 128), 128, 0, mcs>>>(h->nm, h->macro_ids, as<V4<T>>(h->pos),
                                                                    as<V4<T>>(h->size), dc, h->corner);
      count_launch(h, ST_SCATTER);
    }
  }
  {
    StageScope sc(h, ST_PREFIX, s);
    const int rows = h->ny * h->nz;
    if (h->nm > 0) {
      k_scan_rows<long long, long long, false><<<grid_for(rows, 8), 256, 0, mcs>>>(rows, h->nx, h->corner, 1,
                                                                                  h->corner);
      count_launch(h, ST_PREFIX);
      k_scan_cols<long long, false><<<dim3(grid_for(h->nx, 32), h->nz), 1024, 0, mcs>>>(h->nx, h->ny, h->corner);
      count_launch(h, ST_PREFIX);
      if (split) {
        P3D_CUDA(h, cudaEventRecord(h->ev_mac, mcs));
        P3D_CUDA(h, cudaStreamWaitEvent(s, h->ev_mac, 0));
      }
    }
    if (h->tc) {
      p3d_tc::densify(h->tc, s, h->nx * h->ny, h->nz, h->q, h->nm > 0 ? h->corner : nullptr, as<float>(h->part_d));
    } else {
      k_densify<T><<<grid_for((long long)h->nx * h->ny, 256), 256, 0, s>>>(
          h->nx * h->ny, h->nz, h->q, h->nm > 0 ? h->corner : nullptr, OutPlain<T>{as<T>(h->rho)}, as<T>(h->part_d));
    }
    count_launch(h, ST_PREFIX);
    // density overflow (sum of max(rho - 1, 0) and of rho) from densify's per-warp rows
    const int orow = grid_for((long long)h->nx * h->ny, 256) * 8;
    if (ms != s) {  // nothing on the density chain waits for it
      P3D_CUDA(h, cudaEventRecord(h->ev_z, s));
      P3D_CUDA(h, cudaStreamWaitEvent(ms, h->ev_z, 0));
    }
    if (h->tc)
      k_sum_parts<2, float><<<sum_grid(orow), 256, 0, ms>>>(as<float>(h->part_d), orow, h->scal + S_OVFL);
    else
      k_sum_parts<2, T><<<sum_grid(orow), 256, 0, ms>>>(as<T>(h->part_d), orow, h->scal + S_OVFL);
    count_launch(h, ST_PREFIX);
  }
  if (h->tc)
    run_transforms_tc(h, s, ms);
  else
    run_transforms<T>(h, s, ms);
  if (h->nm > 0 && h->macro_direct) {
    if (split) {
      P3D_CUDA(h, cudaEventRecord(h->ev_field, s));
      P3D_CUDA(h, cudaStreamWaitEvent(mcs, h->ev_field, 0));
    }
    StageScope sc(h, ST_MACRO_GATHER, mcs);
    P3D_CUDA(h, cudaMemsetAsync(h->mgrad, 0, sizeof(double) * 3 * h->nm, mcs));
    k_macro_gather_direct<T><<<dim3(h->nm, 16), 256, 0, mcs>>>(h->macro_ids, as<V4<T>>(h->pos), as<V4<T>>(h->size),
                                                              dc, as<V4<T>>(h->e4), h->mgrad);
    count_launch(h, ST_MACRO_GATHER);
  } else if (h->nm > 0) {
    StageScope sc(h, ST_MACRO_GATHER, s);
    const int rows = h->ny * h->nz;
    for (int comp = 0; comp < 3; ++comp) {
      const T *E = as<T>(h->e4) + comp;  // one component of the interleaved field map
      k_scan_rows<T, double, true><<<grid_for(rows, 8), 256, 0, s>>>(rows, h->nx, E, 4, h->suffix + comp * h->nb);
      count_launch(h, ST_MACRO_GATHER);
    }
    k_scan_cols<double, true><<<dim3(grid_for(h->nx, 32), h->nz * 3), 1024, 0, s>>>(h->nx, h->ny, h->suffix);
    count_launch(h, ST_MACRO_GATHER);
    P3D_CUDA(h, cudaMemsetAsync(h->mgrad, 0, sizeof(double) * 3 * h->nm, s));
    k_macro_gather<T><<<grid_for(h->nm * 8, 128), 128, 0, s>>>(h->nm, h->macro_ids, as<V4<T>>(h->pos),
                                                               as<V4<T>>(h->size), dc, h->suffix, h->nb, h->mgrad);
    count_launch(h, ST_MACRO_GATHER);
  }
  FinalC<T> fc;
  fc.alpha = (T)h->alpha;
  fc.volb = (T)(h->mode2d ? h->wb * h->hb : h->wb * h->hb * h->db);  // 2D: bin area
  fc.scal = h->scal;
  fc.lam_dev = lam_dev<T>(h);
  fc.g = T(0);
  fc.mode2d = h->mode2d ? 1 : 0;
  // host-mapped outputs: the per-cell gather, whose stores to host memory
  // (coalesced, by instance) overlap its computation
  const bool tiled_final = n > 0 && h->tiles && !h->host_out;
  if (tiled_final) {
    StageScope sc(h, ST_FINAL, s);
    cudaStream_t mgs = h->nm > 0 && h->macro_direct ? mcs : s;  // the macros' field gather ran there
    launch_final_dens<T>(h, s, mgs, dc, fc);
    if (mgs != s) {
      P3D_CUDA(h, cudaEventRecord(h->ev_mgrad, mgs));
      P3D_CUDA(h, cudaStreamWaitEvent(s, h->ev_mgrad, 0));
    }
  }
  // ---------------- join + final assembly ----------------
  P3D_CUDA(h, cudaStreamWaitEvent(s, bh ? bh->wl_done : h->ev_join, 0));
  {
    StageScope sc(h, ST_FINAL, s);
    const bool direct = mem == PLACE3D_MEM_DEVICE && gx && gy && gz;
    const int odt = direct ? dtype : (sizeof(T) == 8 ? PLACE3D_F64 : PLACE3D_F32);
    void *ox = direct ? gx : h->gout;
    void *oy = direct ? gy : (char *)h->gout + (size_t)n * sizeof(T);
    void *oz = direct ? gz : (char *)h->gout + (size_t)2 * n * sizeof(T);
    if (tiled_final) {  // the wirelength part and the density force, per instance
      if (odt == PLACE3D_F64)
        k_combine<T, double><<<grid_for(n, 256), 256, 0, s>>>(n, as<V4<T>>(h->acc), as<V4<T>>(h->g4), h->flags_d, fc,
                                                              (double *)ox, (double *)oy, (double *)oz);
      else
        k_combine<T, float><<<grid_for(n, 256), 256, 0, s>>>(n, as<V4<T>>(h->acc), as<V4<T>>(h->g4), h->flags_d, fc,
                                                             (float *)ox, (float *)oy, (float *)oz);
      count_launch(h, ST_FINAL);
    } else if (n > 0) {
      if (odt == PLACE3D_F64)
        k_final<T, double><<<grid_for(n, 256), 256, 0, s>>>(n, as<V4<T>>(h->pos), as<V4<T>>(h->size), h->flags_d,
                                                            h->macro_slot, dc, as<V4<T>>(h->e4),
                                                            h->mgrad, as<V4<T>>(h->acc), fc, (double *)ox, (double *)oy,
                                                            (double *)oz, split ? 1 : 0);
      else
        k_final<T, float><<<grid_for(n, 256), 256, 0, s>>>(n, as<V4<T>>(h->pos), as<V4<T>>(h->size), h->flags_d,
                                                           h->macro_slot, dc, as<V4<T>>(h->e4),
                                                           h->mgrad, as<V4<T>>(h->acc), fc, (float *)ox, (float *)oy,
                                                           (float *)oz, split ? 1 : 0);
      count_launch(h, ST_FINAL);
      if (split) {  // the macros, once their field gather is done
        P3D_CUDA(h, cudaEventRecord(h->ev_mgrad, ms));
        P3D_CUDA(h, cudaStreamWaitEvent(s, h->ev_mgrad, 0));
        if (odt == PLACE3D_F64)
          k_final_macro_out<T, double><<<grid_for(h->nm, 128), 128, 0, s>>>(
              h->nm, h->macro_ids, as<V4<T>>(h->pos), h->flags_d, h->mgrad, as<V4<T>>(h->acc), fc, dc.zmid,
              (double *)ox, (double *)oy, (double *)oz);
        else
          k_final_macro_out<T, float><<<grid_for(h->nm, 128), 128, 0, s>>>(
              h->nm, h->macro_ids, as<V4<T>>(h->pos), h->flags_d, h->mgrad, as<V4<T>>(h->acc), fc, dc.zmid,
              (float *)ox, (float *)oy, (float *)oz);
        count_launch(h, ST_FINAL);
      }
    }
    if (!direct && gx && gy && gz && n > 0) {
      // host outputs (or device outputs of another dtype): copy / convert
      const size_t tb = sizeof(T);
      const size_t ob = dtype == PLACE3D_F64 ? 8 : 4;
      if (ob != tb) return fail(h, PLACE3D_ERR_INVALID_ARG, "host gradient dtype must match the handle precision");
      cudaMemcpyKind k = mem == PLACE3D_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
      P3D_CUDA(h, cudaMemcpyAsync(gx, ox, (size_t)n * tb, k, s));
      P3D_CUDA(h, cudaMemcpyAsync(gy, oy, (size_t)n * tb, k, s));
      P3D_CUDA(h, cudaMemcpyAsync(gz, oz, (size_t)n * tb, k, s));
    }
  }
  if (ms != s) {  // the third stream's reductions
    P3D_CUDA(h, cudaEventRecord(h->ev_mgrad, ms));
    P3D_CUDA(h, cudaStreamWaitEvent(caller, h->ev_mgrad, 0));
  }
  if (s != caller) {
    P3D_CUDA(h, cudaEventRecord(h->ev_dens, s));
    P3D_CUDA(h, cudaStreamWaitEvent(caller, h->ev_dens, 0));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
  if (h->profiling) h->prof_evals++;
  return PLACE3D_OK;
}

void fill_result(const place3d_handle *h, place3d_result *r) {
  const double *s = h->host_scal;
  const double volb = h->wb * h->hb * h->db;
  r->wl_bi = s[S_WL_BI];
  r->wl_z = s[S_WL_Z];
  r->hpwl_d2d = s[S_HPWL];
  r->n_cross = s[S_NCROSS];
  r->energy = 0.5 * volb * (double)h->nb * s[S_ESUM];
  r->s_x = s[S_SX];
  r->s_y = s[S_SY];
  r->s_z = s[S_SZ];
  r->g_scale = s[S_SZ] > 0 ? (s[S_SX] + s[S_SY]) / (2.0 * s[S_SZ]) : 0.0;
  r->obj = r->wl_bi + h->alpha * r->wl_z + h->lambda * r->energy;
  r->overflow = s[S_RHO] > 0 ? s[S_OVFL] / s[S_RHO] : 0.0;
  for (int l = 0; l < 3; ++l) r->energy_layer[l] = 0.0;
  if (h->mode2d) {
    // eq. 2d-place: U_l = 1/2 A_b N_x N_y sum c_j c_k a^2 / w^2 per layer
    const double ab = h->wb * h->hb, nxy = (double)h->nx * h->ny;
    r->energy = 0.0;
    r->obj = r->wl_bi;
    for (int l = 0; l < 3; ++l) {
      r->energy_layer[l] = 0.5 * ab * nxy * s[S_EL0 + l];
      r->energy += r->energy_layer[l];
      r->obj += h->lam_layer[l] * r->energy_layer[l];
    }
  }
}

void free_all(place3d_handle *h) {
  void *bufs[] = {h->pos,   h->size,  h->off,   h->acc,   h->flags_d, h->macro_ids, h->macro_slot,
                  h->net_start, h->pin_inst, h->q, h->corner, h->rho, h->t1, h->t2, h->czpsi,
                  h->szpsi, h->xinv, h->x2, h->e4, h->mats, h->suffix, h->mgrad,
                  h->scal, h->zc, h->gout, h->stage_in, h->check_flag, h->tkey, h->titems,
                  h->part_w, h->part_d, h->d_lam, h->npins, h->nest, h->part_n,
                  h->tcount, h->tstart, h->tnitems, h->trec, h->g4, h->big_chunk, h->big_net,
                  h->big_done, h->big_ext_part, h->big_sum_part, h->big_ext, h->big_sums};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (h->tc) p3d_tc::destroy(h->tc);
  for (auto &e : h->ev_pool) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (auto &e : h->ev_live) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_dens) cudaEventDestroy(h->ev_dens);
  if (h->ev_param) cudaEventDestroy(h->ev_param);
  if (h->ev_mac) cudaEventDestroy(h->ev_mac);
  if (h->ev_field) cudaEventDestroy(h->ev_field);
  if (h->ev_mgrad) cudaEventDestroy(h->ev_mgrad);
  if (h->ev_z) cudaEventDestroy(h->ev_z);
  if (h->mac) cudaStreamDestroy(h->mac);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->side2) cudaStreamDestroy(h->side2);
  if (h->ev_w2a) cudaEventDestroy(h->ev_w2a);
  if (h->ev_w2b) cudaEventDestroy(h->ev_w2b);
  if (h->dens) cudaStreamDestroy(h->dens);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->egexec) cudaGraphExecDestroy(h->egexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
}

template <typename T>
int upload_typed(place3d_handle *h, const place3d_problem *p, const std::vector<int> &order,
                 const std::vector<int> &new_start) {
  const int n = h->n;
  // instance sizes (w_bot, h_bot, w_top, h_top)
  std::vector<V4<T>> sz(std::max(n, 1));
  for (int i = 0; i < n; ++i) {
    sz[i].x = (T)p->w_bot[i];
    sz[i].y = (T)p->h_bot[i];
    sz[i].z = (T)p->w_top[i];
    sz[i].w = (T)p->h_top[i];
  }
  P3D_CUDA(h, cudaMemcpy(h->size, sz.data(), sizeof(V4<T>) * n, cudaMemcpyHostToDevice));
  // pins in bucket order
  std::vector<V4<T>> off(std::max(h->npin, 1));
  std::vector<int> pin(std::max(h->npin, 1));
  size_t k = 0;
  for (int e : order) {
    for (int q = p->net_start[e]; q < p->net_start[e + 1]; ++q, ++k) {
      pin[k] = p->pin_inst[q];
      if (h->mode2d && p->is_hbt && p->is_hbt[pin[k]]) pin[k] = ~pin[k];  // HBT pin: both partial nets
      off[k].x = (T)p->pin_off_bot_x[q];
      off[k].y = (T)p->pin_off_bot_y[q];
      off[k].z = (T)p->pin_off_top_x[q];
      off[k].w = (T)p->pin_off_top_y[q];
    }
  }
  P3D_CUDA(h, cudaMemcpy(h->off, off.data(), sizeof(V4<T>) * k, cudaMemcpyHostToDevice));
  P3D_CUDA(h, cudaMemcpy(h->pin_inst, pin.data(), sizeof(int) * k, cudaMemcpyHostToDevice));
  P3D_CUDA(h, cudaMemcpy(h->net_start, new_start.data(), sizeof(int) * new_start.size(), cudaMemcpyHostToDevice));
  // transform matrices
  std::vector<T> Fx, Cx, Sx, Fy, Cy, Sy;
  host_mats<T>(h->nx, h->dx, Fx, Cx, Sx);
  host_mats<T>(h->ny, h->dy, Fy, Cy, Sy);
  const size_t nx2 = (size_t)h->nx * h->nx, ny2 = (size_t)h->ny * h->ny;
  h->mat_off[0] = 0;
  h->mat_off[1] = nx2;
  h->mat_off[2] = nx2 + ny2;
  h->mat_off[3] = 3 * nx2 + ny2;
  h->mat_off[4] = 3 * nx2 + 2 * ny2;
  std::vector<T> all(3 * nx2 + 3 * ny2);
  std::copy(Fx.begin(), Fx.end(), all.begin());
  std::copy(Fy.begin(), Fy.end(), all.begin() + h->mat_off[1]);
  std::copy(Sx.begin(), Sx.end(), all.begin() + h->mat_off[2]);
  std::copy(Cx.begin(), Cx.end(), all.begin() + h->mat_off[2] + nx2);
  std::copy(Cy.begin(), Cy.end(), all.begin() + h->mat_off[3]);
  std::copy(Sy.begin(), Sy.end(), all.begin() + h->mat_off[4]);
  {
    const cudaError_t e = p3d_malloc(&h->mats, sizeof(T) * all.size());
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");  // OOM for an allocation failure
  }
  P3D_CUDA(h, cudaMemcpy(h->mats, all.data(), sizeof(T) * all.size(), cudaMemcpyHostToDevice));
  return PLACE3D_OK;
}

}  // namespace

extern "C" {

void place3d_debug_fail_alloc(int nth) { g_fail_alloc = nth > 0 ? nth : 0; }

namespace {
__global__ void k_ll2f_check(const long long *v, float *out, int n, int *bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = r_ll2f(v[i]), b = __ll2float_rn(v[i]);
  out[i] = a;
  if (__float_as_uint(a) != __float_as_uint(b)) atomicAdd(bad, 1);
}
}  // namespace

int place3d_ll2f_selftest(const long long *vals, float *out, int n, int *mismatches) {
  if (!vals || !out || !mismatches || n < 0) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "bad selftest arguments");
  *mismatches = 0;
  if (n == 0) return PLACE3D_OK;
  long long *dv = nullptr;
  float *dout = nullptr;
  int *dbad = nullptr;
  int rc = PLACE3D_ERR_CUDA;
  if (cudaMalloc(&dv, sizeof(long long) * n) == cudaSuccess && cudaMalloc(&dout, sizeof(float) * n) == cudaSuccess &&
      cudaMalloc(&dbad, sizeof(int)) == cudaSuccess && cudaMemset(dbad, 0, sizeof(int)) == cudaSuccess &&
      cudaMemcpy(dv, vals, sizeof(long long) * n, cudaMemcpyHostToDevice) == cudaSuccess) {
    k_ll2f_check<<<grid_for(n, 256), 256>>>(dv, dout, n, dbad);
    if (cudaGetLastError() == cudaSuccess &&
        cudaMemcpy(out, dout, sizeof(float) * n, cudaMemcpyDeviceToHost) == cudaSuccess &&
        cudaMemcpy(mismatches, dbad, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
      rc = PLACE3D_OK;
  }
  cudaFree(dv);
  cudaFree(dout);
  cudaFree(dbad);
  return rc == PLACE3D_OK ? rc : fail(nullptr, rc, "conversion self-test failed");
}

double place3d_alpha(double dx, double dz, double beta, double w_hbt, double rh_top, double rh_bot) {
  const double eta = 2.0 * w_hbt / (rh_top + rh_bot);
  return 3.5e-3 * (dx * eta * eta / dz) * std::log(90.0 * beta * eta - 1.0);
}

int place3d_create(const place3d_problem *p, int device, void *cuda_stream, place3d_handle **out) {
  if (!p || !out) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL problem or output handle pointer");
  *out = nullptr;
  if (p->n_inst < 0 || p->n_net < 0 || p->n_pin < 0)
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "negative instance, net or pin count");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nz > kMaxNz)
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "bin grid must have nx, ny >= 1 and 1 <= nz <= 16");
  if (!(p->xh > p->xl) || !(p->yh > p->yl) || !std::isfinite(p->xl) || !std::isfinite(p->yl) ||
      !std::isfinite(p->xh) || !std::isfinite(p->yh))
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "region must satisfy xh > xl and yh > yl (finite)");
  if (!(p->gamma > 0) || !std::isfinite(p->gamma) || !std::isfinite(p->alpha) || !std::isfinite(p->lambda))
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "gamma must be > 0; alpha, lambda finite");
  if (p->precision != PLACE3D_FP64 && p->precision != PLACE3D_FP32 && p->precision != PLACE3D_FP32_TC)
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "unknown precision mode");
  const int n = p->n_inst;
  if (n > 0 && (!p->is_macro || !p->w_bot || !p->h_bot || !p->w_top || !p->h_top))
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL instance array");
  if (p->mode != PLACE3D_MODE_3D && p->mode != PLACE3D_MODE_2D)
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "unknown placement mode");
  if (p->mode == PLACE3D_MODE_2D) {
    if (p->nz != 3) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "2D mode needs nz = 3 layers");
    for (int l = 0; l < 3; ++l)
      if (!std::isfinite(p->lam_layer[l])) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "lam_layer must be finite");
    if (p->is_hbt)
      for (int i = 0; i < n; ++i)
        if (p->is_hbt[i] && p->is_macro[i])
          return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "an HBT cannot be a macro");
  } else if (p->is_hbt) {
    for (int i = 0; i < n; ++i)
      if (p->is_hbt[i]) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "HBT instances need 2D mode");
  }
  for (int i = 0; i < n; ++i)
    if (!(p->w_bot[i] >= 0) || !(p->h_bot[i] >= 0) || !(p->w_top[i] >= 0) || !(p->h_top[i] >= 0) ||
        !std::isfinite(p->w_bot[i] + p->h_bot[i] + p->w_top[i] + p->h_top[i]))
      return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "instance sizes must be finite and >= 0");
  if (!p->net_start) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL net_start");
  if (p->net_start[0] != 0 || p->net_start[p->n_net] != p->n_pin)
    return fail(nullptr, PLACE3D_ERR_BAD_CSR, "net_start[0] must be 0 and net_start[n_net] == n_pin");
  if (p->n_pin > 0 && (!p->pin_inst || !p->pin_off_bot_x || !p->pin_off_bot_y || !p->pin_off_top_x ||
                       !p->pin_off_top_y))
    return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL pin array");
  std::vector<int> stamp(std::max(n, 1), -1);
  for (int e = 0; e < p->n_net; ++e) {
    if (p->net_start[e + 1] < p->net_start[e]) return fail(nullptr, PLACE3D_ERR_BAD_CSR, "net_start decreases");
    for (int q = p->net_start[e]; q < p->net_start[e + 1]; ++q) {
      const int i = p->pin_inst[q];
      if (i < 0 || i >= n) return fail(nullptr, PLACE3D_ERR_BAD_CSR, "pin_inst out of range");
      if (stamp[i] == e)
        return fail(nullptr, PLACE3D_ERR_BAD_CSR, "an instance holds two pins of one net (net " + std::to_string(e) + ")");
      stamp[i] = e;
      if (!std::isfinite(p->pin_off_bot_x[q] + p->pin_off_bot_y[q] + p->pin_off_top_x[q] + p->pin_off_top_y[q]))
        return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "pin offsets must be finite");
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(nullptr, PLACE3D_ERR_CUDA, "no such CUDA device");
  if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, PLACE3D_ERR_CUDA, "cudaSetDevice failed");

  place3d_handle *h = new place3d_handle();
  h->device = device;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->precision = p->precision;
  h->flags = p->flags;
  h->n = n;
  h->nx = p->nx;
  h->ny = p->ny;
  h->nz = p->nz;
  h->nb = (size_t)p->nx * p->ny * p->nz;
  h->dx = p->xh - p->xl;
  h->dy = p->yh - p->yl;
  h->wb = h->dx / p->nx;
  h->hb = h->dy / p->ny;
  h->db = 0.5 * (h->wb + h->hb);
  h->dz = p->nz * h->db;
  h->gamma = p->gamma;
  h->gamma_z = p->gamma_z;
  h->alpha = p->alpha;
  h->lambda = p->lambda;
  h->esz = p->precision == PLACE3D_FP64 ? 8 : 4;
  std::memset(h->stage_ms, 0, sizeof(h->stage_ms));
  std::memset(h->stage_launch, 0, sizeof(h->stage_launch));
  h->xl = p->xl;
  h->yl = p->yl;
  h->xh = p->xh;
  h->yh = p->yh;
  h->mode2d = p->mode == PLACE3D_MODE_2D;
  for (int l = 0; l < 3; ++l) h->lam_layer[l] = h->mode2d ? p->lam_layer[l] : 0.0;
  auto bail = [&](int code) {
    free_all(h);
    g_thread_err = h->err;
    delete h;
    return code;
  };

  // net-degree classes: nets of degree < 2 are dropped (they contribute 0)
  std::vector<std::vector<int>> cls(kNumClasses);
  for (int e = 0; e < p->n_net; ++e) {
    const int d = p->net_start[e + 1] - p->net_start[e];
    if (d < 2) continue;
    int k = 0;
    while (d > kClassMax[k]) ++k;
    cls[k].push_back(e);
  }
  // within a class, nets by ascending degree (stable): the nets that one
  // warp of a group form reduces then have about the same degree, so the
  // warp skips the pin slots that none of its nets fills
  for (auto &v : cls)
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
      return p->net_start[a + 1] - p->net_start[a] < p->net_start[b + 1] - p->net_start[b];
    });
  std::vector<int> order, new_start(1, 0);
  for (int k = 0; k < kNumClasses; ++k) {
    if (cls[k].empty()) continue;
    int dmax = 0;
    for (int e : cls[k]) dmax = std::max(dmax, p->net_start[e + 1] - p->net_start[e]);
    h->fine.push_back({(int)order.size(), (int)cls[k].size(), dmax, 0, 0, new_start.back()});
    for (int e : cls[k]) {
      order.push_back(e);
      new_start.push_back(new_start.back() + (p->net_start[e + 1] - p->net_start[e]));
    }
  }
  default_groups(h);
  h->nnet = (int)order.size();
  h->npin = new_start.back();
  // macros
  std::vector<int> mids, mslot(std::max(n, 1), -1);
  std::vector<uint8_t> fl(std::max(n, 1), 0);
  for (int i = 0; i < n; ++i) {
    if (p->is_macro[i]) {
      mslot[i] = (int)mids.size();
      mids.push_back(i);
      fl[i] |= 1;
    }
    if (p->z_fixed && p->z_fixed[i]) fl[i] |= 2;
    if (h->mode2d && p->is_hbt && p->is_hbt[i]) fl[i] |= 4;
  }
  h->nm = (int)mids.size();
  // macro gather form: direct when the macros' bins (at their larger size) are
  // fewer than twice the grid, Theorem 1's suffix-sum adjoint otherwise
  {
    double covered = 0;
    const double wbv = (p->xh - p->xl) / p->nx, hbv = (p->yh - p->yl) / p->ny;
    for (int i : mids) {
      const double w = std::max(p->w_bot[i], p->w_top[i]), hh = std::max(p->h_bot[i], p->h_top[i]);
      covered += (std::ceil(std::max(w, std::sqrt(2.0) * wbv) / wbv) + 1) *
                 (std::ceil(std::max(hh, std::sqrt(2.0) * hbv) / hbv) + 1) * (p->nz / 2 + 2);
    }
    h->macro_direct = covered <= 2.0 * (double)p->nx * p->ny * p->nz;
    if (p->flags & PLACE3D_FLAG_MACRO_GATHER_SCAN) h->macro_direct = false;
    if (p->flags & PLACE3D_FLAG_MACRO_GATHER_DIRECT) h->macro_direct = true;
  }
  // tile windows: halo R covers the largest std-cell footprint (stretched)
  {
    const double wbv = (p->xh - p->xl) / p->nx, hbv = (p->yh - p->yl) / p->ny;
    double hw = std::sqrt(2.0) * wbv, hh = std::sqrt(2.0) * hbv;
    for (int i = 0; i < n; ++i)
      if (!p->is_macro[i]) {
        hw = std::max(hw, std::max(p->w_bot[i], p->w_top[i]));
        hh = std::max(hh, std::max(p->h_bot[i], p->h_top[i]));
      }
    // a cell's centre lies in its tile, so a halo of ceil(half the stretched
    // footprint) bins holds the whole footprint
    const int R = std::max(1, (int)std::max(std::ceil(0.5 * hw / wbv), std::ceil(0.5 * hh / hbv)));
    h->tcfg.ntx = (p->nx + kTile - 1) / kTile;
    h->tcfg.nty = (p->ny + kTile - 1) / kTile;
    h->tcfg.R = R;
    h->tcfg.WX = kTile + 2 * R;
    h->tcfg.WY = kTile + 2 * R;
    h->ntiles = h->tcfg.ntx * h->tcfg.nty;
    const size_t wbins = (size_t)h->tcfg.WX * h->tcfg.WY * p->nz;
    h->smem_scatter = wbins * 8;  // two 32-bit words per bin
    h->smem_final = wbins * 4 * (p->precision == PLACE3D_FP64 ? 8 : 4);  // one (E_x, E_y, E_z, -) vector per bin
    // small problems are launch-bound: the sort's extra launches do not pay
    // below kTileMinInst instances; in 2D mode an instance covers one layer
    // (about 6 bins instead of 17), too little work per cell for the sort to
    // pay; PLACE3D_FLAG_TILES asks for tiles anyway
    const bool want = (p->flags & PLACE3D_FLAG_TILES) || (n >= kTileMinInst && p->mode != PLACE3D_MODE_2D);
    h->tiles = want && !(p->flags & PLACE3D_FLAG_NO_TILES) && R <= 8 && h->ntiles <= 8192 && n < (1 << 24) &&
               h->smem_final <= 200 * 1024 && h->smem_scatter <= 200 * 1024;
    h->max_items = (n + kChunk - 1) / kChunk + h->ntiles;
  }

  // device allocation
  const size_t es = h->esz, nb = h->nb, nn = std::max(n, 1);
  const size_t v4 = es * 4;
  struct A {
    void **p;
    size_t bytes;
  } allocs[] = {
      {&h->pos, v4 * nn}, {&h->size, v4 * nn}, {&h->off, v4 * (size_t)std::max(h->npin, 1)}, {&h->acc, v4 * nn},
      {(void **)&h->flags_d, nn}, {(void **)&h->macro_ids, sizeof(int) * (size_t)std::max(h->nm, 1)},
      {(void **)&h->macro_slot, sizeof(int) * nn}, {(void **)&h->net_start, sizeof(int) * (size_t)(h->nnet + 1)},
      {(void **)&h->pin_inst, sizeof(int) * (size_t)std::max(h->npin, 1)}, {(void **)&h->q, 8 * nb},
      {(void **)&h->corner, h->nm ? 8 * nb : (size_t)8}, {&h->rho, es * nb}, {&h->t1, es * nb}, {&h->t2, es * nb},
      {&h->czpsi, es * nb}, {&h->szpsi, es * nb}, {&h->xinv, 2 * es * nb}, {&h->x2, es * nb},
      {&h->e4, 4 * es * nb},
      {(void **)&h->suffix, h->nm && !h->macro_direct ? 3 * 8 * nb : (size_t)8}, {(void **)&h->mgrad, (size_t)24 * std::max(h->nm, 1)},
      {(void **)&h->scal, sizeof(double) * S_COUNT}, {(void **)&h->zc, sizeof(ZStageC)},
      {&h->d_lam, 8 * sizeof(double)},
      {(void **)&h->npins, sizeof(float) * nn}, {(void **)&h->nest, sizeof(NestState)},
      {&h->part_n, sizeof(double) * 8 * (size_t)grid_for((long long)nn, 256)},
      {&h->gout, 3 * es * nn}, {(void **)&h->check_flag, sizeof(int)},
      {(void **)&h->tkey, sizeof(int2) * nn},
      {&h->trec, (p->precision == PLACE3D_FP64 ? sizeof(TileRec<double>) : sizeof(TileRec<float>)) * nn},
      {&h->g4, v4 * nn},
      {(void **)&h->tcount, sizeof(int) * kCountPad * (size_t)(h->ntiles + 1)},  // counters, then the ticket
      {(void **)&h->tstart, sizeof(int) * (size_t)(h->ntiles + 1)},
      {(void **)&h->titems, sizeof(int2) * (size_t)std::max(h->max_items, 1)}, {(void **)&h->tnitems, sizeof(int)}};
  for (auto &a : allocs) {
    cudaError_t e = p3d_malloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      cuda_fail(h, e, "cudaMalloc");
      return bail(e == cudaErrorMemoryAllocation ? PLACE3D_ERR_OOM : PLACE3D_ERR_CUDA);
    }
  }
  {
    // partial-sum rows (one per warp) for the largest grids any bucket form
    // may use (G <= 32)
    const int bs = h->precision == PLACE3D_FP64 ? wl_block<double>() : wl_block<float>();
    // rows of any grouping of the classes: a group of c nets writes at most
    // c * G / 32 + bs / 32 rows (G <= 32), the 2-pin form fewer
    size_t rw = 1216 * 8;  // k_norms
    for (const Bucket &b : h->fine) rw += (size_t)b.count + (size_t)bs / 32 + 8;
    const size_t rd = (size_t)std::max(grid_for((long long)h->nx * h->ny, 256), 1) * 8;
    if (p3d_malloc((void **)&h->part_w, sizeof(double) * 4 * rw) != cudaSuccess ||
        p3d_malloc((void **)&h->part_d, sizeof(double) * 3 * rd) != cudaSuccess) {
      fail(h, PLACE3D_ERR_OOM, "cudaMalloc (partial-sum rows)");
      return bail(PLACE3D_ERR_OOM);
    }
  }
  // chunks of the nets above 128 pins (the block-form bucket, G = 0)
  for (const Bucket &b : h->buckets) {
    if (b.G != 0) continue;
    std::vector<int4> chunks;
    std::vector<int2> nets;
    for (int t = 0; t < b.count; ++t) {
      const int e = b.first + t, s0 = new_start[e], d = new_start[e + 1] - s0;
      const int nch = (d + kWlChunk - 1) / kWlChunk;
      nets.push_back(make_int2((int)chunks.size(), nch));
      for (int k = 0; k < nch; ++k) chunks.push_back(make_int4(e, s0 + k * kWlChunk, std::min(kWlChunk, d - k * kWlChunk), t));
    }
    h->big_nchunks = (int)chunks.size();
    h->big_nnets = (int)nets.size();
    const size_t ne = h->precision == PLACE3D_FP64 ? sizeof(NetExt<double>) : sizeof(NetExt<float>);
    const size_t ns = h->precision == PLACE3D_FP64 ? sizeof(Sums<double>) : sizeof(Sums<float>);
    if (p3d_malloc((void **)&h->big_chunk, sizeof(int4) * chunks.size()) != cudaSuccess ||
        p3d_malloc((void **)&h->big_net, sizeof(int2) * nets.size()) != cudaSuccess ||
        p3d_malloc((void **)&h->big_done, sizeof(int) * nets.size()) != cudaSuccess ||
        p3d_malloc(&h->big_ext_part, ne * chunks.size()) != cudaSuccess ||
        p3d_malloc(&h->big_sum_part, ns * chunks.size()) != cudaSuccess ||
        p3d_malloc(&h->big_ext, ne * nets.size()) != cudaSuccess ||
        p3d_malloc(&h->big_sums, ns * nets.size()) != cudaSuccess) {
      fail(h, PLACE3D_ERR_OOM, "cudaMalloc (high-fanout net chunks)");
      return bail(PLACE3D_ERR_OOM);
    }
    if (cudaMemcpy(h->big_chunk, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->big_net, nets.data(), sizeof(int2) * nets.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->big_done, 0, sizeof(int) * nets.size()) != cudaSuccess) {
      fail(h, PLACE3D_ERR_CUDA, "upload failed");
      return bail(PLACE3D_ERR_CUDA);
    }
  }
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_w2a, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_w2b, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithPriority(&h->dens, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_dens, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_param, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithPriority(&h->mac, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_mac, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_field, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_mgrad, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_z, cudaEventDisableTiming) != cudaSuccess) {
    fail(h, PLACE3D_ERR_CUDA, "stream/event creation failed");
    return bail(PLACE3D_ERR_CUDA);
  }
  int rc = h->precision == PLACE3D_FP64 ? upload_typed<double>(h, p, order, new_start)
                                        : upload_typed<float>(h, p, order, new_start);
  if (rc != PLACE3D_OK) return bail(rc);
  {
    std::vector<float> np(nn, 0.0f);
    for (int k = 0; k < p->n_pin; ++k) np[p->pin_inst[k]] += 1.0f;
    if (cudaMemcpy(h->npins, np.data(), sizeof(float) * nn, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->nest, 0, sizeof(NestState)) != cudaSuccess) {
      fail(h, PLACE3D_ERR_CUDA, "upload failed");
      return bail(PLACE3D_ERR_CUDA);
    }
  }
  if (cudaMemcpy(h->flags_d, fl.data(), nn, cudaMemcpyHostToDevice) != cudaSuccess ||
      (h->nm && cudaMemcpy(h->macro_ids, mids.data(), sizeof(int) * h->nm, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(h->macro_slot, mslot.data(), sizeof(int) * nn, cudaMemcpyHostToDevice) != cudaSuccess) {
    fail(h, PLACE3D_ERR_CUDA, "upload failed");
    return bail(PLACE3D_ERR_CUDA);
  }
  ZStageC zc;
  std::memset(&zc, 0, sizeof(zc));
  zc.nx = h->nx;
  zc.ny = h->ny;
  zc.nz = h->nz;
  zc.mode2d = h->mode2d ? 1 : 0;
  const double pi = 3.14159265358979323846;
  zc.pi_dx = pi / h->dx;
  zc.pi_dy = pi / h->dy;
  zc.pi_dz = pi / h->dz;
  // 2D mode: each layer's coefficients are normalised by its own N_x N_y bins
  zc.inv_n = 1.0 / (h->mode2d ? (double)h->nx * h->ny : (double)h->nb);
  zc.pi_dx_f = (float)zc.pi_dx;
  zc.pi_dy_f = (float)zc.pi_dy;
  zc.pi_dz_f = (float)zc.pi_dz;
  zc.inv_n_f = (float)zc.inv_n;
  for (int l = 0; l < h->nz; ++l)
    for (int z = 0; z < h->nz; ++z) {
      const double arg = pi * l * (z + 0.5) / h->nz;
      zc.cz[l * kMaxNz + z] = std::cos(arg);
      zc.sz[l * kMaxNz + z] = (l * pi / h->dz) * std::sin(arg);
      zc.cz_f[l * kMaxNz + z] = (float)zc.cz[l * kMaxNz + z];
      zc.sz_f[l * kMaxNz + z] = (float)zc.sz[l * kMaxNz + z];
    }
  if (cudaMemcpy(h->zc, &zc, sizeof(zc), cudaMemcpyHostToDevice) != cudaSuccess) {
    fail(h, PLACE3D_ERR_CUDA, "upload failed");
    return bail(PLACE3D_ERR_CUDA);
  }
  if (h->tiles && std::max(h->smem_scatter, h->smem_final) > 48 * 1024) {
    // The limit is a property of the kernel, shared by every handle: raise it
    // to the device's opt-in maximum (never lower it, which would break the
    // launches of a handle with larger windows captured earlier)
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    const bool f64 = h->precision == PLACE3D_FP64;
    cudaError_t e1 = f64 ? cudaFuncSetAttribute(k_scatter_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                optin)
                         : cudaFuncSetAttribute(k_scatter_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                optin);
    cudaError_t e2 = f64 ? cudaFuncSetAttribute(k_final_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                optin)
                         : cudaFuncSetAttribute(k_final_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                optin);
    if (e1 != cudaSuccess || e2 != cudaSuccess || (size_t)optin < std::max(h->smem_scatter, h->smem_final)) {
      (void)cudaGetLastError();
      h->tiles = false;
    }
  }
  if (h->precision == PLACE3D_FP32_TC) {
    std::string why;
    h->tc = p3d_tc::create(h->device, h->nx, h->ny, h->nz, h->dx, h->dy, h->dz, h->e4, h->zc, &why);
    if (!h->tc) {
      fail(h, PLACE3D_ERR_UNSUPPORTED, "FP32_TC: " + why);
      return bail(PLACE3D_ERR_UNSUPPORTED);
    }
  }
  {
    const int rl = upload_lam(h);
    if (rl != PLACE3D_OK) return bail(rl);
  }
  *out = h;
  return PLACE3D_OK;
}

int place3d_geometry(const place3d_handle *h, double out[6]) {
  if (!h || !out) return PLACE3D_ERR_INVALID_ARG;
  out[0] = h->wb;
  out[1] = h->hb;
  out[2] = h->db;
  out[3] = h->dx;
  out[4] = h->dy;
  out[5] = h->dz;
  return PLACE3D_OK;
}

// Pack device positions into the handle's float4/double4 buffer (no checks,
// no host copies: usable inside a stream capture).
static int enqueue_pack(place3d_handle *h, const void *px, const void *py, const void *pz, int dtype) {
  cudaStream_t s = h->stream;
  const int n = h->n;
  const int g = grid_for(n, 256);
  if (n == 0) return PLACE3D_OK;
  if (h->precision == PLACE3D_FP64) {
    if (dtype == PLACE3D_F64)
      k_pack<double, double><<<g, 256, 0, s>>>(n, (const double *)px, (const double *)py, (const double *)pz,
                                               as<V4<double>>(h->pos), 0, 0, nullptr);
    else
      k_pack<float, double><<<g, 256, 0, s>>>(n, (const float *)px, (const float *)py, (const float *)pz,
                                              as<V4<double>>(h->pos), 0, 0, nullptr);
  } else {
    if (dtype == PLACE3D_F64)
      k_pack<double, float><<<g, 256, 0, s>>>(n, (const double *)px, (const double *)py, (const double *)pz,
                                              as<V4<float>>(h->pos), 0, 0, nullptr);
    else
      k_pack<float, float><<<g, 256, 0, s>>>(n, (const float *)px, (const float *)py, (const float *)pz,
                                             as<V4<float>>(h->pos), 0, 0, nullptr);
  }
  count_launch(h, ST_PREP);
  return PLACE3D_OK;
}

// Device address of a host array of `bytes` bytes when its first and last
// bytes are both in page-locked host memory the device can address (the
// host memory is then read or written by the kernels directly, over the
// CPU-GPU link, with no staging copy); nullptr for pageable memory.
static const void *host_direct(const void *p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  const void *ends[2] = {p, static_cast<const char *>(p) + bytes - 1};
  const void *dev[2] = {nullptr, nullptr};
  for (int k = 0; k < 2; ++k) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ends[k]) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    dev[k] = a.devicePointer;
  }
  if (static_cast<const char *>(dev[1]) - static_cast<const char *>(dev[0]) != (std::ptrdiff_t)(bytes - 1))
    return nullptr;
  return dev[0];
}

int place3d_set_positions(place3d_handle *h, const void *x, const void *y, const void *z, int dtype, int mem) {
  if (!h) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL handle");
  if (h->n == 0) return PLACE3D_OK;
  if (!x || !y || !z) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL position array");
  if ((dtype != PLACE3D_F64 && dtype != PLACE3D_F32) || (mem != PLACE3D_MEM_HOST && mem != PLACE3D_MEM_DEVICE))
    return fail(h, PLACE3D_ERR_INVALID_ARG, "bad dtype or memory kind");
  P3D_CUDA(h, cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const int n = h->n;
  const size_t eb = dtype == PLACE3D_F64 ? 8 : 4;
  const void *px = x, *py = y, *pz = z;
  StageScope sc(h, ST_PREP, s);
  const void *dx = mem == PLACE3D_MEM_HOST ? host_direct(x, eb * n) : nullptr;
  const void *dy = dx ? host_direct(y, eb * n) : nullptr;
  const void *dz = dy ? host_direct(z, eb * n) : nullptr;
  if (dz) {  // page-locked host arrays: the pack kernel reads them directly
    px = dx;
    py = dy;
    pz = dz;
  } else if (mem == PLACE3D_MEM_HOST) {
    if (!h->stage_in) P3D_CUDA(h, cudaMalloc(&h->stage_in, 3 * 8 * (size_t)n));
    char *st = static_cast<char *>(h->stage_in);
    P3D_CUDA(h, cudaMemcpyAsync(st, x, eb * n, cudaMemcpyHostToDevice, s));
    P3D_CUDA(h, cudaMemcpyAsync(st + eb * n, y, eb * n, cudaMemcpyHostToDevice, s));
    P3D_CUDA(h, cudaMemcpyAsync(st + 2 * eb * n, z, eb * n, cudaMemcpyHostToDevice, s));
    px = st;
    py = st + eb * n;
    pz = st + 2 * eb * n;
  }
  const bool check = h->flags & PLACE3D_FLAG_CHECKS;
  int *bad = check ? h->check_flag : nullptr;
  if (check) P3D_CUDA(h, cudaMemsetAsync(h->check_flag, 0, sizeof(int), s));
  const double zlo = 0.25 * h->dz, zhi = 0.75 * h->dz;
  const int g = grid_for(n, 256);
  if (h->precision == PLACE3D_FP64) {
    if (dtype == PLACE3D_F64)
      k_pack<double, double><<<g, 256, 0, s>>>(n, (const double *)px, (const double *)py, (const double *)pz,
                                               as<V4<double>>(h->pos), zlo, zhi, bad);
    else
      k_pack<float, double><<<g, 256, 0, s>>>(n, (const float *)px, (const float *)py, (const float *)pz,
                                              as<V4<double>>(h->pos), zlo, zhi, bad);
  } else {
    if (dtype == PLACE3D_F64)
      k_pack<double, float><<<g, 256, 0, s>>>(n, (const double *)px, (const double *)py, (const double *)pz,
                                              as<V4<float>>(h->pos), zlo, zhi, bad);
    else
      k_pack<float, float><<<g, 256, 0, s>>>(n, (const float *)px, (const float *)py, (const float *)pz,
                                             as<V4<float>>(h->pos), zlo, zhi, bad);
  }
  count_launch(h, ST_PREP);
  P3D_CUDA(h, cudaGetLastError());
  if (check) {
    int flag = 0;
    P3D_CUDA(h, cudaMemcpyAsync(&flag, h->check_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    P3D_CUDA(h, cudaStreamSynchronize(s));
    if (flag) return fail(h, PLACE3D_ERR_OUT_OF_RANGE, "a position is non-finite or z is outside [d_z/4, 3 d_z/4]");
  }
  return PLACE3D_OK;
}

// Make *exec run `graph` (consumed).  An existing executable graph is
// updated in place when the new capture has the same shape (a parameter or
// buffer change only alters kernel arguments), which costs far less than a
// fresh instantiation; otherwise it is replaced.
static cudaError_t install_graph(cudaGraphExec_t *exec, cudaGraph_t graph) {
  if (*exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(*exec, graph, &info) == cudaSuccess) {
      cudaGraphDestroy(graph);
      return cudaSuccess;
    }
    (void)cudaGetLastError();
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  const cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

// Evaluate (positions already packed) as one CUDA-graph launch on the
// handle's stream, writing the gradient into tgt (device arrays of the
// handle's dtype); recaptured (and the executable graph updated in place)
// when tgt or the parameter version changes.
static int eval_via_graph(place3d_handle *h, void *const tgt[3], bool host_out) {
  const bool same = h->egexec && h->egversion == h->version && h->egptr[0] == tgt[0] && h->egptr[1] == tgt[1] &&
                    h->egptr[2] == tgt[2];
  if (!same) {
    if (!h->cap_stream) P3D_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    P3D_CUDA(h, cudaStreamSynchronize(h->stream));
    cudaStream_t keep = h->stream;
    h->stream = h->cap_stream;
    P3D_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int hdt = h->precision == PLACE3D_FP64 ? PLACE3D_F64 : PLACE3D_F32;
    h->host_out = host_out;
    const int rc = h->precision == PLACE3D_FP64 ? eval_impl<double>(h, tgt[0], tgt[1], tgt[2], hdt, PLACE3D_MEM_DEVICE)
                                                : eval_impl<float>(h, tgt[0], tgt[1], tgt[2], hdt, PLACE3D_MEM_DEVICE);
    h->host_out = false;
    h->stream = keep;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (rc != PLACE3D_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    const cudaError_t ei = install_graph(&h->egexec, graph);
    if (ei != cudaSuccess) return cuda_fail(h, ei, "cudaGraphInstantiate");
    for (int k = 0; k < 3; ++k) h->egptr[k] = tgt[k];
    h->egversion = h->version;
    ++h->captures;
  }
  P3D_CUDA(h, cudaGraphLaunch(h->egexec, h->stream));
  return PLACE3D_OK;
}

int place3d_eval_objective_and_grad(place3d_handle *h, place3d_result *out, void *gx, void *gy, void *gz,
                                    int dtype, int mem) {
  if (!h) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL handle");
  const int ng = (gx != nullptr) + (gy != nullptr) + (gz != nullptr);
  if (ng != 0 && ng != 3) return fail(h, PLACE3D_ERR_INVALID_ARG, "pass all three gradient arrays or none");
  if (ng && ((dtype != PLACE3D_F64 && dtype != PLACE3D_F32) || (mem != PLACE3D_MEM_HOST && mem != PLACE3D_MEM_DEVICE)))
    return fail(h, PLACE3D_ERR_INVALID_ARG, "bad dtype or memory kind");
  P3D_CUDA(h, cudaSetDevice(h->device));
  const int hdt = h->precision == PLACE3D_FP64 ? PLACE3D_F64 : PLACE3D_F32;
  if (!h->profiling && (!ng || dtype == hdt)) {
    // one graph launch into the handle's own gradient buffer (a fixed
    // target: no recapture when the caller's arrays move), then copies
    const size_t es = h->esz, n = (size_t)h->n;
    void *tgt[3] = {h->gout, (char *)h->gout + n * es, (char *)h->gout + 2 * n * es};
    // page-locked host gradient arrays: the final kernel writes them directly
    void *hd[3] = {nullptr, nullptr, nullptr};
    bool direct = ng && mem == PLACE3D_MEM_HOST && n > 0;
    for (int k = 0; k < 3 && direct; ++k) {
      hd[k] = const_cast<void *>(host_direct(k == 0 ? gx : k == 1 ? gy : gz, n * es));
      direct = hd[k] != nullptr;
    }
    if (direct)
      for (int k = 0; k < 3; ++k) tgt[k] = hd[k];
    const int rc = eval_via_graph(h, tgt, direct);
    if (rc != PLACE3D_OK) return rc;
    if (ng && n > 0 && !direct) {
      const cudaMemcpyKind kind = mem == PLACE3D_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
      for (int k = 0; k < 3; ++k)
        P3D_CUDA(h, cudaMemcpyAsync(k == 0 ? gx : k == 1 ? gy : gz, tgt[k], n * es, kind, h->stream));
    }
    h->gout_fresh = !direct;
  } else {
    const int rc = h->precision == PLACE3D_FP64 ? eval_impl<double>(h, gx, gy, gz, dtype, mem)
                                                : eval_impl<float>(h, gx, gy, gz, dtype, mem);
    if (rc != PLACE3D_OK) return rc;
    h->gout_fresh = !(mem == PLACE3D_MEM_DEVICE && ng);  // eval_impl writes device outputs directly
  }
  h->have_result = true;
  if (out || (ng && mem == PLACE3D_MEM_HOST)) {
    P3D_CUDA(h, cudaMemcpyAsync(h->host_scal, h->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, h->stream));
    P3D_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->tc && p3d_tc::error_code(h->tc) != 0)
      return fail(h, PLACE3D_ERR_TIMEOUT, "a tensor-core transform wait expired");
    if (out) fill_result(h, out);
  }
  return PLACE3D_OK;
}

int place3d_get_result(place3d_handle *h, place3d_result *out) {
  if (!h || !out) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL argument");
  if (!h->have_result) return fail(h, PLACE3D_ERR_INVALID_ARG, "no evaluation has been enqueued");
  P3D_CUDA(h, cudaSetDevice(h->device));
  P3D_CUDA(h, cudaStreamSynchronize(h->stream));
  P3D_CUDA(h, cudaMemcpy(h->host_scal, h->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost));
  if (h->tc && p3d_tc::error_code(h->tc) != 0)
    return fail(h, PLACE3D_ERR_TIMEOUT, "a tensor-core transform wait expired");
  fill_result(h, out);
  return PLACE3D_OK;
}

int place3d_copy_map(place3d_handle *h, int which, void *dst, int mem) {
  if (!h || !dst) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL argument");
  P3D_CUDA(h, cudaSetDevice(h->device));
  const void *src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case PLACE3D_MAP_RHO_FIXED: src = h->q; bytes = 8 * h->nb; break;
    case PLACE3D_MAP_EX:
    case PLACE3D_MAP_EY:
    case PLACE3D_MAP_EZ: src = h->e4; bytes = h->esz * h->nb; break;
    default: return fail(h, PLACE3D_ERR_INVALID_ARG, "unknown map");
  }
  if (which != PLACE3D_MAP_RHO_FIXED) {
    // one component of the interleaved (E_x, E_y, E_z, 0) map
    const int comp = which - PLACE3D_MAP_EX;
    std::vector<unsigned char> all(4 * bytes), one(bytes);
    P3D_CUDA(h, cudaStreamSynchronize(h->stream));
    P3D_CUDA(h, cudaMemcpy(all.data(), h->e4, all.size(), cudaMemcpyDeviceToHost));
    for (size_t b = 0; b < h->nb; ++b)
      std::memcpy(one.data() + b * h->esz, all.data() + (4 * b + comp) * h->esz, h->esz);
    if (mem == PLACE3D_MEM_HOST)
      std::memcpy(dst, one.data(), bytes);
    else
      P3D_CUDA(h, cudaMemcpy(dst, one.data(), bytes, cudaMemcpyHostToDevice));
    return PLACE3D_OK;
  }
  if (which == PLACE3D_MAP_RHO_FIXED) {
    // the fixed-point map of the last evaluation = cell counts + prefix-summed macro corners
    std::vector<long long> a(h->nb), c;
    P3D_CUDA(h, cudaStreamSynchronize(h->stream));
    P3D_CUDA(h, cudaMemcpy(a.data(), h->q, bytes, cudaMemcpyDeviceToHost));
    if (h->nm > 0) {
      c.resize(h->nb);
      P3D_CUDA(h, cudaMemcpy(c.data(), h->corner, bytes, cudaMemcpyDeviceToHost));
      // corner holds x/y-scanned corners; finish the z prefix here (integers, exact)
      const size_t pl = (size_t)h->nx * h->ny;
      for (size_t t = 0; t < pl; ++t) {
        long long acc = 0;
        for (int z = 0; z < h->nz; ++z) {
          acc += c[z * pl + t];
          a[z * pl + t] += acc;
        }
      }
    }
    if (mem == PLACE3D_MEM_HOST)
      std::memcpy(dst, a.data(), bytes);
    else
      P3D_CUDA(h, cudaMemcpy(dst, a.data(), bytes, cudaMemcpyHostToDevice));
    return PLACE3D_OK;
  }
  P3D_CUDA(h, cudaStreamSynchronize(h->stream));
  P3D_CUDA(h, cudaMemcpy(dst, src, bytes, mem == PLACE3D_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
  return PLACE3D_OK;
}

int place3d_copy_wl_parts(place3d_handle *h, double *gx, double *gy, double *gfd, double *gwaz) {
  if (!h) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL handle");
  P3D_CUDA(h, cudaSetDevice(h->device));
  P3D_CUDA(h, cudaStreamSynchronize(h->stream));
  const int n = h->n;
  std::vector<double> v(4 * (size_t)n);
  if (h->precision == PLACE3D_FP64) {
    P3D_CUDA(h, cudaMemcpy(v.data(), h->acc, 32 * (size_t)n, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> f(4 * (size_t)n);
    P3D_CUDA(h, cudaMemcpy(f.data(), h->acc, 16 * (size_t)n, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < f.size(); ++k) v[k] = f[k];
  }
  for (int i = 0; i < n; ++i) {
    if (gx) gx[i] = v[4 * i + 0];
    if (gy) gy[i] = v[4 * i + 1];
    if (gfd) gfd[i] = v[4 * i + 2];
    if (gwaz) gwaz[i] = v[4 * i + 3];
  }
  return PLACE3D_OK;
}

// Result scalars on the device (one thread): obj, wl_bi, wl_z, energy,
// hpwl_d2d, n_cross, g_scale, s_x, s_y, s_z (the place3d_result order).
// 2D mode (l2 != NULL): energy = sum of the layer energies ef * S_EL*, obj = wl + sum_l l2[l] U_l.
struct Lam3 {
  double v[3];
};
__global__ void k_result(const double *__restrict__ s, double alpha, double lambda, double ef, int mode2d, Lam3 l2,
                         double *__restrict__ out) {
  double energy = ef * s[S_ESUM], obj = s[S_WL_BI] + alpha * s[S_WL_Z] + lambda * energy;
  if (mode2d) {
    energy = 0.0;
    obj = s[S_WL_BI];
    for (int l = 0; l < 3; ++l) {
      energy += ef * s[S_EL0 + l];
      obj += l2.v[l] * ef * s[S_EL0 + l];
    }
  }
  out[0] = obj;
  out[1] = s[S_WL_BI];
  out[2] = s[S_WL_Z];
  out[3] = energy;
  out[4] = s[S_HPWL];
  out[5] = s[S_NCROSS];
  out[6] = s[S_SZ] > 0 ? (s[S_SX] + s[S_SY]) / (2.0 * s[S_SZ]) : 0.0;
  out[7] = s[S_SX];
  out[8] = s[S_SY];
  out[9] = s[S_SZ];
}

int place3d_result_to_device(place3d_handle *h, double *dst) {
  if (!h || !dst) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL argument");
  P3D_CUDA(h, cudaSetDevice(h->device));
  const double ef = h->mode2d ? 0.5 * (h->wb * h->hb) * (double)h->nx * h->ny
                              : 0.5 * (h->wb * h->hb * h->db) * (double)h->nb;
  Lam3 l2{{h->lam_layer[0], h->lam_layer[1], h->lam_layer[2]}};
  k_result<<<1, 1, 0, h->stream>>>(h->scal, h->alpha, h->lambda, ef, h->mode2d ? 1 : 0, l2, dst);
  P3D_CUDA(h, cudaGetLastError());
  return PLACE3D_OK;
}

int place3d_set_params(place3d_handle *h, double gamma, double gamma_z, double alpha, double lambda) {
  if (!h) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL handle");
  if (!(gamma > 0) || !std::isfinite(gamma) || !std::isfinite(gamma_z) || !std::isfinite(alpha) ||
      !std::isfinite(lambda))
    return fail(h, PLACE3D_ERR_INVALID_ARG, "gamma must be > 0; gamma_z, alpha, lambda finite");
  P3D_CUDA(h, cudaSetDevice(h->device));
  // gamma, gamma_z and alpha are kernel arguments (a change re-captures the
  // graphs at their next launch); lambda is read from the device
  if (gamma != h->gamma || gamma_z != h->gamma_z || alpha != h->alpha) ++h->version;
  h->gamma = gamma;
  h->gamma_z = gamma_z;
  h->alpha = alpha;
  h->lambda = lambda;
  return upload_lam(h);
}

int place3d_set_layer_weights(place3d_handle *h, const double lam[3]) {
  if (!h || !lam) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL argument");
  if (!h->mode2d) return fail(h, PLACE3D_ERR_INVALID_ARG, "layer weights need a 2D-mode handle");
  for (int l = 0; l < 3; ++l)
    if (!std::isfinite(lam[l])) return fail(h, PLACE3D_ERR_INVALID_ARG, "layer weights must be finite");
  P3D_CUDA(h, cudaSetDevice(h->device));
  for (int l = 0; l < 3; ++l) h->lam_layer[l] = lam[l];
  return upload_lam(h);  // read from the device: graphs stay valid
}

int place3d_autotune(place3d_handle *h, int repeats) {
  if (!h) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL handle");
  P3D_CUDA(h, cudaSetDevice(h->device));
  if (repeats < 1) repeats = 3;
  cudaStream_t w = h->side;
  cudaEvent_t e0, e1;
  P3D_CUDA(h, cudaEventCreate(&e0));
  P3D_CUDA(h, cudaEventCreate(&e1));
  P3D_CUDA(h, cudaStreamSynchronize(h->stream));
  // the fastest of `repeats` timed runs of one launch group, after one warm-up run
  auto time_group = [&](const Bucket &b) -> float {
    float ms = 1e30f;
    for (int r = 0; r <= repeats; ++r) {
      cudaEventRecord(e0, w);
      if (h->precision == PLACE3D_FP64)
        launch_wl<double>(h, b, b.G, b.PPL, w, wl_consts<double>(h), as<double>(h->part_w));
      else
        launch_wl<float>(h, b, b.G, b.PPL, w, wl_consts<float>(h), as<float>(h->part_w));
      cudaEventRecord(e1, w);
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) ms = std::min(ms, t);
    }
    return ms;
  };
  // Degree thresholds and forms: the classes up to 128 pins are split into
  // runs of adjacent classes, one launch each.  Every run with every form
  // that fits it is timed alone; best[j] is the least total time of classes
  // 0..j-1 over all splits whose runs span at most `span` classes (dynamic
  // programming over the measured times).
  const int nf = (int)h->fine.size();
  int nd = nf;
  while (nd > 0 && h->fine[nd - 1].dmax > 128) --nd;
  std::vector<float> tt((size_t)nd * nd * kNumForms, -1.0f);  // [i][j][form], -1: does not fit
  bool bad = false;
  for (int j = 0; j < nd && !bad; ++j)
    for (int i = 0; i <= j && !bad; ++i)
      for (int f = 0; f < kNumForms; ++f) {
        const int G = kForms[f][0], PPL = kForms[f][1];
        if (!form_fits(h, h->fine[j].dmax, G, PPL)) continue;
        const float t = time_group(make_group_of(h, i, j, G, PPL));
        if (t < 0) {
          bad = true;
          break;
        }
        tt[((size_t)i * nd + j) * kNumForms + f] = t;
      }
  // near ties between forms of one run (within 3 %) go to the fewest lanes per net
  int lanes[kNumForms];
  for (int f = 0; f < kNumForms; ++f) lanes[f] = kForms[f][0];
  if (!bad) p3d_plan::break_ties(tt, nd, kNumForms, lanes, 0.03f);
  auto plan_for = [&](int span) {
    std::vector<Bucket> groups;
    for (const p3d_plan::Run &r : p3d_plan::best_split(tt, nd, kNumForms, span))
      groups.push_back(make_group_of(h, r.i, r.j, kForms[r.f][0], kForms[r.f][1]));
    if (groups.empty()) return h->buckets;  // some class fits no form: keep the current plan
    if (nd < nf) groups.push_back(make_group_of(h, nd, nf - 1, 0, 0));  // above 128 pins: the chunked form
    return groups;
  };
  // the tensor-core products' tile widths, each product group timed alone
  if (!bad && h->tc && p3d_tc::autotune(h->tc, w, repeats) != 0) bad = true;
  if (!bad && nd > 0) {
    // Candidates: the least total time alone, and the same with runs of at
    // most 2 classes and of single classes.  The wirelength launches run
    // beside the density path, where finer runs can do better than their
    // serial times say, so the candidates are compared by timing whole
    // evaluations (one graph launch each, at the current positions) and the
    // fastest is kept.
    std::vector<std::vector<Bucket>> cand;
    for (int span : {nd, 2, 1}) {
      std::vector<Bucket> g = plan_for(span);
      bool dup = false;
      for (const auto &c : cand) {
        bool same = c.size() == g.size();
        for (size_t k = 0; same && k < g.size(); ++k)
          same = c[k].dmax == g[k].dmax && c[k].G == g[k].G && c[k].PPL == g[k].PPL;
        dup = dup || same;
      }
      if (!dup) cand.push_back(g);
    }
    size_t pick = 0;
    if (cand.size() > 1 && !h->profiling && h->n > 0) {
      const size_t es = h->esz, n = (size_t)h->n;
      void *tgt[3] = {h->gout, (char *)h->gout + n * es, (char *)h->gout + 2 * n * es};
      std::vector<float> tbest(cand.size(), 1e30f);
      const int rounds = std::max(2 * repeats, 6), per = 8;  // the candidates differ by a few percent
      for (int r = 0; r <= rounds && !bad; ++r)  // pass 0 captures and warms up
        for (size_t k = 0; k < cand.size() && !bad; ++k) {
          h->buckets = cand[k];
          ++h->version;
          if (eval_via_graph(h, tgt, false) != PLACE3D_OK) {
            bad = true;
            break;
          }
          cudaEventRecord(e0, h->stream);
          for (int q = 0; q < per; ++q)
            if (eval_via_graph(h, tgt, false) != PLACE3D_OK) bad = true;
          cudaEventRecord(e1, h->stream);
          if (bad || cudaEventSynchronize(e1) != cudaSuccess) {
            bad = true;
            break;
          }
          float t = 0;
          cudaEventElapsedTime(&t, e0, e1);
          if (r > 0) tbest[k] = std::min(tbest[k], t);
        }
      for (size_t k = 1; k < cand.size(); ++k)
        if (tbest[k] < tbest[pick]) pick = k;
      // the timed evaluations ran at the current positions: their results
      // (scalars, and the gradient in the handle's buffer) are the last
      // evaluation's
      h->have_result = !bad;
      h->gout_fresh = !bad;
    }
    h->buckets = cand[pick];
  }
  ++h->version;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (bad) return cuda_fail(h, cudaGetLastError(), "autotune");
  P3D_CUDA(h, cudaGetLastError());
  return PLACE3D_OK;
}

int place3d_set_wl_plan(place3d_handle *h, const int32_t *dmax, const int32_t *lanes, const int32_t *pins,
                        int count) {
  if (!h || count < 0 || (count > 0 && (!dmax || !lanes || !pins)))
    return fail(h, PLACE3D_ERR_INVALID_ARG, "bad launch plan arguments");
  if (count == 0) {
    default_groups(h);
    ++h->version;
    return PLACE3D_OK;
  }
  std::vector<Bucket> groups;
  const int nf = (int)h->fine.size();
  int i = 0;
  for (int g = 0; g < count; ++g) {
    if (i >= nf) return fail(h, PLACE3D_ERR_INVALID_ARG, "the plan has more groups than the netlist's degrees");
    if (h->fine[i].dmax > dmax[g])
      return fail(h, PLACE3D_ERR_INVALID_ARG, "a group's largest degree is below its first class");
    int j = i;
    while (j + 1 < nf && h->fine[j + 1].dmax <= dmax[g]) ++j;
    const Bucket b = make_group_of(h, i, j, lanes[g], pins[g]);
    if (b.dmax != dmax[g] || !form_fits(h, b.dmax, b.G, b.PPL))
      return fail(h, PLACE3D_ERR_INVALID_ARG, "the plan does not match this netlist's degree classes");
    groups.push_back(b);
    i = j + 1;
  }
  if (i != nf) return fail(h, PLACE3D_ERR_INVALID_ARG, "the plan leaves degree classes uncovered");
  h->buckets = groups;
  ++h->version;
  return PLACE3D_OK;
}

int place3d_tc_tiles(const place3d_handle *h, int32_t *cols, int cap) {
  if (!h || !h->tc) return 0;
  for (int k = 0; k < 4 && k < cap; ++k)
    if (cols) cols[k] = p3d_tc::tile_columns(h->tc, k);
  return 4;
}

int place3d_set_tc_tiles(place3d_handle *h, const int32_t *cols, int count) {
  if (!h || !cols || count != 4) return fail(h, PLACE3D_ERR_INVALID_ARG, "four tile widths expected");
  if (!h->tc) return fail(h, PLACE3D_ERR_INVALID_ARG, "the handle has no tensor-core transforms");
  for (int k = 0; k < 4; ++k)
    if (cols[k] != 64 && cols[k] != 128) return fail(h, PLACE3D_ERR_INVALID_ARG, "tile widths are 64 or 128");
  for (int k = 0; k < 4; ++k) p3d_tc::set_tile_columns(h->tc, k, cols[k]);
  ++h->version;
  return PLACE3D_OK;
}

int place3d_set_wl_form(place3d_handle *h, int bucket, int lanes, int pins) {
  if (!h || bucket < 0 || bucket >= (int)h->buckets.size()) return fail(h, PLACE3D_ERR_INVALID_ARG, "bad bucket");
  Bucket &b = h->buckets[bucket];
  if (b.G == 0) return lanes == 0 && pins == 0 ? PLACE3D_OK : fail(h, PLACE3D_ERR_INVALID_ARG, "block-form bucket");
  for (int f = 0; f < kNumForms; ++f)
    if (kForms[f][0] == lanes && kForms[f][1] == pins &&
        (lanes * pins >= b.dmax || (lanes == 1 && pins == 1 && b.dmax == 2 && !h->mode2d))) {
      b.G = lanes;
      b.PPL = pins;
      ++h->version;
      return PLACE3D_OK;
    }
  return fail(h, PLACE3D_ERR_INVALID_ARG, "unsupported form for this bucket");
}

int place3d_wl_forms(const place3d_handle *h, int32_t *dmax, int32_t *lanes, int32_t *pins, int cap) {
  if (!h) return 0;
  int k = 0;
  for (const Bucket &b : h->buckets) {
    if (k < cap) {
      if (dmax) dmax[k] = b.dmax;
      if (lanes) lanes[k] = b.G;
      if (pins) pins[k] = b.PPL;
    }
    ++k;
  }
  return k;
}

// Capture pack + evaluation of one handle on `cs` (the handle's streams are
// redirected to cs for the capture; the side stream forks from it).
static int capture_eval(place3d_handle *h, cudaStream_t cs, const void *const *ptr, int dtype,
                        const BatchHook *bh = nullptr) {
  const bool prof = h->profiling;
  cudaStream_t keep = h->stream;
  h->profiling = false;
  h->stream = cs;
  int rc = bh ? PLACE3D_OK : enqueue_pack(h, ptr[0], ptr[1], ptr[2], dtype);  // (the batch packs)
  if (rc == PLACE3D_OK)
    rc = h->precision == PLACE3D_FP64
             ? eval_impl<double>(h, const_cast<void *>(ptr[3]), const_cast<void *>(ptr[4]), const_cast<void *>(ptr[5]),
                                 dtype, PLACE3D_MEM_DEVICE, bh)
             : eval_impl<float>(h, const_cast<void *>(ptr[3]), const_cast<void *>(ptr[4]), const_cast<void *>(ptr[5]),
                                dtype, PLACE3D_MEM_DEVICE, bh);
  h->stream = keep;
  h->profiling = prof;
  return rc;
}

int place3d_eval_graph(place3d_handle *h, const void *x, const void *y, const void *z, void *gx, void *gy, void *gz,
                       int dtype) {
  if (!h) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL handle");
  if (!x || !y || !z || !gx || !gy || !gz) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL device array");
  if (dtype != PLACE3D_F64 && dtype != PLACE3D_F32) return fail(h, PLACE3D_ERR_INVALID_ARG, "bad dtype");
  P3D_CUDA(h, cudaSetDevice(h->device));
  const void *ptr[6] = {x, y, z, gx, gy, gz};
  bool same = h->gexec && h->gdtype == dtype && h->gversion == h->version;
  for (int k = 0; k < 6 && same; ++k) same = h->gptr[k] == ptr[k];
  if (!same) {
    if (!h->cap_stream) P3D_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    P3D_CUDA(h, cudaStreamSynchronize(h->stream));
    P3D_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = capture_eval(h, h->cap_stream, ptr, dtype);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (rc != PLACE3D_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    const cudaError_t ei = install_graph(&h->gexec, graph);
    if (ei != cudaSuccess) return cuda_fail(h, ei, "cudaGraphInstantiate");
    for (int k = 0; k < 6; ++k) h->gptr[k] = ptr[k];
    h->gdtype = dtype;
    h->gversion = h->version;
    ++h->captures;
  }
  P3D_CUDA(h, cudaGraphLaunch(h->gexec, h->stream));
  h->have_result = true;
  h->gout_fresh = false;
  return PLACE3D_OK;
}

long long place3d_graph_captures(const place3d_handle *h) { return h ? h->captures : -1; }

// ---------------- Nesterov loop helpers ----------------
// The sums dv2, dg2 and gmax start at 0 (create, and k_nest_step clears them
// after each use); the gradient preconditioned is the last evaluation's, in
// the handle's own gradient buffer.
extern "C++" {
template <typename T>
static int nest_precond(place3d_handle *h, void *gx, void *gy, void *gz, double init_step) {
  cudaStream_t s = h->stream;
  const int n = h->n, g = grid_for(n, 256);
  if (n > 0) {
    const T *G = as<T>(h->gout);
    k_nest_precond<T><<<g, 256, 0, s>>>(n, G, G + n, G + 2 * (size_t)n, (T *)gx, (T *)gy, (T *)gz,
                                        as<V4<T>>(h->pos), as<V4<T>>(h->size), h->flags_d, h->npins, lam_dev<T>(h),
                                        (T)(0.5 * h->dz), (T)(0.5 * h->dz), as<T>(h->part_n),
                                        init_step > 0 ? &h->nest->gmax_bits : nullptr);
    k_sum_parts<1, T><<<sum_grid(g * 8), 256, 0, s>>>(as<T>(h->part_n), g * 8, &h->nest->dg2);
  }
  k_nest_step<<<1, 1, 0, s>>>(h->nest, init_step);
  P3D_CUDA(h, cudaGetLastError());
  return PLACE3D_OK;
}
}  // extern "C++"

static int nest_check(place3d_handle *h, const void *const *ptrs, int count, bool need_grad) {
  if (!h) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL handle");
  if (h->mode2d) return fail(h, PLACE3D_ERR_INVALID_ARG, "the Nesterov helpers need a 3D-mode handle");
  for (int k = 0; k < count; ++k)
    if (!ptrs[k] && h->n > 0) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL device array");
  if (need_grad && !h->gout_fresh)
    return fail(h, PLACE3D_ERR_INVALID_ARG,
                "the last evaluation did not keep its gradient in the handle (see place3d_nesterov_precondition)");
  P3D_CUDA(h, cudaSetDevice(h->device));
  return PLACE3D_OK;
}

int place3d_nesterov_precondition(place3d_handle *h, void *gx, void *gy, void *gz) {
  const void *ptrs[3] = {gx, gy, gz};
  const int rc = nest_check(h, ptrs, 3, true);
  if (rc != PLACE3D_OK) return rc;
  return h->precision == PLACE3D_FP64 ? nest_precond<double>(h, gx, gy, gz, 0.0)
                                      : nest_precond<float>(h, gx, gy, gz, 0.0);
}

int place3d_nesterov_init(place3d_handle *h, void *gx, void *gy, void *gz, double init_step) {
  const void *ptrs[3] = {gx, gy, gz};
  const int rc = nest_check(h, ptrs, 3, true);
  if (rc != PLACE3D_OK) return rc;
  if (!(init_step > 0) || !std::isfinite(init_step)) return fail(h, PLACE3D_ERR_INVALID_ARG, "init_step must be > 0");
  const size_t es = h->esz * (size_t)h->n;
  cudaStream_t s = h->stream;
  for (void *p : {gx, gy, gz})  // the previous preconditioned gradient starts at 0
    if (es) P3D_CUDA(h, cudaMemsetAsync(p, 0, es, s));
  return h->precision == PLACE3D_FP64 ? nest_precond<double>(h, gx, gy, gz, init_step)
                                      : nest_precond<float>(h, gx, gy, gz, init_step);
}

extern "C++" {
template <typename T>
static int nest_update(place3d_handle *h, void *const *u, void *const *v, const void *const *g, double coef) {
  cudaStream_t s = h->stream;
  const int n = h->n, gr = grid_for(n, 256);
  NestBox<T> b;
  b.lo[0] = (T)h->xl;
  b.hi[0] = (T)h->xh;
  b.lo[1] = (T)h->yl;
  b.hi[1] = (T)h->yh;
  b.lo[2] = (T)(0.25 * h->dz);
  b.hi[2] = (T)(0.75 * h->dz);
  if (n > 0) {
    k_nest_update<T><<<gr, 256, 0, s>>>(n, (T *)u[0], (T *)u[1], (T *)u[2], (T *)v[0], (T *)v[1], (T *)v[2],
                                        (const T *)g[0], (const T *)g[1], (const T *)g[2], h->nest, (T)coef, b,
                                        as<V4<T>>(h->pos), as<T>(h->part_n));
    k_sum_parts<1, T><<<sum_grid(gr * 8), 256, 0, s>>>(as<T>(h->part_n), gr * 8, &h->nest->dv2);
  }
  P3D_CUDA(h, cudaGetLastError());
  return PLACE3D_OK;
}
}  // extern "C++"

int place3d_nesterov_update(place3d_handle *h, void *ux, void *uy, void *uz, void *vx, void *vy, void *vz,
                            const void *gx, const void *gy, const void *gz, double coef) {
  const void *ptrs[9] = {ux, uy, uz, vx, vy, vz, gx, gy, gz};
  const int rc = nest_check(h, ptrs, 9, false);
  if (rc != PLACE3D_OK) return rc;
  if (!std::isfinite(coef)) return fail(h, PLACE3D_ERR_INVALID_ARG, "coef must be finite");
  void *u[3] = {ux, uy, uz}, *v[3] = {vx, vy, vz};
  const void *g[3] = {gx, gy, gz};
  return h->precision == PLACE3D_FP64 ? nest_update<double>(h, u, v, g, coef) : nest_update<float>(h, u, v, g, coef);
}

int place3d_nesterov_step(place3d_handle *h, double *step) {
  if (!h || !step) return fail(h, PLACE3D_ERR_INVALID_ARG, "NULL argument");
  P3D_CUDA(h, cudaSetDevice(h->device));
  NestState st;
  P3D_CUDA(h, cudaMemcpyAsync(&st, h->nest, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  P3D_CUDA(h, cudaStreamSynchronize(h->stream));
  *step = st.step;
  return PLACE3D_OK;
}

int place3d_set_profiling(place3d_handle *h, int on) {
  if (!h) return PLACE3D_ERR_INVALID_ARG;
  h->profiling = on != 0;
  return PLACE3D_OK;
}

int place3d_num_stages(void) { return ST_COUNT; }

const char *place3d_stage_name(int stage) {
  return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : "";
}

int place3d_stage_times(place3d_handle *h, double *ms, int64_t *launches, int64_t *evals, int reset) {
  if (!h) return PLACE3D_ERR_INVALID_ARG;
  P3D_CUDA(h, cudaSetDevice(h->device));
  for (auto &e : h->ev_live) {
    P3D_CUDA(h, cudaEventSynchronize(e.b));
    float t = 0;
    P3D_CUDA(h, cudaEventElapsedTime(&t, e.a, e.b));
    h->stage_ms[e.stage] += t;
    h->ev_pool.push_back(e);
  }
  h->ev_live.clear();
  for (int k = 0; k < ST_COUNT; ++k) {
    if (ms) ms[k] = h->stage_ms[k];
    if (launches) launches[k] = h->stage_launch[k];
  }
  if (evals) *evals = h->prof_evals;
  if (reset) {
    std::memset(h->stage_ms, 0, sizeof(h->stage_ms));
    std::memset(h->stage_launch, 0, sizeof(h->stage_launch));
    h->prof_evals = 0;
  }
  return PLACE3D_OK;
}

int place3d_launches_per_eval(const place3d_handle *h) { return h ? h->launches : 0; }

struct place3d_batch {
  std::vector<place3d_handle *> hs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaStream_t root = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void *> ptrs;
  std::vector<unsigned> versions;  // each handle's parameter version at capture
  int dtype = -1, device = 0;
  std::string err;
  // shared wirelength stage (one launch per stage for every instance):
  // its stream, the events after the packing and after the stage, the
  // per-instance descriptors and the block-prefix tables of its launches
  bool shared_wl = false;
  cudaStream_t wls = nullptr;
  cudaEvent_t ev_prep = nullptr, ev_wl = nullptr;
  BWl *d_wl = nullptr;
  int *d_tab = nullptr;
};

// Host plan of the shared wirelength stage: per launch, its kernel form,
// its grid, and the offset of its block-prefix table in d_tab.
struct BatchWlPlan {
  int ngroups = 0;
  int G[kBatchGroups], PPL[kBatchGroups];
  int grid[kBatchGroups + 4], tab[kBatchGroups + 4];  // groups, then prep, sum, norms, norm sums
  int norm_rows_tab = 0;                              // offset of the per-instance norm-row counts
};

static void batch_free(place3d_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->wls) cudaStreamDestroy(b->wls);
  if (b->ev_prep) cudaEventDestroy(b->ev_prep);
  if (b->ev_wl) cudaEventDestroy(b->ev_wl);
  if (b->d_wl) cudaFree(b->d_wl);
  if (b->d_tab) cudaFree(b->d_tab);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->root) cudaStreamDestroy(b->root);
  delete b;
}

int place3d_batch_create(place3d_handle *const *handles, int count, place3d_batch **out) {
  if (!handles || count < 1 || !out) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  const int dev = handles[0] ? handles[0]->device : -1;
  for (int i = 0; i < count; ++i)
    if (!handles[i] || handles[i]->device != dev)
      return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "batch handles must be non-NULL and on one device");
  if (cudaSetDevice(dev) != cudaSuccess) return fail(nullptr, PLACE3D_ERR_CUDA, "cudaSetDevice failed");
  place3d_batch *b = new place3d_batch();
  b->device = dev;
  b->hs.assign(handles, handles + count);
  bool ok = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < count && ok; ++i) {
    cudaStream_t s;
    cudaEvent_t e;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
      b->streams.push_back(s);
      b->done.push_back(e);
    }
  }
  if (!ok) {
    batch_free(b);
    return fail(nullptr, PLACE3D_ERR_CUDA, "batch stream/event creation failed");
  }
  *out = b;
  return PLACE3D_OK;
}

// Whether every instance can join the shared wirelength stage (FP32
// arithmetic, 3D mode, float positions, no net above 128 pins), and the
// common launch groups: the plan of the instance with the most nets, if its
// forms fit every instance's degree classes, else the default plan.
static bool batch_wl_plan(const place3d_batch *b, int dtype, BatchWlPlan &pl, std::vector<BWl> &desc,
                          std::vector<int> &tab, const std::vector<const void *> &ptr) {
  if (dtype != PLACE3D_F32) return false;
  const place3d_handle *big = nullptr;
  for (const place3d_handle *h : b->hs) {
    if (h->precision == PLACE3D_FP64 || h->mode2d || h->profiling) return false;
    if (!h->fine.empty() && h->fine.back().dmax > 128) return false;
    if (!big || h->nnet > big->nnet) big = h;
  }
  std::vector<int> bound, fg, fp;
  for (const Bucket &g : big->buckets) {
    bound.push_back(g.dmax);
    fg.push_back(g.G);
    fp.push_back(g.PPL);
  }
  if (!bound.empty()) bound.back() = 128;  // the last group takes every class up to 128 pins
  auto fits = [&](void) {
    for (const place3d_handle *h : b->hs)
      for (const Bucket &c : h->fine) {
        size_t g = 0;
        while (g < bound.size() && c.dmax > bound[g]) ++g;
        if (g == bound.size() || !form_fits(h, c.dmax, fg[g], fp[g])) return false;
      }
    return true;
  };
  if (bound.empty() || (int)bound.size() > kBatchGroups || !fits()) {
    bound.assign(kDefaultGroupMax, kDefaultGroupMax + 7);
    fg.clear();
    fp.clear();
    for (int g = 0; g < 7; ++g) {
      fg.push_back(kDefaultForm[g][0]);
      fp.push_back(kDefaultForm[g][1]);
    }
    if (!fits()) return false;
  }
  const int ng = (int)bound.size(), nh = (int)b->hs.size();
  pl.ngroups = ng;
  for (int g = 0; g < ng; ++g) {
    pl.G[g] = fg[g];
    pl.PPL[g] = fp[g];
  }
  desc.assign(nh, BWl{});
  std::vector<std::vector<int>> blocks(ng + 4, std::vector<int>(nh, 0));
  std::vector<int> nrows(nh, 0);
  constexpr int BS = wl_block<float>();
  for (int i = 0; i < nh; ++i) {
    const place3d_handle *h = b->hs[i];
    BWl &w = desc[i];
    w.n = h->n;
    w.x = (const float *)ptr[6 * i];
    w.y = (const float *)ptr[6 * i + 1];
    w.z = (const float *)ptr[6 * i + 2];
    w.pos = as<V4<float>>(h->pos);
    w.acc = as<V4<float>>(h->acc);
    w.off = as<V4<float>>(h->off);
    w.net_start = h->net_start;
    w.pin_inst = h->pin_inst;
    w.part = as<float>(h->part_w);
    w.scal = h->scal;
    w.c = wl_consts<float>(h);
    int row = 0;
    size_t k = 0;
    for (int g = 0; g < ng; ++g) {
      w.gfirst[g] = w.gcount[g] = w.gpin0[g] = 0;
      bool first = true;
      while (k < h->fine.size() && h->fine[k].dmax <= bound[g]) {
        if (first) {
          w.gfirst[g] = h->fine[k].first;
          w.gpin0[g] = h->fine[k].pin0;
          first = false;
        }
        w.gcount[g] += h->fine[k].count;
        ++k;
      }
      const bool pair = fg[g] == 1 && fp[g] == 1;
      const int nb = w.gcount[g] == 0 ? 0
                     : pair       ? grid_for(w.gcount[g], 256 * kPairNets)
                                  : grid_for((long long)w.gcount[g] * fg[g], BS);
      blocks[g][i] = nb;
      w.grow[g] = row;
      row += nb * (pair ? 256 / 32 : BS / 32);
    }
    w.rows_wl = row;
    const int gn = std::min(grid_for(std::max(h->n, 1), 256), 1216);
    blocks[ng][i] = std::min(grid_for(std::max(h->n, 1), 256), 1024);  // prep
    blocks[ng + 1][i] = sum_grid(std::max(row, 1));                     // WL rows -> scalars
    blocks[ng + 2][i] = gn;                                              // norms
    nrows[i] = gn * 8;
    blocks[ng + 3][i] = sum_grid(gn * 8);                                // norm rows -> scalars
  }
  tab.clear();
  for (int l = 0; l < ng + 4; ++l) {
    pl.tab[l] = (int)tab.size();
    int acc = 0;
    for (int i = 0; i < nh; ++i) {
      tab.push_back(acc);
      acc += blocks[l][i];
    }
    tab.push_back(acc);
    pl.grid[l] = acc;
  }
  pl.norm_rows_tab = (int)tab.size();
  tab.insert(tab.end(), nrows.begin(), nrows.end());
  return true;
}

// The shared wirelength stage's launches on stream w.
static void batch_wl_launch(const place3d_batch *b, const BatchWlPlan &pl, cudaStream_t w) {
  const int nh = (int)b->hs.size(), ng = pl.ngroups;
  for (int g = 0; g < ng; ++g) {
    const int grid = pl.grid[g];
    if (grid == 0) continue;
    const int *t = b->d_tab + pl.tab[g];
    const int G = pl.G[g], PPL = pl.PPL[g];
    if (G == 1 && PPL == 1) {
      k_b_wl_pair<<<grid, 256, 0, w>>>(b->d_wl, t, nh, g);
      continue;
    }
#define P3D_BWL(GG, PP) \
  if (G == GG && PPL == PP) k_b_wl_group<GG, PP><<<grid, wl_block<float>(), 0, w>>>(b->d_wl, t, nh, g);
    P3D_BWL(1, 2) P3D_BWL(1, 4) P3D_BWL(2, 2) P3D_BWL(4, 1) P3D_BWL(2, 4) P3D_BWL(8, 1) P3D_BWL(4, 4)
    P3D_BWL(16, 1) P3D_BWL(8, 4) P3D_BWL(32, 1) P3D_BWL(16, 4) P3D_BWL(32, 2) P3D_BWL(32, 4)
#undef P3D_BWL
  }
  k_b_sum_wl<<<pl.grid[ng + 1], 256, 0, w>>>(b->d_wl, b->d_tab + pl.tab[ng + 1], nh);
  k_b_norms<<<pl.grid[ng + 2], 256, 0, w>>>(b->d_wl, b->d_tab + pl.tab[ng + 2], nh);
  k_b_sum_norms<<<pl.grid[ng + 3], 256, 0, w>>>(b->d_wl, b->d_tab + pl.tab[ng + 3], b->d_tab + pl.norm_rows_tab,
                                                 nh);
}

int place3d_batch_eval(place3d_batch *b, const void *const *xs, const void *const *ys, const void *const *zs,
                       void *const *gxs, void *const *gys, void *const *gzs, int dtype, void *cuda_stream) {
  if (!b || !xs || !ys || !zs || !gxs || !gys || !gzs) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL argument");
  if (dtype != PLACE3D_F64 && dtype != PLACE3D_F32) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "bad dtype");
  P3D_CUDA(nullptr, cudaSetDevice(b->device));
  const int n = (int)b->hs.size();
  std::vector<const void *> ptr;
  for (int i = 0; i < n; ++i) {
    const void *pi[6] = {xs[i], ys[i], zs[i], gxs[i], gys[i], gzs[i]};
    for (int k = 0; k < 6; ++k) {
      if (!pi[k]) return fail(nullptr, PLACE3D_ERR_INVALID_ARG, "NULL instance array");
      ptr.push_back(pi[k]);
    }
  }
  std::vector<unsigned> vers;
  for (auto *h : b->hs) vers.push_back(h->version);
  if (!b->exec || b->dtype != dtype || b->ptrs != ptr || b->versions != vers) {
    for (auto *h : b->hs) P3D_CUDA(nullptr, cudaStreamSynchronize(h->stream));
    // shared wirelength stage: descriptors and block tables uploaded before
    // the capture (they hold this capture's pointers and plans)
    BatchWlPlan pl;
    std::vector<BWl> desc;
    std::vector<int> tab;
    b->shared_wl = batch_wl_plan(b, dtype, pl, desc, tab, ptr);
    if (b->shared_wl) {
      if (!b->wls) {
        P3D_CUDA(nullptr, cudaStreamCreateWithFlags(&b->wls, cudaStreamNonBlocking));
        P3D_CUDA(nullptr, cudaEventCreateWithFlags(&b->ev_prep, cudaEventDisableTiming));
        P3D_CUDA(nullptr, cudaEventCreateWithFlags(&b->ev_wl, cudaEventDisableTiming));
      }
      if (b->d_wl) cudaFree(b->d_wl);
      if (b->d_tab) cudaFree(b->d_tab);
      b->d_wl = nullptr;
      b->d_tab = nullptr;
      P3D_CUDA(nullptr, cudaMalloc((void **)&b->d_wl, sizeof(BWl) * desc.size()));
      P3D_CUDA(nullptr, cudaMalloc((void **)&b->d_tab, sizeof(int) * tab.size()));
      P3D_CUDA(nullptr, cudaMemcpy(b->d_wl, desc.data(), sizeof(BWl) * desc.size(), cudaMemcpyHostToDevice));
      P3D_CUDA(nullptr, cudaMemcpy(b->d_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice));
    }
    P3D_CUDA(nullptr, cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal));
    int rc = PLACE3D_OK;
    std::string why;
    cudaError_t ce = cudaEventRecord(b->fork, b->root);
    if (ce != cudaSuccess) {
      rc = PLACE3D_ERR_CUDA;
      why = std::string("cudaEventRecord(fork): ") + cudaGetErrorString(ce);
    }
    BatchHook hook{b->ev_wl};
    cudaEvent_t start = b->fork;
    if (rc == PLACE3D_OK && b->shared_wl) {
      // scalars and accumulators zeroed, positions packed: one launch, then
      // the wirelength stage of every instance on its own stream
      const int ng = pl.ngroups;
      k_b_prep<<<pl.grid[ng], 256, 0, b->root>>>(b->d_wl, b->d_tab + pl.tab[ng], n);
      if ((ce = cudaGetLastError()) != cudaSuccess || (ce = cudaEventRecord(b->ev_prep, b->root)) != cudaSuccess ||
          (ce = cudaStreamWaitEvent(b->wls, b->ev_prep, 0)) != cudaSuccess) {
        rc = PLACE3D_ERR_CUDA;
        why = std::string("shared wirelength stage: ") + cudaGetErrorString(ce);
      } else {
        batch_wl_launch(b, pl, b->wls);
        if ((ce = cudaGetLastError()) != cudaSuccess || (ce = cudaEventRecord(b->ev_wl, b->wls)) != cudaSuccess) {
          rc = PLACE3D_ERR_CUDA;
          why = std::string("shared wirelength stage: ") + cudaGetErrorString(ce);
        }
      }
      start = b->ev_prep;
    }
    for (int i = 0; i < n && rc == PLACE3D_OK; ++i) {
      if ((ce = cudaStreamWaitEvent(b->streams[i], start, 0)) != cudaSuccess) {
        rc = PLACE3D_ERR_CUDA;
        why = std::string("cudaStreamWaitEvent(fork): ") + cudaGetErrorString(ce);
        break;
      }
      rc = capture_eval(b->hs[i], b->streams[i], &ptr[6 * i], dtype, b->shared_wl ? &hook : nullptr);
      if (rc != PLACE3D_OK) {
        why = "instance " + std::to_string(i) + ": " + b->hs[i]->err;
        break;
      }
      if ((ce = cudaEventRecord(b->done[i], b->streams[i])) != cudaSuccess ||
          (ce = cudaStreamWaitEvent(b->root, b->done[i], 0)) != cudaSuccess) {
        rc = PLACE3D_ERR_CUDA;
        why = std::string("joining instance ") + std::to_string(i) + ": " + cudaGetErrorString(ce);
      }
    }
    if (rc == PLACE3D_OK && b->shared_wl && (ce = cudaStreamWaitEvent(b->root, b->ev_wl, 0)) != cudaSuccess) {
      rc = PLACE3D_ERR_CUDA;
      why = std::string("joining the shared wirelength stage: ") + cudaGetErrorString(ce);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->root, &graph);
    if (rc != PLACE3D_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (rc != PLACE3D_OK) return fail(nullptr, rc, "batch capture: " + why);
      return cuda_fail(nullptr, e, "cudaStreamEndCapture (batch)");
    }
    P3D_CUDA(nullptr, install_graph(&b->exec, graph));
    b->ptrs = ptr;
    b->versions = vers;
    b->dtype = dtype;
  }
  // density weights written by set_params on the handles' streams come first
  for (auto *h : b->hs) P3D_CUDA(nullptr, cudaStreamWaitEvent(static_cast<cudaStream_t>(cuda_stream), h->ev_param, 0));
  P3D_CUDA(nullptr, cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)));
  for (auto *h : b->hs) {
    h->have_result = true;
    h->gout_fresh = false;
  }
  return PLACE3D_OK;
}

int place3d_batch_shared_stages(const place3d_batch *b) { return b && b->exec && b->shared_wl ? 1 : 0; }

void place3d_batch_destroy(place3d_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  batch_free(b);
}

const char *place3d_last_error(const place3d_handle *h) { return h ? h->err.c_str() : g_thread_err.c_str(); }

void place3d_destroy(place3d_handle *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->side2) cudaStreamSynchronize(h->side2);
  if (h->dens) cudaStreamSynchronize(h->dens);
  free_all(h);
  delete h;
}

}  // extern "C"
