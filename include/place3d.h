/*
 * place3d: one evaluation of the 3D die-to-die placement objective and its
 * gradient on a GB300 GPU (sm_103a), after "Analytical Heterogeneous
 * Die-to-Die 3D Placement with Macros" (arXiv 2403.09070).
 *
 * The objective (eq. analytical-placement with the wirelength of eq.
 * wl-model) is
 *
 *     f(x, y, z) = sum_e W^_e,Bi + alpha sum_e p^_e(z) + lambda U^
 *
 * - W^_e,Bi: bistratal weighted-average wirelength, eq. wl-obj with every
 *   partial HPWL p() smoothed by eq. wa-model-approx (Sec. III-A);
 * - p^_e(z): the WA depth span that models the HBT cost (eq. wl-model);
 * - U^: eDensity3D energy (Sec. III-A), density by eq. density-map-accum
 *   (cells) and Theorem 1 (macros), potential and field by eqs. density-coef,
 *   poisson-sol-potential and possion-sol-force.
 *
 * The gradient returned is (d/dx, d/dy, g + alpha d p^(z)/dz) of the
 * wirelength (eq. fda-normalize, with g the normalised FD depth gradient of
 * eq. fda-grad) plus lambda times the density force (field gather).
 *
 * Conventions for every entry point:
 * - Return value: PLACE3D_OK (0) or a negative PLACE3D_ERR_* code; the
 *   message is available from place3d_last_error().
 * - A handle is not thread-safe; use one handle per host thread.  All GPU
 *   work of a handle is enqueued on the stream given at creation.
 * - Device pointers passed in are used in place on that stream (no copy);
 *   host pointers are copied.  The caller owns every buffer it passes.
 */
#ifndef PLACE3D_H
#define PLACE3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PLACE3D_OK 0
#define PLACE3D_ERR_INVALID_ARG (-1) /* NULL pointer, bad size, bad enum */
#define PLACE3D_ERR_BAD_CSR (-2)     /* net_start/pin_inst inconsistent */
#define PLACE3D_ERR_OUT_OF_RANGE (-3) /* value outside its domain (checks) */
#define PLACE3D_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define PLACE3D_ERR_OOM (-5)         /* device allocation failed */
#define PLACE3D_ERR_TIMEOUT (-6)     /* a bounded device-side wait gave up */
#define PLACE3D_ERR_UNSUPPORTED (-7) /* mode not available on this device */

/* ---- precision modes (place3d_problem.precision) ---- */
#define PLACE3D_FP64 0    /* every step in FP64 (the plain path) */
#define PLACE3D_FP32 1    /* FP32 steps, FP32 CUDA-core transforms, FP64 scalars */
#define PLACE3D_FP32_TC 2 /* FP32 steps, split-BF16 tcgen05 transforms */

/* ---- flags (place3d_problem.flags) ---- */
#define PLACE3D_FLAG_CHECKS 1 /* validate positions on every set_positions */
/* Macro field gather: by default the library picks the bin-parallel direct
 * form when the macros cover fewer bins than twice the grid, else Theorem 1's
 * adjoint (suffix sums of the field, 8 corners per macro, Sec. IV-A).  These
 * flags force one form (both give the same gradient up to rounding). */
#define PLACE3D_FLAG_MACRO_GATHER_SCAN 2
#define PLACE3D_FLAG_MACRO_GATHER_DIRECT 4
/* Run the wirelength path on the caller's stream after the density path
 * instead of concurrently on a second stream (for profiling one kernel at a
 * time). */
#define PLACE3D_FLAG_SERIAL 8
/* Cell scatter and field gather.  By default the std cells are sorted per
 * evaluation by the 16x16-bin tile holding their centre (a counting sort)
 * and scattered / gathered through shared-memory windows of a tile plus a
 * halo, one block per chunk of a tile (Sec. IV-A's instance parallelism for
 * std cells, with the charge staged in shared memory: global atomics once
 * per window bin instead of once per cell and bin).  PLACE3D_FLAG_NO_TILES
 * uses one thread per cell
 * with global int64 atomics and global field loads instead.  Both give the
 * same fixed-point map bit for bit and the same gradient up to rounding.
 * The tiled form is the default in 3D mode from 100,000 instances up (below
 * that the sort's extra launches cost more than they save, and in 2D mode an
 * instance covers too few bins for the sort to pay); PLACE3D_FLAG_TILES asks
 * for it in any case.  It needs fewer than 2^24 instances, at most 8192
 * tiles and a halo of at most 8 bins (cells at most ~16 bins wide);
 * otherwise the per-cell form is used.  An evaluation whose gradient goes
 * to page-locked host arrays gathers per cell (its host stores then overlap
 * the computation) after the tiled scatter. */
#define PLACE3D_FLAG_TILES 16
#define PLACE3D_FLAG_NO_TILES 32

/* ---- placement mode (place3d_problem.mode) ---- */
#define PLACE3D_MODE_3D 0 /* 3D mixed-size placement, eq. analytical-placement */
#define PLACE3D_MODE_2D 1 /* multi-die 2D placement, eq. 2d-place */

/* ---- dtype and memory kind of caller buffers ---- */
#define PLACE3D_F64 0
#define PLACE3D_F32 1
#define PLACE3D_MEM_HOST 0
#define PLACE3D_MEM_DEVICE 1

/*
 * Problem statement (Sec. II-B "Problem Formulation", Sec. III-A, Sec. V-A).
 * All arrays are HOST arrays, read during place3d_create() only (deep copy).
 *
 * Instances i in [0, n_inst): std cells, macros and fillers.  Sizes are per
 * die: (w_bot, h_bot) on the bottom die, (w_top, h_top) on the top die
 * (eq. std-size-tech for cells; eq. macro-size-tech interpolates macros).
 * Fillers are instances without pins; z_fixed marks instances whose
 * z-gradient is forced to 0 (Sec. III-A z-fixed fillers).
 *
 * Netlist: CSR over nets; net e owns pins [net_start[e], net_start[e+1]),
 * pin p sits on instance pin_inst[p] at offset (pin_off_bot_x/y) from its
 * centre on the bottom die and (pin_off_top_x/y) on the top die (offsets
 * follow the partition, Sec. III-A).  An instance may hold at most one pin
 * of a net.  Nets with fewer than 2 pins contribute nothing.
 *
 * Region and bins: Omega = [xl,xh] x [yl,yh] x [0,d_z] with N_x x N_y x N_z
 * bins, w_b = (xh-xl)/N_x, h_b = (yh-yl)/N_y, d_b = (w_b+h_b)/2 and
 * d_z = N_z d_b (Sec. V-A).  Instance depth is d_z/2, movable
 * z in [d_z/4, 3 d_z/4] (Sec. III-A).
 *
 * gamma: WA smoothing of x and y; gamma_z: of z (<= 0 means gamma).
 * alpha: HBT weight of eq. wl-model (place3d_alpha() gives the paper's
 * default); lambda: density weight of eq. analytical-placement.
 */
typedef struct place3d_problem {
  int32_t n_inst;
  const uint8_t *is_macro; /* [n_inst] 1 = macro */
  const uint8_t *z_fixed;  /* [n_inst] 1 = z-gradient forced to 0; may be NULL */
  const double *w_bot, *h_bot, *w_top, *h_top; /* [n_inst] */
  int32_t n_net, n_pin;
  const int32_t *net_start; /* [n_net+1], net_start[0]=0, nondecreasing, last=n_pin */
  const int32_t *pin_inst;  /* [n_pin], values in [0, n_inst) */
  const double *pin_off_bot_x, *pin_off_bot_y; /* [n_pin] offsets on the bottom die */
  const double *pin_off_top_x, *pin_off_top_y; /* [n_pin] offsets on the top die */
  double xl, yl, xh, yh;
  int32_t nx, ny, nz;
  double gamma, gamma_z;
  double alpha, lambda;
  int32_t precision; /* PLACE3D_FP64 | PLACE3D_FP32 | PLACE3D_FP32_TC */
  int32_t flags;     /* PLACE3D_FLAG_* */
  /* Multi-die 2D global placement (Sec. V-B, eq. 2d-place) when mode =
   * PLACE3D_MODE_2D; zero-initialise these three for the 3D placer.
   * In 2D mode the grid has nz = 3 layers (0 bottom die, 1 top die, 2 HBT
   * layer), each an independent 2D electrostatic field; the partition is
   * fixed: a non-HBT instance is on the top die iff z > d_z/2 (d_z = 3 d_b),
   * its footprint is that die's (macros too).  is_hbt marks the hybrid
   * bonding terminals: instances of the HBT layer with footprint w_bot x
   * h_bot whose pins (one per crossing net, offsets normally 0) belong to
   * both partial nets (eq. exact-wirelength).  lam_layer weights the three
   * layers' energies; lambda is not used.  There is no z-gradient (0). */
  int32_t mode;           /* PLACE3D_MODE_3D (0) | PLACE3D_MODE_2D (1) */
  const uint8_t *is_hbt;  /* [n_inst] or NULL; 2D mode only */
  double lam_layer[3];    /* 2D mode: (lambda-, lambda+, lambda') */
} place3d_problem;

/* Scalars of one evaluation (FP64). */
typedef struct place3d_result {
  double obj;      /* f = wl_bi + alpha wl_z + lambda energy */
  double wl_bi;    /* sum_e W^_e,Bi (eq. wl-obj on WA-smoothed spans) */
  double wl_z;     /* sum_e p^_e(z) (eq. wl-model, unscaled) */
  double energy;   /* U^ = 1/2 vol(b) sum_b rho_b phi_b */
  double hpwl_d2d; /* exact D2D HPWL, sum_e W_ex + W_ey (eq. wl-obj) */
  double n_cross;  /* #crossing nets = sum_e C_e (Sec. II-B), i.e. #HBTs */
  double g_scale;  /* (S_x + S_y) / (2 S_z) of eq. fda-normalize (0 if S_z = 0) */
  double s_x, s_y, s_z; /* L1 norms of the WL gradient in x, y and of eq. fda-grad */
  /* 2D mode: U of the bottom, top and HBT layers (1/2 A_b sum rho phi each);
   * obj = wl_bi + sum_l lam_layer[l] energy_layer[l], energy = their sum,
   * hpwl_d2d = exact D2D HPWL with the HBTs (eq. exact-wirelength).  3D: 0. */
  double energy_layer[3];
  /* Density overflow (the paper's OVFL, target density 1): sum over bins of
   * max(rho_b - 1, 0) divided by the sum of rho_b (all instances, fillers
   * included, in the fixed-point density of eq. density-map-accum). */
  double overflow;
} place3d_result;

typedef struct place3d_handle place3d_handle;

/* Validate and deep-copy the problem, allocate every device buffer on
 * `device`, build the net-degree buckets and the transform matrices.
 * cuda_stream: a cudaStream_t of that device, or NULL for the default
 * stream.  On success *out owns all device memory (freed by destroy).
 * Errors: INVALID_ARG, BAD_CSR, OOM, CUDA, UNSUPPORTED (FP32_TC needs an
 * sm_103 device and N_x, N_y multiples of 128). */
int place3d_create(const place3d_problem *prob, int device, void *cuda_stream,
                   place3d_handle **out);

/* out[6] = {w_b, h_b, d_b, d_x, d_y, d_z} (Sec. V-A). */
int place3d_geometry(const place3d_handle *h, double out[6]);

/* HBT penalty factor of Sec. V-A: alpha0 (d_x eta^2 / d_z) log(90 beta eta - 1)
 * with alpha0 = 3.5e-3 and eta = 2 w_hbt / (rh_top + rh_bot). */
double place3d_alpha(double dx, double dz, double beta, double w_hbt,
                     double rh_top, double rh_bot);

/* Set instance centres x, y, z ([n_inst] each, dtype PLACE3D_F32/F64, mem
 * HOST or DEVICE).  Device buffers must stay valid until the next
 * evaluation has been enqueued; they are read on the handle's stream.
 * HOST arrays in page-locked memory the device can address (cudaHostAlloc,
 * torch pin_memory) are read by the packing kernel directly over the
 * CPU-GPU link (no staging copy) and must stay valid until the stream has
 * passed the packing kernel; other host arrays are copied first.
 * z is expected in [d_z/4, 3 d_z/4]; with PLACE3D_FLAG_CHECKS a value
 * outside, or a non-finite coordinate, returns OUT_OF_RANGE (after a sync). */
int place3d_set_positions(place3d_handle *h, const void *x, const void *y,
                          const void *z, int dtype, int mem);

/* Enqueue one evaluation of f and its gradient at the current positions.
 * gx, gy, gz: [n_inst] outputs (dtype, mem) or all NULL (gradient kept on
 * the device only).  If out != NULL the call synchronises the stream and
 * fills *out; with out == NULL it returns right after enqueueing and
 * place3d_get_result() fetches the scalars later.  Host gradient buffers
 * imply a synchronisation; page-locked ones (all three, in the handle's
 * precision) are written by the final kernel directly over the CPU-GPU
 * link instead of through a device copy. */
int place3d_eval_objective_and_grad(place3d_handle *h, place3d_result *out,
                                    void *gx, void *gy, void *gz, int dtype,
                                    int mem);

/* Autotune the launch configuration at the current positions (call after
 * place3d_set_positions; synchronises the device):
 * - degree thresholds and reduction forms of the wirelength stage: the nets
 *   are held in degree classes (2, 3, 4, 5-6, 7-8, 9-12, 13-16, 17-24,
 *   25-32, 33-48, 49-64, 65-128, above 128); every run of adjacent classes
 *   up to 128 pins is timed alone `repeats` times with every (lanes per
 *   net, pins per lane) form that fits it (of forms within 3 % of a run's
 *   fastest, the one with the fewest lanes per net); the splits into runs (one launch
 *   each) with the least total time, with runs of at most two classes and
 *   with single classes are found by dynamic programming, and of these up
 *   to three plans the one whose whole evaluations (one graph launch each,
 *   beside the density path as usual) run fastest is kept; nets above 128
 *   pins keep the chunked form;
 * - with PLACE3D_FP32_TC, the tile width (64 or 128 columns) of each of the
 *   four tensor-core product groups (each group timed alone).
 * The timed evaluations run at the current positions, so afterwards
 * place3d_get_result reports them.  Results are unchanged up to
 * floating-point summation order. */
int place3d_autotune(place3d_handle *h, int repeats);

/* The wirelength launch groups and their forms: writes up to cap entries of
 * (largest degree, lanes per net (0 = the chunked form for nets above 128
 * pins), pins per lane) and returns the number of groups. */
int place3d_wl_forms(const place3d_handle *h, int32_t *dmax, int32_t *lanes,
                     int32_t *pins, int cap);

/* Force the form of one launch group (index as listed by place3d_wl_forms):
 * lanes per net in {1,2,4,8,16,32}, pins per lane in {1,2,4} with
 * lanes*pins at least the group's largest degree (the supported pairs are
 * those the autotuner tries).  INVALID_ARG otherwise. */
int place3d_set_wl_form(place3d_handle *h, int bucket, int lanes, int pins);

/* Set the whole wirelength launch plan, as place3d_wl_forms lists it
 * (typically another handle's autotuned plan for the same netlist): group g
 * covers the degree classes above group g-1's largest degree up to
 * dmax[g], with form (lanes[g], pins[g]).  count = 0 restores the default
 * plan.  INVALID_ARG when the plan does not match this netlist's classes or
 * a form does not fit. */
int place3d_set_wl_plan(place3d_handle *h, const int32_t *dmax,
                        const int32_t *lanes, const int32_t *pins, int count);

/* PLACE3D_FP32_TC: the tile width (64 or 128 output columns) of the four
 * tensor-core product groups (x forward, y forward, x inverse, y inverse).
 * place3d_tc_tiles writes up to cap of them and returns 4 (0 without
 * tensor-core transforms); place3d_set_tc_tiles sets all four (INVALID_ARG
 * for other widths or a handle without them). */
int place3d_tc_tiles(const place3d_handle *h, int32_t *cols, int cap);
int place3d_set_tc_tiles(place3d_handle *h, const int32_t *cols, int count);

/* Synchronise the handle's stream and return the scalars of the last
 * evaluation. */
int place3d_get_result(place3d_handle *h, place3d_result *out);

/* One evaluation as a CUDA graph: position packing (as set_positions with
 * DEVICE arrays) plus the whole evaluation, writing the gradient to DEVICE
 * arrays gx, gy, gz.  The first call (and any call with other pointers or
 * dtype, or after gamma, gamma_z, alpha or a reduction form changed)
 * captures the graph on a private stream and instantiates it (or updates
 * the executable graph in place when its shape is unchanged); every call
 * launches it on the handle's stream.  The pointers are baked into the
 * graph: the arrays must stay allocated while the handle replays it.
 * Results: place3d_get_result / place3d_result_to_device. */
int place3d_eval_graph(place3d_handle *h, const void *x, const void *y,
                       const void *z, void *gx, void *gy, void *gz, int dtype);

/* Batches of independent placement problems (possibly of uneven sizes and
 * precisions) evaluated by ONE CUDA-graph launch: every handle's packing and
 * evaluation is captured on its own stream, forked from and joined to one
 * root, so the instances run concurrently.  handles stay owned by the
 * caller and must outlive the batch; all on one device.  place3d_batch_eval
 * takes per-instance DEVICE pointers (arrays of count pointers, dtype as in
 * place3d_eval_graph), captures on first use or when any pointer or any
 * handle's gamma, gamma_z, alpha or reduction form changes (updating the
 * executable graph in place when it can), and launches on cuda_stream after
 * the handles' last parameter writes (see place3d_batch_shared_stages for
 * the launches the instances share).  Per-instance results via
 * place3d_get_result.  Errors: INVALID_ARG, CUDA (the message, naming the
 * failing call or instance, from place3d_last_error(NULL) on the calling
 * thread). */
typedef struct place3d_batch place3d_batch;
int place3d_batch_create(place3d_handle *const *handles, int count,
                         place3d_batch **out);
int place3d_batch_eval(place3d_batch *b, const void *const *xs,
                       const void *const *ys, const void *const *zs,
                       void *const *gxs, void *const *gys, void *const *gzs,
                       int dtype, void *cuda_stream);
void place3d_batch_destroy(place3d_batch *b);
/* Stages the last captured batch graph runs as one launch shared by all its
 * instances: 1 when the wirelength stage (with the zeroing of the scalars
 * and accumulators, the position packing, the L1 norms and their
 * reductions) is shared -- every instance FP32 or FP32_TC in 3D mode, float
 * positions, no net above 128 pins; its launch groups are those of the
 * instance with the most nets when their forms fit every instance, else the
 * default plan -- and 0 when each instance runs its own (FP64, 2D mode,
 * high-fanout nets).  The density path and the transforms stay per
 * instance (one graph branch each). */
int place3d_batch_shared_stages(const place3d_batch *b);

/* Enqueue, on the handle's stream, a copy of the last evaluation's scalars
 * into dst (a DEVICE buffer of 10 doubles, in place3d_result order: obj,
 * wl_bi, wl_z, energy, hpwl_d2d, n_cross, g_scale, s_x, s_y, s_z) without
 * synchronising (for optimisers that keep the objective on the device). */
int place3d_result_to_device(place3d_handle *h, double *dst);

/* Change gamma, gamma_z, alpha and lambda for the following evaluations (a
 * placement loop anneals gamma and raises lambda, eq. analytical-placement).
 * lambda lives in device memory and is rewritten on the handle's stream
 * (ordered before every later evaluation on that stream; batch launches
 * wait for it), so changing lambda alone leaves captured CUDA graphs as
 * they are and does not synchronise.  A batch launched earlier on another
 * stream must have finished first (the write is not ordered after it).  gamma, gamma_z and alpha are kernel
 * arguments: a change makes the next graph launch re-capture (and update
 * the executable graph in place).
 * Errors: INVALID_ARG (gamma <= 0 or a non-finite value), CUDA. */
int place3d_set_params(place3d_handle *h, double gamma, double gamma_z,
                       double alpha, double lambda);

/* 2D mode: set the three layers' density weights (lambda-, lambda+,
 * lambda') for the following evaluations; device-resident and
 * stream-ordered like lambda in place3d_set_params.  Errors: INVALID_ARG
 * (3D handle or a non-finite weight), CUDA. */
int place3d_set_layer_weights(place3d_handle *h, const double lam[3]);

/* Read an intermediate map of the last evaluation into dst (host or device,
 * [N_z][N_y][N_x] with x fastest):
 *   PLACE3D_MAP_RHO_FIXED: int64 density counts of 2^-36 (the fixed-point
 *     density of eq. density-map-accum + Theorem 1), 8 bytes per bin;
 *   PLACE3D_MAP_EX/EY/EZ: the field of eq. possion-sol-force at bin centres,
 *     in the handle's precision (8 bytes per bin for FP64, else 4).
 * Errors: INVALID_ARG for an unknown map or NULL dst. */
#define PLACE3D_MAP_RHO_FIXED 0
#define PLACE3D_MAP_EX 1
#define PLACE3D_MAP_EY 2
#define PLACE3D_MAP_EZ 3
int place3d_copy_map(place3d_handle *h, int which, void *dst, int mem);

/* Read the per-instance wirelength gradient parts of the last evaluation as
 * FP64 host arrays [n_inst] (any may be NULL): d sum W^_Bi / dx, / dy, the FD
 * depth gradient of eq. fda-grad, and d sum p^_e(z) / dz. */
int place3d_copy_wl_parts(place3d_handle *h, double *gx, double *gy,
                          double *gfd, double *gwaz);

/* Per-stage GPU timing.  With profiling on, every evaluation records CUDA
 * events around its stages on the stream they run on; place3d_stage_times()
 * returns the accumulated milliseconds and launch counts per stage since the
 * last reset (arrays of length place3d_num_stages()), and the stage names. */
int place3d_set_profiling(place3d_handle *h, int on);
int place3d_num_stages(void);
const char *place3d_stage_name(int stage);
int place3d_stage_times(place3d_handle *h, double *ms, int64_t *launches,
                        int64_t *evals, int reset);

/* Number of kernel launches one evaluation enqueues with this handle. */
int place3d_launches_per_eval(const place3d_handle *h);

/*
 * Allocation-free density map.
 *
 * Some callers cannot allocate device memory when they need this map: code
 * that runs inside another framework's memory arena (all device memory is
 * already handed out by that framework's allocator, so a cudaMalloc here
 * would fail or steal from it), or code in a phase where an allocation would
 * implicitly synchronise the device and stall streams it does not own.  This
 * entry point serves them: it computes the same fixed-point density map as a
 * place3d_create handle in PLACE3D_FP64 mode (FP64 contribution arithmetic,
 * counts of 2^-36, macros through corner maps and integer prefix sums) and
 * writes rho[z][y][x] = counts * 2^-36 to a buffer the caller provides,
 * without allocating anything.  The paper has no counterpart of this entry
 * point.
 *
 * Its two int64 accumulator maps live in one array of
 * 2 * PLACE3D_NOALLOC_MAX_BINS int64 (4 MiB) compiled into the library; every
 * GPU that loads the library's device code holds that array until the process
 * exits.
 *
 * All pointers are DEVICE pointers of the current device: x, y, z, w_bot,
 * h_bot, w_top, h_top ([n_inst] doubles, as in place3d_problem), is_macro
 * ([n_inst] bytes) and rho ([nz*ny*nx] doubles, written).  The region and the
 * grid follow place3d_problem.  Work is enqueued on cuda_stream (NULL = the
 * default stream) and the call returns without synchronising.
 * - Warm-up: the first call on a device (and the first after that device's
 *   context was reset or re-created) looks up the array's device address.
 *   With CUDA's lazy module loading (the default) that first call is also
 *   where the library's device code, and with it the array, is loaded onto
 *   the device, which allocates device memory and may synchronise.  Make one
 *   call on each device before entering the phase or arena in which nothing
 *   may allocate, and before any stream capture on that device.
 * - Every call on a device uses the same array and clears it first.  Calls
 *   whose work overlaps on the GPU (other streams or host threads without
 *   ordering between them) race on it and produce wrong maps: order them.
 * - Positions are not checked: for a non-finite coordinate, or z outside
 *   [d_z/4, 3 d_z/4], the map is undefined (every access stays inside the
 *   grid; the counts are simply wrong).
 * Errors: OUT_OF_RANGE if nx*ny*nz > PLACE3D_NOALLOC_MAX_BINS, INVALID_ARG for
 * a bad grid, region or NULL pointer, CUDA for a failed launch or lookup.
 */
#define PLACE3D_NOALLOC_MAX_BINS 262144
int place3d_density_map_noalloc(int n_inst, const double *x, const double *y,
                                const double *z, const double *w_bot,
                                const double *h_bot, const double *w_top,
                                const double *h_top, const uint8_t *is_macro,
                                double xl, double yl, double xh, double yh,
                                int nx, int ny, int nz, double *rho,
                                void *cuda_stream);

/*
 * Self-test of the tensor-core product used by PLACE3D_FP32_TC: out[b][n][m]
 * = sum_k A[b][m][k] W[n][k] with both operands split into BF16 hi/lo planes
 * and FP32 accumulation (the split-precision form of the per-axis transforms
 * of eqs. density-coef .. possion-sol-force).  A: [batches][M][K], W: [N][K],
 * out: [batches][N][M], all HOST FP32 row-major; M a multiple of 128, N and K
 * multiples of 64.  Runs on the current device (sm_103 only) and
 * synchronises it.  *wait_error (may be NULL) receives the kernel's error
 * code (0 = none; 1..3 = a bounded mbarrier wait expired).  Errors:
 * INVALID_ARG, UNSUPPORTED (not an sm_103 device), CUDA, TIMEOUT.
 */
int place3d_tc_selftest(int M, int N, int K, int batches, const float *A,
                        const float *W, float *out, int *wait_error);

/* Failure-path self-test of the bounded waits (the paper has no counterpart;
 * a test hook).  Runs one 128x64x64 tensor-core product whose TMA producer
 * arms and loads nothing, with every mbarrier wait bounded by wait_cycles
 * SM clocks (about wait_cycles / 2e9 seconds): the MMA thread's first wait
 * runs out (or the epilogue's, whichever budget expires first), the CTA
 * records the error code of that wait (1 operands, 2 free stage, 3
 * accumulator), stops issuing work, frees its tensor memory and exits.
 * Returns PLACE3D_ERR_TIMEOUT with *wait_error > 0; the CUDA context stays
 * usable.
 * UNSUPPORTED off sm_103; INVALID_ARG for wait_cycles <= 0. */
int place3d_tc_timeout_selftest(long long wait_cycles, int *wait_error);

/* Failure injection on the host (a test hook; the paper has no
 * counterpart): with nth > 0, the nth device allocation made by a later
 * place3d_create on the calling thread fails as if the device were out of
 * memory (nothing is allocated for it).  place3d_create then returns
 * PLACE3D_ERR_OOM and frees everything it had allocated.  nth <= 0 clears
 * the hook; it also clears itself once it has fired. */
void place3d_debug_fail_alloc(int nth);

/* Nesterov placement loop on the device (Sec. III-A: the gradient-based 3D
 * global placement; eq. improved-precond; the movable range of the centres:
 * x, y in the region, z in [d_z/4, 3 d_z/4]).  All arrays are device arrays
 * of n_inst elements in the handle's precision (F64 for FP64 handles, F32
 * otherwise), all work is enqueued on the handle's stream and nothing
 * synchronises: the step length and the norms it is estimated from stay on
 * the device.  3D-mode handles only (INVALID_ARG otherwise).  Start:
 *   place3d_set_positions(v); place3d_eval_objective_and_grad(h, NULL,
 *   NULL, NULL, NULL, ...); place3d_nesterov_init(g, init_step);
 * then per iteration:
 *   place3d_nesterov_update(u, v, g, (a_k - 1)/a_{k+1});
 *   place3d_eval_objective_and_grad(h, NULL, NULL, NULL, NULL, ...);
 *   place3d_nesterov_precondition(g);
 *
 * place3d_nesterov_precondition: takes the gradient G of the last
 * evaluation, which must have been place3d_eval_objective_and_grad (that
 * keeps the gradient in the handle unless profiling is on or the gradient
 * arrays are device arrays of the other precision; INVALID_ARG after those,
 * after place3d_eval_graph or a batch), and forms g_new = G / H
 * with H_i = max(1, |E_i| + lambda q_i) for macros (|E_i| = the instance's
 * pin count) and max(1, lambda q_i) otherwise, q_i = w_i h_i d_z/2 with the
 * die sizes at the evaluated z; the z component is 0 for z-fixed instances.
 * Stores g_new into g and sets the step length to |v_new - v| / |g_new - g|
 * (2-norms over all 3 n_inst components) when both are positive,
 * |v_new - v| being the one of the last update.
 * place3d_nesterov_init: the same with the previous g taken as 0 and the
 * step length set to init_step / max |g_new| (init_step > 0, in the
 * positions' units).
 * place3d_nesterov_update: u_new = P(v - step g), v_new = P(u_new + coef
 * (u_new - u)) with P the clamp to the movable range; u <- u_new,
 * v <- v_new, and v_new becomes the handle's positions for the next
 * evaluation (as place3d_set_positions would set them).
 * place3d_nesterov_step reads the current step length (synchronises). */
int place3d_nesterov_init(place3d_handle *h, void *gx, void *gy, void *gz, double init_step);
int place3d_nesterov_precondition(place3d_handle *h, void *gx, void *gy, void *gz);
int place3d_nesterov_update(place3d_handle *h, void *ux, void *uy, void *uz, void *vx,
                            void *vy, void *vz, const void *gx, const void *gy,
                            const void *gz, double coef);
int place3d_nesterov_step(place3d_handle *h, double *step);

/* Number of CUDA-graph captures the handle has made so far (place3d_eval_graph
 * and the graph behind place3d_eval_objective_and_grad; a capture follows a
 * change of the output buffers, of gamma / gamma_z / alpha, or of the
 * reduction forms).  -1 for a NULL handle. */
long long place3d_graph_captures(const place3d_handle *h);

/* Self-test of the int64 -> FP32 conversion the FP32 density pass uses (a
 * test hook): converts the n host values vals[] on the current device with
 * it, writes the results to the host array out[] (n floats) and sets
 * *mismatches to the number of values whose result differs, bit for bit,
 * from the hardware's round-to-nearest-even conversion.
 * Errors: INVALID_ARG (NULL pointer, n < 0), CUDA. */
int place3d_ll2f_selftest(const long long *vals, float *out, int n, int *mismatches);

/* Last error message of the handle, or of the calling thread when h is NULL
 * (creation errors).  Never NULL. */
const char *place3d_last_error(const place3d_handle *h);

/* Free every resource of the handle (synchronises its stream). */
void place3d_destroy(place3d_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* PLACE3D_H */
