/*
 * fp.h - C ABI of the GB300 free-stream-preserving (FP) upwind finite-difference
 * residual library (libfpgb300.so).
 *
 * Method: Su, Cai, Pan & Hu, "Reformulated dissipation for the free-stream
 * preserving of the conservative finite difference schemes on curvilinear grids",
 * arXiv 2101.05886.  The library advances the compressible Euler equations on
 * stationary curvilinear grids (Sec. 2.1, Eq. NS without the viscous terms).  At
 * every cell face it forms the reference face state Q* (Eq. Q_star), subtracts
 * the reference flux from every cell value of the upwind stencil, reconstructs
 * with unmodified WENO5-JS or linear upwind under characteristic local
 * Lax-Friedrichs splitting, adds back the metric-weighted reference flux
 * (Eqs. my_point1 to my_point3) and differences the face fluxes into the
 * residual (Eq. aderivative).  Time integration is third-order TVD Runge-Kutta.
 *
 * Conventions for every entry point
 *  - Plain C types only.  No C++ type or exception crosses this boundary, and
 *    nothing here calls exit() or abort().
 *  - Pointers named *_dev are CUDA device pointers.  Pointers named *_host are
 *    host pointers.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Calls are stream-ordered and asynchronous unless stated.
 *  - State layout: conserved variables (rho, rho u, rho v, rho w, rho E) as a
 *    C-contiguous array [5][nk][nj][ni] (i fastest) of interior points only.
 *    The element type is double for FP_F64 and float for FP_F32_MIXED.  Ghost
 *    values come from the boundary codes when they are read; they are never
 *    stored.  The caller owns every state and output buffer.
 *  - Errors: every call returns an fp_status.  FP_ERR_ARG means the call was
 *    rejected before any GPU work was queued.  FP_ERR_CUDA reports a CUDA error,
 *    which may come from earlier asynchronous work.  fp_last_error() gives a
 *    one-line message for the last failing call on a context.
 *  - A context is not thread-safe: use it from one host thread at a time.
 */
#ifndef FP_GB300_H
#define FP_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FP_OK = 0,
  FP_ERR_ARG = 1,          /* invalid argument, nothing was queued */
  FP_ERR_CUDA = 2,         /* CUDA runtime error (possibly from earlier async work) */
  FP_ERR_OOM = 3,          /* device allocation failed */
  FP_ERR_NONFINITE = 4,    /* a kernel produced a non-finite state value */
  FP_ERR_TIMEOUT = 5,      /* reserved: a bounded device-side wait gave up.  No kernel of this
                              library waits on another (work items are assigned statically and
                              no launch waits on a flag), so no call returns it at present */
  FP_ERR_UNSUPPORTED = 6,  /* valid but not implemented combination */
  FP_ERR_BOUNDS = 7        /* bounds-checking build only (fp_bounds_checking() == 1): a kernel met
                              an element index outside its array; the access went to the array's
                              first element instead, so results are wrong but nothing faulted */
} fp_status;

enum { FP_WENO5_JS = 0, FP_LINEAR_UPWIND5 = 1, FP_WENO7_JS = 2, FP_WENOCU6 = 3 };
/* reconstruction: WENO5-JS and linear upwind per Sec. 2.2.2; WENO7-JS and WENOCU6 per
   Remark 2 (WENOCU6: six-point adaptive central-upwind, linear limit the M6 central face
   value, C = 20, power 2, epsilon 1e-40) */
enum { FP_F64 = 0, FP_F32_MIXED = 1 };                      /* precision of the sweep */
enum { FP_BC_PERIODIC = 0, FP_BC_FARFIELD = 1, FP_BC_EXTRAP = 2, FP_BC_SLIP_WALL = 3, FP_BC_CUT = 4,
       FP_BC_BLOCK = 5, FP_BC_HALO = 6 };
enum { FP_XI = 0, FP_ETA = 1, FP_ZETA = 2 };

typedef struct {
  int dims;                   /* 2 or 3 */
  int n[3];                   /* solution points ni, nj, nk (nk = 1 when dims == 2) */
  int metric_order;           /* M in {2,4,6,8}: order of metrics, Jacobian and every
                                 face interpolation (Sec. 3 Eq. metric_discret, Remark 3) */
  int scheme;                 /* FP_WENO5_JS, FP_LINEAR_UPWIND5, FP_WENO7_JS or FP_WENOCU6 */
  int free_stream_preserving; /* 1 = the paper's FP face flux, 0 = plain scheme (control) */
  int characteristic;         /* 1 = Roe characteristic-wise splitting (paper), 0 = component-wise */
  int precision;              /* FP_F64, or FP_F32_MIXED: metrics built in FP64, sweep in FP32 */
  int bc[3][2];               /* per direction (lo, hi), ghost values produced on read:
                                 FP_BC_PERIODIC  wrap around the block;
                                 FP_BC_FARFIELD  q_inf;
                                 FP_BC_EXTRAP    copy of the boundary cell (zero gradient);
                                 FP_BC_SLIP_WALL the wall is the boundary face: ghost x' mirrors
                                   cell x (-1-x, or 2n-1-x) with its momentum reflected about
                                   the face's normal k/|k|, k the order-M face metric of that
                                   grid line (Sec. 4.2 slip walls; the discrete rule is ours);
                                 FP_BC_CUT       C-grid cut: the boundary face meets the block
                                   itself with the first transverse index t reversed (t = j for
                                   the i direction, t = i for j and k): ghost x' is the mirror
                                   cell on line n_t-1-t, unchanged; lines with
                                   cut_width <= t < n_t - cut_width are slip wall (the body);
                                 FP_BC_BLOCK     another block of a batch (fp_batch_create_linked):
                                   ghost x' beyond this side is the linked block's cell next to
                                   its opposite side (x - n or n_linked + x), same transverse
                                   indices, read at the same RK stage; single-block calls
                                   (fp_rhs, fp_rk3_step, fp_rhs_noalloc) reject such blocks;
                                 FP_BC_HALO      cells another process holds (a block split into
                                   slabs across GPUs): ghost x' is read from the caller's halo
                                   buffer of that side (fp_set_halo), which the caller refreshes
                                   before every RK stage (fp_pack_halo on the neighbour, an
                                   exchange, fp_rk3_stage); the ghost nodes given to
                                   fp_init_grid there must be the neighbour's nodes */
  double gamma;               /* ratio of specific heats (Sec. 2.1 Eq. EOS: 1.4) */
  double q_inf[5];            /* far-field state; also the reference state of the FP32 form.
                                 With FP_F32_MIXED it is used as float values, like the state
                                 (a far-field ghost is a float state value) */
  int global_lf;              /* 0 = local Lax-Friedrichs speeds (max over the face's stencil),
                                 1 = global speeds (max over the block, per direction and
                                 characteristic field, refreshed every RK stage); Sec. 4 uses
                                 global splitting for its shock cases */
  int cut_width;              /* FP_BC_CUT sides only: wake cells at each end of t that meet
                                 across the cut (>= n_t/2: the whole side is a cut) */
} fp_grid_desc;

typedef struct fp_ctx fp_ctx;
typedef struct fp_batch fp_batch;

/* Ghost width G of the stored metrics: max(3, M/2), or max(4, M/2) for WENO7 (the
   stencil reach past a face versus the order-M face interpolation). */
int fp_ghost_width(int metric_order, int scheme);
/* Node ghost layers required by fp_init_grid: G + 3M/2 (the metric products,
   the metrics and the Jacobian are all formed by the same order-M central
   operator, so every cell a stencil can reach satisfies the discrete surface
   conservation law, Sec. 2.1 Eq. SCL). */
int fp_node_ghost_width(int metric_order, int scheme);

/* Build a block: copies the node coordinates to the device and forms, in FP64,
   the symmetric conservative metrics (Eq. JBabc), the Jacobian (Eq. JB), the
   face metrics of every direction (Eq. xidJ at order M) and the work lists.
   xyz_nodes_host: double [dims][nk+2g][nj+2g][ni+2g] (2-D: [2][nj+2g][ni+2g]),
   g = ghost_nodes >= fp_node_ghost_width(M, scheme); read during the call only.
   Allocates device memory owned by the context.  Synchronises `stream`. */
int fp_init_grid(const fp_grid_desc *desc, const double *xyz_nodes_host, int ghost_nodes,
                 void *stream, fp_ctx **out);

/* dqdt_dev = -J * sum_d (F'_{d,i+1/2} - F'_{d,i-1/2}) (Eq. aderivative, Delta xi = 1).
   q_dev is read only; dqdt_dev has the state layout and type.  Uses the
   context's residual scratch. */
int fp_rhs(fp_ctx *ctx, const void *q_dev, void *dqdt_dev, void *stream);

/* One third-order TVD Runge-Kutta step (Gottlieb & Shu) of size dt, in place on
   q_dev.  Uses the context's two stage buffers and residual scratch.  A stage
   whose updated state is not finite sets a device flag that fp_get_device_status()
   reports. */
int fp_rk3_step(fp_ctx *ctx, void *q_dev, double dt, void *stream);

/* One of the three stages of fp_rk3_step (stage 0, 1, 2 in order, the same dt; stage 0 reads
   q_dev, stage 2 writes the step's result into q_dev).  For blocks with FP_BC_HALO sides,
   whose halos must hold the neighbours' cells of the same stage before each stage runs
   (Sec. 2.2 third-order TVD Runge-Kutta, split at its stages).  fp_rk3_step rejects such
   blocks; any block may be advanced this way. */
int fp_rk3_stage(fp_ctx *ctx, void *q_dev, double dt, int stage, void *stream);

/* Halo of an FP_BC_HALO side (dir, side): halo_dev is a caller-owned device buffer of
   fp_halo_bytes(ctx, dir) bytes holding the G = fp_ghost_width cells beyond that side, laid
   out like the state with the extent n_dir replaced by G; its index along dir follows the grid
   index (cells -G..-1 below the low side, or n..n+G-1 above the high side, are halo indices
   0..G-1).  Kept by the context and read by every later pass until replaced.  FP_ERR_ARG if
   that side is not FP_BC_HALO. */
int fp_set_halo(fp_ctx *ctx, int dir, int side, void *halo_dev);
size_t fp_halo_bytes(const fp_ctx *ctx, int dir);

/* The G cells next to side (dir, side) of stage state `stage` (0: q_dev, 1 and 2: the
   context's stage buffers, as left by fp_rk3_stage of the previous stage), written to out_dev
   in the layout of the halo the neighbour across that side reads (low side: cells 0..G-1,
   high side: cells n-G..n-1).  Stream-ordered; allocates nothing. */
int fp_pack_halo(fp_ctx *ctx, const void *q_dev, int stage, int dir, int side, void *out_dev, void *stream);

/* dt = cfl / max over points of sum_d (|U_d| + c |grad d|), grad d = J (d_x, d_y, d_z)/J.
   Synchronises `stream` to return the value in *dt_out (host). */
int fp_cfl_dt(fp_ctx *ctx, const void *q_dev, double cfl, double *dt_out, void *stream);

/* Copy the stored cell metrics to host memory: double [10][nk+2G][nj+2G][ni+2G], G = fp_ghost_width
   (2-D: [10][1][nj+2G][ni+2G]); entry 3d+a is (d-th coordinate)_{x_a}/J, entry 9
   is 1/J.  Values are those the sweep uses (rounded to float for FP_F32_MIXED). */
int fp_get_metrics(fp_ctx *ctx, double *host_out);

/* Copy the face metrics of direction dir to host memory: double [3][faces], faces
   ordered like the state with n_dir+1 faces along dir (face f+1/2, f = -1..n-1). */
int fp_get_face_metrics(fp_ctx *ctx, int dir, double *host_out);

/* Synchronise `stream`, read and clear the device status word.  Returns FP_OK, or
   FP_ERR_NONFINITE when an RK stage produced a non-finite state value since the last read, or
   (bounds-checking build) FP_ERR_BOUNDS when a kernel met an out-of-range index. */
int fp_get_device_status(fp_ctx *ctx, void *stream);

/* 1 in the bounds-checking build of the library (libfpgb300_check.so, compiled with
   -DFPK_BOUNDS_CHECK; no counterpart in the paper), 0 in the normal build.  In the checking
   build every global element the sweep, the halo packing and the speed and time-step
   reductions access is checked against its array, and every shared-ring offset against the
   ring, before the access; a violation is redirected and reported as FP_ERR_BOUNDS by
   fp_get_device_status.  The metric kernels of fp_init_grid are not checked. */
int fp_bounds_checking(void);

/* Allocation-free residual (no counterpart in the paper; an interface of this library).
   Computes what fp_rhs computes, bit for bit, without allocating or freeing anything, for
   callers that cannot allocate device memory at the point where they evaluate a residual:
   a host framework that hands out device memory only from a pool it reserved up front, a
   solver loop that runs under a fixed device-memory budget, or a real-time loop that must
   not stall in the allocator.
   The residual accumulator that the three direction passes share is a file-scope static
   device array of 8 MiB, and the block descriptor its kernels read a static device variable;
   the descriptor travels as a kernel argument.  Both arrays come into existence on a device
   with the first fp_init_grid there (which also looks up their device addresses) and stay
   until the process exits.  Blocks that need more than 8 MiB of accumulator (more than
   209,715 points in FP64, 419,430 in FP32) are rejected with FP_ERR_ARG and a message in
   fp_last_error().  The context's device must be current.  Every call on a device shares
   the static arrays, which keep the last call's contents (each call rewrites the whole
   accumulator before reading it, so nothing needs clearing): calls that may overlap on the
   GPU (different streams, several host threads) race with each other and must be
   serialised by the caller.  q_dev, dqdt_dev and the context as in fp_rhs. */
int fp_rhs_noalloc(fp_ctx *ctx, const void *q_dev, void *dqdt_dev, void *stream);

/* Measured arithmetic peaks of the current device (no counterpart in the paper; the
   denominators of the sweep's roofline).  Times, with CUDA events on `stream` (best of
   three after a warm-up), kernels in which every thread runs independent fused
   multiply-add chains on all SMs: scalar FP32 FFMA, packed FP32x2 FFMA2 and FP64 DFMA.
   Writes TFLOP/s (an FMA counts two flops, an FFMA2 four) to the three outputs.  Allocates
   and frees a few MB of device memory; synchronises `stream`.  FP_ERR_ARG for a null output. */
int fp_probe_peaks(double *fp32_tflops, double *fp32x2_tflops, double *fp64_tflops, void *stream);

/* Host-side failure injection: the n-th device or page-locked allocation made by the
   library from now on (n = 0: the next one) fails as if memory were exhausted, so that the
   FP_ERR_OOM paths of fp_init_grid, fp_batch_create and fp_pipe_create (which release
   everything allocated so far and return nothing) can be exercised without exhausting a
   device.  n < 0 cancels a pending failure.  Process-wide; returns FP_OK. */
int fp_debug_fail_allocation(int n);

/* Bytes of one state array of the block: 5 x n_i x n_j x n_k elements of the precision's
   type (double for FP_F64, float for FP_F32_MIXED); 0 for a NULL context. */
size_t fp_state_bytes(const fp_ctx *ctx);

/* Number of kernel launches one fp_rhs / fp_rk3_step call queues. */
int fp_launches_per_rhs(const fp_ctx *ctx);
int fp_launches_per_step(const fp_ctx *ctx);

/* Threads per CTA of the context's sweep (no counterpart in the paper): the primary size, and
   an alternative one (0 if none; the folded FP32 sweeps have one, which a batch's autotuner
   may pick per direction).  A tile has faces x lines equal to one of them. */
int fp_get_cta_sizes(const fp_ctx *ctx, int *primary, int *alternative);
/* Tile shape used for direction dir: faces per chunk and lines per tile.  Defaults: 32 faces
   along xi; 8 faces along eta and zeta, or 32 there when 8 would give fewer work items than
   the device holds resident CTAs (small blocks); lines = the primary CTA size / faces.
   Results do not depend on it. */
int fp_get_tile(const fp_ctx *ctx, int dir, int *faces, int *lines);
/* Override the tile shape: faces in {8,16,32}, faces x lines one of fp_get_cta_sizes; a size
   whose xi rings are unpadded takes 32 faces along xi only (FP_ERR_ARG otherwise). */
int fp_set_tile(fp_ctx *ctx, int dir, int faces, int lines);

const char *fp_last_error(const fp_ctx *ctx);
const char *fp_status_string(int status);
void fp_free(fp_ctx *ctx);                 /* NULL-safe; synchronises the device */

/* ---------------- batched multi-block advance ----------------
   Multi-block grids: a block side with bc FP_BC_BLOCK is linked to another block of the
   batch by an fp_block_link.  The ghost nodes the caller passes to fp_init_grid for that
   side must be the linked block's nodes, so that every metric a stencil reaches is the
   one the unsplit grid would have.  All blocks of a batch advance through the same RK
   stages together, and a pass never writes the stage state that it reads, so the linked
   reads need no synchronisation beyond the launch order.
   A batch advances many independent blocks (same precision, scheme, metric order)
   together: one persistent launch per direction pass covers the work of every
   block, the three RK stages are captured once into a CUDA graph, and each call
   replays it.  Unlinked batches with local Lax-Friedrichs speeds are captured as up to
   four independent chains of the graph, each advancing a group of the blocks of about equal
   point count, so the chains' launches run side by side on the GPU (then one launch per
   chain covers that chain's blocks).  A batch runs one CTA shape of the sweep in every
   direction (fp_get_cta_sizes; the folded FP32 linear-upwind sweep its alternative one),
   with the blocks' tiles where they are of that shape and the defaults elsewhere.  The
   batch keeps pointers to the contexts (they must outlive it) and to the caller's state
   buffers q_devs[b] given at creation.  When autotune is nonzero, fp_batch_create times each
   candidate tile of that shape on the blocks and keeps the fastest per size class
   (fp_batch_get_tile); it may run kernels on the blocks' buffers. */
int fp_batch_create(fp_ctx *const *blocks, int nblocks, void *const *q_devs, int autotune,
                    void *stream, fp_batch **out);
/* Side `side` (0 = low, 1 = high) of direction `dir` of block `a` (index into the batch's
   block list) takes its ghost cells from block `b`. */
typedef struct {
  int a, dir, side, b;
} fp_block_link;
/* fp_batch_create with block links.  Every FP_BC_BLOCK side of every block must be linked
   exactly once, the linked blocks must have the same extents in the two other directions,
   and no other side may be linked; otherwise FP_ERR_ARG and nothing is created.
   fp_batch_create is this call with no links. */
int fp_batch_create_linked(fp_ctx *const *blocks, int nblocks, void *const *q_devs,
                           const fp_block_link *links, int nlinks, int autotune, void *stream,
                           fp_batch **out);
/* One RK3 step of size dt on every block (graph replay). */
int fp_batch_rk3_step(fp_batch *batch, double dt, void *stream);
/* dqdt for every block (no graph); dqdt_devs[b] has block b's state layout. */
int fp_batch_rhs(fp_batch *batch, void *const *dqdt_devs, void *stream);
int fp_batch_launches_per_step(const fp_batch *batch);
/* Tile shape the batch runs block `block` with in direction dir (after autotuning, if any). */
int fp_batch_get_tile(const fp_batch *batch, int block, int dir, int *faces, int *lines);
const char *fp_batch_last_error(const fp_batch *batch);
void fp_batch_free(fp_batch *batch);       /* NULL-safe */

/* ---------------- host-resident states, copies overlapped by compute ----------------
   A pipe advances blocks whose states live in host memory.  It splits the blocks into
   `ngroups` groups of about equal size, each a batch (as fp_batch_create) with device state
   buffers and a stream of its own.  One step issues, group by group on the group's stream,
   the copies of the group's states to the device, the group's RK3 step and the copies back,
   so the copy engines move one group's states while the SMs advance another.  Host states
   should be page-locked (cudaHostAlloc / pinned tensors) for the copies to overlap.  The
   pipe keeps pointers to the contexts (they must outlive it). */
typedef struct fp_pipe fp_pipe;
/* q_host[b]: block b's state in host memory (read once to initialise the device copies, and
   to autotune when autotune is nonzero).  Allocates the device states and the batches. */
int fp_pipe_create(fp_ctx *const *blocks, int nblocks, const void *const *q_host, int ngroups,
                   int autotune, fp_pipe **out);
/* One RK3 step of size dt: q_host[b] is copied in, advanced and copied back, in place.  Each
   group's work follows that group's work of the previous step (its own stream), so consecutive
   steps overlap; `stream` waits for all of it, and the host states are complete once `stream`
   is synchronised.  The pipe's work is not ordered after work the caller queued earlier on
   `stream`, so the pipe's contexts (and their stage and residual scratch) must not be used by
   other calls (fp_rhs, fp_rk3_step, a batch) while a pipe step may be in flight: synchronise
   `stream` before such a call, or switch the pipe to ordered steps (fp_pipe_set_ordered). */
int fp_pipe_rk3_step_host(fp_pipe *pipe, void *const *q_host, double dt, void *stream);
/* Ordered steps (ordered nonzero): every step of the pipe also follows the work queued on the
   step's `stream` before the call, as a call on one stream would, so that work may fill the host
   states (a device-to-host copy, a host function) or use the pipe's contexts.  The price is the
   overlap of consecutive steps: a step's first uploads then wait for the previous step's last
   group.  Off (0) by default.  FP_ERR_ARG for a NULL pipe. */
int fp_pipe_set_ordered(fp_pipe *pipe, int ordered);
int fp_pipe_groups(const fp_pipe *pipe);
int fp_pipe_launches_per_step(const fp_pipe *pipe);
const char *fp_pipe_last_error(const fp_pipe *pipe);
void fp_pipe_free(fp_pipe *pipe);          /* NULL-safe; synchronises the pipe's streams */

/* ---------------- host helper (no counterpart in the paper) ----------------
   The partition behind the graph branches of fp_batch_create (weights = points per block)
   and the groups of fp_pipe_create (weights = state bytes per block).  Items go one at a
   time, heaviest first (equal weights in index order), each into the currently lightest of
   `ngroups` groups (the lowest index among equally light ones); group_of[k] receives the
   group of item k.  Host only: no CUDA call, no allocation visible to the caller.
   FP_ERR_ARG for a null pointer with n > 0, n < 0, ngroups < 1 or a negative weight. */
int fp_balanced_groups(const long long *weights, int n, int ngroups, int *group_of);

#ifdef __cplusplus
}
#endif
#endif /* FP_GB300_H */
