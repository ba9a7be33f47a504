// api.cu - C ABI of libfpgb300.so (declared in include/fp.h): block contexts,
// residual and Runge-Kutta drivers, the batched multi-block advance captured in a
// CUDA graph, and the tile autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fp.h"
#include "fp_internal.h"

using fpk::BlockDev;
using fpk::DirDev;

struct fp_ctx {
  fp_grid_desc desc;
  int G = 0;
  int is_f32 = 0;
  size_t esize = 8;
  long long ncells = 0;
  long long nmet = 0;                 // points of one metric component (ghosted box)
  long long nface[3] = {0, 0, 0};     // faces per direction
  void *met = nullptr;                // T [10][nmet]
  void *fmet[3] = {nullptr, nullptr, nullptr};
  void *dk[3] = {nullptr, nullptr, nullptr};
  void *q1 = nullptr, *q2 = nullptr, *racc = nullptr;
  int *status = nullptr;
  double *dt_dev = nullptr;
  unsigned long long *cfl_bits = nullptr;
  void *lamg = nullptr;               // T [3][3] global Lax-Friedrichs speeds
  int2 *lam_items = nullptr;          // (block 0, first point) chunks for the speed reduction
  int nlam_items = 0;
  BlockDev hblk;
  BlockDev *dblk = nullptr;
  BlockDev uploaded;                  // last BlockDev copied to dblk
  std::vector<int2> hitems[3];
  int2 *items[3] = {nullptr, nullptr, nullptr};
  int nitems[3] = {0, 0, 0};
  int nsm = 152;
  // CTA shapes of the context's sweep: [0] the primary one, [1] the alternative (nshape == 2,
  // the folded FP32 sweeps): threads (faces per chunk x lines per tile), xi rings padded (every
  // tile shape conflict-free) or not (S = 32 only), resident CTAs per SM
  int nshape = 1;
  int nt[2] = {128, 128}, pad[2] = {1, 1}, per_sm[2] = {1, 1};
  int dev = 0;                        // the device the context's memory lives on
  double dt_host = 0.0;
  std::string err;
};

struct fp_batch {
  std::vector<fp_ctx *> ctx;
  std::vector<BlockDev> hblk;
  BlockDev *dblk = nullptr;
  int2 *items[3] = {nullptr, nullptr, nullptr};
  int nitems[3] = {0, 0, 0};
  double *dt_dev = nullptr;
  double *dt_host = nullptr;   // page-locked, so the per-step upload is asynchronous
  cudaEvent_t dt_ready = nullptr;  // the last upload of dt_host has been consumed
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int dims = 3, M = 6, scheme = 0, charwise = 1, fp = 1, is_f32 = 1, global_lf = 0;
  int bnd[3] = {0, 0, 0};   // some block has a slip-wall or cut side in direction d
  // Graph branches: groups of blocks whose RK steps run as independent chains of the graph,
  // so one group's launches fill the end-of-pass tail of another's.  One branch when blocks
  // are linked (a block reads its neighbours' stage states) or the LF speeds are global.
  static constexpr int kMaxBranch = 4;
  int nbranch = 1;
  int2 *bitems[kMaxBranch][3] = {};
  int bnitems[kMaxBranch][3] = {};
  int nsm = 152;
  int nshape = 1, nt[2] = {128, 128}, pad[2] = {1, 1}, per_sm[2] = {1, 1};   // as fp_ctx (shared by all blocks)
  int shape = 0;                     // the one CTA shape the batch runs (sweep_batch_shape)
  int2 *lam_items = nullptr;
  int nlam_items = 0;
  std::string err;
};

// ----------------------------------------------------------------- allocations
//
// Every device and page-locked allocation of the library goes through dev_malloc and
// host_malloc.  fp_debug_fail_allocation arms a countdown on the host: the allocation that
// finds it at zero returns cudaErrorMemoryAllocation without calling CUDA, so the failure
// paths (FP_ERR_OOM, with everything allocated so far released) can be exercised without
// exhausting a device.
namespace {
std::atomic<long long> g_fail_countdown{-1};   // -1: no failure armed

bool take_scheduled_failure() {
  long long cur = g_fail_countdown.load();
  while (cur >= 0 && !g_fail_countdown.compare_exchange_weak(cur, cur - 1)) {
  }
  return cur == 0;
}
}  // namespace

namespace fpk {
cudaError_t dev_malloc(void **p, size_t bytes) {
  *p = nullptr;
  if (take_scheduled_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}
cudaError_t host_malloc(void **p, size_t bytes) {
  *p = nullptr;
  if (take_scheduled_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}
}  // namespace fpk

// ----------------------------------------------------------------- static scratch of fp_rhs_noalloc
//
// The residual accumulator that fp_rhs_noalloc's three direction passes share, and the block
// descriptor its kernels read, live in file-scope device arrays rather than in memory the
// call would have to allocate.  Host code cannot use the arrays' names as device addresses
// (on the host they name a stand-in), so their addresses are looked up once per device with
// that device current, in fp_init_grid: a call that allocates anyway, and the first use of
// this file's module on the device, which is when the arrays come into existence there.
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;      // 8 MiB per device
constexpr int kNoAllocMaxDevices = 64;
__device__ __align__(256) unsigned char g_noalloc_racc[kNoAllocScratchBytes];
__device__ __align__(256) BlockDev g_noalloc_block;

struct NoAllocDevice {
  void *racc = nullptr;
  BlockDev *blk = nullptr;
  std::atomic<bool> ready{false};
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// once per device, with that device current; safe from several host threads
cudaError_t noalloc_prepare(int dev) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaSuccess;   // fp_rhs_noalloc refuses such devices
  NoAllocDevice &S = g_noalloc_dev[dev];
  if (S.ready.load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (S.ready.load(std::memory_order_relaxed)) return cudaSuccess;
  void *racc = nullptr, *blk = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&racc, g_noalloc_racc);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&blk, g_noalloc_block);
  if (e != cudaSuccess) return e;
  S.racc = racc;
  S.blk = static_cast<BlockDev *>(blk);
  S.ready.store(true, std::memory_order_release);
  return cudaSuccess;
}

// the descriptor arrives as a kernel argument (copied by value at launch) and is stored
// into the static descriptor that the passes read
__global__ void k_noalloc_store_block(BlockDev b) { g_noalloc_block = b; }
}  // namespace

namespace {

int fail(fp_ctx *c, int st, const std::string &msg) {
  if (c) c->err = msg;
  return st;
}

int cuda_fail(fp_ctx *c, cudaError_t e, const char *where) {
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
}

int bfail(fp_batch *b, int st, const std::string &msg) {
  if (b) b->err = msg;
  return st;
}

// ghost width: the stencil reach past a face (3, or 4 for WENO7) or the face interpolation's M/2
// direction d of a block has a slip-wall or cut side (those rules are compiled into a
// separate sweep variant, so blocks without them run a sweep without their code)
int has_bnd(const fp_grid_desc &d, int dir) { return d.bc[dir][0] >= FP_BC_SLIP_WALL || d.bc[dir][1] >= FP_BC_SLIP_WALL; }

// some side of the block takes its ghosts from another block (batch only)
int has_link(const fp_grid_desc &d) {
  for (int k = 0; k < d.dims; ++k)
    for (int s = 0; s < 2; ++s)
      if (d.bc[k][s] == FP_BC_BLOCK) return 1;
  return 0;
}

// some side of the block takes its ghosts from a caller's halo buffer
int has_halo(const fp_grid_desc &d) {
  for (int k = 0; k < d.dims; ++k)
    for (int s = 0; s < 2; ++s)
      if (d.bc[k][s] == FP_BC_HALO) return 1;
  return 0;
}

int ghost_of(int M, int scheme) { return std::max(scheme == FP_WENO7_JS ? 4 : 3, M / 2); }

// resident CTAs per SM of the sweep variants a context runs (folded switches or not; the fewer
// of the plain and the boundary-rule instantiation), after opting every variant in to its
// dynamic shared memory
int prepare(int is_f32, int M, int scheme, int fix) {
  using P = int (*)(int, int);
  const P f32[6] = {fpk::prepare_sweep_f32, fpk::prepare_sweep_f32_fix, fpk::prepare_sweep_f32_fix2,
                    fpk::prepare_sweep_f32_bnd, fpk::prepare_sweep_f32_bnd_fix, fpk::prepare_sweep_f32_bnd_fix2};
  const P f64[6] = {fpk::prepare_sweep_f64, fpk::prepare_sweep_f64_fix, nullptr,
                    fpk::prepare_sweep_f64_bnd, fpk::prepare_sweep_f64_bnd_fix, nullptr};
  const P *p = is_f32 ? f32 : f64;
  int nb[6] = {1 << 20, 1 << 20, 1 << 20, 1 << 20, 1 << 20, 1 << 20};
  for (int v = 0; v < 6; ++v)
    if (p[v]) nb[v] = p[v](M, scheme);
  return std::min(nb[fix], nb[3 + fix]);
}

// the CTA shapes of a sweep (fp_internal.h sweep_threads) and their resident CTAs per SM
template <typename C>
void set_shapes(C *c, int is_f32, int M, int scheme, int fix) {
  c->nshape = fpk::sweep_has_alt(is_f32, scheme, fix) ? 2 : 1;
  for (int a = 0; a < c->nshape; ++a) {
    const int f = fix + a;   // fix = 2: the alternative shape
    c->nt[a] = fpk::sweep_threads(is_f32, scheme, f);
    c->pad[a] = fpk::sweep_padded(is_f32, scheme, f) ? 1 : 0;
    c->per_sm[a] = prepare(is_f32, M, scheme, f);
  }
  if (c->nshape == 1) { c->nt[1] = c->nt[0]; c->pad[1] = c->pad[0]; c->per_sm[1] = c->per_sm[0]; }
}

// the shape (0 primary, 1 alternative) of a direction's tile
template <typename C>
int shape_of(const C *c, const fpk::DirDev &D) {
  return c->nshape == 2 && D.S * D.TT == c->nt[1] ? 1 : 0;
}

// the switches are folded for characteristic FP sweeps with local speeds (not for WENOCU6,
// whose sweep measured 1 % slower with them folded)
int fix_of(int scheme, int charwise, int fp, int global_lf) {
  return charwise && fp && !global_lf && scheme != FP_WENOCU6 ? 1 : 0;
}

// the variant of the launch: boundary rules compiled in when some block of the launch has such a
// side in its direction, the switches folded as fix_of says
cudaError_t launch(int is_f32, const fpk::SweepLaunch &L, int M, int scheme, int charwise, int fp,
                   cudaStream_t s) {
  using F = cudaError_t (*)(const fpk::SweepLaunch &, int, int, int, int, cudaStream_t);
  const F f32[4] = {fpk::launch_sweep_f32, fpk::launch_sweep_f32_fix, fpk::launch_sweep_f32_bnd,
                    fpk::launch_sweep_f32_bnd_fix};
  const F f64[4] = {fpk::launch_sweep_f64, fpk::launch_sweep_f64_fix, fpk::launch_sweep_f64_bnd,
                    fpk::launch_sweep_f64_bnd_fix};
  const int fix = fix_of(scheme, charwise, fp, L.glf);
  if (is_f32 && fix && L.alt)
    return (L.bnd ? fpk::launch_sweep_f32_bnd_fix2 : fpk::launch_sweep_f32_fix2)(L, M, scheme, charwise, fp, s);
  return (is_f32 ? f32 : f64)[(L.bnd ? 2 : 0) + fix](L, M, scheme, charwise, fp, s);
}

// default tile of a direction for a CTA of nt threads: 32 faces along xi, 8 across lines
// elsewhere (32 lines of 8 faces at 256 threads)
void default_tile(int dir, int nt, int *S, int *TT) {
  *S = dir == 0 ? 32 : 8;
  *TT = nt / *S;
}

void fill_dirs(fp_ctx *c) {
  const int ni = c->desc.n[0], nj = c->desc.n[1], nk = c->desc.n[2], G = c->G;
  const int dims = c->desc.dims;
  const long long qs1 = ni, qs2 = (long long)ni * nj;
  const long long ei = ni + 2 * G, ej = nj + 2 * G;
  const long long ms1 = ei, ms2 = ei * ej;
  BlockDev &B = c->hblk;
  // direction 0: lines along i, transverse (j, k)
  {
    DirDev &D = B.dir[0];
    D.nd = ni; D.nt1 = nj; D.nlines = (long long)nj * nk;
    D.qT1 = qs1; D.qT2 = qs2; D.qsd = 1;
    D.mT1 = ms1; D.mT2 = ms2; D.msd = 1;
    D.fT1 = ni + 1; D.fT2 = (long long)(ni + 1) * nj; D.fsd = 1;
  }
  // direction 1: lines along j, transverse (i, k)
  {
    DirDev &D = B.dir[1];
    D.nd = nj; D.nt1 = ni; D.nlines = (long long)ni * nk;
    D.qT1 = 1; D.qT2 = qs2; D.qsd = qs1;
    D.mT1 = 1; D.mT2 = ms2; D.msd = ms1;
    D.fT1 = 1; D.fT2 = (long long)ni * (nj + 1); D.fsd = ni;
  }
  // direction 2: lines along k, transverse (i, j)
  {
    DirDev &D = B.dir[2];
    D.nd = nk; D.nt1 = ni; D.nlines = (long long)ni * nj;
    D.qT1 = 1; D.qT2 = qs1; D.qsd = qs2;
    D.mT1 = 1; D.mT2 = ms1; D.msd = ms2;
    D.fT1 = 1; D.fT2 = ni; D.fsd = (long long)ni * nj;
  }
  for (int d = 0; d < 3; ++d) {
    DirDev &D = B.dir[d];
    D.fc = c->nface[d];
    D.bclo = c->desc.bc[d][0];
    D.bchi = c->desc.bc[d][1];
    D.fmet = c->fmet[d];
    D.dk = c->dk[d];
    D.halo[0] = D.halo[1] = nullptr;
    // halo layout: the state layout with this direction's extent replaced by G
    {
      long long e[3] = {ni, nj, nk};
      e[d] = G;
      const long long s1 = e[0], s2 = e[0] * e[1];
      const long long st[3] = {1, s1, s2};
      const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;   // the line's t1 and t2 directions
      D.hsd = st[d];
      D.hT1 = st[ta];
      D.hT2 = st[tb];
      D.hc = e[0] * e[1] * e[2];
    }
    default_tile(d, c->nt[0], &D.S, &D.TT);
    if (d >= dims) D.nlines = 0;
  }
  B.dims = dims;
  B.G = G;
  B.qc = (long long)ni * nj * nk;
  B.mc = c->nmet;
  B.moff = G + G * ms1 + (dims == 3 ? G * ms2 : 0);
  B.met = c->met;
  B.q[0] = nullptr; B.q[1] = c->q1; B.q[2] = c->q2;
  B.racc = c->racc;
  B.dqdt = nullptr;
  for (int v = 0; v < 5; ++v) B.qbar[v] = c->desc.q_inf[v];
  B.gamma = c->desc.gamma;
  B.status = c->status;
  B.global_lf = c->desc.global_lf;
  B.lamg = c->lamg;
  B.cut = c->desc.cut_width;
  for (int d = 0; d < 3; ++d) B.nbr[d][0] = B.nbr[d][1] = -1;
}

void make_items(const BlockDev &B, int bidx, int d, std::vector<int2> &out) {
  const DirDev &D = B.dir[d];
  for (long long L0 = 0; L0 < D.nlines; L0 += D.TT) out.push_back(make_int2(bidx, (int)L0));
}

int upload_items(fp_ctx *c) {
  for (int d = 0; d < 3; ++d) {
    if (c->items[d]) { cudaFree(c->items[d]); c->items[d] = nullptr; }
    c->hitems[d].clear();
    if (d < c->desc.dims) make_items(c->hblk, 0, d, c->hitems[d]);
    c->nitems[d] = (int)c->hitems[d].size();
    if (c->nitems[d] == 0) continue;
    cudaError_t e = fpk::dev_alloc(&c->items[d], c->hitems[d].size() * sizeof(int2));
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(items)");
    e = cudaMemcpy(c->items[d], c->hitems[d].data(), c->hitems[d].size() * sizeof(int2),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy(items)");
  }
  return FP_OK;
}

int sync_block(fp_ctx *c, cudaStream_t s) {
  if (std::memcmp(&c->uploaded, &c->hblk, sizeof(BlockDev)) == 0) return FP_OK;
  cudaError_t e = cudaMemcpyAsync(c->dblk, &c->hblk, sizeof(BlockDev), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "upload block descriptor");
  c->uploaded = c->hblk;
  return FP_OK;
}

int grid_for(int per_sm, int nsm, int nitems) {
  long long g = (long long)per_sm * nsm;
  if (g > nitems) g = nitems;
  return g < 1 ? 1 : (int)g;
}

int validate(const fp_grid_desc *d, int ghost_nodes, std::string &why) {
  if (!d) { why = "desc is NULL"; return 0; }
  if (d->dims != 2 && d->dims != 3) { why = "dims must be 2 or 3"; return 0; }
  const int M = d->metric_order;
  if (M != 2 && M != 4 && M != 6 && M != 8) { why = "metric_order must be 2, 4, 6 or 8"; return 0; }
  if (d->scheme != FP_WENO5_JS && d->scheme != FP_LINEAR_UPWIND5 && d->scheme != FP_WENO7_JS &&
      d->scheme != FP_WENOCU6) { why = "unknown scheme"; return 0; }
  const int G = ghost_of(M, d->scheme);
  for (int k = 0; k < 3; ++k) {
    if (d->n[k] < 1) { why = "n must be positive"; return 0; }
    if (k < d->dims && d->n[k] < G) { why = "each swept extent must be at least the ghost width"; return 0; }
    if (k < d->dims && (long long)d->n[k] > (1LL << 20)) { why = "extent too large"; return 0; }
  }
  if (d->dims == 2 && d->n[2] != 1) { why = "n[2] must be 1 in 2-D"; return 0; }
  if ((long long)d->n[0] * d->n[1] * d->n[2] > (1LL << 31) - 1) { why = "too many points"; return 0; }
  if (d->precision != FP_F64 && d->precision != FP_F32_MIXED) { why = "unknown precision"; return 0; }
  if (d->free_stream_preserving != 0 && d->free_stream_preserving != 1) { why = "free_stream_preserving must be 0 or 1"; return 0; }
  if (d->characteristic != 0 && d->characteristic != 1) { why = "characteristic must be 0 or 1"; return 0; }
  if (d->global_lf != 0 && d->global_lf != 1) { why = "global_lf must be 0 or 1"; return 0; }
  for (int k = 0; k < d->dims; ++k)
    for (int s = 0; s < 2; ++s)
      if (d->bc[k][s] < 0 || d->bc[k][s] > FP_BC_HALO) { why = "unknown boundary code"; return 0; }
  if (d->global_lf && has_halo(*d)) { why = "global_lf with FP_BC_HALO sides (the speeds would be per block)"; return 0; }
  if (d->cut_width < 0) { why = "cut_width must be non-negative"; return 0; }
  if (!(d->gamma > 1.0) || !std::isfinite(d->gamma)) { why = "gamma must exceed 1"; return 0; }
  const double rho = d->q_inf[0];
  if (!(rho > 0.0)) { why = "q_inf density must be positive"; return 0; }
  double ke = 0.5 * (d->q_inf[1] * d->q_inf[1] + d->q_inf[2] * d->q_inf[2] + d->q_inf[3] * d->q_inf[3]) / rho;
  if (!((d->gamma - 1.0) * (d->q_inf[4] - ke) > 0.0)) { why = "q_inf pressure must be positive"; return 0; }
  if (ghost_nodes < G + 3 * (M / 2)) { why = "ghost_nodes below fp_node_ghost_width(metric_order, scheme)"; return 0; }
  return 1;
}

}  // namespace

extern "C" {

int fp_ghost_width(int metric_order, int scheme) { return ghost_of(metric_order, scheme); }
int fp_node_ghost_width(int metric_order, int scheme) {
  return ghost_of(metric_order, scheme) + 3 * (metric_order / 2);
}

size_t fp_state_bytes(const fp_ctx *c) { return c ? (size_t)5 * (size_t)c->ncells * c->esize : 0; }

const char *fp_status_string(int st) {
  switch (st) {
    case FP_OK: return "ok";
    case FP_ERR_ARG: return "invalid argument";
    case FP_ERR_CUDA: return "CUDA error";
    case FP_ERR_OOM: return "device out of memory";
    case FP_ERR_NONFINITE: return "non-finite state";
    case FP_ERR_TIMEOUT: return "device wait timed out";
    case FP_ERR_UNSUPPORTED: return "unsupported combination";
    case FP_ERR_BOUNDS: return "index outside its array (bounds-checking build)";
    default: return "unknown status";
  }
}

const char *fp_last_error(const fp_ctx *c) { return c ? c->err.c_str() : "null context"; }

void fp_free(fp_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cudaFree(c->met);
  for (int d = 0; d < 3; ++d) { cudaFree(c->fmet[d]); cudaFree(c->dk[d]); cudaFree(c->items[d]); }
  cudaFree(c->q1); cudaFree(c->q2); cudaFree(c->racc);
  cudaFree(c->status); cudaFree(c->dt_dev); cudaFree(c->cfl_bits); cudaFree(c->dblk);
  cudaFree(c->lamg); cudaFree(c->lam_items);
  delete c;
}

int fp_init_grid(const fp_grid_desc *desc, const double *xyz, int ghost_nodes, void *stream,
                 fp_ctx **out) {
  if (!out) return FP_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (!validate(desc, ghost_nodes, why) || !xyz) return FP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  fp_ctx *c = new fp_ctx();
  std::memset(&c->hblk, 0, sizeof(BlockDev));
  std::memset(&c->uploaded, 0xff, sizeof(BlockDev));
  c->desc = *desc;
  const int dims = desc->dims, M = desc->metric_order;
  c->G = ghost_of(M, desc->scheme);
  c->is_f32 = desc->precision == FP_F32_MIXED;
  c->esize = c->is_f32 ? sizeof(float) : sizeof(double);
  const int *n = desc->n;
  c->ncells = (long long)n[0] * n[1] * n[2];
  const int G = c->G, Gn = ghost_nodes, h = M / 2;
  auto ext = [&](int d, int g) -> long long { return d < dims ? n[d] + 2LL * g : 1LL; };
  const long long nnode = ext(0, Gn) * ext(1, Gn) * ext(2, Gn);
  const long long nb1 = ext(0, G + M) * ext(1, G + M) * ext(2, G + M);
  const long long nb2 = ext(0, G + h) * ext(1, G + h) * ext(2, G + h);
  c->nmet = ext(0, G) * ext(1, G) * ext(2, G);
  for (int d = 0; d < 3; ++d)
    c->nface[d] = d < dims ? c->ncells / n[d] * (n[d] + 1) : 0;

  cudaError_t e;
  double *nodes = nullptr, *met64 = nullptr, *scratch = nullptr, *fm64[3] = {nullptr, nullptr, nullptr};
  double *dk64[3] = {nullptr, nullptr, nullptr};
  auto cleanup_tmp = [&]() {
    cudaFree(nodes); cudaFree(scratch);
    if (c->is_f32) {
      cudaFree(met64);
      for (int d = 0; d < 3; ++d) { cudaFree(fm64[d]); cudaFree(dk64[d]); }
    }
  };
#define FP_TRY(call, where)                         \
  do {                                              \
    e = (call);                                     \
    if (e != cudaSuccess) {                         \
      int st = cuda_fail(c, e, where);              \
      cleanup_tmp();                                \
      std::fprintf(stderr, "fp_init_grid: %s\n", c->err.c_str()); \
      fp_free(c);                                   \
      return st;                                    \
    }                                               \
  } while (0)
  FP_TRY(fpk::dev_alloc(&nodes, (size_t)dims * nnode * sizeof(double)), "cudaMalloc(nodes)");
  FP_TRY(cudaGetDevice(&c->dev), "cudaGetDevice");
  FP_TRY(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev), "device attribute");
  FP_TRY(noalloc_prepare(c->dev), "static scratch of fp_rhs_noalloc");
  FP_TRY(cudaMemcpyAsync(nodes, xyz, (size_t)dims * nnode * sizeof(double), cudaMemcpyHostToDevice, s),
         "copy nodes");
  FP_TRY(fpk::dev_alloc(&met64, (size_t)10 * c->nmet * sizeof(double)), "cudaMalloc(metrics)");
  for (int d = 0; d < dims; ++d) {
    FP_TRY(fpk::dev_alloc(&fm64[d], (size_t)3 * c->nface[d] * sizeof(double)), "cudaMalloc(face metrics)");
    FP_TRY(fpk::dev_alloc(&dk64[d], (size_t)3 * c->ncells * sizeof(double)), "cudaMalloc(metric differences)");
  }
  FP_TRY(fpk::dev_alloc(&scratch, (size_t)9 * (nb1 + nb2) * sizeof(double)), "cudaMalloc(metric scratch)");
  fpk::MetricJob J;
  J.dims = dims; J.M = M; J.G = G; J.Gn = Gn;
  for (int d = 0; d < 3; ++d) { J.n[d] = n[d]; J.fmet[d] = fm64[d]; J.dk[d] = dk64[d]; }
  J.nodes = nodes; J.met = met64; J.scratch = scratch;
  FP_TRY(fpk::build_metrics(J, s), "build metrics");
  if (c->is_f32) {
    FP_TRY(fpk::dev_alloc(&c->met, (size_t)10 * c->nmet * sizeof(float)), "cudaMalloc(metrics f32)");
    FP_TRY(fpk::convert_f64_to_f32(met64, (float *)c->met, 10 * c->nmet, s), "convert metrics");
    for (int d = 0; d < dims; ++d) {
      FP_TRY(fpk::dev_alloc(&c->fmet[d], (size_t)3 * c->nface[d] * sizeof(float)), "cudaMalloc(face f32)");
      FP_TRY(fpk::convert_f64_to_f32(fm64[d], (float *)c->fmet[d], 3 * c->nface[d], s), "convert face metrics");
      FP_TRY(fpk::dev_alloc(&c->dk[d], (size_t)3 * c->ncells * sizeof(float)), "cudaMalloc(differences f32)");
      FP_TRY(fpk::convert_f64_to_f32(dk64[d], (float *)c->dk[d], 3 * c->ncells, s), "convert differences");
    }
  } else {
    c->met = met64;
    for (int d = 0; d < 3; ++d) { c->fmet[d] = fm64[d]; c->dk[d] = dk64[d]; }
  }
  FP_TRY(cudaStreamSynchronize(s), "metric construction");
  cleanup_tmp();
  nodes = nullptr; scratch = nullptr;
  if (c->is_f32) { met64 = nullptr; for (int d = 0; d < 3; ++d) { fm64[d] = nullptr; dk64[d] = nullptr; } }
  const size_t sbytes = (size_t)5 * c->ncells * c->esize;
  FP_TRY(fpk::dev_alloc(&c->q1, sbytes), "cudaMalloc(stage 1)");
  FP_TRY(fpk::dev_alloc(&c->q2, sbytes), "cudaMalloc(stage 2)");
  FP_TRY(fpk::dev_alloc(&c->racc, sbytes), "cudaMalloc(residual)");
  FP_TRY(fpk::dev_alloc(&c->status, sizeof(int)), "cudaMalloc(status)");
  FP_TRY(cudaMemset(c->status, 0, sizeof(int)), "clear status");
  FP_TRY(fpk::dev_alloc(&c->dt_dev, sizeof(double)), "cudaMalloc(dt)");
  FP_TRY(fpk::dev_alloc(&c->cfl_bits, sizeof(unsigned long long)), "cudaMalloc(cfl)");
  FP_TRY(fpk::dev_alloc(&c->dblk, sizeof(BlockDev)), "cudaMalloc(block)");
  FP_TRY(fpk::dev_alloc(&c->lamg, 9 * c->esize), "cudaMalloc(global speeds)");
  FP_TRY(cudaMemset(c->lamg, 0, 9 * c->esize), "clear global speeds");
  {
    std::vector<int2> li;
    for (long long p0 = 0; p0 < c->ncells; p0 += fpk::kLamChunk) li.push_back(make_int2(0, (int)p0));
    c->nlam_items = (int)li.size();
    FP_TRY(fpk::dev_alloc(&c->lam_items, li.size() * sizeof(int2)), "cudaMalloc(speed items)");
    FP_TRY(cudaMemcpy(c->lam_items, li.data(), li.size() * sizeof(int2), cudaMemcpyHostToDevice),
           "copy speed items");
  }
  {
    const int fix = fix_of(desc->scheme, desc->characteristic, desc->free_stream_preserving, desc->global_lf);
    set_shapes(c, c->is_f32, M, desc->scheme, fix);
    fill_dirs(c);
  }
  FP_TRY(cudaGetLastError(), "prepare sweep kernels");
  // a block too small to fill the resident CTAs with the default tiles of the eta and zeta
  // passes (8 faces per chunk) takes 32 faces per chunk there: four times the work items,
  // each a quarter as long (batches pick their tiles by timing them instead)
  for (int d = 1; d < c->desc.dims; ++d) {
    DirDev &D = c->hblk.dir[d];
    if ((D.nlines + D.TT - 1) / D.TT < (long long)c->per_sm[0] * c->nsm) { D.S = 32; D.TT = c->nt[0] / 32; }
  }
  int st = upload_items(c);
  if (st != FP_OK) { fp_free(c); return st; }
#undef FP_TRY
  *out = c;
  return FP_OK;
}

// the direction passes of one RK stage (rk = 1: the last pass applies the stage update) or
// of one residual (rk = 0)
static int run_stage(fp_ctx *c, int stage, int rk, cudaStream_t s) {
  const int dims = c->desc.dims, M = c->desc.metric_order;
  if (c->desc.global_lf) {
    cudaError_t e = fpk::launch_lambda(c->dblk, 1, c->lam_items, c->nlam_items, c->is_f32,
                                       c->desc.characteristic, stage, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "global speed launch");
  }
  for (int d = 0; d < dims; ++d) {
    fpk::SweepLaunch L;
    L.blocks = c->dblk;
    L.items = c->items[d];
    L.nitems = c->nitems[d];
    L.dir = d;
    L.mode = d == 0 ? fpk::MODE_WRITE : (d == dims - 1 ? (rk ? fpk::MODE_RK : fpk::MODE_RHS) : fpk::MODE_ADD);
    L.stage = stage;
    L.dt = c->dt_dev;
    L.alt = shape_of(c, c->hblk.dir[d]);
    L.grid = grid_for(c->per_sm[L.alt], c->nsm, L.nitems);
    L.bnd = has_bnd(c->desc, d);
    L.glf = c->desc.global_lf;
    cudaError_t e = launch(c->is_f32, L, M, c->desc.scheme, c->desc.characteristic,
                           c->desc.free_stream_preserving, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep launch");
  }
  return FP_OK;
}

static int run_passes(fp_ctx *c, int rk, cudaStream_t s) {
  for (int stage = 0; stage < (rk ? 3 : 1); ++stage) {
    int st = run_stage(c, stage, rk, s);
    if (st) return st;
  }
  return FP_OK;
}

// every FP_BC_HALO side has its buffer
static int halos_set(fp_ctx *c, const char *who) {
  for (int d = 0; d < c->desc.dims; ++d)
    for (int sd = 0; sd < 2; ++sd)
      if (c->desc.bc[d][sd] == FP_BC_HALO && !c->hblk.dir[d].halo[sd])
        return fail(c, FP_ERR_ARG, std::string(who) + ": an FP_BC_HALO side has no halo buffer (fp_set_halo)");
  return FP_OK;
}

int fp_rhs(fp_ctx *c, const void *q, void *dqdt, void *stream) {
  if (!c) return FP_ERR_ARG;
  if (!q || !dqdt) return fail(c, FP_ERR_ARG, "fp_rhs: null buffer");
  if (has_link(c->desc)) return fail(c, FP_ERR_ARG, "fp_rhs: FP_BC_BLOCK sides need a linked batch");
  if (int st = halos_set(c, "fp_rhs")) return st;
  cudaStream_t s = (cudaStream_t)stream;
  c->hblk.q[0] = const_cast<void *>(q);
  c->hblk.dqdt = dqdt;
  int st = sync_block(c, s);
  if (st) return st;
  return run_passes(c, 0, s);
}

int fp_rk3_step(fp_ctx *c, void *q, double dt, void *stream) {
  if (!c) return FP_ERR_ARG;
  if (!q) return fail(c, FP_ERR_ARG, "fp_rk3_step: null state");
  if (!std::isfinite(dt)) return fail(c, FP_ERR_ARG, "fp_rk3_step: dt not finite");
  if (has_link(c->desc)) return fail(c, FP_ERR_ARG, "fp_rk3_step: FP_BC_BLOCK sides need a linked batch");
  if (has_halo(c->desc))
    return fail(c, FP_ERR_ARG, "fp_rk3_step: FP_BC_HALO sides need their halos refreshed between stages (fp_rk3_stage)");
  cudaStream_t s = (cudaStream_t)stream;
  c->hblk.q[0] = q;
  int st = sync_block(c, s);
  if (st) return st;
  c->dt_host = dt;
  cudaError_t e = cudaMemcpyAsync(c->dt_dev, &c->dt_host, sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "upload dt");
  return run_passes(c, 1, s);
}

int fp_rk3_stage(fp_ctx *c, void *q, double dt, int stage, void *stream) {
  if (!c) return FP_ERR_ARG;
  if (!q) return fail(c, FP_ERR_ARG, "fp_rk3_stage: null state");
  if (stage < 0 || stage > 2) return fail(c, FP_ERR_ARG, "fp_rk3_stage: stage must be 0, 1 or 2");
  if (!std::isfinite(dt)) return fail(c, FP_ERR_ARG, "fp_rk3_stage: dt not finite");
  if (has_link(c->desc)) return fail(c, FP_ERR_ARG, "fp_rk3_stage: FP_BC_BLOCK sides need a linked batch");
  if (int st = halos_set(c, "fp_rk3_stage")) return st;
  cudaStream_t s = (cudaStream_t)stream;
  c->hblk.q[0] = q;
  int st = sync_block(c, s);
  if (st) return st;
  if (stage == 0) {   // one dt for the three stages of a step
    c->dt_host = dt;
    cudaError_t e = cudaMemcpyAsync(c->dt_dev, &c->dt_host, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload dt");
  }
  return run_stage(c, stage, 1, s);
}

int fp_set_halo(fp_ctx *c, int dir, int side, void *halo_dev) {
  if (!c) return FP_ERR_ARG;
  if (dir < 0 || dir >= c->desc.dims || side < 0 || side > 1 || !halo_dev)
    return fail(c, FP_ERR_ARG, "fp_set_halo: bad direction, side or buffer");
  if (c->desc.bc[dir][side] != FP_BC_HALO) return fail(c, FP_ERR_ARG, "fp_set_halo: that side is not FP_BC_HALO");
  c->hblk.dir[dir].halo[side] = halo_dev;
  return FP_OK;
}

size_t fp_halo_bytes(const fp_ctx *c, int dir) {
  if (!c || dir < 0 || dir >= c->desc.dims) return 0;
  return (size_t)5 * (size_t)(c->ncells / c->desc.n[dir]) * (size_t)c->G * c->esize;
}

int fp_pack_halo(fp_ctx *c, const void *q, int stage, int dir, int side, void *out_dev, void *stream) {
  if (!c) return FP_ERR_ARG;
  if (!q || !out_dev || stage < 0 || stage > 2 || dir < 0 || dir >= c->desc.dims || side < 0 || side > 1)
    return fail(c, FP_ERR_ARG, "fp_pack_halo: bad argument");
  const void *src = stage == 0 ? q : (stage == 1 ? c->q1 : c->q2);
  cudaError_t e =
      fpk::launch_pack_halo(src, c->is_f32, dir, side, c->G, c->desc.n, out_dev, c->status, (cudaStream_t)stream);
  return e == cudaSuccess ? FP_OK : cuda_fail(c, e, "fp_pack_halo");
}

int fp_cfl_dt(fp_ctx *c, const void *q, double cfl, double *dt_out, void *stream) {
  if (!c) return FP_ERR_ARG;
  if (!q || !dt_out || !(cfl > 0.0)) return fail(c, FP_ERR_ARG, "fp_cfl_dt: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  c->hblk.q[0] = const_cast<void *>(q);
  int st = sync_block(c, s);
  if (st) return st;
  cudaError_t e = cudaMemsetAsync(c->cfl_bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "cfl clear");
  e = fpk::launch_cfl(c->dblk, c->is_f32, c->ncells, c->desc.n, c->desc.dims, c->cfl_bits, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "cfl launch");
  unsigned long long bits = 0;
  e = cudaMemcpyAsync(&bits, c->cfl_bits, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "cfl readback");
  double mx;
  std::memcpy(&mx, &bits, sizeof(mx));
  if (!(mx > 0.0) || !std::isfinite(mx)) return fail(c, FP_ERR_NONFINITE, "fp_cfl_dt: spectral radius not positive");
  *dt_out = cfl / mx;
  return FP_OK;
}

int fp_get_metrics(fp_ctx *c, double *host_out) {
  if (!c) return FP_ERR_ARG;
  if (!host_out) return fail(c, FP_ERR_ARG, "fp_get_metrics: null output");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "fp_get_metrics");
  const long long n = 10 * c->nmet;
  if (c->is_f32) {
    std::vector<float> tmp(n);
    e = cudaMemcpy(tmp.data(), c->met, n * sizeof(float), cudaMemcpyDeviceToHost);
    for (long long i = 0; i < n; ++i) host_out[i] = tmp[i];
  } else {
    e = cudaMemcpy(host_out, c->met, n * sizeof(double), cudaMemcpyDeviceToHost);
  }
  return e == cudaSuccess ? FP_OK : cuda_fail(c, e, "fp_get_metrics copy");
}

int fp_get_face_metrics(fp_ctx *c, int dir, double *host_out) {
  if (!c) return FP_ERR_ARG;
  if (!host_out || dir < 0 || dir >= c->desc.dims) return fail(c, FP_ERR_ARG, "fp_get_face_metrics: bad argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "fp_get_face_metrics");
  const long long n = 3 * c->nface[dir];
  if (c->is_f32) {
    std::vector<float> tmp(n);
    e = cudaMemcpy(tmp.data(), c->fmet[dir], n * sizeof(float), cudaMemcpyDeviceToHost);
    for (long long i = 0; i < n; ++i) host_out[i] = tmp[i];
  } else {
    e = cudaMemcpy(host_out, c->fmet[dir], n * sizeof(double), cudaMemcpyDeviceToHost);
  }
  return e == cudaSuccess ? FP_OK : cuda_fail(c, e, "fp_get_face_metrics copy");
}

int fp_get_device_status(fp_ctx *c, void *stream) {
  if (!c) return FP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, c->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "fp_get_device_status");
  if (word & fpk::ST_BOUNDS) return fail(c, FP_ERR_BOUNDS, "a kernel met an index outside its array (access redirected)");
  if (word & fpk::ST_NONFINITE) return fail(c, FP_ERR_NONFINITE, "a stage produced a non-finite state");
  return FP_OK;
}

int fp_bounds_checking(void) {
#ifdef FPK_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

int fp_launches_per_rhs(const fp_ctx *c) { return c ? c->desc.dims + (c->desc.global_lf ? 2 : 0) : 0; }
int fp_launches_per_step(const fp_ctx *c) { return c ? 3 * fp_launches_per_rhs(c) : 0; }

int fp_get_cta_sizes(const fp_ctx *c, int *primary, int *alternative) {
  if (!c || !primary || !alternative) return FP_ERR_ARG;
  *primary = c->nt[0];
  *alternative = c->nshape == 2 ? c->nt[1] : 0;
  return FP_OK;
}

int fp_get_tile(const fp_ctx *c, int dir, int *faces, int *lines) {
  if (!c || dir < 0 || dir > 2 || !faces || !lines) return FP_ERR_ARG;
  *faces = c->hblk.dir[dir].S;
  *lines = c->hblk.dir[dir].TT;
  return FP_OK;
}

int fp_set_tile(fp_ctx *c, int dir, int faces, int lines) {
  if (!c) return FP_ERR_ARG;
  if (dir < 0 || dir >= c->desc.dims) return fail(c, FP_ERR_ARG, "fp_set_tile: bad direction");
  const int a = c->nshape == 2 && faces * lines == c->nt[1] ? 1 : 0;
  if (!(faces == 8 || faces == 16 || faces == 32) || faces * lines != c->nt[a])
    return fail(c, FP_ERR_ARG, "fp_set_tile: faces in {8,16,32} and faces*lines one of the sweep's CTA sizes "
                               "(fp_get_cta_sizes)");
  if (dir == 0 && !c->pad[a] && faces != 32)
    return fail(c, FP_ERR_ARG, "fp_set_tile: this CTA size's xi rings are unpadded: 32 faces per chunk only");
  c->hblk.dir[dir].S = faces;
  c->hblk.dir[dir].TT = lines;
  return upload_items(c);
}

// ----------------------------------------------------------------- batches

void fp_batch_free(fp_batch *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->dblk);
  for (int d = 0; d < 3; ++d) cudaFree(b->items[d]);
  for (int g = 0; g < fp_batch::kMaxBranch; ++g)
    for (int d = 0; d < 3; ++d) cudaFree(b->bitems[g][d]);
  cudaFree(b->dt_dev);
  if (b->dt_host) cudaFreeHost(b->dt_host);
  if (b->dt_ready) cudaEventDestroy(b->dt_ready);
  cudaFree(b->lam_items);
  delete b;
}

const char *fp_batch_last_error(const fp_batch *b) { return b ? b->err.c_str() : "null batch"; }

int fp_batch_get_tile(const fp_batch *b, int block, int dir, int *faces, int *lines) {
  if (!b || block < 0 || block >= (int)b->hblk.size() || dir < 0 || dir > 2 || !faces || !lines) return FP_ERR_ARG;
  *faces = b->hblk[block].dir[dir].S;
  *lines = b->hblk[block].dir[dir].TT;
  return FP_OK;
}

int fp_batch_launches_per_step(const fp_batch *b) {
  return b ? b->nbranch * 3 * (b->dims + (b->global_lf ? 2 : 0)) : 0;
}

static int batch_items_into(fp_batch *b, int d, const std::vector<int> *only_blocks, int2 **dst, int *ndst);

static int batch_items(fp_batch *b, int d, const std::vector<int> *only_blocks) {
  return batch_items_into(b, d, only_blocks, &b->items[d], &b->nitems[d]);
}

static int batch_items_into(fp_batch *b, int d, const std::vector<int> *only_blocks, int2 **dst, int *ndst) {
  std::vector<std::pair<long long, int2>> work;
  for (size_t k = 0; k < b->hblk.size(); ++k) {
    if (only_blocks && std::find(only_blocks->begin(), only_blocks->end(), (int)k) == only_blocks->end())
      continue;
    const DirDev &D = b->hblk[k].dir[d];
    for (long long L0 = 0; L0 < D.nlines; L0 += D.TT) {
      long long lines = std::min<long long>(D.TT, D.nlines - L0);
      work.push_back({(long long)D.nd * lines, make_int2((int)k, (int)L0)});
    }
  }
  // largest items first: the persistent grid takes them in order
  std::stable_sort(work.begin(), work.end(),
                   [](const std::pair<long long, int2> &x, const std::pair<long long, int2> &y) {
                     return x.first > y.first;
                   });
  std::vector<int2> it(work.size());
  for (size_t k = 0; k < work.size(); ++k) it[k] = work[k].second;
  cudaFree(*dst);
  *dst = nullptr;
  *ndst = (int)it.size();
  if (it.empty()) return FP_OK;
  cudaError_t e = fpk::dev_alloc(dst, it.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, it.data(), it.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess)
    return bfail(b, e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA,
                 std::string("batch items: ") + cudaGetErrorString(e));
  return FP_OK;
}

static int batch_upload(fp_batch *b, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b->dblk, b->hblk.data(), b->hblk.size() * sizeof(BlockDev),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  return FP_OK;
}

static int batch_pass_items(fp_batch *b, int d, int mode, int stage, cudaStream_t s, const int2 *items,
                            int nitems) {
  fpk::SweepLaunch L;
  L.blocks = b->dblk;
  L.items = items;
  L.nitems = nitems;
  L.dir = d;
  L.mode = mode;
  L.stage = stage;
  L.dt = b->dt_dev;
  L.alt = shape_of(b, b->hblk[0].dir[d]);   // every block of a batch pass has the same shape
  L.grid = grid_for(b->per_sm[L.alt], b->nsm, L.nitems);
  L.bnd = b->bnd[d];
  L.glf = b->global_lf;
  cudaError_t e = launch(b->is_f32, L, b->M, b->scheme, b->charwise, b->fp, s);
  if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("batch sweep: ") + cudaGetErrorString(e));
  return FP_OK;
}

static int batch_pass(fp_batch *b, int d, int mode, int stage, cudaStream_t s) {
  return batch_pass_items(b, d, mode, stage, s, b->items[d], b->nitems[d]);
}

// Autotuner: for the batch's CTA shape, each direction and each line-length class, time every
// tile of that shape on the blocks of that class and keep the best (tiles[a][d][k]: block k's
// faces per chunk in direction d).
static int batch_autotune(fp_batch *b, cudaStream_t s, std::vector<int> tiles[2][3]) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  constexpr int nclass = 3;
  int st = FP_OK;
  for (int a = b->shape; a == b->shape && !st; ++a)
    for (int d = 0; d < 3 && !st; ++d) {
      tiles[a][d].assign(b->hblk.size(), 32);
      if (d >= b->dims) continue;
      std::vector<int> members[nclass];
      for (size_t k = 0; k < b->hblk.size(); ++k) {
        const int nd = b->hblk[k].dir[d].nd;
        members[nd < 64 ? 0 : (nd < 96 ? 1 : 2)].push_back((int)k);
      }
      for (auto &B : b->hblk) { B.dir[d].S = 32; B.dir[d].TT = b->nt[a] / 32; }   // the pass's shape: a
      for (int cl = 0; cl < nclass && !st; ++cl) {
        if (members[cl].empty()) continue;
        float best = 1e30f;
        int bestS = 32;
        for (int S : {32, 16, 8}) {
          if (d == 0 && !b->pad[a] && S != 32) continue;   // unpadded xi rings: S = 32 only
          for (int k : members[cl]) { b->hblk[k].dir[d].S = S; b->hblk[k].dir[d].TT = b->nt[a] / S; }
          st = batch_upload(b, s);
          if (!st) st = batch_items(b, d, &members[cl]);
          if (!st) st = batch_pass(b, d, fpk::MODE_WRITE, 0, s);           // warm-up
          if (st) break;
          cudaEventRecord(e0, s);
          for (int r = 0; r < 3; ++r) batch_pass(b, d, fpk::MODE_WRITE, 0, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best) { best = ms; bestS = S; }
        }
        for (int k : members[cl]) tiles[a][d][k] = bestS;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  return FP_OK;
}

// the tiles of shape a from the autotuner's table
static void batch_set_tiles(fp_batch *b, int a, std::vector<int> tiles[2][3]) {
  for (int d = 0; d < b->dims; ++d)
    for (size_t k = 0; k < b->hblk.size(); ++k) {
      b->hblk[k].dir[d].S = tiles[a][d][k];
      b->hblk[k].dir[d].TT = b->nt[a] / tiles[a][d][k];
    }
}

int fp_batch_create(fp_ctx *const *blocks, int nblocks, void *const *q_devs, int autotune,
                    void *stream, fp_batch **out) {
  return fp_batch_create_linked(blocks, nblocks, q_devs, nullptr, 0, autotune, stream, out);
}

int fp_batch_create_linked(fp_ctx *const *blocks, int nblocks, void *const *q_devs,
                           const fp_block_link *links, int nlinks, int autotune, void *stream,
                           fp_batch **out) {
  if (!out) return FP_ERR_ARG;
  *out = nullptr;
  if (!blocks || !q_devs || nblocks < 1 || nlinks < 0 || (nlinks > 0 && !links)) return FP_ERR_ARG;
  for (int k = 0; k < nblocks; ++k)
    if (!blocks[k] || !q_devs[k] || has_halo(blocks[k]->desc)) return FP_ERR_ARG;
  // every FP_BC_BLOCK side linked exactly once, to a block with the same transverse extents
  std::vector<int> nbr((size_t)nblocks * 6, -1);
  for (int l = 0; l < nlinks; ++l) {
    const fp_block_link &L = links[l];
    if (L.a < 0 || L.a >= nblocks || L.b < 0 || L.b >= nblocks || L.side < 0 || L.side > 1) return FP_ERR_ARG;
    const fp_grid_desc &da = blocks[L.a]->desc, &db = blocks[L.b]->desc;
    if (L.dir < 0 || L.dir >= da.dims || da.bc[L.dir][L.side] != FP_BC_BLOCK) return FP_ERR_ARG;
    for (int e = 0; e < 3; ++e)
      if (e != L.dir && da.n[e] != db.n[e]) return FP_ERR_ARG;
    int &slot = nbr[(size_t)L.a * 6 + L.dir * 2 + L.side];
    if (slot >= 0) return FP_ERR_ARG;
    slot = L.b;
  }
  for (int k = 0; k < nblocks; ++k)
    for (int d = 0; d < blocks[k]->desc.dims; ++d)
      for (int sd = 0; sd < 2; ++sd)
        if (blocks[k]->desc.bc[d][sd] == FP_BC_BLOCK && nbr[(size_t)k * 6 + d * 2 + sd] < 0) return FP_ERR_ARG;
  const fp_grid_desc &d0 = blocks[0]->desc;
  for (int k = 1; k < nblocks; ++k) {
    const fp_grid_desc &d = blocks[k]->desc;
    if (d.dims != d0.dims || d.metric_order != d0.metric_order || d.scheme != d0.scheme ||
        d.precision != d0.precision || d.characteristic != d0.characteristic ||
        d.free_stream_preserving != d0.free_stream_preserving || d.global_lf != d0.global_lf)
      return FP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  fp_batch *b = new fp_batch();
  b->dims = d0.dims; b->M = d0.metric_order; b->scheme = d0.scheme;
  b->charwise = d0.characteristic; b->fp = d0.free_stream_preserving;
  b->is_f32 = d0.precision == FP_F32_MIXED;
  b->global_lf = d0.global_lf;
  b->nshape = blocks[0]->nshape;
  for (int a = 0; a < 2; ++a) {
    b->nt[a] = blocks[0]->nt[a];
    b->pad[a] = blocks[0]->pad[a];
    b->per_sm[a] = blocks[0]->per_sm[a];
  }
  b->shape = fpk::sweep_batch_shape(b->is_f32, b->scheme, fix_of(b->scheme, b->charwise, b->fp, b->global_lf));
  b->nsm = blocks[0]->nsm;
  for (int k = 0; k < nblocks; ++k) {
    b->ctx.push_back(blocks[k]);
    for (int d = 0; d < 3; ++d) b->bnd[d] |= has_bnd(blocks[k]->desc, d);
    BlockDev B = blocks[k]->hblk;
    B.q[0] = q_devs[k];
    B.dqdt = nullptr;
    for (int d = 0; d < 3; ++d)
      for (int sd = 0; sd < 2; ++sd) B.nbr[d][sd] = nbr[(size_t)k * 6 + d * 2 + sd];
    b->hblk.push_back(B);
  }
  // the batch runs one CTA shape: the blocks' own tiles where they are of that shape, the
  // defaults of that shape elsewhere
  for (int d = 0; d < 3; ++d)
    for (auto &B : b->hblk)
      if (B.dir[d].S * B.dir[d].TT != b->nt[b->shape]) default_tile(d, b->nt[b->shape], &B.dir[d].S, &B.dir[d].TT);
  cudaError_t e = fpk::dev_alloc(&b->dblk, nblocks * sizeof(BlockDev));
  if (e == cudaSuccess) e = fpk::dev_alloc(&b->dt_dev, sizeof(double));
  if (e == cudaSuccess) e = fpk::host_malloc(reinterpret_cast<void **>(&b->dt_host), sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->dt_ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dt_dev, 0, sizeof(double), s);
  if (e != cudaSuccess) { fp_batch_free(b); return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA; }
  {
    std::vector<int2> li;
    for (int k = 0; k < nblocks; ++k)
      for (long long p0 = 0; p0 < blocks[k]->ncells; p0 += fpk::kLamChunk) li.push_back(make_int2(k, (int)p0));
    b->nlam_items = (int)li.size();
    e = fpk::dev_alloc(&b->lam_items, li.size() * sizeof(int2));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->lam_items, li.data(), li.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { fp_batch_free(b); return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA; }
  }
  int st = FP_OK;
  if (autotune) {
    std::vector<int> tiles[2][3];
    st = batch_autotune(b, s, tiles);
    if (!st) batch_set_tiles(b, b->shape, tiles);
  }
  if (!st) st = batch_upload(b, s);
  for (int d = 0; d < b->dims && !st; ++d) st = batch_items(b, d, nullptr);
  if (st) { std::fprintf(stderr, "fp_batch_create: %s\n", b->err.c_str()); fp_batch_free(b); return st; }
  // graph branches: blocks split into groups of about equal point count, each group's
  // items built separately
  if (!b->global_lf && nlinks == 0 && nblocks >= 2) {
    b->nbranch = std::min(nblocks, (int)fp_batch::kMaxBranch);
    std::vector<long long> weight(nblocks);
    for (int k = 0; k < nblocks; ++k) weight[k] = blocks[k]->ncells;
    std::vector<int> group_of(nblocks);
    fp_balanced_groups(weight.data(), nblocks, b->nbranch, group_of.data());
    std::vector<std::vector<int>> grp(b->nbranch);
    for (int k = 0; k < nblocks; ++k) grp[group_of[k]].push_back(k);
    for (int g = 0; g < b->nbranch && !st; ++g)
      for (int d = 0; d < b->dims && !st; ++d) st = batch_items_into(b, d, &grp[g], &b->bitems[g][d], &b->bnitems[g][d]);
    if (st) { fp_batch_free(b); return st; }
  }
  // capture the three RK stages x directions into one graph (one chain per branch)
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) { fp_batch_free(b); return FP_ERR_CUDA; }
  cudaStream_t bs[fp_batch::kMaxBranch] = {};
  cudaEvent_t fork = nullptr, join[fp_batch::kMaxBranch] = {};
  if (b->nbranch > 1) {
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int g = 0; g < b->nbranch && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&bs[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[g], cudaEventDisableTiming);
    }
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess && b->nbranch > 1) {
    e = cudaEventRecord(fork, cs);
    for (int g = 0; g < b->nbranch && e == cudaSuccess && !st; ++g) {
      e = cudaStreamWaitEvent(bs[g], fork, 0);
      for (int stage = 0; stage < 3 && !st && e == cudaSuccess; ++stage)
        for (int d = 0; d < b->dims && !st; ++d) {
          int mode = d == 0 ? fpk::MODE_WRITE : (d == b->dims - 1 ? fpk::MODE_RK : fpk::MODE_ADD);
          st = batch_pass_items(b, d, mode, stage, bs[g], b->bitems[g][d], b->bnitems[g][d]);
        }
      if (e == cudaSuccess) e = cudaEventRecord(join[g], bs[g]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, join[g], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
    if (e == cudaSuccess) e = e2;
  } else if (e == cudaSuccess) {
    for (int stage = 0; stage < 3 && !st; ++stage) {
      if (b->global_lf) {
        cudaError_t el = fpk::launch_lambda(b->dblk, (int)b->hblk.size(), b->lam_items, b->nlam_items,
                                            b->is_f32, b->charwise, stage, cs);
        if (el != cudaSuccess) st = bfail(b, FP_ERR_CUDA, "batch speed launch");
      }
      for (int d = 0; d < b->dims && !st; ++d) {
        int mode = d == 0 ? fpk::MODE_WRITE : (d == b->dims - 1 ? fpk::MODE_RK : fpk::MODE_ADD);
        st = batch_pass(b, d, mode, stage, cs);
      }
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && !st) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cs);
  for (int g = 0; g < fp_batch::kMaxBranch; ++g) {
    if (bs[g]) cudaStreamDestroy(bs[g]);
    if (join[g]) cudaEventDestroy(join[g]);
  }
  if (fork) cudaEventDestroy(fork);
  if (e != cudaSuccess || st) {
    std::fprintf(stderr, "fp_batch_create: graph: %s %s\n", cudaGetErrorString(e), b->err.c_str());
    fp_batch_free(b);
    return st ? st : FP_ERR_CUDA;
  }
  *out = b;
  return FP_OK;
}

int fp_batch_rk3_step(fp_batch *b, double dt, void *stream) {
  if (!b) return FP_ERR_ARG;
  if (!std::isfinite(dt)) return bfail(b, FP_ERR_ARG, "dt not finite");
  cudaStream_t s = (cudaStream_t)stream;
  // the previous step's upload must have been consumed before the pinned value is reused
  cudaError_t e = cudaEventSynchronize(b->dt_ready);
  if (e == cudaSuccess) {
    *b->dt_host = dt;
    e = cudaMemcpyAsync(b->dt_dev, b->dt_host, sizeof(double), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->dt_ready, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
  return FP_OK;
}

int fp_batch_rhs(fp_batch *b, void *const *dqdt_devs, void *stream) {
  if (!b) return FP_ERR_ARG;
  if (!dqdt_devs) return bfail(b, FP_ERR_ARG, "null outputs");
  cudaStream_t s = (cudaStream_t)stream;
  for (size_t k = 0; k < b->hblk.size(); ++k) {
    if (!dqdt_devs[k]) return bfail(b, FP_ERR_ARG, "null output");
    b->hblk[k].dqdt = dqdt_devs[k];
  }
  int st = batch_upload(b, s);
  if (!st && b->global_lf) {
    cudaError_t el = fpk::launch_lambda(b->dblk, (int)b->hblk.size(), b->lam_items, b->nlam_items, b->is_f32,
                                        b->charwise, 0, s);
    if (el != cudaSuccess) st = bfail(b, FP_ERR_CUDA, "batch speed launch");
  }
  for (int d = 0; d < b->dims && !st; ++d) {
    int mode = d == 0 ? fpk::MODE_WRITE : (d == b->dims - 1 ? fpk::MODE_RHS : fpk::MODE_ADD);
    st = batch_pass(b, d, mode, 0, s);
  }
  return st;
}

}  // extern "C"

// ----------------------------------------------------------------- allocation-free residual
//
// fp_rhs_noalloc: the residual of fp_rhs for callers that cannot allocate device memory
// where they evaluate it.  Same kernels, same data, same result bit for bit; the shared
// residual accumulator is the static scratch above instead of context memory.
extern "C" int fp_rhs_noalloc(fp_ctx *c, const void *q, void *dqdt, void *stream) {
  if (!c) return FP_ERR_ARG;
  if (!q || !dqdt) return fail(c, FP_ERR_ARG, "fp_rhs_noalloc: null buffer");
  if (has_link(c->desc)) return fail(c, FP_ERR_ARG, "fp_rhs_noalloc: FP_BC_BLOCK sides need a linked batch");
  if (int st = halos_set(c, "fp_rhs_noalloc")) return st;
  const size_t need = (size_t)5 * (size_t)c->ncells * c->esize;
  if (need > kNoAllocScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "fp_rhs_noalloc: the block needs %zu bytes of residual scratch but the static "
                  "scratch holds %zu (at most %zu points in FP64, %zu in FP32)",
                  need, kNoAllocScratchBytes, kNoAllocScratchBytes / 40, kNoAllocScratchBytes / 20);
    return fail(c, FP_ERR_ARG, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "fp_rhs_noalloc: cudaGetDevice");
  if (dev != c->dev) return fail(c, FP_ERR_ARG, "fp_rhs_noalloc: the context's device must be current");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(c, FP_ERR_UNSUPPORTED, "fp_rhs_noalloc: device ordinal beyond 63");
  const NoAllocDevice &S = g_noalloc_dev[dev];
  if (!S.ready.load(std::memory_order_acquire))     // set by the fp_init_grid that made c
    return fail(c, FP_ERR_CUDA, "fp_rhs_noalloc: static scratch not set up on this device");
  cudaStream_t s = (cudaStream_t)stream;
  BlockDev b = c->hblk;
  b.q[0] = const_cast<void *>(q);
  b.dqdt = dqdt;
  b.racc = S.racc;                     // fully written by the first pass: nothing to clear
  k_noalloc_store_block<<<1, 1, 0, s>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "fp_rhs_noalloc: descriptor store");
  const int dims = c->desc.dims, M = c->desc.metric_order;
  if (c->desc.global_lf) {
    e = fpk::launch_lambda(S.blk, 1, c->lam_items, c->nlam_items, c->is_f32, c->desc.characteristic, 0, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "fp_rhs_noalloc: global speed launch");
  }
  for (int d = 0; d < dims; ++d) {
    fpk::SweepLaunch L;
    L.blocks = S.blk;
    L.items = c->items[d];
    L.nitems = c->nitems[d];
    L.dir = d;
    L.mode = d == 0 ? fpk::MODE_WRITE : (d == dims - 1 ? fpk::MODE_RHS : fpk::MODE_ADD);
    L.stage = 0;
    L.dt = c->dt_dev;
    L.alt = shape_of(c, c->hblk.dir[d]);
    L.grid = grid_for(c->per_sm[L.alt], c->nsm, L.nitems);
    L.bnd = has_bnd(c->desc, d);
    L.glf = c->desc.global_lf;
    e = launch(c->is_f32, L, M, c->desc.scheme, c->desc.characteristic, c->desc.free_stream_preserving, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "fp_rhs_noalloc: sweep launch");
  }
  return FP_OK;
}

// ----------------------------------------------------------------- failure injection
extern "C" int fp_debug_fail_allocation(int n) {
  g_fail_countdown.store(n < 0 ? -1 : (long long)n);
  return FP_OK;
}
