// fp_internal.h - device-side descriptors shared by the kernels and the C ABI of
// libfpgb300.so.  Not part of the public interface (include/fp.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fpk {

constexpr int kCellFields = 17;      // per-cell values staged in shared memory
constexpr int kFaceFields = 10;      // per-face values staged in shared memory (W, delta)
constexpr int kNextFields = 15;      // staged per thread: next chunk's cell (Q, k, 1/J), face metrics x2
constexpr int kEpiFields = 13;       // epilogue operands staged per thread (accumulator, Q^n, dk)

// CTA shape of a sweep variant (precision, scheme, fix: 0 switches read at run time, 1 folded,
// 2 folded with the alternative shape): its threads, which equal faces per chunk x lines per
// tile, whether the rings of the xi pass (lines of 2S slots, one after the other) are padded to
// 3S slots per line so that every tile shape is free of bank conflicts (unpadded, the xi pass
// takes S = 32 only), and the CTAs one SM holds.
// Small CTAs pay: the warps of a CTA meet at two barriers per chunk, so with fewer warps per
// CTA the phases of the chunk (staging, FMA-heavy faces, epilogue) of different CTAs overlap
// instead of running in step.  Large ones pay where the eta and zeta passes coalesce across
// more lines (TT): a 256^3 block runs linear upwind 12 % faster at 128 threads (TT = 16) than
// at 64 (TT = 8), a batch of blocks up to 128^3 12 % slower.  So the folded FP32 sweeps have
// two shapes, and a batch's autotuner picks one per direction:
//   WENO5-JS:       64 threads, unpadded, 8 CTAs per SM  |  alternative 128, padded, 4
//   linear upwind: 128 threads, padded, 4                |  alternative  64, unpadded, 8
//   WENO7-JS:      128 threads, padded, 2 (255 registers) |  alternative  64, unpadded, 4
// Every other sweep: 128 threads, padded, 4 CTAs (FP32) or 2 (FP64, and WENO7).
// Single blocks run the primary shape; batches the shape sweep_batch_shape names, which was
// the faster one on the 64-block workload (its step graph runs two branches side by side, and
// kernels of two shapes there would not share SMs, so a batch runs one shape throughout):
// linear upwind the alternative (64 threads: +12 %), the others the primary.
__host__ __device__ constexpr bool sweep_has_alt(bool f32, int scheme, int fix) {
  return f32 && fix != 0 && scheme >= 0 && scheme <= 2;
}
__host__ __device__ constexpr int sweep_batch_shape(bool f32, int scheme, int fix) {
  return sweep_has_alt(f32, scheme, fix) && scheme == 1 ? 1 : 0;
}
__host__ __device__ constexpr int sweep_threads(bool f32, int scheme, int fix) {
  return !sweep_has_alt(f32, scheme, fix) ? 128
         : ((scheme == 0) != (fix == 2) ? 64 : 128);   // WENO5 primary 64, the others' alternative 64
}
__host__ __device__ constexpr bool sweep_padded(bool f32, int scheme, int fix) {
  return sweep_threads(f32, scheme, fix) != 64;
}
__host__ __device__ constexpr int sweep_ring(bool f32, int scheme, int fix) {
  return (sweep_padded(f32, scheme, fix) ? 3 : 2) * sweep_threads(f32, scheme, fix);
}
__host__ __device__ constexpr int sweep_min_ctas(bool f32, int scheme, int fix) {
  return (!f32 || scheme == 2 ? 256 : 512) / sweep_threads(f32, scheme, fix);
}

// Shared-memory field indices of a staged cell.
enum : int {
  CF_Q = 0,      // 0..4 conserved variables
  CF_K = 5,      // 5..7 metric vector of the swept direction (d_x, d_y, d_z)/J
  CF_INVJ = 8,   // 1/J
  CF_RINV = 9,   // 1/rho
  CF_U = 10,     // 10..12 velocity
  CF_H = 13,     // total enthalpy
  CF_SQR = 14,   // sqrt(rho)
  CF_UC = 15,    // contravariant velocity u . grad(d), grad(d) = J k
  CF_AC = 16     // c |grad(d)|
};

enum : int { MODE_WRITE = 0, MODE_ADD = 1, MODE_RHS = 2, MODE_RK = 3 };

// Status word bits set by the kernels.
enum : int { ST_NONFINITE = 1, ST_BOUNDS = 2 };

// Bounds-checking builds (compiled with -DFPK_BOUNDS_CHECK, libfpgb300_check.so): before every
// global access of the sweep, the halo packing and the speed and time-step reductions, the
// element is checked against the array it belongs to, and every shared-ring offset against the
// ring.  An element outside records ST_BOUNDS in the status word and the access goes to the
// array's first element instead, so a wrong index shows as FP_ERR_BOUNDS, not as a fault.  In
// the normal build FPK_CHK_ONLY(...) expands to nothing and FPK_IN(p, ...) to p.
#ifdef FPK_BOUNDS_CHECK
#define FPK_CHK_ONLY(...) __VA_ARGS__
template <typename P>
__device__ __forceinline__ P fpk_in(P p, P base, long long n, int *status) {
  if (p >= base && p < base + n) return p;
  atomicOr(status, ST_BOUNDS);
  return base;
}
#define FPK_IN(p, base, n, status) ::fpk::fpk_in((p), (base), (long long)(n), (status))
#else
#define FPK_CHK_ONLY(...)
#define FPK_IN(p, base, n, status) (p)
#endif

// One swept direction of one block.  A "line" runs along the swept direction; the
// lines of a block are numbered by a flattened transverse index L = t1 + nt1 * t2.
struct DirDev {
  int nd;              // points along the line
  int nt1;             // extent of the first transverse coordinate
  long long nlines;    // number of lines
  long long qT1, qT2, qsd;  // state offsets: t1, t2 and along-line strides
  long long mT1, mT2, msd;  // metric offsets (ghosted arrays)
  long long fT1, fT2, fsd;  // face-metric offsets, face f+1/2 at (f+1)*fsd
  long long fc;        // face-metric component stride
  int bclo, bchi;      // boundary codes at the two line ends
  int S, TT;           // faces per chunk, lines per tile (S * TT == the variant's sweep_threads)
  const void *fmet;    // T [3][faces]
  const void *dk;      // T [3][cells]: k_{i+1/2} - k_{i-1/2} along this direction (FP64-formed)
  // FP_BC_HALO sides: the caller's buffers of the G cells beyond each side, laid out like the
  // state with this direction's extent replaced by G (strides: t1, t2, along the line, component)
  const void *halo[2];
  long long hT1, hT2, hsd, hc;
};

// 16-byte aligned and padded so that the sweep can copy a descriptor into shared memory in
// 16-byte cp.async pieces
struct alignas(16) BlockDev {
  DirDev dir[3];
  int dims;
  int G;               // metric ghost width
  long long qc;        // state component stride (ni*nj*nk)
  long long mc;        // metric component stride
  long long moff;      // offset of point (0,0,0) in the metric arrays
  const void *met;     // T [10][...] cell metrics with G ghosts
  void *q[3];          // stage states: 0 = Q^n (caller), 1 = Q^(1), 2 = Q^(2)
  void *racc;          // residual accumulator, state layout
  void *dqdt;          // output of the rhs mode
  double qbar[5];      // reference state (far-field state)
  double gamma;
  int *status;         // device status word: ST_NONFINITE, ST_BOUNDS
  int global_lf;       // 1: Lax-Friedrichs speeds from lamg instead of the stencil
  void *lamg;          // T [3 directions][3]: max |U - c|grad||, |U|, |U + c|grad|| over the block
  int cut;             // FP_BC_CUT sides: lines t1 < cut or t1 >= nt1 - cut meet across the cut
  int nbr[3][2];       // FP_BC_BLOCK sides: index of the linked block in the launch's block table
};

struct SweepLaunch {
  const BlockDev *blocks;
  const int2 *items;   // (block index, first line) per work item
  int nitems;
  int dir;
  int mode;
  int stage;           // RK stage 0,1,2 (input q[stage], output q[(stage+1)%3])
  const double *dt;    // device scalar
  int grid;            // CTAs of the persistent launch
  int bnd = 0;         // some block of the launch has a slip-wall or cut side in `dir`
  int glf = 0;         // the blocks of the launch use global Lax-Friedrichs speeds
  int alt = 0;         // the blocks' tiles in `dir` are of the alternative CTA shape
};

// Launchers of the sweep, one per translation unit (sweep_<NAME>.cu): precision f32 / f64,
// `_bnd` with the slip-wall, cut, link and halo rules compiled in, `_fix` with the
// characteristic decomposition and the FP form fixed on, `_fix2` the same in the alternative
// CTA shape (FP32 only).  Each returns the cudaError_t of the
// launch; prepare_sweep_<NAME> opts in to the dynamic shared memory of its 16 (M, scheme)
// variants and returns the resident CTAs per SM of the given one.
cudaError_t launch_sweep_f32(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f32_fix(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f32_bnd(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f32_bnd_fix(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f32_fix2(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f32_bnd_fix2(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f64(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f64_fix(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f64_bnd(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
cudaError_t launch_sweep_f64_bnd_fix(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s);
int prepare_sweep_f32(int M, int scheme);
int prepare_sweep_f32_fix(int M, int scheme);
int prepare_sweep_f32_bnd(int M, int scheme);
int prepare_sweep_f32_bnd_fix(int M, int scheme);
int prepare_sweep_f32_fix2(int M, int scheme);
int prepare_sweep_f32_bnd_fix2(int M, int scheme);
int prepare_sweep_f64(int M, int scheme);
int prepare_sweep_f64_fix(int M, int scheme);
int prepare_sweep_f64_bnd(int M, int scheme);
int prepare_sweep_f64_bnd_fix(int M, int scheme);

// Every device and page-locked allocation of the library goes through these two, so the
// host-side hook fp_debug_fail_allocation can make a chosen one fail as if the device (or
// the pinned host pool) were out of memory.  Defined in api.cu.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t host_malloc(void **p, size_t bytes);
template <typename P> inline cudaError_t dev_alloc(P **p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void **>(p), bytes);
}

// Metric construction (metrics.cu), FP64.
struct MetricJob {
  int dims, M, G, Gn;
  int n[3];
  const double *nodes;     // device, [dims][..] with Gn ghosts
  double *met;             // device, [10][B3]
  double *fmet[3];         // device, face metrics per direction [3][faces]
  double *dk[3];           // device, per-point face-metric difference per direction [3][cells]
  double *scratch;         // device, 9 * |B2| doubles
};
cudaError_t build_metrics(const MetricJob &J, cudaStream_t s);
cudaError_t convert_f64_to_f32(const double *src, float *dst, long long n, cudaStream_t s);

// Global Lax-Friedrichs speeds (cfl.cu): zero, then max over (block, first point) items of
// kLamChunk points each.
constexpr int kLamChunk = 8192;
cudaError_t launch_lambda(const BlockDev *blocks, int nblocks, const int2 *items, int nitems,
                          int is_f32, int charwise, int stage, cudaStream_t s);

// CFL reduction (cfl.cu).
cudaError_t launch_cfl(const BlockDev *blk, int is_f32, long long ncells, const int *n, int dims,
                       unsigned long long *out_bits, cudaStream_t s);

// Halo packing (cfl.cu): the G cells of stage state `stage` next to side `side` of direction
// `dir` into `out`, in the halo layout of DirDev (the receiving block's view of them); `status`
// is the context's status word (bounds-checking builds record there).
cudaError_t launch_pack_halo(const void *q, int is_f32, int dir, int side, int G, const int *n, void *out,
                             int *status, cudaStream_t s);

}  // namespace fpk
