// pipe.cu - batched advance of host-resident states with the host<->device copies
// overlapped by compute (C ABI in include/fp.h: fp_pipe_*), and the balanced partition that the
// pipe's groups and the batch graph's branches use (fp_balanced_groups).
//
// The blocks are split into groups of about equal size.  Each group is a batch
// (fp_batch_create: one persistent launch per direction pass, the three RK stages in
// one CUDA graph) with its own device state buffers and its own stream.  A step issues,
// group by group on the group's stream, the copies of the group's states to the device,
// the group's graph and the copies back.  The copy engines then move one group's states
// while the SMs advance another, so only the first group's upload and the last group's
// download are exposed.  Built on the public batch calls; no kernel of its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/fp.h"
#include "fp_internal.h"

struct fp_pipe {
  std::vector<fp_ctx *> ctx;
  std::vector<void *> qdev;                 // device state of each block (owned)
  std::vector<size_t> bytes;                // state bytes of each block
  std::vector<std::vector<int>> groups;     // block indices of each group
  std::vector<fp_batch *> batch;            // one batch per group
  std::vector<cudaStream_t> st;             // one stream per group
  std::vector<cudaEvent_t> done;            // end of each group's step
  cudaEvent_t start = nullptr;              // the caller's stream at the start of a step (ordered mode)
  int ordered = 0;
  std::string err;
};

namespace {

int pipe_fail(fp_pipe *p, int status, const std::string &msg) {
  if (p) p->err = msg;
  return status;
}

}  // namespace

extern "C" {

void fp_pipe_free(fp_pipe *p) {
  if (!p) return;
  for (cudaStream_t s : p->st)
    if (s) cudaStreamSynchronize(s);
  for (fp_batch *b : p->batch) fp_batch_free(b);
  for (void *q : p->qdev) cudaFree(q);
  for (cudaStream_t s : p->st)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : p->done)
    if (e) cudaEventDestroy(e);
  if (p->start) cudaEventDestroy(p->start);
  delete p;
}

int fp_pipe_create(fp_ctx *const *blocks, int nblocks, const void *const *q_host, int ngroups,
                   int autotune, fp_pipe **out) {
  if (!out) return FP_ERR_ARG;
  *out = nullptr;
  if (!blocks || !q_host || nblocks < 1 || ngroups < 1) return FP_ERR_ARG;
  for (int k = 0; k < nblocks; ++k)
    if (!blocks[k] || !q_host[k] || fp_state_bytes(blocks[k]) == 0) return FP_ERR_ARG;
  ngroups = std::min(ngroups, nblocks);
  fp_pipe *p = new fp_pipe();
  std::vector<long long> weight(nblocks);
  for (int k = 0; k < nblocks; ++k) {
    p->ctx.push_back(blocks[k]);
    p->bytes.push_back(fp_state_bytes(blocks[k]));
    weight[k] = (long long)p->bytes[k];
  }
  // groups of about equal size (block indices ascending within a group)
  std::vector<int> group_of(nblocks);
  fp_balanced_groups(weight.data(), nblocks, ngroups, group_of.data());
  p->groups.assign(ngroups, {});
  for (int k = 0; k < nblocks; ++k) p->groups[group_of[k]].push_back(k);
  // device states, initialised from the host states (so autotuning runs on real data)
  p->qdev.assign(nblocks, nullptr);
  for (int k = 0; k < nblocks; ++k) {
    cudaError_t e = fpk::dev_malloc(&p->qdev[k], p->bytes[k]);
    if (e == cudaSuccess) e = cudaMemcpy(p->qdev[k], q_host[k], p->bytes[k], cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      fp_pipe_free(p);
      return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  for (int g = 0; g < ngroups && e == cudaSuccess; ++g) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    p->st.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    p->done.push_back(ev);
  }
  if (e != cudaSuccess) {
    fp_pipe_free(p);
    return FP_ERR_CUDA;
  }
  for (int g = 0; g < ngroups; ++g) {
    std::vector<fp_ctx *> c;
    std::vector<void *> q;
    for (int k : p->groups[g]) {
      c.push_back(p->ctx[k]);
      q.push_back(p->qdev[k]);
    }
    fp_batch *b = nullptr;
    const int st = fp_batch_create(c.data(), (int)c.size(), q.data(), autotune, p->st[g], &b);
    if (st != FP_OK) {
      fp_pipe_free(p);
      return st;
    }
    p->batch.push_back(b);
  }
  *out = p;
  return FP_OK;
}

int fp_pipe_rk3_step_host(fp_pipe *p, void *const *q_host, double dt, void *stream) {
  if (!p) return FP_ERR_ARG;
  if (!q_host) return pipe_fail(p, FP_ERR_ARG, "fp_pipe_rk3_step_host: null states");
  for (size_t k = 0; k < p->ctx.size(); ++k)
    if (!q_host[k]) return pipe_fail(p, FP_ERR_ARG, "fp_pipe_rk3_step_host: null state");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  // ordered mode: every group's work also follows what was queued on `stream` before the call
  if (p->ordered) e = cudaEventRecord(p->start, s);
  // each group's work follows that group's previous step on its own stream, so one step's
  // first uploads overlap the previous step's last groups; `stream` waits for every group
  for (size_t g = 0; g < p->groups.size() && e == cudaSuccess; ++g) {
    cudaStream_t gs = p->st[g];
    if (p->ordered) e = cudaStreamWaitEvent(gs, p->start, 0);
    for (int k : p->groups[g])
      if (e == cudaSuccess) e = cudaMemcpyAsync(p->qdev[k], q_host[k], p->bytes[k], cudaMemcpyHostToDevice, gs);
    if (e != cudaSuccess) break;
    const int st = fp_batch_rk3_step(p->batch[g], dt, gs);
    if (st != FP_OK) return pipe_fail(p, st, std::string("fp_pipe_rk3_step_host: ") + fp_batch_last_error(p->batch[g]));
    for (int k : p->groups[g])
      if (e == cudaSuccess) e = cudaMemcpyAsync(q_host[k], p->qdev[k], p->bytes[k], cudaMemcpyDeviceToHost, gs);
    if (e == cudaSuccess) e = cudaEventRecord(p->done[g], gs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->done[g], 0);
  }
  if (e != cudaSuccess)
    return pipe_fail(p, FP_ERR_CUDA, std::string("fp_pipe_rk3_step_host: ") + cudaGetErrorString(e));
  return FP_OK;
}

int fp_pipe_set_ordered(fp_pipe *p, int ordered) {
  if (!p) return FP_ERR_ARG;
  p->ordered = ordered ? 1 : 0;
  return FP_OK;
}

int fp_pipe_groups(const fp_pipe *p) { return p ? (int)p->groups.size() : 0; }

int fp_pipe_launches_per_step(const fp_pipe *p) {
  if (!p) return 0;
  int n = 0;
  for (fp_batch *b : p->batch) n += fp_batch_launches_per_step(b);
  return n;
}

const char *fp_pipe_last_error(const fp_pipe *p) { return p ? p->err.c_str() : "null pipe"; }

int fp_balanced_groups(const long long *weights, int n, int ngroups, int *group_of) {
  if (n < 0 || ngroups < 1 || (n > 0 && (!weights || !group_of))) return FP_ERR_ARG;
  for (int k = 0; k < n; ++k)
    if (weights[k] < 0) return FP_ERR_ARG;
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return weights[a] > weights[b]; });
  std::vector<long long> load(ngroups, 0);
  for (int k : order) {
    const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    group_of[k] = g;
    load[g] += weights[k];
  }
  return FP_OK;
}

}  // extern "C"
