// Batched Radon operators over many z-slices with uneven view counts.
//
// Slices are independent (the paper's motivation is real-time reconstruction
// of whole tomographic volumes, section "Introduction").  A batch binds one
// plan per slice (clones of one plan per distinct geometry share its tables
// and bins) and the slices' device buffers, and captures every slice's kernel
// chain once in a CUDA graph: slices are dealt, longest first, round robin
// onto concurrent graph branches, so one graph launch runs the whole volume
// with no per-kernel launch cost and with small slices filling the GPU
// around large ones.
#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"

struct cpct_batch {
  int batch = 0;
  int mode = 0;
  int branches = 0;
  long long samples = 0;  // polar samples per operator application, all slices
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int ensure_stage_sino(cpct_plan* p) {
  if (p->d_stage_sino) return CPCT_OK;
  if (cudaMalloc(&p->d_stage_sino, sizeof(float) * (size_t)p->m * p->ns) != cudaSuccess) {
    p->d_stage_sino = nullptr;
    return CPCT_ENOMEM;
  }
  p->device_bytes += sizeof(float) * (size_t)p->m * p->ns;
  return CPCT_OK;
}

int enqueue_slice(cpct_plan* p, int mode, const float* in, float* out, cudaStream_t s) {
  switch (mode) {
    case CPCT_BATCH_FWD: return cpct_launch_fwd(p, in, out, s);
    case CPCT_BATCH_ADJ: return cpct_launch_adj(p, in, out, s);
    default: {
      int rc = cpct_launch_fwd(p, in, p->d_stage_sino, s);
      return rc ? rc : cpct_launch_adj(p, p->d_stage_sino, out, s);
    }
  }
}

}  // namespace

extern "C" int cpct_batch_create(cpct_batch** out, cpct_plan* const* plans, int batch, const float* const* d_in,
                                 float* const* d_out, int mode, int branches, cudaStream_t stream) {
  if (!out) return CPCT_EINVAL;
  *out = nullptr;
  if (!plans || batch < 1 || !d_in || !d_out) return CPCT_EINVAL;
  if (mode != CPCT_BATCH_FWD && mode != CPCT_BATCH_ADJ && mode != CPCT_BATCH_PAIR) return CPCT_EINVAL;
  for (int i = 0; i < batch; ++i) {
    if (!plans[i] || !d_in[i] || !d_out[i]) return CPCT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_in[i]) & 15u) || (reinterpret_cast<uintptr_t>(d_out[i]) & 15u))
      return CPCT_EINVAL;
  }
  {
    std::vector<cpct_plan*> sorted(plans, plans + batch);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return CPCT_EINVAL;  // one plan per slice
  }
  if (branches <= 0) branches = 16;
  branches = std::min(branches, batch);
  cpct_batch* b = new (std::nothrow) cpct_batch;
  if (!b) return CPCT_ENOMEM;
  b->batch = batch;
  b->mode = mode;
  b->branches = branches;
  for (int i = 0; i < batch; ++i) b->samples += (long long)plans[i]->m * plans[i]->ns;
  int rc = CPCT_OK;
  std::vector<cudaStream_t> br(branches, nullptr);
  std::vector<cudaEvent_t> joins(branches, nullptr);
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  bool capturing = false;
  // longest slices first, dealt round robin onto the branches
  std::vector<int> order(batch);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return (long long)plans[a]->m * plans[a]->ns > (long long)plans[c]->m * plans[c]->ns;
  });
  for (int i = 0; i < batch && rc == CPCT_OK; ++i) {
    cpct_profile_enable(plans[i], 0);  // no event records inside the graph
    if (mode == CPCT_BATCH_PAIR) rc = ensure_stage_sino(plans[i]);
  }
  // one eager pass: loads every kernel module (not allowed while capturing)
  // and sizes the persistent grids
  for (int i = 0; i < batch && rc == CPCT_OK; ++i) rc = enqueue_slice(plans[i], mode, d_in[i], d_out[i], stream);
  if (rc == CPCT_OK && cudaStreamSynchronize(stream) != cudaSuccess) rc = CPCT_ECUDA;
  if (rc == CPCT_OK && (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess))
    rc = CPCT_ECUDA;
  for (int k = 0; k < branches && rc == CPCT_OK; ++k)
    if (cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming) != cudaSuccess)
      rc = CPCT_ECUDA;
  if (rc == CPCT_OK && cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = CPCT_ECUDA;
  if (rc == CPCT_OK) {
    capturing = true;
    cudaEventRecord(fork, cap);
    for (int k = 0; k < branches; ++k) cudaStreamWaitEvent(br[k], fork, 0);
    for (int i = 0; i < batch && rc == CPCT_OK; ++i) {
      const int sl = order[i];
      rc = enqueue_slice(plans[sl], mode, d_in[sl], d_out[sl], br[i % branches]);
    }
    for (int k = 0; k < branches; ++k) {
      cudaEventRecord(joins[k], br[k]);
      cudaStreamWaitEvent(cap, joins[k], 0);
    }
    capturing = false;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess) {
      if (rc == CPCT_OK) rc = CPCT_ECUDA;
    } else if (rc == CPCT_OK) {
      b->graph = g;
      if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) rc = CPCT_ECUDA;
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  if (capturing) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cap, &g);
    if (g) cudaGraphDestroy(g);
  }
  for (auto e : joins)
    if (e) cudaEventDestroy(e);
  for (auto s : br)
    if (s) cudaStreamDestroy(s);
  if (fork) cudaEventDestroy(fork);
  if (cap) cudaStreamDestroy(cap);
  if (rc != CPCT_OK) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return rc;
  }
  *out = b;
  return CPCT_OK;
}

extern "C" int cpct_batch_run(cpct_batch* b, cudaStream_t stream) {
  if (!b || !b->exec) return CPCT_EINVAL;
  return cudaGraphLaunch(b->exec, stream) == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

extern "C" int cpct_batch_info(const cpct_batch* b, int* batch, long long* samples, int* branches) {
  if (!b) return CPCT_EINVAL;
  if (batch) *batch = b->batch;
  if (samples) *samples = b->samples;
  if (branches) *branches = b->branches;
  return CPCT_OK;
}

extern "C" int cpct_batch_destroy(cpct_batch* b) {
  if (!b) return CPCT_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
  return CPCT_OK;
}
