// Exported operator entry points (C ABI, declared in include/cpct.h).
#include <cstdint>
#include <new>

#include "common.cuh"

namespace {
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

extern "C" int radon_fwd(cpct_plan* plan, const float* d_img, float* d_sino, cudaStream_t stream) {
  if (!plan || !d_img || !d_sino || !aligned16(d_img) || !aligned16(d_sino)) return CPCT_EINVAL;
  return cpct_graph_run(plan, 0, d_img, d_sino, stream);
}

extern "C" int radon_adj(cpct_plan* plan, const float* d_sino, float* d_img, cudaStream_t stream) {
  if (!plan || !d_img || !d_sino || !aligned16(d_img) || !aligned16(d_sino)) return CPCT_EINVAL;
  return cpct_graph_run(plan, 1, d_sino, d_img, stream);
}

extern "C" int radon_fwd_c(cpct_plan* plan, const float* d_img, void* d_sino_c, cudaStream_t stream) {
  if (!plan || !d_img || !d_sino_c || !aligned16(d_img) || !aligned16(d_sino_c)) return CPCT_EINVAL;
  return cpct_launch_fwd_c(plan, d_img, static_cast<float2*>(d_sino_c), stream);
}

extern "C" int radon_adj_c(cpct_plan* plan, const void* d_sino_c, float* d_img, cudaStream_t stream) {
  if (!plan || !d_img || !d_sino_c || !aligned16(d_img) || !aligned16(d_sino_c)) return CPCT_EINVAL;
  return cpct_launch_adj_c(plan, static_cast<const float2*>(d_sino_c), d_img, stream);
}

extern "C" int radon_fbp(cpct_plan* plan, const float* d_sino, float* d_img, cudaStream_t stream) {
  if (!plan || !d_img || !d_sino || !aligned16(d_img) || !aligned16(d_sino)) return CPCT_EINVAL;
  const double ramp = 3.14159265358979323846 / ((double)plan->m * plan->ns);
  return cpct_launch_adj_ramp(plan, d_sino, d_img, (float)ramp, nullptr, stream);
}

namespace {
int ensure_staging(cpct_plan* p) {
  if (!p->d_stage_img) {
    if (cudaMalloc(&p->d_stage_img, sizeof(float) * (size_t)p->n * p->n) != cudaSuccess) {
      p->d_stage_img = nullptr;
      return CPCT_ENOMEM;
    }
    p->device_bytes += sizeof(float) * (size_t)p->n * p->n;
  }
  if (!p->d_stage_sino) {
    if (cudaMalloc(&p->d_stage_sino, sizeof(float) * (size_t)p->m * p->ns) != cudaSuccess) {
      p->d_stage_sino = nullptr;
      return CPCT_ENOMEM;
    }
    p->device_bytes += sizeof(float) * (size_t)p->m * p->ns;
  }
  return CPCT_OK;
}
}  // namespace

extern "C" int radon_fwd_host(cpct_plan* p, const float* h_img, float* h_sino, cudaStream_t s) {
  if (!p || !h_img || !h_sino) return CPCT_EINVAL;
  int rc = ensure_staging(p);
  if (rc) return rc;
  CPCT_CUDA_TRY(cudaMemcpyAsync(p->d_stage_img, h_img, sizeof(float) * (size_t)p->n * p->n, cudaMemcpyHostToDevice, s));
  rc = cpct_graph_run(p, 0, p->d_stage_img, p->d_stage_sino, s);
  if (rc) return rc;
  CPCT_CUDA_TRY(cudaMemcpyAsync(h_sino, p->d_stage_sino, sizeof(float) * (size_t)p->m * p->ns, cudaMemcpyDeviceToHost, s));
  CPCT_CUDA_TRY(cudaStreamSynchronize(s));
  return CPCT_OK;
}

extern "C" int radon_adj_host(cpct_plan* p, const float* h_sino, float* h_img, cudaStream_t s) {
  if (!p || !h_img || !h_sino) return CPCT_EINVAL;
  int rc = ensure_staging(p);
  if (rc) return rc;
  CPCT_CUDA_TRY(cudaMemcpyAsync(p->d_stage_sino, h_sino, sizeof(float) * (size_t)p->m * p->ns, cudaMemcpyHostToDevice, s));
  rc = cpct_graph_run(p, 1, p->d_stage_sino, p->d_stage_img, s);
  if (rc) return rc;
  CPCT_CUDA_TRY(cudaMemcpyAsync(h_img, p->d_stage_img, sizeof(float) * (size_t)p->n * p->n, cudaMemcpyDeviceToHost, s));
  CPCT_CUDA_TRY(cudaStreamSynchronize(s));
  return CPCT_OK;
}

// What radon_pair_host_stream keeps in the plan between calls: two device
// buffer sets (image, sinogram, adjoint), a clone of the plan (the same
// tables, its own workspaces) so that two slices' kernels can run at once,
// the copy streams, the second compute stream and the events.  Created by
// the first call that needs them, freed with the plan or before the plan's
// configuration changes.
struct HostStream {
  float* buf = nullptr;
  size_t bytes = 0;
  cpct_plan* clone = nullptr;
  cudaStream_t up = nullptr, down = nullptr, comp1 = nullptr;
  cudaEvent_t ev[4][2] = {};  // uploaded, forward done, adjoint done, downloaded
};

void cpct_host_stream_release(cpct_plan* p) {
  if (!p || !p->hstream) return;
  HostStream* h = p->hstream;
  p->hstream = nullptr;
  if (h->down) cudaStreamSynchronize(h->down);
  if (h->up) cudaStreamSynchronize(h->up);
  if (h->comp1) cudaStreamSynchronize(h->comp1);
  if (h->clone) cpct_plan_destroy(h->clone);
  for (auto& e2 : h->ev)
    for (auto& e : e2)
      if (e) cudaEventDestroy(e);
  if (h->up) cudaStreamDestroy(h->up);
  if (h->down) cudaStreamDestroy(h->down);
  if (h->comp1) cudaStreamDestroy(h->comp1);
  if (h->buf) cudaFree(h->buf);
  delete h;
}

namespace {
// the plan's host-stream resources, created on first use (a clone only
// when two slices or more are streamed)
int host_stream_setup(cpct_plan* p, bool want_clone, cudaStream_t s) {
  const size_t ni = (size_t)p->n * p->n, ns = (size_t)p->m * p->ns;
  const size_t bytes = 2 * sizeof(float) * (2 * ni + ns);
  if (!p->hstream) {
    HostStream* h = new (std::nothrow) HostStream;
    if (!h) return CPCT_ENOMEM;
    p->hstream = h;
    bool ok = cudaMalloc(&h->buf, bytes) == cudaSuccess;
    if (!ok) h->buf = nullptr;
    h->bytes = bytes;
    ok = ok && cudaStreamCreateWithFlags(&h->up, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&h->down, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&h->comp1, cudaStreamNonBlocking) == cudaSuccess;
    for (auto& e2 : h->ev)
      for (auto& e : e2) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      const int status = h->buf ? CPCT_ECUDA : CPCT_ENOMEM;
      cpct_host_stream_release(p);
      return status;
    }
  }
  if (want_clone && !p->hstream->clone && cpct_plan_clone(p, &p->hstream->clone, s) != CPCT_OK)
    p->hstream->clone = nullptr;  // one plan then
  // the clone follows the plan's launch mode
  cpct_plan* c = p->hstream->clone;
  if (c && c->graph_mode != p->graph_mode) cpct_plan_set_graphs(c, p->graph_mode);
  return CPCT_OK;
}
}  // namespace

extern "C" int radon_pair_host_stream(cpct_plan* p, const float* const* h_imgs, float* const* h_sinos,
                                      float* const* h_outs, int count, cudaStream_t s) {
  if (!p || !h_imgs || !h_sinos || !h_outs || count < 1) return CPCT_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!h_imgs[i] || !h_sinos[i] || !h_outs[i]) return CPCT_EINVAL;
  const size_t ni = (size_t)p->n * p->n, ns = (size_t)p->m * p->ns;
  const size_t bi = sizeof(float) * ni, bs = sizeof(float) * ns;
  int rc = host_stream_setup(p, count > 1, s);
  if (rc != CPCT_OK) return rc;
  HostStream* h = p->hstream;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == CPCT_OK) rc = CPCT_ECUDA;
    return rc == CPCT_OK;
  };
  // set k runs on plan k and compute stream k (with one plan both sets
  // share the caller's stream)
  cpct_plan* const plan_of[2] = {p, h->clone ? h->clone : p};
  cudaStream_t const comp[2] = {s, h->clone ? h->comp1 : s};
  cudaStream_t const up = h->up, down = h->down;
  auto& ev = h->ev;
  enum { IN = 0, FWD = 1, ADJ = 2, OUT = 3 };
  // the buffers are free once the previous call's work on them is done
  for (int k = 0; k < 2; ++k) {
    ok(cudaStreamWaitEvent(up, ev[OUT][k], 0));
    ok(cudaStreamWaitEvent(comp[k], ev[OUT][k], 0));
  }
  for (int i = 0; i < count && rc == CPCT_OK; ++i) {
    const int k = i & 1;
    float* img = h->buf + k * (2 * ni + ns);
    float* sino = img + ni;
    float* out = sino + ns;
    cudaStream_t cs = comp[k];
    // upload: the image buffer is free once slice i - 2's forward has read it
    if (i >= 2 && !ok(cudaStreamWaitEvent(up, ev[FWD][k], 0))) break;
    if (!ok(cudaMemcpyAsync(img, h_imgs[i], bi, cudaMemcpyHostToDevice, up))) break;
    if (!ok(cudaEventRecord(ev[IN][k], up))) break;
    // operators: after the upload, and once slice i - 2's downloads have
    // read this set's sinogram and adjoint buffers
    if (!ok(cudaStreamWaitEvent(cs, ev[IN][k], 0))) break;
    if (i >= 2 && !ok(cudaStreamWaitEvent(cs, ev[OUT][k], 0))) break;
    if ((rc = cpct_graph_run(plan_of[k], 0, img, sino, cs)) != CPCT_OK) break;
    if (!ok(cudaEventRecord(ev[FWD][k], cs))) break;
    if ((rc = cpct_graph_run(plan_of[k], 1, sino, out, cs)) != CPCT_OK) break;
    if (!ok(cudaEventRecord(ev[ADJ][k], cs))) break;
    // downloads: the sinogram while the adjoint runs, then the adjoint
    if (!ok(cudaStreamWaitEvent(down, ev[FWD][k], 0))) break;
    if (!ok(cudaMemcpyAsync(h_sinos[i], sino, bs, cudaMemcpyDeviceToHost, down))) break;
    if (!ok(cudaStreamWaitEvent(down, ev[ADJ][k], 0))) break;
    if (!ok(cudaMemcpyAsync(h_outs[i], out, bi, cudaMemcpyDeviceToHost, down))) break;
    if (!ok(cudaEventRecord(ev[OUT][k], down))) break;
  }
  // every copy has landed in host memory before the call returns
  ok(cudaStreamSynchronize(down));
  ok(cudaStreamSynchronize(up));
  if (h->clone) ok(cudaStreamSynchronize(h->comp1));
  ok(cudaStreamSynchronize(s));
  return rc;
}

extern "C" const char* cpct_strerror(int status) {
  switch (status) {
    case CPCT_OK: return "ok";
    case CPCT_EINVAL: return "invalid argument";
    case CPCT_ENOMEM: return "out of memory";
    case CPCT_ECUDA: return "CUDA error";
    case CPCT_ETIMEOUT: return "bounded device wait expired";
    case CPCT_ENONFINITE: return "non-finite value";
    case CPCT_ENOTCONV: return "iteration limit reached";
    case CPCT_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}
