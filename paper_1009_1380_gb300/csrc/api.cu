// Exported operator entry points (C ABI, declared in include/cpct.h).
#include <cstdint>

#include "common.cuh"

namespace {
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

extern "C" int radon_fwd(cpct_plan* plan, const float* d_img, float* d_sino, cudaStream_t stream) {
  if (!plan || !d_img || !d_sino || !aligned16(d_img) || !aligned16(d_sino)) return CPCT_EINVAL;
  return cpct_launch_fwd(plan, d_img, d_sino, stream);
}

extern "C" int radon_adj(cpct_plan* plan, const float* d_sino, float* d_img, cudaStream_t stream) {
  if (!plan || !d_img || !d_sino || !aligned16(d_img) || !aligned16(d_sino)) return CPCT_EINVAL;
  return cpct_launch_adj(plan, d_sino, d_img, stream);
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
  rc = cpct_launch_fwd(p, p->d_stage_img, p->d_stage_sino, s);
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
  rc = cpct_launch_adj(p, p->d_stage_sino, p->d_stage_img, s);
  if (rc) return rc;
  CPCT_CUDA_TRY(cudaMemcpyAsync(h_img, p->d_stage_img, sizeof(float) * (size_t)p->n * p->n, cudaMemcpyDeviceToHost, s));
  CPCT_CUDA_TRY(cudaStreamSynchronize(s));
  return CPCT_OK;
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
