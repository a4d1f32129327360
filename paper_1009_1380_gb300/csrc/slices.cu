// Per-slice statistics and scaling used by the learned warm start (the paper
// has no counterpart): the network sees every filtered back-projection scaled
// by its own standard deviation, and the starting radius of SPGL1 is
// estimated from the l1 norm of a soft-thresholded prediction.
//
// A batch is `batch` slices of n contiguous float32 values each.  Every
// reduction is deterministic: a fixed grid of blocks per slice, FP64
// per-thread sums, warp shuffles in a fixed pattern, block partials summed
// in block order by one thread per slice.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kT = 256;          // threads per block
constexpr int kMaxBlocks = 64;   // blocks per slice

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of v; thread 0 returns the total
__device__ double block_sum_d(double v) {
  __shared__ double sh[kT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum_d(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kT / 32; ++i) t += sh[i];
  __syncthreads();
  return t;
}

// mode 0: sum of x (partial of the slice's block);
// mode 1: sum of (x - mean_s)^2 with mean_s = aux[s];
// mode 2: sum of max(|x| - aux[s], 0)
__global__ void __launch_bounds__(kT) k_slice_partials(const float* __restrict__ x, long long n, int mode,
                                                       const double* __restrict__ aux, double* __restrict__ part) {
  const int s = blockIdx.y, nb = gridDim.x;
  const float* xs = x + (size_t)s * n;
  const double a = mode ? aux[s] : 0.0;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)nb * kT) {
    const double v = (double)xs[i];
    if (mode == 0) acc += v;
    else if (mode == 1) acc += (v - a) * (v - a);
    else acc += fmax(fabs(v) - a, 0.0);
  }
  const double t = block_sum_d(acc);
  if (threadIdx.x == 0) part[(size_t)s * nb + blockIdx.x] = t;
}

// out[s] = sum over the slice's block partials, in block order
__global__ void k_slice_finish(const double* __restrict__ part, int nb, int batch, double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += part[(size_t)s * nb + b];
  out[s] = t;
}

__global__ void __launch_bounds__(kT) k_slice_scale(const float* __restrict__ in, float* __restrict__ out,
                                                    long long n, const double* __restrict__ factor) {
  const int s = blockIdx.y;
  const float f = (float)factor[s];
  const float* src = in + (size_t)s * n;
  float* dst = out + (size_t)s * n;
  for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT)
    dst[i] = src[i] * f;
}

int blocks_per_slice(long long n) {
  const long long b = (n + kT * 8 - 1) / (kT * 8);
  return (int)std::max(1LL, std::min<long long>(kMaxBlocks, b));
}

bool args_ok(const void* d, int batch, long long n) { return d && batch >= 1 && batch <= 65535 && n >= 1; }

// Workspace of one call: per-slice partials, one auxiliary value and one
// result per slice (stream-ordered allocation, freed on the same stream).
struct SliceWork {
  double* part = nullptr;
  double* aux = nullptr;
  double* res = nullptr;
  cudaStream_t s = nullptr;
  ~SliceWork() {
    if (part) cudaFreeAsync(part, s);
    if (aux) cudaFreeAsync(aux, s);
    if (res) cudaFreeAsync(res, s);
  }
};

int alloc_work(SliceWork& w, int batch, int nb, cudaStream_t s) {
  w.s = s;
  if (cudaMallocAsync((void**)&w.part, sizeof(double) * (size_t)batch * nb, s) != cudaSuccess) return CPCT_ENOMEM;
  if (cudaMallocAsync((void**)&w.aux, sizeof(double) * batch, s) != cudaSuccess) return CPCT_ENOMEM;
  if (cudaMallocAsync((void**)&w.res, sizeof(double) * batch, s) != cudaSuccess) return CPCT_ENOMEM;
  return CPCT_OK;
}

// one reduction pass: res[s] = sum over slice s of the mode's term
int reduce_pass(const float* d_x, int batch, long long n, int mode, SliceWork& w, cudaStream_t s) {
  const int nb = blocks_per_slice(n);
  k_slice_partials<<<dim3(nb, batch), kT, 0, s>>>(d_x, n, mode, w.aux, w.part);
  k_slice_finish<<<(batch + 127) / 128, 128, 0, s>>>(w.part, nb, batch, w.res);
  return cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

}  // namespace

extern "C" int cpct_slice_moments(const float* d_x, int batch, long long n, double* h_mean, double* h_std,
                                  cudaStream_t stream) {
  if (!args_ok(d_x, batch, n) || (!h_mean && !h_std)) return CPCT_EINVAL;
  SliceWork w;
  int rc = alloc_work(w, batch, blocks_per_slice(n), stream);
  if (rc) return rc;
  std::vector<double> sum(batch), ss(batch);
  if ((rc = reduce_pass(d_x, batch, n, 0, w, stream))) return rc;
  if (cudaMemcpyAsync(sum.data(), w.res, sizeof(double) * batch, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return CPCT_ECUDA;
  for (int i = 0; i < batch; ++i) sum[i] /= (double)n;  // means
  if (h_std) {
    // second pass about the mean: the sample variance without cancellation
    if (cudaMemcpyAsync(w.aux, sum.data(), sizeof(double) * batch, cudaMemcpyHostToDevice, stream) != cudaSuccess)
      return CPCT_ECUDA;
    if ((rc = reduce_pass(d_x, batch, n, 1, w, stream))) return rc;
    if (cudaMemcpyAsync(ss.data(), w.res, sizeof(double) * batch, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return CPCT_ECUDA;
    for (int i = 0; i < batch; ++i) h_std[i] = n > 1 ? std::sqrt(ss[i] / (double)(n - 1)) : 0.0;
  }
  if (h_mean)
    for (int i = 0; i < batch; ++i) h_mean[i] = sum[i];
  return CPCT_OK;
}

extern "C" int cpct_slice_soft_l1(const float* d_x, int batch, long long n, const double* h_thresh, double* h_out,
                                  cudaStream_t stream) {
  if (!args_ok(d_x, batch, n) || !h_thresh || !h_out) return CPCT_EINVAL;
  for (int i = 0; i < batch; ++i)
    if (!(h_thresh[i] >= 0.0) || !std::isfinite(h_thresh[i])) return CPCT_EINVAL;
  SliceWork w;
  int rc = alloc_work(w, batch, blocks_per_slice(n), stream);
  if (rc) return rc;
  if (cudaMemcpyAsync(w.aux, h_thresh, sizeof(double) * batch, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return CPCT_ECUDA;
  if ((rc = reduce_pass(d_x, batch, n, 2, w, stream))) return rc;
  if (cudaMemcpyAsync(h_out, w.res, sizeof(double) * batch, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return CPCT_ECUDA;
  return CPCT_OK;
}

extern "C" int cpct_slice_scale(const float* d_in, float* d_out, int batch, long long n, const double* h_factor,
                                cudaStream_t stream) {
  if (!args_ok(d_in, batch, n) || !d_out || !h_factor) return CPCT_EINVAL;
  for (int i = 0; i < batch; ++i)
    if (!std::isfinite(h_factor[i])) return CPCT_EINVAL;
  SliceWork w;
  w.s = stream;
  if (cudaMallocAsync((void**)&w.aux, sizeof(double) * batch, stream) != cudaSuccess) return CPCT_ENOMEM;
  if (cudaMemcpyAsync(w.aux, h_factor, sizeof(double) * batch, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return CPCT_ECUDA;
  const int nb = blocks_per_slice(n);
  k_slice_scale<<<dim3(nb, batch), kT, 0, stream>>>(d_in, d_out, n, w.aux);
  if (cudaGetLastError() != cudaSuccess) return CPCT_ECUDA;
  // the factors are read by the kernel before the workspace is freed on the
  // same stream; the host array may be reused once this call returns
  if (cudaStreamSynchronize(stream) != cudaSuccess) return CPCT_ECUDA;
  return CPCT_OK;
}
