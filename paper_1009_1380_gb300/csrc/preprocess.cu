// Preprocessing front end (section "Introduction", Fig. 1): background
// normalization of the near and far radiographs and their difference, the
// propagation-based phase-contrast image, regrouped into one sinogram per
// detector row (slice).
//
//   n = (I - D) / (F - D)                (0 where F - D <= 0)
//   sino_z[j, s] = n_near[j, z, s] - n_far[j, z, s]
//
// Frames are (angle j, detector row z, column s) uint16 camera counts; the
// output is (z, j, s) float32.  Both are contiguous in s, so the regrouping
// is a reordering of whole rows: every block handles one (j, z) row, reads
// its counts and writes its sinogram row with coalesced accesses.  The
// reciprocals of the flat-field denominators are formed once per call.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kT = 256;

// rden[z, s] = 1 / (F - D), or 0 for a dead or saturated reference pixel
__global__ void __launch_bounds__(kT) k_pc_recip(const float* __restrict__ flat, const float* __restrict__ dark,
                                                 float* __restrict__ rden, long long total) {
  for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < total; i += (long long)gridDim.x * kT) {
    const float den = flat[i] - dark[i];
    rden[i] = den > 0.f ? 1.f / den : 0.f;
  }
}

__global__ void __launch_bounds__(kT) k_pc_diff(const uint16_t* __restrict__ near, const uint16_t* __restrict__ far,
                                                const float* __restrict__ rn, const float* __restrict__ rf,
                                                const float* __restrict__ dark, float* __restrict__ sinos, int M,
                                                int rows, int ns) {
  const int j = blockIdx.x % M, z = blockIdx.x / M;  // consecutive blocks: consecutive angles of one slice
  const size_t in_row = ((size_t)j * rows + z) * ns, cal_row = (size_t)z * ns;
  float* out = sinos + ((size_t)z * M + j) * ns;
  for (int s = threadIdx.x; s < ns; s += kT) {
    const float d = dark[cal_row + s];
    const float a = ((float)near[in_row + s] - d) * rn[cal_row + s];
    const float b = ((float)far[in_row + s] - d) * rf[cal_row + s];
    out[s] = a - b;
  }
}

}  // namespace

extern "C" int cpct_preprocess_pc(const uint16_t* d_near, const uint16_t* d_far, const float* d_flat_near,
                                  const float* d_flat_far, const float* d_dark, int n_views, int n_rows, int n_det,
                                  float* d_sinos, cudaStream_t stream) {
  if (!d_near || !d_far || !d_flat_near || !d_flat_far || !d_dark || !d_sinos) return CPCT_EINVAL;
  if (n_views < 1 || n_rows < 1 || n_det < 1 || (long long)n_views * n_rows > (1LL << 31) - 1) return CPCT_EINVAL;
  const long long cal = (long long)n_rows * n_det;
  float* rden = nullptr;
  if (cudaMallocAsync((void**)&rden, sizeof(float) * 2 * cal, stream) != cudaSuccess) return CPCT_ENOMEM;
  const int g = (int)std::min<long long>(4096, (cal + kT - 1) / kT);
  k_pc_recip<<<g, kT, 0, stream>>>(d_flat_near, d_dark, rden, cal);
  k_pc_recip<<<g, kT, 0, stream>>>(d_flat_far, d_dark, rden + cal, cal);
  k_pc_diff<<<n_views * n_rows, kT, 0, stream>>>(d_near, d_far, rden, rden + cal, d_dark, d_sinos, n_views, n_rows,
                                                 n_det);
  int rc = cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
  cudaFreeAsync(rden, stream);
  return rc;
}
