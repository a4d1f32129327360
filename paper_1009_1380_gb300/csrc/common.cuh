// Internal definitions shared by the CUDA translation units of libcpct.
//
// Data layout in HBM (one plan, one slice):
//   image       N x N float32, row-major (row p = y, column q = x)
//   H1          (N+1) x N complex64: column-transformed image (forward) or
//               row-inverse-transformed spectrum (adjoint); rows b = 0..N
//   Hx          extended half spectrum, (N+8) x LDH complex64, LDH = G+8:
//               buffer row r holds frequency row b = r-2 (b = -2..N+3),
//               buffer column c holds frequency column a = c mod G
//               (c = 0..G+5).  Rows b < 0 and b > N are the Hermitian
//               mirrors conj(H[-b mod G][-a mod G]); columns G..G+5 repeat
//               columns 0..5.  Every 6x6 kernel footprint of a polar sample
//               with v >= 0 is then a plain rectangle of this buffer.
//   Ax          same shape as Hx, accumulator of the adjoint spread
//               (zero outside the tiles that receive samples).
//   Q           M x LDQ complex64, LDQ = Ns/2+2: polar samples k = 0..Ns/2
//               of every ray (the k < 0 half is their complex conjugate
//               because the image is real).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cpct.h"

#define CPCT_W 6          // Kaiser-Bessel kernel width (taps per axis)
#define CPCT_TILE 32      // tile side of the gather / spread bins
#define CPCT_HALO 5       // CPCT_W - 1
#define CPCT_NPOLY 5      // coefficients of each even/odd polynomial part

// error bits recorded by kernels in plan->d_err
#define CPCT_ERR_TIMEOUT 1
#define CPCT_ERR_BIN 2

// Kaiser-Bessel tap weights as polynomials in s = 2z-1, z = frac(u) in [0,1):
// tap i (grid point floor(u)-2+i) has weight g(z+2-i); by the symmetry of g,
// w_{5-i}(s) = w_i(-s), so w_i = E_i(s^2) + s O_i(s^2) and
// w_{5-i} = E_i(s^2) - s O_i(s^2) for i = 0, 1, 2.
struct KBPoly {
  float e[3][CPCT_NPOLY];
  float o[3][CPCT_NPOLY];
};

// per ray: (c_hi, c_lo, s_hi, s_lo) with c = (G/Ns) cos(theta) = c_hi + c_lo
// and s = (G/Ns) sin(theta) = s_hi + s_lo (float32 pairs, built in FP64).

// kernel identifiers for the per-kernel event profiler
enum CpctKernelId {
  KID_FWD_COL = 0, KID_FWD_ROW, KID_FWD_INTERP, KID_FWD_RAY,
  KID_ADJ_RAY, KID_ADJ_SPREAD, KID_ADJ_REDUCE, KID_ADJ_ROW, KID_ADJ_COL,
  KID_COUNT
};

struct CpctProfiler;  // event pairs of profiled launches (profile.cu)

struct cpct_plan {
  int n, ns, m, G, K;       // K = Ns/2
  int logn, logG, logNs;
  int ldh, ext_rows, ldq;
  int flags;
  double scale;             // G / Ns

  KBPoly poly;              // FP32 copy, passed by value to kernels
  double* d_poly64;         // FP64 Chebyshev-fitted monomial coefficients [6][10]
  float4* d_ray;            // [M]
  float* d_deapod;          // [N]
  float2* d_twG;            // twiddles of the G-point FFT passes
  float2* d_twNs;           // twiddles of the Ns-point FFT passes
  float2* d_Hx;             // forward extended spectrum
  float2* d_Ax;             // adjoint accumulator (same shape)
  float2* d_H1;             // (N+1) x N
  float2* d_Q;              // M x LDQ
  // bins: squares of T x T grid points (T = 16, 32, 64; class c = 0, 1, 2);
  // work items are grouped by class, a bin's origin packed as y0 << 16 | x0
  // forward gather work items (origin, first sample, end sample, 0)
  int n_fwd_items;
  int fwd_cls[4];           // items of class c: [fwd_cls[c], fwd_cls[c + 1])
  int4* d_fwd_items;
  uint32_t* d_fwd_ids;      // sample ids (j << 16 | k), grouped by bin
  // adjoint spread work items (origin, first round, end round, partial offset or -1)
  int n_adj_items;
  int adj_cls[4];
  int4* d_adj_items;
  uint32_t* d_adj_ids;      // rounds of 32 lanes
  int n_slots;              // partial-tile space in units of 32 x 32 tiles (rounded up)
  long long partial_elems;  // complex values of the partial tiles of split bins
  float2* d_partials;
  int n_split;
  int split_cls[4];
  int4* d_split;            // (origin, partial offset, pieces, T), grouped by class
  int fwd_kind, fwd_tile, adj_kind, adj_tile;  // bin plans (kind 0 uniform, 1 quadtree)
  int round_lanes;          // samples per adjoint round (16, 32 or 64)
  // staging for the host-buffer entry points
  float* d_stage_img;
  float* d_stage_sino;
  int* d_err;
  CUtensorMap tmap_Hx[3];   // TMA windows of 16, 32 and 64 point bins
  size_t device_bytes;
  int fwd_interp_grid[3];   // persistent grids of the forward gather per class (0 = not yet sized)
  int adj_row_grid;         // persistent grid of the adjoint row transform (0 = not yet sized)
  int fwd_col_grid;         // persistent grid of the forward column transform (0 = not yet sized)
  CUtensorMap tmap_img;     // TMA descriptor of the last image given to the forward column transform
  const float* tmap_img_ptr;  // the image tmap_img was encoded for (null: none)
  // plans with bins of several sizes run the per-size launches concurrently:
  // two side streams fork from the launch stream and join it again
  cudaStream_t side[2];
  cudaEvent_t ev_fork, ev_join[2];
  int fwd_cap, adj_cap;     // work-item caps (samples / rounds per item), tunable
  int concurrency;          // slices expected to run at once (automatic caps; 0 = 1)
  int fwd_cap_set, adj_cap_set;  // 1 once cpct_plan_set_caps fixed the cap (else automatic)
  struct PlanShared* shared;  // read-only geometry shared with clones (refcounted)
  long long launches;       // kernels launched by this plan's operators
  CpctProfiler* prof;       // NULL unless profiling is enabled
  // graph replay of the operators (cpct_plan_set_graphs): 0 = direct launches
  int graph_mode;
  struct GraphCache* graphs;  // captured operator graphs (NULL: none yet)
  struct GraphCapture* capturing;  // set while an operator is being captured
  struct HostStream* hstream;  // buffers, clone and streams of radon_pair_host_stream (NULL: none yet)
};

// Read-only data of one geometry, shared by a plan and its clones: the
// tables and bin lists (device) and the bin pointers kept on the host so the
// work items can be rebuilt with other caps.  Freed with the last plan.
#include <atomic>
#include <vector>
struct PlanShared {
  std::atomic<int> refs{1};
  std::vector<float4> ray;          // per-ray geometry (host copy)
  std::vector<int4> fwd_bins;       // forward bins (x0, y0, T, 0)
  std::vector<int> fwd_ptr;         // forward bins: samples, bins + 1
  std::vector<int4> adj_bins;       // adjoint bins
  std::vector<int> round_ptr;       // adjoint rounds per bin: bins + 1
};

// bracket a kernel launch: counts it and, if its id is profiled, records a
// CUDA event pair on the launch stream (profile.cu)
void cpct_prof_begin(cpct_plan* p, int kid, cudaStream_t s);
void cpct_prof_end(cpct_plan* p, int kid, cudaStream_t s);
void cpct_prof_free(cpct_plan* p);

// TMA descriptor of a caller's image for the forward column transform
// (boxes of 8 columns by min(N, 256) rows), cached in the plan by address
int cpct_image_cols_map(cpct_plan* p, const float* img, const CUtensorMap** out);
// image columns per block of the forward column transform (radon.cu)
int cpct_col_block_width();

// graph replay of the operators (graphs.cu): run op 0 (forward, in = image,
// out = sinogram) or 1 (adjoint, in = sinogram, out = image) through the
// plan's graph cache when graph mode is on, else launch directly
int cpct_graph_run(cpct_plan* p, int op, const void* in, void* out, cudaStream_t s);
// drop every captured graph (the launch configuration changed)
void cpct_graph_clear(cpct_plan* p);
// free the graph cache (plan destruction)
void cpct_graph_free(cpct_plan* p);
// free what radon_pair_host_stream keeps between calls (api.cu)
void cpct_host_stream_release(cpct_plan* p);
// while capturing: record a profiling event as a graph node (profile.cu)
void cpct_graph_prof_event(cpct_plan* p, int kid, bool begin, cudaEvent_t ev, cudaStream_t s);

// side streams and events of a plan (created with the plan and each clone)
int cpct_plan_streams_create(cpct_plan* p);
void cpct_plan_streams_destroy(cpct_plan* p);

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Sample coordinate u = k * (hi + lo) split into an integer floor and a
// fraction z in [0,1), with the product k*hi carried exactly (FMA residual) so
// that the fraction is accurate to ~6e-8 grid units for |u| up to 4096.  The
// host bin builder performs the identical IEEE operations.
__device__ __forceinline__ void split_coord(float k, float hi, float lo, int& fl_out, float& z) {
  float p = __fmul_rn(k, hi);
  float e = __fmaf_rn(k, hi, -p);
  float corr = __fmaf_rn(k, lo, e);
  float fl = floorf(p);
  float zz = __fadd_rn(__fsub_rn(p, fl), corr);
  if (zz < 0.f) {
    float t = __fadd_rn(zz, 1.f);
    if (t < 1.f) { zz = t; fl = __fsub_rn(fl, 1.f); } else { zz = 0.f; }
  } else if (zz >= 1.f) {
    zz = __fsub_rn(zz, 1.f);
    fl = __fadd_rn(fl, 1.f);
  }
  fl_out = (int)fl;
  z = zz;
}

// the six Kaiser-Bessel weights of a sample with fraction z
__device__ __forceinline__ void kb_weights(const KBPoly& P, float z, float w[CPCT_W]) {
  const float s = fmaf(2.f, z, -1.f);
  const float s2 = s * s;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float E = P.e[i][CPCT_NPOLY - 1];
    float O = P.o[i][CPCT_NPOLY - 1];
#pragma unroll
    for (int d = CPCT_NPOLY - 2; d >= 0; --d) {
      E = fmaf(E, s2, P.e[i][d]);
      O = fmaf(O, s2, P.o[i][d]);
    }
    w[i] = fmaf(s, O, E);
    w[5 - i] = fmaf(-s, O, E);
  }
  // open support: the tap at distance exactly W/2 has weight 0
  if (z == 0.f) w[5] = 0.f;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------------------
// mbarrier + TMA (bulk tensor copy) helpers; every wait is bounded
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of `bar` for at most ~`max_cycles` SM clocks.
// Returns false on timeout (the caller records the error and bails out).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long max_cycles) {
  long long t0 = clock64();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > max_cycles) return false;
  }
  return false;
}
// 2-D tiled TMA load of a box into shared memory, completion on `bar`.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// plain bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to shared memory, completion on `bar`
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// order this thread's earlier shared-memory accesses (generic proxy) before
// its later bulk copies into shared memory (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
#define CPCT_CUDA_TRY(expr)                      \
  do {                                           \
    cudaError_t e__ = (expr);                    \
    if (e__ != cudaSuccess) return CPCT_ECUDA;   \
  } while (0)

// FFT pass decomposition shared by the kernels and the twiddle-table builder:
// greedy radix-16 passes, the last pass takes the remaining factor (2..16).
__host__ __device__ constexpr int fft_npass(int logn) { return (logn + 3) / 4; }
__host__ __device__ constexpr int fft_lr(int logn, int p) {
  return p < fft_npass(logn) - 1 ? 4 : logn - 4 * (fft_npass(logn) - 1);
}
__host__ __device__ constexpr int fft_ll(int p) { return 4 * p; }
__host__ __device__ constexpr int fft_tw_offset(int logn, int p) {
  int off = 0;
  for (int q = 1; q < p; ++q) off += ((1 << fft_lr(logn, q)) - 1) << fft_ll(q);
  return off;
}
__host__ __device__ constexpr int fft_tw_size(int logn) { return fft_tw_offset(logn, fft_npass(logn)); }

// launchers implemented in radon.cu
int cpct_launch_fwd(cpct_plan* p, const float* d_img, float* d_sino, cudaStream_t s);
int cpct_launch_adj(cpct_plan* p, const float* d_sino, float* d_img, cudaStream_t s);
// the adjoint with the ray spectra weighted by ramp * |k| (ramp = 0: none)
// and every kernel skipped while *skip != 0 (skip: device flag or null)
int cpct_launch_adj_ramp(cpct_plan* p, const float* d_sino, float* d_img, float ramp, const int* skip,
                         cudaStream_t s);
// the forward with every kernel skipped while *skip != 0
int cpct_launch_fwd_skip(cpct_plan* p, const float* d_img, float* d_sino, const int* skip, cudaStream_t s);
int cpct_launch_fwd_c(cpct_plan* p, const float* d_img, float2* d_sino_c, cudaStream_t s);
int cpct_launch_adj_c(cpct_plan* p, const float2* d_sino_c, float* d_img, cudaStream_t s);
int cpct_radon_setup_attributes(int logG, int logNs);
// resident CTAs of a gridding kernel on the current GPU (SMs x CTAs per SM):
// which 0 the gather of T x T bins, 1 the spread with `threads` threads per
// item; 0 if unknown
int cpct_gridding_resident(int which, int T, int threads);
