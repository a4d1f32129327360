// Plan construction: geometry, Kaiser-Bessel kernel approximation and
// deapodization (built on the device in FP64), FFT twiddle tables, and the
// bin plans of the polar samples.
//
// Gridding (section "fast radon transform") convolves the irregular polar
// samples with a kernel on the regular grid.  The paper divides the sample
// plane into bins (one thread block per bin) chosen by a quadtree on the cost
// samples x grid points.  A plan's bins are either a uniform tiling (16, 32
// or 64 grid points; 32 by default) or that quadtree (bins.cu), chosen per
// operator by cpct_plan_set_bins or the autotuner; every bin whose list is
// longer than a cap is split into several work items (ordered longest
// first), which balances the load around the origin where all rays meet.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "bins.cuh"
#include "common.cuh"

namespace {

constexpr int kPolyDeg = 9;            // Chebyshev interpolation degree per tap
constexpr int kCapAuto = 0;            // work-item caps chosen from the geometry (auto_*_cap)
constexpr int kRoundLanes = 32;        // samples per adjoint round (32; 16 and 64 are tuner options)

// ---------------------------------------------------------------------------
// FP64 device builders (kernel table, deapodization, twiddles)
// ---------------------------------------------------------------------------
// I0(x) = sum_m (x^2/4)^m / (m!)^2  (all terms positive: no cancellation)
__device__ double i0_series(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int m = 1; m < 400; ++m) {
    term *= q / ((double)m * (double)m);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  return sum;
}

// g(t) = (I0(beta sqrt(1 - (2t/W)^2)) - 1) / (I0(beta) - 1), |t| < W/2: the
// Kaiser-Bessel window minus its edge pedestal (continuous at |t| = W/2)
__device__ double kb_g(double t, double beta, double W) {
  const double a = 2.0 * t / W;
  const double w = 1.0 - a * a;
  if (w <= 0.0) return 0.0;
  return (i0_series(beta * sqrt(w)) - 1.0) / (i0_series(beta) - 1.0);
}

// One thread per tap i: Chebyshev interpolation of w_i(s) = g(z + 2 - i),
// z = (s+1)/2, at the kPolyDeg+1 Chebyshev nodes, converted to monomials in s.
__global__ void k_build_poly(double* __restrict__ out, double beta, double W) {
  const int i = threadIdx.x;
  if (i >= CPCT_W) return;
  constexpr int n = kPolyDeg + 1;
  double f[n], c[n];
  for (int mm = 0; mm < n; ++mm) {
    const double s = cospi((mm + 0.5) / n);
    f[mm] = kb_g(0.5 * (s + 1.0) + 2.0 - i, beta, W);
  }
  for (int k = 0; k < n; ++k) {
    double acc = 0.0;
    for (int mm = 0; mm < n; ++mm) acc += f[mm] * cospi(k * (mm + 0.5) / n);
    c[k] = (k == 0 ? 1.0 : 2.0) * acc / n;
  }
  // T_0 = 1, T_1 = s, T_{k+1} = 2 s T_k - T_{k-1}
  double Tm[n], T0[n], T1[n], mono[n];
  for (int d = 0; d < n; ++d) { T0[d] = 0.0; T1[d] = 0.0; mono[d] = 0.0; Tm[d] = 0.0; }
  T0[0] = 1.0;
  T1[1] = 1.0;
  mono[0] += c[0];
  for (int d = 0; d < n; ++d) mono[d] += c[1] * T1[d];
  for (int k = 2; k < n; ++k) {
    for (int d = 0; d < n; ++d) Tm[d] = (d > 0 ? 2.0 * T1[d - 1] : 0.0) - T0[d];
    for (int d = 0; d < n; ++d) { T0[d] = T1[d]; T1[d] = Tm[d]; mono[d] += c[k] * Tm[d]; }
  }
  for (int d = 0; d < n; ++d) out[i * n + d] = mono[d];
}

// c[q] = 1 / ghat((q - N/2)/G) with the continuous Fourier transform of g:
// ghat(xi) = W (sinh(z)/z - sin(pi W xi)/(pi W xi)) / (I0(beta) - 1),
// z = sqrt(beta^2 - (pi W xi)^2) > 0 for |xi| <= 1/4
__global__ void k_build_deapod(float* __restrict__ out, int n, int G, double beta, double W) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double xi = (double)(q - n / 2) / (double)G;
  const double pw = 3.14159265358979323846 * W * xi;
  const double z = sqrt(beta * beta - pw * pw);
  const double pedestal = (q == n / 2) ? 1.0 : sinpi(W * xi) / pw;
  const double ghat = W * (sinh(z) / z - pedestal) / (i0_series(beta) - 1.0);
  out[q] = (float)(1.0 / ghat);
}

// twiddles of pass (offset, L, R): entry (m-1)*L + j = exp(-2 pi i m j / (L R))
__global__ void k_build_twiddles(float2* __restrict__ tw, int offset, int L, int R) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (R - 1) * L) return;
  const int m = idx / L + 1, j = idx % L;
  double s, c;
  sincospi(-2.0 * (double)m * (double)j / ((double)L * R), &s, &c);
  tw[offset + idx] = make_float2((float)c, (float)s);
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// geometry limits shared by plan creation and the host-side introspection
bool geom_ok(const cpct_geom* g) {
  if (!g) return false;
  const int W = g->kb_width ? g->kb_width : 6;
  const double sigma = g->oversamp != 0.0 ? g->oversamp : 2.0;
  if (W != 6 || sigma != 2.0) return false;
  if (!is_pow2(g->n) || g->n < 32 || g->n > 2048) return false;
  if (!is_pow2(g->n_det) || g->n_det < g->n || g->n_det > 4096) return false;
  if (g->n_views < 1 || g->n_views > 32768) return false;
  if (g->angles)
    for (int j = 0; j < g->n_views; ++j)
      if (!(g->angles[j] >= 0.0 && g->angles[j] < M_PI)) return false;
  return true;
}

struct Alloc {
  cpct_plan* p;
  bool fail_next;
  int operator()(void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (fail_next) { fail_next = false; return CPCT_ENOMEM; }
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) { *ptr = nullptr; return CPCT_ENOMEM; }
    p->device_bytes += bytes;
    return CPCT_OK;
  }
};

template <class T>
int upload(Alloc& al, T** dst, const std::vector<T>& src, cudaStream_t s) {
  int rc = al((void**)dst, src.size() * sizeof(T));
  if (rc) return rc;
  if (!src.empty())
    CPCT_CUDA_TRY(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return CPCT_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}


void free_plan(cpct_plan* p) {
  if (!p) return;
  cpct_host_stream_release(p);
  cpct_graph_free(p);
  cpct_prof_free(p);
  cpct_plan_streams_destroy(p);
  // per-plan workspaces
  void* own[] = {p->d_Hx, p->d_Ax, p->d_H1, p->d_Q, p->d_partials, p->d_stage_img, p->d_stage_sino, p->d_err};
  for (void* q : own)
    if (q) cudaFree(q);
  // geometry data, shared with clones: freed with the last plan
  const bool last = !p->shared || --p->shared->refs == 0;
  if (last) {
    void* geo[] = {p->d_poly64, p->d_ray, p->d_deapod, p->d_twG, p->d_twNs, p->d_fwd_items, p->d_fwd_ids,
                   p->d_adj_items, p->d_adj_ids, p->d_split};
    for (void* q : geo)
      if (q) cudaFree(q);
    delete p->shared;
  }
  delete p;
}

// TMA descriptors of the forward extended spectrum (viewed as float32 pairs),
// one per bin size: boxes of T + 5 rows of T + 6 complex values
int encode_hx_map(cpct_plan* p) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return CPCT_EUNSUPPORTED;
  for (int c = 0; c < cpct_detail::kNumTileClasses; ++c) {
    const int T = cpct_detail::class_tile(c);
    cuuint64_t dims[2] = {(cuuint64_t)2 * p->ldh, (cuuint64_t)p->ext_rows};
    cuuint64_t strides[1] = {(cuuint64_t)p->ldh * sizeof(float2)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * (T + CPCT_HALO + 1)), (cuuint32_t)(T + CPCT_HALO)};
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = enc(&p->tmap_Hx[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->d_Hx, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return CPCT_ECUDA;
  }
  return CPCT_OK;
}

// domains of the bins: forward, the first points (columns 0..G-1, rows up to
// the largest first row); adjoint, every cell a footprint touches
void fwd_domain(const cpct_detail::Samples& s, int G, int* W, int* H) {
  int mr = 0;
  for (int r : s.rb0) mr = std::max(mr, r);
  *W = G;
  *H = mr + 1;
}
void adj_domain(const cpct_detail::Samples& s, int G, int* W, int* H) {
  int mr = 0;
  for (int r : s.rb0) mr = std::max(mr, r);
  *W = G + CPCT_HALO;
  *H = mr + CPCT_HALO + 1;
}

constexpr double kQuadAlpha = 2.0;  // quadtree: split while cost > alpha x mean leaf cost

void make_layout(const cpct_detail::Samples& s, int W, int H, int kind, int tile, cpct_detail::BinLayout& L) {
  if (kind == cpct_detail::BIN_QUADTREE) cpct_detail::quadtree_layout(s, W, H, kQuadAlpha, L);
  else cpct_detail::uniform_layout(tile, W, H, L);
}

bool bins_args_ok(int kind, int tile) {
  return kind == cpct_detail::BIN_QUADTREE || (kind == cpct_detail::BIN_UNIFORM && (tile == 16 || tile == 32 || tile == 64));
}

}  // namespace

// TMA descriptor of a caller's N x N float32 image for the forward column
// transform: boxes of 8 columns (32 bytes) by min(N, 256) rows.  Kept in the
// plan with the image address it was encoded for, so a repeated address
// costs nothing.
int cpct_image_cols_map(cpct_plan* p, const float* img, const CUtensorMap** out) {
  if (p->tmap_img_ptr != img) {
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) return CPCT_EUNSUPPORTED;
    cuuint64_t dims[2] = {(cuuint64_t)p->n, (cuuint64_t)p->n};
    cuuint64_t strides[1] = {(cuuint64_t)p->n * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)cpct_col_block_width(), (cuuint32_t)std::min(p->n, 256)};
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = enc(&p->tmap_img, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(img), dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
      p->tmap_img_ptr = nullptr;
      return CPCT_ECUDA;
    }
    p->tmap_img_ptr = img;
  }
  *out = &p->tmap_img;
  return CPCT_OK;
}


// ---------------------------------------------------------------------------
// bin lists (exported for host-side tests: no GPU needed)
// ---------------------------------------------------------------------------
namespace {

struct HostBins {
  cpct_detail::Samples s;
  cpct_detail::BinLayout fl, al;
  cpct_detail::BinLists fwd, adj;
  int fW, fH, aW, aH;
};

int host_bins(const cpct_geom* g, int kind, int tile, HostBins& h, bool rounds_order = true) {
  if (!geom_ok(g) || !bins_args_ok(kind, tile)) return CPCT_EINVAL;
  const int G = 2 * g->n;
  std::vector<float4> ray;
  cpct_detail::make_rays(g->n, g->n_det, g->n_views, g->angles, (double)G / g->n_det, ray);
  cpct_detail::make_samples(g->n_det, g->n_views, G, ray, h.s);
  fwd_domain(h.s, G, &h.fW, &h.fH);
  adj_domain(h.s, G, &h.aW, &h.aH);
  make_layout(h.s, h.fW, h.fH, kind, tile, h.fl);
  make_layout(h.s, h.aW, h.aH, kind, tile, h.al);
  cpct_detail::assign_fwd(h.s, h.fW, h.fH, h.fl, h.fwd);
  cpct_detail::assign_adj(h.s, h.aW, h.aH, h.al, h.adj);
  (void)rounds_order;
  return CPCT_OK;
}

// every invariant of a bin plan: bins are disjoint squares of 16/32/64
// aligned to their size; forward lists partition the samples by first point;
// adjoint lists hold each sample once in every bin its footprint touches;
// rounds hold every adjoint entry once, footprints of a round disjoint,
// lane = bank class
int check_plan(const HostBins& h, const cpct_detail::Rounds& rd, int* n_packed) {
  int ok = 1;
  const auto& s = h.s;
  auto disjoint = [&](const cpct_detail::BinLayout& L) {
    std::vector<std::pair<int, int>> cells;
    for (const int4& b : L.bins) {
      if (!(b.z == 16 || b.z == 32 || b.z == 64) || b.x % b.z || b.y % b.z) return false;
      for (int y = b.y; y < b.y + b.z; y += 16)
        for (int x = b.x; x < b.x + b.z; x += 16) cells.push_back({y, x});
    }
    std::sort(cells.begin(), cells.end());
    return std::adjacent_find(cells.begin(), cells.end()) == cells.end();
  };
  if (!disjoint(h.fl) || !disjoint(h.al)) ok = 0;
  const size_t ns = s.a0.size();
  std::vector<int> seen(ns, 0);
  for (size_t t = 0; t + 1 < h.fwd.ptr.size() && ok; ++t) {
    const int4 b = h.fl.bins[t];
    for (int e = h.fwd.ptr[t]; e < h.fwd.ptr[t + 1]; ++e) {
      const uint32_t id = h.fwd.ids[e];
      const size_t i = (size_t)(id >> 16) * (s.K + 1) + (id & 0xffffu);
      seen[i]++;
      if (s.a0[i] < b.x || s.a0[i] >= b.x + b.z || s.rb0[i] < b.y || s.rb0[i] >= b.y + b.z) ok = 0;
    }
  }
  for (size_t i = 0; i < ns && ok; ++i)
    if (seen[i] != 1) ok = 0;
  // adjoint: a footprint touches bin [x0, x0 + T) x [y0, y0 + T) iff its
  // first point lies in [x0 - 5, x0 + T - 1] x [y0 - 5, y0 + T - 1]; the
  // number of such samples per bin from 2D prefix sums of the first points
  {
    const int PW = h.aW + 1, PH = h.aH + 1;
    std::vector<int> pre((size_t)(PH + 1) * (PW + 1), 0);
    for (size_t i = 0; i < ns; ++i) pre[(size_t)(s.rb0[i] + 1) * (PW + 1) + s.a0[i] + 1]++;
    for (int y = 1; y <= PH; ++y)
      for (int x = 1; x <= PW; ++x)
        pre[(size_t)y * (PW + 1) + x] += pre[(size_t)(y - 1) * (PW + 1) + x] + pre[(size_t)y * (PW + 1) + x - 1] -
                                         pre[(size_t)(y - 1) * (PW + 1) + x - 1];
    auto count = [&](int x0, int y0, int x1, int y1) {  // first points in [x0, x1) x [y0, y1)
      x0 = std::max(0, std::min(x0, PW));
      x1 = std::max(0, std::min(x1, PW));
      y0 = std::max(0, std::min(y0, PH));
      y1 = std::max(0, std::min(y1, PH));
      if (x1 <= x0 || y1 <= y0) return 0;
      const int w = PW + 1;
      return pre[(size_t)y1 * w + x1] - pre[(size_t)y0 * w + x1] - pre[(size_t)y1 * w + x0] + pre[(size_t)y0 * w + x0];
    };
    for (size_t t = 0; t + 1 < h.adj.ptr.size() && ok; ++t) {
      const int4 b = h.al.bins[t];
      const int want = count(b.x - CPCT_HALO, b.y - CPCT_HALO, b.x + b.z, b.y + b.z);
      if (h.adj.ptr[t + 1] - h.adj.ptr[t] != want) ok = 0;
    }
  }
  int packed = 0;
  const bool grp = rd.lanes == cpct_detail::kGroupLanes;
  const int words = cpct_detail::round_words(rd.lanes);
  for (size_t t = 0; t + 1 < rd.ptr.size() && ok; ++t) {
    const int4 b = h.al.bins[t];
    const int ld = cpct_detail::round_pitch(b.z);
    std::vector<uint32_t> got;
    for (int r = rd.ptr[t]; r < rd.ptr[t + 1] && ok; ++r) {
      std::vector<int> cells;
      const uint32_t* w = rd.ids.data() + (size_t)r * words;
      int base = -1;
      for (int l = 0; l < (grp ? cpct_detail::kGroupSlots : rd.lanes); ++l) {
        const uint32_t id = grp ? w[4 * l] : w[l];
        if (id == 0xffffffffu) {
          if (grp && l == 0) ok = 0;  // slot 0 opens every group
          continue;
        }
        got.push_back(id);
        const size_t i = (size_t)(id >> 16) * (s.K + 1) + (id & 0xffffu);
        const int ar = s.a0[i] - b.x + CPCT_HALO, br = s.rb0[i] - b.y + CPCT_HALO;
        if (ar < 0 || br < 0 || ar > b.z + CPCT_HALO - 1 || br > b.z + CPCT_HALO - 1) ok = 0;
        const int cls = (br * ld + ar) & 15;
        if (grp) {
          // slot classes follow the conflict-free pattern; the payload is the
          // sample's fractions and accumulator coordinates
          if (l == 0) base = cls;
          if (cls != ((base + cpct_detail::kGroupPattern[l]) & 15)) ok = 0;
          uint32_t zu, zv;
          std::memcpy(&zu, &s.zu[i], 4);
          std::memcpy(&zv, &s.zv[i], 4);
          if (w[4 * l + 1] != zu || w[4 * l + 2] != zv || w[4 * l + 3] != ((uint32_t)ar | ((uint32_t)br << 16))) ok = 0;
        } else if (cls != (l & 15)) {
          ok = 0;
        }
        for (int q = 0; q < CPCT_W; ++q)
          for (int c = 0; c < CPCT_W; ++c) cells.push_back((br + q) * ld + ar + c);
      }
      std::sort(cells.begin(), cells.end());
      if (std::adjacent_find(cells.begin(), cells.end()) != cells.end()) ok = 0;
    }
    std::vector<uint32_t> want_ids(h.adj.ids.begin() + h.adj.ptr[t], h.adj.ids.begin() + h.adj.ptr[t + 1]);
    std::sort(got.begin(), got.end());
    std::sort(want_ids.begin(), want_ids.end());
    if (got != want_ids) ok = 0;
    packed += (int)got.size();
  }
  if (n_packed) *n_packed = packed;
  return ok;
}

}  // namespace

// conflict-free rounds or column groups of the adjoint bins
void pack_adj(const cpct_detail::Samples& s, const cpct_detail::BinLayout& L, const cpct_detail::BinLists& b,
              int lanes, cpct_detail::Rounds& rd) {
  if (lanes == cpct_detail::kGroupLanes) cpct_detail::pack_groups(s, L, b, rd);
  else cpct_detail::pack_rounds(s, L, b, lanes, rd);
}

bool lanes_ok(int lanes) { return lanes == 16 || lanes == 32 || lanes == 64 || lanes == cpct_detail::kGroupLanes; }

// Round packing of the adjoint bins of a geometry (default bin plan, host
// only): number of rounds, number of packed samples, and 1 if every round
// is footprint- and bank-conflict free and every bin entry appears exactly
// once, else 0.
extern "C" int cpct_debug_rounds(const cpct_geom* g, int* n_rounds, int* n_packed, int* valid) {
  HostBins h;
  int rc = host_bins(g, cpct_detail::BIN_UNIFORM, CPCT_TILE, h);
  if (rc) return rc;
  cpct_detail::Rounds rd;
  pack_adj(h.s, h.al, h.adj, kRoundLanes, rd);
  const int ok = check_plan(h, rd, n_packed);
  if (n_rounds) *n_rounds = (int)(rd.ids.size() / cpct_detail::round_words(rd.lanes));
  if (valid) *valid = ok;
  return CPCT_OK;
}

// A bin plan of a geometry (host only): kind 0 uniform tiles of `tile`
// points, kind 1 the quadtree, adjoint rounds of `lanes` samples (0: the
// default width).  Reports the forward and adjoint bin counts, the bins of
// each size class (T = 16, 32, 64) of the adjoint plan, the rounds and 1 if
// every invariant holds (check_plan).
extern "C" int cpct_debug_binplan(const cpct_geom* g, int kind, int tile, int lanes, int* n_fwd_bins,
                                  int* n_adj_bins, int* adj_class_bins, int* n_rounds, int* valid) {
  if (lanes == 0) lanes = kRoundLanes;
  if (!lanes_ok(lanes)) return CPCT_EINVAL;
  HostBins h;
  int rc = host_bins(g, kind, tile, h);
  if (rc) return rc;
  cpct_detail::Rounds rd;
  pack_adj(h.s, h.al, h.adj, lanes, rd);
  if (valid) *valid = check_plan(h, rd, nullptr);
  if (n_fwd_bins) *n_fwd_bins = (int)h.fl.bins.size();
  if (n_adj_bins) *n_adj_bins = (int)h.al.bins.size();
  if (adj_class_bins) {
    for (int c = 0; c < cpct_detail::kNumTileClasses; ++c) adj_class_bins[c] = 0;
    for (const int4& b : h.al.bins) adj_class_bins[cpct_detail::tile_class(b.z)]++;
  }
  if (n_rounds) *n_rounds = (int)(rd.ids.size() / cpct_detail::round_words(rd.lanes));
  return CPCT_OK;
}

// which = 0: forward bins, 1: adjoint bins (default bin plan).  Reports the
// number of bins, the number of entries and a checksum sum(id * (position +
// 1)) of the id list.
extern "C" int cpct_debug_bins(const cpct_geom* g, int which, int* n_tiles, int* n_entries, int64_t* checksum) {
  HostBins h;
  int rc = host_bins(g, cpct_detail::BIN_UNIFORM, CPCT_TILE, h);
  if (rc) return rc;
  const cpct_detail::BinLists& b = which ? h.adj : h.fwd;
  if (n_tiles) *n_tiles = (int)b.ptr.size() - 1;
  if (n_entries) *n_entries = (int)b.ids.size();
  if (checksum) {
    int64_t cs = 0;
    for (size_t i = 0; i < b.ids.size(); ++i) cs += (int64_t)b.ids[i] * (int64_t)(i % 1000003 + 1);
    *checksum = cs;
  }
  return CPCT_OK;
}

// Copy the bin list of bin `tile` (which = 0 forward, 1 adjoint; default bin
// plan) into ids (capacity cap); returns the number of entries or a negative
// status.
extern "C" int cpct_debug_bin_tile(const cpct_geom* g, int which, int tile, uint32_t* ids, int cap) {
  HostBins h;
  int rc = host_bins(g, cpct_detail::BIN_UNIFORM, CPCT_TILE, h);
  if (rc) return rc;
  const cpct_detail::BinLists& b = which ? h.adj : h.fwd;
  if (tile < 0 || tile >= (int)b.ptr.size() - 1) return CPCT_EINVAL;
  const int cnt = b.ptr[tile + 1] - b.ptr[tile];
  for (int i = 0; i < cnt && i < cap; ++i) ids[i] = b.ids[b.ptr[tile] + i];
  return cnt;
}

// Sample coordinate split exactly as the kernels do it (host mirror).
extern "C" int cpct_debug_split(float k, float hi, float lo, int* fl, float* z) {
  cpct_detail::host_split(k, hi, lo, fl, z);
  return CPCT_OK;
}

namespace {

// replace a device array by a new upload of `src` (at least one element)
template <class T>
int replace_upload(cpct_plan* p, T** dst, const std::vector<T>& src, cudaStream_t s) {
  T* d = nullptr;
  const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  if (cudaMalloc((void**)&d, bytes) != cudaSuccess) return CPCT_ENOMEM;
  if (!src.empty() && cudaMemcpyAsync(d, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaFree(d);
    return CPCT_ECUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaFree(d);
    return CPCT_ECUDA;
  }
  if (*dst) cudaFree(*dst);
  *dst = d;
  p->device_bytes += bytes;
  return CPCT_OK;
}

// Automatic work-item sizes.  The items of a launch run their samples or
// rounds one after another, so the longest item bounds the launch: items
// are cut to about the work one resident CTA gets when the work is spread
// evenly.  Spread: 1.2 x rounds / resident items, 8..64 rounds; gather:
// 0.67 x samples / resident CTAs of the persistent grid, a multiple of 64,
// 256..4096 samples.  Measured on GB300 from 512^2 / 90 views to 2048^2 /
// 1024 views: within a few percent of the best fixed cap at every size
// (fixed caps of 64 rounds and 1024 samples left the smaller geometries
// bound by their longest items: 1024^2 / 128 views, spread 45 -> 14 us,
// gather 16 -> 10 us).  Without a GPU, a GB300's resident counts are used
// (152 SMs; 14 spread items or 9 gather CTAs of 32 x 32 bins per SM).
constexpr int kNominalSpreadResident = 152 * 14;
constexpr int kNominalGatherResident = 152 * 9;

// resident CTAs per slice when `concurrency` slices share the GPU
int share(int resident, int nominal, int concurrency) {
  if (resident <= 0) resident = nominal;
  return std::max(1, resident / std::max(1, concurrency));
}

int auto_adj_cap(long long rounds, int resident, int lanes) {
  if (resident <= 0) resident = kNominalSpreadResident;
  // a column group holds up to 5 samples, a round up to 16 .. 64: the same
  // bounds in samples
  const int lo = lanes == cpct_detail::kGroupLanes ? 24 : 8, hi = 8 * lo;
  const long long c = (12 * rounds / resident + 5) / 10;
  return (int)std::min<long long>(hi, std::max<long long>(lo, c));
}

int auto_fwd_cap(long long samples, int resident) {
  if (resident <= 0) resident = kNominalGatherResident;
  const long long c = (67 * samples / resident) / 100 / 64 * 64;
  return (int)std::min<long long>(4096, std::max<long long>(256, c));
}

// forward work items of the installed bin plan with `cap` samples per item
// (kCapAuto: auto_fwd_cap)
int install_fwd_items(cpct_plan* p, int cap, cudaStream_t s) {
  cpct_graph_clear(p);  // captured graphs hold the old work items
  if (cap == kCapAuto)
    cap = auto_fwd_cap(p->shared->fwd_ptr.empty() ? 0 : p->shared->fwd_ptr.back(),
                       share(cpct_gridding_resident(0, p->fwd_tile ? p->fwd_tile : CPCT_TILE, 0),
                             kNominalGatherResident, p->concurrency));
  cpct_detail::BinLayout L;
  L.bins = p->shared->fwd_bins;
  cpct_detail::Items it;
  cpct_detail::fwd_items(L, p->shared->fwd_ptr, cap, it);
  int rc = replace_upload(p, &p->d_fwd_items, it.items, s);
  if (rc) return rc;
  p->n_fwd_items = (int)it.items.size();
  for (int c = 0; c <= cpct_detail::kNumTileClasses; ++c) p->fwd_cls[c] = it.cls[c];
  p->fwd_cap = cap;
  return CPCT_OK;
}

// adjoint work items (and split list, partial tiles) with `cap` rounds per
// item (kCapAuto: auto_adj_cap)
int install_adj_items(cpct_plan* p, int cap, cudaStream_t s) {
  cpct_graph_clear(p);  // captured graphs hold the old work items
  if (cap == kCapAuto)
    cap = auto_adj_cap(p->shared->round_ptr.empty() ? 0 : p->shared->round_ptr.back(),
                       share(cpct_gridding_resident(1, p->adj_tile ? p->adj_tile : CPCT_TILE, p->round_lanes == 64 ? 64 : 32),
                             kNominalSpreadResident, p->concurrency),
                       p->round_lanes);
  cpct_detail::BinLayout L;
  L.bins = p->shared->adj_bins;
  cpct_detail::Items it;
  cpct_detail::adj_items(L, p->shared->round_ptr, cap, it);
  int rc = replace_upload(p, &p->d_adj_items, it.items, s);
  if (!rc) rc = replace_upload(p, &p->d_split, it.split, s);
  if (rc) return rc;
  if (it.partial_elems > p->partial_elems || !p->d_partials) {
    float2* dp = nullptr;
    if (cudaMalloc(&dp, sizeof(float2) * (size_t)std::max(1LL, it.partial_elems)) != cudaSuccess) return CPCT_ENOMEM;
    if (p->d_partials) cudaFree(p->d_partials);
    p->d_partials = dp;
  }
  p->n_adj_items = (int)it.items.size();
  for (int c = 0; c <= cpct_detail::kNumTileClasses; ++c) {
    p->adj_cls[c] = it.cls[c];
    p->split_cls[c] = it.split_cls[c];
  }
  p->n_split = (int)it.split.size();
  p->partial_elems = it.partial_elems;
  p->n_slots = (int)((it.partial_elems + 1023) / 1024);
  p->adj_cap = cap;
  return CPCT_OK;
}

// build and upload a bin plan for the forward gather
int install_fwd_plan(cpct_plan* p, int kind, int tile, int cap, cudaStream_t s) {
  cpct_detail::Samples smp;
  cpct_detail::make_samples(p->ns, p->m, p->G, p->shared->ray, smp);
  int W, H;
  fwd_domain(smp, p->G, &W, &H);
  cpct_detail::BinLayout L;
  make_layout(smp, W, H, kind, tile, L);
  cpct_detail::BinLists b;
  cpct_detail::assign_fwd(smp, W, H, L, b);
  cpct_detail::order_fwd(smp, L, b);
  int rc = replace_upload(p, &p->d_fwd_ids, b.ids, s);
  if (rc) return rc;
  p->shared->fwd_bins = L.bins;
  p->shared->fwd_ptr = b.ptr;
  p->fwd_kind = kind;
  p->fwd_tile = kind == cpct_detail::BIN_UNIFORM ? tile : 0;
  return install_fwd_items(p, cap, s);
}

// build and upload a bin plan for the adjoint spread (bins, rounds)
int install_adj_plan(cpct_plan* p, int kind, int tile, int cap, cudaStream_t s, int lanes = 0) {
  if (lanes == 0) lanes = p->round_lanes ? p->round_lanes : kRoundLanes;
  cpct_detail::Samples smp;
  cpct_detail::make_samples(p->ns, p->m, p->G, p->shared->ray, smp);
  int W, H;
  adj_domain(smp, p->G, &W, &H);
  cpct_detail::BinLayout L;
  make_layout(smp, W, H, kind, tile, L);
  cpct_detail::BinLists b;
  cpct_detail::assign_adj(smp, W, H, L, b);
  cpct_detail::Rounds rd;
  pack_adj(smp, L, b, lanes, rd);
  int rc = replace_upload(p, &p->d_adj_ids, rd.ids, s);
  if (rc) return rc;
  p->round_lanes = lanes;
  p->shared->adj_bins = L.bins;
  p->shared->round_ptr = rd.ptr;
  p->adj_kind = kind;
  p->adj_tile = kind == cpct_detail::BIN_UNIFORM ? tile : 0;
  return install_adj_items(p, cap, s);
}

}  // namespace

extern "C" int cpct_plan_create(cpct_plan** out, const cpct_geom* g, cudaStream_t stream) {
  if (!out) return CPCT_EINVAL;
  *out = nullptr;
  if (!g) return CPCT_EINVAL;
  if (!geom_ok(g)) return CPCT_EINVAL;
  const int n = g->n, ns = g->n_det, m = g->n_views;
  const int W = 6;
  const double sigma = 2.0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CPCT_ECUDA;

  cpct_plan* p = new (std::nothrow) cpct_plan;
  if (!p) return CPCT_ENOMEM;
  std::memset(p, 0, sizeof(*p));
  p->n = n;
  p->ns = ns;
  p->m = m;
  p->G = 2 * n;
  p->K = ns / 2;
  p->logn = ilog2(n);
  p->logG = ilog2(p->G);
  p->logNs = ilog2(ns);
  p->ldh = p->G + 8;
  p->ext_rows = n + 8;
  p->ldq = p->K + 2;
  p->flags = g->flags;
  p->scale = (double)p->G / (double)ns;
  Alloc al{p, (g->flags & CPCT_PLAN_FAIL_ALLOC) != 0};
  int rc = CPCT_OK;
#define TRY(x)                         \
  do {                                 \
    rc = (x);                          \
    if (rc != CPCT_OK) goto fail;      \
  } while (0)
#define TRYC(x)                                      \
  do {                                               \
    if ((x) != cudaSuccess) { rc = CPCT_ECUDA; goto fail; } \
  } while (0)

  {
    int rca = cpct_radon_setup_attributes(p->logG, p->logNs);
    if (rca != CPCT_OK) { rc = rca; goto fail; }
    TRY(cpct_plan_streams_create(p));
    // geometry
    std::vector<float4> ray;
    cpct_detail::make_rays(n, ns, m, g->angles, p->scale, ray);
    TRY(upload(al, &p->d_ray, ray, stream));
    // kernel approximation, deapodization, twiddles (FP64 on the device)
    const double beta = M_PI * std::sqrt((W / sigma) * (W / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
    TRY(al((void**)&p->d_poly64, sizeof(double) * CPCT_W * (kPolyDeg + 1)));
    k_build_poly<<<1, 32, 0, stream>>>(p->d_poly64, beta, (double)W);
    TRY(al((void**)&p->d_deapod, sizeof(float) * n));
    k_build_deapod<<<(n + 127) / 128, 128, 0, stream>>>(p->d_deapod, n, p->G, beta, (double)W);
    TRY(al((void**)&p->d_twG, sizeof(float2) * std::max(1, fft_tw_size(p->logG))));
    TRY(al((void**)&p->d_twNs, sizeof(float2) * std::max(1, fft_tw_size(p->logNs))));
    for (int which = 0; which < 2; ++which) {
      const int lg = which ? p->logNs : p->logG;
      float2* tw = which ? p->d_twNs : p->d_twG;
      for (int pp = 1; pp < fft_npass(lg); ++pp) {
        const int L = 1 << fft_ll(pp), R = 1 << fft_lr(lg, pp);
        const int cnt = (R - 1) * L;
        k_build_twiddles<<<(cnt + 255) / 256, 256, 0, stream>>>(tw, fft_tw_offset(lg, pp), L, R);
      }
    }
    TRYC(cudaGetLastError());
    // workspaces
    const size_t hx_bytes = sizeof(float2) * (size_t)p->ext_rows * p->ldh;
    TRY(al((void**)&p->d_Hx, hx_bytes));
    TRY(al((void**)&p->d_Ax, hx_bytes));
    TRY(al((void**)&p->d_H1, sizeof(float2) * (size_t)(n + 1) * n));
    TRY(al((void**)&p->d_Q, sizeof(float2) * (size_t)m * p->ldq));
    TRY(al((void**)&p->d_err, sizeof(int)));
    TRYC(cudaMemsetAsync(p->d_Hx, 0, hx_bytes, stream));
    TRYC(cudaMemsetAsync(p->d_Ax, 0, hx_bytes, stream));
    TRYC(cudaMemsetAsync(p->d_Q, 0, sizeof(float2) * (size_t)m * p->ldq, stream));
    TRYC(cudaMemsetAsync(p->d_err, 0, sizeof(int), stream));
    // bins: uniform 32 x 32 tiles for both operators (cpct_plan_set_bins and
    // the autotuner choose others)
    p->shared = new (std::nothrow) PlanShared;
    if (!p->shared) { rc = CPCT_ENOMEM; goto fail; }
    p->shared->ray = ray;
    TRY(install_fwd_plan(p, cpct_detail::BIN_UNIFORM, CPCT_TILE, kCapAuto, stream));
    TRY(install_adj_plan(p, cpct_detail::BIN_UNIFORM, CPCT_TILE, kCapAuto, stream));
    // TMA descriptor of the forward extended spectrum (viewed as float32 pairs)
    TRY(encode_hx_map(p));
    // FP32 copy of the even/odd polynomial parts
    double poly[CPCT_W * (kPolyDeg + 1)];
    TRYC(cudaMemcpyAsync(poly, p->d_poly64, sizeof(poly), cudaMemcpyDeviceToHost, stream));
    TRYC(cudaStreamSynchronize(stream));
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < CPCT_NPOLY; ++d) {
        p->poly.e[i][d] = (float)poly[i * (kPolyDeg + 1) + 2 * d];
        p->poly.o[i][d] = (float)poly[i * (kPolyDeg + 1) + 2 * d + 1];
      }
    TRYC(cudaGetLastError());
  }
#undef TRY
#undef TRYC
  *out = p;
  return CPCT_OK;
fail:
  cudaStreamSynchronize(stream);
  free_plan(p);
  return rc;
}

extern "C" int cpct_plan_destroy(cpct_plan* plan) {
  if (!plan) return CPCT_OK;
  cudaDeviceSynchronize();
  free_plan(plan);
  return CPCT_OK;
}

extern "C" int cpct_plan_info(const cpct_plan* p, int* n, int* n_det, int* n_views, int* grid, size_t* bytes) {
  if (!p) return CPCT_EINVAL;
  if (n) *n = p->n;
  if (n_det) *n_det = p->ns;
  if (n_views) *n_views = p->m;
  if (grid) *grid = p->G;
  if (bytes) *bytes = p->device_bytes;
  return CPCT_OK;
}

extern "C" int cpct_plan_sync(cpct_plan* p, cudaStream_t stream) {
  if (!p) return CPCT_EINVAL;
  int err = 0;
  CPCT_CUDA_TRY(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CPCT_CUDA_TRY(cudaStreamSynchronize(stream));
  if (err) {
    CPCT_CUDA_TRY(cudaMemsetAsync(p->d_err, 0, sizeof(int), stream));
    CPCT_CUDA_TRY(cudaStreamSynchronize(stream));
    return (err & CPCT_ERR_TIMEOUT) ? CPCT_ETIMEOUT : CPCT_ECUDA;
  }
  return CPCT_OK;
}

// FP64 polynomial coefficients [6][10] (monomials in s = 2z-1 per tap) and
// the FP32 deapodization vector [N], copied to host buffers (either may be NULL).
extern "C" int cpct_debug_tables(cpct_plan* p, double* h_poly64, float* h_deapod) {
  if (!p) return CPCT_EINVAL;
  if (h_poly64)
    CPCT_CUDA_TRY(cudaMemcpy(h_poly64, p->d_poly64, sizeof(double) * CPCT_W * (kPolyDeg + 1), cudaMemcpyDeviceToHost));
  if (h_deapod) CPCT_CUDA_TRY(cudaMemcpy(h_deapod, p->d_deapod, sizeof(float) * p->n, cudaMemcpyDeviceToHost));
  return CPCT_OK;
}

// ---------------------------------------------------------------------------
// clones and the work-item autotuner
// ---------------------------------------------------------------------------
extern "C" int cpct_plan_clone(const cpct_plan* src, cpct_plan** out, cudaStream_t stream) {
  if (!src || !out || !src->shared) return CPCT_EINVAL;
  *out = nullptr;
  cpct_plan* p = new (std::nothrow) cpct_plan;
  if (!p) return CPCT_ENOMEM;
  std::memcpy(p, src, sizeof(*p));
  // fresh per-plan state; the geometry pointers stay shared
  p->side[0] = p->side[1] = nullptr;
  p->ev_fork = p->ev_join[0] = p->ev_join[1] = nullptr;
  if (cpct_plan_streams_create(p) != CPCT_OK) {
    cpct_plan_streams_destroy(p);
    delete p;
    return CPCT_ECUDA;
  }
  p->d_Hx = p->d_Ax = p->d_H1 = p->d_Q = p->d_partials = nullptr;
  p->d_stage_img = p->d_stage_sino = nullptr;
  p->d_err = nullptr;
  p->prof = nullptr;
  p->graphs = nullptr;
  p->capturing = nullptr;
  p->hstream = nullptr;
  p->launches = 0;
  p->device_bytes = 0;
  p->shared->refs++;
  Alloc al{p, false};
  int rc = CPCT_OK;
  const size_t hx_bytes = sizeof(float2) * (size_t)p->ext_rows * p->ldh;
  if ((rc = al((void**)&p->d_Hx, hx_bytes)) || (rc = al((void**)&p->d_Ax, hx_bytes)) ||
      (rc = al((void**)&p->d_H1, sizeof(float2) * (size_t)(p->n + 1) * p->n)) ||
      (rc = al((void**)&p->d_Q, sizeof(float2) * (size_t)p->m * p->ldq)) || (rc = al((void**)&p->d_err, sizeof(int))) ||
      (rc = al((void**)&p->d_partials, sizeof(float2) * (size_t)std::max(1LL, p->partial_elems)))) {
    free_plan(p);
    return rc;
  }
  if (cudaMemsetAsync(p->d_Hx, 0, hx_bytes, stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_Ax, 0, hx_bytes, stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_Q, 0, sizeof(float2) * (size_t)p->m * p->ldq, stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_err, 0, sizeof(int), stream) != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess) {
    free_plan(p);
    return CPCT_ECUDA;
  }
  if ((rc = encode_hx_map(p)) != CPCT_OK) {
    free_plan(p);
    return rc;
  }
  *out = p;
  return CPCT_OK;
}

// Autotuner of the bin plans and work-item sizes: for each operator the bin
// plans (uniform 16, 32, 64 and the quadtree) are timed at the default cap,
// then the caps of the fastest plan (gather: 256..4096 samples per item;
// spread: 16..256 rounds per item); every candidate is the median of `reps`
// launches (CUDA events on `stream`) and the fastest is kept.
extern "C" int cpct_plan_tune(cpct_plan* p, int reps, int* fwd_cap, int* adj_cap, cudaStream_t stream) {
  if (!p || !p->shared) return CPCT_EINVAL;
  cpct_host_stream_release(p);  // its cached clone shares this plan's tables
  if (p->shared->refs != 1) return CPCT_EINVAL;  // tune before cloning
  if (reps < 1) reps = 5;
  float *img = nullptr, *sino = nullptr;
  if (cudaMalloc(&img, sizeof(float) * (size_t)p->n * p->n) != cudaSuccess) return CPCT_ENOMEM;
  if (cudaMalloc(&sino, sizeof(float) * (size_t)p->m * p->ns) != cudaSuccess) {
    cudaFree(img);
    return CPCT_ENOMEM;
  }
  cudaMemsetAsync(img, 0, sizeof(float) * (size_t)p->n * p->n, stream);
  cudaMemsetAsync(sino, 0, sizeof(float) * (size_t)p->m * p->ns, stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_op = [&](bool fwd) {
    std::vector<float> t;
    for (int r = 0; r < reps + 1; ++r) {
      cudaEventRecord(e0, stream);
      if (fwd) cpct_launch_fwd(p, img, sino, stream);
      else cpct_launch_adj(p, sino, img, stream);
      cudaEventRecord(e1, stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) t.push_back(ms);  // the first launch warms up
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
  };
  struct Cand {
    int kind, tile;
  };
  const Cand plans[] = {{cpct_detail::BIN_UNIFORM, 16}, {cpct_detail::BIN_UNIFORM, 32}, {cpct_detail::BIN_UNIFORM, 64},
                        {cpct_detail::BIN_QUADTREE, 0}};
  int rc = CPCT_OK;
  for (int op = 0; op < 2 && rc == CPCT_OK; ++op) {
    const bool fwd = op == 0;
    const int cap0 = kCapAuto;
    Cand best = plans[1];
    float tb = 1e30f;
    for (const Cand& c : plans) {
      rc = fwd ? install_fwd_plan(p, c.kind, c.tile, cap0, stream) : install_adj_plan(p, c.kind, c.tile, cap0, stream);
      if (rc != CPCT_OK) break;
      const float t = time_op(fwd);
      if (t < tb) {
        tb = t;
        best = c;
      }
    }
    if (rc == CPCT_OK)
      rc = fwd ? install_fwd_plan(p, best.kind, best.tile, cap0, stream)
               : install_adj_plan(p, best.kind, best.tile, cap0, stream);
    if (!fwd && rc == CPCT_OK) {
      // round width of the adjoint: the fastest of 16, 32 and 64 lanes and
      // column groups
      const int widths[] = {16, 32, 64, cpct_detail::kGroupLanes};
      int best_w = p->round_lanes;
      float tw = time_op(false);
      for (int w : widths) {
        if (w == best_w) continue;
        if ((rc = install_adj_plan(p, best.kind, best.tile, cap0, stream, w)) != CPCT_OK) break;
        const float t = time_op(false);
        if (t < tw) {
          tw = t;
          best_w = w;
        }
      }
      if (rc == CPCT_OK && p->round_lanes != best_w) rc = install_adj_plan(p, best.kind, best.tile, cap0, stream, best_w);
    }
    // caps: the automatic one (installed now), then fixed candidates
    const int fc[] = {256, 512, 1024, 2048, 4096};
    const int ac[] = {8, 16, 32, 64, 128};
    int best_cap = fwd ? p->fwd_cap : p->adj_cap;
    tb = time_op(fwd);
    for (int i = 0; i < 5 && rc == CPCT_OK; ++i) {
      const int cap = fwd ? fc[i] : ac[i];
      if (cap == best_cap) continue;
      if ((rc = fwd ? install_fwd_items(p, cap, stream) : install_adj_items(p, cap, stream)) != CPCT_OK) break;
      const float t = time_op(fwd);
      if (t < tb) {
        tb = t;
        best_cap = cap;
      }
    }
    if (rc == CPCT_OK) rc = fwd ? install_fwd_items(p, best_cap, stream) : install_adj_items(p, best_cap, stream);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(img);
  cudaFree(sino);
  if (fwd_cap) *fwd_cap = p->fwd_cap;
  if (adj_cap) *adj_cap = p->adj_cap;
  return rc;
}

// Install work items with the given caps (0 keeps the current one); the
// plan must not have clones.  Synchronous.
extern "C" int cpct_plan_set_caps(cpct_plan* p, int fwd_cap, int adj_cap, cudaStream_t stream) {
  if (!p || !p->shared || fwd_cap < 0 || adj_cap < 0) return CPCT_EINVAL;
  cpct_host_stream_release(p);  // its cached clone shares this plan's tables
  if (p->shared->refs != 1) return CPCT_EINVAL;
  int rc = CPCT_OK;
  if (fwd_cap > 0) {
    rc = install_fwd_items(p, fwd_cap, stream);
    p->fwd_cap_set = 1;
  }
  if (rc == CPCT_OK && adj_cap > 0) {
    rc = install_adj_items(p, adj_cap, stream);
    p->adj_cap_set = 1;
  }
  return rc;
}

// Automatic caps for `concurrent` slices running at once (each gets that
// share of the resident CTAs).  The plan must not have clones.  Synchronous.
extern "C" int cpct_plan_auto_caps(cpct_plan* p, int concurrent, cudaStream_t stream) {
  if (!p || !p->shared || concurrent < 1) return CPCT_EINVAL;
  cpct_host_stream_release(p);  // its cached clone shares this plan's tables
  if (p->shared->refs != 1) return CPCT_EINVAL;
  p->concurrency = concurrent;
  p->fwd_cap_set = p->adj_cap_set = 0;
  int rc = install_fwd_items(p, kCapAuto, stream);
  if (rc == CPCT_OK) rc = install_adj_items(p, kCapAuto, stream);
  return rc;
}

// Install a bin plan for one operator (which 0 forward, 1 adjoint): kind 0
// uniform tiles of `tile` points (16, 32, 64), kind 1 the quadtree; keeps a
// cap fixed by cpct_plan_set_caps, else takes the automatic cap of the new
// bins.  The plan must not have clones.  Synchronous.
extern "C" int cpct_plan_set_bins(cpct_plan* p, int which, int kind, int tile, cudaStream_t stream) {
  if (!p || !p->shared || (which != 0 && which != 1) || !bins_args_ok(kind, tile)) return CPCT_EINVAL;
  cpct_host_stream_release(p);  // its cached clone shares this plan's tables
  if (p->shared->refs != 1) return CPCT_EINVAL;
  return which == 0 ? install_fwd_plan(p, kind, tile, p->fwd_cap_set ? p->fwd_cap : kCapAuto, stream)
                    : install_adj_plan(p, kind, tile, p->adj_cap_set ? p->adj_cap : kCapAuto, stream);
}

// Width of the adjoint's conflict-free rounds: 16 (one sample per bank
// class, the lower half-warp only), 32 (two per class, one warp) or 64 (four
// per class, two warps); re-packs the installed adjoint bins.  The plan must
// not have clones.  Synchronous.
extern "C" int cpct_plan_set_rounds(cpct_plan* p, int lanes, cudaStream_t stream) {
  if (!p || !p->shared || !lanes_ok(lanes)) return CPCT_EINVAL;
  cpct_host_stream_release(p);  // its cached clone shares this plan's tables
  if (p->shared->refs != 1) return CPCT_EINVAL;
  return install_adj_plan(p, p->adj_kind, p->adj_tile ? p->adj_tile : CPCT_TILE, p->adj_cap_set ? p->adj_cap : kCapAuto,
                          stream, lanes);
}

extern "C" int cpct_plan_rounds(const cpct_plan* p) { return p ? p->round_lanes : CPCT_EINVAL; }

// The bin plans of a plan: kind (0 uniform, 1 quadtree) and tile (uniform
// size, 0 for a quadtree) of each operator, and per operator the bins of
// each size class (T = 16, 32, 64; arrays of 3, may be NULL).
extern "C" int cpct_plan_bins(const cpct_plan* p, int* fwd_kind, int* fwd_tile, int* adj_kind, int* adj_tile,
                              int* fwd_class_bins, int* adj_class_bins) {
  if (!p || !p->shared) return CPCT_EINVAL;
  if (fwd_kind) *fwd_kind = p->fwd_kind;
  if (fwd_tile) *fwd_tile = p->fwd_tile;
  if (adj_kind) *adj_kind = p->adj_kind;
  if (adj_tile) *adj_tile = p->adj_tile;
  for (int which = 0; which < 2; ++which) {
    int* out = which ? adj_class_bins : fwd_class_bins;
    if (!out) continue;
    for (int c = 0; c < cpct_detail::kNumTileClasses; ++c) out[c] = 0;
    for (const int4& b : which ? p->shared->adj_bins : p->shared->fwd_bins) out[cpct_detail::tile_class(b.z)]++;
  }
  return CPCT_OK;
}

// Work-item counts of a plan: forward gather items, adjoint spread items,
// split heavy bins and their partial-tile space in 32 x 32 tiles (slots).
extern "C" int cpct_plan_work(const cpct_plan* p, int* n_fwd_items, int* n_adj_items, int* n_split, int* n_slots) {
  if (!p) return CPCT_EINVAL;
  if (n_fwd_items) *n_fwd_items = p->n_fwd_items;
  if (n_adj_items) *n_adj_items = p->n_adj_items;
  if (n_split) *n_split = p->n_split;
  if (n_slots) *n_slots = p->n_slots;
  return CPCT_OK;
}

// The adjoint work items a plan of geometry g gets with its default bin plan
// and `cap` rounds per item (0: the default cap), built on the host exactly
// as cpct_plan_create / cpct_plan_set_caps build them.  No GPU needed.
extern "C" int cpct_debug_adj_items(const cpct_geom* g, int cap, int* n_items, int* n_split, int* n_slots) {
  if (cap < 0) return CPCT_EINVAL;
  HostBins h;
  int rc = host_bins(g, cpct_detail::BIN_UNIFORM, CPCT_TILE, h);
  if (rc) return rc;
  cpct_detail::Rounds rd;
  pack_adj(h.s, h.al, h.adj, kRoundLanes, rd);
  cpct_detail::Items it;
  cpct_detail::adj_items(h.al, rd.ptr, cap > 0 ? cap : auto_adj_cap(rd.ptr.back(), cpct_gridding_resident(1, CPCT_TILE, 32), rd.lanes), it);
  if (n_items) *n_items = (int)it.items.size();
  if (n_split) *n_split = (int)it.split.size();
  if (n_slots) *n_slots = (int)((it.partial_elems + 1023) / 1024);
  return CPCT_OK;
}

int cpct_plan_streams_create(cpct_plan* p) {
  for (int i = 0; i < 2; ++i)
    if (cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking) != cudaSuccess) return CPCT_ECUDA;
  if (cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess) return CPCT_ECUDA;
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&p->ev_join[i], cudaEventDisableTiming) != cudaSuccess) return CPCT_ECUDA;
  return CPCT_OK;
}

void cpct_plan_streams_destroy(cpct_plan* p) {
  for (int i = 0; i < 2; ++i) {
    if (p->side[i]) cudaStreamDestroy(p->side[i]);
    if (p->ev_join[i]) cudaEventDestroy(p->ev_join[i]);
    p->side[i] = nullptr;
    p->ev_join[i] = nullptr;
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  p->ev_fork = nullptr;
}
