// Plan construction: geometry, Kaiser-Bessel kernel approximation and
// deapodization (built on the device in FP64), FFT twiddle tables, and the
// tile bin lists of the polar samples.
//
// Gridding (section "fast radon transform") convolves the irregular polar
// samples with a kernel on the regular grid.  The paper divides the sample
// plane into bins (one thread block per bin) chosen by a quadtree on the cost
// samples x grid points; here the bins are fixed 32x32 grid tiles and every
// bin whose sample list is longer than a cap is split into several work items
// (ordered longest first), which balances the load around the origin where all
// rays meet.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kPolyDeg = 9;            // Chebyshev interpolation degree per tap
constexpr int kFwdItemMax = 1024;      // samples per forward gather work item
constexpr int kAdjItemRounds = 64;     // conflict-free rounds per adjoint spread work item

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

// host mirror of split_coord (identical IEEE single-precision operations)
void host_split(float k, float hi, float lo, int* fl_out, float* z) {
  float p = k * hi;
  float e = std::fmaf(k, hi, -p);
  float corr = std::fmaf(k, lo, e);
  float fl = std::floor(p);
  float zz = (p - fl) + corr;
  if (zz < 0.f) {
    float t = zz + 1.f;
    if (t < 1.f) { zz = t; fl = fl - 1.f; } else { zz = 0.f; }
  } else if (zz >= 1.f) {
    zz = zz - 1.f;
    fl = fl + 1.f;
  }
  *fl_out = (int)fl;
  *z = zz;
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
  cpct_prof_free(p);
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

int encode_hx_map(cpct_plan* p) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return CPCT_EUNSUPPORTED;
  cuuint64_t dims[2] = {(cuuint64_t)2 * p->ldh, (cuuint64_t)p->ext_rows};
  cuuint64_t strides[1] = {(cuuint64_t)p->ldh * sizeof(float2)};
  cuuint32_t box[2] = {2 * (CPCT_TILE + CPCT_HALO + 1), CPCT_TILE + CPCT_HALO};
  cuuint32_t estr[2] = {1, 1};
  CUresult cr = enc(&p->tmap_Hx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->d_Hx, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS ? CPCT_OK : CPCT_ECUDA;
}

}  // namespace

// ---------------------------------------------------------------------------
// bin lists (exported for host-side tests: no GPU needed)
// ---------------------------------------------------------------------------
extern "C" int cpct_debug_bins(const cpct_geom* g, int which, int* n_tiles, int* n_entries, int64_t* checksum);

namespace cpct_detail {

struct Bins {
  int tiles_x, tiles_y;
  std::vector<int> ptr;          // tiles + 1
  std::vector<uint32_t> ids;     // grouped by tile, increasing id inside a tile
};

struct RayTab {
  std::vector<float4> ray;
};

void make_rays(int n, int ns, int m, const double* angles, double scale, std::vector<float4>& ray) {
  ray.resize(m);
  for (int j = 0; j < m; ++j) {
    const double th = angles ? angles[j] : M_PI * (double)j / (double)m;
    const double c = scale * std::cos(th), s = scale * std::sin(th);
    const float ch = (float)c, sh = (float)s;
    ray[j] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
  }
}

// forward bins: every sample (j, k >= 0) lands in the tile of its footprint's
// first grid point (a0 = floor(u)-2 mod G, buffer row floor(v)); adjoint bins:
// every tile of the extended spectrum that its 6x6 footprint touches.
void build_bins(int n, int ns, int m, int G, const std::vector<float4>& ray, Bins& fwd, Bins& adj,
                std::vector<int>* a0_out = nullptr, std::vector<int>* rb0_out = nullptr) {
  const int K = ns / 2;
  const int T = CPCT_TILE;
  fwd.tiles_x = G / T;
  fwd.tiles_y = n / T + 1;
  adj.tiles_x = G / T + 1;
  adj.tiles_y = (n + 5) / T + 1;
  const int nf = fwd.tiles_x * fwd.tiles_y, na = adj.tiles_x * adj.tiles_y;
  std::vector<int> cf(nf + 1, 0), ca(na + 1, 0);
  std::vector<int> fa0((size_t)m * (K + 1)), frb((size_t)m * (K + 1));
  for (int j = 0; j < m; ++j) {
    for (int k = 0; k <= K; ++k) {
      int fu, fv;
      float zu, zv;
      host_split((float)k, ray[j].x, ray[j].y, &fu, &zu);
      host_split((float)k, ray[j].z, ray[j].w, &fv, &zv);
      const int a0 = (fu - 2) & (G - 1);
      const int rb0 = fv;  // buffer row of the first tap: (floor(v) - 2) + 2
      const size_t sidx = (size_t)j * (K + 1) + k;
      fa0[sidx] = a0;
      frb[sidx] = rb0;
      cf[(rb0 / T) * fwd.tiles_x + a0 / T + 1]++;
      for (int ty = rb0 / T; ty <= (rb0 + CPCT_HALO) / T; ++ty)
        for (int tx = a0 / T; tx <= (a0 + CPCT_HALO) / T; ++tx) ca[ty * adj.tiles_x + tx + 1]++;
    }
  }
  for (int i = 0; i < nf; ++i) cf[i + 1] += cf[i];
  for (int i = 0; i < na; ++i) ca[i + 1] += ca[i];
  fwd.ptr = cf;
  adj.ptr = ca;
  fwd.ids.resize(cf[nf]);
  adj.ids.resize(ca[na]);
  std::vector<int> pf(cf.begin(), cf.end() - 1), pa(ca.begin(), ca.end() - 1);
  for (int j = 0; j < m; ++j) {
    for (int k = 0; k <= K; ++k) {
      const size_t sidx = (size_t)j * (K + 1) + k;
      const int a0 = fa0[sidx], rb0 = frb[sidx];
      const uint32_t id = ((uint32_t)j << 16) | (uint32_t)k;
      fwd.ids[pf[(rb0 / T) * fwd.tiles_x + a0 / T]++] = id;
      for (int ty = rb0 / T; ty <= (rb0 + CPCT_HALO) / T; ++ty)
        for (int tx = a0 / T; tx <= (a0 + CPCT_HALO) / T; ++tx) adj.ids[pa[ty * adj.tiles_x + tx]++] = id;
    }
  }
  if (a0_out) a0_out->swap(fa0);
  if (rb0_out) rb0_out->swap(frb);
}

// Pack the samples of every adjoint tile into rounds of at most 32 samples
// whose 6x6 footprints (clipped to the tile plus a 5-cell halo) are pairwise
// disjoint, so that one warp can add a whole round with one lane per sample
// and no two lanes touching the same accumulator.  The lane of a sample is
// fixed by the 64-bit shared-memory bank pair of its footprint's first cell
// (lanes c and c+16 for bank pair c), which makes every accumulator access of
// a round bank-conflict free.  Greedy first fit in bin order (deterministic).
struct Rounds {
  std::vector<int> tile_ptr;      // tiles + 1, in rounds
  std::vector<uint32_t> ids;      // 32 per round, 0xffffffff = empty lane
};

constexpr int kRoundLd = CPCT_TILE + 2 * CPCT_HALO + 2;  // 44 complex per accumulator row

void pack_rounds(const Bins& adj, int G, const std::vector<int>& fa0, const std::vector<int>& frb, int K,
                 Rounds& out) {
  const int nt = (int)adj.ptr.size() - 1;
  out.tile_ptr.assign(nt + 1, 0);
  out.ids.clear();
  struct R {
    uint64_t occ[CPCT_TILE + 2 * CPCT_HALO];
    uint32_t lanes;
    int count;
  };
  std::vector<R> rounds;
  for (int t = 0; t < nt; ++t) {
    const int TC = (t % adj.tiles_x) * CPCT_TILE, TR = (t / adj.tiles_x) * CPCT_TILE;
    rounds.clear();
    size_t first_open = 0;
    std::vector<std::array<uint32_t, 32>> lanes_of;
    for (int e = adj.ptr[t]; e < adj.ptr[t + 1]; ++e) {
      const uint32_t id = adj.ids[e];
      const size_t sidx = (size_t)(id >> 16) * (K + 1) + (id & 0xffffu);
      const int ar = fa0[sidx] - TC + CPCT_HALO, br = frb[sidx] - TR + CPCT_HALO;  // 0..36
      const int cls = ((br * kRoundLd + ar) & 15);
      const uint64_t fm = 0x3Full << ar;
      size_t r = first_open;
      for (; r < rounds.size(); ++r) {
        R& rd = rounds[r];
        if (rd.count == 32) continue;
        if ((rd.lanes >> cls) & (rd.lanes >> (cls + 16)) & 1u) continue;
        bool clash = false;
        for (int q = 0; q < CPCT_W && !clash; ++q) clash = (rd.occ[br + q] & fm) != 0;
        if (!clash) break;
      }
      if (r == rounds.size()) {
        rounds.push_back(R{});
        std::memset(&rounds.back(), 0, sizeof(R));
        std::array<uint32_t, 32> empty;
        empty.fill(0xffffffffu);
        lanes_of.push_back(empty);
      }
      R& rd = rounds[r];
      const int lane = ((rd.lanes >> cls) & 1u) ? cls + 16 : cls;
      rd.lanes |= 1u << lane;
      rd.count++;
      for (int q = 0; q < CPCT_W; ++q) rd.occ[br + q] |= fm;
      lanes_of[r][lane] = id;
      while (first_open < rounds.size() && rounds[first_open].count == 32) ++first_open;
    }
    for (auto& l : lanes_of) out.ids.insert(out.ids.end(), l.begin(), l.end());
    out.tile_ptr[t + 1] = out.tile_ptr[t] + (int)rounds.size();
  }
}

// Order the samples of every forward bin so that within each group of 16
// consecutive samples (one half-warp) the first cells of their 6x6 windows
// fall in distinct 64-bit bank pairs of the staged 37 x 38 window: every tap
// load of the gather is then bank-conflict free.  Round-robin over the bank
// classes, each class in bin order (deterministic).
void order_fwd_bins(Bins& fwd, int K, const std::vector<int>& fa0, const std::vector<int>& frb, int win_ld) {
  const int nt = (int)fwd.ptr.size() - 1;
  std::vector<uint32_t> cls[16];
  for (int t = 0; t < nt; ++t) {
    const int C0 = (t % fwd.tiles_x) * CPCT_TILE, R0 = (t / fwd.tiles_x) * CPCT_TILE;
    for (auto& c : cls) c.clear();
    for (int e = fwd.ptr[t]; e < fwd.ptr[t + 1]; ++e) {
      const uint32_t id = fwd.ids[e];
      const size_t sidx = (size_t)(id >> 16) * (K + 1) + (id & 0xffffu);
      const int ar = fa0[sidx] - C0, br = frb[sidx] - R0;
      cls[(br * win_ld + ar) & 15].push_back(id);
    }
    size_t pos[16] = {0};
    int e = fwd.ptr[t];
    while (e < fwd.ptr[t + 1]) {
      for (int c = 0; c < 16; ++c)
        if (pos[c] < cls[c].size()) fwd.ids[e++] = cls[c][pos[c]++];
    }
  }
}

// split bins into work items of at most `cap` entries, longest first
void make_items(const Bins& b, int cap, bool slots, std::vector<int4>& items, std::vector<int4>& split,
                int* n_slots) {
  const int nt = (int)b.ptr.size() - 1;
  items.clear();
  split.clear();
  int slot = 0;
  for (int t = 0; t < nt; ++t) {
    const int beg = b.ptr[t], end = b.ptr[t + 1];
    if (end == beg) continue;
    const int pieces = (end - beg + cap - 1) / cap;
    if (pieces == 1 || !slots) {
      for (int q = 0; q < pieces; ++q)
        items.push_back(make_int4(t, beg + q * cap, std::min(end, beg + (q + 1) * cap), -1));
    } else {
      split.push_back(make_int4(t, slot, pieces, 0));
      for (int q = 0; q < pieces; ++q)
        items.push_back(make_int4(t, beg + q * cap, std::min(end, beg + (q + 1) * cap), slot + q));
      slot += pieces;
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const int4& a, const int4& c) { return (a.z - a.y) > (c.z - c.y); });
  if (n_slots) *n_slots = slot;
}

// work items over rounds: at most `cap` rounds per item, longest first; tiles
// split over several items accumulate into partial-tile slots
void make_round_items(const Rounds& rd, int cap, std::vector<int4>& items, std::vector<int4>& split, int* n_slots,
                      std::vector<int>& item_split) {
  const int nt = (int)rd.tile_ptr.size() - 1;
  items.clear();
  split.clear();
  int slot = 0;
  for (int t = 0; t < nt; ++t) {
    const int beg = rd.tile_ptr[t], end = rd.tile_ptr[t + 1];
    if (end == beg) continue;
    const int pieces = (end - beg + cap - 1) / cap;
    if (pieces == 1) {
      items.push_back(make_int4(t, beg, end, -1));
    } else {
      split.push_back(make_int4(t, slot, pieces, 0));
      for (int q = 0; q < pieces; ++q)
        items.push_back(make_int4(t, beg + q * cap, std::min(end, beg + (q + 1) * cap), slot + q));
      slot += pieces;
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const int4& a, const int4& c) { return (a.z - a.y) > (c.z - c.y); });
  *n_slots = slot;
  // split index of every item (slots of split k are contiguous from split[k].y)
  item_split.assign(items.size(), -1);
  for (size_t i = 0; i < items.size(); ++i) {
    if (items[i].w < 0) continue;
    int lo = 0, hi = (int)split.size() - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (split[mid].y <= items[i].w) lo = mid; else hi = mid - 1;
    }
    item_split[i] = lo;
  }
}

}  // namespace cpct_detail

// Round packing of the adjoint bins of a geometry (host only): number of
// rounds, number of packed samples, and 1 if every round is footprint- and
// bank-conflict free and every bin entry appears exactly once, else 0.
extern "C" int cpct_debug_rounds(const cpct_geom* g, int* n_rounds, int* n_packed, int* valid) {
  if (!geom_ok(g)) return CPCT_EINVAL;
  const int G = 2 * g->n, K = g->n_det / 2;
  std::vector<float4> ray;
  cpct_detail::make_rays(g->n, g->n_det, g->n_views, g->angles, (double)G / g->n_det, ray);
  cpct_detail::Bins f, a;
  std::vector<int> fa0, frb;
  cpct_detail::build_bins(g->n, g->n_det, g->n_views, G, ray, f, a, &fa0, &frb);
  cpct_detail::Rounds rd;
  cpct_detail::pack_rounds(a, G, fa0, frb, K, rd);
  const int nt = (int)a.ptr.size() - 1;
  int ok = 1, packed = 0;
  for (int t = 0; t < nt && ok; ++t) {
    const int TC = (t % a.tiles_x) * CPCT_TILE, TR = (t / a.tiles_x) * CPCT_TILE;
    std::vector<uint32_t> seen;
    for (int r = rd.tile_ptr[t]; r < rd.tile_ptr[t + 1] && ok; ++r) {
      std::vector<int> cells;
      for (int l = 0; l < 32; ++l) {
        const uint32_t id = rd.ids[(size_t)r * 32 + l];
        if (id == 0xffffffffu) continue;
        seen.push_back(id);
        const size_t sidx = (size_t)(id >> 16) * (K + 1) + (id & 0xffffu);
        const int ar = fa0[sidx] - TC + CPCT_HALO, br = frb[sidx] - TR + CPCT_HALO;
        if (ar < 0 || br < 0 || ar > CPCT_TILE + CPCT_HALO - 1 || br > CPCT_TILE + CPCT_HALO - 1) ok = 0;
        if (((br * cpct_detail::kRoundLd + ar) & 15) != (l & 15)) ok = 0;
        for (int q = 0; q < CPCT_W; ++q)
          for (int c = 0; c < CPCT_W; ++c) cells.push_back((br + q) * cpct_detail::kRoundLd + ar + c);
      }
      std::sort(cells.begin(), cells.end());
      if (std::adjacent_find(cells.begin(), cells.end()) != cells.end()) ok = 0;
    }
    std::vector<uint32_t> want(a.ids.begin() + a.ptr[t], a.ids.begin() + a.ptr[t + 1]);
    std::sort(seen.begin(), seen.end());
    std::sort(want.begin(), want.end());
    if (seen != want) ok = 0;
    packed += (int)seen.size();
  }
  if (n_rounds) *n_rounds = (int)(rd.ids.size() / 32);
  if (n_packed) *n_packed = packed;
  if (valid) *valid = ok;
  return CPCT_OK;
}

// which = 0: forward bins, 1: adjoint bins.  Reports the number of tiles, the
// number of entries and a checksum sum(id * (position + 1)) of the id list.
extern "C" int cpct_debug_bins(const cpct_geom* g, int which, int* n_tiles, int* n_entries, int64_t* checksum) {
  if (!geom_ok(g)) return CPCT_EINVAL;
  const int G = 2 * g->n;
  std::vector<float4> ray;
  cpct_detail::make_rays(g->n, g->n_det, g->n_views, g->angles, (double)G / g->n_det, ray);
  cpct_detail::Bins f, a;
  cpct_detail::build_bins(g->n, g->n_det, g->n_views, G, ray, f, a);
  const cpct_detail::Bins& b = which ? a : f;
  if (n_tiles) *n_tiles = (int)b.ptr.size() - 1;
  if (n_entries) *n_entries = (int)b.ids.size();
  if (checksum) {
    int64_t cs = 0;
    for (size_t i = 0; i < b.ids.size(); ++i) cs += (int64_t)b.ids[i] * (int64_t)(i % 1000003 + 1);
    *checksum = cs;
  }
  return CPCT_OK;
}

// Copy the bin list of tile `tile` (which = 0 forward, 1 adjoint) into ids
// (capacity cap); returns the number of entries or a negative status.
extern "C" int cpct_debug_bin_tile(const cpct_geom* g, int which, int tile, uint32_t* ids, int cap) {
  if (!geom_ok(g)) return CPCT_EINVAL;
  const int G = 2 * g->n;
  std::vector<float4> ray;
  cpct_detail::make_rays(g->n, g->n_det, g->n_views, g->angles, (double)G / g->n_det, ray);
  cpct_detail::Bins f, a;
  cpct_detail::build_bins(g->n, g->n_det, g->n_views, G, ray, f, a);
  const cpct_detail::Bins& b = which ? a : f;
  if (tile < 0 || tile >= (int)b.ptr.size() - 1) return CPCT_EINVAL;
  const int cnt = b.ptr[tile + 1] - b.ptr[tile];
  for (int i = 0; i < cnt && i < cap; ++i) ids[i] = b.ids[b.ptr[tile] + i];
  return cnt;
}

// Sample coordinate split exactly as the kernels do it (host mirror).
extern "C" int cpct_debug_split(float k, float hi, float lo, int* fl, float* z) {
  host_split(k, hi, lo, fl, z);
  return CPCT_OK;
}

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
    // bins
    cpct_detail::Bins fb, ab;
    std::vector<int> fa0, frb;
    cpct_detail::build_bins(n, ns, m, p->G, ray, fb, ab, &fa0, &frb);
    cpct_detail::Rounds rounds;
    cpct_detail::pack_rounds(ab, p->G, fa0, frb, p->K, rounds);
    cpct_detail::order_fwd_bins(fb, p->K, fa0, frb, CPCT_TILE + CPCT_HALO + 1);
    p->tiles_x_fwd = fb.tiles_x;
    p->tiles_y_fwd = fb.tiles_y;
    p->tiles_x_adj = ab.tiles_x;
    p->tiles_y_adj = ab.tiles_y;
    std::vector<int4> fitems, aitems, fsplit, asplit;
    cpct_detail::make_items(fb, kFwdItemMax, false, fitems, fsplit, nullptr);
    std::vector<int> item_split;
    p->fwd_cap = kFwdItemMax;
    p->adj_cap = kAdjItemRounds;
    cpct_detail::make_round_items(rounds, kAdjItemRounds, aitems, asplit, &p->n_slots, item_split);
    p->shared = new (std::nothrow) PlanShared;
    if (!p->shared) { rc = CPCT_ENOMEM; goto fail; }
    p->shared->fwd_tile_ptr = fb.ptr;
    p->shared->round_tile_ptr = rounds.tile_ptr;
    p->n_fwd_items = (int)fitems.size();
    p->n_adj_items = (int)aitems.size();
    p->n_split = (int)asplit.size();
    TRY(upload(al, &p->d_fwd_items, fitems, stream));
    TRY(upload(al, &p->d_fwd_ids, fb.ids, stream));
    TRY(upload(al, &p->d_adj_items, aitems, stream));
    TRY(upload(al, &p->d_adj_ids, rounds.ids, stream));
    TRY(upload(al, &p->d_split, asplit, stream));
    TRY(al((void**)&p->d_partials, sizeof(float2) * (size_t)std::max(1, p->n_slots) * CPCT_TILE * CPCT_TILE));
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
  p->d_Hx = p->d_Ax = p->d_H1 = p->d_Q = p->d_partials = nullptr;
  p->d_stage_img = p->d_stage_sino = nullptr;
  p->d_err = nullptr;
  p->prof = nullptr;
  p->launches = 0;
  p->device_bytes = 0;
  p->shared->refs++;
  Alloc al{p, false};
  int rc = CPCT_OK;
  const size_t hx_bytes = sizeof(float2) * (size_t)p->ext_rows * p->ldh;
  if ((rc = al((void**)&p->d_Hx, hx_bytes)) || (rc = al((void**)&p->d_Ax, hx_bytes)) ||
      (rc = al((void**)&p->d_H1, sizeof(float2) * (size_t)(p->n + 1) * p->n)) ||
      (rc = al((void**)&p->d_Q, sizeof(float2) * (size_t)p->m * p->ldq)) || (rc = al((void**)&p->d_err, sizeof(int))) ||
      (rc = al((void**)&p->d_partials, sizeof(float2) * (size_t)std::max(1, p->n_slots) * CPCT_TILE * CPCT_TILE))) {
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

namespace {

// install forward items built with `cap` samples per item
int install_fwd_items(cpct_plan* p, int cap, cudaStream_t s) {
  cpct_detail::Bins b;
  b.ptr = p->shared->fwd_tile_ptr;
  b.tiles_x = p->tiles_x_fwd;
  b.tiles_y = p->tiles_y_fwd;
  std::vector<int4> items, split;
  cpct_detail::make_items(b, cap, false, items, split, nullptr);
  int4* d = nullptr;
  if (cudaMalloc(&d, sizeof(int4) * std::max<size_t>(1, items.size())) != cudaSuccess) return CPCT_ENOMEM;
  if (cudaMemcpyAsync(d, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaFree(d);
    return CPCT_ECUDA;
  }
  cudaFree(p->d_fwd_items);
  p->d_fwd_items = d;
  p->n_fwd_items = (int)items.size();
  p->fwd_cap = cap;
  return CPCT_OK;
}

// install adjoint items (and split list, partial tiles) with `cap` rounds per item
int install_adj_items(cpct_plan* p, int cap, cudaStream_t s) {
  cpct_detail::Rounds r;
  r.tile_ptr = p->shared->round_tile_ptr;
  std::vector<int4> items, split;
  std::vector<int> item_split;
  int n_slots = 0;
  cpct_detail::make_round_items(r, cap, items, split, &n_slots, item_split);
  int4 *di = nullptr, *ds = nullptr;
  float2* dp = nullptr;
  if (cudaMalloc(&di, sizeof(int4) * std::max<size_t>(1, items.size())) != cudaSuccess ||
      cudaMalloc(&ds, sizeof(int4) * std::max<size_t>(1, split.size())) != cudaSuccess ||
      cudaMalloc(&dp, sizeof(float2) * (size_t)std::max(1, n_slots) * CPCT_TILE * CPCT_TILE) != cudaSuccess) {
    if (di) cudaFree(di);
    if (ds) cudaFree(ds);
    return CPCT_ENOMEM;
  }
  cudaMemcpyAsync(di, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s);
  if (!split.empty()) cudaMemcpyAsync(ds, split.data(), sizeof(int4) * split.size(), cudaMemcpyHostToDevice, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaFree(di);
    cudaFree(ds);
    cudaFree(dp);
    return CPCT_ECUDA;
  }
  cudaFree(p->d_adj_items);
  cudaFree(p->d_split);
  cudaFree(p->d_partials);
  p->d_adj_items = di;
  p->d_split = ds;
  p->d_partials = dp;
  p->n_adj_items = (int)items.size();
  p->n_split = (int)split.size();
  p->n_slots = n_slots;
  p->adj_cap = cap;
  return CPCT_OK;
}

}  // namespace

// Autotuner of the work-item caps (how many samples a forward gather item and
// how many rounds an adjoint spread item may hold): every candidate is timed
// (median of `reps` launches, CUDA events on `stream`) and the fastest kept.
extern "C" int cpct_plan_tune(cpct_plan* p, int reps, int* fwd_cap, int* adj_cap, cudaStream_t stream) {
  if (!p || !p->shared) return CPCT_EINVAL;
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
  int rc = CPCT_OK;
  const int fcands[] = {256, 512, 1024, 2048, 4096};
  const int acands[] = {16, 32, 64, 128, 256};
  int best_f = p->fwd_cap, best_a = p->adj_cap;
  float tf = 1e30f, ta = 1e30f;
  for (int c : fcands) {
    if ((rc = install_fwd_items(p, c, stream)) != CPCT_OK) break;
    const float t = time_op(true);
    if (t < tf) { tf = t; best_f = c; }
  }
  if (rc == CPCT_OK) rc = install_fwd_items(p, best_f, stream);
  for (int c : acands) {
    if (rc != CPCT_OK) break;
    if ((rc = install_adj_items(p, c, stream)) != CPCT_OK) break;
    const float t = time_op(false);
    if (t < ta) { ta = t; best_a = c; }
  }
  if (rc == CPCT_OK) rc = install_adj_items(p, best_a, stream);
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
  if (p->shared->refs != 1) return CPCT_EINVAL;
  int rc = CPCT_OK;
  if (fwd_cap > 0) rc = install_fwd_items(p, fwd_cap, stream);
  if (rc == CPCT_OK && adj_cap > 0) rc = install_adj_items(p, adj_cap, stream);
  return rc;
}

// Work-item counts of a plan: forward gather items, adjoint spread items,
// split heavy tiles and their partial tiles (slots).
extern "C" int cpct_plan_work(const cpct_plan* p, int* n_fwd_items, int* n_adj_items, int* n_split, int* n_slots) {
  if (!p) return CPCT_EINVAL;
  if (n_fwd_items) *n_fwd_items = p->n_fwd_items;
  if (n_adj_items) *n_adj_items = p->n_adj_items;
  if (n_split) *n_split = p->n_split;
  if (n_slots) *n_slots = p->n_slots;
  return CPCT_OK;
}

// The adjoint work items a plan of geometry g would get with `cap` rounds per
// item (0: the default cap), built on the host exactly as cpct_plan_create
// and cpct_plan_set_caps build them.  No GPU needed.
extern "C" int cpct_debug_adj_items(const cpct_geom* g, int cap, int* n_items, int* n_split, int* n_slots) {
  if (!geom_ok(g) || cap < 0) return CPCT_EINVAL;
  const int G = 2 * g->n, K = g->n_det / 2;
  std::vector<float4> ray;
  cpct_detail::make_rays(g->n, g->n_det, g->n_views, g->angles, (double)G / g->n_det, ray);
  cpct_detail::Bins f, a;
  std::vector<int> fa0, frb;
  cpct_detail::build_bins(g->n, g->n_det, g->n_views, G, ray, f, a, &fa0, &frb);
  cpct_detail::Rounds rd;
  cpct_detail::pack_rounds(a, G, fa0, frb, K, rd);
  std::vector<int4> items, split;
  std::vector<int> item_split;
  int slots = 0;
  cpct_detail::make_round_items(rd, cap > 0 ? cap : kAdjItemRounds, items, split, &slots, item_split);
  if (n_items) *n_items = (int)items.size();
  if (n_split) *n_split = (int)split.size();
  if (n_slots) *n_slots = slots;
  return CPCT_OK;
}
