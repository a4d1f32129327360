// Bin plans of the gridding kernels: uniform tilings and the paper's
// cost-driven quadtree, sample lists, conflict-free rounds and work items
// (host code; see bins.cuh).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <queue>

#include "bins.cuh"

namespace cpct_detail {

// host mirror of the kernels' split of u = k (hi + lo) into floor and
// fraction (identical IEEE single-precision operations)
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

void make_rays(int n, int ns, int m, const double* angles, double scale, std::vector<float4>& ray) {
  (void)n;
  (void)ns;
  ray.resize(m);
  for (int j = 0; j < m; ++j) {
    const double th = angles ? angles[j] : M_PI * (double)j / (double)m;
    const double c = scale * std::cos(th), s = scale * std::sin(th);
    const float ch = (float)c, sh = (float)s;
    ray[j] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
  }
}

void make_samples(int ns, int m, int G, const std::vector<float4>& ray, Samples& s) {
  const int K = ns / 2;
  s.m = m;
  s.K = K;
  s.a0.resize((size_t)m * (K + 1));
  s.rb0.resize((size_t)m * (K + 1));
  s.zu.resize((size_t)m * (K + 1));
  s.zv.resize((size_t)m * (K + 1));
  for (int j = 0; j < m; ++j)
    for (int k = 0; k <= K; ++k) {
      int fu, fv;
      float zu, zv;
      host_split((float)k, ray[j].x, ray[j].y, &fu, &zu);
      host_split((float)k, ray[j].z, ray[j].w, &fv, &zv);
      const size_t i = (size_t)j * (K + 1) + k;
      s.a0[i] = (fu - 2) & (G - 1);
      s.rb0[i] = fv;  // buffer row of the first tap: (floor(v) - 2) + 2
      s.zu[i] = zu;
      s.zv[i] = zv;
    }
}

void uniform_layout(int T, int W, int H, BinLayout& L) {
  L.kind = BIN_UNIFORM;
  L.tile = T;
  L.bins.clear();
  const int tx = (W + T - 1) / T, ty = (H + T - 1) / T;
  for (int y = 0; y < ty; ++y)
    for (int x = 0; x < tx; ++x) L.bins.push_back(make_int4(x * T, y * T, T, 0));
}

namespace {

// counts of first points per 16 x 16 cell, with 2D prefix sums
struct CellCounts {
  int cw = 0, ch = 0;
  std::vector<long long> pre;  // (ch + 1) x (cw + 1)
  long long sum(int cx0, int cy0, int cx1, int cy1) const {  // cells [cx0, cx1) x [cy0, cy1)
    cx0 = std::max(0, std::min(cx0, cw));
    cx1 = std::max(0, std::min(cx1, cw));
    cy0 = std::max(0, std::min(cy0, ch));
    cy1 = std::max(0, std::min(cy1, ch));
    if (cx1 <= cx0 || cy1 <= cy0) return 0;
    const int w = cw + 1;
    return pre[(size_t)cy1 * w + cx1] - pre[(size_t)cy0 * w + cx1] - pre[(size_t)cy1 * w + cx0] +
           pre[(size_t)cy0 * w + cx0];
  }
};

CellCounts count_cells(const Samples& s, int W, int H) {
  CellCounts c;
  c.cw = (W + 15) / 16;
  c.ch = (H + 15) / 16;
  std::vector<long long> cnt((size_t)c.cw * c.ch, 0);
  for (size_t i = 0; i < s.a0.size(); ++i) {
    const int cx = s.a0[i] / 16, cy = s.rb0[i] / 16;
    if (cx >= 0 && cx < c.cw && cy >= 0 && cy < c.ch) cnt[(size_t)cy * c.cw + cx]++;
  }
  const int w = c.cw + 1;
  c.pre.assign((size_t)(c.ch + 1) * w, 0);
  for (int y = 0; y < c.ch; ++y)
    for (int x = 0; x < c.cw; ++x)
      c.pre[(size_t)(y + 1) * w + x + 1] = cnt[(size_t)y * c.cw + x] + c.pre[(size_t)y * w + x + 1] +
                                           c.pre[(size_t)(y + 1) * w + x] - c.pre[(size_t)y * w + x];
  return c;
}

}  // namespace

void quadtree_layout(const Samples& s, int W, int H, double alpha, BinLayout& L) {
  L.kind = BIN_QUADTREE;
  L.tile = 0;
  L.bins.clear();
  const CellCounts cc = count_cells(s, W, H);
  int P = 16;
  while (P < W || P < H) P <<= 1;
  struct Bin {
    int x0, y0, T;
    double cost;
    long long samples;
  };
  auto make = [&](int x0, int y0, int T) {
    const long long sm = cc.sum(x0 / 16, y0 / 16, (x0 + T) / 16, (y0 + T) / 16);
    const long long pts = (long long)std::max(0, std::min(W, x0 + T) - x0) * std::max(0, std::min(H, y0 + T) - y0);
    return Bin{x0, y0, T, (double)sm * (double)pts, sm};
  };
  auto cmp = [](const Bin& a, const Bin& b) {
    if (a.cost != b.cost) return a.cost < b.cost;
    if (a.y0 != b.y0) return a.y0 > b.y0;
    return a.x0 > b.x0;
  };
  std::priority_queue<Bin, std::vector<Bin>, decltype(cmp)> q(cmp);
  std::vector<Bin> done;
  q.push(make(0, 0, P));
  double cost_sum = q.top().cost;
  long long nonempty = q.top().samples > 0 ? 1 : 0;
  // the most intensive bin is divided into four while it is larger than the
  // kernels' largest bin (64), or its cost exceeds alpha times the mean cost
  // of the non-empty leaves and it is larger than 16
  while (!q.empty()) {
    const Bin b = q.top();
    const double mean = nonempty > 0 ? cost_sum / (double)nonempty : 0.0;
    if (b.T <= 64 && (b.T <= 16 || b.cost <= alpha * mean)) break;
    q.pop();
    cost_sum -= b.cost;
    if (b.samples > 0) nonempty--;
    const int h = b.T / 2;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int x0 = b.x0 + dx * h, y0 = b.y0 + dy * h;
        if (x0 >= W || y0 >= H) continue;
        const Bin c = make(x0, y0, h);
        cost_sum += c.cost;
        if (c.samples > 0) nonempty++;
        q.push(c);
      }
  }
  while (!q.empty()) {
    done.push_back(q.top());
    q.pop();
  }
  // leaves above the kernels' largest bin are tiled with 64 x 64 bins
  for (const Bin& b : done) {
    if (b.T <= 64) {
      L.bins.push_back(make_int4(b.x0, b.y0, b.T, 0));
      continue;
    }
    for (int y = b.y0; y < b.y0 + b.T && y < H; y += 64)
      for (int x = b.x0; x < b.x0 + b.T && x < W; x += 64) L.bins.push_back(make_int4(x, y, 64, 0));
  }
  // deterministic order: row-major by origin
  std::sort(L.bins.begin(), L.bins.end(), [](const int4& a, const int4& b) {
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
}

namespace {

// bin index of every 16 x 16 cell of the domain (every bin is a union of
// whole cells, aligned to its size)
struct CellMap {
  int cw = 0, ch = 0;
  std::vector<int> bin;
  int at(int x, int y) const {
    const int cx = x / 16, cy = y / 16;
    if (x < 0 || y < 0 || cx >= cw || cy >= ch) return -1;
    return bin[(size_t)cy * cw + cx];
  }
};

CellMap map_cells(const BinLayout& L, int W, int H) {
  CellMap m;
  int maxx = W, maxy = H;
  for (const int4& b : L.bins) {
    maxx = std::max(maxx, b.x + b.z);
    maxy = std::max(maxy, b.y + b.z);
  }
  m.cw = (maxx + 15) / 16;
  m.ch = (maxy + 15) / 16;
  m.bin.assign((size_t)m.cw * m.ch, -1);
  for (size_t i = 0; i < L.bins.size(); ++i) {
    const int4 b = L.bins[i];
    for (int cy = b.y / 16; cy < (b.y + b.z) / 16; ++cy)
      for (int cx = b.x / 16; cx < (b.x + b.z) / 16; ++cx) m.bin[(size_t)cy * m.cw + cx] = (int)i;
  }
  return m;
}

template <class F>
void fill_lists(const Samples& s, size_t nbins, F&& bins_of, BinLists& out) {
  std::vector<int> cnt(nbins + 1, 0);
  int tmp[4];
  for (int j = 0; j < s.m; ++j)
    for (int k = 0; k <= s.K; ++k) {
      const int nb = bins_of((size_t)j * (s.K + 1) + k, tmp);
      for (int q = 0; q < nb; ++q) cnt[tmp[q] + 1]++;
    }
  for (size_t i = 0; i < nbins; ++i) cnt[i + 1] += cnt[i];
  out.ptr = cnt;
  out.ids.resize(cnt[nbins]);
  std::vector<int> pos(cnt.begin(), cnt.end() - 1);
  for (int j = 0; j < s.m; ++j)
    for (int k = 0; k <= s.K; ++k) {
      const int nb = bins_of((size_t)j * (s.K + 1) + k, tmp);
      const uint32_t id = ((uint32_t)j << 16) | (uint32_t)k;
      for (int q = 0; q < nb; ++q) out.ids[pos[tmp[q]]++] = id;
    }
}

}  // namespace

void assign_fwd(const Samples& s, int W, int H, const BinLayout& L, BinLists& out) {
  const CellMap cm = map_cells(L, W, H);
  fill_lists(s, L.bins.size(),
             [&](size_t i, int* b) {
               b[0] = cm.at(s.a0[i], s.rb0[i]);
               return b[0] >= 0 ? 1 : 0;
             },
             out);
}

void assign_adj(const Samples& s, int W, int H, const BinLayout& L, BinLists& out) {
  const CellMap cm = map_cells(L, W, H);
  fill_lists(s, L.bins.size(),
             [&](size_t i, int* b) {
               int nb = 0;
               const int a0 = s.a0[i], r0 = s.rb0[i];
               const int xs[2] = {a0, a0 + CPCT_HALO}, ys[2] = {r0, r0 + CPCT_HALO};
               for (int yi = 0; yi < 2; ++yi)
                 for (int xi = 0; xi < 2; ++xi) {
                   const int bi = cm.at(xs[xi], ys[yi]);
                   if (bi < 0) continue;
                   bool seen = false;
                   for (int q = 0; q < nb; ++q) seen = seen || b[q] == bi;
                   if (!seen) b[nb++] = bi;
                 }
               // bins touched, in increasing bin order
               std::sort(b, b + nb);
               return nb;
             },
             out);
}

void order_fwd(const Samples& s, const BinLayout& L, BinLists& b) {
  std::vector<uint32_t> cls[16];
  for (size_t t = 0; t + 1 < b.ptr.size(); ++t) {
    const int4 bn = L.bins[t];
    const int ld = bn.z + CPCT_HALO + 1;  // window row pitch (complex)
    for (auto& c : cls) c.clear();
    for (int e = b.ptr[t]; e < b.ptr[t + 1]; ++e) {
      const uint32_t id = b.ids[e];
      const size_t i = (size_t)(id >> 16) * (s.K + 1) + (id & 0xffffu);
      const int ar = s.a0[i] - bn.x, br = s.rb0[i] - bn.y;
      cls[(br * ld + ar) & 15].push_back(id);
    }
    size_t pos[16] = {0};
    int e = b.ptr[t];
    while (e < b.ptr[t + 1])
      for (int c = 0; c < 16; ++c)
        if (pos[c] < cls[c].size()) b.ids[e++] = cls[c][pos[c]++];
  }
}

void pack_rounds(const Samples& s, const BinLayout& L, const BinLists& adj, int lanes, Rounds& out) {
  const int nt = (int)adj.ptr.size() - 1;
  out.lanes = lanes;
  out.ptr.assign(nt + 1, 0);
  out.ids.clear();
  constexpr int kMaxRows = 64 + 2 * CPCT_HALO;
  struct R {
    uint64_t occ[kMaxRows][2];  // accumulator columns 0..127 per row
    uint64_t lanes;             // occupied lanes
    int count;
  };
  const int per_class = lanes / 16;  // lanes c, c + 16, ... of bank class c
  std::vector<R> rounds;
  std::vector<std::array<uint32_t, 64>> lanes_of;
  for (int t = 0; t < nt; ++t) {
    const int4 bn = L.bins[t];
    const int T = bn.z, ld = round_pitch(T);
    const int TC = bn.x, TR = bn.y;
    rounds.clear();
    lanes_of.clear();
    size_t first_open = 0;
    for (int e = adj.ptr[t]; e < adj.ptr[t + 1]; ++e) {
      const uint32_t id = adj.ids[e];
      const size_t i = (size_t)(id >> 16) * (s.K + 1) + (id & 0xffffu);
      const int ar = s.a0[i] - TC + CPCT_HALO, br = s.rb0[i] - TR + CPCT_HALO;  // 0 .. T + 4
      const int cls = ((br * ld + ar) & 15);
      // footprint columns ar .. ar + 5 as two 64-bit masks
      uint64_t fm[2] = {0ull, 0ull};
      for (int c = 0; c < CPCT_W; ++c) fm[(ar + c) >> 6] |= 1ull << ((ar + c) & 63);
      size_t r = first_open;
      for (; r < rounds.size(); ++r) {
        R& rd = rounds[r];
        if (rd.count == lanes) continue;
        int used = 0;
        for (int h = 0; h < per_class; ++h) used += (int)((rd.lanes >> (cls + 16 * h)) & 1ull);
        if (used == per_class) continue;
        bool clash = false;
        for (int q = 0; q < CPCT_W && !clash; ++q)
          clash = ((rd.occ[br + q][0] & fm[0]) | (rd.occ[br + q][1] & fm[1])) != 0;
        if (!clash) break;
      }
      if (r == rounds.size()) {
        rounds.emplace_back();
        std::memset(&rounds.back(), 0, sizeof(R));
        std::array<uint32_t, 64> empty;
        empty.fill(0xffffffffu);
        lanes_of.push_back(empty);
      }
      R& rd = rounds[r];
      int lane = cls;
      while ((rd.lanes >> lane) & 1ull) lane += 16;
      rd.lanes |= 1ull << lane;
      rd.count++;
      for (int q = 0; q < CPCT_W; ++q) {
        rd.occ[br + q][0] |= fm[0];
        rd.occ[br + q][1] |= fm[1];
      }
      lanes_of[r][lane] = id;
      while (first_open < rounds.size() && rounds[first_open].count == lanes) ++first_open;
    }
    for (auto& l : lanes_of) out.ids.insert(out.ids.end(), l.begin(), l.begin() + lanes);
    out.ptr[t + 1] = out.ptr[t] + (int)rounds.size();
  }
}

void pack_groups(const Samples& s, const BinLayout& L, const BinLists& adj, Rounds& out) {
  const int nt = (int)adj.ptr.size() - 1;
  out.lanes = kGroupLanes;
  out.ptr.assign(nt + 1, 0);
  out.ids.clear();
  struct Gp {
    int base;                          // bank class of slot 0
    int used;                          // occupied slots (bits)
    int ar[kGroupSlots], br[kGroupSlots];
    uint32_t w[kGroupWords];
  };
  std::vector<Gp> groups;
  for (int t = 0; t < nt; ++t) {
    const int4 bn = L.bins[t];
    const int ld = round_pitch(bn.z);
    groups.clear();
    size_t first_open = 0;
    for (int e = adj.ptr[t]; e < adj.ptr[t + 1]; ++e) {
      const uint32_t id = adj.ids[e];
      const size_t i = (size_t)(id >> 16) * (s.K + 1) + (id & 0xffffu);
      const int ar = s.a0[i] - bn.x + CPCT_HALO, br = s.rb0[i] - bn.y + CPCT_HALO;  // 0 .. T + 4
      const int cls = (br * ld + ar) & 15;
      size_t g = first_open;
      int slot = -1;
      for (; g < groups.size() && slot < 0; ++g) {
        const Gp& gp = groups[g];
        if (gp.used == (1 << kGroupSlots) - 1) continue;
        for (int j = 1; j < kGroupSlots && slot < 0; ++j) {
          if (((gp.used >> j) & 1) || ((gp.base + kGroupPattern[j]) & 15) != cls) continue;
          bool clash = false;
          for (int q = 0; q < kGroupSlots && !clash; ++q)
            clash = ((gp.used >> q) & 1) && std::abs(gp.ar[q] - ar) < CPCT_W && std::abs(gp.br[q] - br) < CPCT_W;
          if (!clash) slot = j;
        }
        if (slot >= 0) break;
      }
      if (slot < 0) {  // a new group with this sample in slot 0
        Gp gp;
        gp.base = cls;
        gp.used = 0;
        for (int q = 0; q < kGroupWords; ++q) gp.w[q] = 0xffffffffu;
        groups.push_back(gp);
        g = groups.size() - 1;
        slot = 0;
      }
      Gp& gp = groups[g];
      gp.used |= 1 << slot;
      gp.ar[slot] = ar;
      gp.br[slot] = br;
      uint32_t zu, zv;
      std::memcpy(&zu, &s.zu[i], 4);
      std::memcpy(&zv, &s.zv[i], 4);
      gp.w[4 * slot + 0] = id;
      gp.w[4 * slot + 1] = zu;
      gp.w[4 * slot + 2] = zv;
      gp.w[4 * slot + 3] = (uint32_t)ar | ((uint32_t)br << 16);
      while (first_open < groups.size() && groups[first_open].used == (1 << kGroupSlots) - 1) ++first_open;
    }
    for (const Gp& gp : groups) out.ids.insert(out.ids.end(), gp.w, gp.w + kGroupWords);
    out.ptr[t + 1] = out.ptr[t] + (int)groups.size();
  }
}

namespace {

void group_by_class(std::vector<int4>& v, int* cls, const std::vector<int>& tile_of, bool by_len) {
  // stable: class first, then (optionally) longest first
  std::vector<size_t> idx(v.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    const int ca = tile_class(tile_of[a]), cb = tile_class(tile_of[b]);
    if (ca != cb) return ca < cb;
    return by_len && (v[a].z - v[a].y) > (v[b].z - v[b].y);
  });
  std::vector<int4> out(v.size());
  for (int c = 0; c <= kNumTileClasses; ++c) cls[c] = 0;
  for (size_t i = 0; i < idx.size(); ++i) {
    out[i] = v[idx[i]];
    cls[tile_class(tile_of[idx[i]]) + 1]++;
  }
  for (int c = 0; c < kNumTileClasses; ++c) cls[c + 1] += cls[c];
  v.swap(out);
}

}  // namespace

void fwd_items(const BinLayout& L, const std::vector<int>& ptr, int cap, Items& out) {
  out.items.clear();
  out.split.clear();
  out.partial_elems = 0;
  std::vector<int> tile_of;
  for (size_t t = 0; t + 1 < ptr.size(); ++t) {
    const int beg = ptr[t], end = ptr[t + 1];
    if (end == beg) continue;
    const int4 bn = L.bins[t];
    for (int q = beg; q < end; q += cap) {
      out.items.push_back(make_int4(pack_xy(bn.x, bn.y), q, std::min(end, q + cap), 0));
      tile_of.push_back(bn.z);
    }
  }
  group_by_class(out.items, out.cls, tile_of, true);
  for (int c = 0; c <= kNumTileClasses; ++c) out.split_cls[c] = 0;
}

void adj_items(const BinLayout& L, const std::vector<int>& rptr, int cap, Items& out) {
  out.items.clear();
  out.split.clear();
  std::vector<int> tile_of, split_tile;
  long long off = 0;
  for (size_t t = 0; t + 1 < rptr.size(); ++t) {
    const int beg = rptr[t], end = rptr[t + 1];
    if (end == beg) continue;
    const int4 bn = L.bins[t];
    const int xy = pack_xy(bn.x, bn.y);
    const int pieces = (end - beg + cap - 1) / cap;
    if (pieces == 1) {
      out.items.push_back(make_int4(xy, beg, end, -1));
      tile_of.push_back(bn.z);
      continue;
    }
    const long long tile_elems = (long long)bn.z * bn.z;
    out.split.push_back(make_int4(xy, (int)off, pieces, bn.z));
    split_tile.push_back(bn.z);
    for (int q = 0; q < pieces; ++q) {
      out.items.push_back(make_int4(xy, beg + q * cap, std::min(end, beg + (q + 1) * cap), (int)(off + q * tile_elems)));
      tile_of.push_back(bn.z);
    }
    off += pieces * tile_elems;
  }
  out.partial_elems = off;
  group_by_class(out.items, out.cls, tile_of, true);
  group_by_class(out.split, out.split_cls, split_tile, false);
}

}  // namespace cpct_detail
