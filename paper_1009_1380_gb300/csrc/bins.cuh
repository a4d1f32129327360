// Bin plans of the gridding kernels (host side; no device code).
//
// Section "fast radon transform": the sample plane is divided into bins
// with one thread block per bin; the paper chooses them with a quadtree that
// starts from one bin holding every sample and repeatedly divides the most
// computationally intensive bin into four equal bins, the intensity being
// the number of samples times the number of grid points of the bin.
//
// Here a bin is a square of T x T grid points (T = 16, 32 or 64, aligned to
// T) of the extended half spectrum.  A bin plan is either a uniform tiling
// with one T, or the paper's quadtree (leaves of 16..64 points).  The
// forward gather puts every polar sample in the bin holding the first grid
// point of its 6x6 footprint; the adjoint spread puts it in every bin its
// footprint touches, packed into conflict-free rounds.  Bins whose lists are
// longer than a cap are split into several work items (the adjoint's write
// partial tiles, summed afterwards in a fixed order).
#pragma once

#include <cstdint>
#include <vector>

#include "common.cuh"

namespace cpct_detail {

constexpr int kNumTileClasses = 3;  // T = 16, 32, 64
inline int tile_class(int T) { return T <= 16 ? 0 : T <= 32 ? 1 : 2; }
inline int class_tile(int c) { return 16 << c; }
inline int pack_xy(int x0, int y0) { return (y0 << 16) | x0; }

enum BinKind { BIN_UNIFORM = 0, BIN_QUADTREE = 1 };

// host mirror of the kernels' split of u = k (hi + lo) into floor and
// fraction (identical IEEE single-precision operations)
void host_split(float k, float hi, float lo, int* fl_out, float* z);

// first grid point of every polar sample's 6x6 footprint: column
// a0 = floor(u) - 2 mod G and buffer row rb0 = floor(v) of the extended
// spectrum, for sample (j, k), k = 0..K, at index j (K + 1) + k
struct Samples {
  int m = 0, K = 0;
  std::vector<int> a0, rb0;
  std::vector<float> zu, zv;  // fractions of u and v (the kernels' split)
};

void make_rays(int n, int ns, int m, const double* angles, double scale, std::vector<float4>& ray);
void make_samples(int ns, int m, int G, const std::vector<float4>& ray, Samples& s);

struct BinLayout {
  int kind = BIN_UNIFORM;
  int tile = 32;             // uniform tile size (0 for a quadtree)
  std::vector<int4> bins;    // (x0, y0, T, 0)
};

// uniform tiling of the domain [0, W) x [0, H) with T x T bins
void uniform_layout(int T, int W, int H, BinLayout& L);
// the paper's quadtree over [0, W) x [0, H): split the bin of largest
// samples x points (first points counted) into four while that cost exceeds
// alpha times the mean cost of the non-empty leaves and the bin is larger
// than 16; leaves larger than 64 are then tiled with 64 x 64 bins
void quadtree_layout(const Samples& s, int W, int H, double alpha, BinLayout& L);

struct BinLists {
  std::vector<int> ptr;        // bins + 1
  std::vector<uint32_t> ids;   // sample ids (j << 16 | k), grouped by bin, increasing inside a bin
};
void assign_fwd(const Samples& s, int W, int H, const BinLayout& L, BinLists& out);
void assign_adj(const Samples& s, int W, int H, const BinLayout& L, BinLists& out);

// forward: order every bin's samples so that within each group of 16 the
// first cells fall in distinct 64-bit bank pairs of the staged window
void order_fwd(const Samples& s, const BinLayout& L, BinLists& b);

// adjoint: rounds of samples with pairwise disjoint footprints in the bin's
// (T + 10) x (T + 13) accumulator; the 64-bit bank pair of a sample's first
// cell is its class (the odd pitch shifts the classes of consecutive rows by
// 13).  A round of `lanes` samples holds at most lanes / 16 per class, in
// lanes c, c + 16, ...: every half-warp's 64-bit access is then served in
// one pass.  16-lane rounds use the lower half-warp only, 32-lane rounds one
// warp, 64-lane rounds two warps (the larger tiles have room for 64
// disjoint footprints).
struct Rounds {
  int lanes = 32;               // samples per round (16, 32 or 64), or kGroupLanes
  std::vector<int> ptr;         // bins + 1, in rounds
  std::vector<uint32_t> ids;    // round_words(lanes) per round, 0xffffffff = empty lane
};
inline int round_pitch(int T) { return T + 2 * CPCT_HALO + 3; }
void pack_rounds(const Samples& s, const BinLayout& L, const BinLists& adj, int lanes, Rounds& out);

// Column groups (round width kGroupLanes): five samples per warp, lane
// 6 s + c applies column c of sample s's footprint, rows 0..5 in turn, so a
// sample's 36 taps take six accesses of six lanes.  A half-warp then holds
// the columns of up to three samples; its accesses are conflict free when
// the first cells' bank classes of slots 0..4 are b, b + 6, b + 12, b + 2,
// b + 8 (mod 16) for the group's base class b (half-warp 0: slot 0 columns
// on classes b..b+5, slot 1 on b+6..b+11, slot 2's first four on
// b+12..b+15; half-warp 1: slot 2's last two on b, b+1, slot 3 on
// b+2..b+7, slot 4 on b+8..b+13).  The footprints of a group are pairwise
// disjoint.  Each entry carries what the kernel would otherwise recompute
// per lane: (id, zu bits, zv bits, ar | br << 16), accumulator coordinates
// relative to the bin's halo origin; an empty slot has id 0xffffffff.
constexpr int kGroupLanes = 5;      // the round-width value of column groups
constexpr int kGroupSlots = 5;
constexpr int kGroupWords = 4 * kGroupSlots;  // uint32 words per group
constexpr int kGroupPattern[kGroupSlots] = {0, 6, 12, 2, 8};
void pack_groups(const Samples& s, const BinLayout& L, const BinLists& adj, Rounds& out);
// uint32 words per round of a width (rounds: one id per lane)
inline int round_words(int lanes) { return lanes == kGroupLanes ? kGroupWords : lanes; }

// work items, grouped by tile class and longest first within a class
struct Items {
  std::vector<int4> items;   // forward (xy, begin, end, 0); adjoint (xy, begin, end, partial offset or -1)
  int cls[kNumTileClasses + 1] = {0, 0, 0, 0};
  std::vector<int4> split;   // adjoint: (xy, partial offset, pieces, T), grouped by class
  int split_cls[kNumTileClasses + 1] = {0, 0, 0, 0};
  long long partial_elems = 0;  // complex values of all partial tiles
};
void fwd_items(const BinLayout& L, const std::vector<int>& ptr, int cap, Items& out);
void adj_items(const BinLayout& L, const std::vector<int>& rptr, int cap, Items& out);

}  // namespace cpct_detail
