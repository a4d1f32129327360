// Fourier-slice Radon transform by gridding, and its exact adjoint
// (section "fast radon transform").
//
// Forward  y = Re(A x)   (real image x -> real sinogram y):
//   1. k_fwd_col   deapodize x[p,q] c(Y) c(X), place at (Y mod G), G-point FFT
//                  of two real columns packed into one complex FFT, keep the
//                  non-negative frequency rows b = 0..N        -> H1 (N+1) x N
//   2. k_fwd_row   G-point FFT along x of every row b = 0..N, write the
//                  extended half spectrum (Hermitian mirror rows, wrapped
//                  columns)                                     -> Hx
//   3. k_fwd_interp  polar samples k = 0..Ns/2 of every ray: 6x6 Kaiser-Bessel
//                  interpolation; the 37x38 grid window of each 32x32 bin is
//                  staged in shared memory by one TMA tensor copy -> Q
//   4. k_fwd_ray   Hermitian completion + (-1)^k centring, Ns-point inverse
//                  FFT of two rays packed into one complex FFT, 1/Ns -> y
// Adjoint  x = Re(A^H w) is the transpose of these four real-linear maps,
// applied in reverse order:
//   5. k_adj_ray   Ns-point FFT of two packed sinogram rows, weights
//                  (1, 2, ..., 2, 1) (-1)^k / Ns               -> Q~
//   6. k_adj_spread  gridding as a deterministic gather: each 32x32 tile of
//                  the extended spectrum owns its output; its samples were
//                  packed at plan time into rounds of <= 32 samples with
//                  disjoint footprints; one warp applies the rounds in order,
//                  one sample per lane, into a shared-memory tile; no atomics
//   7. k_adj_reduce  the few heavy tiles (near the origin, where all rays
//                  meet) are split into several work items writing partial
//                  tiles, summed here in a fixed order           -> Ax
//   8. k_adj_row   fold the extension (mirror rows, wrapped columns), G-point
//                  inverse FFT along x, keep X = -N/2..N/2-1    -> H1
//   9. k_adj_col   Hermitian-symmetrise the rows b = 0..N of two columns,
//                  pack, G-point inverse FFT, crop Y, deapodize  -> x
#include <algorithm>
#include <mutex>

#include "bins.cuh"
#include "common.cuh"
#include "fft.cuh"

using cpct::fpad;
using cpct::SmemFFT;

namespace {

constexpr int kEcol = 32;              // FFT values per thread, column kernels
constexpr int kErow = 16;              // FFT values per thread, row and ray kernels
constexpr int kColFFTs = 4;            // packed column FFTs per CTA (2 kColFFTs image columns)
constexpr int kThreads = 256;          // threads of the row / ray FFT kernels
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

template <int LOG>
constexpr int fft_threads() { return (1 << LOG) / kErow; }
template <int LOG>
constexpr int rows_per_cta() { return kThreads / fft_threads<LOG>() > 0 ? kThreads / fft_threads<LOG>() : 1; }
template <int LOG>
constexpr size_t fft_smem(int nfft) { return (size_t)nfft * SmemFFT<LOG, kErow, -1>::PADN * sizeof(float2); }

// ---------------------------------------------------------------------------
// 1. forward column transform
// ---------------------------------------------------------------------------
// Persistent: each CTA takes blocks of 2 kColFFTs image columns in turn (FFT f packs
// the deapodized columns q0+2f (real part) and q0+2f+1 (imaginary part)).  A
// block arrives in shared memory by 2-D TMA tile copies (all its columns x min(N,
// 256) rows each); the copy of the CTA's next block is issued as soon as the
// first FFT pass has read the current one, so it lands while the other
// passes, the unpack and the stores run.  The deapodization vector is staged
// once per CTA.  Every wait is bounded: on a timeout the CTA records
// CPCT_ERR_TIMEOUT, lets its copy in flight land and returns.
template <int LOGG>
struct FwdColSmem {
  static constexpr int G = 1 << LOGG, N = G / 2;
  static constexpr int BR = N < 256 ? N : 256;  // rows per TMA box
  static constexpr int FFTS = kColFFTs * SmemFFT<LOGG, kEcol, -1, true, false>::PADN;  // complex values
  static constexpr int CW = 2 * kColFFTs;        // image columns per block
  static constexpr size_t bytes = (size_t)N * CW * sizeof(float)  // the block: N rows x CW columns
                                  + (size_t)FFTS * sizeof(float2) + (size_t)N * sizeof(float) + 128;
};

template <int LOGG>
__global__ void __launch_bounds__(kColFFTs*(1 << LOGG) / kEcol, LOGG >= 12 ? 1 : 2)
    k_fwd_col(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ dp, float2* __restrict__ H1,
              const float2* __restrict__ tw, int* __restrict__ err, const int* __restrict__ skip) {
  if (skip && *skip) return;
  // the padding half [N/2, G - N/2) is zero: the FFT skips it (PIN)
  using FFT = SmemFFT<LOGG, kEcol, -1, true, false>;
  using S = FwdColSmem<LOGG>;
  constexpr int G = 1 << LOGG, N = G / 2, nthr = kColFFTs * G / kEcol;
  constexpr int nblocks = N / (2 * kColFFTs);
  extern __shared__ __align__(128) unsigned char fwd_col_raw[];
  float* blk = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(fwd_col_raw) + 127) & ~(uintptr_t)127);
  float2* sm = reinterpret_cast<float2*>(blk + N * S::CW);
  float* sdp = reinterpret_cast<float*>(sm + S::FFTS);
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  for (int i = tid; i < N; i += nthr) sdp[i] = dp[i];
  __syncthreads();
  // thread 0: copy the columns of block q of every row into blk
  const auto issue = [&](int q) {
    mbar_arrive_expect_tx(&bar, (uint32_t)(N * S::CW * sizeof(float)));
    for (int r = 0; r < N; r += S::BR) tma_load_2d(blk + r * S::CW, &tmap, q * S::CW, r, &bar);
  };
  int q = blockIdx.x;
  if (tid == 0 && q < nblocks) issue(q);
  // the FFTs interleave over the lanes (f = tid mod 4): the first pass's
  // shared-memory reads of one row are 32 contiguous bytes per 4 lanes
  const int f = tid % kColFFTs, t = tid / kColFFTs;
  uint32_t phase = 0;
  for (; q < nblocks; q += gridDim.x) {
    const bool ok = mbar_wait_bounded(&bar, phase, kWaitCycles);
    // (also orders the previous block's unpack reads of sm before this
    // block's first-pass writes)
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(err, CPCT_ERR_TIMEOUT);
        mbar_wait_bounded(&bar, phase, kWaitCycles / 4);
      }
      return;
    }
    phase ^= 1u;
    const int q0 = q * (2 * kColFFTs);
    const float dq0 = sdp[q0 + 2 * f], dq1 = sdp[q0 + 2 * f + 1];
    // input x[pos] = image row (pos + N/2) mod G (the zero half is skipped)
    const auto ld = [&](int pos) -> float2 {
      const int p = (pos + N / 2) & (G - 1);
      const float2 v = *reinterpret_cast<const float2*>(blk + p * S::CW + 2 * f);
      const float cp = sdp[p];
      return make_float2(v.x * cp * dq0, v.y * cp * dq1);
    };
    const int qn = q + gridDim.x;
    const auto prefetch = [&]() {
      if (tid == 0 && qn < nblocks) {
        fence_proxy_async_smem();
        issue(qn);
      }
    };
    FFT::template run_io<false>(sm + f * FFT::PADN, tw, t, ld, typename FFT::NoStore(), prefetch);
    // unpack the two real columns: C1 = (Z[b] + conj Z[G-b])/2, C2 = (Z[b] - conj Z[G-b])/(2i)
    for (int idx = tid; idx < (N + 1) * kColFFTs; idx += nthr) {
      const int b = idx / kColFFTs, fo = idx % kColFFTs;
      const float2 Z = sm[fo * FFT::PADN + fpad(b)];
      const float2 Zm = sm[fo * FFT::PADN + fpad((G - b) & (G - 1))];
      const float4 o =
          make_float4(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y), 0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
      *reinterpret_cast<float4*>(H1 + (size_t)b * N + q0 + 2 * fo) = o;
    }
  }
}

// ---------------------------------------------------------------------------
// 2. forward row transform + extension
// ---------------------------------------------------------------------------
template <int LOGG>
__global__ void __launch_bounds__(kThreads, 4)
    k_fwd_row(const float2* __restrict__ H1, float2* __restrict__ Hx, const float2* __restrict__ tw, int ldh,
              const int* __restrict__ skip) {
  if (skip && *skip) return;
  // the padding half [N/2, G - N/2) is zero: the FFT skips it (PIN)
  using FFT = SmemFFT<LOGG, kErow, -1, true, false>;
  constexpr int G = 1 << LOGG, N = G / 2, T = FFT::T, RPC = rows_per_cta<LOGG>();
  extern __shared__ float2 sm[];
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = sm + f * FFT::PADN;
  const int b = blockIdx.x * RPC + f;
  const bool valid = b <= N;
  // Hermitian mirrors: ext row -b (b = 1, 2) and ext row G-b (b = N-3..N-1)
  int mrow = -1;
  if (b == 1 || b == 2) mrow = 2 - b;
  else if (b >= N - 3 && b <= N - 1) mrow = (2 * N - b) + 2;
  const float2* src = H1 + (size_t)(valid ? b : 0) * N;
  float2* dst = Hx + (size_t)(b + 2) * ldh;
  float2* md = Hx + (size_t)(mrow < 0 ? 0 : mrow) * ldh;
  // FFT input x[pos] = H1[b, (pos + N/2) mod G]: the first pass reads the row
  // straight from global memory (the zero half [N/2, G - N/2) is skipped);
  // the last pass writes the extended row (columns G..G+5 repeat 0..5) and
  // the conjugated mirror row straight to global memory
  const auto ld = [&](int pos) -> float2 {
    return valid ? src[(pos + N / 2) & (G - 1)] : make_float2(0.f, 0.f);
  };
  const auto st = [&](int a, float2 v) {
    if (!valid) return;
    dst[a] = v;
    if (a < 6) dst[a + G] = v;
    if (mrow >= 0) {
      const int am = (-a) & (G - 1);
      const float2 c = cconj(v);
      md[am] = c;
      if (am < 6) md[am + G] = c;
    }
  };
  FFT::template run_io<true>(buf, tw, t, ld, st);
}

// ---------------------------------------------------------------------------
// 3. forward interpolation onto the polar grid (TMA-staged bins)
// ---------------------------------------------------------------------------
struct FwdInterpArgs {
  const int4* items;
  const uint32_t* ids;
  const float4* ray;
  const float2* Hx;
  float2* Q;
  int* err;
  const int* skip;  // the launch does nothing while *skip != 0 (may be null)
  int G, ldq, ldh;
  KBPoly poly;
};

// window of a T x T bin: T + 5 rows of T + 6 complex values (the 6x6
// footprints of every sample whose first point lies in the bin)
template <int T>
struct Win {
  static constexpr int R = T + CPCT_HALO;
  static constexpr int C = T + CPCT_HALO + 1;
  // buffer stride: a TMA tensor copy into shared memory must start on a
  // 128-byte boundary, so each window buffer is padded to a multiple of 128 bytes
  static constexpr int stride = ((R * C * (int)sizeof(float2) + 127) / 128) * 128 / (int)sizeof(float2);
  static constexpr size_t smem = 2 * (size_t)stride * sizeof(float2);
};

// interpolate one polar sample from the staged window (or, if the bin does not
// hold it -- never expected -- from global memory, recording the mismatch)
template <int T>
__device__ __forceinline__ void interp_sample(const FwdInterpArgs& a, const float2* win, int C0, int R0, uint32_t id,
                                              float4 r) {
  constexpr int kWinC = Win<T>::C;
  const int j = (int)(id >> 16), k = (int)(id & 0xffffu);
  int fu, fv;
  float zu, zv;
  split_coord((float)k, r.x, r.y, fu, zu);
  split_coord((float)k, r.z, r.w, fv, zv);
  const int a0 = (fu - 2) & (a.G - 1);
  float wu[CPCT_W], wv[CPCT_W];
  kb_weights(a.poly, zu, wu);
  kb_weights(a.poly, zv, wv);
  const int ar = a0 - C0, br = fv - R0;
  float2 acc = make_float2(0.f, 0.f);
  if ((unsigned)ar < (unsigned)T && (unsigned)br < (unsigned)T) {
#pragma unroll
    for (int rr = 0; rr < CPCT_W; ++rr) {
      const float2* row = win + (br + rr) * kWinC + ar;
      float2 rs = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < CPCT_W; ++c) {
        const float2 h = row[c];
        rs.x = fmaf(wu[c], h.x, rs.x);
        rs.y = fmaf(wu[c], h.y, rs.y);
      }
      acc.x = fmaf(wv[rr], rs.x, acc.x);
      acc.y = fmaf(wv[rr], rs.y, acc.y);
    }
  } else {
    atomicOr(a.err, CPCT_ERR_BIN);
    for (int rr = 0; rr < CPCT_W; ++rr) {
      const float2* row = a.Hx + (size_t)(fv + rr) * a.ldh + a0;
      float2 rs = make_float2(0.f, 0.f);
      for (int c = 0; c < CPCT_W; ++c) {
        rs.x = fmaf(wu[c], row[c].x, rs.x);
        rs.y = fmaf(wu[c], row[c].y, rs.y);
      }
      acc.x = fmaf(wv[rr], rs.x, acc.x);
      acc.y = fmaf(wv[rr], rs.y, acc.y);
    }
  }
  a.Q[(size_t)j * a.ldq + k] = acc;
}

// Persistent CTAs walk the work items (bin, sample range) of one bin size T
// round robin; the (T + 5) x (T + 6) grid window of the next item is copied
// by TMA into the second buffer while the current one is interpolated, and
// the next item's first sample id and ray are prefetched into registers.
// 32 x 32 bins hold ~130 samples on average (1024 at most): 128 threads per
// CTA keep most threads busy on every bin
constexpr int kInterpThreads = 128;

template <int T>
__global__ void __launch_bounds__(kInterpThreads)
    k_fwd_interp(const __grid_constant__ CUtensorMap tmap, const FwdInterpArgs a, int n_items) {
  if (a.skip && *a.skip) return;
  constexpr int kWinStride = Win<T>::stride;
  extern __shared__ __align__(128) unsigned char win_raw[];
  // TMA destinations start on a 128-byte boundary (the launch adds 128 bytes)
  float2* win0 = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(win_raw) + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int item, int buf) {
    const int4 itn = a.items[item];
    const int c0 = itn.x & 0xffff, r0 = itn.x >> 16;
    mbar_arrive_expect_tx(&bar[buf], (uint32_t)(Win<T>::R * Win<T>::C * sizeof(float2)));
    tma_load_2d(win0 + buf * kWinStride, &tmap, 2 * c0, r0, &bar[buf]);
  };
  int item = blockIdx.x;
  if (tid == 0 && item < n_items) issue(item, 0);
  uint32_t phase0 = 0, phase1 = 0;
  // prefetched first sample of the current item
  uint32_t pid = 0xffffffffu;
  float4 pray = make_float4(0.f, 0.f, 0.f, 0.f);
  if (item < n_items) {
    const int4 it0 = a.items[item];
    if (it0.y + tid < it0.z) {
      pid = a.ids[it0.y + tid];
      pray = a.ray[pid >> 16];
    }
  }
  for (int iter = 0; item < n_items; ++iter, item += gridDim.x) {
    const int cur = iter & 1;
    const int next = item + gridDim.x;
    if (tid == 0 && next < n_items) issue(next, cur ^ 1);
    const int4 it = a.items[item];
    // prefetch the next item's first sample before waiting
    uint32_t nid = 0xffffffffu;
    float4 nray = make_float4(0.f, 0.f, 0.f, 0.f);
    if (next < n_items) {
      const int4 itn = a.items[next];
      if (itn.y + tid < itn.z) {
        nid = a.ids[itn.y + tid];
        nray = a.ray[nid >> 16];
      }
    }
    const uint32_t ph = cur ? phase1 : phase0;
    const bool ok = mbar_wait_bounded(&bar[cur], ph, kWaitCycles);
    if (cur) phase1 ^= 1u; else phase0 ^= 1u;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(a.err, CPCT_ERR_TIMEOUT);
        // let copies in flight land before the CTA exits
        mbar_wait_bounded(&bar[cur], ph, kWaitCycles / 4);
        if (next < n_items) mbar_wait_bounded(&bar[cur ^ 1], cur ? phase0 : phase1, kWaitCycles / 4);
      }
      return;
    }
    const int C0 = it.x & 0xffff, R0 = it.x >> 16;
    const float2* wcur = win0 + cur * kWinStride;
    if (pid != 0xffffffffu) interp_sample<T>(a, wcur, C0, R0, pid, pray);
    for (int idx = it.y + tid + (int)blockDim.x; idx < it.z; idx += blockDim.x) {
      const uint32_t id = a.ids[idx];
      interp_sample<T>(a, wcur, C0, R0, id, a.ray[id >> 16]);
    }
    pid = nid;
    pray = nray;
    __syncthreads();  // buffer `cur` is free for the copy issued next iteration
  }
}

// ---------------------------------------------------------------------------
// 4. forward ray transform (c2r of the Hermitian-completed rays)
// ---------------------------------------------------------------------------
template <int LOGNS, bool CPLX>
__global__ void __launch_bounds__(kThreads)
    k_fwd_ray(const float2* __restrict__ Q, float* __restrict__ sino, const float2* __restrict__ tw, int M, int ldq,
              const int* __restrict__ skip) {
  if (skip && *skip) return;
  using FFT = SmemFFT<LOGNS, kErow, +1>;
  constexpr int NS = 1 << LOGNS, T = FFT::T, PPC = rows_per_cta<LOGNS>(), K = NS / 2;
  extern __shared__ float2 sm[];
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = sm + f * FFT::PADN;
  const int j1 = 2 * (blockIdx.x * PPC + f), j2 = j1 + 1;
  const bool v1 = j1 < M, v2 = j2 < M;
  // the first pass reads the two rays straight from Q: Hermitian completion
  // (k > K from Q[Ns - k], conjugated), (-1)^k centring, packed as q1 + i q2
  const auto ld = [&](int k) -> float2 {
    const int kk = k <= K ? k : NS - k;
    const float sg = (kk & 1) ? -1.f : 1.f;
    float2 q1 = v1 ? Q[(size_t)j1 * ldq + kk] : make_float2(0.f, 0.f);
    float2 q2 = v2 ? Q[(size_t)j2 * ldq + kk] : make_float2(0.f, 0.f);
    q1 = cscale(q1, sg);
    q2 = cscale(q2, sg);
    if (kk == 0 || kk == K) { q1.y = 0.f; q2.y = 0.f; }
    if (k > K) { q1.y = -q1.y; q2.y = -q2.y; }
    return make_float2(q1.x - q2.y, q1.y + q2.x);
  };
  const float inv = 1.f / (float)NS;
  // the last pass writes the sinogram rows straight to global memory
  if constexpr (CPLX) {
    // complex sinogram y = A x (interleaved re, im).  Its real part is the
    // real kernel's output; its imaginary part comes only from the Nyquist
    // frequency k = -Ns/2, whose sample P[j, -K] = conj(Q[j, K]) has no
    // Hermitian partner:  Im y[j, s] = -Im(Q[j, K]) (-1)^(s - K) / Ns.
    const float i1 = v1 ? -Q[(size_t)j1 * ldq + K].y * inv : 0.f;
    const float i2 = v2 ? -Q[(size_t)j2 * ldq + K].y * inv : 0.f;
    float2* out = reinterpret_cast<float2*>(sino);
    const auto st = [&](int s_, float2 w) {
      const float sg = ((s_ + K) & 1) ? -1.f : 1.f;
      if (v1) out[(size_t)j1 * NS + s_] = make_float2(w.x * inv, sg * i1);
      if (v2) out[(size_t)j2 * NS + s_] = make_float2(w.y * inv, sg * i2);
    };
    FFT::template run_io<true>(buf, tw, t, ld, st);
  } else {
    const auto st = [&](int s_, float2 w) {
      if (v1) sino[(size_t)j1 * NS + s_] = w.x * inv;
      if (v2) sino[(size_t)j2 * NS + s_] = w.y * inv;
    };
    FFT::template run_io<true>(buf, tw, t, ld, st);
  }
}

// ---------------------------------------------------------------------------
// 5. adjoint ray transform (transpose of step 4)
// ---------------------------------------------------------------------------
template <int LOGNS, bool CPLX>
__global__ void __launch_bounds__(kThreads)
    k_adj_ray(const float* __restrict__ sino, float2* __restrict__ Q, const float2* __restrict__ tw, int M, int ldq,
              float ramp, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using FFT = SmemFFT<LOGNS, kErow, -1>;
  constexpr int NS = 1 << LOGNS, T = FFT::T, PPC = rows_per_cta<LOGNS>(), K = NS / 2;
  extern __shared__ float2 sm[];
  // complex input: per-thread partial sums of Im(w[s]) (-1)^s of both rays
  __shared__ float nyq[2][CPLX ? kThreads : 1];
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = sm + f * FFT::PADN;
  const int j1 = 2 * (blockIdx.x * PPC + f), j2 = j1 + 1;
  const bool v1 = j1 < M, v2 = j2 < M;
  if constexpr (CPLX) {
    // the real parts go through the packed FFT as in the real kernel; the
    // imaginary parts only reach the Nyquist sample (see below)
    const float2* in = reinterpret_cast<const float2*>(sino);
    float a1 = 0.f, a2 = 0.f;
    for (int s = t; s < NS; s += T) {
      const float2 w1 = v1 ? in[(size_t)j1 * NS + s] : make_float2(0.f, 0.f);
      const float2 w2 = v2 ? in[(size_t)j2 * NS + s] : make_float2(0.f, 0.f);
      buf[fpad(s)] = make_float2(w1.x, w2.x);
      const float sg = (s & 1) ? -1.f : 1.f;
      a1 = fmaf(sg, w1.y, a1);
      a2 = fmaf(sg, w2.y, a2);
    }
    nyq[0][threadIdx.x] = a1;
    nyq[1][threadIdx.x] = a2;
    __syncthreads();
    FFT::run(buf, tw, t);
  } else {
    // the first pass reads the two sinogram rows straight from global memory
    const auto ld = [&](int s_) -> float2 {
      return make_float2(v1 ? sino[(size_t)j1 * NS + s_] : 0.f, v2 ? sino[(size_t)j2 * NS + s_] : 0.f);
    };
    FFT::template run_io<false>(buf, tw, t, ld, typename FFT::NoStore());
  }
  const float inv = 1.f / (float)NS;
  for (int k = t; k <= K; k += T) {
    const float2 W = buf[fpad(k)];
    const float2 Wm = buf[fpad((NS - k) & (NS - 1))];
    float2 d1 = make_float2(0.5f * (W.x + Wm.x), 0.5f * (W.y - Wm.y));
    float2 d2 = make_float2(0.5f * (W.y + Wm.y), -0.5f * (W.x - Wm.x));
    float sc = ((k & 1) ? -inv : inv);
    if (k == 0 || k == K) { d1.y = 0.f; d2.y = 0.f; } else { sc *= 2.f; }
    if constexpr (CPLX) {
      // adjoint of the forward's Nyquist term conj(Q[j, K]) (-1)^(s-K) / Ns
      // under the real inner product: Im Q~[j, K] = -(1/Ns) sum_s Im(w[j, s])
      // (-1)^(s-K), i.e. sc * (-sum_s Im(w[j, s]) (-1)^s) with sc = (-1)^K / Ns;
      // the thread's partials are summed in thread order (deterministic)
      if (k == K) {
        float s1 = 0.f, s2 = 0.f;
        for (int i = 0; i < T; ++i) {
          s1 += nyq[0][f * T + i];
          s2 += nyq[1][f * T + i];
        }
        d1.y = -s1;
        d2.y = -s2;
      }
    }
    // filtered back-projection: ramp weight (pi / M) |k| / Ns, the DC bin
    // weighted by the mean of |k| over its width (1/4)
    if (ramp > 0.f) sc *= ramp * (k == 0 ? 0.25f : (float)k);
    if (v1) Q[(size_t)j1 * ldq + k] = cscale(d1, sc);
    if (v2) Q[(size_t)j2 * ldq + k] = cscale(d2, sc);
  }
}

// ---------------------------------------------------------------------------
// 6. adjoint spread: deterministic tile-owned gather (one warp per work item)
// ---------------------------------------------------------------------------
struct AdjSpreadArgs {
  const int4* items;
  const uint32_t* ids;
  const float4* ray;
  const float2* Qt;
  float2* Ax;
  float2* partials;
  int* err;
  const int* skip;  // the launch does nothing while *skip != 0 (may be null)
  int G, ldq, ldh, ext_rows;
  int lanes;  // samples per round: 16 (lanes 0..15), 32 (one warp), 64 (two warps), or column groups
  KBPoly poly;
};

// accumulator of a T x T bin: T + 10 rows (a 5-cell halo on both sides) of
// T + 13 complex values (the odd row pitch the bank classes of the rounds
// use; 45 for T = 32)
template <int T>
struct Acc {
  static constexpr int rows = T + 2 * CPCT_HALO;
  static constexpr int ld = rows + 3;
};

// One warp (two for 64-lane rounds) per work item: a run of conflict-free
// rounds of one tile.  In a round, thread l holds one sample (or none); the
// 6x6 footprints of the round's samples are pairwise disjoint and their
// first cells fall in distinct 64-bit bank pairs within each half-warp, so
// every thread updates its 36 accumulator cells with plain shared-memory
// loads and stores: no atomics, no conflicts.  Rounds are applied in their
// fixed plan order (a barrier of the item's threads between rounds), hence
// every output element receives its contributions in the same order on
// every run.
template <int T>
__global__ void __launch_bounds__(64) k_adj_spread(const AdjSpreadArgs a) {
  if (a.skip && *a.skip) return;
  constexpr int kRRows = Acc<T>::rows, kRLd = Acc<T>::ld;
  __shared__ __align__(16) float2 acc[kRRows * kRLd];
  const int lane = threadIdx.x, nt = blockDim.x;
  const bool two_warps = nt > 32;
  const int4 it = a.items[blockIdx.x];
  const int TC = it.x & 0xffff, TR = it.x >> 16;
  for (int i = lane; i < kRRows * kRLd; i += nt) acc[i] = make_float2(0.f, 0.f);
  // software pipeline: ids two rounds ahead, sample data one round ahead;
  // with 16-lane rounds the upper half-warp holds no sample
  const int L = a.lanes;
  const bool act = lane < L;
  uint32_t id0 = act && it.y < it.z ? a.ids[(size_t)it.y * L + lane] : 0xffffffffu;
  uint32_t id1 = act && it.y + 1 < it.z ? a.ids[(size_t)(it.y + 1) * L + lane] : 0xffffffffu;
  float4 ray0 = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 val0 = make_float2(0.f, 0.f);
  if (id0 != 0xffffffffu) {
    ray0 = a.ray[id0 >> 16];
    val0 = a.Qt[(size_t)(id0 >> 16) * a.ldq + (id0 & 0xffffu)];
  }
  if (two_warps) __syncthreads();
  else __syncwarp();
  for (int r = it.y; r < it.z; ++r) {
    const uint32_t id2 = act && r + 2 < it.z ? a.ids[(size_t)(r + 2) * L + lane] : 0xffffffffu;
    float4 ray1 = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 val1 = make_float2(0.f, 0.f);
    if (id1 != 0xffffffffu) {
      ray1 = a.ray[id1 >> 16];
      val1 = a.Qt[(size_t)(id1 >> 16) * a.ldq + (id1 & 0xffffu)];
    }
    if (id0 != 0xffffffffu) {
      const float k = (float)(id0 & 0xffffu);
      int fu, fv;
      float zu, zv;
      split_coord(k, ray0.x, ray0.y, fu, zu);
      split_coord(k, ray0.z, ray0.w, fv, zv);
      const int ar = ((fu - 2) & (a.G - 1)) - TC + CPCT_HALO, br = fv - TR + CPCT_HALO;
      if ((unsigned)ar <= (unsigned)(T + CPCT_HALO - 1) && (unsigned)br <= (unsigned)(T + CPCT_HALO - 1)) {
        float wu[CPCT_W], wv[CPCT_W];
        kb_weights(a.poly, zu, wu);
        kb_weights(a.poly, zv, wv);
        float2* base = acc + br * kRLd + ar;
        float2 t[CPCT_W * CPCT_W];
#pragma unroll
        for (int q = 0; q < CPCT_W; ++q)
#pragma unroll
          for (int c = 0; c < CPCT_W; ++c) t[q * CPCT_W + c] = base[q * kRLd + c];
#pragma unroll
        for (int q = 0; q < CPCT_W; ++q) {
          const float2 vq = cscale(val0, wv[q]);
#pragma unroll
          for (int c = 0; c < CPCT_W; ++c) {
            t[q * CPCT_W + c].x = fmaf(wu[c], vq.x, t[q * CPCT_W + c].x);
            t[q * CPCT_W + c].y = fmaf(wu[c], vq.y, t[q * CPCT_W + c].y);
          }
        }
#pragma unroll
        for (int q = 0; q < CPCT_W; ++q)
#pragma unroll
          for (int c = 0; c < CPCT_W; ++c) base[q * kRLd + c] = t[q * CPCT_W + c];
      } else {
        atomicOr(a.err, CPCT_ERR_BIN);
      }
    }
    if (two_warps) __syncthreads();
    else __syncwarp();
    id0 = id1;
    ray0 = ray1;
    val0 = val1;
    id1 = id2;
  }
  if (it.w < 0) {
    for (int i = lane; i < T * T; i += nt) {
      const int rr = i / T, cc = i % T;
      const int gr = TR + rr, gc = TC + cc;
      if (gr < a.ext_rows && gc < a.ldh)
        a.Ax[(size_t)gr * a.ldh + gc] = acc[(rr + CPCT_HALO) * kRLd + cc + CPCT_HALO];
    }
  } else {
    float2* dst = a.partials + (size_t)it.w;
    for (int i = lane; i < T * T; i += nt) dst[i] = acc[(i / T + CPCT_HALO) * kRLd + i % T + CPCT_HALO];
  }
}

// Column groups (round width cpct_detail::kGroupLanes): one warp per work
// item, five samples per group; lane 6 s + c applies column c of slot s's
// footprint, row after row, so a sample's 36 taps take six accesses of six
// lanes and a group's 30 lanes cover five samples.  The slots' first cells
// follow a bank pattern that keeps each half-warp's accesses conflict free
// (the packer's invariant), and the footprints of a group are disjoint.  The
// entries carry the sample's fractions and accumulator coordinates (the host
// computed them with the kernels' own split), so a lane evaluates only its
// column's weight and the six row weights.  Groups are applied in plan
// order: the result is bitwise reproducible, with per-tap products equal to
// the rounds' (only the order of the additions into a cell differs).
template <int T>
__global__ void __launch_bounds__(32) k_adj_spread_cols(const AdjSpreadArgs a) {
  if (a.skip && *a.skip) return;
  constexpr int kRRows = Acc<T>::rows, kRLd = Acc<T>::ld;
  constexpr uint32_t kEmpty = 0xffffffffu;
  __shared__ __align__(16) float2 acc[kRRows * kRLd];
  const int lane = threadIdx.x;
  const int slot = lane / CPCT_W, c = lane - CPCT_W * slot;
  const bool act = slot < cpct_detail::kGroupSlots;
  // this lane's column tap: pair min(c, 5 - c) of the even / odd split
  const int pi = c < 3 ? c : CPCT_W - 1 - c;
  float E[CPCT_NPOLY], O[CPCT_NPOLY];
#pragma unroll
  for (int d = 0; d < CPCT_NPOLY; ++d) {
    E[d] = pi == 0 ? a.poly.e[0][d] : pi == 1 ? a.poly.e[1][d] : a.poly.e[2][d];
    O[d] = pi == 0 ? a.poly.o[0][d] : pi == 1 ? a.poly.o[1][d] : a.poly.o[2][d];
  }
  const int4 it = a.items[blockIdx.x];
  const int TC = it.x & 0xffff, TR = it.x >> 16;
  for (int i = lane; i < kRRows * kRLd; i += 32) acc[i] = make_float2(0.f, 0.f);
  const uint4* ent = reinterpret_cast<const uint4*>(a.ids);
  const uint4 none = make_uint4(kEmpty, 0u, 0u, 0u);
  // software pipeline over a register ring: a group is about a sixth of a
  // round's work, so entries are fetched 2 kDepth groups ahead and the
  // sample values (a gather from the polar samples) kDepth ahead
  constexpr int kDepth = 4;
  uint4 e[2 * kDepth];
  float2 v[kDepth];
  auto fetch_e = [&](int g) { return act && g < it.z ? ent[(size_t)g * cpct_detail::kGroupSlots + slot] : none; };
  auto fetch_v = [&](const uint4& x) {
    return x.x != kEmpty ? a.Qt[(size_t)(x.x >> 16) * a.ldq + (x.x & 0xffffu)] : make_float2(0.f, 0.f);
  };
#pragma unroll
  for (int k = 0; k < 2 * kDepth; ++k) e[k] = fetch_e(it.y + k);
#pragma unroll
  for (int k = 0; k < kDepth; ++k) v[k] = fetch_v(e[k]);
  __syncwarp();
  for (int r = it.y; r < it.z; r += kDepth) {
#pragma unroll
    for (int k = 0; k < kDepth; ++k) {
      const uint4 e0 = e[k];
      const float2 v0 = v[k];
      // refill: this slot's value for group r + k + kDepth (its entry was
      // fetched kDepth groups ago), its entry for group r + k + 2 kDepth
      v[k] = fetch_v(e[k + kDepth]);
      e[k] = e[k + kDepth];
      e[k + kDepth] = fetch_e(r + k + 2 * kDepth);
      if (e0.x != kEmpty) {
        const int ar = (int)(e0.w & 0xffffu), br = (int)(e0.w >> 16);
        if (ar <= T + CPCT_HALO - 1 && br <= T + CPCT_HALO - 1) {
          const float zu = __uint_as_float(e0.y), zv = __uint_as_float(e0.z);
          float wv[CPCT_W];
          kb_weights(a.poly, zv, wv);
          const float su = fmaf(2.f, zu, -1.f), su2 = su * su;
          float Eu = E[CPCT_NPOLY - 1], Ou = O[CPCT_NPOLY - 1];
#pragma unroll
          for (int d = CPCT_NPOLY - 2; d >= 0; --d) {
            Eu = fmaf(Eu, su2, E[d]);
            Ou = fmaf(Ou, su2, O[d]);
          }
          float wu = fmaf(c < 3 ? su : -su, Ou, Eu);
          if (c == CPCT_W - 1 && zu == 0.f) wu = 0.f;  // open support, as kb_weights
          float2* col = acc + br * kRLd + ar + c;
#pragma unroll
          for (int q = 0; q < CPCT_W; ++q) {
            const float2 vq = cscale(v0, wv[q]);
            float2 t = col[q * kRLd];
            t.x = fmaf(wu, vq.x, t.x);
            t.y = fmaf(wu, vq.y, t.y);
            col[q * kRLd] = t;
          }
        } else {
          atomicOr(a.err, CPCT_ERR_BIN);
        }
      }
      __syncwarp();
    }
  }
  if (it.w < 0) {
    for (int i = lane; i < T * T; i += 32) {
      const int rr = i / T, cc = i % T;
      const int gr = TR + rr, gc = TC + cc;
      if (gr < a.ext_rows && gc < a.ldh)
        a.Ax[(size_t)gr * a.ldh + gc] = acc[(rr + CPCT_HALO) * kRLd + cc + CPCT_HALO];
    }
  } else {
    float2* dst = a.partials + (size_t)it.w;
    for (int i = lane; i < T * T; i += 32) dst[i] = acc[(i / T + CPCT_HALO) * kRLd + i % T + CPCT_HALO];
  }
}

// 7. fixed-order sum of the partial tiles of a split T x T bin (piece order
// q = 0, 1, ...); kReduceThreads threads per part of a bin, blockIdx.y the
// part.  Every thread issues the loads of up to 16 pieces at once (one
// round trip for a bin of at most 16 pieces) and adds them in piece order.
constexpr int kReduceThreads = 256;

template <int T>
__global__ void __launch_bounds__(kReduceThreads)
    k_adj_reduce(const int4* __restrict__ split, const float2* __restrict__ partials, float2* __restrict__ Ax,
                 int ldh, int ext_rows, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int4 sp = split[blockIdx.x];
  const int TC = sp.x & 0xffff, TR = sp.x >> 16;
  constexpr size_t S = (size_t)T * T;
  const int i = blockIdx.y * kReduceThreads + threadIdx.x;
  if (i >= T * T) return;
  const float2* src = partials + (size_t)sp.y + i;
  float2 sum = make_float2(0.f, 0.f);
  for (int q0 = 0; q0 < sp.z; q0 += 16) {
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = q0 + k < sp.z ? src[(size_t)(q0 + k) * S] : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (q0 + k < sp.z) sum = cadd(sum, v[k]);
  }
  const int gr = TR + i / T, gc = TC + i % T;
  if (gr < ext_rows && gc < ldh) Ax[(size_t)gr * ldh + gc] = sum;
}

// ---------------------------------------------------------------------------
// 8. adjoint row transform with the fold of the extension
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 wrapped(const float2* __restrict__ row, int a, int G) {
  float2 v = row[a];
  if (a < 6) v = cadd(v, row[a + G]);
  return v;
}

// Persistent: each CTA takes groups of RPC rows (b = g RPC + f) in turn.  The
// raw rows (G + 6 values: the wrapped columns included) arrive in shared
// memory by bulk copies; the copy of the CTA's next group is issued as soon
// as the first FFT pass has read the current one, so it lands while the
// remaining passes and the stores run.  Mirror rows (5 rows) are read from
// global memory.  Every wait is bounded: on a timeout the CTA records
// CPCT_ERR_TIMEOUT, lets its copy in flight land and returns.
template <int LOGG>
struct AdjRowSmem {
  static constexpr int G = 1 << LOGG;
  static constexpr int RPC = rows_per_cta<LOGG>();
  static constexpr int RAWS = (G + 6 + 15) / 16 * 16;  // raw row stride (128-byte multiple)
  static constexpr uint32_t RAW_BYTES = (uint32_t)(G + 6) * sizeof(float2);  // a multiple of 16
  static constexpr size_t bytes = (size_t)RPC * (RAWS + SmemFFT<LOGG, kErow, +1, false, true>::PADN) * sizeof(float2) + 128;
};

template <int LOGG>
__global__ void __launch_bounds__(kThreads, 3)
    k_adj_row(const float2* __restrict__ Ax, float2* __restrict__ H1, const float2* __restrict__ tw, int ldh,
              int* __restrict__ err, const int* __restrict__ skip) {
  if (skip && *skip) return;
  // only X = -N/2 .. N/2-1 is kept: the FFT skips the other outputs (POUT)
  using FFT = SmemFFT<LOGG, kErow, +1, false, true>;
  using S = AdjRowSmem<LOGG>;
  constexpr int G = 1 << LOGG, N = G / 2, T = FFT::T, RPC = S::RPC;
  constexpr int ngroups = (N + 1 + RPC - 1) / RPC;
  extern __shared__ __align__(128) unsigned char adj_row_raw[];
  float2* raw0 = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(adj_row_raw) + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int f = tid / T, t = tid % T;
  float2* raw = raw0 + f * S::RAWS;
  float2* buf = raw0 + RPC * S::RAWS + f * FFT::PADN;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0: copy the rows of group g into the raw buffers
  const auto issue = [&](int g) {
    const int nv = min(RPC, N + 1 - g * RPC);
    mbar_arrive_expect_tx(&bar, (uint32_t)nv * S::RAW_BYTES);
    for (int ff = 0; ff < nv; ++ff)
      bulk_load(raw0 + ff * S::RAWS, Ax + (size_t)(g * RPC + ff + 2) * ldh, S::RAW_BYTES, &bar);
  };
  int g = blockIdx.x;
  if (tid == 0 && g < ngroups) issue(g);
  uint32_t phase = 0;
  for (; g < ngroups; g += gridDim.x) {
    const bool ok = mbar_wait_bounded(&bar, phase, kWaitCycles);
    // (also orders the previous group's last-pass reads of buf before this
    // group's first-pass writes)
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(err, CPCT_ERR_TIMEOUT);
        mbar_wait_bounded(&bar, phase, kWaitCycles / 4);
      }
      return;
    }
    phase ^= 1u;
    const int b = g * RPC + f;
    const bool valid = b <= N;
    int mrow = -1;
    if (b == 1 || b == 2) mrow = 2 - b;
    else if (b >= N - 3 && b <= N - 1) mrow = (2 * N - b) + 2;
    const float2* mr = Ax + (size_t)(mrow < 0 ? 0 : mrow) * ldh;
    // fold the extension into the first pass's input: wrapped columns
    // G..G+5 and, for rows 1, 2, N-3..N-1, the conjugated mirror row
    const auto ld = [&](int a) -> float2 {
      if (!valid) return make_float2(0.f, 0.f);
      float2 v = raw[a];
      if (a < 6) v = cadd(v, raw[a + G]);
      if (mrow >= 0) v = cadd(v, cconj(wrapped(mr, (-a) & (G - 1), G)));
      return v;
    };
    float2* out = H1 + (size_t)b * N;
    const auto st = [&](int k, float2 v) {
      if (valid) out[(k + N / 2) & (G - 1)] = v;
    };
    const int gn = g + gridDim.x;
    const auto prefetch = [&]() {
      if (tid == 0 && gn < ngroups) {
        fence_proxy_async_smem();
        issue(gn);
      }
    };
    FFT::template run_io<true>(buf, tw, t, ld, st, prefetch);
  }
}

// ---------------------------------------------------------------------------
// 9. adjoint column transform: Re of the inverse transform over b = 0..N
// ---------------------------------------------------------------------------
template <int LOGG>
__global__ void __launch_bounds__(kColFFTs*(1 << LOGG) / kEcol)
    k_adj_col(const float2* __restrict__ H1, const float* __restrict__ dp, float* __restrict__ img,
              const float2* __restrict__ tw, const int* __restrict__ skip) {
  if (skip && *skip) return;
  // only Y = -N/2 .. N/2-1 is kept: the FFT skips the other outputs (POUT)
  using FFT = SmemFFT<LOGG, kEcol, +1, false, true>;
  constexpr int G = 1 << LOGG, N = G / 2;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int q0 = blockIdx.x * (2 * kColFFTs);
  // FFT f packs columns q0+2f and q0+2f+1; the FFTs interleave over the lanes
  // (f = tid mod 4).  The first pass reads H1 straight from global memory and
  // Hermitian-symmetrises it: x[b] and x[G-b] both come from row b of the
  // two columns z1 = (z.x, z.y), z2 = (z.z, z.w)
  const int f = tid % kColFFTs, t = tid / kColFFTs;
  const auto ld = [&](int pos) -> float2 {
    const int b = pos <= N ? pos : G - pos;
    const float4 z = *reinterpret_cast<const float4*>(H1 + (size_t)b * N + q0 + 2 * f);
    if (b == 0 || b == N) return make_float2(z.x, z.z);
    if (pos < N) return make_float2(0.5f * (z.x - z.w), 0.5f * (z.y + z.z));
    return make_float2(0.5f * (z.x + z.w), 0.5f * (z.z - z.y));
  };
  // the last pass writes the cropped, deapodized columns straight to the image
  const float2 dq = *reinterpret_cast<const float2*>(dp + q0 + 2 * f);
  const auto st = [&](int k, float2 w) {
    const int p = (k + N / 2) & (G - 1);
    const float cp = dp[p];
    *reinterpret_cast<float2*>(img + (size_t)p * N + q0 + 2 * f) = make_float2(w.x * cp * dq.x, w.y * cp * dq.y);
  };
  FFT::template run_io<true>(sm + f * FFT::PADN, tw, t, ld, st);
}

// ---------------------------------------------------------------------------
// size dispatch
// ---------------------------------------------------------------------------
template <class F>
void max_carveout(F f) {
  cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

template <int LOGG>
int set_attr_G() {
  max_carveout(k_fwd_col<LOGG>);
  max_carveout(k_adj_col<LOGG>);
  max_carveout(k_fwd_row<LOGG>);
  max_carveout(k_adj_row<LOGG>);
  if (cudaFuncSetAttribute(k_fwd_col<LOGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FwdColSmem<LOGG>::bytes) != cudaSuccess) return CPCT_ECUDA;
  if (cudaFuncSetAttribute(k_adj_col<LOGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem<LOGG>(kColFFTs)) != cudaSuccess) return CPCT_ECUDA;
  if (cudaFuncSetAttribute(k_fwd_row<LOGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem<LOGG>(rows_per_cta<LOGG>())) != cudaSuccess) return CPCT_ECUDA;
  if (cudaFuncSetAttribute(k_adj_row<LOGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdjRowSmem<LOGG>::bytes) != cudaSuccess) return CPCT_ECUDA;
  return CPCT_OK;
}
template <int LOGNS, bool CPLX>
int set_attr_Ns_one() {
  max_carveout(k_fwd_ray<LOGNS, CPLX>);
  max_carveout(k_adj_ray<LOGNS, CPLX>);
  if (cudaFuncSetAttribute(k_fwd_ray<LOGNS, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem<LOGNS>(rows_per_cta<LOGNS>())) != cudaSuccess) return CPCT_ECUDA;
  if (cudaFuncSetAttribute(k_adj_ray<LOGNS, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem<LOGNS>(rows_per_cta<LOGNS>())) != cudaSuccess) return CPCT_ECUDA;
  return CPCT_OK;
}
template <int LOGNS>
int set_attr_Ns() {
  const int rc = set_attr_Ns_one<LOGNS, false>();
  return rc ? rc : set_attr_Ns_one<LOGNS, true>();
}

template <int LOGG>
int launch_fwd_G(cpct_plan* p, const float* img, const int* skip, cudaStream_t s) {
  constexpr int G = 1 << LOGG;
  const int nthr = kColFFTs * G / kEcol, nblocks = p->n / (2 * kColFFTs);
  if (p->fwd_col_grid <= 0) {
    // persistent grid: every CTA resident at once
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_col<LOGG>, nthr, FwdColSmem<LOGG>::bytes);
    p->fwd_col_grid = std::max(1, sms * std::max(1, per_sm));
  }
  const CUtensorMap* tm = nullptr;
  if (cpct_image_cols_map(p, img, &tm) != CPCT_OK) return CPCT_ECUDA;
  cpct_prof_begin(p, KID_FWD_COL, s);
  k_fwd_col<LOGG><<<std::min(nblocks, p->fwd_col_grid), nthr, FwdColSmem<LOGG>::bytes, s>>>(
      *tm, p->d_deapod, p->d_H1, p->d_twG, p->d_err, skip);
  cpct_prof_end(p, KID_FWD_COL, s);
  constexpr int RPC = rows_per_cta<LOGG>();
  cpct_prof_begin(p, KID_FWD_ROW, s);
  k_fwd_row<LOGG><<<(p->n + 1 + RPC - 1) / RPC, RPC * (G / kErow), fft_smem<LOGG>(RPC), s>>>(p->d_H1, p->d_Hx, p->d_twG, p->ldh, skip);
  cpct_prof_end(p, KID_FWD_ROW, s);
  return CPCT_OK;
}
template <int LOGNS>
void launch_fwd_Ns(cpct_plan* p, float* sino, bool cplx, const int* skip, cudaStream_t s) {
  constexpr int NS = 1 << LOGNS, PPC = rows_per_cta<LOGNS>();
  const int pairs = (p->m + 1) / 2;
  const dim3 grid((pairs + PPC - 1) / PPC), block(PPC * (NS / kErow));
  cpct_prof_begin(p, KID_FWD_RAY, s);
  if (cplx)
    k_fwd_ray<LOGNS, true><<<grid, block, fft_smem<LOGNS>(PPC), s>>>(p->d_Q, sino, p->d_twNs, p->m, p->ldq, skip);
  else
    k_fwd_ray<LOGNS, false><<<grid, block, fft_smem<LOGNS>(PPC), s>>>(p->d_Q, sino, p->d_twNs, p->m, p->ldq, skip);
  cpct_prof_end(p, KID_FWD_RAY, s);
}
template <int LOGNS>
void launch_adj_Ns(cpct_plan* p, const float* sino, bool cplx, float ramp, const int* skip, cudaStream_t s) {
  constexpr int NS = 1 << LOGNS, PPC = rows_per_cta<LOGNS>();
  const int pairs = (p->m + 1) / 2;
  const dim3 grid((pairs + PPC - 1) / PPC), block(PPC * (NS / kErow));
  cpct_prof_begin(p, KID_ADJ_RAY, s);
  if (cplx)
    k_adj_ray<LOGNS, true><<<grid, block, fft_smem<LOGNS>(PPC), s>>>(sino, p->d_Q, p->d_twNs, p->m, p->ldq, ramp, skip);
  else
    k_adj_ray<LOGNS, false><<<grid, block, fft_smem<LOGNS>(PPC), s>>>(sino, p->d_Q, p->d_twNs, p->m, p->ldq, ramp, skip);
  cpct_prof_end(p, KID_ADJ_RAY, s);
}
template <int LOGG>
void launch_adj_G(cpct_plan* p, float* img, const int* skip, cudaStream_t s) {
  constexpr int G = 1 << LOGG;
  constexpr int RPC = rows_per_cta<LOGG>();
  const int groups = (p->n + 1 + RPC - 1) / RPC;
  if (p->adj_row_grid <= 0) {
    // persistent grid: every CTA resident at once
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_row<LOGG>, RPC * (G / kErow), AdjRowSmem<LOGG>::bytes);
    p->adj_row_grid = std::max(1, sms * std::max(1, per_sm));
  }
  cpct_prof_begin(p, KID_ADJ_ROW, s);
  k_adj_row<LOGG><<<std::min(groups, p->adj_row_grid), RPC * (G / kErow), AdjRowSmem<LOGG>::bytes, s>>>(
      p->d_Ax, p->d_H1, p->d_twG, p->ldh, p->d_err, skip);
  cpct_prof_end(p, KID_ADJ_ROW, s);
  cpct_prof_begin(p, KID_ADJ_COL, s);
  k_adj_col<LOGG><<<p->n / (2 * kColFFTs), kColFFTs * G / kEcol, fft_smem<LOGG>(kColFFTs), s>>>(p->d_H1, p->d_deapod, img, p->d_twG, skip);
  cpct_prof_end(p, KID_ADJ_COL, s);
}

#define CPCT_DISPATCH_G(lg, CALL)   \
  switch (lg) {                     \
    case 6: CALL(6); break;         \
    case 7: CALL(7); break;         \
    case 8: CALL(8); break;         \
    case 9: CALL(9); break;         \
    case 10: CALL(10); break;       \
    case 11: CALL(11); break;       \
    case 12: CALL(12); break;       \
    default: return CPCT_EINVAL;    \
  }
#define CPCT_DISPATCH_NS(lg, CALL)  \
  switch (lg) {                     \
    case 5: CALL(5); break;         \
    case 6: CALL(6); break;         \
    case 7: CALL(7); break;         \
    case 8: CALL(8); break;         \
    case 9: CALL(9); break;         \
    case 10: CALL(10); break;       \
    case 11: CALL(11); break;       \
    case 12: CALL(12); break;       \
    default: return CPCT_EINVAL;    \
  }

constexpr int kBinClasses = 3;  // bins of 16, 32 and 64 grid points

template <int T>
int set_attr_interp() {
  if (cudaFuncSetAttribute(k_fwd_interp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Win<T>::smem + 128) !=
      cudaSuccess)
    return CPCT_ECUDA;
  return CPCT_OK;
}

template <int T>
void launch_fwd_interp(cpct_plan* p, const FwdInterpArgs& a, int n_items, cudaStream_t s) {
  const int c = T == 16 ? 0 : T == 32 ? 1 : 2;
  if (p->fwd_interp_grid[c] <= 0) {
    // persistent grid: every CTA resident at once
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_interp<T>, kInterpThreads, Win<T>::smem + 128);
    p->fwd_interp_grid[c] = std::max(1, sms * std::max(1, per_sm));
  }
  const int grid = std::min(n_items, p->fwd_interp_grid[c]);
  k_fwd_interp<T><<<grid, kInterpThreads, Win<T>::smem + 128, s>>>(p->tmap_Hx[c], a, n_items);
}

}  // namespace

int cpct_col_block_width() { return 2 * kColFFTs; }

int cpct_gridding_resident(int which, int T, int threads) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  cudaError_t e;
  if (which == 0)
    e = T == 16   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fwd_interp<16>, kInterpThreads, Win<16>::smem + 128)
        : T == 64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fwd_interp<64>, kInterpThreads, Win<64>::smem + 128)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fwd_interp<32>, kInterpThreads, Win<32>::smem + 128);
  else
    e = T == 16   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adj_spread<16>, threads, 0)
        : T == 64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adj_spread<64>, threads, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adj_spread<32>, threads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per;
}

int cpct_radon_setup_attributes(int logG, int logNs) {
  int rc = set_attr_interp<16>();
  if (!rc) rc = set_attr_interp<32>();
  if (!rc) rc = set_attr_interp<64>();
  if (rc) return rc;
#define SETG(L) rc = set_attr_G<L>()
#define SETN(L) rc = set_attr_Ns<L>()
  CPCT_DISPATCH_G(logG, SETG);
  if (rc) return rc;
  CPCT_DISPATCH_NS(logNs, SETN);
#undef SETG
#undef SETN
  return rc;
}

namespace {

// forward operator; `sino` is M x Ns float32 (cplx = false) or M x Ns
// interleaved complex64 (cplx = true)
int launch_fwd_impl(cpct_plan* p, const float* d_img, float* d_sino, bool cplx, const int* skip, cudaStream_t s) {
#define FG(L)                                        \
  {                                                  \
    const int rc_ = launch_fwd_G<L>(p, d_img, skip, s); \
    if (rc_ != CPCT_OK) return rc_;                  \
  }
  CPCT_DISPATCH_G(p->logG, FG);
#undef FG
  FwdInterpArgs a;
  a.ids = p->d_fwd_ids;
  a.ray = p->d_ray;
  a.Hx = p->d_Hx;
  a.Q = p->d_Q;
  a.err = p->d_err;
  a.G = p->G;
  a.ldq = p->ldq;
  a.ldh = p->ldh;
  a.poly = p->poly;
  a.skip = skip;
  if (p->n_fwd_items > 0) {
    // one profiling bracket around the launches of every bin size; with
    // bins of several sizes the per-size launches run concurrently on side
    // streams forked from `s` (they read disjoint item lists and write
    // disjoint polar samples)
    cpct_prof_begin(p, KID_FWD_INTERP, s);
    int cls[kBinClasses], nc = 0;
    for (int c = 0; c < kBinClasses; ++c)
      if (p->fwd_cls[c + 1] > p->fwd_cls[c]) cls[nc++] = c;
    p->launches += nc - 1;
    if (nc > 1) cudaEventRecord(p->ev_fork, s);
    for (int i = 0; i < nc; ++i) {
      const int c = cls[i];
      cudaStream_t si = i == 0 ? s : p->side[i - 1];
      if (i > 0) cudaStreamWaitEvent(si, p->ev_fork, 0);
      a.items = p->d_fwd_items + p->fwd_cls[c];
      const int n_items = p->fwd_cls[c + 1] - p->fwd_cls[c];
      if (c == 0) launch_fwd_interp<16>(p, a, n_items, si);
      else if (c == 1) launch_fwd_interp<32>(p, a, n_items, si);
      else launch_fwd_interp<64>(p, a, n_items, si);
      if (i > 0) cudaEventRecord(p->ev_join[i - 1], si);
    }
    for (int i = 1; i < nc; ++i) cudaStreamWaitEvent(s, p->ev_join[i - 1], 0);
    cpct_prof_end(p, KID_FWD_INTERP, s);
  }
#define FN(L) launch_fwd_Ns<L>(p, d_sino, cplx, skip, s)
  CPCT_DISPATCH_NS(p->logNs, FN);
#undef FN
  return cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

// adjoint operator; `partials` holds the partial tiles of the split heavy
// tiles (the plan's own buffer, or the allocation-free entry point's array)
int launch_adj_impl(cpct_plan* p, const float* d_sino, float* d_img, bool cplx, float ramp, const int* skip,
                    float2* partials, cudaStream_t s) {
#define AN(L) launch_adj_Ns<L>(p, d_sino, cplx, ramp, skip, s)
  CPCT_DISPATCH_NS(p->logNs, AN);
#undef AN
  AdjSpreadArgs a;
  a.ids = p->d_adj_ids;
  a.ray = p->d_ray;
  a.Qt = p->d_Q;
  a.Ax = p->d_Ax;
  a.partials = partials;
  a.err = p->d_err;
  a.G = p->G;
  a.ldq = p->ldq;
  a.ldh = p->ldh;
  a.ext_rows = p->ext_rows;
  a.lanes = p->round_lanes;
  a.poly = p->poly;
  a.skip = skip;
  // every partial tile is written in full by its work item before the
  // reduce reads it, so the partial tiles need no clearing between calls
  int cls[kBinClasses], nc = 0;
  for (int c = 0; c < kBinClasses; ++c)
    if (p->adj_cls[c + 1] > p->adj_cls[c]) cls[nc++] = c;
  auto spread = [&](int c, cudaStream_t si) {
    a.items = p->d_adj_items + p->adj_cls[c];
    const int n_items = p->adj_cls[c + 1] - p->adj_cls[c];
    if (a.lanes == cpct_detail::kGroupLanes) {
      if (c == 0) k_adj_spread_cols<16><<<n_items, 32, 0, si>>>(a);
      else if (c == 1) k_adj_spread_cols<32><<<n_items, 32, 0, si>>>(a);
      else k_adj_spread_cols<64><<<n_items, 32, 0, si>>>(a);
      return;
    }
    const int nt = a.lanes > 32 ? 64 : 32;
    if (c == 0) k_adj_spread<16><<<n_items, nt, 0, si>>>(a);
    else if (c == 1) k_adj_spread<32><<<n_items, nt, 0, si>>>(a);
    else k_adj_spread<64><<<n_items, nt, 0, si>>>(a);
  };
  auto reduce = [&](int c, cudaStream_t si) {
    const int n = p->split_cls[c + 1] - p->split_cls[c];
    if (n <= 0) return false;
    const int4* sp = p->d_split + p->split_cls[c];
    const int T = c == 0 ? 16 : c == 1 ? 32 : 64;
    const dim3 grid(n, (T * T + kReduceThreads - 1) / kReduceThreads);
    if (c == 0) k_adj_reduce<16><<<grid, kReduceThreads, 0, si>>>(sp, partials, p->d_Ax, p->ldh, p->ext_rows, skip);
    else if (c == 1) k_adj_reduce<32><<<grid, kReduceThreads, 0, si>>>(sp, partials, p->d_Ax, p->ldh, p->ext_rows, skip);
    else k_adj_reduce<64><<<grid, kReduceThreads, 0, si>>>(sp, partials, p->d_Ax, p->ldh, p->ext_rows, skip);
    return true;
  };
  if (nc == 1) {
    cpct_prof_begin(p, KID_ADJ_SPREAD, s);
    spread(cls[0], s);
    cpct_prof_end(p, KID_ADJ_SPREAD, s);
    if (p->n_split > 0) {
      cpct_prof_begin(p, KID_ADJ_REDUCE, s);
      reduce(cls[0], s);
      cpct_prof_end(p, KID_ADJ_REDUCE, s);
    }
  } else if (nc > 1) {
    // bins of several sizes: each size's spread and reduce run as one chain
    // on its own stream (disjoint output regions and partial tiles); the
    // bracket of k_adj_spread covers the whole fork..join, reduce included
    cpct_prof_begin(p, KID_ADJ_SPREAD, s);
    cudaEventRecord(p->ev_fork, s);
    for (int i = 0; i < nc; ++i) {
      cudaStream_t si = i == 0 ? s : p->side[i - 1];
      if (i > 0) cudaStreamWaitEvent(si, p->ev_fork, 0);
      spread(cls[i], si);
      if (i > 0) p->launches++;
      if (reduce(cls[i], si)) p->launches++;
      if (i > 0) cudaEventRecord(p->ev_join[i - 1], si);
    }
    for (int i = 1; i < nc; ++i) cudaStreamWaitEvent(s, p->ev_join[i - 1], 0);
    cpct_prof_end(p, KID_ADJ_SPREAD, s);
  }
#define AG(L) launch_adj_G<L>(p, d_img, skip, s)
  CPCT_DISPATCH_G(p->logG, AG);
#undef AG
  return cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

}  // namespace

int cpct_launch_fwd(cpct_plan* p, const float* d_img, float* d_sino, cudaStream_t s) {
  return launch_fwd_impl(p, d_img, d_sino, false, nullptr, s);
}

int cpct_launch_fwd_skip(cpct_plan* p, const float* d_img, float* d_sino, const int* skip, cudaStream_t s) {
  return launch_fwd_impl(p, d_img, d_sino, false, skip, s);
}

int cpct_launch_fwd_c(cpct_plan* p, const float* d_img, float2* d_sino_c, cudaStream_t s) {
  return launch_fwd_impl(p, d_img, reinterpret_cast<float*>(d_sino_c), true, nullptr, s);
}

int cpct_launch_adj(cpct_plan* p, const float* d_sino, float* d_img, cudaStream_t s) {
  return launch_adj_impl(p, d_sino, d_img, false, 0.f, nullptr, p->d_partials, s);
}

int cpct_launch_adj_ramp(cpct_plan* p, const float* d_sino, float* d_img, float ramp, const int* skip,
                         cudaStream_t s) {
  return launch_adj_impl(p, d_sino, d_img, false, ramp, skip, p->d_partials, s);
}

int cpct_launch_adj_c(cpct_plan* p, const float2* d_sino_c, float* d_img, cudaStream_t s) {
  return launch_adj_impl(p, reinterpret_cast<const float*>(d_sino_c), d_img, true, 0.f, nullptr, p->d_partials, s);
}

// ---------------------------------------------------------------------------
// Allocation-free adjoint: the same operator as radon_adj, with the spread's
// only per-call scratch (the partial tiles of split heavy tiles) in a fixed
// static device array instead of plan memory.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxSlots = CPCT_NOALLOC_MAX_SLOTS;
constexpr int kNoAllocMaxDevices = 64;

// Every device that loads this library holds this array until the process
// exits.  Host code must not use its name as a device address: the device
// address is looked up per device with cudaGetSymbolAddress below.
static __device__ __align__(256) float2 g_noalloc_partials[(size_t)kNoAllocMaxSlots * 1024];

std::mutex g_noalloc_mutex;
float2* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// device address of g_noalloc_partials on the current device (looked up once
// per device, with that device current); nullptr on failure
float2* noalloc_scratch(int* status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    *status = CPCT_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr) {
      *status = CPCT_ECUDA;
      return nullptr;
    }
    g_noalloc_ptr[dev] = static_cast<float2*>(ptr);
  }
  *status = CPCT_OK;
  return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" int radon_adj_noalloc(cpct_plan* p, const float* d_sino, float* d_img, cudaStream_t s) {
  if (!p || !d_sino || !d_img) return CPCT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_sino) & 15u) || (reinterpret_cast<uintptr_t>(d_img) & 15u)) return CPCT_EINVAL;
  // the plan's split bins need more partial-tile space than the array holds
  if (p->partial_elems > (long long)kNoAllocMaxSlots * 1024) return CPCT_EINVAL;
  int status = CPCT_OK;
  float2* partials = noalloc_scratch(&status);
  if (!partials) return status;
  // the same kernels, in the same order and with the same profiling
  // brackets, as radon_adj; only the partial tiles live elsewhere
  return launch_adj_impl(p, d_sino, d_img, false, 0.f, nullptr, partials, s);
}
