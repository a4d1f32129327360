// Shared-memory Stockham FFT used by every transform of the Radon operator
// (section "fast radon transform": the 2D FFT on the oversampled grid and the
// 1D FFTs along the rays).
//
// One FFT of length N = 2^LOGN lives in shared memory in natural order with a
// padded index (q + q/16, so that the strided stores of the radix-16 passes
// are bank-conflict free).  T = N/E threads cooperate; in every pass each
// thread loads E values into registers, applies the inter-pass twiddles and
// radix-R DFTs (R = 16, last pass 2..16) and writes the Stockham
// self-sorting output back.  Twiddles come from a per-pass table laid out
// [m-1][j] so that consecutive threads read consecutive entries (built in FP64
// by the plan); a DFT reads three entries and forms the other powers.  Several FFTs run side by side in one CTA; every thread of the
// CTA must call run() (it contains __syncthreads()).
#pragma once

#include "common.cuh"

namespace cpct {

__device__ __forceinline__ int fpad(int q) { return q + (q >> 4); }

// multiply by exp(DIR * 2 pi i idx / 16), idx in [0, 8); idx is a
// compile-time constant after unrolling, so the switch folds away
template <int DIR>
__device__ __forceinline__ float2 tw16(float2 v, int idx) {
  const float c1 = 0.92387953251128675613f;  // cos(pi/8)
  const float s1 = 0.38268343236508977173f;  // sin(pi/8)
  const float r2 = 0.70710678118654752440f;  // cos(pi/4)
  const float d = (float)DIR;
  switch (idx) {
    case 0: return v;
    case 1: return cmul(v, make_float2(c1, d * s1));
    case 2: return cmul(v, make_float2(r2, d * r2));
    case 3: return cmul(v, make_float2(s1, d * c1));
    case 4: return make_float2(-d * v.y, d * v.x);
    case 5: return cmul(v, make_float2(-s1, d * c1));
    case 6: return cmul(v, make_float2(-r2, d * r2));
    default: return cmul(v, make_float2(-c1, d * s1));
  }
}

__host__ __device__ constexpr int bitrev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// in-register DFT of R = 2^LR points, natural order in and out:
// X[m'] = sum_m x[m] exp(DIR 2 pi i m m' / R)  (radix-2 decimation in frequency)
template <int LR, int DIR>
__device__ __forceinline__ void dft_reg(float2* x) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int start = 0; start < R; start += 2 * span) {
#pragma unroll
      for (int k = 0; k < span; ++k) {
        float2 a = x[start + k], b = x[start + k + span];
        x[start + k] = cadd(a, b);
        x[start + k + span] = tw16<DIR>(csub(a, b), (8 * k) / span);
      }
    }
  }
  float2 y[R];
#pragma unroll
  for (int i = 0; i < R; ++i) y[bitrev(i, LR)] = x[i];
#pragma unroll
  for (int i = 0; i < R; ++i) x[i] = y[i];
}

// PIN: the input is zero outside the circular window [-N/4, N/4) (a signal
// of N/2 values zero-padded to N); in the first pass (radix R >= 4) those
// zeros are exactly the inputs m = R/4 .. 3R/4-1 of every DFT, which are
// then neither loaded nor computed on (constant zeros fold away), and the
// caller need not write them.  POUT: only the outputs in [-N/4, N/4) are needed; the last pass
// stores only the outputs m < R/4 and m >= 3R/4 of every DFT, and the others
// are left unwritten.
template <int LOGN, int E, int DIR, bool PIN = false, bool POUT = false>
struct SmemFFT {
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / E;  // threads per FFT
  // buffers of the FFTs of one CTA start 4 complex values (two 16-byte bank
  // groups) apart modulo 128 bytes: reads of one index from several FFTs
  // fall in distinct banks
  static constexpr int PADN = N + (N >> 4) + 4;
  static constexpr int NPASS = fft_npass(LOGN);
  static_assert(E >= 16 && (N % E) == 0, "E must be >= 16 and divide N");

  // One Stockham pass P.  SRCG (first pass only): the R inputs of every DFT
  // come from ld(q), q = i + m N/R, instead of the buffer -- consecutive
  // threads read consecutive q, so a caller reading global memory reads it
  // coalesced, and no barrier separates the reads from the buffer writes.
  // DSTG (last pass only): output k = i + m N/R goes to st(k, value) instead
  // of the buffer (natural order, consecutive threads at consecutive k), and
  // no barrier follows.
  template <int P, bool SRCG, bool DSTG, class LD, class ST>
  __device__ static __forceinline__ void pass(float2* buf, const float2* __restrict__ tw, int t, const LD& ld,
                                              const ST& st) {
    constexpr int LR = fft_lr(LOGN, P);
    constexpr int R = 1 << LR;
    constexpr int L = 1 << fft_ll(P);
    constexpr int NB = E / R;
    static_assert(E % R == 0, "radix must divide E");
    static_assert(!SRCG || P == 0, "only the first pass reads through ld");
    static_assert(!DSTG || P == NPASS - 1, "only the last pass writes through st");
    // inter-pass twiddles w^m = exp(DIR 2 pi i m j / (R L)), m = 1..R-1: the
    // table entries for m = 1, 4, 8 (built in FP64) are loaded before the
    // barrier, the other powers are products of at most four of them
    float2 w1[NB], w4[NB], w8[NB];
    if (L > 1) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = (t + b * T) & (L - 1);
        const float2* twp = tw + fft_tw_offset(LOGN, P) + j;
        w1[b] = __ldg(&twp[0]);
        if (R > 4) w4[b] = __ldg(&twp[3 * L]);
        if (R > 8) w8[b] = __ldg(&twp[7 * L]);
      }
    }
    float2 v[E];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = t + b * T;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (PIN && R >= 4 && P == 0 && m >= R / 4 && m < 3 * R / 4) v[b * R + m] = make_float2(0.f, 0.f);
        else if constexpr (SRCG) v[b * R + m] = ld(i + m * (N / R));
        else v[b * R + m] = buf[fpad(i + m * (N / R))];
      }
    }
    // in place: every read of the pass before any write (a pass that reads
    // through ld or writes through st shares nothing with the buffer)
    if constexpr (!SRCG && !DSTG) __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = t + b * T;
      const int j = i & (L - 1);
      float2* x = &v[b * R];
      if (L > 1) {
        float2 w[R];
        w[1] = w1[b];
        if (DIR > 0) w[1].y = -w[1].y;
        if (R > 2) w[2] = cmul(w[1], w[1]);
        if (R > 3) w[3] = cmul(w[2], w[1]);
        if (R > 4) {
          w[4] = w4[b];
          if (DIR > 0) w[4].y = -w[4].y;
#pragma unroll
          for (int m = 5; m < 8 && m < R; ++m) w[m] = cmul(w[4], w[m - 4]);
        }
        if (R > 8) {
          w[8] = w8[b];
          if (DIR > 0) w[8].y = -w[8].y;
#pragma unroll
          for (int m = 9; m < R; ++m) w[m] = cmul(w[8], w[m - 8]);
        }
#pragma unroll
        for (int m = 1; m < R; ++m) x[m] = cmul(x[m], w[m]);
      }
      dft_reg<LR, DIR>(x);
      const int base = (i - j) * R + j;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        // (for R >= 4 the outputs i + m N/R, i < N/R, outside [-N/4, N/4)
        // are exactly m = R/4 .. 3R/4-1; a radix-2 last pass writes all of
        // them to the buffer and hands only the kept ones to st)
        if (POUT && R >= 4 && P == NPASS - 1 && m >= R / 4 && m < 3 * R / 4) continue;
        if constexpr (DSTG) {
          // st() only ever sees kept outputs: a radix-2 last pass checks k
          const int k = base + m * L;
          if (POUT && R < 4 && k >= N / 4 && k < 3 * N / 4) continue;
          st(k, x[m]);
        } else {
          buf[fpad(base + m * L)] = x[m];
        }
      }
    }
    if constexpr (!DSTG) __syncthreads();
  }

  // after_first() runs once the first pass is complete in every thread (the
  // first pass ends with a barrier when more passes follow): from then on
  // the source that ld() read may be overwritten
  template <int P, bool SRCG, bool DSTG, class LD, class ST, class AF>
  __device__ static __forceinline__ void passes(float2* buf, const float2* __restrict__ tw, int t, const LD& ld,
                                                const ST& st, const AF& after_first) {
    constexpr bool last = P + 1 == NPASS;
    pass<P, SRCG && P == 0, DSTG && last>(buf, tw, t, ld, st);
    if constexpr (P == 0) after_first();
    if constexpr (!last) passes<P + 1, SRCG, DSTG>(buf, tw, t, ld, st, after_first);
  }

  struct NoLoad {
    __device__ float2 operator()(int) const { return make_float2(0.f, 0.f); }
  };
  struct NoStore {
    __device__ void operator()(int, float2) const {}
  };
  struct NoHook {
    __device__ void operator()() const {}
  };

  // In-place transform of buf[fpad(q)], q = 0..N-1 (unnormalised):
  // DIR = -1: X[k] = sum_q x[q] exp(-2 pi i k q / N); DIR = +1: conjugate kernel.
  // Every thread of the CTA must call it (it contains __syncthreads()), so
  // callers give each thread a valid t.
  __device__ static __forceinline__ void run(float2* buf, const float2* __restrict__ tw, int t) {
    passes<0, false, false>(buf, tw, t, NoLoad(), NoStore(), NoHook());
  }

  // The same transform with the input read through ld(q) in the first pass
  // (x[q] = ld(q); with PIN only q outside [N/4, 3N/4) are asked for) and,
  // with DSTG, the output handed to st(k, X[k]) by the last pass (with POUT
  // only k outside [N/4, 3N/4)); buf is then scratch of N + N/16 values.
  // The input never visits shared memory, and with DSTG neither does the
  // output: NPASS - 1 shared-memory round trips instead of NPASS + 1 for a
  // staged input and output, and 2 NPASS - 3 barriers instead of 2 NPASS + 1
  // (3 instead of 7 for three passes).  Every thread of the CTA must call
  // it.  Without DSTG the output is in buf after the call, as with run(),
  // and the call ends with a barrier.
  template <bool DSTG, class LD, class ST>
  __device__ static __forceinline__ void run_io(float2* buf, const float2* __restrict__ tw, int t, const LD& ld,
                                                const ST& st) {
    passes<0, true, DSTG>(buf, tw, t, ld, st, NoHook());
  }
  // run_io with after_first() called when every thread has finished the
  // first pass, i.e. has read all of its input through ld() (needs NPASS >= 2)
  template <bool DSTG, class LD, class ST, class AF>
  __device__ static __forceinline__ void run_io(float2* buf, const float2* __restrict__ tw, int t, const LD& ld,
                                                const ST& st, const AF& after_first) {
    static_assert(NPASS >= 2, "the first pass must end with a barrier");
    passes<0, true, DSTG>(buf, tw, t, ld, st, after_first);
  }
};

}  // namespace cpct
