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

  template <int P>
  __device__ static __forceinline__ void pass(float2* buf, const float2* __restrict__ tw, int t) {
    constexpr int LR = fft_lr(LOGN, P);
    constexpr int R = 1 << LR;
    constexpr int L = 1 << fft_ll(P);
    constexpr int NB = E / R;
    static_assert(E % R == 0, "radix must divide E");
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
        else v[b * R + m] = buf[fpad(i + m * (N / R))];
      }
    }
    __syncthreads();
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
        // are exactly m = R/4 .. 3R/4-1; a radix-2 last pass stores all)
        if (POUT && R >= 4 && P == NPASS - 1 && m >= R / 4 && m < 3 * R / 4) continue;
        buf[fpad(base + m * L)] = x[m];
      }
    }
    __syncthreads();
  }

  template <int P>
  __device__ static __forceinline__ void passes(float2* buf, const float2* __restrict__ tw, int t) {
    pass<P>(buf, tw, t);
    if constexpr (P + 1 < NPASS) passes<P + 1>(buf, tw, t);
  }

  // In-place transform of buf[fpad(q)], q = 0..N-1 (unnormalised):
  // DIR = -1: X[k] = sum_q x[q] exp(-2 pi i k q / N); DIR = +1: conjugate kernel.
  // Threads with t >= T must still call (pass t = -1 ... no: every thread of
  // the CTA must reach the barriers), so callers give each thread a valid t.
  __device__ static __forceinline__ void run(float2* buf, const float2* __restrict__ tw, int t) {
    passes<0>(buf, tw, t);
  }
};

}  // namespace cpct
