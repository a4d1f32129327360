// Learned warm start: the convolutional denoiser (U-Net) and its training.
//
// The paper has no learned component.  The network maps a filtered
// back-projection of the data to a starting point of SPGL1 (the solver of the
// paper's L1 problem, section "Introduction"); its function is fixed in the
// C header (cpct_unet_*).  Layout and precision:
//   * activations and their gradients: FP32, NHWC (channel fastest);
//   * weights: FP32 master copy (Adam), BF16 copies in [Cout][3][3][Cin]
//     (forward) and [Cin][3][3][Cout] with flipped taps (data gradient);
//   * every 3x3 convolution is an implicit GEMM with BF16 operands and FP32
//     accumulation.  Forward and data-gradient convolutions run on the
//     fifth-generation tensor cores (k_conv3x3_tc: TMA operand boxes,
//     tcgen05.mma into tensor memory, persistent and warp-specialized);
//     they read BF16 copies that the producers of their inputs write beside
//     the FP32 tensors.  Weight gradients run on mma.sync m16n8k16 from the
//     same BF16 copies.  The FP32-staging mma.sync kernels remain for shapes
//     the others do not take;
//   * the first layer (one input channel) is a direct kernel; for its weight
//     gradient the training pass stores the input with 32 channels
//     (channel 0 = image), so every GEMM reduction chunk is 32 channels of
//     one tap;
//   * inference (cpct_unet_forward) skips the FP32 copies that only the
//     backward pass reads, and computes the 1x1 head in the last
//     convolution's epilogue.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int kCT = 256;     // threads of the convolution kernels
constexpr int kBM = 128;     // pixels per forward tile
constexpr int kBK = 32;      // reduction chunk: 32 channels of one tap
constexpr int kEW = 256;     // threads of elementwise kernels

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// A tile row of 32 BF16 (64 B = four 16-byte chunks); chunk c of row r is
// stored at chunk c ^ ((r >> 1) & 3): the eight rows an ldmatrix phase reads
// then fall in eight distinct 16-byte bank groups
__device__ __forceinline__ int sw64(int r, int c) { return r * 4 + (c ^ ((r >> 1) & 3)); }

struct ConvArgs {
  // input activations: channels [0, C1) from x1, [C1, C1 + C2) from x2
  const float* x1;
  const float* x2;
  int C1, C2;
  const __nv_bfloat16* W;  // [Cout][3][3][Cin] (Cin = C1 + C2)
  const float* bias;       // [Cout] or null
  // output: channels [0, O1) to y1 (stride O1), [O1, Cout) to y2
  float* y1;
  float* y2;
  // optional ReLU masks of the outputs (same layout as y1 / y2): an output
  // element is zeroed where its mask is not positive (data gradients land
  // on ReLU outputs as pre-activation gradients)
  const float* om1;
  const float* om2;
  // forward pass: BF16 copies of the inputs (read instead of x1 / x2 by the
  // BF16-input kernel) and of the output (written beside y1 if given)
  const __nv_bfloat16* xb1;
  const __nv_bfloat16* xb2;
  __nv_bfloat16* yb1;
  int O1, Cout;
  int relu;                // apply max(., 0) in the epilogue
  int B, H, Wd;            // batch, height, width
  int* err;                // device error flag (bounded waits of the tensor-memory kernel)
  // fused 1x1 head (tensor-memory kernel, one N tile covering Cout): if
  // head_out is set, head_out[p] = head_x[p] + head_b[0] + sum_c head_w[c] y[p, c]
  // (FP32, channel order)
  const float* head_w;
  const float* head_b;
  const float* head_x;
  float* head_out;
};

constexpr int kStages = 3;  // cp.async pipeline depth of the convolution GEMMs

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0));
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// FP32 staging rows of 32 channels padded to 36 floats (144 B): rows start 4
// banks apart, so the conversion's 16-byte reads of 8 threads (4 rows x 2
// halves) fall in 32 distinct banks
constexpr int kAfLd = kBK + 4;

template <int BN>
constexpr size_t conv_smem() {
  return (size_t)kStages * (kBM * kAfLd * 4 + BN * kBK * 2) + kBM * kBK * 2;
}

// Implicit-GEMM 3x3 convolution (zero padding 1): M = B*H*W pixels, N = Cout,
// K = 9 * Cin in chunks of 32 channels of one tap.  256 threads, tile
// 128 pixels x BN output channels, warps 4 (M) x 2 (N).  A 3-stage cp.async
// pipeline stages the FP32 activation chunk (zero-filled outside the image)
// and the BF16 weight chunk; each chunk's activations are converted once to a
// swizzled BF16 tile that ldmatrix feeds to mma.sync.
template <int BN>
__global__ void __launch_bounds__(kCT) k_conv3x3(const ConvArgs a) {
  constexpr int WN = BN / 2;        // warp tile N (32 or 16)
  constexpr int NT = WN / 8;        // n8 tiles per warp
  extern __shared__ __align__(128) unsigned char smraw[];
  float* Af = reinterpret_cast<float*>(smraw);                                     // [kStages][kBM][kAfLd]
  uint32_t* sB = reinterpret_cast<uint32_t*>(smraw + (size_t)kStages * kBM * kAfLd * 4);  // [kStages][BN * kBK / 2]
  uint32_t* sA = sB + kStages * BN * kBK / 2;                                   // [kBM * kBK / 2]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;
  const int HW = a.H * a.Wd, P = a.B * HW;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int Cin = a.C1 + a.C2, cchunks = Cin / kBK, nk = 9 * cchunks;

  // A copies: this thread's 16-byte chunk c16 of rows r0 + 32 i, i = 0..3
  const int c16 = tid & 7, r0 = tid >> 3;
  int py[4], px[4], pb[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pm = m0 + r0 + 32 * i;
    pb[i] = -1;
    if (pm < P) {
      pb[i] = pm / HW;
      const int r = pm - pb[i] * HW;
      py[i] = r / a.Wd;
      px[i] = r - py[i] * a.Wd;
    }
  }
  auto load_stage = [&](int kc, int st) {
    const int tap = kc / cchunks, ci0 = (kc - tap * cchunks) * kBK;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const float* base = ci0 < a.C1 ? a.x1 : a.x2;
    const int cs = ci0 < a.C1 ? a.C1 : a.C2, co = (ci0 < a.C1 ? ci0 : ci0 - a.C1) + 4 * c16;
    float* dst = Af + (size_t)st * kBM * kAfLd;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int sy = py[i] + dy, sx = px[i] + dx;
      const bool ok = pb[i] >= 0 && sy >= 0 && sy < a.H && sx >= 0 && sx < a.Wd;
      const float* src = ok ? base + (((size_t)pb[i] * a.H + sy) * a.Wd + sx) * cs + co : base;
      cp_async16_zfill(smem_u32(dst + (r0 + 32 * i) * kAfLd + 4 * c16), src, ok);
    }
    if (tid < BN * 4) {
      const int r = tid >> 2, c = tid & 3;
      const __nv_bfloat16* src = a.W + ((size_t)(n0 + r) * 9 + tap) * Cin + ci0 + c * 8;
      cp_async16(smem_u32(sB + (size_t)st * BN * kBK / 2 + 4 * sw64(r, c)), src);
    }
  };
  // FP32 chunk -> swizzled BF16 tile: thread -> (row, 16-channel half)
  auto convert = [&](int st) {
    const int row = tid >> 1, half = tid & 1;
    const float4* src = reinterpret_cast<const float4*>(Af + (size_t)st * kBM * kAfLd + row * kAfLd + half * 16);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float4 u = src[2 * c], v = src[2 * c + 1];
      uint4 q;
      q.x = pack_bf16(u.x, u.y);
      q.y = pack_bf16(u.z, u.w);
      q.z = pack_bf16(v.x, v.y);
      q.w = pack_bf16(v.z, v.w);
      *reinterpret_cast<uint4*>(sA + 4 * sw64(row, half * 2 + c)) = q;
    }
  };

  float acc[2][NT][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (st < nk) load_stage(st, st);
    cp_async_commit();
  }
  for (int kc = 0; kc < nk; ++kc) {
    const int cur = kc % kStages;
    cp_async_wait<kStages - 2>();
    __syncthreads();  // chunk kc landed for every thread; chunk kc-1 fully consumed
    convert(cur);
    {
      const int nx = kc + kStages - 1;
      if (nx < nk) load_stage(nx, nx % kStages);
      cp_async_commit();
    }
    __syncthreads();  // BF16 tile of chunk kc visible
    const uint32_t* sBc = sB + (size_t)cur * BN * kBK / 2;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {  // two k16 steps per chunk
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + (lane & 15);
        const int c = ks * 2 + (lane >> 4);
        ldsm_x4(smem_u32(sA + 4 * sw64(r, c)), af[i][0], af[i][1], af[i][2], af[i][3]);
      }
#pragma unroll
      for (int j = 0; j < NT; j += 2) {
        // two n8 tiles: lanes 0-7 n 0-7 k0, 8-15 n 0-7 k8, 16-23 n 8-15 k0, 24-31 n 8-15 k8
        const int r = wn * WN + j * 8 + (lane & 7) + ((lane >> 4) << 3);
        const int c = ks * 2 + ((lane >> 3) & 1);
        uint32_t b0, b1, b2, b3;
        ldsm_x4(smem_u32(sBc + 4 * sw64(r, c)), b0, b1, b2, b3);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][j], af[i], b0, b1);
          mma_bf16(acc[i][j + 1], af[i], b2, b3);
        }
      }
    }
  }
  cp_async_wait<0>();
  // epilogue: rows lane/4 and lane/4 + 8, columns 2 (lane % 4) + {0, 1}
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
      if (m >= P) continue;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int n = n0 + wn * WN + j * 8 + 2 * (lane & 3);
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (a.bias) {
          v0 += a.bias[n];
          v1 += a.bias[n + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        const bool first = n < a.O1;
        const size_t off = first ? (size_t)m * a.O1 + n : (size_t)m * (a.Cout - a.O1) + (n - a.O1);
        const float* mk = first ? a.om1 : a.om2;
        if (mk) {
          const float2 mv = *reinterpret_cast<const float2*>(mk + off);
          v0 = mv.x > 0.f ? v0 : 0.f;
          v1 = mv.y > 0.f ? v1 : 0.f;
        }
        *reinterpret_cast<float2*>((first ? a.y1 : a.y2) + off) = make_float2(v0, v1);
        if (a.yb1 && first) *reinterpret_cast<uint32_t*>(a.yb1 + off) = pack_bf16(v0, v1);
      }
    }
}

constexpr int kStagesB = 4;  // pipeline depth of the BF16-input forward GEMM

// pixels per tile of the BF16-input kernel: every warp computes 32 x 32
// (4 x 2 warps of 128 x 64, or 8 x 1 warps of 256 x 32 for 32 channels)
template <int BN>
constexpr int bm_b16() { return 8192 / BN; }

template <int BN>
constexpr size_t conv_smem_b16() {
  return (size_t)kStagesB * (bm_b16<BN>() * kBK * 2 + BN * kBK * 2);
}

// The forward convolution reading the BF16 copies of its inputs: a 4-stage
// cp.async pipeline copies the operand tiles (zero-filled outside the image)
// straight into the swizzled layout that ldmatrix reads; no conversion, one
// barrier per chunk.  Results equal k_conv3x3's (the same round-to-nearest
// BF16 operands, the same accumulation order).
template <int BN>
__global__ void __launch_bounds__(kCT) k_conv3x3_b16(const ConvArgs a) {
  constexpr int BM = bm_b16<BN>();
  constexpr int WARPS_M = BM / 32;  // 4 or 8
  constexpr int WN = 32;
  constexpr int NT = WN / 8;
  constexpr int RPT = BM / 64;      // A rows per thread
  extern __shared__ __align__(128) unsigned char smraw[];
  uint32_t* sA = reinterpret_cast<uint32_t*>(smraw);      // [kStagesB][BM * kBK / 2]
  uint32_t* sB = sA + kStagesB * BM * kBK / 2;            // [kStagesB][BN * kBK / 2]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % WARPS_M, wn = warp / WARPS_M;
  const int HW = a.H * a.Wd, P = a.B * HW;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int Cin = a.C1 + a.C2, cchunks = Cin / kBK, nk = 9 * cchunks;
  // A copies: 16-byte chunk c (0..3) of rows r0 + 64 i
  const int c = tid & 3, r0 = tid >> 2;
  int py[RPT], px[RPT], pb[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int pm = m0 + r0 + 64 * i;
    pb[i] = -1;
    if (pm < P) {
      pb[i] = pm / HW;
      const int r = pm - pb[i] * HW;
      py[i] = r / a.Wd;
      px[i] = r - py[i] * a.Wd;
    }
  }
  auto load_stage = [&](int kc, int st) {
    const int tap = kc / cchunks, ci0 = (kc - tap * cchunks) * kBK;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const __nv_bfloat16* base = ci0 < a.C1 ? a.xb1 : a.xb2;
    const int cs = ci0 < a.C1 ? a.C1 : a.C2, co = (ci0 < a.C1 ? ci0 : ci0 - a.C1) + 8 * c;
    uint32_t* dA = sA + (size_t)st * BM * kBK / 2;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int sy = py[i] + dy, sx = px[i] + dx;
      const bool ok = pb[i] >= 0 && sy >= 0 && sy < a.H && sx >= 0 && sx < a.Wd;
      const __nv_bfloat16* src = ok ? base + (((size_t)pb[i] * a.H + sy) * a.Wd + sx) * cs + co : base;
      cp_async16_zfill(smem_u32(dA + 4 * sw64(r0 + 64 * i, c)), src, ok);
    }
    if (tid < BN * 4) {
      const int r = tid >> 2, cc = tid & 3;
      const __nv_bfloat16* src = a.W + ((size_t)(n0 + r) * 9 + tap) * Cin + ci0 + cc * 8;
      cp_async16(smem_u32(sB + (size_t)st * BN * kBK / 2 + 4 * sw64(r, cc)), src);
    }
  };

  float acc[2][NT][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
#pragma unroll
  for (int st = 0; st < kStagesB - 1; ++st) {
    if (st < nk) load_stage(st, st);
    cp_async_commit();
  }
  for (int kc = 0; kc < nk; ++kc) {
    const int cur = kc % kStagesB;
    cp_async_wait<kStagesB - 2>();
    __syncthreads();  // chunk kc landed for every thread; chunk kc-1 fully consumed
    {
      const int nx = kc + kStagesB - 1;
      if (nx < nk) load_stage(nx, nx % kStagesB);
      cp_async_commit();
    }
    const uint32_t* sAc = sA + (size_t)cur * BM * kBK / 2;
    const uint32_t* sBc = sB + (size_t)cur * BN * kBK / 2;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + (lane & 15);
        const int cc = ks * 2 + (lane >> 4);
        ldsm_x4(smem_u32(sAc + 4 * sw64(r, cc)), af[i][0], af[i][1], af[i][2], af[i][3]);
      }
#pragma unroll
      for (int j = 0; j < NT; j += 2) {
        const int r = wn * WN + j * 8 + (lane & 7) + ((lane >> 4) << 3);
        const int cc = ks * 2 + ((lane >> 3) & 1);
        uint32_t b0, b1, b2, b3;
        ldsm_x4(smem_u32(sBc + 4 * sw64(r, cc)), b0, b1, b2, b3);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][j], af[i], b0, b1);
          mma_bf16(acc[i][j + 1], af[i], b2, b3);
        }
      }
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
      if (m >= P) continue;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int n = n0 + wn * WN + j * 8 + 2 * (lane & 3);
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (a.bias) {
          v0 += a.bias[n];
          v1 += a.bias[n + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        const size_t off = (size_t)m * a.Cout + n;
        if (a.y1) *reinterpret_cast<float2*>(a.y1 + off) = make_float2(v0, v1);
        if (a.yb1) *reinterpret_cast<uint32_t*>(a.yb1 + off) = pack_bf16(v0, v1);
      }
    }
}

// Persistent warp-specialized forward convolution on the tensor cores.
constexpr int kTcLag = 2;         // chunks a cp.async producer keeps in flight before signalling one
constexpr long long kTcWait = 2000000000LL;  // bounded waits (~1 s at 2 GHz)

// threads: warps 0-3 epilogue, then the producers (4 warps of cp.async
// copies, or one warp whose lane 0 issues TMA loads), then one MMA warp
template <bool TMA>
constexpr int tc_threads() {
  return TMA ? 6 * 32 : 9 * 32;
}

// shared-memory budget of the stage ring: two CTAs per SM for N tiles up to
// 128 columns, one for 256
// (at least 3 stages for TMA, kTcLag + 2 for cp.async producers)
template <int BN, int KC, bool TMA>
constexpr int tc_stages() {
  constexpr int budget = (BN >= 256 ? 192 : 100) * 1024, per = (128 + BN) * KC * 2, lo = TMA ? 3 : kTcLag + 2;
  return budget / per > 12 ? 12 : budget / per < lo ? lo : budget / per;
}
template <int BN, int KC, bool TMA>
constexpr size_t conv_smem_tc() {
  return (size_t)tc_stages<BN, KC, TMA>() * (128 + BN) * KC * 2 + 1024;  // + alignment slack
}

// wait on an mbarrier phase; gives up (and raises the CTA's abort flag) after
// kTcWait cycles, or as soon as another role has raised it
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kTcWait) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// Tiles of the TMA path: Wb x Hb pixels of one image (Wb Hb = 128).  The
// operand boxes come from 4-D tensor maps {C, W, H, B} of the BF16 input
// copies (box {KC, Wb, Hb, 1}: zero fill outside the image is the
// convolution's padding) and a 2-D map {9 Cin, Cout} of the weights (box
// {KC, BN}), with the 128-byte (KC = 64) or 64-byte (KC = 32) swizzle: each
// pixel / output channel is one row of KC channels, the K-major swizzled
// layout the MMA descriptors name.
struct TcMaps {
  CUtensorMap a1, a2, w;
  int Wb, Hb;
};

// Implicit GEMM: M = 128 pixels per tile, N = BN output channels, K = 9 Cin
// in chunks of KC (32 or 64) channels of one tap (tap-major, then channel).
// Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... (N tile
// fastest); the chunks of all its tiles flow through one ring of S stages:
// * producers fill a stage with a chunk's BF16 operand tiles in a K-major
//   layout and signal its "full" barrier: TMA (one thread, swizzled rows,
//   the barrier completes on the transaction bytes), or cp.async copies by 128
//   threads (zero-filled outside the image; element (row, k) at byte
//   (row / 8) * 16 KC + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2, eight
//   consecutive threads on eight consecutive rows), each thread arriving
//   once its copies of the chunk have landed (kTcLag chunks later) and were
//   fenced for the async proxy;
// * one MMA thread waits for "full", issues KC / 16 MMAs (K = 16) into one
//   of two FP32 accumulators in tensor memory and commits them to the
//   stage's "empty" barrier (the producers refill the stage after it), and
//   after a tile's last chunk to the accumulator's "tfull" barrier;
// * the epilogue (warps 0-3, warp w on tile rows 32 w .. 32 w + 31) waits for
//   "tfull", reads the accumulator with tcgen05.ld, adds the bias, applies
//   the ReLU, writes FP32 and BF16 outputs and releases the accumulator
//   ("tempty"), so that a tile's epilogue overlaps the next tile's MMAs.
// Every wait is bounded; on expiry the CTA's abort flag stops all roles, the
// MMA thread waits (bounded) for its MMAs in flight, and the error flag is
// raised before the tensor memory is freed.
template <int BN, int KC, bool TMA>
__global__ void __launch_bounds__(tc_threads<TMA>(), BN >= 256 ? 1 : 2)
    k_conv3x3_tc(const ConvArgs a, const __grid_constant__ TcMaps maps) {
  constexpr int S = tc_stages<BN, KC, TMA>();
  constexpr int NCH = KC / 8;                  // 16-byte pieces per row
  constexpr int APT = NCH;                     // A pieces per cp.async producer thread
  constexpr int RSTEP = 128 / (8 * NCH);       // 8-row groups between a thread's pieces
  constexpr uint32_t A_BYTES = 128 * KC * 2, B_BYTES = BN * KC * 2;
  // descriptors: swizzled rows of KC channels (TMA) or core matrices (cp.async)
  constexpr uint32_t LAYOUT = TMA ? (KC == 64 ? cpct::kTcSwizzle128 : cpct::kTcSwizzle64) : cpct::kTcNoSwizzle;
  constexpr uint32_t LBO = TMA ? 16 : 128, SBO = 16 * KC;     // SBO: 8 rows of KC channels either way
  constexpr uint32_t KSTEP = TMA ? 32 : 256;                  // start advance per K = 16
  constexpr int MMA_WARP = TMA ? 5 : 8;
  extern __shared__ unsigned char smtc_raw[];
  // 1024-byte aligned stage ring
  unsigned char* smtc = smtc_raw + ((1024 - (smem_u32(smtc_raw) & 1023)) & 1023);
  unsigned char* sA = smtc;                           // [S][A_BYTES]
  unsigned char* sB = smtc + (size_t)S * A_BYTES;     // [S][B_BYTES]
  __shared__ __align__(8) uint64_t full[S], empty[S], tfull[2], tempty[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HW = a.H * a.Wd, P = a.B * HW;
  const int ntn = a.Cout / BN, ntiles = ((P + 127) / 128) * ntn;
  const int Cin = a.C1 + a.C2, cchunks = Cin / KC, nk = 9 * cchunks;
  const int txn = TMA ? a.Wd / maps.Wb : 1, tyn = TMA ? a.H / maps.Hb : 1;  // TMA tiles per image row / column
  if (warp == MMA_WARP) {
    cpct::tc_alloc(smem_u32(&tslot), 2 * BN);
    cpct::tc_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], TMA ? 1 : 128);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 128);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  cpct::tc_fence_before();
  __syncthreads();
  cpct::tc_fence_after();
  const uint32_t tbase = tslot;

  if (TMA && warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int g = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int mt = t / ntn, n0 = (t % ntn) * BN;
        const int b = mt / (txn * tyn), rem = mt - b * (txn * tyn);
        const int y0 = (rem / txn) * maps.Hb, x0 = (rem % txn) * maps.Wb;
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int st = g % S;
          if (g >= S && !tc_wait(&empty[st], (uint32_t)(((g / S) - 1) & 1), abort)) {
            ok = false;
            break;
          }
          const int tap = kc / cchunks, ci0 = (kc - tap * cchunks) * KC;
          const int dy = tap / 3 - 1, dx = tap % 3 - 1;
          mbar_arrive_expect_tx(&full[st], A_BYTES + B_BYTES);
          const bool first = ci0 < a.C1;
          cpct::tma_load_4d(smem_u32(sA + (size_t)st * A_BYTES), first ? &maps.a1 : &maps.a2,
                            first ? ci0 : ci0 - a.C1, x0 + dx, y0 + dy, b, &full[st]);
          cpct::tma_load_2d_u32(smem_u32(sB + (size_t)st * B_BYTES), &maps.w, tap * Cin + ci0, n0, &full[st]);
        }
        if (!ok) break;
      }
      // on abort: loads still in flight land before the CTA exits
      if (*abort)
        for (int q = g - S < 0 ? 0 : g - S; q < g; ++q) mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), kTcWait);
    }
    __syncwarp();
  } else if (!TMA && warp >= 4 && warp < 8) {
    // ---------------- cp.async producers ----------------
    const int pt = tid - 128, c = (pt >> 3) % NCH;
    int g = 0;  // chunks issued by this CTA
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int m0 = (t / ntn) * 128, n0 = (t % ntn) * BN;
      int py[APT], px[APT], pb[APT];
#pragma unroll
      for (int i = 0; i < APT; ++i) {
        const int pm = m0 + 8 * (i * RSTEP + pt / (8 * NCH)) + (pt & 7);
        pb[i] = -1;
        if (pm < P) {
          pb[i] = pm / HW;
          const int q = pm - pb[i] * HW;
          py[i] = q / a.Wd;
          px[i] = q - py[i] * a.Wd;
        }
      }
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int st = g % S;
        if (g >= S && !tc_wait(&empty[st], (uint32_t)(((g / S) - 1) & 1), abort)) break;
        const int tap = kc / cchunks, ci0 = (kc - tap * cchunks) * KC;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const __nv_bfloat16* base = ci0 < a.C1 ? a.xb1 : a.xb2;
        const int cs = ci0 < a.C1 ? a.C1 : a.C2, co = (ci0 < a.C1 ? ci0 : ci0 - a.C1) + 8 * c;
        unsigned char* dA = sA + (size_t)st * A_BYTES;
#pragma unroll
        for (int i = 0; i < APT; ++i) {
          const int r = 8 * (i * RSTEP + pt / (8 * NCH)) + (pt & 7);
          const int sy = py[i] + dy, sx = px[i] + dx;
          const bool ok = pb[i] >= 0 && sy >= 0 && sy < a.H && sx >= 0 && sx < a.Wd;
          const __nv_bfloat16* src = ok ? base + (((size_t)pb[i] * a.H + sy) * a.Wd + sx) * cs + co : base;
          cp_async16_zfill(smem_u32(dA + (r >> 3) * SBO + c * 128 + (r & 7) * 16), src, ok);
        }
        unsigned char* dB = sB + (size_t)st * B_BYTES;
#pragma unroll
        for (int q = pt; q < BN * NCH; q += 128) {
          const int r = 8 * ((q >> 3) / NCH) + (q & 7), cc = (q >> 3) % NCH;
          const __nv_bfloat16* src = a.W + ((size_t)(n0 + r) * 9 + tap) * Cin + ci0 + cc * 8;
          cp_async16(smem_u32(dB + (r >> 3) * SBO + cc * 128 + (r & 7) * 16), src);
        }
        cp_async_commit();
        if (g >= kTcLag) {
          cp_async_wait<kTcLag>();  // chunk g - kTcLag landed
          cpct::fence_proxy_async_smem();
          cpct::mbar_arrive(&full[(g - kTcLag) % S]);
        }
      }
      if (*abort) break;
    }
    cp_async_wait<0>();
    cpct::fence_proxy_async_smem();
    for (int q = g - kTcLag < 0 ? 0 : g - kTcLag; q < g; ++q) cpct::mbar_arrive(&full[q % S]);
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = cpct::tc_idesc_bf16(128, BN);
      int g = 0, it = 0;
      uint64_t* last = nullptr;  // barrier of the last commit, and its phase
      uint32_t last_par = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        const int acc = it & 1;
        if (it >= 2 && !tc_wait(&tempty[acc], (uint32_t)(((it >> 1) - 1) & 1), abort)) break;
        cpct::tc_fence_after();
        const uint32_t d = tbase + acc * BN;
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int st = g % S;
          if (!tc_wait(&full[st], (uint32_t)((g / S) & 1), abort)) {
            ok = false;
            break;
          }
          cpct::tc_fence_after();
          const uint32_t a0 = smem_u32(sA + (size_t)st * A_BYTES);
          const uint32_t b0 = smem_u32(sB + (size_t)st * B_BYTES);
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk)
            cpct::tc_mma_bf16(d, cpct::tc_smem_desc(a0 + kk * KSTEP, LBO, SBO, LAYOUT),
                              cpct::tc_smem_desc(b0 + kk * KSTEP, LBO, SBO, LAYOUT), idesc, kc > 0 || kk > 0);
          cpct::tc_commit(&empty[st]);
          last = &empty[st];
          last_par = (uint32_t)((g / S) & 1);
        }
        if (!ok) break;
        cpct::tc_commit(&tfull[acc]);
        last = &tfull[acc];
        last_par = (uint32_t)((it >> 1) & 1);
      }
      // MMAs still in flight must finish before the tensor memory is freed
      if (*abort && last) mbar_wait_bounded(last, last_par, kTcWait);
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---------------- epilogue ----------------
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int acc = it & 1;
      if (!tc_wait(&tfull[acc], (uint32_t)((it >> 1) & 1), abort)) break;
      cpct::tc_fence_after();
      const int mt = t / ntn, n0 = (t % ntn) * BN, p = warp * 32 + lane;
      float hs = a.head_out ? a.head_b[0] : 0.f;  // fused head: FP32, channel order
      int m;
      if (TMA) {
        const int b = mt / (txn * tyn), rem = mt - b * (txn * tyn);
        const int y = (rem / txn) * maps.Hb + p / maps.Wb, x = (rem % txn) * maps.Wb + p % maps.Wb;
        m = (b * a.H + y) * a.Wd + x;
      } else {
        m = mt * 128 + p;
      }
#pragma unroll 1
      for (int j = 0; j < BN / 16; ++j) {
        float v[16];
        cpct::tc_ld16(tbase + ((uint32_t)(warp * 32) << 16) + acc * BN + j * 16, v);
        cpct::tc_wait_ld();
        if (m < P) {
          const int n = n0 + j * 16;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float x = v[i] + (a.bias ? a.bias[n + i] : 0.f);
            v[i] = a.relu ? fmaxf(x, 0.f) : x;
          }
          if (a.head_out) {
#pragma unroll
            for (int i = 0; i < 16; ++i) hs = fmaf(a.head_w[n + i], v[i], hs);
          }
          // channels [0, O1) go to y1 (row stride O1), [O1, Cout) to y2
          // (stride Cout - O1); an optional ReLU mask of the same layout
          // zeroes an output where it is not positive
          const bool first = n < a.O1;
          const size_t off = first ? (size_t)m * a.O1 + n : (size_t)m * (a.Cout - a.O1) + (n - a.O1);
          const float* mk = first ? a.om1 : a.om2;
          if (mk) {
            const float4* mv = reinterpret_cast<const float4*>(mk + off);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float4 q = mv[i];
              v[4 * i] = q.x > 0.f ? v[4 * i] : 0.f;
              v[4 * i + 1] = q.y > 0.f ? v[4 * i + 1] : 0.f;
              v[4 * i + 2] = q.z > 0.f ? v[4 * i + 2] : 0.f;
              v[4 * i + 3] = q.w > 0.f ? v[4 * i + 3] : 0.f;
            }
          }
          float* yo = first ? a.y1 : a.y2;
          if (yo) {
            float4* dst = reinterpret_cast<float4*>(yo + off);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          }
          if (a.yb1 && first) {
            uint4* db = reinterpret_cast<uint4*>(a.yb1 + off);
            db[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                               pack_bf16(v[6], v[7]));
            db[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                               pack_bf16(v[14], v[15]));
          }
        }
      }
      if (a.head_out && m < P) a.head_out[m] = a.head_x[m] + hs;
      cpct::tc_fence_before();
      cpct::mbar_arrive(&tempty[acc]);
    }
  }
  cpct::tc_fence_before();
  __syncthreads();
  if (tid == 0 && abort_flag) atomicOr(a.err, 1);
  if (warp == MMA_WARP) {
    cpct::tc_fence_after();
    cpct::tc_dealloc(tbase, 2 * BN);
  }
}

// swizzled 16-byte chunk index of a row of CPR chunks (CPR = 4 or 8)
template <int CPR>
__device__ __forceinline__ int swz(int r, int c) {
  return CPR == 8 ? r * 8 + (c ^ (r & 7)) : r * 4 + (c ^ ((r >> 1) & 3));
}

struct WgradArgs {
  const float* dz;   // [P][Cout] gradient of the layer's pre-activation
  const float* x1;   // layer input channels [0, C1)
  const float* x2;   // channels [C1, C1 + C2)
  // BF16 copies (read by the BF16 kernel instead of dz, x1, x2)
  const __nv_bfloat16* dzb;
  const __nv_bfloat16* xb1;
  const __nv_bfloat16* xb2;
  int C1, C2, Cout;
  int B, H, Wd;
  int chunks_per_split;  // 32-pixel chunks per split
  float* part;       // [splits][Cout][9][Cin]
};

template <int BM, int BN>
constexpr size_t wgrad_smem() {
  return (size_t)kStages * kBK * (BM + BN) * 4 + (size_t)kBK * (BM + BN) * 2;
}

// Weight gradient dW[co][tap][ci] = sum_p dZ[p][co] X[p + tap][ci] as a GEMM
// with M = Cout, N = 9 Cin (tiles inside one tap), K = pixels, split over
// blockIdx.z.  Both FP32 operand chunks ([pixel][channel], 32 pixels) are
// staged by a 3-stage cp.async pipeline (shifted pixels outside the image
// zero-filled), converted to swizzled BF16 tiles and read with
// ldmatrix.trans.  Warp tile 16 x 16, (BM / 16) x (BN / 16) warps.
template <int BM, int BN>
__global__ void __launch_bounds__((BM / 16) * (BN / 16) * 32) k_conv3x3_wgrad(const WgradArgs a) {
  constexpr int NW_N = BN / 16, NTH = (BM / 16) * NW_N * 32;
  constexpr int CA = BM / 8, CB = BN / 8;  // 16-byte chunks per BF16 row
  extern __shared__ __align__(128) unsigned char smraw[];
  float* Af = reinterpret_cast<float*>(smraw);                 // [kStages][kBK][BM]
  float* Bf = Af + (size_t)kStages * kBK * BM;                 // [kStages][kBK][BN]
  uint32_t* sA = reinterpret_cast<uint32_t*>(Bf + (size_t)kStages * kBK * BN);  // [kBK][BM] bf16
  uint32_t* sB = sA + kBK * BM / 2;                            // [kBK][BN] bf16
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / NW_N, wn = warp % NW_N;
  const int Cin = a.C1 + a.C2, ctiles = Cin / BN;
  const int m0 = blockIdx.x * BM;
  const int tap = blockIdx.y / ctiles, ci0 = (blockIdx.y % ctiles) * BN;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int HW = a.H * a.Wd, P = a.B * HW;
  const int c_begin = blockIdx.z * a.chunks_per_split;
  const int c_end = min(c_begin + a.chunks_per_split, (P + kBK - 1) / kBK);
  const float* xs = ci0 < a.C1 ? a.x1 : a.x2;
  const int xc = ci0 < a.C1 ? a.C1 : a.C2, xo = ci0 < a.C1 ? ci0 : ci0 - a.C1;

  constexpr int NA16 = kBK * BM / 4, NB16 = kBK * BN / 4;  // 16-byte chunks per stage
  auto load_stage = [&](int ch, int st) {
    const int p0 = ch * kBK;
    float* da = Af + (size_t)st * kBK * BM;
    float* db = Bf + (size_t)st * kBK * BN;
    for (int idx = tid; idx < NA16; idx += NTH) {
      const int r = idx / (BM / 4), c4 = idx % (BM / 4), p = p0 + r;
      const bool ok = p < P;
      const float* src = ok ? a.dz + (size_t)p * a.Cout + m0 + 4 * c4 : a.dz;
      cp_async16_zfill(smem_u32(da + r * BM + 4 * c4), src, ok);
    }
    for (int idx = tid; idx < NB16; idx += NTH) {
      const int r = idx / (BN / 4), c4 = idx % (BN / 4), p = p0 + r;
      bool ok = p < P;
      const float* src = xs;
      if (ok) {
        const int b = p / HW, rem = p - b * HW;
        const int py = rem / a.Wd + dy, px = rem % a.Wd + dx;
        ok = py >= 0 && py < a.H && px >= 0 && px < a.Wd;
        if (ok) src = xs + (((size_t)b * a.H + py) * a.Wd + px) * xc + xo + 4 * c4;
      }
      cp_async16_zfill(smem_u32(db + r * BN + 4 * c4), src, ok);
    }
  };
  auto convert = [&](int st) {
    const float* da = Af + (size_t)st * kBK * BM;
    const float* db = Bf + (size_t)st * kBK * BN;
    for (int idx = tid; idx < NA16; idx += NTH) {
      const int r = idx / (BM / 4), c4 = idx % (BM / 4);
      const float4 v = *reinterpret_cast<const float4*>(da + r * BM + 4 * c4);
      *reinterpret_cast<uint2*>(sA + 4 * swz<CA>(r, c4 >> 1) + 2 * (c4 & 1)) =
          make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
    }
    for (int idx = tid; idx < NB16; idx += NTH) {
      const int r = idx / (BN / 4), c4 = idx % (BN / 4);
      const float4 v = *reinterpret_cast<const float4*>(db + r * BN + 4 * c4);
      *reinterpret_cast<uint2*>(sB + 4 * swz<CB>(r, c4 >> 1) + 2 * (c4 & 1)) =
          make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
    }
  };

  float acc[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  const int nch = max(0, c_end - c_begin);
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (st < nch) load_stage(c_begin + st, st);
    cp_async_commit();
  }
  for (int k = 0; k < nch; ++k) {
    cp_async_wait<kStages - 2>();
    __syncthreads();
    convert(k % kStages);
    {
      const int nx = k + kStages - 1;
      if (nx < nch) load_stage(c_begin + nx, nx % kStages);
      cp_async_commit();
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int q = lane >> 3;
      uint32_t af[4];
      {
        const int kk = ks * 16 + (lane & 7) + ((q >> 1) << 3);
        const int c = wm * 2 + (q & 1);
        ldsm_x4_t(smem_u32(sA + 4 * swz<CA>(kk, c)), af[0], af[1], af[2], af[3]);
      }
      uint32_t b0, b1, b2, b3;
      {
        const int kk = ks * 16 + (lane & 7) + ((q & 1) << 3);
        const int c = wn * 2 + (q >> 1);
        ldsm_x4_t(smem_u32(sB + 4 * swz<CB>(kk, c)), b0, b1, b2, b3);
      }
      mma_bf16(acc[0], af, b0, b1);
      mma_bf16(acc[1], af, b2, b3);
    }
  }
  cp_async_wait<0>();
  float* dst = a.part + (size_t)blockIdx.z * a.Cout * 9 * Cin;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int co = m0 + wm * 16 + (lane >> 2) + h * 8;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int ci = ci0 + wn * 16 + j * 8 + 2 * (lane & 3);
      *reinterpret_cast<float2*>(dst + ((size_t)co * 9 + tap) * Cin + ci) =
          make_float2(acc[j][2 * h], acc[j][2 * h + 1]);
    }
  }
}

// The weight gradient from BF16 copies of dZ and of the layer input: cp.async
// copies the 16-byte chunks straight into the XOR-swizzled [pixel][channel]
// tiles that ldmatrix.trans reads (a 4-stage pipeline, one barrier per
// chunk of 32 pixels), every warp a 32 x 32 block of (co, ci).  The same
// BF16 operands and the same K order per split as the FP32-input kernel.
constexpr int kStagesW = 4;
template <int BM, int BN>
constexpr size_t wgrad_smem_b16() {
  return (size_t)kStagesW * kBK * (BM + BN) * 2;
}
template <int BM, int BN>
__global__ void __launch_bounds__((BM / 32) * (BN / 32) * 32) k_conv3x3_wgrad_b16(const WgradArgs a) {
  constexpr int WN = BN / 32, NTH = (BM / 32) * WN * 32;
  constexpr int CA = BM / 8, CB = BN / 8;  // 16-byte chunks per row
  extern __shared__ __align__(128) unsigned char smraw[];
  uint32_t* sA = reinterpret_cast<uint32_t*>(smraw);  // [kStagesW][kBK][BM] bf16
  uint32_t* sB = sA + kStagesW * kBK * BM / 2;        // [kStagesW][kBK][BN] bf16
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / WN, wn = warp % WN;
  const int Cin = a.C1 + a.C2, ctiles = Cin / BN;
  const int m0 = blockIdx.x * BM;
  const int tap = blockIdx.y / ctiles, ci0 = (blockIdx.y % ctiles) * BN;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int HW = a.H * a.Wd, P = a.B * HW;
  const int c_begin = blockIdx.z * a.chunks_per_split;
  const int c_end = min(c_begin + a.chunks_per_split, (P + kBK - 1) / kBK);
  const __nv_bfloat16* xs = ci0 < a.C1 ? a.xb1 : a.xb2;
  const int xc = ci0 < a.C1 ? a.C1 : a.C2, xo = ci0 < a.C1 ? ci0 : ci0 - a.C1;
  auto load_stage = [&](int ch, int st) {
    const int p0 = ch * kBK;
    uint32_t* da = sA + (size_t)st * kBK * BM / 2;
    uint32_t* db = sB + (size_t)st * kBK * BN / 2;
    for (int idx = tid; idx < kBK * CA; idx += NTH) {
      const int r = idx / CA, c = idx % CA, p = p0 + r;
      const bool ok = p < P;
      const __nv_bfloat16* src = ok ? a.dzb + (size_t)p * a.Cout + m0 + 8 * c : a.dzb;
      cp_async16_zfill(smem_u32(da + 4 * swz<CA>(r, c)), src, ok);
    }
    for (int idx = tid; idx < kBK * CB; idx += NTH) {
      const int r = idx / CB, c = idx % CB, p = p0 + r;
      bool ok = p < P;
      const __nv_bfloat16* src = xs;
      if (ok) {
        const int b = p / HW, rem = p - b * HW;
        const int py = rem / a.Wd + dy, px = rem % a.Wd + dx;
        ok = py >= 0 && py < a.H && px >= 0 && px < a.Wd;
        if (ok) src = xs + (((size_t)b * a.H + py) * a.Wd + px) * xc + xo + 8 * c;
      }
      cp_async16_zfill(smem_u32(db + 4 * swz<CB>(r, c)), src, ok);
    }
  };
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const int nch = max(0, c_end - c_begin);
#pragma unroll
  for (int st = 0; st < kStagesW - 1; ++st) {
    if (st < nch) load_stage(c_begin + st, st);
    cp_async_commit();
  }
  for (int k = 0; k < nch; ++k) {
    cp_async_wait<kStagesW - 2>();
    __syncthreads();  // chunk k landed for every thread; chunk k - 1 fully consumed
    {
      const int nx = k + kStagesW - 1;
      if (nx < nch) load_stage(c_begin + nx, nx % kStagesW);
      cp_async_commit();
    }
    const uint32_t* sAc = sA + (size_t)(k % kStagesW) * kBK * BM / 2;
    const uint32_t* sBc = sB + (size_t)(k % kStagesW) * kBK * BN / 2;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int q = lane >> 3;
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int kk = ks * 16 + (lane & 7) + ((q >> 1) << 3);
        const int c = wm * 4 + i * 2 + (q & 1);
        ldsm_x4_t(smem_u32(sAc + 4 * swz<CA>(kk, c)), af[i][0], af[i][1], af[i][2], af[i][3]);
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int kk = ks * 16 + (lane & 7) + ((q & 1) << 3);
        const int c = wn * 4 + jj * 2 + (q >> 1);
        uint32_t b0, b1, b2, b3;
        ldsm_x4_t(smem_u32(sBc + 4 * swz<CB>(kk, c)), b0, b1, b2, b3);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][2 * jj], af[i], b0, b1);
          mma_bf16(acc[i][2 * jj + 1], af[i], b2, b3);
        }
      }
    }
  }
  cp_async_wait<0>();
  float* dst = a.part + (size_t)blockIdx.z * a.Cout * 9 * Cin;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int co = m0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int ci = ci0 + wn * 32 + j * 8 + 2 * (lane & 3);
        *reinterpret_cast<float2*>(dst + ((size_t)co * 9 + tap) * Cin + ci) =
            make_float2(acc[i][j][2 * h], acc[i][j][2 * h + 1]);
      }
    }
}

// out[i] (+)= sum_s part[s][i], s in order (deterministic split reduction)
__global__ void __launch_bounds__(kEW) k_split_sum(const float* __restrict__ part, int splits, long long n,
                                                   float* __restrict__ out, int accumulate) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * n + i];
    out[i] = accumulate ? out[i] + s : s;
  }
}

// per-channel sums of dZ = dy * (y > 0) over pixel ranges: part[split][c]
// (lane <-> channel within a 32-channel group, 8 pixel rows per block)
__global__ void __launch_bounds__(kEW) k_colsum(const float* __restrict__ dy, const float* __restrict__ y, int P, int C,
                                                int rows_per_split, float* __restrict__ part) {
  __shared__ float sh[8][33];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31), r = threadIdx.x >> 5;
  const int p0 = blockIdx.y * rows_per_split, p1 = min(P, p0 + rows_per_split);
  float s = 0.f;
  if (c < C)
    for (int p = p0 + r; p < p1; p += 8) {
      const float v = dy[(size_t)p * C + c];
      s += (!y || y[(size_t)p * C + c] > 0.f) ? v : 0.f;
    }
  sh[r][threadIdx.x & 31] = s;
  __syncthreads();
  if (r == 0 && c < C) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += sh[i][threadIdx.x & 31];
    part[(size_t)blockIdx.y * C + c] = t;
  }
}

// level-0 input: X0[p][0] = x[p], channels 1..31 zero (and its BF16 copy)
__global__ void __launch_bounds__(kEW) k_pack_input(const float* __restrict__ x, float* __restrict__ X0,
                                                    __nv_bfloat16* __restrict__ Xb, int P) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float4* d = reinterpret_cast<float4*>(X0 + (size_t)p * 32);
    d[0] = make_float4(x[p], 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 1; i < 8; ++i) d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (Xb) {
      uint4* db = reinterpret_cast<uint4*>(Xb + (size_t)p * 32);
      db[0] = make_uint4(pack_bf16(x[p], 0.f), 0u, 0u, 0u);
#pragma unroll
      for (int i = 1; i < 4; ++i) db[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// The first 3x3 convolution (one input channel): z[p, co] = b[co] +
// sum_tap bf16(x[p + tap]) w[co, tap] with the BF16 weights of the layer
// (channel 0 of its [Cout][3][3][32] copy), FP32 accumulation in tap order,
// ReLU; outputs FP32 (if y is set) and BF16.  Grid: x over the pixels of an
// image row, y over the rows (b, row) of the batch; one thread per pixel,
// all output channels (weights broadcast from shared memory).
constexpr int kFirstMaxC = 1024;
__global__ void __launch_bounds__(kEW) k_conv_first(const float* __restrict__ x, const __nv_bfloat16* __restrict__ wf,
                                                    const float* __restrict__ bias, float* __restrict__ y,
                                                    __nv_bfloat16* __restrict__ yb, int B, int H, int W, int C) {
  __shared__ float sw[9 * kFirstMaxC];
  __shared__ float sb[kFirstMaxC];
  for (int i = threadIdx.x; i < 9 * C; i += blockDim.x) sw[i] = __bfloat162float(wf[(size_t)i * 32]);
  for (int i = threadIdx.x; i < C; i += blockDim.x) sb[i] = bias[i];
  __syncthreads();
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= W) return;
  for (int row = blockIdx.y; row < B * H; row += gridDim.y) {
    const int py = row % H;
    const size_t img = (size_t)(row - py) * W;  // first pixel of the image
    float xv[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int sy = py + t / 3 - 1, sx = px + t % 3 - 1;
      const bool ok = sy >= 0 && sy < H && sx >= 0 && sx < W;
      xv[t] = ok ? __bfloat162float(__float2bfloat16_rn(x[img + (size_t)sy * W + sx])) : 0.f;
    }
    const size_t p = (size_t)row * W + px;
    for (int g = 0; g < C / 8; ++g) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int co = g * 8 + j;
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < 9; ++t) acc = fmaf(xv[t], sw[co * 9 + t], acc);
        v[j] = fmaxf(acc + sb[co], 0.f);
      }
      const size_t off = p * C + g * 8;
      if (y) {
        float4* d = reinterpret_cast<float4*>(y + off);
        d[0] = make_float4(v[0], v[1], v[2], v[3]);
        d[1] = make_float4(v[4], v[5], v[6], v[7]);
      }
      *reinterpret_cast<uint4*>(yb + off) =
          make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
  }
}

// launch shape of the row kernels: x over `per_row` items, y over rows
inline dim3 row_grid(int per_row, int rows) {
  return dim3((per_row + kEW - 1) / kEW, std::min(rows, 65535));
}

// 2x2 average pooling: (B, H, W, C) -> (B, H/2, W/2, C), float4 over
// channels; FP32 output if y is set, BF16 copy if yb is set.  Grid:
// row_grid(W/2 * C/4, B * H/2).
__global__ void __launch_bounds__(kEW) k_avgpool(const float* __restrict__ x, float* __restrict__ y,
                                                 __nv_bfloat16* __restrict__ yb, int B, int H, int W, int C) {
  const int H2 = H / 2, W2 = W / 2, C4 = C / 4;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= W2 * C4) return;
  const int ox = e / C4, c4 = e - ox * C4;
  const float4* s = reinterpret_cast<const float4*>(x);
  for (int orow = blockIdx.y; orow < B * H2; orow += gridDim.y) {
    const int oy = orow % H2, b = orow / H2;
    const size_t r0 = (((size_t)b * H + 2 * oy) * W + 2 * ox) * C4 + c4, r1 = r0 + (size_t)W * C4;
    const float4 a0 = s[r0], a1 = s[r0 + C4], a2 = s[r1], a3 = s[r1 + C4];
    const float4 o = make_float4(0.25f * (a0.x + a1.x + a2.x + a3.x), 0.25f * (a0.y + a1.y + a2.y + a3.y),
                                 0.25f * (a0.z + a1.z + a2.z + a3.z), 0.25f * (a0.w + a1.w + a2.w + a3.w));
    const size_t i = (size_t)orow * W2 * C4 + e;
    if (y) reinterpret_cast<float4*>(y)[i] = o;
    if (yb) reinterpret_cast<uint2*>(yb)[i] = make_uint2(pack_bf16(o.x, o.y), pack_bf16(o.z, o.w));
  }
}
// adjoint of the pooling plus the skip gradient: g[p] = gp[p/2] / 4 + gs[p],
// zeroed where the ReLU mask mk (if given) is not positive.  Grid:
// row_grid(W * C/4, B * H) over g.
__global__ void __launch_bounds__(kEW) k_avgpool_bwd(const float* __restrict__ gp, const float* __restrict__ gs,
                                                     const float* __restrict__ mk, float* __restrict__ g, int B, int H,
                                                     int W, int C) {
  const int C4 = C / 4;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= W * C4) return;
  const int x = e / C4, c4 = e - x * C4;
  for (int row = blockIdx.y; row < B * H; row += gridDim.y) {
    const int yy = row % H, b = row / H;
    const size_t i = (size_t)row * W * C4 + e;
    const float4 v = reinterpret_cast<const float4*>(gp)[(((size_t)b * (H / 2) + yy / 2) * (W / 2) + x / 2) * C4 + c4];
    float4 o = make_float4(0.25f * v.x, 0.25f * v.y, 0.25f * v.z, 0.25f * v.w);
    if (gs) {
      const float4 s = reinterpret_cast<const float4*>(gs)[i];
      o.x += s.x;
      o.y += s.y;
      o.z += s.z;
      o.w += s.w;
    }
    if (mk) {
      const float4 m = reinterpret_cast<const float4*>(mk)[i];
      o.x = m.x > 0.f ? o.x : 0.f;
      o.y = m.y > 0.f ? o.y : 0.f;
      o.z = m.z > 0.f ? o.z : 0.f;
      o.w = m.w > 0.f ? o.w : 0.f;
    }
    reinterpret_cast<float4*>(g)[i] = o;
  }
}

// nearest 2x upsampling: (B, H, W, C) -> (B, 2H, 2W, C); each thread reads
// one float4 of the input and writes its 2x2 block (FP32 if y is set, BF16
// if yb is set).  Grid: row_grid(W * C/4, B * H) over the input.
__global__ void __launch_bounds__(kEW) k_upsample(const float* __restrict__ x, float* __restrict__ y,
                                                  __nv_bfloat16* __restrict__ yb, int B, int H, int W, int C) {
  const int C4 = C / 4;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= W * C4) return;
  const int ix = e / C4, c4 = e - ix * C4;
  for (int irow = blockIdx.y; irow < B * H; irow += gridDim.y) {
    const float4 o = reinterpret_cast<const float4*>(x)[(size_t)irow * W * C4 + e];
    const uint2 ob = make_uint2(pack_bf16(o.x, o.y), pack_bf16(o.z, o.w));
    const int iy = irow % H, b = irow / H;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const size_t i = (((size_t)b * 2 * H + 2 * iy + (d >> 1)) * 2 * W + 2 * ix + (d & 1)) * C4 + c4;
      if (y) reinterpret_cast<float4*>(y)[i] = o;
      if (yb) reinterpret_cast<uint2*>(yb)[i] = ob;
    }
  }
}

// adjoint of the upsampling: sum of the 2x2 block, zeroed where the ReLU
// mask mk (if given) is not positive
__global__ void __launch_bounds__(kEW) k_upsample_bwd(const float* __restrict__ g, const float* __restrict__ mk,
                                                      float* __restrict__ gx, int B, int H, int W, int C) {
  const int C4 = C / 4;
  const long long n = (long long)B * H * W * C4;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c4 = (int)(i % C4);
    long long q = i / C4;
    const int x = (int)(q % W);
    q /= W;
    const int yy = (int)(q % H);
    const int b = (int)(q / H);
    const float4* s = reinterpret_cast<const float4*>(g);
    const size_t r0 = (((size_t)b * 2 * H + 2 * yy) * 2 * W + 2 * x) * C4 + c4, r1 = r0 + (size_t)2 * W * C4;
    const float4 a0 = s[r0], a1 = s[r0 + C4], a2 = s[r1], a3 = s[r1 + C4];
    float4 o = make_float4(a0.x + a1.x + a2.x + a3.x, a0.y + a1.y + a2.y + a3.y, a0.z + a1.z + a2.z + a3.z,
                           a0.w + a1.w + a2.w + a3.w);
    if (mk) {
      const float4 m = reinterpret_cast<const float4*>(mk)[i];
      o.x = m.x > 0.f ? o.x : 0.f;
      o.y = m.y > 0.f ? o.y : 0.f;
      o.z = m.z > 0.f ? o.z : 0.f;
      o.w = m.w > 0.f ? o.w : 0.f;
    }
    reinterpret_cast<float4*>(gx)[i] = o;
  }
}

// head: out[p] = x[p] + bh + sum_c Wh[c] h[p][c]   (one warp per pixel group)
__global__ void __launch_bounds__(kEW) k_head(const float* __restrict__ x, const float* __restrict__ h,
                                              const float* __restrict__ wh, const float* __restrict__ bh,
                                              float* __restrict__ out, int P, int C) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float s = bh[0];
    const float4* hp = reinterpret_cast<const float4*>(h + (size_t)p * C);
    for (int c4 = 0; c4 < C / 4; ++c4) {
      const float4 v = hp[c4];
      s = fmaf(wh[4 * c4], v.x, s);
      s = fmaf(wh[4 * c4 + 1], v.y, s);
      s = fmaf(wh[4 * c4 + 2], v.z, s);
      s = fmaf(wh[4 * c4 + 3], v.w, s);
    }
    out[p] = x[p] + s;
  }
}

// loss partials and the output gradient g = (out - t) / P
__global__ void __launch_bounds__(kEW) k_loss(const float* __restrict__ out, const float* __restrict__ t,
                                              float* __restrict__ g, int P, double* __restrict__ part) {
  __shared__ double sh[kEW / 32];
  double s = 0.0;
  const float inv = 1.f / (float)P;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const float d = out[p] - t[p];
    g[p] = d * inv;
    s += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tt = 0.0;
    for (int i = 0; i < kEW / 32; ++i) tt += sh[i];
    part[blockIdx.x] = tt;
  }
}

// head backward: gh[p][c] = g[p] Wh[c] where h[p][c] > 0 (h is a ReLU output)
__global__ void __launch_bounds__(kEW) k_head_bwd(const float* __restrict__ g, const float* __restrict__ wh,
                                                  const float* __restrict__ h, float* __restrict__ gh, int P, int C) {
  const long long n = (long long)P * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    gh[i] = h[i] > 0.f ? g[i / C] * wh[i % C] : 0.f;
}

// BF16 copy (round to nearest even) of n floats
__global__ void __launch_bounds__(kEW) k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                                 long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// the same conversion, four elements per thread (n a multiple of 4)
__global__ void __launch_bounds__(kEW) k_to_bf16x4(const float4* __restrict__ x, uint2* __restrict__ y,
                                                   long long n4) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = x[i];
    y[i] = make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
  }
}

// dz = dy where y > 0, else 0
__global__ void __launch_bounds__(kEW) k_relu_mask(const float* __restrict__ dy, const float* __restrict__ y,
                                                   float* __restrict__ dz, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dz[i] = y[i] > 0.f ? dy[i] : 0.f;
}

// head weight gradient partials: part[s][c] = sum_p g[p] h[p][c] (c < C),
// part[s][C] = sum_p g[p]
__global__ void __launch_bounds__(kEW) k_head_wgrad(const float* __restrict__ g, const float* __restrict__ h, int P,
                                                    int C, int rows_per_split, float* __restrict__ part) {
  __shared__ float sh[8][33];
  const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int p0 = blockIdx.x * rows_per_split, p1 = min(P, p0 + rows_per_split);
  for (int cb = 0; cb <= C; cb += 32) {
    const int cc = cb + c;
    float s = 0.f;
    if (cc <= C)
      for (int p = p0 + r; p < p1; p += 8) s += g[p] * (cc < C ? h[(size_t)p * C + cc] : 1.f);
    sh[r][c] = s;
    __syncthreads();
    if (r == 0 && cc <= C) {
      float t = 0.f;
      for (int i = 0; i < 8; ++i) t += sh[i][c];
      part[(size_t)blockIdx.x * (C + 1) + cc] = t;
    }
    __syncthreads();
  }
}

// squared L2 norm of the gradient: FP32 per thread and warp, FP64 per block
__global__ void __launch_bounds__(kEW) k_sumsq(const float* __restrict__ g, long long n, double* __restrict__ part) {
  __shared__ double sh[kEW / 32];
  float s = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fmaf(g[i], g[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kEW / 32; ++i) t += sh[i];
    part[blockIdx.x] = t;
  }
}

// gradient scale min(1, max_norm / ||g||) (max_norm <= 0: 1) from the block
// partials in a fixed order; also stores ||g||
__global__ void k_clip_scale(const double* __restrict__ part, int nb, float max_norm, float* __restrict__ scale,
                             double* __restrict__ norm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nb; ++i) t += part[i];
  const double nrm = sqrt(t);
  *norm = nrm;
  *scale = (max_norm > 0.f && nrm > (double)max_norm) ? (float)((double)max_norm / nrm) : 1.f;
}

// Adam on the FP32 master parameters (bias-corrected step size lr_t), the
// gradient multiplied by *gscale
__global__ void __launch_bounds__(kEW) k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, long long n, float lr_t, float b1, float b2,
                                              float eps, const float* __restrict__ gscale) {
  const float sc = *gscale;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] * sc;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr_t * mi / (sqrtf(vi) + eps);
  }
}

// BF16 weight copies of one 3x3 layer: Wf[co][tap][ci] (forward) and
// Wt[ci][8 - tap][co] (data gradient: transposed channels, flipped taps)
__global__ void __launch_bounds__(kEW) k_weights_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wf,
                                                      __nv_bfloat16* __restrict__ wt, int Cout, int Cin) {
  const long long n = (long long)Cout * 9 * Cin;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(i % Cin);
    const int tap = (int)((i / Cin) % 9);
    const int co = (int)(i / ((long long)9 * Cin));
    const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
    wf[i] = b;
    wt[((size_t)ci * 9 + (8 - tap)) * Cout + co] = b;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct Layer {
  int cout, cin, cin_pad, k;    // k = 3 (convolution) or 1 (head)
  int c1, c2, lv;               // input channels from the first / second tensor, level
  size_t w_off, b_off;          // into the padded FP32 parameter vector
  size_t bf_off;                // into the BF16 weight arrays (3x3 layers)
  size_t host_off;              // into the caller's (unpadded) parameter vector
};

struct Net {
  int L, base, maxB, H, W;
  std::vector<int> c;           // channels per level
  std::vector<Layer> layers;    // enc0.a, enc0.b, ..., dec(L-2).up/a/b, ..., head
  size_t n_param = 0, n_bf = 0;
  long long host_count = 0;
  std::vector<void*> allocs;
  float *param = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  __nv_bfloat16 *wf = nullptr, *wt = nullptr;
  int adam_t = 0;
  // activations and gradients (indexed by level)
  float* X0 = nullptr;
  std::vector<float*> ea, eb, pool, upin, upout, da, db;
  // BF16 copies of every convolution input of the forward pass
  std::vector<__nv_bfloat16*> eab, ebb, poolb, upinb, upoutb, dab;
  std::vector<float*> g_ea, g_eb, g_pool, g_upin, g_upout, g_da, g_db, g_skip;
  float *out = nullptr, *g_out = nullptr, *g_in = nullptr;
  float* part = nullptr;        // split partials
  size_t part_floats = 0;
  double* loss_part = nullptr;
  double* norm_part = nullptr;   // gradient-norm block partials
  double* d_gnorm = nullptr;     // ||g|| of the last Adam step
  float* d_gscale = nullptr;     // clipping factor of the last Adam step
  int* d_err = nullptr;          // device error flag (CPCT_ERR_* bits)
  __nv_bfloat16* gradb = nullptr;  // BF16 copy of the gradient entering a data-gradient convolution
  int last_batch = 0;
};

int enc_a(int l) { return 2 * l; }
int enc_b(int l) { return 2 * l + 1; }
int dec_up(const Net& n, int l) { return 2 * n.L + 3 * (n.L - 2 - l); }
int dec_a(const Net& n, int l) { return dec_up(n, l) + 1; }
int dec_b(const Net& n, int l) { return dec_up(n, l) + 2; }
int head_idx(const Net& n) { return (int)n.layers.size() - 1; }

int grid_for(long long n) { return (int)std::min<long long>((n + kEW - 1) / kEW, 152LL * 16); }

// pixel rows per split of the per-channel sums (at most 65535 splits: the
// grid's y extent)
long long colsum_rows(long long P) { return std::max<long long>(2048, (P + 65534) / 65535); }

bool build_layers(Net& n) {
  n.c.resize(n.L);
  for (int l = 0; l < n.L; ++l) n.c[l] = n.base << l;
  auto add = [&](int cout, int cin, int k, int lv, bool concat) {
    Layer y;
    y.cout = cout;
    y.cin = cin;
    y.cin_pad = (k == 3 && cin < 32) ? 32 : cin;
    y.c1 = concat ? cin / 2 : y.cin_pad;
    y.c2 = concat ? cin / 2 : 0;
    y.lv = lv;
    y.k = k;
    y.w_off = n.n_param;
    n.n_param += (size_t)cout * k * k * y.cin_pad;
    y.b_off = n.n_param;
    n.n_param += cout;
    y.bf_off = n.n_bf;
    if (k == 3) n.n_bf += (size_t)cout * 9 * y.cin_pad;
    y.host_off = (size_t)n.host_count;
    n.host_count += (long long)cout * k * k * cin + cout;
    n.layers.push_back(y);
  };
  for (int l = 0; l < n.L; ++l) {
    add(n.c[l], l == 0 ? 1 : n.c[l - 1], 3, l, false);
    add(n.c[l], n.c[l], 3, l, false);
  }
  for (int l = n.L - 2; l >= 0; --l) {
    add(n.c[l], n.c[l + 1], 3, l, false);
    add(n.c[l], 2 * n.c[l], 3, l, true);
    add(n.c[l], n.c[l], 3, l, false);
  }
  add(1, n.c[0], 1, 0, false);
  return true;
}

template <class T>
bool dalloc(Net& n, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) return false;
  n.allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}

void free_net(Net* n) {
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

// the largest split-partial buffer any layer needs (floats)
// tiles of the weight gradient (an N tile must not straddle the two input
// tensors of a concatenation) and the split of the pixel reduction
// tiles and pixel splits of a weight gradient: enough CTAs for about 32
// warps per SM (warps per CTA: (BM/16)(BN/16) for the FP32-input kernel,
// (BM/32)(BN/32) for the BF16 one)
size_t wgrad_splits(int cout, int c1, int c2, long long P, int* bm, int* bn, int* splits, int* cps, bool b16 = true) {
  const int cin = c1 + c2;
  *bm = cout % 64 == 0 ? 64 : 32;
  *bn = (c1 % 64 == 0 && c2 % 64 == 0) ? 64 : 32;
  const long long tiles = (long long)(cout / *bm) * 9 * (cin / *bn);
  const long long warps = b16 ? (*bm / 32) * (*bn / 32) : (*bm / 16) * (*bn / 16);
  const long long chunks = (P + kBK - 1) / kBK;
  const long long want = (32LL * 152 + tiles * warps - 1) / (tiles * warps);
  long long s = std::max<long long>(1, std::min<long long>(want, chunks));
  const long long per = (chunks + s - 1) / s;
  s = (chunks + per - 1) / per;
  *splits = (int)s;
  *cps = (int)per;
  return (size_t)s * cout * 9 * cin;
}

// the pipelined kernels need more than the default 48 KB of dynamic shared
// memory: raise the limit once per process (per kernel)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                   cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? reinterpret_cast<EncodeTiledFn>(ptr)
               : nullptr;
  }();
  return fn;
}

// 4-D map {C, W, H, B} of a BF16 NHWC activation, box {KC, Wb, Hb, 1},
// 128-byte (KC = 64) or 64-byte (KC = 32) swizzle
bool encode_act_map(CUtensorMap* m, const __nv_bfloat16* x, int C, int B, int H, int W, int Wb, int Hb, int KC) {
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)KC, (cuuint32_t)Wb, (cuuint32_t)Hb, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(x), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, KC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor maps of the TMA forward convolution; false where the image does
// not tile into 128-pixel boxes (or no encoder is available)
bool encode_conv_maps(const ConvArgs& a, int bn, int kc, TcMaps* maps) {
  if (!encode_fn()) return false;
  const int Wb = a.Wd >= 128 ? 128 : a.Wd;
  if (Wb < 1 || a.Wd % Wb || 128 % Wb) return false;
  const int Hb = 128 / Wb;
  if (a.H % Hb) return false;
  maps->Wb = Wb;
  maps->Hb = Hb;
  const int Cin = a.C1 + a.C2;
  if (!encode_act_map(&maps->a1, a.xb1, a.C1, a.B, a.H, a.Wd, Wb, Hb, kc)) return false;
  if (a.C2 == 0)
    maps->a2 = maps->a1;  // unused
  else if (!encode_act_map(&maps->a2, a.xb2, a.C2, a.B, a.H, a.Wd, Wb, Hb, kc))
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)9 * Cin, (cuuint64_t)a.Cout};
  const cuuint64_t strides[1] = {(cuuint64_t)9 * Cin * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kc, (cuuint32_t)bn};
  const cuuint32_t estr[2] = {1, 1};
  return encode_fn()(&maps->w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(a.W), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool smem_attrs_set() {
  static const bool ok = [] {
    bool r = true;
    r &= cudaFuncSetAttribute(k_conv3x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<64>()) ==
         cudaSuccess;
    r &= cudaFuncSetAttribute(k_conv3x3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<32>()) ==
         cudaSuccess;
    r &= cudaFuncSetAttribute(k_conv3x3_b16<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)conv_smem_b16<64>()) == cudaSuccess;
    r &= cudaFuncSetAttribute(k_conv3x3_b16<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)conv_smem_b16<32>()) == cudaSuccess;
#define CPCT_TC_ATTR(BN, KC)                                                                       \
  r &= cudaFuncSetAttribute(k_conv3x3_tc<BN, KC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                            (int)conv_smem_tc<BN, KC, true>()) == cudaSuccess;                           \
  r &= cudaFuncSetAttribute(k_conv3x3_tc<BN, KC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                            (int)conv_smem_tc<BN, KC, false>()) == cudaSuccess;
    CPCT_TC_ATTR(256, 32)
    CPCT_TC_ATTR(128, 32)
    CPCT_TC_ATTR(64, 32)
    CPCT_TC_ATTR(32, 32)
    CPCT_TC_ATTR(256, 64)
    CPCT_TC_ATTR(128, 64)
    CPCT_TC_ATTR(64, 64)
    CPCT_TC_ATTR(32, 64)
#undef CPCT_TC_ATTR
    r &= cudaFuncSetAttribute(k_conv3x3_wgrad<64, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)wgrad_smem<64, 64>()) == cudaSuccess;
    r &= cudaFuncSetAttribute(k_conv3x3_wgrad<64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)wgrad_smem<64, 32>()) == cudaSuccess;
    r &= cudaFuncSetAttribute(k_conv3x3_wgrad<32, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)wgrad_smem<32, 64>()) == cudaSuccess;
    r &= cudaFuncSetAttribute(k_conv3x3_wgrad<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)wgrad_smem<32, 32>()) == cudaSuccess;
    return r;
  }();
  return ok;
}

// N tile of the tensor-memory kernel for Cout (0: not eligible)
int tc_bn(int Cout) {
  return Cout % 256 == 0 ? 256 : (Cout == 128 || Cout == 64 || Cout == 32) ? Cout : 0;
}

void launch_conv(const ConvArgs& a, cudaStream_t s, bool force_cp_async = false) {
  const int P = a.B * a.H * a.Wd;
  smem_attrs_set();  // if this failed, the launch below reports the error
  // forward pass on the tensor-memory kernel: N tiles of 32, 64, 128 or 256
  // channels (a power of two: the tensor memory allocation's granularity)
  const int bn = tc_bn(a.Cout);
  if (a.xb1 && a.err && bn) {
    // persistent: one CTA (N tile of 256) or two per SM over all tiles;
    // 64-channel chunks where both inputs split into them
    static const int sms = [] {
      int dev = 0, n = 0;
      cudaGetDevice(&dev);
      return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 1;
    }();
    const bool k64 = a.C1 % 64 == 0 && a.C2 % 64 == 0;
    const long long ntiles = (long long)((P + 127) / 128) * (a.Cout / bn);
    const int grid = (int)std::min<long long>(ntiles, (long long)sms * (bn >= 256 ? 1 : 2));
    TcMaps maps;
    const bool tma = !force_cp_async && encode_conv_maps(a, bn, k64 ? 64 : 32, &maps);
    if (!tma) memset(&maps, 0, sizeof(maps));
#define CPCT_TC_LAUNCH(BN, KC)                                                                           \
  do {                                                                                                  \
    if (tma)                                                                                            \
      k_conv3x3_tc<BN, KC, true><<<grid, tc_threads<true>(), conv_smem_tc<BN, KC, true>(), s>>>(a, maps);   \
    else                                                                                                    \
      k_conv3x3_tc<BN, KC, false><<<grid, tc_threads<false>(), conv_smem_tc<BN, KC, false>(), s>>>(a, maps); \
  } while (0)
    if (bn == 256) { if (k64) CPCT_TC_LAUNCH(256, 64); else CPCT_TC_LAUNCH(256, 32); }
    else if (bn == 128) { if (k64) CPCT_TC_LAUNCH(128, 64); else CPCT_TC_LAUNCH(128, 32); }
    else if (bn == 64) { if (k64) CPCT_TC_LAUNCH(64, 64); else CPCT_TC_LAUNCH(64, 32); }
    else { if (k64) CPCT_TC_LAUNCH(32, 64); else CPCT_TC_LAUNCH(32, 32); }
#undef CPCT_TC_LAUNCH
    return;
  }
  if (a.xb1) {  // forward pass with BF16 input copies (single output tensor)
    if (a.Cout % 64 == 0) {
      dim3 grid((P + bm_b16<64>() - 1) / bm_b16<64>(), a.Cout / 64);
      k_conv3x3_b16<64><<<grid, kCT, conv_smem_b16<64>(), s>>>(a);
    } else {
      dim3 grid((P + bm_b16<32>() - 1) / bm_b16<32>(), a.Cout / 32);
      k_conv3x3_b16<32><<<grid, kCT, conv_smem_b16<32>(), s>>>(a);
    }
    return;
  }
  if (a.Cout % 64 == 0) {
    dim3 grid((P + kBM - 1) / kBM, a.Cout / 64);
    k_conv3x3<64><<<grid, kCT, conv_smem<64>(), s>>>(a);
  } else {
    dim3 grid((P + kBM - 1) / kBM, a.Cout / 32);
    k_conv3x3<32><<<grid, kCT, conv_smem<32>(), s>>>(a);
  }
}

void launch_wgrad_b16(const WgradArgs& a, int bm, int bn, int splits, cudaStream_t s) {
  const int Cin = a.C1 + a.C2;
  dim3 grid(a.Cout / bm, 9 * (Cin / bn), splits);
  if (bm == 64 && bn == 64) k_conv3x3_wgrad_b16<64, 64><<<grid, 4 * 32, wgrad_smem_b16<64, 64>(), s>>>(a);
  else if (bm == 64) k_conv3x3_wgrad_b16<64, 32><<<grid, 2 * 32, wgrad_smem_b16<64, 32>(), s>>>(a);
  else if (bn == 64) k_conv3x3_wgrad_b16<32, 64><<<grid, 2 * 32, wgrad_smem_b16<32, 64>(), s>>>(a);
  else k_conv3x3_wgrad_b16<32, 32><<<grid, 32, wgrad_smem_b16<32, 32>(), s>>>(a);
}

void launch_wgrad(const WgradArgs& a, int bm, int bn, int splits, cudaStream_t s) {
  const int Cin = a.C1 + a.C2;
  smem_attrs_set();
  dim3 grid(a.Cout / bm, 9 * (Cin / bn), splits);
  if (bm == 64 && bn == 64) k_conv3x3_wgrad<64, 64><<<grid, 16 * 32, wgrad_smem<64, 64>(), s>>>(a);
  else if (bm == 64) k_conv3x3_wgrad<64, 32><<<grid, 8 * 32, wgrad_smem<64, 32>(), s>>>(a);
  else if (bn == 64) k_conv3x3_wgrad<32, 64><<<grid, 8 * 32, wgrad_smem<32, 64>(), s>>>(a);
  else k_conv3x3_wgrad<32, 32><<<grid, 4 * 32, wgrad_smem<32, 32>(), s>>>(a);
}

// forward of one 3x3 layer: y = relu(conv(x1 | x2) + b)
void conv_fwd(Net& n, int li, const float* x1, const __nv_bfloat16* xb1, int C1, const float* x2,
              const __nv_bfloat16* xb2, int C2, float* y, __nv_bfloat16* yb, int B, int lv, cudaStream_t s,
              const float* head_x = nullptr, float* head_out = nullptr) {
  const Layer& L = n.layers[li];
  ConvArgs a{};
  a.x1 = x1;
  a.x2 = x2;
  a.xb1 = xb1;
  a.xb2 = xb2;
  a.yb1 = yb;
  a.C1 = C1;
  a.C2 = C2;
  a.W = n.wf + L.bf_off;
  a.bias = n.param + L.b_off;
  a.y1 = y;
  a.y2 = nullptr;
  a.O1 = L.cout;
  a.Cout = L.cout;
  a.relu = 1;
  a.B = B;
  a.H = n.H >> lv;
  a.Wd = n.W >> lv;
  a.err = n.d_err;
  if (head_out) {
    const Layer& Hd = n.layers[head_idx(n)];
    a.head_w = n.param + Hd.w_off;
    a.head_b = n.param + Hd.b_off;
    a.head_x = head_x;
    a.head_out = head_out;
  }
  launch_conv(a, s);
}

// backward of one 3x3 layer at dz = dL/dz, z its pre-activation: data
// gradient into (dx1 | dx2) if dx1 is given -- each part zeroed where its
// mask (om1 / om2, the ReLU output it lands on) is not positive, so it is
// again a pre-activation gradient -- and the weight and bias gradients into
// n.grad
// backward of one 3x3 layer: data gradient (if dx1) and weight / bias
// gradients; xb1 / xb2 are the BF16 copies of the layer's inputs (null: the
// FP32-input weight-gradient kernel)
void conv_bwd(Net& n, int li, const float* dz, const float* x1, const __nv_bfloat16* xb1, int C1, const float* x2,
              const __nv_bfloat16* xb2, int C2, float* dx1, float* dx2, const float* om1, const float* om2, int B,
              int lv, cudaStream_t s) {
  const Layer& L = n.layers[li];
  const int H = n.H >> lv, W = n.W >> lv;
  const long long P = (long long)B * H * W;
  const bool tc_dgrad = dx1 && tc_bn(C1 + C2);
  const bool b16_wgrad = xb1 && (C2 == 0 || xb2);
  if (tc_dgrad || b16_wgrad) {
    // a BF16 copy of dz (the rounding the FP32 kernels apply while
    // staging); the largest dz is level 0's P0 x c0
    const long long nz4 = P * L.cout / 4;
    k_to_bf16x4<<<grid_for(nz4), kEW, 0, s>>>(reinterpret_cast<const float4*>(dz), reinterpret_cast<uint2*>(n.gradb),
                                               nz4);
  }
  if (dx1) {
    ConvArgs a{};
    a.x1 = dz;
    a.x2 = nullptr;
    if (tc_dgrad) {
      a.xb1 = n.gradb;
      a.err = n.d_err;
    }
    a.C1 = L.cout;
    a.C2 = 0;
    a.W = n.wt + L.bf_off;
    a.bias = nullptr;
    a.y1 = dx1;
    a.y2 = dx2;
    a.om1 = om1;
    a.om2 = om2;
    a.O1 = C1;
    a.Cout = C1 + C2;
    a.relu = 0;
    a.B = B;
    a.H = H;
    a.Wd = W;
    launch_conv(a, s);
  }
  int bm, bn, splits, cps;
  wgrad_splits(L.cout, C1, C2, P, &bm, &bn, &splits, &cps, b16_wgrad);
  WgradArgs w{};
  w.dz = dz;
  w.x1 = x1;
  w.x2 = x2;
  w.dzb = n.gradb;
  w.xb1 = xb1;
  w.xb2 = xb2;
  w.C1 = C1;
  w.C2 = C2;
  w.Cout = L.cout;
  w.B = B;
  w.H = H;
  w.Wd = W;
  w.chunks_per_split = cps;
  w.part = n.part;
  if (b16_wgrad)
    launch_wgrad_b16(w, bm, bn, splits, s);
  else
    launch_wgrad(w, bm, bn, splits, s);
  const long long nw = (long long)L.cout * 9 * (C1 + C2);
  k_split_sum<<<grid_for(nw), kEW, 0, s>>>(n.part, splits, nw, n.grad + L.w_off, 0);
  // bias: per-channel sums of dz over pixel ranges, then the fixed-order sum
  const int rows = (int)colsum_rows(P), sp = (int)((P + rows - 1) / rows);
  dim3 cg((L.cout + 31) / 32, sp);
  k_colsum<<<cg, kEW, 0, s>>>(dz, nullptr, (int)P, L.cout, rows, n.part);
  k_split_sum<<<grid_for(L.cout), kEW, 0, s>>>(n.part, sp, L.cout, n.grad + L.b_off, 0);
}

void refresh_bf16(Net& n, cudaStream_t s) {
  for (const Layer& L : n.layers)
    if (L.k == 3) {
      const long long cnt = (long long)L.cout * 9 * L.cin_pad;
      k_weights_bf16<<<grid_for(cnt), kEW, 0, s>>>(n.param + L.w_off, n.wf + L.bf_off, n.wt + L.bf_off, L.cout,
                                                   L.cin_pad);
    }
}

// forward pass; `train` keeps the FP32 copies that only the backward pass
// reads (outputs whose forward consumers read their BF16 copies: enc a, the
// pooled and upsampled maps, dec up and dec a) and the padded FP32 input
void forward_pass(Net& n, const float* x, int B, cudaStream_t s, bool train) {
  const int P0 = B * n.H * n.W;
  if (train) k_pack_input<<<grid_for(P0), kEW, 0, s>>>(x, n.X0, nullptr, P0);
  {
    const Layer& L0 = n.layers[enc_a(0)];
    k_conv_first<<<row_grid(n.W, B * n.H), kEW, 0, s>>>(x, n.wf + L0.bf_off, n.param + L0.b_off,
                                                        train ? n.ea[0] : nullptr, n.eab[0], B, n.H, n.W, n.c[0]);
  }
  const float* h = nullptr;
  const __nv_bfloat16* hb = nullptr;
  int hc = 0;
  for (int l = 0; l < n.L; ++l) {
    if (l > 0) conv_fwd(n, enc_a(l), h, hb, hc, nullptr, nullptr, 0, train ? n.ea[l] : nullptr, n.eab[l], B, l, s);
    conv_fwd(n, enc_b(l), n.ea[l], n.eab[l], n.c[l], nullptr, nullptr, 0, n.eb[l], n.ebb[l], B, l, s);
    if (l < n.L - 1) {
      k_avgpool<<<row_grid((n.W >> (l + 1)) * n.c[l] / 4, B * (n.H >> (l + 1))), kEW, 0, s>>>(
          n.eb[l], train ? n.pool[l] : nullptr, n.poolb[l], B, n.H >> l, n.W >> l, n.c[l]);
      h = n.pool[l];
      hb = n.poolb[l];
      hc = n.c[l];
    }
  }
  h = n.eb[n.L - 1];
  for (int l = n.L - 2; l >= 0; --l) {
    k_upsample<<<row_grid((n.W >> (l + 1)) * n.c[l + 1] / 4, B * (n.H >> (l + 1))), kEW, 0, s>>>(
        h, train ? n.upin[l] : nullptr, n.upinb[l], B, n.H >> (l + 1), n.W >> (l + 1), n.c[l + 1]);
    conv_fwd(n, dec_up(n, l), n.upin[l], n.upinb[l], n.c[l + 1], nullptr, nullptr, 0, train ? n.upout[l] : nullptr,
             n.upoutb[l], B, l, s);
    conv_fwd(n, dec_a(n, l), n.eb[l], n.ebb[l], n.c[l], n.upout[l], n.upoutb[l], n.c[l], train ? n.da[l] : nullptr,
             n.dab[l], B, l, s);
    // the last layer carries the head in its epilogue where the tensor-memory
    // kernel takes all c0 channels in one N tile; its output is then read
    // only by the backward pass
    const bool fuse = l == 0 && tc_bn(n.c[0]) == n.c[0];
    conv_fwd(n, dec_b(n, l), n.da[l], n.dab[l], n.c[l], nullptr, nullptr, 0, fuse && !train ? nullptr : n.db[l],
             nullptr, B, l, s, fuse ? x : nullptr, fuse ? n.out : nullptr);
    if (fuse) return;
    h = n.db[l];
  }
  const Layer& Hd = n.layers[head_idx(n)];
  k_head<<<grid_for(P0), kEW, 0, s>>>(x, h, n.param + Hd.w_off, n.param + Hd.b_off, n.out, P0, n.c[0]);
}

void backward_pass(Net& n, const float* x, const float* t, int B, cudaStream_t s) {
  // every gradient buffer of a ReLU output holds the pre-activation gradient
  // dL/dz of the layer that produced it (the ReLU mask is applied where the
  // gradient is formed)
  const int P0 = B * n.H * n.W;
  const int lg = std::min(1024, (P0 + kEW - 1) / kEW);
  k_loss<<<lg, kEW, 0, s>>>(n.out, t, n.g_out, P0, n.loss_part);
  const float* h = n.L > 1 ? n.db[0] : n.eb[0];
  float* gh = n.L > 1 ? n.g_db[0] : n.g_eb[0];
  const Layer& Hd = n.layers[head_idx(n)];
  k_head_bwd<<<grid_for((long long)P0 * n.c[0]), kEW, 0, s>>>(n.g_out, n.param + Hd.w_off, h, gh, P0, n.c[0]);
  {
    const int rows = 2048, sp = (P0 + rows - 1) / rows;
    k_head_wgrad<<<sp, kEW, 0, s>>>(n.g_out, h, P0, n.c[0], rows, n.part);
    k_split_sum<<<grid_for(n.c[0] + 1), kEW, 0, s>>>(n.part, sp, n.c[0] + 1, n.grad + Hd.w_off, 0);
  }
  for (int l = 0; l <= n.L - 2; ++l) {
    conv_bwd(n, dec_b(n, l), n.g_db[l], n.da[l], n.dab[l], n.c[l], nullptr, nullptr, 0, n.g_da[l], nullptr, n.da[l],
             nullptr, B, l, s);
    // the skip part is summed with the pooled path before its mask applies
    conv_bwd(n, dec_a(n, l), n.g_da[l], n.eb[l], n.ebb[l], n.c[l], n.upout[l], n.upoutb[l], n.c[l], n.g_skip[l],
             n.g_upout[l], nullptr, n.upout[l], B, l, s);
    conv_bwd(n, dec_up(n, l), n.g_upout[l], n.upin[l], n.upinb[l], n.c[l + 1], nullptr, nullptr, 0, n.g_upin[l],
             nullptr, nullptr, nullptr, B, l, s);
    float* gnext = l + 1 <= n.L - 2 ? n.g_db[l + 1] : n.g_eb[n.L - 1];
    const float* mnext = l + 1 <= n.L - 2 ? n.db[l + 1] : n.eb[n.L - 1];
    const long long cnt = (long long)B * (n.H >> (l + 1)) * (n.W >> (l + 1)) * n.c[l + 1] / 4;
    k_upsample_bwd<<<grid_for(cnt), kEW, 0, s>>>(n.g_upin[l], mnext, gnext, B, n.H >> (l + 1), n.W >> (l + 1),
                                                 n.c[l + 1]);
  }
  for (int l = n.L - 1; l >= 0; --l) {
    if (l < n.L - 1) {
      k_avgpool_bwd<<<row_grid((n.W >> l) * n.c[l] / 4, B * (n.H >> l)), kEW, 0, s>>>(
          n.g_pool[l], n.g_skip[l], n.eb[l], n.g_eb[l], B, n.H >> l, n.W >> l, n.c[l]);
    }
    conv_bwd(n, enc_b(l), n.g_eb[l], n.ea[l], n.eab[l], n.c[l], nullptr, nullptr, 0, n.g_ea[l], nullptr, n.ea[l],
             nullptr, B, l, s);
    if (l > 0)
      conv_bwd(n, enc_a(l), n.g_ea[l], n.pool[l - 1], n.poolb[l - 1], n.c[l - 1], nullptr, nullptr, 0,
               n.g_pool[l - 1], nullptr, nullptr, nullptr, B, l, s);
    else
      conv_bwd(n, enc_a(0), n.g_ea[0], n.X0, nullptr, 32, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, B,
               0, s);
  }
}

}  // namespace

struct cpct_unet {
  Net* net;
};

extern "C" long long cpct_unet_param_count(int levels, int base) {
  if (levels < 1 || levels > 6 || base < 32 || base % 32) return -1;
  Net n;
  n.L = levels;
  n.base = base;
  build_layers(n);
  return n.host_count;
}

extern "C" int cpct_unet_create(cpct_unet** out, int levels, int base, int max_batch, int height, int width,
                                cudaStream_t stream) {
  if (!out) return CPCT_EINVAL;
  *out = nullptr;
  if (levels < 1 || levels > 6 || base < 32 || base % 32 || (base << (levels - 1)) > 1024 || max_batch < 1)
    return CPCT_EINVAL;
  const int div = 1 << (levels - 1);
  if (height < div || width < div || height % div || width % div) return CPCT_EINVAL;
  if ((long long)max_batch * height * width > (1LL << 30)) return CPCT_EINVAL;
  Net* n = new (std::nothrow) Net;
  if (!n) return CPCT_ENOMEM;
  n->L = levels;
  n->base = base;
  n->maxB = max_batch;
  n->H = height;
  n->W = width;
  build_layers(*n);
  bool ok = dalloc(*n, &n->param, n->n_param) && dalloc(*n, &n->grad, n->n_param) &&
            dalloc(*n, &n->adam_m, n->n_param) && dalloc(*n, &n->adam_v, n->n_param) &&
            dalloc(*n, &n->wf, n->n_bf) && dalloc(*n, &n->wt, n->n_bf);
  const int L = levels;
  n->ea.assign(L, nullptr);
  n->eb.assign(L, nullptr);
  n->pool.assign(L, nullptr);
  n->upin.assign(L, nullptr);
  n->upout.assign(L, nullptr);
  n->da.assign(L, nullptr);
  n->db.assign(L, nullptr);
  n->g_ea.assign(L, nullptr);
  n->g_eb.assign(L, nullptr);
  n->g_pool.assign(L, nullptr);
  n->g_upin.assign(L, nullptr);
  n->g_upout.assign(L, nullptr);
  n->g_da.assign(L, nullptr);
  n->g_db.assign(L, nullptr);
  n->g_skip.assign(L, nullptr);
  n->eab.assign(L, nullptr);
  n->ebb.assign(L, nullptr);
  n->poolb.assign(L, nullptr);
  n->upinb.assign(L, nullptr);
  n->upoutb.assign(L, nullptr);
  n->dab.assign(L, nullptr);
  const size_t P0 = (size_t)max_batch * height * width;
  for (int l = 0; l < L && ok; ++l) {
    const size_t Pl = P0 >> (2 * l), cl = n->c[l];
    ok = dalloc(*n, &n->eab[l], Pl * cl) && dalloc(*n, &n->ebb[l], Pl * cl);
    if (ok && l < L - 1)
      ok = dalloc(*n, &n->poolb[l], (Pl / 4) * cl) && dalloc(*n, &n->upinb[l], Pl * (size_t)n->c[l + 1]) &&
           dalloc(*n, &n->upoutb[l], Pl * cl) && dalloc(*n, &n->dab[l], Pl * cl);
  }
  ok = ok && dalloc(*n, &n->X0, P0 * 32) && dalloc(*n, &n->out, P0) && dalloc(*n, &n->g_out, P0) &&
       dalloc(*n, &n->loss_part, 1024) && dalloc(*n, &n->norm_part, 152 * 16) && dalloc(*n, &n->d_gnorm, 1) &&
       dalloc(*n, &n->d_gscale, 1) && dalloc(*n, &n->d_err, 1) && dalloc(*n, &n->gradb, P0 * n->c[0]);
  for (int l = 0; l < L && ok; ++l) {
    const size_t Pl = P0 >> (2 * l), cl = n->c[l];
    ok = dalloc(*n, &n->ea[l], Pl * cl) && dalloc(*n, &n->eb[l], Pl * cl) && dalloc(*n, &n->g_ea[l], Pl * cl) &&
         dalloc(*n, &n->g_eb[l], Pl * cl);
    if (ok && l < L - 1) {
      const size_t c1 = n->c[l + 1];
      ok = dalloc(*n, &n->pool[l], (Pl / 4) * cl) && dalloc(*n, &n->g_pool[l], (Pl / 4) * cl) &&
           dalloc(*n, &n->upin[l], Pl * c1) && dalloc(*n, &n->g_upin[l], Pl * c1) &&
           dalloc(*n, &n->upout[l], Pl * cl) && dalloc(*n, &n->g_upout[l], Pl * cl) &&
           dalloc(*n, &n->da[l], Pl * cl) && dalloc(*n, &n->g_da[l], Pl * cl) && dalloc(*n, &n->db[l], Pl * cl) &&
           dalloc(*n, &n->g_db[l], Pl * cl) && dalloc(*n, &n->g_skip[l], Pl * cl);
    }
  }
  // split partials: the largest weight-gradient split of any layer, the
  // bias and head sums
  size_t part = 0;
  for (int li = 0; li < (int)n->layers.size() && ok; ++li) {
    const Layer& Ly = n->layers[li];
    if (Ly.k != 3) continue;
    int bm, bn, sp, cps;
    for (const bool b16 : {false, true})
      part = std::max(part,
                      wgrad_splits(Ly.cout, Ly.c1, Ly.c2, (long long)(P0 >> (2 * Ly.lv)), &bm, &bn, &sp, &cps, b16));
    const long long Pl = (long long)(P0 >> (2 * Ly.lv));
    part = std::max(part, (size_t)((Pl + colsum_rows(Pl) - 1) / colsum_rows(Pl)) * (size_t)Ly.cout);
  }
  part = std::max(part, (size_t)((P0 + 2047) / 2048) * (size_t)(n->c[0] + 1));
  ok = ok && dalloc(*n, &n->part, part);
  n->part_floats = part;
  if (ok) {
    ok = cudaMemsetAsync(n->param, 0, sizeof(float) * n->n_param, stream) == cudaSuccess &&
         cudaMemsetAsync(n->grad, 0, sizeof(float) * n->n_param, stream) == cudaSuccess &&
         cudaMemsetAsync(n->adam_m, 0, sizeof(float) * n->n_param, stream) == cudaSuccess &&
         cudaMemsetAsync(n->adam_v, 0, sizeof(float) * n->n_param, stream) == cudaSuccess &&
         cudaMemsetAsync(n->d_err, 0, sizeof(int), stream) == cudaSuccess;
    refresh_bf16(*n, stream);
    ok = ok && cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(stream) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_net(n);
    return CPCT_ENOMEM;
  }
  cpct_unet* h = new (std::nothrow) cpct_unet;
  if (!h) {
    free_net(n);
    return CPCT_ENOMEM;
  }
  h->net = n;
  *out = h;
  return CPCT_OK;
}

extern "C" int cpct_unet_destroy(cpct_unet* net) {
  if (!net) return CPCT_OK;
  cudaDeviceSynchronize();
  free_net(net->net);
  delete net;
  return CPCT_OK;
}

// copy between the caller's layout (per layer: W (Cout, k, k, Cin), b) and
// the padded device layout; to_device selects the direction
static int params_copy(Net& n, float* h, const float* dev_src, float* dev_dst, cudaStream_t s, bool to_device) {
  std::vector<float> pad(n.n_param, 0.f);
  if (!to_device) {
    if (cudaMemcpyAsync(pad.data(), dev_src, sizeof(float) * n.n_param, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return CPCT_ECUDA;
  }
  for (const Layer& L : n.layers) {
    const int kk = L.k * L.k;
    for (int co = 0; co < L.cout; ++co)
      for (int t = 0; t < kk; ++t)
        for (int ci = 0; ci < L.cin; ++ci) {
          const size_t hi = L.host_off + ((size_t)co * kk + t) * L.cin + ci;
          const size_t di = L.w_off + ((size_t)co * kk + t) * L.cin_pad + ci;
          if (to_device) pad[di] = h[hi];
          else h[hi] = pad[di];
        }
    const size_t hb = L.host_off + (size_t)L.cout * kk * L.cin;
    for (int co = 0; co < L.cout; ++co) {
      if (to_device) pad[L.b_off + co] = h[hb + co];
      else h[hb + co] = pad[L.b_off + co];
    }
  }
  if (to_device) {
    if (cudaMemcpyAsync(dev_dst, pad.data(), sizeof(float) * n.n_param, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return CPCT_ECUDA;
  }
  return CPCT_OK;
}

extern "C" int cpct_unet_set_params(cpct_unet* net, const float* h_params, cudaStream_t stream) {
  if (!net || !h_params) return CPCT_EINVAL;
  Net& n = *net->net;
  int rc = params_copy(n, const_cast<float*>(h_params), nullptr, n.param, stream, true);
  if (rc) return rc;
  if (cudaMemsetAsync(n.adam_m, 0, sizeof(float) * n.n_param, stream) != cudaSuccess ||
      cudaMemsetAsync(n.adam_v, 0, sizeof(float) * n.n_param, stream) != cudaSuccess)
    return CPCT_ECUDA;
  n.adam_t = 0;
  refresh_bf16(n, stream);
  return cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(stream) == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

extern "C" int cpct_unet_get_params(cpct_unet* net, float* h_params, cudaStream_t stream) {
  if (!net || !h_params) return CPCT_EINVAL;
  return params_copy(*net->net, h_params, net->net->param, nullptr, stream, false);
}

extern "C" int cpct_unet_get_grads(cpct_unet* net, float* h_grads, cudaStream_t stream) {
  if (!net || !h_grads) return CPCT_EINVAL;
  return params_copy(*net->net, h_grads, net->net->grad, nullptr, stream, false);
}

static bool unet_ptr_ok(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

extern "C" int cpct_unet_forward(cpct_unet* net, const float* d_in, float* d_out, int batch, cudaStream_t stream) {
  if (!net || !unet_ptr_ok(d_in) || !unet_ptr_ok(d_out)) return CPCT_EINVAL;
  Net& n = *net->net;
  if (batch < 1 || batch > n.maxB) return CPCT_EINVAL;
  forward_pass(n, d_in, batch, stream, false);
  const size_t P0 = (size_t)batch * n.H * n.W;
  if (cudaMemcpyAsync(d_out, n.out, sizeof(float) * P0, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
    return CPCT_ECUDA;
  return cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

extern "C" int cpct_unet_sync(cpct_unet* net, cudaStream_t stream) {
  if (!net) return CPCT_EINVAL;
  Net& n = *net->net;
  int err = 0;
  if (cudaMemcpyAsync(&err, n.d_err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return CPCT_ECUDA;
  if (err) {
    if (cudaMemsetAsync(n.d_err, 0, sizeof(int), stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return CPCT_ECUDA;
    return CPCT_ETIMEOUT;
  }
  return CPCT_OK;
}

extern "C" int cpct_unet_backward(cpct_unet* net, const float* d_in, const float* d_target, int batch, double* loss,
                                  cudaStream_t stream) {
  if (!net || !unet_ptr_ok(d_in) || !unet_ptr_ok(d_target)) return CPCT_EINVAL;
  Net& n = *net->net;
  if (batch < 1 || batch > n.maxB) return CPCT_EINVAL;
  forward_pass(n, d_in, batch, stream, true);
  backward_pass(n, d_in, d_target, batch, stream);
  if (cudaGetLastError() != cudaSuccess) return CPCT_ECUDA;
  if (loss) {
    const int P0 = batch * n.H * n.W;
    const int lg = std::min(1024, (P0 + kEW - 1) / kEW);
    std::vector<double> part(lg);
    if (cudaMemcpyAsync(part.data(), n.loss_part, sizeof(double) * lg, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return CPCT_ECUDA;
    double s = 0.0;
    for (double v : part) s += v;
    *loss = s / (2.0 * P0);
  }
  return CPCT_OK;
}

extern "C" int cpct_unet_adam_step(cpct_unet* net, float lr, float max_grad_norm, double* grad_norm,
                                   cudaStream_t stream) {
  if (!net || !(lr > 0.f) || !(max_grad_norm >= 0.f)) return CPCT_EINVAL;
  Net& n = *net->net;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  n.adam_t++;
  const double lr_t = lr * std::sqrt(1.0 - std::pow((double)b2, n.adam_t)) / (1.0 - std::pow((double)b1, n.adam_t));
  const int nb = grid_for((long long)n.n_param);
  k_sumsq<<<nb, kEW, 0, stream>>>(n.grad, (long long)n.n_param, n.norm_part);
  k_clip_scale<<<1, 32, 0, stream>>>(n.norm_part, nb, max_grad_norm, n.d_gscale, n.d_gnorm);
  k_adam<<<nb, kEW, 0, stream>>>(n.param, n.grad, n.adam_m, n.adam_v, (long long)n.n_param, (float)lr_t, b1, b2,
                                 eps, n.d_gscale);
  refresh_bf16(n, stream);
  if (cudaGetLastError() != cudaSuccess) return CPCT_ECUDA;
  if (grad_norm) {
    if (cudaMemcpyAsync(grad_norm, n.d_gnorm, sizeof(double), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return CPCT_ECUDA;
  }
  return CPCT_OK;
}

// One network operation on caller tensors (NHWC, device float32), for tests:
//   op 0: y = relu(conv3x3([a | b]) + bias), weights h_w (host float32,
//         [Cout][3][3][C1 + C2] followed by Cout biases)
//   op 1: y = 2x2 average pool of a (C1 channels)
//   op 2: y = nearest 2x upsampling of a
//   op 3: y = adjoint of the pooling applied to a (half-size), plus b
//   op 4: y = adjoint of the upsampling applied to a (double-size)
//   op 5: y = data gradient of op 0 at output gradient a with ReLU mask b
//         (a, b: Cout channels; y: C1 + C2 channels, one tensor)
//   op 7: op 0 through the forward kernel that reads BF16 copies of a, b
//   op 6: y = weight and bias gradients of op 0's convolution (no mask) at
//         input a (C1 channels) and output gradient b (Cout channels):
//         [Cout][3][3][C1] weights, then Cout biases
extern "C" int cpct_unet_debug_op(int op, const float* d_a, const float* d_b, float* d_y, const float* h_w, int B,
                                  int H, int W, int C1, int C2, int Cout, cudaStream_t stream) {
  if (op == 10) {
    // first layer: one input channel, weights [Cout][3][3][1] + bias
    if (!d_a || !d_y || !h_w || B < 1 || H < 1 || W < 1 || C1 != 1 || C2 != 0 || Cout < 8 || Cout % 8 ||
        Cout > kFirstMaxC)
      return CPCT_EINVAL;
    const size_t nw = (size_t)Cout * 9 * 32;
    std::vector<float> hp(nw + Cout, 0.f);
    for (int co = 0; co < Cout; ++co)
      for (int t = 0; t < 9; ++t) hp[((size_t)co * 9 + t) * 32] = h_w[co * 9 + t];
    for (int co = 0; co < Cout; ++co) hp[nw + co] = h_w[(size_t)Cout * 9 + co];
    float* dw = nullptr;
    __nv_bfloat16* bf = nullptr;
    if (cudaMalloc(&dw, sizeof(float) * (nw + Cout)) != cudaSuccess) return CPCT_ENOMEM;
    if (cudaMalloc(&bf, sizeof(__nv_bfloat16) * 2 * nw) != cudaSuccess) {
      cudaFree(dw);
      return CPCT_ENOMEM;
    }
    int rc = cudaMemcpyAsync(dw, hp.data(), sizeof(float) * hp.size(), cudaMemcpyHostToDevice, stream) == cudaSuccess
                 ? CPCT_OK
                 : CPCT_ECUDA;
    if (rc == CPCT_OK) {
      k_weights_bf16<<<grid_for((long long)nw), kEW, 0, stream>>>(dw, bf, bf + nw, Cout, 32);
      __nv_bfloat16* yb = nullptr;
      if (cudaMalloc(&yb, sizeof(__nv_bfloat16) * B * H * W * Cout) != cudaSuccess) rc = CPCT_ENOMEM;
      if (rc == CPCT_OK)
        k_conv_first<<<row_grid(W, B * H), kEW, 0, stream>>>(d_a, bf, dw + nw, d_y, yb, B, H, W, Cout);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess) rc = CPCT_ECUDA;
      if (yb) cudaFree(yb);
    }
    cudaFree(bf);
    cudaFree(dw);
    return rc;
  }
  if (!d_a || !d_y || B < 1 || H < 1 || W < 1 || C1 < 1 || C1 % 32 || C2 < 0 || C2 % 32) return CPCT_EINVAL;
  if (op == 6 || op == 12) {
    if (!d_b || C2 != 0 || Cout < 32 || Cout % 32) return CPCT_EINVAL;
    const long long P = (long long)B * H * W;
    const bool b16 = op == 12;
    int bm, bn, sp, cps;
    size_t need = wgrad_splits(Cout, C1, 0, P, &bm, &bn, &sp, &cps, b16);
    const int rows = (int)colsum_rows(P), csp = (int)((P + rows - 1) / rows);
    need = std::max(need, (size_t)csp * Cout);
    float* part = nullptr;
    if (cudaMalloc(&part, sizeof(float) * need) != cudaSuccess) return CPCT_ENOMEM;
    __nv_bfloat16* cb = nullptr;  // op 12: BF16 copies of x (P x C1) and dz (P x Cout)
    if (b16) {
      if (cudaMalloc(&cb, sizeof(__nv_bfloat16) * P * (C1 + Cout)) != cudaSuccess) {
        cudaFree(part);
        return CPCT_ENOMEM;
      }
      k_to_bf16x4<<<grid_for(P * C1 / 4), kEW, 0, stream>>>(reinterpret_cast<const float4*>(d_a),
                                                             reinterpret_cast<uint2*>(cb), P * C1 / 4);
      k_to_bf16x4<<<grid_for(P * Cout / 4), kEW, 0, stream>>>(reinterpret_cast<const float4*>(d_b),
                                                               reinterpret_cast<uint2*>(cb + P * C1), P * Cout / 4);
    }
    WgradArgs w{};
    w.dz = d_b;
    w.x1 = d_a;
    w.x2 = nullptr;
    w.C1 = C1;
    w.C2 = 0;
    w.Cout = Cout;
    w.B = B;
    w.H = H;
    w.Wd = W;
    w.chunks_per_split = cps;
    w.part = part;
    w.xb1 = cb;
    w.dzb = cb ? cb + P * C1 : nullptr;
    if (b16)
      launch_wgrad_b16(w, bm, bn, sp, stream);
    else
      launch_wgrad(w, bm, bn, sp, stream);
    const long long nw = (long long)Cout * 9 * C1;
    k_split_sum<<<grid_for(nw), kEW, 0, stream>>>(part, sp, nw, d_y, 0);
    dim3 cg((Cout + 31) / 32, csp);
    k_colsum<<<cg, kEW, 0, stream>>>(d_b, nullptr, (int)P, Cout, rows, part);
    k_split_sum<<<grid_for(Cout), kEW, 0, stream>>>(part, csp, Cout, d_y + nw, 0);
    const int rc = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(stream) == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
    if (cb) cudaFree(cb);
    cudaFree(part);
    return rc;
  }
  if (op == 0 || op == 5 || op == 7 || op == 8 || op == 9 || op == 11) {
    if (!h_w || Cout < 32 || Cout % 32 || ((op == 5 || op == 11) && !d_b)) return CPCT_EINVAL;
    if ((op == 8 || op == 9) && !tc_bn(Cout)) return CPCT_EINVAL;
    if (op == 11 && (C2 != 0 || !tc_bn(C1))) return CPCT_EINVAL;
    const int Cin = C1 + C2;
    const size_t nw = (size_t)Cout * 9 * Cin;
    float* dw = nullptr;
    __nv_bfloat16* bf = nullptr;
    if (cudaMalloc(&dw, sizeof(float) * (nw + Cout)) != cudaSuccess) return CPCT_ENOMEM;
    if (cudaMalloc(&bf, sizeof(__nv_bfloat16) * 2 * nw) != cudaSuccess) {
      cudaFree(dw);
      return CPCT_ENOMEM;
    }
    int rc = CPCT_OK;
    if (cudaMemcpyAsync(dw, h_w, sizeof(float) * (nw + Cout), cudaMemcpyHostToDevice, stream) != cudaSuccess)
      rc = CPCT_ECUDA;
    if (rc == CPCT_OK) {
      k_weights_bf16<<<grid_for((long long)nw), kEW, 0, stream>>>(dw, bf, bf + nw, Cout, Cin);
      ConvArgs a{};
      a.B = B;
      a.H = H;
      a.Wd = W;
      __nv_bfloat16* xb = nullptr;
      int* derr = nullptr;
      if (op == 0 || op == 7 || op == 8 || op == 9) {
        a.x1 = d_a;
        a.x2 = d_b;
        a.C1 = C1;
        a.C2 = C2;
        a.W = bf;
        a.bias = dw + nw;
        a.y1 = d_y;
        a.O1 = Cout;
        a.Cout = Cout;
        a.relu = 1;
        if (op >= 8) {
          if (cudaMalloc(&derr, sizeof(int)) != cudaSuccess ||
              cudaMemsetAsync(derr, 0, sizeof(int), stream) != cudaSuccess)
            rc = CPCT_ENOMEM;
          a.err = derr;
        }
        if (op >= 7) {
          const long long n1 = (long long)B * H * W * C1, n2 = (long long)B * H * W * C2;
          if (cudaMalloc(&xb, sizeof(__nv_bfloat16) * (n1 + n2 + 8)) != cudaSuccess) rc = CPCT_ENOMEM;
          if (rc == CPCT_OK) {
            k_to_bf16<<<grid_for(n1), kEW, 0, stream>>>(d_a, xb, n1);
            a.xb1 = xb;
            if (C2) {
              k_to_bf16<<<grid_for(n2), kEW, 0, stream>>>(d_b, xb + n1, n2);
              a.xb2 = xb + n1;
            }
          }
        }
      } else {
        // pre-activation gradient dz = a * (b > 0), then the data gradient
        float* dz = nullptr;
        const long long nz = (long long)B * H * W * Cout;
        if (cudaMalloc(&dz, sizeof(float) * nz) != cudaSuccess) rc = CPCT_ENOMEM;
        if (rc == CPCT_OK) {
          k_relu_mask<<<grid_for(nz), kEW, 0, stream>>>(d_a, d_b, dz, nz);
          if (op == 11) {
            // tensor-memory kernel on the BF16 copy of dz
            if (cudaMalloc(&xb, sizeof(__nv_bfloat16) * nz) != cudaSuccess ||
                cudaMalloc(&derr, sizeof(int)) != cudaSuccess || cudaMemsetAsync(derr, 0, sizeof(int), stream) != cudaSuccess)
              rc = CPCT_ENOMEM;
            if (rc == CPCT_OK)
              k_to_bf16x4<<<grid_for(nz / 4), kEW, 0, stream>>>(reinterpret_cast<const float4*>(dz),
                                                                reinterpret_cast<uint2*>(xb), nz / 4);
            a.xb1 = xb;
            a.err = derr;
          }
          a.x1 = dz;
          a.C1 = Cout;
          a.C2 = 0;
          a.W = bf + nw;
          a.y1 = d_y;
          a.O1 = Cin;
          a.Cout = Cin;
          if (rc == CPCT_OK) launch_conv(a, stream);
          if (cudaStreamSynchronize(stream) != cudaSuccess) rc = CPCT_ECUDA;
          cudaFree(dz);
        }
      }
      if (rc == CPCT_OK && (op == 0 || op == 7 || op == 8 || op == 9)) launch_conv(a, stream, op == 9);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess) rc = CPCT_ECUDA;
      if (derr) {
        int e = 0;
        if (rc == CPCT_OK && cudaMemcpy(&e, derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = CPCT_ECUDA;
        if (rc == CPCT_OK && e) rc = CPCT_ETIMEOUT;
        cudaFree(derr);
      }
      if (xb) cudaFree(xb);
    }
    cudaFree(bf);
    cudaFree(dw);
    return rc;
  }
  const long long n4 = (long long)B * H * W * C1 / 4;
  switch (op) {
    case 1:
      k_avgpool<<<row_grid((W / 2) * C1 / 4, B * (H / 2)), kEW, 0, stream>>>(d_a, d_y, nullptr, B, H, W, C1);
      break;
    case 2:
      k_upsample<<<row_grid(W * C1 / 4, B * H), kEW, 0, stream>>>(d_a, d_y, nullptr, B, H, W, C1);
      break;
    case 3:
      k_avgpool_bwd<<<row_grid(W * C1 / 4, B * H), kEW, 0, stream>>>(d_a, d_b, nullptr, d_y, B, H, W, C1);
      break;
    case 4:
      k_upsample_bwd<<<grid_for(n4), kEW, 0, stream>>>(d_a, nullptr, d_y, B, H, W, C1);
      break;
    default:
      return CPCT_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(stream) == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

// ---------------------------------------------------------------------------
// tcgen05 check: D (128 x N, FP32) = A (128 x K, BF16) * B (N x K, BF16)^T with
// one CTA, the accumulator in tensor memory (for tests of the descriptors and
// of the MMA / commit / load sequence)
// ---------------------------------------------------------------------------
namespace {

constexpr long long kTcWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

template <int N>
__global__ void __launch_bounds__(128) k_tc_gemm_check(const __nv_bfloat16* __restrict__ A,
                                                       const __nv_bfloat16* __restrict__ B, float* __restrict__ D,
                                                       int K, int* __restrict__ err) {
  __shared__ __align__(1024) unsigned char sA[128 * 32 * 2];
  __shared__ __align__(1024) unsigned char sB[N * 32 * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    cpct::tc_alloc(smem_u32(&tslot), N);
    cpct::tc_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  cpct::tc_fence_before();
  __syncthreads();
  cpct::tc_fence_after();
  const uint32_t tbase = tslot;
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K && ok; k0 += 32) {
    // K-major core-matrix layout: (row / 8) * 512 + (k / 8) * 128 + (row % 8) * 16
    for (int q = tid; q < 128 * 4; q += 128) {
      const int r = q >> 2, c = q & 3;
      cp_async16(smem_u32(sA + (r >> 3) * 512 + c * 128 + (r & 7) * 16), A + (size_t)r * K + k0 + 8 * c);
    }
    for (int q = tid; q < N * 4; q += 128) {
      const int r = q >> 2, c = q & 3;
      cp_async16(smem_u32(sB + (r >> 3) * 512 + c * 128 + (r & 7) * 16), B + (size_t)r * K + k0 + 8 * c);
    }
    cp_async_commit();
    cp_async_wait_all();
    cpct::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      cpct::tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint64_t ad = cpct::tc_smem_desc(smem_u32(sA) + kk * 256, 128, 512);
        const uint64_t bd = cpct::tc_smem_desc(smem_u32(sB) + kk * 256, 128, 512);
        cpct::tc_mma_bf16(tbase, ad, bd, cpct::tc_idesc_bf16(128, N), k0 > 0 || kk > 0);
      }
      cpct::tc_commit(&bar);
    }
    const bool w = mbar_wait_bounded(&bar, phase, kTcWaitCycles);
    phase ^= 1u;
    ok = __syncthreads_and(w);
    cpct::tc_fence_after();
  }
  if (ok) {
#pragma unroll
    for (int j = 0; j < N / 8; ++j) {
      float v[8];
      cpct::tc_ld8(tbase + ((uint32_t)(warp * 32) << 16) + j * 8, v);
      cpct::tc_wait_ld();
      const int row = warp * 32 + lane;
#pragma unroll
      for (int i = 0; i < 8; ++i) D[(size_t)row * N + j * 8 + i] = v[i];
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  cpct::tc_fence_before();
  __syncthreads();
  if (warp == 0) cpct::tc_dealloc(tbase, N);
}

}  // namespace

// D = A * B^T on the tensor cores (tcgen05); A 128 x K, B N x K (BF16,
// row-major, device), D 128 x N (FP32, device); K a multiple of 32, N in
// {32, 64, 128}.  Test introspection only.
extern "C" int cpct_debug_tc_gemm(const void* d_a, const void* d_b, float* d_d, int n, int k, cudaStream_t stream) {
  if (!d_a || !d_b || !d_d || k < 32 || k % 32 || (n != 32 && n != 64 && n != 128)) return CPCT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_a) & 15u) || (reinterpret_cast<uintptr_t>(d_b) & 15u)) return CPCT_EINVAL;
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return CPCT_ENOMEM;
  int rc = cudaMemsetAsync(err, 0, sizeof(int), stream) == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
  const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(d_a);
  const __nv_bfloat16* B = static_cast<const __nv_bfloat16*>(d_b);
  if (rc == CPCT_OK) {
    if (n == 32) k_tc_gemm_check<32><<<1, 128, 0, stream>>>(A, B, d_d, k, err);
    else if (n == 64) k_tc_gemm_check<64><<<1, 128, 0, stream>>>(A, B, d_d, k, err);
    else k_tc_gemm_check<128><<<1, 128, 0, stream>>>(A, B, d_d, k, err);
  }
  int h_err = 0;
  if (rc == CPCT_OK && (cudaGetLastError() != cudaSuccess ||
                        cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                        cudaStreamSynchronize(stream) != cudaSuccess))
    rc = CPCT_ECUDA;
  cudaFree(err);
  if (rc == CPCT_OK && h_err) rc = CPCT_ETIMEOUT;
  return rc;
}
