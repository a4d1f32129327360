// Ring-artifact filter and the SPGL1 basis-pursuit solver on the device.
//
// Section "Introduction": the reconstruction solves
//     min ||x||_1  subject to  ||filter(Radon{x} - data)||_2 < eps
// with SPGL1 (van den Berg and Friedlander 2008), which needs only the
// operator and its adjoint.  The filter is a 3rd-order polynomial
// subtraction; read here as the orthogonal projector
//     F y = y - 1_M (m - Pi_3 m),  m[s] = mean_j y[j, s],
// with Pi_3 the least-squares cubic fit over the detector coordinate s.
// Because F is a projector the problem is SPGL1 on A = F R with b = F data.
//
// The solver runs as a state machine on the device: every "tick" is the same
// fixed sequence of kernels (projection onto the l1 ball, forward operator,
// filter + residual, a mid-tick FP64 controller, the adjoint, gradient
// update, an end-of-tick FP64 controller), captured once in a CUDA graph and
// replayed; the controllers take every data-dependent decision (Armijo test,
// step halving, Barzilai-Borwein step, duality gap, Newton update of tau on
// the Pareto curve, termination) in FP64, so the host only replays the graph
// and polls a done flag.  All reductions are deterministic: fixed grids,
// per-block partials, fixed-order trees.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kRB = 256;        // threads of the reduction / vector kernels
constexpr int kRG = 256;        // blocks of the grid-stride vector kernels

// ---------------------------------------------------------------------------
// deterministic block reductions (warp shuffles in a fixed pattern, then the
// warps' results in warp order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// sums NQ values over the block; thread 0 gets the result (others: undefined)
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ]) {
  __shared__ double sh[NQ][kRB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    v[q] = warp_sum(v[q]);
    if (lane == 0) sh[q][w] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[q][i];
      v[q] = s;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// ring filter
// ---------------------------------------------------------------------------
// Orthonormal basis Q (Ns x 4, FP64) of cubics on s = 0..Ns-1, by modified
// Gram-Schmidt on the monomials of t = (s - (Ns-1)/2) / (Ns/2).  One block.
__global__ void __launch_bounds__(kRB) k_build_cubic(double* __restrict__ Q, int ns) {
  for (int d = 0; d < 4; ++d) {
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
      const double t = (s - 0.5 * (ns - 1)) / (0.5 * ns);
      Q[d * ns + s] = d == 0 ? 1.0 : d == 1 ? t : d == 2 ? t * t : t * t * t;
    }
    __syncthreads();
    for (int e = 0; e <= d; ++e) {
      double v[1] = {0.0};
      for (int s = threadIdx.x; s < ns; s += blockDim.x)
        v[0] += (e < d ? Q[e * ns + s] : Q[d * ns + s]) * Q[d * ns + s];
      block_sum<1>(v);
      __shared__ double coef;
      if (threadIdx.x == 0) coef = v[0];
      __syncthreads();
      const double c = coef;
      for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        if (e < d) Q[d * ns + s] -= c * Q[e * ns + s];
        else Q[d * ns + s] /= sqrt(c);
      }
      __syncthreads();
    }
  }
}

// column means m[s] = (1/M) sum_j y[j, s]: 32 columns x 8 row slices per
// block, slices summed in order
__global__ void __launch_bounds__(kRB) k_ring_colmean(const float* __restrict__ y, double* __restrict__ m, int M,
                                                      int ns) {
  __shared__ double part[8][33];
  const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + c;
  double acc = 0.0;
  if (s < ns)
    for (int j = r; j < M; j += 8) acc += (double)y[(size_t)j * ns + s];
  part[r][c] = acc;
  __syncthreads();
  if (r == 0 && s < ns) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += part[i][c];
    m[s] = t / M;
  }
}

// offset removed from every row: d[s] = m[s] - (Pi_3 m)[s]
__global__ void __launch_bounds__(kRB) k_ring_offset(const double* __restrict__ Q, const double* __restrict__ m,
                                                     float* __restrict__ d, int ns) {
  double c[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s = threadIdx.x; s < ns; s += blockDim.x)
    for (int q = 0; q < 4; ++q) c[q] += Q[q * ns + s] * m[s];
  block_sum<4>(c);
  __shared__ double cc[4];
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) cc[q] = c[q];
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    double fit = 0.0;
    for (int q = 0; q < 4; ++q) fit += cc[q] * Q[q * ns + s];
    d[s] = (float)(m[s] - fit);
  }
}

__global__ void __launch_bounds__(kRB) k_ring_apply(const float* __restrict__ y, const float* __restrict__ d,
                                                    float* __restrict__ out, int M, int ns) {
  const size_t total = (size_t)M * ns;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    out[i] = y[i] - d[i % ns];
}

}  // namespace

// filter workspace of a plan (basis + column means + offsets), built lazily
struct RingWork {
  double* Q = nullptr;
  double* m = nullptr;
  float* d = nullptr;
  int ns = 0;
};

static int ring_work(int ns, RingWork& w, cudaStream_t s) {
  if (cudaMalloc(&w.Q, sizeof(double) * 4 * ns) != cudaSuccess) return CPCT_ENOMEM;
  if (cudaMalloc(&w.m, sizeof(double) * ns) != cudaSuccess) return CPCT_ENOMEM;
  if (cudaMalloc(&w.d, sizeof(float) * ns) != cudaSuccess) return CPCT_ENOMEM;
  w.ns = ns;
  k_build_cubic<<<1, kRB, 0, s>>>(w.Q, ns);
  return cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

static void ring_free(RingWork& w) {
  if (w.Q) cudaFree(w.Q);
  if (w.m) cudaFree(w.m);
  if (w.d) cudaFree(w.d);
  w = RingWork();
}

static void ring_launch(const RingWork& w, const float* y, float* out, int M, int ns, cudaStream_t s) {
  k_ring_colmean<<<(ns + 31) / 32, kRB, 0, s>>>(y, w.m, M, ns);
  k_ring_offset<<<1, kRB, 0, s>>>(w.Q, w.m, w.d, ns);
  if (out) k_ring_apply<<<kRG, kRB, 0, s>>>(y, w.d, out, M, ns);
}

extern "C" int cpct_ring_filter(cpct_plan* p, const float* d_in, float* d_out, cudaStream_t stream) {
  if (!p || !d_in || !d_out) return CPCT_EINVAL;
  RingWork w;
  int rc = ring_work(p->ns, w, stream);
  if (rc == CPCT_OK) {
    ring_launch(w, d_in, d_out, p->m, p->ns, stream);
    rc = cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = CPCT_ECUDA;
  }
  ring_free(w);
  return rc;
}

// ---------------------------------------------------------------------------
// SPGL1 state machine
// ---------------------------------------------------------------------------
namespace {

// tick types: the initial point, the initial step length (projected
// gradient, no operator), the projection onto a shrunk ball, a trial on the
// projection arc, a trial along the fixed feasible direction
enum TickType { T_INIT = 0, T_PG = 1, T_PROJX = 2, T_TRIAL = 3, T_FEAS = 4 };
constexpr int kHist = 8;        // objective history capacity (memory <= 8)
// l1-ball projection by radix selection on the FP32 bit patterns of |v|
// (non-negative floats order like their patterns): three passes over bits
// 30..20, 19..9 and 8..0; a bin of any pass holds values of one exponent, so
// its sum is an exact integer sum of 24-bit significands times a power of 2
constexpr int kRadixPasses = 3;
constexpr int kBins = 2048;
__host__ __device__ constexpr int radix_shift(int p) { return p == 0 ? 20 : p == 1 ? 9 : 0; }
__host__ __device__ constexpr int radix_bits(int p) { return p == 2 ? 9 : 11; }

struct SpgState {
  // options
  double sigma, opt_tol, bp_tol, ls_tol, dec_tol, gamma, step_min, step_max;
  int max_iter, max_line, memory, single_tau;
  // solver scalars (FP64)
  double tau, bnorm, f, f_old, fmax, gstep, rtb, ginf, gnorm2;
  double fhist[kHist];
  double rel_gap, rnorm;
  int upd_last, line_errors_left, n_newton, n_line_errors;
  // this tick
  int type, accept_x, accept_r, update_g, stationary, go_feas, line_err, store_dir;
  double ps;      // trial point P_tau(x - ps g) (arc, init, projected gradient)
  double feas_t;  // trial point x + feas_t d (feasible direction)
  // the arc search of this iteration
  double step, scale, sn_prev, f1, gtd1;
  int nsafe, n_line, n_feas, n_safeguard, n_stationary;
  int n_nodescent;   // consecutive iterations whose first arc trial had no descent
  int pg_end_iter;   // the T_PG tick ends an iteration (step restart) rather than the set-up
  // projection of v = x - ps g onto the l1 ball of radius tau
  double theta, c_above, s_above;  // threshold; count and sum of |v| above the selected prefix
  unsigned prefix;                  // selected high bits of the pattern of theta
  int proj_done, proj_identity, proj_zero;
  // mid-tick results
  double ft, gtd, dn2, dinf, rtb_t;
  // counters / status
  int iter, status, done, ticks, n_trials;
  // the tick's adjoint operator is skipped (its output unused) while set:
  // no gradient update, or the slice is done
  int skip_adj;
  // the tick's forward operator is skipped while set: the slice is done, or
  // the tick is the projected-gradient step-length tick (T_PG), which reads
  // only x and g and accepts nothing
  int skip_fwd;
};

// SPGL1 status codes (spgl1_info.status)
enum {
  S_RUNNING = 0, S_ROOT = 1, S_BP = 2, S_ITER = 3, S_LINE = 4, S_NONFINITE = 5, S_LS = 6, S_SUBOPT = 7,
  S_OPTIMAL = 8
};

struct SpgVec {
  float *x, *xt, *xold, *g, *gold, *gtmp;  // image space, n
  float* dir;                              // image space, n: feasible direction d
  float *y, *rt, *r, *bf;                  // sinogram space, m
  double* part;                            // per-block partials
  unsigned* hcnt;                          // radix histogram: counts (kBins)
  unsigned long long* hsum;                // radix histogram: significand sums (kBins)
  SpgState* st;
  long long n, m;
};

// partial buffer regions (each kRG doubles per quantity)
constexpr int P_APPLY = 0;                  // 3: gtd, dn2, dinf
constexpr int P_RES = P_APPLY + 3;          // 2: sum rt^2, sum rt*bf
constexpr int P_GRAD = P_RES + 2;           // 4: sts, sty, ginf, gnorm2
constexpr int P_TOTAL = P_GRAD + 4;

// FP64 throughput is a small fraction of FP32 on this GPU, so every
// per-element operation and per-thread / per-warp partial is FP32 (counts are
// integers) and FP64 only combines the 8 warp partials of a block and the 256
// block partials of a grid, in a fixed order.
template <int NQ>
__device__ __forceinline__ void block_sum_f(float (&v)[NQ], double (&out)[NQ]) {
  __shared__ float sh[NQ][kRB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float t = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh[q][w] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double t = 0.0;
      for (int i = 0; i < kRB / 32; ++i) t += (double)sh[q][i];
      out[q] = t;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float block_max_f(float v) {
  __shared__ float sh[kRB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i < kRB / 32; ++i) v = fmaxf(v, sh[i]);
  __syncthreads();
  return v;
}

__device__ __forceinline__ void put(double* part, int q, double v) { part[(size_t)q * kRG + blockIdx.x] = v; }

// v_i = x_i - ps g_i (FP32)
__device__ __forceinline__ float vval(const SpgVec& V, float ps, long long i) { return fmaf(-ps, V.g[i], V.x[i]); }

#define SPG_LOOP(i, len) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (len); i += (long long)gridDim.x * blockDim.x)

// histogram of the patterns u of |v_i| that carry the prefix selected so far
// (pass 0: all), binned by the pass's bits; zeros are skipped (they never lie
// above a threshold >= 0).  Shared-memory integer atomics, then one global
// integer atomic per non-empty bin: the result is independent of order.
__global__ void __launch_bounds__(kRB) k_spg_radix_hist(SpgVec V, int pass) {
  const SpgState* st = V.st;
  if (st->done || st->type == T_FEAS || (pass > 0 && st->proj_done)) return;
  __shared__ unsigned hc[kBins];
  __shared__ unsigned long long hs[kBins];
  for (int b = threadIdx.x; b < kBins; b += kRB) {
    hc[b] = 0u;
    hs[b] = 0ull;
  }
  __syncthreads();
  const float ps = (float)st->ps;
  const int shift = radix_shift(pass), top = shift + radix_bits(pass);
  const unsigned mask = (1u << radix_bits(pass)) - 1u;
  const unsigned prefix = pass > 0 ? st->prefix : 0u;
  SPG_LOOP(i, V.n) {
    const unsigned u = __float_as_uint(fabsf(vval(V, ps, i)));
    if (u == 0u || (u >> top) != prefix) continue;
    const unsigned e = u >> 23;
    const unsigned sig = (u & 0x7fffffu) | (e ? 0x800000u : 0u);
    const unsigned b = (u >> shift) & mask;
    atomicAdd(&hc[b], 1u);
    atomicAdd(&hs[b], (unsigned long long)sig);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += kRB)
    if (hc[b]) {
      atomicAdd(&V.hcnt[b], hc[b]);
      atomicAdd(&V.hsum[b], hs[b]);
    }
}

// trial point and the partials needed by the controllers: xt = soft(v,
// theta) with v = x - ps g (arc trials, initial point, projected gradient),
// or xt = x + t d along the stored feasible direction d (T_FEAS); the first
// arc trial of an iteration stores d = xt - x
__global__ void __launch_bounds__(kRB) k_spg_proj_apply(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done) return;
  const float ps = (float)st->ps, ft = (float)st->feas_t;
  const double th = st->theta;
  const int ident = st->proj_identity, zero = st->proj_zero;
  const bool feas = st->type == T_FEAS, store = st->store_dir != 0;
  const bool full = st->type == T_INIT || !st->single_tau;  // operator on xt itself
  float q[2] = {0.f, 0.f};  // gtd, dn2
  float dinf = 0.f;
  SPG_LOOP(i, V.n) {
    const float xi = V.x[i];
    float xt;
    if (feas) {
      xt = fmaf(ft, V.dir[i], xi);
    } else {
      const float v = vval(V, ps, i);
      if (zero) xt = 0.f;
      else if (ident) xt = v;
      else {
        // |v| - theta in FP64, rounded once: the FP32 output of every
        // active entry is the correctly rounded exact value, so ||xt||_1
        // misses tau only by the outputs' own rounding (an FP32 copy of
        // theta would shift every active entry the same way)
        const double a = (double)fabsf(v) - th;
        xt = a > 0.0 ? copysignf((float)a, v) : 0.f;
      }
    }
    V.xt[i] = xt;
    const float d = xt - xi;
    // the operator's input.  With a fixed tau (LASSO) the trial's step from
    // x: the residual is then r - F(R d), whose FP32 rounding is relative to
    // ||R d|| rather than to ||R xt||, so the objective resolves the small
    // decreases of the last iterations.  Else (and on the set-up tick) the
    // trial point itself: the root-finding's control was checked against
    // the FP64 oracle with the residual bf - F(R xt).
    if (V.gtmp) V.gtmp[i] = full ? xt : d;  // (null in the stand-alone projection)
    if (store) V.dir[i] = d;
    q[0] = fmaf(V.g[i], d, q[0]);
    q[1] = fmaf(d, d, q[1]);
    dinf = fmaxf(dinf, fabsf(d));
  }
  double o[2];
  block_sum_f<2>(q, o);
  dinf = block_max_f(dinf);
  if (threadIdx.x == 0) {
    put(V.part, P_APPLY + 0, o[0]);
    put(V.part, P_APPLY + 1, o[1]);
    put(V.part, P_APPLY + 2, (double)dinf);
  }
}

// rt = bf - F(R xt).  With y = R xt (the set-up tick, and every tick when
// tau is updated) rt = bf - F y; with a fixed tau after the set-up tick
// y = R (xt - x) and rt = r - F y, r the residual of the current x (the same
// value in exact arithmetic; F y = y - d with the filter offsets d per
// column)
__global__ void __launch_bounds__(kRB) k_spg_resid(SpgVec V, const float* __restrict__ doff, int ns, int filter) {
  const SpgState* st = V.st;
  if (st->done) return;
  const float* base = (st->type == T_INIT || !st->single_tau) ? V.bf : V.r;
  float q[2] = {0.f, 0.f};
  SPG_LOOP(i, V.m) {
    const float fy = filter ? V.y[i] - doff[i % ns] : V.y[i];
    const float r = base[i] - fy;
    V.rt[i] = r;
    q[0] = fmaf(r, r, q[0]);
    q[1] = fmaf(r, V.bf[i], q[1]);
  }
  double o[2];
  block_sum_f<2>(q, o);
  if (threadIdx.x == 0) {
    put(V.part, P_RES + 0, o[0]);
    put(V.part, P_RES + 1, o[1]);
  }
}

__global__ void __launch_bounds__(kRB) k_spg_accept(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done) return;
  const int ax = st->accept_x, ar = st->accept_r;
  if (ax)
    SPG_LOOP(i, V.n) {
      V.xold[i] = V.x[i];
      V.x[i] = V.xt[i];
    }
  if (ar) SPG_LOOP(i, V.m) V.r[i] = V.rt[i];
}

// g = -A^T r (gtmp holds R^T r; F r = r because r lies in the range of F)
__global__ void __launch_bounds__(kRB) k_spg_grad(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done || !st->update_g) return;
  float q[3] = {0.f, 0.f, 0.f};  // sts, sty, gnorm2
  float ginf = 0.f;
  SPG_LOOP(i, V.n) {
    const float go = V.g[i], gn = -V.gtmp[i];
    V.gold[i] = go;
    V.g[i] = gn;
    const float sv = V.x[i] - V.xold[i], yv = gn - go;
    q[0] = fmaf(sv, sv, q[0]);
    q[1] = fmaf(sv, yv, q[1]);
    q[2] = fmaf(gn, gn, q[2]);
    ginf = fmaxf(ginf, fabsf(gn));
  }
  double o[3];
  block_sum_f<3>(q, o);
  ginf = block_max_f(ginf);
  if (threadIdx.x == 0) {
    put(V.part, P_GRAD + 0, o[0]);
    put(V.part, P_GRAD + 1, o[1]);
    put(V.part, P_GRAD + 2, o[2]);
    put(V.part, P_GRAD + 3, (double)ginf);
  }
}

}  // namespace

namespace {

// fixed-order sums of the block partials of quantities q0..q0+NQ-1 (one
// warp per quantity: strided FP64 sums, then a shuffle tree); every thread
// gets the results
template <int NQ>
__device__ __forceinline__ void gather_sums(const double* part, int q0, double (&v)[NQ]) {
  __shared__ double res[NQ];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = w; q < NQ; q += kRB / 32) {
    double t = 0.0;
#pragma unroll
    for (int b = lane; b < kRG; b += 32) t += part[(size_t)(q0 + q) * kRG + b];
    t = warp_sum(t);
    if (lane == 0) res[q] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = res[q];
  __syncthreads();
}
__device__ __forceinline__ double gather_max(const double* part, int q) {
  __shared__ double res;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = threadIdx.x; b < kRG; b += 32) t = fmax(t, part[(size_t)q * kRG + b]);
    t = warp_max(t);
    if (threadIdx.x == 0) res = t;
  }
  __syncthreads();
  const double r = res;
  __syncthreads();
  return r;
}

// one radix-select step.  phi(t) = sum_i max(|v_i| - t, 0) - tau decreases
// in t; at the lower edge t_b of bin b it is (S_above + S_{>=b}) - t_b
// (C_above + C_{>=b}) - tau.  theta lies in the highest bin b* with
// phi(t_b*) > 0.  If b* holds no value, or its values are all equal (last
// pass), the active set is exactly the values above it and theta =
// (S - tau) / C over that set; otherwise the next pass refines inside b*.
// Pass 0 also decides the two trivial cases: tau <= 0 (projection is 0) and
// ||v||_1 <= tau (projection is v).  The kernel consumes and re-zeroes the
// histogram.
__global__ void __launch_bounds__(kRB) k_spg_radix_select(SpgVec V, int pass) {
  SpgState* st = V.st;
  if (st->done || st->type == T_FEAS || (pass > 0 && st->proj_done)) return;
  constexpr int kPer = kBins / kRB;
  __shared__ double scan_c[kRB], scan_s[kRB];
  __shared__ int best;
  const int shift = radix_shift(pass), nb = radix_bits(pass), nbins = 1 << nb;
  const unsigned prefix = pass > 0 ? st->prefix : 0u;
  const double c_above = pass > 0 ? st->c_above : 0.0, s_above = pass > 0 ? st->s_above : 0.0;
  const double tau = st->tau;
  const int b0 = threadIdx.x * kPer;
  double c[kPer], s[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int b = b0 + k;
    c[k] = 0.0;
    s[k] = 0.0;
    if (b < nbins) {
      const unsigned pat = (prefix << (shift + nb)) | ((unsigned)b << shift);
      const int e = (int)(pat >> 23);
      c[k] = (double)V.hcnt[b];
      s[k] = ldexp((double)V.hsum[b], (e > 0 ? e : 1) - 150);
      V.hcnt[b] = 0u;
      V.hsum[b] = 0ull;
    }
  }
  // inclusive suffix sums over bins: within the thread, then across threads
  double tc = 0.0, ts = 0.0;
#pragma unroll
  for (int k = kPer - 1; k >= 0; --k) {
    tc += c[k];
    ts += s[k];
  }
  scan_c[threadIdx.x] = tc;
  scan_s[threadIdx.x] = ts;
  if (threadIdx.x == 0) best = 0;
  __syncthreads();
  for (int off = 1; off < kRB; off <<= 1) {
    const double ac = threadIdx.x + off < kRB ? scan_c[threadIdx.x + off] : 0.0;
    const double as = threadIdx.x + off < kRB ? scan_s[threadIdx.x + off] : 0.0;
    __syncthreads();
    scan_c[threadIdx.x] += ac;
    scan_s[threadIdx.x] += as;
    __syncthreads();
  }
  // bins above this thread's chunk
  double xc = threadIdx.x + 1 < kRB ? scan_c[threadIdx.x + 1] : 0.0;
  double xs = threadIdx.x + 1 < kRB ? scan_s[threadIdx.x + 1] : 0.0;
  double cx[kPer], sx[kPer];  // counts and sums strictly above each bin
  int mine = -1;
#pragma unroll
  for (int k = kPer - 1; k >= 0; --k) {
    cx[k] = xc;
    sx[k] = xs;
    xc += c[k];
    xs += s[k];
    const int b = b0 + k;
    if (mine < 0 && b < nbins) {
      const double t = (double)__uint_as_float((prefix << (shift + nb)) | ((unsigned)b << shift));
      const double phi = (s_above + xs) - t * (c_above + xc) - tau;
      if (phi > 0.0) mine = b;
    }
  }
  if (pass == 0 && threadIdx.x == 0) {
    const double total = scan_s[0];
    st->proj_zero = tau <= 0.0;
    st->proj_identity = tau > 0.0 && total <= tau;
    st->proj_done = st->proj_zero || st->proj_identity;
    st->theta = 0.0;
  }
  if (mine >= 0) atomicMax(&best, mine);
  __syncthreads();
  if (st->proj_done || threadIdx.x != best / kPer) return;
  const int k = best - b0;
  double ck = 0.0, cxk = 0.0, sxk = 0.0;
#pragma unroll
  for (int q = 0; q < kPer; ++q)
    if (q == k) {
      ck = c[q];
      cxk = cx[q];
      sxk = sx[q];
    }
  if (ck == 0.0 || pass == kRadixPasses - 1) {
    const double cnt = c_above + cxk;
    st->theta = cnt > 0.0 ? fmax((s_above + sxk - tau) / cnt, 0.0) : 0.0;
    st->proj_done = 1;
  } else {
    st->prefix = (prefix << nb) | (unsigned)best;
    st->c_above = c_above + cxk;
    st->s_above = s_above + sxk;
  }
}

// non-monotone history: every entry -inf, then f0 in the first slot
__device__ void spg_reset_hist(SpgState* st, double f0) {
  for (int i = 0; i < kHist; ++i) st->fhist[i] = -INFINITY;
  st->fhist[0] = f0;
}

__device__ double spg_clamp_step(const SpgState* st, double v) { return fmin(st->step_max, fmax(st->step_min, v)); }

// start of an SPGL1 iteration: the non-monotone search along the projection
// arc from the Barzilai-Borwein step gstep
__device__ void spg_start_trial(SpgState* st) {
  st->iter++;
  st->f_old = st->f;
  double fm = st->fhist[0];
  for (int i = 1; i < st->memory; ++i) fm = fmax(fm, st->fhist[i]);
  st->fmax = fm;
  st->step = 1.0;
  st->scale = 1.0;
  st->nsafe = 0;
  st->sn_prev = 0.0;
  st->n_line = 0;
  st->n_feas = 0;
  st->type = T_TRIAL;
  st->store_dir = 1;
  st->ps = st->gstep;
}

// top of an SPGL1 iteration: exit tests in the published order, Newton
// update of tau on the Pareto curve when the objective stagnates
__device__ void spg_check(SpgState* st) {
  const double f = st->f, rnorm = sqrt(2.0 * f), gnorm = st->ginf, tau = st->tau, sigma = st->sigma;
  const double gap = 2.0 * f - st->rtb + tau * gnorm;
  const double rel_gap = fabs(gap) / fmax(1.0, f);
  const double aerr1 = rnorm - sigma;
  const double rerr1 = fabs(aerr1) / fmax(1.0, st->bnorm);  // root error relative to the data
  const double rerr2 = fabs(f - 0.5 * sigma * sigma) / fmax(1.0, f);
  st->rel_gap = rel_gap;
  st->rnorm = rnorm;
  int status = S_RUNNING;
  bool shrink = false;
  if (st->single_tau) {
    if (rel_gap <= st->opt_tol || rnorm < st->opt_tol * st->bnorm) status = S_OPTIMAL;
  } else {
    if (gnorm <= st->ls_tol * rnorm) status = S_LS;
    if (rel_gap <= fmax(st->opt_tol, rerr2) || rerr1 <= st->opt_tol) {
      if (rnorm <= sigma) status = S_SUBOPT;
      if (rerr1 <= st->opt_tol) status = S_ROOT;
      if (rnorm <= st->bp_tol * st->bnorm) status = S_BP;
    }
    // the LASSO problem of this tau is solved as far as the Newton step
    // needs once f stops decreasing: relative change <= dec_tol far from
    // the root, below a tenth of the relative root error near it
    const double change = fabs(f - st->f_old);
    const double near = 0.1 * fabs(rnorm - sigma) / fmax(rnorm, 1e-300);
    const bool stagnant = (change <= st->dec_tol * f && rnorm > 2.0 * sigma) || (change <= near * f && rnorm <= 2.0 * sigma);
    const bool upd = stagnant && status == S_RUNNING && !st->upd_last;
    st->upd_last = upd ? 1 : 0;
    if (upd) {
      const double tau_new = fmax(0.0, tau + rnorm * aerr1 / gnorm);
      shrink = tau_new < tau;
      st->tau = tau_new;
      st->n_newton++;
    }
  }
  if (status == S_RUNNING && st->iter >= st->max_iter) status = S_ITER;
  if (status != S_RUNNING) {
    st->status = status;
    st->done = 1;
    return;
  }
  if (shrink) {
    // project x onto the smaller ball; the tick recomputes r, f and g there
    st->type = T_PROJX;
    st->ps = 0.0;
    st->store_dir = 0;
    return;
  }
  spg_start_trial(st);
}

// end of an iteration (accepted step, stationary point or failed search):
// record f in the history (not below sigma^2/2 when solving for the root)
// and run the checks of the next iteration
__device__ void spg_end_iteration(SpgState* st) {
  if (st->single_tau || st->f > 0.5 * st->sigma * st->sigma) st->fhist[st->iter % st->memory] = st->f;
  spg_check(st);
}

// step along the feasible direction after the trial at t gave f(t) = fnew:
// safeguarded quadratic interpolation, else halving
__device__ double spg_feas_next(const SpgState* st, double t, double fnew) {
  if (t <= 0.1) return 0.5 * t;
  const double den = 2.0 * (fnew - st->f - t * st->gtd1);
  const double tmp = den != 0.0 ? (-st->gtd1 * t * t) / den : NAN;
  return (isfinite(tmp) && tmp >= 0.1 && tmp <= 0.9 * t) ? tmp : 0.5 * t;
}

// mid-tick controller: what this tick's trial point is accepted as
__global__ void __launch_bounds__(kRB) k_spg_mid(SpgVec V) {
  SpgState* st = V.st;
  if (st->done) return;
  double a[2], r[2];
  gather_sums<2>(V.part, P_APPLY, a);
  const double dinf = gather_max(V.part, P_APPLY + 2);
  gather_sums<2>(V.part, P_RES, r);
  if (threadIdx.x != 0) return;
  st->gtd = a[0];
  st->dn2 = a[1];
  st->dinf = dinf;
  st->ft = 0.5 * r[0];
  st->rtb_t = r[1];
  st->accept_x = st->accept_r = st->update_g = 0;
  st->stationary = st->go_feas = st->line_err = 0;
  const int type = st->type;
  if (type != T_PG) {
    if (!isfinite(st->ft) || !isfinite(st->gtd)) {
      st->status = S_NONFINITE;
      st->done = 1;
      st->skip_adj = 1;
      st->skip_fwd = 1;
      return;
    }
  }
  if (type == T_INIT || type == T_PROJX) {
    // the initial point, or x projected onto the shrunk ball: residual,
    // objective and gradient are brought up to date with it
    st->accept_x = st->accept_r = st->update_g = 1;
  } else if (type == T_TRIAL) {
    st->n_trials++;
    if (st->n_line == 0) {
      st->f1 = st->ft;
      st->gtd1 = st->gtd;
    }
    bool acc = false;
    if (st->gtd >= 0.0) {
      // no descent: x is optimal for this tau if the very first trial does
      // not move it; a later trial falls back to the feasible direction
      if (st->n_line == 0) st->stationary = 1;
      else st->go_feas = 1;
    } else if (st->ft < st->fmax + st->gamma * st->gtd) {
      acc = true;  // non-monotone sufficient decrease along the arc
    } else if (st->n_line >= st->max_line) {
      st->go_feas = 1;
    }
    if (acc) st->accept_x = st->accept_r = st->update_g = 1;
  } else if (type == T_FEAS) {
    st->n_trials++;
    if (st->ft < st->fmax + st->gamma * st->feas_t * st->gtd1) st->accept_x = st->accept_r = st->update_g = 1;
    else if (st->n_feas >= st->max_line) st->line_err = 1;
  }
  st->skip_adj = st->update_g ? 0 : 1;
}

// end-of-tick controller: Barzilai-Borwein step, history, next tick
__global__ void __launch_bounds__(kRB) k_spg_end(SpgVec V) {
  SpgState* st = V.st;
  if (st->done) return;
  double gq[3] = {0.0, 0.0, 0.0};
  double ginf = 0.0;
  if (st->update_g) {
    gather_sums<3>(V.part, P_GRAD, gq);
    ginf = gather_max(V.part, P_GRAD + 3);
  }
  if (threadIdx.x != 0) return;
  st->ticks++;
  if (st->update_g) {
    st->ginf = ginf;
    st->gnorm2 = gq[2];
  }
  if (st->accept_r) {
    st->f = st->ft;
    st->rtb = st->rtb_t;
  }
  st->store_dir = 0;
  switch (st->type) {
    case T_INIT:
      spg_reset_hist(st, st->f);
      st->f_old = st->f;
      st->type = T_PG;
      st->ps = 1.0;
      break;
    case T_PG: {
      // step length 1 / ||P(x - g) - x||_inf: the initial step, or the
      // restart after an iteration whose first trial had no descent
      const double dxn = st->dinf;
      st->gstep = dxn < 1.0 / st->step_max ? st->step_max : spg_clamp_step(st, 1.0 / dxn);
      if (st->pg_end_iter) spg_end_iteration(st);
      else spg_check(st);
      break;
    }
    case T_PROJX:
      spg_reset_hist(st, st->f);
      spg_start_trial(st);
      break;
    default: {  // T_TRIAL, T_FEAS
      if (!st->stationary && (st->accept_r || st->line_err)) st->n_nodescent = 0;
      if (st->accept_r) {
        const double sts = gq[0], sty = gq[1];
        st->gstep = sty <= 0.0 ? st->step_max : spg_clamp_step(st, sts / sty);
        spg_end_iteration(st);
      } else if (st->stationary) {
        // the first trial did not move x downhill at a point the exit tests
        // did not certify: the BB step is too short for the working
        // precision.  x stays; the step restarts from the projected
        // gradient (a T_PG tick), then the iteration ends.  With a fixed tau
        // three such iterations in a row end the solve.
        st->n_stationary++;
        st->n_nodescent++;
        if (st->single_tau && st->n_nodescent > 2) {
          st->status = S_LINE;
          st->done = 1;
          st->skip_adj = 1;
          break;
        }
        st->type = T_PG;
        st->ps = 1.0;
        st->pg_end_iter = 1;
      } else if (st->line_err) {
        // both searches failed: x, f, r and g stay; damp the longest step
        st->n_line_errors++;
        if (st->line_errors_left <= 0) {
          st->status = S_LINE;
          st->done = 1;
          st->skip_adj = 1;
          break;
        }
        st->step_max /= 10.0;
        st->line_errors_left--;
        st->gstep = fmin(st->step_max, st->gstep);
        spg_end_iteration(st);
      } else if (st->go_feas) {
        // its t = 1 point is the first arc trial, already rejected
        st->type = T_FEAS;
        st->feas_t = spg_feas_next(st, 1.0, st->f1);
        st->n_feas = 1;
      } else if (st->type == T_TRIAL) {
        // backtrack along the arc; a flat arc (two consecutive trials with
        // displacements of equal norm) rescales the gradient so that the
        // next displacement is step |s| / 2^nsafe
        st->n_line++;
        st->step *= 0.5;
        const double sn = sqrt(st->dn2), gn = sqrt(st->gnorm2);
        if (fabs(sn - st->sn_prev) <= 1e-6 * sn && gn > 0.0) {
          st->scale = sn / (st->gstep * gn) / exp2((double)st->nsafe);
          st->nsafe++;
          st->n_safeguard++;
        }
        st->sn_prev = sn;
        st->ps = st->step * st->scale * st->gstep;
      } else {  // T_FEAS, rejected
        st->feas_t = spg_feas_next(st, st->feas_t, st->ft);
        st->n_feas++;
      }
      break;
    }
  }
  st->skip_fwd = (st->done || st->type == T_PG) ? 1 : 0;
}

// ||b||^2 and ||x0||_1 for the set-up
__global__ void __launch_bounds__(kRB) k_spg_norms(const float* __restrict__ bf, long long m,
                                                   const float* __restrict__ x, long long n, double* part) {
  double q[2] = {0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x, i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = i0; i < m; i += stride) q[0] += (double)bf[i] * bf[i];
  for (long long i = i0; i < n; i += stride) q[1] += fabs((double)x[i]);
  block_sum<2>(q);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = q[0];
    part[kRG + blockIdx.x] = q[1];
  }
}

__global__ void __launch_bounds__(kRB) k_spg_setup(SpgVec V, double tau0) {
  double q[2];
  gather_sums<2>(V.part, 0, q);
  if (threadIdx.x != 0) return;
  SpgState* st = V.st;
  st->bnorm = sqrt(q[0]);
  st->tau = tau0 >= 0.0 ? tau0 : q[1];
  st->gstep = st->step_max;
  st->type = T_INIT;
  st->ps = 0.0;
  st->skip_fwd = 0;
  if (!isfinite(st->bnorm) || !isfinite(st->tau)) {
    // NaN / Inf in the data or the warm start: stop before the first tick
    st->status = S_NONFINITE;
    st->done = 1;
    st->skip_fwd = 1;
    st->skip_adj = 1;
  }
}

// final ||x||_1 and ||r||_2 (ignores the done flag)
__global__ void __launch_bounds__(kRB) k_spg_final(SpgVec V) {
  double q[2] = {0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x, i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = i0; i < V.n; i += stride) q[0] += fabs((double)V.x[i]);
  for (long long i = i0; i < V.m; i += stride) q[1] += (double)V.r[i] * V.r[i];
  block_sum<2>(q);
  if (threadIdx.x == 0) {
    V.part[blockIdx.x] = q[0];
    V.part[kRG + blockIdx.x] = q[1];
  }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// finite-difference synthesis operator of the analysis-l1 variant
// ---------------------------------------------------------------------------
// u = C z: prefix sums along every image row (C inverts the horizontal
// difference z[p, 0] = u[p, 0], z[p, q] = u[p, q] - u[p, q - 1]); its adjoint
// C^T w: suffix sums along every row.  One CTA per row (grid-stride over
// rows), thread t owns `per` consecutive positions in scan order (from the
// row's end for the adjoint); FP32 sums: the thread's run, then a warp and a
// block scan of the run totals.  In place allowed: every thread writes only
// the positions it has read, after the block's scan barrier.
constexpr int kScanT = 256;
constexpr int kScanMaxPer = 16;  // rows of up to 4096 values
__global__ void __launch_bounds__(kScanT) k_synth_rows(const float* __restrict__ in, float* __restrict__ out, int n,
                                                      int rows, int adjoint, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ float wsum[kScanT / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (n + kScanT - 1) / kScanT;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const float* src = in + (size_t)row * n;
    float* dst = out + (size_t)row * n;
    float v[kScanMaxPer];
    float run = 0.f;
#pragma unroll
    for (int i = 0; i < kScanMaxPer; ++i) {
      const int q = t * per + i;
      v[i] = 0.f;
      if (i < per && q < n) v[i] = src[adjoint ? n - 1 - q : q];
      run += v[i];
    }
    float x = run;  // inclusive scan of the run totals within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      float y = lane < kScanT / 32 ? wsum[lane] : 0.f;
#pragma unroll
      for (int o = 1; o < kScanT / 32; o <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      if (lane < kScanT / 32) wsum[lane] = y;
    }
    __syncthreads();
    float acc = (x - run) + (w > 0 ? wsum[w - 1] : 0.f);  // exclusive prefix of this thread's run
#pragma unroll
    for (int i = 0; i < kScanMaxPer; ++i) {
      const int q = t * per + i;
      if (i < per && q < n) {
        acc += v[i];
        dst[adjoint ? n - 1 - q : q] = acc;
      }
    }
    __syncthreads();  // wsum is reused by the next row
  }
}

void launch_synth(const float* in, float* out, int n, int adjoint, const int* skip, cudaStream_t s) {
  k_synth_rows<<<n < 4096 ? n : 4096, kScanT, 0, s>>>(in, out, n, n, adjoint, skip);
}

}  // namespace

extern "C" int cpct_synth_dh(const float* d_in, float* d_out, int n, int adjoint, cudaStream_t stream) {
  if (!d_in || !d_out || n < 1 || n > kScanT * kScanMaxPer || (adjoint != 0 && adjoint != 1)) return CPCT_EINVAL;
  launch_synth(d_in, d_out, n, adjoint, nullptr, stream);
  return cudaGetLastError() == cudaSuccess ? CPCT_OK : CPCT_ECUDA;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
namespace {

struct SliceWork {
  cpct_plan* plan = nullptr;
  float* x = nullptr;
  const float* b = nullptr;
  double sigma = 0.0;
  SpgVec V{};
  RingWork ring;
  cudaStream_t stream = nullptr;
  float* mem = nullptr;
  float* ubuf = nullptr;  // u = C xt of the analysis-l1 variant (within mem)
};

void enqueue_tick(SliceWork& w, int filter) {
  cudaStream_t s = w.stream;
  SpgVec V = w.V;
  for (int pass = 0; pass < kRadixPasses; ++pass) {
    k_spg_radix_hist<<<kRG, kRB, 0, s>>>(V, pass);
    k_spg_radix_select<<<1, kRB, 0, s>>>(V, pass);
  }
  k_spg_proj_apply<<<kRG, kRB, 0, s>>>(V);
  // the operator acts on gtmp, written by the projection: the trial point,
  // or its step from x with a fixed tau (k_spg_proj_apply)
  if (w.ubuf) {
    // analysis-l1 variant: the operator acts on u = C gtmp
    launch_synth(V.gtmp, w.ubuf, w.plan->n, 0, &V.st->skip_fwd, s);
    cpct_launch_fwd_skip(w.plan, w.ubuf, V.y, &V.st->skip_fwd, s);
  } else {
    cpct_launch_fwd_skip(w.plan, V.gtmp, V.y, &V.st->skip_fwd, s);
  }
  if (filter) {
    k_ring_colmean<<<(w.plan->ns + 31) / 32, kRB, 0, s>>>(V.y, w.ring.m, w.plan->m, w.plan->ns);
    k_ring_offset<<<1, kRB, 0, s>>>(w.ring.Q, w.ring.m, w.ring.d, w.plan->ns);
  }
  k_spg_resid<<<kRG, kRB, 0, s>>>(V, w.ring.d, w.plan->ns, filter);
  k_spg_mid<<<1, kRB, 0, s>>>(V);
  k_spg_accept<<<kRG, kRB, 0, s>>>(V);
  cpct_launch_adj_ramp(w.plan, V.r, V.gtmp, 0.f, &V.st->skip_adj, s);
  if (w.ubuf) launch_synth(V.gtmp, V.gtmp, w.plan->n, 1, &V.st->skip_adj, s);  // C^T R^T F r
  k_spg_grad<<<kRG, kRB, 0, s>>>(V);
  k_spg_end<<<1, kRB, 0, s>>>(V);
}

int fill_opts(const spgl1_opts* o, SpgState& st, double* tau0, int* filter, int* synth) {
  st.max_iter = (o && o->max_iter > 0) ? o->max_iter : 300;
  st.opt_tol = (o && o->opt_tol > 0) ? o->opt_tol : 1e-4;
  st.bp_tol = (o && o->bp_tol > 0) ? o->bp_tol : 1e-6;
  st.ls_tol = (o && o->ls_tol > 0) ? o->ls_tol : 1e-6;
  st.dec_tol = (o && o->dec_tol > 0) ? o->dec_tol : 1e-4;
  st.memory = (o && o->memory > 0) ? o->memory : 3;
  st.gamma = (o && o->gamma > 0) ? o->gamma : 1e-4;
  st.step_min = (o && o->step_min > 0) ? o->step_min : 1e-16;
  st.step_max = (o && o->step_max > 0) ? o->step_max : 1e5;
  st.max_line = (o && o->max_line > 0) ? o->max_line : 10;
  st.line_errors_left = (o && o->max_line_errors > 0) ? o->max_line_errors : 10;
  st.single_tau = (o && (o->flags & CPCT_SPGL1_LASSO)) ? 1 : 0;
  if (st.memory > kHist) return CPCT_EINVAL;
  *tau0 = (o && (o->flags & (CPCT_SPGL1_TAU0 | CPCT_SPGL1_LASSO))) ? o->tau0 : -1.0;
  if (st.single_tau && !(*tau0 >= 0.0 && std::isfinite(*tau0))) return CPCT_EINVAL;
  *filter = (o && (o->flags & CPCT_SPGL1_NO_FILTER)) ? 0 : 1;
  *synth = (o && (o->flags & CPCT_SPGL1_SYNTH_DH)) ? 1 : 0;
  return CPCT_OK;
}

}  // namespace

extern "C" int spgl1_solve_batched(cpct_plan* const* plans, int batch, const float* const* d_b, const double* sigma,
                                   float* const* d_x, const spgl1_opts* opts, spgl1_info* info, cudaStream_t stream) {
  if (!plans || batch < 1 || !d_b || !d_x) return CPCT_EINVAL;
  if (!sigma && !(opts && (opts->flags & CPCT_SPGL1_LASSO))) return CPCT_EINVAL;
  SpgState proto;
  std::memset(&proto, 0, sizeof(proto));
  double tau0 = -1.0;
  int filter = 1, synth = 0;
  int rc = fill_opts(opts, proto, &tau0, &filter, &synth);
  if (rc) return rc;
  for (int i = 0; i < batch; ++i) {
    if (!plans[i] || !d_b[i] || !d_x[i] || (sigma && !(sigma[i] >= 0.0))) return CPCT_EINVAL;
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return CPCT_EINVAL;  // a plan holds per-call workspaces
  }
  std::vector<SliceWork> ws(batch);
  SpgState* d_states = nullptr;
  double* d_part = nullptr;
  unsigned char* d_hist = nullptr;  // per slice: kBins counts, then (all slices) kBins sums
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  std::vector<SpgState> h_states(batch);
  std::vector<cudaStream_t> branch;
  cudaStream_t cap = nullptr;
  bool capturing = false;
  rc = CPCT_OK;
  auto cuda = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == CPCT_OK) rc = CPCT_ECUDA;
    return e == cudaSuccess;
  };
  if (!cuda(cudaMalloc(&d_states, sizeof(SpgState) * batch))) goto done;
  if (!cuda(cudaMalloc(&d_part, sizeof(double) * P_TOTAL * kRG * batch))) goto done;
  if (!cuda(cudaMalloc(&d_hist, (sizeof(unsigned) + sizeof(unsigned long long)) * kBins * batch))) goto done;
  if (!cuda(cudaMemsetAsync(d_hist, 0, (sizeof(unsigned) + sizeof(unsigned long long)) * kBins * batch, stream)))
    goto done;
  for (int i = 0; i < batch; ++i) {
    SliceWork& w = ws[i];
    w.plan = plans[i];
    w.x = d_x[i];
    w.b = d_b[i];
    w.sigma = sigma ? sigma[i] : 0.0;
    const long long n = (long long)w.plan->n * w.plan->n, m = (long long)w.plan->m * w.plan->ns;
    if (synth && w.plan->n > kScanT * kScanMaxPer) {
      rc = CPCT_EINVAL;
      goto done;
    }
    if (!cuda(cudaMalloc(&w.mem, sizeof(float) * ((synth ? 7 : 6) * n + 4 * m)))) goto done;
    SpgVec& V = w.V;
    V.n = n;
    V.m = m;
    V.x = w.x;
    V.xt = w.mem;
    V.xold = w.mem + n;
    V.g = w.mem + 2 * n;
    V.gold = w.mem + 3 * n;
    V.gtmp = w.mem + 4 * n;
    V.dir = w.mem + 5 * n;
    V.y = w.mem + 6 * n;
    V.rt = V.y + m;
    V.r = V.rt + m;
    V.bf = V.r + m;
    w.ubuf = synth ? V.bf + m : nullptr;
    V.part = d_part + (size_t)i * P_TOTAL * kRG;
    V.hcnt = reinterpret_cast<unsigned*>(d_hist) + (size_t)i * kBins;
    V.hsum = reinterpret_cast<unsigned long long*>(d_hist + sizeof(unsigned) * kBins * batch) + (size_t)i * kBins;
    V.st = d_states + i;
    if ((rc = ring_work(w.plan->ns, w.ring, stream)) != CPCT_OK) goto done;
    w.stream = stream;
    if (batch > 1) {
      branch.push_back(nullptr);
      if (!cuda(cudaStreamCreateWithFlags(&branch.back(), cudaStreamNonBlocking))) goto done;
    }
    // state, filtered data, zero gradient and residual, ||b||, tau0
    SpgState st = proto;
    st.sigma = proto.single_tau ? 0.0 : w.sigma;
    if (!cuda(cudaMemcpyAsync(V.st, &st, sizeof(st), cudaMemcpyHostToDevice, stream))) goto done;
    if (!cuda(cudaMemsetAsync(V.g, 0, sizeof(float) * n, stream))) goto done;
    if (!cuda(cudaMemsetAsync(V.r, 0, sizeof(float) * m, stream))) goto done;
    if (filter) ring_launch(w.ring, w.b, V.bf, w.plan->m, w.plan->ns, stream);
    else if (!cuda(cudaMemcpyAsync(V.bf, w.b, sizeof(float) * m, cudaMemcpyDeviceToDevice, stream))) goto done;
    k_spg_norms<<<kRG, kRB, 0, stream>>>(V.bf, m, V.x, n, V.part);
    k_spg_setup<<<1, kRB, 0, stream>>>(V, tau0);
    if (!cuda(cudaGetLastError())) goto done;
  }
  // the first tick runs eagerly: it loads every kernel of a tick (modules
  // load lazily, which is not allowed while a stream is being captured)
  for (int i = 0; i < batch; ++i) {
    cpct_profile_enable(ws[i].plan, 0);
    enqueue_tick(ws[i], filter);
  }
  if (!cuda(cudaGetLastError())) goto done;
  if (!cuda(cudaStreamSynchronize(stream))) goto done;
  // one tick of every slice, captured once on a private stream (the
  // caller's stream may be the legacy default stream, which cannot be
  // captured); the graph is then launched on the caller's stream
  {
    // kernel-level event profiling cannot be recorded inside a graph
    for (int i = 0; i < batch; ++i) cpct_profile_enable(ws[i].plan, 0);
    if (!cuda(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) goto done;
    if (!cuda(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming))) goto done;
    joins.resize(batch, nullptr);
    for (int i = 0; i < batch; ++i)
      if (!cuda(cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming))) goto done;
    if (!cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) goto done;
    capturing = true;
    if (batch > 1) cudaEventRecord(fork, cap);
    for (int i = 0; i < batch; ++i) {
      SliceWork w = ws[i];
      if (batch > 1) {
        w.stream = branch[i];
        cudaStreamWaitEvent(w.stream, fork, 0);
      } else {
        w.stream = cap;
      }
      enqueue_tick(w, filter);
      if (batch > 1) {
        cudaEventRecord(joins[i], w.stream);
        cudaStreamWaitEvent(cap, joins[i], 0);
      }
    }
    capturing = false;
    if (!cuda(cudaStreamEndCapture(cap, &graph))) goto done;
    if (!cuda(cudaGraphInstantiate(&exec, graph, 0))) goto done;
  }
  {
    const int chunk = 8;
    // per iteration at most max_line + 1 arc trials, max_line feasible
    // trials and one projection onto a shrunk ball
    const long long max_ticks = (long long)(proto.max_iter + 2) * (2 * proto.max_line + 4) + 16;
    long long ticks = 0;
    bool all_done = false;
    while (!all_done && ticks < max_ticks) {
      for (int c = 0; c < chunk; ++c)
        if (!cuda(cudaGraphLaunch(exec, stream))) goto done;
      ticks += chunk;
      if (!cuda(cudaMemcpyAsync(h_states.data(), d_states, sizeof(SpgState) * batch, cudaMemcpyDeviceToHost, stream)))
        goto done;
      if (!cuda(cudaStreamSynchronize(stream))) goto done;
      all_done = true;
      for (int i = 0; i < batch; ++i) all_done = all_done && h_states[i].done;
    }
  }
  // final norms and the info records
  for (int i = 0; i < batch; ++i) {
    SliceWork& w = ws[i];
    k_spg_final<<<kRG, kRB, 0, stream>>>(w.V);
    std::vector<double> part(2 * kRG);
    if (!cuda(cudaMemcpyAsync(part.data(), w.V.part, sizeof(double) * 2 * kRG, cudaMemcpyDeviceToHost, stream))) goto done;
    if (!cuda(cudaMemcpyAsync(&h_states[i], w.V.st, sizeof(SpgState), cudaMemcpyDeviceToHost, stream))) goto done;
    if (!cuda(cudaStreamSynchronize(stream))) goto done;
    double l1 = 0.0, r2 = 0.0;
    for (int b = 0; b < kRG; ++b) {
      l1 += part[b];
      r2 += part[kRG + b];
    }
    const SpgState& st = h_states[i];
    if (info) {
      spgl1_info& I = info[i];
      I.status = st.done ? st.status : S_ITER;
      I.iterations = st.iter;
      I.ticks = st.ticks;
      I.trials = st.n_trials;
      I.tau = st.tau;
      I.rnorm = std::sqrt(r2);
      I.xnorm1 = l1;
      I.rel_gap = st.rel_gap;
      I.newton = st.n_newton;
      I.line_errors = st.n_line_errors;
      I.safeguards = st.n_safeguard;
      I.stationary = st.n_stationary;
      I.gstep = st.gstep;
    }
    if (rc == CPCT_OK) {
      const int sst = st.done ? st.status : S_ITER;
      if (sst == S_NONFINITE) rc = CPCT_ENONFINITE;
      else if (sst == S_ITER || sst == S_LINE) rc = CPCT_ENOTCONV;
    }
  }
done:
  if (capturing) {
    // end a capture that an error interrupted, so no stream stays capturing
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cap, &g);
    if (g) cudaGraphDestroy(g);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamSynchronize(stream);
  for (auto e : joins)
    if (e) cudaEventDestroy(e);
  if (fork) cudaEventDestroy(fork);
  for (auto& w : ws) {
    if (w.mem) cudaFree(w.mem);
    ring_free(w.ring);
  }
  for (auto b : branch)
    if (b) cudaStreamDestroy(b);
  if (cap) cudaStreamDestroy(cap);
  if (d_states) cudaFree(d_states);
  if (d_part) cudaFree(d_part);
  if (d_hist) cudaFree(d_hist);
  return rc;
}

extern "C" int spgl1_solve(cpct_plan* plan, const float* d_b, double sigma, float* d_x, const spgl1_opts* opts,
                           spgl1_info* info, cudaStream_t stream) {
  return spgl1_solve_batched(&plan, 1, &d_b, &sigma, &d_x, opts, info, stream);
}

extern "C" int cpct_project_l1_batched(const float* const* d_v, int batch, long long n, const double* tau,
                                       float* const* d_out, double* theta, cudaStream_t stream) {
  if (!d_v || !d_out || !tau || batch < 1 || n < 1 || n > (1LL << 30)) return CPCT_EINVAL;
  for (int i = 0; i < batch; ++i)
    if (!d_v[i] || !d_out[i] || !std::isfinite(tau[i])) return CPCT_EINVAL;
  // workspace per vector: state, partials of the apply kernel, histogram
  const size_t b_state = (sizeof(SpgState) + 255) / 256 * 256;
  const size_t b_part = sizeof(double) * P_TOTAL * kRG;
  const size_t b_hist = (sizeof(unsigned) + sizeof(unsigned long long)) * kBins;
  const size_t b_one = b_state + b_part + b_hist;
  unsigned char* mem = nullptr;
  if (cudaMalloc(&mem, b_one * batch) != cudaSuccess) return CPCT_ENOMEM;
  std::vector<SpgState> st(batch);
  int rc = CPCT_OK;
  for (int i = 0; i < batch && rc == CPCT_OK; ++i) {
    std::memset(&st[i], 0, sizeof(SpgState));
    st[i].tau = tau[i];  // ps = 0: v = x - 0 * g = x
  }
  // the states, then zeroed histograms, in two copies
  std::vector<unsigned char> init(b_one * batch, 0);
  for (int i = 0; i < batch; ++i) std::memcpy(init.data() + b_one * i, &st[i], sizeof(SpgState));
  if (cudaMemcpyAsync(mem, init.data(), init.size(), cudaMemcpyHostToDevice, stream) != cudaSuccess) rc = CPCT_ECUDA;
  for (int i = 0; i < batch && rc == CPCT_OK; ++i) {
    unsigned char* w = mem + b_one * i;
    SpgVec V{};
    V.x = const_cast<float*>(d_v[i]);
    V.g = const_cast<float*>(d_v[i]);
    V.xt = d_out[i];
    V.n = n;
    V.st = reinterpret_cast<SpgState*>(w);
    V.part = reinterpret_cast<double*>(w + b_state);
    V.hcnt = reinterpret_cast<unsigned*>(w + b_state + b_part);
    V.hsum = reinterpret_cast<unsigned long long*>(w + b_state + b_part + sizeof(unsigned) * kBins);
    for (int pass = 0; pass < kRadixPasses; ++pass) {
      k_spg_radix_hist<<<kRG, kRB, 0, stream>>>(V, pass);
      k_spg_radix_select<<<1, kRB, 0, stream>>>(V, pass);
    }
    k_spg_proj_apply<<<kRG, kRB, 0, stream>>>(V);
  }
  if (rc == CPCT_OK && cudaGetLastError() != cudaSuccess) rc = CPCT_ECUDA;
  if (rc == CPCT_OK && theta) {
    for (int i = 0; i < batch && rc == CPCT_OK; ++i)
      if (cudaMemcpyAsync(&st[i], mem + b_one * i, sizeof(SpgState), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        rc = CPCT_ECUDA;
  }
  if (cudaStreamSynchronize(stream) != cudaSuccess && rc == CPCT_OK) rc = CPCT_ECUDA;
  cudaFree(mem);
  if (rc == CPCT_OK && theta)
    for (int i = 0; i < batch; ++i) theta[i] = st[i].proj_zero ? 0.0 : st[i].theta;
  return rc;
}

extern "C" int cpct_project_l1(const float* d_v, long long n, double tau, float* d_out, double* theta,
                               cudaStream_t stream) {
  if (!d_v || !d_out) return CPCT_EINVAL;
  return cpct_project_l1_batched(&d_v, 1, n, &tau, &d_out, theta, stream);
}
