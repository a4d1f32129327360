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

__device__ __forceinline__ double block_max(double v) {
  __shared__ double sh[kRB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sh[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, sh[i]);
    v = m;
  }
  __syncthreads();
  return v;
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

enum TickType { T_INIT = 0, T_PG = 1, T_PROJX = 2, T_TRIAL = 3 };
enum AfterPG { PG_THEN_CHECK = 0, PG_THEN_TRIAL = 1 };
constexpr int kHist = 8;        // objective history capacity (memory <= 8)
constexpr int kCand = 16;       // candidate thresholds per multi-section pass
constexpr int kPasses = 8;      // multi-section passes per projection
constexpr double kDecTol = 1e-4;  // stagnation threshold of the inexact Newton test

struct SpgState {
  // options
  double sigma, opt_tol, bp_tol, gamma, step_min, step_max;
  int max_iter, max_line, memory, pad0;
  // solver scalars (FP64)
  double tau, bnorm, f, f_old, fmax, alpha, step, dn_prev, rtb, ginf, gnorm2;
  double fhist[kHist];
  int nhist, hpos;
  double rel_gap, rnorm;
  // this tick
  int type, pg_then, accept_x, accept_r, update_g, line_fail;
  double ps;
  // projection of v = x - ps g onto the l1 ball of radius tau
  double lo, hi, theta, c_lo, s_lo;
  int proj_done, proj_identity, proj_zero, pad1;
  // mid-tick results
  double ft, gtd, dn2, dinf, rtb_t;
  // counters / status
  int iter, n_line, status, done, ticks, n_trials, stationary, n_stationary;
};

// SPGL1 status codes (spgl1_info.status)
enum { S_RUNNING = 0, S_ROOT = 1, S_BP = 2, S_ITER = 3, S_LINE = 4, S_NONFINITE = 5 };

struct SpgVec {
  float *x, *xt, *xold, *g, *gold, *gtmp;  // image space, n
  float *y, *rt, *r, *bf;                  // sinogram space, m
  double* part;                            // per-block partials
  SpgState* st;
  long long n, m;
};

// partial buffer regions (each kRG doubles per quantity)
constexpr int P_VSTAT = 0;                  // 2: sum|v|, max|v|
constexpr int P_PROJ = 2;                   // 2*(kCand+1): counts, sums
constexpr int P_APPLY = P_PROJ + 2 * (kCand + 1);  // 3: gtd, dn2, dinf
constexpr int P_RES = P_APPLY + 3;          // 2: sum rt^2, sum rt*bf
constexpr int P_GRAD = P_RES + 2;           // 4: sts, sty, ginf, gnorm2
constexpr int P_TOTAL = P_GRAD + 4;

__device__ __forceinline__ double pget(const double* part, int q, int b) { return part[(size_t)q * kRG + b]; }

// v_i = x_i - ps g_i
__device__ __forceinline__ float vval(const SpgVec& V, double ps, long long i) {
  return (float)((double)V.x[i] - ps * (double)V.g[i]);
}

__global__ void __launch_bounds__(kRB) k_spg_vstats(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done) return;
  const double ps = st->ps;
  double s[1] = {0.0};
  double mx = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V.n; i += (long long)gridDim.x * blockDim.x) {
    const double a = fabs((double)vval(V, ps, i));
    s[0] += a;
    mx = fmax(mx, a);
  }
  block_sum<1>(s);
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    V.part[(size_t)(P_VSTAT + 0) * kRG + blockIdx.x] = s[0];
    V.part[(size_t)(P_VSTAT + 1) * kRG + blockIdx.x] = mx;
  }
}

// one multi-section pass: counts and sums of |v| above kCand+1 thresholds
// t_c = lo + (hi - lo) c / kCand, c = 0..kCand
__global__ void __launch_bounds__(kRB) k_spg_proj_pass(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done || st->proj_done) return;
  const double ps = st->ps, lo = st->lo, w = (st->hi - st->lo) / kCand;
  double cnt[kCand + 1], sum[kCand + 1];
#pragma unroll
  for (int c = 0; c <= kCand; ++c) { cnt[c] = 0.0; sum[c] = 0.0; }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V.n; i += (long long)gridDim.x * blockDim.x) {
    const double a = fabs((double)vval(V, ps, i));
    if (a <= lo) continue;
#pragma unroll
    for (int c = 0; c <= kCand; ++c) {
      const bool above = a > lo + w * c;
      cnt[c] += above ? 1.0 : 0.0;
      sum[c] += above ? a : 0.0;
    }
  }
  block_sum<kCand + 1>(cnt);
  block_sum<kCand + 1>(sum);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c <= kCand; ++c) {
      V.part[(size_t)(P_PROJ + c) * kRG + blockIdx.x] = cnt[c];
      V.part[(size_t)(P_PROJ + kCand + 1 + c) * kRG + blockIdx.x] = sum[c];
    }
  }
}

// xt = soft(v, theta) and the partials needed by the controllers
__global__ void __launch_bounds__(kRB) k_spg_proj_apply(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done) return;
  const double ps = st->ps, th = st->theta;
  const int ident = st->proj_identity, zero = st->proj_zero;
  double q[2] = {0.0, 0.0};  // gtd, dn2
  double dinf = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V.n; i += (long long)gridDim.x * blockDim.x) {
    const float v = vval(V, ps, i);
    float xt;
    if (zero) xt = 0.f;
    else if (ident) xt = v;
    else {
      const double a = fabs((double)v) - th;
      xt = a > 0.0 ? copysignf((float)a, v) : 0.f;
    }
    V.xt[i] = xt;
    const double d = (double)xt - (double)V.x[i];
    q[0] += (double)V.g[i] * d;
    q[1] += d * d;
    dinf = fmax(dinf, fabs(d));
  }
  block_sum<2>(q);
  dinf = block_max(dinf);
  if (threadIdx.x == 0) {
    V.part[(size_t)(P_APPLY + 0) * kRG + blockIdx.x] = q[0];
    V.part[(size_t)(P_APPLY + 1) * kRG + blockIdx.x] = q[1];
    V.part[(size_t)(P_APPLY + 2) * kRG + blockIdx.x] = dinf;
  }
}

// rt = bf - F(R xt) = bf - (y - d), with the filter offsets d per column
__global__ void __launch_bounds__(kRB) k_spg_resid(SpgVec V, const float* __restrict__ doff, int ns, int filter) {
  const SpgState* st = V.st;
  if (st->done) return;
  double q[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V.m; i += (long long)gridDim.x * blockDim.x) {
    const float fy = filter ? V.y[i] - doff[i % ns] : V.y[i];
    const float r = V.bf[i] - fy;
    V.rt[i] = r;
    q[0] += (double)r * r;
    q[1] += (double)r * V.bf[i];
  }
  block_sum<2>(q);
  if (threadIdx.x == 0) {
    V.part[(size_t)(P_RES + 0) * kRG + blockIdx.x] = q[0];
    V.part[(size_t)(P_RES + 1) * kRG + blockIdx.x] = q[1];
  }
}

__global__ void __launch_bounds__(kRB) k_spg_accept(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done) return;
  const int ax = st->accept_x, ar = st->accept_r;
  const long long stride = (long long)gridDim.x * blockDim.x, i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ax)
    for (long long i = i0; i < V.n; i += stride) {
      V.xold[i] = V.x[i];
      V.x[i] = V.xt[i];
    }
  if (ar)
    for (long long i = i0; i < V.m; i += stride) V.r[i] = V.rt[i];
}

// g = -A^T r (gtmp holds R^T r; F r = r because r lies in the range of F)
__global__ void __launch_bounds__(kRB) k_spg_grad(SpgVec V) {
  const SpgState* st = V.st;
  if (st->done || !st->update_g) return;
  double q[3] = {0.0, 0.0, 0.0};  // sts, sty, gnorm2
  double ginf = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V.n; i += (long long)gridDim.x * blockDim.x) {
    const float go = V.g[i], gn = -V.gtmp[i];
    V.gold[i] = go;
    V.g[i] = gn;
    const double s = (double)V.x[i] - (double)V.xold[i], yv = (double)gn - (double)go;
    q[0] += s * s;
    q[1] += s * yv;
    q[2] += (double)gn * gn;
    ginf = fmax(ginf, fabs((double)gn));
  }
  block_sum<3>(q);
  ginf = block_max(ginf);
  if (threadIdx.x == 0) {
    V.part[(size_t)(P_GRAD + 0) * kRG + blockIdx.x] = q[0];
    V.part[(size_t)(P_GRAD + 1) * kRG + blockIdx.x] = q[1];
    V.part[(size_t)(P_GRAD + 2) * kRG + blockIdx.x] = q[2];
    V.part[(size_t)(P_GRAD + 3) * kRG + blockIdx.x] = ginf;
  }
}

}  // namespace

namespace {

// block-parallel fixed-order sum of partials q0..q0+NQ-1 (thread 0 gets them)
template <int NQ>
__device__ __forceinline__ void gather_sums(const double* part, int q0, double (&v)[NQ]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = threadIdx.x < kRG ? part[(size_t)(q0 + q) * kRG + threadIdx.x] : 0.0;
  block_sum<NQ>(v);
}
__device__ __forceinline__ double gather_max(const double* part, int q) {
  return block_max(threadIdx.x < kRG ? part[(size_t)q * kRG + threadIdx.x] : 0.0);
}

// choose the sub-interval of the bracket that holds theta (block-parallel
// reduction of the pass partials); finish when it holds no |v_i|: the active
// set is then fixed and theta = (sum of active |v_i| - tau) / their count
__global__ void __launch_bounds__(kRB) k_spg_proj_pick2(SpgVec V, int last_pass) {
  SpgState* st = V.st;
  if (st->done || st->proj_done) return;
  double C[kCand + 1], S[kCand + 1];
  gather_sums<kCand + 1>(V.part, P_PROJ, C);
  gather_sums<kCand + 1>(V.part, P_PROJ + kCand + 1, S);
  if (threadIdx.x != 0) return;
  const double lo = st->lo, w = (st->hi - st->lo) / kCand, tau = st->tau;
  int c = 1;
  for (; c < kCand; ++c)
    if (S[c] - (lo + w * c) * C[c] - tau <= 0.0) break;
  if (C[c - 1] == C[c] || last_pass || w <= 1e-15 * st->hi) {
    const double t0 = lo + w * (c - 1), t1 = lo + w * c;
    const double th = C[c] > 0.0 ? (S[c] - tau) / C[c] : t1;
    st->theta = C[c - 1] == C[c] ? th : fmin(fmax(th, t0), t1);
    st->proj_done = 1;
  } else {
    st->lo = lo + w * (c - 1);
    st->hi = lo + w * c;
  }
}

// start of the projection: the threshold theta solves
// sum_i max(|v_i| - theta, 0) = tau; it lies in [max(0, max|v| - tau), max|v|]
__global__ void __launch_bounds__(kRB) k_spg_proj_begin2(SpgVec V) {
  SpgState* st = V.st;
  if (st->done) return;
  double s[1];
  gather_sums<1>(V.part, P_VSTAT, s);
  const double mx = gather_max(V.part, P_VSTAT + 1);
  if (threadIdx.x != 0) return;
  st->proj_identity = 0;
  st->proj_zero = 0;
  if (st->tau <= 0.0) {
    st->proj_zero = 1;
    st->proj_done = 1;
    st->theta = mx;
  } else if (s[0] <= st->tau) {
    st->proj_identity = 1;
    st->proj_done = 1;
    st->theta = 0.0;
  } else {
    st->proj_done = 0;
    st->lo = fmax(0.0, mx - st->tau);
    st->hi = mx;
  }
}

__device__ void spg_push_hist(SpgState* st, double f) {
  st->fhist[st->hpos] = f;
  st->hpos = (st->hpos + 1) % st->memory;
  if (st->nhist < st->memory) st->nhist++;
}

__device__ void spg_start_trial(SpgState* st) {
  st->iter++;
  st->f_old = st->f;
  double fm = st->fhist[0];
  for (int i = 1; i < st->nhist; ++i) fm = fmax(fm, st->fhist[i]);
  st->fmax = fm;
  st->step = st->alpha;
  st->n_line = 0;
  st->dn_prev = -1.0;
  st->type = T_TRIAL;
  st->ps = st->step;
}

// top of an SPGL1 iteration: duality gap, root error, termination, Newton
// update of tau on the Pareto curve
__device__ void spg_check(SpgState* st) {
  const double f = st->f, rnorm = sqrt(2.0 * f), gnorm = st->ginf, tau = st->tau, sigma = st->sigma;
  const double gap = 2.0 * f - st->rtb + tau * gnorm;
  const double rel_gap = fabs(gap) / fmax(1.0, f);
  const double err_root = fabs(rnorm - sigma) / fmax(1.0, st->bnorm);
  const double err_f = fabs(f - 0.5 * sigma * sigma) / fmax(1.0, f);
  st->rel_gap = rel_gap;
  st->rnorm = rnorm;
  // the LASSO problem counts as solved when its duality gap is small or it
  // stagnates (relative decrease of f below 1e-4 far from the root, below a
  // tenth of the relative root error near it); f_old = 0 before the first step
  bool solved = rel_gap <= fmax(st->opt_tol, err_f);
  if (st->f_old > 0.0 && f > 0.0) {
    const double dec = fabs(f - st->f_old) / f;
    solved = solved || (rnorm > 2.0 * sigma ? dec <= kDecTol : dec <= 0.1 * fabs(rnorm - sigma) / fmax(rnorm, 1e-300));
  }
  int status = S_RUNNING;
  if (solved) {
    if (err_root <= st->opt_tol) status = S_ROOT;
    else if (gnorm <= st->bp_tol * rnorm || rnorm <= st->bp_tol * st->bnorm) status = S_BP;
  }
  if (status == S_RUNNING && st->iter >= st->max_iter) status = S_ITER;
  if (status != S_RUNNING) {
    st->status = status;
    st->done = 1;
    return;
  }
  if (solved && gnorm > 0.0) {
    const double tau_new = fmax(0.0, tau + (rnorm - sigma) * rnorm / gnorm);
    const bool shrink = tau_new < tau;
    st->tau = tau_new;
    st->pg_then = PG_THEN_TRIAL;
    st->type = shrink ? T_PROJX : T_PG;
    st->ps = shrink ? 0.0 : 1.0;
    return;
  }
  spg_start_trial(st);
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
  st->accept_x = st->accept_r = st->update_g = st->line_fail = st->stationary = 0;
  const int type = st->type;
  if (type == T_INIT || type == T_TRIAL) {
    if (!isfinite(st->ft) || !isfinite(st->gtd)) {
      st->status = S_NONFINITE;
      st->done = 1;
      return;
    }
  }
  if (type == T_INIT) {
    st->accept_x = st->accept_r = st->update_g = 1;
  } else if (type == T_PROJX) {
    // x projected onto the shrunk ball: residual, objective and gradient
    // are brought up to date with it
    st->accept_x = st->accept_r = st->update_g = 1;
  } else if (type == T_TRIAL) {
    st->n_trials++;
    bool acc = false;
    if (st->gtd >= 0.0) st->stationary = 1;                       // no descent: x is stationary
    else if (st->ft < st->fmax + st->gamma * st->gtd) acc = true;  // non-monotone Armijo
    else if (st->n_line >= st->max_line) {                         // last halving
      if (st->ft < st->f_old) acc = true;
      else st->stationary = 1;  // no measurable decrease left at this tau
    }
    if (acc) st->accept_x = st->accept_r = st->update_g = 1;
  }
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
  switch (st->type) {
    case T_INIT:
      spg_push_hist(st, st->f);
      st->type = T_PG;
      st->pg_then = PG_THEN_CHECK;
      st->ps = 1.0;
      break;
    case T_PG: {
      const double dxn = st->dinf;
      st->alpha = dxn < 1.0 / st->step_max ? st->step_max : fmin(st->step_max, fmax(st->step_min, 1.0 / dxn));
      if (st->pg_then == PG_THEN_CHECK) spg_check(st);
      else spg_start_trial(st);
      break;
    }
    case T_PROJX:
      st->type = T_PG;
      st->pg_then = PG_THEN_TRIAL;
      st->ps = 1.0;
      break;
    default: {  // T_TRIAL
      if (st->line_fail) {
        st->status = S_LINE;
        st->done = 1;
        break;
      }
      if (st->stationary) {
        // x is stationary for the current LASSO problem: check the root /
        // take the Newton step (unchanged f registers as stagnation);
        // repeated stationarity without progress is a failure
        if (++st->n_stationary > 3) {
          st->status = S_LINE;
          st->done = 1;
          break;
        }
        spg_check(st);
        break;
      }
      if (st->accept_r) {
        st->n_stationary = 0;
        const double sts = gq[0], sty = gq[1];
        st->alpha = sty <= 0.0 ? st->step_max : fmin(st->step_max, fmax(st->step_min, sts / sty));
        if (st->f > 0.5 * st->sigma * st->sigma) spg_push_hist(st, st->f);
        spg_check(st);
      } else {
        // backtrack along the projection arc; a flat arc (same displacement
        // norm as the previous trial) jumps to half the displacement scale
        const double dn = sqrt(st->dn2), gn = sqrt(st->gnorm2);
        if (st->dn_prev >= 0.0 && fabs(dn - st->dn_prev) <= 1e-6 * dn && gn > 0.0)
          st->step = fmin(0.5 * st->step, 0.5 * dn / gn);
        else
          st->step *= 0.5;
        st->dn_prev = dn;
        st->n_line++;
        st->ps = st->step;
      }
      break;
    }
  }
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
  st->type = T_INIT;
  st->ps = 0.0;
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
};

void enqueue_tick(SliceWork& w, int filter) {
  cudaStream_t s = w.stream;
  SpgVec V = w.V;
  k_spg_vstats<<<kRG, kRB, 0, s>>>(V);
  k_spg_proj_begin2<<<1, kRB, 0, s>>>(V);
  for (int pass = 0; pass < kPasses; ++pass) {
    k_spg_proj_pass<<<kRG, kRB, 0, s>>>(V);
    k_spg_proj_pick2<<<1, kRB, 0, s>>>(V, pass == kPasses - 1);
  }
  k_spg_proj_apply<<<kRG, kRB, 0, s>>>(V);
  cpct_launch_fwd(w.plan, V.xt, V.y, s);
  if (filter) {
    k_ring_colmean<<<(w.plan->ns + 31) / 32, kRB, 0, s>>>(V.y, w.ring.m, w.plan->m, w.plan->ns);
    k_ring_offset<<<1, kRB, 0, s>>>(w.ring.Q, w.ring.m, w.ring.d, w.plan->ns);
  }
  k_spg_resid<<<kRG, kRB, 0, s>>>(V, w.ring.d, w.plan->ns, filter);
  k_spg_mid<<<1, kRB, 0, s>>>(V);
  k_spg_accept<<<kRG, kRB, 0, s>>>(V);
  cpct_launch_adj(w.plan, V.r, V.gtmp, s);
  k_spg_grad<<<kRG, kRB, 0, s>>>(V);
  k_spg_end<<<1, kRB, 0, s>>>(V);
}

int fill_opts(const spgl1_opts* o, SpgState& st, double* tau0, int* filter) {
  st.max_iter = (o && o->max_iter > 0) ? o->max_iter : 300;
  st.opt_tol = (o && o->opt_tol > 0) ? o->opt_tol : 1e-4;
  st.bp_tol = (o && o->bp_tol > 0) ? o->bp_tol : 1e-6;
  st.memory = (o && o->memory > 0) ? o->memory : 3;
  st.gamma = (o && o->gamma > 0) ? o->gamma : 1e-4;
  st.step_min = (o && o->step_min > 0) ? o->step_min : 1e-16;
  st.step_max = (o && o->step_max > 0) ? o->step_max : 1e5;
  st.max_line = (o && o->max_line > 0) ? o->max_line : 30;
  if (st.memory > kHist) return CPCT_EINVAL;
  *tau0 = (o && (o->flags & CPCT_SPGL1_TAU0)) ? o->tau0 : -1.0;
  *filter = (o && (o->flags & CPCT_SPGL1_NO_FILTER)) ? 0 : 1;
  return CPCT_OK;
}

}  // namespace

extern "C" int spgl1_solve_batched(cpct_plan* const* plans, int batch, const float* const* d_b, const double* sigma,
                                   float* const* d_x, const spgl1_opts* opts, spgl1_info* info, cudaStream_t stream) {
  if (!plans || batch < 1 || !d_b || !sigma || !d_x) return CPCT_EINVAL;
  SpgState proto;
  std::memset(&proto, 0, sizeof(proto));
  double tau0 = -1.0;
  int filter = 1;
  int rc = fill_opts(opts, proto, &tau0, &filter);
  if (rc) return rc;
  for (int i = 0; i < batch; ++i) {
    if (!plans[i] || !d_b[i] || !d_x[i] || !(sigma[i] >= 0.0)) return CPCT_EINVAL;
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return CPCT_EINVAL;  // a plan holds per-call workspaces
  }
  std::vector<SliceWork> ws(batch);
  SpgState* d_states = nullptr;
  double* d_part = nullptr;
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
  for (int i = 0; i < batch; ++i) {
    SliceWork& w = ws[i];
    w.plan = plans[i];
    w.x = d_x[i];
    w.b = d_b[i];
    w.sigma = sigma[i];
    const long long n = (long long)w.plan->n * w.plan->n, m = (long long)w.plan->m * w.plan->ns;
    if (!cuda(cudaMalloc(&w.mem, sizeof(float) * (5 * n + 4 * m)))) goto done;
    SpgVec& V = w.V;
    V.n = n;
    V.m = m;
    V.x = w.x;
    V.xt = w.mem;
    V.xold = w.mem + n;
    V.g = w.mem + 2 * n;
    V.gold = w.mem + 3 * n;
    V.gtmp = w.mem + 4 * n;
    V.y = w.mem + 5 * n;
    V.rt = V.y + m;
    V.r = V.rt + m;
    V.bf = V.r + m;
    V.part = d_part + (size_t)i * P_TOTAL * kRG;
    V.st = d_states + i;
    if ((rc = ring_work(w.plan->ns, w.ring, stream)) != CPCT_OK) goto done;
    w.stream = stream;
    if (batch > 1) {
      branch.push_back(nullptr);
      if (!cuda(cudaStreamCreateWithFlags(&branch.back(), cudaStreamNonBlocking))) goto done;
    }
    // state, filtered data, zero gradient and residual, ||b||, tau0
    SpgState st = proto;
    st.sigma = w.sigma;
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
    const long long max_ticks = (long long)(proto.max_iter + 2) * (proto.max_line + 4) + 16;
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
  return rc;
}

extern "C" int spgl1_solve(cpct_plan* plan, const float* d_b, double sigma, float* d_x, const spgl1_opts* opts,
                           spgl1_info* info, cudaStream_t stream) {
  return spgl1_solve_batched(&plan, 1, &d_b, &sigma, &d_x, opts, info, stream);
}
