// Per-kernel CUDA-event profiler and launch counter of a plan.
//
// Profiling is off by default.  When a kernel id is enabled, each of its
// launches is bracketed by a pair of CUDA events recorded on the launch
// stream; cpct_profile_read() synchronizes on those events and reports the
// summed device time and the number of launches per kernel.
#include <vector>

#include "common.cuh"

struct CpctProfiler {
  unsigned mask = 0;
  struct Rec {
    int kid;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open_a = nullptr;
  int open_kid = -1;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
};

void cpct_prof_begin(cpct_plan* p, int kid, cudaStream_t s) {
  p->launches++;
  CpctProfiler* pr = p->prof;
  if (!pr || !(pr->mask & (1u << kid))) return;
  if (p->capturing) {
    // inside a graph capture: an event-record node whose event the replay sets
    cpct_graph_prof_event(p, kid, true, pr->get(), s);
    return;
  }
  pr->open_a = pr->get();
  pr->open_kid = kid;
  if (pr->open_a) cudaEventRecord(pr->open_a, s);
}

void cpct_prof_end(cpct_plan* p, int kid, cudaStream_t s) {
  CpctProfiler* pr = p->prof;
  if (!pr || !(pr->mask & (1u << kid))) return;
  if (p->capturing) {
    cpct_graph_prof_event(p, kid, false, pr->get(), s);
    return;
  }
  if (pr->open_kid != kid || !pr->open_a) return;
  cudaEvent_t b = pr->get();
  if (!b) return;
  cudaEventRecord(b, s);
  pr->recs.push_back({kid, pr->open_a, b});
  pr->open_a = nullptr;
  pr->open_kid = -1;
}

void cpct_prof_free(cpct_plan* p) {
  if (!p->prof) return;
  for (auto& r : p->prof->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p->prof->pool) cudaEventDestroy(e);
  delete p->prof;
  p->prof = nullptr;
}

// events of the plan's profiler pool, for graph replays (graphs.cu)
cudaEvent_t cpct_prof_event(cpct_plan* p) { return p->prof ? p->prof->get() : nullptr; }
void cpct_prof_push(cpct_plan* p, int kid, cudaEvent_t a, cudaEvent_t b) {
  if (p->prof) p->prof->recs.push_back({kid, a, b});
}
void cpct_prof_release(cpct_plan* p, cudaEvent_t e) {
  if (p->prof && e) p->prof->pool.push_back(e);
}
unsigned cpct_prof_mask(const cpct_plan* p) { return p->prof ? p->prof->mask : 0u; }

extern "C" int cpct_profile_enable(cpct_plan* p, unsigned mask) {
  if (!p) return CPCT_EINVAL;
  if (!p->prof) p->prof = new (std::nothrow) CpctProfiler;
  if (!p->prof) return CPCT_ENOMEM;
  p->prof->mask = mask;
  return CPCT_OK;
}

extern "C" int cpct_profile_read(cpct_plan* p, double* total_ms, long long* launches) {
  if (!p || !total_ms || !launches) return CPCT_EINVAL;
  for (int k = 0; k < KID_COUNT; ++k) {
    total_ms[k] = 0.0;
    launches[k] = 0;
  }
  if (!p->prof) return CPCT_OK;
  for (auto& r : p->prof->recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return CPCT_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return CPCT_ECUDA;
    total_ms[r.kid] += ms;
    launches[r.kid] += 1;
    p->prof->pool.push_back(r.a);
    p->prof->pool.push_back(r.b);
  }
  p->prof->recs.clear();
  return CPCT_OK;
}

extern "C" const char* cpct_kernel_name(int kid) {
  static const char* names[KID_COUNT] = {"k_fwd_col", "k_fwd_row", "k_fwd_interp", "k_fwd_ray", "k_adj_ray",
                                         "k_adj_spread", "k_adj_reduce", "k_adj_row", "k_adj_col"};
  return (kid >= 0 && kid < KID_COUNT) ? names[kid] : "";
}

extern "C" long long cpct_launch_count(cpct_plan* p, int reset) {
  if (!p) return -1;
  long long n = p->launches;
  if (reset) p->launches = 0;
  return n;
}
