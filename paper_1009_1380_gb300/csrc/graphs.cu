// Graph replay of the Radon operators (cpct_plan_set_graphs).
//
// A forward or adjoint application launches four or five kernels; launched
// one by one from the host each costs the GPU front end about two
// microseconds more than the same kernel inside a CUDA graph.  In graph mode
// the first call with a given (operator, input, output, profiling mask)
// captures the launch sequence on a private stream into a CUDA graph; later
// calls with the same key replay it on the caller's stream.  Calls made while
// the caller's stream is itself being captured (batched operators, SPGL1
// ticks) launch directly, so they land in the caller's graph.  Profiled
// kernels keep their CUDA-event brackets: they are captured as event-record
// nodes, and every replay points those nodes at fresh events of the plan's
// profiler before the launch.  Any change of the launch configuration (bin
// plans, work-item caps, round width) drops the cache.
#include <vector>

#include "common.cuh"

cudaEvent_t cpct_prof_event(cpct_plan* p);
void cpct_prof_push(cpct_plan* p, int kid, cudaEvent_t a, cudaEvent_t b);
void cpct_prof_release(cpct_plan* p, cudaEvent_t e);
unsigned cpct_prof_mask(const cpct_plan* p);

namespace {

struct EvNode {
  int kid;
  bool begin;
  cudaGraphNode_t node;
  cudaEvent_t placeholder;  // the event captured into the node
};

constexpr int kMaxGraphs = 8;

}  // namespace

// an operator graph being captured: its event-record nodes in capture order
struct GraphCapture {
  std::vector<EvNode> ev;
  bool failed = false;
};

struct GraphEntry {
  int op = -1;
  const void* in = nullptr;
  void* out = nullptr;
  unsigned mask = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long n_launch = 0;  // kernels of one application
  std::vector<EvNode> ev;
  unsigned long long last_use = 0;
};

struct GraphCache {
  std::vector<GraphEntry> e;
  cudaStream_t cap = nullptr;  // private capture stream
  unsigned long long tick = 0;
};

namespace {

void free_entry(cpct_plan* p, GraphEntry& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  for (auto& n : g.ev) cpct_prof_release(p, n.placeholder);
  g = GraphEntry();
}

int launch_direct(cpct_plan* p, int op, const void* in, void* out, cudaStream_t s) {
  if (op == 0) return cpct_launch_fwd(p, static_cast<const float*>(in), static_cast<float*>(out), s);
  return cpct_launch_adj(p, static_cast<const float*>(in), static_cast<float*>(out), s);
}

}  // namespace

void cpct_graph_prof_event(cpct_plan* p, int kid, bool begin, cudaEvent_t ev, cudaStream_t s) {
  GraphCapture* c = p->capturing;
  if (!c || !ev) {
    if (c) c->failed = true;
    return;
  }
  // an external event-record node, then the node itself from the capture's
  // current dependency set (the node just added)
  if (cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) != cudaSuccess) {
    c->failed = true;
    cpct_prof_release(p, ev);
    return;
  }
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess || nd != 1 || !deps) {
    c->failed = true;
    return;
  }
  c->ev.push_back({kid, begin, deps[0], ev});
}

void cpct_graph_clear(cpct_plan* p) {
  if (!p || !p->graphs) return;
  for (auto& g : p->graphs->e) free_entry(p, g);
  p->graphs->e.clear();
}

void cpct_graph_free(cpct_plan* p) {
  if (!p || !p->graphs) return;
  cpct_graph_clear(p);
  if (p->graphs->cap) cudaStreamDestroy(p->graphs->cap);
  delete p->graphs;
  p->graphs = nullptr;
}

namespace {

// capture one application into a new cache entry; false: not captured
bool capture(cpct_plan* p, int op, const void* in, void* out, unsigned mask, GraphEntry& g) {
  GraphCache* gc = p->graphs;
  if (!gc->cap && cudaStreamCreateWithFlags(&gc->cap, cudaStreamNonBlocking) != cudaSuccess) {
    gc->cap = nullptr;
    return false;
  }
  GraphCapture c;
  const long long l0 = p->launches;
  if (cudaStreamBeginCapture(gc->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  p->capturing = &c;
  const int rc = launch_direct(p, op, in, out, gc->cap);
  p->capturing = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(gc->cap, &graph);
  const long long n = p->launches - l0;
  p->launches = l0;
  bool ok = rc == CPCT_OK && ec == cudaSuccess && graph && !c.failed;
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& e : c.ev) cpct_prof_release(p, e.placeholder);
    cudaGetLastError();  // clear a capture error so the direct launch can run
    return false;
  }
  g.op = op;
  g.in = in;
  g.out = out;
  g.mask = mask;
  g.graph = graph;
  g.exec = exec;
  g.n_launch = n;
  g.ev = std::move(c.ev);
  return true;
}

// point the entry's event nodes at fresh profiler events, then launch
int replay(cpct_plan* p, GraphEntry& g, cudaStream_t s) {
  for (size_t i = 0; i + 1 < g.ev.size(); i += 2) {
    const EvNode& a = g.ev[i];
    const EvNode& b = g.ev[i + 1];
    if (!a.begin || b.begin || a.kid != b.kid) return CPCT_ECUDA;
    cudaEvent_t ea = cpct_prof_event(p), eb = cpct_prof_event(p);
    if (!ea || !eb) return CPCT_ECUDA;
    if (cudaGraphExecEventRecordNodeSetEvent(g.exec, a.node, ea) != cudaSuccess ||
        cudaGraphExecEventRecordNodeSetEvent(g.exec, b.node, eb) != cudaSuccess)
      return CPCT_ECUDA;
    cpct_prof_push(p, a.kid, ea, eb);
  }
  if (cudaGraphLaunch(g.exec, s) != cudaSuccess) return CPCT_ECUDA;
  p->launches += g.n_launch;
  return CPCT_OK;
}

}  // namespace

int cpct_graph_run(cpct_plan* p, int op, const void* in, void* out, cudaStream_t s) {
  if (!p->graph_mode) return launch_direct(p, op, in, out, s);
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone)
    return launch_direct(p, op, in, out, s);
  if (!p->graphs) {
    p->graphs = new (std::nothrow) GraphCache;
    if (!p->graphs) return launch_direct(p, op, in, out, s);
  }
  GraphCache* gc = p->graphs;
  const unsigned mask = cpct_prof_mask(p);
  ++gc->tick;
  for (auto& g : gc->e)
    if (g.op == op && g.in == in && g.out == out && g.mask == mask) {
      g.last_use = gc->tick;
      return replay(p, g, s);
    }
  GraphEntry g;
  if (!capture(p, op, in, out, mask, g)) return launch_direct(p, op, in, out, s);
  g.last_use = gc->tick;
  if ((int)gc->e.size() >= kMaxGraphs) {
    size_t lru = 0;
    for (size_t i = 1; i < gc->e.size(); ++i)
      if (gc->e[i].last_use < gc->e[lru].last_use) lru = i;
    free_entry(p, gc->e[lru]);
    gc->e.erase(gc->e.begin() + lru);
  }
  gc->e.push_back(std::move(g));
  return replay(p, gc->e.back(), s);
}

extern "C" int cpct_plan_set_graphs(cpct_plan* p, int enable) {
  if (!p || (enable != 0 && enable != 1)) return CPCT_EINVAL;
  p->graph_mode = enable;
  if (!enable) cpct_graph_clear(p);
  return CPCT_OK;
}

extern "C" int cpct_plan_graphs(const cpct_plan* p) {
  if (!p) return CPCT_EINVAL;
  return p->graphs ? (int)p->graphs->e.size() : 0;
}
