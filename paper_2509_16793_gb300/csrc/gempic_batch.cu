// Batched parameter scan: independent simulations stepped together in one persistent launch
// per call (the paper has no counterpart; include/gempic.h, gempic_batch_*).
//
// Work items are (simulation, march index c), c = 0 .. n-1 for the s-steps k .. k+n-1 of the
// call, laid out s-step by s-step with the costliest simulations first.  The persistent kernel
// (batch_kernel, one CTA per SM) takes them from a queue; the march of a simulation's s-step
// k+c waits slice by slice for its s-step k+c-1 (the wavefront of a single simulation), so a
// large simulation marches several s-steps at once while small ones fill the remaining SMs,
// and the makespan is no longer the largest simulation's n s-steps one after another.
//
// The costs come from a small autotuner run at creation: for every size class (grid and
// species of a simulation) it times one s-step of a representative simulation at each
// candidate CTA size (256 and 512 threads), keeps the per-class times, launches the batch at
// the CTA size with the smallest total over the simulations, and orders the items by their
// class's measured time.  Each call's work is a CUDA graph (parameter upload, queue reset,
// persistent launch) built once per number of s-steps and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "gempic.h"
#include "gempic_internal.h"

namespace gempic {
gempic_status batch_prepare(gempic_sim* s, int nthreads, int nsteps, Params* out);
void batch_advance(gempic_sim* s, int n);
int batch_precision(const gempic_sim* s);
}  // namespace gempic

namespace {

constexpr int kBatchDepth = 16;                 // s-steps per launch (per simulation in flight)
constexpr int kCandidates[2] = {256, 512};      // CTA sizes the autotuner tries

}  // namespace

struct gempic_batch {
  std::vector<gempic_sim*> sims;
  cudaStream_t stream = nullptr;
  int precision = 32;
  int nthreads = 512;
  int smem = 0, grid = 0;
  std::vector<int> order;                       // simulations by descending measured cost
  std::vector<double> cost_ms;                  // per simulation: its class's ms per s-step
  std::vector<std::vector<double>> class_ms;    // per simulation: ms per s-step per candidate
  gempic::Params* d_params = nullptr;
  gempic::Params* h_params = nullptr;           // pinned: read by the graph's upload
  int* d_head = nullptr;
  int2* d_items = nullptr;
  int items_n = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_n = 0;
  cudaEvent_t done = nullptr;
  bool launched = false;
};

namespace {

void release(gempic_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (gempic_sim* sim : b->sims) gempic_destroy(sim);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_params) cudaFree(b->d_params);
  if (b->h_params) cudaFreeHost(b->h_params);
  if (b->d_head) cudaFree(b->d_head);
  if (b->d_items) cudaFree(b->d_items);
  if (b->done) cudaEventDestroy(b->done);
  if (b->stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
}

// ms per s-step of one simulation of this config at CTA size nt: a throw-away simulation on
// the batch's stream, one warm-up s-step, then two timed ones (CUDA events); <0 if the size
// does not apply
double time_class(const gempic_config& cfg, int nt, cudaStream_t stream) {
  gempic_config c = cfg;
  c.cuda_stream = stream;
  c.pipeline_depth = 1;
  c.beam = nullptr;
  gempic_sim* sim = nullptr;
  if (gempic_create(&c, &sim) != GEMPIC_OK) return -1.0;
  double ms = -1.0;
  gempic::Params q;
  if (gempic::batch_prepare(sim, nt, 1, &q) == GEMPIC_OK && gempic_step(sim, 1) == GEMPIC_OK) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, stream);
    const gempic_status st = gempic_step(sim, 2);
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    if (st == GEMPIC_OK) ms = t / 2.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  gempic_destroy(sim);
  cudaGetLastError();
  return ms;
}

gempic_status autotune(gempic_batch* b, const gempic_config* cfgs, int n) {
  // size class: grid, precision, species and flags decide the per-slice work
  std::map<std::tuple<int, int, int, int, int, unsigned>, std::vector<double>> classes;
  b->class_ms.assign(n, {});
  for (int i = 0; i < n; ++i) {
    const gempic_config& c = cfgs[i];
    int ppc = 0;
    for (int j = 0; j < c.nspecies; ++j) ppc += c.species[j].ppc;
    const auto key = std::make_tuple(c.grid.nx, c.grid.ny, c.grid.nzeta, c.precision, ppc, c.flags);
    auto it = classes.find(key);
    if (it == classes.end()) {
      std::vector<double> t;
      for (int nt : kCandidates) t.push_back(time_class(c, nt, b->stream));
      it = classes.emplace(key, t).first;
    }
    b->class_ms[i] = it->second;
  }
  // the CTA size of the launch: smallest total over the simulations (every one must run)
  double best = -1.0;
  for (int ci = 0; ci < 2; ++ci) {
    double tot = 0.0;
    bool ok = true;
    for (int i = 0; i < n; ++i) {
      if (b->class_ms[i][ci] < 0) ok = false;
      tot += b->class_ms[i][ci];
    }
    if (ok && (best < 0 || tot < best)) {
      best = tot;
      b->nthreads = kCandidates[ci];
    }
  }
  if (best < 0) return GEMPIC_EINVAL;
  const int ci = b->nthreads == kCandidates[0] ? 0 : 1;
  b->cost_ms.resize(n);
  for (int i = 0; i < n; ++i) b->cost_ms[i] = b->class_ms[i][ci];
  b->order.resize(n);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int a, int c) { return b->cost_ms[a] > b->cost_ms[c]; });
  return GEMPIC_OK;
}

// the work items of a call of m s-steps: s-step by s-step, costliest simulation first
cudaError_t build_items(gempic_batch* b, int m) {
  if (b->items_n == m) return cudaSuccess;
  std::vector<int2> items;
  for (int c = 0; c < m; ++c)
    for (int i : b->order) items.push_back(make_int2(i, c));
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  cudaError_t e = cudaMalloc(&b->d_items, items.size() * sizeof(int2));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
  b->items_n = e == cudaSuccess ? m : 0;
  return e;
}

// the call as a graph: upload of the launch parameters, queue reset, persistent launch
cudaError_t build_graph(gempic_batch* b, int m) {
  if (b->exec && b->graph_n == m) return cudaSuccess;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  const int n = (int)b->sims.size();
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaMemcpyAsync(b->d_params, b->h_params, n * sizeof(gempic::Params), cudaMemcpyHostToDevice,
                  b->stream);
  cudaMemsetAsync(b->d_head, 0, sizeof(int), b->stream);
  gempic::launch_batch(b->precision, b->d_params, b->d_items, n * m, b->d_head, b->grid,
                       b->nthreads, b->smem, b->stream);
  e = cudaStreamEndCapture(b->stream, &b->graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  b->graph_n = e == cudaSuccess ? m : 0;
  return e;
}

}  // namespace

extern "C" {

void gempic_batch_destroy(gempic_batch* b) {
  if (b) release(b);
}

gempic_status gempic_batch_create(const gempic_config* cfgs, int32_t n, gempic_batch** out) {
  if (!out) return GEMPIC_EINVAL;
  *out = nullptr;
  if (!cfgs || n < 1) return GEMPIC_EINVAL;
  for (int32_t i = 1; i < n; ++i)
    if (cfgs[i].precision != cfgs[0].precision) return GEMPIC_EINVAL;
  gempic_batch* b = new gempic_batch;
  b->precision = cfgs[0].precision;
  gempic_status st = GEMPIC_OK;
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    release(b);
    return GEMPIC_ECUDA;
  }
  for (int32_t i = 0; i < n && st == GEMPIC_OK; ++i) {
    gempic_config c = cfgs[i];
    c.cuda_stream = b->stream;
    c.pipeline_depth = kBatchDepth;
    gempic_sim* sim = nullptr;
    st = gempic_create(&c, &sim);
    if (st == GEMPIC_OK) b->sims.push_back(sim);
  }
  if (st == GEMPIC_OK) st = autotune(b, cfgs, n);
  // every simulation at the chosen CTA size; the launch takes the largest shared memory
  gempic::Params q;
  for (int32_t i = 0; i < n && st == GEMPIC_OK; ++i) {
    st = gempic::batch_prepare(b->sims[i], b->nthreads, 1, &q);
    b->smem = std::max(b->smem, q.smem_bytes);
  }
  cudaError_t e = cudaSuccess;
  if (st == GEMPIC_OK) {
    int dev = 0, nsm = 0, occ = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = gempic::configure_batch(b->precision, b->smem);
    if (e == cudaSuccess) e = gempic::batch_occupancy(b->precision, b->nthreads, b->smem, &occ);
    b->grid = nsm * std::max(1, occ);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_params, n * sizeof(gempic::Params));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_params, n * sizeof(gempic::Params));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_head, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
  }
  if (st != GEMPIC_OK) {
    release(b);
    return st;
  }
  *out = b;
  return GEMPIC_OK;
}

gempic_status gempic_batch_step_async(gempic_batch* b, int32_t n) {
  if (!b || n < 0) return GEMPIC_EINVAL;
  const int ns = (int)b->sims.size();
  for (int32_t done = 0; done < n;) {
    const int m = std::min(kBatchDepth, n - done);
    // the previous call's upload has read the pinned parameters: they may be rewritten
    if (b->launched && cudaEventSynchronize(b->done) != cudaSuccess) return GEMPIC_ECUDA;
    for (int i = 0; i < ns; ++i) {
      const gempic_status st = gempic::batch_prepare(b->sims[i], b->nthreads, m, &b->h_params[i]);
      if (st != GEMPIC_OK) return st;
    }
    cudaError_t e = build_items(b, m);
    if (e == cudaSuccess) e = build_graph(b, m);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return GEMPIC_ECUDA;
    }
    b->launched = true;
    for (int i = 0; i < ns; ++i) gempic::batch_advance(b->sims[i], m);
    done += m;
  }
  return GEMPIC_OK;
}

gempic_status gempic_batch_sync(gempic_batch* b) {
  if (!b) return GEMPIC_EINVAL;
  gempic_status first = GEMPIC_OK;
  for (gempic_sim* sim : b->sims) {
    const gempic_status st = gempic_sync(sim);
    if (first == GEMPIC_OK) first = st;
  }
  return first;
}

gempic_status gempic_batch_step(gempic_batch* b, int32_t n) {
  const gempic_status st = gempic_batch_step_async(b, n);
  const gempic_status ss = b ? gempic_batch_sync(b) : GEMPIC_EINVAL;
  return st != GEMPIC_OK ? st : ss;
}

int32_t gempic_batch_size(const gempic_batch* b) { return b ? (int32_t)b->sims.size() : 0; }

gempic_sim* gempic_batch_sim(gempic_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->sims.size()) return nullptr;
  return b->sims[i];
}

void* gempic_batch_stream(gempic_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->sims.size()) return nullptr;
  return (void*)b->stream;
}

gempic_status gempic_batch_tuning(const gempic_batch* b, int32_t i, int32_t* nthreads,
                                  double* ms_per_step) {
  if (!b || i < 0 || i >= (int32_t)b->sims.size()) return GEMPIC_EINVAL;
  if (nthreads) *nthreads = b->nthreads;
  if (ms_per_step) *ms_per_step = b->cost_ms[i];
  return GEMPIC_OK;
}

}  // extern "C"
