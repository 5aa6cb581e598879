// Batched parameter scan: independent simulations stepped side by side, built on the public
// C-ABI.  Each instance owns a non-blocking stream and marches one s-step at a time (a single
// cluster per instance), so concurrently running instances never wait on one another; one
// step call submits one persistent launch per instance.
#include <cuda_runtime.h>

#include <vector>

#include "gempic.h"

struct gempic_batch {
  std::vector<gempic_sim*> sims;
  std::vector<cudaStream_t> streams;
};

extern "C" {

void gempic_batch_destroy(gempic_batch* b) {
  if (!b) return;
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  for (gempic_sim* sim : b->sims) gempic_destroy(sim);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  delete b;
}

gempic_status gempic_batch_create(const gempic_config* cfgs, int32_t n, gempic_batch** out) {
  if (!out) return GEMPIC_EINVAL;
  *out = nullptr;
  if (!cfgs || n < 1) return GEMPIC_EINVAL;
  gempic_batch* b = new gempic_batch;
  gempic_status st = GEMPIC_OK;
  for (int32_t i = 0; i < n; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      st = GEMPIC_ECUDA;
      break;
    }
    b->streams.push_back(s);
    gempic_config c = cfgs[i];
    c.cuda_stream = s;
    c.pipeline_depth = 1;
    gempic_sim* sim = nullptr;
    st = gempic_create(&c, &sim);
    if (st != GEMPIC_OK) break;
    b->sims.push_back(sim);
  }
  if (st != GEMPIC_OK) {
    gempic_batch_destroy(b);
    return st;
  }
  *out = b;
  return GEMPIC_OK;
}

gempic_status gempic_batch_step_async(gempic_batch* b, int32_t n) {
  if (!b || n < 0) return GEMPIC_EINVAL;
  for (gempic_sim* sim : b->sims) {
    const gempic_status st = gempic_step_async(sim, n);
    if (st != GEMPIC_OK) return st;
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
  if (!b || i < 0 || i >= (int32_t)b->streams.size()) return nullptr;
  return (void*)b->streams[i];
}

}  // extern "C"
