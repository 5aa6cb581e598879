// Allocation-free variant of one GEM-PIC s-step (gempic_step_noalloc, include/gempic.h).
//
// Some callers cannot allocate device memory themselves or through a library: programs whose
// host framework owns every device allocation under a fixed budget, plug-ins that are not
// allowed to call cudaMalloc, or code that must not add the implicit synchronisation of an
// allocation to a latency-critical loop.  For them this entry point advances a spectral state
// that the caller owns by one s-step and allocates nothing: its working memory is the
// file-scope array below, of a fixed size, which every GPU that loads the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/gempic.h"
#include "gempic_internal.h"
#include "gempic_setup.h"

namespace {

// Limits of the allocation-free step (checked before anything runs).
constexpr int kMaxNx = 1024;
constexpr int kMaxNy = 1024;
constexpr int kMaxNzeta = 4096;
constexpr int kRing = 3;         // s-levels k+1, k+2 of the (empty) particle stores
constexpr int kMaxCluster = 16;

// Byte layout of the scratch array.
constexpr size_t kTablesBytes = 64 * 1024;                      // twiddles, shifts, kx, ky
constexpr size_t kOffErr = kTablesBytes;                        // int error word
constexpr size_t kOffProgress = kOffErr + 256;                  // unused progress word
constexpr size_t kOffDiag = kOffProgress + 256;                 // kNDiag x C doubles
constexpr size_t kOffOnaxis = kOffDiag + 2048;                  // nzeta doubles
constexpr size_t kOffStCnt = kOffOnaxis + kMaxNzeta * 8;        // ring x nzeta ints
constexpr size_t kOffRqCnt = kOffStCnt + kRing * kMaxNzeta * 4; // ring x nzeta ints
constexpr size_t kOffJflag = kOffRqCnt + kRing * kMaxNzeta * 4; // ring x nzeta ints
constexpr size_t kScratchBytes = kOffJflag + kRing * kMaxNzeta * 4;
static_assert(kScratchBytes == 248320, "the documented size of the scratch array");
// the largest tables (nx = ny = 1024, FP64) take 53 248 bytes
static_assert((512 + 512 + 512 + 1024) * 16 + (512 + 1024) * 8 <= kTablesBytes,
              "tables of the largest grid exceed their part of the scratch");
static_assert(kMaxCluster * gempic::kNDiag * 8 <= 2048, "diagnostic partials do not fit");

// The working memory.  In host code this name is only a stand-in for the device array: its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[64] = {};

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace

extern "C" gempic_status gempic_step_noalloc(const gempic_config* cfg, int64_t step, void* state,
                                             size_t state_bytes, gempic_diag* diag_out,
                                             double* onaxis_out) {
  using gempic::Params;
  if (!cfg || !state || step < 0) return GEMPIC_EINVAL;
  const gempic_grid& g = cfg->grid;
  if (!pow2(g.nx) || g.nx < 8 || g.nx > kMaxNx) return GEMPIC_EINVAL;
  if (!pow2(g.ny) || g.ny > kMaxNy) return GEMPIC_EINVAL;
  if (g.nzeta < 2 || g.nzeta > kMaxNzeta) return GEMPIC_EINVAL;
  if (!(g.hx > 0) || !(g.hy > 0) || !(g.h > 0) || !(cfg->delta >= 0)) return GEMPIC_EINVAL;
  if (cfg->precision != 32 && cfg->precision != 64) return GEMPIC_EINVAL;
  if (cfg->hz) return GEMPIC_EINVAL;               // uniform zeta-step only
  if (cfg->beam) return GEMPIC_EINVAL;             // no stored-particle store for a bunch
  // no snapshot buffer and no continuity-residual output here
  if (cfg->flags & (GEMPIC_FLAG_SNAPSHOT | GEMPIC_FLAG_RESIDUAL)) return GEMPIC_EINVAL;
  {
    // the host-side tables (twiddles, shifts, kx, ky) must fit their part of the scratch
    const size_t nyh = g.ny > 1 ? g.ny / 2 : 1;
    const size_t eb0 = cfg->precision == 64 ? 8 : 4;
    const size_t tb = (g.nx / 2 + nyh + g.nx / 2 + g.ny) * 2 * eb0 + (g.nx / 2 + g.ny) * eb0;
    if (tb > kTablesBytes) return GEMPIC_EINVAL;
  }
  const int eb = cfg->precision == 64 ? 8 : 4;
  const size_t need = (size_t)6 * g.nzeta * g.ny * (g.nx / 2) * 2 * eb;
  if (state_bytes < need) return GEMPIC_EINVAL;

  Params p{};
  {
    const gempic_status st = gempic::setup_species(cfg, p);
    if (st != GEMPIC_OK) return st;
  }
  const int ppc_sum = p.ppc_sum;
  p.nx = g.nx;
  p.ny = g.ny;
  p.nz = g.nzeta;
  p.lognx = ilog2(g.nx);
  p.logny = ilog2(g.ny);
  p.hx = g.hx;
  p.hy = g.hy;
  p.h = g.h;
  p.delta = cfg->delta;
  p.delta_field = cfg->delta;
  p.seed = cfg->seed;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int smem_optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return GEMPIC_ECUDA;

  // launch shape: as gempic_create (no stored particles rejoin here, but particles still
  // move between bands)
  const int nxh = g.nx / 2;
  const int C0 = cfg->cluster_ctas;
  bool chosen = false;
  for (int cand = (C0 > 0 ? C0 : 1); cand <= (C0 > 0 ? C0 : kMaxCluster); cand *= 2) {
    if (g.ny % cand || nxh % cand || cand > kMaxCluster) continue;
    if (g.ny == 1 && cand != 1) continue;
    // 3-D bands need two rows or more (the current halo reaches two rows above the band)
    if (g.ny > 1 && g.ny / cand < 2) continue;
    const int RB = g.ny / cand, KB = nxh / cand, M = KB * g.ny;
    if (M > 512) continue;
    const int fresh = RB * g.nx * ppc_sum;
    int NT = std::max(M, fresh / 4);
    NT = std::min(512, std::max(128, (NT + 31) / 32 * 32));
    p.C = cand;
    p.RB = RB;
    p.KB = KB;
    p.M = M;
    p.logRB = ilog2(RB);
    p.logKB = ilog2(KB);
    p.nthreads = NT;
    // streaming slots beyond the fresh layer take particles that move in from other bands
    // (transverse compression): as many as the shared memory allows, up to max(256, fresh)
    for (int head = std::max(256, fresh); head >= 32; head -= 32) {
      p.pcap = fresh + head;
      if (gempic::smem_layout(p, eb) <= smem_optin) {
        chosen = true;
        break;
      }
    }
    if (chosen) break;
  }
  if (!chosen) return GEMPIC_EINVAL;

  // set-up, once per device, with that device current: the device address of the scratch
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess || !a) return GEMPIC_ECUDA;
      g_scratch_addr[dev] = a;
    }
    base = g_scratch_addr[dev];
  }
  char* b = (char*)base;
  p.tables = b;
  p.err = (int*)(b + kOffErr);
  p.progress = (unsigned long long*)(b + kOffProgress);
  p.diag_out = (double*)(b + kOffDiag);
  p.onaxis = (double*)(b + kOffOnaxis);
  p.st.cnt = (int*)(b + kOffStCnt);
  p.rq.cnt = (int*)(b + kOffRqCnt);
  p.jflag = (int*)(b + kOffJflag);
  // no stored-particle store: with capacity 0 a trapped particle sets the overflow bit
  p.bcap = 0;
  p.ring = kRing;
  gempic::PartStore* stores[2] = {&p.st, &p.rq};
  for (gempic::PartStore* S : stores) {
    S->cell = (int*)(b + kOffJflag);
    S->fx = S->fy = S->fz = S->ux = S->uy = S->uz = S->q = b + kOffJflag;
  }
  p.jbeam = b + kOffJflag;
  // no overflow slots: a band that outgrows its shared memory keeps the extra particles in
  // their old band (generic path) and, if even that fails, reports an overflow
  p.gcap = 0;
  p.pover = b + kOffJflag;
  p.snap = nullptr;
  p.timers = nullptr;
  p.state = state;
  p.k0 = step;
  p.nsteps = 1;
  p.P = 1;
  p.inject = cfg->nspecies > 0 ? 1 : 0;
  p.diag = 1;
  p.snapshot = 0;
  p.gt1 = (cfg->flags & GEMPIC_FLAG_GT1) ? 1 : 0;
  p.wait_spin_limit = 20000000;

  cudaStream_t s = (cudaStream_t)cfg->cuda_stream;
  // the array keeps the previous call's contents: clear what must start at zero
  e = cudaMemsetAsync(b + kOffErr, 0, kScratchBytes - kOffErr, s);
  if (e == cudaSuccess) e = gempic::launch_tables(cfg->precision, p, b, s);
  if (e == cudaSuccess) e = gempic::configure_march_canon(cfg->precision, p.smem_bytes);
  if (e == cudaSuccess) e = gempic::launch_march_canon(cfg->precision, p, s);
  int err = 0;
  double part[gempic::kNDiag * kMaxCluster];
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, p.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part, p.diag_out, sizeof(double) * gempic::kNDiag * p.C,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && onaxis_out)
    e = cudaMemcpyAsync(onaxis_out, p.onaxis, sizeof(double) * g.nzeta, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  if (diag_out) {
    double v[gempic::kNDiag];
    for (int i = 0; i < gempic::kNDiag; ++i) {
      v[i] = 0.0;
      for (int r = 0; r < p.C; ++r) v[i] += part[(size_t)i * p.C + r];
    }
    diag_out->step = step + 1;
    diag_out->field_energy = v[gempic::DG_FIELD];
    diag_out->kinetic_energy = v[gempic::DG_KIN];
    diag_out->charge_flux = v[gempic::DG_FLUX];
    diag_out->n_trapped = (int64_t)std::llround(v[gempic::DG_TRAP]);
    diag_out->n_stored = (int64_t)std::llround(v[gempic::DG_STORED]);
    diag_out->n_rejoined = (int64_t)std::llround(v[gempic::DG_REJOIN]);
    diag_out->pushes = (int64_t)std::llround(v[gempic::DG_PUSH]);
    diag_out->stored_kinetic_energy = v[gempic::DG_KST];
    diag_out->continuity_residual = -1.0;           // not computed by this entry point
    diag_out->gauss_residual = -1.0;
  }
  if (err & gempic::ERR_TIMEOUT) return GEMPIC_ETIMEOUT;
  if (err & gempic::ERR_NONFINITE) return GEMPIC_ENONFINITE;
  if (err & (gempic::ERR_PCAP | gempic::ERR_BCAP | gempic::ERR_QCAP)) return GEMPIC_EOVERFLOW;
  if (err) return GEMPIC_ESTATE;
  return GEMPIC_OK;
}
