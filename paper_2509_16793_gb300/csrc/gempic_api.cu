// Host side of the GEM-PIC C-ABI (include/gempic.h): validation, launch shape, device
// allocations, initial condition, stepping and copies.  All compute runs in the kernels of
// gempic_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "../../include/gempic.h"
#include "gempic_internal.h"
#include "gempic_setup.h"

using gempic::Params;

struct gempic_sim {
  gempic_config cfg;
  gempic_species species[gempic::kMaxSpecies];
  gempic_laser laser;
  bool has_laser = false;
  gempic_channel channel;
  bool has_channel = false;
  gempic_beam beam;                // Gaussian bunch sampled at initialisation (n_macro > 0)
  bool has_beam = false;
  int beam_species = 0;            // species slot of the bunch
  int nspecies_all = 0;            // injected species plus a slot of the bunch's own
  std::vector<double> hz, zp;      // variable zeta-step: slab thicknesses, plane positions
  Params p{};                      // launch template
  int eb = 8;                      // bytes per real
  int pmax = 1;                    // concurrent marches
  cudaStream_t stream = nullptr;
  long long k = 0;                 // s-steps completed
  bool initialized = false;
  gempic_status failed = GEMPIC_OK;
  long long launches = 0;
  int diag_cap = 0;
  long long last_launch_k0 = 0;
  int last_launch_n = 0;
  std::vector<void*> allocs;
  void* stage = nullptr;           // device staging of the public state layout (host copies)
  // learned current denoiser (two passes per s-step) and the current of the last s-step
  gempic_denoiser* dn = nullptr;
  void* jcap = nullptr;            // [nz][3][ny][nx] plain current of the last s-step
  void* jden = nullptr;            // its denoised form
  void* state2 = nullptr;          // provisional level of the first pass
  bool denoised_last = false;      // the last launch was a denoised s-step
  // particles placed before the first step: absolute positions
  std::vector<double> px, py, pz, pux, puy, puz, pq;
  std::vector<int> psp;
  // gempic_step_streamed: input and output levels on the device (public layout), the
  // host-mapped words [ready: pmax][done: pmax], the copy streams (out, in, and the first
  // s-step's input) and their events
  void* io_a = nullptr;
  void* io_b = nullptr;
  unsigned long long* io_host = nullptr;
  unsigned long long* io_dev = nullptr;
  cudaStream_t io_out = nullptr, io_in = nullptr, io_fill = nullptr;
  std::vector<cudaEvent_t> io_events;
  // denoised chain: rings of four plain and denoised currents, host-mapped words [done: 8]
  // [ready: 8], the stream the net runs on
  void* dn_jcap[4] = {};
  void* dn_jden[4] = {};
  unsigned long long* dn_host = nullptr;
  unsigned long long* dn_dev = nullptr;
  cudaStream_t dn_stream = nullptr;
  void* jcap_last = nullptr;       // the plain current of the last s-step
};

namespace {

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

gempic_status cuda_fail(gempic_sim* s, cudaError_t e) {
  if (e == cudaSuccess) return GEMPIC_OK;
  if (s) s->failed = GEMPIC_ECUDA;
  return GEMPIC_ECUDA;
}

#ifdef GEMPIC_PHASE_TIMERS
// profiling builds: 256 words of phase sums, then per (slice, CTA) of the first march of a
// launch the cycles from the slice start to the arrival at and the release from barrier B1
static int timer_words(const gempic::Params& p) { return 256 + 2 * p.nz * p.C; }
#endif

template <typename Tp>
cudaError_t dalloc(gempic_sim* s, Tp** ptr, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return e;
  s->allocs.push_back(v);
  e = cudaMemsetAsync(v, 0, bytes > 0 ? bytes : 16, s->stream);
  *ptr = (Tp*)v;
  return e;
}

gempic_status check_device_error(gempic_sim* s) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, s->p.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (err == 0) return GEMPIC_OK;
  gempic_status st = (err & gempic::ERR_TIMEOUT) ? GEMPIC_ETIMEOUT
                     : (err & gempic::ERR_NONFINITE) ? GEMPIC_ENONFINITE
                     : (err & (gempic::ERR_PCAP | gempic::ERR_BCAP | gempic::ERR_QCAP))
                         ? GEMPIC_EOVERFLOW
                         : GEMPIC_ESTATE;
  s->failed = st;
  return st;
}

cudaError_t ensure_diag_cap(gempic_sim* s, int n) {
  if (n <= s->diag_cap) return cudaSuccess;
  double *d = nullptr, *o = nullptr, *r = nullptr, *gr = nullptr;
  cudaError_t e = dalloc(s, &d, (size_t)n * gempic::kNDiag * s->p.C * sizeof(double));
  if (e != cudaSuccess) return e;
  e = dalloc(s, &o, (size_t)n * s->p.nz * sizeof(double));
  if (e != cudaSuccess) return e;
  e = dalloc(s, &r, (size_t)n * sizeof(double));
  if (e != cudaSuccess) return e;
  e = dalloc(s, &gr, (size_t)n * sizeof(double));
  if (e != cudaSuccess) return e;
  s->p.gauss_out = gr;
  s->p.diag_out = d;
  s->p.onaxis = o;
  s->p.resid_out = r;
  s->diag_cap = n;
  return cudaSuccess;
}

// stored particles given in absolute coordinates -> level-0 buckets (ring slot 0)
gempic_status upload_particles(gempic_sim* s) {
  const size_t n = s->px.size();
  if (n == 0) return GEMPIC_OK;
  const Params& p = s->p;
  const size_t cap = (size_t)p.nz * p.bcap;
  std::vector<int> cnt(p.nz, 0), cell(cap, 0);
  std::vector<double> f[7];
  for (auto& v : f) v.assign(cap, 0.0);
  for (size_t i = 0; i < n; ++i) {
    const double X = s->px[i] / p.hx, Y = p.ny > 1 ? s->py[i] / p.hy : 0.0;
    const double fX = std::floor(X), fY = std::floor(Y);
    int m;
    double fz;
    if (s->zp.empty()) {
      const double Z = s->pz[i] / p.h;
      m = (int)std::ceil(Z) - 1;
      fz = Z - m;
    } else {
      // slab m with zeta_m < zeta <= zeta_{m+1}
      m = (int)(std::lower_bound(s->zp.begin(), s->zp.end(), s->pz[i]) - s->zp.begin()) - 1;
      fz = m >= 0 && m < p.nz ? (s->pz[i] - s->zp[m]) / s->hz[m] : 0.0;
    }
    if (m < 0 || m >= p.nz) continue;
    const int ix = ((int)fX % p.nx + p.nx) % p.nx, iy = ((int)fY % p.ny + p.ny) % p.ny;
    if (cnt[m] >= p.bcap) return GEMPIC_EOVERFLOW;
    const size_t e = (size_t)m * p.bcap + cnt[m]++;
    cell[e] = ix | (iy << 10) | (s->psp[i] << 20);
    f[0][e] = X - fX;
    f[1][e] = Y - fY;
    f[2][e] = fz;
    f[3][e] = s->pux[i];
    f[4][e] = s->puy[i];
    f[5][e] = s->puz[i];
    f[6][e] = s->pq[i];
  }
  cudaError_t e = cudaMemcpyAsync(p.st.cnt, cnt.data(), p.nz * sizeof(int), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p.st.cell, cell.data(), cap * sizeof(int), cudaMemcpyHostToDevice, s->stream);
  void* dst[7] = {p.st.fx, p.st.fy, p.st.fz, p.st.ux, p.st.uy, p.st.uz, p.st.q};
  std::vector<float> ff(cap);
  for (int j = 0; j < 7 && e == cudaSuccess; ++j) {
    if (s->eb == 8) {
      e = cudaMemcpyAsync(dst[j], f[j].data(), cap * 8, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    } else {
      for (size_t i = 0; i < cap; ++i) ff[i] = (float)f[j][i];
      e = cudaMemcpyAsync(dst[j], ff.data(), cap * 4, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_fail(s, e);
}

gempic_status ensure_initialized(gempic_sim* s) {
  if (s->failed != GEMPIC_OK) return GEMPIC_ESTATE;
  if (s->initialized) return GEMPIC_OK;
  const int prec = s->cfg.precision;
  cudaError_t e = cudaSuccess;
  if (s->has_laser) {
    e = gempic::launch_laser_init(prec, s->p, s->laser.a0, s->laser.waist, s->laser.duration,
                                  s->laser.zeta_center, s->laser.pol, s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  gempic_status st = upload_particles(s);
  if (st != GEMPIC_OK) return st;
  if (s->has_beam && s->beam.n_macro > 0) {
    // the bunch is appended to the level-0 buckets after the host-placed particles
    const gempic_beam& b = s->beam;
    const double pi = 3.14159265358979323846;
    const double total = s->p.ny > 1
        ? b.charge * b.n_peak * std::pow(2.0 * pi, 1.5) * b.sigma_r * b.sigma_r * b.sigma_z
        : b.charge * b.n_peak * 2.0 * pi * b.sigma_r * b.sigma_z;
    gempic::BeamArgs a;
    a.xc = 0.5 * s->p.nx * s->p.hx;
    a.yc = s->p.ny > 1 ? 0.5 * s->p.ny * s->p.hy : 0.0;
    a.sr = b.sigma_r;
    a.sz = b.sigma_z;
    a.zc = b.zeta_center;
    a.gamma = b.gamma;
    a.spread = b.rel_spread;
    a.q = total / (double)b.n_macro;
    a.n = b.n_macro;
    a.seed = b.seed;
    a.sp = s->beam_species;
    e = gempic::launch_beam_init(prec, s->p, a, s->stream);
    s->launches++;
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  // Delta = 0 consistency march: R^1 = R^0, fills E_z, B_z, L of the initial laser and
  // pushes the particles placed at level 0 to level 1.
  e = ensure_diag_cap(s, 1);
  if (e != cudaSuccess) return cuda_fail(s, e);
  Params q = s->p;
  q.k0 = -1;
  q.nsteps = 1;
  q.P = 1;
  q.inject = 0;
  q.delta_field = 0.0;
  q.diag = 1;
  q.snapshot = 0;
  e = gempic::launch_march(prec, q, s->stream);
  s->launches++;
  if (e != cudaSuccess) return cuda_fail(s, e);
  st = check_device_error(s);
  if (st != GEMPIC_OK) return st;
  s->initialized = true;
  s->last_launch_k0 = -1;
  s->last_launch_n = 1;
  return GEMPIC_OK;
}

}  // namespace

namespace gempic {

// ---- support of the batched scan (gempic_batch.cu) ---------------------------------------

// Initialise s if needed, give its kernels `nthreads` threads (one spectral mode per thread:
// nthreads >= M; the shared-memory layout is recomputed) and return the parameters of a
// launch of `nsteps` concurrent marches from its current s-step (march index c <-> s-step
// k + c, each waiting for the one before it).
gempic_status batch_prepare(gempic_sim* s, int nthreads, int nsteps, Params* out) {
  if (!s || !out || nsteps < 1) return GEMPIC_EINVAL;
  if (s->dn) return GEMPIC_EINVAL;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  if (nsteps > s->pmax) return GEMPIC_EINVAL;
  if (nthreads != s->p.nthreads) {
    if (nthreads < s->p.M || nthreads > 512 || nthreads % 32) return GEMPIC_EINVAL;
    Params t = s->p;
    t.nthreads = nthreads;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(s, e);
    if (smem_layout(t, s->eb) > optin) return GEMPIC_EINVAL;
    s->p = t;
  }
  cudaError_t e = ensure_diag_cap(s, nsteps);
  if (e != cudaSuccess) return cuda_fail(s, e);
  Params q = s->p;
  q.k0 = s->k;
  q.nsteps = nsteps;
  q.P = nsteps;
  q.inject = q.nspecies > 0 ? 1 : 0;
  q.delta_field = s->p.delta;
  *out = q;
  return GEMPIC_OK;
}

// After a batch launch of n s-steps of s.
void batch_advance(gempic_sim* s, int n) {
  s->last_launch_k0 = s->k;
  s->last_launch_n = n;
  s->k += n;
  s->launches++;
  s->denoised_last = false;
}

int batch_precision(const gempic_sim* s) { return s->cfg.precision; }

}  // namespace gempic

extern "C" {

const char* gempic_strerror(gempic_status s) {
  switch (s) {
    case GEMPIC_OK: return "ok";
    case GEMPIC_EINVAL: return "invalid argument or unsupported size";
    case GEMPIC_ENOMEM: return "out of memory";
    case GEMPIC_ECUDA: return "CUDA runtime error";
    case GEMPIC_EUNSTABLE: return "Delta h omega_p^2 > 4: outside the stability bound";
    case GEMPIC_ETIMEOUT: return "a bounded device wait gave up";
    case GEMPIC_ESTATE: return "simulation failed earlier or call not valid in this state";
    case GEMPIC_EOVERFLOW: return "a fixed-capacity particle store overflowed";
    case GEMPIC_ENONFINITE: return "a non-finite value appeared in the fields or particles";
  }
  return "unknown status";
}

gempic_status gempic_create(const gempic_config* cfg, gempic_sim** out) {
  if (!cfg || !out) return GEMPIC_EINVAL;
  *out = nullptr;
  const gempic_grid& g = cfg->grid;
  if (!pow2(g.nx) || g.nx < 8 || g.nx > 1024) return GEMPIC_EINVAL;
  if (!pow2(g.ny) || g.ny > 1024) return GEMPIC_EINVAL;
  if (g.nzeta < 2 || !(g.hx > 0) || !(g.hy > 0) || !(g.h > 0) || !(cfg->delta >= 0))
    return GEMPIC_EINVAL;
  if (cfg->precision != 32 && cfg->precision != 64) return GEMPIC_EINVAL;
  gempic::Params chk{};
  {
    const gempic_status st = gempic::setup_species(cfg, chk);
    if (st != GEMPIC_OK) return st;
  }
  if (cfg->laser && (!(cfg->laser->fwhm_intensity >= 0) || !std::isfinite(cfg->laser->fwhm_intensity)))
    return GEMPIC_EINVAL;
  // the bunch: validated here; it takes the slot of the species with its charge and mass, or
  // a slot of its own after the injected species
  int beam_slot = -1;
  if (cfg->beam) {
    const gempic_beam& b = *cfg->beam;
    const double v[8] = {b.charge, b.mass, b.n_peak, b.sigma_r, b.sigma_z, b.zeta_center,
                         b.gamma, b.rel_spread};
    for (double x : v)
      if (!std::isfinite(x)) return GEMPIC_EINVAL;
    if (!(b.mass > 0) || !(b.sigma_r > 0) || !(b.sigma_z > 0) || !(b.gamma >= 1) ||
        !(b.rel_spread >= 0) || b.n_macro < 0)
      return GEMPIC_EINVAL;
    for (int i = 0; i < cfg->nspecies && beam_slot < 0; ++i)
      if (cfg->species[i].charge == b.charge && cfg->species[i].mass == b.mass) beam_slot = i;
    if (beam_slot < 0) {
      if (cfg->nspecies >= gempic::kMaxSpecies) return GEMPIC_EINVAL;
      beam_slot = cfg->nspecies;
    }
  }

  gempic_sim* s = new (std::nothrow) gempic_sim();
  if (!s) return GEMPIC_ENOMEM;
  s->cfg = *cfg;
  for (int i = 0; i < cfg->nspecies; ++i) s->species[i] = cfg->species[i];
  s->cfg.species = nullptr;
  if (cfg->laser) {
    s->laser = *cfg->laser;
    s->has_laser = true;
    // intensity ~ exp(-2 phi^2/T^2): its full width at half maximum is T sqrt(2 ln 2)
    if (s->laser.fwhm_intensity > 0)
      s->laser.duration = s->laser.fwhm_intensity / std::sqrt(2.0 * std::log(2.0));
  }
  s->cfg.laser = nullptr;
  s->nspecies_all = cfg->nspecies;
  if (cfg->beam) {
    s->beam = *cfg->beam;
    s->has_beam = true;
    s->beam_species = beam_slot;
    s->nspecies_all = std::max(cfg->nspecies, beam_slot + 1);
  }
  s->cfg.beam = nullptr;
  if (cfg->channel) {
    s->channel = *cfg->channel;
    s->has_channel = true;
  }
  s->cfg.channel = nullptr;
  if (cfg->hz) {
    s->hz.assign(cfg->hz, cfg->hz + g.nzeta);
    s->zp.assign(g.nzeta + 1, 0.0);
    for (int n = 0; n < g.nzeta; ++n) s->zp[n + 1] = s->zp[n] + s->hz[n];
  }
  s->cfg.hz = nullptr;
  s->stream = (cudaStream_t)cfg->cuda_stream;
  s->eb = cfg->precision == 64 ? 8 : 4;

  Params& p = s->p;
  p.resid = (cfg->flags & GEMPIC_FLAG_RESIDUAL) ? 1 : 0;   // sizes shared memory
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
  (void)gempic::setup_species(cfg, p);            // validated at the top of this function
  if (s->has_beam && s->beam_species >= cfg->nspecies) {
    // a slot of the bunch's own: q/m and m/q for its push and energy; never injected
    const int b = s->beam_species;
    p.qm[b] = s->beam.charge / s->beam.mass;
    p.m_over_q[b] = s->beam.charge != 0 ? s->beam.mass / s->beam.charge : 0.0;
    p.Qf[b] = 0.0;
    p.wd[b] = 0.0;
    p.ppc[b] = 0;
    p.poff[b] = p.nlayer;
  }
  const int ppc_sum = p.ppc_sum;

  // launch shape: C CTAs per cluster own ny/C rows and (nx/2)/C kx columns; one spectral
  // mode per thread (M <= 512).
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int smem_optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    delete s;
    return GEMPIC_ECUDA;
  }
  const int nxh = g.nx / 2;
  int C = cfg->cluster_ctas;
  bool chosen = false;
  for (int cand = (C > 0 ? C : 1); cand <= (C > 0 ? C : 16); cand *= 2) {
    if (g.ny % cand || nxh % cand) continue;
    if (g.ny == 1 && cand != 1) continue;
    // 3-D bands need two rows or more (the current halo reaches two rows above the band)
    if (g.ny > 1 && g.ny / cand < 2) continue;
    const int RB = g.ny / cand, KB = nxh / cand, M = KB * g.ny;
    if (M > 512) continue;
    const int fresh = RB * g.nx * ppc_sum;
    int NT = std::max(M, fresh / 4);
    NT = std::min(512, std::max(128, (NT + 31) / 32 * 32));
    // streaming slots beyond the fresh layer hold stored particles that rejoin the march;
    // by default as many as the shared-memory budget allows, up to max(256, fresh)
    int head = cfg->particle_headroom > 0 ? cfg->particle_headroom : std::max(256, fresh);
    p.C = cand;
    p.RB = RB;
    p.KB = KB;
    p.logRB = ilog2(RB);
    p.logKB = ilog2(KB);
    p.M = M;
    p.nthreads = NT;
    for (;;) {
      p.pcap = fresh + head;
      if (gempic::smem_layout(p, s->eb) <= smem_optin) {
        chosen = true;
        break;
      }
      if (cfg->particle_headroom > 0 || head <= 32) break;
      head -= 32;
    }
    // many particles per cell: a fresh layer larger than the shared memory keeps as many
    // slots there as fit and continues in the overflow slots in global memory
    for (int pc = (fresh / 256) * 256; !chosen && cfg->particle_headroom <= 0 && pc >= 512;
         pc -= 256) {
      p.pcap = pc;
      if (gempic::smem_layout(p, s->eb) <= smem_optin) chosen = true;
    }
    if (chosen) break;
  }
  if (!chosen) {
    delete s;
    return GEMPIC_EINVAL;
  }
  p.bcap = cfg->stored_bucket_capacity > 0 ? cfg->stored_bucket_capacity
                                           : std::max(256, g.nx * g.ny * std::max(ppc_sum, 1) / 4);
  if (cfg->stored_bucket_capacity <= 0 && s->has_beam && s->beam.n_macro > 0) {
    // room for the bunch's densest slab: n_macro h_max/(sqrt(2 pi) sigma_z), with a margin
    const double hmax = s->hz.empty() ? g.h : *std::max_element(s->hz.begin(), s->hz.end());
    const double peak = (double)s->beam.n_macro * std::min(1.0, hmax / (2.5066282746310002 * s->beam.sigma_z));
    p.bcap += (int)std::min<double>((double)s->beam.n_macro, std::ceil(1.5 * peak) + 64.0);
  }
  p.wait_spin_limit = 20000000;
  p.diag = (cfg->flags & GEMPIC_FLAG_DIAG) ? 1 : 0;
  p.snapshot = (cfg->flags & GEMPIC_FLAG_SNAPSHOT) ? 1 : 0;
  p.gt1 = (cfg->flags & GEMPIC_FLAG_GT1) ? 1 : 0;

  e = gempic::configure_kernels(cfg->precision, p.smem_bytes, p.C);
  int maxcl = 1;
  if (e == cudaSuccess) e = gempic::max_active_clusters(cfg->precision, p, &maxcl);
  if (e != cudaSuccess) {
    delete s;
    return GEMPIC_ECUDA;
  }
  s->pmax = cfg->pipeline_depth > 0 ? cfg->pipeline_depth : std::max(1, std::min(maxcl, 16));
  if (s->pmax > std::max(1, maxcl)) s->pmax = std::max(1, maxcl);
  p.ring = s->pmax + 2;

  // device memory
  const size_t eb = s->eb;
  const size_t nperp = (size_t)g.nx * g.ny;
  const size_t ring = p.ring;
  const size_t bslots = ring * g.nzeta * (size_t)p.bcap;
#define ALLOC(ptr, bytes)                  \
  do {                                     \
    e = dalloc(s, &(ptr), (bytes));        \
    if (e != cudaSuccess) goto fail;       \
  } while (0)
  {
    ALLOC(p.state, (size_t)(g.nzeta + 1) * 6 * nxh * g.ny * 2 * eb);
    ALLOC(p.progress, (size_t)std::max(s->pmax, 1) * sizeof(unsigned long long));
    ALLOC(p.err, sizeof(int));
    void* tab = nullptr;
    const int nyh = g.ny > 1 ? g.ny / 2 : 1;
    const size_t ncx = nxh + nyh + nxh + g.ny, nr = nxh + g.ny;
    ALLOC(tab, (ncx * 2 + nr) * eb);
    p.tables = tab;
    if (!s->hz.empty()) {
      // variable zeta-step tables: slab thicknesses in the arithmetic type, plane positions
      void* hzt = nullptr;
      double* zpd = nullptr;
      ALLOC(hzt, (size_t)g.nzeta * eb);
      ALLOC(zpd, (size_t)(g.nzeta + 1) * sizeof(double));
      std::vector<unsigned char> hb((size_t)g.nzeta * eb);
      for (int n = 0; n < g.nzeta; ++n) {
        if (eb == 8) ((double*)hb.data())[n] = s->hz[n];
        else ((float*)hb.data())[n] = (float)s->hz[n];
      }
      e = cudaMemcpyAsync(hzt, hb.data(), hb.size(), cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(zpd, s->zp.data(), s->zp.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) goto fail;
      p.hzt = hzt;
      p.zpd = zpd;
      p.varh = 1;
    }
    // twiddles and shifts in FP64 on the host
    std::vector<double> t(ncx * 2 + nr);
    size_t o = 0;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < nxh; ++k, o += 2) { t[o] = std::cos(-2 * pi * k / g.nx); t[o + 1] = std::sin(-2 * pi * k / g.nx); }
    for (int k = 0; k < nyh; ++k, o += 2) {
      const double a = g.ny > 1 ? -2 * pi * k / g.ny : 0.0;
      t[o] = std::cos(a); t[o + 1] = std::sin(a);
    }
    std::vector<double> kx(nxh), ky(g.ny);
    for (int k = 0; k < nxh; ++k) kx[k] = 2 * pi * k / (g.nx * g.hx);
    for (int j = 0; j < g.ny; ++j) {
      // FFT order: j < ny/2 -> j, else j - ny (fftfreq)
      const int f = (g.ny == 1) ? 0 : (j < (g.ny + 1) / 2 ? j : j - g.ny);
      ky[j] = 2 * pi * (double)f / ((double)g.ny * g.hy);
    }
    for (int k = 0; k < nxh; ++k, o += 2) { t[o] = std::cos(-0.5 * kx[k] * g.hx); t[o + 1] = std::sin(-0.5 * kx[k] * g.hx); }
    for (int j = 0; j < g.ny; ++j, o += 2) { t[o] = std::cos(-0.5 * ky[j] * g.hy); t[o + 1] = std::sin(-0.5 * ky[j] * g.hy); }
    for (int k = 0; k < nxh; ++k) t[o++] = kx[k];
    for (int j = 0; j < g.ny; ++j) t[o++] = ky[j];
    if (eb == 8) {
      e = cudaMemcpyAsync(tab, t.data(), t.size() * 8, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    } else {
      std::vector<float> tf(t.begin(), t.end());
      e = cudaMemcpyAsync(tab, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    if (e != cudaSuccess) goto fail;
    gempic::PartStore* stores[2] = {&p.st, &p.rq};
    for (gempic::PartStore* S : stores) {
      ALLOC(S->cnt, ring * g.nzeta * sizeof(int));
      ALLOC(S->cell, bslots * sizeof(int));
      ALLOC(S->fx, bslots * eb);
      ALLOC(S->fy, bslots * eb);
      ALLOC(S->fz, bslots * eb);
      ALLOC(S->ux, bslots * eb);
      ALLOC(S->uy, bslots * eb);
      ALLOC(S->uz, bslots * eb);
      ALLOC(S->q, bslots * eb);
    }
    ALLOC(p.jbeam, ring * g.nzeta * 3 * nperp * eb);
    ALLOC(p.jflag, ring * g.nzeta * sizeof(int));
    // overflow particle slots: bands that gain particles (radial expulsion, rejoining stored
    // particles) spill beyond their shared-memory capacity into these
    p.gcap = std::max(1024, g.nx * (g.ny / p.C) * std::max(ppc_sum, 1) * 2);
    ALLOC(p.pover, (size_t)std::max(s->pmax, 1) * p.C * p.gcap * (4 + 7 * eb));
    if (p.snapshot) ALLOC(p.snap, (size_t)9 * g.nzeta * nperp * eb);
    if (cfg->flags & GEMPIC_FLAG_CURRENT) {
      ALLOC(s->jcap, (size_t)3 * g.nzeta * nperp * eb);
      p.jcap = s->jcap;
    }
#ifdef GEMPIC_PHASE_TIMERS
    ALLOC(p.timers, timer_words(p) * sizeof(unsigned long long));
#endif
  }
#undef ALLOC
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) goto fail;
  *out = s;
  return GEMPIC_OK;
fail:
  for (void* v : s->allocs) cudaFree(v);
  delete s;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
}

gempic_status gempic_add_particles(gempic_sim* s, int64_t n, const double* x, const double* y,
                                   const double* zeta, const double* ux, const double* uy,
                                   const double* uz, const double* weight, const int32_t* species) {
  if (!s) return GEMPIC_EINVAL;
  if (s->failed != GEMPIC_OK || s->initialized) return GEMPIC_ESTATE;
  if (n < 0 || (n > 0 && (!x || !zeta || !ux || !uy || !uz || !weight || !species)))
    return GEMPIC_EINVAL;
  if (s->p.ny > 1 && n > 0 && !y) return GEMPIC_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    if (species[i] < 0 || species[i] >= std::max(1, s->nspecies_all)) return GEMPIC_EINVAL;
    const double L = s->zp.empty() ? s->p.nz * s->p.h : s->zp.back();
    if (!(zeta[i] > 0) || !(zeta[i] <= L)) return GEMPIC_EINVAL;
  }
  for (int64_t i = 0; i < n; ++i) {
    s->px.push_back(x[i]);
    s->py.push_back(y ? y[i] : 0.0);
    s->pz.push_back(zeta[i]);
    s->pux.push_back(ux[i]);
    s->puy.push_back(uy[i]);
    s->puz.push_back(uz[i]);
    s->pq.push_back(weight[i]);
    s->psp.push_back(species[i]);
  }
  return GEMPIC_OK;
}

namespace {

cudaError_t io_event(gempic_sim* s, cudaEvent_t* ev) {
  if (!s->io_events.empty()) {
    *ev = s->io_events.back();
    s->io_events.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
}

struct IoPending {
  int step;          // s-step within the call whose input (H2D) or output (D2H) this is
  int group;
  cudaEvent_t ev;
};

}  // namespace

// Denoised s-steps as one chain of marches in one launch: march 2i is the first pass of s-step
// i (particles, plain deposit, its current kept), march 2i+1 the second (the level from the
// denoised current, the stored set); each march follows the one before it slice by slice as
// the wavefront does.  This thread runs the net on groups of half-slices as soon as the first
// pass has written them and the three half-slices the net reaches beyond them, and releases
// each group to the second pass, which waits for it (bounded) before it reads it.
static gempic_status denoised_chain(gempic_sim* s, int n) {
  const int nz = s->p.nz;
  const size_t nb = (size_t)3 * nz * s->p.ny * s->p.nx * s->eb;
  cudaError_t e = ensure_diag_cap(s, 2 * n);
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    if (!s->dn_jcap[r]) e = dalloc(s, &s->dn_jcap[r], nb);
    if (e == cudaSuccess && !s->dn_jden[r]) e = dalloc(s, &s->dn_jden[r], nb);
  }
  if (e == cudaSuccess && !s->dn_host) {
    void* h = nullptr;
    e = cudaHostAlloc(&h, 16 * sizeof(unsigned long long), cudaHostAllocMapped);
    if (e == cudaSuccess) {
      s->dn_host = (unsigned long long*)h;
      void* d = nullptr;
      e = cudaHostGetDevicePointer(&d, h, 0);
      s->dn_dev = (unsigned long long*)d;
    }
  }
  if (e == cudaSuccess && !s->dn_stream) e = cudaStreamCreateWithFlags(&s->dn_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(s, e);
  // nothing below may allocate or free device memory while the marches run: cudaFree waits
  // for the whole device, and the marches wait for the net
  int rs = gempic::denoise_reserve(s->dn, s->p.nx, s->p.ny, nz);
  if (rs != GEMPIC_OK) return (gempic_status)rs;
  for (int i = 0; i < 4 * nz / std::max(4, (nz + 15) / 16) + 8 && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;           // enough events for every group in flight
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) s->io_events.push_back(ev);
  }
  if (e != cudaSuccess) return cuda_fail(s, e);
  // groups of about a sixteenth of the window; a group needs the first pass three half-slices
  // beyond it (the net's reach along zeta)
  const int chunk = std::max(4, (nz + 15) / 16);
  const int nch = (nz + chunk - 1) / chunk;
  const int lead = 3 % chunk;
  // at most 7 marches in flight: the first pass of s-step i+4 reuses the current buffers of
  // s-step i only after it starts, i.e. after march 2i+8-P, the second pass of s-step i or later,
  // has finished with them.  The net runs on the SMs the marches leave free: unless the
  // configuration sets the depth, the marches take at most two thirds of them (on GB300 at
  // 128 x 128 x 512, 1 ppc, the chain's time per s-step against its depth was 11.5, 7.7, 6.8,
  // 5.5, 5.3 and 7.3 ms for 2 to 7 clusters of 16 CTAs: 6 leaves 56 SMs to the net).
  int dev = 0, nsm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(s, e);
  const int want = s->cfg.pipeline_depth > 0 ? s->cfg.pipeline_depth
                                             : std::max(1, 2 * nsm / (3 * s->p.C));
  const int P = std::min(std::min(std::min(s->pmax, 2 * n), 7), want);
  const long long k0 = s->k;
  unsigned long long* done = s->dn_host;
  unsigned long long* ready = s->dn_host + 8;
  std::memset(s->dn_host, 0, 16 * sizeof(unsigned long long));
  // progress words carry march indices here: start from zero
  e = cudaMemsetAsync(s->p.progress, 0, (size_t)s->pmax * sizeof(unsigned long long), s->stream);
  Params q = s->p;
  q.k0 = k0;
  q.nsteps = 2 * n;
  q.P = P;
  q.inject = q.nspecies > 0 ? 1 : 0;
  q.delta_field = s->p.delta;
  q.jcap = nullptr;
  q.jext = nullptr;
  q.state_out = nullptr;
  q.dn_pipe = 1;
  for (int r = 0; r < 4; ++r) {
    q.dn_jcap[r] = s->dn_jcap[r];
    q.dn_jext[r] = s->dn_jden[r];
  }
  q.dn_scratch = s->state2;
  q.dn_done = s->dn_dev;
  q.dn_ready = s->dn_dev + 8;
  q.dn_chunk = chunk;
  q.dn_nchunk = nch;
  q.dn_lead = lead;
  // the net's stream starts after everything before this launch
  cudaEvent_t start = nullptr;
  if (e == cudaSuccess) e = io_event(s, &start);
  if (e == cudaSuccess) e = cudaEventRecord(start, s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->dn_stream, start, 0);
  if (start) s->io_events.push_back(start);
  if (e == cudaSuccess) e = gempic::launch_march(s->cfg.precision, q, s->stream);
  s->launches++;
  if (e != cudaSuccess) return cuda_fail(s, e);
  std::vector<int> next(n, 0);
  std::deque<IoPending> netq;
  int released = 0;
  int st = GEMPIC_OK;
  auto last_move = std::chrono::steady_clock::now();
  while (released < n * nch && st == GEMPIC_OK && e == cudaSuccess) {
    bool moved = false;
    for (int i = 0; i < n && e == cudaSuccess && st == GEMPIC_OK; ++i) {
      if (next[i] >= nch) continue;
      const long long m1 = 2 * (k0 + i);                 // the first pass's march index
      const unsigned long long v = __atomic_load_n(done + (int)((2 * i) % P), __ATOMIC_ACQUIRE);
      while (next[i] < nch) {
        const int g = next[i];
        const int z1 = nz - g * chunk, z0 = std::max(0, z1 - chunk);
        if (v < gempic::prog_value(m1, nz, std::min(nz, nz - z0 + 3))) break;
        const int kr = (int)((k0 + i) & 3);
        st = gempic::denoise_range(s->dn, (const float*)s->dn_jcap[kr], (float*)s->dn_jden[kr],
                                   s->p.nx, s->p.ny, nz, z0, z1, s->dn_stream);
        s->launches += 4;
        if (st != GEMPIC_OK) break;
        IoPending pd{i, g, nullptr};
        e = io_event(s, &pd.ev);
        if (e == cudaSuccess) e = cudaEventRecord(pd.ev, s->dn_stream);
        if (e != cudaSuccess) break;
        netq.push_back(pd);
        ++next[i];
        moved = true;
      }
    }
    while (e == cudaSuccess && !netq.empty()) {
      const cudaError_t qe = cudaEventQuery(netq.front().ev);
      if (qe == cudaErrorNotReady) break;
      if (qe != cudaSuccess) {
        e = qe;
        break;
      }
      const IoPending pd = netq.front();
      netq.pop_front();
      const long long m2 = 2 * (k0 + pd.step) + 1;      // the second pass's march index
      __atomic_store_n(ready + (int)((k0 + pd.step) & 3), gempic::io_value(m2, nch, pd.group),
                       __ATOMIC_RELEASE);
      s->io_events.push_back(pd.ev);
      ++released;
      moved = true;
    }
    if (e != cudaSuccess || st != GEMPIC_OK) break;
    const auto now = std::chrono::steady_clock::now();
    if (moved) {
      last_move = now;
      continue;
    }
    const cudaError_t me = cudaStreamQuery(s->stream);
    if (me != cudaSuccess && me != cudaErrorNotReady) {
      e = me;
      break;
    }
    if (now - last_move > std::chrono::seconds(120)) {
      st = GEMPIC_ETIMEOUT;
      break;
    }
    std::this_thread::yield();
  }
  const cudaError_t e2 = cudaStreamSynchronize(s->stream);
  const cudaError_t e3 = cudaStreamSynchronize(s->dn_stream);
  for (const IoPending& pd : netq) s->io_events.push_back(pd.ev);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
  // leave the progress words as a plain launch expects them (below any s-step's value)
  if (e == cudaSuccess)
    e = cudaMemsetAsync(s->p.progress, 0, (size_t)s->pmax * sizeof(unsigned long long), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  s->last_launch_k0 = k0;
  s->last_launch_n = 2 * n;
  s->denoised_last = true;
  s->jcap_last = s->dn_jcap[(k0 + n - 1) & 3];
  s->k += n;
  if (st != GEMPIC_OK) {
    s->failed = (gempic_status)st;
    return (gempic_status)st;
  }
  st = gempic::denoise_status(s->dn, s->stream);
  if (st != GEMPIC_OK) s->failed = (gempic_status)st;
  return (gempic_status)st;
}

gempic_status gempic_step_async(gempic_sim* s, int32_t n) {
  if (!s || n < 0) return GEMPIC_EINVAL;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  if (n == 0) return GEMPIC_OK;
  if (s->dn) return denoised_chain(s, n);
  s->denoised_last = false;
  cudaError_t e = ensure_diag_cap(s, n);
  if (e != cudaSuccess) return cuda_fail(s, e);
  Params q = s->p;
  q.k0 = s->k;
  q.nsteps = n;
  q.P = std::min(s->pmax, n);
  q.inject = q.nspecies > 0 ? 1 : 0;
  q.delta_field = s->p.delta;
  e = gempic::launch_march(s->cfg.precision, q, s->stream);
  s->launches++;
  if (e != cudaSuccess) return cuda_fail(s, e);
  s->last_launch_k0 = s->k;
  s->last_launch_n = n;
  s->k += n;
  return GEMPIC_OK;
}

gempic_status gempic_set_delta(gempic_sim* s, double delta) {
  if (!s) return GEMPIC_EINVAL;
  if (!(delta >= 0) || !std::isfinite(delta)) return GEMPIC_EINVAL;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  gempic_config c = s->cfg;
  c.delta = delta;
  c.species = s->species;
  c.channel = s->has_channel ? &s->channel : nullptr;
  c.hz = s->hz.empty() ? nullptr : s->hz.data();
  Params t = s->p;
  st = gempic::setup_species(&c, t);
  if (st != GEMPIC_OK) return st;
  s->cfg.delta = delta;
  s->p = t;
  s->p.delta = delta;
  s->p.delta_field = delta;
  return GEMPIC_OK;
}

gempic_status gempic_set_wait_limit(gempic_sim* s, int64_t polls) {
  if (!s || polls < 0) return GEMPIC_EINVAL;
  if (s->failed != GEMPIC_OK) return GEMPIC_ESTATE;
  s->p.wait_spin_limit = (int)std::min<int64_t>(polls, 2000000000);
  return GEMPIC_OK;
}

gempic_status gempic_sync(gempic_sim* s) {
  if (!s) return GEMPIC_EINVAL;
  if (s->failed != GEMPIC_OK) return GEMPIC_ESTATE;
  return check_device_error(s);
}

gempic_status gempic_step(gempic_sim* s, int32_t n) {
  gempic_status st = gempic_step_async(s, n);
  if (st != GEMPIC_OK) return st;
  return gempic_sync(s);
}

size_t gempic_state_bytes(const gempic_sim* s) {
  if (!s) return 0;
  return (size_t)6 * s->p.nz * s->p.ny * (s->p.nx / 2) * 2 * s->eb;
}

static gempic_status copy_state(gempic_sim* s, void* ptr, size_t bytes, int is_device, bool out) {
  if (!s || !ptr) return GEMPIC_EINVAL;
  if (bytes < gempic_state_bytes(s)) return GEMPIC_EINVAL;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  const size_t nb = gempic_state_bytes(s);
  void* dev = ptr;
  cudaError_t e = cudaSuccess;
  if (!is_device) {
    // one staging buffer per simulation, kept for its lifetime: a host copy every s-step
    // (the end-to-end path) then costs no allocation
    if (!s->stage) {
      e = cudaMalloc(&s->stage, nb);
      if (e != cudaSuccess) {
        s->stage = nullptr;
        return cuda_fail(s, e);
      }
      s->allocs.push_back(s->stage);
    }
    dev = s->stage;
    if (!out) e = cudaMemcpyAsync(dev, ptr, nb, cudaMemcpyHostToDevice, s->stream);
  }
  if (e == cudaSuccess)
    e = out ? gempic::launch_export_state(s->cfg.precision, s->p, dev, s->stream)
            : gempic::launch_import_state(s->cfg.precision, s->p, dev, s->stream);
  s->launches++;
  if (e == cudaSuccess && !is_device && out)
    e = cudaMemcpyAsync(ptr, dev, nb, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_fail(s, e);
}

gempic_status gempic_get_state(gempic_sim* s, void* dst, size_t bytes, int32_t dst_is_device) {
  return copy_state(s, dst, bytes, dst_is_device, true);
}

gempic_status gempic_set_state(gempic_sim* s, const void* src, size_t bytes, int32_t src_is_device) {
  return copy_state(s, const_cast<void*>(src), bytes, src_is_device, false);
}

gempic_status gempic_step_host(gempic_sim* s, int32_t n, const void* state_in, void* state_out,
                               size_t state_bytes, gempic_diag* diag_out) {
  if (!s) return GEMPIC_EINVAL;
  gempic_status st = GEMPIC_OK;
  if (state_in) st = gempic_set_state(s, state_in, state_bytes, 0);
  if (st == GEMPIC_OK) st = gempic_step(s, n);
  if (st == GEMPIC_OK && state_out) st = gempic_get_state(s, state_out, state_bytes, 0);
  if (st == GEMPIC_OK && diag_out) st = gempic_get_diagnostics(s, diag_out);
  return st;
}

// the FP64 diagnostic sums of march `sl` of the last launch: the per-CTA partials added
static cudaError_t diag_sums(gempic_sim* s, int sl, double* v) {
  const Params& p = s->p;
  std::vector<double> d((size_t)gempic::kNDiag * p.C);
  cudaError_t e = cudaMemcpyAsync(d.data(), p.diag_out + (size_t)sl * gempic::kNDiag * p.C,
                                  d.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < gempic::kNDiag; ++i) {
    v[i] = 0.0;
    for (int r = 0; r < p.C; ++r) v[i] += d[(size_t)i * p.C + r];
  }
  return cudaSuccess;
}

static gempic_status diag_record(gempic_sim* s, int sl, long long step, const double* v,
                                 gempic_diag* out) {
  const Params& p = s->p;
  out->step = step;
  out->field_energy = v[gempic::DG_FIELD];
  out->kinetic_energy = v[gempic::DG_KIN];
  out->charge_flux = v[gempic::DG_FLUX];
  out->n_trapped = (int64_t)std::llround(v[gempic::DG_TRAP]);
  out->n_stored = (int64_t)std::llround(v[gempic::DG_STORED]);
  out->n_rejoined = (int64_t)std::llround(v[gempic::DG_REJOIN]);
  out->pushes = (int64_t)std::llround(v[gempic::DG_PUSH]);
  out->stored_kinetic_energy = v[gempic::DG_KST];
  out->continuity_residual = -1.0;
  out->gauss_residual = -1.0;
  if (p.resid) {
    cudaError_t e = cudaMemcpyAsync(&out->continuity_residual, p.resid_out + sl, sizeof(double),
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&out->gauss_residual, p.gauss_out + sl, sizeof(double),
                          cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  return GEMPIC_OK;
}

// ------------------------------------------------------------------------------------------
// s-steps with the state streamed through host memory
// ------------------------------------------------------------------------------------------
namespace {

cudaError_t ensure_stream_io(gempic_sim* s) {
  const size_t nb = gempic_state_bytes(s);
  cudaError_t e = cudaSuccess;
  if (!s->io_a) e = dalloc(s, &s->io_a, nb);
  if (e == cudaSuccess && !s->io_b) e = dalloc(s, &s->io_b, nb);
  if (e == cudaSuccess && !s->io_host) {
    // [ready: pmax + 1][done: pmax]
    const size_t words = 2 * (size_t)s->pmax + 1;
    void* h = nullptr;
    e = cudaHostAlloc(&h, words * sizeof(unsigned long long), cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    std::memset(h, 0, words * sizeof(unsigned long long));
    s->io_host = (unsigned long long*)h;
    void* d = nullptr;
    e = cudaHostGetDevicePointer(&d, h, 0);
    s->io_dev = (unsigned long long*)d;
  }
  if (e == cudaSuccess && !s->io_out) e = cudaStreamCreateWithFlags(&s->io_out, cudaStreamNonBlocking);
  if (e == cudaSuccess && !s->io_in) e = cudaStreamCreateWithFlags(&s->io_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !s->io_fill) e = cudaStreamCreateWithFlags(&s->io_fill, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = gempic::configure_march_canon(s->cfg.precision, s->p.smem_bytes);
  return e;
}

// Copy group j of the public layout [6][nz][ny][nx/2] between the host buffer and a device
// level: blocks [lo, hi) are R_x, R_y, E_z, B_z at slices lo .. hi-1 (below nz) and j_x, j_y at
// half-slices lo-1 .. hi-2 (from 0); one contiguous copy per component (measured faster than
// strided two-dimensional copies of the same bytes).
cudaError_t io_copy(gempic_sim* s, int j, int chunk, void* dev, void* host, bool out,
                    cudaStream_t st) {
  const int nz = s->p.nz;
  const size_t sb = (size_t)s->p.ny * (s->p.nx / 2) * 2 * s->eb;    // one slice of one component
  const size_t cb = (size_t)nz * sb;                                 // one component
  const int hi = nz + 1 - j * chunk, lo = std::max(0, hi - chunk);
  char* d = (char*)dev;
  char* h = (char*)host;
  const cudaMemcpyKind kind = out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < 6 && e == cudaSuccess; ++c) {
    const int s0 = c < 4 ? lo : std::max(lo, 1) - 1;                // fields / currents
    const int s1 = c < 4 ? std::min(hi, nz) : hi - 1;
    if (s1 <= s0) continue;
    const size_t off = (size_t)c * cb + (size_t)s0 * sb, w = (size_t)(s1 - s0) * sb;
    e = out ? cudaMemcpyAsync(h + off, d + off, w, kind, st) : cudaMemcpyAsync(d + off, h + off, w, kind, st);
  }
  return e;
}

}  // namespace

gempic_status gempic_step_streamed(gempic_sim* s, int32_t n, void* host, size_t bytes,
                                   gempic_diag* diag_out) {
  if (!s || n < 0 || !host) return GEMPIC_EINVAL;
  if (bytes < gempic_state_bytes(s)) return GEMPIC_EINVAL;
  if (s->dn) return GEMPIC_ESTATE;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  if (n == 0) return GEMPIC_OK;
  cudaError_t e = ensure_stream_io(s);
  if (e == cudaSuccess) e = ensure_diag_cap(s, n);
  if (e != cudaSuccess) return cuda_fail(s, e);
  const int nz = s->p.nz;
  // groups of at most 8 MiB and at least 8 groups a level (so that the next s-step follows
  // closely), each of at least 2 blocks (a march starts on blocks nz and nz-1)
  const size_t block_bytes = (size_t)6 * s->p.ny * (s->p.nx / 2) * 2 * s->eb;
  const size_t by_bytes = std::max<size_t>(1, ((size_t)8 << 20) / block_bytes);
  const int chunk = (int)std::max<size_t>(2, std::min<size_t>(by_bytes, (size_t)(nz + 8) / 8));
  const int nch = (nz + 1 + chunk - 1) / chunk;
  Params q = s->p;
  q.k0 = s->k;
  q.nsteps = n;
  q.P = std::min(s->pmax, n);
  q.inject = q.nspecies > 0 ? 1 : 0;
  q.delta_field = s->p.delta;
  q.state = s->io_a;
  q.state_out = s->io_b;
  q.io_ready = s->io_dev;
  q.io_done = s->io_dev + s->pmax + 1;
  q.io_chunk = chunk;
  q.io_nchunk = nch;
  q.io_ring = s->pmax + 1;
  unsigned long long* ready = s->io_host;
  const unsigned long long* done = s->io_host + s->pmax + 1;
  const long long k0 = s->k;
  auto slot = [&](int i) { return i % q.P; };
  // the first s-step's input goes in before the launch's marches reach it, on a stream of
  // its own, so that the second s-step's input copies do not queue behind it
  std::deque<IoPending> outq, inq;
  for (int j = 0; j < nch && e == cudaSuccess; ++j) {
    IoPending pd{0, j, nullptr};
    e = io_event(s, &pd.ev);
    if (e == cudaSuccess) e = io_copy(s, j, chunk, s->io_a, host, false, s->io_fill);
    if (e == cudaSuccess) e = cudaEventRecord(pd.ev, s->io_fill);
    if (e == cudaSuccess) inq.push_back(pd);
  }
  if (e == cudaSuccess) e = gempic::launch_march_canon(s->cfg.precision, q, s->stream);
  s->launches++;
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s->io_fill);
    for (const IoPending& pd : inq) s->io_events.push_back(pd.ev);
    return cuda_fail(s, e);
  }
  // Drive the copies: a group of s-step i's result goes out once its march has written it,
  // back in as s-step i+1's input once it is out, and is released to that march once it is
  // in.  Each link waits for the one before it, so the host buffer and both device levels are
  // only rewritten after their last reader is done.
  std::vector<int> next_out(n, 0), blocked;
  int first = 0, outs_done = 0;
  gempic_status result = GEMPIC_OK;
  auto last_move = std::chrono::steady_clock::now();
  while (outs_done < n * nch || !inq.empty()) {
    bool moved = false;
    for (int i = first; i < n && e == cudaSuccess; ++i) {
      if (next_out[i] >= nch) {
        if (i == first) ++first;
        continue;
      }
      const unsigned long long v = __atomic_load_n(done + slot(i), __ATOMIC_ACQUIRE);
      while (next_out[i] < nch && e == cudaSuccess) {
        const int j = next_out[i];
        const int lo = std::max(0, nz + 1 - (j + 1) * chunk);
        const unsigned long long need = gempic::prog_value(k0 + i, nz, std::min(nz, nz - lo + 1));
        if (v < need) break;
        IoPending pd{i, j, nullptr};
        e = io_event(s, &pd.ev);
        if (e == cudaSuccess) e = io_copy(s, j, chunk, s->io_b, host, true, s->io_out);
        if (e == cudaSuccess) e = cudaEventRecord(pd.ev, s->io_out);
        if (e == cudaSuccess) outq.push_back(pd);
        ++next_out[i];
        moved = true;
      }
    }
    while (e == cudaSuccess && !outq.empty()) {
      const cudaError_t qe = cudaEventQuery(outq.front().ev);
      if (qe == cudaErrorNotReady) break;
      if (qe != cudaSuccess) {
        e = qe;
        break;
      }
      IoPending pd = outq.front();
      outq.pop_front();
      ++outs_done;
      moved = true;
      if (pd.step + 1 < n) {
        IoPending nx{pd.step + 1, pd.group, pd.ev};
        e = io_copy(s, pd.group, chunk, s->io_a, host, false, s->io_in);
        if (e == cudaSuccess) e = cudaEventRecord(nx.ev, s->io_in);
        if (e == cudaSuccess) inq.push_back(nx);
      } else {
        s->io_events.push_back(pd.ev);
      }
    }
    // an s-step's groups are released in order (one word per s-step); the first s-step's
    // copies run on their own stream, so the next s-step's may finish before them
    blocked.clear();
    for (size_t qi = 0; e == cudaSuccess && qi < inq.size();) {
      const IoPending pd = inq[qi];
      if (std::find(blocked.begin(), blocked.end(), pd.step) != blocked.end()) {
        ++qi;
        continue;
      }
      const cudaError_t qe = cudaEventQuery(pd.ev);
      if (qe == cudaErrorNotReady) {
        blocked.push_back(pd.step);
        ++qi;
        continue;
      }
      if (qe != cudaSuccess) {
        e = qe;
        break;
      }
      inq.erase(inq.begin() + (std::ptrdiff_t)qi);
      __atomic_store_n(ready + (k0 + pd.step) % q.io_ring,
                       gempic::io_value(k0 + pd.step, nch, pd.group), __ATOMIC_RELEASE);
      s->io_events.push_back(pd.ev);
      moved = true;
    }
    if (e != cudaSuccess) break;
    const auto now = std::chrono::steady_clock::now();
    if (moved) {
      last_move = now;
      continue;
    }
    // a launch that failed publishes nothing more
    const cudaError_t me = cudaStreamQuery(s->stream);
    if (me != cudaSuccess && me != cudaErrorNotReady) {
      e = me;
      break;
    }
    if (now - last_move > std::chrono::seconds(120)) {
      result = GEMPIC_ETIMEOUT;
      break;
    }
    std::this_thread::yield();
  }
  // the marches always finish (their waits are bounded); then the copies
  cudaError_t e2 = cudaStreamSynchronize(s->stream);
  cudaError_t e3 = cudaStreamSynchronize(s->io_out);
  cudaError_t e4 = cudaStreamSynchronize(s->io_in);
  if (e4 == cudaSuccess) e4 = cudaStreamSynchronize(s->io_fill);
  for (const IoPending& pd : outq) s->io_events.push_back(pd.ev);
  for (const IoPending& pd : inq) s->io_events.push_back(pd.ev);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4;
  if (e != cudaSuccess) return cuda_fail(s, e);
  s->last_launch_k0 = s->k;
  s->last_launch_n = n;
  s->denoised_last = false;
  s->k += n;
  if (result != GEMPIC_OK) {
    s->failed = result;
    return result;
  }
  st = check_device_error(s);
  if (st != GEMPIC_OK) return st;
  // the last result becomes the simulation's state
  e = gempic::launch_import_state(s->cfg.precision, s->p, s->io_b, s->stream);
  s->launches++;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (diag_out) {
    for (int i = 0; i < n; ++i) {
      double v[gempic::kNDiag];
      e = diag_sums(s, i, v);
      if (e != cudaSuccess) return cuda_fail(s, e);
      st = diag_record(s, i, k0 + i + 1, v, diag_out + i);
      if (st != GEMPIC_OK) return st;
    }
  }
  return GEMPIC_OK;
}

gempic_status gempic_get_fields(gempic_sim* s, int32_t comp, void* dst, size_t bytes,
                                int32_t dst_is_device) {
  if (!s || !dst || comp < 0 || comp > 8) return GEMPIC_EINVAL;
  if (!s->p.snapshot || s->k == 0) return GEMPIC_ESTATE;
  const size_t nb = (size_t)s->p.nz * s->p.ny * s->p.nx * s->eb;
  if (bytes < nb) return GEMPIC_EINVAL;
  if (s->failed != GEMPIC_OK) return GEMPIC_ESTATE;
  cudaError_t e = cudaMemcpyAsync(dst, (const char*)s->p.snap + (size_t)comp * nb, nb,
                                  dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_fail(s, e);
}

gempic_status gempic_get_particles(gempic_sim* s, int32_t kind, int64_t* n_inout, double* x,
                                   double* y, double* zeta, double* ux, double* uy, double* uz,
                                   double* weight, int32_t* species) {
  if (!s || !n_inout || (kind != 0 && kind != 1)) return GEMPIC_EINVAL;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  const Params& p = s->p;
  const gempic::PartStore& S = kind == 0 ? p.st : p.rq;
  const int slot = (int)((s->k + 1) % p.ring);
  const size_t cap = (size_t)p.nz * p.bcap;
  const size_t base = (size_t)slot * cap;
  std::vector<int> cnt(p.nz), cell(cap);
  std::vector<char> raw[7];
  void* src[7] = {S.fx, S.fy, S.fz, S.ux, S.uy, S.uz, S.q};
  cudaError_t e = cudaMemcpyAsync(cnt.data(), S.cnt + (size_t)slot * p.nz, p.nz * sizeof(int),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cell.data(), S.cell + base, cap * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  for (int j = 0; j < 7 && e == cudaSuccess; ++j) {
    raw[j].resize(cap * s->eb);
    e = cudaMemcpyAsync(raw[j].data(), (const char*)src[j] + base * s->eb, cap * s->eb,
                        cudaMemcpyDeviceToHost, s->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  int64_t total = 0;
  for (int b = 0; b < p.nz; ++b) total += std::min(cnt[b], p.bcap);
  if (total > *n_inout) {
    *n_inout = total;
    return GEMPIC_EINVAL;
  }
  auto val = [&](int j, size_t i) -> double {
    return s->eb == 8 ? ((const double*)raw[j].data())[i] : (double)((const float*)raw[j].data())[i];
  };
  int64_t o = 0;
  for (int b = 0; b < p.nz; ++b) {
    for (int i = 0; i < std::min(cnt[b], p.bcap); ++i, ++o) {
      const size_t e2 = (size_t)b * p.bcap + i;
      const int c = cell[e2];
      const int ix = c & 1023, iy = (c >> 10) & 1023, sp = (c >> 20) & 3;
      if (x) x[o] = (ix + val(0, e2)) * p.hx;
      if (y) y[o] = p.ny > 1 ? (iy + val(1, e2)) * p.hy : 0.0;
      if (zeta) zeta[o] = s->zp.empty() ? (b + val(2, e2)) * p.h : s->zp[b] + val(2, e2) * s->hz[b];
      if (ux) ux[o] = val(3, e2);
      if (uy) uy[o] = val(4, e2);
      if (uz) uz[o] = val(5, e2);
      if (weight) weight[o] = val(6, e2);
      if (species) species[o] = sp;
    }
  }
  *n_inout = total;
  return GEMPIC_OK;
}

gempic_status gempic_get_diagnostics(gempic_sim* s, gempic_diag* out) {
  if (!s || !out) return GEMPIC_EINVAL;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  st = check_device_error(s);
  if (st != GEMPIC_OK) return st;
  const int sl = s->last_launch_n - 1;
  double v[gempic::kNDiag];
  // a denoised s-step: march sl - 1 is its first pass, sl its second
  cudaError_t e = diag_sums(s, s->denoised_last ? sl - 1 : sl, v);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (s->denoised_last) {
    // the second pass holds the fields and the stored set; the first the streaming particles
    double v2[gempic::kNDiag];
    e = diag_sums(s, sl, v2);
    if (e != cudaSuccess) return cuda_fail(s, e);
    v[gempic::DG_FIELD] = v2[gempic::DG_FIELD];
    v[gempic::DG_KIN] += v2[gempic::DG_KIN];
    v[gempic::DG_KST] = v2[gempic::DG_KST];
    v[gempic::DG_STORED] = v2[gempic::DG_STORED];
    v[gempic::DG_LOST] = v2[gempic::DG_LOST];
  }
  return diag_record(s, sl, s->k, v, out);
}

gempic_status gempic_get_onaxis_ez(gempic_sim* s, double* dst, int32_t n) {
  if (!s || !dst || n < s->p.nz) return GEMPIC_EINVAL;
  gempic_status st = ensure_initialized(s);
  if (st != GEMPIC_OK) return st;
  const int sl = s->last_launch_n - 1;                 // a denoised s-step's second pass
  cudaError_t e = cudaMemcpyAsync(dst, s->p.onaxis + (size_t)sl * s->p.nz, s->p.nz * sizeof(double),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_fail(s, e);
}

int64_t gempic_launch_count(const gempic_sim* s) { return s ? s->launches : 0; }

gempic_status gempic_set_denoiser(gempic_sim* s, gempic_denoiser* d) {
  if (!s) return GEMPIC_EINVAL;
  if (s->failed != GEMPIC_OK) return GEMPIC_ESTATE;
  if (d && s->cfg.precision != 32) return GEMPIC_EINVAL;
  if (d) {
    const size_t nb = (size_t)3 * s->p.nz * s->p.ny * s->p.nx * s->eb;
    const size_t sb = (size_t)(s->p.nz + 1) * 6 * (s->p.nx / 2) * s->p.ny * 2 * s->eb;
    cudaError_t e = cudaSuccess;
    (void)nb;
    if (!s->state2) e = dalloc(s, &s->state2, sb);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
    }
  }
  s->dn = d;
  return GEMPIC_OK;
}

gempic_status gempic_get_current(gempic_sim* s, void* dst, size_t bytes, int32_t dst_is_device) {
  if (!s || !dst) return GEMPIC_EINVAL;
  const void* src = s->denoised_last ? s->jcap_last : s->jcap;
  if (!src || s->k == 0) return GEMPIC_ESTATE;
  if (s->failed != GEMPIC_OK) return GEMPIC_ESTATE;
  const size_t nb = (size_t)3 * s->p.nz * s->p.ny * s->p.nx * s->eb;
  if (bytes < nb) return GEMPIC_EINVAL;
  cudaError_t e = cudaMemcpyAsync(dst, src, nb,
                                  dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_fail(s, e);
}

#ifdef GEMPIC_PHASE_TIMERS
// profiling builds only: the raw device error word
int gempic_debug_error_word(gempic_sim* s) {
  int err = -1;
  if (cudaMemcpy(&err, s->p.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -2;
  return err;
}
// profiling builds only: accumulated clock64 cycles per march phase (thread 0 of each CTA)
gempic_status gempic_phase_timers(gempic_sim* s, unsigned long long* out, int32_t n) {
  if (!s || !out || n < 1) return GEMPIC_EINVAL;
  const int tw = timer_words(s->p);
  cudaError_t e = cudaMemcpyAsync(out, s->p.timers, std::min(n, tw) * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->p.timers, 0, tw * sizeof(unsigned long long), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_fail(s, e);
}
#endif

gempic_status gempic_launch_shape(const gempic_sim* s, int32_t* cluster_ctas, int32_t* threads,
                                  int32_t* smem_bytes, int32_t* pipeline) {
  if (!s) return GEMPIC_EINVAL;
  if (cluster_ctas) *cluster_ctas = s->p.C;
  if (threads) *threads = s->p.nthreads;
  if (smem_bytes) *smem_bytes = s->p.smem_bytes;
  if (pipeline) *pipeline = s->pmax;
  return GEMPIC_OK;
}

void gempic_destroy(gempic_sim* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  if (s->io_out) cudaStreamSynchronize(s->io_out);
  if (s->io_in) cudaStreamSynchronize(s->io_in);
  if (s->io_fill) cudaStreamSynchronize(s->io_fill);
  for (cudaEvent_t ev : s->io_events) cudaEventDestroy(ev);
  if (s->io_out) cudaStreamDestroy(s->io_out);
  if (s->io_in) cudaStreamDestroy(s->io_in);
  if (s->io_fill) cudaStreamDestroy(s->io_fill);
  if (s->io_host) cudaFreeHost(s->io_host);
  if (s->dn_stream) {
    cudaStreamSynchronize(s->dn_stream);
    cudaStreamDestroy(s->dn_stream);
  }
  if (s->dn_host) cudaFreeHost(s->dn_host);
  for (void* v : s->allocs) cudaFree(v);
  cudaGetLastError();
  delete s;
}

}  // extern "C"
