// Internal interface between the host API (gempic_api.cu) and the device kernels
// (gempic_kernels.cu).  Not part of the public C-ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gempic {

constexpr int kMaxSpecies = 4;
constexpr int kNDiag = 9;        // per-CTA FP64 diagnostic partials per s-step
enum DiagSlot { DG_FIELD = 0, DG_KIN, DG_FLUX, DG_TRAP, DG_STORED, DG_REJOIN, DG_PUSH, DG_LOST,
                DG_KST };         // DG_KST: the stored set's part of DG_KIN

// Device error word bits.
enum ErrBits : int {
  ERR_TIMEOUT = 1,       // a bounded wait on another march gave up
  ERR_PCAP = 2,          // streaming particle capacity of a CTA exceeded
  ERR_BCAP = 4,          // stored bucket capacity exceeded
  ERR_QCAP = 8,          // rejoin queue capacity exceeded
  ERR_NONFINITE = 16     // a field or kinetic-energy sum was not finite, or a particle moved
                         // more than the sub-step cap across one slice (runaway momentum)
};

// Stored-particle store: ring of s-levels x nzeta buckets x capacity, structure of arrays.
// The cell word packs ix | iy << 10 | species << 20; fx, fy in [0,1) are transverse in-cell
// offsets and fz in (0,1] the in-cell zeta offset: zeta = (bucket + fz) h.
struct PartStore {
  int* cnt;          // [ring][nzeta]
  int* cell;         // [ring][nzeta][cap]
  void* fx; void* fy; void* fz;
  void* ux; void* uy; void* uz; void* q;
};

struct Params {
  // grid and decomposition
  int nx, ny, nz;                 // transverse nodes, slices
  int C, RB, KB, M;               // CTAs per cluster, rows per CTA, kx per CTA, modes per CTA
  int FR, JR, JOFF;               // field rows per CTA (own + halo above), current rows (own +
                                  // halo below/above), row offset of own row 0 in the currents
  int lognx, logny, logRB, logKB;
  int nthreads;
  // physics
  double hx, hy, h, delta, delta_field;
  double jref;                    // FP32 deposit: contributions below jref add in 32-bit fixed
                                  // point with resolution jref / 2^22 (exact integer sums)
  int nspecies, nlayer, ppc_sum;
  double qm[kMaxSpecies];         // q/m
  double wd[kMaxSpecies];         // (rho - j_z) weight Q_f/(hx hy Delta) of a fresh particle
  double Qf[kMaxSpecies];         // fresh macroparticle charge q n hx hy Delta/ppc
  double m_over_q[kMaxSpecies];   // m/q: kinetic energy of N = Q/q particles is Q (m/q)(gamma-1)
  int ppc[kMaxSpecies], poff[kMaxSpecies];
  double chan_a, chan_ir2;        // density channel f(r) = 1 + chan_a exp(-r^2 chan_ir2)
                                  // (Eq. n_plasma); chan_a = 0: uniform
  unsigned long long seed;
  // launch
  long long k0;                   // s-step index of the first march of this launch (-1: init)
  int nsteps;                     // marches in this launch
  int P;                          // concurrent marches (clusters)
  int inject, diag, snapshot;
  int gt1;                        // particle law: 0 = GT2 (Eq. trap2), 1 = GT1 (Eq. trap1)
  int varh;                       // 1: slab thicknesses from hzt (variable zeta-step)
  int resid;                      // 1: continuity and Gauss residuals (verification mode)
  double* resid_out;              // [nsteps] continuity residual maximum per s-step
  double* gauss_out;              // [nsteps] Gauss residual maximum per s-step
  double bg_qn;                   // neutralising background -sum_s q_s n_s (immobile ions)
  const void* hzt;                // [nz] slab thickness h_n (slab n: planes n, n+1), real type
  const double* zpd;              // [nz+1] plane positions zeta_n (plane 0 at the back)
  int pcap;                       // streaming particle slots per CTA in shared memory
  int fcap;                       // entries of the free-slot stack (slots freed and not yet
                                  // reused; further freed slots stay empty this s-step)
  int gcap;                       // further slots per CTA in global memory (overflow)
  int bcap, ring;                 // stored bucket capacity, ring of s-levels
  int wait_spin_limit;            // bounded wait: polls before giving up
  int nwork;                      // FFT work rows per CTA
  int mig_cap;                    // migrating particles a CTA can receive per slice
  // shared-memory layout (byte offsets)
  int o_f0, o_f1, o_j, o_recv, o_sr, o_sc, o_workB, o_workD, o_tw, o_inbox, o_outbox, o_part, o_misc, o_dd,
      smem_bytes;
  // device memory
  void* state;                    // blocks [nz+1][C][6][M] complex
  unsigned long long* progress;   // [P] completed-iteration counters
  int* err;
  const void* tables;             // twx[nx/2], twy[ny/2], shx[nx/2], shy[ny], kx[nx/2], ky[ny]
  PartStore st;                   // stored particles (trapped / beam)
  PartStore rq;                   // rejoin queues
  void* jbeam;                    // [ring][nz][3][ny][nx]
  int* jflag;                     // [ring][nz]
  double* diag_out;               // [nsteps][kNDiag][C]
  double* onaxis;                 // [nsteps][nz]
  void* snap;                     // [9][nz][ny][nx]
  // denoised s-step (two passes): the first marches the particles with the plain deposit,
  // captures its current (jcap) and writes its provisional level to state_out, leaving the
  // stored set for the second (skip_stored); the second takes the denoised current (jext) on
  // the unchanged old level, with no fresh or rejoining particles (fields_only), and pushes
  // the stored set with the final fields
  void* jcap;                     // [nz][3][ny][nx] current of the last march of the launch
  const void* jext;               // [nz][3][ny][nx] current replacing the deposit
  void* state_out;                // new level written here instead of over the old one
  int skip_stored, fields_only;
  void* pover;                    // overflow particle slots [P*C][int cell; 7 reals][gcap]
  unsigned long long* timers;     // phase timers (builds with GEMPIC_PHASE_TIMERS only)
  // state streamed through host memory (gempic_step_streamed): the old level is read from
  // `state`, the new one written to `state_out`, both in the public layout; the blocks go out
  // and back in groups of io_chunk (group j: blocks nz - j io_chunk down to
  // nz + 1 - (j+1) io_chunk).  Words in host-mapped memory:
  unsigned long long* io_ready;   // [io_ring], written by the host: word k % io_ring holds
                                  // io_value(k, io_nchunk, j) once group j of s-step k's input
                                  // is in `state`.  One word per s-step, io_ring > P: the word is
                                  // reused for s-step k + io_ring only after march k has finished
                                  // (a slot's marches run in turn), so no march sees another's
                                  // release
  unsigned long long* io_done;    // [P], written by the march of slot c: prog_value(k, nz,
                                  // completed) each time `completed` reaches a multiple of
                                  // io_chunk, and at the end
  int io_chunk, io_nchunk, io_ring;   // io_chunk = 0: not streamed
  // denoised s-steps as one chain of marches (dn_pipe = 1; nsteps then counts marches): march
  // 2i is the first pass of s-step k0 + i (particles with the plain deposit, its current kept
  // in dn_jcap[k & 3], its level written to dn_scratch and never read), march 2i + 1 the second
  // (the level from the denoised current dn_jext[k & 3] on the unchanged old one, the stored
  // set).  Progress words carry the march index 2k + pass.  The host runs the net on groups of
  // dn_chunk half-slices (group g: nz - (g+1) dn_chunk .. nz - g dn_chunk - 1) as the first
  // pass completes them with their reach, and releases each group to the second pass.
  int dn_pipe;
  void* dn_jcap[4];
  const void* dn_jext[4];
  void* dn_scratch;
  unsigned long long* dn_done;    // host-mapped, per slot: first-pass progress (prog_value of
                                  // its march index) whenever done % dn_chunk == dn_lead, and at
                                  // the end
  unsigned long long* dn_ready;   // host-mapped [4]: word k & 3 holds io_value(2k + 1, dn_nchunk,
                                  // g) once group g of s-step k's denoised current is written
                                  // (one word per s-step, like the current buffers: s-step k + 4
                                  // releases only after s-step k's second pass has finished)
  int dn_chunk, dn_nchunk, dn_lead;
};

// progress word of a march: s-step k has completed `completed` of its nz iterations (they run
// from slice nz-1 down to 0); increasing along the marches a slot runs
__host__ __device__ inline unsigned long long prog_value(long long k, int nz, int completed) {
  return (unsigned long long)(k + 2) * (unsigned long long)(nz + 1) + (unsigned long long)completed;
}
// release word of a streamed input: group j of s-step k's input is in device memory
__host__ __device__ inline unsigned long long io_value(long long k, int nchunk, int j) {
  return (unsigned long long)(k + 2) * (unsigned long long)(nchunk + 1) + (unsigned long long)(j + 1);
}
// group of block b (blocks nz .. 0 from the front)
__host__ __device__ inline int io_group(int nz, int chunk, int b) { return (nz - b) / chunk; }

// Gaussian bunch to sample into the level-0 stored set (gempic_beam, resolved by the host):
// centre (xc, yc), widths, centre and spread along zeta, charge per macroparticle, species slot
struct BeamArgs {
  double xc, yc, sr, sz, zc, gamma, spread, q;
  long long n;
  unsigned long long seed;
  int sp;
};

// Host-side helpers implemented in gempic_kernels.cu
int smem_layout(Params& p, int elem_bytes);           // fills offsets, returns total bytes
cudaError_t configure_kernels(int precision, int smem_bytes, int cluster);
cudaError_t launch_march(int precision, const Params& p, cudaStream_t s);
cudaError_t launch_laser_init(int precision, const Params& p, double a0, double waist,
                              double duration, double zeta_c, int pol, cudaStream_t s);
cudaError_t launch_export_state(int precision, const Params& p, void* dst, cudaStream_t s);
cudaError_t launch_beam_init(int precision, const Params& p, const BeamArgs& b, cudaStream_t s);
// batched scan: one persistent launch over the work items (simulation, march index)
cudaError_t configure_batch(int precision, int smem);
cudaError_t batch_occupancy(int precision, int nthreads, int smem, int* blocks);
cudaError_t launch_batch(int precision, const Params* ps, const int2* items, int nitems, int* head,
                         int grid, int nthreads, int smem, cudaStream_t s);
cudaError_t launch_import_state(int precision, const Params& p, const void* src, cudaStream_t s);
cudaError_t max_active_clusters(int precision, const Params& p, int* n);
// allocation-free entry point: march on a caller's state in the public layout
cudaError_t configure_march_canon(int precision, int smem_bytes);
cudaError_t launch_march_canon(int precision, const Params& p, cudaStream_t s);
cudaError_t launch_tables(int precision, const Params& p, void* dst, cudaStream_t s);
// the denoised chain's march (FP32, p.dn_pipe = 1; compiled in gempic_chain.cu)
cudaError_t configure_chain(int smem_bytes);
cudaError_t launch_march_chain(const Params& p, cudaStream_t s);
// the learned current denoiser on output half-slices [z0, z1) (gempic_denoise.cu); status codes
// of gempic_status
int denoise_range(struct gempic_denoiser* d, const float* j_in, float* j_out, int nx, int ny,
                  int nz, int z0, int z1, cudaStream_t s);
int denoise_status(struct gempic_denoiser* d, cudaStream_t s);
int denoise_reserve(struct gempic_denoiser* d, int nx, int ny, int nz);

}  // namespace gempic
