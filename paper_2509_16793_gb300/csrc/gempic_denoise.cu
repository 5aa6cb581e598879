// Learned current denoiser: a 3-layer 3x3x3 convolutional net (16 hidden channels, ReLU) on
// the current j of the half-slice grid, BF16 operands with FP32 accumulation on the 5th-
// generation tensor cores (tcgen05.mma, accumulators in tensor memory), plus its training
// step (loss, backward pass, Adam).  The paper has no such component: it lets a run with few
// particles per cell stand in for one with many (include/gempic.h, gempic_denoiser_*).
//
// Tensors are channel-last, X[z][y][x][16] in BF16 (z = half-slice, periodic across, zero
// outside the window along zeta).  A convolution is an implicit GEMM: a tile of 128 voxels
// (consecutive in z, y, x order) is the M dimension, the 16 output channels N, and each of the
// 27 taps adds a K = 16 slice (the 16 input channels of the tap's neighbour).  Per tap the
// CTA gathers its tile's 128 neighbour voxels into shared memory in the tensor core's K-major
// layout without swizzle (8-row x 16-byte core matrices: 128 B apart along K, 256 B apart
// along M), one thread issues the MMA, and the 27 MMAs of a tile accumulate in 16 columns of
// tensor memory.  Taps are staged nine at a time into one of two buffers, so the gather of the
// next nine overlaps the MMAs of the last; an mbarrier that tcgen05.commit arrives on tells
// when a buffer is free.  The epilogue reads the accumulators back (tcgen05.ld, one warp per
// 32 rows) and applies the layer's bias, activation or mask.
//
// The backward pass through a layer's input is the same convolution with the kernel mirrored
// and its channels transposed (host-packed operand), masked by the ReLU of the layer below.
// The weight gradients are reductions over the voxels of X_shift^T dY in FP32 on the CUDA
// cores; Adam updates FP32 master weights, which are then repacked into the BF16 operands.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gempic.h"

namespace {

constexpr int kCh = 16;            // channels of every activation tensor (inputs padded)
constexpr int kTaps = 27;
constexpr int kTile = 128;         // voxels per MMA tile (M)
constexpr int kRound = 9;          // taps staged per buffer
constexpr int kThreads = 128;      // 4 warps: one per 32 accumulator rows, one thread per row
static_assert(kThreads == kTile, "the gather gives each thread one row of the tile");
constexpr uint32_t kTapBytesA = kTile * kCh * 2;     // 4096
constexpr uint32_t kTapBytesB = kCh * kCh * 2;       // 512
constexpr uint32_t kLBO = 128;     // byte offset of the core matrix next along K
constexpr uint32_t kSBO = 256;     // byte offset of the core matrix next along M (N)
constexpr int kSpinLimit = 1 << 22;   // polls of an mbarrier before giving up

// instruction descriptor of tcgen05.mma kind::f16: D in FP32, A and B in BF16, both K-major,
// N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kCh >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

enum Mode { MODE_HIDDEN = 0, MODE_LAST = 1, MODE_BWD = 2 };

struct ConvArgs {
  const __nv_bfloat16* x;     // [V][16] input activations
  const __nv_bfloat16* w;     // [27][256] operand B per tap, K-major canonical layout
  const float* bias;          // [16] (MODE_HIDDEN, MODE_LAST)
  int nx, ny, nz;
  int mode;
  __nv_bfloat16* out;         // [V][16] (MODE_HIDDEN, MODE_BWD)
  const __nv_bfloat16* mask;  // [V][16] activations whose sign masks the output (MODE_BWD)
  float* r;                   // [V][4] net output r (MODE_LAST, may be null)
  const float* jres;          // [nz][3][ny][nx] current added to scale r (MODE_LAST, may be null)
  float* jout;                // [nz][3][ny][nx] denoised current (MODE_LAST, may be null)
  float scale;
  int* err;
  int zlo, zhi;               // output half-slices [zlo, zhi) (inputs are read where needed)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1
// (bit 46), no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) |
         ((uint64_t)(kSBO >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase `parity` of an mbarrier: false if it did not complete
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
  for (int i = 0; i < kSpinLimit; ++i)
    if (mbar_test(m, parity)) return true;
  return false;
}

// 16-byte asynchronous copy global -> shared through L1 (neighbouring taps reuse it);
// src_bytes = 0 fills the destination with zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 16 FP32 accumulator columns of this warp's 32 rows (lane = row)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// the layer's output for voxel v from its 16 accumulators: bias + ReLU in BF16 (hidden layers),
// the input's ReLU mask (backward through a layer's input), or bias, the net output r and the
// residual into the FP32 current (last layer)
__device__ __forceinline__ void epilogue(const ConvArgs& a, long long v, const float* acc,
                                         bool add_bias = true) {
  if (a.mode == MODE_HIDDEN) {
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c)
      o[c] = __float2bfloat16_rn(fmaxf(acc[c] + (add_bias ? a.bias[c] : 0.0f), 0.0f));
    uint4* d = reinterpret_cast<uint4*>(a.out + v * kCh);
    d[0] = reinterpret_cast<const uint4*>(o)[0];
    d[1] = reinterpret_cast<const uint4*>(o)[1];
  } else if (a.mode == MODE_BWD) {
    const uint4* mk = reinterpret_cast<const uint4*>(a.mask + v * kCh);
    __align__(16) __nv_bfloat16 m[16];
    reinterpret_cast<uint4*>(m)[0] = mk[0];
    reinterpret_cast<uint4*>(m)[1] = mk[1];
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c)
      o[c] = __float2bfloat16_rn(__bfloat162float(m[c]) > 0.0f ? acc[c] : 0.0f);
    uint4* d = reinterpret_cast<uint4*>(a.out + v * kCh);
    d[0] = reinterpret_cast<const uint4*>(o)[0];
    d[1] = reinterpret_cast<const uint4*>(o)[1];
  } else {
    const float b0 = add_bias ? a.bias[0] : 0.0f, b1 = add_bias ? a.bias[1] : 0.0f,
                b2 = add_bias ? a.bias[2] : 0.0f;
    const float r0 = acc[0] + b0, r1 = acc[1] + b1, r2 = acc[2] + b2;
    if (a.r) *reinterpret_cast<float4*>(a.r + v * 4) = make_float4(r0, r1, r2, 0.0f);
    if (a.jout) {
      const long long plane = (long long)a.nx * a.ny;
      const long long z = v / plane, rem = v - z * plane;
      const long long base = z * 3 * plane + rem;
      const float rr[3] = {r0, r1, r2};
#pragma unroll
      for (int c = 0; c < 3; ++c)
        a.jout[base + c * plane] = __ldcg(a.jres + base + c * plane) + a.scale * rr[c];
    }
  }
}

// neighbour voxel of v for tap t = (dz, dy, dx) + 1 in row-major order, -1 outside the window
__device__ __forceinline__ long long neighbour(long long v, int t, int nx, int ny, int nz) {
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const long long plane = (long long)nx * ny;
  const int z = (int)(v / plane);
  const int rem = (int)(v - (long long)z * plane);
  const int y = rem / nx, x = rem - y * nx;
  const int zz = z + dz;
  if (zz < 0 || zz >= nz) return -1;
  const int yy = (y + dy + ny) % ny, xx = (x + dx + nx) % nx;
  return (long long)zz * plane + (long long)yy * nx + xx;
}

__global__ void __launch_bounds__(kThreads) conv_kernel(ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sB = smem;                                   // 27 x 512
  unsigned char* sA = smem + kTaps * kTapBytesB;              // 2 x 9 x 4096
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long plane0 = (long long)a.nx * a.ny;
  const long long vlo = (long long)a.zlo * plane0;
  const long long V = (long long)a.zhi * plane0;            // output voxels [vlo, V)
  const long long ntiles = (V - vlo + kTile - 1) / kTile;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(
                     smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  // the B operands of the 27 taps
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.w);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < (int)(kTaps * kTapBytesB / 16); i += kThreads) dst[i] = src[i];
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);
  uint32_t phase[2] = {0u, 0u};
  int pending[2] = {0, 0};
  int gr = 0;                                                 // rounds staged so far

  const long long plane = (long long)a.nx * a.ny;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long v0 = vlo + tile * kTile;
    // this thread gathers tile row `tid` (one voxel) for every tap
    const long long vr = v0 + tid;
    const bool valid = vr < V;
    int z = 0, y = 0, x = 0;
    if (valid) {
      z = (int)(vr / plane);
      const int rem = (int)(vr - (long long)z * plane);
      y = rem / a.nx;
      x = rem - y * a.nx;
    }
    for (int round = 0; round < kTaps / kRound; ++round, ++gr) {
      const int buf = gr & 1;
      if (pending[buf]) {                                     // MMAs still reading this buffer
        if (!mbar_wait(&mbar[buf], phase[buf])) atomicExch(&abort_flag, 1);
        phase[buf] ^= 1u;
        pending[buf] = 0;
      }
      // gather: for each tap of the round, this thread's row = the 16 channels (two 16-byte
      // core-matrix rows) of its voxel's neighbour
      // (asynchronous copies: all of a round's loads are in flight at once; a neighbour
      // outside the window copies zero bytes, which fills zeros)
      const uint32_t dstA = aBase + (uint32_t)(buf * kRound) * kTapBytesA + (tid >> 3) * kSBO +
                            (tid & 7) * 16;
#pragma unroll
      for (int s = 0; s < kRound; ++s) {
        const int t = round * kRound + s;
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const int zz = z + dz;
        const bool in = valid && zz >= 0 && zz < a.nz;
        int yy = y + dy, xx = x + dx;
        yy += yy < 0 ? a.ny : 0;
        yy -= yy >= a.ny ? a.ny : 0;
        xx += xx < 0 ? a.nx : 0;
        xx -= xx >= a.nx ? a.nx : 0;
        const __nv_bfloat16* src =
            in ? a.x + ((long long)zz * plane + (long long)yy * a.nx + xx) * kCh : a.x;
        const uint32_t nb = in ? 16u : 0u;
        cp_async16(dstA + (uint32_t)s * kTapBytesA, src, nb);
        cp_async16(dstA + (uint32_t)s * kTapBytesA + kLBO, src + 8, nb);
      }
      cp_async_wait_all();
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0 && !abort_flag) {
        for (int s = 0; s < kRound; ++s) {
          const int t = round * kRound + s;
          umma(tmem, sdesc(aBase + (uint32_t)(buf * kRound + s) * kTapBytesA),
               sdesc(bBase + (uint32_t)t * kTapBytesB), (round > 0 || s > 0) ? 1u : 0u);
        }
        umma_commit(&mbar[buf]);
      }
      pending[buf] = abort_flag ? 0 : 1;                      // uniform after the barrier
    }
    // epilogue: wait for this tile's last MMAs, then one warp per 32 rows
    const int last = (gr - 1) & 1;
    if (pending[last]) {
      if (!mbar_wait(&mbar[last], phase[last])) atomicExch(&abort_flag, 1);
      phase[last] ^= 1u;
      pending[last] = 0;
    }
    tc_fence_after();
    float acc[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), acc);
    const long long v = v0 + warp * 32 + lane;
    if (v < V && !abort_flag) epilogue(a, v, acc);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // no MMA may still be running when the accumulator is released
  for (int b = 0; b < 2; ++b)
    if (pending[b]) {
      if (!mbar_wait(&mbar[b], phase[b])) atomicExch(&abort_flag, 1);
      phase[b] ^= 1u;
    }
  tc_fence_before();
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(a.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// ---- row-staged operands (rows of 128 voxels) ------------------------------------------------
// For nx = 128 an output tile is one row (z, y), and the A operand of tap (dz, dy, dx) is the
// input row (z + dz, y + dy) shifted by dx.  Each input row is staged once in shared memory
// with one halo voxel at each end (x = -1 and x = 128, periodic), a voxel's 16 channels as one
// 32-byte row of the K-major layout with 32-byte swizzling (the two 16-byte halves of a row
// exchanged where bit 7 of its shared-memory address is set; rows 256-byte aligned in groups of
// eight): every tap's operand is then a descriptor into the staged rows, advanced by dx x 32
// bytes, with no per-tap gather.
constexpr int kRowVox = 128;                         // nx of the row path
constexpr int kRowHalo = kRowVox + 2;                // staged voxels: x = -1 .. 128
constexpr uint32_t kRowBytes = 17u * 256u;           // 130 x 32 bytes, rounded to 256

__device__ __forceinline__ uint64_t sdesc_row(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(256u >> 4) << 32) |
         (1ull << 46) | (6ull << 61);
}

// shared-memory address of the 16-byte half h of staged voxel xi in the row at `row`
__device__ __forceinline__ uint32_t swz_addr(uint32_t row, int xi, int h) {
  const uint32_t a = row + (uint32_t)xi * 32u + (uint32_t)h * 16u;
  return a ^ (((a >> 7) & 1u) << 4);
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// ---- warp-specialised row convolution with the three dy taps in one MMA (rows of 128 voxels) -
// An input row (z + dz, r) feeds the output rows r - 1, r, r + 1 of plane z through the taps
// dy = +1, 0, -1.  With the operand B of a (dz, dx) pair holding those three taps' 16 x 16
// weights one under the other (N = 48) and the accumulators of consecutive output rows in
// consecutive 16-column sets of tensor memory, one MMA per (input row, dz, dx) adds all three
// contributions: 9 MMAs per output row instead of 27, each reading its 4 KB operand A once.
// A CTA takes strips of kStripW output rows of one z; the input rows y0 - 1 .. y1 are staged
// as units (three z-planes each) in a ring; set s of tensor memory holds output row
// y0 - 1 + s (sets 0 and kStripW + 1 only collect the contributions to the rows beyond the
// strip, the first and last input rows use N = 16 MMAs of the one tap that reaches into it).
// Roles: two producer warps stage the units with asynchronous copies, wait for them, fence
// them into the tensor core's view and arrive on the unit's `full` mbarrier; one thread issues
// the MMAs (after the epilogue warps zeroed the strip's accumulators), frees each unit through
// `empty` and marks each finished output row through its set's `rowd` mbarrier; four epilogue
// warps zero the accumulators, then read each finished row back and write it.  Every wait is
// bounded: a wait that gives up sets the abort flag and its role stops; the MMA thread waits
// for its MMAs in flight before the tensor memory is freed.
constexpr int kUnits = 6;                            // ring of staged units
constexpr int kLead = 4;                             // units whose copies may be in flight
constexpr int kStripW = 14;                          // output rows per strip
constexpr int kSets = kStripW + 2;                   // accumulator sets (16 columns each)
constexpr int kWsThreads = 224;                      // warps 0-1 produce, 2 issues, 3-6 drain
constexpr uint32_t kUnitBytes = 3u * kRowBytes;      // three z-planes of one row
constexpr uint32_t kWsSmem = (uint32_t)kTaps * kTapBytesB + kUnits * kUnitBytes + 256u;
// instruction descriptors: M = 128, N = 48 (three taps) and N = 16 (one)
constexpr uint32_t kIdesc48 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(48 >> 3) << 17) |
                              ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void umma_n(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// all but the kLead newest groups have landed
__device__ __forceinline__ void cp_async_wait_lead() {
  asm volatile("cp.async.wait_group %0;" ::"n"(kLead) : "memory");
}
// 16-byte asynchronous copy global -> shared through L2 only (a staged row is read once per CTA)
__device__ __forceinline__ void cp_async16_cg(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// zero 16 accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1};" ::"r"(taddr), "r"(z)
      : "memory");
}

__global__ void __launch_bounds__(kWsThreads) conv_ws_kernel(ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sB = smem;                                   // [9 (dz, dx)][3 (dy = +1, 0, -1)][512]
  unsigned char* sU = smem + kTaps * kTapBytesB;              // [kUnits][3 planes][kRowBytes]
  __shared__ __align__(8) uint64_t full[kUnits], empty[kUnits], rowd[kSets], zeroed, drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int u = 0; u < kUnits; ++u) {
      mbar_init(&full[u], 64);
      mbar_init(&empty[u], 1);
    }
    for (int c = 0; c < kSets; ++c) mbar_init(&rowd[c], 1);
    mbar_init(&zeroed, 4);
    mbar_init(&drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  {
    // operand B regrouped by (dz, dx): the taps dy = +1, 0, -1 one under the other
    const uint4* src = reinterpret_cast<const uint4*>(a.w);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    constexpr int kBlk = (int)(kTapBytesB / 16);              // 32 uint4 per tap
    for (int i = tid; i < kTaps * kBlk; i += kWsThreads) {
      const int blk = i / kBlk, e = i - blk * kBlk;
      const int pair = blk / 3, b = blk - pair * 3;           // b = 0, 1, 2: dy = +1, 0, -1
      const int pz = pair / 3, px = pair - pz * 3;
      const int t = pz * 9 + (2 - b) * 3 + px;                // tap (dz, dy, dx) + 1
      dst[i] = src[t * kBlk + e];
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t uBase = smem_u32(sU);
  const int nyb = (a.ny + kStripW - 1) / kStripW;
  const long long nstrips = (long long)(a.zhi - a.zlo) * nyb;
  auto unit_addr = [&](long long u, int plane) -> uint32_t {
    return uBase + (uint32_t)(u % kUnits) * kUnitBytes + (uint32_t)plane * kRowBytes;
  };

  if (warp < 2) {
    // ---- producers: units (z, r) for r = y0-1 .. y1 of every strip, in order ----
    const int pt = tid;                                       // 0 .. 63
    long long uc = 0;
    long long landed = 0;                 // units before this one have been released
    for (long long strip = blockIdx.x; strip < nstrips && !abort_flag; strip += gridDim.x) {
      const int z = a.zlo + (int)(strip / nyb);
      const int y0 = (int)(strip % nyb) * kStripW, y1 = min(a.ny, y0 + kStripW);
      for (int r = y0 - 1; r <= y1; ++r, ++uc) {
        if (!mbar_wait(&empty[uc % kUnits], (uint32_t)(((uc / kUnits) & 1) ^ 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        const int yr = r < 0 ? r + a.ny : (r >= a.ny ? r - a.ny : r);
        for (int dz = -1; dz <= 1; ++dz) {
          const int zz = z + dz;
          if (zz < 0 || zz >= a.nz) continue;                 // its taps are skipped
          const __nv_bfloat16* row = a.x + ((long long)zz * a.ny + yr) * (long long)kRowVox * kCh;
          const uint32_t dst = unit_addr(uc, dz + 1);
          for (int i = pt; i < 2 * kRowHalo; i += 64) {
            const int xi = i >> 1, h = i & 1;
            const int xs = (xi + kRowVox - 1) & (kRowVox - 1);
            cp_async16_cg(swz_addr(dst, xi, h), row + xs * kCh + h * 8);
          }
        }
        cp_async_commit();
        // up to kLead + 1 units in flight (with the one the MMAs read, the whole ring): release
        // the oldest once its copies have landed
        if (uc - landed >= kLead) {
          cp_async_wait_lead();
          fence_async_smem();
          mbar_arrive(&full[landed % kUnits]);
          ++landed;
        }
      }
    }
    cp_async_wait_0();
    fence_async_smem();
    for (; landed < uc; ++landed) mbar_arrive(&full[landed % kUnits]);
  } else if (warp == 2) {
    // ---- MMA issue: one thread ----
    if (lane == 0) {
      const uint64_t bdesc = sdesc(smem_u32(sB));
      constexpr uint64_t kPair = (3u * kTapBytesB) >> 4;     // B of the next (dz, dx) pair
      constexpr uint64_t kTap = kTapBytesB >> 4;
      long long uc = 0, sc = 0;
      bool issued = false;
      for (long long strip = blockIdx.x; strip < nstrips && !abort_flag; strip += gridDim.x, ++sc) {
        const int z = a.zlo + (int)(strip / nyb);
        const int y0 = (int)(strip % nyb) * kStripW, y1 = min(a.ny, y0 + kStripW);
        // the epilogue warps have zeroed the accumulators of this strip
        if (!mbar_wait(&zeroed, (uint32_t)(sc & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        tc_fence_after();
        bool ok = true;
        for (int r = y0 - 1; r <= y1 && ok; ++r, ++uc) {
          if (!mbar_wait(&full[uc % kUnits], (uint32_t)((uc / kUnits) & 1))) {
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          tc_fence_after();
          const int sidx = r - y0;                            // set of output row r - 1
#pragma unroll
          for (int pz = 0; pz < 3; ++pz) {
            if (z + pz - 1 < 0 || z + pz - 1 >= a.nz) continue;
            const uint64_t ad = sdesc_row(unit_addr(uc, pz));
#pragma unroll
            for (int px = 0; px < 3; ++px) {
              const uint64_t bd = bdesc + (uint64_t)(pz * 3 + px) * kPair;
              const uint64_t as = ad + (uint64_t)(2 * px);          // dx: 32 bytes a voxel
              if (r == y0 - 1)            // only dy = -1 reaches the strip (row y0: set 1)
                umma_n(tmem + 16u, as, bd + 2 * kTap, kIdesc);
              else if (r == y1)           // only dy = +1 (row y1 - 1)
                umma_n(tmem + (uint32_t)(16 * (y1 - y0)), as, bd, kIdesc);
              else                        // rows r - 1, r, r + 1: sets r - y0 .. r - y0 + 2
                umma_n(tmem + (uint32_t)(16 * sidx), as, bd, kIdesc48);
            }
          }
          issued = true;
          umma_commit(&empty[uc % kUnits]);
          // output row r - 1 has all its contributions (input rows r - 2 .. r)
          if (r - 1 >= y0) umma_commit(&rowd[r - y0]);
        }
        if (!ok) break;
      }
      if (issued) {
        umma_commit(&drain);
        if (!mbar_wait(&drain, 0u)) atomicExch(&abort_flag, 1);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: warps 3..6 own lanes 32 (warp % 4) .. +31 of the accumulators ----
    const int q = warp & 3;
    float bias[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) bias[c] = (a.bias && a.mode != MODE_BWD) ? a.bias[c] : 0.0f;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    // phase of each row barrier (a short strip at the end of y completes only some of them)
    uint32_t rpar = 0u;                                       // bit c: parity of rowd[c]
    long long sc = 0;
    for (long long strip = blockIdx.x; strip < nstrips && !abort_flag; strip += gridDim.x, ++sc) {
      const int z = a.zlo + (int)(strip / nyb);
      const int y0 = (int)(strip % nyb) * kStripW, y1 = min(a.ny, y0 + kStripW);
      // zero this strip's accumulators (the previous strip's rows have all been read)
      for (int c = 0; c < kSets; ++c) tmem_zero16(tmem + lanes + (uint32_t)(16 * c));
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&zeroed);
      bool ok = true;
      for (int y = y0; y < y1; ++y) {
        const int set = y - y0 + 1;
        if (!mbar_wait(&rowd[set], (rpar >> set) & 1u)) {
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        rpar ^= 1u << set;
        tc_fence_after();
        float acc[16];
        tmem_ld16(tmem + lanes + (uint32_t)(16 * set), acc);
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] += bias[c];
        const long long v = ((long long)z * a.ny + y) * kRowVox + q * 32 + lane;
        epilogue(a, v, acc, false);
      }
      tc_fence_before();
      if (!ok) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(a.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// ---- element-wise kernels ------------------------------------------------------------------

// x0 = bf16(j / scale) channel-last, channels 3..15 zero, on the half-slices [zlo, zhi)
// (j is read through L2: it may have been written by a kernel still running)
__global__ void pack_input_kernel(const float* j, __nv_bfloat16* x0, int nx, int ny, int zlo,
                                  int zhi, float inv_scale) {
  const long long plane = (long long)nx * ny, v0 = plane * zlo, V = plane * zhi;
  for (long long v = v0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    const long long z = v / plane, rem = v - z * plane;
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(0.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      o[c] = __float2bfloat16_rn(__ldcg(j + (z * 3 + c) * plane + rem) * inv_scale);
    uint4* d = reinterpret_cast<uint4*>(x0 + v * kCh);
    d[0] = reinterpret_cast<const uint4*>(o)[0];
    d[1] = reinterpret_cast<const uint4*>(o)[1];
  }
}

// e = j/scale + r - t/scale on the slices [zlo, zhi): loss += e^2 (FP64), dr = bf16(2 e / count)
// channel-last (zero elsewhere and in channels 3..15)
__global__ void loss_kernel(const float* j, const float* t, const float* r, __nv_bfloat16* dr,
                            int nx, int ny, int nz, int zlo, int zhi, float inv_scale,
                            float inv_count2, double* loss) {
  const long long plane = (long long)nx * ny, V = plane * nz;
  double acc = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    const long long z = v / plane, rem = v - z * plane;
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(0.0f);
    if (z >= zlo && z < zhi) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long e0 = (z * 3 + c) * plane + rem;
        const float e = (j[e0] - t[e0]) * inv_scale + r[v * 4 + c];
        acc += (double)e * e;
        o[c] = __float2bfloat16_rn(e * inv_count2);
      }
    }
    uint4* d = reinterpret_cast<uint4*>(dr + v * kCh);
    d[0] = reinterpret_cast<const uint4*>(o)[0];
    d[1] = reinterpret_cast<const uint4*>(o)[1];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// dW[t][ci][co] += sum over voxels of X[v + off(t)][ci] dY[v][co]; db[co] += sum dY[v][co]
// (tap 13 blocks).  Block = one tap x one chunk of voxels; thread = (ci, co).
constexpr int kGradChunk = 1024;
__global__ void __launch_bounds__(256) wgrad_kernel(const __nv_bfloat16* X, const __nv_bfloat16* dY,
                                                    float* dW, float* db, int nx, int ny, int nz,
                                                    int cin, int cout) {
  __shared__ float sx[64][16];
  __shared__ float sy[64][16];
  __shared__ long long snb[64];
  const int t = blockIdx.y;
  const long long V = (long long)nx * ny * nz;
  const long long v0 = (long long)blockIdx.x * kGradChunk;
  const int ci = threadIdx.x >> 4, co = threadIdx.x & 15;
  float acc = 0.0f, accb = 0.0f;
  for (int s = 0; s < kGradChunk; s += 64) {
    if (threadIdx.x < 64) {
      const long long v = v0 + s + threadIdx.x;
      snb[threadIdx.x] = v < V ? neighbour(v, t, nx, ny, nz) : -2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int q = e >> 4, c = e & 15;
      const long long v = v0 + s + q;
      const long long nb = snb[q];
      sy[q][c] = nb > -2 ? __bfloat162float(dY[v * kCh + c]) : 0.0f;
      sx[q][c] = nb >= 0 ? __bfloat162float(X[nb * kCh + c]) : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 64; ++q) {
      acc = fmaf(sx[q][ci], sy[q][co], acc);
      accb += sy[q][co];
    }
    __syncthreads();
  }
  if (ci < cin && co < cout) atomicAdd(dW + ((size_t)t * cin + ci) * cout + co, acc);
  if (t == 13 && ci == 0 && co < cout) atomicAdd(db + co, accb);
}

// Adam (Kingma and Ba 2015) on the FP32 master parameters, bias-corrected
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// operand B of one layer from FP32 weights W[27][cin][cout]: K-major canonical layout,
// B_t[n][k] = W[t][k][n] (forward) or the mirrored tap with channels swapped,
// B_t[n][k] = W[26 - t][n][k] (backward through the input)
__global__ void pack_weights_kernel(const float* W, __nv_bfloat16* B, int cin, int cout, int bwd) {
  const int t = blockIdx.x;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int n = e >> 4, k = e & 15;
    float val = 0.0f;
    if (!bwd) {
      if (k < cin && n < cout) val = W[((size_t)t * cin + k) * cout + n];
    } else {
      if (n < cin && k < cout) val = W[((size_t)(26 - t) * cin + n) * cout + k];
    }
    const uint32_t off = (n >> 3) * kSBO + (k >> 3) * kLBO + (n & 7) * 16 + (k & 7) * 2;
    B[(size_t)t * 256 + off / 2] = __float2bfloat16_rn(val);
  }
}

}  // namespace

// ---- host side ------------------------------------------------------------------------------

struct gempic_denoiser {
  double scale = 1.0;
  int dev = 0, nsm = 0;
  float* p = nullptr;          // FP32 master parameters (layout of gempic_denoiser_params)
  float* g = nullptr;          // gradients
  float* m = nullptr;          // Adam moments
  float* v = nullptr;
  __nv_bfloat16* wf[3] = {};   // forward operands per layer
  __nv_bfloat16* wb[3] = {};   // backward operands (layers 2, 3)
  long long step = 0;
  // activations (grown on demand): x0, h1, h2, dr, dh2, dh1 channel-last; r FP32
  long long cap = 0;
  __nv_bfloat16* act[6] = {};
  float* r = nullptr;
  double* loss = nullptr;
  int* err = nullptr;
};

namespace {

constexpr int kCin[3] = {3, 16, 16}, kCout[3] = {16, 16, 3};
// offsets of W1, b1, W2, b2, W3, b3 in the parameter vector
size_t woff(int l) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)kTaps * kCin[i] * kCout[i] + kCout[i];
  return o;
}
size_t boff(int l) { return woff(l) + (size_t)kTaps * kCin[l] * kCout[l]; }
size_t nparams() { return woff(3); }

size_t conv_smem() { return (size_t)kTaps * kTapBytesB + 2u * kRound * kTapBytesA; }

cudaError_t grow(gempic_denoiser* d, long long V) {
  if (V <= d->cap) return cudaSuccess;
  for (auto*& a : d->act) {
    if (a) cudaFree(a);
    a = nullptr;
  }
  if (d->r) cudaFree(d->r);
  d->r = nullptr;
  d->cap = 0;
  cudaError_t e = cudaSuccess;
  for (auto*& a : d->act)
    if (e == cudaSuccess) e = cudaMalloc(&a, (size_t)V * kCh * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&d->r, (size_t)V * 4 * sizeof(float));
  if (e == cudaSuccess) d->cap = V;
  return e;
}

cudaError_t repack(gempic_denoiser* d, cudaStream_t s) {
  for (int l = 0; l < 3; ++l) {
    pack_weights_kernel<<<kTaps, 256, 0, s>>>(d->p + woff(l), d->wf[l], kCin[l], kCout[l], 0);
    pack_weights_kernel<<<kTaps, 256, 0, s>>>(d->p + woff(l), d->wb[l], kCin[l], kCout[l], 1);
  }
  return cudaGetLastError();
}

cudaError_t conv(gempic_denoiser* d, ConvArgs a, cudaStream_t s) {
  a.err = d->err;
  if (a.zhi <= a.zlo) {                  // whole window unless a range was given
    a.zlo = 0;
    a.zhi = a.nz;
  }
  if (a.nx == kRowVox) {
    const long long strips = (long long)(a.zhi - a.zlo) * ((a.ny + kStripW - 1) / kStripW);
    const int grid = (int)std::min<long long>(strips, 2LL * d->nsm);
    conv_ws_kernel<<<grid, kWsThreads, kWsSmem, s>>>(a);
    return cudaGetLastError();
  }
  const long long V = (long long)a.nx * a.ny * (a.zhi - a.zlo);
  const long long tiles = (V + kTile - 1) / kTile;
  const int grid = (int)std::min<long long>(tiles, 2LL * d->nsm);
  conv_kernel<<<grid, kThreads, conv_smem(), s>>>(a);
  return cudaGetLastError();
}

bool grid_ok(int nx, int ny, int nz) { return nx >= 1 && ny >= 1 && nz >= 1; }

// forward pass of the three layers on x0 = act[0]; h1 -> act[1], h2 -> act[2]; last layer's
// epilogue as requested, for the output half-slices [z0, z1): each layer is computed where the
// next one reads it (one more half-slice on each side per layer below the last)
cudaError_t forward(gempic_denoiser* d, int nx, int ny, int nz, int z0, int z1, const float* jres,
                    float* jout, float* r, cudaStream_t s) {
  ConvArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.zlo = std::max(0, z0 - 2);
  a.zhi = std::min(nz, z1 + 2);
  a.mode = MODE_HIDDEN;
  a.x = d->act[0];
  a.w = d->wf[0];
  a.bias = d->p + boff(0);
  a.out = d->act[1];
  cudaError_t e = conv(d, a, s);
  if (e != cudaSuccess) return e;
  a.x = d->act[1];
  a.w = d->wf[1];
  a.bias = d->p + boff(1);
  a.out = d->act[2];
  a.zlo = std::max(0, z0 - 1);
  a.zhi = std::min(nz, z1 + 1);
  e = conv(d, a, s);
  if (e != cudaSuccess) return e;
  ConvArgs l{};
  l.nx = nx;
  l.ny = ny;
  l.nz = nz;
  l.zlo = z0;
  l.zhi = z1;
  l.mode = MODE_LAST;
  l.x = d->act[2];
  l.w = d->wf[2];
  l.bias = d->p + boff(2);
  l.r = r;
  l.jres = jres;
  l.jout = jout;
  l.scale = (float)d->scale;
  return conv(d, l, s);
}

gempic_status check_err(gempic_denoiser* d, cudaStream_t s) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, d->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  return err ? GEMPIC_ETIMEOUT : GEMPIC_OK;
}

}  // namespace

namespace gempic {

// The net on the output half-slices [z0, z1) of j_in (read where needed: z0 - 3 .. z1 + 2),
// into the same half-slices of j_out, on stream s (no wait).  For the denoised chain of
// marches: j_in may still be written elsewhere outside the half-slices the net reads.
int denoise_range(gempic_denoiser* d, const float* j_in, float* j_out, int nx, int ny, int nz,
                  int z0, int z1, cudaStream_t s) {
  if (!d || !j_in || !j_out || !grid_ok(nx, ny, nz) || z0 < 0 || z1 > nz || z0 >= z1)
    return GEMPIC_EINVAL;
  cudaError_t e = grow(d, (long long)nx * ny * nz);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
  const int p0 = std::max(0, z0 - 3), p1 = std::min(nz, z1 + 3);
  const long long V = (long long)nx * ny * (p1 - p0);
  const int blocks = (int)std::min<long long>((V + 255) / 256, 8LL * d->nsm);
  pack_input_kernel<<<blocks, 256, 0, s>>>(j_in, d->act[0], nx, ny, p0, p1, (float)(1.0 / d->scale));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = forward(d, nx, ny, nz, z0, z1, j_in, j_out, nullptr, s);
  return e == cudaSuccess ? GEMPIC_OK : GEMPIC_ECUDA;
}

// the denoiser's device status word (a bounded wait that gave up): GEMPIC_ETIMEOUT
int denoise_status(gempic_denoiser* d, cudaStream_t s) { return check_err(d, s); }

// working buffers for nx x ny x nz currents, allocated now: growing them frees the old ones,
// and cudaFree waits for the whole device -- while the chain of marches runs, that would wait
// for marches that wait for the net
int denoise_reserve(gempic_denoiser* d, int nx, int ny, int nz) {
  if (!d || !grid_ok(nx, ny, nz)) return GEMPIC_EINVAL;
  cudaError_t e = grow(d, (long long)nx * ny * nz);
  // the net's kernels are loaded now: with lazy module loading a kernel's first launch loads
  // its module, which can wait for the device -- for marches that wait for that kernel
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, pack_input_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv_ws_kernel);
  return e == cudaSuccess ? GEMPIC_OK : e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
}

}  // namespace gempic

extern "C" {

size_t gempic_denoiser_param_count(void) { return nparams(); }

gempic_status gempic_denoiser_create(const float* params, double scale, gempic_denoiser** out) {
  if (!out || !(scale > 0) || !std::isfinite(scale)) return GEMPIC_EINVAL;
  *out = nullptr;
  gempic_denoiser* d = new (std::nothrow) gempic_denoiser();
  if (!d) return GEMPIC_ENOMEM;
  d->scale = scale;
  cudaError_t e = cudaGetDevice(&d->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->nsm, cudaDevAttrMultiProcessorCount, d->dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kWsSmem);
  const size_t n = nparams();
  float** bufs[4] = {&d->p, &d->g, &d->m, &d->v};
  for (float** b : bufs)
    if (e == cudaSuccess) e = cudaMalloc(b, n * sizeof(float));
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    e = cudaMalloc(&d->wf[l], kTaps * 256 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&d->wb[l], kTaps * 256 * sizeof(__nv_bfloat16));
  }
  if (e == cudaSuccess) e = cudaMalloc(&d->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d->m, 0, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(d->v, 0, n * sizeof(float));
  if (e == cudaSuccess) {
    if (params) {
      e = cudaMemcpy(d->p, params, n * sizeof(float), cudaMemcpyHostToDevice);
    } else {
      e = cudaMemset(d->p, 0, n * sizeof(float));   // all zero: the identity on j
    }
  }
  if (e == cudaSuccess) e = repack(d, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    gempic_denoiser_destroy(d);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
  }
  *out = d;
  return GEMPIC_OK;
}

gempic_status gempic_denoiser_set_params(gempic_denoiser* d, const float* params, size_t n) {
  if (!d || !params || n != nparams()) return GEMPIC_EINVAL;
  cudaError_t e = cudaMemcpy(d->p, params, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d->m, 0, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(d->v, 0, n * sizeof(float));
  if (e == cudaSuccess) e = repack(d, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  d->step = 0;
  return e == cudaSuccess ? GEMPIC_OK : GEMPIC_ECUDA;
}

gempic_status gempic_denoiser_get_params(gempic_denoiser* d, float* params, size_t n) {
  if (!d || !params || n != nparams()) return GEMPIC_EINVAL;
  cudaError_t e = cudaMemcpy(params, d->p, n * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? GEMPIC_OK : GEMPIC_ECUDA;
}

gempic_status gempic_denoiser_apply(gempic_denoiser* d, const float* j_in, float* j_out,
                                    int32_t nx, int32_t ny, int32_t nz, void* cuda_stream) {
  if (!d || !j_in || !j_out || !grid_ok(nx, ny, nz)) return GEMPIC_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long V = (long long)nx * ny * nz;
  cudaError_t e = grow(d, V);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
  const int blocks = (int)std::min<long long>((V + 255) / 256, 8LL * d->nsm);
  pack_input_kernel<<<blocks, 256, 0, s>>>(j_in, d->act[0], nx, ny, 0, nz, (float)(1.0 / d->scale));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = forward(d, nx, ny, nz, 0, nz, j_in, j_out, nullptr, s);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  return check_err(d, s);
}

gempic_status gempic_denoiser_grad(gempic_denoiser* d, const float* j_in, const float* j_target,
                                   int32_t nx, int32_t ny, int32_t nz, int32_t z_margin,
                                   double* loss, float* grad_host, void* cuda_stream) {
  if (!d || !j_in || !j_target || !grid_ok(nx, ny, nz) || z_margin < 0 || 2 * z_margin >= nz)
    return GEMPIC_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long V = (long long)nx * ny * nz;
  cudaError_t e = grow(d, V);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GEMPIC_ENOMEM : GEMPIC_ECUDA;
  const int blocks = (int)std::min<long long>((V + 255) / 256, 8LL * d->nsm);
  const size_t n = nparams();
  e = cudaMemsetAsync(d->g, 0, n * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  pack_input_kernel<<<blocks, 256, 0, s>>>(j_in, d->act[0], nx, ny, 0, nz, (float)(1.0 / d->scale));
  e = forward(d, nx, ny, nz, 0, nz, nullptr, nullptr, d->r, s);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  const double count = 3.0 * (double)nx * ny * (nz - 2 * z_margin);
  loss_kernel<<<blocks, 256, 0, s>>>(j_in, j_target, d->r, d->act[3], nx, ny, nz, z_margin,
                                     nz - z_margin, (float)(1.0 / d->scale), (float)(2.0 / count),
                                     d->loss);
  // backward: dr = act[3]; dh2 = mask(h2) conv(dr, W3'); dh1 = mask(h1) conv(dh2, W2')
  __nv_bfloat16* const dr = d->act[3];
  __nv_bfloat16* const dh2 = d->act[4];
  __nv_bfloat16* const dh1 = d->act[5];
  ConvArgs b{};
  b.nx = nx;
  b.ny = ny;
  b.nz = nz;
  b.mode = MODE_BWD;
  b.x = dr;
  b.w = d->wb[2];
  b.mask = d->act[2];
  b.out = dh2;
  e = conv(d, b, s);
  if (e == cudaSuccess) {
    b.x = dh2;
    b.w = d->wb[1];
    b.mask = d->act[1];
    b.out = dh1;
    e = conv(d, b, s);
  }
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  const dim3 gg((unsigned)((V + kGradChunk - 1) / kGradChunk), kTaps);
  const __nv_bfloat16* xs[3] = {d->act[0], d->act[1], d->act[2]};
  const __nv_bfloat16* ds[3] = {dh1, dh2, dr};
  for (int l = 0; l < 3; ++l)
    wgrad_kernel<<<gg, 256, 0, s>>>(xs[l], ds[l], d->g + woff(l), d->g + boff(l), nx, ny, nz,
                                    kCin[l], kCout[l]);
  e = cudaGetLastError();
  double lv = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&lv, d->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, d->g, n * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return GEMPIC_ECUDA;
  if (loss) *loss = lv / count;
  return check_err(d, s);
}

gempic_status gempic_denoiser_train_step(gempic_denoiser* d, const float* j_in,
                                         const float* j_target, int32_t nx, int32_t ny,
                                         int32_t nz, int32_t z_margin, double lr, double* loss,
                                         void* cuda_stream) {
  if (!(lr > 0) || !std::isfinite(lr)) return GEMPIC_EINVAL;
  gempic_status st = gempic_denoiser_grad(d, j_in, j_target, nx, ny, nz, z_margin, loss, nullptr,
                                          cuda_stream);
  if (st != GEMPIC_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  d->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)d->step));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)d->step));
  const int n = (int)nparams();
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(d->p, d->g, d->m, d->v, n, (float)lr, b1, b2, 1e-8f,
                                               c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = repack(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? GEMPIC_OK : GEMPIC_ECUDA;
}

void gempic_denoiser_destroy(gempic_denoiser* d) {
  if (!d) return;
  cudaDeviceSynchronize();
  float* bufs[4] = {d->p, d->g, d->m, d->v};
  for (float* b : bufs)
    if (b) cudaFree(b);
  for (int l = 0; l < 3; ++l) {
    if (d->wf[l]) cudaFree(d->wf[l]);
    if (d->wb[l]) cudaFree(d->wb[l]);
  }
  for (auto* a : d->act)
    if (a) cudaFree(a);
  if (d->r) cudaFree(d->r);
  if (d->loss) cudaFree(d->loss);
  if (d->err) cudaFree(d->err);
  cudaGetLastError();
  delete d;
}

}  // extern "C"
