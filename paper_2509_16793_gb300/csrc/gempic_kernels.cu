// GEM-PIC hot path on sm_103a: the zeta march of one s-step as a persistent kernel run by a
// thread-block cluster, and (optionally) several s-steps in flight as a wavefront.
//
// One cluster of C CTAs marches one s-step (Sec. 4.1: the fields of the next s-level are found
// slice by slice, starting at the front edge of the window).  CTA r owns
//   * real-space rows y in [r RB, (r+1) RB) of every slice plane (fields for the gather,
//     current accumulators for the deposit), and the fresh particles injected into them;
//   * spectral columns kx in [r KB, (r+1) KB) for all ky (per-mode slice solve, App. B),
//     with one mode per thread whose carried state lives in registers.
// Per slice n = nz-1 .. 0 (zeta_n = n h):
//   A  gather E,B of slice n+1 at every streaming particle, push it to plane n along the GT2
//      characteristics (two-pass Boris, budget rule of Eq. trap2), deposit the transverse
//      current by the 2-D Esirkepov decomposition and j_z by CIC into shared memory
//      (distributed shared memory atomics for rows of another CTA); trapped particles go to
//      the stored set; rejoining stored particles join here; the beam current is added.
//   B  row FFTs of the currents, transposed into the kx-owner CTAs (DSMEM stores).
//   C  column FFTs; per mode: corrector of R at slice n+1, write of the new level at slice
//      n+1 to HBM, App. B solve at slice n, fields E,B; inverse column FFTs, transposed back.
//   D  inverse row FFTs: real-space E,B of slice n into shared memory (next gather).
//   E  stored particles in cell (zeta_n, zeta_{n+1}] are pushed along s with the fields of
//      slices n and n+1 (Sec. 5.1, last paragraph), depositing the next level's beam current.
//
// Wavefront: the march of s-step k+1 on another cluster needs, at slice n, only what the march
// of step k produced at slices >= n-1.  Marches publish per-slice progress in global memory
// and wait on their predecessor with bounded spins; every device wait has a limit and sets an
// error bit instead of hanging.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "gempic_internal.h"

namespace cg = cooperative_groups;

namespace gempic {

// ------------------------------------------------------------------------------------------
// small complex / vector helpers
// ------------------------------------------------------------------------------------------
template <typename T>
struct alignas(2 * sizeof(T)) Cx {
  T re, im;
};
template <typename T>
__device__ __forceinline__ Cx<T> cx(T a, T b) { return Cx<T>{a, b}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ Cx<T> operator*(T s, Cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> conjg(Cx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> mul_i(Cx<T> a) { return {-a.im, a.re}; }   // i a

template <typename T>
struct V3 {
  T x, y, z;
};

template <typename T>
__device__ __forceinline__ T gamma_of(V3<T> u) {   // sqrt(1 + ux^2 + uy^2 + uz^2)
  return sqrt(((T(1) + u.x * u.x) + u.y * u.y) + u.z * u.z);
}
// gamma - 1 for the kinetic energy: in FP32 as u^2/(gamma + 1) (sqrt(1 + u^2) - 1 cancels for
// slow particles); in FP64 as gamma - 1, the form the FP64 reference evaluates
template <typename T>
__device__ __forceinline__ T gamma_minus_one(V3<T> u, T g) {
  if constexpr (sizeof(T) == 4)
    return ((u.x * u.x + u.y * u.y) + u.z * u.z) / (g + T(1));
  else
    return g - T(1);
}
// gamma - u_z, as (1 + u_perp^2)/(gamma + u_z) where u_z > 0 (no cancellation).
template <typename T>
__device__ __forceinline__ T gamma_minus_uz(V3<T> u, T g) {
  return u.z > T(0) ? ((T(1) + u.x * u.x) + u.y * u.y) / (g + u.z) : g - u.z;
}

// reciprocal and reciprocal square root: hardware approximations (a few ulp) in FP32, exact
// division in FP64
template <typename T>
__device__ __forceinline__ T rcp(T x) {
  if constexpr (sizeof(T) == 4)
    return __fdividef(1.0f, x);
  else
    return T(1) / x;
}
template <typename T>
__device__ __forceinline__ T rsq(T x) {
  if constexpr (sizeof(T) == 4)
    return rsqrtf(x);
  else
    return T(1) / sqrt(x);
}

// Relativistic Boris rotation over lab time dt: du/dt = (q/m)(E + u x B / gamma).
template <typename T>
__device__ __forceinline__ V3<T> boris(V3<T> u, const T* E, const T* B, T qm, T dt) {
  const T a = T(0.5) * qm * dt;
  V3<T> um{u.x + a * E[0], u.y + a * E[1], u.z + a * E[2]};
  const T ag = a * rsq(T(1) + ((um.x * um.x + um.y * um.y) + um.z * um.z));   // a / gamma
  const T tx = ag * B[0], ty = ag * B[1], tz = ag * B[2];
  V3<T> up{um.x + (um.y * tz - um.z * ty), um.y + (um.z * tx - um.x * tz),
           um.z + (um.x * ty - um.y * tx)};
  const T f = T(2) * rcp(T(1) + ((tx * tx + ty * ty) + tz * tz));
  const T sx = f * tx, sy = f * ty, sz = f * tz;
  V3<T> upl{um.x + (up.y * sz - up.z * sy), um.y + (up.z * sx - up.x * sz),
            um.z + (up.x * sy - up.y * sx)};
  return V3<T>{upl.x + a * E[0], upl.y + a * E[1], upl.z + a * E[2]};
}

// ------------------------------------------------------------------------------------------
// memory-model helpers: data exchanged between clusters is read at L2 (ld.global.cg) and the
// progress word is published / observed with release / acquire at GPU scope.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ Cx<float> ldcg(const Cx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return Cx<float>{v.x, v.y};
}
template <>
__device__ __forceinline__ Cx<double> ldcg(const Cx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return Cx<double>{v.x, v.y};
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// system scope: words in host-mapped memory shared with the calling thread
__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// shared memory of this CTA and of other CTAs of the cluster, addressed explicitly
__device__ __forceinline__ uint32_t sh_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float lds(uint32_t a, float) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ double lds(uint32_t a, double) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float ldc(uint32_t a, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ double ldc(uint32_t a, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void red_local(uint32_t a, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ void red_local(uint32_t a, double v) {
  asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(a), "d"(v));
}
__device__ __forceinline__ void red_local_u32(uint32_t a, int v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v));
}
// the same, predicated on v != 0 (no branch)
__device__ __forceinline__ void red_local_u32_nz(uint32_t a, int v) {
  asm volatile(
      "{\n\t.reg .pred nz;\n\tsetp.ne.s32 nz, %1, 0;\n\t@nz red.shared.add.u32 [%0], %1;\n\t}" ::"r"(a),
      "r"(v));
}
__device__ __forceinline__ void red_cluster(uint32_t a, float v) {
  asm volatile("red.shared::cluster.add.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ void red_cluster(uint32_t a, double v) {
  asm volatile("red.shared::cluster.add.f64 [%0], %1;" ::"r"(a), "d"(v));
}
__device__ __forceinline__ void red_cluster_u32(uint32_t a, int v) {
  asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v));
}

// Counter-based SplitMix64 (Steele, Lea, Flood 2014): output c of the stream seeded with s.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long s,
                                                         unsigned long long c) {
  unsigned long long z = s + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// 24 random bits as a uniform in [0,1), exact in float and double.
__device__ __forceinline__ double uniform24(unsigned long long s, unsigned long long c) {
  return (double)(splitmix64(s, c) >> 40) * (1.0 / 16777216.0);
}

// ------------------------------------------------------------------------------------------
// warp-level FFTs on shared memory (length N = 2^logN, unnormalised, in place).
// tw[k] = exp(-2 pi i k / N), k < N/2; inverse: conjugate twiddles.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Cx<T> twiddle(const Cx<T>* tw, int N, int m, bool inverse) {
  m &= N - 1;
  Cx<T> w = m < (N >> 1) ? tw[m] : cx<T>(-tw[m - (N >> 1)].re, -tw[m - (N >> 1)].im);
  if (inverse) w.im = -w.im;
  return w;
}

// radix-2, any N = 2^logN (used for N < 32 and N > 256)
template <typename T>
__device__ void warp_fft_r2(Cx<T>* d, int logN, const Cx<T>* tw, bool inverse) {
  const int N = 1 << logN;
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < N; i += 32) {
    const int r = (int)(__brev((unsigned)i) >> (32 - logN));
    if (i < r) {
      Cx<T> t = d[i];
      d[i] = d[r];
      d[r] = t;
    }
  }
  __syncwarp();
  for (int s = 1; s <= logN; ++s) {
    const int half = 1 << (s - 1);
    const int tstride = N >> s;
    for (int b = lane; b < N / 2; b += 32) {
      const int grp = b >> (s - 1);
      const int j = b & (half - 1);
      const int i0 = grp * (half << 1) + j;
      const int i1 = i0 + half;
      Cx<T> w = tw[j * tstride];
      if (inverse) w.im = -w.im;
      const Cx<T> t = w * d[i1];
      const Cx<T> u = d[i0];
      d[i0] = u + t;
      d[i1] = u - t;
    }
    __syncwarp();
  }
}

template <typename T>
__device__ __forceinline__ Cx<T> shfl_xor_cx(Cx<T> v, int m) {
  return cx<T>(__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m));
}

// Register FFTs of length N = 32 R (R = 1, 2, 4, 8), one transform per warp.  With
// n = l + 32 r and k = k2 + R k1 the DFT factors as
//   X[k2 + R k1] = sum_l W_32^{l k1} W_N^{l k2} sum_r W_R^{r k2} x[l + 32 r]:
// an R-point DFT in the registers of each lane, a twiddle, and a 32-point DFT across the
// lanes (shuffles).  Two register layouts occur:
//   natural:   lane l, register r holds element l + 32 r;
//   lane order: lane l, register k2 holds element k2 + R bitrev5(l).
// fft_dif_lanes maps natural -> lane order (decimation in frequency across the lanes),
// fft_dit_lanes maps lane order -> natural (decimation in time); both are unnormalised and
// take conjugate twiddles when inverse is set.  Stored with register j of lane l at
// position l + 32 j, both layouts give conflict-free shared-memory rows.

// R-point DFT over the registers of one lane, natural order in and out
template <typename T, int R>
__device__ __forceinline__ void reg_dft(Cx<T> (&a)[R], const Cx<T>* tw, bool inverse) {
  if constexpr (R > 1) {
    constexpr int N = 32 * R;
    constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : 3;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int rr = (int)(__brev((unsigned)r) >> (32 - LR));
      if (r < rr) {
        const Cx<T> t = a[r];
        a[r] = a[rr];
        a[rr] = t;
      }
    }
#pragma unroll
    for (int st = 1; st <= LR; ++st) {
      const int half = 1 << (st - 1);
#pragma unroll
      for (int q = 0; q < R / 2; ++q) {
        const int grp = q >> (st - 1), j = q & (half - 1);
        const int i0 = grp * (half << 1) + j, i1 = i0 + half;
        const Cx<T> w = twiddle(tw, N, j * (N / (half << 1)), inverse);
        const Cx<T> t = w * a[i1];
        const Cx<T> u = a[i0];
        a[i0] = u + t;
        a[i1] = u - t;
      }
    }
  }
}

template <typename T, int R>
__device__ __forceinline__ void fft_dif_lanes(Cx<T> (&a)[R], const Cx<T>* tw, bool inverse) {
  constexpr int N = 32 * R;
  const int l = threadIdx.x & 31;
  reg_dft<T, R>(a, tw, inverse);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) a[k2] = twiddle(tw, N, l * k2, inverse) * a[k2];
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool bottom = (l & half) != 0;
    const Cx<T> w = twiddle(tw, N, (l & (half - 1)) * (16 / half) * R, inverse);
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      const Cx<T> o = shfl_xor_cx(a[k2], half);
      a[k2] = bottom ? w * (o - a[k2]) : a[k2] + o;
    }
  }
}

template <typename T, int R>
__device__ __forceinline__ void fft_dit_lanes(Cx<T> (&a)[R], const Cx<T>* tw, bool inverse) {
  constexpr int N = 32 * R;
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int half = 1; half <= 16; half <<= 1) {
    const bool bottom = (l & half) != 0;
    const Cx<T> w = twiddle(tw, N, (l & (half - 1)) * (16 / half) * R, inverse);
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      const Cx<T> t = bottom ? w * a[k2] : a[k2];
      const Cx<T> o = shfl_xor_cx(t, half);
      a[k2] = bottom ? o - t : t + o;
    }
  }
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) a[k2] = twiddle(tw, N, l * k2, inverse) * a[k2];
  reg_dft<T, R>(a, tw, inverse);
}

// lengths with a register FFT
__host__ __device__ __forceinline__ bool reg_fft_len(int logN) { return logN >= 5 && logN <= 8; }

// Column spectra of the lane-order register FFTs (ny = 32, 64, 256) are kept in lane order:
// position q of a column holds ky index ky_of_pos(q); natural order for other lengths.
__host__ __device__ __forceinline__ int bitrev5(int v) {
  return ((v & 1) << 4) | ((v & 2) << 2) | (v & 4) | ((v & 8) >> 2) | ((v & 16) >> 4);
}
// columns of length 128 use the natural-order transform fft128_h16
__host__ __device__ __forceinline__ bool col_lane_order(int logny) {
  return reg_fft_len(logny) && logny != 7;
}
__host__ __device__ __forceinline__ int ky_of_pos(int logny, int q) {
  if (!col_lane_order(logny)) return q;
  const int R = 1 << (logny - 5);
  return (q >> 5) + R * bitrev5(q & 31);
}
__host__ __device__ __forceinline__ int pos_of_ky(int logny, int ky) {
  if (!col_lane_order(logny)) return ky;
  const int R = 1 << (logny - 5);
  return bitrev5(ky / R) + 32 * (ky % R);
}

// store R consecutive reals (16-byte vectors where the run allows)
template <typename T, int R>
__device__ __forceinline__ void st_run(T* dst, const T (&v)[R]) {
  if constexpr (sizeof(T) == 4 && R >= 4) {
#pragma unroll
    for (int i = 0; i < R; i += 4)
      *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  } else if constexpr (sizeof(T) == 4 && R == 2) {
    *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
  } else if constexpr (sizeof(T) == 8 && R >= 2) {
#pragma unroll
    for (int i = 0; i < R; i += 2) *reinterpret_cast<double2*>(dst + i) = make_double2(v[i], v[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) dst[i] = v[i];
  }
}

// Transforms of length 128 (the 128-cell transverse grids): 16 lanes per transform, 8 values
// per lane, one swizzled transpose through shared memory, compile-time twiddles for the small
// DFTs.  With n = j + 16 r and k = k2 + 8 k1:
//   X[k2 + 8 k1] = sum_j W_16^{j k1} W_128^{j k2} sum_r W_8^{r k2} x[j + 16 r];
// each lane does the 8-point DFT over r and the twiddle W_128^{j k2}; after the transpose lane
// (k2, j0) does the 8-point DFT over j1 of the terms j = 2 j1 + j0, and the pair (j0 = 0, 1)
// finishes the 16-point DFT over j with one radix-2 step across the two lanes.

// a (c - i s) forward, a (c + i s) inverse
template <typename T>
__device__ __forceinline__ Cx<T> cmul_w(Cx<T> a, T c, T s, bool inverse) {
  const T sn = inverse ? s : -s;
  return cx<T>(a.re * c - a.im * sn, a.re * sn + a.im * c);
}

// cos and sin of 2 pi m / 16, m = 0..7
template <typename T>
__device__ __forceinline__ T cos16(int m) {
  return m == 0 ? T(1) : m == 1 ? T(0.92387953251128675613) : m == 2 ? T(0.70710678118654752440)
       : m == 3 ? T(0.38268343236508977173) : m == 4 ? T(0) : m == 5 ? T(-0.38268343236508977173)
       : m == 6 ? T(-0.70710678118654752440) : T(-0.92387953251128675613);
}
template <typename T>
__device__ __forceinline__ T sin16(int m) {
  return m == 0 ? T(0) : m == 1 || m == 7 ? T(0.38268343236508977173)
       : m == 2 || m == 6 ? T(0.70710678118654752440) : m == 3 || m == 5 ? T(0.92387953251128675613)
       : T(1);
}

// 8-point DFT in registers (radix 2, decimation in time on bit-reversed inputs), natural order
// in and out, unnormalised; conjugate twiddles when inverse
template <typename T>
__device__ __forceinline__ void dft8_reg(Cx<T> (&a)[8], bool inverse) {
  { Cx<T> t = a[1]; a[1] = a[4]; a[4] = t; t = a[3]; a[3] = a[6]; a[6] = t; }
#pragma unroll
  for (int st = 1; st <= 3; ++st) {
    const int half = 1 << (st - 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int grp = q >> (st - 1), j = q & (half - 1);
      const int i0 = grp * (half << 1) + j, i1 = i0 + half;
      const int m16 = j * (16 / (half << 1));           // W_{2 half}^j = W_16^{m16}
      Cx<T> t;
      if (m16 == 0)
        t = a[i1];
      else if (m16 == 4)
        t = inverse ? cx<T>(-a[i1].im, a[i1].re) : cx<T>(a[i1].im, -a[i1].re);
      else
        t = cmul_w(a[i1], cos16<T>(m16), sin16<T>(m16), inverse);
      const Cx<T> u = a[i0];
      a[i0] = u + t;
      a[i1] = u - t;
    }
  }
}

// In: lane i = j (i = lane mod 16) holds a[r] = x[j + 16 r].  Out: lane i = 2 k2 + j0 holds
// b[m] = X[k2 + 8 m + 64 j0], m = 0..7.  bufA / bufB: positions 0..63 / 64..127 of 128 entries
// of scratch private to this half-warp; the transpose puts (k2, j) at 16 k2 + (j ^ 2 k2)
// (conflict-free for the writing and the reading lanes).  tw[j] = W_128^j (j < 16).  Every lane
// of the warp calls it (it synchronises the warp); a half with active == false touches no
// memory.
template <typename T>
__device__ __forceinline__ void fft128_h16(Cx<T> (&a)[8], Cx<T>* bufA, Cx<T>* bufB,
                                           const Cx<T>* tw, bool inverse, bool active,
                                           Cx<T> (&b)[8]) {
  const int i = threadIdx.x & 15;
  dft8_reg<T>(a, inverse);
  {
    // W_128^{j k2}, k2 = 1..7, as powers of W_128^j
    Cx<T> w1 = tw[i];
    if (inverse) w1.im = -w1.im;
    const Cx<T> w2 = w1 * w1, w4 = w2 * w2;
    const Cx<T> w3 = w2 * w1, w5 = w4 * w1, w6 = w4 * w2, w7 = w4 * w3;
    a[1] = w1 * a[1];
    a[2] = w2 * a[2];
    a[3] = w3 * a[3];
    a[4] = w4 * a[4];
    a[5] = w5 * a[5];
    a[6] = w6 * a[6];
    a[7] = w7 * a[7];
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      const int pos = 16 * k2 + (i ^ (2 * k2));
      if (k2 < 4)
        bufA[pos] = a[k2];
      else
        bufB[pos - 64] = a[k2];
    }
  }
  __syncwarp();
  const int k2 = i >> 1, j0 = i & 1;
#pragma unroll
  for (int j1 = 0; j1 < 8; ++j1) {
    const int pos = 16 * k2 + ((2 * j1 + j0) ^ (2 * k2));
    b[j1] = active ? (pos < 64 ? bufA[pos] : bufB[pos - 64]) : cx<T>(T(0), T(0));
  }
  dft8_reg<T>(b, inverse);
  // X[k2 + 8 k1] = E[k1] + W_16^{k1} O[k1], X[k2 + 8 (k1 + 8)] = E[k1] - W_16^{k1} O[k1]
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const Cx<T> mine = j0 ? cmul_w(b[m], cos16<T>(m), sin16<T>(m), inverse) : b[m];
    const Cx<T> other = shfl_xor_cx(mine, 1);
    b[m] = j0 ? other - mine : mine + other;
  }
  __syncwarp();
}

// ------------------------------------------------------------------------------------------
// per-kernel shared-memory views
// ------------------------------------------------------------------------------------------
enum CstSlot {
  K_H = 0, K_INVH, K_HX, K_HY, K_D, K_DF, K_WSCALE, K_CX, K_CY, K_INVHX, K_INVHY, K_FLUX,
  K_BEAM, K_JREF, K_JSCALE, K_JINV, K_QM = 16, K_MOQ = 20, K_QF = 24, K_INVD = 28, K_N = 29
};
enum MiscSlot { M_PCOUNT = 0, M_FTOP, M_INBOX, M_RQN, M_JFLAG, M_STN, M_OUTN, M_IOSEEN };
// particles leaving the band during a push wait in a local outbox of this many entries
constexpr int kOutCap = 64;

// Shared memory of one CTA.  Plane sets are [comp][rows][nx]: the fields F keep the CTA's RB
// rows plus one halo row above (FR = RB + 1); the currents J keep rows -1 .. RB + 1 of the
// band (JR = RB + 3, own row 0 at index JOFF = 1).  In 2-D FR = JR = 1, JOFF = 0.
template <typename T>
struct Sm {
  T* F[2];          // [6][FR][nx] real-space fields (Ex,Ey,Ez,Bx,By,Bz)
  T* J;             // [3][JR][nx] current accumulators (jx on x-edges, jy (3-D: y-edges), jz)
  int* Jint;        // [3][JR][nx] fixed-point accumulators of the push phase (FP32; aliases SR)
  T* recv;          // [3][3][nx] halo currents received: rows 0, 1 (from below), RB-1 (above)
  Cx<T>* SR;        // [6][FR][nx/2] row spectra received for the inverse transform
  Cx<T>* SC;        // [6][KB][ny] column spectra (forward: 3 currents; inverse: 6 fields)
  Cx<T>* workB;     // [nwork][nx] row FFT work of the forward transform (aliases SR)
  Cx<T>* workD;     // [nwork][nx] row FFT work of the inverse transform (aliases SC)
  Cx<T>* twx;       // [nx/2]
  Cx<T>* twy;       // [max(ny/2,1)]
  Cx<T>* shx;       // [nx/2]  exp(-i kx hx/2)
  Cx<T>* shy;       // [ny]    exp(-i ky hy/2)
  T* kx;            // [nx/2]
  T* ky;            // [ny]
  T* cst;           // [K_N] constants in the working precision
  int* icell;       // [mig_cap] inbox of particles migrating in
  T *ifx, *ify, *iux, *iuy, *iuz, *isig, *iq;
  int *ocell, *odst;  // [kOutCap] outbox of particles leaving the band (3-D), owner CTA
  T *ofx, *ofy, *oux, *ouy, *ouz, *osig, *oq;
  int* pcell;       // [pcap] ix | iy << 10 | sp << 20, -1 = empty
  T *pfx, *pfy, *pux, *puy, *puz, *psig, *pq;
  int* fstack;      // [fcap] free particle slots
  int* misc;        // MiscSlot
  double* dacc;     // [kNDiag]; dacc[0], dacc[1]: the march's continuity and Gauss residual
                    // maxima (verification mode)
  T* dd;            // [RBe][nx] continuity residual: w CIC(start) - w CIC(end) of the slab's
                    // moves on the own rows (RBe = RB in 3-D, 1 in 2-D)
  T* dn;            // [2][RBe][nx] (rho - j_z) CIC density of the particles reaching a plane,
                    // by plane parity (Gauss residual)
  double* dwarp;    // [nthreads / 32][kNDiag] per-warp FP64 diagnostic sums of this march
};

template <typename T>
__device__ Sm<T> carve(const Params& p, unsigned char* base) {
  Sm<T> s;
  s.F[0] = (T*)(base + p.o_f0);
  s.F[1] = (T*)(base + p.o_f1);
  s.J = (T*)(base + p.o_j);
  s.recv = (T*)(base + p.o_recv);
  s.SR = (Cx<T>*)(base + p.o_sr);
  s.Jint = (int*)(base + p.o_sr);
  s.SC = (Cx<T>*)(base + p.o_sc);
  s.workB = (Cx<T>*)(base + p.o_workB);
  s.workD = (Cx<T>*)(base + p.o_workD);
  Cx<T>* tw = (Cx<T>*)(base + p.o_tw);
  const int nyh = p.ny > 1 ? p.ny / 2 : 1;
  s.twx = tw;
  s.twy = s.twx + p.nx / 2;
  s.shx = s.twy + nyh;
  s.shy = s.shx + p.nx / 2;
  s.kx = (T*)(s.shy + p.ny);
  s.ky = s.kx + p.nx / 2;
  s.cst = s.ky + p.ny;
  unsigned char* ib = base + p.o_inbox;
  const int mcap = p.mig_cap;
  s.icell = (int*)ib;
  T* it = (T*)(ib + ((mcap * 4 + 15) / 16) * 16);
  s.ifx = it;
  s.ify = it + mcap;
  s.iux = it + 2 * mcap;
  s.iuy = it + 3 * mcap;
  s.iuz = it + 4 * mcap;
  s.isig = it + 5 * mcap;
  s.iq = it + 6 * mcap;
  unsigned char* ob = base + p.o_outbox;
  s.ocell = (int*)ob;
  s.odst = s.ocell + kOutCap;
  T* ot = (T*)(ob + 2 * kOutCap * 4);
  s.ofx = ot;
  s.ofy = ot + kOutCap;
  s.oux = ot + 2 * kOutCap;
  s.ouy = ot + 3 * kOutCap;
  s.ouz = ot + 4 * kOutCap;
  s.osig = ot + 5 * kOutCap;
  s.oq = ot + 6 * kOutCap;
  unsigned char* pp = base + p.o_part;
  s.pcell = (int*)pp;
  T* pt = (T*)(pp + ((p.pcap * 4 + 15) / 16) * 16);
  s.pfx = pt;
  s.pfy = pt + p.pcap;
  s.pux = pt + 2 * p.pcap;
  s.puy = pt + 3 * p.pcap;
  s.puz = pt + 4 * p.pcap;
  s.psig = pt + 5 * p.pcap;
  s.pq = pt + 6 * p.pcap;
  s.fstack = (int*)(pt + 7 * p.pcap);
  s.misc = (int*)(base + p.o_misc);
  s.dacc = (double*)(base + p.o_misc + 32);
  s.dwarp = s.dacc + kNDiag;
  s.dd = (T*)(base + p.o_dd);
  s.dn = s.dd + (size_t)(p.ny > 1 ? p.RB : 1) * p.nx;
  return s;
}

// tables built in FP64 on the host (already in the working precision) and the constants
template <typename T>
__device__ void load_tables(const Params& p, const Sm<T>& s) {
  const int nyh = p.ny > 1 ? p.ny / 2 : 1;
  const int ncx = p.nx / 2 + nyh + p.nx / 2 + p.ny;
  const int nr = p.nx / 2 + p.ny;
  const Cx<T>* src = (const Cx<T>*)p.tables;
  for (int i = threadIdx.x; i < ncx; i += blockDim.x) s.twx[i] = src[i];
  const T* srcr = (const T*)(src + ncx);
  for (int i = threadIdx.x; i < nr; i += blockDim.x) s.kx[i] = srcr[i];
  if (threadIdx.x == 0) {
    T* c = s.cst;
    c[K_H] = T(p.h);
    c[K_INVH] = T(1.0 / p.h);
    c[K_HX] = T(p.hx);
    c[K_HY] = T(p.hy);
    c[K_D] = T(p.delta);
    c[K_DF] = T(p.delta_field);
    c[K_WSCALE] = T(1.0 / (p.hx * p.hy * p.delta));
    c[K_CX] = T(p.hx / p.h);
    c[K_CY] = T(p.hy / p.h);
    c[K_INVHX] = T(1.0 / p.hx);
    c[K_INVHY] = T(1.0 / p.hy);
    c[K_FLUX] = T(p.hx * p.hy * p.h);
    c[K_BEAM] = T(1.0 / (p.hx * p.hy * p.h));
    c[K_JREF] = T(p.jref);
    c[K_JSCALE] = T(4194304.0 / p.jref);   // 2^22 / jref
    c[K_JINV] = T(p.jref / 4194304.0);
    c[K_INVD] = p.delta > 0 ? T(1.0 / p.delta) : T(0);
    for (int i = 0; i < kMaxSpecies; ++i) {
      c[K_QM + i] = T(p.qm[i]);
      c[K_MOQ + i] = T(p.m_over_q[i]);
      c[K_QF + i] = T(p.Qf[i]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// phase timers (profiling builds only)
// ------------------------------------------------------------------------------------------
enum Phase { PH_A = 0, PH_B1, PH_BEAM, PH_FWD, PH_B2, PH_COLF, PH_SOLVE, PH_COLI, PH_SCAT, PH_B3,
             PH_INV, PH_B4, PH_E, PH_AG, PH_AM, PH_AD, PH_AW, PH_AR, PH_BF, PH_BI, PH_N };
// Thread 0 of each CTA adds the cycles of each phase straight into global memory (phase ph at
// word ph, PH_AW and PH_AR at 32 + ph): no per-phase registers are carried through the march.
#ifdef GEMPIC_PHASE_TIMERS
__device__ __forceinline__ int timer_word(int ph) { return ph >= PH_AW ? 32 + ph : ph; }
#define TIMER_DECL long long t_last = clock64();
#define TIMER_MARK(ph)                                                                \
  do {                                                                                \
    const long long t_now = clock64();                                                \
    if (threadIdx.x == 0 && p.timers)                                                 \
      atomicAdd(p.timers + timer_word(ph), (unsigned long long)(t_now - t_last));     \
    t_last = t_now;                                                                   \
  } while (0)
#else
#define TIMER_DECL
#define TIMER_MARK(ph) \
  do {                 \
  } while (0)
#endif
// timers inside the push (gather / arithmetic / deposit): their clock reads keep the compiler
// from interleaving the stages, so they are a separate profiling option
#if defined(GEMPIC_PHASE_TIMERS) && defined(GEMPIC_SUB_TIMERS)
#define SUB_DECL long long s_t0 = clock64();
#define SUB_MARK(i)                                                                 \
  do {                                                                              \
    const long long s_t1 = clock64();                                               \
    if (threadIdx.x == 0 && p.timers)                                               \
      atomicAdd(p.timers + PH_AG + (i), (unsigned long long)(s_t1 - s_t0));         \
    s_t0 = s_t1;                                                                    \
  } while (0)
#else
#define SUB_DECL
#define SUB_MARK(i) \
  do {              \
  } while (0)
#endif

// ------------------------------------------------------------------------------------------
// Forward transverse transform of the three current planes J (own rows) into the kx-owner
// CTAs' SC[0..2] (DSMEM).  stagger: apply exp(-i kx hx/2) to j_x (x-edge values).
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void st_cx(const cg::cluster_group& cl, Cx<T>* local, int r, int me,
                                      Cx<T> v) {
  Cx<T>* q = r == me ? local : cl.map_shared_rank(local, r);
  *q = v;
}

// Register path (nx = 32 R): task (row yl, pair pr) transforms u + i v of two real rows; the
// spectra split as U(k) = (Z(k) + conj Z(N-k))/2, V(k) = i (conj Z(N-k) - Z(k))/2.  With Z
// in lane order the partner N - k of register k2 > 0 is register R - k2 of lane l ^ 31, that
// of register 0 is register 0 of lane bitrev5(-bitrev5(l) mod 32); the lanes holding
// k < N/2 are the even ones.  Their values are staged in SR (free until the inverse
// transform) as rows [comp][k2][yl] of 16 + 1 entries (conflict-free both ways), then each
// element (comp, k, yl), yl fastest, goes to its kx owner: a warp's 32 stores go to one CTA.
template <typename T, int R>
__device__ void forward_rows_reg(const cg::cluster_group& cl, const Params& p, const Sm<T>& s,
                                 int me, bool stagger) {
  constexpr int N = 32 * R, NH = N / 2, SP = 17;
  constexpr int LR = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : 3;
  const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int ntask = 2 * p.RB;
  const int k1 = bitrev5(l);
  const int src0 = bitrev5((32 - k1) & 31);
  Cx<T>* stg = s.SR;      // [3][R][RB][SP]
  for (int task = warp; task < ntask; task += nwarps) {
    const int yl = task >> 1, pr = task & 1;
    const T* A = s.J + ((size_t)(pr == 0 ? 0 : 2) * p.JR + yl + p.JOFF) * N;
    const T* B = s.J + ((size_t)1 * p.JR + yl + p.JOFF) * N;
    Cx<T> a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = cx<T>(A[l + 32 * r], pr == 0 ? B[l + 32 * r] : T(0));
    fft_dif_lanes<T, R>(a, s.twx, false);
    Cx<T> zm[R];
    zm[0] = cx<T>(__shfl_sync(0xffffffffu, a[0].re, src0), __shfl_sync(0xffffffffu, a[0].im, src0));
#pragma unroll
    for (int k2 = 1; k2 < R; ++k2) zm[k2] = shfl_xor_cx(a[R - k2], 31);
    if (l & 1) continue;
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      const int k = k2 + R * k1;
      const Cx<T> zc = conjg(zm[k2]);
      Cx<T> X = T(0.5) * (a[k2] + zc);                  // spectrum of the real part
      const Cx<T> Y = T(0.5) * mul_i(zc - a[k2]);       // spectrum of the imaginary part
      if (pr == 0) {
        if (stagger) X = X * s.shx[k];
        stg[((0 * R + k2) * p.RB + yl) * SP + (l >> 1)] = X;
        stg[((1 * R + k2) * p.RB + yl) * SP + (l >> 1)] = Y;
      } else {
        stg[((2 * R + k2) * p.RB + yl) * SP + (l >> 1)] = X;
      }
    }
  }
  __syncthreads();
  const int total = 3 * NH * p.RB;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int yl = i & (p.RB - 1);
    const int rest = i >> p.logRB;
    const int k = rest & (NH - 1), c = rest / NH;
    const Cx<T> v = stg[((c * R + (k & (R - 1))) * p.RB + yl) * SP + (bitrev5(k >> LR) >> 1)];
    const int rd = k >> p.logKB, kxl = k & (p.KB - 1);
    st_cx(cl, s.SC + ((size_t)c * p.KB + kxl) * p.ny + (me << p.logRB) + yl, rd, me, v);
  }
}

// Length 128 with an even number of rows per band: the tasks pair the rows (j_x, j_y) of one
// y and the j_z rows of two y, each as u + i v of one transform, two tasks per warp.  A task's
// two current rows (dead after this phase) are its transform scratch; the split spectra
// U(k) = (Z(k) + conj Z(N-k))/2, V(k) = i (conj Z(N-k) - Z(k))/2 are staged in SR (free
// until the inverse transform) as [3][64][RB + 1] and sent with y fastest, so that a warp's
// distributed-shared stores go to one kx owner.
template <typename T>
__device__ void forward_rows_128(const cg::cluster_group& cl, const Params& p, const Sm<T>& s,
                                 int me, bool stagger) {
  constexpr int N = 128, NH = 64;
  const int warp = threadIdx.x >> 5, hf = (threadIdx.x >> 4) & 1, i = threadIdx.x & 15;
  const int nwarps = blockDim.x >> 5;
  const int ntask = p.RB + p.RB / 2;
  const int SP = p.RB + 1;
  Cx<T>* stg = s.SR;
  for (int t0 = 2 * warp; t0 < ntask; t0 += 2 * nwarps) {
    const int t = min(t0 + hf, ntask - 1);
    const bool live = t0 + hf < ntask;
    // rows of the pair and their (comp, y) destinations
    int ca, ya, cb, yb;
    if (t < p.RB) {
      ca = 0; ya = t; cb = 1; yb = t;
    } else {
      ca = 2; ya = 2 * (t - p.RB); cb = 2; yb = ya + 1;
    }
    T* A = s.J + ((size_t)ca * p.JR + ya + p.JOFF) * N;
    T* B = s.J + ((size_t)cb * p.JR + yb + p.JOFF) * N;
    Cx<T> a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = cx<T>(A[i + 16 * r], B[i + 16 * r]);
    Cx<T> z[8];
    Cx<T>* bufA = reinterpret_cast<Cx<T>*>(A);
    Cx<T>* bufB = reinterpret_cast<Cx<T>*>(B);
    fft128_h16<T>(a, bufA, bufB, s.twx, false, live, z);
    if (live) {
      const int k2 = i >> 1, j0 = i & 1;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int k = k2 + 8 * m + 64 * j0;
        if (k < 64) bufA[k] = z[m]; else bufB[k - 64] = z[m];
      }
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = i + 16 * q;
        const Cx<T> zk = bufA[k];
        const Cx<T> zc = conjg(k == 0 ? bufA[0] : bufB[64 - k]);        // conj Z(N - k)
        Cx<T> X = T(0.5) * (zk + zc);
        const Cx<T> Y = T(0.5) * mul_i(zc - zk);
        if (ca == 0 && stagger) X = X * s.shx[k];
        stg[((size_t)ca * NH + k) * SP + ya] = X;
        stg[((size_t)cb * NH + k) * SP + yb] = Y;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  const int total = 3 * NH * p.RB;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int yl = e & (p.RB - 1);
    const int rest = e >> p.logRB;
    const int k = rest & (NH - 1), c = rest >> 6;
    const Cx<T> v = stg[((size_t)c * NH + k) * SP + yl];
    const int rd = k >> p.logKB, kxl = k & (p.KB - 1);
    st_cx(cl, s.SC + ((size_t)c * p.KB + kxl) * p.ny + (me << p.logRB) + yl, rd, me, v);
  }
}

// the length-256 variants run out of line: inlined, their registers would spill the march's
// carried per-mode state at every length
template <typename T>
__device__ __noinline__ void forward_rows_r8(const cg::cluster_group& cl, const Params& p,
                                             const Sm<T>& s, int me, bool stagger) {
  forward_rows_reg<T, 8>(cl, p, s, me, stagger);
}

// SH = 1: the kernel instantiated for 128 x 128 grids with an even band (only the length-128
// transforms are compiled in; with the other lengths present the compiler schedules them
// markedly worse)
template <typename T, int SH>
__device__ void forward_rows(const cg::cluster_group& cl, const Params& p, const Sm<T>& s,
                             int me, bool stagger) {
  if constexpr (SH == 1) {
    forward_rows_128(cl, p, s, me, stagger);
  } else {
  if (p.lognx == 7 && p.ny > 1 && (p.RB & 1) == 0) {
    forward_rows_128(cl, p, s, me, stagger);
    return;
  }
  switch (p.lognx) {
    case 5: forward_rows_reg<T, 1>(cl, p, s, me, stagger); return;
    case 6: forward_rows_reg<T, 2>(cl, p, s, me, stagger); return;
    case 7: forward_rows_reg<T, 4>(cl, p, s, me, stagger); return;
    case 8: forward_rows_r8<T>(cl, p, s, me, stagger); return;
    default: break;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nxh = p.nx / 2;
  const int ntask = 2 * p.RB;                 // (row, pair): pair 0 = jx + i jy, 1 = jz
  if (warp >= p.nwork) return;
  for (int task = warp; task < ntask; task += p.nwork) {
    Cx<T>* w = s.workB + (size_t)warp * p.nx;
    const int yl = task >> 1, pr = task & 1;
    const T* a = s.J + ((size_t)(pr == 0 ? 0 : 2) * p.JR + yl + p.JOFF) * p.nx;
    const T* b = s.J + ((size_t)1 * p.JR + yl + p.JOFF) * p.nx;
    for (int x = lane; x < p.nx; x += 32) w[x] = cx<T>(a[x], pr == 0 ? b[x] : T(0));
    __syncwarp();
    warp_fft_r2(w, p.lognx, s.twx, false);
    const int y = (me << p.logRB) + yl;
    for (int k = lane; k < nxh; k += 32) {
      const Cx<T> zk = w[k];
      const Cx<T> zm = conjg(w[(p.nx - k) & (p.nx - 1)]);
      Cx<T> X = T(0.5) * (zk + zm);                     // spectrum of the real part
      const Cx<T> Y = T(0.5) * mul_i(zm - zk);          // spectrum of the imaginary part
      const int rd = k >> p.logKB, kxl = k & (p.KB - 1);
      if (pr == 0) {
        if (stagger) X = X * s.shx[k];
        st_cx(cl, s.SC + ((size_t)0 * p.KB + kxl) * p.ny + y, rd, me, X);
        st_cx(cl, s.SC + ((size_t)1 * p.KB + kxl) * p.ny + y, rd, me, Y);
      } else {
        st_cx(cl, s.SC + ((size_t)2 * p.KB + kxl) * p.ny + y, rd, me, X);
      }
    }
    __syncwarp();
  }
  }
}

// one column of length 32 R: forward from natural order to lane order, inverse from lane
// order to natural order; every lane rewrites the positions it read
template <typename T, int R>
__device__ __forceinline__ void col_fft_reg(Cx<T>* d, const Cx<T>* tw, bool inverse) {
  const int l = threadIdx.x & 31;
  Cx<T> a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) a[r] = d[l + 32 * r];
  if (inverse)
    fft_dit_lanes<T, R>(a, tw, true);
  else
    fft_dif_lanes<T, R>(a, tw, false);
#pragma unroll
  for (int r = 0; r < R; ++r) d[l + 32 * r] = a[r];
}

template <typename T>
__device__ __noinline__ void col_fft_r8(Cx<T>* d, const Cx<T>* tw, bool inverse) {
  col_fft_reg<T, 8>(d, tw, inverse);
}

// columns of length 128: two per warp, in place, natural order in and out
template <typename T>
__device__ void column_ffts_128(const Params& p, const Sm<T>& s, int c0, int c1, bool inverse) {
  const int warp = threadIdx.x >> 5, hf = (threadIdx.x >> 4) & 1, i = threadIdx.x & 15;
  const int nwarps = blockDim.x >> 5;
  const int ntask = (c1 - c0) << p.logKB;
  for (int t0 = 2 * warp; t0 < ntask; t0 += 2 * nwarps) {
    const int t = min(t0 + hf, ntask - 1);
    const bool live = t0 + hf < ntask;
    const int c = c0 + (t >> p.logKB), kxl = t & (p.KB - 1);
    Cx<T>* d = s.SC + ((size_t)c * p.KB + kxl) * 128;
    Cx<T> a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = d[i + 16 * r];
    Cx<T> b[8];
    fft128_h16<T>(a, d, d + 64, s.twy, inverse, live, b);
    if (live) {
      const int k2 = i >> 1, j0 = i & 1;
#pragma unroll
      for (int m = 0; m < 8; ++m) d[k2 + 8 * m + 64 * j0] = b[m];
    }
  }
}

// column FFTs of SC[c0..c1) (in place), forward or inverse; with a lane-order register FFT
// the spectra stay in lane order (position q holds ky_of_pos(q))
template <typename T, int SH>
__device__ void column_ffts(const Params& p, const Sm<T>& s, int c0, int c1, bool inverse) {
  if constexpr (SH == 1) {
    column_ffts_128(p, s, c0, c1, inverse);
  } else {
    if (p.ny == 1) return;
    if (p.logny == 7) {
      column_ffts_128(p, s, c0, c1, inverse);
      return;
    }
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int ntask = (c1 - c0) << p.logKB;
    for (int task = warp; task < ntask; task += nwarps) {
      const int c = c0 + (task >> p.logKB), kxl = task & (p.KB - 1);
      Cx<T>* d = s.SC + ((size_t)c * p.KB + kxl) * p.ny;
      switch (p.logny) {
        case 5: col_fft_reg<T, 1>(d, s.twy, inverse); break;
        case 6: col_fft_reg<T, 2>(d, s.twy, inverse); break;
        case 8: col_fft_r8<T>(d, s.twy, inverse); break;
        default: warp_fft_r2(d, p.logny, s.twy, inverse); break;
      }
    }
  }
}

// scatter the 6 inverse-column-transformed field spectra to the row owners' SR; the first row
// of each band also goes to the band below as its halo row FR - 1 = RB.  Element
// (comp, y, kxl), kxl fastest: with KB RB >= 32 a warp's stores go to one owner CTA.
template <typename T>
__device__ void scatter_to_rows(const cg::cluster_group& cl, const Params& p, const Sm<T>& s,
                                int me) {
  const int nxh = p.nx / 2;
  const int kx0 = me << p.logKB;
  const int total = 6 * p.ny * p.KB;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int kxl = i & (p.KB - 1);
    const int y = (i >> p.logKB) & (p.ny - 1);
    const int c = i >> (p.logKB + p.logny);
    const int ro = y >> p.logRB, yl = y & (p.RB - 1);
    const Cx<T> v = s.SC[((size_t)c * p.KB + kxl) * p.ny + y];
    Cx<T>* d0 = s.SR + ((size_t)c * p.FR + yl) * nxh + kx0 + kxl;
    *(ro == me ? d0 : cl.map_shared_rank(d0, ro)) = v;
    if (p.ny > 1 && yl == 0) {
      const int rb = (ro + p.C - 1) & (p.C - 1);
      Cx<T>* d1 = s.SR + ((size_t)c * p.FR + p.RB) * nxh + kx0 + kxl;
      *(rb == me ? d1 : cl.map_shared_rank(d1, rb)) = v;
    }
  }
}

// inverse row transforms: SR pairs (Ex,Ey), (Ez,Bx), (By,Bz) -> real rows of Fdst (own rows
// and the halo row); the field energy counts own rows only.  The spectrum X + iY (with
// X(-k) = conj X(k)) is formed while loading; the real and imaginary parts of the result
// are the two field rows.  Register path (nx = 32 R): each lane ends with R consecutive
// outputs and stores them as vectors.
template <typename T, int R>
__device__ void inverse_rows_reg(const Params& p, const Sm<T>& s, T* Fdst, T& fe) {
  constexpr int N = 32 * R;
  constexpr int nxh = N / 2;
  const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const T scale = T(1.0 / ((double)p.nx * (double)p.ny));
  const int ntask = 3 * p.FR;
  const int k1 = bitrev5(l);
  T acc = T(0);
  for (int t = warp; t < ntask; t += nwarps) {
    const int yl = t / 3, pr = t - 3 * (t / 3);
    const Cx<T>* X = s.SR + ((size_t)(2 * pr) * p.FR + yl) * nxh;
    const Cx<T>* Y = s.SR + ((size_t)(2 * pr + 1) * p.FR + yl) * nxh;
    Cx<T> a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = l + 32 * r;
      Cx<T> v = cx<T>(T(0), T(0));                        // Nyquist projected out
      if (j < nxh) {
        const Cx<T> x = X[j], y = Y[j];
        v = j == 0 ? cx<T>(x.re, y.re)                     // real DC of each field
                   : cx<T>(x.re - y.im, x.im + y.re);      // X + i Y
      } else if (j > nxh) {
        const Cx<T> x = X[N - j], y = Y[N - j];
        v = cx<T>(x.re + y.im, y.re - x.im);               // conj(X) + i conj(Y)
      }
      a[r] = v;
    }
    fft_dif_lanes<T, R>(a, s.twx, true);
    T va[R], vb[R];
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      va[k2] = a[k2].re * scale;
      vb[k2] = a[k2].im * scale;
    }
    st_run<T, R>(Fdst + ((size_t)(2 * pr) * p.FR + yl) * N + R * k1, va);
    st_run<T, R>(Fdst + ((size_t)(2 * pr + 1) * p.FR + yl) * N + R * k1, vb);
    if (yl < p.RB) {
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) acc += va[k2] * va[k2] + vb[k2] * vb[k2];
    }
  }
  fe += acc;
}

// Length 128: two tasks per warp (all 3 FR tasks in one round on 16 warps); a task's two
// spectrum rows X, Y are its transform scratch once read.
template <typename T>
__device__ void inverse_rows_128(const Params& p, const Sm<T>& s, T* Fdst, T& fe) {
  constexpr int N = 128, nxh = 64;
  const int warp = threadIdx.x >> 5, hf = (threadIdx.x >> 4) & 1, i = threadIdx.x & 15;
  const int nwarps = blockDim.x >> 5;
  const T scale = T(1.0 / ((double)p.nx * (double)p.ny));
  const int ntask = 3 * p.FR;
  T acc = T(0);
  for (int t0 = 2 * warp; t0 < ntask; t0 += 2 * nwarps) {
    const int t = min(t0 + hf, ntask - 1);
    const bool live = t0 + hf < ntask;
    const int yl = t / 3, pr = t - 3 * (t / 3);
    Cx<T>* X = s.SR + ((size_t)(2 * pr) * p.FR + yl) * nxh;
    Cx<T>* Y = s.SR + ((size_t)(2 * pr + 1) * p.FR + yl) * nxh;
    Cx<T> a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int n = i + 16 * r;
      Cx<T> v = cx<T>(T(0), T(0));                          // Nyquist projected out
      if (n < nxh) {
        const Cx<T> x = X[n], y = Y[n];
        v = n == 0 ? cx<T>(x.re, y.re)                       // real DC of each field
                   : cx<T>(x.re - y.im, x.im + y.re);        // X + i Y
      } else if (n > nxh) {
        const Cx<T> x = X[N - n], y = Y[N - n];
        v = cx<T>(x.re + y.im, y.re - x.im);                 // conj(X) + i conj(Y)
      }
      a[r] = v;
    }
    Cx<T> b[8];
    fft128_h16<T>(a, X, Y, s.twx, true, live, b);
    if (live) {
      const int k2 = i >> 1, j0 = i & 1;
      T* A = Fdst + ((size_t)(2 * pr) * p.FR + yl) * N;
      T* B = Fdst + ((size_t)(2 * pr + 1) * p.FR + yl) * N;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int k = k2 + 8 * m + 64 * j0;
        const T va = b[m].re * scale, vb = b[m].im * scale;
        A[k] = va;
        B[k] = vb;
        if (yl < p.RB) acc += va * va + vb * vb;
      }
    }
  }
  fe += acc;
}

template <typename T>
__device__ __noinline__ void inverse_rows_r8(const Params& p, const Sm<T>& s, T* Fdst, T& fe) {
  inverse_rows_reg<T, 8>(p, s, Fdst, fe);
}

template <typename T, int SH>
__device__ void inverse_rows(const Params& p, const Sm<T>& s, T* Fdst, T& fe) {
  if constexpr (SH == 1) {
    inverse_rows_128<T>(p, s, Fdst, fe);
  } else {
    switch (p.lognx) {
      case 5: inverse_rows_reg<T, 1>(p, s, Fdst, fe); return;
      case 6: inverse_rows_reg<T, 2>(p, s, Fdst, fe); return;
      case 7: inverse_rows_128<T>(p, s, Fdst, fe); return;
      case 8: inverse_rows_r8<T>(p, s, Fdst, fe); return;
      default: break;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nxh = p.nx / 2;
    const T scale = T(1.0 / ((double)p.nx * (double)p.ny));
    const int ntask = 3 * p.FR;
    for (int task = (warp < p.nwork ? warp : ntask); task < ntask; task += p.nwork) {
      Cx<T>* w = s.workD + (size_t)warp * p.nx;
      const int yl = task / 3, pr = task - 3 * yl;
      const Cx<T>* X = s.SR + ((size_t)(2 * pr) * p.FR + yl) * nxh;
      const Cx<T>* Y = s.SR + ((size_t)(2 * pr + 1) * p.FR + yl) * nxh;
      for (int k = lane; k < nxh; k += 32) {
        Cx<T> x = X[k], y = Y[k];
        if (k == 0) {
          w[0] = cx<T>(x.re, y.re);                         // real DC of each field
        } else {
          w[k] = cx<T>(x.re - y.im, x.im + y.re);           // X + i Y
          w[p.nx - k] = cx<T>(x.re + y.im, y.re - x.im);    // conj(X) + i conj(Y)
        }
      }
      if (lane == 0) w[nxh] = cx<T>(T(0), T(0));            // Nyquist projected out
      __syncwarp();
      warp_fft_r2(w, p.lognx, s.twx, true);
      T* a = Fdst + ((size_t)(2 * pr) * p.FR + yl) * p.nx;
      T* b = Fdst + ((size_t)(2 * pr + 1) * p.FR + yl) * p.nx;
      const bool own = yl < p.RB;
      for (int x = lane; x < p.nx; x += 32) {
        const T va = w[x].re * scale, vb = w[x].im * scale;
        a[x] = va;
        b[x] = vb;
        if (own) fe += va * va + vb * vb;
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------------------------------
// Gather and deposit.  Fast path: a particle in the CTA's own rows reads fields of rows
// yl, yl + 1 (halo) and deposits into current rows yl - 1 .. yl + 2, all in its own shared
// memory.  Generic path (stored particles, particles outside the band, moves reaching past the
// halo): any row of the cluster through distributed shared memory.
// ------------------------------------------------------------------------------------------
template <typename T>
struct RowRef {
  uint32_t a;        // address of (comp 0, row, col 0) in the owner's window (or local)
  bool remote;
};

// row y (global) of a plane set whose own row 0 sits at index `off` of `rows` rows per comp
template <typename T>
__device__ __forceinline__ RowRef<T> row_ref(const Params& p, const T* base, int rows, int off,
                                             int y, int me) {
  const int r = y >> p.logRB;
  const int yl = (y & (p.RB - 1)) + off;
  (void)rows;
  uint32_t a = sh_addr(base + (size_t)yl * p.nx);
  RowRef<T> rr;
  rr.remote = r != me;
  rr.a = rr.remote ? cluster_addr(a, r) : a;
  return rr;
}

template <typename T>
__device__ __forceinline__ T row_ld(const RowRef<T>& rr, uint32_t off_elems) {
  const uint32_t a = rr.a + off_elems * (uint32_t)sizeof(T);
  return rr.remote ? ldc(a, T(0)) : lds(a, T(0));
}

template <typename T>
__device__ __forceinline__ void row_red(const RowRef<T>& rr, uint32_t off_elems, T v) {
  const uint32_t a = rr.a + off_elems * (uint32_t)sizeof(T);
  if (rr.remote)
    red_cluster(a, v);
  else
    red_local(a, v);
}

// CIC gather of the 6 fields at (ix + fx, iy + fy), any row of the cluster
template <typename T>
__device__ __forceinline__ void gather6_g(const Params& p, const T* Fb, int ix, T fx, int iy, T fy,
                                          int me, T* out) {
  const int ix1 = (ix + 1) & (p.nx - 1);
  const uint32_t cs = (uint32_t)(p.FR * p.nx);     // component stride
  if (p.ny == 1) {
    const uint32_t a = sh_addr(Fb);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const uint32_t b = a + (c * cs) * (uint32_t)sizeof(T);
      out[c] = (T(1) - fx) * lds(b + ix * (uint32_t)sizeof(T), T(0)) +
               fx * lds(b + ix1 * (uint32_t)sizeof(T), T(0));
    }
    return;
  }
  const int iy1 = (iy + 1) & (p.ny - 1);
  const RowRef<T> r0 = row_ref(p, Fb, p.FR, 0, iy, me);
  const RowRef<T> r1 = row_ref(p, Fb, p.FR, 0, iy1, me);
  const T w00 = (T(1) - fx) * (T(1) - fy), w10 = fx * (T(1) - fy);
  const T w01 = (T(1) - fx) * fy, w11 = fx * fy;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const uint32_t o = c * cs;
    out[c] = ((w00 * row_ld(r0, o + ix) + w10 * row_ld(r0, o + ix1)) + w01 * row_ld(r1, o + ix)) +
             w11 * row_ld(r1, o + ix1);
  }
}

// the same for a particle in own row yl (rows yl and yl + 1 <= RB are local)
template <typename T>
__device__ __forceinline__ void gather6_l(const Params& p, const T* Fb, int ix, T fx, int yl, T fy,
                                          T* out) {
  const int ix1 = (ix + 1) & (p.nx - 1);
  const uint32_t cs = (uint32_t)(p.FR * p.nx) * (uint32_t)sizeof(T);
  const uint32_t a0 = sh_addr(Fb + (size_t)yl * p.nx);
  const uint32_t i0 = ix * (uint32_t)sizeof(T), i1 = ix1 * (uint32_t)sizeof(T);
  if (p.ny == 1) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const uint32_t b = a0 + c * cs;
      out[c] = (T(1) - fx) * lds(b + i0, T(0)) + fx * lds(b + i1, T(0));
    }
    return;
  }
  const uint32_t a1 = a0 + (uint32_t)p.nx * (uint32_t)sizeof(T);
  const T w00 = (T(1) - fx) * (T(1) - fy), w10 = fx * (T(1) - fy);
  const T w01 = (T(1) - fx) * fy, w11 = fx * fy;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const uint32_t b0 = a0 + c * cs, b1 = a1 + c * cs;
    out[c] = ((w00 * lds(b0 + i0, T(0)) + w10 * lds(b0 + i1, T(0))) + w01 * lds(b1 + i0, T(0))) +
             w11 * lds(b1 + i1, T(0));
  }
}

// Deposit targets.  Sink<T, true>: own current rows (row index relative to the particle's
// row, band rows -1 .. RB + 1), local shared reductions with precomputed addresses; in FP32
// a contribution below jref goes to the 32-bit fixed-point accumulators (native integer
// reductions, exact sums, at most 2^9 such contributions per node), a larger one to the float
// accumulators.  Sink<T, false>: any global row, into the own rows of the CTA that owns it; in
// FP32 below jref through the owner's fixed-point accumulators (a native distributed-shared
// integer reduction; the float one is a compare-and-swap loop some 40 times slower).
template <typename T, bool LOCAL>
struct Sink;

template <typename T>
struct Sink<T, true> {
  uint32_t fbase, ibase;     // address of (comp 0, particle row, col 0): float / fixed point
  uint32_t cstride, rstride; // bytes per component, per row
  T jref, jscale;
  __device__ __forceinline__ Sink(const Params& p, const Sm<T>& s, int yrow0) {
    const uint32_t off = (uint32_t)((yrow0 + p.JOFF) * p.nx) * (uint32_t)sizeof(T);
    fbase = sh_addr(s.J) + off;
    ibase = sh_addr(s.Jint) + (uint32_t)((yrow0 + p.JOFF) * p.nx) * 4u;
    cstride = (uint32_t)(p.JR * p.nx) * (uint32_t)sizeof(T);
    rstride = (uint32_t)p.nx * (uint32_t)sizeof(T);
    jref = s.cst[K_JREF];
    jscale = s.cst[K_JSCALE];
  }
  __device__ __forceinline__ void add(int comp, int yrow, int x, T v) const {
    if (v == T(0)) return;
    const uint32_t off = (uint32_t)comp * cstride + (uint32_t)(yrow * (int)rstride) +
                         (uint32_t)x * (uint32_t)sizeof(T);
    if constexpr (sizeof(T) == 4) {
      if (fabsf(v) < jref) {
        red_local_u32(ibase + off, __float2int_rn(v * jscale));
        return;
      }
    }
    red_local(fbase + off, v);
  }
};

template <typename T>
struct Sink<T, false> {
  const Params& p;
  const T* J;
  const int* Jint;
  int me, y0;                // global row of the particle
  T jref, jscale;
  __device__ __forceinline__ void add(int comp, int yrow, int x, T v) const {
    if (v == T(0)) return;
    const int y = (yrow + y0) & (p.ny - 1);
    if constexpr (sizeof(T) == 4) {
      if (fabsf(v) < jref) {
        const int r = y >> p.logRB;
        const uint32_t a =
            sh_addr(Jint + ((size_t)comp * p.JR + (y & (p.RB - 1)) + p.JOFF) * p.nx + x);
        const int q = __float2int_rn(v * jscale);
        if (r == me)
          red_local_u32(a, q);
        else
          red_cluster_u32(cluster_addr(a, r), q);
        return;
      }
    }
    const RowRef<T> rr = row_ref(p, J, p.JR, p.JOFF, y, me);
    row_red(rr, (uint32_t)(comp * p.JR * p.nx + x), v);
  }
};

// Esirkepov (Comput. Phys. Commun. 135, 2001) transverse current of a move (X0,Y0)->(X1,Y1)
// in cell units relative to node (ix, row 0 of the sink); w is the (rho - j_z) weight.  With
// D = w S the deposit satisfies (D_new - D_old) + h div J = 0 on every node.  A sub-step that
// stays inside one cell column (row) has no current on its second x-edge (y-edge row): those
// sums vanish exactly and are set to zero rather than left to rounding, so they deposit
// nothing.
constexpr int kMaxSub = 256;   // sub-steps of one Esirkepov move at most

template <typename T, bool LOCAL>
__device__ void esirkepov(const Params& p, const Sm<T>& s, const Sink<T, LOCAL>& sk, int ix,
                          T X0, T Y0, T X1, T Y1, T w, T dyo) {
  const T invh = s.cst[K_INVH];
  const T dX = X1 - X0;
  const T dY = Y1 - Y0;
  const T m = fmax(fabs(dX), fabs(dY));
  // a move of more than kMaxSub cells across one slice only comes from a runaway momentum:
  // its sub-steps are capped (the deposit is then wrong, and the error word says so)
  if (m > T(kMaxSub)) atomicOr(p.err, ERR_NONFINITE);
  const int nsub = m > T(1) ? (int)fmin(ceil(m), T(kMaxSub)) : 1;
  const T cx_ = -(w * s.cst[K_CX]);
  const T cy_ = -(w * s.cst[K_CY]);
  const int mx = p.nx - 1;
  for (int sb = 0; sb < nsub; ++sb) {
    const T xa = X0 + dX * (T(sb) / T(nsub));
    const T xb = X0 + dX * (T(sb + 1) / T(nsub));
    // 3-node window from bx = floor(min(xa, xb)); with u = x - bx in [0, 2) the linear shape
    // S(u, a) = max(0, 1 - |u - a|) is (1 - u, u, 0) on [0, 1) and (0, 2 - u, u - 1) on [1, 2)
    const T bx = floor(fmin(xa, xb));
    const T ua = xa - bx, ub = xb - bx;
    const T S0x0 = fmax(T(0), T(1) - ua), S0x1 = T(1) - fabs(ua - T(1)), S0x2 = fmax(T(0), ua - T(1));
    const T S1x0 = fmax(T(0), T(1) - ub), S1x1 = T(1) - fabs(ub - T(1)), S1x2 = fmax(T(0), ub - T(1));
    const bool crossx = floor(fmax(xa, xb)) != bx;
    // x-edge currents: cumulative sums of S1x - S0x; the second edge carries current only
    // when the sub-step crosses into the third node (else its sum vanishes exactly)
    const T dS0 = S1x0 - S0x0;
    const T ex0 = cx_ * dS0;
    const T ex1 = crossx ? cx_ * (dS0 + (S1x1 - S0x1)) : T(0);
    const T hx0 = T(0.5) * (S0x0 + S1x0), hx1 = T(0.5) * (S0x1 + S1x1), hx2 = T(0.5) * (S0x2 + S1x2);
    const int gx = ix + (int)bx;
    const int x0 = gx & mx, x1 = (gx + 1) & mx, x2 = (gx + 2) & mx;
    if (p.ny == 1) {
      sk.add(0, 0, x0, ex0);
      sk.add(0, 0, x1, ex1);
      const T vy = w * ((dyo / T(nsub)) * invh);
      sk.add(1, 0, x0, vy * hx0);
      sk.add(1, 0, x1, vy * hx1);
      sk.add(1, 0, x2, vy * hx2);
      continue;
    }
    const T ya = Y0 + dY * (T(sb) / T(nsub));
    const T yb = Y0 + dY * (T(sb + 1) / T(nsub));
    const T by = floor(fmin(ya, yb));
    const T va = ya - by, vb = yb - by;
    const T S0y0 = fmax(T(0), T(1) - va), S0y1 = T(1) - fabs(va - T(1)), S0y2 = fmax(T(0), va - T(1));
    const T S1y0 = fmax(T(0), T(1) - vb), S1y1 = T(1) - fabs(vb - T(1)), S1y2 = fmax(T(0), vb - T(1));
    const bool crossy = floor(fmax(ya, yb)) != by;
    const T dT0 = S1y0 - S0y0;
    const T ey0 = cy_ * dT0;
    const T ey1 = crossy ? cy_ * (dT0 + (S1y1 - S0y1)) : T(0);
    const T hy0 = T(0.5) * (S0y0 + S1y0), hy1 = T(0.5) * (S0y1 + S1y1), hy2 = T(0.5) * (S0y2 + S1y2);
    const int gy = (int)by;
    // j_x on x-edges (a = 0, 1) of rows b = 0, 1, 2; j_y on y-edges (b = 0, 1) of columns
    // a = 0, 1, 2 (Esirkepov's W = (S1 - S0) along the current times the mean shape across)
    sk.add(0, gy, x0, ex0 * hy0);
    sk.add(0, gy, x1, ex1 * hy0);
    sk.add(0, gy + 1, x0, ex0 * hy1);
    sk.add(0, gy + 1, x1, ex1 * hy1);
    sk.add(0, gy + 2, x0, ex0 * hy2);
    sk.add(0, gy + 2, x1, ex1 * hy2);
    sk.add(1, gy, x0, ey0 * hx0);
    sk.add(1, gy, x1, ey0 * hx1);
    sk.add(1, gy, x2, ey0 * hx2);
    sk.add(1, gy + 1, x0, ey1 * hx0);
    sk.add(1, gy + 1, x1, ey1 * hx1);
    sk.add(1, gy + 1, x2, ey1 * hx2);
  }
}

// Fixed-point quantum of v (|v js| < 2^22): round(v js) to the nearest integer, ties to even,
// by adding 1.5 2^23 in one rounding (the sum's unit in the last place is 1, so its low
// mantissa bits hold the integer) -- an FMA and an integer subtract instead of a conversion.
__device__ __forceinline__ int fixq(float v, float js) {
  return __float_as_int(fmaf(v, js, 12582912.0f)) - 0x4B400000;
}

// FP32 deposit of a move that needs no sub-steps (|dX|, |dY| <= 1) and whose contributions are
// all below jref: the Esirkepov and CIC values of the general path, added to the fixed-point
// accumulators by reductions predicated on a nonzero quantum (no branches).  Every value is a
// shape weight <= 1 times one of ex0, ex1, ey0, ey1 (vy in 2-D) or vz, which bounds them all.
// Returns false (nothing deposited) where it does not apply.
template <typename T>
__device__ __forceinline__ bool deposit_fixed(const Params& p, const Sm<T>& s,
                                              const Sink<T, true>& sk, int ix, T X0, T Y0, T X1,
                                              T Y1, T w, T dyo, T vz) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    const T dX = X1 - X0, dY = Y1 - Y0;
    if (!(fmax(fabs(dX), fabs(dY)) <= T(1))) return false;
    const int mx = p.nx - 1;
    const T bx = floor(fmin(X0, X1));
    const T ua = X0 - bx, ub = X1 - bx;
    const T S0x0 = fmax(T(0), T(1) - ua), S0x1 = T(1) - fabs(ua - T(1)), S0x2 = fmax(T(0), ua - T(1));
    const T S1x0 = fmax(T(0), T(1) - ub), S1x1 = T(1) - fabs(ub - T(1)), S1x2 = fmax(T(0), ub - T(1));
    const bool crossx = floor(fmax(X0, X1)) != bx;
    const T dS0 = S1x0 - S0x0;
    const T cx_ = -(w * s.cst[K_CX]);
    const T ex0 = cx_ * dS0;
    const T ex1 = crossx ? cx_ * (dS0 + (S1x1 - S0x1)) : T(0);
    const T hx0 = T(0.5) * (S0x0 + S1x0), hx1 = T(0.5) * (S0x1 + S1x1), hx2 = T(0.5) * (S0x2 + S1x2);
    const int gx = ix + (int)bx;
    const uint32_t o0 = (uint32_t)(gx & mx) * 4u, o1 = (uint32_t)((gx + 1) & mx) * 4u,
                   o2 = (uint32_t)((gx + 2) & mx) * 4u;
    // CIC of j_z at the end point
    const T fX1 = floor(X1), fx = X1 - fX1;
    const int cz = ix + (int)fX1;
    const uint32_t z0 = (uint32_t)(cz & mx) * 4u, z1 = (uint32_t)((cz + 1) & mx) * 4u;
    const T js = sk.jscale;
    const uint32_t cs = sk.cstride, rs = sk.rstride;
    if (p.ny == 1) {
      const T vy = w * (dyo * s.cst[K_INVH]);
      const T bnd = fmax(fmax(fabs(ex0), fabs(ex1)), fmax(fabs(vy), fabs(vz)));
      if (!(bnd < sk.jref)) return false;
      const uint32_t b = sk.ibase;
      red_local_u32_nz(b + o0, fixq(ex0, js));
      red_local_u32_nz(b + o1, fixq(ex1, js));
      red_local_u32_nz(b + cs + o0, fixq(vy * hx0, js));
      red_local_u32_nz(b + cs + o1, fixq(vy * hx1, js));
      red_local_u32_nz(b + cs + o2, fixq(vy * hx2, js));
      red_local_u32_nz(b + 2 * cs + z0, fixq((T(1) - fx) * vz, js));
      red_local_u32_nz(b + 2 * cs + z1, fixq(fx * vz, js));
      return true;
    }
    const T by = floor(fmin(Y0, Y1));
    const T va = Y0 - by, vb = Y1 - by;
    const T S0y0 = fmax(T(0), T(1) - va), S0y1 = T(1) - fabs(va - T(1)), S0y2 = fmax(T(0), va - T(1));
    const T S1y0 = fmax(T(0), T(1) - vb), S1y1 = T(1) - fabs(vb - T(1)), S1y2 = fmax(T(0), vb - T(1));
    const bool crossy = floor(fmax(Y0, Y1)) != by;
    const T dT0 = S1y0 - S0y0;
    const T cy_ = -(w * s.cst[K_CY]);
    const T ey0 = cy_ * dT0;
    const T ey1 = crossy ? cy_ * (dT0 + (S1y1 - S0y1)) : T(0);
    const T hy0 = T(0.5) * (S0y0 + S1y0), hy1 = T(0.5) * (S0y1 + S1y1), hy2 = T(0.5) * (S0y2 + S1y2);
    const T bnd = fmax(fmax(fmax(fabs(ex0), fabs(ex1)), fmax(fabs(ey0), fabs(ey1))), fabs(vz));
    if (!(bnd < sk.jref)) return false;
    const T fY1 = floor(Y1), fy = Y1 - fY1;
    const uint32_t r0 = sk.ibase + (uint32_t)((int)by * (int)rs);
    const uint32_t r1 = r0 + rs, r2 = r1 + rs;
    red_local_u32_nz(r0 + o0, fixq(ex0 * hy0, js));
    red_local_u32_nz(r0 + o1, fixq(ex1 * hy0, js));
    red_local_u32_nz(r1 + o0, fixq(ex0 * hy1, js));
    red_local_u32_nz(r1 + o1, fixq(ex1 * hy1, js));
    red_local_u32_nz(r2 + o0, fixq(ex0 * hy2, js));
    red_local_u32_nz(r2 + o1, fixq(ex1 * hy2, js));
    red_local_u32_nz(r0 + cs + o0, fixq(ey0 * hx0, js));
    red_local_u32_nz(r0 + cs + o1, fixq(ey0 * hx1, js));
    red_local_u32_nz(r0 + cs + o2, fixq(ey0 * hx2, js));
    red_local_u32_nz(r1 + cs + o0, fixq(ey1 * hx0, js));
    red_local_u32_nz(r1 + cs + o1, fixq(ey1 * hx1, js));
    red_local_u32_nz(r1 + cs + o2, fixq(ey1 * hx2, js));
    const uint32_t q0 = sk.ibase + 2 * cs + (uint32_t)((int)fY1 * (int)rs), q1 = q0 + rs;
    red_local_u32_nz(q0 + z0, fixq(((T(1) - fx) * (T(1) - fy)) * vz, js));
    red_local_u32_nz(q0 + z1, fixq((fx * (T(1) - fy)) * vz, js));
    red_local_u32_nz(q1 + z0, fixq(((T(1) - fx) * fy) * vz, js));
    red_local_u32_nz(q1 + z1, fixq((fx * fy) * vz, js));
    return true;
  }
}

// CIC deposit of value v at (X, Y) relative to node (ix, row 0 of the sink) into comp
template <typename T, bool LOCAL>
__device__ __forceinline__ void cic_add(const Params& p, const Sink<T, LOCAL>& sk, int comp,
                                        int ix, T X, T Y, T v) {
  const T i0 = floor(X);
  const T fx = X - i0;
  const int gx = (ix + (int)i0) & (p.nx - 1);
  const int gx1 = (gx + 1) & (p.nx - 1);
  if (p.ny == 1) {
    sk.add(comp, 0, gx, (T(1) - fx) * v);
    sk.add(comp, 0, gx1, fx * v);
    return;
  }
  const T j0 = floor(Y);
  const T fy = Y - j0;
  const int gy = (int)j0;
  sk.add(comp, gy, gx, ((T(1) - fx) * (T(1) - fy)) * v);
  sk.add(comp, gy, gx1, (fx * (T(1) - fy)) * v);
  sk.add(comp, gy + 1, gx, ((T(1) - fx) * fy) * v);
  sk.add(comp, gy + 1, gx1, (fx * fy) * v);
}

// ------------------------------------------------------------------------------------------
// One streaming push from the plane above to plane n (zeta distance d): gather at the
// particle, budget rule (Eq. trap2), two-pass Boris, deposit.  Returns true if trapped; on
// return the particle state holds the new values (cell-relative position at plane n, or at
// zeta_n + (d - hc) when trapped, reported through fz_trap).
// ------------------------------------------------------------------------------------------
template <typename T>
struct PState {
  int ix, iy, sp;
  T fx, fy;
  V3<T> u;
  T sig, q;
};

template <typename T>
struct SliceAcc {     // per-thread, per-slice diagnostics in the working precision
  T kin, flux;
  int push;
};

// LAW: 0 = GT2, 1 = GT1, -1 = either (read from p.gt1); RES: the continuity-residual
// deposit may be compiled in (taken when p.resid)
// CIC of v at node (ix, iy) + (fx, fy) into a plane of own rows [RBe][nx], reduced into the
// CTA that owns each row (verification mode)
template <typename T>
__device__ __forceinline__ void res_cic(const Params& p, T* plane, int me, int ix, int iy, T fx,
                                        T fy, T v) {
  const int ix1 = (ix + 1) & (p.nx - 1);
  if (p.ny == 1) {
    const uint32_t b = sh_addr(plane);
    red_local(b + (uint32_t)(ix * sizeof(T)), v * (T(1) - fx));
    red_local(b + (uint32_t)(ix1 * sizeof(T)), v * fx);
    return;
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int y = (iy + t) & (p.ny - 1);
    const T wy = t == 0 ? T(1) - fy : fy;
    const int r = y >> p.logRB;
    const uint32_t a = sh_addr(plane + (size_t)(y & (p.RB - 1)) * p.nx);
    const uint32_t a0 = a + (uint32_t)(ix * sizeof(T)), a1 = a + (uint32_t)(ix1 * sizeof(T));
    const T v0 = v * ((T(1) - fx) * wy), v1 = v * (fx * wy);
    if (r == me) {
      red_local(a0, v0);
      red_local(a1, v1);
    } else {
      red_cluster(cluster_addr(a0, r), v0);
      red_cluster(cluster_addr(a1, r), v1);
    }
  }
}

template <typename T, int LAW, bool RES>
__device__ bool stream_push(const Params& p, const Sm<T>& s, const T* Fcur, PState<T>& P, T d,
                            int me, T& fz_trap, SliceAcc<T>& acc, T* dn) {
  SUB_DECL
  const int yl = P.iy - (me << p.logRB);
  const bool own = p.ny == 1 || (yl >= 0 && yl < p.RB);
  T E[6];
  if (own)
    gather6_l(p, Fcur, P.ix, P.fx, p.ny == 1 ? 0 : yl, P.fy, E);
  else
    gather6_g(p, Fcur, P.ix, P.fx, P.iy, P.fy, me, E);
  SUB_MARK(0);
  const T D = s.cst[K_D];
  const T invh = s.cst[K_INVH];
  const T qm = s.cst[K_QM + P.sp];
  V3<T> u = P.u;
  const T g0 = gamma_of(u);
  const T gmu0 = gamma_minus_uz(u, g0);
  // the step ends where the s-budget reaches Delta: GT2 (Eq. trap2) ds~ = v_z dt, so
  // -dzeta <= (Delta - sigma)(gamma - u_z)/u_z; GT1 (Eq. trap1) ds = dt, so
  // -dzeta <= (Delta - sigma)(gamma - u_z)/gamma
  const bool gt1 = LAW < 0 ? p.gt1 != 0 : LAW == 1;
  const T vs = gt1 ? g0 : u.z;
  T hlim = vs > T(0) ? (D - P.sig) * gmu0 / vs : T(INFINITY);
  hlim = fmax(hlim, T(0));
  const bool trap = hlim < d;
  const T hc = trap ? hlim : d;
  // two passes: the lab time of the step is evaluated at the step's mean momentum
  const T dt1 = hc * g0 / gmu0;
  const V3<T> us = boris(u, E, E + 3, qm, dt1);
  const V3<T> ub{T(0.5) * (u.x + us.x), T(0.5) * (u.y + us.y), T(0.5) * (u.z + us.z)};
  const T gb = gamma_of(ub);
  const T dt2 = hc * gb / gamma_minus_uz(ub, gb);
  const V3<T> un = boris(u, E, E + 3, qm, dt2);
  const T gn = gamma_of(un);
  const T hden = hc * rcp(gamma_minus_uz(un, gn));    // h / (gamma - u_z)
  const T dx = hden * un.x, dy = hden * un.y, ds = hden * un.z;
  // deposit: w = Q/(hx hy Delta) is the particle's (rho - j_z) density weight (Sec. 5.1)
  const T w = P.q * s.cst[K_WSCALE];
  const T X1 = P.fx + dx * s.cst[K_INVHX];
  const T Y1 = p.ny > 1 ? P.fy + dy * s.cst[K_INVHY] : P.fy;
  SUB_MARK(1);
  // the move stays inside the band's current rows -1 .. RB + 1 -> local reductions only
  const T lo = floor(fmin(P.fy, Y1)), hi = floor(fmax(P.fy, Y1));
  const bool local = own && (p.ny == 1 || (yl + (int)lo >= -1 && yl + (int)hi + 2 <= p.RB + 1));
  if (local) {
    const Sink<T, true> sk(p, s, p.ny == 1 ? 0 : yl);
    const T vz = w * ds * invh;
    if (!deposit_fixed(p, s, sk, P.ix, P.fx, P.fy, X1, Y1, w, dy, vz)) {
      esirkepov(p, s, sk, P.ix, P.fx, P.fy, X1, Y1, w, dy);
      cic_add(p, sk, 2, P.ix, X1, Y1, vz);
    }
  } else {
    const Sink<T, false> sk{p, s.J, s.Jint, me, P.iy, s.cst[K_JREF], s.cst[K_JSCALE]};
    esirkepov(p, s, sk, P.ix, P.fx, P.fy, X1, Y1, w, dy);
    cic_add(p, sk, 2, P.ix, X1, Y1, w * ds * invh);
  }
  SUB_MARK(2);
  if constexpr (RES) {
    if (p.resid) {
      // verification mode: +w CIC at the start of the move and -w at its end (continuity
      // residual), +w at the end of a move that reaches the plane (its (rho - j_z) density,
      // Gauss residual), into the own rows of the rows' owners
      const T fXe = floor(X1), fe = X1 - fXe;
      const int ie = (P.ix + (int)fXe) & (p.nx - 1);
      int je = 0;
      T ge = T(0);
      if (p.ny > 1) {
        const T fYe = floor(Y1);
        ge = Y1 - fYe;
        je = (P.iy + (int)fYe) & (p.ny - 1);
      }
      res_cic(p, s.dd, me, P.ix, P.iy, P.fx, P.fy, w);
      res_cic(p, s.dd, me, ie, je, fe, ge, -w);
      if (!trap) res_cic(p, dn, me, ie, je, fe, ge, w);
    }
  }
  // diagnostics: kinetic energy N m (gamma-1) dt/Delta, (rho - j_z) flux through plane n
  const T dtl = hden * gn;
  acc.kin += P.q * s.cst[K_MOQ + P.sp] * gamma_minus_one(un, gn) * dtl * s.cst[K_INVD];
  if (!trap) acc.flux += w;
  acc.push += 1;
  // new cell-relative position
  const T fX = floor(X1);
  P.ix = (P.ix + (int)fX) & (p.nx - 1);
  P.fx = X1 - fX;
  if (p.ny > 1) {
    const T fY = floor(Y1);
    P.iy = (P.iy + (int)fY) & (p.ny - 1);
    P.fy = Y1 - fY;
  }
  P.u = un;
  P.sig = P.sig + (gt1 ? dtl : ds);
  fz_trap = (d - hc) * invh;
  return trap;
}

// write a particle into a stored store (ring slot, bucket); false on overflow
template <typename T>
__device__ bool store_append(const PartStore& S, const Params& p, int slot, int bucket,
                             const PState<T>& P, T fz) {
  int* cnt = S.cnt + (size_t)slot * p.nz + bucket;
  const int i = atomicAdd(cnt, 1);
  if (i >= p.bcap) return false;
  const size_t e = ((size_t)slot * p.nz + bucket) * p.bcap + i;
  S.cell[e] = P.ix | (P.iy << 10) | (P.sp << 20);
  ((T*)S.fx)[e] = P.fx;
  ((T*)S.fy)[e] = P.fy;
  ((T*)S.fz)[e] = fz;
  ((T*)S.ux)[e] = P.u.x;
  ((T*)S.uy)[e] = P.u.y;
  ((T*)S.uz)[e] = P.u.z;
  ((T*)S.q)[e] = P.q;
  return true;
}

template <typename T>
__device__ PState<T> store_read(const PartStore& S, const Params& p, size_t e, T& fz) {
  PState<T> P;
  const int c = ldcg(S.cell + e);
  P.ix = c & 1023;
  P.iy = (c >> 10) & 1023;
  P.sp = (c >> 20) & 3;
  P.fx = ldcg((const T*)S.fx + e);
  P.fy = ldcg((const T*)S.fy + e);
  fz = ldcg((const T*)S.fz + e);
  P.u = V3<T>{ldcg((const T*)S.ux + e), ldcg((const T*)S.uy + e), ldcg((const T*)S.uz + e)};
  P.q = ldcg((const T*)S.q + e);
  P.sig = T(0);
  return P;
}

// hand a particle to the CTA that owns its row (its inbox, DSMEM).  An inbox slot is taken only
// while the owner still has room for it (free slots + unused capacity, less a margin for the
// stored particles that may rejoin there in the same slice); otherwise the particle stays and
// is pushed through the generic path.
template <typename T>
__device__ bool migrate(const cg::cluster_group& cl, const Params& p, const Sm<T>& s,
                        const PState<T>& P, int owner) {
  int* rmisc = cl.map_shared_rank(s.misc, owner);
  const int room = p.pcap + p.gcap - rmisc[M_PCOUNT] + min(rmisc[M_FTOP], p.fcap) - 64;
  const int limit = min(p.mig_cap, room);
  int* cnt = rmisc + M_INBOX;
  int e = *(volatile int*)cnt;
  for (;;) {
    if (e >= limit) return false;
    const int prev = atomicCAS(cnt, e, e + 1);
    if (prev == e) break;
    e = prev;
  }
  *cl.map_shared_rank(s.icell + e, owner) = P.ix | (P.iy << 10) | (P.sp << 20);
  *cl.map_shared_rank(s.ifx + e, owner) = P.fx;
  *cl.map_shared_rank(s.ify + e, owner) = P.fy;
  *cl.map_shared_rank(s.iux + e, owner) = P.u.x;
  *cl.map_shared_rank(s.iuy + e, owner) = P.u.y;
  *cl.map_shared_rank(s.iuz + e, owner) = P.u.z;
  *cl.map_shared_rank(s.isig + e, owner) = P.sig;
  *cl.map_shared_rank(s.iq + e, owner) = P.q;
  return true;
}

// Streaming particle slots of a CTA: [0, pcap) in shared memory, [pcap, pcap + gcap) in its
// overflow arrays in global memory (used only when the band holds more particles than fit).
template <typename T>
struct Ovf {
  int* cell;
  T *fx, *fy, *ux, *uy, *uz, *sig, *q;
};

template <typename T>
__device__ __forceinline__ Ovf<T> ovf_view(const Params& p, int cid, int me) {
  Ovf<T> o;
  const size_t g = (size_t)p.gcap;
  char* b = (char*)p.pover + ((size_t)cid * p.C + me) * g * (4 + 7 * sizeof(T));
  o.cell = (int*)b;
  T* t = (T*)(b + 4 * g);
  o.fx = t;
  o.fy = t + g;
  o.ux = t + 2 * g;
  o.uy = t + 3 * g;
  o.uz = t + 4 * g;
  o.sig = t + 5 * g;
  o.q = t + 6 * g;
  return o;
}

template <typename T>
__device__ __forceinline__ int get_cell(const Params& p, const Sm<T>& s, const Ovf<T>& o, int i) {
  return i < p.pcap ? s.pcell[i] : o.cell[i - p.pcap];
}

template <typename T>
__device__ __forceinline__ void set_cell(const Params& p, const Sm<T>& s, const Ovf<T>& o, int i,
                                         int v) {
  if (i < p.pcap)
    s.pcell[i] = v;
  else
    o.cell[i - p.pcap] = v;
}

template <typename T>
__device__ __forceinline__ PState<T> get_particle(const Params& p, const Sm<T>& s,
                                                  const Ovf<T>& o, int i, int cw) {
  PState<T> P;
  P.ix = cw & 1023;
  P.iy = (cw >> 10) & 1023;
  P.sp = (cw >> 20) & 3;
  if (i < p.pcap) {
    P.fx = s.pfx[i];
    P.fy = s.pfy[i];
    P.u = V3<T>{s.pux[i], s.puy[i], s.puz[i]};
    P.sig = s.psig[i];
    P.q = s.pq[i];
  } else {
    const int j = i - p.pcap;
    P.fx = o.fx[j];
    P.fy = o.fy[j];
    P.u = V3<T>{o.ux[j], o.uy[j], o.uz[j]};
    P.sig = o.sig[j];
    P.q = o.q[j];
  }
  return P;
}

template <typename T>
__device__ __forceinline__ void put_particle(const Params& p, const Sm<T>& s, const Ovf<T>& o,
                                             int i, const PState<T>& P) {
  const int cw = P.ix | (P.iy << 10) | (P.sp << 20);
  if (i < p.pcap) {
    s.pcell[i] = cw;
    s.pfx[i] = P.fx;
    s.pfy[i] = P.fy;
    s.pux[i] = P.u.x;
    s.puy[i] = P.u.y;
    s.puz[i] = P.u.z;
    s.psig[i] = P.sig;
    s.pq[i] = P.q;
  } else {
    const int j = i - p.pcap;
    o.cell[j] = cw;
    o.fx[j] = P.fx;
    o.fy[j] = P.fy;
    o.ux[j] = P.u.x;
    o.uy[j] = P.u.y;
    o.uz[j] = P.u.z;
    o.sig[j] = P.sig;
    o.q[j] = P.q;
  }
}

// ------------------------------------------------------------------------------------------
// Stored particle along s (Sec. 5.1: trapped / beam particles are integrated along s):
// bucket n of level k+1, fields of slices n (Fn) and n+1 (Fn1) of that level.
// ------------------------------------------------------------------------------------------
// Adds the warp's sum of v into the warp's row of FP64 diagnostics.  The sum runs in the
// type of v (FP32 sums in FP32: FP64 arithmetic is a small fraction of the FP32 rate), and lane
// 0 adds it in FP64.  Every lane of the warp calls it.
template <typename V>
__device__ __forceinline__ void warp_diag_add(double* dwarp, int slot, V v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) dwarp[(threadIdx.x >> 5) * kNDiag + slot] += (double)v;
}

template <typename T>
__device__ void stored_phase(const Params& p, const Sm<T>& s, const T* Fn, const T* Fn1,
                             int s1, int s2, int n, int me, int cnt_raw, bool varh) {
  // s1, s2: ring slots of the stored sets at levels k+1 and k+2
  T dkin = T(0);
  int dsto = 0, dlost = 0;
  const int cnt = min(cnt_raw, p.bcap);
  const T D = s.cst[K_D], h = s.cst[K_H], invh = s.cst[K_INVH];
  const int mx = p.nx - 1, my = p.ny - 1;
  for (int e0 = me * blockDim.x + threadIdx.x; e0 < cnt; e0 += p.C * blockDim.x) {
    T fz;
    PState<T> P = store_read<T>(p.st, p, ((size_t)s1 * p.nz + n) * p.bcap + e0, fz);
    const T g = gamma_of(P.u);
    dkin += P.q * s.cst[K_MOQ + P.sp] * gamma_minus_one(P.u, g);
    ++dsto;
    const T gmu = gamma_minus_uz(P.u, g);
    // stays stored while it moves less than one cell per s-step: GT2 Delta (1 - v_z)/v_z < h,
    // GT1 Delta (1 - v_z) < h
    const bool spush = p.gt1 ? D * gmu < h * g
                             : (P.u.z > T(0)) && (D * gmu < h * fmax(P.u.z, T(0)));
    if (!spush) {
      // moves more than one cell per s-step: rejoins the next zeta march at this slice
      if (!store_append(p.rq, p, s2, n, P, fz)) atomicOr(p.err, ERR_QCAP);
      continue;
    }
    T lo[6], hi[6], E[6];
    gather6_g(p, Fn, P.ix, P.fx, P.iy, P.fy, me, lo);
    gather6_g(p, Fn1, P.ix, P.fx, P.iy, P.fy, me, hi);
#pragma unroll
    for (int c = 0; c < 6; ++c) E[c] = (T(1) - fz) * lo[c] + fz * hi[c];
    // GT2: the s-step is the distance Delta along z (dt = Delta/v_z); GT1: the lab time Delta
    const T dt = p.gt1 ? D : D * g / P.u.z;
    const V3<T> un = boris(P.u, E, E + 3, s.cst[K_QM + P.sp], dt);
    const T gn = gamma_of(un);
    P.u = un;
    int m = n;
    // displacement per unit of the new velocity's divisor: dr = Delta u/vd
    const T vd = p.gt1 ? gn : un.z;
    if (vd > T(0)) {
      const T X = P.fx + D * un.x / vd * s.cst[K_INVHX];
      const T fX = floor(X);
      P.ix = (P.ix + (int)fX) & mx;
      P.fx = X - fX;
      if (p.ny > 1) {
        const T Y = P.fy + D * un.y / vd * s.cst[K_INVHY];
        const T fY = floor(Y);
        P.iy = (P.iy + (int)fY) & my;
        P.fy = Y - fY;
      }
      const T Z = fz - D * gamma_minus_uz(un, gn) / vd * invh;
      const T* hz = (const T*)p.hzt;
      if (varh) {
        // variable zeta-step: walk down the slabs from plane n (moves are backwards)
        T za = Z * h;                           // distance above plane n
        m = n;
        while (za <= T(0) && m > 0) {
          --m;
          za += hz[m];
        }
        while (m < p.nz - 1 && za > hz[m]) {
          za -= hz[m];
          ++m;
        }
        fz = za / hz[m];
        if (za <= T(0)) m = -1;
      } else {
        const T cZ = ceil(Z) - T(1);
        m = n + (int)cZ;
        fz = Z - cZ;
      }
      if (m < 0) {                              // left the box at the back
        ++dlost;
        continue;
      }
      // beam current of the next level j = Q u/(gamma hx hy h), CIC across, linear in zeta
      // between half-slice centres; with a variable step the centres are zeta_i + h_i/2 and
      // half-slice i divides by its own thickness
      const T amp = varh ? P.q / (T(p.hx * p.hy) * gn) : P.q * s.cst[K_BEAM] / gn;
      int i0;
      T f;
      if (varh) {
        const T hm = hz[m];
        if (fz >= T(0.5)) {
          const T hu = m + 1 < p.nz ? hz[m + 1] : hm;
          i0 = m;
          f = (fz - T(0.5)) * hm / (T(0.5) * (hm + hu));
        } else {
          const T hd = m > 0 ? hz[m - 1] : hm;
          i0 = m - 1;
          f = (T(0.5) * hd + fz * hm) / (T(0.5) * (hd + hm));
        }
      } else {
        const T tz = fz - T(0.5);
        const T ftz = floor(tz);
        i0 = m + (int)ftz;
        f = tz - ftz;
      }
      T* jb = (T*)p.jbeam;
      for (int t = 0; t < 2; ++t) {
        const int iz = i0 + t;
        if (iz < 0 || iz >= p.nz) continue;
        const T a = amp * (t == 0 ? T(1) - f : f) / (varh ? hz[iz] : T(1));
        T* base = jb + (((size_t)s2 * p.nz + iz) * 3) * (size_t)p.nx * p.ny;
        const T vals[3] = {a * un.x, a * un.y, a * un.z};
        for (int c = 0; c < 3; ++c) {
          const T sx = (c == 0) ? T(-0.5) : T(0);
          const T sy = (c == 1 && p.ny > 1) ? T(-0.5) : T(0);
          const T X = P.fx + sx, Y = P.fy + sy;
          const T i0f = floor(X), fx = X - i0f;
          const int gx = (P.ix + (int)i0f) & mx, gx1 = (gx + 1) & mx;
          T* pl = base + (size_t)c * p.nx * p.ny;
          if (p.ny == 1) {
            atomicAdd(pl + gx, (T(1) - fx) * vals[c]);
            atomicAdd(pl + gx1, fx * vals[c]);
          } else {
            const T j0f = floor(Y), fy = Y - j0f;
            const int gy = (P.iy + (int)j0f) & my, gy1 = (gy + 1) & my;
            atomicAdd(pl + (size_t)gy * p.nx + gx, ((T(1) - fx) * (T(1) - fy)) * vals[c]);
            atomicAdd(pl + (size_t)gy * p.nx + gx1, (fx * (T(1) - fy)) * vals[c]);
            atomicAdd(pl + (size_t)gy1 * p.nx + gx, ((T(1) - fx) * fy) * vals[c]);
            atomicAdd(pl + (size_t)gy1 * p.nx + gx1, (fx * fy) * vals[c]);
          }
        }
        atomicExch(p.jflag + (size_t)s2 * p.nz + iz, 1);
      }
    }
    if (!store_append(p.st, p, s2, m, P, fz)) atomicOr(p.err, ERR_BCAP);
  }
  if (p.diag) {
    if (__any_sync(0xffffffffu, (dsto | dlost) != 0)) {
      warp_diag_add(s.dwarp, DG_KIN, dkin);
      warp_diag_add(s.dwarp, DG_KST, dkin);
      warp_diag_add(s.dwarp, DG_STORED, dsto);
      warp_diag_add(s.dwarp, DG_LOST, dlost);
    }
  }
}

// ------------------------------------------------------------------------------------------
// App. B closed form of the slice system (Eqs. RxN..eqall, LyN read with B_z0^1 + B_z1^1,
// eqall with +i k_y, T4 = -2 h Delta E_z0^0 K^2) for one mode.
// ------------------------------------------------------------------------------------------
template <typename T>
struct Mode6 {
  Cx<T> Rx, Ry, Lx, Ly, Ez, Bz;
};

template <typename T>
__device__ __forceinline__ Mode6<T> slice_solve(T kx, T ky, T h, T Dl, const Mode6<T>& n1,
                                                Cx<T> Rxo, Cx<T> Ryo, Cx<T> Ezo, Cx<T> Bzo,
                                                Cx<T> jx0m, Cx<T> jy0m, Cx<T> jx0p, Cx<T> jy0p,
                                                Cx<T> jx1p, Cx<T> jy1p, Cx<T> jz1p) {
  const T K2 = kx * kx + ky * ky;
  const T Dd = T(16) + h * (T(2) * Dl + h) * K2;
  // predictor j^1_{-1/2} := j^1_{+1/2}
  const Cx<T> Jx = (jx0m + jx0p) + T(2) * jx1p;
  const Cx<T> Jy = (jy0m + jy0p) + T(2) * jy1p;
  const Cx<T> Wx = (n1.Rx + Rxo) - T(2) * n1.Lx;
  const Cx<T> Wy = (n1.Ry + Ryo) - T(2) * n1.Ly;
  const Cx<T> Ux = (n1.Rx + Rxo) + T(2) * n1.Lx;
  const Cx<T> Uy = (n1.Ry + Ryo) + T(2) * n1.Ly;
  const T c16 = T(16) - h * h * K2;
  const T hD = h * Dl;
  Cx<T> numE = c16 * n1.Ez - (T(16) * h) * jz1p;
  numE = numE - mul_i(hD * (kx * Jx + ky * Jy));
  numE = numE - (T(2) * hD * K2) * Ezo;
  numE = numE + mul_i((T(2) * h * h) * (kx * jx1p + ky * jy1p));
  numE = numE + mul_i((T(4) * h) * (kx * Wx + ky * Wy));
  Cx<T> numB = c16 * n1.Bz + mul_i((T(2) * h * h) * (kx * jy1p - ky * jx1p));
  numB = numB + mul_i(hD * (kx * Jy - ky * Jx));
  numB = numB - (T(2) * hD * K2) * Bzo;
  numB = numB + mul_i((T(4) * h) * (ky * Ux - kx * Uy));
  const T invD = T(1) / Dd;
  Mode6<T> o;
  o.Ez = invD * numE;
  o.Bz = invD * numB;
  // RxN, RyN (trapezoid in s)
  const Cx<T> sEz = o.Ez + Ezo, sBz = o.Bz + Bzo;
  o.Rx = Rxo + Dl * (mul_i(T(0.5) * (kx * sEz + ky * sBz)) - T(0.25) * Jx);
  o.Ry = Ryo + Dl * (mul_i(T(0.5) * (ky * sEz - kx * sBz)) - T(0.25) * Jy);
  // LxN, LyN (box scheme in zeta)
  const Cx<T> tEz = n1.Ez + o.Ez, tBz = o.Bz + n1.Bz;
  o.Lx = n1.Lx - (T(0.5) * h) * (mul_i(T(0.5) * (kx * tEz - ky * tBz)) + jx1p);
  o.Ly = n1.Ly - (T(0.5) * h) * (mul_i(T(0.5) * (ky * tEz + kx * tBz)) + jy1p);
  return o;
}

// ------------------------------------------------------------------------------------------
// progress / waits between concurrently marching clusters
// ------------------------------------------------------------------------------------------
static __device__ void wait_for(const Params& p, int pcid, unsigned long long target) {
  int spins = 0;
  while (ld_acquire_u64(p.progress + pcid) < target) {
    if (atomicAdd(p.err, 0) & ERR_TIMEOUT) return;
    __nanosleep(200);
    if (++spins > p.wait_spin_limit) {
      atomicOr(p.err, ERR_TIMEOUT);
      return;
    }
  }
}

// wait until the host has released group g of march `key` in the host-mapped word `word`
// (streamed state: the input's groups; denoised chain: the denoised current's groups).
// *seen (shared memory, -1 at the start of a march) is the last group known released.
static __device__ void wait_release(const Params& p, const unsigned long long* word, long long key,
                             int nchunk, int g, int* seen) {
  if (*seen >= g) return;
  const unsigned long long target = io_value(key, nchunk, g);
  unsigned long long v;
  int spins = 0;
  while ((v = ld_acquire_sys_u64(word)) < target) {
    if (atomicAdd(p.err, 0) & ERR_TIMEOUT) return;
    __nanosleep(200);
    if (++spins > p.wait_spin_limit) {
      atomicOr(p.err, ERR_TIMEOUT);
      return;
    }
  }
  // the host releases a march's groups in order and the next march's of this slot only after
  // this one has used them all, so v names a group of this march
  *seen = (int)min((unsigned long long)(nchunk - 1), v - io_value(key, nchunk, 0));
}

// streamed state: the group of block b of s-step k's input
__device__ __forceinline__ void wait_input(const Params& p, long long k, int b, int* seen) {
  wait_release(p, p.io_ready + (k % p.io_ring), k, p.io_nchunk, io_group(p.nz, p.io_chunk, b), seen);
}

// FP64 diagnostics: each warp adds its lanes' sums to its own row (no atomics); the rows are
// summed once at the end of the march.  Every lane of the warp calls it.

// ------------------------------------------------------------------------------------------
// the march of one s-step k (computes level k+1)
// ------------------------------------------------------------------------------------------
// CANON = false: the library's block layout [nz+1][C][6][M].  CANON = true: the public layout
// of gempic_get_state ([6][nz][ny][nx/2]; j at half-slice index n <-> block n+1), used by the
// allocation-free entry point on a caller's buffer.
// DN: the march of a denoised chain (its hooks are compiled into the chain's instantiations
// only); CANON instantiations carry the streamed state's hooks.
template <typename T, bool CANON = false, int SH = 0, bool DN = false>
__device__ void march(const Params& p, const Sm<T>& s, const cg::cluster_group& cl, long long k,
                      int cid, long long item_) {
  // the 128 x 128 instantiation is compiled for GT2 and a uniform zeta-step only (other runs
  // take the generic one)
  constexpr int LAW = SH == 1 ? 0 : -1;
  const bool varh = SH != 1 && p.varh != 0;
  const bool resid = SH != 1 && p.resid != 0;     // continuity and Gauss residuals
  const int rbe = p.ny > 1 ? p.RB : 1;            // own rows of the residual planes
  T rmax = T(0), gmax = T(0);
  const T* hzt = (const T*)p.hzt;
  const int me = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  // march index: k, or 2k + pass in a denoised chain; the previous march of the launch is
  // item - 1
  const long long item = DN ? item_ : k;
  const long long item0 = DN ? 2 * p.k0 : p.k0;
  const bool dn1 = DN && !(item & 1), dn2 = DN && (item & 1);
  const bool waits = p.P > 1 && item > item0;
  const int pcid = (cid + p.P - 1) % p.P;
  const int nz = p.nz;
  const int nxh = p.nx / 2;
  const int s1 = (int)(((k + 1) % p.ring + p.ring) % p.ring);
  const int s2 = (int)(((k + 2) % p.ring + p.ring) % p.ring);
  const T h = s.cst[K_H], Dl = s.cst[K_DF];
  const long long sl = item - item0;                // march index within this launch
  const Ovf<T> ov = ovf_view<T>(p, cid, me);        // overflow particle slots of this CTA
  const int fplane = p.FR * p.nx;                   // elements of one field component
  const int jplane = p.JR * p.nx;                   // elements of one current component
  TIMER_DECL

  // FP64 diagnostics go to per-warp rows in shared memory (section below), not registers
  double fe = 0.0;      // field energy of the march: each slice's FP32 partial added in FP64

  // reset the next level's stored buckets and rejoin queues (free: their last reader, the
  // march of step k+1-ring, has completed)
  for (int b = me * NT + tid; b < nz; b += p.C * NT) {
    p.st.cnt[(size_t)s2 * nz + b] = 0;
    p.rq.cnt[(size_t)s2 * nz + b] = 0;
  }
  // fresh particles at the front ghost plane (Sec. 5.1: Q_f = q n hx hy Delta / ppc)
  if (tid == 0) {
    s.misc[M_PCOUNT] = 0;
    s.misc[M_FTOP] = 0;
    s.misc[M_INBOX] = 0;
    s.misc[M_OUTN] = 0;
  }
  for (int i = tid; i < (NT >> 5) * kNDiag; i += NT) s.dwarp[i] = 0.0;
  if (resid) {
    for (int i = tid; i < 3 * rbe * p.nx; i += NT) s.dd[i] = T(0);
    if (tid == 0) s.dacc[0] = s.dacc[1] = 0.0;
  }
  __syncthreads();
  if (p.inject && !dn2) {
    const int per_row = p.nlayer >> p.logny;        // particles per transverse row
    const int nmine = per_row * p.RB;
    for (int i = tid; i < nmine; i += NT) {
      // storage order: segments of nx particles with fixed (row, species, k); inside a segment
      // position j holds cell ix = 5 j mod nx, so the 32 lanes of a warp deposit into cells 5
      // apart (disjoint stencils, distinct shared-memory banks)
      const int seg = i >> p.lognx, j = i & (p.nx - 1);
      const int yl = seg / p.ppc_sum;
      int kk = seg - yl * p.ppc_sum;
      int sp = 0;
      while (sp + 1 < p.nspecies && kk >= p.ppc[sp]) {
        kk -= p.ppc[sp];
        ++sp;
      }
      const int ix = (5 * j) & (p.nx - 1);
      const int iy = (me << p.logRB) + yl;
      const int cell = iy * p.nx + ix;
      const unsigned long long g =
          (unsigned long long)(p.poff[sp] + cell * p.ppc[sp] + kk);
      const unsigned long long c =
          ((unsigned long long)k * (unsigned long long)p.nlayer + g) * 2ull;
      const T fx = T(uniform24(p.seed, c));
      const T fy = p.ny > 1 ? T(uniform24(p.seed, c + 1)) : T(0);
      T q = s.cst[K_QF + sp];
      if (p.chan_a != 0.0) {
        // density channel (Eq. n_plasma) at the particle's distance from the middle node
        const T dx = (T(ix - (p.nx >> 1)) + fx) * s.cst[K_HX];
        const T dy = p.ny > 1 ? (T(iy - (p.ny >> 1)) + fy) * s.cst[K_HY] : T(0);
        q *= T(1) + T(p.chan_a) * exp(-(dx * dx + dy * dy) * T(p.chan_ir2));
      }
      if (i < p.pcap) {
        s.pcell[i] = ix | (iy << 10) | (sp << 20);
        s.pfx[i] = fx;
        s.pfy[i] = fy;
        s.pux[i] = T(0);
        s.puy[i] = T(0);
        s.puz[i] = T(0);
        s.psig[i] = T(0);
        s.pq[i] = q;
      } else {
        // a fresh layer larger than the shared-memory slots (many particles per cell)
        // continues in the CTA's overflow slots in global memory
        PState<T> P;
        P.ix = ix;
        P.iy = iy;
        P.sp = sp;
        P.fx = fx;
        P.fy = fy;
        P.u = V3<T>{T(0), T(0), T(0)};
        P.sig = T(0);
        P.q = q;
        put_particle(p, s, ov, i, P);
      }
    }
    if (tid == 0) s.misc[M_PCOUNT] = min(nmine, p.pcap + p.gcap);
    if (nmine > p.pcap + p.gcap && tid == 0) atomicOr(p.err, ERR_PCAP);
  }
  // ghost slice: field-free
  T* Fcur = s.F[0];
  T* Fnew = s.F[1];
  for (int i = tid; i < 6 * fplane; i += NT) Fcur[i] = T(0);
  for (int i = tid; i < 3 * jplane; i += NT) s.J[i] = T(0);
  if constexpr (sizeof(T) == 4)
    for (int i = tid; i < 3 * jplane; i += NT) s.Jint[i] = 0;

  // per-mode carried state (one mode per thread): thread m owns column position q of kx
  // column kxl, i.e. the mode (kxl, ky_of_pos(q)).  Block layout: q fastest (a warp's state
  // accesses are 32 consecutive words).  Public layout (kx innermost): kxl fastest, so that a
  // warp reads and writes whole 32-byte runs of its CTA's KB columns in 32 / KB rows, not 32
  // rows one word each
  const int m = tid;
  const bool has_mode = m < p.M;
  const int kxl = !has_mode ? 0 : CANON ? m & (p.KB - 1) : m >> p.logny;
  const int q = !has_mode ? 0 : CANON ? m >> p.logKB : m & (p.ny - 1);
  const int kyi = ky_of_pos(p.logny, q);
  const T kx = has_mode ? s.kx[(me << p.logKB) + kxl] : T(0);
  const T ky = has_mode ? s.ky[kyi] : T(0);
  const bool masked = p.ny > 1 && kyi == p.ny / 2;
  Mode6<T> S1;
  S1.Rx = S1.Ry = S1.Lx = S1.Ly = S1.Ez = S1.Bz = cx<T>(T(0), T(0));
  Cx<T> jpx = cx<T>(T(0), T(0)), jpy = jpx;       // j^1 at n + 3/2 (predictor of the last solve)
  Cx<T> o[6];                                     // old level, block n
  Cx<T> j0px = jpx, j0py = jpx;                   // old level j at n + 1/2
  const Cx<T>* st = (const Cx<T>*)p.state;
  // the new level is written over the old one, or (first pass of a denoised s-step) elsewhere
  Cx<T>* stw = (Cx<T>*)(dn1 ? p.dn_scratch : p.state_out ? p.state_out : p.state);
  auto blk = [&](int b, int c) -> size_t {
    if constexpr (CANON) {
      const int kxg = (me << p.logKB) + kxl;
      const int sl_ = c < 4 ? b : b - 1;
      return (((size_t)c * p.nz + sl_) * p.ny + kyi) * (size_t)nxh + kxg;
    } else {
      return (((size_t)b * p.C + me) * 6 + c) * (size_t)p.M + m;
    }
  };
  // the public layout has no ghost slice and no j at half-slice -1
  auto blk_ok = [&](int b, int c) -> bool {
    if constexpr (CANON) {
      return c < 4 ? b < p.nz : b >= 1;
    } else {
      return true;
    }
  };

  if (waits && tid == 0 && me == 0)
    wait_for(p, pcid, prog_value(item - 1, nz, min(nz, 3)));   // predecessor done down to nz-3
  // streamed state: the input's blocks nz and nz-1
  if (tid == 0 && me == 0) s.misc[M_IOSEEN] = -1;
  if constexpr (CANON)
    if (p.io_chunk && tid == 0 && me == 0) wait_input(p, k, nz - 1, s.misc + M_IOSEEN);
  cl.sync();
  if (has_mode) {
    j0px = ldcg(st + blk(nz, 4));
    j0py = ldcg(st + blk(nz, 5));
#pragma unroll
    for (int c = 0; c < 6; ++c) o[c] = ldcg(st + blk(nz - 1, c));
  }
  const long long klast = DN ? p.k0 + p.nsteps / 2 - 1 : p.k0 + p.nsteps - 1;
  const bool snap_step = p.snapshot && k == klast;
  // the current kept: every first pass of a denoised chain, else the launch's last s-step
  T* const jcap = (T*)(dn1 ? p.dn_jcap[k & 3] : DN ? nullptr : p.jcap);
  const bool cap_step = jcap != nullptr && (dn1 || k == klast);
  // per-slice counters of other marches, read once per CTA and broadcast in shared memory
  if (tid == 0) {
    s.misc[M_RQN] = ldcg(p.rq.cnt + (size_t)s1 * nz + (nz - 1));
    s.misc[M_JFLAG] = ldcg(p.jflag + (size_t)s1 * nz + (nz - 1));
  }
  __syncthreads();

  // per-thread diagnostic sums, flushed to the warp rows every 16 slices (a warp reduction
  // per slice costs more than the push of a particle)
  SliceAcc<T> sa{T(0), T(0), 0};
  int ntrap = 0, nrej = 0;
  T fluxw = T(0);                                  // variable zeta-step: flux weighted by h_n
  for (int n = nz - 1; n >= 0; --n) {
#ifdef GEMPIC_PHASE_TIMERS
    const long long t_slice = clock64();
#endif
    // variable zeta-step: the slab of this slice (planes n, n+1) sets the step-dependent
    // constants (the previous slice's stored phase has finished reading them)
    const T hn = varh ? hzt[n] : h;
    T* const dn_n = s.dn + (size_t)(n & 1) * rbe * p.nx;   // arrival density of plane n
    if (varh) {
      __syncthreads();
      if (tid == 0) {
        T* c = s.cst;
        c[K_H] = hn;
        c[K_INVH] = T(1) / hn;
        c[K_CX] = T(p.hx) / hn;
        c[K_CY] = T(p.hy) / hn;
        c[K_FLUX] = T(p.hx * p.hy) * hn;
        c[K_BEAM] = T(1) / (T(p.hx * p.hy) * hn);
      }
      __syncthreads();
    }
    // ---------------- A: streaming push from plane n+1 to plane n -----------------------
    {
      const int cnt0 = s.misc[M_PCOUNT];
      for (int i = tid; i < cnt0; i += NT) {
        const int cw = get_cell(p, s, ov, i);
        if (cw < 0) continue;
        PState<T> P = get_particle(p, s, ov, i, cw);
        T fzt;
        const bool trap = stream_push<T, LAW, SH != 1>(p, s, Fcur, P, hn, me, fzt, sa, dn_n);
        bool gone = trap;
        if (trap) {
          ++ntrap;
          if (!store_append(p.st, p, s1, n, P, fzt)) atomicOr(p.err, ERR_BCAP);
        } else {
          const int owner = P.iy >> p.logRB;
          // a particle that left the band moves to the owner of its row: queued in the local
          // outbox and sent after the push (directly if the outbox is full; kept here if the
          // owner's inbox is full: it then takes the generic path)
          if (owner != me) {
            const int o = atomicAdd(s.misc + M_OUTN, 1);
            if (o < kOutCap) {
              s.ocell[o] = P.ix | (P.iy << 10) | (P.sp << 20);
              s.odst[o] = owner;
              s.ofx[o] = P.fx;
              s.ofy[o] = P.fy;
              s.oux[o] = P.u.x;
              s.ouy[o] = P.u.y;
              s.ouz[o] = P.u.z;
              s.osig[o] = P.sig;
              s.oq[o] = P.q;
              gone = true;
            } else if (migrate(cl, p, s, P, owner)) {
              gone = true;
            }
          }
        }
        if (gone) {
          set_cell(p, s, ov, i, -1);
          // shared-memory slots are reused; a dead overflow slot stays unused this s-step
          if (i < p.pcap) {
            const int f = atomicAdd(s.misc + M_FTOP, 1);
            if (f < p.fcap) s.fstack[f] = i;
          }
        } else {
          put_particle(p, s, ov, i, P);
        }
      }
      TIMER_MARK(PH_AR);
      // stored particles that rejoin the march at this slice (partial first step), taken by
      // the CTA that owns their row
      const int nq = (p.fields_only || dn2) ? 0 : min(s.misc[M_RQN], p.bcap);
      for (int e = tid; e < nq; e += NT) {
        const size_t ge = ((size_t)s1 * nz + n) * p.bcap + e;
        if ((((ldcg(p.rq.cell + ge) >> 10) & 1023) >> p.logRB) != me) continue;
        T fz;
        PState<T> P = store_read<T>(p.rq, p, ge, fz);
        ++nrej;
        T fzt;
        const bool trap = stream_push<T, LAW, SH != 1>(p, s, Fcur, P, fz * hn, me, fzt, sa, dn_n);
        if (trap) {
          ++ntrap;
          if (!store_append(p.st, p, s1, n, P, fzt)) atomicOr(p.err, ERR_BCAP);
          continue;
        }
        const int owner = P.iy >> p.logRB;
        if (owner != me && migrate(cl, p, s, P, owner)) continue;
        const int slot = atomicAdd(s.misc + M_PCOUNT, 1);
        if (slot < p.pcap + p.gcap) {
          put_particle(p, s, ov, slot, P);
        } else {
          atomicOr(p.err, ERR_PCAP);
#ifdef GEMPIC_PHASE_TIMERS
          if (p.timers && atomicCAS(p.timers + 20, 0ull, 2ull) == 0ull) {
            p.timers[21] = n; p.timers[22] = nq; p.timers[24] = slot; p.timers[26] = me;
            p.timers[27] = (unsigned long long)k;
          }
#endif
        }
      }
    }
    if (varh) {
      fluxw += sa.flux * hn;
      sa.flux = T(0);
    }
    if (p.diag && (n & 15) == 0) {
      warp_diag_add(s.dwarp, DG_KIN, sa.kin);
      warp_diag_add(s.dwarp, DG_FLUX, varh ? fluxw : sa.flux);
      int cnts[3] = {sa.push, ntrap, nrej};
#pragma unroll
      for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) cnts[c] += __shfl_down_sync(0xffffffffu, cnts[c], off);
      if ((tid & 31) == 0) {
        double* row = s.dwarp + (tid >> 5) * kNDiag;
        row[DG_PUSH] += (double)cnts[0];
        row[DG_TRAP] += (double)cnts[1];
        row[DG_REJOIN] += (double)cnts[2];
      }
      sa = SliceAcc<T>{T(0), T(0), 0};
      ntrap = nrej = 0;
      fluxw = T(0);
    }
    TIMER_MARK(PH_A);
    __syncthreads();
    TIMER_MARK(PH_AW);
    // outbox: the lanes of the first warps group their particles by owner; per owner one lane
    // reserves inbox entries (as many as fit) and the lanes write them remotely; a particle
    // that does not fit returns to a slot of this CTA
    if (p.ny > 1) {
      const int nout = min(s.misc[M_OUTN], kOutCap);
      if (tid < ((nout + 31) & ~31)) {
        const int lane = tid & 31;
        const bool have = tid < nout;
        const int dst = have ? s.odst[tid] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, dst);
        const int leader = __ffs(grp) - 1;
        const int rank = __popc(grp & ((1u << lane) - 1u));
        int base = 0, take = 0;
        if (lane == leader && dst >= 0) {
          const int want = __popc(grp);
          int* rmisc = cl.map_shared_rank(s.misc, dst);
          const int room = p.pcap + p.gcap - rmisc[M_PCOUNT] + min(rmisc[M_FTOP], p.fcap) - 64;
          const int limit = min(p.mig_cap, room);
          int* cnt = rmisc + M_INBOX;
          int e = *(volatile int*)cnt;
          for (;;) {
            take = max(0, min(want, limit - e));
            if (take == 0) break;
            const int prev = atomicCAS(cnt, e, e + take);
            if (prev == e) break;
            e = prev;
          }
          base = e;
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        take = __shfl_sync(0xffffffffu, take, leader);
        if (have) {
          PState<T> P;
          const int cw = s.ocell[tid];
          P.ix = cw & 1023;
          P.iy = (cw >> 10) & 1023;
          P.sp = (cw >> 20) & 3;
          P.fx = s.ofx[tid];
          P.fy = s.ofy[tid];
          P.u = V3<T>{s.oux[tid], s.ouy[tid], s.ouz[tid]};
          P.sig = s.osig[tid];
          P.q = s.oq[tid];
          if (rank < take) {
            const int e = base + rank;
            *cl.map_shared_rank(s.icell + e, dst) = cw;
            *cl.map_shared_rank(s.ifx + e, dst) = P.fx;
            *cl.map_shared_rank(s.ify + e, dst) = P.fy;
            *cl.map_shared_rank(s.iux + e, dst) = P.u.x;
            *cl.map_shared_rank(s.iuy + e, dst) = P.u.y;
            *cl.map_shared_rank(s.iuz + e, dst) = P.u.z;
            *cl.map_shared_rank(s.isig + e, dst) = P.sig;
            *cl.map_shared_rank(s.iq + e, dst) = P.q;
          } else {
            const int slot = atomicAdd(s.misc + M_PCOUNT, 1);
            if (slot < p.pcap + p.gcap)
              put_particle(p, s, ov, slot, P);
            else
              atomicOr(p.err, ERR_PCAP);
          }
        }
      }
    }
    // FP32: fold the fixed-point accumulators of the halo rows now (only this CTA's pushes
    // deposit there); own rows also receive other CTAs' fixed-point deposits and are folded
    // after the barrier
    // (FP32: four consecutive elements per thread, 16-byte accesses; rows are nx >= 32 long)
    if (p.ny > 1) {
      const int rb = (me + p.C - 1) & (p.C - 1), ra = (me + 1) & (p.C - 1);
      if constexpr (sizeof(T) == 4) {
        const T jinv = s.cst[K_JINV];
        for (int i = 4 * tid; i < 9 * p.nx; i += 4 * NT) {
          const int rowi = i >> p.lognx, x = i & (p.nx - 1);
          const int c = rowi / 3, which = rowi - 3 * c;
          const int jrow = which == 0 ? 0 : p.RB + p.JOFF + (which - 1);
          const size_t j = ((size_t)c * p.JR + jrow) * p.nx + x;
          float4 v = *reinterpret_cast<const float4*>(s.J + j);
          const int4 q = *reinterpret_cast<const int4*>(s.Jint + j);
          v.x += T(q.x) * jinv;
          v.y += T(q.y) * jinv;
          v.z += T(q.z) * jinv;
          v.w += T(q.w) * jinv;
          // which 0: band row -1 -> row RB-1 of the CTA below (recv slot 2)
          // which 1, 2: band rows RB, RB+1 -> rows 0, 1 of the CTA above (recv slots 0, 1)
          const int dst = which == 0 ? rb : ra;
          const int slot = which == 0 ? 2 : which - 1;
          float4* d = reinterpret_cast<float4*>(s.recv + ((size_t)c * 3 + slot) * p.nx + x);
          *(dst == me ? d : cl.map_shared_rank(d, dst)) = v;
        }
      } else {
        // halo currents (band rows -1, RB, RB+1) to the owners' receive buffers (plain stores)
        for (int i = tid; i < 9 * p.nx; i += NT) {
          const int rowi = i >> p.lognx, x = i & (p.nx - 1);
          const int c = rowi / 3, which = rowi - 3 * c;
          const int jrow = which == 0 ? 0 : p.RB + p.JOFF + (which - 1);
          const T v = s.J[((size_t)c * p.JR + jrow) * p.nx + x];
          const int dst = which == 0 ? rb : ra;
          const int slot = which == 0 ? 2 : which - 1;
          T* q = s.recv + ((size_t)c * 3 + slot) * p.nx + x;
          *(dst == me ? q : cl.map_shared_rank(q, dst)) = v;
        }
      }
    }
    if (tid == 0) {
      if (s.misc[M_PCOUNT] > p.pcap + p.gcap) s.misc[M_PCOUNT] = p.pcap + p.gcap;
      __threadfence();
    }
#ifdef GEMPIC_PHASE_TIMERS
    // per CTA: cycles from the slice start to the arrival at B1 (words 64 + rank); per slice of
    // the launch's first march, arrival and release (words 256 + 2 (n C + rank))
    const long long t_arr = clock64() - t_slice;
    if (tid == 0 && p.timers) atomicAdd(p.timers + 64 + me, (unsigned long long)t_arr);
#endif
    // denoised chain: the second pass reads the denoised current of half-slice n after B1
    if (dn2 && me == 0 && tid == 0)
      wait_release(p, p.dn_ready + (k & 3), item, p.dn_nchunk, (nz - 1 - n) / p.dn_chunk,
                   s.misc + M_IOSEEN);
    cl.sync();                                                      // B1: deposits done
#ifdef GEMPIC_PHASE_TIMERS
    if (tid == 0 && p.timers && k == p.k0) {
      p.timers[256 + 2 * ((size_t)n * p.C + me)] = (unsigned long long)t_arr;
      p.timers[256 + 2 * ((size_t)n * p.C + me) + 1] = (unsigned long long)(clock64() - t_slice);
    }
#endif
    // publish: iteration n+1 complete (its stored phase and this push have been issued)
    if (p.P > 1 && me == 0 && tid == 0 && n + 1 <= nz - 1)
      st_release_u64(p.progress + cid, prog_value(item, nz, nz - (n + 1)));
    // denoised chain: the first pass's current of half-slices >= n + 1 is written
    if (dn1 && me == 0 && tid == 0) {
      const int done = nz - (n + 1);
      if (done > 0 && done % p.dn_chunk == p.dn_lead)
        st_release_sys_u64(p.dn_done + cid, prog_value(item, nz, done));
    }
    // streamed state: blocks >= n + 2 of the new level are written (and blocks >= n of the
    // old level read); the host copies a group out once its last block is
    if constexpr (CANON)
      if (p.io_chunk && me == 0 && tid == 0) {
        const int done = nz - (n + 1);
        if (done > 0 && done % p.io_chunk == 0) st_release_sys_u64(p.io_done + cid, prog_value(k, nz, done));
      }
    // stored particles of cell n at this level (traps of this push included), for phase E;
    // loaded by the last warp, which has no forward-transform task
    if (tid == NT - 32) s.misc[M_STN] = ldcg(p.st.cnt + (size_t)s1 * nz + n);
    TIMER_MARK(PH_B1);
    // own rows: fixed-point accumulators (FP32) and the received halo currents (rows 0, 1
    // from the band below, RB - 1 from the band above); element mapping as in the beam add
    if constexpr (sizeof(T) == 4) {
      const T jinv = s.cst[K_JINV];
      for (int i = 4 * tid; i < 3 * p.RB * p.nx; i += 4 * NT) {
        const int c = i >> (p.logRB + p.lognx);
        const int rem = i & ((p.RB << p.lognx) - 1);
        const int row = rem >> p.lognx, x = rem & (p.nx - 1);
        const size_t j = ((size_t)c * p.JR + p.JOFF) * p.nx + rem;
        float4 v = *reinterpret_cast<const float4*>(s.J + j);
        const int4 q = *reinterpret_cast<const int4*>(s.Jint + j);
        v.x += T(q.x) * jinv;
        v.y += T(q.y) * jinv;
        v.z += T(q.z) * jinv;
        v.w += T(q.w) * jinv;
        if (p.ny > 1) {
          const int slot = row == 0 ? 0 : row == 1 ? 1 : row == p.RB - 1 ? 2 : -1;
          if (slot >= 0) {
            const float4 r = *reinterpret_cast<const float4*>(s.recv + ((size_t)c * 3 + slot) * p.nx + x);
            v.x += r.x;
            v.y += r.y;
            v.z += r.z;
            v.w += r.w;
            if (slot == 1 && p.RB == 2) {     // RB = 2: row 1 is also row RB - 1
              const float4 r2 = *reinterpret_cast<const float4*>(s.recv + ((size_t)c * 3 + 2) * p.nx + x);
              v.x += r2.x;
              v.y += r2.y;
              v.z += r2.z;
              v.w += r2.w;
            }
          }
        }
        *reinterpret_cast<float4*>(s.J + j) = v;
      }
    } else {
      for (int i = tid; i < 3 * p.RB * p.nx; i += NT) {
        const int c = i >> (p.logRB + p.lognx);
        const int rem = i & ((p.RB << p.lognx) - 1);
        const int row = rem >> p.lognx, x = rem & (p.nx - 1);
        const size_t j = ((size_t)c * p.JR + p.JOFF) * p.nx + rem;
        T v = s.J[j];
        if (p.ny > 1) {
          if (row == 0) v += s.recv[((size_t)c * 3 + 0) * p.nx + x];
          if (row == 1) v += s.recv[((size_t)c * 3 + 1) * p.nx + x];
          if (row == p.RB - 1) v += s.recv[((size_t)c * 3 + 2) * p.nx + x];
        }
        s.J[j] = v;
      }
    }
    TIMER_MARK(PH_BF);
    // migrating particles into free slots
    if (p.ny > 1) {
      const int nin = min(s.misc[M_INBOX], p.mig_cap);
      const int ftop = min(s.misc[M_FTOP], p.fcap);
      const int pc = s.misc[M_PCOUNT];
      for (int e = tid; e < nin; e += NT) {
        const int slot = e < ftop ? s.fstack[ftop - 1 - e] : pc + (e - ftop);
        if (slot >= p.pcap + p.gcap) {
          atomicOr(p.err, ERR_PCAP);
#ifdef GEMPIC_PHASE_TIMERS
          if (p.timers && atomicCAS(p.timers + 20, 0ull, 1ull) == 0ull) {
            p.timers[21] = n; p.timers[22] = nin; p.timers[23] = ftop; p.timers[24] = pc;
            p.timers[25] = slot; p.timers[26] = me; p.timers[27] = (unsigned long long)k;
          }
#endif
          continue;
        }
        PState<T> P = get_particle(p, s, ov, 0, s.icell[e]);
        P.fx = s.ifx[e];
        P.fy = s.ify[e];
        P.u = V3<T>{s.iux[e], s.iuy[e], s.iuz[e]};
        P.sig = s.isig[e];
        P.q = s.iq[e];
        put_particle(p, s, ov, slot, P);
      }
      __syncthreads();
      if (tid == 0) {
        s.misc[M_FTOP] = max(0, ftop - nin);
        s.misc[M_PCOUNT] = min(p.pcap + p.gcap, pc + max(0, nin - ftop));
        s.misc[M_INBOX] = 0;
        s.misc[M_OUTN] = 0;
      }
    }
    TIMER_MARK(PH_BI);
    // the inbox drain ends with a barrier that also orders the own-row fold before the beam
    // add and the row transforms; 2-D runs have no inbox
    if (p.ny == 1) __syncthreads();
    if (resid) {
      // (D(start) - D(end))/h_n - div j_perp on every node of the own rows, before the beam
      // current joins j (backward differences: j_x on x-edges, j_y on y-edges).  3-D: the
      // row below the band is the last own row of the CTA below, read once every CTA has
      // folded its rows and before any adds the beam current.  Each thread clears the
      // entries it read.
      if (p.ny > 1) cl.sync();
      const T* jx = s.J + (size_t)p.JOFF * p.nx;
      const T* jy = s.J + ((size_t)p.JR + p.JOFF) * p.nx;
      const T ihx = T(1.0 / p.hx), ihy = T(1.0 / p.hy), ih = T(1) / hn;
      const int below = (me + p.C - 1) & (p.C - 1);
      const uint32_t jyb =
          p.ny > 1 ? cluster_addr(sh_addr(jy + (size_t)(p.RB - 1) * p.nx), below) : 0u;
      for (int i = tid; i < rbe * p.nx; i += NT) {
        const int row = i >> p.lognx, x = i & (p.nx - 1);
        const int o = row * p.nx;
        T div = (jx[o + x] - jx[o + ((x - 1) & (p.nx - 1))]) * ihx;
        if (p.ny > 1) {
          const T jyd = row > 0 ? jy[o - p.nx + x] : ldc(jyb + (uint32_t)(x * sizeof(T)), T(0));
          div += (jy[o + x] - jyd) * ihy;
        }
        rmax = fmax(rmax, fabs(s.dd[i] * ih - div));
        s.dd[i] = T(0);
      }
      if (p.ny > 1)
        cl.sync();
      else
        __syncthreads();
    }
    // beam current of this level at the half-slice n + 1/2 (own rows); the flag is cleared
    // by CTA 0 after B2, once every CTA has read it
    const bool beam_slice = s.misc[M_JFLAG] != 0;
    if (beam_slice) {
      T* jb = (T*)p.jbeam + (((size_t)s1 * nz + n) * 3) * (size_t)p.nx * p.ny;
      for (int i = tid; i < 3 * p.RB * p.nx; i += NT) {
        const int c = i >> (p.logRB + p.lognx);
        const int rem = i & ((p.RB << p.lognx) - 1);
        const size_t g = (size_t)c * p.nx * p.ny + ((size_t)me << p.logRB) * p.nx + rem;
        s.J[((size_t)c * p.JR + p.JOFF) * p.nx + rem] += ldcg(jb + g);
        jb[g] = T(0);
      }
    }
    if (snap_step || cap_step) {
      __syncthreads();
      T* sn = (T*)p.snap;
      T* jc = jcap;
      for (int i = tid; i < 3 * p.RB * p.nx; i += NT) {
        const int c = i >> (p.logRB + p.lognx);
        const int rem = i & ((p.RB << p.lognx) - 1);
        const T v = s.J[((size_t)c * p.JR + p.JOFF) * p.nx + rem];
        if (snap_step) sn[(((size_t)(6 + c) * nz + n) * p.ny + (me << p.logRB)) * p.nx + rem] = v;
        // the current of the s-step in [nzeta][3][ny][nx] (the denoiser's layout)
        if (cap_step) jc[(((size_t)n * 3 + c) * p.ny + (me << p.logRB)) * p.nx + rem] = v;
      }
    }
    const T* const jext = (const T*)(dn2 ? p.dn_jext[k & 3] : DN ? nullptr : p.jext);
    if (jext) {
      // second pass of a denoised s-step: the half-slice's current is the given one
      __syncthreads();
      const T* je = jext;
      for (int i = tid; i < 3 * p.RB * p.nx; i += NT) {
        const int c = i >> (p.logRB + p.lognx);
        const int rem = i & ((p.RB << p.lognx) - 1);
        s.J[((size_t)c * p.JR + p.JOFF) * p.nx + rem] =
            ldcg(je + (((size_t)n * 3 + c) * p.ny + (me << p.logRB)) * p.nx + rem);
      }
    }
    if (beam_slice || snap_step || cap_step || jext) __syncthreads();
    TIMER_MARK(PH_BEAM);
    // ---------------- B: row FFTs of the currents, transposed to the kx owners ------------
    forward_rows<T, SH>(cl, p, s, me, true);
    TIMER_MARK(PH_FWD);
    // streamed state: block n-1 of the input, read after the solve below
    if constexpr (CANON)
      if (p.io_chunk && tid == 0 && me == 0 && n >= 1) wait_input(p, k, n - 1, s.misc + M_IOSEEN);
    cl.sync();                                                      // B2
    if (tid == 0 && me == 0) p.jflag[(size_t)s1 * nz + n] = 0;
    TIMER_MARK(PH_B2);
    // ---------------- C: column FFTs, per-mode solve, inverse column FFTs ------------------
    if constexpr (sizeof(T) == 4) {
      for (int i = 4 * tid; i < 3 * jplane; i += 4 * NT)
        *reinterpret_cast<float4*>(s.J + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (int i = tid; i < 3 * jplane; i += NT) s.J[i] = T(0);
    }
    column_ffts<T, SH>(p, s, 0, 3, false);
    __syncthreads();
    TIMER_MARK(PH_COLF);
    if (has_mode) {
      Cx<T> Jx = s.SC[((size_t)0 * p.KB + kxl) * p.ny + q];
      Cx<T> Jy = s.SC[((size_t)1 * p.KB + kxl) * p.ny + q];
      Cx<T> Jz = s.SC[((size_t)2 * p.KB + kxl) * p.ny + q];
      if (p.ny > 1) Jy = Jy * s.shy[kyi];
      if (masked) Jx = Jy = Jz = cx<T>(T(0), T(0));
      // corrector: R at slice n+1 was built with j_{n+1/2} := j_{n+3/2}
      if (n + 1 < nz) {
        S1.Rx = S1.Rx - (T(0.25) * Dl) * (Jx - jpx);
        S1.Ry = S1.Ry - (T(0.25) * Dl) * (Jy - jpy);
      }
      // new level, block n+1 = {R, E_z, B_z at slice n+1; j at n+1/2}
      if (blk_ok(n + 1, 0)) {
        stw[blk(n + 1, 0)] = S1.Rx;
        stw[blk(n + 1, 1)] = S1.Ry;
        stw[blk(n + 1, 2)] = S1.Ez;
        stw[blk(n + 1, 3)] = S1.Bz;
      }
      stw[blk(n + 1, 4)] = Jx;
      stw[blk(n + 1, 5)] = Jy;
      // old level at slice n; j^0 at n -/+ 1/2
      const Cx<T> j0mx = n > 0 ? o[4] : j0px;
      const Cx<T> j0my = n > 0 ? o[5] : j0py;
      Mode6<T> S0;
      if (masked) {
        S0.Rx = S0.Ry = S0.Lx = S0.Ly = S0.Ez = S0.Bz = cx<T>(T(0), T(0));
      } else {
        S0 = slice_solve(kx, ky, hn, Dl, S1, o[0], o[1], o[2], o[3], j0mx, j0my, j0px, j0py, Jx,
                         Jy, Jz);
      }
      // fields E, B (Eqs. Rx..Ly) for the inverse transform
      Cx<T>* sc = s.SC + (size_t)kxl * p.ny + q;
      const size_t cs = (size_t)p.KB * p.ny;
      sc[0 * cs] = T(0.5) * (S0.Rx + S0.Lx);
      sc[1 * cs] = T(0.5) * (S0.Ry + S0.Ly);
      sc[2 * cs] = S0.Ez;
      sc[3 * cs] = T(0.5) * (S0.Ly - S0.Ry);
      sc[4 * cs] = T(0.5) * (S0.Rx - S0.Lx);
      sc[5 * cs] = S0.Bz;
      S1 = S0;
      jpx = Jx;
      jpy = Jy;
      j0px = j0mx;
      j0py = j0my;
      if (n == 0) {
        stw[blk(0, 0)] = S0.Rx;
        stw[blk(0, 1)] = S0.Ry;
        stw[blk(0, 2)] = S0.Ez;
        stw[blk(0, 3)] = S0.Bz;
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c)
          o[c] = blk_ok(n - 1, c) ? ldcg(st + blk(n - 1, c)) : cx<T>(T(0), T(0));
      }
    }
    __syncthreads();
    TIMER_MARK(PH_SOLVE);
    column_ffts<T, SH>(p, s, 0, 6, true);
    __syncthreads();
    TIMER_MARK(PH_COLI);
    scatter_to_rows(cl, p, s, me);
    TIMER_MARK(PH_SCAT);
    if (waits && tid == 0 && me == 0)
      wait_for(p, pcid, prog_value(item - 1, nz, min(nz, nz - n + 3)));   // down to n-3
    cl.sync();                                                      // B3
    // the predecessor is now known to be done down to slice n-3: counters of slice n-1,
    // loaded by the last warp (no inverse-transform task) so that no transform waits on them
    if (tid == NT - 32 && n > 0) {
      s.misc[M_RQN] = ldcg(p.rq.cnt + (size_t)s1 * nz + (n - 1));
      s.misc[M_JFLAG] = ldcg(p.jflag + (size_t)s1 * nz + (n - 1));
    }
    TIMER_MARK(PH_B3);
    // ---------------- D: inverse rows -> real-space fields of slice n ----------------------
    {
      T fs = T(0);
      inverse_rows<T, SH>(p, s, Fnew, fs);
      fe += (double)(varh ? fs * hn : fs);
    }
    TIMER_MARK(PH_INV);
    if constexpr (sizeof(T) == 4) {
      // SR has been consumed: it holds the fixed-point accumulators of the next push
      __syncthreads();
      for (int i = 4 * tid; i < 3 * jplane; i += 4 * NT)
        *reinterpret_cast<int4*>(s.Jint + i) = make_int4(0, 0, 0, 0);
    }
    cl.sync();                                                      // B4: fields of slice n
    TIMER_MARK(PH_B4);
    if (resid) {
      // Gauss residual on plane n: d_x L_x + d_y L_y - (rho - j_z), L_x = E_x - B_y,
      // L_y = E_y + B_x, central differences; rho - j_z = arrival density + background.  The
      // row above the band is the fields' halo row, the row below the last own row of the CTA
      // below (its fields of slice n stay until its inverse transform of slice n - 2).
      const T* Ex = Fnew;
      const T* Ey = Fnew + fplane;
      const T* Bx = Fnew + 3 * (size_t)fplane;
      const T* By = Fnew + 4 * (size_t)fplane;
      const T hihx = T(0.5 / p.hx), hihy = T(0.5 / p.hy);
      const int below = (me + p.C - 1) & (p.C - 1);
      const size_t lrow = (size_t)(p.RB - 1) * p.nx;
      const uint32_t eyb = p.ny > 1 ? cluster_addr(sh_addr(Ey + lrow), below) : 0u;
      const uint32_t bxb = p.ny > 1 ? cluster_addr(sh_addr(Bx + lrow), below) : 0u;
      for (int i = tid; i < rbe * p.nx; i += NT) {
        const int row = i >> p.lognx, x = i & (p.nx - 1);
        const int o = row * p.nx;
        const int xp = (x + 1) & (p.nx - 1), xm = (x - 1) & (p.nx - 1);
        T g = ((Ex[o + xp] - By[o + xp]) - (Ex[o + xm] - By[o + xm])) * hihx;
        if (p.ny > 1) {
          const T lyu = Ey[o + p.nx + x] + Bx[o + p.nx + x];
          const T lyd = row > 0 ? Ey[o - p.nx + x] + Bx[o - p.nx + x]
                                : ldc(eyb + (uint32_t)(x * sizeof(T)), T(0)) +
                                      ldc(bxb + (uint32_t)(x * sizeof(T)), T(0));
          g += (lyu - lyd) * hihy;
        }
        T bg = T(p.bg_qn);
        if (p.chan_a != 0.0) {
          const T dx = T(x - (p.nx >> 1)) * s.cst[K_HX];
          const T dy = p.ny > 1 ? T((me << p.logRB) + row - (p.ny >> 1)) * s.cst[K_HY] : T(0);
          bg *= T(1) + T(p.chan_a) * exp(-(dx * dx + dy * dy) * T(p.chan_ir2));
        }
        gmax = fmax(gmax, fabs(g - (dn_n[i] + bg)));
        dn_n[i] = T(0);
      }
    }
    if (p.diag) {
      const int yc = p.ny / 2;
      if (tid == 0 && (yc >> p.logRB) == me)
        p.onaxis[sl * nz + n] = (double)Fnew[((size_t)2 * p.FR + (yc & (p.RB - 1))) * p.nx + nxh];
    }
    if (snap_step) {
      T* sn = (T*)p.snap;
      for (int i = tid; i < 6 * p.RB * p.nx; i += NT) {
        const int c = i >> (p.logRB + p.lognx);
        const int rem = i & ((p.RB << p.lognx) - 1);
        sn[(((size_t)c * nz + n) * p.ny + (me << p.logRB)) * p.nx + rem] =
            Fnew[(size_t)c * fplane + rem];
      }
    }
    // ---------------- E: stored particles of cell (zeta_n, zeta_{n+1}] along s -------------
    // (most cells hold no stored particle: the call is skipped, uniformly over the CTA)
    if (s.misc[M_STN] > 0 && !p.skip_stored && !dn1)
      stored_phase(p, s, Fnew, Fcur, s1, s2, n, me, s.misc[M_STN], varh);
    TIMER_MARK(PH_E);
    T* t = Fcur;
    Fcur = Fnew;
    Fnew = t;
  }
  // publish completion of the march
  __syncthreads();
  if (tid == 0) __threadfence();
  cl.sync();
  if (p.P > 1 && me == 0 && tid == 0) st_release_u64(p.progress + cid, prog_value(item, nz, nz));
  if constexpr (CANON)
    if (p.io_chunk && me == 0 && tid == 0) st_release_sys_u64(p.io_done + cid, prog_value(k, nz, nz));
  if (dn1 && me == 0 && tid == 0) st_release_sys_u64(p.dn_done + cid, prog_value(item, nz, nz));

  if (resid) {
    // the march's largest residuals: non-negative doubles order like their bit patterns
    double v[2] = {(double)rmax, (double)gmax};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      for (int off = 16; off > 0; off >>= 1) v[c] = fmax(v[c], __shfl_xor_sync(0xffffffffu, v[c], off));
      if ((tid & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(s.dacc + c),
                  (unsigned long long)__double_as_longlong(v[c]));
    }
    cl.sync();
    // the cluster's maxima: CTA 0 reads every CTA's partial maxima
    if (me == 0 && tid < 2) {
      double m = 0.0;
      for (int r = 0; r < p.C; ++r) m = fmax(m, ldc(cluster_addr(sh_addr(s.dacc + tid), r), 0.0));
      (tid == 0 ? p.resid_out : p.gauss_out)[sl] = m;
    }
    cl.sync();
  }
  // diagnostics: per-CTA FP64 partials
  if (p.diag) {
    warp_diag_add(s.dwarp, DG_FIELD, fe);
    __syncthreads();
    if (tid < kNDiag) {
      double v = 0.0;
      for (int w = 0; w < (NT >> 5); ++w) v += s.dwarp[w * kNDiag + tid];
      // variable zeta-step: each slice's sums were weighted by its slab thickness
      const double hw = p.varh ? 1.0 : p.h;
      const double hv = tid == DG_FIELD ? 0.5 * p.hx * p.hy * hw
                        : tid == DG_FLUX ? p.hx * p.hy * hw
                                         : 1.0;
      p.diag_out[((size_t)sl * kNDiag + tid) * p.C + me] = v * hv;
      // watchdog: a NaN or infinity anywhere in the slice fields or in a particle's momentum
      // reaches these FP64 sums
      if ((tid == DG_FIELD || tid == DG_KIN) && !isfinite(v)) atomicOr(p.err, ERR_NONFINITE);
    }
    __syncthreads();
  }
}

template <typename T, bool CANON, int SH, bool DN>
__device__ __forceinline__ void march_launch(const Params& p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const Sm<T> s = carve<T>(p, smem);
  load_tables(p, s);
  if (threadIdx.x < kNDiag) s.dacc[threadIdx.x] = 0.0;
  __syncthreads();
  const int cid = (int)(blockIdx.x / p.C);
  // a chain's march index is 2k + pass
  for (long long it = cid; it < p.nsteps; it += p.P) {
    const long long item = DN ? 2 * p.k0 + it : p.k0 + it;
    march<T, CANON, SH, DN>(p, s, cl, DN ? item >> 1 : item, cid, item);
  }
}

template <typename T, bool CANON = false, int SH = 0, bool DN = false>
__global__ void __launch_bounds__(512, 1) march_kernel(const Params p) {
  march_launch<T, CANON, SH, DN>(p);
}

#ifndef GEMPIC_CHAIN_TU
// FP64 with at most 256 threads per CTA (the 2-D and small 3-D grids): up to 255 registers a
// thread, so the FP64 march keeps its state in registers instead of spilling it
__global__ void __launch_bounds__(256, 1) march_kernel_fp64_narrow(const Params p) {
  march_launch<double, false, 0, false>(p);
}
#endif

#ifndef GEMPIC_CHAIN_TU
// Batched scan: one persistent launch over independent simulations.  Each CTA takes work
// items (simulation, march index) from a queue in global memory, in the order the host laid
// out (s-step by s-step, the costliest simulations first); the march of s-step k of a
// simulation waits for that simulation's s-step k-1 with the bounded per-slice wavefront wait,
// so a large simulation marches many s-steps at once while small ones fill the other SMs.
// Every CTA of the launch is resident (one per SM), and an item is taken only after all items
// before it, so the march it waits for is already running: no wait can block forever.
template <typename T>
__global__ void __launch_bounds__(512, 1) batch_kernel(const Params* ps, const int2* items,
                                                       int nitems, int* head) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) Params sp;
  __shared__ int item;
  cg::cluster_group cl = cg::this_cluster();
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item = atomicAdd(head, 1);
    __syncthreads();
    const int it = item;
    if (it >= nitems) break;
    const int2 w = items[it];
    const int* src = reinterpret_cast<const int*>(ps + w.x);
    int* dst = reinterpret_cast<int*>(&sp);
    for (int i = threadIdx.x; i < (int)(sizeof(Params) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    const Sm<T> s = carve<T>(sp, smem);
    load_tables(sp, s);
    if (threadIdx.x < kNDiag) s.dacc[threadIdx.x] = 0.0;
    __syncthreads();
    march<T, false, 0, false>(sp, s, cl, sp.k0 + w.y, w.y, sp.k0 + w.y);
  }
}

cudaError_t configure_batch(int precision, int smem) {
  if (precision == 64)
    return cudaFuncSetAttribute(batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return cudaFuncSetAttribute(batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t batch_occupancy(int precision, int nthreads, int smem, int* blocks) {
  if (precision == 64)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_kernel<double>, nthreads, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_kernel<float>, nthreads, smem);
}

cudaError_t launch_batch(int precision, const Params* ps, const int2* items, int nitems, int* head,
                         int grid, int nthreads, int smem, cudaStream_t s) {
  if (precision == 64)
    batch_kernel<double><<<grid, nthreads, smem, s>>>(ps, items, nitems, head);
  else
    batch_kernel<float><<<grid, nthreads, smem, s>>>(ps, items, nitems, head);
  return cudaGetLastError();
}

// tables of the allocation-free entry point, built on the device (same formulas as the host
// tables of gempic_create): twx, twy, shx, shy (complex), kx, ky (real)
template <typename T>
__global__ void tables_kernel(const Params p, void* dst) {
  const double pi = 3.14159265358979323846;
  const int nxh = p.nx / 2, nyh = p.ny > 1 ? p.ny / 2 : 1;
  Cx<T>* c = (Cx<T>*)dst;
  T* r = (T*)(c + nxh + nyh + nxh + p.ny);
  for (int i = threadIdx.x; i < nxh; i += blockDim.x) {
    const double a = -2 * pi * i / p.nx;
    c[i] = cx<T>(T(cos(a)), T(sin(a)));
    const double kx = 2 * pi * i / (p.nx * p.hx);
    c[nxh + nyh + i] = cx<T>(T(cos(-0.5 * kx * p.hx)), T(sin(-0.5 * kx * p.hx)));
    r[i] = T(kx);
  }
  for (int j = threadIdx.x; j < nyh; j += blockDim.x) {
    const double a = p.ny > 1 ? -2 * pi * j / p.ny : 0.0;
    c[nxh + j] = cx<T>(T(cos(a)), T(sin(a)));
  }
  for (int j = threadIdx.x; j < p.ny; j += blockDim.x) {
    const int f = (p.ny == 1) ? 0 : (j < (p.ny + 1) / 2 ? j : j - p.ny);
    const double ky = 2 * pi * (double)f / ((double)p.ny * p.hy);
    c[nxh + nyh + nxh + j] = cx<T>(T(cos(-0.5 * ky * p.hy)), T(sin(-0.5 * ky * p.hy)));
    r[nxh + j] = T(ky);
  }
}

// ------------------------------------------------------------------------------------------
// laser initial condition (Eq. E_laser): R = 2E (forward wave) on every slice, spectral
// ------------------------------------------------------------------------------------------
template <typename T, int SH = 0>
__global__ void __launch_bounds__(512, 1)
    laser_kernel(const Params p, double a0, double waist, double dur, double zc, int pol) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const Sm<T> s = carve<T>(p, smem);
  load_tables(p, s);
  __syncthreads();
  const int me = (int)cl.block_rank();
  const int cid = (int)(blockIdx.x / p.C);
  const int ncl = (int)(gridDim.x / p.C);
  Cx<T>* stw = (Cx<T>*)p.state;
  const double xc = 0.5 * p.nx * p.hx, yc = 0.5 * p.ny * p.hy;
  const int plane = p.RB * p.nx;
  for (int n = cid; n < p.nz; n += ncl) {
    const double phi = (p.varh ? p.zpd[n] : n * p.h) - zc;
    const double env = a0 * cos(phi) * exp(-phi * phi / (dur * dur));
    for (int i = threadIdx.x; i < 3 * plane; i += blockDim.x) {
      const int c = i / plane;
      const int rem = i - c * plane;
      const int yl = rem / p.nx, x = rem - yl * p.nx;
      const double dx = x * p.hx - xc;
      const double dy = p.ny > 1 ? ((me << p.logRB) + yl) * p.hy - yc : 0.0;
      const double E = env * exp(-(dy * dy + dx * dx) / (waist * waist));
      s.J[((size_t)c * p.JR + yl + p.JOFF) * p.nx + x] = (c == 2) ? T(2.0 * E) : T(0);
    }
    __syncthreads();
    forward_rows<T, SH>(cl, p, s, me, false);
    cl.sync();
    column_ffts<T, SH>(p, s, 2, 3, false);
    __syncthreads();
    for (int m = threadIdx.x; m < p.M; m += blockDim.x) {
      const int kxl = m >> p.logny, q = m & (p.ny - 1);
      Cx<T> v = s.SC[((size_t)2 * p.KB + kxl) * p.ny + q];
      if (p.ny > 1 && ky_of_pos(p.logny, q) == p.ny / 2) v = cx<T>(T(0), T(0));
      const Cx<T> z = cx<T>(T(0), T(0));
      for (int c = 0; c < 6; ++c)
        stw[(((size_t)n * p.C + me) * 6 + c) * p.M + m] = (c == pol) ? v : z;
    }
    cl.sync();
  }
}

// ------------------------------------------------------------------------------------------
// Gaussian bunch placed in the box at creation (beam particles of Sec. 5.1, equal charges):
// macroparticle i takes the uniforms ((o >> 11) + 1) 2^-53 in (0, 1] from SplitMix64 outputs
// o = 4 i + j of the bunch's stream and two normal pairs by the Box-Muller transform; it is
// appended to its slab's bucket of the level-0 stored set (ring slot 0).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double uniform53(unsigned long long s, unsigned long long c) {
  return (double)((splitmix64(s, c) >> 11) + 1ull) * (1.0 / 9007199254740992.0);
}

template <typename T>
__global__ void beam_kernel(const Params p, BeamArgs b) {
  const double two_pi = 6.283185307179586476925;
  const double lx = p.nx * p.hx, ly = p.ny * p.hy;
  const double len = p.varh ? p.zpd[p.nz] : p.nz * p.h;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < b.n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long c = 4ull * (unsigned long long)i;
    const double v0 = uniform53(b.seed, c), v1 = uniform53(b.seed, c + 1);
    const double v2 = uniform53(b.seed, c + 2), v3 = uniform53(b.seed, c + 3);
    const double r01 = sqrt(-2.0 * log(v0)), r23 = sqrt(-2.0 * log(v2));
    const double g0 = r01 * cos(two_pi * v1), g1 = r01 * sin(two_pi * v1);
    const double g2 = r23 * cos(two_pi * v3), g3 = r23 * sin(two_pi * v3);
    const double zeta = b.zc + b.sz * g2;
    if (!(zeta > 0.0) || !(zeta <= len)) continue;
    // slab m with zeta_m < zeta <= zeta_{m+1}, in-slab offset fz in (0, 1]
    int m;
    double fz;
    if (p.varh) {
      int lo = 0, hi = p.nz;            // zpd[lo] < zeta <= zpd[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (p.zpd[mid] < zeta) lo = mid; else hi = mid;
      }
      m = lo;
      fz = (zeta - p.zpd[m]) / (p.zpd[m + 1] - p.zpd[m]);
    } else {
      const double Z = zeta / p.h;
      m = (int)ceil(Z) - 1;
      fz = Z - m;
    }
    if (m < 0 || m >= p.nz) continue;
    double x = fmod(b.xc + b.sr * g0, lx);
    if (x < 0.0) x += lx;
    double y = 0.0;
    if (p.ny > 1) {
      y = fmod(b.yc + b.sr * g1, ly);
      if (y < 0.0) y += ly;
    }
    const double X = x / p.hx, Y = p.ny > 1 ? y / p.hy : 0.0;
    const double fX = floor(X), fY = floor(Y);
    PState<T> P;
    P.ix = ((int)fX % p.nx + p.nx) % p.nx;
    P.iy = p.ny > 1 ? ((int)fY % p.ny + p.ny) % p.ny : 0;
    P.sp = b.sp;
    P.fx = T(X - fX);
    P.fy = T(Y - fY);
    const double gi = b.gamma * (1.0 + b.spread * g3);
    P.u = V3<T>{T(0), T(0), T(sqrt(fmax(gi * gi - 1.0, 0.0)))};
    P.q = T(b.q);
    P.sig = T(0);
    if (!store_append(p.st, p, 0, m, P, T(fz))) atomicOr(p.err, ERR_BCAP);
  }
}

// ------------------------------------------------------------------------------------------
// layout conversion of the spectral state: blocks [nz+1][C][6][M] <-> [6][nz][ny][nx/2]
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void export_kernel(const Params p, Cx<T>* dst, const Cx<T>* src, int dir) {
  const size_t nxh = p.nx / 2;
  const size_t total = (size_t)6 * p.nz * p.ny * nxh;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nxh);
    const int ky = (int)((i / nxh) % p.ny);
    const int n = (int)((i / (nxh * p.ny)) % p.nz);
    const int c = (int)(i / (nxh * p.ny * p.nz));
    const int b = c >= 4 ? n + 1 : n;
    const int r = kx / p.KB, kxl = kx % p.KB;
    const size_t e = (((size_t)b * p.C + r) * 6 + c) * p.M + (size_t)kxl * p.ny +
                     pos_of_ky(p.logny, ky);
    if (dir == 0)
      dst[i] = src[e];
    else
      dst[e] = src[i];
  }
}

// ------------------------------------------------------------------------------------------
// host-side launchers
// ------------------------------------------------------------------------------------------
#endif  // GEMPIC_CHAIN_TU

static int align16(int v) { return (v + 15) / 16 * 16; }

#ifndef GEMPIC_CHAIN_TU
int smem_layout(Params& p, int eb) {
  // halo geometry: fields own rows + 1 above, currents rows -1 .. RB + 1 (3-D only)
  p.FR = p.ny > 1 ? p.RB + 1 : 1;
  p.JR = p.ny > 1 ? p.RB + 3 : 1;
  p.JOFF = p.ny > 1 ? 1 : 0;
  p.mig_cap = p.ny > 1 ? 128 : 0;
  p.nwork = std::min(p.nthreads / 32, 3 * p.FR);
  const int nxh = p.nx / 2;
  const int nyh = p.ny > 1 ? p.ny / 2 : 1;
  int o = 0;
  p.o_f0 = o;
  o += align16(6 * p.FR * p.nx * eb);
  p.o_f1 = o;
  o += align16(6 * p.FR * p.nx * eb);
  p.o_j = o;
  o += align16(3 * p.JR * p.nx * eb);
  p.o_recv = o;
  o += align16((p.ny > 1 ? 9 : 1) * p.nx * eb);
  p.o_sr = o;
  const int sr_bytes = align16(6 * p.FR * nxh * 2 * eb);
  o += sr_bytes;
  p.o_sc = o;
  const int sc_bytes = align16(6 * p.KB * p.ny * 2 * eb);
  o += sc_bytes;
  // row-FFT work rows live in SR (forward transform) and SC (inverse) when they fit
  const int work = align16(p.nwork * p.nx * 2 * eb);
  p.o_workB = work <= sr_bytes ? p.o_sr : o;
  if (work > sr_bytes) o += work;
  p.o_workD = work <= sc_bytes ? p.o_sc : o;
  if (work > sc_bytes) o += work;
  p.o_tw = o;
  o += align16((nxh + nyh + nxh + p.ny) * 2 * eb + (nxh + p.ny + 32) * eb);
  p.o_inbox = o;
  o += align16(p.mig_cap * 4) + align16(7 * p.mig_cap * eb);
  p.o_outbox = o;
  if (p.ny > 1) o += align16(2 * kOutCap * 4) + align16(7 * kOutCap * eb);
  p.o_part = o;
  // free-slot stack: bounded (a slot freed beyond it stays empty until the next s-step), so
  // that a particle slot costs 4 + 7 reals of shared memory
  p.fcap = std::min(p.pcap, 512);
  o += align16(p.pcap * 4) + align16(7 * p.pcap * eb + p.fcap * 4);
  // verification mode: start-minus-end CIC densities of the own rows (continuity residual)
  // and two planes of arrival densities (Gauss residual)
  p.o_dd = o;
  if (p.resid) o += align16(3 * (p.ny > 1 ? p.RB : 1) * p.nx * eb);
  p.o_misc = o;
  o += 32 + kNDiag * 8 + (p.nthreads / 32) * kNDiag * 8;
  p.smem_bytes = align16(o);
  return p.smem_bytes;
}

#endif  // GEMPIC_CHAIN_TU

// kernel instantiation for the grid: 1 = FP32 128 x 128 with an even band (length-128
// transforms only), 0 = any size
static int shape_class(int precision, const Params& p) {
  return precision == 32 && p.nx == 128 && p.ny == 128 && (p.RB & 1) == 0 && !p.gt1 && !p.varh &&
                 !p.resid
             ? 1 : 0;
}

// The dynamic shared-memory limit is an attribute of the kernel function, shared by every
// simulation of the process: it is raised to the device's opt-in maximum (each launch asks
// for its own size), never set to one simulation's size, which would break the launches of a
// larger simulation alive at the same time.
template <typename K>
static cudaError_t cfg_kernel(K* k, int smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(smem, optin));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

#ifndef GEMPIC_CHAIN_TU
cudaError_t configure_kernels(int precision, int smem, int) {
  if (precision == 64) {
    cudaError_t e = cfg_kernel(march_kernel<double>, smem);
    if (e == cudaSuccess) e = cfg_kernel(march_kernel_fp64_narrow, smem);
    return e == cudaSuccess ? cfg_kernel(laser_kernel<double>, smem) : e;
  }
  cudaError_t e = cfg_kernel(march_kernel<float>, smem);
  if (e == cudaSuccess) e = cfg_kernel(laser_kernel<float>, smem);
  if (e == cudaSuccess) e = cfg_kernel(march_kernel<float, false, 1>, smem);
  if (e == cudaSuccess) e = cfg_kernel(laser_kernel<float, 1>, smem);
  if (e == cudaSuccess) e = configure_chain(smem);
  return e;
}

#endif  // GEMPIC_CHAIN_TU

static cudaLaunchConfig_t make_cfg(const Params& p, int nclusters, cudaStream_t s,
                                   cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t c = {};
  c.gridDim = dim3((unsigned)(nclusters * p.C), 1, 1);
  c.blockDim = dim3((unsigned)p.nthreads, 1, 1);
  c.dynamicSmemBytes = (size_t)p.smem_bytes;
  c.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  c.attrs = attr;
  c.numAttrs = 1;
  return c;
}

#ifndef GEMPIC_CHAIN_TU
cudaError_t launch_march(int precision, const Params& p, cudaStream_t s) {
  if (p.dn_pipe) return precision == 32 ? launch_march_chain(p, s) : cudaErrorInvalidValue;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t c = make_cfg(p, p.P, s, attr);
  if (precision == 64 && p.nthreads <= 256)
    return cudaLaunchKernelEx(&c, march_kernel_fp64_narrow, p);
  if (precision == 64) return cudaLaunchKernelEx(&c, march_kernel<double>, p);
  if (shape_class(precision, p) == 1) return cudaLaunchKernelEx(&c, march_kernel<float, false, 1>, p);
  return cudaLaunchKernelEx(&c, march_kernel<float>, p);
}

cudaError_t launch_laser_init(int precision, const Params& p, double a0, double waist, double dur,
                              double zc, int pol, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  int ncl = 1;
  max_active_clusters(precision, p, &ncl);
  if (ncl < 1) ncl = 1;
  if (ncl > p.nz) ncl = p.nz;
  cudaLaunchConfig_t c = make_cfg(p, ncl, s, attr);
  if (precision == 64) return cudaLaunchKernelEx(&c, laser_kernel<double>, p, a0, waist, dur, zc, pol);
  if (shape_class(precision, p) == 1)
    return cudaLaunchKernelEx(&c, laser_kernel<float, 1>, p, a0, waist, dur, zc, pol);
  return cudaLaunchKernelEx(&c, laser_kernel<float>, p, a0, waist, dur, zc, pol);
}

cudaError_t launch_beam_init(int precision, const Params& p, const BeamArgs& b, cudaStream_t s) {
  if (b.n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((b.n + 255) / 256, 4096);
  if (precision == 64)
    beam_kernel<double><<<blocks, 256, 0, s>>>(p, b);
  else
    beam_kernel<float><<<blocks, 256, 0, s>>>(p, b);
  return cudaGetLastError();
}

cudaError_t launch_export_state(int precision, const Params& p, void* dst, cudaStream_t s) {
  if (precision == 64)
    export_kernel<double><<<264, 256, 0, s>>>(p, (Cx<double>*)dst, (const Cx<double>*)p.state, 0);
  else
    export_kernel<float><<<264, 256, 0, s>>>(p, (Cx<float>*)dst, (const Cx<float>*)p.state, 0);
  return cudaGetLastError();
}

cudaError_t launch_import_state(int precision, const Params& p, const void* src, cudaStream_t s) {
  if (precision == 64)
    export_kernel<double><<<264, 256, 0, s>>>(p, (Cx<double>*)p.state, (const Cx<double>*)src, 1);
  else
    export_kernel<float><<<264, 256, 0, s>>>(p, (Cx<float>*)p.state, (const Cx<float>*)src, 1);
  return cudaGetLastError();
}

cudaError_t configure_march_canon(int precision, int smem) {
  if (precision == 64) return cfg_kernel(march_kernel<double, true>, smem);
  cudaError_t e = cfg_kernel(march_kernel<float, true>, smem);
  return e == cudaSuccess ? cfg_kernel(march_kernel<float, true, 1>, smem) : e;
}

cudaError_t launch_march_canon(int precision, const Params& p, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t c = make_cfg(p, p.P, s, attr);
  if (precision == 64) return cudaLaunchKernelEx(&c, march_kernel<double, true>, p);
  if (shape_class(precision, p) == 1) return cudaLaunchKernelEx(&c, march_kernel<float, true, 1>, p);
  return cudaLaunchKernelEx(&c, march_kernel<float, true>, p);
}

cudaError_t launch_tables(int precision, const Params& p, void* dst, cudaStream_t s) {
  if (precision == 64)
    tables_kernel<double><<<1, 256, 0, s>>>(p, dst);
  else
    tables_kernel<float><<<1, 256, 0, s>>>(p, dst);
  return cudaGetLastError();
}

cudaError_t max_active_clusters(int precision, const Params& p, int* n) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t c = make_cfg(p, 1, 0, attr);
  if (precision == 64 && p.nthreads <= 256)
    return cudaOccupancyMaxActiveClusters(n, march_kernel_fp64_narrow, &c);
  if (precision == 64) return cudaOccupancyMaxActiveClusters(n, march_kernel<double>, &c);
  if (shape_class(precision, p) == 1)
    return cudaOccupancyMaxActiveClusters(n, march_kernel<float, false, 1>, &c);
  return cudaOccupancyMaxActiveClusters(n, march_kernel<float>, &c);
}

#else  // GEMPIC_CHAIN_TU

// the denoised chain's instantiations of the march (FP32; the 128 x 128 one where it applies)
cudaError_t configure_chain(int smem) {
  cudaError_t e = cfg_kernel(march_kernel<float, false, 0, true>, smem);
  return e == cudaSuccess ? cfg_kernel(march_kernel<float, false, 1, true>, smem) : e;
}

cudaError_t launch_march_chain(const Params& p, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t c = make_cfg(p, p.P, s, attr);
  if (shape_class(32, p) == 1) return cudaLaunchKernelEx(&c, march_kernel<float, false, 1, true>, p);
  return cudaLaunchKernelEx(&c, march_kernel<float, false, 0, true>, p);
}
#endif  // GEMPIC_CHAIN_TU

}  // namespace gempic
