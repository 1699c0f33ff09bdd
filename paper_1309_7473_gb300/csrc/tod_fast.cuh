// Device helpers shared by the two register-FFT paths of A = P^T N^-1 P for FP32
// compute (tod_fast.cu: one detector per complex sequence; tod_pair.cu: two
// detectors per complex sequence): launch shapes of the column FFTs, the
// fixed-point pixel rule, the noise-filter law on the FP32 pipes and the binning
// run accumulator.
#pragma once

#include "common.cuh"
#include "fft_reg.cuh"
#include "tod_common.cuh"

namespace cmm {

// Tuning knobs (compile-time; the defaults are the measured best on GB300).
#ifndef CMM_DETS_PER_CTA
#define CMM_DETS_PER_CTA 1
#endif
#ifndef CMM_COL_THREADS_PER_SM
#define CMM_COL_THREADS_PER_SM 1024
#endif
#ifndef CMM_INV_THREADS_PER_SM
#define CMM_INV_THREADS_PER_SM 768
#endif
#ifndef CMM_FILTER_MINB
#define CMM_FILTER_MINB 4
#endif
#ifndef CMM_GEN_UNROLL
#define CMM_GEN_UNROLL 2
#endif
#ifndef CMM_COLJ_256
#define CMM_COLJ_256 16   // columns per CTA of the column passes at R = 256
#endif
#ifndef CMM_BIN_HALVES
#define CMM_BIN_HALVES 1   // consecutive samples per lane in the binning: 8 x this
#endif
#ifndef CMM_BIN_UNROLL
#define CMM_BIN_UNROLL 1
#endif

constexpr int kDetsPerCta = CMM_DETS_PER_CTA;
constexpr int kGenUnroll = CMM_GEN_UNROLL;
constexpr int kBinUnroll = CMM_BIN_UNROLL;
constexpr int kBinHalves = CMM_BIN_HALVES;
#ifndef CMM_V8
#define CMM_V8 1   // binning: a lane's 8 rotations / cached pixels by 32-byte loads (1) or 16-byte loads (0)
#endif
constexpr int kE = 16;     // elements per thread in the column FFT

// Columns per CTA: 32 (one per lane) for R <= 128, 16 (one per half-warp lane)
// for R = 256; either way a half-warp reads 16 complex = 32 consecutive samples
// and touches 32 different shared-memory banks.
template <int R> struct ColShape {
  static constexpr int J = R >= 256 ? CMM_COLJ_256 : 32;
  static constexpr int THREADS = J * R / kE;
  static constexpr int MINB = CMM_COL_THREADS_PER_SM / THREADS > 0 ? CMM_COL_THREADS_PER_SM / THREADS : 1;
  static constexpr int MINB_INV = CMM_INV_THREADS_PER_SM / THREADS > 0 ? CMM_INV_THREADS_PER_SM / THREADS : 1;
};

// GB300's FP64 unit also executes int <-> float conversions, at a small fraction
// of the FP32 rate; this helper does the one of the filter exactly on the FP32 pipe.

// Exact float of an integer 0 <= k < 2^23 (IEEE-754 single: 2^23 + k has k as its
// mantissa).
__device__ __forceinline__ float small_int_to_float(int k) {
  return __int_as_float(0x4B000000 | k) - 8388608.0f;
}

// exp2 / log2 on the special function unit; relative error of w below 1e-6.
__device__ __forceinline__ float filter_weight_law(const float4 cf, int k) {
  if (cf.w != 0.0f) return cf.x;
  const float kk = small_int_to_float(k == 0 ? 1 : k);
  const float e = exp2f(fmaf(-cf.y, __log2f(kk), cf.z));
  return __fdividef(cf.x, 1.0f + e);
}

// Pixel of a sample for the fast kernels (the rule of sample_pixel).  A sample
// outside the map gets index npix: an extra pixel that is zero in the gather copy
// and whose accumulator is never read, so the kernels take no branch on it.
template <bool PERIODIC>
__device__ __forceinline__ int pixel_fast(const int4 b, const int2 o, int ny, int nx, int npix) {
  const int ox = b.z * o.x - b.w * o.y;
  const int oy = b.w * o.x + b.z * o.y;
  int ix = (b.x + (1 << 15) + (ox >> 6)) >> 16;
  int iy = (b.y + (1 << 15) + (oy >> 6)) >> 16;
  if (PERIODIC) {
    ix %= nx;
    ix += ix < 0 ? nx : 0;
    iy %= ny;
    iy += iy < 0 ? ny : 0;
    return iy * nx + ix;
  }
  const bool in = (unsigned)ix < (unsigned)nx && (unsigned)iy < (unsigned)ny;
  return in ? iy * nx + ix : npix;
}

// w_N^e, 0 <= e < N, from the two tables w_N^(e mod C) and w_R^(e div C)
__device__ __forceinline__ float2 tw_N(const TodArgs& a, const float2* __restrict__ tw, int e) {
  const float2 lo = __ldg(tw + a.twl.Nlo_off + (e & (a.C - 1)));
  const float2 hi = __ldg(tw + a.twl.R_off + (e >> a.logC));
  return cmul(lo, hi);
}

// J interleaved columns: position pos of column cl at J pos + cl, so every access
// of the column FFT puts consecutive lanes on consecutive elements.
template <int J>
struct ColJ {
  float2* buf;
  int cl;
  __device__ __forceinline__ void st(int pos, float2 v) const { buf[pos * J + cl] = v; }
  __device__ __forceinline__ float2 ld(int pos) const { return buf[pos * J + cl]; }
  __device__ __forceinline__ int base(int pos) const { return pos * J + cl; }
  __device__ __forceinline__ void st_at(int b, int o, float2 v) const { buf[b + o * J] = v; }
  __device__ __forceinline__ float2 ld_at(int b, int o) const { return buf[b + o * J]; }
};

template <int R> struct ColPlan;
template <> struct ColPlan<64> {
  template <int SIGN, typename Addr>
  static __device__ __forceinline__ void run(float2 (&x)[kE], int i, const float2* tw, const Addr& ad) {
    rfft<SIGN, kE, 16, 4>(x, i, tw, ad);
  }
};
template <> struct ColPlan<128> {
  template <int SIGN, typename Addr>
  static __device__ __forceinline__ void run(float2 (&x)[kE], int i, const float2* tw, const Addr& ad) {
    rfft<SIGN, kE, 16, 8>(x, i, tw, ad);
  }
};
template <> struct ColPlan<256> {
  template <int SIGN, typename Addr>
  static __device__ __forceinline__ void run(float2 (&x)[kE], int i, const float2* tw, const Addr& ad) {
    rfft<SIGN, kE, 16, 16>(x, i, tw, ad);
  }
};

__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
// One 32-byte read-only load of eight floats (the 256-bit vector load of sm_100 and
// later); p must be 32-byte aligned.  A lane that needs 32 contiguous bytes gets them
// in one request touching one sector, where two 16-byte loads of lanes 32 bytes
// apart would each touch every sector twice.
__device__ __forceinline__ void ld_nc_v8(const void* p, float (&v)[8]) {
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
// The same for eight ints read once (evict-first: streamed pixel indices).
__device__ __forceinline__ void ld_cs_v8(const int* p, int (&v)[8]) {
  asm volatile("ld.global.cs.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(0.0f)
               : "memory");
}

// Run accumulator of one lane's consecutive samples: samples in the same pixel as
// the open run are summed in registers; a new pixel closes the run with one
// reduction into the FP32 partial map.  Runs in the extra pixel `skip` (samples
// outside the map) issue none: every warp would otherwise hit that one address.
struct BinRun {
  int cur = -1;   // pixel of the open run (-1: none)
  float ax = 0.f, ay = 0.f, az = 0.f;
};

template <int NC>
__device__ __forceinline__ void bin_close(float* acc32, const BinRun& r, int skip) {
  if (r.cur >= 0 && r.cur != skip) {
    if (NC == 1) red_add(acc32 + r.cur, r.ax);
    else red_add4(acc32 + 4 * r.cur, r.ax, r.ay, r.az);
  }
}

template <int NC>
__device__ __forceinline__ void bin_push8(float* acc32, BinRun& r, const int (&p)[8], const float (&u)[8],
                                          const float (&c)[8], const float (&s)[8], int skip) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (p[k] != r.cur) {
      bin_close<NC>(acc32, r, skip);
      r.cur = p[k];
      r.ax = 0.f;
      r.ay = 0.f;
      r.az = 0.f;
    }
    r.ax += u[k];
    if (NC == 3) {
      r.ay = fmaf(c[k], u[k], r.ay);
      r.az = fmaf(s[k], u[k], r.az);
    }
  }
}

}  // namespace cmm
