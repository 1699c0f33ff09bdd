// Fast path of A = P^T N^-1 P for FP32 compute (FP32 or BF16 spectrum storage).
//
// The complex length N = n_t / 2 is split as N = R C with short columns
// (R = 64 or 128) and long rows (C = N / R up to 4096):
//
//   k_fast_fwd:     pass T.  A CTA holds 32 adjacent columns; thread (lane cl, warp i)
//                   owns the 16 rows i + e R/16 of column c0 + cl, so every warp
//                   reads 64 consecutive samples at a time (coalesced boresight and
//                   gather loads).  P m is produced on the fly, transformed by a
//                   register-resident R-point FFT and stored times w_N^{c k_r}.
//   k_fast_filter:  pass F.  Row pairs (k_r, R - k_r) of C points: forward FFT, the
//                   real-FFT split, the noise filter w_d(f), the merge, inverse FFT.
//   k_fast_inv_bin: pass T'.  Inverse R-point FFTs; each warp then holds 64
//                   consecutive filtered samples in lane order, and runs of samples
//                   that fall in the same pixel are summed by a warp-level segmented
//                   scan, so that one vector FP32 reduction per run goes to an
//                   L2-resident partial map.
//   k_fast_flush:   adds the FP32 partial map into the FP64 accumulator and clears
//                   it, after every group of at most kFlushDets detectors, so each
//                   FP32 partial sums a bounded number of samples.
#include <math.h>

#include <algorithm>

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
#ifndef CMM_FILTER_MINB
#define CMM_FILTER_MINB 3
#endif
#ifndef CMM_GEN_UNROLL
#define CMM_GEN_UNROLL 2
#endif

constexpr int kDetsPerCta = CMM_DETS_PER_CTA;
constexpr int kGenUnroll = CMM_GEN_UNROLL;
constexpr int kFlushDets = 128;
constexpr int kE = 16;     // elements per thread in the column FFT

// Columns per CTA: 32 (one per lane) for R <= 128, 16 (one per half-warp lane)
// for R = 256; either way a half-warp reads 16 complex = 32 consecutive samples
// and touches 32 different shared-memory banks.
template <int R> struct ColShape {
  static constexpr int J = R >= 256 ? 16 : 32;
  static constexpr int THREADS = J * R / kE;
  static constexpr int MINB = CMM_COL_THREADS_PER_SM / THREADS > 0 ? CMM_COL_THREADS_PER_SM / THREADS : 1;
};

// GB300's FP64 unit also executes int <-> float conversions, at a small fraction
// of the FP32 rate; this helper does the one of the filter exactly on the FP32 pipe.

// Exact float of an integer 0 <= k < 2^23 (IEEE-754 single: 2^23 + k has k as its
// mantissa).
__device__ __forceinline__ float small_int_to_float(int k) {
  return __int_as_float(0x4B000000 | k) - 8388608.0f;
}

// exp2 / log2 on the special function unit; relative error of w below 1e-6.
__device__ __forceinline__ float filter_weight_fast(const float4 cf, int k) {
  if (cf.w != 0.0f) return cf.x;
  const float kk = small_int_to_float(k == 0 ? 1 : k);
  const float e = exp2f(fmaf(-cf.y, __log2f(kk), cf.z));
  return __fdividef(cf.x, 1.0f + e);
}

// (cos 2a, sin 2a) of sample t, a = psi_d + phi_t, from the FP32 (cos 2phi, sin 2phi)
__device__ __forceinline__ void response_fast(const TodArgs& a, int t, const float2 pol, float& c,
                                              float& s) {
  const float2 r2 = __ldg(a.rot2 + t);
  c = pol.x * r2.x - pol.y * r2.y;
  s = pol.y * r2.x + pol.x * r2.y;
}

// w_N^e, 0 <= e < N, from the two tables w_N^(e mod C) and w_R^(e div C)
__device__ __forceinline__ float2 tw_N(const TodArgs& a, const float2* __restrict__ tw, int e) {
  const float2 lo = __ldg(tw + a.twl.Nlo_off + (e & (a.C - 1)));
  const float2 hi = __ldg(tw + a.twl.R_off + (e >> a.logC));
  return cmul(lo, hi);
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

// (P m) at sample t of a detector: gather from the FP32 map copy at the sample's pixel
template <int NC, bool PERIODIC>
__device__ __forceinline__ float project_fast(const TodArgs& a, const int2 off, const float2 pol, int t) {
  const int4 b = __ldg(a.bore + t);
  const int p = pixel_fast<PERIODIC>(b, off, a.ny, a.nx, (int)a.npix);
  if (NC == 1) return __ldg((const float*)a.gather + p);
  const float4 g = __ldg((const float4*)a.gather + p);
  float c, s;
  response_fast(a, t, pol, c, s);
  return fmaf(s, g.z, fmaf(c, g.y, g.x));
}

// J interleaved columns: position pos of column cl at J pos + cl, so every access
// of the column FFT puts consecutive lanes on consecutive elements.
template <int J>
struct ColJ {
  float2* buf;
  int cl;
  __device__ __forceinline__ void st(int pos, float2 v) const { buf[pos * J + cl] = v; }
  __device__ __forceinline__ float2 ld(int pos) const { return buf[pos * J + cl]; }
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

// ------------------------------------------------------------------ pass T (forward)
template <int NC, typename S, int R, bool PERIODIC>
__global__ void __launch_bounds__(ColShape<R>::THREADS, ColShape<R>::MINB) k_fast_fwd(const TodArgs a, int nd) {
  constexpr int TPC = R / kE;
  constexpr int J = ColShape<R>::J;
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float2 smf[];
  const int cl = threadIdx.x % J;
  const int i = threadIdx.x / J;
  const int c = blockIdx.x * J + cl;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  const ColJ<J> ad{smf, cl};
  // element e of the thread: column position kr = i + e TPC, complex index c + kr C,
  // samples t0 + e dt and t0 + e dt + 1
  const int t0 = 2 * (c + i * a.C);
  const int dt = 2 * TPC * a.C;
  const int dl0 = blockIdx.y * kDetsPerCta;
  for (int dd = 0; dd < kDetsPerCta; ++dd) {
    const int dl = dl0 + dd;
    if (dl >= nd) break;
    const int d = a.d0 + dl;
    const int2 off = a.det_off[d];
    const float2 pol = reinterpret_cast<const float2*>(a.pol)[d];
    // samples into the tile (the previous detector's last reads are fenced first)
    __syncthreads();
#pragma unroll kGenUnroll
    for (int e = 0; e < kE; ++e) {
      const int t = t0 + e * dt;
      ad.st(i + e * TPC, make_float2(project_fast<NC, PERIODIC>(a, off, pol, t),
                                     project_fast<NC, PERIODIC>(a, off, pol, t + 1)));
    }
    __syncthreads();
    float2 x[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) x[e] = ad.ld(i + e * TPC);
    ColPlan<R>::template run<-1>(x, i, tw + a.twl.R_off, ad);
    // four-step twiddle w_N^(c kr), kr = i + e TPC, by recurrence over e
    float2 w = tw_N(a, tw, c * i);
    const float2 step = tw_N(a, tw, c * TPC);
    S* Y = reinterpret_cast<S*>(a.spec) + (size_t)dl * a.N + c + i * a.C;
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      Store<float, S>::st(Y + e * (TPC * a.C), cmul(x[e], w));
      w = cmul(w, step);
    }
  }
}

// ------------------------------------------------------------------ pass F (filter)
template <int C, int E> struct FilterShape {
  static constexpr int TPR = C / E;
  static constexpr int THREADS = 2 * TPR > 256 ? 2 * TPR : 256;
  static constexpr int ROWS = THREADS / TPR;
  static constexpr int MINB = THREADS > 256 ? 1 : CMM_FILTER_MINB;
};

template <typename S, int E, int... RC>
__global__ void __launch_bounds__(FilterShape<RadProd<RC...>::value, E>::THREADS,
                                  FilterShape<RadProd<RC...>::value, E>::MINB)
    k_fast_filter(const TodArgs a) {
  constexpr int C = RadProd<RC...>::value;
  constexpr int TPR = C / E;
  constexpr int ROWS = FilterShape<C, E>::ROWS;
  constexpr int PAIRS = ROWS / 2;
  constexpr int PS = clog2(E);
  constexpr int ROWLEN = C + (C >> PS);
  static_assert(ROWS >= 2 && ROWS % 2 == 0, "a CTA holds whole row pairs");
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float2 smf[];
  const int rs = threadIdx.x / TPR;
  const int i = threadIdx.x % TPR;
  const int ps = rs >> 1, side = rs & 1;
  const int pr = blockIdx.x * PAIRS + ps;
  const bool pair_ok = pr <= (a.R >> 1);
  const int ra = pr;
  const int rb = (a.R - pr) & (a.R - 1);
  const bool single = ra == rb;
  const bool active = pair_ok && !(single && side);
  const int row = side ? rb : ra;
  const int dl = blockIdx.y;
  const int d = a.d0 + dl;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  S* Y = reinterpret_cast<S*>(a.spec) + (size_t)dl * a.N;
  const RowAddr<PS> ad{smf + rs * ROWLEN};
  float2 x[E];
#pragma unroll
  for (int e = 0; e < E; ++e)
    x[e] = active ? Store<float, S>::ld(Y + row * C + i + e * TPR) : make_float2(0.f, 0.f);
  rfft<-1, E, RC...>(x, i, tw + a.twl.C_off, ad);
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) ad.st(i + e * TPR, x[e]);
  __syncthreads();
  if (pair_ok) {
    const float4 cf = reinterpret_cast<const float4*>(a.coef)[d];
    const float2 wrow = __ldg(tw + a.twl.N2_off + ra);
    float2* r0 = smf + (2 * ps) * ROWLEN;
    float2* r1 = single ? r0 : r0 + ROWLEN;
    int kc0, step, npairs;
    if (!single) {
      kc0 = side * TPR + i;
      step = 2 * TPR;
      npairs = C;
    } else {
      kc0 = side ? C : i;   // only side 0 works on a single row
      step = TPR;
      npairs = ra == 0 ? C / 2 + 1 : C / 2;
    }
    for (int kc = kc0; kc < npairs; kc += step) {
      int j2;
      if (!single) j2 = C - 1 - kc;
      else if (ra == 0) j2 = (C - kc) & (C - 1);
      else j2 = C - 1 - kc;
      const int i1 = kc + (kc >> PS), i2 = j2 + (j2 >> PS);
      const int k = ra + a.R * kc;   // < N <= 2^19
      const float2 A = r0[i1];
      const float2 B = cconj(r1[i2]);
      const float2 half2{0.5f, 0.5f};
      const float2 Ev = pmul(padd(A, B), half2);
      const float2 Dv = pmul(psub(A, B), half2);
      const float2 O{Dv.y, -Dv.x};
      const float2 W = cmul(wrow, __ldg(tw + a.twl.C2_off + kc));
      const float wk = filter_weight_fast(cf, k);
      const float wm = filter_weight_fast(cf, (int)a.N - k);
      const float ws = 0.5f * (wk + wm), wd = 0.5f * (wk - wm);
      const float2 WO = cmul(W, O);
      const float2 Ep = __ffma2_rn(make_float2(ws, ws), Ev, pmul(make_float2(wd, wd), WO));
      const float2 cWE = cmulc(Ev, W);
      const float2 Op = __ffma2_rn(make_float2(wd, wd), cWE, pmul(make_float2(ws, ws), O));
      r0[i1] = make_float2(Ep.x - Op.y, Ep.y + Op.x);
      if (!(single && i2 == i1)) r1[i2] = make_float2(Ep.x + Op.y, Op.x - Ep.y);
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = ad.ld(i + e * TPR);
  rfft<1, E, RC...>(x, i, tw + a.twl.C_off, ad);
  if (active) {
    // w_N^(row c), c = i + e TPR, by recurrence over e
    float2 w = tw_N(a, tw, row * i);
    const float2 step = tw_N(a, tw, row * TPR);
    S* Yr = Y + row * C + i;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      Store<float, S>::st(Yr + e * TPR, cmulc(x[e], w));
      w = cmul(w, step);
    }
  }
}

// ------------------------------------------------------------------ pass T' (inverse + P^T)

__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(0.0f)
               : "memory");
}

// Bins the two samples of every lane of a warp.  Each group of G consecutive lanes
// holds 2G consecutive samples in lane order (lane l of a group: samples 2l, 2l + 1).
// Items with equal pixels that are adjacent in time are summed (in-lane, then across
// the lanes of a group by a segmented suffix scan); the first item of every run
// issues one reduction.  Runs in the extra pixel `skip` (samples outside the map)
// issue none: every warp would otherwise hit that one address.
template <int NC, int G>
__device__ __forceinline__ void warp_bin(float* acc32, int p0, int p1, float3 v0, float3 v1, int skip) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool group_end = (lane % G) == G - 1;
  const bool two = p1 != p0;
  if (!two) {
    v0.x += v1.x;
    v0.y += v1.y;
    v0.z += v1.z;
  }
  const int g = two ? p1 : p0;                 // pixel of the lane's last item
  const int fnext = __shfl_down_sync(full, p0, 1);
  const bool link = !group_end && g == fnext;   // next lane's first item continues my last run
  const unsigned linkmask = __ballot_sync(full, link);
  const bool linkprev = lane > 0 && ((linkmask >> (lane - 1)) & 1u);
  // y_l = A_l + (single_l && link_l ? y_{l+1} : 0), by a segmented suffix scan
  float3 y = v0;
  bool cont = !two && link;
  unsigned contmask = __ballot_sync(full, cont);
  for (int dist = 1; contmask != 0u && dist < 32; dist <<= 1) {
    const float yx = __shfl_down_sync(full, y.x, dist);
    const float yy = __shfl_down_sync(full, y.y, dist);
    const float yz = __shfl_down_sync(full, y.z, dist);
    const bool other = lane + dist < 32 && ((contmask >> (lane + dist)) & 1u);
    if (cont && lane + dist < 32) {
      y.x += yx;
      y.y += yy;
      y.z += yz;
      cont = other;
    } else {
      cont = false;
    }
    contmask = __ballot_sync(full, cont);
  }
  // carry_l = link_l ? y_{l+1} : 0
  float3 carry;
  carry.x = __shfl_down_sync(full, y.x, 1);
  carry.y = __shfl_down_sync(full, y.y, 1);
  carry.z = __shfl_down_sync(full, y.z, 1);
  if (!link) carry = make_float3(0.f, 0.f, 0.f);
  if (two) {
    if (!linkprev && p0 != skip) {
      if (NC == 1) red_add(acc32 + p0, v0.x);
      else red_add4(acc32 + 4 * p0, v0.x, v0.y, v0.z);
    }
    if (p1 != skip) {
      if (NC == 1) red_add(acc32 + p1, v1.x + carry.x);
      else red_add4(acc32 + 4 * p1, v1.x + carry.x, v1.y + carry.y, v1.z + carry.z);
    }
  } else if (!linkprev && p0 != skip) {
    if (NC == 1) red_add(acc32 + p0, y.x);
    else red_add4(acc32 + 4 * p0, y.x, y.y, y.z);
  }
}

template <int NC, typename S, int R, bool PERIODIC>
__global__ void __launch_bounds__(ColShape<R>::THREADS, ColShape<R>::MINB) k_fast_inv_bin(const TodArgs a, int nd) {
  constexpr int TPC = R / kE;
  constexpr int J = ColShape<R>::J;
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float2 smf[];
  const int cl = threadIdx.x % J;
  const int i = threadIdx.x / J;
  const int c = blockIdx.x * J + cl;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  const ColJ<J> ad{smf, cl};
  const float scale = 1.0f / (float)a.N;
  const int t0 = 2 * (c + i * a.C);
  const int dt = 2 * TPC * a.C;
  const int npix = (int)a.npix;
  const int dl0 = blockIdx.y * kDetsPerCta;
  for (int dd = 0; dd < kDetsPerCta; ++dd) {
    const int dl = dl0 + dd;
    if (dl >= nd) break;
    const int d = a.d0 + dl;
    const S* Y = reinterpret_cast<const S*>(a.spec) + (size_t)dl * a.N + c + i * a.C;
    float2 x[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) x[e] = Store<float, S>::ld(Y + e * (TPC * a.C));
    __syncthreads();   // the previous detector's binning reads of the tile are done
    ColPlan<R>::template run<1>(x, i, tw + a.twl.R_off, ad);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kE; ++e) ad.st(i + e * TPC, x[e]);
    __syncthreads();
    const int2 off = a.det_off[d];
    const float2 pol = reinterpret_cast<const float2*>(a.pol)[d];
#pragma unroll 2
    for (int e = 0; e < kE; ++e) {
      const int t = t0 + e * dt;
      const int4 b0 = __ldg(a.bore + t);
      const int4 b1 = __ldg(a.bore + t + 1);
      const int p0 = pixel_fast<PERIODIC>(b0, off, a.ny, a.nx, npix);
      const int p1 = pixel_fast<PERIODIC>(b1, off, a.ny, a.nx, npix);
      const float2 xe = ad.ld(i + e * TPC);
      const float u0 = xe.x * scale, u1 = xe.y * scale;
      float3 v0 = make_float3(u0, 0.f, 0.f), v1 = make_float3(u1, 0.f, 0.f);
      if (NC == 3) {
        float c0, s0, c1, s1;
        response_fast(a, t, pol, c0, s0);
        response_fast(a, t + 1, pol, c1, s1);
        v0.y = c0 * u0;
        v0.z = s0 * u0;
        v1.y = c1 * u1;
        v1.z = s1 * u1;
      }
      warp_bin<NC, J>(a.acc32, p0, p1, v0, v1, npix);
    }
  }
}

template <int NC>
__global__ void k_fast_flush(float* __restrict__ acc32, double* __restrict__ acc, long long npix,
                             const int* done) {
  if (done && *done) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      const float v = acc32[p];
      if (v != 0.0f) {
        acc[p] += (double)v;
        acc32[p] = 0.0f;
      }
    } else {
      const float4 v = reinterpret_cast<float4*>(acc32)[p];
      if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f) {
        double* o = acc + 4 * p;
        o[0] += (double)v.x;
        o[1] += (double)v.y;
        o[2] += (double)v.z;
        reinterpret_cast<float4*>(acc32)[p] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

// ------------------------------------------------------------------ dispatch

// Fast-path split of N = 2^logN: R = 64 below 2^16, 128 for 2^16 and 2^17, 256 for
// 2^18 and 2^19 (rows C = N / R of 64 to 2048 points).
bool fast_path_sizes(int logN, int prec, int* logR, int* logC) {
  if (prec == CMM_PREC_F64 || logN < 12 || logN > 19) return false;
  *logR = logN < 16 ? 6 : (logN < 18 ? 7 : 8);
  *logC = logN - *logR;
  return true;
}

bool fast_path_ok(const cmm_op* op) {
  int lr, lc;
  return fast_path_sizes(op->logR + op->logC, op->prec, &lr, &lc) && lr == op->logR;
}

template <int NC, typename S, int R, bool PERIODIC>
static int run_T(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  constexpr int J = ColShape<R>::J;
  constexpr int NT = ColShape<R>::THREADS;
  const int smem = (int)(sizeof(float2) * R * J);
  if (attr_only) {
    CMM_CUDA(cudaFuncSetAttribute(k_fast_fwd<NC, S, R, PERIODIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CMM_CUDA(cudaFuncSetAttribute(k_fast_inv_bin<NC, S, R, PERIODIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem));
    return CMM_OK;
  }
  const dim3 g(a.C / J, (nd + kDetsPerCta - 1) / kDetsPerCta);
  if (pass == 0) k_fast_fwd<NC, S, R, PERIODIC><<<g, NT, smem, st>>>(a, nd);
  else k_fast_inv_bin<NC, S, R, PERIODIC><<<g, NT, smem, st>>>(a, nd);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <int NC, typename S, bool PERIODIC>
static int dispatch_T_p(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  if (a.logR == 6) return run_T<NC, S, 64, PERIODIC>(a, nd, pass, st, attr_only);
  if (a.logR == 7) return run_T<NC, S, 128, PERIODIC>(a, nd, pass, st, attr_only);
  return run_T<NC, S, 256, PERIODIC>(a, nd, pass, st, attr_only);
}

template <int NC, typename S>
static int dispatch_T(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  return a.periodic ? dispatch_T_p<NC, S, true>(a, nd, pass, st, attr_only)
                    : dispatch_T_p<NC, S, false>(a, nd, pass, st, attr_only);
}

template <typename S, int E, int... RC>
static int run_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  constexpr int C = RadProd<RC...>::value;
  constexpr int ROWS = FilterShape<C, E>::ROWS;
  constexpr int PAIRS = ROWS / 2;
  constexpr int PS = clog2(E);
  const size_t smem = sizeof(float2) * ROWS * (C + (C >> PS));
  if (attr_only) {
    CMM_CUDA(cudaFuncSetAttribute(k_fast_filter<S, E, RC...>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return CMM_OK;
  }
  const int npairs = a.R / 2 + 1;
  const dim3 g((npairs + PAIRS - 1) / PAIRS, nd);
  k_fast_filter<S, E, RC...><<<g, FilterShape<C, E>::THREADS, smem, st>>>(a);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <typename S>
static int dispatch_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  switch (a.logC) {
    case 6: return run_F<S, 16, 16, 4>(a, nd, st, attr_only);
    case 7: return run_F<S, 16, 16, 8>(a, nd, st, attr_only);
    case 8: return run_F<S, 16, 16, 16>(a, nd, st, attr_only);
    case 9: return run_F<S, 16, 16, 16, 2>(a, nd, st, attr_only);
    case 10: return run_F<S, 16, 16, 16, 4>(a, nd, st, attr_only);
    case 11: return run_F<S, 16, 16, 16, 8>(a, nd, st, attr_only);
    default: return run_F<S, 16, 16, 16, 16>(a, nd, st, attr_only);
  }
}

static int flush(const TodArgs& a, int nc, cudaStream_t st) {
  // npix + 1 entries: the extra pixel is cleared too, so its FP32 sum stays bounded
  const int blocks = (int)std::min<long long>((a.npix + 256) / 256, 4096);
  if (nc == 1) k_fast_flush<1><<<blocks, 256, 0, st>>>(a.acc32, a.acc, a.npix + 1, a.done);
  else k_fast_flush<3><<<blocks, 256, 0, st>>>(a.acc32, a.acc, a.npix + 1, a.done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

// Forward pass from a stored TOD (right-hand side) uses the generic kernel of
// tod.cu; the spectrum layout is the same.
int launch_generic_fwd_from_tod(cmm_op* op, int d0, int nd, const void* tod, int tod_is_f64);

template <typename S>
static int apply_fast_s(cmm_op* op, int d0, int nd, const void* tod, int tod_is_f64, int pass) {
  TodArgs a = make_args(op, d0);
  cudaStream_t st = op->ctx->stream;
  const int nc = op->pt->ncomp;
  if (pass < 0 || pass == 0) {
    if (tod) CMM_TRY(launch_generic_fwd_from_tod(op, d0, nd, tod, tod_is_f64));
    else if (nc == 1) CMM_TRY((dispatch_T<1, S>(a, nd, 0, st, false)));
    else CMM_TRY((dispatch_T<3, S>(a, nd, 0, st, false)));
  }
  if (pass < 0 || pass == 1) CMM_TRY(dispatch_F<S>(a, nd, st, false));
  if (pass < 0 || pass == 2) {
    for (int g0 = 0; g0 < nd; g0 += kFlushDets) {
      TodArgs b = a;
      const int gn = std::min(kFlushDets, nd - g0);
      b.d0 = a.d0 + g0;
      b.spec = reinterpret_cast<S*>(a.spec) + (long long)g0 * a.N;
      if (nc == 1) CMM_TRY((dispatch_T<1, S>(b, gn, 2, st, false)));
      else CMM_TRY((dispatch_T<3, S>(b, gn, 2, st, false)));
      CMM_TRY(flush(b, nc, st));
    }
  }
  return CMM_OK;
}

int launch_apply_chunk_fast(cmm_op* op, int d0, int nd, const void* tod, int tod_is_f64, int pass) {
  if (op->prec == CMM_PREC_BF16) return apply_fast_s<__nv_bfloat162>(op, d0, nd, tod, tod_is_f64, pass);
  return apply_fast_s<float2>(op, d0, nd, tod, tod_is_f64, pass);
}

template <typename S>
static int prepare_fast_s(cmm_op* op) {
  TodArgs a = make_args(op, 0);
  if (op->pt->ncomp == 1) CMM_TRY((dispatch_T<1, S>(a, 0, 0, nullptr, true)));
  else CMM_TRY((dispatch_T<3, S>(a, 0, 0, nullptr, true)));
  return dispatch_F<S>(a, 0, nullptr, true);
}

int prepare_fast(cmm_op* op) {
  return op->prec == CMM_PREC_BF16 ? prepare_fast_s<__nv_bfloat162>(op) : prepare_fast_s<float2>(op);
}

}  // namespace cmm
