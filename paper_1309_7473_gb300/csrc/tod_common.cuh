// Device helpers shared by the time-ordered-data kernels: pointing, response,
// noise-filter weights, spectrum storage and the kernel argument block.
#pragma once

#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace cmm {

// ------------------------------------------------------------------ pointing

// Nearest pixel of sample (bore b, detector offset o), exact 32-bit fixed point:
// the rotated offset (units 2^-22 px, |.| < 2^30) is floored to 2^-16 px and added
// to the boresight (units 2^-16 px); the pixel is floor((x + 2^15) / 2^16).
__device__ __forceinline__ int sample_pixel(const int4 b, const int2 o, int ny, int nx, int periodic) {
  const int ox = b.z * o.x - b.w * o.y;
  const int oy = b.w * o.x + b.z * o.y;
  const int x = b.x + (ox >> 6);
  const int y = b.y + (oy >> 6);
  int ix = (x + (1 << 15)) >> 16;
  int iy = (y + (1 << 15)) >> 16;
  if (periodic) {
    ix %= nx;
    if (ix < 0) ix += nx;
    iy %= ny;
    if (iy < 0) iy += ny;
  } else if ((unsigned)ix >= (unsigned)nx || (unsigned)iy >= (unsigned)ny) {
    return -1;
  }
  return iy * nx + ix;
}

// Response (cos 2a, sin 2a), a = psi_d + phi_t, by angle addition; phi_t is the angle
// of the fixed-point rotation pair (c, s), whose double angle is (c^2 - s^2, 2 c s)
// over c^2 + s^2 (the pair's length differs from one by its rounding).
template <typename T>
__device__ __forceinline__ void sample_response(const int4 b, const V2<T> pol, T& c, T& s) {
  const T cf = (T)b.z, sf = (T)b.w;
  const T r2 = cf * cf + sf * sf;
  const T c2 = (cf * cf - sf * sf) / r2;
  const T s2 = (T)2 * cf * sf / r2;
  c = pol.x * c2 - pol.y * s2;
  s = pol.y * c2 + pol.x * s2;
}

// ------------------------------------------------------------------ noise filter
// w_d(k) = 1/sigma^2 / (1 + (k f_s / (n_t f_knee))^-alpha); k = 0 uses k = 1.
template <typename T>
__device__ __forceinline__ T filter_weight(const V4<T> cf, long long k) {
  if (cf.w != (T)0) return cf.x;
  const T kk = (T)(k == 0 ? 1 : k);
  const T e = exp2(fma(-cf.y, log2(kk), cf.z));
  return cf.x / ((T)1 + e);
}

// w_d(f_k) from the detector's table when the noise has one, else the law
template <typename T>
__device__ __forceinline__ T noise_weight(const void* wtab, long long N, int d, const V4<T> cf, long long k) {
  if (wtab) return reinterpret_cast<const T*>(wtab)[(long long)d * (N + 1) + k];
  return filter_weight<T>(cf, k);
}

// ------------------------------------------------------------------ spectrum storage
template <typename T, typename S> struct Store;
template <typename T> struct Store<T, V2<T>> {
  static __device__ __forceinline__ V2<T> ld(const V2<T>* p) { return *p; }
  static __device__ __forceinline__ void st(V2<T>* p, V2<T> v) { *p = v; }
};
template <> struct Store<float, __nv_bfloat162> {
  static __device__ __forceinline__ float2 ld(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }
};

struct TodArgs {
  const int4* bore;
  const int2* det_off;
  const float2* rot2;   // [n_t] (cos 2phi, sin 2phi) in FP32
  const void* pol;      // V2<T> [n_det]
  const void* coef;     // V4<T> [n_det]
  const void* wtab;     // T [n_det][N + 1] tabulated w_d(f_k), or nullptr (the parametric law)
  int ny, nx, periodic;
  long long n_t, N;
  int R, C, logR, logC, J, logJ;
  const void* tw;       // V2<T> twiddle tables
  TwLayout twl;
  void* spec;           // S [nd][N]
  const void* gather;   // V4<T> / T [npix]
  double* acc;          // [npix][acc_stride]
  float* acc32;         // [npix][acc_stride] FP32 partials (fast path)
  long long acc32_map;  // elements of one partial map in acc32 (pair path: one map per flush group)
  int flush_dets;       // detectors per partial map (the pair path's binning picks map (d - d0) / flush_dets)
  long long npix;
  const void* tod;      // float / double [n_det][n_t]
  const int* pix;       // cached pixel indices [n_det][n_t] or nullptr
  int corr_r;           // correlated noise modes (0: independent detectors)
  const float* corrV;   // [n_det][corr_r]
  const float* corr_minv;   // [N + 1][r][r] slot order
  float2* corr_s;       // [N][r]
  int d0;
  const int* done;
};

template <typename T, int NC>
__device__ __forceinline__ T project_sample(const TodArgs& a, const int2 off, const V2<T> pol, long long t) {
  const int4 b = __ldg(a.bore + t);
  const int p = sample_pixel(b, off, a.ny, a.nx, a.periodic);
  if (p < 0) return (T)0;
  if (NC == 1) return ((const T*)a.gather)[p];
  const V4<T> g = ((const V4<T>*)a.gather)[p];
  T c, s;
  sample_response<T>(b, pol, c, s);
  return g.x + c * g.y + s * g.z;
}

template <typename T, int NC>
__device__ __forceinline__ void bin_sample(const TodArgs& a, const int2 off, const V2<T> pol,
                                           long long t, T u) {
  const int4 b = __ldg(a.bore + t);
  const int p = sample_pixel(b, off, a.ny, a.nx, a.periodic);
  if (p < 0) return;
  if (NC == 1) {
    atomicAdd(a.acc + p, (double)u);
    return;
  }
  T c, s;
  sample_response<T>(b, pol, c, s);
  double* dst = a.acc + 4 * (long long)p;
  atomicAdd(dst + 0, (double)u);
  atomicAdd(dst + 1, (double)(c * u));
  atomicAdd(dst + 2, (double)(s * u));
}

// w_N^e for 0 <= e < N = R C: w_N^(e mod C) * w_R^(e div C)
template <typename T>
__device__ __forceinline__ V2<T> twiddle_N(const TodArgs& a, const V2<T>* tw, long long e) {
  const V2<T> lo = tw[a.twl.Nlo_off + (e & (a.C - 1))];
  const V2<T> hi = tw[a.twl.R_off + (e >> a.logC)];
  return cmul(lo, hi);
}


static inline int ilog2_ll(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

// Columns per CTA of the generic (shared-memory ping-pong) kernels.
static inline int tod_J(const cmm_op* op) {
  const int elems = (op->prec == CMM_PREC_F64) ? 2048 : 4096;
  int J = std::max(1, elems / op->R);
  J = std::min(J, 16);
  J = std::min(J, op->C);
  return J;
}

static inline TodArgs make_args(const cmm_op* op, int d0) {
  const cmm_pointing* pt = op->pt;
  TodArgs a;
  a.bore = pt->bore;
  a.det_off = pt->det_off;
  a.rot2 = pt->rot2;
  const bool f64 = op->prec == CMM_PREC_F64;
  a.pol = f64 ? (const void*)pt->det_pol64 : (const void*)pt->det_pol32;
  a.coef = f64 ? (const void*)op->nz->coef64 : (const void*)op->nz->coef32;
  a.wtab = f64 ? (const void*)op->nz->wtab64 : (const void*)op->nz->wtab32;
  a.ny = pt->ny;
  a.nx = pt->nx;
  a.periodic = pt->periodic;
  a.n_t = pt->n_t;
  a.N = op->N;
  a.R = op->R;
  a.C = op->C;
  a.logR = op->logR;
  a.logC = op->logC;
  a.J = tod_J(op);
  a.logJ = ilog2_ll(a.J);
  a.tw = op->tw;
  a.twl = tw_layout(op->R, op->C);
  a.spec = op->spec;
  a.gather = op->gather;
  a.acc = op->acc;
  a.acc32 = op->acc32;
  a.acc32_map = 0;
  a.flush_dets = 1 << 30;
  a.npix = pt->npix;
  a.tod = nullptr;
  a.pix = op->pix;
  const bool corr = op->nz->corr_r > 0 && op->corr_minv && op->corr_version == op->nz->corr_version;
  a.corr_r = corr ? op->nz->corr_r : 0;
  a.corrV = op->nz->corr_V;
  a.corr_minv = op->corr_minv;
  a.corr_s = op->corr_s;
  a.d0 = d0;
  a.done = op->done;
  return a;
}

// Fast-path kernels (register-resident FFTs) for FP32 compute; tod_fast.cu.
bool fast_path_ok(const cmm_op* op);
int launch_apply_chunk_fast(cmm_op* op, int d0, int nd, const void* tod, int tod_is_f64, int pass);
int prepare_fast(cmm_op* op);

}  // namespace cmm
