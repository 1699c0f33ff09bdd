// Fast path of A = P^T N^-1 P for FP32 compute (FP32 or BF16 spectrum storage):
// the same four-step decomposition as tod.cu, with register-resident FFTs.
//
//   k_fast_fwd:     pass T, R-point column FFTs (E = 8 elements per thread, J = 8
//                   columns per CTA) of samples produced by P on the fly; each CTA
//                   loops over a block of detectors and keeps the four-step
//                   twiddles w_N^{c k_r} in registers.
//   k_fast_filter:  pass F, C-point row FFTs (E = 16 or 32), the real-FFT split with
//                   the noise filter w_d(f) evaluated with the SFU, inverse row FFTs.
//   k_fast_inv_bin: pass T', inverse column FFTs, a transpose through shared memory
//                   so that each thread owns 16 consecutive samples, and P^T with
//                   runs of equal pixels summed in FP32 before one FP64 atomic per
//                   Stokes component (partials over at most 16 samples).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "fft_reg.cuh"
#include "tod_common.cuh"

namespace cmm {

constexpr int kDetsPerCta = 2;

// GB300's FP64 unit also executes int <-> float and float <-> double conversions,
// at a small fraction of the FP32 rate; the helpers below do them exactly on the
// integer and FP32 pipes instead.

// Exact float of an integer 0 <= k < 2^23 (IEEE-754 single: 2^23 + k has k as its
// mantissa).
__device__ __forceinline__ float small_int_to_float(int k) {
  return __int_as_float(0x4B000000 | k) - 8388608.0f;
}

// Exact double of a float, by re-biasing the exponent (bias 127 -> 1023) and
// widening the mantissa (23 -> 52 bits); zeros and subnormals give +-0.
__device__ __forceinline__ double float_to_double_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned sign = u & 0x80000000u;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  const unsigned ed = (e == 0xffu) ? 0x7ffu : e + 896u;
  const unsigned hi = sign | (ed << 20) | ((u & 0x7fffffu) >> 3);
  const unsigned lo = u << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// exp2 / log2 on the special function unit; relative error of w below 1e-6.
__device__ __forceinline__ float filter_weight_fast(const float4 cf, int k) {
  if (cf.w != 0.0f) return cf.x;
  const float kk = small_int_to_float(k == 0 ? 1 : k);
  const float e = exp2f(fmaf(-cf.y, __log2f(kk), cf.z));
  return __fdividef(cf.x, 1.0f + e);
}

// (cos 2a, sin 2a) of sample t, a = psi_d + phi_t, from the FP32 (cos 2phi, sin 2phi)
__device__ __forceinline__ void response_fast(const TodArgs& a, long long t, const float2 pol, float& c, float& s) {
  const float2 r2 = __ldg(a.rot2 + t);
  c = pol.x * r2.x - pol.y * r2.y;
  s = pol.y * r2.x + pol.x * r2.y;
}

__device__ __forceinline__ float2 tw_N(const TodArgs& a, const float2* __restrict__ tw, long long e) {
  const float2 lo = __ldg(tw + a.twl.Nlo_off + (e & (a.C - 1)));
  const float2 hi = __ldg(tw + a.twl.R_off + (e >> a.logC));
  return cmul(lo, hi);
}

template <int NC>
__device__ __forceinline__ float project_fast(const TodArgs& a, const int2 off, const float2 pol, long long t) {
  const int4 b = __ldg(a.bore + t);
  const int p = sample_pixel(b, off, a.ny, a.nx, a.periodic);
  if (p < 0) return 0.0f;
  if (NC == 1) return __ldg((const float*)a.gather + p);
  const float4 g = __ldg((const float4*)a.gather + p);
  float c, s;
  response_fast(a, t, pol, c, s);
  return g.x + c * g.y + s * g.z;
}

// ------------------------------------------------------------------ pass T (forward)
template <int NC, typename S, int... RR>
__global__ void __launch_bounds__(RadProd<RR...>::value, 1024 / RadProd<RR...>::value)
    k_fast_fwd(const TodArgs a, int nd) {
  constexpr int R = RadProd<RR...>::value;
  constexpr int E = 8;
  constexpr int TPC = R / E;
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float2 smf[];
  const int cl = threadIdx.x & 7;
  const int i = threadIdx.x >> 3;
  const int c = (blockIdx.x << 3) + cl;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  const ColAddr ad{smf, cl};
  const int dl0 = blockIdx.y * kDetsPerCta;
  for (int dd = 0; dd < kDetsPerCta; ++dd) {
    const int dl = dl0 + dd;
    if (dl >= nd) break;
    const int d = a.d0 + dl;
    const int2 off = a.det_off[d];
    const float2 pol = reinterpret_cast<const float2*>(a.pol)[d];
    float2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long j = (long long)c + ((long long)(i + e * TPC) << a.logC);
      x[e].x = project_fast<NC>(a, off, pol, 2 * j);
      x[e].y = project_fast<NC>(a, off, pol, 2 * j + 1);
    }
    rfft<-1, E, RR...>(x, i, tw + a.twl.R_off, ad);
    S* Y = reinterpret_cast<S*>(a.spec) + (long long)dl * a.N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int kr = i + e * TPC;
      Store<float, S>::st(Y + ((long long)kr << a.logC) + c, cmul(x[e], tw_N(a, tw, (long long)c * kr)));
    }
  }
}

// ------------------------------------------------------------------ pass F (filter)
template <typename S, int E, int... RC>
__global__ void __launch_bounds__(256, 2) k_fast_filter(const TodArgs a) {
  constexpr int C = RadProd<RC...>::value;
  constexpr int TPR = C / E;
  constexpr int ROWS = 256 / TPR;
  constexpr int PAIRS = ROWS / 2;
  constexpr int PS = clog2(E) <= 4 ? 4 : 5;
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
  S* Y = reinterpret_cast<S*>(a.spec) + (long long)dl * a.N;
  const RowAddr<PS> ad{smf + rs * ROWLEN};
  float2 x[E];
#pragma unroll
  for (int e = 0; e < E; ++e)
    x[e] = active ? Store<float, S>::ld(Y + (long long)row * C + i + e * TPR) : make_float2(0.f, 0.f);
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
      const int k = ra + a.R * kc;   // < N <= 2^20
      const float2 A = r0[i1];
      const float2 B = cconj(r1[i2]);
      const float2 Ev{(A.x + B.x) * 0.5f, (A.y + B.y) * 0.5f};
      const float2 Dv{(A.x - B.x) * 0.5f, (A.y - B.y) * 0.5f};
      const float2 O{Dv.y, -Dv.x};
      const float2 W = cmul(wrow, __ldg(tw + a.twl.C2_off + kc));
      const float wk = filter_weight_fast(cf, k);
      const float wm = filter_weight_fast(cf, (int)a.N - k);
      const float ws = 0.5f * (wk + wm), wd = 0.5f * (wk - wm);
      const float2 WO = cmul(W, O);
      const float2 Ep{ws * Ev.x + wd * WO.x, ws * Ev.y + wd * WO.y};
      const float2 cWE = cmulc(Ev, W);
      const float2 Op{wd * cWE.x + ws * O.x, wd * cWE.y + ws * O.y};
      r0[i1] = make_float2(Ep.x - Op.y, Ep.y + Op.x);
      if (!(single && i2 == i1)) r1[i2] = make_float2(Ep.x + Op.y, Op.x - Ep.y);
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = ad.ld(i + e * TPR);
  rfft<1, E, RC...>(x, i, tw + a.twl.C_off, ad);
  if (active) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = i + e * TPR;
      const float2 w = tw_N(a, tw, (long long)c * row);
      Store<float, S>::st(Y + (long long)row * C + c, cmulc(x[e], w));
    }
  }
}

// ------------------------------------------------------------------ pass T' (inverse + P^T)
template <int NC>
__device__ __forceinline__ void flush_bin(double* acc, int p, float aT, float aQ, float aU) {
  if (p < 0) return;
  if (NC == 1) {
    atomicAdd(acc + p, float_to_double_exact(aT));
    return;
  }
  double* dst = acc + 4 * (long long)p;
  atomicAdd(dst + 0, float_to_double_exact(aT));
  atomicAdd(dst + 1, float_to_double_exact(aQ));
  atomicAdd(dst + 2, float_to_double_exact(aU));
}

template <int NC, typename S, int... RR>
__global__ void __launch_bounds__(RadProd<RR...>::value, 1024 / RadProd<RR...>::value)
    k_fast_inv_bin(const TodArgs a, int nd) {
  constexpr int R = RadProd<RR...>::value;
  constexpr int E = 8;
  constexpr int TPC = R / E;
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float2 smf[];
  const int cl = threadIdx.x & 7;
  const int i = threadIdx.x >> 3;
  const int c0 = blockIdx.x << 3;
  const int c = c0 + cl;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  const ColAddr ad{smf, cl};
  const float scale = 1.0f / (float)a.N;
  const int dl0 = blockIdx.y * kDetsPerCta;
  for (int dd = 0; dd < kDetsPerCta; ++dd) {
    const int dl = dl0 + dd;
    if (dl >= nd) break;
    const int d = a.d0 + dl;
    const S* Y = reinterpret_cast<const S*>(a.spec) + (long long)dl * a.N;
    float2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = Store<float, S>::ld(Y + ((long long)(i + e * TPC) << a.logC) + c);
    rfft<1, E, RR...>(x, i, tw + a.twl.R_off, ad);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) ad.st(i + e * TPC, make_float2(x[e].x * scale, x[e].y * scale));
    __syncthreads();
    // thread r owns time row r: samples 2 (c0 + C r) .. + 15
    const int r = threadIdx.x;
    const int2 off = a.det_off[d];
    const float2 pol = reinterpret_cast<const float2*>(a.pol)[d];
    const long long t0 = 2 * ((long long)c0 + ((long long)r << a.logC));
    const int rbase = (r + (r >> 3)) << 3;
    int cur = -1;
    float aT = 0.f, aQ = 0.f, aU = 0.f;
#pragma unroll
    for (int cq = 0; cq < 8; ++cq) {
      const float2 v = smf[rbase + (cq ^ (r & 7))];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long t = t0 + 2 * cq + h;
        const float u = h ? v.y : v.x;
        const int4 b = __ldg(a.bore + t);
        const int p = sample_pixel(b, off, a.ny, a.nx, a.periodic);
        if (p != cur) {
          flush_bin<NC>(a.acc, cur, aT, aQ, aU);
          cur = p;
          aT = aQ = aU = 0.f;
        }
        if (p >= 0) {
          aT += u;
          if (NC == 3) {
            float cc, ss;
            response_fast(a, t, pol, cc, ss);
            aQ += cc * u;
            aU += ss * u;
          }
        }
      }
    }
    flush_bin<NC>(a.acc, cur, aT, aQ, aU);
  }
}

// ------------------------------------------------------------------ dispatch
bool fast_path_ok(const cmm_op* op) {
  if (op->prec == CMM_PREC_F64) return false;
  return op->logR >= 6 && op->logR <= 9 && op->logC >= 6 && op->logC <= 10;
}

template <int NC, typename S, int... RR>
static int run_T(const TodArgs& a, int nd, int pass, cudaStream_t st) {
  constexpr int R = RadProd<RR...>::value;
  const size_t smem = sizeof(float2) * col_tile_elems(R);
  const dim3 g(a.C / 8, (nd + kDetsPerCta - 1) / kDetsPerCta);
  if (pass == 0) k_fast_fwd<NC, S, RR...><<<g, R, smem, st>>>(a, nd);
  else k_fast_inv_bin<NC, S, RR...><<<g, R, smem, st>>>(a, nd);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <int NC, typename S, int... RR>
static int attr_T() {
  constexpr int R = RadProd<RR...>::value;
  const int smem = (int)(sizeof(float2) * col_tile_elems(R));
  CMM_CUDA(cudaFuncSetAttribute(k_fast_fwd<NC, S, RR...>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CMM_CUDA(cudaFuncSetAttribute(k_fast_inv_bin<NC, S, RR...>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return CMM_OK;
}

template <int NC, typename S>
static int dispatch_T(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  switch (a.logR) {
    case 6: return attr_only ? attr_T<NC, S, 8, 8>() : run_T<NC, S, 8, 8>(a, nd, pass, st);
    case 7: return attr_only ? attr_T<NC, S, 2, 8, 8>() : run_T<NC, S, 2, 8, 8>(a, nd, pass, st);
    case 8: return attr_only ? attr_T<NC, S, 4, 8, 8>() : run_T<NC, S, 4, 8, 8>(a, nd, pass, st);
    default: return attr_only ? attr_T<NC, S, 8, 8, 8>() : run_T<NC, S, 8, 8, 8>(a, nd, pass, st);
  }
}

template <typename S, int E, int... RC>
static size_t smem_F() {
  constexpr int C = RadProd<RC...>::value;
  constexpr int TPR = C / E;
  constexpr int ROWS = 256 / TPR;
  constexpr int PS = clog2(E) <= 4 ? 4 : 5;
  return sizeof(float2) * ROWS * (C + (C >> PS));
}

template <typename S, int E, int... RC>
static int run_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  constexpr int C = RadProd<RC...>::value;
  constexpr int PAIRS = (256 / (C / E)) / 2;
  const size_t smem = smem_F<S, E, RC...>();
  if (attr_only) {
    CMM_CUDA(cudaFuncSetAttribute(k_fast_filter<S, E, RC...>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return CMM_OK;
  }
  const int npairs = a.R / 2 + 1;
  const dim3 g((npairs + PAIRS - 1) / PAIRS, nd);
  k_fast_filter<S, E, RC...><<<g, 256, smem, st>>>(a);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <typename S>
static int dispatch_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  switch (a.logC) {
    case 6: return run_F<S, 16, 4, 16>(a, nd, st, attr_only);
    case 7: return run_F<S, 16, 8, 16>(a, nd, st, attr_only);
    case 8: return run_F<S, 16, 16, 16>(a, nd, st, attr_only);
    case 9: return run_F<S, 16, 2, 16, 16>(a, nd, st, attr_only);
    default: return run_F<S, 16, 4, 16, 16>(a, nd, st, attr_only);
  }
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
    if (nc == 1) CMM_TRY((dispatch_T<1, S>(a, nd, 2, st, false)));
    else CMM_TRY((dispatch_T<3, S>(a, nd, 2, st, false)));
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
