// Fast path of A = P^T N^-1 P for FP32 compute (FP32 or BF16 spectrum storage).
//
// The complex length N = n_t / 2 is split as N = R C with short columns
// (R = 64, 128 or 256) and long rows (C = N / R, 64 to 2048 points):
//
//   k_fast_fwd:     pass T.  A CTA holds J = 32 (R <= 128) or 16 (R = 256) adjacent
//                   columns; thread (cl, i) owns the 16 rows i + e R/16 of column
//                   c0 + cl, so each group of J lanes reads 2J consecutive samples
//                   at a time (coalesced pixel-cache, boresight and rotation loads).
//                   P m is produced into a shared tile, transformed by a
//                   register-resident R-point FFT and stored times w_N^{c k_r}.
//   k_fast_filter:  pass F.  Row pairs (k_r, R - k_r) of C points: forward FFT, the
//                   real-FFT split, the noise filter w_d(f), the merge, inverse FFT.
//   k_fast_inv_bin: pass T'.  Inverse R-point FFTs into a padded shared tile; each
//                   lane then takes 8 consecutive filtered samples, sums runs of
//                   samples in the same pixel in registers and issues one vector FP32
//                   reduction per run into an L2-resident partial map.
//   k_fast_flush:   adds the FP32 partial map into the FP64 accumulator and clears
//                   it, after every group of at most kFlushDets detectors, so each
//                   FP32 partial sums a bounded number of samples (operators with
//                   more samples on a pixel than that allows bin with the generic
//                   kernel instead, see kF32HitLimit).
//   k_fast_flush_maps: the same for the two-detector path, whose binning launch
//                   fills up to kMaxPartialMaps partial maps (one per group of
//                   kFlushDets detectors): sums them in FP64 into the accumulator
//                   and clears them.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "fft_reg.cuh"
#include "tod_common.cuh"
#include "tod_fast.cuh"

namespace cmm {

// w_d(f_k): the detector's tabulated weight when the noise has a table, else the law
__device__ __forceinline__ float filter_weight_fast(const TodArgs& a, int d, const float4 cf, int k) {
  if (a.wtab) return __ldg(reinterpret_cast<const float*>(a.wtab) + (size_t)d * (a.N + 1) + k);
  return filter_weight_law(cf, k);
}

// (cos 2a, sin 2a) of sample t, a = psi_d + phi_t, from the FP32 (cos 2phi, sin 2phi)
__device__ __forceinline__ void response_fast(const TodArgs& a, int t, const float2 pol, float& c,
                                              float& s) {
  const float2 r2 = __ldg(a.rot2 + t);
  c = pol.x * r2.x - pol.y * r2.y;
  s = pol.y * r2.x + pol.x * r2.y;
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

// ------------------------------------------------------------------ pass T (forward)
// The samples t (even) and t + 1 with known pixels (cached pointing): one 16-byte
// load of their two (cos 2phi, sin 2phi).
template <int NC>
__device__ __forceinline__ float2 gather_pair(const TodArgs& a, const int2 p, const float2 pol, int t) {
  if (NC == 1) return make_float2(__ldg((const float*)a.gather + p.x), __ldg((const float*)a.gather + p.y));
  const float4 g0 = __ldg((const float4*)a.gather + p.x);
  const float4 g1 = __ldg((const float4*)a.gather + p.y);
  const float4 r = __ldg(reinterpret_cast<const float4*>(a.rot2 + t));
  const float c0 = pol.x * r.x - pol.y * r.y, s0 = pol.y * r.x + pol.x * r.y;
  const float c1 = pol.x * r.z - pol.y * r.w, s1 = pol.y * r.z + pol.x * r.w;
  return make_float2(fmaf(s0, g0.z, fmaf(c0, g0.y, g0.x)), fmaf(s1, g1.z, fmaf(c1, g1.y, g1.x)));
}

template <int NC, typename S, int R, bool PERIODIC, bool CACHED>
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
    if constexpr (CACHED) {
      // all pixel pairs first (independent loads), then the gathers
      const int2* pp = reinterpret_cast<const int2*>(a.pix + (size_t)d * a.n_t + t0);
      int2 pq[kE];
#pragma unroll
      for (int e = 0; e < kE; ++e) pq[e] = __ldcs(pp + e * (dt / 2));
#pragma unroll
      for (int e = 0; e < kE; ++e) ad.st(i + e * TPC, gather_pair<NC>(a, pq[e], pol, t0 + e * dt));
    } else {
#pragma unroll kGenUnroll
      for (int e = 0; e < kE; ++e) {
        const int t = t0 + e * dt;
        ad.st(i + e * TPC, make_float2(project_fast<NC, PERIODIC>(a, off, pol, t),
                                       project_fast<NC, PERIODIC>(a, off, pol, t + 1)));
      }
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

// Filter-pass modes: kFilterFull applies the per-detector filter (row FFT, split,
// w_d(f), merge, inverse row FFT).  With noise correlated between detectors the pass
// is cut in two around a cross-detector step: kFilterSplit ends after the split and
// stores the real-FFT spectrum X_d(k) in the slot of bin k (row k mod R, column
// k div R; slot 0 holds the two real bins 0 and N as (X(0), X(N))); kFilterMerge
// starts from those slots, applies y = w_d (X - sum_j V_dj s_j) with the
// correlation solution s of k_fast_corr, merges and inverts.
constexpr int kFilterFull = 0, kFilterSplit = 1, kFilterMerge = 2;

// sum_j V_dj s_j(slot) for one detector (complex)
__device__ __forceinline__ float2 corr_mode_sum(const TodArgs& a, const float* vd, int slot) {
  float2 acc = make_float2(0.f, 0.f);
  for (int j = 0; j < a.corr_r; ++j) {
    const float2 sj = a.corr_s[(size_t)slot * a.corr_r + j];
    acc.x = fmaf(vd[j], sj.x, acc.x);
    acc.y = fmaf(vd[j], sj.y, acc.y);
  }
  return acc;
}

template <typename S, int MODE, int E, int... RC>
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
  const int bi = ad.base(i);
  if constexpr (MODE != kFilterMerge) {
#pragma unroll
    for (int e = 0; e < E; ++e)
      x[e] = active ? Store<float, S>::ld(Y + row * C + i + e * TPR) : make_float2(0.f, 0.f);
    rfft<-1, E, RC...>(x, i, tw + a.twl.C_off, ad);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) ad.st_at(bi, e * TPR, x[e]);
  } else {
    // the split spectrum of the row, straight into the padded row buffer
#pragma unroll
    for (int e = 0; e < E; ++e)
      ad.st_at(bi, e * TPR, active ? Store<float, S>::ld(Y + row * C + i + e * TPR) : make_float2(0.f, 0.f));
  }
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
    float vd[kMaxCorrModes];
    if constexpr (MODE == kFilterMerge)
      for (int j = 0; j < a.corr_r; ++j) vd[j] = a.corrV[d * a.corr_r + j];
    for (int kc = kc0; kc < npairs; kc += step) {
      int j2;
      if (!single) j2 = C - 1 - kc;
      else if (ra == 0) j2 = (C - kc) & (C - 1);
      else j2 = C - 1 - kc;
      const int i1 = kc + (kc >> PS), i2 = j2 + (j2 >> PS);
      const int k = ra + a.R * kc;   // < N <= 2^19
      const float2 W = cmul(wrow, __ldg(tw + a.twl.C2_off + kc));
      const float2 half2{0.5f, 0.5f};
      if constexpr (MODE == kFilterFull) {
        const float2 A = r0[i1];
        const float2 B = cconj(r1[i2]);
        const float2 Ev = pmul(padd(A, B), half2);
        const float2 Dv = pmul(psub(A, B), half2);
        const float2 O{Dv.y, -Dv.x};
        const float wk = filter_weight_fast(a, d, cf, k);
        const float wm = filter_weight_fast(a, d, cf, (int)a.N - k);
        const float ws = 0.5f * (wk + wm), wd = 0.5f * (wk - wm);
        const float2 WO = cmul(W, O);
        const float2 Ep = __ffma2_rn(make_float2(ws, ws), Ev, pmul(make_float2(wd, wd), WO));
        const float2 cWE = cmulc(Ev, W);
        const float2 Op = __ffma2_rn(make_float2(wd, wd), cWE, pmul(make_float2(ws, ws), O));
        r0[i1] = make_float2(Ep.x - Op.y, Ep.y + Op.x);
        if (!(single && i2 == i1)) r1[i2] = make_float2(Ep.x + Op.y, Op.x - Ep.y);
      } else if constexpr (MODE == kFilterSplit) {
        // X(k) = Ev + W O and X(N - k) = conj(Ev - W O) into their bins' slots
        const float2 A = r0[i1];
        const float2 B = cconj(r1[i2]);
        const float2 Ev = pmul(padd(A, B), half2);
        const float2 Dv = pmul(psub(A, B), half2);
        const float2 O{Dv.y, -Dv.x};
        const float2 WO = cmul(W, O);
        const float2 Xk = padd(Ev, WO);
        const float2 Xm = cconj(psub(Ev, WO));
        if (ra == 0 && kc == 0) {
          Store<float, S>::st(Y, make_float2(Xk.x, Xm.x));   // the real bins 0 and N
        } else {
          Store<float, S>::st(Y + ra * C + kc, Xk);
          if (!(single && i2 == i1)) Store<float, S>::st(Y + rb * C + j2, Xm);
        }
      } else {
        // y = w (X - V s) at bins k and N - k, merged back into the packed spectrum
        const int sa = ra * C + kc, sb = rb * C + j2;
        const float2 X1 = r0[i1], X2 = r1[i2];
        const float2 S1 = corr_mode_sum(a, vd, sa);
        float2 Yk, Ym;
        if (ra == 0 && kc == 0) {
          Yk = make_float2(filter_weight_fast(a, d, cf, 0) * (X1.x - S1.x), 0.f);
          Ym = make_float2(filter_weight_fast(a, d, cf, (int)a.N) * (X1.y - S1.y), 0.f);
        } else {
          const float2 S2 = (single && i2 == i1) ? S1 : corr_mode_sum(a, vd, sb);
          const float wk = filter_weight_fast(a, d, cf, k);
          const float wm = filter_weight_fast(a, d, cf, (int)a.N - k);
          Yk = pmul(make_float2(wk, wk), psub(X1, S1));
          Ym = cconj(pmul(make_float2(wm, wm), psub(X2, S2)));
        }
        const float2 Ev = pmul(padd(Yk, Ym), half2);
        const float2 Op = cmulc(pmul(psub(Yk, Ym), half2), W);
        r0[i1] = make_float2(Ev.x - Op.y, Ev.y + Op.x);
        if (!(single && i2 == i1)) r1[i2] = make_float2(Ev.x + Op.y, Op.x - Ev.y);
      }
    }
  }
  if constexpr (MODE == kFilterSplit) return;
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = ad.ld_at(bi, e * TPR);
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

// Cross-detector step of correlated noise, one thread per bin slot: t_j = sum_d
// V_dj w_d(k) X_d(k) over all detectors, s = M(k)^-1 t with the per-bin
// M = E^-1 + V^T D^-1 V of corr_minv, stored for kFilterMerge.  Slot 0 carries the
// real bins 0 and N in its two parts (M^-1 of bin N at index N).
template <typename S>
__global__ void k_fast_corr(const TodArgs a, int n_det) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= a.N) return;
  if (a.done && *a.done) return;
  const int r = a.corr_r;
  const int k = (slot & (a.C - 1)) * a.R + (slot >> a.logC);
  const S* X = reinterpret_cast<const S*>(a.spec) + slot;
  const float4* coef = reinterpret_cast<const float4*>(a.coef);
  float2 t[kMaxCorrModes];
  for (int j = 0; j < r; ++j) t[j] = make_float2(0.f, 0.f);
  for (int d = 0; d < n_det; ++d) {
    const float2 x = Store<float, S>::ld(X + (size_t)d * a.N);
    const float4 cf = coef[a.d0 + d];
    const float* vd = a.corrV + (a.d0 + d) * r;
    float wx, wy;
    if (slot == 0) {
      wx = filter_weight_fast(a, a.d0 + d, cf, 0) * x.x;
      wy = filter_weight_fast(a, a.d0 + d, cf, (int)a.N) * x.y;
    } else {
      const float w = filter_weight_fast(a, a.d0 + d, cf, k);
      wx = w * x.x;
      wy = w * x.y;
    }
    for (int j = 0; j < r; ++j) {
      t[j].x = fmaf(vd[j], wx, t[j].x);
      t[j].y = fmaf(vd[j], wy, t[j].y);
    }
  }
  const float* m0 = a.corr_minv + (size_t)slot * r * r;
  const float* m1 = slot == 0 ? a.corr_minv + (size_t)a.N * r * r : m0;   // bin N for the imaginary part
  for (int j = 0; j < r; ++j) {
    float sx = 0.f, sy = 0.f;
    for (int l = 0; l < r; ++l) {
      sx = fmaf(m0[j * r + l], t[l].x, sx);
      sy = fmaf(m1[j * r + l], t[l].y, sy);
    }
    a.corr_s[(size_t)slot * r + j] = make_float2(sx, sy);
  }
}

// M(k)^-1 per bin slot (slot order of the op's split; index N: bin N):
// M = diag(1 / e_j(k)) + sum_d w_d(k) V_d V_d^T, accumulated and inverted in FP64
// (Gauss-Jordan with partial pivoting, r <= 4), stored in FP32.
__global__ void k_corr_minv(const TodArgs a, int n_det, const double* __restrict__ mode_par, double f_samp,
                            float* __restrict__ minv) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot > a.N) return;
  const int r = a.corr_r;
  const int k = slot == (int)a.N ? (int)a.N : (slot & (a.C - 1)) * a.R + (slot >> a.logC);
  double m[kMaxCorrModes][2 * kMaxCorrModes];
  const double f = (double)(k == 0 ? 1 : k) * f_samp / (double)a.n_t;
  for (int j = 0; j < r; ++j) {
    for (int l = 0; l < 2 * r; ++l) m[j][l] = 0.0;
    const double amp = mode_par[3 * j], fk = mode_par[3 * j + 1], al = mode_par[3 * j + 2];
    const double e = amp * amp * (1.0 + pow(f / fk, -al));
    m[j][j] = 1.0 / e;
    m[j][r + j] = 1.0;
  }
  const float4* coef = reinterpret_cast<const float4*>(a.coef);
  for (int d = 0; d < n_det; ++d) {
    const double w = (double)filter_weight_fast(a, d, coef[d], k);
    const float* vd = a.corrV + d * r;
    for (int j = 0; j < r; ++j)
      for (int l = 0; l < r; ++l) m[j][l] += w * (double)vd[j] * (double)vd[l];
  }
  for (int c = 0; c < r; ++c) {
    int piv = c;
    for (int q = c + 1; q < r; ++q)
      if (fabs(m[q][c]) > fabs(m[piv][c])) piv = q;
    if (piv != c)
      for (int l = 0; l < 2 * r; ++l) {
        const double tmp = m[c][l];
        m[c][l] = m[piv][l];
        m[piv][l] = tmp;
      }
    const double inv = 1.0 / m[c][c];
    for (int l = 0; l < 2 * r; ++l) m[c][l] *= inv;
    for (int q = 0; q < r; ++q)
      if (q != c) {
        const double fq = m[q][c];
        for (int l = 0; l < 2 * r; ++l) m[q][l] -= fq * m[c][l];
      }
  }
  for (int j = 0; j < r; ++j)
    for (int l = 0; l < r; ++l) minv[(size_t)slot * r * r + j * r + l] = (float)m[j][r + l];
}

// ------------------------------------------------------------------ pass T' (inverse + P^T)

template <int NC, typename S, int R, bool PERIODIC, bool CACHED>
__global__ void __launch_bounds__(ColShape<R>::THREADS, ColShape<R>::MINB_INV) k_fast_inv_bin(const TodArgs a, int nd) {
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
  const int npix = (int)a.npix;
  // binning layout: BS = row stride of the tile (the 2-complex pad spreads the
  // rows' 16-byte reads over all banks), LPR lanes per row, RPP rows per pass
  constexpr int BS = J + 2;
  constexpr int H = kBinHalves;           // groups of 8 consecutive samples per lane
  constexpr int LPR = J / (4 * H);        // lanes per row
  static_assert(LPR >= 1, "a row must hold the lane's samples");
  constexpr int RPP = ColShape<R>::THREADS / LPR;
  constexpr int PSTR = 2 * J + 4;   // ints per staged pixel row (the pad spreads 16-byte reads over the banks)
  const int bq = threadIdx.x % LPR;
  const int br = threadIdx.x / LPR;
  const int c0 = blockIdx.x * J;
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
    // filtered samples into a tile of rows kr (stride J + 2 complex) for the binning
#pragma unroll
    for (int e = 0; e < kE; ++e) smf[(i + e * TPC) * BS + cl] = x[e];
    __syncthreads();
    const int2 off = a.det_off[d];
    const float2 pol = reinterpret_cast<const float2*>(a.pol)[d];
    const int* pixd = CACHED ? a.pix + (size_t)d * a.n_t : nullptr;
    int* pst = reinterpret_cast<int*>(smf + R * BS);   // pixel staging of one pass (on-the-fly pointing)
    // each lane bins 8 H consecutive samples: 4 H complex of row kr from column 4 H q
#pragma unroll kBinUnroll
    for (int kr0 = 0; kr0 < R; kr0 += RPP) {
      const int kr = kr0 + br;
      const int tq = 2 * (c0 + 4 * H * bq + kr * a.C);
      if constexpr (!CACHED) {
        // pixels of the pass's RPP rows x 2J samples, lanes on consecutive samples
        // (coalesced boresight reads), staged in shared memory
#pragma unroll
        for (int k = 0; k < 8 * H; ++k) {
          const int sidx = threadIdx.x + k * ColShape<R>::THREADS;
          const int rr = sidx / (2 * J), col = sidx % (2 * J);
          const int ts = 2 * (c0 + (kr0 + rr) * a.C) + col;
          pst[rr * PSTR + col] = pixel_fast<PERIODIC>(__ldg(a.bore + ts), off, a.ny, a.nx, npix);
        }
        __syncthreads();
      }
      BinRun run;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int t = tq + 8 * h;
        int p[8];
        int4 P0, P1;
        if constexpr (!CACHED) {
          P0 = *reinterpret_cast<const int4*>(pst + br * PSTR + 8 * H * bq + 8 * h);
          P1 = *reinterpret_cast<const int4*>(pst + br * PSTR + 8 * H * bq + 8 * h + 4);
        } else if constexpr (CMM_V8) {
          ld_cs_v8(pixd + t, p);   // 32-byte aligned: t and n_t are multiples of 8
        } else {
          P0 = __ldcs(reinterpret_cast<const int4*>(pixd + t));
          P1 = __ldcs(reinterpret_cast<const int4*>(pixd + t + 4));
        }
        if constexpr (!CACHED || !CMM_V8) {
          p[0] = P0.x; p[1] = P0.y; p[2] = P0.z; p[3] = P0.w;
          p[4] = P1.x; p[5] = P1.y; p[6] = P1.z; p[7] = P1.w;
        }
        const float4 A = *reinterpret_cast<const float4*>(smf + kr * BS + 4 * H * bq + 4 * h);
        const float4 B = *reinterpret_cast<const float4*>(smf + kr * BS + 4 * H * bq + 4 * h + 2);
        float u[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
        float cc[8], ss[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) u[k] *= scale;
        if (NC == 3) {
#pragma unroll
          for (int k = 0; k < 8; k += 4) {
            float4 r2[2];
            if constexpr (CMM_V8) {
              float v[8];
              ld_nc_v8(a.rot2 + t + k, v);
              r2[0] = make_float4(v[0], v[1], v[2], v[3]);
              r2[1] = make_float4(v[4], v[5], v[6], v[7]);
            } else {
              r2[0] = __ldg(reinterpret_cast<const float4*>(a.rot2 + t + k));
              r2[1] = __ldg(reinterpret_cast<const float4*>(a.rot2 + t + k + 2));
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int kk = k + 2 * j;
              cc[kk] = pol.x * r2[j].x - pol.y * r2[j].y;
              ss[kk] = pol.y * r2[j].x + pol.x * r2[j].y;
              cc[kk + 1] = pol.x * r2[j].z - pol.y * r2[j].w;
              ss[kk + 1] = pol.y * r2[j].z + pol.x * r2[j].w;
            }
          }
        }
        bin_push8<NC>(a.acc32, run, p, u, cc, ss, npix);
      }
      bin_close<NC>(a.acc32, run, npix);
      if constexpr (!CACHED) __syncthreads();   // the staging is rewritten by the next pass
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

// ------------------------------------------------------------------ pointing cache
// pix[d][t] = pixel of sample t of detector d (npix outside the map), by the rule
// of the on-the-fly kernels.
template <bool PERIODIC>
__global__ void k_fill_pixels(const TodArgs a, int n_det, int* __restrict__ pix) {
  const long long total = (long long)n_det * a.n_t;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int d = (int)(q / a.n_t);
    const int t = (int)(q - (long long)d * a.n_t);
    pix[q] = pixel_fast<PERIODIC>(__ldg(a.bore + t), a.det_off[d], a.ny, a.nx, (int)a.npix);
  }
}

int launch_fill_pixels(cmm_op* op) {
  TodArgs a = make_args(op, 0);
  const long long total = (long long)op->pt->n_det * op->pt->n_t;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  if (a.periodic) k_fill_pixels<true><<<blocks, 256, 0, op->ctx->stream>>>(a, op->pt->n_det, op->pix);
  else k_fill_pixels<false><<<blocks, 256, 0, op->ctx->stream>>>(a, op->pt->n_det, op->pix);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
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

template <int NC, typename S, int R, bool PERIODIC, bool CACHED>
static int run_T_c(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  constexpr int J = ColShape<R>::J;
  constexpr int NT = ColShape<R>::THREADS;
  // forward: FFT tile R x J complex.  inverse: binning tile R x (J + 2) complex,
  // then the pixel staging of one binning pass, (threads / (J / 4)) rows x (2 J + 4) ints
  const int smem_f = (int)(sizeof(float2) * R * J);
  const int smem_i = (int)(sizeof(float2) * R * (J + 2) + sizeof(int) * (NT / (J / (4 * kBinHalves))) * (2 * J + 4));
  if (attr_only) {
    CMM_CUDA(cudaFuncSetAttribute(k_fast_fwd<NC, S, R, PERIODIC, CACHED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_f));
    CMM_CUDA(cudaFuncSetAttribute(k_fast_inv_bin<NC, S, R, PERIODIC, CACHED>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem_i));
    return CMM_OK;
  }
  const dim3 g(a.C / J, (nd + kDetsPerCta - 1) / kDetsPerCta);
  if (pass == 0) k_fast_fwd<NC, S, R, PERIODIC, CACHED><<<g, NT, smem_f, st>>>(a, nd);
  else k_fast_inv_bin<NC, S, R, PERIODIC, CACHED><<<g, NT, smem_i, st>>>(a, nd);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

// The cached-pixel kernels exist only for the non-periodic map (the periodic
// boundary is a test geometry).
template <int NC, typename S, int R, bool PERIODIC>
static int run_T(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  if constexpr (!PERIODIC) {
    if (attr_only) CMM_TRY((run_T_c<NC, S, R, false, true>(a, nd, pass, st, true)));
    else if (a.pix) return run_T_c<NC, S, R, false, true>(a, nd, pass, st, false);
  }
  return run_T_c<NC, S, R, PERIODIC, false>(a, nd, pass, st, attr_only);
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

template <typename S, int MODE, int E, int... RC>
static int run_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  constexpr int C = RadProd<RC...>::value;
  constexpr int ROWS = FilterShape<C, E>::ROWS;
  constexpr int PAIRS = ROWS / 2;
  constexpr int PS = clog2(E);
  const size_t smem = sizeof(float2) * ROWS * (C + (C >> PS));
  if (attr_only) {
    CMM_CUDA(cudaFuncSetAttribute(k_fast_filter<S, MODE, E, RC...>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    return CMM_OK;
  }
  const int npairs = a.R / 2 + 1;
  const dim3 g((npairs + PAIRS - 1) / PAIRS, nd);
  k_fast_filter<S, MODE, E, RC...><<<g, FilterShape<C, E>::THREADS, smem, st>>>(a);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <typename S, int MODE>
static int dispatch_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  switch (a.logC) {
    case 6: return run_F<S, MODE, 16, 16, 4>(a, nd, st, attr_only);
    case 7: return run_F<S, MODE, 16, 16, 8>(a, nd, st, attr_only);
    case 8: return run_F<S, MODE, 16, 16, 16>(a, nd, st, attr_only);
    case 9: return run_F<S, MODE, 16, 16, 16, 2>(a, nd, st, attr_only);
    case 10: return run_F<S, MODE, 16, 16, 16, 4>(a, nd, st, attr_only);
    case 11: return run_F<S, MODE, 16, 16, 16, 8>(a, nd, st, attr_only);
    default: return run_F<S, MODE, 16, 16, 16, 16>(a, nd, st, attr_only);
  }
}

// Flush of `maps` FP32 partial maps (map_elems elements apart) into the FP64 map:
// per pixel the partials are summed in FP64, added once, and cleared.
template <int NC>
__global__ void k_fast_flush_maps(float* __restrict__ acc32, int maps, long long map_elems, double* __restrict__ acc,
                                  long long npix, const int* done) {
  if (done && *done) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      double s = 0.0;
      bool any = false;
      for (int g = 0; g < maps; ++g) {
        float* q = acc32 + g * map_elems + p;
        const float v = *q;
        if (v != 0.0f) {
          s += (double)v;
          *q = 0.0f;
          any = true;
        }
      }
      if (any) acc[p] += s;
    } else {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      bool any = false;
      for (int g = 0; g < maps; ++g) {
        float4* q = reinterpret_cast<float4*>(acc32 + g * map_elems) + p;
        const float4 v = *q;
        if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f) {
          s0 += (double)v.x;
          s1 += (double)v.y;
          s2 += (double)v.z;
          *q = make_float4(0.f, 0.f, 0.f, 0.f);
          any = true;
        }
      }
      if (any) {
        double* d = acc + 4 * p;
        d[0] += s0;
        d[1] += s1;
        d[2] += s2;
      }
    }
  }
}

int launch_flush(const TodArgs& a, int nc, cudaStream_t st);

int launch_flush_maps(const TodArgs& a, int nc, int maps, cudaStream_t st) {
  if (maps <= 1) return launch_flush(a, nc, st);
  const int blocks = (int)std::min<long long>((a.npix + 256) / 256, 4096);
  if (nc == 1) k_fast_flush_maps<1><<<blocks, 256, 0, st>>>(a.acc32, maps, a.acc32_map, a.acc, a.npix + 1, a.done);
  else k_fast_flush_maps<3><<<blocks, 256, 0, st>>>(a.acc32, maps, a.acc32_map, a.acc, a.npix + 1, a.done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_flush(const TodArgs& a, int nc, cudaStream_t st) {
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
  if (pass < 0 || pass == 1) {
    if (a.corr_r > 0) {
      // correlated noise: split, cross-detector solve over the whole chunk, merge
      CMM_TRY((dispatch_F<S, kFilterSplit>(a, nd, st, false)));
      k_fast_corr<S><<<(int)((a.N + 255) / 256), 256, 0, st>>>(a, nd);
      CMM_LAUNCH_CHECK();
      CMM_TRY((dispatch_F<S, kFilterMerge>(a, nd, st, false)));
    } else {
      CMM_TRY((dispatch_F<S, kFilterFull>(a, nd, st, false)));
    }
  }
  if (pass < 0 || pass == 2) {
    for (int g0 = 0; g0 < nd; g0 += kFlushDets) {
      TodArgs b = a;
      const int gn = std::min(kFlushDets, nd - g0);
      b.d0 = a.d0 + g0;
      b.spec = reinterpret_cast<S*>(a.spec) + (long long)g0 * a.N;
      if (nc == 1) CMM_TRY((dispatch_T<1, S>(b, gn, 2, st, false)));
      else CMM_TRY((dispatch_T<3, S>(b, gn, 2, st, false)));
      CMM_TRY(launch_flush(b, nc, st));
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
  CMM_TRY((dispatch_F<S, kFilterFull>(a, 0, nullptr, true)));
  CMM_TRY((dispatch_F<S, kFilterSplit>(a, 0, nullptr, true)));
  return dispatch_F<S, kFilterMerge>(a, 0, nullptr, true);
}

int launch_corr_minv(cmm_op* op, const double* mode_par_dev, float* minv) {
  TodArgs a = make_args(op, 0);
  a.corr_r = op->nz->corr_r;   // the tables are being built: make_args does not count them yet
  const long long n = op->N + 1;
  k_corr_minv<<<(int)((n + 127) / 128), 128, 0, op->ctx->stream>>>(a, op->pt->n_det, mode_par_dev, op->nz->f_samp,
                                                                  minv);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int prepare_fast(cmm_op* op) {
  return op->prec == CMM_PREC_BF16 ? prepare_fast_s<__nv_bfloat162>(op) : prepare_fast_s<float2>(op);
}

}  // namespace cmm
