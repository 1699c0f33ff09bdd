// Pair-packed fast path of A = P^T N^-1 P (Eq. 2; pointing of Eq. 1 with the response
// of Sec. Test setup; N^-1 the per-detector Fourier-diagonal noise filter of the
// Introduction and Sec. Test setup) for FP32 compute (FP32 or BF16 spectrum storage),
// detectors with independent noise.
//
// Two detectors d1, d2 share one complex sequence of n_t points, z(t) = s1(t) +
// i s2(t): each complex element is one time sample of both detectors, so the
// boresight and rotation tables are read once per element for the two of them, by
// lanes on consecutive samples (coalesced).  With Z = FFT(z), the real spectra are
// S1(k) = (Z(k) + conj Z(n_t - k)) / 2 and i S2(k) = (Z(k) - conj Z(n_t - k)) / 2, so
// the filtered sequence y = y1 + i y2 has
//     Y(k) = a Z(k) + b conj Z(n_t - k),  a = (w1 + w2) / 2,  b = (w1 - w2) / 2,
// w_j = w_dj at the frequency index min(k, n_t - k) of the n_t-point DFT: each bin
// pair (k, n_t - k) is filtered with four real products and no split twiddle.
// n_t = R C as a four-step FFT over t = c + C kr (c < C contiguous, kr < R):
//
//   k_pair_fwd:     P m for both detectors at (c, kr), the R-point column FFTs over
//                   kr (register-resident, one shared-memory exchange), times
//                   w_{n_t}^{c k1}.
//   k_pair_filter:  row pairs (k1, R - k1): C-point row FFTs, the pair filter in
//                   registers (each thread against the elements of one partner
//                   thread), the inverse row FFTs and the conjugate twiddle.
//   k_pair_inv_bin: inverse column FFTs into a padded tile; each lane then takes 8
//                   consecutive samples of a row and bins them for each detector
//                   with a run accumulator (one vector FP32 reduction per run into
//                   the L2-resident partial map of its group of kFlushDets = 256
//                   detectors).
//   k_fast_flush_maps (tod_fast.cu) sums a launch's partial maps in FP64 into the
//   FP64 map, so no FP32 sum covers more than 256 detectors.
//
// A chunk with an odd number of detectors pairs its last detector with nothing
// (the imaginary part stays zero and is not binned).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "fft_reg.cuh"
#include "tod_common.cuh"
#include "tod_fast.cuh"

namespace cmm {

// Tuning knobs of this path (compile-time; the defaults are the measured best).
#ifndef CMM_PAIR_ROT
#define CMM_PAIR_ROT 1     // forward pass: 0 = (cos 2phi, sin 2phi) from the FP32 table, 1 = from the boresight record
#endif
#ifndef CMM_PAIR_XOR
#define CMM_PAIR_XOR 1     // pixel staging: 0 = rows padded to J + 8 ints, 1 = XOR-swizzled 16-byte chunks (no pad)
#endif
#ifndef CMM_PAIR_FILTER_THREADS_PER_SM
#define CMM_PAIR_FILTER_THREADS_PER_SM 1024
#endif

// A binning run in the frame of the scan rotation: for samples of one detector on
// one pixel, sums of u, u cos 2phi_t and u sin 2phi_t; the detector angle psi_d
// enters once, when the run is reduced: sum u cos 2(psi + phi) = cos 2psi * sum u
// cos 2phi - sin 2psi * sum u sin 2phi (and the sine likewise), with the inverse
// FFT's 1/N folded into (sx, sy) = (cos 2psi, sin 2psi) / N and st = 1/N.
struct PairRun {
  int cur = -1;
  float t = 0.f, c = 0.f, s = 0.f;
};

template <int NC>
__device__ __forceinline__ void pair_run_close(float* acc32, const PairRun& r, int skip, float st, float sx, float sy) {
  if (r.cur >= 0 && r.cur != skip) {
    if (NC == 1) red_add(acc32 + r.cur, st * r.t);
    else red_add4(acc32 + 4 * r.cur, st * r.t, fmaf(sx, r.c, -sy * r.s), fmaf(sy, r.c, sx * r.s));
  }
}

// (cos 2phi, sin 2phi) of the fixed-point pair (c, s) of a boresight record, in FP32:
// (c^2 - s^2, 2 c s) / (c^2 + s^2), the integers converted exactly on the FP32 pipe
__device__ __forceinline__ float2 rot2_of_bore(const int4 b) {
  const float cf = small_int_to_float(b.z + 32768) - 32768.0f;
  const float sf = small_int_to_float(b.w + 32768) - 32768.0f;
  const float inv = __fdividef(1.0f, fmaf(cf, cf, sf * sf));
  return make_float2((cf - sf) * (cf + sf) * inv, 2.0f * cf * sf * inv);
}

// w_d at frequency index kf (0 <= kf <= n_t / 2): the detector's table, else the law
__device__ __forceinline__ float pair_weight(const TodArgs& a, int d, const float4 cf, int kf) {
  if (a.wtab) return __ldg(reinterpret_cast<const float*>(a.wtab) + (size_t)d * (a.n_t / 2 + 1) + kf);
  return filter_weight_law(cf, kf);
}

// w_d1 and w_d2 at frequency index kf: the tables, else the law with log2(kf) shared
__device__ __forceinline__ void pair_weights(const TodArgs& a, int d1, int d2, const float4 cf1, const float4 cf2,
                                             bool two, int kf, float& w1, float& w2) {
  if (a.wtab) {
    w1 = pair_weight(a, d1, cf1, kf);
    w2 = two ? pair_weight(a, d2, cf2, kf) : 0.f;
    return;
  }
  const float lk = __log2f(small_int_to_float(kf == 0 ? 1 : kf));
  w1 = cf1.w != 0.0f ? cf1.x : __fdividef(cf1.x, 1.0f + exp2f(fmaf(-cf1.y, lk, cf1.z)));
  w2 = !two ? 0.f : cf2.w != 0.0f ? cf2.x : __fdividef(cf2.x, 1.0f + exp2f(fmaf(-cf2.y, lk, cf2.z)));
}

// (P m)(t) of one detector from its pixel, the response table entry and the gather copy
template <int NC>
__device__ __forceinline__ float pair_project(const TodArgs& a, int p, const float2 pol, const float2 r2) {
  if (NC == 1) return __ldg((const float*)a.gather + p);
  const float4 g = __ldg((const float4*)a.gather + p);
  const float c = pol.x * r2.x - pol.y * r2.y;
  const float s = pol.y * r2.x + pol.x * r2.y;
  return fmaf(s, g.z, fmaf(c, g.y, g.x));
}

// ------------------------------------------------------------------ pass T (forward)
template <int NC, typename S, int R, bool PERIODIC, bool CACHED>
__global__ void __launch_bounds__(ColShape<R>::THREADS, ColShape<R>::MINB) k_pair_fwd(const TodArgs a, int nd) {
  constexpr int TPC = R / kE;
  constexpr int J = ColShape<R>::J;
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float2 smf[];
  const int cl = threadIdx.x % J;
  const int i = threadIdx.x / J;
  const int c = blockIdx.x * J + cl;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  const ColJ<J> ad{smf, cl};
  const int q = blockIdx.y;   // pair within the chunk
  const bool two = 2 * q + 1 < nd;
  const int d1 = a.d0 + 2 * q, d2 = two ? d1 + 1 : d1;
  const int2 off1 = a.det_off[d1], off2 = a.det_off[d2];
  const float2* pol = reinterpret_cast<const float2*>(a.pol);
  const float2 pol1 = pol[d1], pol2 = pol[d2];
  const int npix = (int)a.npix;
  float2 x[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const int t = c + (i + e * TPC) * a.C;
    int p1, p2;
    float2 r2 = make_float2(0.f, 0.f);
    if constexpr (CACHED) {
      p1 = __ldcs(a.pix + (size_t)d1 * a.n_t + t);
      p2 = __ldcs(a.pix + (size_t)d2 * a.n_t + t);
      if (NC == 3) r2 = __ldg(a.rot2 + t);
    } else {
      const int4 b = __ldg(a.bore + t);
      p1 = pixel_fast<PERIODIC>(b, off1, a.ny, a.nx, npix);
      p2 = pixel_fast<PERIODIC>(b, off2, a.ny, a.nx, npix);
      if (NC == 3) r2 = CMM_PAIR_ROT ? rot2_of_bore(b) : __ldg(a.rot2 + t);
    }
    const float v1 = pair_project<NC>(a, p1, pol1, r2);
    const float v2 = pair_project<NC>(a, p2, pol2, r2);
    x[e] = make_float2(v1, two ? v2 : 0.f);
  }
  ColPlan<R>::template run<-1>(x, i, tw + a.twl.R_off, ad);
  // four-step twiddle w_N^(c kr), kr = i + e TPC, by recurrence over e
  float2 w = tw_N(a, tw, c * i);
  const float2 step = tw_N(a, tw, c * TPC);
  S* Y = reinterpret_cast<S*>(a.spec) + (size_t)q * a.N + c + i * a.C;
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    Store<float, S>::st(Y + e * (TPC * a.C), cmul(x[e], w));
    w = cmul(w, step);
  }
}

// ------------------------------------------------------------------ pass F (filter)
template <int C, int E> struct PairFilterShape {
  static constexpr int TPR = C / E;
  static constexpr int THREADS = 2 * TPR > 256 ? 2 * TPR : 256;
  static constexpr int ROWS = THREADS / TPR;
  static constexpr int MINB = THREADS >= CMM_PAIR_FILTER_THREADS_PER_SM ? 1 : CMM_PAIR_FILTER_THREADS_PER_SM / THREADS;
};

template <typename S, int E, int... RC>
__global__ void __launch_bounds__(PairFilterShape<RadProd<RC...>::value, E>::THREADS,
                                  PairFilterShape<RadProd<RC...>::value, E>::MINB)
    k_pair_filter(const TodArgs a, int nd) {
  constexpr int C = RadProd<RC...>::value;
  constexpr int TPR = C / E;
  constexpr int ROWS = PairFilterShape<C, E>::ROWS;
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
  const int q = blockIdx.y;
  const bool two = 2 * q + 1 < nd;
  const int d1 = a.d0 + 2 * q, d2 = two ? d1 + 1 : d1;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  S* Y = reinterpret_cast<S*>(a.spec) + (size_t)q * a.N;
  const RowAddr<PS> ad{smf + rs * ROWLEN};
  float2 x[E];
  const int bi = ad.base(i);
#pragma unroll
  for (int e = 0; e < E; ++e)
    x[e] = active ? Store<float, S>::ld(Y + row * C + i + e * TPR) : make_float2(0.f, 0.f);
  rfft<-1, E, RC...>(x, i, tw + a.twl.C_off, ad);
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) ad.st_at(bi, e * TPR, x[e]);
  const bool wrap = row == 0;
  const int n = (int)a.N;
  __syncthreads();
  // Each thread filters its own elements in registers.  Position pos of row `row`
  // holds Z(k), k = row + R pos; Z(n - k) sits at position C - 1 - pos of row
  // R - row (for row 0: (C - pos) mod C of row 0), held by one partner thread;
  // both threads form a Z + b conj(partner) with the same (a, b), since
  // min(k, n - k) is the same for the two.  The inverse FFT's first stage starts
  // with a barrier, so the partner reads below finish before the buffer is reused.
  if (active) {
    const float4 cf1 = reinterpret_cast<const float4*>(a.coef)[d1];
    const float4 cf2 = reinterpret_cast<const float4*>(a.coef)[d2];
    const RowAddr<PS> pa{smf + (single ? rs : (rs ^ 1)) * ROWLEN};
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int pos = i + e * TPR;
      const int pp = wrap ? ((C - pos) & (C - 1)) : (C - 1 - pos);
      const float2 B = pa.ld(pp);
      const int k = row + a.R * pos;
      const int kf = min(k, n - k);
      float w1, w2;
      pair_weights(a, d1, d2, cf1, cf2, two, kf, w1, w2);
      const float ha = 0.5f * (w1 + w2), hb = 0.5f * (w1 - w2);
      x[e] = make_float2(fmaf(ha, x[e].x, hb * B.x), fmaf(ha, x[e].y, -hb * B.y));
    }
  }
  rfft<1, E, RC...>(x, i, tw + a.twl.C_off, ad);
  if (active) {
    // w_N^(row c), c = i + e TPR, by recurrence over e
    float2 w = tw_N(a, tw, row * i);
    const float2 stp = tw_N(a, tw, row * TPR);
    S* Yr = Y + row * C + i;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      Store<float, S>::st(Yr + e * TPR, cmulc(x[e], w));
      w = cmul(w, stp);
    }
  }
}

// ------------------------------------------------------------------ pass T' (inverse + P^T)
template <int NC, typename S, int R, bool PERIODIC, bool CACHED>
__global__ void __launch_bounds__(ColShape<R>::THREADS, ColShape<R>::MINB_INV) k_pair_inv_bin(const TodArgs a, int nd) {
  constexpr int TPC = R / kE;
  constexpr int J = ColShape<R>::J;
  constexpr int NT = ColShape<R>::THREADS;
  constexpr int BS = J + 2;    // row stride of the binning tile (the pad spreads rows over the banks)
  constexpr int SPL = 8;              // consecutive samples per lane
  constexpr int LPR = J / SPL;        // lanes per row
  constexpr int RPP = NT / LPR;       // rows per binning pass
  // Pixel staging: row stride PS ints; a lane's 8 pixels are two 16-byte chunks
  // interleaved with its row neighbour's (chunk h of lane bq at word 8h + 4bq of a
  // 16-sample group), so that the eight lanes of a quarter-warp load hit eight
  // distinct 4-bank groups (PS = 24 words = 8 mod 32 shifts consecutive rows).
  constexpr int PS = CMM_PAIR_XOR ? J + (J == 32 ? 8 : 0) : J + 8;
  static_assert(LPR >= 1 && RPP <= R && R % RPP == 0 && (RPP * J) % NT == 0, "binning layout");
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float2 smf[];
  const int cl = threadIdx.x % J;
  const int i = threadIdx.x / J;
  const int c = blockIdx.x * J + cl;
  const int c0 = blockIdx.x * J;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  const ColJ<J> ad{smf, cl};
  const int q = blockIdx.y;
  const bool two = 2 * q + 1 < nd;
  const int d1 = a.d0 + 2 * q, d2 = two ? d1 + 1 : d1;
  // the FP32 partial map of this pair's group of detectors (whole pairs per group)
  float* const acc32 = a.acc32 + (long long)((2 * q) / a.flush_dets) * a.acc32_map;
  const float scale = 1.0f / (float)a.N;
  const int npix = (int)a.npix;
  const S* Y = reinterpret_cast<const S*>(a.spec) + (size_t)q * a.N + c + i * a.C;
  float2 x[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) x[e] = Store<float, S>::ld(Y + e * (TPC * a.C));
  ColPlan<R>::template run<1>(x, i, tw + a.twl.R_off, ad);
  __syncthreads();
  // y(t) for t = c + C kr into a tile of rows kr
#pragma unroll
  for (int e = 0; e < kE; ++e) smf[(i + e * TPC) * BS + cl] = x[e];
  __syncthreads();
  const int bq = threadIdx.x % LPR;
  const int br = threadIdx.x / LPR;
  const float2* pol = reinterpret_cast<const float2*>(a.pol);
  const float2 pol1 = pol[d1], pol2 = pol[d2];
  const int2 off1 = a.det_off[d1], off2 = a.det_off[d2];
  int* pst = reinterpret_cast<int*>(smf + R * BS);   // pixels of one pass: [detector][RPP][PS]
  const float4* smf4 = reinterpret_cast<const float4*>(smf);
  for (int kr0 = 0; kr0 < R; kr0 += RPP) {
    const int kr = kr0 + br;
    const int tq = c0 + SPL * bq + kr * a.C;   // the lane's first sample
    // the lane's 8 rotations (64 bytes, 64-byte aligned: tq is a multiple of 8),
    // issued before the staging so that they are in flight across its barrier
    float2 r2[8];
    if (NC == 3) {
      if constexpr (CMM_V8) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[8];
          ld_nc_v8(a.rot2 + tq + 4 * h, v);
#pragma unroll
          for (int k = 0; k < 4; ++k) r2[4 * h + k] = make_float2(v[2 * k], v[2 * k + 1]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(a.rot2 + tq + k));
          r2[k] = make_float2(v.x, v.y);
          r2[k + 1] = make_float2(v.z, v.w);
        }
      }
    }
    if constexpr (!CACHED) {
      // pixels of both detectors for the pass's RPP x J samples, lanes on
      // consecutive samples (coalesced boresight reads)
#pragma unroll
      for (int k = 0; k < RPP * J / NT; ++k) {
        const int sidx = threadIdx.x + k * NT;
        const int rr = sidx / J, col = sidx % J;
        const int4 b = __ldg(a.bore + c0 + col + (kr0 + rr) * a.C);
        // column col = 16 g + 8 bq + 4 h + w of the row goes to word 16 g + 8 h + 4 bq + w
        // (padded rows), or to chunk (2 h + bq) ^ (row & 3) of its 16-word group
        const int sw = CMM_PAIR_XOR ? (col & ~15) | (((((col >> 1) & 2) | ((col >> 3) & 1)) ^ (rr & 3)) << 2) | (col & 3)
                                    : (col & ~15) | ((col & 4) << 1) | ((col & 8) >> 1) | (col & 3);
        pst[rr * PS + sw] = pixel_fast<PERIODIC>(b, off1, a.ny, a.nx, npix);
        pst[(RPP + rr) * PS + sw] = pixel_fast<PERIODIC>(b, off2, a.ny, a.nx, npix);
      }
      __syncthreads();
    }
    // the lane's 8 filtered samples of both detectors (real part: d1, imaginary: d2)
    float4 yv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) yv[j] = smf4[(kr * BS + 8 * bq) / 2 + j];
#pragma unroll
    for (int dd = 0; dd < 2; ++dd) {
      if (dd == 1 && !two) break;
      int p[8];
      int4 P0, P1;
      if constexpr (CACHED && CMM_V8) {
        // 32 bytes, 32-byte aligned (tq and n_t are multiples of 8)
        ld_cs_v8(a.pix + (size_t)(dd ? d2 : d1) * a.n_t + tq, p);
        P0 = make_int4(p[0], p[1], p[2], p[3]);
        P1 = make_int4(p[4], p[5], p[6], p[7]);
      } else if constexpr (CACHED) {
        const int* pixd = a.pix + (size_t)(dd ? d2 : d1) * a.n_t + tq;
        P0 = __ldcs(reinterpret_cast<const int4*>(pixd));
        P1 = __ldcs(reinterpret_cast<const int4*>(pixd + 4));
      } else {
        const int* prow = pst + (dd * RPP + br) * PS + ((bq >> 1) << 4);
        if (CMM_PAIR_XOR) {
          // chunks (2 h + bq % 2) ^ (row & 3) of the 16-word group
          P0 = *reinterpret_cast<const int4*>(prow + (((bq & 1) ^ (br & 3)) << 2));
          P1 = *reinterpret_cast<const int4*>(prow + (((2 | (bq & 1)) ^ (br & 3)) << 2));
        } else {
          // chunks h = 0, 1 of the lane's 8 pixels at words 16 (bq / 2) + 4 (bq % 2) + 8 h
          const int4* ps = reinterpret_cast<const int4*>(prow + ((bq & 1) << 2));
          P0 = ps[0];
          P1 = ps[2];
        }
      }
      p[0] = P0.x; p[1] = P0.y; p[2] = P0.z; p[3] = P0.w;
      p[4] = P1.x; p[5] = P1.y; p[6] = P1.z; p[7] = P1.w;
      const float2 pl = dd ? pol2 : pol1;
      const float sx = scale * pl.x, sy = scale * pl.y;
      PairRun run;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 v = yv[k >> 1];
        const float u = dd ? ((k & 1) ? v.w : v.y) : ((k & 1) ? v.z : v.x);
        if (p[k] != run.cur) {
          pair_run_close<NC>(acc32, run, npix, scale, sx, sy);
          run.cur = p[k];
          run.t = 0.f;
          run.c = 0.f;
          run.s = 0.f;
        }
        run.t += u;
        if (NC == 3) {
          run.c = fmaf(r2[k].x, u, run.c);
          run.s = fmaf(r2[k].y, u, run.s);
        }
      }
      pair_run_close<NC>(acc32, run, npix, scale, sx, sy);
    }
    if constexpr (!CACHED) __syncthreads();   // the staging is rewritten by the next pass
  }
}

// ------------------------------------------------------------------ dispatch

// Split of the pair sequence, n_t = 2^log_nt points: R = 64 below 2^16, 128 for 2^16
// and 2^17, 256 from 2^18 (rows C = n_t / R of 128 to 4096 points).
bool pair_path_sizes(int log_nt, int prec, int* logR, int* logC) {
  if (prec == CMM_PREC_F64 || log_nt < 13 || log_nt > 20) return false;
  *logR = log_nt < 16 ? 6 : (log_nt < 18 ? 7 : 8);
  *logC = log_nt - *logR;
  return true;
}

bool pair_path_ok(const cmm_op* op) {
  return op->pair && op->pR > 0 && op->tw_pair && op->nz->corr_r == 0 && op->pt->max_hits <= kF32HitLimit;
}

static TodArgs pair_args(const cmm_op* op, int d0) {
  TodArgs a = make_args(op, d0);
  a.N = op->pt->n_t;
  a.R = op->pR;
  a.C = op->pC;
  a.logR = op->plogR;
  a.logC = op->plogC;
  a.tw = op->tw_pair;
  a.twl = tw_layout(op->pR, op->pC);
  return a;
}

template <int NC, typename S, int R, bool PERIODIC, bool CACHED>
static int run_pair_T_c(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  constexpr int J = ColShape<R>::J;
  constexpr int NT = ColShape<R>::THREADS;
  // forward: FFT tile R x J complex.  inverse: binning tile R x (J + 2) complex, the
  // pixel staging of one pass (2 detectors x RPP rows x (J + 8) ints) and, when the
  // rotation is staged, RPP rows x (J + 2) complex
  constexpr int RPP = NT / (J / 8);   // rows per binning pass
  const int smem_f = (int)(sizeof(float2) * R * J);
  constexpr int PS = CMM_PAIR_XOR ? J + (J == 32 ? 8 : 0) : J + 8;
  // (the pixel-cache instances stage no pixels: less shared memory leaves more L1)
  const int smem_i = (int)(sizeof(float2) * R * (J + 2) + (CACHED ? 0 : sizeof(int) * 2 * RPP * PS));
  if (attr_only) {
    CMM_CUDA(cudaFuncSetAttribute(k_pair_fwd<NC, S, R, PERIODIC, CACHED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_f));
    CMM_CUDA(cudaFuncSetAttribute(k_pair_inv_bin<NC, S, R, PERIODIC, CACHED>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem_i));
    return CMM_OK;
  }
  const dim3 g(a.C / J, (nd + 1) / 2);
  if (pass == 0) k_pair_fwd<NC, S, R, PERIODIC, CACHED><<<g, NT, smem_f, st>>>(a, nd);
  else k_pair_inv_bin<NC, S, R, PERIODIC, CACHED><<<g, NT, smem_i, st>>>(a, nd);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

// The cached-pixel kernels exist only for the non-periodic map.
template <int NC, typename S, int R, bool PERIODIC>
static int run_pair_T(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  if constexpr (!PERIODIC) {
    if (attr_only) CMM_TRY((run_pair_T_c<NC, S, R, false, true>(a, nd, pass, st, true)));
    else if (a.pix) return run_pair_T_c<NC, S, R, false, true>(a, nd, pass, st, false);
  }
  return run_pair_T_c<NC, S, R, PERIODIC, false>(a, nd, pass, st, attr_only);
}

template <int NC, typename S, bool PERIODIC>
static int dispatch_pair_T_p(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  if (a.logR == 6) return run_pair_T<NC, S, 64, PERIODIC>(a, nd, pass, st, attr_only);
  if (a.logR == 7) return run_pair_T<NC, S, 128, PERIODIC>(a, nd, pass, st, attr_only);
  return run_pair_T<NC, S, 256, PERIODIC>(a, nd, pass, st, attr_only);
}

template <int NC, typename S>
static int dispatch_pair_T(const TodArgs& a, int nd, int pass, cudaStream_t st, bool attr_only) {
  return a.periodic ? dispatch_pair_T_p<NC, S, true>(a, nd, pass, st, attr_only)
                    : dispatch_pair_T_p<NC, S, false>(a, nd, pass, st, attr_only);
}

template <typename S, int E, int... RC>
static int run_pair_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  constexpr int C = RadProd<RC...>::value;
  constexpr int ROWS = PairFilterShape<C, E>::ROWS;
  constexpr int PAIRS = ROWS / 2;
  constexpr int PS = clog2(E);
  const size_t smem = sizeof(float2) * ROWS * (C + (C >> PS));
  if (attr_only) {
    CMM_CUDA(cudaFuncSetAttribute(k_pair_filter<S, E, RC...>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return CMM_OK;
  }
  const int nrp = a.R / 2 + 1;
  const dim3 g((nrp + PAIRS - 1) / PAIRS, (nd + 1) / 2);
  k_pair_filter<S, E, RC...><<<g, PairFilterShape<C, E>::THREADS, smem, st>>>(a, nd);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <typename S>
static int dispatch_pair_F(const TodArgs& a, int nd, cudaStream_t st, bool attr_only) {
  switch (a.logC) {
    case 7: return run_pair_F<S, 16, 16, 8>(a, nd, st, attr_only);
    case 8: return run_pair_F<S, 16, 16, 16>(a, nd, st, attr_only);
    case 9: return run_pair_F<S, 16, 16, 16, 2>(a, nd, st, attr_only);
    case 10: return run_pair_F<S, 16, 16, 16, 4>(a, nd, st, attr_only);
    case 11: return run_pair_F<S, 16, 16, 16, 8>(a, nd, st, attr_only);
    case 12: return run_pair_F<S, 16, 16, 16, 16>(a, nd, st, attr_only);
    default: return fail(CMM_ERR_UNSUPPORTED, "pair path: row length out of range");
  }
}

int launch_flush(const TodArgs& a, int nc, cudaStream_t st);
int launch_flush_maps(const TodArgs& a, int nc, int maps, cudaStream_t st);

template <typename S>
static int apply_pair_s(cmm_op* op, int d0, int nd, int pass) {
  TodArgs a = pair_args(op, d0);
  cudaStream_t st = op->ctx->stream;
  const int nc = op->pt->ncomp;
  if (pass < 0 || pass == 0) {
    TraceRange tr("A: P m + column FFTs (two detectors per sequence)");
    if (nc == 1) CMM_TRY((dispatch_pair_T<1, S>(a, nd, 0, st, false)));
    else CMM_TRY((dispatch_pair_T<3, S>(a, nd, 0, st, false)));
  }
  if (pass < 0 || pass == 1) {
    TraceRange tr("A: row FFTs + N^-1");
    CMM_TRY((dispatch_pair_F<S>(a, nd, st, false)));
  }
  if (pass < 0 || pass == 2) {
    TraceRange tr("A: inverse column FFTs + P^T");
    // one launch bins up to acc32_maps groups of kFlushDets detectors, each group
    // into its own FP32 partial map; one flush then adds them all into FP64
    const int per_launch = op->acc32_maps * kFlushDets;   // even: whole pairs per group
    for (int g0 = 0; g0 < nd; g0 += per_launch) {
      TodArgs b = a;
      const int gn = std::min(per_launch, nd - g0);
      b.d0 = a.d0 + g0;
      b.spec = reinterpret_cast<S*>(a.spec) + (long long)(g0 / 2) * a.N;
      b.flush_dets = kFlushDets;
      b.acc32_map = (long long)op->acc_stride * (a.npix + 1);
      if (nc == 1) CMM_TRY((dispatch_pair_T<1, S>(b, gn, 2, st, false)));
      else CMM_TRY((dispatch_pair_T<3, S>(b, gn, 2, st, false)));
      CMM_TRY(launch_flush_maps(b, nc, (gn + kFlushDets - 1) / kFlushDets, st));
    }
  }
  return CMM_OK;
}

int launch_apply_chunk_pair(cmm_op* op, int d0, int nd, int pass) {
  if (op->prec == CMM_PREC_BF16) return apply_pair_s<__nv_bfloat162>(op, d0, nd, pass);
  return apply_pair_s<float2>(op, d0, nd, pass);
}

template <typename S>
static int prepare_pair_s(cmm_op* op) {
  TodArgs a = pair_args(op, 0);
  if (op->pt->ncomp == 1) CMM_TRY((dispatch_pair_T<1, S>(a, 0, 0, nullptr, true)));
  else CMM_TRY((dispatch_pair_T<3, S>(a, 0, 0, nullptr, true)));
  return dispatch_pair_F<S>(a, 0, nullptr, true);
}

// Twiddle tables of the pair split (w_R, w_C, w_{n_t} low part) and the kernels'
// shared-memory attributes; the split is fixed by n_samp.
int prepare_pair(cmm_op* op) {
  int lr = 0, lc = 0;
  if (!pair_path_sizes(ilog2_ll(op->pt->n_t), op->prec, &lr, &lc)) return CMM_OK;
  op->plogR = lr;
  op->plogC = lc;
  op->pR = 1 << lr;
  op->pC = 1 << lc;
  if (!op->tw_pair) {
    const TwLayout l = tw_layout(op->pR, op->pC);
    std::vector<float2> h(l.total);
    auto fill = [&](int64_t off, int count, double L) {
      for (int e = 0; e < count; ++e) {
        const double ang = -2.0 * M_PI * (double)e / L;
        h[off + e] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
    };
    fill(l.R_off, op->pR, op->pR);
    fill(l.C_off, op->pC, op->pC);
    fill(l.Nlo_off, op->pC, (double)op->pt->n_t);
    void* d = nullptr;
    if (cudaMalloc(&d, sizeof(float2) * l.total) != cudaSuccess) {
      cudaGetLastError();
      return fail(CMM_ERR_OOM, "twiddle table allocation failed");
    }
    op->tw_pair = d;
    CMM_CUDA(cudaMemcpy(op->tw_pair, h.data(), sizeof(float2) * l.total, cudaMemcpyHostToDevice));
  }
  return op->prec == CMM_PREC_BF16 ? prepare_pair_s<__nv_bfloat162>(op) : prepare_pair_s<float2>(op);
}

}  // namespace cmm
