// Shared-memory FFT engines.
//
// * Power-of-two lengths (time-ordered data): Stockham auto-sort radix-2/4/8/16
//   passes; each butterfly is a small DFT held in registers (iterative radix-2
//   decimation in time with constant twiddles), passes ping-pong between two
//   shared-memory buffers.
// * 2/3/5-smooth lengths (map FFTs): the same Stockham schedule with radices
//   2, 3, 4, 5 and table twiddles.
//
// A Stockham pass of radix R over a length-L sequence, after passes whose radices
// multiply to p, takes for butterfly i (0 <= i < L/R, k = i mod p) the inputs
// x_m = in[i + m L/R], multiplies x_m by w_{pR}^{m k}, forms the R-point DFT y and
// writes y_q to out[(i - k) R + k + q p]; after the last pass the output is in
// natural order.  w_L = exp(SIGN * 2 pi i / L), SIGN = -1 forward, +1 inverse.
#pragma once

#include "common.cuh"

namespace cmm {

// cos(2 pi k / 32) for integer k (exact constants of the 32nd roots of unity).
// Written without recursion: a recursive constexpr function is a real call when its
// argument is not a constant expression (rot32's m is a function parameter), so
// the compiler kept it out of line, with a stack frame and double-precision
// conversions, inside every register FFT.
__host__ __device__ constexpr double cos32(int k) {
  k &= 31;
  if (k > 16) k = 32 - k;            // cos is even
  const double sg = k > 8 ? -1.0 : 1.0;
  if (k > 8) k = 16 - k;             // cos(pi - x) = -cos x
  switch (k) {
    case 0: return sg;
    case 1: return sg * 0.98078528040323044913;
    case 2: return sg * 0.92387953251128675613;
    case 3: return sg * 0.83146961230254523708;
    case 4: return sg * 0.70710678118654752440;
    case 5: return sg * 0.55557023301960222474;
    case 6: return sg * 0.38268343236508977173;
    case 7: return sg * 0.19509032201612826785;
    default: return 0.0;
  }
}
__host__ __device__ constexpr double sin32(int k) { return cos32(k - 8); }

// v * exp(SIGN * 2 pi i m / 32), m known at compile time after unrolling
template <typename T, int SIGN>
__device__ __forceinline__ V2<T> rot32(V2<T> v, int m) {
  m &= 31;
  if (m == 0) return v;
  if (m == 16) return V2<T>{-v.x, -v.y};
  if (m == 8) return SIGN < 0 ? V2<T>{v.y, -v.x} : V2<T>{-v.y, v.x};
  if (m == 24) return SIGN < 0 ? V2<T>{-v.y, v.x} : V2<T>{v.y, -v.x};
  const T c = (T)cos32(m);
  const T s = (T)(SIGN * sin32(m));
  return V2<T>{v.x * c - v.y * s, v.x * s + v.y * c};
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// 4-point DFT in place: (x0, x1, x2, x3) <- their transform (w_4 = exp(SIGN i pi / 2))
template <typename T, int SIGN>
__device__ __forceinline__ void dft4_reg(V2<T>& x0, V2<T>& x1, V2<T>& x2, V2<T>& x3) {
  const V2<T> a0 = padd(x0, x2), a1 = psub(x0, x2), a2 = padd(x1, x3);
  const V2<T> d = psub(x1, x3);
  const V2<T> a3 = SIGN < 0 ? V2<T>{d.y, -d.x} : V2<T>{-d.y, d.x};   // d w_4
  x0 = padd(a0, a2);
  x2 = psub(a0, a2);
  x1 = padd(a1, a3);
  x3 = psub(a1, a3);
}

// In-register DFT of size R = 2^LR by bit reversal and LR radix-2 stages
template <typename T, int LR, int SIGN>
__device__ __forceinline__ void dft_reg_radix2(V2<T>* x) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = bitrev(i, LR);
    if (i < j) {
      V2<T> t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < R; half *= 2) {
#pragma unroll
    for (int start = 0; start < R; start += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const V2<T> t = rot32<T, SIGN>(x[start + j + half], j * (32 / (2 * half)));
        const V2<T> u = x[start + j];
        x[start + j] = padd(u, t);
        x[start + j + half] = psub(u, t);
      }
    }
  }
}

// In-register DFT of size R = 2^LR (R <= 32): x_q <- sum_j x_j w_R^{j q}
template <typename T, int LR, int SIGN>
__device__ __forceinline__ void dft_reg(V2<T>* x) {
  if constexpr (LR == 4) {
    // 16 = 4 x 4 (index n1 + 4 n2 -> k2 + 4 k1): 4-point DFTs over n2, twiddles
    // w_16^(n1 k2), 4-point DFTs over n1.  Same transform as four radix-2 stages
    // with fewer live registers (fewer spills in the 64-register kernels).
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) dft4_reg<T, SIGN>(x[n1], x[n1 + 4], x[n1 + 8], x[n1 + 12]);
#pragma unroll
    for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
      for (int k2 = 1; k2 < 4; ++k2) x[n1 + 4 * k2] = rot32<T, SIGN>(x[n1 + 4 * k2], 2 * n1 * k2);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) dft4_reg<T, SIGN>(x[4 * k2], x[4 * k2 + 1], x[4 * k2 + 2], x[4 * k2 + 3]);
    // x[4 k2 + k1] holds X[k2 + 4 k1]: transpose the 4 x 4 index (register renaming)
    V2<T> t[16];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2)
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) t[k2 + 4 * k1] = x[4 * k2 + k1];
#pragma unroll
    for (int e = 0; e < 16; ++e) x[e] = t[e];
  } else {
    dft_reg_radix2<T, LR, SIGN>(x);
  }
}

// One power-of-two Stockham pass of radix 2^LR over `1 << lognseq` sequences of
// length 2^logL; element e of sequence s sits at buf[s * sstride + e * estride].
// tw holds w_L^e = exp(-2 pi i e / L), e < L (forward sign; conjugated for SIGN > 0).
template <typename T, int LR, int SIGN>
__device__ __forceinline__ void pow2_pass(const V2<T>* __restrict__ in, V2<T>* __restrict__ out,
                                          int logL, int lp, int lognseq, int sstride, int estride,
                                          const V2<T>* __restrict__ tw) {
  constexpr int R = 1 << LR;
  const int lognbf = logL - LR;
  const int total = 1 << (lognbf + lognseq);
  const int p = 1 << lp;
  const int twsh = logL - lp - LR;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int s, i;
    if (sstride == 1) {  // sequences interleaved: consecutive threads take consecutive sequences
      s = t & ((1 << lognseq) - 1);
      i = t >> lognseq;
    } else {
      i = t & ((1 << lognbf) - 1);
      s = t >> lognbf;
    }
    const int k = i & (p - 1);
    const V2<T>* src = in + s * sstride;
    V2<T> x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = src[(i + (m << lognbf)) * estride];
    if (k != 0) {
#pragma unroll
      for (int m = 1; m < R; ++m) {
        V2<T> w = tw[(m * k) << twsh];
        if (SIGN > 0) w.y = -w.y;
        x[m] = cmul(x[m], w);
      }
    }
    dft_reg<T, LR, SIGN>(x);
    const int base = ((i - k) << LR) + k;
    V2<T>* dst = out + s * sstride;
#pragma unroll
    for (int m = 0; m < R; ++m) dst[(base + (m << lp)) * estride] = x[m];
  }
}

// Full power-of-two FFT on data in `a` (scratch `b`); returns the buffer that holds
// the result.  Radices are spread evenly over ceil(logL / 4) passes.
template <typename T, int SIGN>
__device__ V2<T>* block_fft_pow2(V2<T>* a, V2<T>* b, int logL, int lognseq, int sstride,
                                 int estride, const V2<T>* __restrict__ tw) {
  int rem = logL, lp = 0;
  const int nst = (logL + 3) / 4;
  for (int st = 0; st < nst; ++st) {
    const int left = nst - st;
    const int lr = (rem + left - 1) / left;
    switch (lr) {
      case 1: pow2_pass<T, 1, SIGN>(a, b, logL, lp, lognseq, sstride, estride, tw); break;
      case 2: pow2_pass<T, 2, SIGN>(a, b, logL, lp, lognseq, sstride, estride, tw); break;
      case 3: pow2_pass<T, 3, SIGN>(a, b, logL, lp, lognseq, sstride, estride, tw); break;
      default: pow2_pass<T, 4, SIGN>(a, b, logL, lp, lognseq, sstride, estride, tw); break;
    }
    __syncthreads();
    V2<T>* t = a;
    a = b;
    b = t;
    lp += lr;
    rem -= lr;
  }
  return a;
}

// ------------------------------------------------------------------ mixed radix
constexpr int kMaxFactors = 24;
struct MixedPlan {
  int L;
  int nrad;
  int rad[kMaxFactors];
  // per stage: magic multipliers of the divisions by L / rad and by p (the product
  // of the earlier radices; 0 where p = 1), see fast_div
  unsigned mnbf[kMaxFactors];
  unsigned mp[kMaxFactors];
};

// t / d for 0 <= t < 2^16 and 2 <= d < 2^16 as __umulhi(t, m), m = floor((2^32 - 1) / d) + 1:
// t m / 2^32 exceeds t / d by less than t / 2^32 < 2^-16 < 1 / d, so its floor is
// floor(t / d).  A magic of 0 stands for d = 1.
__host__ __device__ constexpr unsigned fast_div_magic(unsigned d) { return d > 1 ? 0xFFFFFFFFu / d + 1u : 0u; }
__device__ __forceinline__ int fast_div(int t, unsigned m) { return m ? (int)__umulhi((unsigned)t, m) : t; }

// R-point DFTs for R = 2, 3, 4, 5, y_q = sum_m x_m w^(m q), w = exp(sign 2 pi i / R):
// sums and differences of conjugate pairs, then the real cosines and the sines
// times sign i (the standard short transforms).
template <typename T>
__device__ __forceinline__ V2<T> times_i(V2<T> v, T sg) { return V2<T>{-sg * v.y, sg * v.x}; }

template <typename T, int R>
__device__ __forceinline__ void dft_small(V2<T> (&x)[R], T sg) {
  if constexpr (R == 2) {
    const V2<T> a = x[0], b = x[1];
    x[0] = V2<T>{a.x + b.x, a.y + b.y};
    x[1] = V2<T>{a.x - b.x, a.y - b.y};
  } else if constexpr (R == 3) {
    const T h = (T)0.86602540378443864676;   // sin(2 pi / 3)
    const V2<T> t1{x[1].x + x[2].x, x[1].y + x[2].y};
    const V2<T> t2{x[0].x - (T)0.5 * t1.x, x[0].y - (T)0.5 * t1.y};
    const V2<T> u = times_i(V2<T>{h * (x[1].x - x[2].x), h * (x[1].y - x[2].y)}, sg);
    x[0] = V2<T>{x[0].x + t1.x, x[0].y + t1.y};
    x[1] = V2<T>{t2.x + u.x, t2.y + u.y};
    x[2] = V2<T>{t2.x - u.x, t2.y - u.y};
  } else if constexpr (R == 4) {
    const V2<T> a{x[0].x + x[2].x, x[0].y + x[2].y}, b{x[1].x + x[3].x, x[1].y + x[3].y};
    const V2<T> c{x[0].x - x[2].x, x[0].y - x[2].y};
    const V2<T> d = times_i(V2<T>{x[1].x - x[3].x, x[1].y - x[3].y}, sg);
    x[0] = V2<T>{a.x + b.x, a.y + b.y};
    x[1] = V2<T>{c.x + d.x, c.y + d.y};
    x[2] = V2<T>{a.x - b.x, a.y - b.y};
    x[3] = V2<T>{c.x - d.x, c.y - d.y};
  } else {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;   // cos(2 pi / 5), cos(4 pi / 5)
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;    // sin(2 pi / 5), sin(4 pi / 5)
    const V2<T> a1{x[1].x + x[4].x, x[1].y + x[4].y}, a2{x[2].x + x[3].x, x[2].y + x[3].y};
    const V2<T> b1{x[1].x - x[4].x, x[1].y - x[4].y}, b2{x[2].x - x[3].x, x[2].y - x[3].y};
    const V2<T> t1{x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y};
    const V2<T> t2{x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y};
    const V2<T> u1 = times_i(V2<T>{s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y}, sg);
    const V2<T> u2 = times_i(V2<T>{s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y}, sg);
    x[0] = V2<T>{x[0].x + a1.x + a2.x, x[0].y + a1.y + a2.y};
    x[1] = V2<T>{t1.x + u1.x, t1.y + u1.y};
    x[4] = V2<T>{t1.x - u1.x, t1.y - u1.y};
    x[2] = V2<T>{t2.x + u2.x, t2.y + u2.y};
    x[3] = V2<T>{t2.x - u2.x, t2.y - u2.y};
  }
}

// cos and sin of 2 pi j / R for the radices of the map FFT (R in {2, 3, 4, 5})
template <int R> struct RootsR;
template <> struct RootsR<2> {
  static __device__ __forceinline__ double c(int j) { return j ? -1.0 : 1.0; }
  static __device__ __forceinline__ double s(int) { return 0.0; }
};
template <> struct RootsR<3> {
  static __device__ __forceinline__ double c(int j) { return j ? -0.5 : 1.0; }
  static __device__ __forceinline__ double s(int j) {
    return j == 0 ? 0.0 : (j == 1 ? 0.86602540378443864676 : -0.86602540378443864676);
  }
};
template <> struct RootsR<4> {
  static __device__ __forceinline__ double c(int j) { return j == 0 ? 1.0 : (j == 2 ? -1.0 : 0.0); }
  static __device__ __forceinline__ double s(int j) { return j == 1 ? 1.0 : (j == 3 ? -1.0 : 0.0); }
};
template <> struct RootsR<5> {
  static __device__ __forceinline__ double c(int j) {
    return j == 0 ? 1.0 : ((j == 1 || j == 4) ? 0.30901699437494742410 : -0.80901699437494742410);
  }
  static __device__ __forceinline__ double s(int j) {
    return j == 0 ? 0.0
                  : (j == 1 ? 0.95105651629515357212
                            : (j == 2 ? 0.58778525229247312917 : (j == 3 ? -0.58778525229247312917 : -0.95105651629515357212)));
  }
};

// One mixed-radix Stockham pass of compile-time radix R; tw holds w_L^e, e < L.
// The R-point DFT is dft_small, only the inter-stage twiddles come from the table;
// the butterfly and sequence indices come from multiplicative divisions (mnbf, mp:
// the plan's magics of this stage; ns: of nseq).
template <typename T, int R>
__device__ __forceinline__ void mixed_pass_r(const V2<T>* __restrict__ in, V2<T>* __restrict__ out, int L, int p,
                                             int nseq, int sstride, int estride, const V2<T>* __restrict__ tw,
                                             int sign, unsigned mnbf, unsigned mp, unsigned ns) {
  const int nbf = L / R;
  const int total = nbf * nseq;
  const int step = L / (p * R);
  const T sg = (T)sign;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int s, i;
    if (sstride == 1) {
      s = t - fast_div(t, ns) * nseq;
      i = fast_div(t, ns);
    } else {
      s = fast_div(t, mnbf);
      i = t - s * nbf;
    }
    const int k = i - fast_div(i, mp) * p;
    const V2<T>* src = in + s * sstride;
    V2<T> x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const V2<T> v = src[(i + m * nbf) * estride];
      if (m == 0 || k == 0) {
        x[m] = v;
      } else {
        V2<T> w = tw[m * k * step];
        if (sign > 0) w.y = -w.y;
        x[m] = cmul(v, w);
      }
    }
    dft_small<T, R>(x, sg);
    const int base = (i - k) * R + k;
    V2<T>* dst = out + s * sstride;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[(base + q * p) * estride] = x[q];
  }
}

// One mixed-radix Stockham pass (radix R in {2,3,4,5}).
template <typename T>
__device__ __forceinline__ void mixed_pass(const V2<T>* __restrict__ in, V2<T>* __restrict__ out,
                                           int L, int R, int p, int nseq, int sstride, int estride,
                                           const V2<T>* __restrict__ tw, int sign, unsigned mnbf, unsigned mp,
                                           unsigned ns) {
  switch (R) {
    case 2: mixed_pass_r<T, 2>(in, out, L, p, nseq, sstride, estride, tw, sign, mnbf, mp, ns); break;
    case 3: mixed_pass_r<T, 3>(in, out, L, p, nseq, sstride, estride, tw, sign, mnbf, mp, ns); break;
    case 4: mixed_pass_r<T, 4>(in, out, L, p, nseq, sstride, estride, tw, sign, mnbf, mp, ns); break;
    default: mixed_pass_r<T, 5>(in, out, L, p, nseq, sstride, estride, tw, sign, mnbf, mp, ns); break;
  }
}

template <typename T>
__device__ V2<T>* block_fft_mixed(V2<T>* a, V2<T>* b, const MixedPlan& plan, int nseq, int sstride,
                                  int estride, const V2<T>* __restrict__ tw, int sign) {
  int p = 1;
  const unsigned ns = fast_div_magic((unsigned)nseq);
  for (int st = 0; st < plan.nrad; ++st) {
    const int R = plan.rad[st];
    mixed_pass<T>(a, b, plan.L, R, p, nseq, sstride, estride, tw, sign, plan.mnbf[st], plan.mp[st], ns);
    __syncthreads();
    V2<T>* t = a;
    a = b;
    b = t;
    p *= R;
  }
  return a;
}

}  // namespace cmm
