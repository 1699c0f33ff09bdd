// Register-resident Stockham FFT used by the fast-path time-ordered-data kernels.
//
// A thread owns E elements of one length-L sequence (L = product of the stage
// radices, every radix divides E): on entry x[e] holds the element at position
// i + e (L/E), 0 <= i < L/E, and on exit x[e] holds the transform at that same
// position.  Every stage's butterflies read their inputs from those natural
// positions (butterfly ib = i + (L/E) u, input m at ib + m L/R is register
// u + m E/R), so only the outputs of non-final stages go through shared memory:
// a sequence of S stages costs S - 1 exchanges, each one store and one load per
// element, instead of a load and a store per stage.  Twiddles w_{PR}^{mk} come
// from a table of w_L^e, e < L (forward sign, conjugated for SIGN > 0): the powers
// of two are loaded and the other exponents formed as products.
#pragma once

#include "common.cuh"
#include "fft.cuh"

// Stage twiddles w^m, m < R: 1 (default) by recurrence from one loaded w (two live
// registers, relative error growing to ~R ulp); 0 from the loaded w, w^2, w^4, w^8
// and products (at most three roundings, more live registers).
#ifndef CMM_TW_MODE
#define CMM_TW_MODE 1
#endif

namespace cmm {

constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v / 2); }

template <int... Rs> struct RadProd;
template <> struct RadProd<> { static constexpr int value = 1; };
template <int R, int... Rs> struct RadProd<R, Rs...> { static constexpr int value = R * RadProd<Rs...>::value; };

template <int SIGN, int E, int L, int P, typename Addr, int R, int... REST>
__device__ __forceinline__ void rfft_stages(float2 (&x)[E], const int i, const float2* __restrict__ tw,
                                            const Addr& ad) {
  static_assert(E % R == 0, "every radix must divide the elements per thread");
  constexpr int NB = E / R;
  constexpr bool LAST = sizeof...(REST) == 0;
  if constexpr (!LAST) __syncthreads();
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int ib = i + (L / E) * u;
    const int k = ib & (P - 1);
    float2 z[R];
#pragma unroll
    for (int m = 0; m < R; ++m) z[m] = x[u + m * NB];
    if constexpr (P > 1) {
      // one or four L1 loads per butterfly instead of R - 1, the rest on the FP32 pipe
      const int b = k * (L / (P * R));
#if CMM_TW_MODE == 1
      // w^m by recurrence from w (two live twiddles)
      float2 w1 = __ldg(tw + b);
      if (SIGN > 0) w1.y = -w1.y;
      float2 wm = w1;
#pragma unroll
      for (int m = 1; m < R; ++m) {
        z[m] = cmul(z[m], wm);
        if (m + 1 < R) wm = cmul(wm, w1);
      }
#else
      float2 wp[R];
#pragma unroll
      for (int m = 1; m < R; m *= 2) {
        wp[m] = __ldg(tw + m * b);
        if (SIGN > 0) wp[m].y = -wp[m].y;
      }
#pragma unroll
      for (int m = 3; m < R; ++m)
        if (m & (m - 1)) wp[m] = cmul(wp[m & (m - 1)], wp[m & -m]);
#pragma unroll
      for (int m = 1; m < R; ++m) z[m] = cmul(z[m], wp[m]);
#endif
    }
    dft_reg<float, clog2(R), SIGN>(z);
    if constexpr (LAST) {
#pragma unroll
      for (int q = 0; q < R; ++q) x[u + q * NB] = z[q];
    } else {
      // outputs at (ib - k) R + k + q P: one base index, constant offsets
      const int b = ad.base((ib - k) * R + k);
#pragma unroll
      for (int q = 0; q < R; ++q) ad.st_at(b, q * P, z[q]);
    }
  }
  if constexpr (!LAST) {
    __syncthreads();
    const int b = ad.base(i);
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = ad.ld_at(b, e * (L / E));
    rfft_stages<SIGN, E, L, P * R, Addr, REST...>(x, i, tw, ad);
  }
}

template <int SIGN, int E, int... RS, typename Addr>
__device__ __forceinline__ void rfft(float2 (&x)[E], const int i, const float2* __restrict__ tw, const Addr& ad) {
  rfft_stages<SIGN, E, RadProd<RS...>::value, 1, Addr, RS...>(x, i, tw, ad);
}

// One contiguous row (pass F), padded by one element every 2^PS positions.
// st_at / ld_at address position pos + o from base(pos) with a constant offset o;
// exact whenever the low PS bits of pos and o do not carry into each other, which
// holds for every access of the register FFT (either pos is a multiple of 2^PS
// and o < 2^PS, or o is a multiple of 2^PS, or o is a multiple of a power of two
// p < 2^PS and pos < p).
template <int PS>
struct RowAddr {
  float2* buf;
  __device__ __forceinline__ int idx(int pos) const { return pos + (pos >> PS); }
  __device__ __forceinline__ void st(int pos, float2 v) const { buf[idx(pos)] = v; }
  __device__ __forceinline__ float2 ld(int pos) const { return buf[idx(pos)]; }
  __device__ __forceinline__ int base(int pos) const { return idx(pos); }
  __device__ __forceinline__ void st_at(int b, int o, float2 v) const { buf[b + o + (o >> PS)] = v; }
  __device__ __forceinline__ float2 ld_at(int b, int o) const { return buf[b + o + (o >> PS)]; }
};

}  // namespace cmm
