// U-Net of the learned preconditioner correction: BF16 weights and activations,
// FP32 accumulation and gradients, Adam in FP32 master weights.
//
// Architecture (widths w_1..w_L, 3 input and 3 output channels): encoder level l
// = two 3x3 convolutions with ReLU, 2x2 average pooling between levels; decoder
// level l (from L-1 down to 1) = 2x2 stride-2 transposed convolution, channel
// concatenation [up, skip], two 3x3 convolutions with ReLU; output = 1x1
// convolution.  Parameters are one flat FP32 vector, per layer weights then
// biases (conv weights [cout][cin][k][k], transposed-conv weights [cin][cout][2][2]).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <string>
#include <vector>

#include "common.cuh"
#include "map_kernels.cuh"

namespace cmm {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ bool stopped(const int* done) { return done && *done; }

// ------------------------------------------------------------------ 3x3 convolution
// out[b][o][y][x] = sum_i sum_{dy,dx} Wv(o,i,dy,dx) in[b][i][y+dy-1][x+dx-1] (+ bias[o]),
// zero padded.  Forward: Wv = W[o][i][dy][dx].  FLIP (gradient w.r.t. the input of a
// forward convolution with weights W[co][ci]): o = ci, i = co, Wv = W[i][o][2-dy][2-dx].
// A CTA computes a 16x16 pixel tile for 16 output channels; input channels are
// staged 16 at a time through shared memory.
template <typename TIN, typename TOUT, bool RELU, bool FLIP>
__global__ void __launch_bounds__(256) k_conv3(const TIN* __restrict__ in, const bf16* __restrict__ w,
                                               const float* __restrict__ bias, TOUT* __restrict__ out,
                                               int Cin, int Cout, int H, int W, const int* done) {
  if (stopped(done)) return;
  __shared__ float s_in[16][18][19];
  __shared__ float s_w[16][16][9];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int tiles_x = (W + 15) / 16;
  const int x0 = (blockIdx.x % tiles_x) * 16, y0 = (blockIdx.x / tiles_x) * 16;
  const int o0 = blockIdx.y * 16;
  const int b = blockIdx.z;
  const int ox = x0 + tx, oy = y0 + ty;
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.f;
  // weight tensor dims of the forward layer: FLIP reads W[i][o] with i < Cin(this) = Cout(fwd)
  const int Wo = FLIP ? Cin : Cout;   // forward output channels
  const int Wi = FLIP ? Cout : Cin;   // forward input channels
  for (int i0 = 0; i0 < Cin; i0 += 16) {
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * 18 * 18; t += 256) {
      const int ci = t / 324, r = t % 324, yy = r / 18, xx = r % 18;
      const int gi = i0 + ci, gy = y0 + yy - 1, gx = x0 + xx - 1;
      float v = 0.f;
      if (gi < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = ldf(in + (((long long)b * Cin + gi) * H + gy) * W + gx);
      s_in[ci][yy][xx] = v;
    }
    for (int t = threadIdx.x; t < 16 * 16 * 9; t += 256) {
      const int oo = t / 144, r = t % 144, ii = r / 9, k = r % 9;
      const int go = o0 + oo, gi = i0 + ii;
      float v = 0.f;
      if (go < Cout && gi < Cin) {
        if (!FLIP) v = __bfloat162float(w[((long long)go * Wi + gi) * 9 + k]);
        else v = __bfloat162float(w[((long long)gi * Wi + go) * 9 + (8 - k)]);
      }
      s_w[oo][ii][k] = v;
    }
    (void)Wo;
    __syncthreads();
    const int nci = min(16, Cin - i0);
    for (int ci = 0; ci < nci; ++ci) {
      float v[9];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) v[dy * 3 + dx] = s_in[ci][ty + dy][tx + dx];
#pragma unroll
      for (int oo = 0; oo < 16; ++oo) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) s = fmaf(s_w[oo][ci][k], v[k], s);
        acc[oo] += s;
      }
    }
  }
  if (ox >= W || oy >= H) return;
#pragma unroll
  for (int oo = 0; oo < 16; ++oo) {
    const int go = o0 + oo;
    if (go >= Cout) break;
    float r = acc[oo] + (bias ? bias[go] : 0.f);
    if (RELU) r = fmaxf(r, 0.f);
    stf(out + (((long long)b * Cout + go) * H + oy) * W + ox, r);
  }
}

// ------------------------------------------------------------------ tensor-core 3x3 convolution
// The same convolutions as implicit GEMMs on the tensor cores: BF16 operands, FP32
// accumulation, warp-level mma.sync m16n8k16 (row-major A, column-major B).
// Fragment layout of one m16n8k16 (g = lane / 4, q = lane % 4; each .b32 register
// holds two BF16, the lower index in the low half):
//   A (16 x 16, M x K): a0 (row g, k 2q..2q+1), a1 (row g+8, same k),
//                       a2 (row g, k 2q+8..2q+9), a3 (row g+8, k 2q+8..2q+9)
//   B (16 x 8, K x N):  b0 (k 2q..2q+1, col g), b1 (k 2q+8..2q+9, col g)
//   C (16 x 8, FP32):   c0, c1 (row g, cols 2q, 2q+1), c2, c3 (row g+8, same cols)
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t lds32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Channel stride (BF16 elements) of the staged tiles: 24 (= 12 words) puts the eight
// row or column groups of a fragment load on distinct banks.
constexpr int kCP = 24;

template <typename T> __device__ __forceinline__ void st2(T* p, float a, float b);
template <> __device__ __forceinline__ void st2(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
template <> __device__ __forceinline__ void st2(bf16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}

// out = conv3(in) as k_conv3 (same FLIP convention).  GEMM: M = output channels
// (MT x 16 per CTA), N = the CTA's pixel tile (256 / TW rows x TW columns, eight
// n8 tiles per warp), K = input channels (16 per chunk) x 9 taps.  Each chunk
// stages the input tile with its one-pixel halo as [y][x][channel] and the weights
// as [tap][o][i] in BF16; every tap is then one A fragment per m16 tile and one B
// fragment per n8 tile read straight from the staged tile shifted by (dy, dx).
template <typename TIN, typename TOUT, bool RELU, bool FLIP, int MT, int TW>
__global__ void __launch_bounds__(128) k_conv3_mma(const TIN* __restrict__ in, const bf16* __restrict__ w,
                                                   const float* __restrict__ bias, TOUT* __restrict__ out, int Cin,
                                                   int Cout, int H, int W, const int* done, int ks = 1,
                                                   float* __restrict__ part = nullptr) {
  if (stopped(done)) return;
  constexpr int TH = 256 / TW;   // tile rows
  constexpr int RPW = TH / 4;    // rows per warp
  constexpr int NPR = TW / 8;    // n8 tiles per row
  constexpr int NT = RPW * NPR;  // n8 tiles per warp (8)
  constexpr int MO = MT * 16;    // output channels per CTA
  constexpr int SX = TW + 2;
  __shared__ __align__(16) bf16 s_in[(TH + 2) * SX * kCP];
  __shared__ __align__(16) bf16 s_w[9 * MO * kCP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int tiles_x = (W + TW - 1) / TW;
  const int x0 = (blockIdx.x % tiles_x) * TW, y0 = (blockIdx.x / tiles_x) * TH;
  const int o0 = blockIdx.y * MO;
  const int b = blockIdx.z / ks;
  // split K: slice blockIdx.z % ks of the input channels, in whole 16-channel chunks
  const int cps = ((Cin + 15) / 16 + ks - 1) / ks;
  const int c_lo = (blockIdx.z % ks) * cps * 16, c_hi = min(Cin, c_lo + cps * 16);
  const int Wi = FLIP ? Cout : Cin;   // input channels of the forward layer's weight tensor
  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[m][n][c] = 0.f;
  for (int i0 = c_lo; i0 < c_hi; i0 += 16) {
    __syncthreads();
    // unrolled so that a thread has several loads in flight: with few CTAs (one map)
    // the staging is latency-bound
#pragma unroll 8
    for (int t = threadIdx.x; t < 16 * (TH + 2) * SX; t += 128) {
      const int xx = t % SX, r = t / SX, yy = r % (TH + 2), ci = r / (TH + 2);
      const int gi = i0 + ci, gy = y0 + yy - 1, gx = x0 + xx - 1;
      float v = 0.f;
      if (gi < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = ldf(in + (((long long)b * Cin + gi) * H + gy) * W + gx);
      s_in[(yy * SX + xx) * kCP + ci] = __float2bfloat16_rn(v);
    }
#pragma unroll 8
    for (int t = threadIdx.x; t < 9 * MO * 16; t += 128) {
      const int k = t % 9, r = t / 9, ii = r % 16, oo = r / 16;
      const int go = o0 + oo, gi = i0 + ii;
      bf16 v = __float2bfloat16_rn(0.f);
      if (go < Cout && gi < Cin)
        v = FLIP ? w[((long long)gi * Wi + go) * 9 + (8 - k)] : w[((long long)go * Wi + gi) * 9 + k];
      s_w[(k * MO + oo) * kCP + ii] = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < 9; ++k) {
      const int dy = k / 3, dx = k - 3 * dy;
      uint32_t a[MT][4];
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        const bf16* pa = s_w + (k * MO + m * 16 + g) * kCP + 2 * q;
        a[m][0] = lds32(pa);
        a[m][1] = lds32(pa + 8 * kCP);
        a[m][2] = lds32(pa + 8);
        a[m][3] = lds32(pa + 8 * kCP + 8);
      }
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const int r = warp * RPW + n / NPR, xb = (n % NPR) * 8;
        const bf16* pb = s_in + ((r + dy) * SX + xb + g + dx) * kCP + 2 * q;
        const uint32_t b0 = lds32(pb), b1 = lds32(pb + 8);
#pragma unroll
        for (int m = 0; m < MT; ++m) mma_bf16_16816(acc[m][n], a[m], b0, b1);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int r = warp * RPW + n / NPR, xb = (n % NPR) * 8;
      const int y = y0 + r, x = x0 + xb + 2 * q;
      if (y >= H || x >= W) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int o = o0 + m * 16 + g + 8 * h;
        if (o >= Cout) continue;
        if (part) {
          // partial sum of this K slice; bias and activation follow in k_bias_act
          float* dst = part + (((long long)b * Cout + o) * H + y) * W + x;
          atomicAdd(dst, acc[m][n][2 * h]);
          if (x + 1 < W) atomicAdd(dst + 1, acc[m][n][2 * h + 1]);
          continue;
        }
        const float bo = bias ? bias[o] : 0.f;
        float v0 = acc[m][n][2 * h] + bo, v1 = acc[m][n][2 * h + 1] + bo;
        if (RELU) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        TOUT* dst = out + (((long long)b * Cout + o) * H + y) * W + x;
        if (x + 1 < W) st2(dst, v0, v1);
        else stf(dst, v0);
      }
    }
}

// Weight and bias gradients of a 3x3 convolution on the tensor cores:
// gw[o][i][tap] += sum_p g[o][p] in[i][p + tap offset].  GEMM per tap: M = 16
// output channels, N = 16 input channels (two n8 tiles), K = pixels, 16 at a time
// along a row.  The CTA walks its slice of (image, row) rows; each row stages g
// (BF16, [o][x]) and the three input rows y-1..y+1 twice ([dy][i][x], once shifted
// by one pixel so that every tap's pixel pairs are 32-bit aligned); warp w
// accumulates the taps w, w + 4, w + 8.  Partial sums go to the zeroed FP32
// gradient with atomics.
__global__ void __launch_bounds__(128) k_conv3_wgrad_mma(const bf16* __restrict__ in, const float* __restrict__ g,
                                                         float* __restrict__ gw, float* __restrict__ gb, int Cin,
                                                         int Cout, int H, int W, int B, int rows_per_cta) {
  constexpr int WMAX = 64;
  constexpr int SG = WMAX + 8;        // row stride (BF16) of the staged g rows
  constexpr int SI = WMAX + 8;        // row stride of the staged input rows
  __shared__ __align__(16) bf16 s_g[16 * SG];
  __shared__ __align__(16) bf16 s_a[3 * 16 * SI];   // in[x - 1] at index x (halo at 0)
  __shared__ __align__(16) bf16 s_b[3 * 16 * SI];   // in[x] at index x
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gq = lane >> 2, q = lane & 3;
  const int o0 = blockIdx.x * 16, i0 = blockIdx.y * 16;
  const int Wp = (W + 15) & ~15;      // K extent of a row, zero padded to whole chunks
  const int ntap = warp == 0 ? 3 : 2;
  float acc[3][2][4];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[j][n][c] = 0.f;
  float accb = 0.f;
  const int r0 = blockIdx.z * rows_per_cta;
  const int r1 = min(B * H, r0 + rows_per_cta);
  for (int row = r0; row < r1; ++row) {
    const int b = row / H, y = row % H;
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * Wp; t += 128) {
      const int oo = t / Wp, x = t % Wp;
      float v = 0.f;
      if (o0 + oo < Cout && x < W) v = g[(((long long)b * Cout + o0 + oo) * H + y) * W + x];
      s_g[oo * SG + x] = __float2bfloat16_rn(v);
    }
    for (int t = threadIdx.x; t < 3 * 16 * (Wp + 2); t += 128) {
      const int xs = t % (Wp + 2), r = t / (Wp + 2), ii = r % 16, dy = r / 16;
      const int yy = y + dy - 1, x = xs - 1;
      bf16 v = __float2bfloat16_rn(0.f);
      if (i0 + ii < Cin && yy >= 0 && yy < H && x >= 0 && x < W) v = in[(((long long)b * Cin + i0 + ii) * H + yy) * W + x];
      s_a[(dy * 16 + ii) * SI + xs] = v;
      if (xs < Wp) {
        bf16 u = __float2bfloat16_rn(0.f);
        if (i0 + ii < Cin && yy >= 0 && yy < H && xs < W) u = in[(((long long)b * Cin + i0 + ii) * H + yy) * W + xs];
        s_b[(dy * 16 + ii) * SI + xs] = u;
      }
    }
    __syncthreads();
    if (threadIdx.x < 16 && o0 + (int)threadIdx.x < Cout) {
      const float* gr = g + (((long long)b * Cout + o0 + threadIdx.x) * H + y) * W;
      for (int x = 0; x < W; ++x) accb += gr[x];
    }
    for (int c0 = 0; c0 < Wp; c0 += 16) {
      uint32_t a[4];
      const bf16* pa = s_g + gq * SG + c0 + 2 * q;
      a[0] = lds32(pa);
      a[1] = lds32(pa + 8 * SG);
      a[2] = lds32(pa + 8);
      a[3] = lds32(pa + 8 * SG + 8);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (j >= ntap) break;
        const int k = warp + 4 * j;
        const int dy = k / 3, dx = k - 3 * dy;
        // pixel p needs in[p + dx - 1]: s_a[p + dx] for dx = 0, 2 and s_b[p] for dx = 1
        const bf16* base = (dx == 1 ? s_b + c0 : s_a + c0 + dx) + (dy * 16) * SI + 2 * q;
#pragma unroll
        for (int n = 0; n < 2; ++n) {
          const bf16* pb = base + (n * 8 + gq) * SI;
          mma_bf16_16816(acc[j][n], a, lds32(pb), lds32(pb + 8));
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (j >= ntap) break;
    const int k = warp + 4 * j;
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int o = o0 + gq + 8 * (c >> 1), i = i0 + n * 8 + 2 * q + (c & 1);
        if (o < Cout && i < Cin) atomicAdd(gw + ((long long)o * Cin + i) * 9 + k, acc[j][n][c]);
      }
  }
  if (threadIdx.x < 16 && blockIdx.y == 0 && o0 + (int)threadIdx.x < Cout) atomicAdd(gb + o0 + threadIdx.x, accb);
}

// Per-pixel channel GEMMs on the tensor cores: the 2x2 stride-2 transposed
// convolution (TAPS = 4: out[b][o][2y+dy][2x+dx] = sum_i in[b][i][y][x] W[i][o][dy][dx]
// + bias[o], BF16 out) and the 1x1 output convolution (TAPS = 1: out[b][o][p] =
// sum_i W[o][i] in[b][i][p] + bias[o], FP32 out).  GEMM per tap: M = output
// channels (MT x 16 per CTA), N = 128 pixels (four warps x four n8 tiles), K = input
// channels, 16 per chunk; the pixel tile is staged once per chunk as [pixel][channel]
// and reused by every tap.
template <int TAPS, typename TOUT, int MT>
__global__ void __launch_bounds__(128) k_pointwise_mma(const bf16* __restrict__ in, const bf16* __restrict__ w,
                                                       const float* __restrict__ bias, TOUT* __restrict__ out,
                                                       int Cin, int Cout, int H, int W, const int* done, int ks = 1,
                                                       float* __restrict__ part = nullptr) {
  if (stopped(done)) return;
  constexpr int NP = 128;       // pixels per CTA
  constexpr int MO = MT * 16;
  __shared__ __align__(16) bf16 s_in[NP * kCP];
  __shared__ __align__(16) bf16 s_w[TAPS * MO * kCP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int HW = H * W;
  const int p0 = blockIdx.x * NP;
  const int o0 = blockIdx.y * MO;
  const int b = blockIdx.z / ks;
  const int cps = ((Cin + 15) / 16 + ks - 1) / ks;
  const int c_lo = (blockIdx.z % ks) * cps * 16, c_hi = min(Cin, c_lo + cps * 16);
  float acc[TAPS][MT][4][4];
#pragma unroll
  for (int t = 0; t < TAPS; ++t)
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[t][m][n][c] = 0.f;
  for (int i0 = c_lo; i0 < c_hi; i0 += 16) {
    __syncthreads();
#pragma unroll 8
    for (int e = threadIdx.x; e < 16 * NP; e += 128) {
      const int px = e % NP, ci = e / NP;
      const int gi = i0 + ci, gp = p0 + px;
      s_in[px * kCP + ci] = (gi < Cin && gp < HW) ? in[((long long)b * Cin + gi) * HW + gp] : __float2bfloat16_rn(0.f);
    }
#pragma unroll 8
    for (int e = threadIdx.x; e < TAPS * MO * 16; e += 128) {
      const int ii = e % 16, r = e / 16, oo = r % MO, t = r / MO;
      const int go = o0 + oo, gi = i0 + ii;
      bf16 v = __float2bfloat16_rn(0.f);
      if (go < Cout && gi < Cin) v = TAPS == 4 ? w[((long long)gi * Cout + go) * 4 + t] : w[(long long)go * Cin + gi];
      s_w[(t * MO + oo) * kCP + ii] = v;
    }
    __syncthreads();
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const bf16* pb = s_in + (warp * 32 + n * 8 + g) * kCP + 2 * q;
      const uint32_t b0 = lds32(pb), b1 = lds32(pb + 8);
#pragma unroll
      for (int t = 0; t < TAPS; ++t)
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const bf16* pa = s_w + (t * MO + m * 16 + g) * kCP + 2 * q;
          uint32_t a[4] = {lds32(pa), lds32(pa + 8 * kCP), lds32(pa + 8), lds32(pa + 8 * kCP + 8)};
          mma_bf16_16816(acc[t][m][n], a, b0, b1);
        }
    }
  }
#pragma unroll
  for (int t = 0; t < TAPS; ++t)
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int o = o0 + m * 16 + g + 8 * (c >> 1);
          const int p = p0 + warp * 32 + n * 8 + 2 * q + (c & 1);
          if (o >= Cout || p >= HW) continue;
          long long idx;
          if (TAPS == 4) {
            const int y = p / W, x = p - (p / W) * W;
            const int Y = 2 * y + (t >> 1), X = 2 * x + (t & 1);
            idx = (((long long)b * Cout + o) * 2 * H + Y) * 2 * W + X;
          } else {
            idx = ((long long)b * Cout + o) * HW + p;
          }
          if (part) atomicAdd(part + idx, acc[t][m][n][c]);
          else stf(out + idx, acc[t][m][n][c] + bias[o]);
        }
}

// out = act(part + bias[o]) over [B][Cout][hw] and part reset to zero: the end of a
// split-K convolution, whose K slices added their partial sums into part.
template <typename TOUT, bool RELU>
__global__ void k_bias_act(float* __restrict__ part, const float* __restrict__ bias, TOUT* __restrict__ out,
                           int Cout, long long hw, long long n, const int* done) {
  if (stopped(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int o = (int)((i / hw) % Cout);
    float v = part[i] + (bias ? bias[o] : 0.f);
    if (RELU) v = fmaxf(v, 0.f);
    stf(out + i, v);
    part[i] = 0.f;
  }
}

// Weight and bias gradients of a 3x3 convolution: gw[o][i][dy][dx] +=
// sum_{b,y,x} g[b][o][y][x] in[b][i][y+dy-1][x+dx-1], gb[o] += sum g[b][o].
// CTA: 16 output x 16 input channels, one image row at a time over its slice of the
// (b, y) rows; partial sums are added to the zeroed FP32 gradient with atomics.
__global__ void __launch_bounds__(256) k_conv3_wgrad(const bf16* __restrict__ in, const float* __restrict__ g,
                                                     float* __restrict__ gw, float* __restrict__ gb, int Cin,
                                                     int Cout, int H, int W, int B, int rows_per_cta) {
  __shared__ float s_g[16][64];
  __shared__ float s_in[16][3][66];
  const int ol = threadIdx.x >> 4, il = threadIdx.x & 15;
  const int o0 = blockIdx.x * 16, i0 = blockIdx.y * 16;
  const int go = o0 + ol, gi = i0 + il;
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  float accb = 0.f;
  const int r0 = blockIdx.z * rows_per_cta;
  const int r1 = min(B * H, r0 + rows_per_cta);
  for (int row = r0; row < r1; ++row) {
    const int b = row / H, y = row % H;
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * W; t += 256) {
      const int oo = t / W, x = t % W;
      s_g[oo][x] = (o0 + oo < Cout) ? g[(((long long)b * Cout + o0 + oo) * H + y) * W + x] : 0.f;
    }
    for (int t = threadIdx.x; t < 16 * 3 * (W + 2); t += 256) {
      const int ii = t / (3 * (W + 2)), r = t % (3 * (W + 2)), dy = r / (W + 2), xx = r % (W + 2);
      const int yy = y + dy - 1, gx = xx - 1;
      float v = 0.f;
      if (i0 + ii < Cin && yy >= 0 && yy < H && gx >= 0 && gx < W)
        v = __bfloat162float(in[(((long long)b * Cin + i0 + ii) * H + yy) * W + gx]);
      s_in[ii][dy][xx] = v;
    }
    __syncthreads();
    for (int x = 0; x < W; ++x) {
      const float gv = s_g[ol][x];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) acc[dy * 3 + dx] = fmaf(gv, s_in[il][dy][x + dx], acc[dy * 3 + dx]);
      if (il == 0) accb += gv;
    }
  }
  if (go < Cout && gi < Cin) {
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(gw + ((long long)go * Cin + gi) * 9 + k, acc[k]);
  }
  if (il == 0 && blockIdx.y == 0 && go < Cout) atomicAdd(gb + go, accb);
}

// ------------------------------------------------------------------ 2x2 transposed convolution
// out[b][o][2y+dy][2x+dx] = sum_i in[b][i][y][x] W[i][o][dy][dx] + bias[o]
__global__ void k_tconv_fwd(const bf16* __restrict__ in, const bf16* __restrict__ w, const float* __restrict__ bias,
                            bf16* __restrict__ out, int Cin, int Cout, int H, int W, int B, const int* done) {
  if (stopped(done)) return;
  const long long n = (long long)B * Cout * 4 * H * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int X = t % (2 * W);
    const int Y = (t / (2 * W)) % (2 * H);
    const int o = (t / (4LL * H * W)) % Cout;
    const int b = t / (4LL * H * W * Cout);
    const int y = Y >> 1, x = X >> 1, k = (Y & 1) * 2 + (X & 1);
    float s = bias[o];
    for (int i = 0; i < Cin; ++i)
      s = fmaf(__bfloat162float(in[(((long long)b * Cin + i) * H + y) * W + x]),
               __bfloat162float(w[((long long)i * Cout + o) * 4 + k]), s);
    out[t] = __float2bfloat16_rn(s);
  }
}

// gin[b][i][y][x] = sum_o sum_k g[b][o][2y+dy][2x+dx] W[i][o][k]
__global__ void k_tconv_bwd_data(const float* __restrict__ g, const bf16* __restrict__ w, float* __restrict__ gin,
                                 int Cin, int Cout, int H, int W, int B) {
  const long long n = (long long)B * Cin * H * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int x = t % W;
    const int y = (t / W) % H;
    const int i = (t / ((long long)H * W)) % Cin;
    const int b = t / ((long long)H * W * Cin);
    float s = 0.f;
    for (int o = 0; o < Cout; ++o) {
      const float* gp = g + (((long long)b * Cout + o) * 2 * H + 2 * y) * 2 * W + 2 * x;
      const bf16* wp = w + ((long long)i * Cout + o) * 4;
      s = fmaf(gp[0], __bfloat162float(wp[0]), s);
      s = fmaf(gp[1], __bfloat162float(wp[1]), s);
      s = fmaf(gp[2 * W], __bfloat162float(wp[2]), s);
      s = fmaf(gp[2 * W + 1], __bfloat162float(wp[3]), s);
    }
    gin[t] = s;
  }
}

// gw[i][o][k] += sum_{b,y,x} in[b][i][y][x] g[b][o][2y+dy][2x+dx]; gb[o] += sum g[b][o]
__global__ void __launch_bounds__(256) k_tconv_wgrad(const bf16* __restrict__ in, const float* __restrict__ g,
                                                     float* __restrict__ gw, float* __restrict__ gb, int Cin,
                                                     int Cout, int H, int W, int B, int rows_per_cta) {
  __shared__ float s_in[16][64];
  __shared__ float s_g[16][2][128];
  const int ol = threadIdx.x >> 4, il = threadIdx.x & 15;
  const int o0 = blockIdx.x * 16, i0 = blockIdx.y * 16;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float accb = 0.f;
  const int r0 = blockIdx.z * rows_per_cta;
  const int r1 = min(B * H, r0 + rows_per_cta);
  for (int row = r0; row < r1; ++row) {
    const int b = row / H, y = row % H;
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * W; t += 256) {
      const int ii = t / W, x = t % W;
      s_in[ii][x] = (i0 + ii < Cin) ? __bfloat162float(in[(((long long)b * Cin + i0 + ii) * H + y) * W + x]) : 0.f;
    }
    for (int t = threadIdx.x; t < 16 * 2 * 2 * W; t += 256) {
      const int oo = t / (4 * W), r = t % (4 * W), dy = r / (2 * W), X = r % (2 * W);
      s_g[oo][dy][X] = (o0 + oo < Cout) ? g[(((long long)b * Cout + o0 + oo) * 2 * H + 2 * y + dy) * 2 * W + X] : 0.f;
    }
    __syncthreads();
    for (int x = 0; x < W; ++x) {
      const float iv = s_in[il][x];
      acc[0] = fmaf(iv, s_g[ol][0][2 * x], acc[0]);
      acc[1] = fmaf(iv, s_g[ol][0][2 * x + 1], acc[1]);
      acc[2] = fmaf(iv, s_g[ol][1][2 * x], acc[2]);
      acc[3] = fmaf(iv, s_g[ol][1][2 * x + 1], acc[3]);
      if (il == 0) accb += s_g[ol][0][2 * x] + s_g[ol][0][2 * x + 1] + s_g[ol][1][2 * x] + s_g[ol][1][2 * x + 1];
    }
  }
  const int go = o0 + ol, gi = i0 + il;
  if (go < Cout && gi < Cin)
    for (int k = 0; k < 4; ++k) atomicAdd(gw + ((long long)gi * Cout + go) * 4 + k, acc[k]);
  if (il == 0 && blockIdx.y == 0 && go < Cout) atomicAdd(gb + go, accb);
}

// ------------------------------------------------------------------ 1x1 output convolution (FP32 out)
__global__ void k_conv1_fwd(const bf16* __restrict__ in, const bf16* __restrict__ w, const float* __restrict__ bias,
                            float* __restrict__ out, int Cin, int Cout, long long HW, int B, const int* done) {
  if (stopped(done)) return;
  const long long n = (long long)B * Cout * HW;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t % HW;
    const int o = (t / HW) % Cout;
    const int b = t / (HW * Cout);
    float s = bias[o];
    for (int i = 0; i < Cin; ++i)
      s = fmaf(__bfloat162float(w[o * Cin + i]), __bfloat162float(in[((long long)b * Cin + i) * HW + p]), s);
    out[t] = s;
  }
}

__global__ void k_conv1_bwd_data(const float* __restrict__ g, const bf16* __restrict__ w, float* __restrict__ gin,
                                 int Cin, int Cout, long long HW, int B) {
  const long long n = (long long)B * Cin * HW;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t % HW;
    const int i = (t / HW) % Cin;
    const int b = t / (HW * Cin);
    float s = 0.f;
    for (int o = 0; o < Cout; ++o) s = fmaf(__bfloat162float(w[o * Cin + i]), g[((long long)b * Cout + o) * HW + p], s);
    gin[t] = s;
  }
}

// gw[o][i] += sum_{b,p} g[b][o][p] in[b][i][p]; gb[o] += sum g[b][o]: one CTA per (o, i) pair
__global__ void k_conv1_wgrad(const bf16* __restrict__ in, const float* __restrict__ g, float* __restrict__ gw,
                              float* __restrict__ gb, int Cin, int Cout, long long HW, int B) {
  const int o = blockIdx.x / Cin, i = blockIdx.x % Cin;
  float s = 0.f, sb = 0.f;
  for (long long t = threadIdx.x; t < (long long)B * HW; t += blockDim.x) {
    const long long p = t % HW;
    const int b = t / HW;
    const float gv = g[((long long)b * Cout + o) * HW + p];
    s = fmaf(gv, __bfloat162float(in[((long long)b * Cin + i) * HW + p]), s);
    sb += gv;
  }
  __shared__ float sh[256], shb[256];
  sh[threadIdx.x] = s;
  shb[threadIdx.x] = sb;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      sh[threadIdx.x] += sh[threadIdx.x + k];
      shb[threadIdx.x] += shb[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    gw[o * Cin + i] += sh[0];
    if (i == 0) gb[o] += shb[0];
  }
}

// ------------------------------------------------------------------ elementwise pieces
__global__ void k_pool_fwd(const bf16* __restrict__ in, bf16* __restrict__ out, int C, int H, int W, int B,
                           const int* done) {
  if (stopped(done)) return;
  const int h = H / 2, w = W / 2;
  const long long n = (long long)B * C * h * w;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int x = t % w;
    const int y = (t / w) % h;
    const long long bc = t / ((long long)h * w);
    const bf16* p = in + (bc * H + 2 * y) * W + 2 * x;
    out[t] = __float2bfloat16_rn(0.25f * (__bfloat162float(p[0]) + __bfloat162float(p[1]) + __bfloat162float(p[W]) +
                                          __bfloat162float(p[W + 1])));
  }
}

// g[b][c][y][x] = gp[b][c][y/2][x/2] / 4 + gskip[b][c][y][x]
__global__ void k_pool_bwd_add(const float* __restrict__ gp, const float* __restrict__ gskip, float* __restrict__ g,
                               int C, int H, int W, int B) {
  const long long n = (long long)B * C * H * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int x = t % W;
    const int y = (t / W) % H;
    const long long bc = t / ((long long)H * W);
    g[t] = 0.25f * gp[(bc * (H / 2) + y / 2) * (W / 2) + x / 2] + gskip[t];
  }
}

// cat[b] = [u[b] (Cu channels), s[b] (Cs channels)]
__global__ void k_cat(const bf16* __restrict__ u, const bf16* __restrict__ s, bf16* __restrict__ cat, int Cu, int Cs,
                      long long HW, int B, const int* done) {
  if (stopped(done)) return;
  const long long n = (long long)B * (Cu + Cs) * HW;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t % HW;
    const int c = (t / HW) % (Cu + Cs);
    const int b = t / (HW * (Cu + Cs));
    cat[t] = c < Cu ? u[((long long)b * Cu + c) * HW + p] : s[((long long)b * Cs + c - Cu) * HW + p];
  }
}

// gu, gs = split of gcat
__global__ void k_split(const float* __restrict__ gcat, float* __restrict__ gu, float* __restrict__ gs, int Cu, int Cs,
                        long long HW, int B) {
  const long long n = (long long)B * (Cu + Cs) * HW;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t % HW;
    const int c = (t / HW) % (Cu + Cs);
    const int b = t / (HW * (Cu + Cs));
    if (c < Cu) gu[((long long)b * Cu + c) * HW + p] = gcat[t];
    else gs[((long long)b * Cs + c - Cu) * HW + p] = gcat[t];
  }
}

// g *= (act > 0): gradient through the ReLU
__global__ void k_relu_mask(float* __restrict__ g, const bf16* __restrict__ act, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(act[t]) > 0.f)) g[t] = 0.f;
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long long n, const int* done) {
  if (stopped(done)) return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = __float2bfloat16_rn(x[t]);
}

// loss partials of 0.5 (y - t)^2 and g = (y - t) / n
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ tgt, float* __restrict__ g, long long n,
                      double* __restrict__ partial) {
  double acc = 0.0;
  const float inv = 1.0f / (float)n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float d = y[t] - tgt[t];
    g[t] = d * inv;
    acc += 0.5 * (double)d * (double)d;
  }
  block_sum_store(acc, partial);
}

__global__ void k_adam(float* __restrict__ w, bf16* __restrict__ wb, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    const float wt = w[t] - lr * (mt * c1) / (sqrtf(vt * c2) + eps);
    w[t] = wt;
    wb[t] = __float2bfloat16_rn(wt);
  }
}

// ------------------------------------------------------------------ correction inside flexible CG
// s = ||z||; in = z / s (FP32); z = mask * (z + s * out) afterwards
__global__ void k_corr_prep(const double* __restrict__ z, const double* __restrict__ partial, float* __restrict__ in,
                            long long n, const int* done) {
  if (stopped(done)) return;
  __shared__ double s_norm;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kRedBlocks; ++k) s += partial[k];
    s_norm = s > 0.0 ? sqrt(s) : 1.0;
  }
  __syncthreads();
  const double inv = 1.0 / s_norm;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    in[t] = (float)(z[t] * inv);
}

// Per-block sums of r.z and r.y over unmasked entries (z: M_C r, y: the network
// output); written to partial[kRedBlocks + b] and partial[2 kRedBlocks + b].
__global__ void k_corr_dots(const double* __restrict__ r, const double* __restrict__ z, const float* __restrict__ y,
                            const uint8_t* __restrict__ mask, long long npix, int ncomp, double* __restrict__ partial,
                            const int* done) {
  if (stopped(done)) return;
  const long long n = npix * ncomp;
  double rz = 0.0, ry = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    if (mask[t % npix]) {
      rz += r[t] * z[t];
      ry += r[t] * (double)y[t];
    }
  block_sum_store(rz, partial + kRedBlocks);
  block_sum_store(ry, partial + 2 * kRedBlocks);
}

// z <- mask(z + theta s y), s = ||z||.  theta = 1 unless that would leave
// r.z_new < kCorrKeep r.z; then theta shrinks the correction to make
// r.z_new = kCorrKeep r.z, so the corrected direction stays a descent direction
// whatever the network outputs (flexible CG needs r.z > 0 to make progress).
constexpr double kCorrKeep = 0.25;

__global__ void k_corr_apply(double* __restrict__ z, const double* __restrict__ partial, const float* __restrict__ out,
                             const uint8_t* __restrict__ mask, long long npix, int ncomp, const int* done) {
  if (stopped(done)) return;
  const double zz = block_sum_all(partial, kRedBlocks);
  const double rz = block_sum_all(partial + kRedBlocks, kRedBlocks);
  const double ry = block_sum_all(partial + 2 * kRedBlocks, kRedBlocks);
  const double s = zz > 0.0 ? sqrt(zz) : 1.0;
  double theta = 1.0;
  if (rz > 0.0 && rz + s * ry < kCorrKeep * rz) theta = (kCorrKeep - 1.0) * rz / (s * ry);
  if (!(rz > 0.0)) theta = 0.0;
  const double f = theta * s;
  const long long n = npix * ncomp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    z[t] = mask[t % npix] ? z[t] + f * (double)out[t] : 0.0;
}

}  // namespace cmm

// ------------------------------------------------------------------ handle
using namespace cmm;

namespace {
struct Layer {
  int kind;        // 0 conv3, 1 tconv, 2 conv1
  int cin, cout;
  long long woff, boff;
};
}  // namespace

struct cmm_unet {
  int refs = 1;
  int tensor_cores = 1;        // 3x3 convolutions on the tensor cores (0: the FP32 CUDA-core kernels)
  cmm_ctx* ctx = nullptr;
  int ny = 0, nx = 0, L = 0, batch_max = 0;
  int widths[4] = {0, 0, 0, 0};
  long long n_params = 0;
  std::vector<Layer> layers;
  float* master = nullptr;
  bf16* wbf = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  long long step = 0;
  // activations (BF16), indexed as in the forward schedule
  bf16* x_in = nullptr;
  std::vector<bf16*> enc_a, enc_b, pooled, up, cat, dec_a, dec_b;
  float* y_out = nullptr;
  // gradients (FP32)
  float *g0 = nullptr, *g1 = nullptr, *g2 = nullptr;
  std::vector<float*> gskip;
  double* partial = nullptr;
  float* part = nullptr;       // zeroed FP32 partial sums of the split-K forward convolutions
};

namespace {

int grid_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8192)); }

int level_h(const cmm_unet* u, int l) { return u->ny >> l; }
int level_w(const cmm_unet* u, int l) { return u->nx >> l; }

// K slices for a forward launch of `ctas` CTAs over Cin input channels: enough to
// put about two CTAs on every SM when the output alone gives too few (a single map,
// the deep levels), in whole 16-channel chunks and without empty slices.
int k_slices(int ctas, int Cin) {
  const int chunks = (Cin + 15) / 16;
  if (ctas >= 152 || chunks < 2) return 1;
  const int want = std::min(chunks, (2 * 152 + ctas - 1) / ctas);
  const int cps = (chunks + want - 1) / want;
  return (chunks + cps - 1) / cps;
}

template <typename TOUT, bool RELU>
int bias_act(const cmm_unet* u, const float* bias, TOUT* out, int Cout, long long hw, int B, const int* done) {
  const long long n = (long long)B * Cout * hw;
  k_bias_act<TOUT, RELU><<<grid_n(n), 256, 0, u->ctx->stream>>>(u->part, bias, out, Cout, hw, n, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <typename TIN, typename TOUT, bool RELU, bool FLIP, int MT, int TW>
int conv3_tc(const cmm_unet* u, const TIN* in, const bf16* w, const float* bias, TOUT* out, int Cin, int Cout, int H,
             int W, int B, const int* done) {
  constexpr int TH = 256 / TW;
  const int gx = ((W + TW - 1) / TW) * ((H + TH - 1) / TH), gy = (Cout + MT * 16 - 1) / (MT * 16);
  // split K only in the forward layers (FLIP is the input gradient of the backward pass)
  const int ks = (!FLIP && u->part) ? k_slices(gx * gy * B, Cin) : 1;
  const dim3 g(gx, gy, B * ks);
  k_conv3_mma<TIN, TOUT, RELU, FLIP, MT, TW><<<g, 128, 0, u->ctx->stream>>>(in, w, bias, out, Cin, Cout, H, W, done,
                                                                           ks, ks > 1 ? u->part : nullptr);
  CMM_LAUNCH_CHECK();
  if (ks > 1) return bias_act<TOUT, RELU>(u, bias, out, Cout, (long long)H * W, B, done);
  return CMM_OK;
}

// k_pointwise_mma over Cin -> Cout at H x W inputs (TAPS = 4: the 2x2 transposed
// convolution to 2H x 2W; TAPS = 1: a 1x1 convolution), split K as conv3_tc.
template <int TAPS, typename TOUT, int MT>
int pointwise_tc(const cmm_unet* u, const bf16* in, const bf16* w, const float* bias, TOUT* out, int Cin, int Cout,
                 int H, int W, int B, const int* done) {
  const int gx = (H * W + 127) / 128, gy = (Cout + MT * 16 - 1) / (MT * 16);
  const int ks = u->part ? k_slices(gx * gy * B, Cin) : 1;
  const dim3 g(gx, gy, B * ks);
  k_pointwise_mma<TAPS, TOUT, MT><<<g, 128, 0, u->ctx->stream>>>(in, w, bias, out, Cin, Cout, H, W, done, ks,
                                                                 ks > 1 ? u->part : nullptr);
  CMM_LAUNCH_CHECK();
  if (ks > 1) return bias_act<TOUT, false>(u, bias, out, Cout, (long long)H * W * TAPS, B, done);
  return CMM_OK;
}

template <typename TIN, typename TOUT, bool RELU, bool FLIP>
int conv3(const cmm_unet* u, const TIN* in, const bf16* w, const float* bias, TOUT* out, int Cin, int Cout, int H,
          int W, int B, const int* done) {
  if (u->tensor_cores) {
    // two m16 tiles per CTA where there are 32 or more output channels; 8-wide
    // pixel tiles for maps narrower than 16
    if (Cout >= 32) {
      return W >= 16 ? conv3_tc<TIN, TOUT, RELU, FLIP, 2, 16>(u, in, w, bias, out, Cin, Cout, H, W, B, done)
                     : conv3_tc<TIN, TOUT, RELU, FLIP, 2, 8>(u, in, w, bias, out, Cin, Cout, H, W, B, done);
    }
    return W >= 16 ? conv3_tc<TIN, TOUT, RELU, FLIP, 1, 16>(u, in, w, bias, out, Cin, Cout, H, W, B, done)
                   : conv3_tc<TIN, TOUT, RELU, FLIP, 1, 8>(u, in, w, bias, out, Cin, Cout, H, W, B, done);
  }
  const dim3 g(((W + 15) / 16) * ((H + 15) / 16), (Cout + 15) / 16, B);
  k_conv3<TIN, TOUT, RELU, FLIP><<<g, 256, 0, u->ctx->stream>>>(in, w, bias, out, Cin, Cout, H, W, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int conv3_wgrad(const cmm_unet* u, const bf16* in, const float* g, float* gw, float* gb, int Cin, int Cout, int H,
                int W, int B) {
  const int rows = B * H;
  const int ctas_ij = ((Cout + 15) / 16) * ((Cin + 15) / 16);
  const int slices = std::max(1, std::min(rows, 608 / std::max(1, ctas_ij)));
  const int per = (rows + slices - 1) / slices;
  const dim3 gr((Cout + 15) / 16, (Cin + 15) / 16, (rows + per - 1) / per);
  if (u->tensor_cores) k_conv3_wgrad_mma<<<gr, 128, 0, u->ctx->stream>>>(in, g, gw, gb, Cin, Cout, H, W, B, per);
  else k_conv3_wgrad<<<gr, 256, 0, u->ctx->stream>>>(in, g, gw, gb, Cin, Cout, H, W, B, per);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int tconv_wgrad(const cmm_unet* u, const bf16* in, const float* g, float* gw, float* gb, int Cin, int Cout, int H,
                int W, int B) {
  const int rows = B * H;
  const int ctas_ij = ((Cout + 15) / 16) * ((Cin + 15) / 16);
  const int slices = std::max(1, std::min(rows, 608 / std::max(1, ctas_ij)));
  const int per = (rows + slices - 1) / slices;
  const dim3 gr((Cout + 15) / 16, (Cin + 15) / 16, (rows + per - 1) / per);
  k_tconv_wgrad<<<gr, 256, 0, u->ctx->stream>>>(in, g, gw, gb, Cin, Cout, H, W, B, per);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

void build_layers(cmm_unet* u) {
  long long o = 0;
  auto add = [&](int kind, int cin, int cout) {
    Layer l;
    l.kind = kind;
    l.cin = cin;
    l.cout = cout;
    const long long nw = (long long)cin * cout * (kind == 0 ? 9 : (kind == 1 ? 4 : 1));
    l.woff = o;
    o += nw;
    l.boff = o;
    o += cout;
    u->layers.push_back(l);
  };
  int c = 3;
  for (int l = 0; l < u->L; ++l) {
    add(0, c, u->widths[l]);
    add(0, u->widths[l], u->widths[l]);
    c = u->widths[l];
  }
  for (int l = u->L - 2; l >= 0; --l) {
    add(1, u->widths[l + 1], u->widths[l]);
    add(0, 2 * u->widths[l], u->widths[l]);
    add(0, u->widths[l], u->widths[l]);
  }
  add(2, u->widths[0], 3);
  u->n_params = o;
}

template <typename P>
int dalloc_u(P** p, size_t bytes) {
  if (cudaMalloc((void**)p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    return fail(CMM_ERR_OOM, "U-Net allocation failed");
  }
  return CMM_OK;
}

// Forward pass for `B` inputs already in u->x_in; output FP32 in u->y_out.
int unet_forward(cmm_unet* u, int B, const int* done) {
  const int L = u->L;
  const bf16* h = u->x_in;
  int c = 3;
  size_t li = 0;
  for (int l = 0; l < L; ++l) {
    const int H = level_h(u, l), W = level_w(u, l), w = u->widths[l];
    const Layer& a = u->layers[li++];
    const Layer& b = u->layers[li++];
    CMM_TRY((conv3<bf16, bf16, true, false>(u, h, u->wbf + a.woff, u->master + a.boff, u->enc_a[l], c, w, H, W, B, done)));
    CMM_TRY((conv3<bf16, bf16, true, false>(u, u->enc_a[l], u->wbf + b.woff, u->master + b.boff, u->enc_b[l], w, w, H, W, B, done)));
    h = u->enc_b[l];
    c = w;
    if (l < L - 1) {
      k_pool_fwd<<<grid_n((long long)B * w * H * W / 4), 256, 0, u->ctx->stream>>>(h, u->pooled[l], w, H, W, B, done);
      CMM_LAUNCH_CHECK();
      h = u->pooled[l];
    }
  }
  for (int l = L - 2; l >= 0; --l) {
    const int H = level_h(u, l), W = level_w(u, l), w = u->widths[l];
    const Layer& t = u->layers[li++];
    const Layer& a = u->layers[li++];
    const Layer& b = u->layers[li++];
    if (u->tensor_cores) {
      CMM_TRY((pointwise_tc<4, bf16, 2>(u, h, u->wbf + t.woff, u->master + t.boff, u->up[l], c, w, H / 2, W / 2, B,
                                         done)));
    } else {
      k_tconv_fwd<<<grid_n((long long)B * w * H * W), 256, 0, u->ctx->stream>>>(h, u->wbf + t.woff, u->master + t.boff,
                                                                                u->up[l], c, w, H / 2, W / 2, B, done);
      CMM_LAUNCH_CHECK();
    }
    k_cat<<<grid_n((long long)B * 2 * w * H * W), 256, 0, u->ctx->stream>>>(u->up[l], u->enc_b[l], u->cat[l], w, w,
                                                                            (long long)H * W, B, done);
    CMM_LAUNCH_CHECK();
    CMM_TRY((conv3<bf16, bf16, true, false>(u, u->cat[l], u->wbf + a.woff, u->master + a.boff, u->dec_a[l], 2 * w, w, H, W, B, done)));
    CMM_TRY((conv3<bf16, bf16, true, false>(u, u->dec_a[l], u->wbf + b.woff, u->master + b.boff, u->dec_b[l], w, w, H, W, B, done)));
    h = u->dec_b[l];
    c = w;
  }
  const Layer& o = u->layers[li++];
  const long long HW = (long long)u->ny * u->nx;
  if (u->tensor_cores)
    return pointwise_tc<1, float, 1>(u, h, u->wbf + o.woff, u->master + o.boff, u->y_out, c, 3, u->ny, u->nx, B, done);
  k_conv1_fwd<<<grid_n((long long)B * 3 * HW), 256, 0, u->ctx->stream>>>(h, u->wbf + o.woff, u->master + o.boff,
                                                                        u->y_out, c, 3, HW, B, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

// Backward pass from dL/dy in u->g0 ([B][3][ny][nx]); accumulates into u->grad (zeroed here).
int unet_backward(cmm_unet* u, int B) {
  cudaStream_t st = u->ctx->stream;
  CMM_CUDA(cudaMemsetAsync(u->grad, 0, sizeof(float) * u->n_params, st));
  const int L = u->L;
  const long long HW = (long long)u->ny * u->nx;
  int li = (int)u->layers.size() - 1;
  float* g = u->g0;      // current gradient
  float* gn = u->g1;     // next
  // output 1x1
  {
    const Layer& o = u->layers[li--];
    const bf16* hin = L > 1 ? u->dec_b[0] : u->enc_b[0];
    k_conv1_wgrad<<<o.cout * o.cin, 256, 0, st>>>(hin, g, u->grad + o.woff, u->grad + o.boff, o.cin, o.cout, HW, B);
    CMM_LAUNCH_CHECK();
    k_conv1_bwd_data<<<grid_n((long long)B * o.cin * HW), 256, 0, st>>>(g, u->wbf + o.woff, gn, o.cin, o.cout, HW, B);
    CMM_LAUNCH_CHECK();
    std::swap(g, gn);
  }
  auto conv_back = [&](const Layer& ly, const bf16* in, const bf16* out, int H, int W) -> int {
    const long long n = (long long)B * ly.cout * H * W;
    k_relu_mask<<<grid_n(n), 256, 0, st>>>(g, out, n);
    CMM_LAUNCH_CHECK();
    CMM_TRY(conv3_wgrad(u, in, g, u->grad + ly.woff, u->grad + ly.boff, ly.cin, ly.cout, H, W, B));
    CMM_TRY((conv3<float, float, false, true>(u, g, u->wbf + ly.woff, nullptr, gn, ly.cout, ly.cin, H, W, B, nullptr)));
    std::swap(g, gn);
    return CMM_OK;
  };
  // decoder, in reverse order of the forward pass
  for (int l = 0; l <= L - 2; ++l) {
    const int H = level_h(u, l), W = level_w(u, l), w = u->widths[l];
    const Layer& b = u->layers[li--];
    const Layer& a = u->layers[li--];
    const Layer& t = u->layers[li--];
    CMM_TRY(conv_back(b, u->dec_a[l], u->dec_b[l], H, W));
    CMM_TRY(conv_back(a, u->cat[l], u->dec_a[l], H, W));
    // g is now dL/dcat [B][2w][H][W]
    k_split<<<grid_n((long long)B * 2 * w * H * W), 256, 0, st>>>(g, gn, u->gskip[l], w, w, (long long)H * W, B);
    CMM_LAUNCH_CHECK();
    std::swap(g, gn);   // g = dL/dup
    const bf16* tin = (l + 1 <= L - 2) ? u->dec_b[l + 1] : u->enc_b[L - 1];
    CMM_TRY(tconv_wgrad(u, tin, g, u->grad + t.woff, u->grad + t.boff, t.cin, t.cout, H / 2, W / 2, B));
    k_tconv_bwd_data<<<grid_n((long long)B * t.cin * (H / 2) * (W / 2)), 256, 0, st>>>(g, u->wbf + t.woff, gn, t.cin,
                                                                                         t.cout, H / 2, W / 2, B);
    CMM_LAUNCH_CHECK();
    std::swap(g, gn);
  }
  // encoder, deepest level first
  for (int l = L - 1; l >= 0; --l) {
    const int H = level_h(u, l), W = level_w(u, l);
    const Layer& b = u->layers[li--];
    const Layer& a = u->layers[li--];
    CMM_TRY(conv_back(b, u->enc_a[l], u->enc_b[l], H, W));
    const bf16* ain = l > 0 ? u->pooled[l - 1] : u->x_in;
    if (l > 0) {
      CMM_TRY(conv_back(a, ain, u->enc_a[l], H, W));
      // g = dL/dpooled[l-1]; through the pool plus the skip gradient of level l-1
      const int Hp = level_h(u, l - 1), Wp = level_w(u, l - 1);
      k_pool_bwd_add<<<grid_n((long long)B * u->widths[l - 1] * Hp * Wp), 256, 0, st>>>(g, u->gskip[l - 1], gn,
                                                                                        u->widths[l - 1], Hp, Wp, B);
      CMM_LAUNCH_CHECK();
      std::swap(g, gn);
    } else {
      // first layer: only the weight gradient is needed
      const long long n = (long long)B * a.cout * H * W;
      k_relu_mask<<<grid_n(n), 256, 0, st>>>(g, u->enc_a[0], n);
      CMM_LAUNCH_CHECK();
      CMM_TRY(conv3_wgrad(u, ain, g, u->grad + a.woff, u->grad + a.boff, a.cin, a.cout, H, W, B));
    }
  }
  return CMM_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

static void free_unet(cmm_unet* u) {
  cudaSetDevice(u->ctx->device);
  cudaStreamSynchronize(u->ctx->stream);
  for (void* p : {(void*)u->master, (void*)u->wbf, (void*)u->grad, (void*)u->m, (void*)u->v, (void*)u->x_in,
                  (void*)u->y_out, (void*)u->g0, (void*)u->g1, (void*)u->g2, (void*)u->partial, (void*)u->part})
    if (p) cudaFree(p);
  for (auto* vec : {&u->enc_a, &u->enc_b, &u->pooled, &u->up, &u->cat, &u->dec_a, &u->dec_b})
    for (auto* p : *vec)
      if (p) cudaFree(p);
  for (auto* p : u->gskip)
    if (p) cudaFree(p);
  cmm_ctx* c = u->ctx;
  delete u;
  ctx_release(c);
}

}  // extern "C"

namespace cmm {
void unet_retain(cmm_unet* u) { u->refs++; }
void unet_release(cmm_unet* u) {
  if (--u->refs == 0) free_unet(u);
}
}  // namespace cmm

extern "C" {

int cmm_unet_destroy(cmm_unet* u) {
  if (u) unet_release(u);
  return CMM_OK;
}

int cmm_unet_create(cmm_ctx* ctx, int32_t ny, int32_t nx, int32_t levels, const int32_t* widths, int32_t batch_max,
                    cmm_unet** out) {
  if (!ctx || !widths || !out) return fail(CMM_ERR_ARG, "null argument");
  *out = nullptr;
  if (levels < 1 || levels > 4 || batch_max < 1) return fail(CMM_ERR_ARG, "levels must be 1..4, batch_max >= 1");
  if (ny % (1 << (levels - 1)) || nx % (1 << (levels - 1)))
    return fail(CMM_ERR_ARG, "map sides must be divisible by 2^(levels-1)");
  if (nx > 64) return fail(CMM_ERR_UNSUPPORTED, "U-Net maps wider than 64 pixels are not supported");
  for (int l = 0; l < levels; ++l)
    if (widths[l] < 1 || widths[l] > 256) return fail(CMM_ERR_ARG, "bad width");
  CMM_CUDA(cudaSetDevice(ctx->device));
  cmm_unet* u = new cmm_unet();
  u->ctx = ctx;
  ctx_retain(ctx);
  u->ny = ny;
  u->nx = nx;
  u->L = levels;
  u->batch_max = batch_max;
  for (int l = 0; l < levels; ++l) u->widths[l] = widths[l];
  build_layers(u);
  const long long B = batch_max;
  int s = CMM_OK;
  auto A = [&](auto** p, size_t bytes) {
    if (s == CMM_OK) s = dalloc_u(p, bytes);
  };
  A(&u->master, sizeof(float) * u->n_params);
  A(&u->wbf, sizeof(bf16) * u->n_params);
  A(&u->grad, sizeof(float) * u->n_params);
  A(&u->m, sizeof(float) * u->n_params);
  A(&u->v, sizeof(float) * u->n_params);
  A(&u->x_in, sizeof(bf16) * B * 3 * ny * nx);
  A(&u->y_out, sizeof(float) * B * 3 * ny * nx);
  A(&u->partial, sizeof(double) * 3 * kRedBlocks);
  long long gmax = 3;
  u->enc_a.assign(levels, nullptr);
  u->enc_b.assign(levels, nullptr);
  u->pooled.assign(levels, nullptr);
  u->up.assign(levels, nullptr);
  u->cat.assign(levels, nullptr);
  u->dec_a.assign(levels, nullptr);
  u->dec_b.assign(levels, nullptr);
  u->gskip.assign(levels, nullptr);
  for (int l = 0; l < levels; ++l) {
    const long long hw = (long long)(ny >> l) * (nx >> l), w = widths[l];
    A(&u->enc_a[l], sizeof(bf16) * B * w * hw);
    A(&u->enc_b[l], sizeof(bf16) * B * w * hw);
    gmax = std::max(gmax, 2 * w * hw);
    if (l < levels - 1) {
      A(&u->pooled[l], sizeof(bf16) * B * w * hw / 4);
      A(&u->up[l], sizeof(bf16) * B * w * hw);
      A(&u->cat[l], sizeof(bf16) * B * 2 * w * hw);
      A(&u->dec_a[l], sizeof(bf16) * B * w * hw);
      A(&u->dec_b[l], sizeof(bf16) * B * w * hw);
      A(&u->gskip[l], sizeof(float) * B * w * hw);
    }
  }
  A(&u->g0, sizeof(float) * B * gmax);
  A(&u->g1, sizeof(float) * B * gmax);
  A(&u->g2, sizeof(float) * B * gmax);
  // split-K partial sums: the largest forward output, [B][w_l][ny >> l][nx >> l] or the 3-channel output
  long long pmax = 3LL * ny * nx;
  for (int l = 0; l < levels; ++l) pmax = std::max(pmax, (long long)widths[l] * (ny >> l) * (nx >> l));
  A(&u->part, sizeof(float) * B * pmax);
  if (s == CMM_OK && cudaMemset(u->part, 0, sizeof(float) * B * pmax) != cudaSuccess) {
    cudaGetLastError();
    s = fail(CMM_ERR_CUDA, "cudaMemset of the U-Net partial sums failed");
  }
  if (s != CMM_OK) {
    cmm_unet_destroy(u);
    return s;
  }
  *out = u;
  return CMM_OK;
}

int cmm_unet_set_tensor_cores(cmm_unet* u, int32_t enable) {
  if (!u) return fail(CMM_ERR_ARG, "null argument");
  u->tensor_cores = enable ? 1 : 0;
  return CMM_OK;
}

int cmm_unet_param_count(cmm_unet* u, int64_t* n) {
  if (!u || !n) return fail(CMM_ERR_ARG, "null argument");
  *n = u->n_params;
  return CMM_OK;
}

int cmm_unet_set_params(cmm_unet* u, const float* params) {
  if (!u || !params) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(u->ctx->device));
  cudaStream_t st = u->ctx->stream;
  CMM_CUDA(cudaMemcpyAsync(u->master, params, sizeof(float) * u->n_params, cudaMemcpyDeviceToDevice, st));
  k_to_bf16<<<grid_n(u->n_params), 256, 0, st>>>(u->master, u->wbf, u->n_params, nullptr);
  CMM_LAUNCH_CHECK();
  CMM_CUDA(cudaMemsetAsync(u->m, 0, sizeof(float) * u->n_params, st));
  CMM_CUDA(cudaMemsetAsync(u->v, 0, sizeof(float) * u->n_params, st));
  u->step = 0;
  return CMM_OK;
}

int cmm_unet_init(cmm_unet* u, uint64_t seed) {
  if (!u) return fail(CMM_ERR_ARG, "null argument");
  std::vector<float> h((size_t)u->n_params, 0.0f);
  std::mt19937_64 gen(seed);
  std::normal_distribution<double> normal(0.0, 1.0);
  for (size_t i = 0; i < u->layers.size(); ++i) {
    const Layer& a = u->layers[i];
    const long long fan_in = (long long)a.cin * (a.kind == 0 ? 9 : a.kind == 1 ? 4 : 1);
    const long long nw = a.boff - a.woff;
    const double scale = std::sqrt(2.0 / (double)fan_in) * (i + 1 == u->layers.size() ? 1e-2 : 1.0);
    for (long long k = 0; k < nw; ++k) h[a.woff + k] = (float)(normal(gen) * scale);
  }
  float* d = nullptr;
  CMM_CUDA(cudaSetDevice(u->ctx->device));
  CMM_CUDA(cudaMalloc(&d, sizeof(float) * u->n_params));
  cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(float) * u->n_params, cudaMemcpyHostToDevice, u->ctx->stream);
  int st = e == cudaSuccess ? cmm_unet_set_params(u, d) : cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
  if (st == CMM_OK) {
    e = cudaStreamSynchronize(u->ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
  }
  cudaFree(d);
  return st;
}

int cmm_unet_get_params(cmm_unet* u, float* params) {
  if (!u || !params) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(u->ctx->device));
  CMM_CUDA(cudaMemcpyAsync(params, u->master, sizeof(float) * u->n_params, cudaMemcpyDeviceToDevice, u->ctx->stream));
  return CMM_OK;
}

int cmm_unet_forward(cmm_unet* u, int32_t batch, const float* in, float* out) {
  if (!u || !in || !out || batch < 1 || batch > u->batch_max) return fail(CMM_ERR_ARG, "bad argument");
  CMM_CUDA(cudaSetDevice(u->ctx->device));
  const long long n = (long long)batch * 3 * u->ny * u->nx;
  k_to_bf16<<<grid_n(n), 256, 0, u->ctx->stream>>>(in, u->x_in, n, nullptr);
  CMM_LAUNCH_CHECK();
  CMM_TRY(unet_forward(u, batch, nullptr));
  CMM_CUDA(cudaMemcpyAsync(out, u->y_out, sizeof(float) * n, cudaMemcpyDeviceToDevice, u->ctx->stream));
  return CMM_OK;
}

int cmm_unet_loss_grad(cmm_unet* u, int32_t batch, const float* in, const float* target, float* grad,
                       double* loss_host) {
  if (!u || !in || !target || batch < 1 || batch > u->batch_max) return fail(CMM_ERR_ARG, "bad argument");
  CMM_CUDA(cudaSetDevice(u->ctx->device));
  cudaStream_t st = u->ctx->stream;
  const long long n = (long long)batch * 3 * u->ny * u->nx;
  k_to_bf16<<<grid_n(n), 256, 0, st>>>(in, u->x_in, n, nullptr);
  CMM_LAUNCH_CHECK();
  CMM_TRY(unet_forward(u, batch, nullptr));
  k_mse<<<kRedBlocks, 256, 0, st>>>(u->y_out, target, u->g0, n, u->partial);
  CMM_LAUNCH_CHECK();
  CMM_TRY(unet_backward(u, batch));
  if (grad) CMM_CUDA(cudaMemcpyAsync(grad, u->grad, sizeof(float) * u->n_params, cudaMemcpyDeviceToDevice, st));
  if (loss_host) {
    std::vector<double> h(kRedBlocks);
    CMM_CUDA(cudaMemcpyAsync(h.data(), u->partial, sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
    CMM_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : h) s += v;
    *loss_host = s / (double)n;
  }
  return CMM_OK;
}

int cmm_unet_train_step(cmm_unet* u, int32_t batch, const float* in, const float* target, float lr,
                        double* loss_host) {
  CMM_TRY(cmm_unet_loss_grad(u, batch, in, target, nullptr, loss_host));
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f / (1.0f - powf(b1, (float)u->step));
  const float c2 = 1.0f / (1.0f - powf(b2, (float)u->step));
  k_adam<<<grid_n(u->n_params), 256, 0, u->ctx->stream>>>(u->master, u->wbf, u->grad, u->m, u->v, u->n_params, lr, b1,
                                                          b2, eps, c1, c2);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

}  // extern "C"

namespace cmm {

bool unet_matches(const cmm_unet* u, const cmm_ctx* ctx, int ny, int nx) {
  return u->ctx == ctx && u->ny == ny && u->nx == nx;
}

// z <- mask (z + ||z|| U(z / ||z||)) for a batch of one map, all on the device.
int unet_correct(cmm_unet* u, const double* r, double* z, const uint8_t* mask, int64_t npix, int ncomp,
                 const int* done, cudaStream_t st) {
  if (ncomp != 3 || npix != (int64_t)u->ny * u->nx) return fail(CMM_ERR_ARG, "U-Net shape does not match the map");
  const long long n = 3 * npix;
  CMM_TRY(launch_dot_partial(z, z, n, u->partial, done, st));
  float* in = u->g2;   // FP32 staging of the normalised input
  k_corr_prep<<<grid_n(n), 256, 0, st>>>(z, u->partial, in, n, done);
  CMM_LAUNCH_CHECK();
  k_to_bf16<<<grid_n(n), 256, 0, st>>>(in, u->x_in, n, done);
  CMM_LAUNCH_CHECK();
  CMM_TRY(unet_forward(u, 1, done));
  k_corr_dots<<<kRedBlocks, 256, 0, st>>>(r, z, u->y_out, mask, npix, ncomp, u->partial, done);
  CMM_LAUNCH_CHECK();
  k_corr_apply<<<grid_n(n), 256, 0, st>>>(z, u->partial, u->y_out, mask, npix, ncomp, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

}  // namespace cmm
