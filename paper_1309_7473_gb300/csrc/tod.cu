// The operator A = P^T N^-1 P (Eq. 2) on the time-ordered data.
//
// Per detector the n_t real samples are packed as N = n_t / 2 complex values
// z_j = x_{2j} + i x_{2j+1} and transformed by a two-pass (four-step) FFT with
// N = R * C, j = c + C r, k = k_r + R k_c:
//   pass T  (k_tod_fwd):    for each column c, an R-point FFT over r of the samples
//                           generated on the fly by P (pointing + map gather, Eq. 1),
//                           times w_N^{c k_r}; stored as Y[k_r][c].
//   pass F  (k_tod_filter): for each row pair (k_r, R - k_r), C-point FFTs over c,
//                           the real-FFT split, the filter w_d(f) of N^-1, the real
//                           inverse merge, inverse C-point FFTs, times w_N^{-c k_r}.
//   pass T' (k_tod_inv_bin): inverse R-point FFTs per column and the binning P^T of
//                           each sample into the FP64 map accumulator.
// The half-spectrum crosses HBM twice (forward and inverse exchange); the map
// copy used by the gather and the accumulator stay resident in L2.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "tod_common.cuh"

namespace cmm {

// ------------------------------------------------------------------ pass T (forward)
// SRC 0: samples are P m; 1: float TOD; 2: double TOD.
template <typename T, int NC, int SRC, typename S>
__global__ void __launch_bounds__(256) k_tod_fwd(const TodArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C2 = V2<T>;
  C2* b0 = reinterpret_cast<C2*>(smem_raw);
  C2* b1 = b0 + (a.J << a.logR);
  const int dl = blockIdx.y;
  const int d = a.d0 + dl;
  const int c0 = blockIdx.x << a.logJ;
  const int nel = a.J << a.logR;
  const int2 off = a.det_off[d];
  const V2<T> pol = reinterpret_cast<const V2<T>*>(a.pol)[d];
  const C2* tw = reinterpret_cast<const C2*>(a.tw);
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    const int cl = idx & (a.J - 1);
    const int r = idx >> a.logJ;
    const long long j = (long long)(c0 + cl) + ((long long)r << a.logC);
    const long long t0 = 2 * j;
    T v0, v1;
    if (SRC == 0) {
      v0 = project_sample<T, NC>(a, off, pol, t0);
      v1 = project_sample<T, NC>(a, off, pol, t0 + 1);
    } else if (SRC == 1) {
      const float2 v = *reinterpret_cast<const float2*>((const float*)a.tod + (long long)d * a.n_t + t0);
      v0 = (T)v.x;
      v1 = (T)v.y;
    } else {
      const double2 v = *reinterpret_cast<const double2*>((const double*)a.tod + (long long)d * a.n_t + t0);
      v0 = (T)v.x;
      v1 = (T)v.y;
    }
    b0[idx] = C2{v0, v1};
  }
  __syncthreads();
  C2* res = block_fft_pow2<T, -1>(b0, b1, a.logR, a.logJ, 1, a.J, tw + a.twl.R_off);
  S* Y = reinterpret_cast<S*>(a.spec) + (long long)dl * a.N;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    const int cl = idx & (a.J - 1);
    const int kr = idx >> a.logJ;
    const long long e = (long long)(c0 + cl) * kr;
    const C2 v = cmul(res[idx], twiddle_N<T>(a, tw, e));
    Store<T, S>::st(Y + (long long)kr * a.C + c0 + cl, v);
  }
}

// ------------------------------------------------------------------ pass F (filter)
template <typename T, typename S>
__global__ void __launch_bounds__(256) k_tod_filter(const TodArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C2 = V2<T>;
  const int C = a.C;
  C2* b0 = reinterpret_cast<C2*>(smem_raw);
  C2* b1 = b0 + 2 * C;
  const int ra = blockIdx.x;                 // 0 .. R/2
  const int rb = (a.R - ra) & (a.R - 1);
  const int nrows = (ra == rb) ? 1 : 2;
  const int dl = blockIdx.y;
  const int d = a.d0 + dl;
  const C2* tw = reinterpret_cast<const C2*>(a.tw);
  S* Y = reinterpret_cast<S*>(a.spec) + (long long)dl * a.N;
  for (int idx = threadIdx.x; idx < nrows * C; idx += blockDim.x) {
    const int s = idx >> a.logC;
    const int e = idx & (C - 1);
    const int row = s ? rb : ra;
    b0[idx] = Store<T, S>::ld(Y + (long long)row * C + e);
  }
  __syncthreads();
  C2* res = block_fft_pow2<T, -1>(b0, b1, a.logC, nrows - 1, C, 1, tw + a.twl.C_off);
  C2* other = (res == b0) ? b1 : b0;
  // real-FFT split, filter, merge: for each pair (k, N - k)
  const V4<T> cf = reinterpret_cast<const V4<T>*>(a.coef)[d];
  const C2 wrow = tw[a.twl.N2_off + ra];     // w_{2N}^{k_r}
  int npairs;
  if (nrows == 2) npairs = C;
  else if (ra == 0) npairs = C / 2 + 1;
  else npairs = C / 2;
  for (int kc = threadIdx.x; kc < npairs; kc += blockDim.x) {
    int i1 = kc, i2;
    if (nrows == 2) i2 = C + (C - 1 - kc);
    else if (ra == 0) i2 = (C - kc) & (C - 1);
    else i2 = C - 1 - kc;
    const long long k = (long long)ra + (long long)a.R * kc;
    const C2 A = res[i1];
    const C2 B = cconj(res[i2]);
    const C2 E{(A.x + B.x) * (T)0.5, (A.y + B.y) * (T)0.5};
    const C2 D{(A.x - B.x) * (T)0.5, (A.y - B.y) * (T)0.5};
    const C2 O{D.y, -D.x};                   // (A - B) / (2i)
    const C2 W = cmul(wrow, tw[a.twl.C2_off + kc]);   // w_{2N}^k
    const T wk = noise_weight<T>(a.wtab, a.N, d, cf, k);
    const T wm = noise_weight<T>(a.wtab, a.N, d, cf, a.N - k);
    const T ws = (T)0.5 * (wk + wm), wd = (T)0.5 * (wk - wm);
    const C2 WO = cmul(W, O);
    const C2 Ep{ws * E.x + wd * WO.x, ws * E.y + wd * WO.y};
    const C2 cWE = cmulc(E, W);              // conj(W) E
    const C2 Op{wd * cWE.x + ws * O.x, wd * cWE.y + ws * O.y};
    res[i1] = C2{Ep.x - Op.y, Ep.y + Op.x};  // E' + i O'
    if (i2 != i1) res[i2] = C2{Ep.x + Op.y, Op.x - Ep.y};  // conj(E') + i conj(O')
  }
  __syncthreads();
  C2* res2 = block_fft_pow2<T, 1>(res, other, a.logC, nrows - 1, C, 1, tw + a.twl.C_off);
  for (int idx = threadIdx.x; idx < nrows * C; idx += blockDim.x) {
    const int s = idx >> a.logC;
    const int c = idx & (C - 1);
    const int row = s ? rb : ra;
    const C2 w = twiddle_N<T>(a, tw, (long long)c * row);
    Store<T, S>::st(Y + (long long)row * C + c, cmulc(res2[idx], w));
  }
}

// ------------------------------------------------------------------ pass T' (inverse + P^T)
template <typename T, int NC, typename S>
__global__ void __launch_bounds__(256) k_tod_inv_bin(const TodArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C2 = V2<T>;
  C2* b0 = reinterpret_cast<C2*>(smem_raw);
  C2* b1 = b0 + (a.J << a.logR);
  const int dl = blockIdx.y;
  const int d = a.d0 + dl;
  const int c0 = blockIdx.x << a.logJ;
  const int nel = a.J << a.logR;
  const C2* tw = reinterpret_cast<const C2*>(a.tw);
  const S* Y = reinterpret_cast<const S*>(a.spec) + (long long)dl * a.N;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    const int cl = idx & (a.J - 1);
    const int kr = idx >> a.logJ;
    b0[idx] = Store<T, S>::ld(Y + (long long)kr * a.C + c0 + cl);
  }
  __syncthreads();
  C2* res = block_fft_pow2<T, 1>(b0, b1, a.logR, a.logJ, 1, a.J, tw + a.twl.R_off);
  const int2 off = a.det_off[d];
  const V2<T> pol = reinterpret_cast<const V2<T>*>(a.pol)[d];
  const T scale = (T)1 / (T)a.N;
  for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
    const int cl = idx & (a.J - 1);
    const int r = idx >> a.logJ;
    const long long j = (long long)(c0 + cl) + ((long long)r << a.logC);
    const C2 z = res[idx];
    bin_sample<T, NC>(a, off, pol, 2 * j, z.x * scale);
    bin_sample<T, NC>(a, off, pol, 2 * j + 1, z.y * scale);
  }
}

// ------------------------------------------------------------------ map <-> resident copies
template <typename T, int NC>
__global__ void k_map_to_gather(const double* __restrict__ m, const uint8_t* __restrict__ mask,
                                void* gather, double* acc, int acc_stride, long long npix,
                                const int* done) {
  if (done && *done) return;
  // the extra pixel npix: zero in the gather copy, accumulator cleared
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (NC == 1) reinterpret_cast<T*>(gather)[npix] = (T)0;
    else reinterpret_cast<V4<T>*>(gather)[npix] = V4<T>{(T)0, (T)0, (T)0, (T)0};
    for (int c = 0; c < acc_stride; ++c) acc[npix * acc_stride + c] = 0.0;
  }
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    const bool ok = mask[p] != 0;
    if (NC == 1) {
      reinterpret_cast<T*>(gather)[p] = ok ? (T)m[p] : (T)0;
    } else {
      V4<T> g;
      g.x = ok ? (T)m[p] : (T)0;
      g.y = ok ? (T)m[npix + p] : (T)0;
      g.z = ok ? (T)m[2 * npix + p] : (T)0;
      g.w = (T)0;
      reinterpret_cast<V4<T>*>(gather)[p] = g;
    }
    for (int c = 0; c < acc_stride; ++c) acc[p * acc_stride + c] = 0.0;
  }
}

template <int NC>
__global__ void k_acc_to_map(const double* __restrict__ acc, const uint8_t* __restrict__ mask,
                             double* __restrict__ out, int acc_stride, long long npix, const int* done) {
  if (done && *done) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    const bool ok = mask[p] != 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c * npix + p] = ok ? acc[p * acc_stride + c] : 0.0;
  }
}

// tod[d][t] = (P m)_{d,t}: pointing + gather only (used to synthesise noise-free data)
template <typename T, int NC, typename OUT>
__global__ void k_project(const TodArgs a, OUT* __restrict__ tod) {
  const int d = blockIdx.y;
  const int2 off = a.det_off[d];
  const V2<T> pol = reinterpret_cast<const V2<T>*>(a.pol)[d];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < a.n_t;
       t += (long long)gridDim.x * blockDim.x)
    tod[(long long)d * a.n_t + t] = (OUT)project_sample<T, NC>(a, off, pol, t);
}

// Per-pixel blocks sum_t u_d P_t P_t^T (Eq. 3-5): [npix][6] = (TT, TQ, TU, QQ, QU, UU)
// for TQU maps, [npix] for T maps.  u_d = det_weight[d] (or 1); masked pixels skipped.
template <int NC>
__global__ void k_hit_blocks(const int4* __restrict__ bore, const int2* __restrict__ det_off,
                             const double2* __restrict__ pol, int ny, int nx, int periodic,
                             long long n_t, const double* __restrict__ det_weight,
                             const uint8_t* __restrict__ mask, double* __restrict__ blocks,
                             const int* done) {
  if (done && *done) return;
  const int d = blockIdx.y;
  const int2 off = det_off[d];
  const double2 pl = pol[d];
  const double u = det_weight ? det_weight[d] : 1.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_t;
       t += (long long)gridDim.x * blockDim.x) {
    const int4 b = bore[t];
    const int p = sample_pixel(b, off, ny, nx, periodic);
    if (p < 0) continue;
    if (mask && !mask[p]) continue;
    if (NC == 1) {
      atomicAdd(blocks + p, u);
    } else {
      double c, s;
      sample_response<double>(b, pl, c, s);
      double* dst = blocks + 6 * (long long)p;
      atomicAdd(dst + 0, u);
      atomicAdd(dst + 1, u * c);
      atomicAdd(dst + 2, u * s);
      atomicAdd(dst + 3, u * c * c);
      atomicAdd(dst + 4, u * c * s);
      atomicAdd(dst + 5, u * s * s);
    }
  }
}

// ------------------------------------------------------------------ host side

template <typename T>
static void fill_table(std::vector<V2<T>>& dst, int64_t off, int count, double L) {
  for (int e = 0; e < count; ++e) {
    const double ang = -2.0 * M_PI * (double)e / L;
    dst[off + e] = V2<T>{(T)std::cos(ang), (T)std::sin(ang)};
  }
}

template <typename T>
static int init_tw(cmm_op* op) {
  const TwLayout l = tw_layout(op->R, op->C);
  std::vector<V2<T>> h(l.total);
  fill_table<T>(h, l.R_off, op->R, op->R);
  fill_table<T>(h, l.C_off, op->C, op->C);
  fill_table<T>(h, l.Nlo_off, op->C, (double)op->N);
  fill_table<T>(h, l.N2_off, op->R, 2.0 * (double)op->N);
  fill_table<T>(h, l.C2_off, op->C, 2.0 * op->C);
  if (cudaMalloc(&op->tw, sizeof(V2<T>) * l.total) != cudaSuccess)
    return fail(CMM_ERR_OOM, "twiddle table allocation failed");
  CMM_CUDA(cudaMemcpy(op->tw, h.data(), sizeof(V2<T>) * l.total, cudaMemcpyHostToDevice));
  return CMM_OK;
}

int op_init_twiddles(cmm_op* op) {
  return op->prec == CMM_PREC_F64 ? init_tw<double>(op) : init_tw<float>(op);
}

template <typename T, int NC>
static int map_to_gather_t(cmm_op* op, const double* m) {
  const long long npix = op->pt->npix;
  const int blocks = (int)std::min<long long>((npix + 255) / 256, 4096);
  k_map_to_gather<T, NC><<<blocks, 256, 0, op->ctx->stream>>>(m, op->pt->mask, op->gather, op->acc,
                                                              op->acc_stride, npix, op->done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_map_to_gather(cmm_op* op, const double* m) {
  const bool f64 = op->prec == CMM_PREC_F64;
  if (op->pt->ncomp == 1) return f64 ? map_to_gather_t<double, 1>(op, m) : map_to_gather_t<float, 1>(op, m);
  return f64 ? map_to_gather_t<double, 3>(op, m) : map_to_gather_t<float, 3>(op, m);
}

int launch_acc_to_map(cmm_op* op, double* out) {
  const long long npix = op->pt->npix;
  const int blocks = (int)std::min<long long>((npix + 255) / 256, 4096);
  if (op->pt->ncomp == 1)
    k_acc_to_map<1><<<blocks, 256, 0, op->ctx->stream>>>(op->acc, op->pt->mask, out, op->acc_stride, npix, op->done);
  else
    k_acc_to_map<3><<<blocks, 256, 0, op->ctx->stream>>>(op->acc, op->pt->mask, out, op->acc_stride, npix, op->done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

// pass: 0 = forward (k_tod_fwd), 1 = filter (k_tod_filter), 2 = inverse + binning
// (k_tod_inv_bin); -1 = all three in order.
template <typename T, int NC, int SRC, typename S>
static int apply_chunk_t(cmm_op* op, int d0, int nd, const void* tod, int pass) {
  TodArgs a = make_args(op, d0);
  a.tod = tod;
  cudaStream_t st = op->ctx->stream;
  const size_t smem_t = 2 * sizeof(V2<T>) * ((size_t)a.J << a.logR);
  const size_t smem_f = 4 * sizeof(V2<T>) * (size_t)a.C;
  const dim3 gt(op->C / a.J, nd);
  const dim3 gf(op->R / 2 + 1, nd);
  if (pass < 0 || pass == 0) {
    k_tod_fwd<T, NC, SRC, S><<<gt, 256, smem_t, st>>>(a);
    CMM_LAUNCH_CHECK();
  }
  if (pass < 0 || pass == 1) {
    k_tod_filter<T, S><<<gf, 256, smem_f, st>>>(a);
    CMM_LAUNCH_CHECK();
  }
  if (pass < 0 || pass == 2) {
    k_tod_inv_bin<T, NC, S><<<gt, 256, smem_t, st>>>(a);
    CMM_LAUNCH_CHECK();
  }
  return CMM_OK;
}

template <typename T, int NC, typename S>
static int prepare_t() {
  const int mx = 200 * 1024;
  CMM_CUDA(cudaFuncSetAttribute(k_tod_fwd<T, NC, 0, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CMM_CUDA(cudaFuncSetAttribute(k_tod_fwd<T, NC, 1, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CMM_CUDA(cudaFuncSetAttribute(k_tod_fwd<T, NC, 2, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CMM_CUDA(cudaFuncSetAttribute(k_tod_filter<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CMM_CUDA(cudaFuncSetAttribute(k_tod_inv_bin<T, NC, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  return CMM_OK;
}

template <int NC>
static int prepare_nc(int prec) {
  switch (prec) {
    case CMM_PREC_F64: return prepare_t<double, NC, double2>();
    case CMM_PREC_BF16: return prepare_t<float, NC, __nv_bfloat162>();
    default: return prepare_t<float, NC, float2>();
  }
}

// Opt every kernel of this operator's variant into large dynamic shared memory
// (done once, before any stream capture).
int op_prepare_kernels(cmm_op* op) {
  if (fast_path_ok(op)) CMM_TRY(prepare_fast(op));
  if (op->prec != CMM_PREC_F64) CMM_TRY(prepare_pair(op));
  return op->pt->ncomp == 1 ? prepare_nc<1>(op->prec) : prepare_nc<3>(op->prec);
}

template <int NC, int SRC>
static int apply_chunk_nc(cmm_op* op, int d0, int nd, const void* tod, int pass) {
  switch (op->prec) {
    case CMM_PREC_F64: return apply_chunk_t<double, NC, SRC, double2>(op, d0, nd, tod, pass);
    case CMM_PREC_BF16: return apply_chunk_t<float, NC, SRC, __nv_bfloat162>(op, d0, nd, tod, pass);
    default: return apply_chunk_t<float, NC, SRC, float2>(op, d0, nd, tod, pass);
  }
}

int launch_apply_chunk(cmm_op* op, int d0, int nd, const void* tod, int tod_is_f64, int pass) {
  const int nc = op->pt->ncomp;
  if (!tod && pair_path_ok(op)) return launch_apply_chunk_pair(op, d0, nd, pass);
  if (fast_path_ok(op)) {
    if (op->pt->max_hits <= kF32HitLimit || pass == 0 || pass == 1)
      return launch_apply_chunk_fast(op, d0, nd, tod, tod_is_f64, pass);
    // more samples on one pixel than the FP32 partial map takes: fast forward and
    // filter passes, then the generic binning into the FP64 map (same spectrum layout)
    if (pass < 0) {
      CMM_TRY(launch_apply_chunk_fast(op, d0, nd, tod, tod_is_f64, 0));
      CMM_TRY(launch_apply_chunk_fast(op, d0, nd, tod, tod_is_f64, 1));
    }
    return nc == 1 ? apply_chunk_nc<1, 0>(op, d0, nd, nullptr, 2) : apply_chunk_nc<3, 0>(op, d0, nd, nullptr, 2);
  }
  if (!tod) return nc == 1 ? apply_chunk_nc<1, 0>(op, d0, nd, nullptr, pass) : apply_chunk_nc<3, 0>(op, d0, nd, nullptr, pass);
  if (tod_is_f64) return nc == 1 ? apply_chunk_nc<1, 2>(op, d0, nd, tod, pass) : apply_chunk_nc<3, 2>(op, d0, nd, tod, pass);
  return nc == 1 ? apply_chunk_nc<1, 1>(op, d0, nd, tod, pass) : apply_chunk_nc<3, 1>(op, d0, nd, tod, pass);
}

int launch_generic_fwd_from_tod(cmm_op* op, int d0, int nd, const void* tod, int tod_is_f64) {
  const int nc = op->pt->ncomp;
  if (tod_is_f64) return nc == 1 ? apply_chunk_nc<1, 2>(op, d0, nd, tod, 0) : apply_chunk_nc<3, 2>(op, d0, nd, tod, 0);
  return nc == 1 ? apply_chunk_nc<1, 1>(op, d0, nd, tod, 0) : apply_chunk_nc<3, 1>(op, d0, nd, tod, 0);
}

template <typename T, int NC>
static int project_t(cmm_op* op, void* tod, int tod_is_f64) {
  TodArgs a = make_args(op, 0);
  const long long n_t = op->pt->n_t;
  const int bx = (int)std::min<long long>((n_t + 255) / 256, 1024);
  dim3 g(bx, op->pt->n_det);
  if (tod_is_f64)
    k_project<T, NC, double><<<g, 256, 0, op->ctx->stream>>>(a, (double*)tod);
  else
    k_project<T, NC, float><<<g, 256, 0, op->ctx->stream>>>(a, (float*)tod);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_project(cmm_op* op, const double* m, void* tod, int tod_is_f64) {
  CMM_TRY(launch_map_to_gather(op, m));
  const bool f64 = op->prec == CMM_PREC_F64;
  if (op->pt->ncomp == 1) return f64 ? project_t<double, 1>(op, tod, tod_is_f64) : project_t<float, 1>(op, tod, tod_is_f64);
  return f64 ? project_t<double, 3>(op, tod, tod_is_f64) : project_t<float, 3>(op, tod, tod_is_f64);
}

int launch_hit_blocks(cmm_pointing* pt, const double* det_weight, const uint8_t* mask, double* blocks,
                      const int* done) {
  const long long n_t = pt->n_t;
  const int bx = (int)std::min<long long>((n_t + 255) / 256, 1024);
  dim3 g(bx, pt->n_det);
  cudaStream_t st = pt->ctx->stream;
  if (pt->ncomp == 1)
    k_hit_blocks<1><<<g, 256, 0, st>>>(pt->bore, pt->det_off, pt->det_pol64, pt->ny, pt->nx, pt->periodic,
                                       n_t, det_weight, mask, blocks, done);
  else
    k_hit_blocks<3><<<g, 256, 0, st>>>(pt->bore, pt->det_off, pt->det_pol64, pt->ny, pt->nx, pt->periodic,
                                       n_t, det_weight, mask, blocks, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

}  // namespace cmm
