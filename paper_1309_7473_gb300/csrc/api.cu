// Host runtime and C ABI of the map-maker (include/cmm.h).
#include <math.h>

#include <cmath>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "map_kernels.cuh"

// ------------------------------------------------------------------ errors
namespace cmm {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  g_err = std::string(cudaGetErrorString(e)) + " in " + what + " (" + file + ":" + std::to_string(line) + ")";
  return e == cudaErrorMemoryAllocation ? CMM_ERR_OOM : CMM_ERR_CUDA;
}

template <typename P>
static int dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CMM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  return CMM_OK;
}

static void dfree(void* p) {
  if (p) cudaFree(p);
}


// diag(N^-1) per detector: deterministic FP64 sum of w over the two-sided grid
__global__ void k_noise_diag(const double4_32a* __restrict__ coef, long long n_t, double* __restrict__ out) {
  const int d = blockIdx.x;
  const double4_32a cf = coef[d];
  const long long N = n_t / 2;
  double acc = 0.0;
  for (long long k = threadIdx.x; k <= N; k += blockDim.x) {
    double w;
    if (cf.w != 0.0) {
      w = cf.x;
    } else {
      const double kk = (double)(k == 0 ? 1 : k);
      w = cf.x / (1.0 + exp2(fma(-cf.y, log2(kk), cf.z)));
    }
    acc += (k == 0 || k == N) ? w : 2.0 * w;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[d] = sh[0] / (double)n_t;
}

// (cos 2phi, sin 2phi) per sample, phi the angle of the 2^-15 fixed-point rotation
// pair (c, s): the double angle of the normalised pair, (c^2 - s^2, 2 c s) / (c^2 + s^2),
// in FP64 (the integer products are exact), stored in FP32.
__global__ void k_rot2(const int4* __restrict__ bore, long long n, float2* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int4 b = bore[t];
    const double cf = (double)b.z, sf = (double)b.w;
    const double r2 = cf * cf + sf * sf;
    out[t] = make_float2((float)((cf * cf - sf * sf) / r2), (float)(2.0 * cf * sf / r2));
  }
}

__global__ void k_set_unit(double* __restrict__ v, long long idx) { v[idx] = 1.0; }

}  // namespace cmm

extern "C" {
static void free_ctx(cmm_ctx* c);
}

namespace cmm {
void ctx_retain(cmm_ctx* c) { c->refs++; }
void ctx_release(cmm_ctx* c) {
  if (--c->refs == 0) free_ctx(c);
}

// inputs = z / ||z||, targets = (x* - x_k - z) / ||z|| (FP32), ||z||^2 from partials
__global__ void k_pair(const double* __restrict__ z, const double* __restrict__ xs, const double* __restrict__ xk,
                       const double* __restrict__ partial, float* __restrict__ in, float* __restrict__ tgt, long long n) {
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kRedBlocks; ++k) s += partial[k];
    s_inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    in[t] = (float)(z[t] * s_inv);
    tgt[t] = (float)((xs[t] - xk[t] - z[t]) * s_inv);
  }
}

}  // namespace cmm

using namespace cmm;

struct cmm_precon {
  int refs = 1;
  cmm_op* op = nullptr;
  int kind = 0;
  double* inv = nullptr;       // binned / Jacobi: inverse blocks
  double* sig = nullptr;       // circulant: Sigma
  double* sig_inv = nullptr;   // circulant: Sigma^-1
  float* sig_inv32 = nullptr;  // its FP32 copy, for the apply of FP32/BF16 operators
  double* hinv = nullptr;      // circulant: per-mode packed inverse
  float* hinv32 = nullptr;     // its FP32 copy, applied with the FP32 map FFTs of FP32/BF16 operators
  void* planes = nullptr;      // complex workspace [ncomp][npix]
  double* tmp = nullptr;       // [ncomp * npix]
  Fft2Plan plan;
  int64_t n_clamped = 0;
  int64_t ref = -1;
  double taper = 0.0;
  cmm_unet* unet = nullptr;    // learned correction (CIRC_LEARNED)
  std::vector<cmm_precon*> parts;   // CIRC_TILED: one circulant per tile
  double* sqrt_phi = nullptr;  // CIRC_TILED: [tiles][npix] square roots of the partition of unity
  double* ttmp = nullptr;      // CIRC_TILED: [2][ncomp * npix]
};

extern "C" {

const char* cmm_last_error(void) { return g_err.c_str(); }

const char* cmm_version(void) { return "cmm 0.1 (sm_103a)"; }

int cmm_ctx_create(int device, void* stream, cmm_ctx** out) {
  if (!out) return fail(CMM_ERR_ARG, "out is null");
  *out = nullptr;
  int n = 0;
  CMM_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(CMM_ERR_ARG, "bad device index");
  CMM_CUDA(cudaSetDevice(device));
  cmm_ctx* c = new cmm_ctx();
  c->device = device;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
    }
    c->own_stream = true;
  }
  int s = dalloc(&c->d_partial, sizeof(double) * (kRedBlocks + 16));
  if (s == CMM_OK) s = dalloc(&c->d_scalar, sizeof(double) * 16);
  if (s == CMM_OK && cudaMallocHost(&c->h_scalar, sizeof(double) * 64) != cudaSuccess) s = fail(CMM_ERR_OOM, "pinned alloc");
  if (s != CMM_OK) {
    cmm_ctx_destroy(c);
    return s;
  }
  *out = c;
  return CMM_OK;
}

static void free_ctx(cmm_ctx* c) {
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  dfree(c->d_partial);
  dfree(c->d_scalar);
  if (c->h_scalar) cudaFreeHost(c->h_scalar);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int cmm_ctx_destroy(cmm_ctx* c) {
  if (c) ctx_release(c);
  return CMM_OK;
}

// ------------------------------------------------------------------ pointing
static void free_pointing(cmm_pointing* pt) {
  cudaSetDevice(pt->ctx->device);
  cudaStreamSynchronize(pt->ctx->stream);
  dfree(pt->bore);
  dfree(pt->det_off);
  dfree(pt->det_pol64);
  dfree(pt->det_pol32);
  dfree(pt->rot2);
  dfree(pt->mask);
  cmm_ctx* c = pt->ctx;
  delete pt;
  ctx_release(c);
}

static void pointing_release(cmm_pointing* pt) {
  if (--pt->refs == 0) free_pointing(pt);
}

int cmm_pointing_destroy(cmm_pointing* pt) {
  if (pt) pointing_release(pt);
  return CMM_OK;
}

int cmm_pointing_create(cmm_ctx* ctx, const cmm_map_geom* geom, int32_t n_det, const int32_t* det_off,
                        const double* det_pol, int64_t n_samp, const int32_t* bore, cmm_pointing** out) {
  if (!ctx || !geom || !det_off || !det_pol || !bore || !out) return fail(CMM_ERR_ARG, "null argument");
  *out = nullptr;
  // 4 (npix + 1) accumulator entries must stay below 2^31 for the kernels' 32-bit indices
  if (geom->ny <= 0 || geom->nx <= 0 || (long long)geom->ny * geom->nx > (1LL << 28))
    return fail(CMM_ERR_ARG, "bad map size (1 <= ny * nx <= 2^28)");
  if (geom->ncomp != 1 && geom->ncomp != 3) return fail(CMM_ERR_ARG, "ncomp must be 1 or 3");
  if (n_det <= 0 || n_samp <= 0 || n_det > 65535) return fail(CMM_ERR_ARG, "bad detector or sample count");
  // ranges under which the fixed-point pointing is exact in int32
  for (int d = 0; d < n_det; ++d)
    if (std::abs((long long)det_off[2 * d]) >= (1 << 14) || std::abs((long long)det_off[2 * d + 1]) >= (1 << 14))
      return fail(CMM_ERR_ARG, "detector offset out of range (|dx|, |dy| < 2^14)");
  for (int64_t t = 0; t < n_samp; ++t) {
    const int32_t* b = bore + 4 * t;
    if (std::abs((long long)b[0]) > (1LL << 30) - (1LL << 25) || std::abs((long long)b[1]) > (1LL << 30) - (1LL << 25) ||
        std::abs((long long)b[2]) > (1 << 15) || std::abs((long long)b[3]) > (1 << 15))
      return fail(CMM_ERR_ARG, "boresight entry out of range");
  }
  CMM_CUDA(cudaSetDevice(ctx->device));
  cmm_pointing* pt = new cmm_pointing();
  pt->ctx = ctx;
  ctx_retain(ctx);
  pt->ny = geom->ny;
  pt->nx = geom->nx;
  pt->ncomp = geom->ncomp;
  pt->periodic = geom->periodic ? 1 : 0;
  pt->n_det = n_det;
  pt->n_t = n_samp;
  pt->npix = (int64_t)geom->ny * geom->nx;
  std::vector<float2> pol32(n_det);
  for (int d = 0; d < n_det; ++d) pol32[d] = float2{(float)det_pol[2 * d], (float)det_pol[2 * d + 1]};
  double* blocks = nullptr;
  const int nb = pt->ncomp == 1 ? 1 : 6;
  int s = dalloc(&pt->bore, sizeof(int4) * n_samp);
  if (s == CMM_OK) s = dalloc(&pt->det_off, sizeof(int2) * n_det);
  if (s == CMM_OK) s = dalloc(&pt->det_pol64, sizeof(double2) * n_det);
  if (s == CMM_OK) s = dalloc(&pt->det_pol32, sizeof(float2) * n_det);
  if (s == CMM_OK) s = dalloc(&pt->mask, pt->npix);
  if (s == CMM_OK) s = dalloc(&pt->rot2, sizeof(float2) * n_samp);
  if (s == CMM_OK) s = dalloc(&blocks, sizeof(double) * nb * pt->npix);
  if (s != CMM_OK) {
    dfree(blocks);
    cmm_pointing_destroy(pt);
    return s;
  }
  cudaStream_t st = ctx->stream;
  auto run = [&]() -> int {
    CMM_CUDA(cudaMemcpyAsync(pt->bore, bore, sizeof(int4) * n_samp, cudaMemcpyHostToDevice, st));
    CMM_CUDA(cudaMemcpyAsync(pt->det_off, det_off, sizeof(int2) * n_det, cudaMemcpyHostToDevice, st));
    CMM_CUDA(cudaMemcpyAsync(pt->det_pol64, det_pol, sizeof(double2) * n_det, cudaMemcpyHostToDevice, st));
    CMM_CUDA(cudaMemcpyAsync(pt->det_pol32, pol32.data(), sizeof(float2) * n_det, cudaMemcpyHostToDevice, st));
    k_rot2<<<(int)std::min<long long>((n_samp + 255) / 256, 4096), 256, 0, st>>>(pt->bore, n_samp, pt->rot2);
    CMM_LAUNCH_CHECK();
    CMM_CUDA(cudaMemsetAsync(blocks, 0, sizeof(double) * nb * pt->npix, st));
    CMM_TRY(launch_hit_blocks(pt, nullptr, nullptr, blocks, nullptr));
    CMM_TRY(launch_mask_from_hits(pt, blocks));
    CMM_CUDA(cudaStreamSynchronize(st));
    return CMM_OK;
  };
  s = run();
  dfree(blocks);
  if (s != CMM_OK) {
    cmm_pointing_destroy(pt);
    return s;
  }
  *out = pt;
  return CMM_OK;
}

int cmm_pointing_mask(cmm_pointing* pt, uint8_t* mask_host, int64_t* n_good) {
  if (!pt) return fail(CMM_ERR_ARG, "null pointing");
  CMM_CUDA(cudaSetDevice(pt->ctx->device));
  if (mask_host) {
    CMM_CUDA(cudaMemcpyAsync(mask_host, pt->mask, pt->npix, cudaMemcpyDeviceToHost, pt->ctx->stream));
    CMM_CUDA(cudaStreamSynchronize(pt->ctx->stream));
  }
  if (n_good) *n_good = pt->n_good;
  return CMM_OK;
}

// ------------------------------------------------------------------ noise
static void free_noise(cmm_noise* nz) {
  cudaSetDevice(nz->ctx->device);
  cudaStreamSynchronize(nz->ctx->stream);
  dfree(nz->coef64);
  dfree(nz->coef32);
  dfree(nz->diag);
  dfree(nz->white);
  dfree(nz->corr_V);
  dfree(nz->corr_par);
  dfree(nz->wtab64);
  dfree(nz->wtab32);
  cmm_ctx* c = nz->ctx;
  delete nz;
  ctx_release(c);
}

static void noise_release(cmm_noise* nz) {
  if (--nz->refs == 0) free_noise(nz);
}

int cmm_noise_destroy(cmm_noise* nz) {
  if (nz) noise_release(nz);
  return CMM_OK;
}

int cmm_noise_create(cmm_ctx* ctx, int32_t n_det, int64_t n_samp, double f_samp, const double* sigma,
                     const double* fknee, const double* alpha, cmm_noise** out) {
  if (!ctx || !sigma || !fknee || !alpha || !out) return fail(CMM_ERR_ARG, "null argument");
  *out = nullptr;
  if (n_det <= 0 || n_samp < 2 || !(f_samp > 0)) return fail(CMM_ERR_ARG, "bad noise sizes");
  std::vector<double4_32a> c64(n_det);
  std::vector<float4> c32(n_det);
  std::vector<double> white(n_det);
  for (int d = 0; d < n_det; ++d) {
    if (!(sigma[d] > 0) || fknee[d] < 0 || !std::isfinite(alpha[d])) return fail(CMM_ERR_ARG, "bad noise parameter");
    const double iv = 1.0 / (sigma[d] * sigma[d]);
    white[d] = iv;
    if (fknee[d] == 0.0) {
      c64[d] = double4_32a{iv, 0.0, 0.0, 1.0};
    } else {
      const double sc = f_samp / ((double)n_samp * fknee[d]);
      c64[d] = double4_32a{iv, alpha[d], -alpha[d] * std::log2(sc), 0.0};
    }
    c32[d] = float4{(float)c64[d].x, (float)c64[d].y, (float)c64[d].z, (float)c64[d].w};
  }
  CMM_CUDA(cudaSetDevice(ctx->device));
  cmm_noise* nz = new cmm_noise();
  nz->ctx = ctx;
  ctx_retain(ctx);
  nz->n_det = n_det;
  nz->n_t = n_samp;
  nz->f_samp = f_samp;
  int s = dalloc(&nz->coef64, sizeof(double4_32a) * n_det);
  if (s == CMM_OK) s = dalloc(&nz->coef32, sizeof(float4) * n_det);
  if (s == CMM_OK) s = dalloc(&nz->diag, sizeof(double) * n_det);
  if (s == CMM_OK) s = dalloc(&nz->white, sizeof(double) * n_det);
  if (s != CMM_OK) {
    cmm_noise_destroy(nz);
    return s;
  }
  auto run = [&]() -> int {
    cudaStream_t st = ctx->stream;
    CMM_CUDA(cudaMemcpyAsync(nz->coef64, c64.data(), sizeof(double4_32a) * n_det, cudaMemcpyHostToDevice, st));
    CMM_CUDA(cudaMemcpyAsync(nz->coef32, c32.data(), sizeof(float4) * n_det, cudaMemcpyHostToDevice, st));
    CMM_CUDA(cudaMemcpyAsync(nz->white, white.data(), sizeof(double) * n_det, cudaMemcpyHostToDevice, st));
    k_noise_diag<<<n_det, 256, 0, st>>>(nz->coef64, n_samp, nz->diag);
    CMM_LAUNCH_CHECK();
    nz->diag_host.resize(n_det);
    CMM_CUDA(cudaMemcpyAsync(nz->diag_host.data(), nz->diag, sizeof(double) * n_det, cudaMemcpyDeviceToHost, st));
    CMM_CUDA(cudaStreamSynchronize(st));
    return CMM_OK;
  };
  s = run();
  if (s != CMM_OK) {
    cmm_noise_destroy(nz);
    return s;
  }
  *out = nz;
  return CMM_OK;
}

int cmm_noise_diag(cmm_noise* nz, double* diag_host) {
  if (!nz || !diag_host) return fail(CMM_ERR_ARG, "null argument");
  std::memcpy(diag_host, nz->diag_host.data(), sizeof(double) * nz->n_det);
  return CMM_OK;
}

// ------------------------------------------------------------------ operator
static void free_op(cmm_op* op) {
  cudaSetDevice(op->ctx->device);
  cudaStreamSynchronize(op->ctx->stream);
  dfree(op->spec);
  dfree(op->gather);
  dfree(op->acc);
  dfree(op->acc32);
  dfree(op->tw);
  dfree(op->tw_pair);
  dfree(op->tmp_a);
  dfree(op->tmp_b);
  dfree(op->pix);
  dfree(op->corr_minv);
  dfree(op->corr_s);
  dfree(op->sol);
  dfree(op->sol_state);
  dfree(op->host_bx);
  dfree(op->fcg);
  cmm_ctx* c = op->ctx;
  cmm_pointing* pt = op->pt;
  cmm_noise* nz = op->nz;
  delete op;
  pointing_release(pt);
  noise_release(nz);
  ctx_release(c);
}

static void op_release(cmm_op* op) {
  if (--op->refs == 0) free_op(op);
}

int cmm_op_destroy(cmm_op* op) {
  if (op) op_release(op);
  return CMM_OK;
}

int cmm_op_create(cmm_ctx* ctx, cmm_pointing* pt, cmm_noise* nz, int32_t precision, int32_t det_chunk,
                  cmm_op** out) {
  if (!ctx || !pt || !nz || !out) return fail(CMM_ERR_ARG, "null argument");
  *out = nullptr;
  if (pt->n_det != nz->n_det || pt->n_t != nz->n_t) return fail(CMM_ERR_ARG, "pointing and noise sizes differ");
  if (precision < CMM_PREC_F64 || precision > CMM_PREC_BF16) return fail(CMM_ERR_ARG, "bad precision");
  const int64_t n_t = pt->n_t;
  if (n_t < 32 || n_t > (1LL << 22) || (n_t & (n_t - 1)))
    return fail(CMM_ERR_UNSUPPORTED, "n_samp must be a power of two in [32, 2^22]");
  CMM_CUDA(cudaSetDevice(ctx->device));
  cmm_op* op = new cmm_op();
  op->ctx = ctx;
  op->pt = pt;
  op->nz = nz;
  ctx_retain(ctx);
  pt->refs++;
  nz->refs++;
  op->prec = precision;
  op->N = n_t / 2;
  int logN = 0;
  while ((1LL << logN) < op->N) ++logN;
  if (!fast_path_sizes(logN, precision, &op->logR, &op->logC)) {
    op->logR = logN / 2;
    op->logC = logN - op->logR;
  }
  op->R = 1 << op->logR;
  op->C = 1 << op->logC;
  const size_t elt = precision == CMM_PREC_F64 ? 16 : (precision == CMM_PREC_BF16 ? 4 : 8);
  const size_t per_det = elt * (size_t)op->N;
  int chunk = det_chunk > 0 ? det_chunk : (int)std::max<size_t>(1, (size_t(8) << 30) / per_det);
  chunk = std::min(chunk, pt->n_det);
  op->chunk = chunk;
  const int64_t npix = pt->npix;
  const int nc = pt->ncomp;
  op->acc_stride = nc == 1 ? 1 : 4;
  const size_t gel = precision == CMM_PREC_F64 ? 8 : 4;
  // an even number of detector slots: the two-detector path fills whole pairs
  int s = dalloc(&op->spec, per_det * (chunk + (chunk & 1)));
  // map-sized buffers carry one extra pixel (index npix): the fast kernels send
  // samples outside the map there (zero in the gather copy, never read back)
  if (s == CMM_OK) s = dalloc(&op->gather, gel * (nc == 1 ? 1 : 4) * (npix + 1));
  if (s == CMM_OK) s = dalloc(&op->acc, sizeof(double) * op->acc_stride * (npix + 1));
  // one FP32 partial map per group of kFlushDets detectors of a chunk (at most
  // kMaxPartialMaps): the two-detector path bins a whole chunk in one launch
  op->acc32_maps = precision == CMM_PREC_F64 ? 1 : std::max(1, std::min(kMaxPartialMaps, (chunk + kFlushDets - 1) / kFlushDets));
  const size_t acc32_elems = (size_t)op->acc32_maps * op->acc_stride * (npix + 1);
  if (s == CMM_OK) s = dalloc(&op->acc32, sizeof(float) * acc32_elems);
  if (s == CMM_OK) s = (cudaMemset(op->acc32, 0, sizeof(float) * acc32_elems) == cudaSuccess) ? CMM_OK : fail(CMM_ERR_CUDA, "memset");
  if (s == CMM_OK) s = dalloc(&op->tmp_a, sizeof(double) * nc * npix);
  if (s == CMM_OK) s = dalloc(&op->tmp_b, sizeof(double) * nc * npix);
  if (s == CMM_OK) s = op_init_twiddles(op);
  if (s == CMM_OK) s = op_prepare_kernels(op);
  if (s != CMM_OK) {
    cmm_op_destroy(op);
    return s;
  }
  *out = op;
  return CMM_OK;
}

// Re-split N = R C (logR given) for the time-ordered FFTs: new twiddle tables and
// kernel attributes.  The spectrum buffer holds N complex per detector either way.
static int op_set_split(cmm_op* op, int logR) {
  const int logN = op->logR + op->logC;
  if (logR < 1 || logR >= logN) return fail(CMM_ERR_ARG, "bad split");
  if (op->tw) {
    CMM_CUDA(cudaStreamSynchronize(op->ctx->stream));
    dfree(op->tw);
    op->tw = nullptr;
  }
  op->logR = logR;
  op->logC = logN - logR;
  op->R = 1 << op->logR;
  op->C = 1 << op->logC;
  op->corr_version = -1;   // the correlated-noise tables are in the old split's slot order
  CMM_TRY(op_init_twiddles(op));
  return op_prepare_kernels(op);
}

int cmm_noise_set_table(cmm_noise* nz, const double* w_host) {
  if (!nz) return fail(CMM_ERR_ARG, "null argument");
  const int64_t K = nz->n_t / 2 + 1;
  const int n_det = nz->n_det;
  if (w_host)
    for (int64_t q = 0; q < (int64_t)n_det * K; ++q)
      if (!(w_host[q] >= 0) || !std::isfinite(w_host[q])) return fail(CMM_ERR_ARG, "weights must be finite and >= 0");
  CMM_CUDA(cudaSetDevice(nz->ctx->device));
  cudaStream_t st = nz->ctx->stream;
  CMM_CUDA(cudaStreamSynchronize(st));
  dfree(nz->wtab64);
  dfree(nz->wtab32);
  nz->wtab64 = nullptr;
  nz->wtab32 = nullptr;
  nz->corr_version++;   // correlated-noise tables depend on the weights
  std::vector<double> diag(n_det);
  if (!w_host) {
    k_noise_diag<<<n_det, 256, 0, st>>>(nz->coef64, nz->n_t, nz->diag);
    CMM_LAUNCH_CHECK();
    CMM_CUDA(cudaMemcpyAsync(nz->diag_host.data(), nz->diag, sizeof(double) * n_det, cudaMemcpyDeviceToHost, st));
    CMM_CUDA(cudaStreamSynchronize(st));
    return CMM_OK;
  }
  std::vector<float> w32((size_t)n_det * K);
  for (int d = 0; d < n_det; ++d) {
    const double* w = w_host + (size_t)d * K;
    double inner = 0.0;   // R3: mean of w over the full two-sided grid
    for (int64_t k = 1; k < K - 1; ++k) inner += w[k];
    diag[d] = (w[0] + 2.0 * inner + w[K - 1]) / (double)nz->n_t;
    for (int64_t k = 0; k < K; ++k) w32[(size_t)d * K + k] = (float)w[k];
  }
  CMM_TRY(dalloc(&nz->wtab64, sizeof(double) * (size_t)n_det * K));
  CMM_TRY(dalloc(&nz->wtab32, sizeof(float) * (size_t)n_det * K));
  CMM_CUDA(cudaMemcpy(nz->wtab64, w_host, sizeof(double) * (size_t)n_det * K, cudaMemcpyHostToDevice));
  CMM_CUDA(cudaMemcpy(nz->wtab32, w32.data(), sizeof(float) * (size_t)n_det * K, cudaMemcpyHostToDevice));
  CMM_CUDA(cudaMemcpy(nz->diag, diag.data(), sizeof(double) * n_det, cudaMemcpyHostToDevice));
  nz->diag_host = diag;
  return CMM_OK;
}

int cmm_noise_set_correlated(cmm_noise* nz, int32_t r, const double* modes, const double* amp, const double* fknee,
                             const double* alpha) {
  if (!nz || r < 0 || r > kMaxCorrModes) return fail(CMM_ERR_ARG, "bad noise handle or mode count (0..4)");
  if (r > 0 && (!modes || !amp || !fknee || !alpha)) return fail(CMM_ERR_ARG, "null argument");
  for (int j = 0; j < r; ++j)
    if (!(amp[j] >= 0) || !(fknee[j] > 0) || !std::isfinite(alpha[j])) return fail(CMM_ERR_ARG, "bad mode parameter");
  CMM_CUDA(cudaSetDevice(nz->ctx->device));
  CMM_CUDA(cudaStreamSynchronize(nz->ctx->stream));
  dfree(nz->corr_V);
  dfree(nz->corr_par);
  nz->corr_V = nullptr;
  nz->corr_par = nullptr;
  nz->corr_r = 0;
  nz->corr_version++;
  if (r == 0) return CMM_OK;
  std::vector<float> v((size_t)nz->n_det * r);
  for (size_t q = 0; q < v.size(); ++q) v[q] = (float)modes[q];
  std::vector<double> par(3 * r);
  for (int j = 0; j < r; ++j) {
    par[3 * j] = amp[j];
    par[3 * j + 1] = fknee[j];
    par[3 * j + 2] = alpha[j];
  }
  CMM_TRY(dalloc(&nz->corr_V, sizeof(float) * v.size()));
  CMM_TRY(dalloc(&nz->corr_par, sizeof(double) * par.size()));
  CMM_CUDA(cudaMemcpy(nz->corr_V, v.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice));
  CMM_CUDA(cudaMemcpy(nz->corr_par, par.data(), sizeof(double) * par.size(), cudaMemcpyHostToDevice));
  nz->corr_r = r;
  return CMM_OK;
}

int cmm_op_set_pixel_cache(cmm_op* op, int32_t enable) {
  if (!op) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  if (!enable) {
    if (op->pix) {
      CMM_CUDA(cudaStreamSynchronize(op->ctx->stream));
      dfree(op->pix);
      op->pix = nullptr;
    }
    return CMM_OK;
  }
  if (op->pix) return CMM_OK;
  if (!fast_path_ok(op) || op->pt->periodic)
    return fail(CMM_ERR_UNSUPPORTED, "the pixel cache needs the FP32/BF16 fast path and a non-periodic map");
  const size_t bytes = sizeof(int32_t) * (size_t)op->pt->n_det * (size_t)op->pt->n_t;
  CMM_TRY(dalloc(&op->pix, bytes));
  const int s = launch_fill_pixels(op);
  if (s != CMM_OK) {
    dfree(op->pix);
    op->pix = nullptr;
  }
  return s;
}

int cmm_op_set_pair_packing(cmm_op* op, int32_t enable) {
  if (!op) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  CMM_CUDA(cudaStreamSynchronize(op->ctx->stream));
  op->pair = enable ? 1 : 0;
  return CMM_OK;
}

}  // extern "C"

namespace cmm {
// Brings the operator's correlated-noise tables up to its noise's current model
// (allocates; call before any stream capture).
int op_sync_corr(cmm_op* op) {
  cmm_noise* nz = op->nz;
  if (op->corr_version == nz->corr_version) return CMM_OK;
  CMM_CUDA(cudaStreamSynchronize(op->ctx->stream));
  dfree(op->corr_minv);
  dfree(op->corr_s);
  op->corr_minv = nullptr;
  op->corr_s = nullptr;
  if (nz->corr_r > 0) {
    if (!fast_path_ok(op))
      return fail(CMM_ERR_UNSUPPORTED, "correlated noise needs the FP32/BF16 operator at a fast-path size");
    if (op->chunk < op->pt->n_det)
      return fail(CMM_ERR_UNSUPPORTED, "correlated noise needs every detector in one chunk (det_chunk)");
    const int r = nz->corr_r;
    CMM_TRY(dalloc(&op->corr_minv, sizeof(float) * (size_t)(op->N + 1) * r * r));
    CMM_TRY(dalloc(&op->corr_s, sizeof(float2) * (size_t)op->N * r));
    CMM_TRY(launch_corr_minv(op, nz->corr_par, op->corr_minv));
    CMM_CUDA(cudaStreamSynchronize(op->ctx->stream));
  }
  op->corr_version = nz->corr_version;
  return CMM_OK;
}
}  // namespace cmm

extern "C" {

static int apply_A_dev(cmm_op* op, const double* m_in, double* m_out) {
  TraceRange tr("cmm: A = P^T N^-1 P");
  CMM_TRY(launch_map_to_gather(op, m_in));
  for (int d0 = 0; d0 < op->pt->n_det; d0 += op->chunk) {
    const int nd = std::min(op->chunk, op->pt->n_det - d0);
    CMM_TRY(launch_apply_chunk(op, d0, nd, nullptr, 0));
  }
  return launch_acc_to_map(op, m_out);
}

int cmm_apply_A(cmm_op* op, const double* m_in, double* m_out) {
  if (!op || !m_in || !m_out) return fail(CMM_ERR_ARG, "null argument");
  if (m_in == m_out) return fail(CMM_ERR_ARG, "m_in and m_out must not alias");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  CMM_TRY(op_sync_corr(op));
  return apply_A_dev(op, m_in, m_out);
}

int cmm_profile_apply(cmm_op* op, const double* m_in, double* m_out, int32_t reps, double* ms_host) {
  if (!op || !m_in || !m_out || !ms_host || reps <= 0) return fail(CMM_ERR_ARG, "bad argument");
  if (m_in == m_out) return fail(CMM_ERR_ARG, "m_in and m_out must not alias");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  CMM_TRY(op_sync_corr(op));
  cudaStream_t st = op->ctx->stream;
  const int nchunk = (op->pt->n_det + op->chunk - 1) / op->chunk;
  const int nev = 2 + reps * (1 + 3 * nchunk + 1);
  std::vector<cudaEvent_t> ev(nev, nullptr);
  for (auto& e : ev) CMM_CUDA(cudaEventCreate(&e));
  int s = [&]() -> int {
    int k = 0;
    CMM_CUDA(cudaEventRecord(ev[k++], st));
    for (int r = 0; r < reps; ++r) {
      CMM_TRY(launch_map_to_gather(op, m_in));
      CMM_CUDA(cudaEventRecord(ev[k++], st));
      for (int d0 = 0; d0 < op->pt->n_det; d0 += op->chunk) {
        const int nd = std::min(op->chunk, op->pt->n_det - d0);
        for (int pass = 0; pass < 3; ++pass) {
          CMM_TRY(launch_apply_chunk(op, d0, nd, nullptr, 0, pass));
          CMM_CUDA(cudaEventRecord(ev[k++], st));
        }
      }
      CMM_TRY(launch_acc_to_map(op, m_out));
      CMM_CUDA(cudaEventRecord(ev[k++], st));
    }
    CMM_CUDA(cudaEventRecord(ev[k++], st));
    CMM_CUDA(cudaEventSynchronize(ev[k - 1]));
    double acc[5] = {0, 0, 0, 0, 0};
    float t = 0;
    k = 1;
    for (int r = 0; r < reps; ++r) {
      CMM_CUDA(cudaEventElapsedTime(&t, ev[k - 1], ev[k]));
      acc[3] += t;  // gather copy + accumulator clear
      ++k;
      for (int c = 0; c < nchunk; ++c)
        for (int pass = 0; pass < 3; ++pass) {
          CMM_CUDA(cudaEventElapsedTime(&t, ev[k - 1], ev[k]));
          acc[pass] += t;
          ++k;
        }
      CMM_CUDA(cudaEventElapsedTime(&t, ev[k - 1], ev[k]));
      acc[3] += t;
      ++k;
    }
    CMM_CUDA(cudaEventElapsedTime(&t, ev[0], ev[k]));
    acc[4] = t;
    for (int i = 0; i < 3; ++i) ms_host[i] = acc[i] / (reps * nchunk);
    ms_host[3] = acc[3] / reps;
    ms_host[4] = acc[4] / reps;
    return CMM_OK;
  }();
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return s;
}

int cmm_apply_A_host(cmm_op* op, const double* m_in_host, double* m_out_host) {
  if (!op || !m_in_host || !m_out_host) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  CMM_TRY(op_sync_corr(op));
  const size_t bytes = sizeof(double) * op->pt->ncomp * op->pt->npix;
  cudaStream_t st = op->ctx->stream;
  CMM_CUDA(cudaMemcpyAsync(op->tmp_a, m_in_host, bytes, cudaMemcpyHostToDevice, st));
  CMM_TRY(apply_A_dev(op, op->tmp_a, op->tmp_b));
  CMM_CUDA(cudaMemcpyAsync(m_out_host, op->tmp_b, bytes, cudaMemcpyDeviceToHost, st));
  CMM_CUDA(cudaStreamSynchronize(st));
  return CMM_OK;
}

int cmm_project(cmm_op* op, const double* m, void* tod, int32_t tod_is_f64) {
  if (!op || !m || !tod) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  return launch_project(op, m, tod, tod_is_f64);
}

int cmm_rhs(cmm_op* op, const void* tod, int32_t tod_is_f64, double* b) {
  TraceRange tr("cmm: rhs P^T N^-1 d");
  if (!op || !tod || !b) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  CMM_TRY(op_sync_corr(op));
  CMM_CUDA(cudaMemsetAsync(op->acc, 0, sizeof(double) * op->acc_stride * op->pt->npix, op->ctx->stream));
  for (int d0 = 0; d0 < op->pt->n_det; d0 += op->chunk) {
    const int nd = std::min(op->chunk, op->pt->n_det - d0);
    CMM_TRY(launch_apply_chunk(op, d0, nd, tod, tod_is_f64));
  }
  return launch_acc_to_map(op, b);
}

int cmm_dot(cmm_op* op, const double* x, const double* y, int64_t n, double* result_host) {
  if (!op || !x || !y || !result_host || n < 0) return fail(CMM_ERR_ARG, "bad argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  cmm_ctx* c = op->ctx;
  CMM_TRY(launch_dot(x, y, n, c->d_partial, c->d_scalar, nullptr, c->stream));
  CMM_CUDA(cudaMemcpyAsync(c->h_scalar, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CMM_CUDA(cudaStreamSynchronize(c->stream));
  *result_host = c->h_scalar[0];
  return CMM_OK;
}

// ------------------------------------------------------------------ preconditioners
int cmm_precon_destroy(cmm_precon* pc) {
  if (!pc) return CMM_OK;
  if (--pc->refs > 0) return CMM_OK;
  cudaSetDevice(pc->op->ctx->device);
  cudaStreamSynchronize(pc->op->ctx->stream);
  dfree(pc->inv);
  dfree(pc->sig);
  dfree(pc->sig_inv);
  dfree(pc->sig_inv32);
  dfree(pc->hinv);
  dfree(pc->hinv32);
  dfree(pc->planes);
  dfree(pc->tmp);
  dfree(pc->plan.tw);
  dfree(pc->sqrt_phi);
  dfree(pc->ttmp);
  for (cmm_precon* q : pc->parts) cmm_precon_destroy(q);
  cmm_op* op = pc->op;
  cmm_unet* net = pc->unet;
  delete pc;
  if (net) unet_release(net);
  op_release(op);
  return CMM_OK;
}

}  // extern "C"

// Raised-cosine windows on n pixels, t of them, summing to 1 (centres (i + 1/2) n/t,
// half-width n/t, the outer ones held at 1 towards the edges).
static std::vector<double> tile_windows_1d(int n, int t) {
  std::vector<double> w((size_t)t * n, 0.0);
  const double h = (double)n / t;
  for (int i = 0; i < t; ++i) {
    const double c = (i + 0.5) * h;
    for (int y = 0; y < n; ++y) {
      const double u = (y - c) / h;
      double v = std::fabs(u) <= 1.0 ? std::pow(std::cos(0.5 * M_PI * u), 2) : 0.0;
      if (i == 0 && y <= c) v = 1.0;
      if (i == t - 1 && y >= c) v = 1.0;
      w[(size_t)i * n + y] = v;
    }
  }
  return w;
}

// the unmasked pixel nearest (cy, cx), ties to the lowest index
static int64_t nearest_unmasked(const std::vector<uint8_t>& mask, int nx, long long cy, long long cx) {
  int64_t best = -1;
  long long bd = -1;
  for (int64_t p = 0; p < (int64_t)mask.size(); ++p) {
    if (!mask[p]) continue;
    const long long dy = p / nx - cy, dx = p % nx - cx;
    const long long d2 = dy * dy + dx * dx;
    if (best < 0 || d2 < bd) {
      best = p;
      bd = d2;
    }
  }
  return best;
}

static int tiled_build(cmm_precon* pc, const cmm_precon_opts* o) {
  cmm_op* op = pc->op;
  cmm_pointing* pt = op->pt;
  const int ny = pt->ny, nx = pt->nx, nc = pt->ncomp;
  const int64_t npix = pt->npix;
  const int ty = (o && o->tiles_y > 0) ? o->tiles_y : 2, tx = (o && o->tiles_x > 0) ? o->tiles_x : 2;
  if (ty > ny || tx > nx || ty * tx > 64) return fail(CMM_ERR_ARG, "bad tile grid (at most 64 tiles)");
  std::vector<uint8_t> mask(npix);
  CMM_CUDA(cudaMemcpy(mask.data(), pt->mask, npix, cudaMemcpyDeviceToHost));
  const std::vector<double> wy = tile_windows_1d(ny, ty), wx = tile_windows_1d(nx, tx);
  std::vector<double> sp((size_t)ty * tx * npix);
  for (int i = 0; i < ty; ++i)
    for (int j = 0; j < tx; ++j)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
          sp[((size_t)(i * tx + j) * ny + y) * nx + x] = std::sqrt(wy[(size_t)i * ny + y] * wx[(size_t)j * nx + x]);
  CMM_TRY(dalloc(&pc->sqrt_phi, sizeof(double) * sp.size()));
  CMM_TRY(dalloc(&pc->ttmp, sizeof(double) * 2 * nc * npix));
  CMM_CUDA(cudaMemcpy(pc->sqrt_phi, sp.data(), sizeof(double) * sp.size(), cudaMemcpyHostToDevice));
  for (int i = 0; i < ty; ++i)
    for (int j = 0; j < tx; ++j) {
      cmm_precon_opts co{};
      if (o) co = *o;
      co.ref_pixel = nearest_unmasked(mask, nx, (long long)((i + 0.5) * ny / ty), (long long)((j + 0.5) * nx / tx));
      if (co.ref_pixel < 0) return fail(CMM_ERR_ARG, "no unmasked pixel");
      cmm_precon* part = nullptr;
      CMM_TRY(cmm_precon_create(op, CMM_PRECON_CIRCULANT, &co, &part));
      pc->parts.push_back(part);
    }
  return CMM_OK;
}

extern "C" {

static int64_t pick_reference(const std::vector<uint8_t>& mask, int ny, int nx) {
  const int64_t p0 = (int64_t)(ny / 2) * nx + nx / 2;
  if (mask[p0]) return p0;
  int64_t best = -1;
  long long bd = -1;
  for (int64_t p = 0; p < (int64_t)mask.size(); ++p) {
    if (!mask[p]) continue;
    const long long dy = p / nx - ny / 2, dx = p % nx - nx / 2;
    const long long d2 = dy * dy + dx * dx;
    if (best < 0 || d2 < bd) {
      best = p;
      bd = d2;
    }
  }
  return best;
}

}  // extern "C"

// Detector weights diag(N^-1)_d of Eq. 3 and Eq. 7: the exact diagonal of the
// circulant filter, or with opts->white_diag the white level 1 / sigma_d^2.
static const double* precon_weights(const cmm_op* op, const cmm_precon_opts* o) {
  return (o && o->white_diag) ? op->nz->white : op->nz->diag;
}

template <typename T>
static int circulant_build(cmm_precon* pc, const cmm_precon_opts* o) {
  cmm_op* op = pc->op;
  cmm_pointing* pt = op->pt;
  cudaStream_t st = op->ctx->stream;
  const int nc = pt->ncomp;
  const int64_t npix = pt->npix;
  const int nb = nc == 1 ? 1 : 6;
  CMM_TRY(fft2_plan_init<T>(pc->plan, pt->ny, pt->nx));
  // the build (q, its transform and the per-mode inverse) is FP64 in every precision
  // mode; only the apply's transforms follow the operator's precision
  Fft2Plan plan64;
  CMM_TRY(fft2_plan_init<double>(plan64, pt->ny, pt->nx));
  double* blocks = nullptr;
  double* rows = nullptr;
  double2* qplanes = nullptr;
  unsigned long long* scratch = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    dfree(blocks);
    dfree(rows);
    dfree(qplanes);
    dfree(scratch);
    dfree(plan64.tw);
  };
  auto run = [&]() -> int {
    CMM_TRY(dalloc(&blocks, sizeof(double) * nb * npix));
    CMM_TRY(dalloc(&rows, sizeof(double) * nc * nc * npix));
    CMM_TRY(dalloc(&qplanes, sizeof(double2) * nc * nc * npix));
    CMM_TRY(dalloc(&scratch, sizeof(unsigned long long) * 2));
    CMM_TRY(dalloc(&pc->sig, sizeof(double) * nb * npix));
    CMM_TRY(dalloc(&pc->sig_inv, sizeof(double) * nb * npix));
    CMM_TRY(dalloc(&pc->hinv, sizeof(double) * (nc == 1 ? 1 : 9) * npix));
    CMM_TRY(dalloc(&pc->planes, sizeof(V2<T>) * nc * npix));
    CMM_TRY(dalloc(&pc->tmp, sizeof(double) * nc * npix));
    // Eq. 7: Sigma^T Sigma = binned blocks
    CMM_CUDA(cudaMemsetAsync(blocks, 0, sizeof(double) * nb * npix, st));
    CMM_TRY(launch_hit_blocks(pt, precon_weights(op, o), pt->mask, blocks, nullptr));
    CMM_TRY(launch_block_sqrt(nc, npix, blocks, pt->mask, pc->sig, pc->sig_inv, st));
    // reference pixel
    std::vector<uint8_t> mask(npix);
    CMM_CUDA(cudaMemcpyAsync(mask.data(), pt->mask, npix, cudaMemcpyDeviceToHost, st));
    CMM_CUDA(cudaStreamSynchronize(st));
    int64_t ref = (o && o->ref_pixel >= 0) ? o->ref_pixel : pick_reference(mask, pt->ny, pt->nx);
    if (ref < 0 || ref >= npix || !mask[ref]) return fail(CMM_ERR_ARG, "no usable reference pixel");
    pc->ref = ref;
    // Eq. 6: rows A e_{ref, gamma}
    for (int g = 0; g < nc; ++g) {
      CMM_CUDA(cudaMemsetAsync(op->tmp_a, 0, sizeof(double) * nc * npix, st));
      k_set_unit<<<1, 1, 0, st>>>(op->tmp_a, (long long)g * npix + ref);
      CMM_LAUNCH_CHECK();
      CMM_TRY(apply_A_dev(op, op->tmp_a, rows + (size_t)g * nc * npix));
    }
    // Eq. 13 + symmetrisation + Gaussian taper, then Eq. 11: H = conj(F q)
    double taper = (o && o->taper_sigma_px > 0 && std::isfinite(o->taper_sigma_px)) ? o->taper_sigma_px : 0.0;
    pc->taper = taper;
    CMM_TRY(launch_circ_q<double>(nc, rows, pc->sig_inv, (int)ref, pt->ny, pt->nx, taper, qplanes, st));
    CMM_TRY(fft2<double>(plan64, qplanes, nc * nc, -1, nullptr, st));
    const double eps = (o && o->pd_eps > 0) ? o->pd_eps : 1e-6;
    CMM_TRY(launch_mode_inverse<double>(nc, qplanes, npix, eps, pc->hinv, scratch, st));
    if (op->prec != CMM_PREC_F64) {
      // the apply of an FP32 operator multiplies FP32 spectra: FP32 blocks (GB300's
      // FP64 pipe would otherwise bound the per-mode products)
      const int64_t nh = (int64_t)(nc == 1 ? 1 : 9) * npix;
      CMM_TRY(dalloc(&pc->hinv32, sizeof(float) * nh));
      CMM_TRY(launch_to_f32(pc->hinv, pc->hinv32, nh, st));
      CMM_TRY(dalloc(&pc->sig_inv32, sizeof(float) * nb * npix));
      CMM_TRY(launch_to_f32(pc->sig_inv, pc->sig_inv32, nb * npix, st));
    }
    unsigned long long h[2];
    CMM_CUDA(cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    CMM_CUDA(cudaStreamSynchronize(st));
    pc->n_clamped = (int64_t)(h[1] / 2);
    return CMM_OK;
  };
  int s = run();
  cleanup();
  return s;
}

extern "C" {

int cmm_precon_create(cmm_op* op, int32_t kind, const cmm_precon_opts* opts, cmm_precon** out) {
  TraceRange tr("cmm: preconditioner build");
  if (!op || !out) return fail(CMM_ERR_ARG, "null argument");
  *out = nullptr;
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  CMM_TRY(op_sync_corr(op));
  if (kind < CMM_PRECON_BINNED || kind > CMM_PRECON_CIRC_TILED || kind == CMM_PRECON_CIRC_LEARNED)
    return fail(CMM_ERR_ARG, "bad preconditioner kind");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  cmm_precon* pc = new cmm_precon();
  pc->op = op;
  op->refs++;
  pc->kind = kind;
  cmm_pointing* pt = op->pt;
  const int nb = pt->ncomp == 1 ? 1 : 6;
  cudaStream_t st = op->ctx->stream;
  int s = CMM_OK;
  if (kind == CMM_PRECON_BINNED || kind == CMM_PRECON_JACOBI) {
    double* blocks = nullptr;
    s = dalloc(&blocks, sizeof(double) * nb * pt->npix);
    if (s == CMM_OK) s = dalloc(&pc->inv, sizeof(double) * nb * pt->npix);
    if (s == CMM_OK) {
      auto run = [&]() -> int {
        CMM_CUDA(cudaMemsetAsync(blocks, 0, sizeof(double) * nb * pt->npix, st));
        CMM_TRY(launch_hit_blocks(pt, kind == CMM_PRECON_BINNED ? precon_weights(op, opts) : nullptr, pt->mask,
                                  blocks, nullptr));
        CMM_TRY(launch_block_inverse(pt->ncomp, pt->npix, blocks, pt->mask, pc->inv, st));
        CMM_CUDA(cudaStreamSynchronize(st));
        return CMM_OK;
      };
      s = run();
    }
    dfree(blocks);
  } else if (kind == CMM_PRECON_CIRCULANT) {
    s = op->prec == CMM_PREC_F64 ? circulant_build<double>(pc, opts) : circulant_build<float>(pc, opts);
  } else if (kind == CMM_PRECON_CIRC_TILED) {
    s = tiled_build(pc, opts);
  }
  if (s != CMM_OK) {
    cmm_precon_destroy(pc);
    return s;
  }
  *out = pc;
  return CMM_OK;
}

}  // extern "C"

// z = M r; when `partial` is given, also the per-block partials of r^T z.
template <typename T>
static int circulant_apply(cmm_precon* pc, const double* r, double* z, double* partial, const int* done) {
  cmm_op* op = pc->op;
  const int nc = op->pt->ncomp;
  const int64_t npix = op->pt->npix;
  cudaStream_t st = op->ctx->stream;
  V2<T>* planes = (V2<T>*)pc->planes;
  // z = Sigma^-1 F^-1 H^-1 F Sigma^-1 r (Eq. 12), the block applies fused with the
  // moves into and out of the complex planes; TQU maps travel as two complex planes
  // (T + i Q and U), so three real transforms take two complex ones
  if (nc == 3) {
    if constexpr (sizeof(T) == 4) {
      if (pc->hinv32 && pc->sig_inv32) {
        // FP32 operator: Sigma^-1 and the mode blocks in FP32 (FP64 build, FP32 copies)
        CMM_TRY((launch_block_to_planes_packed<T, float>(npix, pc->sig_inv32, r, planes, done, st)));
        CMM_TRY(fft2<T>(pc->plan, planes, 2, -1, done, st));
        CMM_TRY((launch_mode_apply_packed<T, float>(planes, pc->hinv32, op->pt->ny, op->pt->nx, done, st)));
        CMM_TRY(fft2<T>(pc->plan, planes, 2, 1, done, st));
        return launch_planes_block_dot_packed<T, float>(npix, planes, 1.0 / (double)npix, pc->sig_inv32, z, r,
                                                        partial, done, st);
      }
    }
    CMM_TRY((launch_block_to_planes_packed<T, double>(npix, pc->sig_inv, r, planes, done, st)));
    CMM_TRY(fft2<T>(pc->plan, planes, 2, -1, done, st));
    CMM_TRY((launch_mode_apply_packed<T, double>(planes, pc->hinv, op->pt->ny, op->pt->nx, done, st)));
    CMM_TRY(fft2<T>(pc->plan, planes, 2, 1, done, st));
    return launch_planes_block_dot_packed<T, double>(npix, planes, 1.0 / (double)npix, pc->sig_inv, z, r, partial,
                                                     done, st);
  }
  CMM_TRY(launch_block_to_planes<T>(nc, npix, pc->sig_inv, r, planes, done, st));
  CMM_TRY(fft2<T>(pc->plan, planes, nc, -1, done, st));
  CMM_TRY(launch_mode_apply<T>(nc, planes, pc->hinv, npix, done, st));
  CMM_TRY(fft2<T>(pc->plan, planes, nc, 1, done, st));
  return launch_planes_block_dot<T>(nc, npix, planes, 1.0 / (double)npix, pc->sig_inv, z, r, partial, done, st);
}

extern "C" {

static int precon_apply_dev(cmm_precon* pc, const double* r, double* z, double* partial, const int* done) {
  cmm_op* op = pc->op;
  const int nc = op->pt->ncomp;
  const int64_t npix = op->pt->npix;
  cudaStream_t st = op->ctx->stream;
  switch (pc->kind) {
    case CMM_PRECON_BINNED:
    case CMM_PRECON_JACOBI:
      return launch_block_apply_dot(nc, npix, pc->inv, r, z, r, partial, done, st);
    case CMM_PRECON_CIRCULANT:
      return op->prec == CMM_PREC_F64 ? circulant_apply<double>(pc, r, z, partial, done)
                                      : circulant_apply<float>(pc, r, z, partial, done);
    case CMM_PRECON_CIRC_TILED: {
      // z = sum_t D_t M_t D_t r
      double* a = pc->ttmp;
      double* b = pc->ttmp + nc * npix;
      for (size_t t = 0; t < pc->parts.size(); ++t) {
        const double* d = pc->sqrt_phi + t * npix;
        CMM_TRY(launch_window_mul(d, r, a, npix, nc, done, st));
        CMM_TRY(precon_apply_dev(pc->parts[t], a, b, nullptr, done));
        CMM_TRY(launch_window_acc(d, b, z, npix, nc, t == 0, done, st));
      }
      if (partial) CMM_TRY(launch_dot_partial(r, z, nc * npix, partial, done, st));
      return CMM_OK;
    }
    case CMM_PRECON_CIRC_LEARNED:
      CMM_TRY(op->prec == CMM_PREC_F64 ? circulant_apply<double>(pc, r, z, nullptr, done)
                                       : circulant_apply<float>(pc, r, z, nullptr, done));
      CMM_TRY(unet_correct(pc->unet, r, z, op->pt->mask, npix, nc, done, st));
      if (partial) CMM_TRY(launch_dot_partial(r, z, nc * npix, partial, done, st));
      return CMM_OK;
    default:
      CMM_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * nc * npix, cudaMemcpyDeviceToDevice, st));
      if (partial) CMM_TRY(launch_dot_partial(r, z, nc * npix, partial, done, st));
      return CMM_OK;
  }
}

int cmm_precon_apply(cmm_precon* pc, const double* r, double* z) {
  TraceRange tr("cmm: preconditioner apply");
  if (!pc || !r || !z) return fail(CMM_ERR_ARG, "null argument");
  if (r == z) return fail(CMM_ERR_ARG, "r and z must not alias");
  CMM_CUDA(cudaSetDevice(pc->op->ctx->device));
  return precon_apply_dev(pc, r, z, nullptr, nullptr);
}

int cmm_precon_set_correction(cmm_precon* pc, cmm_unet* net) {
  if (!pc) return fail(CMM_ERR_ARG, "null preconditioner");
  if (pc->kind != CMM_PRECON_CIRCULANT && pc->kind != CMM_PRECON_CIRC_LEARNED)
    return fail(CMM_ERR_ARG, "the learned correction follows the circulant preconditioner");
  if (!net) {
    if (pc->unet) unet_release(pc->unet);
    pc->unet = nullptr;
    pc->kind = CMM_PRECON_CIRCULANT;
    return CMM_OK;
  }
  if (!unet_matches(net, pc->op->ctx, pc->op->pt->ny, pc->op->pt->nx) || pc->op->pt->ncomp != 3)
    return fail(CMM_ERR_ARG, "the U-Net must share the operator's context and its TQU map shape");
  unet_retain(net);
  if (pc->unet) unet_release(pc->unet);
  pc->unet = net;
  pc->kind = CMM_PRECON_CIRC_LEARNED;
  return CMM_OK;
}

int cmm_harvest_pairs(cmm_precon* pc, const double* snapshots, int32_t count, const double* x_star, float* inputs,
                      float* targets) {
  if (!pc || !snapshots || !x_star || !inputs || !targets || count < 0) return fail(CMM_ERR_ARG, "bad argument");
  cmm_op* op = pc->op;
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  cudaStream_t st = op->ctx->stream;
  const long long n = (long long)op->pt->ncomp * op->pt->npix;
  double* z = op->tmp_b;
  for (int k = 0; k < count; ++k) {
    const double* xk = snapshots + (long long)k * 2 * n;
    const double* rk = xk + n;
    CMM_TRY(precon_apply_dev(pc, rk, z, nullptr, nullptr));
    CMM_TRY(launch_dot_partial(z, z, n, op->ctx->d_partial, nullptr, st));
    k_pair<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(z, x_star, xk, op->ctx->d_partial,
                                                                             inputs + (long long)k * n,
                                                                             targets + (long long)k * n, n);
    CMM_LAUNCH_CHECK();
  }
  return CMM_OK;
}

int cmm_precon_clamped(cmm_precon* pc, int64_t* n_clamped) {
  if (!pc || !n_clamped) return fail(CMM_ERR_ARG, "null argument");
  *n_clamped = pc->n_clamped;
  return CMM_OK;
}

// ------------------------------------------------------------------ solver
struct SolveBufs {
  double *r, *z, *p, *q, *r_old, *p1, *p2, *p3;
  bool cg_f32 = false;   // FP32 CG: z is rounded to FP32 before its dot products
};

// ||b - A x|| / ||b|| recomputed from x (one A-application), in the op's CG
// scratch (q and z slots: r, p and r_old stay as the solve left them, for a
// checkpoint); the check the recursive residual is compared with.
static int true_residual(cmm_op* op, const double* b, const double* x, double bnorm2, double* out) {
  const int64_t n = (int64_t)op->pt->ncomp * op->pt->npix;
  double* q = op->sol + 3 * n;
  double* r = op->sol + n;
  CMM_TRY(apply_A_dev(op, x, q));
  CMM_TRY(launch_sub(r, b, q, n, op->ctx->stream));
  double rr = 0.0;
  CMM_TRY(cmm_dot(op, r, r, n, &rr));
  *out = std::sqrt(rr / bnorm2);
  return CMM_OK;
}

// z = M r (and the learned correction when the preconditioner has one), then the
// CG dot products of z.
static int precon_step(cmm_op* op, cmm_precon* pc, const SolveBufs& v, SolverDev* dst, bool flexible) {
  const int64_t n = (int64_t)op->pt->ncomp * op->pt->npix;
  cudaStream_t st = op->ctx->stream;
  // FP64 PCG: the preconditioner's last kernel forms the partials of r^T z itself
  if (!flexible && !v.cg_f32) return precon_apply_dev(pc, v.r, v.z, v.p1, &dst->done);
  CMM_TRY(precon_apply_dev(pc, v.r, v.z, nullptr, &dst->done));
  return launch_solver_z(v.z, v.r, flexible ? v.r_old : nullptr, n, dst, v.p1, flexible ? v.p3 : nullptr, st);
}

struct Snap {
  double* buf = nullptr;
  int every = 0, max = 0;
};

// Rings of truncated flexible CG, FCG(m): P, Q [win][n] and the window partials
struct Fcg {
  double *P = nullptr, *Q = nullptr, *wpart = nullptr;
  int win = 1;
};

static int solve_iteration(cmm_op* op, cmm_precon* pc, double* x, const SolveBufs& v, SolverDev* dst,
                           double* hist, double* anorm, bool flexible, const Snap& snap = Snap(),
                           const Fcg& fcg = Fcg()) {
  const int64_t n = (int64_t)op->pt->ncomp * op->pt->npix;
  cudaStream_t st = op->ctx->stream;
  const bool ring = fcg.win > 1;
  CMM_TRY(apply_A_dev(op, v.p, v.q));
  CMM_TRY(launch_dot_partial_cg(v.p, v.q, n, dst, v.p1, st));
  CMM_TRY(launch_solver_alpha(dst, v.p1, anorm, st));
  if (ring) CMM_TRY(launch_update_xr_ring(x, v.r, v.p, v.q, n, dst, fcg.P, fcg.Q, v.p2, st));
  else CMM_TRY(launch_update_xr(x, v.r, flexible ? v.r_old : nullptr, v.p, v.q, n, dst, v.p2, st));
  CMM_TRY(launch_solver_check(dst, v.p2, hist, st));
  if (snap.buf) CMM_TRY(launch_snapshot(x, v.r, n, dst, snap.every, snap.max, snap.buf, st));
  if (ring) {
    // z = M r, then p = z made A-conjugate to the kept directions, rho = p^T r
    CMM_TRY(precon_step(op, pc, v, dst, false));
    CMM_TRY(launch_window_dots(v.z, fcg.Q, n, dst, fcg.wpart, st));
    CMM_TRY(launch_window_beta(dst, fcg.wpart, st));
    CMM_TRY(launch_update_p_window(v.p, v.z, fcg.P, v.r, n, dst, v.p2, st));
    return launch_solver_rho_pr(dst, v.p2, st);
  }
  CMM_TRY(precon_step(op, pc, v, dst, flexible));
  CMM_TRY(launch_solver_beta(dst, v.p1, flexible ? v.p3 : nullptr, st));
  CMM_TRY(launch_update_p(v.p, v.z, n, dst, st));
  return CMM_OK;
}

// ------------------------------------------------------------------ checkpoint / resume
// State layout (doubles): r_k [n], p_{k-1} [n], r_{k-1} [n], then kStateScalars
// scalars: rho_{k-1}, k, ||r_k|| / ||b||, FP32-CG flag, a format tag.
constexpr int kStateScalars = 8;
constexpr double kStateTag = 1309.7473;

int cmm_solve_state_size(cmm_op* op, int64_t* n_doubles) {
  if (!op || !n_doubles) return fail(CMM_ERR_ARG, "null argument");
  *n_doubles = 3 * (int64_t)op->pt->ncomp * op->pt->npix + kStateScalars;
  return CMM_OK;
}

int cmm_solve_state_save(cmm_op* op, double* state) {
  if (!op || !state) return fail(CMM_ERR_ARG, "null argument");
  if (!op->sol || !op->sol_state) return fail(CMM_ERR_ARG, "the operator has no solve to save");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  const int64_t n = (int64_t)op->pt->ncomp * op->pt->npix;
  cudaStream_t st = op->ctx->stream;
  SolverDev h{};
  CMM_CUDA(cudaMemcpyAsync(&h, op->sol_state, sizeof(h), cudaMemcpyDeviceToHost, st));
  CMM_CUDA(cudaStreamSynchronize(st));
  if (h.status == CMM_ERR_BREAKDOWN) return fail(CMM_ERR_ARG, "the last solve broke down: nothing to resume");
  CMM_CUDA(cudaMemcpyAsync(state, op->sol, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));              // r
  CMM_CUDA(cudaMemcpyAsync(state + n, op->sol + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));  // p
  CMM_CUDA(cudaMemcpyAsync(state + 2 * n, op->sol + 4 * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));  // r_old
  const double sc[kStateScalars] = {h.rho, (double)h.iter, h.rel, (double)h.f32, kStateTag, 0, 0, 0};
  CMM_CUDA(cudaMemcpyAsync(state + 3 * n, sc, sizeof(sc), cudaMemcpyHostToDevice, st));
  CMM_CUDA(cudaStreamSynchronize(st));
  return CMM_OK;
}

int cmm_solve_state_load(cmm_op* op, const double* state) {
  if (!op || !state) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  const int64_t n = (int64_t)op->pt->ncomp * op->pt->npix;
  cudaStream_t st = op->ctx->stream;
  double sc[kStateScalars];
  CMM_CUDA(cudaMemcpyAsync(sc, state + 3 * n, sizeof(sc), cudaMemcpyDeviceToHost, st));
  CMM_CUDA(cudaStreamSynchronize(st));
  if (sc[4] != kStateTag || !(sc[1] >= 0) || !std::isfinite(sc[0]))
    return fail(CMM_ERR_ARG, "not a solver state of cmm_solve_state_save");
  if (!op->sol) CMM_TRY(dalloc(&op->sol, sizeof(double) * (5 * n + 3 * kRedBlocks)));
  if (!op->sol_state) CMM_TRY(dalloc(&op->sol_state, sizeof(SolverDev)));
  CMM_CUDA(cudaMemcpyAsync(op->sol, state, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  CMM_CUDA(cudaMemcpyAsync(op->sol + 2 * n, state + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  CMM_CUDA(cudaMemcpyAsync(op->sol + 4 * n, state + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  op->resume_rho = sc[0];
  op->resume_iter = (int)sc[1];
  op->resume_rel = sc[2];
  op->resume_ready = 1;
  CMM_CUDA(cudaStreamSynchronize(st));
  return CMM_OK;
}

int cmm_solve(cmm_op* op, cmm_precon* pc, const double* b, double* x, const cmm_solve_opts* opts,
              double* resid_hist, double* anorm_terms, double* snapshots, cmm_solve_info* info) {
  TraceRange tr("cmm: solve");
  if (!op || !pc || !b || !x || !opts || !info) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  CMM_TRY(op_sync_corr(op));
  if (snapshots && (opts->snapshot_every < 1 || opts->snapshot_max < 1)) return fail(CMM_ERR_ARG, "bad snapshot options");
  Snap snap;
  if (snapshots) {
    snap.buf = snapshots;
    snap.every = opts->snapshot_every;
    snap.max = opts->snapshot_max;
  }
  if (pc->op != op) return fail(CMM_ERR_ARG, "preconditioner belongs to another operator");
  if (opts->maxit < 0 || !(opts->tol >= 0) || opts->resid_replace < 0) return fail(CMM_ERR_ARG, "bad solve options");
  if (opts->resume && !op->resume_ready) return fail(CMM_ERR_ARG, "resume without a loaded solver state");
  if (opts->fcg_window < 0 || opts->fcg_window > kMaxWin) return fail(CMM_ERR_ARG, "fcg_window must be 0..8");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  const auto t0 = std::chrono::steady_clock::now();
  cmm_ctx* c = op->ctx;
  cudaStream_t st = c->stream;
  const int64_t n = (int64_t)op->pt->ncomp * op->pt->npix;
  const bool flexible = opts->flexible != 0 || pc->kind == CMM_PRECON_CIRC_LEARNED;
  Fcg fcg;
  fcg.win = flexible ? std::max(1, (int)opts->fcg_window) : 1;
  if (fcg.win > 1 && (opts->resume || opts->resid_replace > 0))
    return fail(CMM_ERR_UNSUPPORTED, "fcg_window > 1 with resume or residual replacement");
  if (!op->sol) CMM_TRY(dalloc(&op->sol, sizeof(double) * (5 * n + 3 * kRedBlocks)));
  if (!op->sol_state) CMM_TRY(dalloc(&op->sol_state, sizeof(SolverDev)));
  if (fcg.win > 1) {
    const int64_t need = 2 * (int64_t)fcg.win * n + (int64_t)fcg.win * kRedBlocks;
    if (op->fcg_doubles < need) {
      CMM_CUDA(cudaStreamSynchronize(op->ctx->stream));
      dfree(op->fcg);
      op->fcg = nullptr;
      op->fcg_doubles = 0;
      CMM_TRY(dalloc(&op->fcg, sizeof(double) * need));
      op->fcg_doubles = need;
    }
    fcg.P = op->fcg;
    fcg.Q = op->fcg + (int64_t)fcg.win * n;
    fcg.wpart = op->fcg + 2 * (int64_t)fcg.win * n;
  }
  SolveBufs v;
  v.cg_f32 = opts->cg_f32 != 0;
  v.r = op->sol;
  v.z = v.r + n;
  v.p = v.z + n;
  v.q = v.p + n;
  v.r_old = v.q + n;
  v.p1 = v.r_old + n;
  v.p2 = v.p1 + kRedBlocks;
  v.p3 = v.p2 + kRedBlocks;
  SolverDev* dst = (SolverDev*)op->sol_state;
  double bnorm2 = 0.0;
  CMM_TRY(cmm_dot(op, b, b, n, &bnorm2));
  SolverDev h{};
  h.bnorm2 = bnorm2 > 0 ? bnorm2 : 1.0;
  h.tol = opts->tol;
  h.maxit = opts->maxit;
  h.f32 = opts->cg_f32 ? 1 : 0;
  h.win = fcg.win;
  if (!std::isfinite(bnorm2)) {
    // a non-finite right-hand side: no iteration is meaningful
    h.done = 1;
    h.status = CMM_ERR_BREAKDOWN;
    CMM_CUDA(cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    CMM_CUDA(cudaStreamSynchronize(st));
    op->resume_ready = 0;
    info->iterations = 0;
    info->status = CMM_ERR_BREAKDOWN;
    info->rel_resid = -1.0;
    info->true_rel_resid = -1.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return CMM_OK;
  }
  const bool resume = opts->resume != 0;
  if (resume) {
    h.rho = op->resume_rho;
    h.iter = op->resume_iter;
    h.rel = op->resume_rel;
    h.status = CMM_ERR_NOT_CONVERGED;
    h.done = h.iter >= h.maxit ? 1 : 0;
    op->resume_ready = 0;
  }
  CMM_CUDA(cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  if (!(bnorm2 > 0)) {
    CMM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    CMM_CUDA(cudaStreamSynchronize(st));
    info->iterations = 0;
    info->status = CMM_OK;
    info->rel_resid = 0.0;
    info->true_rel_resid = 0.0;
    info->seconds = 0.0;
    return CMM_OK;
  }
  if (resume) {
    // continue from the loaded state (r_k, p_{k-1}, r_{k-1}, rho_{k-1}, k) and the
    // caller's x_k: the tail of iteration k that the interrupted solve skipped,
    // z_k = M r_k, beta, p_k = z_k + beta p_{k-1}
    CMM_TRY(precon_step(op, pc, v, dst, flexible));
    CMM_TRY(launch_solver_beta(dst, v.p1, flexible ? v.p3 : nullptr, st));
    CMM_TRY(launch_update_p(v.p, v.z, n, dst, st));
  } else {
    // r0 = b - A x0 (rounded in FP32 CG), z0 = M r0, p0 = z0
    if (opts->x0_given) {
      CMM_TRY(apply_A_dev(op, x, v.q));
    } else {
      CMM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
      CMM_CUDA(cudaMemsetAsync(v.q, 0, sizeof(double) * n, st));
    }
    CMM_TRY(launch_residual(v.r, b, v.q, n, dst, v.p2, st));
    CMM_CUDA(cudaMemcpyAsync(v.r_old, v.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    CMM_TRY(precon_step(op, pc, v, dst, false));
    CMM_TRY(launch_solver_init(dst, v.p1, v.p2, resid_hist, st));
    if (snap.buf) CMM_TRY(launch_snapshot(x, v.r, n, dst, snap.every, snap.max, snap.buf, st));
    CMM_CUDA(cudaMemcpyAsync(v.p, v.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  }
  int per = std::max(1, opts->check_every);
  if (opts->resid_replace > 0) per = std::min(per, opts->resid_replace);
  while (opts->resid_replace > 0 && opts->resid_replace % per) --per;   // per divides the replacement period
  op->done = &dst->done;
  cudaGraphExec_t exec = nullptr;
  int status = CMM_OK;
  if (opts->use_graph) {
    cudaGraph_t graph = nullptr;
    status = [&]() -> int {
      CMM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int s2 = CMM_OK;
      for (int i = 0; i < per && s2 == CMM_OK; ++i)
        s2 = solve_iteration(op, pc, x, v, dst, resid_hist, anorm_terms, flexible, snap, fcg);
      cudaError_t e = cudaStreamEndCapture(st, &graph);
      if (s2 != CMM_OK) return s2;
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      CMM_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      return CMM_OK;
    }();
    if (graph) cudaGraphDestroy(graph);
  }
  SolverDev* hs = (SolverDev*)c->h_scalar;
  int launched = 0;
  while (status == CMM_OK) {
    if (exec) {
      cudaError_t e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) {
        status = cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__);
        break;
      }
    } else {
      for (int i = 0; i < per && status == CMM_OK; ++i)
        status = solve_iteration(op, pc, x, v, dst, resid_hist, anorm_terms, flexible, snap, fcg);
      if (status != CMM_OK) break;
    }
    launched += per;
    cudaError_t e = cudaMemcpyAsync(hs, dst, sizeof(SolverDev), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      status = cuda_fail(e, "solver state readback", __FILE__, __LINE__);
      break;
    }
    if (hs->done) break;
    if (launched > opts->maxit + per) break;
    if (opts->resid_replace > 0 && hs->iter % opts->resid_replace == 0) {
      // residual replacement: r = b - A x, z = M r, rho = r^T z; p is kept
      status = [&]() -> int {
        CMM_TRY(apply_A_dev(op, x, v.q));
        CMM_TRY(launch_residual(v.r, b, v.q, n, dst, v.p2, st));
        CMM_TRY(precon_step(op, pc, v, dst, false));
        return launch_solver_rho(dst, v.p1, st);
      }();
    }
  }
  op->done = nullptr;
  if (exec) cudaGraphExecDestroy(exec);
  if (status != CMM_OK) return status;
  info->iterations = hs->iter;
  info->status = hs->status;
  info->rel_resid = hs->rel;
  info->true_rel_resid = -1.0;
  if (!opts->skip_true_resid) CMM_TRY(true_residual(op, b, x, h.bnorm2, &info->true_rel_resid));
  info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return CMM_OK;
}

int cmm_solve_host(cmm_op* op, cmm_precon* pc, const double* b_host, double* x_host, const cmm_solve_opts* opts,
                   cmm_solve_info* info) {
  if (!op || !pc || !b_host || !x_host || !opts || !info) return fail(CMM_ERR_ARG, "null argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  const int64_t n = (int64_t)op->pt->ncomp * op->pt->npix;
  if (!op->host_bx) CMM_TRY(dalloc(&op->host_bx, sizeof(double) * 2 * n));
  double* b = op->host_bx;
  double* x = op->host_bx + n;
  cudaStream_t st = op->ctx->stream;
  CMM_CUDA(cudaMemcpyAsync(b, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if (opts->x0_given || opts->resume)
    CMM_CUDA(cudaMemcpyAsync(x, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  CMM_TRY(cmm_solve(op, pc, b, x, opts, nullptr, nullptr, nullptr, info));
  CMM_CUDA(cudaMemcpyAsync(x_host, x, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CMM_CUDA(cudaStreamSynchronize(st));
  return CMM_OK;
}

// ------------------------------------------------------------------ autotuner
namespace {
struct TuneKey {
  int64_t n_t;
  int n_det, prec, ncomp;
  bool operator==(const TuneKey& o) const {
    return n_t == o.n_t && n_det == o.n_det && prec == o.prec && ncomp == o.ncomp;
  }
};
std::vector<std::pair<TuneKey, int>> g_tune_cache;
}  // namespace

// Decision values of the tuner (process cache and file): 0 = two-detector packing
// (its split is fixed by n_samp), lr > 0 = one-detector packing with R = 2^lr.
static int apply_decision(cmm_op* op, int v) {
  if (v == 0) {
    op->pair = 1;
    return CMM_OK;
  }
  op->pair = 0;
  return v != op->logR ? op_set_split(op, v) : CMM_OK;
}

static void report_decision(const cmm_op* op, int v, int32_t* chosen_logR, int32_t* chosen_pair) {
  if (chosen_pair) *chosen_pair = v == 0 ? 1 : 0;
  if (chosen_logR) *chosen_logR = v == 0 ? op->plogR : v;
}

int cmm_autotune(cmm_op* op, int32_t reps, const char* cache_path, int32_t* chosen_logR, int32_t* chosen_pair,
                 double* best_ms) {
  if (!op || reps <= 0) return fail(CMM_ERR_ARG, "bad argument");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  const TuneKey key{op->pt->n_t, op->pt->n_det, op->prec, op->pt->ncomp};
  const int logN = op->logR + op->logC;
  const bool pair_ok = op->pR > 0 && op->tw_pair && op->nz->corr_r == 0 && op->pt->max_hits <= kF32HitLimit;
  auto valid = [&](int v) { return (v == 0 && pair_ok) || (v > 0 && v < logN); };
  // cached decision (process-wide, then the optional file)
  for (auto& e : g_tune_cache)
    if (e.first == key && valid(e.second)) {
      CMM_TRY(apply_decision(op, e.second));
      report_decision(op, e.second, chosen_logR, chosen_pair);
      if (best_ms) *best_ms = -1.0;
      return CMM_OK;
    }
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      long long nt;
      int nd, pr, nc, v;
      while (std::fscanf(f, "%lld %d %d %d %d", &nt, &nd, &pr, &nc, &v) == 5)
        if (TuneKey{nt, nd, pr, nc} == key && valid(v)) {
          std::fclose(f);
          g_tune_cache.push_back({key, v});
          CMM_TRY(apply_decision(op, v));
          report_decision(op, v, chosen_logR, chosen_pair);
          if (best_ms) *best_ms = -1.0;
          return CMM_OK;
        }
      std::fclose(f);
    }
  }
  // candidates: the two-detector packing where it applies, and every split of the
  // one-detector packing that the fast kernels support (else the current one)
  std::vector<int> cand;
  if (pair_ok) cand.push_back(0);
  for (int lr = 6; lr <= 8; ++lr)
    if (logN - lr >= 6 && logN - lr <= 12 && op->prec != CMM_PREC_F64) cand.push_back(lr);
  if (cand.empty()) cand.push_back(op->logR);
  const size_t bytes = sizeof(double) * op->pt->ncomp * op->pt->npix;
  CMM_CUDA(cudaMemsetAsync(op->tmp_a, 0, bytes, op->ctx->stream));
  cudaEvent_t e0, e1;
  CMM_CUDA(cudaEventCreate(&e0));
  CMM_CUDA(cudaEventCreate(&e1));
  int best = cand[0];
  double best_t = 1e300;
  int s = CMM_OK;
  for (int v : cand) {
    s = apply_decision(op, v);
    if (s != CMM_OK) break;
    s = apply_A_dev(op, op->tmp_a, op->tmp_b);   // warm-up
    if (s != CMM_OK) break;
    cudaEventRecord(e0, op->ctx->stream);
    for (int r = 0; r < reps && s == CMM_OK; ++r) s = apply_A_dev(op, op->tmp_a, op->tmp_b);
    cudaEventRecord(e1, op->ctx->stream);
    if (s != CMM_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / reps < best_t) {
      best_t = ms / reps;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != CMM_OK) return s;
  CMM_TRY(apply_decision(op, best));
  g_tune_cache.push_back({key, best});
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%lld %d %d %d %d\n", (long long)key.n_t, key.n_det, key.prec, key.ncomp, best);
      std::fclose(f);
    }
  }
  report_decision(op, best, chosen_logR, chosen_pair);
  if (best_ms) *best_ms = best_t;
  return CMM_OK;
}

// ------------------------------------------------------------------ batched solves
int cmm_batch_solve(int32_t n, cmm_op* const* ops, cmm_precon* const* pcs, const double* const* b,
                    double* const* x, const cmm_solve_opts* opts, cmm_solve_info* infos) {
  TraceRange tr("cmm: batch solve");
  if (n <= 0 || !ops || !pcs || !b || !x || !opts || !infos) return fail(CMM_ERR_ARG, "null argument");
  for (int i = 0; i < n; ++i) {
    if (!ops[i] || !pcs[i] || !b[i] || !x[i]) return fail(CMM_ERR_ARG, "null entry in batch");
    if (pcs[i]->op != ops[i]) return fail(CMM_ERR_ARG, "preconditioner belongs to another operator");
    if (ops[i]->ctx->device != ops[0]->ctx->device) return fail(CMM_ERR_ARG, "batch spans devices");
    for (int j = 0; j < i; ++j)
      if (ops[j] == ops[i]) return fail(CMM_ERR_ARG, "an operator appears twice in the batch");
  }
  if (opts->maxit < 0 || !(opts->tol >= 0) || opts->resid_replace != 0 || opts->fcg_window > 1)
    return fail(CMM_ERR_ARG, "bad batch solve options (residual replacement and fcg_window are per solve)");
  CMM_CUDA(cudaSetDevice(ops[0]->ctx->device));
  for (int i = 0; i < n; ++i) CMM_TRY(op_sync_corr(ops[i]));
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t main_st = ops[0]->ctx->stream;
  std::vector<SolveBufs> vb(n);
  std::vector<SolverDev*> dst(n);
  std::vector<bool> flex(n);
  // per-solve set-up on each solve's own stream
  for (int i = 0; i < n; ++i) {
    cmm_op* op = ops[i];
    const int64_t m = (int64_t)op->pt->ncomp * op->pt->npix;
    cudaStream_t st = op->ctx->stream;
    if (!op->sol) CMM_TRY(dalloc(&op->sol, sizeof(double) * (5 * m + 3 * kRedBlocks)));
    if (!op->sol_state) CMM_TRY(dalloc(&op->sol_state, sizeof(SolverDev)));
    SolveBufs& v = vb[i];
    v.cg_f32 = opts->cg_f32 != 0;
    v.r = op->sol;
    v.z = v.r + m;
    v.p = v.z + m;
    v.q = v.p + m;
    v.r_old = v.q + m;
    v.p1 = v.r_old + m;
    v.p2 = v.p1 + kRedBlocks;
    v.p3 = v.p2 + kRedBlocks;
    dst[i] = (SolverDev*)op->sol_state;
    flex[i] = opts->flexible != 0 || pcs[i]->kind == CMM_PRECON_CIRC_LEARNED;
    double bnorm2 = 0.0;
    CMM_TRY(cmm_dot(op, b[i], b[i], m, &bnorm2));
    SolverDev h{};
    h.bnorm2 = bnorm2 > 0 ? bnorm2 : 1.0;
    h.tol = opts->tol;
    h.maxit = opts->maxit;
    h.f32 = opts->cg_f32 ? 1 : 0;
    CMM_CUDA(cudaMemcpyAsync(dst[i], &h, sizeof(h), cudaMemcpyHostToDevice, st));
    if (opts->x0_given) {
      CMM_TRY(apply_A_dev(op, x[i], v.q));
    } else {
      CMM_CUDA(cudaMemsetAsync(x[i], 0, sizeof(double) * m, st));
      CMM_CUDA(cudaMemsetAsync(v.q, 0, sizeof(double) * m, st));
    }
    CMM_TRY(launch_residual(v.r, b[i], v.q, m, dst[i], v.p2, st));
    CMM_CUDA(cudaMemcpyAsync(v.r_old, v.r, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    CMM_TRY(precon_step(op, pcs[i], v, dst[i], false));
    CMM_TRY(launch_solver_init(dst[i], v.p1, v.p2, nullptr, st));
    CMM_CUDA(cudaMemcpyAsync(v.p, v.z, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    op->done = &dst[i]->done;
  }
  for (int i = 0; i < n; ++i) CMM_CUDA(cudaStreamSynchronize(ops[i]->ctx->stream));
  const int per = std::max(1, opts->check_every);
  // lanes: solves sorted by samples, each to the least loaded lane
  std::vector<long long> work(n);
  for (int i = 0; i < n; ++i) work[i] = (long long)ops[i]->pt->n_det * ops[i]->pt->n_t;
  long long total = 0;
  for (long long w : work) total += w;
  // automatic width: one lane when the solves average 10^8 samples or more (their
  // passes fill the GPU and concurrent solves only share the L2), else 8 lanes (64
  // solves of 128 detectors x 2^18 samples on 256x256 maps: 0.442 s in 8 lanes
  // against 0.539 s one after another)
  int width = opts->batch_width > 0 ? opts->batch_width : (total / n >= 100000000LL ? 1 : 8);
  width = std::max(1, std::min(width, n));
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return work[p] > work[q]; });
  std::vector<std::vector<int>> lanes(width);
  std::vector<long long> load(width, 0);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[l].push_back(i);
    load[l] += work[i];
  }
  // one graph per `per` batch iterations: the lanes are parallel branches, the
  // solves of a lane follow one another
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev(n + 1, nullptr);
  int status = [&]() -> int {
    for (auto& e : ev) CMM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CMM_CUDA(cudaStreamBeginCapture(main_st, cudaStreamCaptureModeThreadLocal));
    int s2 = CMM_OK;
    cudaError_t e = cudaEventRecord(ev[n], main_st);
    for (int l = 0; l < width && s2 == CMM_OK && e == cudaSuccess; ++l) {
      cudaEvent_t prev = ev[n];   // the lane starts at the fork
      for (size_t q = 0; q < lanes[l].size() && s2 == CMM_OK && e == cudaSuccess; ++q) {
        const int i = lanes[l][q];
        cudaStream_t st = ops[i]->ctx->stream;
        e = cudaStreamWaitEvent(st, prev, 0);
        for (int k = 0; k < per && s2 == CMM_OK && e == cudaSuccess; ++k)
          s2 = solve_iteration(ops[i], pcs[i], x[i], vb[i], dst[i], nullptr, nullptr, flex[i]);
        if (e == cudaSuccess) e = cudaEventRecord(ev[i], st);
        prev = ev[i];
      }
      if (e == cudaSuccess && prev != ev[n]) e = cudaStreamWaitEvent(main_st, prev, 0);   // join
    }
    // every stream that took part rejoins the capturing stream
    for (int i = 0; i < n && s2 == CMM_OK && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(main_st, ev[i], 0);
    cudaError_t e2 = cudaStreamEndCapture(main_st, &graph);
    if (s2 != CMM_OK) return s2;
    if (e != cudaSuccess) return cuda_fail(e, "batch graph capture", __FILE__, __LINE__);
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
    CMM_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    return CMM_OK;
  }();
  if (graph) cudaGraphDestroy(graph);
  std::vector<SolverDev> hs(n);
  SolverDev* pinned = nullptr;
  if (status == CMM_OK && cudaMallocHost(&pinned, sizeof(SolverDev) * n) != cudaSuccess)
    status = fail(CMM_ERR_OOM, "pinned allocation failed");
  int launched = 0;
  while (status == CMM_OK) {
    cudaError_t e = cudaGraphLaunch(exec, main_st);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(pinned + i, dst[i], sizeof(SolverDev), cudaMemcpyDeviceToHost, main_st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(main_st);
    if (e != cudaSuccess) {
      status = cuda_fail(e, "batch solve", __FILE__, __LINE__);
      break;
    }
    launched += per;
    bool all = true;
    for (int i = 0; i < n; ++i) all = all && pinned[i].done;
    if (all || launched > opts->maxit + per) break;
  }
  for (int i = 0; i < n; ++i) ops[i]->done = nullptr;
  if (exec) cudaGraphExecDestroy(exec);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (status == CMM_OK)
    for (int i = 0; i < n && status == CMM_OK; ++i) {
      infos[i].iterations = pinned[i].iter;
      infos[i].status = pinned[i].status;
      infos[i].rel_resid = pinned[i].rel;
      infos[i].true_rel_resid = -1.0;
      if (!opts->skip_true_resid)
        status = true_residual(ops[i], b[i], x[i], pinned[i].bnorm2, &infos[i].true_rel_resid);
    }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (status == CMM_OK)
    for (int i = 0; i < n; ++i) infos[i].seconds = secs;
  if (pinned) cudaFreeHost(pinned);
  return status;
}

}  // extern "C"
