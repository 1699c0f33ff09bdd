// Internal definitions shared by the CUDA translation units of the map-maker.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cmm.h"

namespace cmm {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CMM_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return ::cmm::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define CMM_LAUNCH_CHECK() CMM_CUDA(cudaGetLastError())

#define CMM_TRY(call)            \
  do {                           \
    int s_ = (call);             \
    if (s_ != CMM_OK) return s_; \
  } while (0)

// ------------------------------------------------------------------ tracing
// NVTX range for the lifetime of the object (a name per A-application pass and
// per solver phase, seen by Nsight tools; free when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// ------------------------------------------------------------------ vector types
template <typename T> struct V2t;
template <> struct V2t<float> { using t = float2; };
template <> struct V2t<double> { using t = double2; };
template <typename T> using V2 = typename V2t<T>::t;

template <typename T> struct V4t;
template <> struct V4t<float> { using t = float4; };
template <> struct V4t<double> { using t = double4_32a; };
template <typename T> using V4 = typename V4t<T>::t;

template <typename V>
__host__ __device__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename V>
__host__ __device__ __forceinline__ V cmulc(V a, V b) {  // a * conj(b)
  return V{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename V>
__host__ __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V>
__host__ __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V>
__host__ __device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }

// Complex add / subtract for butterflies: FP32 pairs use the packed two-wide
// FP32 instructions of sm_100+ (one instruction for both components).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return double2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return double2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return double2{a.x * b.x, a.y * b.y}; }

// ------------------------------------------------------------------ handles
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace cmm

struct cmm_ctx {
  int refs = 1;                // owner reference + one per dependent handle
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double* d_partial = nullptr;   // reduction partials [kRedBlocks]
  double* d_scalar = nullptr;    // small scalar scratch [16]
  double* h_scalar = nullptr;    // pinned host mirror [16]
};

struct cmm_pointing {
  int refs = 1;                // owner reference + one per dependent handle
  cmm_ctx* ctx = nullptr;
  int ny = 0, nx = 0, ncomp = 0, periodic = 0;
  int n_det = 0;
  int64_t n_t = 0, npix = 0, n_good = 0;
  int4* bore = nullptr;        // [n_t] (bx, by, cphi, sphi)
  int2* det_off = nullptr;     // [n_det] (dx, dy)
  double2* det_pol64 = nullptr;  // [n_det] (cos 2psi, sin 2psi)
  float2* det_pol32 = nullptr;
  float2* rot2 = nullptr;      // [n_t] (cos 2phi, sin 2phi) rounded to FP32 (FP32 response)
  uint8_t* mask = nullptr;     // [npix]
  int64_t max_hits = 0;        // largest number of samples (all detectors) on one pixel
};

// Above this many samples (all detectors) on one pixel the fast path's FP32
// partial map would sum too many terms between flushes: its error grows with the
// number of adds, and where the added values are exact ties the rounding is
// biased.  The binning pass of such operators runs the generic kernel, which
// reduces every sample straight into the FP64 map.
constexpr int64_t kF32HitLimit = 8192;
// Detectors whose samples share one FP32 partial sum before it is added into the
// FP64 map, and the most partial maps an operator keeps (one per such group of a
// chunk, so that a chunk's binning is one launch).
#ifndef CMM_FLUSH_DETS
#define CMM_FLUSH_DETS 256
#endif
constexpr int kFlushDets = CMM_FLUSH_DETS;
constexpr int kMaxPartialMaps = 8;

struct cmm_noise {
  int refs = 1;                // owner reference + one per dependent handle
  cmm_ctx* ctx = nullptr;
  int n_det = 0;
  int64_t n_t = 0;
  double f_samp = 0;
  // per detector (1/sigma^2, alpha, -alpha*log2(f_samp/(n_t*fknee)), white ? 1 : 0)
  double4_32a* coef64 = nullptr;
  float4* coef32 = nullptr;
  double* wtab64 = nullptr;    // optional [n_det][n_t/2 + 1] tabulated w_d(f_k) (replaces the law)
  float* wtab32 = nullptr;
  double* diag = nullptr;      // [n_det] diag(N^-1)
  double* white = nullptr;     // [n_det] 1 / sigma^2, the white level of the law
  std::vector<double> diag_host;
  // noise correlated between detectors: N(f) = D(f) + V E(f) V^T (r modes, 0 = none)
  int corr_r = 0;
  int corr_version = 0;        // bumped by every cmm_noise_set_correlated
  float* corr_V = nullptr;     // [n_det][r] templates V
  double* corr_par = nullptr;  // [r][3] (amp, fknee, alpha) of the mode spectra
};

struct cmm_op {
  int refs = 1;                // owner reference + one per dependent handle
  cmm_ctx* ctx = nullptr;
  cmm_pointing* pt = nullptr;
  cmm_noise* nz = nullptr;
  int prec = CMM_PREC_F32;
  int64_t N = 0;               // complex length n_t / 2
  int R = 0, C = 0, logR = 0, logC = 0;
  int chunk = 0;               // detectors per pass through `spec`
  void* spec = nullptr;        // [chunk][N] complex intermediate
  void* gather = nullptr;      // [npix] map copy for the projection gather
  double* acc = nullptr;       // [npix][acc_stride] FP64 accumulator of P^T
  float* acc32 = nullptr;      // [maps][npix + 1][acc_stride] FP32 partial accumulators (fast path)
  int acc32_maps = 1;          // partial maps in acc32: one per group of detectors between flushes
  int acc_stride = 0;
  void* tw = nullptr;          // twiddle tables in the op's compute type
  int32_t* pix = nullptr;      // optional [n_det][n_samp] pixel index per sample (npix: outside)
  int pair = 1;                // A-applications on the two-detector path where it applies (tod_pair.cu)
  int pR = 0, pC = 0, plogR = 0, plogC = 0;   // split n_samp = pR pC of the two-detector sequences
  void* tw_pair = nullptr;     // their twiddle tables (FP32)
  int corr_version = 0;        // noise correlation version the tables below were built for
  float* corr_minv = nullptr;  // [N + 1][r][r] per-bin M^-1 in slot order (index N: bin N)
  float2* corr_s = nullptr;    // [N][r] cross-detector solution per bin slot
  double* tmp_a = nullptr;     // [ncomp*npix] device temporaries
  double* tmp_b = nullptr;
  const int* done = nullptr;   // solver stop flag seen by every kernel (nullptr: none)
  double* sol = nullptr;       // PCG vectors r, z, p, q, r_old and reduction partials
  void* sol_state = nullptr;   // PCG scalars (SolverDev)
  double* host_bx = nullptr;   // [2][ncomp*npix] device b and x of cmm_solve_host
  double* fcg = nullptr;       // rings of truncated flexible CG (directions, A times them, partials)
  int64_t fcg_doubles = 0;
  int resume_ready = 0;        // a solver state was loaded (cmm_solve_state_load)
  int resume_iter = 0;         // its iteration count, rho and relative residual
  double resume_rho = 0.0, resume_rel = 0.0;
};

namespace cmm {

constexpr int kRedBlocks = 1024;   // fixed grid of the deterministic reductions
constexpr int kMaxCorrModes = 4;   // correlated noise modes

// twiddle table offsets inside cmm_op::tw (in elements of V2<T>)
struct TwLayout {
  int64_t R_off, C_off, Nlo_off, N2_off, C2_off, total;
};
inline TwLayout tw_layout(int R, int C) {
  TwLayout l;
  l.R_off = 0;            // w_R^e, e < R
  l.C_off = R;            // w_C^e, e < C
  l.Nlo_off = R + C;      // w_N^e, e < C
  l.N2_off = R + 2 * C;   // w_{2N}^e, e < R
  l.C2_off = 2 * R + 2 * C;  // w_{2C}^e, e < C
  l.total = 2 * R + 3 * C;
  return l;
}

// ---- launchers implemented in tod.cu
int launch_map_to_gather(cmm_op* op, const double* m);
int launch_acc_to_map(cmm_op* op, double* out);
int launch_apply_chunk(cmm_op* op, int d0, int nd, const void* tod, int tod_is_f64, int pass = -1);
int launch_project(cmm_op* op, const double* m, void* tod, int tod_is_f64);
int launch_hit_blocks(cmm_pointing* pt, const double* det_weight, const uint8_t* mask,
                      double* blocks, const int* done);
int op_init_twiddles(cmm_op* op);
int op_prepare_kernels(cmm_op* op);
int launch_fill_pixels(cmm_op* op);
int launch_corr_minv(cmm_op* op, const double* mode_par_dev, float* minv);
int op_sync_corr(cmm_op* op);
bool fast_path_ok(const cmm_op* op);
bool fast_path_sizes(int logN, int prec, int* logR, int* logC);
// ---- two-detector path (tod_pair.cu)
bool pair_path_ok(const cmm_op* op);
bool pair_path_sizes(int log_nt, int prec, int* logR, int* logC);
int launch_apply_chunk_pair(cmm_op* op, int d0, int nd, int pass);
int prepare_pair(cmm_op* op);

// ---- handle lifetimes: a handle stays alive while handles made from it exist, so
// they may be destroyed in any order (api.cu, unet.cu)
void ctx_retain(cmm_ctx* c);
void ctx_release(cmm_ctx* c);
void unet_retain(cmm_unet* u);
void unet_release(cmm_unet* u);

// ---- learned correction (unet.cu)
int unet_correct(cmm_unet* u, const double* r, double* z, const uint8_t* mask, int64_t npix, int ncomp,
                 const int* done, cudaStream_t st);
bool unet_matches(const cmm_unet* u, const cmm_ctx* ctx, int ny, int nx);

// ---- launchers implemented in map.cu
int launch_mask_from_hits(cmm_pointing* pt, const double* blocks);
int launch_block_inverse(int ncomp, int64_t npix, const double* blocks, const uint8_t* mask,
                         double* inv, cudaStream_t s);
int launch_block_sqrt(int ncomp, int64_t npix, const double* blocks, const uint8_t* mask,
                      double* sig, double* sig_inv, cudaStream_t s);
int launch_block_apply(int ncomp, int64_t npix, const double* blocks, const double* x,
                       double* y, const int* done, cudaStream_t s);
int launch_dot(const double* x, const double* y, int64_t n, double* partial, double* out,
               const int* done, cudaStream_t s);
int launch_sub(double* r, const double* b, const double* q, int64_t n, cudaStream_t s);

}  // namespace cmm
