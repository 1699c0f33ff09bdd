// Declarations shared between map.cu (pixel-space kernels) and api.cu (host runtime).
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace cmm {

// Scalars of one PCG solve, kept in device memory so that an iteration can be
// replayed as a CUDA graph; every kernel of the loop returns early once `done`.
constexpr int kMaxWin = 8;   // directions kept by truncated flexible CG, FCG(m)

struct SolverDev {
  double rho, pq, alpha, beta, rr, rel, bnorm2, tol;
  int iter, maxit, done, status;
  int f32;        // FP32 CG vectors and scalars
  int win;        // FCG(m): m > 1 directions kept (ring slot j mod m); <= 1: PCG / Polak-Ribiere
  double pq_ring[kMaxWin];   // p_j^T A p_j of the kept directions
  double beta_w[kMaxWin];    // coefficients of the new direction on them
};

struct Fft2Plan {
  int ny = 0, nx = 0;
  bool f64 = false;
  MixedPlan py{}, px{};
  void* tw = nullptr;   // [nx] w_nx^e then [ny] w_ny^e
};

// Block-wide (256 threads) sum of `v`, stored to partial[blockIdx.x] (fixed order).
__device__ __forceinline__ void block_sum_store(double v, double* partial) {
  __shared__ double sh[256];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// Sum of n partials by one block of 256 threads in a fixed order; result in every thread.
__device__ __forceinline__ double block_sum_all(const double* partial, int n) {
  __shared__ double sh2[256];
  __syncthreads();
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  sh2[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh2[threadIdx.x] += sh2[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh2[0];
  __syncthreads();
  return r;
}

int launch_block_apply_dot(int ncomp, int64_t npix, const double* blk, const double* x, double* y,
                           const double* w, double* partial, const int* done, cudaStream_t s);
// y = d .* x and z = (first ? 0 : z) + d .* x on every Stokes component (d [npix])
int launch_window_mul(const double* d, const double* x, double* y, int64_t npix, int ncomp, const int* done,
                      cudaStream_t s);
int launch_window_acc(const double* d, const double* x, double* z, int64_t npix, int ncomp, bool first,
                      const int* done, cudaStream_t s);
int launch_dot_partial(const double* x, const double* y, int64_t n, double* partial, const int* done,
                       cudaStream_t s);
int launch_copy_sub(double* dst, const double* a, const double* b, int64_t n, cudaStream_t s);
int launch_solver_init(SolverDev* st, const double* prz, const double* prr, double* hist, cudaStream_t s);
int launch_solver_alpha(SolverDev* st, const double* partial, double* anorm, cudaStream_t s);
int launch_update_xr(double* x, double* r, double* r_old, const double* p, const double* q, int64_t n,
                     const SolverDev* st, double* partial, cudaStream_t s);
int launch_dot_partial_cg(const double* x, const double* y, int64_t n, const SolverDev* st, double* partial,
                          cudaStream_t s);
int launch_solver_z(double* z, const double* r, const double* r_old, int64_t n, const SolverDev* st,
                    double* p_rz, double* p_flex, cudaStream_t s);
int launch_residual(double* r, const double* b, const double* q, int64_t n, const SolverDev* st, double* partial,
                    cudaStream_t s);
int launch_solver_rho(SolverDev* st, const double* p_rz, cudaStream_t s);
int launch_snapshot(const double* x, const double* r, int64_t n, const SolverDev* st, int every, int max,
                    double* snaps, cudaStream_t s);
int launch_solver_check(SolverDev* st, const double* partial, double* hist, cudaStream_t s);
int launch_solver_beta(SolverDev* st, const double* p_rz, const double* p_flex, cudaStream_t s);
int launch_update_p(double* p, const double* z, int64_t n, const SolverDev* st, cudaStream_t s);
// FCG(m): x, r update storing p and q = A p in the ring; z^T Q_j partials; the
// coefficients; p = z + sum_j beta_j P_j with the partials of p^T r; rho = p^T r.
int launch_update_xr_ring(double* x, double* r, const double* p, const double* q, int64_t n, const SolverDev* st,
                          double* P, double* Q, double* partial, cudaStream_t s);
int launch_window_dots(const double* z, const double* Q, int64_t n, const SolverDev* st, double* wpart,
                       cudaStream_t s);
int launch_window_beta(SolverDev* st, const double* wpart, cudaStream_t s);
int launch_update_p_window(double* p, const double* z, const double* P, const double* r, int64_t n,
                           const SolverDev* st, double* partial, cudaStream_t s);
int launch_solver_rho_pr(SolverDev* st, const double* partial, cudaStream_t s);

template <typename T> int fft2_plan_init(Fft2Plan& p, int ny, int nx);
template <typename T> int fft2(const Fft2Plan& p, V2<T>* data, int nplanes, int sign, const int* done, cudaStream_t s);
template <typename T>
int launch_circ_q(int ncomp, const double* rows, const double* sig_inv, int ref, int ny, int nx,
                  double taper_sigma, V2<T>* planes, cudaStream_t s);
template <typename T>
int launch_mode_inverse(int ncomp, const V2<T>* planes, long long npix, double eps, double* hinv,
                        unsigned long long* scratch2, cudaStream_t s);
template <typename T>
int launch_real_to_planes(const double* x, V2<T>* planes, long long n, const int* done, cudaStream_t s);
template <typename T>
int launch_block_to_planes(int ncomp, int64_t npix, const double* blk, const double* x, V2<T>* planes,
                           const int* done, cudaStream_t s);
template <typename T>
int launch_planes_block_dot(int ncomp, int64_t npix, const V2<T>* planes, double scale, const double* blk, double* y,
                            const double* w, double* partial, const int* done, cudaStream_t s);
template <typename T>
int launch_planes_to_real(const V2<T>* planes, double* x, long long n, double scale, const int* done,
                          cudaStream_t s);
template <typename T, typename H>
int launch_mode_apply(int ncomp, V2<T>* planes, const H* hinv, long long npix, const int* done,
                      cudaStream_t s);
int launch_to_f32(const double* x, float* y, long long n, cudaStream_t s);
template <typename T, typename B>
int launch_block_to_planes_packed(int64_t npix, const B* blk, const double* x, V2<T>* planes, const int* done,
                                  cudaStream_t s);
template <typename T, typename B>
int launch_planes_block_dot_packed(int64_t npix, const V2<T>* planes, double scale, const B* blk, double* y,
                                   const double* w, double* partial, const int* done, cudaStream_t s);
template <typename T, typename H>
int launch_mode_apply_packed(V2<T>* planes, const H* hinv, int ny, int nx, const int* done, cudaStream_t s);

}  // namespace cmm
