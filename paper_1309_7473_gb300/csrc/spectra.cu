// Flat-sky angular power spectra of TQU maps, binned in multipole: the convergence
// diagnostic of the paper's Results section (spectra of the PCG iterates against
// the spectrum of the input map, in units of cosmic variance).
//
// For a map of ny x nx square pixels of side `pix` (radians) the 2-D DFT X(k) of
// each component gives the modes l = 2 pi (ky / (ny pix), kx / (nx pix)) with signed
// frequencies; E and B are the rotations of (Q, U) by twice the mode's angle
// phi = atan2(ly, lx): E = Q cos 2phi + U sin 2phi, B = -Q sin 2phi + U cos 2phi.
// C_b = pix^2 / (ny nx) * mean over the modes of bin b of |X|^2, for TT, EE and BB;
// bin b holds lmax b / nbins <= |l| < lmax (b + 1) / nbins (l = 0 excluded).
// cmm_spectra_converged_at turns the spectra of a sequence of iterates into the
// Results section's count: the iteration from which each bin stays within a
// fraction of cosmic variance of the input map's spectrum (host arithmetic on a
// few hundred numbers).
#include <cmath>

#include <vector>

#include "common.cuh"
#include "map_kernels.cuh"

namespace cmm {
namespace {

// Per-block bin sums in shared memory, then one global atomic per bin and block.
__global__ void k_spectra_bin(const double2* __restrict__ planes, int ny, int nx, double pix, int nbins,
                              double lmax, double* __restrict__ sums, unsigned long long* __restrict__ counts) {
  extern __shared__ double sh[];   // [3][nbins] sums, then [nbins] counts
  double* s = sh;
  double* c = sh + 3 * nbins;
  for (int q = threadIdx.x; q < 4 * nbins; q += blockDim.x) sh[q] = 0.0;
  __syncthreads();
  const long long npix = (long long)ny * nx;
  const double two_pi = 6.283185307179586476925287;
  const double bw = lmax / nbins;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < npix;
       f += (long long)gridDim.x * blockDim.x) {
    const int ky = (int)(f / nx), kx = (int)(f - (long long)ky * nx);
    const int sy = ky <= ny / 2 ? ky : ky - ny;
    const int sx = kx <= nx / 2 ? kx : kx - nx;
    const double ly = two_pi * sy / (ny * pix), lx = two_pi * sx / (nx * pix);
    const double l = sqrt(lx * lx + ly * ly);
    if (l == 0.0) continue;
    const int b = (int)(l / bw);
    if (b >= nbins) continue;
    const double phi = atan2(ly, lx);
    double s2, c2;
    sincos(2.0 * phi, &s2, &c2);
    const double2 T = planes[f], Q = planes[npix + f], U = planes[2 * npix + f];
    const double Er = Q.x * c2 + U.x * s2, Ei = Q.y * c2 + U.y * s2;
    const double Br = -Q.x * s2 + U.x * c2, Bi = -Q.y * s2 + U.y * c2;
    atomicAdd(&s[b], T.x * T.x + T.y * T.y);
    atomicAdd(&s[nbins + b], Er * Er + Ei * Ei);
    atomicAdd(&s[2 * nbins + b], Br * Br + Bi * Bi);
    atomicAdd(&c[b], 1.0);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 3 * nbins; q += blockDim.x)
    if (s[q] != 0.0) atomicAdd(&sums[q], s[q]);
  for (int q = threadIdx.x; q < nbins; q += blockDim.x)
    if (c[q] != 0.0) atomicAdd(&counts[q], (unsigned long long)c[q]);
}

}  // namespace
}  // namespace cmm

using namespace cmm;

extern "C" {

int cmm_spectra(cmm_ctx* ctx, int32_t ny, int32_t nx, double pix_rad, int32_t nmaps, const double* maps,
                int32_t nbins, double lmax, double* cls_host, int64_t* nmodes_host) {
  if (!ctx || !maps || !cls_host || ny <= 0 || nx <= 0 || nmaps <= 0 || nbins <= 0 || nbins > 1024 ||
      !(pix_rad > 0) || !(lmax > 0))
    return fail(CMM_ERR_ARG, "bad argument");
  CMM_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const long long npix = (long long)ny * nx;
  Fft2Plan plan;
  CMM_TRY(fft2_plan_init<double>(plan, ny, nx));
  double2* planes = nullptr;
  double* sums = nullptr;
  unsigned long long* counts = nullptr;
  int s = CMM_OK;
  if (cudaMalloc(&planes, sizeof(double2) * 3 * npix) != cudaSuccess ||
      cudaMalloc(&sums, sizeof(double) * 3 * nbins) != cudaSuccess ||
      cudaMalloc(&counts, sizeof(unsigned long long) * nbins) != cudaSuccess)
    s = fail(CMM_ERR_OOM, "spectra work buffers");
  std::vector<double> h(3 * nbins);
  std::vector<unsigned long long> hc(nbins);
  const int blocks = (int)std::min<long long>((npix + 255) / 256, 1024);
  const size_t smem = sizeof(double) * 4 * nbins;
  for (int m = 0; m < nmaps && s == CMM_OK; ++m) {
    s = [&]() -> int {
      CMM_TRY(launch_real_to_planes<double>(maps + (size_t)m * 3 * npix, planes, 3 * npix, nullptr, st));
      CMM_TRY(fft2<double>(plan, planes, 3, -1, nullptr, st));
      CMM_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * 3 * nbins, st));
      CMM_CUDA(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * nbins, st));
      k_spectra_bin<<<blocks, 256, smem, st>>>(planes, ny, nx, pix_rad, nbins, lmax, sums, counts);
      CMM_LAUNCH_CHECK();
      CMM_CUDA(cudaMemcpyAsync(h.data(), sums, sizeof(double) * 3 * nbins, cudaMemcpyDeviceToHost, st));
      CMM_CUDA(cudaMemcpyAsync(hc.data(), counts, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, st));
      CMM_CUDA(cudaStreamSynchronize(st));
      const double norm = pix_rad * pix_rad / (double)npix;
      for (int c = 0; c < 3; ++c)
        for (int b = 0; b < nbins; ++b)
          cls_host[((size_t)m * 3 + c) * nbins + b] = hc[b] ? h[c * nbins + b] * norm / (double)hc[b] : 0.0;
      if (m == 0 && nmodes_host)
        for (int b = 0; b < nbins; ++b) nmodes_host[b] = (int64_t)hc[b];
      return CMM_OK;
    }();
  }
  cudaStreamSynchronize(st);
  if (planes) cudaFree(planes);
  if (sums) cudaFree(sums);
  if (counts) cudaFree(counts);
  if (plan.tw) cudaFree(plan.tw);
  return s;
}

int cmm_spectra_converged_at(int32_t n_snap, const int32_t* iters, int32_t nspec, int32_t nbins,
                             const double* cls_iter, const double* cls_true, const int64_t* nmodes, double level,
                             int32_t* out) {
  if (n_snap <= 0 || nspec <= 0 || nbins <= 0 || !iters || !cls_iter || !cls_true || !nmodes || !out ||
      !(level > 0))
    return fail(CMM_ERR_ARG, "bad argument");
  for (int c = 0; c < nspec; ++c)
    for (int b = 0; b < nbins; ++b) {
      const size_t cb = (size_t)c * nbins + b;
      // cosmic variance of the bin: C_b sqrt(2 / n_b) over its n_b modes
      const double sigma = cls_true[cb] * std::sqrt(2.0 / (double)std::max<int64_t>(nmodes[b], 1));
      int last_far = -1;   // last snapshot whose error is level sigma or more
      for (int k = 0; k < n_snap; ++k) {
        const double e = std::fabs(cls_iter[(size_t)k * nspec * nbins + cb] - cls_true[cb]);
        if (sigma > 0 ? e >= level * sigma : false) last_far = k;
      }
      out[cb] = last_far + 1 < n_snap ? iters[last_far + 1] : -1;
    }
  return CMM_OK;
}

}  // extern "C"
