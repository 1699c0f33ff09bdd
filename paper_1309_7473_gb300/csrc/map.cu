// Pixel-space work of the map-maker: pixel masks, the binned / Jacobi block
// preconditioners (Eq. 3-5), the circulant preconditioner (Eq. 7-13), the 2-D map
// FFTs it needs, and the FP64 vector kernels of preconditioned conjugate gradients.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "map_kernels.cuh"

namespace cmm {

// ------------------------------------------------------------------ small dense algebra

// Cyclic Jacobi eigen-decomposition of a real symmetric n x n matrix (n <= 6):
// a is overwritten (its diagonal holds the eigenvalues), v receives eigenvectors
// as columns.
template <int n>
__device__ void jacobi_eigen(double (&a)[n][n], double (&v)[n][n]) {
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = 0; j < n; ++j) v[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0, diag = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      diag += a[i][i] * a[i][i];
#pragma unroll
      for (int j = i + 1; j < n; ++j) off += a[i][j] * a[i][j];
    }
    if (off <= 1e-34 * diag || off == 0.0) break;
#pragma unroll
    for (int p = 0; p < n - 1; ++p) {
#pragma unroll
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
        double t;
        if (fabs(theta) > 1e150) t = 0.5 / theta;
        else t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0);
        const double s = t * c;
        // A <- G^T A G with G = I except G_pp = G_qq = c, G_pq = s, G_qp = -s
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        a[p][q] = 0.0;
        a[q][p] = 0.0;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
    }
  }
}

__device__ __forceinline__ void sym3_load(const double* b, double (&a)[3][3]) {
  a[0][0] = b[0]; a[0][1] = b[1]; a[0][2] = b[2];
  a[1][0] = b[1]; a[1][1] = b[3]; a[1][2] = b[4];
  a[2][0] = b[2]; a[2][1] = b[4]; a[2][2] = b[5];
}

__device__ __forceinline__ void sym3_store(double* b, const double (&a)[3][3]) {
  b[0] = a[0][0]; b[1] = a[0][1]; b[2] = a[0][2];
  b[3] = a[1][1]; b[4] = a[1][2]; b[5] = a[2][2];
}

// ------------------------------------------------------------------ masks and blocks

// A pixel is kept when its unit-weight hit block has hits and reciprocal condition
// number >= 1e-3 (eigenvalues of the symmetric 3x3 block).
template <int NC>
__global__ void k_mask_from_hits(const double* __restrict__ blocks, uint8_t* __restrict__ mask,
                                 long long npix, unsigned long long* __restrict__ n_good,
                                 unsigned long long* __restrict__ max_hits) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    bool ok;
    if (NC == 1) {
      ok = blocks[p] > 0.0;
    } else {
      double a[3][3], v[3][3];
      sym3_load(blocks + 6 * p, a);
      jacobi_eigen<3>(a, v);
      const double l0 = a[0][0], l1 = a[1][1], l2 = a[2][2];
      const double lmax = fmax(l0, fmax(l1, l2));
      const double lmin = fmin(l0, fmin(l1, l2));
      ok = (lmax > 0.0) && (lmin >= 1e-3 * lmax);
    }
    mask[p] = ok ? 1 : 0;
    if (ok) atomicAdd(n_good, 1ULL);
    // unit-weight blocks: the (T, T) entry is the pixel's sample count
    const double hits = NC == 1 ? blocks[p] : blocks[6 * p];
    if (hits > 0.0) atomicMax(max_hits, (unsigned long long)hits);
  }
}

// inv = B^-1 per unmasked pixel (0 on masked pixels), B symmetric packed.
template <int NC>
__global__ void k_block_inverse(const double* __restrict__ blocks, const uint8_t* __restrict__ mask,
                                double* __restrict__ inv, long long npix) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      inv[p] = mask[p] ? 1.0 / blocks[p] : 0.0;
      continue;
    }
    const double* b = blocks + 6 * p;
    double* o = inv + 6 * p;
    if (!mask[p]) {
      for (int i = 0; i < 6; ++i) o[i] = 0.0;
      continue;
    }
    const double a00 = b[0], a01 = b[1], a02 = b[2], a11 = b[3], a12 = b[4], a22 = b[5];
    const double c00 = a11 * a22 - a12 * a12;
    const double c01 = a02 * a12 - a01 * a22;
    const double c02 = a01 * a12 - a02 * a11;
    const double c11 = a00 * a22 - a02 * a02;
    const double c12 = a01 * a02 - a00 * a12;
    const double c22 = a00 * a11 - a01 * a01;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    const double r = 1.0 / det;
    o[0] = c00 * r; o[1] = c01 * r; o[2] = c02 * r;
    o[3] = c11 * r; o[4] = c12 * r; o[5] = c22 * r;
  }
}

// Sigma = B^(1/2), Sigma^-1 = B^(-1/2) (symmetric) per unmasked pixel.
template <int NC>
__global__ void k_block_sqrt(const double* __restrict__ blocks, const uint8_t* __restrict__ mask,
                             double* __restrict__ sig, double* __restrict__ sig_inv, long long npix) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      const double b = blocks[p];
      sig[p] = mask[p] ? sqrt(b) : 0.0;
      sig_inv[p] = mask[p] ? 1.0 / sqrt(b) : 0.0;
      continue;
    }
    double* s = sig + 6 * p;
    double* si = sig_inv + 6 * p;
    if (!mask[p]) {
      for (int i = 0; i < 6; ++i) s[i] = si[i] = 0.0;
      continue;
    }
    double a[3][3], v[3][3];
    sym3_load(blocks + 6 * p, a);
    jacobi_eigen<3>(a, v);
    double r[3], ri[3];
    for (int k = 0; k < 3; ++k) {
      r[k] = sqrt(a[k][k]);
      ri[k] = 1.0 / r[k];
    }
    double m[3][3], mi[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double x = 0, y = 0;
        for (int k = 0; k < 3; ++k) {
          x += v[i][k] * r[k] * v[j][k];
          y += v[i][k] * ri[k] * v[j][k];
        }
        m[i][j] = x;
        mi[i][j] = y;
      }
    sym3_store(s, m);
    sym3_store(si, mi);
  }
}

// y = blk x per pixel (blk symmetric packed); optional partial of dot(w, y).
template <int NC>
__global__ void k_block_apply(const double* __restrict__ blk, const double* __restrict__ x,
                              double* __restrict__ y, long long npix, const double* __restrict__ w,
                              double* __restrict__ partial, const int* done) {
  if (done && *done) return;
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      const double v = blk[p] * x[p];
      y[p] = v;
      if (w) acc += w[p] * v;
    } else {
      const double* b = blk + 6 * p;
      const double x0 = x[p], x1 = x[npix + p], x2 = x[2 * npix + p];
      const double y0 = b[0] * x0 + b[1] * x1 + b[2] * x2;
      const double y1 = b[1] * x0 + b[3] * x1 + b[4] * x2;
      const double y2 = b[2] * x0 + b[4] * x1 + b[5] * x2;
      y[p] = y0;
      y[npix + p] = y1;
      y[2 * npix + p] = y2;
      if (w) acc += w[p] * y0 + w[npix + p] * y1 + w[2 * npix + p] * y2;
    }
  }
  if (partial) block_sum_store(acc, partial);
}

// ------------------------------------------------------------------ reductions
// r = b - q (the true residual once A x is in q)
__global__ void k_sub(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ q,
                      long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - q[i];
}

__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, long long n,
                              double* __restrict__ partial, const int* done) {
  if (done && *done) return;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  block_sum_store(acc, partial);
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out,
                               const int* done) {
  if (done && *done) return;
  const double s = block_sum_all(partial, n);
  if (threadIdx.x == 0) *out = s;
}

// ------------------------------------------------------------------ PCG state machine
// With st->f32 the CG vectors, dot products and scalars are rounded to FP32
// (the FP32-CG precision mode); the operator and preconditioner are unchanged.
__device__ __forceinline__ double cg_round(const SolverDev* st, double v) { return st->f32 ? (double)(float)v : v; }

__device__ __forceinline__ double cg_acc(const SolverDev* st, double acc, double term) {
  return st->f32 ? (double)((float)acc + (float)term) : acc + term;
}

__global__ void k_solver_alpha(SolverDev* st, const double* __restrict__ partial, double* anorm_terms) {
  if (st->done) return;
  const double pq = block_sum_all(partial, kRedBlocks);
  if (threadIdx.x == 0) {
    st->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(st->rho)) {
      st->status = CMM_ERR_BREAKDOWN;
      st->done = 1;
      st->alpha = 0.0;
      return;
    }
    st->alpha = cg_round(st, st->rho / pq);
    if (anorm_terms) anorm_terms[st->iter] = st->alpha * st->rho;
    if (st->win > 1) st->pq_ring[st->iter % st->win] = pq;
  }
}

__global__ void k_dot_partial_cg(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                 const SolverDev* st, double* __restrict__ partial) {
  if (st->done) return;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = cg_acc(st, acc, x[i] * y[i]);
  block_sum_store(acc, partial);
}

// x += alpha p; r -= alpha q (r_old keeps the previous residual for flexible CG)
__global__ void k_update_xr(double* __restrict__ x, double* __restrict__ r, double* __restrict__ r_old,
                            const double* __restrict__ p, const double* __restrict__ q, long long n,
                            const SolverDev* st, double* __restrict__ partial) {
  if (st->done) return;
  const double alpha = st->alpha;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = cg_round(st, x[i] + alpha * p[i]);
    const double r0 = r[i];
    if (r_old) r_old[i] = r0;
    const double ri = cg_round(st, r0 - alpha * q[i]);
    r[i] = ri;
    acc = cg_acc(st, acc, ri * ri);
  }
  block_sum_store(acc, partial);
}

__global__ void k_solver_check(SolverDev* st, const double* __restrict__ partial, double* hist) {
  if (st->done) return;
  const double rr = block_sum_all(partial, kRedBlocks);
  if (threadIdx.x == 0) {
    st->rr = rr;
    st->iter += 1;
    const double rel = sqrt(rr / st->bnorm2);
    if (hist) hist[st->iter] = rel;
    if (!isfinite(rr)) {
      st->status = CMM_ERR_BREAKDOWN;   // st->rel keeps the last finite residual
      st->done = 1;
      return;
    }
    st->rel = rel;
    if (rel <= st->tol) {
      st->status = CMM_OK;
      st->done = 1;
    } else if (st->iter >= st->maxit) {
      st->status = CMM_ERR_NOT_CONVERGED;
      st->done = 1;
    }
  }
}

// After z = M r: round z (FP32 CG), partials of r^T z and, for flexible CG, of
// z^T (r - r_old).
__global__ void k_solver_z(double* __restrict__ z, const double* __restrict__ r, const double* __restrict__ r_old,
                           long long n, const SolverDev* st, double* __restrict__ p_rz,
                           double* __restrict__ p_flex) {
  if (st->done) return;
  double a1 = 0.0, a2 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double zi = cg_round(st, z[i]);
    z[i] = zi;
    const double ri = r[i];
    a1 = cg_acc(st, a1, ri * zi);
    if (r_old) a2 = cg_acc(st, a2, zi * (ri - r_old[i]));
  }
  block_sum_store(a1, p_rz);
  if (r_old) {
    __syncthreads();
    block_sum_store(a2, p_flex);
  }
}

// beta = rz_new / rz (Fletcher-Reeves form of PCG) or z^T (r - r_old) / rz (flexible)
__global__ void k_solver_beta(SolverDev* st, const double* __restrict__ p_rz, const double* __restrict__ p_flex) {
  if (st->done) return;
  const double rz = block_sum_all(p_rz, kRedBlocks);
  double fl = 0.0;
  if (p_flex) fl = block_sum_all(p_flex, kRedBlocks);
  if (threadIdx.x == 0) {
    if (!(rz > 0.0) || !isfinite(rz) || !isfinite(fl)) {
      st->status = CMM_ERR_BREAKDOWN;
      st->done = 1;
      return;
    }
    st->beta = cg_round(st, (p_flex ? fl : rz) / st->rho);
    st->rho = rz;
  }
}

__global__ void k_update_p(double* __restrict__ p, const double* __restrict__ z, long long n,
                           const SolverDev* st) {
  if (st->done) return;
  const double beta = st->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = cg_round(st, z[i] + beta * p[i]);
}

// Initialisation after r0, z0 are known: rho = r^T z (partial), bnorm2 set by host.
__global__ void k_solver_init(SolverDev* st, const double* __restrict__ partial_rz,
                              const double* __restrict__ partial_rr, double* hist) {
  const double rz = block_sum_all(partial_rz, kRedBlocks);
  __syncthreads();
  const double rr = block_sum_all(partial_rr, kRedBlocks);
  if (threadIdx.x == 0) {
    st->rho = rz;
    st->iter = 0;
    const double rel = sqrt(rr / st->bnorm2);
    st->rel = isfinite(rel) ? rel : -1.0;   // -1: the starting residual is not finite
    if (hist) hist[0] = rel;
    st->done = 0;
    st->status = CMM_ERR_NOT_CONVERGED;
    if (rel <= st->tol) {
      st->status = CMM_OK;
      st->done = 1;
    } else if (!isfinite(rel) || !(rz > 0.0) || !isfinite(rz)) {
      st->status = CMM_ERR_BREAKDOWN;
      st->done = 1;
    } else if (st->maxit <= 0) {
      st->done = 1;
    }
  }
}

// ------------------------------------------------------------------ truncated flexible CG, FCG(m)
// The last m = st->win directions p_j and q_j = A p_j live in rings P, Q ([m][n],
// direction of iteration j in slot j mod m) with p_j^T q_j in st->pq_ring.  The new
// direction is z made A-conjugate to them, p = z - sum_j (z^T q_j / p_j^T q_j) p_j,
// and the step uses rho = p^T r (Notay's FCG).

// x += alpha p; r -= alpha q; p and q into ring slot iter mod m; partials of r^T r
__global__ void k_update_xr_ring(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                                 const double* __restrict__ q, long long n, const SolverDev* st,
                                 double* __restrict__ P, double* __restrict__ Q, double* __restrict__ partial) {
  if (st->done) return;
  const double alpha = st->alpha;
  const long long slot = st->iter % st->win;
  double* Ps = P + slot * n;
  double* Qs = Q + slot * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double pi = p[i], qi = q[i];
    x[i] = cg_round(st, x[i] + alpha * pi);
    const double ri = cg_round(st, r[i] - alpha * qi);
    r[i] = ri;
    Ps[i] = pi;
    Qs[i] = qi;
    acc = cg_acc(st, acc, ri * ri);
  }
  block_sum_store(acc, partial);
}

// partials of z^T Q_j for the kept directions j < min(iter, m): wpart[j][block]
__global__ void k_window_dots(const double* __restrict__ z, const double* __restrict__ Q, long long n,
                              const SolverDev* st, double* __restrict__ wpart) {
  if (st->done) return;
  const int nv = min(st->iter, st->win);
  double acc[kMaxWin];
#pragma unroll
  for (int j = 0; j < kMaxWin; ++j) acc[j] = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double zi = z[i];
#pragma unroll
    for (int j = 0; j < kMaxWin; ++j)
      if (j < nv) acc[j] = cg_acc(st, acc[j], zi * Q[j * n + i]);
  }
#pragma unroll
  for (int j = 0; j < kMaxWin; ++j) {
    if (j < nv) {
      __syncthreads();
      block_sum_store(acc[j], wpart + (long long)j * kRedBlocks);
    }
  }
}

// beta_j = -z^T q_j / p_j^T q_j
__global__ void k_window_beta(SolverDev* st, const double* __restrict__ wpart) {
  if (st->done) return;
  const int nv = min(st->iter, st->win);
  for (int j = 0; j < nv; ++j) {
    const double zq = block_sum_all(wpart + (long long)j * kRedBlocks, kRedBlocks);
    if (threadIdx.x == 0) {
      const double b = -zq / st->pq_ring[j];
      st->beta_w[j] = cg_round(st, b);
      if (!isfinite(b)) {
        st->status = CMM_ERR_BREAKDOWN;
        st->done = 1;
      }
    }
  }
}

// p = z + sum_j beta_j P_j; partials of p^T r
__global__ void k_update_p_window(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ P,
                                  const double* __restrict__ r, long long n, const SolverDev* st,
                                  double* __restrict__ partial) {
  if (st->done) return;
  const int nv = min(st->iter, st->win);
  double beta[kMaxWin];
#pragma unroll
  for (int j = 0; j < kMaxWin; ++j) beta[j] = j < nv ? st->beta_w[j] : 0.0;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double v = z[i];
#pragma unroll
    for (int j = 0; j < kMaxWin; ++j)
      if (j < nv) v += beta[j] * P[j * n + i];
    v = cg_round(st, v);
    p[i] = v;
    acc = cg_acc(st, acc, v * r[i]);
  }
  block_sum_store(acc, partial);
}

// rho = p^T r, the numerator of the next step
__global__ void k_solver_rho_pr(SolverDev* st, const double* __restrict__ partial) {
  if (st->done) return;
  const double pr = block_sum_all(partial, kRedBlocks);
  if (threadIdx.x == 0) {
    if (!(pr > 0.0) || !isfinite(pr)) {
      st->status = CMM_ERR_BREAKDOWN;
      st->done = 1;
      return;
    }
    st->rho = cg_round(st, pr);
  }
}

// Iterate snapshots: at iterations k = 0, every, 2 every, ... (slot k / every < max)
// (x_k, r_k) are copied to snaps[slot][0] and snaps[slot][1].
__global__ void k_snapshot(const double* __restrict__ x, const double* __restrict__ r, long long n,
                           const SolverDev* st, int every, int max, double* __restrict__ snaps) {
  const int it = st->iter;
  if (it % every) return;
  const int slot = it / every;
  if (slot >= max) return;
  double* dst = snaps + (long long)slot * 2 * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    dst[i] = x[i];
    dst[n + i] = r[i];
  }
}

// Residual replacement: r = b - A x (already in q as A x), rounded for FP32 CG.
__global__ void k_residual(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ q,
                           long long n, const SolverDev* st, double* __restrict__ partial) {
  if (st->done) return;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ri = cg_round(st, b[i] - q[i]);
    r[i] = ri;
    acc = cg_acc(st, acc, ri * ri);
  }
  block_sum_store(acc, partial);
}

// After a residual replacement: rho = r^T z of the new residual.
__global__ void k_solver_rho(SolverDev* st, const double* __restrict__ p_rz) {
  if (st->done) return;
  const double rz = block_sum_all(p_rz, kRedBlocks);
  if (threadIdx.x == 0) {
    if (!(rz > 0.0) || !isfinite(rz)) {
      st->status = CMM_ERR_BREAKDOWN;
      st->done = 1;
      return;
    }
    st->rho = rz;
  }
}

__global__ void k_copy_sub(double* __restrict__ dst, const double* __restrict__ a, const double* __restrict__ b,
                           long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = b ? a[i] - b[i] : a[i];
}

// ------------------------------------------------------------------ circulant preconditioner

// q_{ab}(k) = 1/2 (Q_{ref a, ref+k b} + Q_{ref b, ref-k a}) g(k), with
// Q_{ref a, j b} = sum_{g,d} Sigma^-1_{ref}[g][a] rows[g][d][j] Sigma^-1_j[d][b] (Eq. 13),
// g(k) the Gaussian over wrapped offsets; written as complex planes [a][b][ny][nx].
template <typename T, int NC>
__global__ void k_circ_q(const double* __restrict__ rows, const double* __restrict__ sig_inv,
                         int ref, int ny, int nx, double inv2s2, V2<T>* __restrict__ planes) {
  const long long npix = (long long)ny * nx;
  const int ry = ref / nx, rx = ref % nx;
  double sr[NC][NC];
  if (NC == 1) {
    sr[0][0] = sig_inv[ref];
  } else {
    double t[3][3];
    sym3_load(sig_inv + 6 * (long long)ref, t);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) sr[i][j] = t[i][j];
  }
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < npix;
       k += (long long)gridDim.x * blockDim.x) {
    const int ky = (int)(k / nx), kx = (int)(k % nx);
    const int j1 = ((ry + ky) % ny) * nx + (rx + kx) % nx;
    const int j2 = ((ry - ky + ny) % ny) * nx + (rx - kx + nx) % nx;
    const int wy = (ky < (ny + 1) / 2) ? ky : ky - ny;
    const int wx = (kx < (nx + 1) / 2) ? kx : kx - nx;
    const double g = exp(-((double)wy * wy + (double)wx * wx) * inv2s2);
    double q1[NC][NC], q2[NC][NC];
    const int js[2] = {j1, j2};
    for (int w = 0; w < 2; ++w) {
      const int j = js[w];
      double sj[NC][NC];
      if (NC == 1) {
        sj[0][0] = sig_inv[j];
      } else {
        double t[3][3];
        sym3_load(sig_inv + 6 * (long long)j, t);
        for (int i = 0; i < 3; ++i)
          for (int i2 = 0; i2 < 3; ++i2) sj[i][i2] = t[i][i2];
      }
      // tmp[a][d] = sum_g sr[g][a] rows[g][d][j]
      double tmp[NC][NC];
      for (int a = 0; a < NC; ++a)
        for (int d = 0; d < NC; ++d) {
          double s = 0;
          for (int gg = 0; gg < NC; ++gg) s += sr[gg][a] * rows[((long long)gg * NC + d) * npix + j];
          tmp[a][d] = s;
        }
      for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
          double s = 0;
          for (int d = 0; d < NC; ++d) s += tmp[a][d] * sj[d][b];
          if (w == 0) q1[a][b] = s;
          else q2[a][b] = s;
        }
    }
    for (int a = 0; a < NC; ++a)
      for (int b = 0; b < NC; ++b)
        planes[(long long)(a * NC + b) * npix + k] = V2<T>{(T)(0.5 * (q1[a][b] + q2[b][a]) * g), (T)0};
  }
}

// Per Fourier mode: H_f = conj(F q)_f (Hermitian NC x NC, Eq. 11).  Pass 1 finds the
// largest eigenvalue over all modes; pass 2 writes the floored inverse, packed as
// (re d0, re d1, re d2, re/im h01, re/im h02, re/im h12) for TQU, (d0) for T.
template <typename T, int NC>
__device__ void mode_matrix(const V2<T>* __restrict__ planes, long long npix, long long f,
                            double (&m)[2 * NC][2 * NC]) {
  // real embedding [[Re H, -Im H], [Im H, Re H]] of H = conj(Fq)
  for (int a = 0; a < NC; ++a)
    for (int b = 0; b < NC; ++b) {
      const V2<T> v = planes[(long long)(a * NC + b) * npix + f];
      const double re = (double)v.x, im = -(double)v.y;   // conjugate
      m[a][b] = re;
      m[a + NC][b + NC] = re;
      m[a][b + NC] = -im;
      m[a + NC][b] = im;
    }
  // enforce exact symmetry of the embedding (H Hermitian up to rounding)
  for (int i = 0; i < 2 * NC; ++i)
    for (int j = i + 1; j < 2 * NC; ++j) {
      const double s = 0.5 * (m[i][j] + m[j][i]);
      m[i][j] = s;
      m[j][i] = s;
    }
}

template <typename T, int NC>
__global__ void k_mode_maxeig(const V2<T>* __restrict__ planes, long long npix,
                              unsigned long long* __restrict__ maxbits) {
  double local = 0.0;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < npix;
       f += (long long)gridDim.x * blockDim.x) {
    double m[2 * NC][2 * NC], v[2 * NC][2 * NC];
    mode_matrix<T, NC>(planes, npix, f, m);
    jacobi_eigen<2 * NC>(m, v);
    for (int i = 0; i < 2 * NC; ++i) local = fmax(local, m[i][i]);
  }
  if (local > 0.0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(local));
}

template <typename T, int NC>
__global__ void k_mode_inverse(const V2<T>* __restrict__ planes, long long npix,
                               const unsigned long long* __restrict__ maxbits, double eps,
                               double* __restrict__ hinv, unsigned long long* __restrict__ nclamp) {
  const double floor_ = eps * __longlong_as_double((long long)*maxbits);
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < npix;
       f += (long long)gridDim.x * blockDim.x) {
    double m[2 * NC][2 * NC], v[2 * NC][2 * NC];
    mode_matrix<T, NC>(planes, npix, f, m);
    jacobi_eigen<2 * NC>(m, v);
    double il[2 * NC];
    int nc = 0;
    for (int i = 0; i < 2 * NC; ++i) {
      double l = m[i][i];
      if (l < floor_) {
        l = floor_;
        ++nc;
      }
      il[i] = 1.0 / l;
    }
    if (nc) atomicAdd(nclamp, (unsigned long long)nc);
    // F = V diag(il) V^T in the embedding; H^-1 = F[0:NC,0:NC] + i F[NC:2NC, 0:NC]
    double re[NC][NC], im[NC][NC];
    for (int a = 0; a < NC; ++a)
      for (int b = 0; b < NC; ++b) {
        double sr = 0, si = 0;
        for (int k = 0; k < 2 * NC; ++k) {
          sr += v[a][k] * il[k] * v[b][k];
          si += v[a + NC][k] * il[k] * v[b][k];
        }
        re[a][b] = sr;
        im[a][b] = si;
      }
    double* o = hinv + (long long)(NC == 1 ? 1 : 9) * f;
    if (NC == 1) {
      o[0] = re[0][0];
    } else {
      o[0] = re[0][0]; o[1] = re[1][1]; o[2] = re[2][2];
      o[3] = 0.5 * (re[0][1] + re[1][0]); o[4] = 0.5 * (im[0][1] - im[1][0]);
      o[5] = 0.5 * (re[0][2] + re[2][0]); o[6] = 0.5 * (im[0][2] - im[2][0]);
      o[7] = 0.5 * (re[1][2] + re[2][1]); o[8] = 0.5 * (im[1][2] - im[2][1]);
    }
  }
}

// x (real map [NC][npix]) -> complex planes
template <typename T>
__global__ void k_real_to_planes(const double* __restrict__ x, V2<T>* __restrict__ planes, long long n,
                                 const int* done) {
  if (done && *done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    planes[i] = V2<T>{(T)x[i], (T)0};
}

template <typename T>
__global__ void k_planes_to_real(const V2<T>* __restrict__ planes, double* __restrict__ x, long long n,
                                 double scale, const int* done) {
  if (done && *done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = (double)planes[i].x * scale;
}

// planes = (Sigma^-1 x, 0): the first step of the circulant apply (the 3x3 block
// apply of k_block_apply) written straight into the complex FFT planes.
template <typename T, int NC>
__global__ void k_block_to_planes(const double* __restrict__ blk, const double* __restrict__ x,
                                  V2<T>* __restrict__ planes, long long npix, const int* done) {
  if (done && *done) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      planes[p] = V2<T>{(T)(blk[p] * x[p]), (T)0};
    } else {
      const double* b = blk + 6 * p;
      const double x0 = x[p], x1 = x[npix + p], x2 = x[2 * npix + p];
      planes[p] = V2<T>{(T)(b[0] * x0 + b[1] * x1 + b[2] * x2), (T)0};
      planes[npix + p] = V2<T>{(T)(b[1] * x0 + b[3] * x1 + b[4] * x2), (T)0};
      planes[2 * npix + p] = V2<T>{(T)(b[2] * x0 + b[4] * x1 + b[5] * x2), (T)0};
    }
  }
}

// y = Sigma^-1 (scale Re planes) and the partial sums of w^T y: the last step of the
// circulant apply (k_planes_to_real followed by k_block_apply) in one pass.
template <typename T, int NC>
__global__ void k_planes_block_dot(const V2<T>* __restrict__ planes, double scale, const double* __restrict__ blk,
                                   double* __restrict__ y, long long npix, const double* __restrict__ w,
                                   double* __restrict__ partial, const int* done) {
  if (done && *done) return;
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      const double v = blk[p] * ((double)planes[p].x * scale);
      y[p] = v;
      if (w) acc += w[p] * v;
    } else {
      const double* b = blk + 6 * p;
      const double x0 = (double)planes[p].x * scale, x1 = (double)planes[npix + p].x * scale,
                   x2 = (double)planes[2 * npix + p].x * scale;
      const double y0 = b[0] * x0 + b[1] * x1 + b[2] * x2;
      const double y1 = b[1] * x0 + b[3] * x1 + b[4] * x2;
      const double y2 = b[2] * x0 + b[4] * x1 + b[5] * x2;
      y[p] = y0;
      y[npix + p] = y1;
      y[2 * npix + p] = y2;
      if (w) acc += w[p] * y0 + w[npix + p] * y1 + w[2 * npix + p] * y2;
    }
  }
  if (partial) block_sum_store(acc, partial);
}

// The three real planes of a TQU map packed into two complex ones: plane 0 holds
// T + i Q, plane 1 U (a real plane's spectrum is Hermitian, so the FFT of T + i Q
// carries both, X_T(f) = (Z(f) + conj Z(-f)) / 2 and X_Q(f) = (Z(f) - conj Z(-f)) / 2i).
// First step of the circulant apply: plane 0 = (Sigma^-1 x)_T + i (Sigma^-1 x)_Q,
// plane 1 = (Sigma^-1 x)_U.
// B: the type of Sigma^-1 and of its products (double, or float for FP32 operators,
// whose spectra are FP32: GB300's FP64 pipe bounds the FP64 form)
template <typename T, typename B>
__global__ void k_block_to_planes_packed(const B* __restrict__ blk, const double* __restrict__ x,
                                         V2<T>* __restrict__ planes, long long npix, const int* done) {
  if (done && *done) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    const B* b = blk + 6 * p;
    const B x0 = (B)x[p], x1 = (B)x[npix + p], x2 = (B)x[2 * npix + p];
    planes[p] = V2<T>{(T)(b[0] * x0 + b[1] * x1 + b[2] * x2), (T)(b[1] * x0 + b[3] * x1 + b[4] * x2)};
    planes[npix + p] = V2<T>{(T)(b[2] * x0 + b[4] * x1 + b[5] * x2), (T)0};
  }
}

// Last step, from the packed planes: t = scale (Re P0, Im P0, Re P1), y = Sigma^-1 t,
// and the partial sums of w^T y.
template <typename T, typename B>
__global__ void k_planes_block_dot_packed(const V2<T>* __restrict__ planes, double scale,
                                          const B* __restrict__ blk, double* __restrict__ y, long long npix,
                                          const double* __restrict__ w, double* __restrict__ partial,
                                          const int* done) {
  if (done && *done) return;
  double acc = 0.0;
  const B sc = (B)scale;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    const B* b = blk + 6 * p;
    const V2<T> z0 = planes[p];
    const B x0 = (B)z0.x * sc, x1 = (B)z0.y * sc, x2 = (B)planes[npix + p].x * sc;
    const double y0 = (double)(b[0] * x0 + b[1] * x1 + b[2] * x2);
    const double y1 = (double)(b[1] * x0 + b[3] * x1 + b[4] * x2);
    const double y2 = (double)(b[2] * x0 + b[4] * x1 + b[5] * x2);
    y[p] = y0;
    y[npix + p] = y1;
    y[2 * npix + p] = y2;
    if (w) acc += w[p] * y0 + w[npix + p] * y1 + w[2 * npix + p] * y2;
  }
  if (partial) block_sum_store(acc, partial);
}

// Y = H^-1 X for one mode from its packed Hermitian block (d0 d1 d2, h01 h02 h12)
template <typename H>
__device__ __forceinline__ void mode_mul3(const H* __restrict__ o, const H (&xr)[3], const H (&xi)[3], H (&yr)[3],
                                          H (&yi)[3]) {
  const H h01r = o[3], h01i = o[4], h02r = o[5], h02i = o[6], h12r = o[7], h12i = o[8];
  yr[0] = o[0] * xr[0] + (h01r * xr[1] - h01i * xi[1]) + (h02r * xr[2] - h02i * xi[2]);
  yi[0] = o[0] * xi[0] + (h01r * xi[1] + h01i * xr[1]) + (h02r * xi[2] + h02i * xr[2]);
  yr[1] = (h01r * xr[0] + h01i * xi[0]) + o[1] * xr[1] + (h12r * xr[2] - h12i * xi[2]);
  yi[1] = (h01r * xi[0] - h01i * xr[0]) + o[1] * xi[1] + (h12r * xi[2] + h12i * xr[2]);
  yr[2] = (h02r * xr[0] + h02i * xi[0]) + (h12r * xr[1] + h12i * xi[1]) + o[2] * xr[2];
  yi[2] = (h02r * xi[0] - h02i * xr[0]) + (h12r * xi[1] - h12i * xr[1]) + o[2] * xi[2];
}

// The per-mode products on the packed spectra: each thread takes a mode f and its
// mirror g = -f (when f <= g in index order), unpacks X_T, X_Q from plane 0 at f and
// g and X_U from plane 1, multiplies X(f) and X(g) = conj X(f) by their own blocks,
// and packs Y_T + i Y_Q and Y_U back at f and g.
template <typename T, typename H>
__global__ void k_mode_apply_packed(V2<T>* __restrict__ planes, const H* __restrict__ hinv, int ny, int nx,
                                    const int* done) {
  if (done && *done) return;
  const long long npix = (long long)ny * nx;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < npix;
       f += (long long)gridDim.x * blockDim.x) {
    const int ky = (int)(f / nx), kx = (int)(f - (long long)ky * nx);
    const long long g = (long long)(ky ? ny - ky : 0) * nx + (kx ? nx - kx : 0);
    if (g < f) continue;
    const V2<T> z0f = planes[f], z0g = planes[g], z1f = planes[npix + f], z1g = planes[npix + g];
    H xr[3], xi[3];
    xr[0] = (H)0.5 * ((H)z0f.x + (H)z0g.x);
    xi[0] = (H)0.5 * ((H)z0f.y - (H)z0g.y);
    xr[1] = (H)0.5 * ((H)z0f.y + (H)z0g.y);
    xi[1] = (H)0.5 * ((H)z0g.x - (H)z0f.x);
    xr[2] = (H)z1f.x;
    xi[2] = (H)z1f.y;
    H yr[3], yi[3];
    mode_mul3<H>(hinv + 9 * f, xr, xi, yr, yi);
    planes[f] = V2<T>{(T)(yr[0] - yi[1]), (T)(yi[0] + yr[1])};
    planes[npix + f] = V2<T>{(T)yr[2], (T)yi[2]};
    if (g == f) continue;
    H gr[3], gi[3], vr[3], vi[3];
    gr[0] = xr[0];
    gi[0] = -xi[0];
    gr[1] = xr[1];
    gi[1] = -xi[1];
    gr[2] = (H)z1g.x;
    gi[2] = (H)z1g.y;
    mode_mul3<H>(hinv + 9 * g, gr, gi, vr, vi);
    planes[g] = V2<T>{(T)(vr[0] - vi[1]), (T)(vi[0] + vr[1])};
    planes[npix + g] = V2<T>{(T)vr[2], (T)vi[2]};
  }
}

// y_f = H_f^-1 x_f per mode (Hermitian packed)
template <typename T, int NC, typename H>
__global__ void k_mode_apply(V2<T>* __restrict__ planes, const H* __restrict__ hinv, long long npix,
                             const int* done) {
  if (done && *done) return;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < npix;
       f += (long long)gridDim.x * blockDim.x) {
    if (NC == 1) {
      const H h = hinv[f];
      V2<T> v = planes[f];
      planes[f] = V2<T>{(T)(h * v.x), (T)(h * v.y)};
      continue;
    }
    const H* o = hinv + 9 * f;
    H xr[3], xi[3];
    for (int a = 0; a < 3; ++a) {
      const V2<T> v = planes[a * npix + f];
      xr[a] = v.x;
      xi[a] = v.y;
    }
    // H = [[d0, h01, h02], [conj h01, d1, h12], [conj h02, conj h12, d2]]
    const H h01r = o[3], h01i = o[4], h02r = o[5], h02i = o[6], h12r = o[7], h12i = o[8];
    const H y0r = o[0] * xr[0] + (h01r * xr[1] - h01i * xi[1]) + (h02r * xr[2] - h02i * xi[2]);
    const H y0i = o[0] * xi[0] + (h01r * xi[1] + h01i * xr[1]) + (h02r * xi[2] + h02i * xr[2]);
    const H y1r = (h01r * xr[0] + h01i * xi[0]) + o[1] * xr[1] + (h12r * xr[2] - h12i * xi[2]);
    const H y1i = (h01r * xi[0] - h01i * xr[0]) + o[1] * xi[1] + (h12r * xi[2] + h12i * xr[2]);
    const H y2r = (h02r * xr[0] + h02i * xi[0]) + (h12r * xr[1] + h12i * xi[1]) + o[2] * xr[2];
    const H y2i = (h02r * xi[0] - h02i * xr[0]) + (h12r * xi[1] - h12i * xr[1]) + o[2] * xi[2];
    planes[f] = V2<T>{(T)y0r, (T)y0i};
    planes[npix + f] = V2<T>{(T)y1r, (T)y1i};
    planes[2 * npix + f] = V2<T>{(T)y2r, (T)y2i};
  }
}

// Batched line FFTs over 2-D planes: `nlines` lines of length L per plane, element e
// of line l at data[plane * plane_stride + l * line_stride + e * elem_stride].
template <typename T>
__global__ void k_fft_lines(V2<T>* __restrict__ data, MixedPlan plan, int nlines, long long line_stride,
                            long long elem_stride, long long plane_stride, int lines_per_cta,
                            const V2<T>* __restrict__ tw, int sign, const int* done) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = plan.L;
  V2<T>* b0 = reinterpret_cast<V2<T>*>(smem_raw);
  V2<T>* b1 = b0 + (long long)lines_per_cta * L;
  const int l0 = blockIdx.x * lines_per_cta;
  const int nl = min(lines_per_cta, nlines - l0);
  V2<T>* base = data + blockIdx.y * plane_stride + l0 * line_stride;
  const bool minor = (elem_stride != 1);   // column lines: interleave lines in smem
  const int total = nl * L;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, e;
    if (minor) {
      l = t % nl;
      e = t / nl;
      b0[e * nl + l] = base[l * line_stride + e * elem_stride];
    } else {
      e = t % L;
      l = t / L;
      b0[l * L + e] = base[l * line_stride + e];
    }
  }
  __syncthreads();
  V2<T>* res = minor ? block_fft_mixed<T>(b0, b1, plan, nl, 1, nl, tw, sign)
                     : block_fft_mixed<T>(b0, b1, plan, nl, L, 1, tw, sign);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, e;
    if (minor) {
      l = t % nl;
      e = t / nl;
      base[l * line_stride + e * elem_stride] = res[e * nl + l];
    } else {
      e = t % L;
      l = t / L;
      base[l * line_stride + e] = res[l * L + e];
    }
  }
}

// ------------------------------------------------------------------ host launchers
static int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

int launch_mask_from_hits(cmm_pointing* pt, const double* blocks) {
  unsigned long long* d_cnt = nullptr;   // [0] unmasked pixels, [1] largest hit count
  CMM_CUDA(cudaMalloc(&d_cnt, 2 * sizeof(unsigned long long)));
  CMM_CUDA(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), pt->ctx->stream));
  if (pt->ncomp == 1)
    k_mask_from_hits<1><<<grid_for(pt->npix), 256, 0, pt->ctx->stream>>>(blocks, pt->mask, pt->npix, d_cnt,
                                                                         d_cnt + 1);
  else
    k_mask_from_hits<3><<<grid_for(pt->npix), 256, 0, pt->ctx->stream>>>(blocks, pt->mask, pt->npix, d_cnt,
                                                                         d_cnt + 1);
  CMM_LAUNCH_CHECK();
  unsigned long long h[2] = {0, 0};
  CMM_CUDA(cudaMemcpyAsync(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, pt->ctx->stream));
  CMM_CUDA(cudaStreamSynchronize(pt->ctx->stream));
  CMM_CUDA(cudaFree(d_cnt));
  pt->n_good = (int64_t)h[0];
  pt->max_hits = (int64_t)h[1];
  return CMM_OK;
}

int launch_block_inverse(int ncomp, int64_t npix, const double* blocks, const uint8_t* mask, double* inv,
                         cudaStream_t s) {
  if (ncomp == 1) k_block_inverse<1><<<grid_for(npix), 256, 0, s>>>(blocks, mask, inv, npix);
  else k_block_inverse<3><<<grid_for(npix), 256, 0, s>>>(blocks, mask, inv, npix);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_block_sqrt(int ncomp, int64_t npix, const double* blocks, const uint8_t* mask, double* sig,
                      double* sig_inv, cudaStream_t s) {
  if (ncomp == 1) k_block_sqrt<1><<<grid_for(npix), 256, 0, s>>>(blocks, mask, sig, sig_inv, npix);
  else k_block_sqrt<3><<<grid_for(npix), 256, 0, s>>>(blocks, mask, sig, sig_inv, npix);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_block_apply_dot(int ncomp, int64_t npix, const double* blk, const double* x, double* y,
                           const double* w, double* partial, const int* done, cudaStream_t s) {
  const int g = partial ? kRedBlocks : grid_for(npix);
  if (ncomp == 1) k_block_apply<1><<<g, 256, 0, s>>>(blk, x, y, npix, w, partial, done);
  else k_block_apply<3><<<g, 256, 0, s>>>(blk, x, y, npix, w, partial, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_block_apply(int ncomp, int64_t npix, const double* blk, const double* x, double* y,
                       const int* done, cudaStream_t s) {
  return launch_block_apply_dot(ncomp, npix, blk, x, y, nullptr, nullptr, done, s);
}

int launch_dot_partial(const double* x, const double* y, int64_t n, double* partial, const int* done,
                       cudaStream_t s) {
  k_dot_partial<<<kRedBlocks, 256, 0, s>>>(x, y, n, partial, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_sub(double* r, const double* b, const double* q, int64_t n, cudaStream_t s) {
  k_sub<<<grid_for(n), 256, 0, s>>>(r, b, q, n);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_dot(const double* x, const double* y, int64_t n, double* partial, double* out, const int* done,
               cudaStream_t s) {
  CMM_TRY(launch_dot_partial(x, y, n, partial, done, s));
  k_sum_partials<<<1, 256, 0, s>>>(partial, kRedBlocks, out, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_copy_sub(double* dst, const double* a, const double* b, int64_t n, cudaStream_t s) {
  k_copy_sub<<<grid_for(n), 256, 0, s>>>(dst, a, b, n);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_solver_init(SolverDev* st, const double* prz, const double* prr, double* hist, cudaStream_t s) {
  k_solver_init<<<1, 256, 0, s>>>(st, prz, prr, hist);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_solver_alpha(SolverDev* st, const double* partial, double* anorm, cudaStream_t s) {
  k_solver_alpha<<<1, 256, 0, s>>>(st, partial, anorm);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_update_xr(double* x, double* r, double* r_old, const double* p, const double* q, int64_t n,
                     const SolverDev* st, double* partial, cudaStream_t s) {
  k_update_xr<<<kRedBlocks, 256, 0, s>>>(x, r, r_old, p, q, n, st, partial);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_dot_partial_cg(const double* x, const double* y, int64_t n, const SolverDev* st, double* partial,
                          cudaStream_t s) {
  k_dot_partial_cg<<<kRedBlocks, 256, 0, s>>>(x, y, n, st, partial);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_solver_z(double* z, const double* r, const double* r_old, int64_t n, const SolverDev* st,
                    double* p_rz, double* p_flex, cudaStream_t s) {
  k_solver_z<<<kRedBlocks, 256, 0, s>>>(z, r, r_old, n, st, p_rz, p_flex);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_residual(double* r, const double* b, const double* q, int64_t n, const SolverDev* st, double* partial,
                    cudaStream_t s) {
  k_residual<<<kRedBlocks, 256, 0, s>>>(r, b, q, n, st, partial);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_snapshot(const double* x, const double* r, int64_t n, const SolverDev* st, int every, int max,
                    double* snaps, cudaStream_t s) {
  k_snapshot<<<grid_for(n), 256, 0, s>>>(x, r, n, st, every, max, snaps);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_solver_rho(SolverDev* st, const double* p_rz, cudaStream_t s) {
  k_solver_rho<<<1, 256, 0, s>>>(st, p_rz);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_solver_check(SolverDev* st, const double* partial, double* hist, cudaStream_t s) {
  k_solver_check<<<1, 256, 0, s>>>(st, partial, hist);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_solver_beta(SolverDev* st, const double* p_rz, const double* p_flex, cudaStream_t s) {
  k_solver_beta<<<1, 256, 0, s>>>(st, p_rz, p_flex);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_update_p(double* p, const double* z, int64_t n, const SolverDev* st, cudaStream_t s) {
  k_update_p<<<grid_for(n), 256, 0, s>>>(p, z, n, st);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_update_xr_ring(double* x, double* r, const double* p, const double* q, int64_t n, const SolverDev* st,
                          double* P, double* Q, double* partial, cudaStream_t s) {
  k_update_xr_ring<<<kRedBlocks, 256, 0, s>>>(x, r, p, q, n, st, P, Q, partial);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_window_dots(const double* z, const double* Q, int64_t n, const SolverDev* st, double* wpart,
                       cudaStream_t s) {
  k_window_dots<<<kRedBlocks, 256, 0, s>>>(z, Q, n, st, wpart);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_window_beta(SolverDev* st, const double* wpart, cudaStream_t s) {
  k_window_beta<<<1, 256, 0, s>>>(st, wpart);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_update_p_window(double* p, const double* z, const double* P, const double* r, int64_t n,
                           const SolverDev* st, double* partial, cudaStream_t s) {
  k_update_p_window<<<kRedBlocks, 256, 0, s>>>(p, z, P, r, n, st, partial);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_solver_rho_pr(SolverDev* st, const double* partial, cudaStream_t s) {
  k_solver_rho_pr<<<1, 256, 0, s>>>(st, partial);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

// ---- 2-D FFT plans
static bool factor_smooth(int L, MixedPlan& plan) {
  plan.L = L;
  plan.nrad = 0;
  int n = L;
  while (n % 4 == 0 && plan.nrad < kMaxFactors) { plan.rad[plan.nrad++] = 4; n /= 4; }
  while (n % 2 == 0 && plan.nrad < kMaxFactors) { plan.rad[plan.nrad++] = 2; n /= 2; }
  while (n % 3 == 0 && plan.nrad < kMaxFactors) { plan.rad[plan.nrad++] = 3; n /= 3; }
  while (n % 5 == 0 && plan.nrad < kMaxFactors) { plan.rad[plan.nrad++] = 5; n /= 5; }
  int p = 1;
  for (int st = 0; st < plan.nrad; ++st) {
    plan.mnbf[st] = fast_div_magic((unsigned)(L / plan.rad[st]));
    plan.mp[st] = fast_div_magic((unsigned)p);
    p *= plan.rad[st];
  }
  return n == 1;
}

template <typename T>
int fft2_plan_init(Fft2Plan& p, int ny, int nx) {
  p.ny = ny;
  p.nx = nx;
  p.f64 = sizeof(T) == 8;
  if (!factor_smooth(ny, p.py) || !factor_smooth(nx, p.px))
    return fail(CMM_ERR_UNSUPPORTED, "map dimensions must factor into 2, 3 and 5");
  if (ny >= 65536 || nx >= 65536)   // the index divisions of the line FFTs (fast_div)
    return fail(CMM_ERR_UNSUPPORTED, "map sides must be below 65536 pixels");
  std::vector<V2<T>> h(ny + nx);
  for (int e = 0; e < nx; ++e) {
    const double a = -2.0 * M_PI * e / nx;
    h[e] = V2<T>{(T)std::cos(a), (T)std::sin(a)};
  }
  for (int e = 0; e < ny; ++e) {
    const double a = -2.0 * M_PI * e / ny;
    h[nx + e] = V2<T>{(T)std::cos(a), (T)std::sin(a)};
  }
  CMM_CUDA(cudaFuncSetAttribute(k_fft_lines<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  CMM_CUDA(cudaMalloc(&p.tw, sizeof(V2<T>) * (ny + nx)));
  CMM_CUDA(cudaMemcpy(p.tw, h.data(), sizeof(V2<T>) * (ny + nx), cudaMemcpyHostToDevice));
  return CMM_OK;
}
template int fft2_plan_init<float>(Fft2Plan&, int, int);
template int fft2_plan_init<double>(Fft2Plan&, int, int);

#ifndef CMM_FFT_ROW_KB
#define CMM_FFT_ROW_KB 96
#endif
#ifndef CMM_FFT_COL_KB
#define CMM_FFT_COL_KB 64
#endif

template <typename T>
static int lines_launch(const Fft2Plan& p, V2<T>* data, int nplanes, bool rows, int sign, const int* done,
                        cudaStream_t s) {
  const int L = rows ? p.nx : p.ny;
  const int nlines = rows ? p.ny : p.nx;
  const long long line_stride = rows ? p.nx : 1;
  const long long elem_stride = rows ? 1 : p.nx;
  const long long plane_stride = (long long)p.ny * p.nx;
  const int budget = (rows ? CMM_FFT_ROW_KB : CMM_FFT_COL_KB) * 1024;   // shared memory per CTA
  int lpc = std::max(1, std::min(rows ? 4 : 16, budget / (int)(2 * sizeof(V2<T>) * L)));
  const size_t smem = 2 * sizeof(V2<T>) * (size_t)lpc * L;
  const V2<T>* tw = reinterpret_cast<const V2<T>*>(p.tw) + (rows ? 0 : p.nx);
  dim3 g((nlines + lpc - 1) / lpc, nplanes);
  k_fft_lines<T><<<g, 256, smem, s>>>(data, rows ? p.px : p.py, nlines, line_stride, elem_stride,
                                      plane_stride, lpc, tw, sign, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

template <typename T>
int fft2(const Fft2Plan& p, V2<T>* data, int nplanes, int sign, const int* done, cudaStream_t s) {
  CMM_TRY(lines_launch<T>(p, data, nplanes, true, sign, done, s));
  CMM_TRY(lines_launch<T>(p, data, nplanes, false, sign, done, s));
  return CMM_OK;
}
template int fft2<float>(const Fft2Plan&, float2*, int, int, const int*, cudaStream_t);
template int fft2<double>(const Fft2Plan&, double2*, int, int, const int*, cudaStream_t);

template <typename T>
int launch_circ_q(int ncomp, const double* rows, const double* sig_inv, int ref, int ny, int nx,
                  double taper_sigma, V2<T>* planes, cudaStream_t s) {
  const double inv2s2 = (taper_sigma > 0 && std::isfinite(taper_sigma)) ? 1.0 / (2.0 * taper_sigma * taper_sigma) : 0.0;
  const long long npix = (long long)ny * nx;
  if (ncomp == 1) k_circ_q<T, 1><<<grid_for(npix), 256, 0, s>>>(rows, sig_inv, ref, ny, nx, inv2s2, planes);
  else k_circ_q<T, 3><<<grid_for(npix), 256, 0, s>>>(rows, sig_inv, ref, ny, nx, inv2s2, planes);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_circ_q<float>(int, const double*, const double*, int, int, int, double, float2*, cudaStream_t);
template int launch_circ_q<double>(int, const double*, const double*, int, int, int, double, double2*, cudaStream_t);

template <typename T>
int launch_mode_inverse(int ncomp, const V2<T>* planes, long long npix, double eps, double* hinv,
                        unsigned long long* scratch2, cudaStream_t s) {
  CMM_CUDA(cudaMemsetAsync(scratch2, 0, 2 * sizeof(unsigned long long), s));
  if (ncomp == 1) {
    k_mode_maxeig<T, 1><<<grid_for(npix), 256, 0, s>>>(planes, npix, scratch2);
    k_mode_inverse<T, 1><<<grid_for(npix), 256, 0, s>>>(planes, npix, scratch2, eps, hinv, scratch2 + 1);
  } else {
    k_mode_maxeig<T, 3><<<grid_for(npix), 128, 0, s>>>(planes, npix, scratch2);
    k_mode_inverse<T, 3><<<grid_for(npix), 128, 0, s>>>(planes, npix, scratch2, eps, hinv, scratch2 + 1);
  }
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_mode_inverse<float>(int, const float2*, long long, double, double*, unsigned long long*, cudaStream_t);
template int launch_mode_inverse<double>(int, const double2*, long long, double, double*, unsigned long long*, cudaStream_t);

template <typename T>
int launch_real_to_planes(const double* x, V2<T>* planes, long long n, const int* done, cudaStream_t s) {
  k_real_to_planes<T><<<grid_for(n), 256, 0, s>>>(x, planes, n, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_real_to_planes<float>(const double*, float2*, long long, const int*, cudaStream_t);
template int launch_real_to_planes<double>(const double*, double2*, long long, const int*, cudaStream_t);

template <typename T>
int launch_planes_to_real(const V2<T>* planes, double* x, long long n, double scale, const int* done,
                          cudaStream_t s) {
  k_planes_to_real<T><<<grid_for(n), 256, 0, s>>>(planes, x, n, scale, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_planes_to_real<float>(const float2*, double*, long long, double, const int*, cudaStream_t);
template int launch_planes_to_real<double>(const double2*, double*, long long, double, const int*, cudaStream_t);

template <typename T>
int launch_block_to_planes(int ncomp, int64_t npix, const double* blk, const double* x, V2<T>* planes,
                           const int* done, cudaStream_t s) {
  if (ncomp == 1) k_block_to_planes<T, 1><<<grid_for(npix), 256, 0, s>>>(blk, x, planes, npix, done);
  else k_block_to_planes<T, 3><<<grid_for(npix), 256, 0, s>>>(blk, x, planes, npix, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_block_to_planes<float>(int, int64_t, const double*, const double*, float2*, const int*,
                                           cudaStream_t);
template int launch_block_to_planes<double>(int, int64_t, const double*, const double*, double2*, const int*,
                                            cudaStream_t);

template <typename T>
int launch_planes_block_dot(int ncomp, int64_t npix, const V2<T>* planes, double scale, const double* blk, double* y,
                            const double* w, double* partial, const int* done, cudaStream_t s) {
  const int g = partial ? kRedBlocks : grid_for(npix);
  if (ncomp == 1) k_planes_block_dot<T, 1><<<g, 256, 0, s>>>(planes, scale, blk, y, npix, w, partial, done);
  else k_planes_block_dot<T, 3><<<g, 256, 0, s>>>(planes, scale, blk, y, npix, w, partial, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_planes_block_dot<float>(int, int64_t, const float2*, double, const double*, double*,
                                            const double*, double*, const int*, cudaStream_t);
template int launch_planes_block_dot<double>(int, int64_t, const double2*, double, const double*, double*,
                                             const double*, double*, const int*, cudaStream_t);

template <typename T, typename B>
int launch_block_to_planes_packed(int64_t npix, const B* blk, const double* x, V2<T>* planes, const int* done,
                                  cudaStream_t s) {
  k_block_to_planes_packed<T, B><<<grid_for(npix), 256, 0, s>>>(blk, x, planes, npix, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_block_to_planes_packed<float, float>(int64_t, const float*, const double*, float2*, const int*,
                                                         cudaStream_t);
template int launch_block_to_planes_packed<float, double>(int64_t, const double*, const double*, float2*,
                                                          const int*, cudaStream_t);
template int launch_block_to_planes_packed<double, double>(int64_t, const double*, const double*, double2*,
                                                           const int*, cudaStream_t);

template <typename T, typename B>
int launch_planes_block_dot_packed(int64_t npix, const V2<T>* planes, double scale, const B* blk, double* y,
                                   const double* w, double* partial, const int* done, cudaStream_t s) {
  const int g = partial ? kRedBlocks : grid_for(npix);
  k_planes_block_dot_packed<T, B><<<g, 256, 0, s>>>(planes, scale, blk, y, npix, w, partial, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_planes_block_dot_packed<float, float>(int64_t, const float2*, double, const float*, double*,
                                                          const double*, double*, const int*, cudaStream_t);
template int launch_planes_block_dot_packed<float, double>(int64_t, const float2*, double, const double*, double*,
                                                           const double*, double*, const int*, cudaStream_t);
template int launch_planes_block_dot_packed<double, double>(int64_t, const double2*, double, const double*,
                                                            double*, const double*, double*, const int*,
                                                            cudaStream_t);

template <typename T, typename H>
int launch_mode_apply_packed(V2<T>* planes, const H* hinv, int ny, int nx, const int* done, cudaStream_t s) {
  k_mode_apply_packed<T, H><<<grid_for((long long)ny * nx), 256, 0, s>>>(planes, hinv, ny, nx, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_mode_apply_packed<float, float>(float2*, const float*, int, int, const int*, cudaStream_t);
template int launch_mode_apply_packed<float, double>(float2*, const double*, int, int, const int*, cudaStream_t);
template int launch_mode_apply_packed<double, double>(double2*, const double*, int, int, const int*, cudaStream_t);

template <typename T, typename H>
int launch_mode_apply(int ncomp, V2<T>* planes, const H* hinv, long long npix, const int* done,
                      cudaStream_t s) {
  if (ncomp == 1) k_mode_apply<T, 1, H><<<grid_for(npix), 256, 0, s>>>(planes, hinv, npix, done);
  else k_mode_apply<T, 3, H><<<grid_for(npix), 256, 0, s>>>(planes, hinv, npix, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}
template int launch_mode_apply<float, double>(int, float2*, const double*, long long, const int*, cudaStream_t);
template int launch_mode_apply<float, float>(int, float2*, const float*, long long, const int*, cudaStream_t);
template int launch_mode_apply<double, double>(int, double2*, const double*, long long, const int*, cudaStream_t);

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

int launch_to_f32(const double* x, float* y, long long n, cudaStream_t s) {
  k_to_f32<<<grid_for(n), 256, 0, s>>>(x, y, n);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

__global__ void k_window(const double* __restrict__ d, const double* __restrict__ x, double* __restrict__ y,
                         long long npix, int ncomp, int mode, const int* done) {
  if (done && *done) return;
  const long long n = npix * ncomp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = d[i % npix] * x[i];
    y[i] = mode == 2 ? y[i] + v : v;   // 0: y = d x, 1: first accumulation, 2: y += d x
  }
}

int launch_window_mul(const double* d, const double* x, double* y, int64_t npix, int ncomp, const int* done,
                      cudaStream_t s) {
  k_window<<<grid_for(npix * ncomp), 256, 0, s>>>(d, x, y, npix, ncomp, 0, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

int launch_window_acc(const double* d, const double* x, double* z, int64_t npix, int ncomp, bool first,
                      const int* done, cudaStream_t s) {
  k_window<<<grid_for(npix * ncomp), 256, 0, s>>>(d, x, z, npix, ncomp, first ? 1 : 2, done);
  CMM_LAUNCH_CHECK();
  return CMM_OK;
}

}  // namespace cmm
