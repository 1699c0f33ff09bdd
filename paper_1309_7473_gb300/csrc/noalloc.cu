// cmm_apply_A_noalloc: A = P^T N^-1 P with every temporary in one fixed,
// statically allocated device array instead of the operator's own buffers.
//
// Who needs it: callers that cannot have device memory allocated or freed for
// them around an apply.  cudaMalloc and cudaFree can block on work queued on the
// device's other streams and can fail when memory is short, so a caller that
// keeps its device memory inside its own caching allocator, or one that runs
// close to the device's capacity, may forbid them.  This entry point makes no
// cudaMalloc, cudaFree or other allocating call.  Its temporaries (the spectrum
// of a chunk of detectors, the gather copy of the map and the FP64 and FP32
// accumulators) live in kNoAllocScratchBytes of static device memory, which every
// GPU that loads the library holds until the process exits.  All calls in the
// process share that array.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Address of the static array on `device` (current on the calling thread).  The
// first call on each device looks it up; later calls reuse the cached pointer.
int scratch_for_device(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cmm::fail(CMM_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cmm::cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_ptr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[device]);
  return CMM_OK;
}

size_t round_up(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

using namespace cmm;

extern "C" {

int cmm_apply_A_noalloc(cmm_op* op, const double* m_in, double* m_out) {
  if (!op || !m_in || !m_out) return fail(CMM_ERR_ARG, "null argument");
  if (m_in == m_out) return fail(CMM_ERR_ARG, "m_in and m_out must not alias");
  CMM_CUDA(cudaSetDevice(op->ctx->device));
  if (op->nz->corr_r > 0) return fail(CMM_ERR_UNSUPPORTED, "noise correlated between detectors is not supported here");
  const int64_t npix = op->pt->npix;
  const int nc = op->pt->ncomp;
  const size_t elt = op->prec == CMM_PREC_F64 ? 16 : (op->prec == CMM_PREC_BF16 ? 4 : 8);
  const size_t gel = op->prec == CMM_PREC_F64 ? 8 : 4;
  const size_t acc_bytes = round_up(sizeof(double) * op->acc_stride * (npix + 1));
  const size_t acc32_bytes = round_up(sizeof(float) * op->acc_stride * (npix + 1));
  const size_t gather_bytes = round_up(gel * (nc == 1 ? 1 : 4) * (npix + 1));
  const size_t per_det = elt * (size_t)op->N;
  const size_t fixed = acc_bytes + acc32_bytes + gather_bytes;
  if (fixed + per_det > kNoAllocScratchBytes)
    return fail(CMM_ERR_UNSUPPORTED,
                "operator too large for the 32 MiB static scratch (map buffers plus one detector's spectrum)");
  unsigned char* base = nullptr;
  CMM_TRY(scratch_for_device(op->ctx->device, &base));

  // A shallow copy of the operator whose scratch pointers point into the array.
  cmm_op v = *op;
  v.acc = reinterpret_cast<double*>(base);
  v.acc32 = reinterpret_cast<float*>(base + acc_bytes);
  v.acc32_maps = 1;
  v.gather = base + acc_bytes + acc32_bytes;
  v.spec = base + fixed;
  v.chunk = (int)std::min<size_t>((kNoAllocScratchBytes - fixed) / per_det, (size_t)op->pt->n_det);
  v.done = nullptr;
  // the two-detector path fills whole pairs of spectrum slots: an even chunk, or
  // the one-detector path when the array holds a single spectrum
  if (pair_path_ok(&v)) {
    if (v.chunk >= 2) v.chunk &= ~1;
    else v.pair = 0;
  }

  // The array keeps whatever the previous call left: the FP32 partial map must
  // start at zero (the FP64 accumulator is cleared by the gather kernel).
  CMM_CUDA(cudaMemsetAsync(v.acc32, 0, sizeof(float) * op->acc_stride * (npix + 1), op->ctx->stream));
  CMM_TRY(launch_map_to_gather(&v, m_in));
  for (int d0 = 0; d0 < op->pt->n_det; d0 += v.chunk) {
    const int nd = std::min(v.chunk, op->pt->n_det - d0);
    CMM_TRY(launch_apply_chunk(&v, d0, nd, nullptr, 0));
  }
  return launch_acc_to_map(&v, m_out);
}

}  // extern "C"
