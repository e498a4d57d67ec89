// <Z> without any device allocation.
//
// qc_expect_z keeps its per-CTA partial sums in device memory that the
// circuit handle allocates (and grows) on first use.  Some callers cannot
// allocate at that point: their device memory is entirely held by another
// allocator (a framework's caching pool, a fixed budget reserved at start-up),
// or a cudaMalloc, which may synchronise the whole device, is not acceptable
// inside their loop.  qc_expect_z_noalloc runs the same kernels with the
// partial sums in a fixed array that is part of this library's device image,
// so it allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/qlayer.h"
#include "qc_internal.h"
#include "qc_kernels.h"

namespace {

// Partial sums of one call: batch * 2^(n - min(n, 14)) CTAs x (n + 1) values.
constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 20;  // 8 MiB on every device
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once per
// device, with that device current).
qc_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return qc::set_error(QC_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return qc::set_error(QC_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      std::string m = std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e);
      return qc::set_error(QC_ERR_CUDA, m.c_str());
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return QC_OK;
}

}  // namespace

extern "C" QC_API qc_status qc_expect_z_noalloc(qc_circuit* c, int batch, const void* psi,
                                                double* ez, void* stream) {
  if (!c) return qc::set_error(QC_ERR_INVALID, "circuit handle is NULL");
  if (batch <= 0 || !psi || !ez) return qc::set_error(QC_ERR_INVALID, "bad batch, psi or ez");
  int n = 0, dtype = 0;
  qc::circuit_shape(c, &n, &dtype);
  const int cb = n < 14 ? n : 14;
  const size_t need = ((size_t)batch << (n - cb)) * (size_t)(n + 1);
  if (need > kNoAllocScratchDoubles) {
    std::string m = "qc_expect_z_noalloc: batch * 2^(n-min(n,14)) * (n+1) = " + std::to_string(need) +
                    " partial sums exceed the static scratch of " +
                    std::to_string(kNoAllocScratchDoubles) + "; use qc_expect_z";
    return qc::set_error(QC_ERR_INVALID, m.c_str());
  }
  double* scratch = nullptr;
  qc_status s = scratch_address(&scratch);
  if (s != QC_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = dtype == QC_C64 ? qc::launch_expect<float>(n, cb, batch, psi, scratch, ez, st)
                                  : qc::launch_expect<double>(n, cb, batch, psi, scratch, ez, st);
  if (e != cudaSuccess) return qc::set_error(QC_ERR_CUDA, cudaGetErrorString(e));
  return QC_OK;
}
