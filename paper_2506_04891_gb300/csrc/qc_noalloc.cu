// <Z> without any device allocation.
//
// qc_expect_z keeps its per-CTA partial sums in device memory that the
// circuit handle allocates when it is created.  Some callers cannot let the
// library own device memory, or cannot allocate at the point where they
// measure: their device memory is entirely held by another allocator (a
// framework's caching pool, a fixed budget reserved at start-up), or a
// cudaMalloc / cudaFree, which may synchronise the whole device, is not
// acceptable inside their loop.  qc_expect_z_noalloc runs the same kernels
// with the partial sums in a fixed array that is part of this library's
// device image, so it allocates nothing.
//
// Each .cu file of the library is its own device module, and with lazy module
// loading a module (code and static arrays) is loaded, which allocates device
// memory, when it is first used.  noalloc_prepare(), which qc_create calls on
// the current device, makes that first use happen at set-up: it resolves the
// array's address (loading this module and committing the array) and loads
// the <Z> kernels.  A call made on a device where set-up has not run does it
// itself, so such a first call should stay outside stream capture.
#include <cuda_runtime.h>

#include <string>

#include "../../include/qlayer.h"
#include "qc_internal.h"
#include "qc_kernels.h"

namespace {

// Partial sums of one call: batch * 2^(n - min(n, 14)) CTAs x (n + 1) values.
constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 20;  // 8 MiB on every device
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of the scratch array in the current context.  The host-side
// name g_noalloc_scratch is only a stand-in for the device symbol, so kernels
// get this address.  It is looked up on every call (cheap once the module is
// loaded), so a context that was reset and reloaded never sees a stale one.
qc_status scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::string m = std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e);
    return qc::set_error(QC_ERR_CUDA, m.c_str());
  }
  *out = (double*)p;
  return QC_OK;
}

}  // namespace

namespace qc {
void noalloc_prepare(int n, int dtype) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;  // no usable device (e.g. host-only planning): the first call sets up
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) == cudaSuccess) {
    if (dtype == QC_C64) preload_expect<float>(n);
    else preload_expect<double>(n);
  }
  cudaGetLastError();
}
}  // namespace qc

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
