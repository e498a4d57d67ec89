// TMA-staged tile passes of the backward sweep (complex64).
#include "qc_tile_tma_impl.cuh"

namespace qc {

cudaError_t launch_tile_tma_bwd(const TilePass& P, int rb, int batch, int cps, const void* coef, const void* s0,
                                void* d0, const void* s1, void* d1, double* part, cudaStream_t st) {
  return launch_tma_ns<2>(P, rb, batch, cps, coef, s0, d0, s1, d1, part, st);
}

unsigned long long tma_take_timeouts_bwd() {
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_tma_timeouts, sizeof(v)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_tma_timeouts, &z, sizeof(z)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}

}  // namespace qc
