// Tile-pass instantiations for the backward (NS = 2) sweep, in a translation unit of
// their own so the build compiles them in parallel with the other kernels.
#include "qc_tile.cuh"

// QC_INST_R: 4 float, 8 double, 0 both (the build compiles one object per precision)
#ifndef QC_INST_R
#define QC_INST_R 0
#endif

namespace qc {

template <class R>
cudaError_t launch_tile_bwd(const TilePass& P, int rb, int batch, int cps, const void* coef,
                             const void* s0, void* d0, const void* s1, void* d1, double* part,
                             cudaStream_t st) {
  switch (rb) {
    case 1: return launch_tile_rb<R, 2, 1>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
    case 2: return launch_tile_rb<R, 2, 2>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
    case 3: return launch_tile_rb<R, 2, 3>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
    case 4: return launch_tile_rb<R, 2, 4>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
  }
  return cudaErrorInvalidValue;
}

#if QC_INST_R != 8
template cudaError_t launch_tile_bwd<float>(const TilePass&, int, int, int, const void*, const void*, void*,
                                             const void*, void*, double*, cudaStream_t);
#endif
#if QC_INST_R != 4
template cudaError_t launch_tile_bwd<double>(const TilePass&, int, int, int, const void*, const void*, void*,
                                              const void*, void*, double*, cudaStream_t);
#endif

}  // namespace qc
