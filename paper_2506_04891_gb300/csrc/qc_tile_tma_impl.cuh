// Host side of the TMA-staged tile pass: tensor maps of a pass's tile
// geometry and the launch templates.  Included by qc_tile_tma_fwd.cu and
// qc_tile_tma_bwd.cu (one sweep each, compiled in parallel).
#pragma once
#include "qc_tile_tma.cuh"

namespace qc {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The tile of a pass (local bits [0, c) of the sample index, then [h0, h0+m),
// c + m = 12) as a 5-dimensional box of 8-byte elements: 16 amplitudes (bits
// 0..3), bits 4..c-1, the gap [c, h0) (one element), bits [h0, h0+m), and the
// bits above merged with the batch.  The kernel's coordinates of tile f of
// sample b: (0, 0, f mod 2^(h0-c), 0, b 2^(n-h0-m) + f / 2^(h0-c)).
static cudaError_t make_tile_map(CUtensorMap* tm, const void* base, const TilePass& P, int batch) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return cudaErrorNotSupported;
  const int n = P.n, c = P.c, h0 = P.h0, m = kTmaT - c, gap = h0 - c;
  if (c < 4 || m < 0 || m > 8 || gap < 0 || h0 + m > n || ((uintptr_t)base & 15)) return cudaErrorInvalidValue;
  const cuuint64_t dims[5] = {16, 1ull << (c - 4), 1ull << gap, 1ull << m, (cuuint64_t)batch << (n - h0 - m)};
  const cuuint64_t strides[4] = {128, 8ull << c, 8ull << h0, 8ull << (h0 + m)};
  const cuuint32_t box[5] = {16, 1u << (c - 4), 1, 1u << m, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_INT64, 5, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int NS, int RB, int KIND, int PRE, bool XL = false>
static cudaError_t launch_tma_k(const TilePass& P, int batch, int cps, const void* coef, const void* s0,
                                void* d0, const void* s1, void* d1, double* part, cudaStream_t st) {
  // companion gradients only occur in backward single-qubit passes
  constexpr bool kMayComp = NS == 2 && KIND != 2 && KIND != 3;
  const bool comp = kMayComp && P.ncomp > 0;
  CUtensorMap tm0, tm1;
  cudaError_t e = make_tile_map(&tm0, s0, P, batch);
  if (e != cudaSuccess) return e;
  if (NS == 2) {
    e = make_tile_map(&tm1, s1, P, batch);
    if (e != cudaSuccess) return e;
  } else {
    tm1 = tm0;
  }
  const size_t smem = tma_smem_bytes(P, NS);
  auto kern = comp ? k_tile_tma<NS, RB, KIND, PRE, kMayComp, XL> : k_tile_tma<NS, RB, KIND, PRE, false, XL>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = (long long)batch * cps;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(P, tm0, tm1, (const float*)coef, (float2*)d0, (float2*)d1, part, cps);
  return cudaGetLastError();
}

// Kinds and register bits the TMA pass is built for: single-qubit layers
// (complex, real, constant SX) at 3 or 4 register bits, brick layers at
// 2 .. 4; the fused diagonal variants at 4.
template <int NS>
static cudaError_t launch_tma_ns(const TilePass& P, int rb, int batch, int cps, const void* coef, const void* s0,
                                 void* d0, const void* s1, void* d1, double* part, cudaStream_t st) {
#define QC_TMA_L(RB_, K_, PRE_) launch_tma_k<NS, RB_, K_, PRE_>(P, batch, cps, coef, s0, d0, s1, d1, part, st)
#define QC_TMA_X(RB_, K_, PRE_) launch_tma_k<NS, RB_, K_, PRE_, true>(P, batch, cps, coef, s0, d0, s1, d1, part, st)
  if (P.xload) {
    // a fused X layer (complemented loads): built for the forward brick pass
    // and the backward SX pass with its diagonal undone in round 0
    if constexpr (NS == 1) {
      if (P.kind == 2 && !P.pre && !P.post) {
        if (rb == 3) return QC_TMA_X(3, 2, 0);
        if (rb == 4) return QC_TMA_X(4, 2, 0);
      }
    } else {
      if (P.kind == 0 && P.sx && P.pre && rb == 4)
        return P.pre_zmode == Z_RINGXOR ? QC_TMA_X(4, 3, 2) : QC_TMA_X(4, 3, 1);
    }
    return cudaErrorInvalidValue;
  }
  if (P.kind == 2) {
    if (P.pre || P.post) return cudaErrorInvalidValue;
    switch (rb) {
      case 2: return QC_TMA_L(2, 2, 0);
      case 3: return QC_TMA_L(3, 2, 0);
      case 4: return QC_TMA_L(4, 2, 0);
    }
    return cudaErrorInvalidValue;
  }
  const bool diag = NS == 2 ? P.pre != 0 : P.post != 0;
  // constant SX passes run the additions-only variant (kind 3)
  const bool sx = P.kind == 0 && P.sx;
  if (diag) {
    if (rb != 4) return cudaErrorInvalidValue;
    const bool ring = (NS == 2 ? P.pre_zmode : P.post_zmode) == Z_RINGXOR;
    // backward 1 / 2 identity / ring; forward 3 / 2 identity / ring
    if constexpr (NS == 2) {
      if (P.kind == 1) return ring ? QC_TMA_L(4, 1, 2) : QC_TMA_L(4, 1, 1);
      if (sx) return ring ? QC_TMA_L(4, 3, 2) : QC_TMA_L(4, 3, 1);
      return ring ? QC_TMA_L(4, 0, 2) : QC_TMA_L(4, 0, 1);
    } else {
      if (P.kind == 1) return ring ? QC_TMA_L(4, 1, 2) : QC_TMA_L(4, 1, 3);
      if (sx) return ring ? QC_TMA_L(4, 3, 2) : QC_TMA_L(4, 3, 3);
      return ring ? QC_TMA_L(4, 0, 2) : QC_TMA_L(4, 0, 3);
    }
  }
  if (rb == 3) return P.kind == 1 ? QC_TMA_L(3, 1, 0) : sx ? QC_TMA_L(3, 3, 0) : QC_TMA_L(3, 0, 0);
  if (rb == 4) return P.kind == 1 ? QC_TMA_L(4, 1, 0) : sx ? QC_TMA_L(4, 3, 0) : QC_TMA_L(4, 0, 0);
#undef QC_TMA_L
#undef QC_TMA_X
  return cudaErrorInvalidValue;
}

}  // namespace qc
