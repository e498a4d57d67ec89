// Host-side launch wrappers of the kernels in qc_kernels.cu.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "qc_internal.h"

namespace qc {

// Coefficient job: one layer's gate matrices / generators / phase tables.
struct CoefJob {
  int cls, kind, source, offset, parity;
  int ngates;
  int per_sample;
  int has_phase;
  int tb;
  int pstride;    // parameter j at offset + pstride * j
  int rot_phase;  // RZ part of a Rot (see LayerInfo)
  long long coef_off;
  long long bstride;
};

constexpr int kMaxLeading = 32;
struct ProdVecJob {
  int nl;
  int kind[kMaxLeading], source[kMaxLeading], offset[kMaxLeading];
  int pstride[kMaxLeading], rot_phase[kMaxLeading];
};

template <class R>
cudaError_t launch_coef(const CoefJob* jobs_dev, int njobs, int n, int batch, int n_in,
                        const double* x, const double* theta, void* coef, cudaStream_t st);
template <class R>
cudaError_t launch_prodvec(const ProdVecJob& P, int n, int batch, int n_in, const double* x,
                           const double* theta, void* pv, cudaStream_t st);
template <class R>
cudaError_t launch_prodinit(int n, int cb, int batch, const void* pv, void* psi,
                           const void* post_tabs, long long post_bstride, int post_tb,
                           int post_zmode, cudaStream_t st);
template <class R>
cudaError_t launch_tile(const TilePass& P, int rb, int ns, int batch, int cps, const void* coef,
                        const void* s0, void* d0, const void* s1, void* d1, double* part,
                        cudaStream_t st);
// the two sweeps' tile instantiations (qc_tile_fwd.cu, qc_tile_bwd.cu)
template <class R>
cudaError_t launch_tile_fwd(const TilePass& P, int rb, int batch, int cps, const void* coef,
                            const void* s0, void* d0, const void* s1, void* d1, double* part,
                            cudaStream_t st);
template <class R>
cudaError_t launch_tile_bwd(const TilePass& P, int rb, int batch, int cps, const void* coef,
                            const void* s0, void* d0, const void* s1, void* d1, double* part,
                            cudaStream_t st);
// TMA-staged complex64 tile passes (qc_tile_tma_fwd.cu / qc_tile_tma_bwd.cu)
cudaError_t launch_tile_tma_fwd(const TilePass& P, int rb, int batch, int cps, const void* coef, const void* s0,
                                void* d0, const void* s1, void* d1, double* part, cudaStream_t st);
cudaError_t launch_tile_tma_bwd(const TilePass& P, int rb, int batch, int cps, const void* coef, const void* s0,
                                void* d0, const void* s1, void* d1, double* part, cudaStream_t st);
size_t tile_tma_smem_bytes(const TilePass& P, int ns);
// tensor-core dense block of a forward real pass (qc_tile_tc.cu, experiment)
bool tile_tc_ok(const TilePass& P, int ns);
cudaError_t launch_tile_tc(const TilePass& P, int batch, int cps, const void* coef, const void* s0, void* d0,
                           cudaStream_t st);
unsigned long long tc_take_timeouts();
unsigned long long tma_take_timeouts_fwd();
unsigned long long tma_take_timeouts_bwd();
template <class R>
cudaError_t launch_diag(const DiagPass& P, int ns, int batch, const void* coef, const void* s0,
                        void* d0, const void* s1, void* d1, double* part, cudaStream_t st);
template <class R>
cudaError_t launch_ring(const RingPass& P, int ns, int batch, const void* s0, void* d0,
                        const void* s1, void* d1, const double* gez, const void* coef, double* part,
                        cudaStream_t st);
template <class R>
cudaError_t launch_expect(int n, int cb, int batch, const void* psi, double* part, double* ez,
                          cudaStream_t st);
template <class R>
cudaError_t launch_laminit(int n, int cb, int batch, const double* gez, const void* psi, void* lam,
                           cudaStream_t st);
template <class R>
cudaError_t launch_smem(const SmemLayer* prog_dev, int nl, int n, int batch, int bwd,
                        const void* coef, const void* psi_in, void* psi_out, double* ez,
                        const double* gez, double* part, int nslots, cudaStream_t st);
cudaError_t launch_reduce(const RedJob* jobs, const long long* row0, const int* out0, int njobs,
                          long long rowbase, long long nrows, int outbase, int nout,
                          const RedOut* outs, int batch, int n_in, const double* part, double* V,
                          double* d_theta, double* d_x, cudaStream_t st);

// copies `bytes` host bytes to device memory `dst` in stream order through
// kernel parameters (no allocation, no synchronisation)
cudaError_t launch_upload(const void* host, size_t bytes, void* dst, cudaStream_t st);
template <class R>
cudaError_t preload_expect(int n);

size_t tile_smem_bytes(const TilePass& P, int ns, int rsize);
size_t ring_smem_bytes(const RingPass& P, int rsize);
size_t smem_circuit_bytes(int n, int bwd, int rsize);
long long diag_grid(const DiagPass& P, int batch);

}  // namespace qc
