// Tensor-core dense block (experiment): a forward real single-qubit layer
// (RY) on the 7 high bits of a strided tile pass as one 128 x 128 real
// matrix product on the 5th-generation tensor cores (tcgen05.mma kind::tf32),
// with the split-precision 3xTF32 scheme so that the result keeps FP32
// accuracy.  This is the paper's Unitary Operation technique (Sec. 2.2.1:
// apply the layer's matrix, here the Kronecker product of the 7 gates it
// holds on those bits) on a sub-block of the tile instead of the whole state.
//
// Tile (2^12 amplitudes, contiguous bits 0..4 and gate bits h0..h0+6): the
// TMA box is ordered [bit 4][gate row g][bits 0..3], so shared memory holds X
// as two 16 KB blocks of 128 rows of 128 bytes (16 complex amplitudes, 32
// floats), 128-byte swizzled.  The threads transpose it into the K-major
// B operand of D = K X (N = 64 floats: 32 amplitudes x (re, im); K = 128 gate
// rows; a probe showed the MN-major form of this operand multiplying to
// zero), which frees the landing buffer for the next tile's copy before the
// MMAs run.  K (M = 128 output rows) is built per CTA from the staged gate
// records in K-major layout.  3xTF32: X = Xh + Xl with Xh the TF32 truncation the tensor core
// applies and Xl = X - Xh (exact), the same for K; D = Kh Xh + Kh Xl + Kl Xh
// accumulates in tensor memory (128 lanes x 64 FP32 columns), is read back by
// tcgen05.ld and stored to global memory.
//
// One CTA of 256 threads per SM (224 KB of operands); one thread issues the
// TMA copies and the 48 MMAs of a tile and commits them to an mbarrier; every
// wait is bounded in time (a CTA that gives up counts it in a timeout counter
// that qc_kernel_timeouts reads, waits again with a bound for what it has in
// flight, frees its tensor memory and leaves).
#include "qc_tile_tma_impl.cuh"

namespace qc {

namespace {

constexpr int kTcThreads = 256;
constexpr unsigned kTcCols = 64;                       // tensor-memory columns of D
constexpr size_t kTcA = 4 * 128 * 128;                 // bytes of one A (K-matrix) copy: 4 K-atoms x 16 KB
constexpr size_t kTcB = 2 * 128 * 128;                 // bytes of one tile: 4096 complex64
constexpr size_t kTcSmem = 2 * kTcA + 3 * kTcB + 1024;  // Ah, Al, landing tile, Bh, Bl + alignment slack
static __device__ unsigned long long g_tc_timeouts;

__device__ __forceinline__ uint64_t umma_sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}
// D f32, A and B tf32, both K-major, N = 64, M = 128
constexpr unsigned kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_tf32(unsigned dt, uint64_t da, uint64_t db, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ float tf32_lo(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}
// byte offset of element (row, k) in a K-major 128-byte swizzled block of rows of 32 floats
__device__ __forceinline__ unsigned sw128(unsigned row, unsigned k) {
  return row * 128u + ((((k >> 2) ^ (row & 7u))) << 4) + (k & 3u) * 4u;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tile_tc(const __grid_constant__ TilePass P, const __grid_constant__ CUtensorMap tm, const float* __restrict__ coef,
              float2* dst, int cps) {
  extern __shared__ unsigned char smraw_tc[];
  const unsigned raw_sa = smem_u32(smraw_tc);
  unsigned char* sm = smraw_tc + (((raw_sa + 1023u) & ~1023u) - raw_sa);
  unsigned char* sAh = sm;
  unsigned char* sAl = sm + kTcA;
  unsigned char* sX = sm + 2 * kTcA;  // TMA landing buffer: [bit 4][gate row g][16 amplitudes], swizzled
  unsigned char* sBh = sX + kTcB;      // B = X in K-major layout: 4 K-atoms (32 g each) x 64 n-rows x 128 B
  unsigned char* sBl = sBh + kTcB;
  __shared__ unsigned long long bar_tma, bar_mma;
  __shared__ unsigned taddr_s;
  __shared__ float rec[7][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = P.n, h0 = P.h0;
  const long long tps = 1LL << (n - kTmaT);
  const int b = blockIdx.x / cps, r0 = blockIdx.x % cps;
  const int gap = h0 - P.c;  // P.c = 5, m = 7
  float2* db = dst + ((long long)b << n);

  // the 7 gate records (ops sorted by bit: op k acts on bit k of the row index)
  if (tid < 28) {
    const TileOp& o = P.ops[tid >> 2];
    rec[tid >> 2][tid & 3] = coef[o.coef + (long long)b * o.bstride + (tid & 3)];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar_tma)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar_mma)) : "memory");
    mbar_init_fence();
  }
  __syncthreads();
  // K[g'][g] = prod_q M_q[g'_q][g_q] with M_q = (m00, m01; m10, m11); split into TF32 hi / lo
  for (int e = tid; e < 128 * 128; e += kTcThreads) {
    const int gr = e >> 7, gc = e & 127;
    float v = 1.f;
#pragma unroll
    for (int q = 0; q < 7; ++q) v *= rec[q][(((gr >> q) & 1) << 1) | ((gc >> q) & 1)];
    const unsigned off = (unsigned)(gc >> 5) * (128u * 128u) + sw128((unsigned)gr, (unsigned)(gc & 31));
    *reinterpret_cast<float*>(sAh + off) = v;
    *reinterpret_cast<float*>(sAl + off) = tf32_lo(v);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&taddr_s)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned taddr = taddr_s;

  auto issue = [&](long long f) {  // thread 0
    const int c3 = (int)(f & ((1LL << gap) - 1));
    const int c4 = (int)(((long long)b << (n - h0 - 7)) | (f >> gap));
    const unsigned bar = smem_u32(&bar_tma);
    mbar_expect_tx(bar, (unsigned)kTcB);
    tma_load_5d(smem_u32(sX), &tm, 0, 0, 0, c3, c4, bar);
  };
  unsigned ph_tma = 0, ph_mma = 0;
  long long f = r0;
  if (tid == 0 && f < tps) issue(f);
  bool bad = false;
  for (; f < tps && !bad; f += cps) {
    if (!mbar_wait_bounded(smem_u32(&bar_tma), ph_tma, kTmaWaitNs)) bad = true;
    ph_tma ^= 1u;
    if (__syncthreads_or(bad)) { bad = true; break; }
    // B = X transposed into the K-major layout (the MN-major form of this
    // operand did not multiply correctly), split into TF32 hi and lo: each
    // thread reads one 16-byte chunk (4 floats n = 4c .. 4c+3 of row g) and
    // writes 4 elements (n, g); a warp covers 32 consecutive rows of one
    // chunk column, so reads hit 8 distinct chunks per quarter warp and the
    // writes of each n fill one 128-byte row
    for (int q = tid; q < (int)(kTcB / 16); q += kTcThreads) {
      const int jh = q >> 10, cc = (q >> 7) & 7, g = q & 127;
      const float4 x = *reinterpret_cast<const float4*>(sX + jh * 16384 + g * 128 + ((cc ^ (g & 7)) << 4));
      const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const unsigned nn = (unsigned)(32 * jh + 4 * cc + e);
        const unsigned off = (unsigned)(g >> 5) * 8192u + nn * 128u + (((((unsigned)g & 31u) >> 2) ^ (nn & 7u)) << 4) +
                             ((unsigned)g & 3u) * 4u;
        *reinterpret_cast<float*>(sBh + off) = xv[e];
        *reinterpret_cast<float*>(sBl + off) = tf32_lo(xv[e]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // the landing buffer is free: the next tile's copy overlaps the MMAs
      if (f + cps < tps) issue(f + cps);
      const unsigned ah = smem_u32(sAh), al = smem_u32(sAl), xh = smem_u32(sBh), xl = smem_u32(sBl);
      // k-step s: A and B atom s / 4, at +32 bytes per step inside it
      for (int pass = 0; pass < 3; ++pass) {
        const unsigned a0 = pass == 2 ? al : ah, b0 = pass == 1 ? xl : xh;
        for (int s = 0; s < 16; ++s) {
          const uint64_t da = umma_sdesc(a0 + (unsigned)(s >> 2) * (128u * 128u) + (unsigned)(s & 3) * 32u, 16, 1024);
          const uint64_t dB = umma_sdesc(b0 + (unsigned)(s >> 2) * 8192u + (unsigned)(s & 3) * 32u, 16, 1024);
          umma_tf32(taddr, da, dB, (pass | s) != 0);
        }
      }
      umma_commit(smem_u32(&bar_mma));
    }
    if (!mbar_wait_bounded(smem_u32(&bar_mma), ph_mma, kTmaWaitNs)) bad = true;
    ph_mma ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (__syncthreads_or(bad)) { bad = true; break; }
    // warp w reads lanes (rows g') 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31
    // = amplitudes j = 16 (w / 4) .. + 15 of row g'
    {
      unsigned r[32];
      const unsigned ta = taddr + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(32 * (warp >> 2));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          // the load is asynchronous: wait in the same statement, so that no
          // copy of a destination register can be placed before the data lands
          "tcgen05.wait::ld.sync.aligned;\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(ta)
          : "memory");
      const int gr = 32 * (warp & 3) + lane, j0 = 16 * (warp >> 2);
      const int kb = (int)(((f & ((1LL << gap) - 1)) << 5) | ((f >> gap) << (h0 + 7)));
      float4* o = reinterpret_cast<float4*>(db + (kb | j0 | (gr << h0)));
#pragma unroll
      for (int q = 0; q < 8; ++q)
        o[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                           __uint_as_float(r[4 * q + 3]));
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // tensor memory and the operand buffers are free for the next tile
  }
  if (bad && tid == 0) {
    atomicAdd(&g_tc_timeouts, 1ull);
    // bounded waits for whatever this CTA still has in flight
    mbar_wait_bounded(smem_u32(&bar_tma), ph_tma, kTmaWaitNs);
    mbar_wait_bounded(smem_u32(&bar_mma), ph_mma, kTmaWaitNs);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(kTcCols) : "memory");
}

// The tile as the B operand: dims [bits 0..3][gate bits h0..h0+6][bit 4][gap][above, with the batch]
cudaError_t make_tc_map(CUtensorMap* tmap, const void* base, const TilePass& P, int batch) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return cudaErrorNotSupported;
  const int n = P.n, c = P.c, h0 = P.h0, gap = h0 - c;
  if (c != 5 || P.t != 12 || h0 + 7 > n || ((uintptr_t)base & 15)) return cudaErrorInvalidValue;
  const cuuint64_t dims[5] = {16, 128, 2, 1ull << gap, (cuuint64_t)batch << (n - h0 - 7)};
  const cuuint64_t strides[4] = {8ull << h0, 128, 8ull << c, 8ull << (h0 + 7)};
  const cuuint32_t box[5] = {16, 128, 2, 1, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(tmap, CU_TENSOR_MAP_DATA_TYPE_INT64, 5, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// Whether the tensor-core block can run a forward pass: a real single-qubit
// layer with one gate on each of the 7 high bits of a 2^12 tile whose
// contiguous part is 32 amplitudes, nothing fused.
bool tile_tc_ok(const TilePass& P, int ns) {
  if (ns != 1 || P.kind != 1 || P.t != 12 || P.c != 5 || P.gather || P.pre || P.post || P.scatter) return false;
  if (P.nops != 7) return false;
  for (int k = 0; k < 7; ++k)
    if (P.ops[k].l != 5 + k || P.ops[k].nco != 4) return false;
  return true;
}

cudaError_t launch_tile_tc(const TilePass& P, int batch, int cps, const void* coef, const void* s0, void* d0,
                           cudaStream_t st) {
  CUtensorMap tmap;
  cudaError_t e = make_tc_map(&tmap, s0, P, batch);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tile_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  k_tile_tc<<<(unsigned)((long long)batch * cps), kTcThreads, kTcSmem, st>>>(P, tmap, (const float*)coef,
                                                                              (float2*)d0, cps);
  return cudaGetLastError();
}

unsigned long long tc_take_timeouts() {
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof(v)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_tc_timeouts, &z, sizeof(z)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}

}  // namespace qc
