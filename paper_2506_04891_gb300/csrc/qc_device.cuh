// Device helpers shared by the kernel translation units: complex
// arithmetic on interleaved float2 / double2, packed FP32x2 ops, warp sums,
// the CNOT-ring index maps and the diagonal-layer z map and phase tables.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "qc_internal.h"

// resident CTAs per SM the tile passes are compiled for: the complex64
// forward passes of real single-qubit gates (RY; also the variant that
// multiplies a following diagonal in its last round) fit three (80
// registers, no spills), the others two (a three-CTA backward spills and
// measured slower)
#ifndef QC_BWD_MINB
#define QC_BWD_MINB 2
#endif
#ifndef QC_FWD_MINB
#define QC_FWD_MINB 2
#endif
#ifndef QC_REAL_MINB
#define QC_REAL_MINB 3
#endif
#ifndef QC_PRE_MINB
#define QC_PRE_MINB 2
#endif

namespace qc {

template <class R> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };
template <class R> using cx = typename CT<R>::C;

template <class R> __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> r; r.x = a; r.y = b; return r; }
template <class R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <class R> __device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// m * v + acc
template <class R> __device__ __forceinline__ cx<R> cfma(cx<R> m, cx<R> v, cx<R> acc) {
  return mk<R>(fma(m.x, v.x, fma(-m.y, v.y, acc.x)), fma(m.x, v.y, fma(m.y, v.x, acc.y)));
}
// conj(m) * v + acc
template <class R> __device__ __forceinline__ cx<R> cfmac(cx<R> m, cx<R> v, cx<R> acc) {
  return mk<R>(fma(m.x, v.x, fma(m.y, v.y, acc.x)), fma(m.x, v.y, fma(-m.y, v.x, acc.y)));
}
template <class R> __device__ __forceinline__ R re_cdot(cx<R> l, cx<R> v) {  // Re(conj(l) v)
  return l.x * v.x + l.y * v.y;
}
template <class R> __device__ __forceinline__ R im_cdot(cx<R> l, cx<R> v) {  // Im(conj(l) v)
  return l.x * v.y - l.y * v.x;
}
template <class R> __device__ __forceinline__ cx<R> ldc(const R* p) { return mk<R>(p[0], p[1]); }
// Four consecutive R from a 16-byte aligned address (shared-memory staged
// coefficients): one 16-byte load for float, two for double.
template <class R>
__device__ __forceinline__ void ld4(const R* p, R& a, R& b, R& c, R& d) {
  if constexpr (std::is_same<R, float>::value) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
  } else {
    const double2 u = *reinterpret_cast<const double2*>(p), v = *reinterpret_cast<const double2*>(p + 2);
    a = u.x; b = u.y; c = v.x; d = v.y;
  }
}
// Two consecutive complex values (a 2x2 matrix row or column pair).
template <class R>
__device__ __forceinline__ void ldc2(const R* p, cx<R>& u, cx<R>& v) {
  R a, b, c, d;
  ld4<R>(p, a, b, c, d);
  u = mk<R>(a, b);
  v = mk<R>(c, d);
}

// Real coefficient times complex value, packed over (re, im): one FMUL2 /
// FFMA2 on sm_100+ for float, two scalar ops for double.
template <class R>
__device__ __forceinline__ cx<R> rmul(R a, cx<R> x) {
  if constexpr (std::is_same<R, float>::value) return __fmul2_rn(make_float2(a, a), x);
  else return mk<R>(a * x.x, a * x.y);
}
template <class R>
__device__ __forceinline__ cx<R> rfma(R a, cx<R> x, cx<R> acc) {
  if constexpr (std::is_same<R, float>::value) return __ffma2_rn(make_float2(a, a), x, acc);
  else return mk<R>(fma(a, x.x, acc.x), fma(a, x.y, acc.y));
}
// componentwise l * v + acc (sum of the components = Re(conj(l) v) contributions)
template <class R>
__device__ __forceinline__ cx<R> pfma(cx<R> l, cx<R> v, cx<R> acc) {
  if constexpr (std::is_same<R, float>::value) return __ffma2_rn(l, v, acc);
  else return mk<R>(fma(l.x, v.x, acc.x), fma(l.y, v.y, acc.y));
}

// 16-byte asynchronous global -> shared copy (Ampere+ LDGSTS path)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// butterfly sum in the state's real type: every lane gets the total
template <class R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sums of nv per-thread values val(v): each warp adds its lanes in R
// (butterfly) and lane 0 keeps the warp total in wred[v * kWarps + warp]
// (nv * kWarps entries of R); after a barrier thread v adds the kWarps warp
// totals in FP64 and calls out(v, total). Only those last additions run on
// the FP64 pipe, slow on this part (a per-warp FP64 butterfly for every value
// stalled the end of each pass); the order of the sums is fixed.
template <class R, class Val, class Out>
__device__ __forceinline__ void block_sums(R* wred, int nv, Val val, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = 0; v < nv; ++v) {
    const R s = warp_sum_r<R>(val(v));
    if (lane == 0) wred[v * kWarps + warp] = s;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += kThreads) {
    double s = 0;
    for (int w = 0; w < kWarps; ++w) s += (double)wred[v * kWarps + w];
    out(v, s);
  }
}

// Ring = CNOT(q->q+1 mod n) for q = 0..n-1.  With bit p = n-1-q:
//   forward  f(k):   bit p = parity(k >> p) for p <= n-2, bit n-1 = parity(k mod 2^(n-1))
//   inverse  f^-1(k) = k ^ (k >> 1) ^ (k & 1 ? 3 << (n-2) : 0)
__device__ __forceinline__ long long ring_finv(long long k, int n) {
  return k ^ (k >> 1) ^ ((k & 1) ? (3LL << (n - 2)) : 0LL);
}
// ring_finv for offsets below 2^30 (3 << (n - 2) fits for n <= 30)
__device__ __forceinline__ int ring_finv32(int k, int n) {
  return k ^ (k >> 1) ^ ((k & 1) ? (3 << (n - 2)) : 0);
}
__device__ __forceinline__ int par64(long long v) { return __popcll((unsigned long long)v) & 1; }
__device__ __forceinline__ long long ring_f(long long k, int n) {
  // prefix parities from the top: s_p = parity(k >> p)
  unsigned long long s = (unsigned long long)k;
  s ^= s >> 1; s ^= s >> 2; s ^= s >> 4; s ^= s >> 8; s ^= s >> 16; s ^= s >> 32;
  const long long low = (long long)(s & ((1ULL << (n - 1)) - 1));
  const long long top = (long long)par64(k & ((1LL << (n - 1)) - 1));
  return low | (top << (n - 1));
}
__device__ __forceinline__ int gray_inv(int x) {
  x ^= x >> 1; x ^= x >> 2; x ^= x >> 4; x ^= x >> 8; x ^= x >> 16;
  return x;
}

// compile-time z(j << 8) bits above bit 7 for the marginal accumulators
template <int ZM>
__device__ __forceinline__ constexpr int zj_bits(int j) {
  return ZM == Z_RINGXOR ? ((j << 8) ^ (j << 7)) : (j << 8);
}
__device__ __forceinline__ long long ztrans(long long k, int n, int zm) {
  if (zm == Z_RINGXOR) return k ^ ((k >> 1) | ((k & 1) << (n - 1)));
  return k;
}

// 32-bit forms for in-sample indices (n <= 30)
__device__ __forceinline__ int ztrans32(int k, int n, int zm) {
  if (zm == Z_RINGXOR) return k ^ ((k >> 1) | ((k & 1) << (n - 1)));
  return k;
}
template <class R>
__device__ __forceinline__ cx<R> diag_phase32(const R* tabs, int tb, int z) {
  const int mask = (1 << tb) - 1, T = 1 << tb;
  const cx<R> a = ldc<R>(tabs + 2 * (z & mask));
  const cx<R> b = ldc<R>(tabs + 2 * (T + ((z >> tb) & mask)));
  const cx<R> c = ldc<R>(tabs + 2 * (2 * T + ((z >> (2 * tb)) & mask)));
  return cmul<R>(cmul<R>(a, b), c);
}

// phase(z) = T0[z0] T1[z1] T2[z2]
template <class R>
__device__ __forceinline__ cx<R> diag_phase(const R* tabs, int tb, long long z) {
  const long long mask = (1LL << tb) - 1;
  const long long T = 1LL << tb;
  cx<R> a = ldc<R>(tabs + 2 * (z & mask));
  cx<R> b = ldc<R>(tabs + 2 * (T + ((z >> tb) & mask)));
  cx<R> c = ldc<R>(tabs + 2 * (2 * T + ((z >> (2 * tb)) & mask)));
  return cmul<R>(cmul<R>(a, b), c);
}

}  // namespace qc
