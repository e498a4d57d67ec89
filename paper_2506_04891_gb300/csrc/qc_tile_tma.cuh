// Tile pass with TMA-staged tiles (complex64, 2^12-amplitude tiles).
//
// The same method as the tile pass in qc_tile.cuh (the gates of one layer
// applied, or undone with their gradients, on the index bits a tile holds:
// Sec. 2.2.2's Einsum restricted to a tile of the state), with the copy in
// done by the Tensor Memory Accelerator instead of per-thread copies: one
// thread issues one cp.async.bulk.tensor per state and tile, completion is
// tracked by an mbarrier (transaction bytes), and the tile lands in shared
// memory in the 128-byte swizzled layout, which the rounds read without bank
// conflicts:
//   * the tile's local index i (bits [0, c) of the sample index, then
//     [h0, h0 + m)) is a 5-dimensional box of the state: 16 amplitudes (bits
//     0..3, 128 bytes, the swizzle span), bits 4..c-1, the gap [c, h0) (one
//     element of the box), bits [h0, h0 + m) and, merged with the batch, the
//     bits above;
//   * element i sits at i ^ (((i >> 4) & 7) << 1) (16-byte chunks XORed with
//     the 128-byte row), a GF(2)-linear map, so a round's element addresses
//     are one base XOR compile-time combinations of per-bit offsets;
//   * a round on bits 0..RB-1 reads and writes amplitude pairs as 16-byte
//     accesses (8 lanes of a quarter warp hit 8 distinct chunks); a round on
//     higher bits uses 8-byte accesses whose half warps cover 16 distinct
//     8-byte bank pairs (the planner checks this for every round).
// psi and lambda (backward) sit in two separate arrays.  Waits on an mbarrier
// are bounded in time; a CTA that gives up records it in a device counter
// (qc_kernel_timeouts) and leaves after waiting, again bounded, for its copies
// in flight.
#pragma once
#include <cuda.h>

#include "qc_tile.cuh"

namespace qc {

constexpr int kTmaT = 12;  // log2 amplitudes of a TMA-staged tile

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// true once the phase with this parity has completed; false after limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_load_5d(unsigned dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            int c4, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// the same box fetched into L2 only (no completion to wait for)
__device__ __forceinline__ void tma_prefetch_5d(const CUtensorMap* tm, int c0, int c1, int c2, int c3, int c4) {
  asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];\n" ::"l"(
                   reinterpret_cast<unsigned long long>(tm)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
               : "memory");
}

// element i of a TMA tile (8-byte elements, 128-byte swizzle)
__device__ __forceinline__ int tma_swz(int i) { return i ^ (((i >> 4) & 7) << 1); }

// CTAs that gave up waiting for a tile copy (one counter per translation
// unit, which is its own device module; read and cleared by qc_kernel_timeouts)
static __device__ unsigned long long g_tma_timeouts;
constexpr unsigned long long kTmaWaitNs = 2000000000ull;  // 2 s: far above any tile copy

// Shared-memory carve-out, from the 1024-byte aligned base: tile buffers
// [stages][NS][2^12] float2, one mbarrier per stage, staged coefficients,
// per-warp gradient sums, deferred companion sums, backward pre-diagonal
// marginals and running sums, phase block.
struct TmaSmem {
  size_t buf, bar, sco, sred, sdef, smarg, smacc, fph, end;
};
__host__ __device__ inline TmaSmem tma_smem_layout(const TilePass& P, int ns) {
  TmaSmem L;
  L.buf = 0;
  L.bar = L.buf + (size_t)P.nstage * ns * ((size_t)1 << kTmaT) * 8;
  L.sco = tsm_align16(L.bar + 8 * (size_t)P.nstage);
  L.sred = tsm_align16(L.sco + (size_t)P.ncoef * 4);
  L.sdef = tsm_align16(L.sred + (size_t)kWarps * (P.nslots > 0 ? P.nslots : 1) * sizeof(double));
  L.smarg = tsm_align16(L.sdef + (ns == 2 ? (size_t)tile_defer_slots(P) * kThreads * 4 : 0));
  const bool pre = ns == 2 && P.pre;
  L.smacc = tsm_align16(L.smarg + (pre ? (size_t)kWarps * (P.n + 1) * sizeof(double) : 0));
  L.fph = tsm_align16(L.smacc + (pre ? (size_t)kPreAcc * kThreads * 4 : 0));
  const size_t nfph = ns == 1 ? (P.post ? 1 : 0) : (pre ? 1 : 0);
  L.end = tsm_align16(L.fph + nfph * kFphBytes(4));
  return L;
}
// dynamic shared memory of a launch: the carve-out plus alignment slack
__host__ __device__ inline size_t tma_smem_bytes(const TilePass& P, int ns) {
  return tma_smem_layout(P, ns).end + 1024;
}

constexpr int tma_minb(int ns, int kind) { return (ns == 1 && kind == 1) ? 3 : 2; }

// Real single-qubit gates (RY) in scaled form (the square-root-free "fast
// Givens" rotation, Gentleman 1973): with c = M00 = M11, the rotation of a
// pair is c * (x0 + tau0 x1, x1 + tau1 x0), so a gate costs one packed FMA
// per output when the factor c is carried along instead of applied.  Every
// gate of the pass runs in this form (its record holds tau0, tau1 and the
// gradient factor gf), and after the pass's last gate the held amplitudes are
// multiplied by the product C of the factors, so the outputs are exact.
// Between gates the held amplitudes of psi and lambda are the true ones
// divided by the product of the factors so far, so a gate's gradient products
// carry that product squared, which gf (the product squared, including the
// gate's own factor) puts back.  The forward applies M, the backward M^T.
// The form is chosen per pass, so the round loop is compiled once per form
// with no per-gate branch between them (a per-gate choice had the compiler
// reconcile the two forms' registers with moves after every gate).
template <int RB, int I>
__device__ __forceinline__ void ap1t(float2* v, const float* m) {
  float t0, t1, gf, unused;
  ld4<float>(m, t0, t1, gf, unused);
#pragma unroll
  for (int a = 0; a < (1 << RB); ++a)
    if (!(a & (1 << I))) {
      const float2 x0 = v[a], x1 = v[a | (1 << I)];
      v[a] = rfma<float>(t0, x1, x0);
      v[a | (1 << I)] = rfma<float>(t1, x0, x1);
    }
}
template <int RB, int I, bool MAYCK>
__device__ __forceinline__ void bw1t(float2* p, float2* l, const float* m, int np, int ck_in, float* acc) {
  using C = float2;
  const int ck = MAYCK ? ck_in : 0;
  float t0, t1, gf, unused;
  ld4<float>(m, t0, t1, gf, unused);
  C ga = make_float2(0, 0), gb = make_float2(0, 0), hc = make_float2(0, 0);
  float hs = 0;
#pragma unroll
  for (int a = 0; a < (1 << RB); ++a)
    if (!(a & (1 << I))) {
      const int a1 = a | (1 << I);
      const C x0 = p[a], x1 = p[a1];
      const C y0 = rfma<float>(t0, x1, x0), y1 = rfma<float>(t1, x0, x1);
      p[a] = y0;
      p[a1] = y1;
      const C u0 = l[a], u1 = l[a1];
      const C w0 = rfma<float>(t0, u1, u0), w1 = rfma<float>(t1, u0, u1);
      l[a] = w0;
      l[a1] = w1;
      // 2 Re <l|(-i/2 Y)|p> = Re(l1* p0) - Re(l0* p1)
      ga = pfma<float>(w1, y0, ga);
      gb = pfma<float>(w0, y1, gb);
      if (ck == 1) {
        // companion RX: Im(l0* p1 + l1* p0), packed as l * swap(p)
        hc = pfma<float>(w0, make_float2(y1.y, y1.x), hc);
        hc = pfma<float>(w1, make_float2(y0.y, y0.x), hc);
      } else if (ck == 2) {
        hs += pauli_grad<float>(2, w0, w1, y0, y1);
      }
    }
  if (np) acc[I * 3] += gf * ((ga.x + ga.y) - (gb.x + gb.y));
  if (ck == 1) acc[I * 3 + 1] += gf * (hc.x - hc.y);
  else if (ck == 2) acc[I * 3 + 1] += gf * hs;
}

// Complex single-qubit gates with equal diagonal entries d = M00 = M11 (RX,
// SX, GPI2) in the same scaled form: M = d (I + T), T off-diagonal, so a
// gate costs one complex multiply-add per output instead of two.  Forward
// records (tau0, tau1) = (M01 / d, M10 / d): y0 = x0 + tau0 x1, y1 = x1 +
// tau1 x0.  Backward (M^dagger = conj(d) (I + T^dagger)): (sig0, sig1) =
// (M10 / d, M01 / d), y0 = x0 + conj(sig0) x1, y1 = x1 + conj(sig1) x0, then
// gf = |product of the factors so far|^2 and the record's A (unchanged) for
// the gradient.  After the last gate the held amplitudes are multiplied by
// the product C of the factors (backward: its conjugate).
// FIXED: every scaled record of the pass is tau0 = tau1 = -i (SX, RX(pi/2),
// GPI2(0): constant gates without gradients), so the gate is additions only.
template <int RB, int I, bool FIXED = false>
__device__ __forceinline__ void ap1tc(float2* v, const float* m) {
  float2 t0 = make_float2(0.f, -1.f), t1 = make_float2(0.f, -1.f);
  if (!FIXED) ldc2<float>(m, t0, t1);
#pragma unroll
  for (int a = 0; a < (1 << RB); ++a)
    if (!(a & (1 << I))) {
      const float2 x0 = v[a], x1 = v[a | (1 << I)];
      v[a] = cfma<float>(t0, x1, x0);
      v[a | (1 << I)] = cfma<float>(t1, x0, x1);
    }
}
template <int RB, int I, bool MAYCK, bool FIXED = false>
__device__ __forceinline__ void bw1tc(float2* p, float2* l, const float* m, int np_in, int gk, int ck_in,
                                      float* acc) {
  using C = float2;
  const int ck = MAYCK && !FIXED ? ck_in : 0;
  const int np = FIXED ? 0 : np_in;
  C s0 = make_float2(0.f, -1.f), s1 = make_float2(0.f, -1.f);
  if (!FIXED) ldc2<float>(m, s0, s1);
  const float gf = FIXED ? 1.f : m[4];
  float g = 0, h = 0;
  GenGrad<float> gg;
#pragma unroll
  for (int a = 0; a < (1 << RB); ++a)
    if (!(a & (1 << I))) {
      const int a1 = a | (1 << I);
      const C x0 = p[a], x1 = p[a1];
      const C y0 = cfmac<float>(s0, x1, x0), y1 = cfmac<float>(s1, x0, x1);
      p[a] = y0;
      p[a1] = y1;
      const C u0 = l[a], u1 = l[a1];
      const C w0 = cfmac<float>(s0, u1, u0), w1 = cfmac<float>(s1, u0, u1);
      l[a] = w0;
      l[a1] = w1;
      if (np) {
        if (gk == 1) {
          g += im_cdot<float>(w0, y1) + im_cdot<float>(w1, y0);
        } else {
          gg.add(w0, w1, y0, y1);
        }
      }
      if (ck) h += pauli_grad<float>(ck, w0, w1, y0, y1);
    }
  if (np) acc[I * 3] += gf * (gk == 1 ? g : gg.value(m + 8));
  if (ck) acc[I * 3 + 1] += gf * h;
}

// Rewrites a complex pass's staged records for the scaled form (one thread,
// per CTA), when every factor has |d| >= 2^-10, their running product stays
// >= 2^-60 in magnitude and M11 == M00 exactly; else returns false and leaves
// them.  *corr gets the factor the held amplitudes take after the last gate:
// C forward, conj(C) backward.  The ratios and the running product are formed
// in FP64 from the staged FP32 entries and rounded once (in FP32 their three
// roundings per ratio left the pass's output norm off by ~5e-7 on a 12-gate
// pass, 8x the full form's).
template <bool FWD>
__device__ bool scale_complex_records(float* sco, int nops, int nco, float2* corr) {
  if (nops < 1 || nco != (FWD ? 8 : 16)) return false;
  double cr = 1.0, ci = 0.0;
  for (int k = 0; k < nops; ++k) {
    const float* r = sco + nco * k;
    if (r[6] != r[0] || r[7] != r[1]) return false;
    const double dr = r[0], di = r[1];
    if (!(dr * dr + di * di >= 0x1p-20)) return false;
    const double nr = cr * dr - ci * di, ni = cr * di + ci * dr;
    cr = nr;
    ci = ni;
    if (!(cr * cr + ci * ci >= 0x1p-120)) return false;
  }
  cr = 1.0;
  ci = 0.0;
  for (int k = 0; k < nops; ++k) {
    float* r = sco + nco * k;
    const double dr = r[0], di = r[1], inv = 1.0 / (dr * dr + di * di);
    const double nr = cr * dr - ci * di, ni = cr * di + ci * dr;
    cr = nr;
    ci = ni;
    // x / d = x conj(d) / |d|^2
    const double m01r = r[2], m01i = r[3], m10r = r[4], m10i = r[5];
    const double q01r = (m01r * dr + m01i * di) * inv, q01i = (m01i * dr - m01r * di) * inv;
    const double q10r = (m10r * dr + m10i * di) * inv, q10i = (m10i * dr - m10r * di) * inv;
    r[0] = (float)(FWD ? q01r : q10r);
    r[1] = (float)(FWD ? q01i : q10i);
    r[2] = (float)(FWD ? q10r : q01r);
    r[3] = (float)(FWD ? q10i : q01i);
    r[4] = (float)(cr * cr + ci * ci);
    r[5] = r[6] = r[7] = 0.f;
  }
  *corr = make_float2((float)cr, (float)(FWD ? ci : -ci));
  return true;
}

// Rewrites a real pass's staged records for the scaled form (one thread, per
// CTA: the records are shared by the CTA's tiles).  Returns false, leaving the
// records as they are, when a factor is small (|c| < 2^-10) or their product
// would leave the normal range (< 2^-60); the pass then runs every gate in
// full form.  FWD: records become (M01 / M00, M10 / M11, gf, 0), else
// (M10 / M00, M01 / M11, gf, 0); *corr = (C, 0).  Ratios and product in FP64,
// rounded once (as above).
template <bool FWD>
__device__ bool scale_real_records(float* sco, int nops, int nco, float2* corr) {
  if (nops < 1 || nco != 4) return false;
  double cacc = 1.0;
  for (int k = 0; k < nops; ++k) {
    const float* r = sco + 4 * k;
    const float cc = r[0];
    if (!(fabsf(cc) >= 0x1p-10f) || r[3] != cc) return false;
    cacc *= cc;
    if (!(fabs(cacc) >= 0x1p-60)) return false;
  }
  cacc = 1.0;
  for (int k = 0; k < nops; ++k) {
    float* r = sco + 4 * k;
    const double m00 = r[0], m01 = r[1], m10 = r[2], m11 = r[3];
    cacc *= m00;
    r[0] = (float)(FWD ? m01 / m00 : m10 / m00);
    r[1] = (float)(FWD ? m10 / m11 : m01 / m11);
    r[2] = (float)(cacc * cacc);
    r[3] = 0.f;
  }
  *corr = make_float2((float)cacc, 0.f);
  return true;
}

// The op on register bit I of a round, if any: round r's ops are numbered
// from rop[r] in increasing bit order (the planner sorts them), every op of a
// pass stages the same number of coefficients (nco) and has the same
// gradient count and generator kinds, so the op's index and coefficient
// block follow from the round's presence mask without per-op lookups.
// SC, the pass's form: 0 full matrices, 1 scaled (single-qubit kinds 0 and
// 1), 2 scaled -i butterflies (kind 3: constant SX, additions only), -1 the
// runtime flag sc_rt chooses between 1 and 0 (complex kind 0: a round loop
// per form spilled registers there, the branch measured faster; for real
// passes the branch measured 1.6% slower on zz26 than a loop per form).
// FULL: every register bit of the round carries an op (the presence test and
// its branch are compiled out).
template <int NS, int RB, int KIND, int I, bool COMP, int SC, bool FULL = false>
__device__ __forceinline__ void tma_bit(unsigned rmask, int k0, int nco, int np, int gk, int ck, int pat,
                                        int sc_rt, float2* v0, float2* v1, const float* sco, float* acc) {
  using R = float;
  if (KIND == 2 && I + 1 >= RB) return;
  if (!FULL && !((rmask >> I) & 1u)) return;
  const int k = FULL ? k0 + I : k0 + __popc(rmask & ((1u << I) - 1u));
  const R* mc = sco + k * nco;
  if constexpr (KIND == 3) {
    // constant SX without gradients: -i butterflies, or the full matrices
    // when the records did not scale
    if constexpr (SC == 2) {
      if (NS == 1) ap1tc<RB, I, true>(v0, mc);
      else bw1tc<RB, I, false, true>(v0, v1, mc, 0, 0, 0, acc);
    } else {
      if (NS == 1) ap1<float, RB, I>(v0, mc, 0);
      else bw1<float, RB, I, false>(v0, v1, mc, 0, 0, 0, 0, acc);
    }
    return;
  }
  if constexpr (SC == 1 && KIND == 1) {
    if (NS == 1) ap1t<RB, I>(v0, mc);
    else bw1t<RB, I, COMP>(v0, v1, mc, np, ck, acc);
    return;
  }
  if constexpr ((SC == 1 || SC == -1) && KIND == 0) {
    if (SC == 1 || sc_rt) {
      if (NS == 1) ap1tc<RB, I>(v0, mc);
      else bw1tc<RB, I, COMP>(v0, v1, mc, np, gk, ck, acc);
      return;
    }
  }
  constexpr int I2 = (KIND == 2 && I + 1 < RB) ? I : 0;
  if (NS == 1) {
    if (KIND == 2) {
      if (pat) ap2<R, RB, I2, 1>(v0, mc);
      else ap2<R, RB, I2, 0>(v0, mc);
    } else {
      ap1<R, RB, I>(v0, mc, KIND == 1);
    }
  } else {
    if (KIND == 2) {
      if (pat) bw2<R, RB, I2, 1>(v0, v1, mc, np, acc);
      else bw2<R, RB, I2, 0>(v0, v1, mc, np, acc);
    } else {
      bw1<R, RB, I, COMP>(v0, v1, mc, KIND == 1, np, gk, ck, acc);
    }
  }
}

// NS = 1 forward, 2 backward.  PRE: backward 1 / 2 = undo a diagonal layer
// (identity / ring z map) in round 0 (contiguous pass, round 0 on bits 0..3);
// forward 2 / 3 = a following diagonal's phase in the last round (contiguous
// pass, last round on bits 8..11).
// COMP: the pass also takes companion gradients (a folded preceding RX / RY
// layer); without them that code is compiled out.
// XL: the pass first undoes (backward) or applies (forward) an X layer on
// every qubit, k -> ~k: each tile is loaded from the mirrored box and its
// elements are addressed in reversed order (local index i ^ (T - 1)), which
// the XOR swizzle and the register bases keep linear.
template <int NS, int RB, int KIND, int PRE, bool COMP, bool XL = false>
__global__ void __launch_bounds__(kThreads, tma_minb(NS, KIND))
    k_tile_tma(const __grid_constant__ TilePass P, const __grid_constant__ CUtensorMap tm0,
               const __grid_constant__ CUtensorMap tm1, const float* __restrict__ coef, float2* dst0,
               float2* dst1, double* __restrict__ part, int cps) {
  using R = float;
  using C = float2;
  constexpr int t = kTmaT;
  constexpr int T = 1 << t;
  extern __shared__ unsigned char smraw_tma[];
  const unsigned raw_sa = smem_u32(smraw_tma);
  unsigned char* sm = smraw_tma + (((raw_sa + 1023u) & ~1023u) - raw_sa);
  const TmaSmem lay = tma_smem_layout(P, NS);
  C* buf = reinterpret_cast<C*>(sm + lay.buf);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(sm + lay.bar);
  R* sco = reinterpret_cast<R*>(sm + lay.sco);
  double* sred = reinterpret_cast<double*>(sm + lay.sred);
  R* sdef = reinterpret_cast<R*>(sm + lay.sdef);
  double* smarg = reinterpret_cast<double*>(sm + lay.smarg);
  R* macc = reinterpret_cast<R*>(sm + lay.smacc) + threadIdx.x;
  unsigned char* fph = sm + lay.fph;

  const int n = P.n, c = P.c, h0 = P.h0;
  const int m = t - c, gap = h0 - c;
  const int nst = P.nstage;
  const long long tps = 1LL << (n - t);
  const int b = blockIdx.x / cps;
  const int r0 = blockIdx.x % cps;
  const int cmask = (1 << c) - 1;
  const long long sb = (long long)b << n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  C* d0b = dst0 + sb;
  C* d1b = NS == 2 ? dst1 + sb : nullptr;
  auto tile_base = [&](long long f) -> int {
    return (int)(((f & ((1LL << gap) - 1)) << c) | ((f >> gap) << (h0 + m)));
  };
  auto elem_off = [&](int i) -> int { return (i & cmask) | ((i >> c) << h0); };

  for (int k = 0; k < P.nops; ++k) {
    const TileOp& o = P.ops[k];
    const R* s = coef + o.coef + (long long)b * o.bstride;
    for (int i = threadIdx.x; i < o.nco; i += kThreads) sco[o.soff + i] = s[i];
  }
  // per-pass op data (uniform over the pass's ops) and the presence mask of
  // every round's register bits (4 bits per round)
  const int op_nco = P.ops[0].nco, op_np = P.ops[0].np, op_gk = P.ops[0].gk, op_ck = COMP ? P.ops[0].ck : 0;
  const int op_pat = P.ops[0].pat;
  unsigned rmask_all = 0;
  for (int r = 0; r < P.nrounds; ++r)
#pragma unroll
    for (int i = 0; i < RB; ++i)
      if (P.rbit[r][i] >= 0) rmask_all |= 1u << (4 * r + i);
  if (NS == 2) {
    for (int i = threadIdx.x; i < kWarps * P.nslots; i += kThreads) sred[i] = 0;
    for (int s = 0, nd = tile_defer_slots(P); s < nd; ++s) sdef[s * kThreads + threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(smem_u32(&bars[s]), 1);
    mbar_init_fence();
  }

  constexpr int kAR = RB == 4 ? 3 : 4;
  R acct[kAR][4];
#pragma unroll
  for (int r = 0; r < kAR; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) acct[r][i] = 0;

  // backward pre-diagonal (round 0 holds bits 0..3 of group g = tid: local
  // indices g << 4 | a): the element z bits are 0..3 (and n - 1 for the ring
  // map, through index bit 0); bits whose z depends on the tile are warp
  // uniform (index bits >= 9 only); the others depend on the thread alone
  constexpr bool pre_b = NS == 2 && PRE >= 1;
  constexpr int zmc = PRE == 2 ? Z_RINGXOR : Z_IDENT;
  const R* ptabs = coef + P.pre_coef + (long long)b * P.pre_bstride;
  int zT = 0, fmask = 0;
  bool lane_f = false;
  if (pre_b) {
    fph_setup<R>(fph, ptabs, P.pre_tb, zmc, n, t, c, h0, 0, 4);
    const int sem = reinterpret_cast<const FwdPhaseMeta*>(fph)->semask;
    zT = ztrans32(threadIdx.x << 4, n, zmc);
    for (int q = t; q < n; ++q) fmask |= ztrans32(1 << q, n, zmc);
    fmask &= ~sem;
    lane_f = ((fmask >> lane) & 1) != 0;
    for (int j = 0; j < kPreAcc; ++j) macc[j * kThreads] = 0;
  }
  // forward post phase in the last round (bits 8..11 of a contiguous pass)
  const R* fpost_tabs = coef + P.post_coef + (long long)b * P.post_bstride;
  const int rlast = P.nrounds - 1;
  if (NS == 1 && PRE >= 2 && P.post)
    fph_setup<R>(fph, fpost_tabs, P.post_tb, P.post_zmode, n, t, c, h0, P.rlo[rlast], RB);
  const bool fpost_ok = NS == 1 && PRE >= 2 && P.post && reinterpret_cast<const FwdPhaseMeta*>(fph)->ok;
  // the last round stores straight from registers unless the pass scatters
  // (or stores nothing); the single-buffer backward then starts the next
  // tile's copy as soon as every thread holds its last-round elements
  const bool dstore = P.store && !P.scatter;
  const bool early = NS == 2 && nst == 1 && dstore && RB == 4;
  // single-qubit passes: switch the records to the scaled form when every
  // gate allows it (kind 3: when every raw record is d (I - i X), M01 = M10 =
  // -i M00, M11 = M00); s_corr is the factor the held amplitudes take after
  // the pass's last gate
  __shared__ int s_sc;
  __shared__ float2 s_corr;
  if (KIND != 2) {
    __syncthreads();  // the records are staged
    if (threadIdx.x == 0) {
      float2 corr = make_float2(1.f, 0.f);
      int sc = 0;
      if (KIND == 3) {
        bool fx = op_np == 0 && op_ck == 0;
        for (int k = 0; fx && k < P.nops; ++k) {
          const float* r = sco + op_nco * k;
          fx = r[6] == r[0] && r[7] == r[1] && r[2] == r[1] && r[3] == -r[0] && r[4] == r[1] && r[5] == -r[0];
        }
        if (fx && scale_complex_records<NS == 1>(sco, P.nops, op_nco, &corr)) sc = 2;
      } else if (KIND == 1) {
        if (scale_real_records<NS == 1>(sco, P.nops, op_nco, &corr)) sc = 1;
      } else {
        if (scale_complex_records<NS == 1>(sco, P.nops, op_nco, &corr)) sc = 1;
      }
      s_sc = sc;
      s_corr = corr;
    }
  }
  __syncthreads();
  const int pass_sc = KIND != 2 ? s_sc : 0;
  const float2 corr = s_corr;

  unsigned pending = 0, phase = 0;
  // box coordinates of tile f (XL: of the mirrored tile, every index bit
  // outside the box complemented; the batch bits above them are not)
  const long long hmask = (1LL << (n - h0 - m)) - 1;
  auto coord2 = [&](long long f) { return (int)((f & ((1LL << gap) - 1)) ^ (XL ? ((1LL << gap) - 1) : 0)); };
  auto coord4 = [&](long long f) {
    return (int)(((long long)b << (n - h0 - m)) | ((f >> gap) ^ (XL ? hmask : 0)));
  };
  auto issue = [&](long long f, int s) {  // thread 0
    const int c2 = coord2(f);
    const int c4 = coord4(f);
    const unsigned bar = smem_u32(&bars[s]);
    mbar_expect_tx(bar, (unsigned)(NS * T * sizeof(C)));
    tma_load_5d(smem_u32(buf + (size_t)s * NS * T), &tm0, 0, 0, c2, 0, c4, bar);
    if (NS == 2) tma_load_5d(smem_u32(buf + (size_t)s * NS * T + T), &tm1, 0, 0, c2, 0, c4, bar);
    pending |= 1u << s;
  };
  // the tile after the ones in flight, pulled into L2 while this one is
  // processed, so its copy into shared memory does not wait on DRAM
  auto prefetch = [&](long long f) {  // thread 0
    const int c2 = coord2(f);
    const int c4 = coord4(f);
    tma_prefetch_5d(&tm0, 0, 0, c2, 0, c4);
    if (NS == 2) tma_prefetch_5d(&tm1, 0, 0, c2, 0, c4);
  };
  long long f = r0;
  int slot = 0;
  if (threadIdx.x == 0)
    for (int j = 0; j < nst; ++j)
      if (f + (long long)j * cps < tps) issue(f + (long long)j * cps, j);

  for (; f < tps; f += cps) {
    const bool ok = mbar_wait_bounded(smem_u32(&bars[slot]), (phase >> slot) & 1u, kTmaWaitNs);
    phase ^= 1u << slot;
    pending &= ~(1u << slot);
    if (__syncthreads_or(!ok)) {
      // a copy did not complete in time: record it, wait (bounded) for the
      // copies this CTA still has in flight, and leave
      if (threadIdx.x == 0) {
        atomicAdd(&g_tma_timeouts, 1ull);
        for (int s = 0; s < nst; ++s)
          if (((pending >> s) & 1u) || s == slot)
            mbar_wait_bounded(smem_u32(&bars[s]), ((phase ^ (s == slot ? 1u << s : 0u)) >> s) & 1u, kTmaWaitNs);
      }
      __syncthreads();
      return;
    }
    C* S0 = buf + (size_t)slot * NS * T;
    C* S1 = S0 + T;
    const int kb = tile_base(f);
    if (threadIdx.x == 0 && f + (long long)nst * cps < tps) prefetch(f + (long long)nst * cps);

    // the round loop, compiled once per form of the pass
    auto rounds = [&](auto form) {
      constexpr int SC = decltype(form)::value;
#pragma unroll 1
    for (int r = 0; r < P.nrounds; ++r) {
      const int lo = P.rlo[r];
      const bool last = r == rlast;
      const unsigned rmask = (rmask_all >> (4 * r)) & 15u;
      const int k0 = P.rop[r];
      R acc[RB * 3];
#pragma unroll
      for (int i = 0; i < RB * 3; ++i) acc[i] = 0;
      int basis[RB], eo[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        basis[j] = tma_swz(1 << (lo + j));
        eo[j] = elem_off(1 << (lo + j));  // global offset of register bit j (disjoint bits)
      }
      // the group loop, compiled for rounds whose register bits all carry a
      // gate (FULL: no presence branch after each gate, whose join had the
      // compiler move the held amplitudes between registers) and for the rest
      auto groups = [&](auto full_c) {
        constexpr bool FULL = decltype(full_c)::value;
      for (int g = threadIdx.x; g < (T >> RB); g += kThreads) {
        const int li = (g & ((1 << lo) - 1)) | ((g >> lo) << (lo + RB));
        const int pb = tma_swz(XL ? (li ^ (T - 1)) : li);
        C v0[1 << RB], v1[NS == 2 ? (1 << RB) : 1];
        if (lo == 0) {
          // amplitude pairs (bit 0) as 16-byte accesses; the swizzle keeps bit 0
          // (XL: the pair's elements sit in reversed order at pb ^ 1, pb)
#pragma unroll
          for (int a = 0; a < (1 << RB); a += 2) {
            int ad = XL ? (pb ^ 1) : pb;
#pragma unroll
            for (int j = 1; j < RB; ++j)
              if (a & (1 << j)) ad ^= basis[j];
            const float4 q = *reinterpret_cast<const float4*>(&S0[ad]);
            v0[a] = XL ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
            v0[a + 1] = XL ? make_float2(q.x, q.y) : make_float2(q.z, q.w);
            if constexpr (NS == 2) {
              const float4 u = *reinterpret_cast<const float4*>(&S1[ad]);
              v1[a] = XL ? make_float2(u.z, u.w) : make_float2(u.x, u.y);
              v1[a + 1] = XL ? make_float2(u.x, u.y) : make_float2(u.z, u.w);
            }
          }
        } else {
#pragma unroll
          for (int a = 0; a < (1 << RB); ++a) {
            int ad = pb;
#pragma unroll
            for (int j = 0; j < RB; ++j)
              if (a & (1 << j)) ad ^= basis[j];
            v0[a] = S0[ad];
            if constexpr (NS == 2) v1[a] = S1[ad];
          }
        }
        if constexpr (pre_b) {
          if (r == 0) {
            // undo the diagonal layer on psi and lambda: element a has z =
            // z0 ^ z(a) with the compile-time pattern a ^ (a >> 1) (| a_0 at
            // z bit n - 1, pattern bit 4) for the ring map, a for the identity;
            // w = Im(conj(lambda) psi) is unchanged by the phase
            constexpr int nse = PRE == 2 ? 5 : 4;
            const int z0 = ztrans32(kb | li, n, zmc);
            const int semask = PRE == 2 ? (15 | (1 << (n - 1))) : 15;
            const int z0se = (z0 & 15) | (PRE == 2 ? ((z0 >> (n - 1)) & 1) << 4 : 0);
            const C p0 = diag_phase32<R>(ptabs, P.pre_tb, z0 & ~semask);
            const C* ratio = reinterpret_cast<const C*>(fph + ((sizeof(FwdPhaseMeta) + 15) & ~(size_t)15));
            R Wt = 0, Ase[5] = {0, 0, 0, 0, 0};
#pragma unroll
            for (int a = 0; a < (1 << RB); ++a) {
              const int pat = PRE == 2 ? ((a ^ (a >> 1)) | ((a & 1) << 4)) : a;
              const C ph = cmul<R>(p0, ratio[z0se ^ pat]);
              const R w = im_cdot<R>(v1[a], v0[a]);
              v0[a] = cmulc<R>(ph, v0[a]);
              v1[a] = cmulc<R>(ph, v1[a]);
              Wt += w;
#pragma unroll
              for (int j = 0; j < nse; ++j)
                if ((pat >> j) & 1) Ase[j] += w;
            }
            if (P.pre_grad) {
#pragma unroll
              for (int j = 0; j < nse; ++j)
                if ((z0se >> j) & 1) Ase[j] = Wt - Ase[j];
              macc[0] += Wt;
#pragma unroll
              for (int j = 0; j < nse; ++j) macc[(1 + j) * kThreads] += Ase[j];
              const R sw = warp_sum_r<R>(Wt);
              if (lane_f && ((z0 >> lane) & 1)) macc[11 * kThreads] += sw;
            }
          }
        }
        if (early && last) {
          // every thread holds its elements of the last round: the buffer is
          // free for the next tile's copy
          __syncthreads();
          if (threadIdx.x == 0 && f + cps < tps) issue(f + cps, 0);
        }
        tma_bit<NS, RB, KIND, 0, COMP, SC, FULL>(rmask, k0, op_nco, op_np, op_gk, op_ck, op_pat, pass_sc, v0, v1, sco, acc);
        if (RB > 1)
          tma_bit<NS, RB, KIND, (RB > 1 ? 1 : 0), COMP, SC, FULL>(rmask, k0, op_nco, op_np, op_gk, op_ck, op_pat, pass_sc, v0, v1,
                                                           sco, acc);
        if (RB > 2)
          tma_bit<NS, RB, KIND, (RB > 2 ? 2 : 0), COMP, SC, FULL>(rmask, k0, op_nco, op_np, op_gk, op_ck, op_pat, pass_sc, v0, v1,
                                                           sco, acc);
        if (RB > 3)
          tma_bit<NS, RB, KIND, (RB > 3 ? 3 : 0), COMP, SC, FULL>(rmask, k0, op_nco, op_np, op_gk, op_ck, op_pat, pass_sc, v0, v1,
                                                           sco, acc);
        if ((SC > 0 || (SC < 0 && pass_sc)) && last) {
          // the pass's gates are all applied: restore the product of the
          // scaled form's factors (folded into the phase below where there
          // is one)
          if (!(NS == 1 && PRE >= 2 && fpost_ok)) {
#pragma unroll
            for (int a = 0; a < (1 << RB); ++a) {
              if (KIND == 1) {
                v0[a] = rmul<R>(corr.x, v0[a]);
                if constexpr (NS == 2) v1[a] = rmul<R>(corr.x, v1[a]);
              } else {
                v0[a] = cmul<R>(corr, v0[a]);
                if constexpr (NS == 2) v1[a] = cmul<R>(corr, v1[a]);
              }
            }
          }
        }
        if (NS == 1 && PRE >= 2 && fpost_ok && last) {
          // group g = tid holds local indices g | a << 8 of a contiguous pass:
          // z = z0 ^ z(a << 8) with the compile-time pattern a ^ (a << 1)
          // (ring) or a (identity) over z bits zlo .. 11
          constexpr int zlo = PRE == 2 ? 7 : 8, nse = 12 - zlo;
          constexpr int semask = ((1 << nse) - 1) << zlo;
          const int z0 = ztrans32(kb | li, n, PRE == 2 ? Z_RINGXOR : Z_IDENT);
          const int z0se = (z0 >> zlo) & ((1 << nse) - 1);
          C p0 = diag_phase32<R>(fpost_tabs, P.post_tb, z0 & ~semask);
          if (SC > 0 || (SC < 0 && pass_sc)) p0 = cmul<R>(p0, corr);
          const C* ratio = reinterpret_cast<const C*>(fph + ((sizeof(FwdPhaseMeta) + 15) & ~(size_t)15));
#pragma unroll
          for (int a = 0; a < (1 << RB); ++a) {
            const int pat = PRE == 2 ? (a ^ (a << 1)) : a;
            v0[a] = cmul<R>(cmul<R>(p0, ratio[z0se ^ pat]), v0[a]);
          }
        }
        if (last && dstore) {
          // element a sits at gb + (sum of eo[j] over the set bits j of a)
          const int gb = kb | elem_off(li);
          C* o0 = d0b + gb;
          C* o1 = NS == 2 ? d1b + gb : nullptr;
#pragma unroll
          for (int a = 0; a < (1 << RB); ++a) {
            int go = 0;
#pragma unroll
            for (int j = 0; j < RB; ++j)
              if (a & (1 << j)) go += eo[j];
            o0[go] = v0[a];
            if constexpr (NS == 2) o1[go] = v1[a];
          }
        } else if (lo == 0) {
#pragma unroll
          for (int a = 0; a < (1 << RB); a += 2) {
            int ad = XL ? (pb ^ 1) : pb;
#pragma unroll
            for (int j = 1; j < RB; ++j)
              if (a & (1 << j)) ad ^= basis[j];
            const int e0 = XL ? a + 1 : a, e1 = XL ? a : a + 1;
            *reinterpret_cast<float4*>(&S0[ad]) = make_float4(v0[e0].x, v0[e0].y, v0[e1].x, v0[e1].y);
            if constexpr (NS == 2)
              *reinterpret_cast<float4*>(&S1[ad]) = make_float4(v1[e0].x, v1[e0].y, v1[e1].x, v1[e1].y);
          }
        } else {
#pragma unroll
          for (int a = 0; a < (1 << RB); ++a) {
            int ad = pb;
#pragma unroll
            for (int j = 0; j < RB; ++j)
              if (a & (1 << j)) ad ^= basis[j];
            S0[ad] = v0[a];
            if constexpr (NS == 2) S1[ad] = v1[a];
          }
        }
      }
      };
      if constexpr (KIND != 2) {
        if (rmask == (1u << RB) - 1u) groups(std::true_type{});
        else groups(std::false_type{});
      } else {
        groups(std::false_type{});
      }
      if (NS == 2) {
        if (P.defer == 1) {
#pragma unroll
          for (int rr = 0; rr < kAR; ++rr)
            if (rr == r) {
#pragma unroll
              for (int i = 0; i < (RB < 4 ? RB : 4); ++i) acct[rr][i] += acc[i * 3];
            }
          if (P.ncomp) {
#pragma unroll
            for (int i = 0; i < (RB < 4 ? RB : 4); ++i) {
              const int cs = P.rcslot[r][i];
              if (cs >= 0) sdef[(cs - P.nslots + P.ncomp) * kThreads + threadIdx.x] += acc[i * 3 + 1];
            }
          }
        } else if (P.defer == 2) {
          // the thread's column of every slot in shared memory (each thread
          // touches only its own words: no barrier needed)
#pragma unroll
          for (int i = 0; i < RB; ++i) {
            const int k = P.rbit[r][i];
            if (k < 0) continue;
            const TileOp& o = P.ops[k];
            R* col = sdef + (int)o.slot * kThreads + threadIdx.x;
#pragma unroll
            for (int q = 0; q < 3; ++q)
              if (q < o.np) col[q * kThreads] += acc[i * 3 + q];
            if (o.ck) sdef[(int)o.cslot * kThreads + threadIdx.x] += acc[i * 3 + 1];
          }
        } else {
#pragma unroll
          for (int i = 0; i < RB; ++i) {
            const int k = P.rbit[r][i];
            if (k < 0) continue;
            const TileOp& o = P.ops[k];
#pragma unroll
            for (int q = 0; q < 3; ++q)
              if (q < o.np) {
                const double v = warp_sum((double)acc[i * 3 + q]);
                if (lane == 0) sred[warp * P.nslots + o.slot + q] += v;
              }
            if (o.ck) {
              const double v = warp_sum((double)acc[i * 3 + 1]);
              if (lane == 0) sred[warp * P.nslots + o.cslot] += v;
            }
          }
        }
      }
      __syncthreads();
    }

    };
    if (KIND == 0) rounds(std::integral_constant<int, -1>{});
    else if (KIND == 3 && pass_sc == 2) rounds(std::integral_constant<int, KIND == 3 ? 2 : 0>{});
    else if (KIND == 1 && pass_sc == 1) rounds(std::integral_constant<int, KIND == 1 ? 1 : 0>{});
    else rounds(std::integral_constant<int, 0>{});

    if (P.store && P.scatter) {
      // backward scatter through the CNOT ring's inverse map f^-1, in 16-byte
      // pairs: f^-1(k ^ 1 ^ 2^(n-1)) = f^-1(k) ^ 1, and this top pass holds
      // index bit 0 (local 0) and bit n-1 (local t-1)
      for (int i = threadIdx.x; i < (T >> 1); i += kThreads) {
        const int d = ring_finv32(kb | elem_off(i), n);
        const int pa = tma_swz(i), pp = tma_swz(i ^ 1 ^ (T >> 1));
        const C qa = S0[pa], qb = S0[pp];
        const bool odd = d & 1;
        const int dd = d & ~1;
        *reinterpret_cast<float4*>(&d0b[dd]) = odd ? make_float4(qb.x, qb.y, qa.x, qa.y)
                                                   : make_float4(qa.x, qa.y, qb.x, qb.y);
        if constexpr (NS == 2) {
          const C ua = S1[pa], ub = S1[pp];
          *reinterpret_cast<float4*>(&d1b[dd]) = odd ? make_float4(ub.x, ub.y, ua.x, ua.y)
                                                     : make_float4(ua.x, ua.y, ub.x, ub.y);
        }
      }
    }
    __syncthreads();  // the stage is free
    const long long fn = f + (long long)nst * cps;
    if (!early && threadIdx.x == 0 && fn < tps) issue(fn, slot);
    slot = slot + 1 == nst ? 0 : slot + 1;
  }

  if constexpr (NS == 2) {
    // gradient sums over the block: per-warp totals in R, FP64 across warps
    const long long nblk = gridDim.x;
    auto slot_out = [&](int v, double sum) { part[(long long)v * nblk + blockIdx.x] = sum; };
    if (P.defer == 2) {
      block_sums<R>(reinterpret_cast<R*>(sred), P.nslots,
                    [&](int v) { return sdef[v * kThreads + threadIdx.x]; }, slot_out);
    } else if (P.defer == 1) {
      // rounds' register sums (one per slot), then the companions' columns
      const int nr = P.nslots - P.ncomp;
      block_sums<R>(
          reinterpret_cast<R*>(sred), P.nslots,
          [&](int v) -> R {
            if (v >= nr) return sdef[(v - nr) * kThreads + threadIdx.x];
            R a = 0;
#pragma unroll
            for (int r = 0; r < kAR; ++r)
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (P.rslot[r][i] == v) a = acct[r][i];
            return a;
          },
          slot_out);
    } else if (P.nslots > 0) {
      // per-round sums: sred holds every warp's FP64 totals
      __syncthreads();
      for (int s = threadIdx.x; s < P.nslots; s += kThreads) {
        double v = 0;
        for (int w = 0; w < kWarps; ++w) v += sred[w * P.nslots + s];
        slot_out(s, v);
      }
    }
    if (pre_b && P.pre_grad) {
      // u_p = sum over the thread's elements of w * z_p: element bits exactly,
      // the rest from the thread's total and its tile-independent z bits; the
      // tile-dependent (warp-uniform) bits were summed per warp into lane p's
      // mF, which lane p adds to its u_p
      const FwdPhaseMeta* pm = reinterpret_cast<const FwdPhaseMeta*>(fph);
      const R mW = macc[0], mF = macc[11 * kThreads];
      block_sums<R>(
          reinterpret_cast<R*>(smarg), n + 1,
          [&](int v) -> R {
            if (v == 0) return mW;
            const int p = v - 1;
            R u;
            int js = -1;
            for (int j = 0; j < pm->nse; ++j)
              if (pm->sepos[j] == p) js = j;
            if (js >= 0) u = macc[(1 + js) * kThreads];
            else if ((fmask >> p) & 1) u = 0;
            else u = ((zT >> p) & 1) ? mW : (R)0;
            return lane == p ? u + mF : u;
          },
          [&](int v, double sum) { part[P.pre_moff + (long long)v * nblk + blockIdx.x] = sum; });
    }
  }
}

}  // namespace qc
