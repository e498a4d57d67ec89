// Tile pass: the persistent kernel that applies (forward) or undoes with
// gradients (backward) the gates of one layer on a tile of 2^t amplitudes
// staged in shared memory, and its launch templates.  Instantiated by
// qc_tile_fwd.cu (NS = 1) and qc_tile_bwd.cu (NS = 2).
#pragma once
#include "qc_device.cuh"
#include "qc_kernels.h"

namespace qc {

// ---------------------------------------------------------------------------
// Tile pass: register-blocked single-qubit and two-qubit gate ops
// ---------------------------------------------------------------------------

// forward single-qubit op on register bit I
// `m` is the staged record: the packed real matrix for a real op, else M
// (2x2 complex) followed, backward, by A = M^dagger dM.
template <class R, int RB, int I>
__device__ __forceinline__ void ap1(cx<R>* v, const R* m, int real) {
  using C = cx<R>;
  if (real) {
    R m00, m01, m10, m11;
    ld4<R>(m, m00, m01, m10, m11);
#pragma unroll
    for (int a = 0; a < (1 << RB); ++a)
      if (!(a & (1 << I))) {
        C x0 = v[a], x1 = v[a | (1 << I)];
        v[a] = rfma<R>(m01, x1, rmul<R>(m00, x0));
        v[a | (1 << I)] = rfma<R>(m11, x1, rmul<R>(m10, x0));
      }
  } else {
    C m00, m01, m10, m11;
    ldc2<R>(m, m00, m01);
    ldc2<R>(m + 4, m10, m11);
#pragma unroll
    for (int a = 0; a < (1 << RB); ++a)
      if (!(a & (1 << I))) {
        C x0 = v[a], x1 = v[a | (1 << I)];
        v[a] = cfma<R>(m01, x1, cmul<R>(m00, x0));
        v[a | (1 << I)] = cfma<R>(m11, x1, cmul<R>(m10, x0));
      }
  }
}

// 2 Re <l|(-i/2 G)|p> on one amplitude pair, G = X (ck 1) or Y (ck 2):
// Im(l0* p1 + l1* p0) and Re(l1* p0) - Re(l0* p1).
template <class R>
__device__ __forceinline__ R pauli_grad(int ck, cx<R> w0, cx<R> w1, cx<R> y0, cx<R> y1) {
  if (ck == 1) return im_cdot<R>(w0, y1) + im_cdot<R>(w1, y0);
  return re_cdot<R>(w1, y0) - re_cdot<R>(w0, y1);
}

// backward single-qubit op: undo M on psi and lambda, then accumulate
// 2 Re <lambda| A |psi> on the gate's input side into acc[3 I].  With a
// companion generator ck, also the gradient of the preceding layer's RX / RY
// gate on the same qubit into acc[3 I + 1]: its generator commutes with that
// gate, so the pair just undone (that layer's output side) gives it.
// MAYCK = false compiles the companion code out (ck is then ignored): the
// compiler otherwise evaluates it for every pair and selects the result.
// Gradient of a single-qubit gate with a generic generator, 2 Re <w|A|y>
// summed over a thread's pairs, A = M^dagger dM.  M is unitary, so A is
// anti-Hermitian: A00 = i a0 and A11 = i a1 with a0, a1 real, A10 = -conj(A01),
// and
//   2 Re <w|A|y> = 2 Re(A01 D) - 2 a0 Im(w0* y0) - 2 a1 Im(w1* y1),
//   D = w0* y1 - w1 conj(y0).
// A thread sums the componentwise products behind Im(w0* y0), Im(w1* y1) and
// D over its pairs (six packed multiply-adds per pair, where the dense
// form took two complex matrix-vector products and two inner products) and
// applies A once per gate.
template <class R>
struct GenGrad {
  cx<R> pa, pb, pc, pd, pe, pf;
  __device__ __forceinline__ GenGrad() {
    pa = pb = pc = pd = pe = pf = mk<R>(0, 0);
  }
  __device__ __forceinline__ void add(cx<R> w0, cx<R> w1, cx<R> y0, cx<R> y1) {
    const cx<R> s0 = mk<R>(y0.y, y0.x), s1 = mk<R>(y1.y, y1.x);
    pa = pfma<R>(w0, y1, pa);  // Re(w0* y1) = pa.x + pa.y
    pb = pfma<R>(w1, y0, pb);  // Re(w1 conj(y0)) = pb.x + pb.y
    pc = pfma<R>(w0, s1, pc);  // Im(w0* y1) = pc.x - pc.y
    pd = pfma<R>(w1, s0, pd);  // -Im(w1 conj(y0)) = pd.x - pd.y
    pe = pfma<R>(w0, s0, pe);  // Im(w0* y0) = pe.x - pe.y
    pf = pfma<R>(w1, s1, pf);  // Im(w1* y1) = pf.x - pf.y
  }
  // a: the record's A (row-major 2x2 complex: A00, A01, A10, A11)
  __device__ __forceinline__ R value(const R* a) const {
    const R a0 = a[1], a01r = a[2], a01i = a[3], a1 = a[7];
    const R dre = (pa.x + pa.y) - (pb.x + pb.y);
    const R dim = (pc.x - pc.y) + (pd.x - pd.y);
    return 2 * (a01r * dre - a01i * dim) - 2 * (a0 * (pe.x - pe.y) + a1 * (pf.x - pf.y));
  }
};

template <class R, int RB, int I, bool MAYCK = true>
__device__ __forceinline__ void bw1(cx<R>* p, cx<R>* l, const R* m, int real, int np, int gk, int ck_in,
                                    R* acc) {
  using C = cx<R>;
  const int ck = MAYCK ? ck_in : 0;
  if (real) {
    // RY (the only real gate; m is its packed real matrix): undo with M^T;
    // 2 Re <l|(-i/2 Y)|p> = Re(l1* p0) - Re(l0* p1)
    R m00, m01, m10, m11;
    ld4<R>(m, m00, m01, m10, m11);
    C ga = mk<R>(0, 0), gb = mk<R>(0, 0);
    if (ck == 1) {
      // companion RX: Im(l0* p1 + l1* p0), packed as l * swap(p)
      C hc = mk<R>(0, 0);
#pragma unroll
      for (int a = 0; a < (1 << RB); ++a)
        if (!(a & (1 << I))) {
          const int a1 = a | (1 << I);
          C x0 = p[a], x1 = p[a1];
          C y0 = rfma<R>(m10, x1, rmul<R>(m00, x0));
          C y1 = rfma<R>(m11, x1, rmul<R>(m01, x0));
          p[a] = y0; p[a1] = y1;
          C u0 = l[a], u1 = l[a1];
          C w0 = rfma<R>(m10, u1, rmul<R>(m00, u0));
          C w1 = rfma<R>(m11, u1, rmul<R>(m01, u0));
          l[a] = w0; l[a1] = w1;
          ga = pfma<R>(w1, y0, ga);
          gb = pfma<R>(w0, y1, gb);
          hc = pfma<R>(w0, mk<R>(y1.y, y1.x), hc);
          hc = pfma<R>(w1, mk<R>(y0.y, y0.x), hc);
        }
      acc[I * 3 + 1] += hc.x - hc.y;
    } else {
#pragma unroll
      for (int a = 0; a < (1 << RB); ++a)
        if (!(a & (1 << I))) {
          const int a1 = a | (1 << I);
          C x0 = p[a], x1 = p[a1];
          C y0 = rfma<R>(m10, x1, rmul<R>(m00, x0));
          C y1 = rfma<R>(m11, x1, rmul<R>(m01, x0));
          p[a] = y0; p[a1] = y1;
          C u0 = l[a], u1 = l[a1];
          C w0 = rfma<R>(m10, u1, rmul<R>(m00, u0));
          C w1 = rfma<R>(m11, u1, rmul<R>(m01, u0));
          l[a] = w0; l[a1] = w1;
          ga = pfma<R>(w1, y0, ga);
          gb = pfma<R>(w0, y1, gb);
          if (ck) acc[I * 3 + 1] += pauli_grad<R>(ck, w0, w1, y0, y1);
        }
    }
    if (np) acc[I * 3] += (ga.x + ga.y) - (gb.x + gb.y);
    return;
  }
  {
    C m00, m01, m10, m11;
    ldc2<R>(m, m00, m01);
    ldc2<R>(m + 4, m10, m11);
    R g = 0;
    GenGrad<R> gg;
#pragma unroll
    for (int a = 0; a < (1 << RB); ++a)
      if (!(a & (1 << I))) {
        const int a1 = a | (1 << I);
        C x0 = p[a], x1 = p[a1];
        // y = M^dagger x: y0 = conj(m00) x0 + conj(m10) x1; y1 = conj(m01) x0 + conj(m11) x1
        C y0 = cfmac<R>(m10, x1, cfmac<R>(m00, x0, mk<R>(0, 0)));
        C y1 = cfmac<R>(m11, x1, cfmac<R>(m01, x0, mk<R>(0, 0)));
        p[a] = y0; p[a1] = y1;
        C u0 = l[a], u1 = l[a1];
        C w0 = cfmac<R>(m10, u1, cfmac<R>(m00, u0, mk<R>(0, 0)));
        C w1 = cfmac<R>(m11, u1, cfmac<R>(m01, u0, mk<R>(0, 0)));
        l[a] = w0; l[a1] = w1;
        if (np) {
          if (gk == 1) {
            // RX: 2 Re <l|(-i/2 X)|p> = Im(l0* p1 + l1* p0)
            g += im_cdot<R>(w0, y1) + im_cdot<R>(w1, y0);
          } else if constexpr (sizeof(R) == 4) {
            gg.add(w0, w1, y0, y1);
          } else {
            // complex128: the dense form (the packed sums' 24 extra live
            // registers spilled at four register bits)
            C a00, a01, a10, a11;
            ldc2<R>(m + 8, a00, a01);
            ldc2<R>(m + 12, a10, a11);
            C t0 = cfma<R>(a01, y1, cmul<R>(a00, y0));
            C t1 = cfma<R>(a11, y1, cmul<R>(a10, y0));
            g += 2 * (re_cdot<R>(w0, t0) + re_cdot<R>(w1, t1));
          }
        }
        if (ck) acc[I * 3 + 1] += pauli_grad<R>(ck, w0, w1, y0, y1);
      }
    if (np) acc[I * 3] += (gk == 1 || sizeof(R) != 4) ? g : gg.value(m + 8);
  }
}

// Two-qubit ops on register bits (I, I+1); 4x4 index = 2*bit(I+1) + bit(I),
// the gate's first qubit the high bit.  Every brick gate has at most two
// nonzeros per row, in columns r ^ P and r ^ Q: (P, Q) = (0, 3) for MS, CZ
// and SWAP, (1, 3) for ECR (SP = 1).  M^dagger has the same pattern, and
// A = M^dagger dM the pattern {0, P ^ Q}.  The staged records are the dense
// 4x4 matrices; only the pattern's entries are read (the others are exact
// zeros), so a gate costs 8 complex multiply-adds per 4 amplitudes, not 16.
template <int SP>
struct Pat2 {
  static constexpr int P = SP ? 1 : 0, Q = 3, D = P ^ Q;
};

// forward: y = M x
template <class R, int RB, int I, int SP>
__device__ __forceinline__ void ap2(cx<R>* v, const R* m) {
  using C = cx<R>;
  constexpr int P = Pat2<SP>::P, Q = Pat2<SP>::Q;
#pragma unroll
  for (int a = 0; a < (1 << RB); ++a)
    if (!(a & (3 << I))) {
      C x[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) x[s] = v[a | (s << I)];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        v[a | (r << I)] = cfma<R>(ldc<R>(m + 2 * (r * 4 + (r ^ Q))), x[r ^ Q],
                                  cmul<R>(ldc<R>(m + 2 * (r * 4 + (r ^ P))), x[r ^ P]));
    }
}

// backward: undo M on psi and lambda (y = M^dagger x, w = M^dagger u).  The
// only parametrised brick gate is MS (np = 3): M = c I - i s K with c, s =
// cos, sin(pi theta) and K[r][r ^ 3] = e_r (e_0 = conj(e_3) = exp(-i alpha),
// e_1 = conj(e_2) = exp(-i beta), alpha = 2 pi (phi0 + phi1), beta =
// 2 pi (phi1 - phi0)), staged after M.  Gradients 2 Re <u| dM |y> (u the
// lambda before the undo): alpha and beta enter only the entries M[r][r ^ 3],
// d/d alpha of M[0][3], M[3][0] is -i, +i times the entry (beta: M[1][2],
// M[2][1]), so with R_r = conj(u_r) M[r][r ^ 3] y[r ^ 3]
//   g_alpha = 2 Im(R_0 - R_3),  g_beta = 2 Im(R_1 - R_2),
// and d/d phi0 = 2 pi (g_alpha - g_beta), d/d phi1 = 2 pi (g_alpha + g_beta);
// K commutes with M, so M^dagger dM/d theta = -i pi K and
//   d/d theta = 2 pi Im <w| K |y>.
template <class R, int RB, int I, int SP>
__device__ __forceinline__ void bw2(cx<R>* p, cx<R>* l, const R* m, int np, R* acc) {
  using C = cx<R>;
  constexpr int P = Pat2<SP>::P, Q = Pat2<SP>::Q;
  constexpr R kTwoPi = (R)6.283185307179586;
#pragma unroll
  for (int a = 0; a < (1 << RB); ++a)
    if (!(a & (3 << I))) {
      C x[4], u[4], y[4], w[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) { x[s] = p[a | (s << I)]; u[s] = l[a | (s << I)]; }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        // (M^dagger)[r][s] = conj(M[s][r]), nonzero for s = r ^ P, r ^ Q
        const C mp = ldc<R>(m + 2 * ((r ^ P) * 4 + r)), mq = ldc<R>(m + 2 * ((r ^ Q) * 4 + r));
        y[r] = cfmac<R>(mq, x[r ^ Q], cfmac<R>(mp, x[r ^ P], mk<R>(0, 0)));
        w[r] = cfmac<R>(mq, u[r ^ Q], cfmac<R>(mp, u[r ^ P], mk<R>(0, 0)));
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) { p[a | (s << I)] = y[s]; l[a | (s << I)] = w[s]; }
      if (SP == 0 && np) {
        R imr[4], kw = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          imr[r] = im_cdot<R>(u[r], cmul<R>(ldc<R>(m + 2 * (r * 4 + (r ^ 3))), y[r ^ 3]));
          kw += im_cdot<R>(w[r], cmul<R>(ldc<R>(m + kRec2qK + 2 * r), y[r ^ 3]));
        }
        const R ga = 2 * (imr[0] - imr[3]), gb = 2 * (imr[1] - imr[2]);
        acc[I * 3 + 0] += kTwoPi * (ga - gb);
        acc[I * 3 + 1] += kTwoPi * (ga + gb);
        acc[I * 3 + 2] += kTwoPi * kw;
      }
    }
}

// Applies the round's op on register bit I (if any).  KIND is uniform over a
// pass: 0 complex single-qubit, 1 real single-qubit, 2 two-qubit on (I, I+1).
template <class R, int NS, int RB, int KIND, int I>
__device__ __forceinline__ void tile_bit(const TilePass& P, int r, cx<R>* v0, cx<R>* v1,
                                         const R* sco, R* acc) {
  if (KIND == 2 && I + 1 >= RB) return;
  const int k = P.rbit[r][I];
  if (k < 0) return;
  const TileOp& o = P.ops[k];
  const R* mc = sco + o.soff;
  constexpr int I2 = (KIND == 2 && I + 1 < RB) ? I : 0;
  if (NS == 1) {
    if (KIND == 2) {
      if (o.pat) ap2<R, RB, I2, 1>(v0, mc);
      else ap2<R, RB, I2, 0>(v0, mc);
    } else {
      ap1<R, RB, I>(v0, mc, KIND == 1);
    }
  } else {
    if (KIND == 2) {
      if (o.pat) bw2<R, RB, I2, 1>(v0, v1, mc, o.np, acc);
      else bw2<R, RB, I2, 0>(v0, v1, mc, o.np, acc);
    } else {
      bw1<R, RB, I>(v0, v1, mc, KIND == 1, o.np, o.gk, o.ck, acc);
    }
  }
}

// Tile-pass shared-memory layout: an XOR swizzle that folds index bits 4..7
// (8-byte elements: complex64 forward, 16 per 128-byte wavefront) or 3..6
// (16-byte elements: complex128, or an interleaved complex64 (psi, lambda)
// pair; 8 per wavefront) into the bank bits, with
// fold columns (15, 10, 12, 8) and (7, 5, 6, 4) packed as nibble tables.
// With these columns every round's accesses (register bits [lo, lo + RB) for
// any lo and RB <= 4), the copy loop and the paired complex64 store hit
// distinct banks; an exhaustive host-side count of wavefronts fixed them (the
// plain fold of bits 4..7 onto bits 0..3 is 2-way conflicted at lo = 3,
// RB = 3).  The map is linear over GF(2), so the address of (base | a << lo)
// is swz(base) ^ swz(a << lo), and it leaves bits >= 8 alone, so
// swz(i + k * 256) = swz(i) + k * 256.
template <int EB>
__device__ __forceinline__ int tswz(int i) {
  if constexpr (EB == 8)
    return i ^ (int)((0x1eb4d278963c5af0ull >> (4 * ((i >> 4) & 15))) & 15);
  else
    return i ^ (int)((0x0752613443162570ull >> (4 * ((i >> 3) & 15))) & 15);
}

// the same with a shared-space address (advanced by the caller)
template <int BYTES>
__device__ __forceinline__ void cp_async_sa(unsigned sa, const void* gmem) {
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Bulk prefetch of a global segment into L2 (address 16-byte aligned, size a
// multiple of 16); no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Persistent tile pass.  CTA (b, r) of the cps CTAs of sample b handles tiles
// f = r, r + cps, ... of that sample through a ring of P.nstage shared-memory
// buffers: the next nstage - 1 tiles are in flight while one is processed.
// NS = 1: forward (apply M to psi).  NS = 2: backward (undo M on psi and
// lambda, accumulate gradient partials into part[slot][block]).
// Forward diagonal phase multiplied into a tile (pre: after the load, post:
// at the store).  Thread tid handles the elements i = tid + 256 k; with
// off() the tile's element-to-index map (linear over GF(2)) and z linear,
// z(base | off(i)) = z0 ^ zK(k), z0 = z(base | off(tid)), zK(k) = z(off(256 k)).
// zK touches a few "element" bits SE, so phase(z) = phase(z0 without SE) *
// ratio[pattern of z on SE], ratio[] the products of the per-bit phase ratios
// d_p[1] / d_p[0] (from the factored tables), set up once per CTA.
// ebit0 / KB: the element index bits are ebit0 .. ebit0 + KB - 1 of the tile's
// local index (the store loop: 8 .. t-1; a register round: lo .. lo + RB - 1).
template <class R>
__device__ void fph_setup(unsigned char* blk, const R* tabs, int tb, int zm, int n, int t, int c,
                          int h0, int ebit0 = 8, int KB = -1) {
  FwdPhaseMeta* M = reinterpret_cast<FwdPhaseMeta*>(blk);
  cx<R>* ratio = reinterpret_cast<cx<R>*>(blk + ((sizeof(FwdPhaseMeta) + 15) & ~(size_t)15));
  if (KB < 0) KB = t > 8 ? t - 8 : 0;
  if (threadIdx.x == 0) {
    const int cm = (1 << c) - 1;
    auto eoff = [&](int i) { return (i & cm) | ((i >> c) << h0); };
    int zk[4] = {0, 0, 0, 0}, se = 0;
    M->ok = KB <= 4;
    if (M->ok) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < KB) {
          zk[j] = ztrans32(eoff(1 << (ebit0 + j)), n, zm);
          se |= zk[j];
        }
      M->ok = __popc(se) <= kFphMaxSE;
    }
    if (M->ok) {
      int nse = 0;
      for (int p = 0; p < n; ++p)
        if ((se >> p) & 1) M->sepos[nse++] = p;
      M->nse = nse;
      M->semask = se;
      for (int k = 0; k < (1 << KB); ++k) {
        int z = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < KB && ((k >> j) & 1)) z ^= zk[j];
        int pat = 0;
        for (int j = 0; j < nse; ++j)
          if ((z >> M->sepos[j]) & 1) pat |= 1 << j;
        M->patk[k] = pat;
      }
    }
  }
  __syncthreads();
  if (!M->ok) return;
  const int nse = M->nse;
  for (int e = threadIdx.x; e < (1 << nse); e += kThreads) {
    cx<R> v = mk<R>(1, 0);
    for (int j = 0; j < nse; ++j) {
      if (!((e >> j) & 1)) continue;
      const int p = M->sepos[j];
      const int sblk = p / tb, i = p % tb;
      const R* tt = tabs + 2LL * sblk * (1LL << tb);
      v = cmul<R>(v, cmulc<R>(ldc<R>(tt), ldc<R>(tt + 2 * (1 << i))));  // T[1 << i] conj(T[0])
    }
    ratio[e] = v;
  }
}
// per (thread, tile): the base phase and the element-bit pattern of z0
template <class R>
__device__ __forceinline__ void fph_tile(const unsigned char* blk, const R* tabs, int tb, int z0,
                                         cx<R>& p0, int& z0se) {
  const FwdPhaseMeta* M = reinterpret_cast<const FwdPhaseMeta*>(blk);
  z0se = 0;
  for (int j = 0; j < M->nse; ++j) z0se |= ((z0 >> M->sepos[j]) & 1) << j;
  p0 = diag_phase32<R>(tabs, tb, z0 & ~M->semask);
}
template <class R>
__device__ __forceinline__ cx<R> fph_elem(const unsigned char* blk, cx<R> p0, int z0se, int k) {
  const FwdPhaseMeta* M = reinterpret_cast<const FwdPhaseMeta*>(blk);
  const cx<R>* ratio = reinterpret_cast<const cx<R>*>(blk + ((sizeof(FwdPhaseMeta) + 15) & ~(size_t)15));
  return cmul<R>(p0, ratio[z0se ^ M->patk[k]]);
}

// PRE, backward: 1 / 2 undo a diagonal layer (identity / ring z map) in a
// sweep before the rounds (P.pre).  PRE, forward: 1 multiplies a following
// diagonal's phase in the last round with table-driven element patterns, 2 / 3
// the same on a contiguous 2^12 pass with compile-time patterns (ring /
// identity z map).
constexpr int tile_minb(int rsize, int ns, int kind, int pre) {
  return (rsize == 4 && kind == 1 && ns == 1) ? QC_REAL_MINB
         : (ns == 2 && pre > 0) ? QC_PRE_MINB
         : (ns == 2 ? QC_BWD_MINB : QC_FWD_MINB);
}
template <class R, int NS, int RB, int KIND, int PRE>
__global__ void __launch_bounds__(kThreads, tile_minb(sizeof(R), NS, KIND, PRE)) k_tile(const __grid_constant__ TilePass P,
                                                      const R* __restrict__ coef,
                                                      const cx<R>* src0, cx<R>* dst0,
                                                      const cx<R>* src1, cx<R>* dst1,
                                                      double* __restrict__ part, int cps) {
  using C = cx<R>;
  // complex64 backward: psi and lambda of one index side by side (one 16-byte
  // element), so a round moves both with one 16-byte shared access
  constexpr bool IL = NS == 2 && sizeof(R) == 4;
  constexpr int EB = (IL || sizeof(C) == 16) ? 16 : 8;  // shared-memory element bytes
  extern __shared__ __align__(16) unsigned char smraw[];
  const int t = P.t, n = P.n, c = P.c, h0 = P.h0;
  const int T = 1 << t;
  const int nst = P.nstage;
  const TileSmem lay = tile_smem_layout(P, NS, (int)sizeof(R));
  C* buf = reinterpret_cast<C*>(smraw + lay.buf);        // [nst][NS][T], or [nst][T][2] interleaved
  R* sco = reinterpret_cast<R*>(smraw + lay.sco);
  double* sred = reinterpret_cast<double*>(smraw + lay.sred);  // [kWarps][nslots]
  R* sdef = reinterpret_cast<R*>(smraw + lay.sdef);            // [ncomp][kThreads]
  // backward pre-diagonal: [kWarps][n + 1] marginal sums, then the phase
  // ratio table over the element-varying z bits
  double* smarg = reinterpret_cast<double*>(smraw + lay.smarg);
  // forward pre / post phase blocks
  unsigned char* fph_pre = smraw + lay.fph;
  unsigned char* fph_post = smraw + lay.fph + (P.pre ? kFphBytes((int)sizeof(R)) : 0);

  const long long tps = 1LL << (n - t);
  const int b = blockIdx.x / cps;
  const int r0 = blockIdx.x % cps;
  const int m = t - c, gap = h0 - c;
  const int cmask = (1 << c) - 1;
  const long long sb = (long long)b << n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sw_tid = tswz<EB>(threadIdx.x), sw_tid2 = tswz<EB>(2 * threadIdx.x);

  for (int k = 0; k < P.nops; ++k) {
    const TileOp& o = P.ops[k];
    const R* s = coef + o.coef + (long long)b * o.bstride;
    for (int i = threadIdx.x; i < o.nco; i += kThreads) sco[o.soff + i] = s[i];
  }
  if (NS == 2) {
    for (int i = threadIdx.x; i < kWarps * P.nslots; i += kThreads) sred[i] = 0;
    for (int s = 0, nd = tile_defer_slots(P); s < nd; ++s) sdef[s * kThreads + threadIdx.x] = 0;
  }

  constexpr int kAR = RB == 4 ? 3 : 4;  // deferred rounds (the planner matches)
  R acct[kAR][4];
#pragma unroll
  for (int r = 0; r < kAR; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) acct[r][i] = 0;

  // Backward pre-diagonal (PRE = 1 identity, 2 ring z map): before round 0 a
  // sweep over the tile undoes a diagonal layer D on psi and lambda and sums
  // the bit marginals of w = Im(conj(lambda) psi), which D leaves unchanged.
  // The pass is contiguous (c = t), thread tid holds elements i = tid + 256 k,
  // and z is linear over GF(2): z(base | i) = z0 ^ zK(k), z0 = z(base | tid).
  // The phase comes from the forward helper (base phase x per-bit ratios).
  // Marginals: the element bits SE (those zK touches) add each element's
  // exact bit; bits that vary with both the tile and the lane (the ring map's
  // n-1) are summed per thread and tile; tile-only bits are warp-uniform and
  // lane p keeps bit p after one warp sum per tile; every other bit follows
  // from the thread's total W at the end.  Running sums sit in this thread's
  // shared-memory columns: [0] W, [1 .. 8] SE bits, [9 .. 10] tile-and-lane
  // bits, [11] the lane's tile-only bit.
  constexpr bool pre_b = NS == 2 && PRE >= 1;
  constexpr int zmc = PRE == 2 ? Z_RINGXOR : Z_IDENT;
  const R* ptabs = coef + P.pre_coef + (long long)b * P.pre_bstride;
  unsigned char* fph_bpre = smraw + lay.fph;
  R* macc = reinterpret_cast<R*>(smraw + lay.smacc) + threadIdx.x;
  int zT = 0, fmask = 0, flmask = 0, flpos0 = -1, flpos1 = -1;
  bool lane_f = false;
  if (pre_b) {
    fph_setup<R>(fph_bpre, ptabs, P.pre_tb, zmc, n, t, c, h0);
    zT = ztrans32(threadIdx.x, n, zmc);
    int lmask = 0;
    for (int q = t; q < n; ++q) fmask |= ztrans32(1 << q, n, zmc);
    for (int q = 0; q < 5; ++q) lmask |= ztrans32(1 << q, n, zmc);
    const int sem = reinterpret_cast<const FwdPhaseMeta*>(fph_bpre)->semask;
    flmask = fmask & lmask & ~sem;  // one bit (n-1) for the ring map, none for the identity
    for (int p = 0; p < n; ++p)
      if ((flmask >> p) & 1) {
        if (flpos0 < 0) flpos0 = p;
        else flpos1 = p;
      }
    lane_f = (((fmask & ~lmask & ~sem) >> lane) & 1) != 0;
    for (int j = 0; j < kPreAcc; ++j) macc[j * kThreads] = 0;
  }

  const R* fpre_tabs = coef + P.pre_coef + (long long)b * P.pre_bstride;
  const R* fpost_tabs = coef + P.post_coef + (long long)b * P.post_bstride;
  if (NS == 1 && P.pre) fph_setup<R>(fph_pre, fpre_tabs, P.pre_tb, P.pre_zmode, n, t, c, h0);
  // the post phase is applied in the last round, on its RB register bits
  const int rlast = P.nrounds - 1;
  if (NS == 1 && P.post) {
    if (PRE >= 1) fph_setup<R>(fph_post, fpost_tabs, P.post_tb, P.post_zmode, n, t, c, h0, P.rlo[rlast], RB);
    else fph_setup<R>(fph_post, fpost_tabs, P.post_tb, P.post_zmode, n, t, c, h0);
  }
  const bool fpre_ok = NS == 1 && P.pre && reinterpret_cast<const FwdPhaseMeta*>(fph_pre)->ok;
  // forward: the PRE >= 1 variants multiply the post phase in the last round
  // (PRE = 2 / 3: ring / identity z map on a contiguous 2^12 pass whose last
  // round holds bits 8 .. 11, with compile-time element patterns)
  const bool fpost_ok = NS == 1 && PRE >= 1 && P.post && reinterpret_cast<const FwdPhaseMeta*>(fph_post)->ok;
  // The last round stores straight to global memory when it holds local bits
  // 8 .. 11 of a 2^12 tile: thread g has the local indices g | a << 8, at
  // global base | off(g) | a << dshift (dshift = 8 for a contiguous pass, 8 -
  // c + h0 when c <= 8), and the lanes of a warp cover the contiguous low bits
  // (c >= 5), so each a is 32 consecutive amplitudes.  The shared-memory
  // write of that round and the store loop are skipped.
  const int dshift = c >= t ? 8 : (c <= 8 ? 8 - c + h0 : -1);
  const bool dstore = RB == 4 && P.store && !P.scatter && t == 12 && c >= 5 && dshift >= 0 &&
                      P.nrounds >= 1 && P.rlo[P.nrounds - 1] == 8 && !(NS == 1 && P.post && !fpost_ok);

  // Offsets inside one sample (< 2^30) stay 32-bit; the sample base is in the
  // pointers.  Tile bits [c, h0) and [h0 + m, n) are disjoint from element
  // bits [0, c) and [h0, h0 + m).
  const C* s0b = src0 + sb;
  const C* s1b = NS == 2 ? src1 + sb : nullptr;
  C* d0b = dst0 + sb;
  C* d1b = NS == 2 ? dst1 + sb : nullptr;
  auto tile_base = [&](long long f) -> int {
    return (int)(((f & ((1LL << gap) - 1)) << c) | ((f >> gap) << (h0 + m)));
  };
  auto elem_off = [&](int i) -> int { return (i & cmask) | ((i >> c) << h0); };
  // elem_off(i0 + k * step) = elem_off(i0) + k * lin_step(step) when the step
  // keeps clear of the split between the contiguous and the high bits (c >= t,
  // or step a multiple of 2^c); -1 otherwise.  The loops below then advance
  // the offset by one add per element instead of re-deriving it.
  auto lin_step = [&](int step) -> int {
    if (c >= t) return step;
    return (step & cmask) == 0 ? ((step >> c) << h0) : -1;
  };
  const int ds_half = lin_step(kThreads / 2), ds_full = lin_step(kThreads),
            ds_pair = lin_step(2 * kThreads);
  // interleaved copies: each run of 16 threads moves psi then lambda of 8
  // consecutive indices (16 distinct bank pairs in shared memory, two 64-byte
  // segments in global memory)
  const int il_i = ((threadIdx.x >> 4) << 3) | (threadIdx.x & 7);
  const int il_s = (threadIdx.x >> 3) & 1;
  const C* il_src = il_s ? s1b : s0b;
  const int il_si = 2 * tswz<EB>(il_i) + il_s;
  auto issue = [&](long long f, int slot) {
    const int base = tile_base(f);
    C* d0 = buf + slot * NS * T;
    if constexpr (IL) {
      if (ds_half >= 0 && !P.gather) {
        // one pointer and one shared-space address, each advanced by a constant
        const C* gp = il_src + (base | elem_off(il_i));
        unsigned sa = (unsigned)__cvta_generic_to_shared(&d0[il_si]);
#pragma unroll 4
        for (int i = il_i; i < T; i += kThreads / 2, sa += kThreads * sizeof(C), gp += ds_half)
          cp_async_sa<sizeof(C)>(sa, gp);
      } else if (ds_half >= 0) {
        int gi = base | elem_off(il_i);
#pragma unroll 4
        for (int i = il_i, si = il_si; i < T; i += kThreads / 2, si += kThreads, gi += ds_half)
          cp_async_elem<sizeof(C)>(&d0[si], &il_src[ring_finv32(gi, n)]);
      } else {
        for (int i = il_i, si = il_si; i < T; i += kThreads / 2, si += kThreads) {
          int gi = base | elem_off(i);
          if (P.gather) gi = ring_finv32(gi, n);
          cp_async_elem<sizeof(C)>(&d0[si], &il_src[gi]);
        }
      }
    } else if (ds_full >= 0 && !P.gather) {
      const int g0 = base | elem_off(threadIdx.x);
      const C* gp0 = s0b + g0;
      const C* gp1 = NS == 2 ? s1b + g0 : nullptr;
      unsigned sa = (unsigned)__cvta_generic_to_shared(&d0[sw_tid]);
      for (int i = threadIdx.x; i < T; i += kThreads, sa += kThreads * sizeof(C), gp0 += ds_full) {
        cp_async_sa<sizeof(C)>(sa, gp0);
        if (NS == 2) {
          cp_async_sa<sizeof(C)>(sa + T * sizeof(C), gp1);
          gp1 += ds_full;
        }
      }
    } else if (ds_full >= 0) {
      int gi = base | elem_off(threadIdx.x);
      for (int i = threadIdx.x, si = sw_tid; i < T; i += kThreads, si += kThreads, gi += ds_full) {
        const int g2 = ring_finv32(gi, n);
        cp_async_elem<sizeof(C)>(&d0[si], &s0b[g2]);
        if (NS == 2) cp_async_elem<sizeof(C)>(&d0[T + si], &s1b[g2]);
      }
    } else {
      for (int i = threadIdx.x, si = sw_tid; i < T; i += kThreads, si += kThreads) {
        int gi = base | elem_off(i);
        if (P.gather) gi = ring_finv32(gi, n);
        cp_async_elem<sizeof(C)>(&d0[si], &s0b[gi]);
        if (NS == 2) cp_async_elem<sizeof(C)>(&d0[T + si], &s1b[gi]);
      }
    }
  };

  // Backward, one buffer and a direct-store last round: the next tile's copy
  // starts as soon as every thread holds its last-round elements (the buffer
  // is free then), so it overlaps that round's gates and stores.
  const bool early = NS == 2 && nst == 1 && dstore;
  long long f = r0;
  int slot = 0;
  for (int j = 0; j + 1 < nst; ++j) {
    if (f + (long long)j * cps < tps) issue(f + (long long)j * cps, j);
    cp_async_commit();
  }
  for (; f < tps; f += cps) {
    // every iteration commits one group (possibly empty), so the group of
    // tile f is complete once at most nst - 1 newer groups are pending
    const long long fn = f + (long long)(nst - 1) * cps;
    const int sn = slot + nst - 1 < nst ? slot + nst - 1 : slot - 1;
    if (fn < tps && !(early && f != r0)) issue(fn, sn);  // early: already in flight
    cp_async_commit();
    if (nst == 3) cp_async_wait_group<2>();
    else if (nst == 2) cp_async_wait_group<1>();
    else cp_async_wait_group<0>();  // one buffer: the tile just issued
    // one buffer: while this tile is processed, pull the next one into L2 so
    // its copies do not wait on DRAM (one bulk prefetch per contiguous
    // segment of 2^c amplitudes and state; not for gathered loads)
    if (nst == 1 && !P.gather && f + cps < tps) {
      const int nb = tile_base(f + cps);
      const int nseg = 1 << m;                      // rows of the tile
      const unsigned bytes = (unsigned)(sizeof(C) << c);
      for (int j = threadIdx.x; j < nseg * NS; j += kThreads) {
        const int row = j & (nseg - 1), st = j >> m;
        const int off = nb | (row << h0);
        prefetch_l2((st ? s1b : s0b) + off, bytes);
      }
    }
    __syncthreads();
    C* S0 = buf + (long long)slot * NS * T;
    C* S1 = S0 + T;
    if (NS == 1 && P.pre) {
      const int base = tile_base(f);
      if (fpre_ok) {
        if (threadIdx.x < T) {
          C p0;
          int z0se;
          fph_tile<R>(fph_pre, fpre_tabs, P.pre_tb, ztrans32(base | elem_off(threadIdx.x), n, P.pre_zmode),
                      p0, z0se);
          for (int i = threadIdx.x, pi = sw_tid, k = 0; i < T; i += kThreads, pi += kThreads, ++k)
            S0[pi] = cmul<R>(fph_elem<R>(fph_pre, p0, z0se, k), S0[pi]);
        }
      } else {
        for (int i = threadIdx.x, pi = sw_tid; i < T; i += kThreads, pi += kThreads) {
          const int k = base | elem_off(i);
          S0[pi] = cmul<R>(diag_phase32<R>(fpre_tabs, P.pre_tb, ztrans32(k, n, P.pre_zmode)), S0[pi]);
        }
      }
      __syncthreads();
    }
    if (pre_b) {
      const int base = tile_base(f);
      const FwdPhaseMeta* pm = reinterpret_cast<const FwdPhaseMeta*>(fph_bpre);
      const int nse = pm->nse;
      const int z0 = ztrans32(base | threadIdx.x, n, zmc);  // c = t: elem_off(i) = i
      // Contiguous pass: element k is index bits 8 .. t-1, so the element z
      // bits are 7 .. t-1 (ring: z_p = k_p ^ k_{p+1}) or 8 .. t-1 (identity)
      // and the pattern of element k is k ^ (k << 1) or k -- compile-time
      // constants in the unrolled loop below (the per-CTA table's bit order).
      constexpr int zlo = PRE == 2 ? 7 : 8;
      const int z0se = (z0 >> zlo) & ((1 << nse) - 1);  // nse = t - 7 (ring) or t - 8
      const C p0 = diag_phase32<R>(ptabs, P.pre_tb, z0 & ~pm->semask);
      const C* ratio = reinterpret_cast<const C*>(fph_bpre + ((sizeof(FwdPhaseMeta) + 15) & ~(size_t)15));
      R Wt = 0, Ase[5] = {0, 0, 0, 0, 0};
      auto load = [&](int si, C& x, C& l) {
        if constexpr (IL) {
          const float4 q = *reinterpret_cast<const float4*>(&S0[2 * si]);
          x = mk<R>(q.x, q.y);
          l = mk<R>(q.z, q.w);
        } else {
          x = S0[si];
          l = S1[si];
        }
      };
      auto store = [&](int si, C y, C u) {
        if constexpr (IL) {
          *reinterpret_cast<float4*>(&S0[2 * si]) = make_float4(y.x, y.y, u.x, u.y);
        } else {
          S0[si] = y;
          S1[si] = u;
        }
      };
      const int ne = T >> 8;  // 2 .. 16 elements per thread
#pragma unroll
      for (int k = 0; k < 16; k += 2) {
        if (k < ne) {
          const int si = sw_tid + k * kThreads;  // the swizzle only folds bits below 8
          C x0, l0, x1, l1;
          load(si, x0, l0);
          load(si + kThreads, x1, l1);
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int kk = k + e;
            const int pat = PRE == 2 ? (kk ^ (kk << 1)) : kk;
            const C ph = cmul<R>(p0, ratio[z0se ^ pat]);
            const C y = cmulc<R>(ph, e ? x1 : x0), u = cmulc<R>(ph, e ? l1 : l0);
            store(si + e * kThreads, y, u);
            const R w = im_cdot<R>(u, y);
            Wt += w;
            // the element bit j of z is z0se_j ^ pat_j: sum w where pat_j is
            // set, and fold z0se in when the tile is done
#pragma unroll
            for (int j = 0; j < 5; ++j)
              if ((pat >> j) & 1) Ase[j] += w;
          }
        }
      }
      // Ase[j] so far sums w over pat_j = 1; z_j = z0se_j ^ pat_j
#pragma unroll
      for (int j = 0; j < 5; ++j)
        if ((z0se >> j) & 1) Ase[j] = Wt - Ase[j];
      if (P.pre_grad) {
        macc[0] += Wt;
#pragma unroll
        for (int j = 0; j < 5; ++j)
          if (j < nse) macc[(1 + j) * kThreads] += Ase[j];
        if (flpos0 >= 0 && ((z0 >> flpos0) & 1)) macc[9 * kThreads] += Wt;
        if (flpos1 >= 0 && ((z0 >> flpos1) & 1)) macc[10 * kThreads] += Wt;
        const R sw = warp_sum_r<R>(Wt);
        if (lane_f && ((z0 >> lane) & 1)) macc[11 * kThreads] += sw;
      }
      __syncthreads();
    }

#pragma unroll 1
    for (int r = 0; r < P.nrounds; ++r) {
      const int lo = P.rlo[r];
      R acc[RB * 3];
#pragma unroll
      for (int i = 0; i < RB * 3; ++i) acc[i] = 0;
      // address of register element a = pb ^ (XOR of basis[j] over set bits j of a)
      int basis[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) basis[j] = tswz<EB>(1 << (lo + j));
      for (int g = threadIdx.x; g < (T >> RB); g += kThreads) {
        const int pb = tswz<EB>((g & ((1 << lo) - 1)) | ((g >> lo) << (lo + RB)));
        C v0[1 << RB], v1[NS == 2 ? (1 << RB) : 1];
#pragma unroll
        for (int a = 0; a < (1 << RB); ++a) {
          int ad = pb;
#pragma unroll
          for (int j = 0; j < RB; ++j)
            if (a & (1 << j)) ad ^= basis[j];
          if constexpr (IL) {
            const float4 q = *reinterpret_cast<const float4*>(&S0[2 * ad]);
            v0[a] = mk<R>(q.x, q.y);
            v1[a] = mk<R>(q.z, q.w);
          } else {
            v0[a] = S0[ad];
            if (NS == 2) v1[a] = S1[ad];
          }
        }
        if constexpr (NS == 2) {
          if (early && r == rlast) {
            // every thread holds its elements of this round (one group each):
            // the buffer is free for the next tile
            __syncthreads();
            if (f + cps < tps) issue(f + cps, 0);
            cp_async_commit();
          }
        }
        tile_bit<R, NS, RB, KIND, 0>(P, r, v0, v1, sco, acc);
        if (RB > 1) tile_bit<R, NS, RB, KIND, (RB > 1 ? 1 : 0)>(P, r, v0, v1, sco, acc);
        if (RB > 2) tile_bit<R, NS, RB, KIND, (RB > 2 ? 2 : 0)>(P, r, v0, v1, sco, acc);
        if (RB > 3) tile_bit<R, NS, RB, KIND, (RB > 3 ? 3 : 0)>(P, r, v0, v1, sco, acc);
        if (NS == 1 && PRE == 1 && fpost_ok && r == rlast) {
          // the layer's gates are all applied to these elements: multiply in
          // the following diagonal layer's phase (element a = local index
          // bits lo .. lo + RB - 1 of this group)
          const int lidx = (g & ((1 << lo) - 1)) | ((g >> lo) << (lo + RB));
          C p0;
          int z0se;
          fph_tile<R>(fph_post, fpost_tabs, P.post_tb,
                      ztrans32(tile_base(f) | elem_off(lidx), n, P.post_zmode), p0, z0se);
#pragma unroll
          for (int a = 0; a < (1 << RB); ++a) v0[a] = cmul<R>(fph_elem<R>(fph_post, p0, z0se, a), v0[a]);
        } else if (NS == 1 && PRE >= 2 && fpost_ok && r == rlast) {
          // group g = tid holds local indices g | a << 8 (c = t = 12, lo = 8):
          // z = z0 ^ z(a << 8), and z(a << 8) covers z bits zlo .. 11 with the
          // compile-time pattern a ^ (a << 1) (ring) or a (identity); the
          // per-CTA ratio table is indexed in that bit order
          constexpr int zlo = PRE == 2 ? 7 : 8, nse = 12 - zlo;
          constexpr int semask = ((1 << nse) - 1) << zlo;
          const int z0 = ztrans32(tile_base(f) | g, n, PRE == 2 ? Z_RINGXOR : Z_IDENT);
          const int z0se = (z0 >> zlo) & ((1 << nse) - 1);
          const C p0 = diag_phase32<R>(fpost_tabs, P.post_tb, z0 & ~semask);
          const C* ratio = reinterpret_cast<const C*>(fph_post + ((sizeof(FwdPhaseMeta) + 15) & ~(size_t)15));
#pragma unroll
          for (int a = 0; a < (1 << RB); ++a) {
            const int pat = PRE == 2 ? (a ^ (a << 1)) : a;
            v0[a] = cmul<R>(cmul<R>(p0, ratio[z0se ^ pat]), v0[a]);
          }
        }
        if (dstore && r == rlast) {
          const int gb = tile_base(f) | elem_off(g);
          C* o0 = d0b + gb;
          C* o1 = NS == 2 ? d1b + gb : nullptr;
          if (c >= t) {  // contiguous: compile-time offsets a << 8
#pragma unroll
            for (int a = 0; a < (1 << RB); ++a) {
              o0[a << 8] = v0[a];
              if constexpr (NS == 2) o1[a << 8] = v1[a];
            }
          } else {
#pragma unroll
            for (int a = 0; a < (1 << RB); ++a) {
              o0[a << dshift] = v0[a];
              if constexpr (NS == 2) o1[a << dshift] = v1[a];
            }
          }
        } else {
#pragma unroll
          for (int a = 0; a < (1 << RB); ++a) {
            int ad = pb;
#pragma unroll
            for (int j = 0; j < RB; ++j)
              if (a & (1 << j)) ad ^= basis[j];
            if constexpr (IL) {
              *reinterpret_cast<float4*>(&S0[2 * ad]) = make_float4(v0[a].x, v0[a].y, v1[a].x, v1[a].y);
            } else {
              S0[ad] = v0[a];
              if (NS == 2) S1[ad] = v1[a];
            }
          }
        }
      }
      if (NS == 2) {
        if (P.defer == 1) {
          // keep per-thread sums across tiles, reduced once after the last
          // tile: the pass's own slots in registers, companion slots in this
          // thread's column of shared memory
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
          // per op of the round, by its (lower) register bit: every acc index
          // is a compile-time constant, so acc stays in registers
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

    if (P.store && !dstore) {
      const int base = tile_base(f);
      if (IL && P.scatter) {
        // backward scatter through the CNOT ring's inverse map f^-1, in
        // 16-byte pairs: f^-1(k ^ 1 ^ 2^(n-1)) = f^-1(k) ^ 1, and this top
        // pass holds both index bit 0 (local 0) and bit n-1 (local t-1), so
        // the thread takes local i < T/2 with its partner i ^ 1 ^ T/2
        for (int i = threadIdx.x, si = sw_tid; i < (T >> 1); i += kThreads, si += kThreads) {
          const int d = ring_finv32(base | elem_off(i), n);
          const int sp = tswz<EB>(i ^ 1 ^ (T >> 1));
          const float4 qa = *reinterpret_cast<const float4*>(&S0[2 * si]);
          const float4 qb = *reinterpret_cast<const float4*>(&S0[2 * sp]);
          const bool odd = d & 1;
          const int dd = d & ~1;
          *reinterpret_cast<float4*>(&d0b[dd]) =
              odd ? make_float4(qb.x, qb.y, qa.x, qa.y) : make_float4(qa.x, qa.y, qb.x, qb.y);
          *reinterpret_cast<float4*>(&d1b[dd]) =
              odd ? make_float4(qb.z, qb.w, qa.z, qa.w) : make_float4(qa.z, qa.w, qb.z, qb.w);
        }
      } else if ((NS == 1 && P.post && !(PRE >= 1 && fpost_ok)) || P.scatter) {
        // forward post not applied in the round: the store-loop decomposition
        const bool loop_ok = NS == 1 && P.post && PRE == 0 &&
                             reinterpret_cast<const FwdPhaseMeta*>(fph_post)->ok;
        C p0 = mk<R>(1, 0);
        int z0se = 0;
        if (loop_ok && threadIdx.x < T)
          fph_tile<R>(fph_post, fpost_tabs, P.post_tb, ztrans32(base | elem_off(threadIdx.x), n, P.post_zmode),
                      p0, z0se);
        for (int i = threadIdx.x, pi = sw_tid, k = 0; i < T; i += kThreads, pi += kThreads, ++k) {
          const int kl = base | elem_off(i);
          C e = S0[pi];
          if (NS == 1 && P.post)
            e = cmul<R>(loop_ok ? fph_elem<R>(fph_post, p0, z0se, k)
                                : diag_phase32<R>(fpost_tabs, P.post_tb, ztrans32(kl, n, P.post_zmode)),
                        e);
          const int gd = P.scatter ? ring_finv32(kl, n) : kl;
          if constexpr (IL) {
            d0b[gd] = S0[2 * pi];
            d1b[gd] = S0[2 * pi + 1];
          } else {
            d0b[gd] = e;
            if (NS == 2) d1b[gd] = S1[pi];
          }
        }
      } else if (NS == 1 && sizeof(C) == 8 && ds_pair >= 0) {
        // forward paired 16-byte stores, i = 2 tid + k * 2 kThreads, with the
        // global and shared-memory pointers advanced by constants: the swizzle
        // leaves bits >= 8 alone, so the partner pi ^ 1 sits at a fixed
        // distance dp = +-1 from pi (the backward keeps the indexed loop below,
        // measured faster there)
        C* q0p = d0b + (base | elem_off(2 * threadIdx.x));
        const int dp = (sw_tid2 ^ 1) - sw_tid2;
        const C* sp = S0 + sw_tid2;
#pragma unroll 2
        for (int i = 2 * threadIdx.x; i < T; i += 2 * kThreads, sp += 2 * kThreads, q0p += ds_pair) {
          const C e0 = sp[0], e1 = sp[dp];
          *reinterpret_cast<float4*>(q0p) = make_float4(e0.x, e0.y, e1.x, e1.y);
        }
      } else if (sizeof(C) == 8) {
        // paired 16-byte stores: i = 2 tid + k * 2 kThreads (c >= 1 here, so the
        // pair never straddles the contiguous segment)
        int gi_step = base | elem_off(2 * threadIdx.x);
#pragma unroll 2
        for (int i = 2 * threadIdx.x, pi = sw_tid2; i < T;
             i += 2 * kThreads, pi += 2 * kThreads, gi_step += (ds_pair >= 0 ? ds_pair : 0)) {
          const int gi = ds_pair >= 0 ? gi_step : (base | elem_off(i));
          if constexpr (IL) {
            const float4 q0 = *reinterpret_cast<const float4*>(&S0[2 * pi]);
            const float4 q1 = *reinterpret_cast<const float4*>(&S0[2 * (pi ^ 1)]);
            *reinterpret_cast<float4*>(&d0b[gi]) = make_float4(q0.x, q0.y, q1.x, q1.y);
            *reinterpret_cast<float4*>(&d1b[gi]) = make_float4(q0.z, q0.w, q1.z, q1.w);
          } else {
            C e0 = S0[pi], e1 = S0[pi ^ 1];
            *reinterpret_cast<float4*>(&d0b[gi]) = make_float4(e0.x, e0.y, e1.x, e1.y);
            if (NS == 2) {
              C u0 = S1[pi], u1 = S1[pi ^ 1];
              *reinterpret_cast<float4*>(&d1b[gi]) = make_float4(u0.x, u0.y, u1.x, u1.y);
            }
          }
        }
      } else {
        int gi_step = base | elem_off(threadIdx.x);
        for (int i = threadIdx.x, pi = sw_tid; i < T;
             i += kThreads, pi += kThreads, gi_step += (ds_full >= 0 ? ds_full : 0)) {
          const int gi = ds_full >= 0 ? gi_step : (base | elem_off(i));
          d0b[gi] = S0[pi];
          if (NS == 2) d1b[gi] = S1[pi];
        }
      }
    }
    __syncthreads();
    slot = slot + 1 == nst ? 0 : slot + 1;
  }
  cp_async_wait_group<0>();
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
      const FwdPhaseMeta* pm = reinterpret_cast<const FwdPhaseMeta*>(fph_bpre);
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
            else if (p == flpos0) u = macc[9 * kThreads];
            else if (p == flpos1) u = macc[10 * kThreads];
            else if ((fmask >> p) & 1) u = 0;
            else u = ((zT >> p) & 1) ? mW : (R)0;
            return lane == p ? u + mF : u;
          },
          [&](int v, double sum) { part[P.pre_moff + (long long)v * nblk + blockIdx.x] = sum; });
    }
  }
}

template <class R, int NS, int RB, int KIND, int PRE>
static cudaError_t launch_tile_k(const TilePass& P, int batch, int cps, const void* coef,
                                 const void* s0, void* d0, const void* s1, void* d1, double* part,
                                 cudaStream_t st) {
  size_t smem = tile_smem_bytes(P, NS, sizeof(R));
  auto kern = k_tile<R, NS, RB, KIND, PRE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long long grid = (long long)batch * cps;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(P, (const R*)coef, (const cx<R>*)s0, (cx<R>*)d0,
                                               (const cx<R>*)s1, (cx<R>*)d1, part, cps);
  return cudaGetLastError();
}

template <class R, int NS, int RB>
static cudaError_t launch_tile_rb(const TilePass& P, int batch, int cps, const void* coef,
                                  const void* s0, void* d0, const void* s1, void* d1, double* part,
                                  cudaStream_t st) {
  // forward: passes with a post phase and single-qubit gates at RB = 3 or 4
  // run the variant that applies it in the last round
  if constexpr (NS == 1 && (RB == 3 || RB == 4)) {
    if (P.post && P.kind != 2) {
      if constexpr (RB == 4 && sizeof(R) == 4) {
        // contiguous 2^12 pass whose last round holds bits 8 .. 11
        if (fwd_post_contig(P)) {
          const bool ring = P.post_zmode == Z_RINGXOR;
          if (P.kind == 1)
            return ring ? launch_tile_k<R, NS, RB, 1, 2>(P, batch, cps, coef, s0, d0, s1, d1, part, st)
                        : launch_tile_k<R, NS, RB, 1, 3>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
          return ring ? launch_tile_k<R, NS, RB, 0, 2>(P, batch, cps, coef, s0, d0, s1, d1, part, st)
                      : launch_tile_k<R, NS, RB, 0, 3>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
        }
      }
      if (P.kind == 1) return launch_tile_k<R, NS, RB, 1, 1>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
      return launch_tile_k<R, NS, RB, 0, 1>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
    }
  }
  // the pre-diagonal variant exists for backward single-qubit passes with
  // RB = 3 or 4 (the planner only fuses those)
  // (a forward pass's P.pre is the plain phase multiply inside PRE = 0)
  constexpr bool kPre = NS == 2 && (RB == 3 || RB == 4);
  if (NS == 2 && P.pre) {
    if (!kPre || P.kind == 2) return cudaErrorInvalidValue;
    switch (P.kind) {
      case 0:
        if (P.pre_zmode == Z_RINGXOR)
          return launch_tile_k<R, NS, RB, 0, kPre ? 2 : 0>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
        return launch_tile_k<R, NS, RB, 0, kPre ? 1 : 0>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
      case 1:
        if (P.pre_zmode == Z_RINGXOR)
          return launch_tile_k<R, NS, RB, 1, kPre ? 2 : 0>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
        return launch_tile_k<R, NS, RB, 1, kPre ? 1 : 0>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (P.kind) {
    case 0: return launch_tile_k<R, NS, RB, 0, 0>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
    case 1: return launch_tile_k<R, NS, RB, 1, 0>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
    case 2: return launch_tile_k<R, NS, RB, 2, 0>(P, batch, cps, coef, s0, d0, s1, d1, part, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qc
