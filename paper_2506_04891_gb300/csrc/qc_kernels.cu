// CUDA kernels of the layered state-vector simulator (sm_103a): coefficients,
// product-state init, diagonal and complement passes, <Z>, the CNOT ring,
// reductions and the whole-circuit shared-memory kernel.  The tile passes
// live in qc_tile.cuh (instantiated by qc_tile_fwd.cu / qc_tile_bwd.cu).
//
// State: psi[b][k] interleaved complex (float2 / double2), qubit q = bit n-1-q.
// Every kernel here is bandwidth-shaped: a CTA streams a tile or a contiguous
// chunk of one sample's state through shared memory or registers once.
#include <string.h>

#include "qc_device.cuh"
#include "qc_gates.cuh"
#include "qc_kernels.h"

// QC_INST_R selects the precision this object instantiates (4: float, 8:
// double, 0: both); the build compiles the file once per precision, and the
// non-template definitions go into the float object only
#ifndef QC_INST_R
#define QC_INST_R 0
#endif

namespace qc {
// ---------------------------------------------------------------------------
// Coefficients: gate matrices, generators, diagonal phase tables
// ---------------------------------------------------------------------------

__device__ __forceinline__ double param_of(const CoefJob& J, int b, int j, const double* x,
                                           const double* theta, int n_in) {
  const int idx = J.offset + J.pstride * j;
  if (J.source == QC_SRC_THETA) return theta[idx];
  if (J.source == QC_SRC_INPUT) return x[(long long)b * n_in + idx];
  return 0.0;
}

template <class R>
__global__ void k_coef(const CoefJob* __restrict__ jobs, int njobs, int n, int batch, int n_in,
                       const double* __restrict__ x, const double* __restrict__ theta,
                       R* __restrict__ coef) {
  const CoefJob J = jobs[blockIdx.x];
  const int b = blockIdx.y;
  if (!J.per_sample && b > 0) return;
  R* out = coef + J.coef_off + (long long)b * J.bstride;
  __shared__ dc dvec[kMaxQubits][2];
  if (J.cls == LC_ROT1) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      double t = param_of(J, b, q, x, theta, n_in);
      dc M[4], D[4], A[4];
      gate1q(J.kind, t, M);
      dgate1q(J.kind, t, D);
      mdag_mul(M, D, A, 2);
      R* o = out + (long long)q * kRec1q;
      for (int i = 0; i < 4; ++i) {
        o[2 * i] = (R)M[i].x; o[2 * i + 1] = (R)M[i].y;
        o[8 + 2 * i] = (R)A[i].x; o[8 + 2 * i + 1] = (R)A[i].y;
        o[kRealOff + i] = (R)M[i].x;
      }
    }
  } else if (J.cls == LC_DENSE2) {
    for (int g = threadIdx.x; g < J.ngates; g += blockDim.x) {
      dc M[16], D[16], A[16];
      R* o = out + (long long)g * kRec2q;
      for (int i = 0; i < kRec2q; ++i) o[i] = (R)0;
      if (J.kind == QC_L_MS_BRICK) {
        double p0 = param_of(J, b, 3 * g, x, theta, n_in);
        double p1 = param_of(J, b, 3 * g + 1, x, theta, n_in);
        double th = param_of(J, b, 3 * g + 2, x, theta, n_in);
        gate_ms(p0, p1, th, M);
        const double wt = 2.0 * kPi;
        const dc e[4] = {dexpi(-wt * (p0 + p1)), dexpi(-wt * (p1 - p0)), dexpi(-wt * (p0 - p1)),
                         dexpi(wt * (p0 + p1))};
        for (int r = 0; r < 4; ++r) {
          o[kRec2qK + 2 * r] = (R)e[r].x;
          o[kRec2qK + 2 * r + 1] = (R)e[r].y;
        }
        for (int w = 0; w < 3; ++w) {
          dgate_ms(p0, p1, th, w, D);
          mdag_mul(M, D, A, 4);
          for (int i = 0; i < 16; ++i) {
            o[kRec2qA + 32 * w + 2 * i] = (R)A[i].x;
            o[kRec2qA + 32 * w + 2 * i + 1] = (R)A[i].y;
          }
        }
      } else if (J.kind == QC_L_CZ_BRICK) {
        gate_cz(M);
      } else if (J.kind == QC_L_SWAP_BRICK) {
        gate_swap(M);
      } else {
        gate_ecr(M);
      }
      for (int i = 0; i < 16; ++i) { o[2 * i] = (R)M[i].x; o[2 * i + 1] = (R)M[i].y; }
    }
  } else if (J.cls == LC_DIAG || J.cls == LC_XCOMP) {
    if (!J.has_phase) return;
    // per-bit phase pair d_p = (phase if z-bit p = 0, phase if z-bit p = 1)
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      int j;
      if (J.kind == QC_L_ISINGZZ_RING) j = ((n - 2 - p) % n + n) % n;
      else j = n - 1 - p;
      double t = param_of(J, b, j, x, theta, n_in);
      if (J.kind == QC_L_GPI) {
        dvec[p][0] = dexpi(2.0 * kPi * t);
        dvec[p][1] = dexpi(-2.0 * kPi * t);
      } else if (J.kind == QC_L_Z) {
        dvec[p][0] = dmk(1, 0);
        dvec[p][1] = dmk(-1, 0);
      } else if (J.kind == QC_L_S) {
        dvec[p][0] = dmk(1, 0);
        dvec[p][1] = dmk(0, 1);
      } else {  // RZ, IsingZZ: exp(-i t/2 * (+1 / -1))
        dvec[p][0] = dexpi(-0.5 * t);
        dvec[p][1] = dexpi(0.5 * t);
        if (J.rot_phase) {
          // RZ(phi) part of Rot(theta, phi, lambda): times e^{i (phi + lambda) / 2}
          CoefJob Jl = J;
          Jl.offset += 1;
          const dc g = dexpi(0.5 * (t + param_of(Jl, b, j, x, theta, n_in)));
          dvec[p][0] = dmul(dvec[p][0], g);
          dvec[p][1] = dmul(dvec[p][1], g);
        }
      }
    }
    __syncthreads();
    const int tb = J.tb, T = 1 << tb;
    for (int e = threadIdx.x; e < kDiagTables * T; e += blockDim.x) {
      int s = e / T, idx = e % T;
      dc v = dmk(1, 0);
      for (int i = 0; i < tb; ++i) {
        int p = s * tb + i;
        if (p >= n) break;
        v = dmul(v, dvec[p][(idx >> i) & 1]);
      }
      out[2LL * e] = (R)v.x;
      out[2LL * e + 1] = (R)v.y;
    }
  }
}

// Product state of the leading single-qubit layers: v[b][p] = M_m ... M_1 |0>
// for qubit q = n-1-p (two complex numbers per qubit).
template <class R>
__global__ void k_prodvec(ProdVecJob P, int n, int batch, int n_in, const double* __restrict__ x,
                          const double* __restrict__ theta, R* __restrict__ pv) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= batch * n) return;
  int b = idx / n, q = idx % n;
  dc v0 = dmk(1, 0), v1 = dmk(0, 0);
  for (int l = 0; l < P.nl; ++l) {
    CoefJob J;
    J.source = P.source[l];
    J.offset = P.offset[l];
    J.pstride = P.pstride[l];
    double t = param_of(J, b, q, x, theta, n_in);
    dc M[4];
    gate1q(P.kind[l], t, M);
    if (P.rot_phase[l]) {  // RZ(phi) part of a Rot: times e^{i (phi + lambda) / 2}
      J.offset += 1;
      const dc g = dexpi(0.5 * (t + param_of(J, b, q, x, theta, n_in)));
      for (int i = 0; i < 4; ++i) M[i] = dmul(M[i], g);
    }
    dc a = dadd(dmul(M[0], v0), dmul(M[1], v1));
    dc c = dadd(dmul(M[2], v0), dmul(M[3], v1));
    v0 = a; v1 = c;
  }
  int p = n - 1 - q;
  R* o = pv + ((long long)b * n + p) * 4;
  o[0] = (R)v0.x; o[1] = (R)v0.y; o[2] = (R)v1.x; o[3] = (R)v1.y;
}

// two adjacent amplitudes at an even index: one 16-byte store for complex64
template <class R>
__device__ __forceinline__ void store_pair(cx<R>* p, cx<R> a, cx<R> b) {
  if constexpr (sizeof(R) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// psi[b][k] = prod_p v[b][p][bit_p(k)], one contiguous chunk of 2^cb per CTA.
// With post_tabs != NULL the product state is multiplied by the diagonal
// phase of the following diagonal layer (tables as in k_diag).
template <class R>
__global__ void __launch_bounds__(kThreads) k_prodinit(int n, int cb, const R* __restrict__ pv,
                                                       cx<R>* __restrict__ psi,
                                                       const R* __restrict__ post_tabs,
                                                       long long post_bstride, int post_tb,
                                                       int post_zmode) {
  using C = cx<R>;
  __shared__ C Ta[64], Tb[64];
  const int nch_bits = n - cb;
  const long long blk = blockIdx.x;
  const int b = (int)(blk >> nch_bits);
  const long long chunk = blk & ((1LL << nch_bits) - 1);
  const long long base = chunk << cb;
  // the sample's per-qubit vectors, staged once: the product chains below then
  // wait on shared-memory latency instead of one global load per link
  __shared__ __align__(16) R v[kMaxQubits * 4];
  for (int i = threadIdx.x; i < n * 4; i += blockDim.x) v[i] = pv[(long long)b * n * 4 + i];
  __syncthreads();
  const int la = cb < 6 ? cb : 6, lb = cb - la;
  // constant factor of the chunk's fixed high bits
  C H = mk<R>(1, 0);
  for (int p = cb; p < n; ++p) {
    int bit = (int)((base >> p) & 1);
    H = cmul<R>(H, ldc<R>(v + p * 4 + 2 * bit));
  }
  for (int e = threadIdx.x; e < 128; e += blockDim.x) {
    if (e < 64) {
      C a = mk<R>(1, 0);
      for (int i = 0; i < la; ++i) a = cmul<R>(a, ldc<R>(v + i * 4 + 2 * ((e >> i) & 1)));
      Ta[e] = a;
    } else {
      int f = e - 64;
      C a = H;
      for (int i = 0; i < lb; ++i) a = cmul<R>(a, ldc<R>(v + (la + i) * 4 + 2 * ((f >> i) & 1)));
      Tb[f] = a;
    }
  }
  __syncthreads();
  C* out = psi + ((long long)b << n) + base;
  const int CH = 1 << cb, ma = (1 << la) - 1;
  if (post_tabs) {
    // the first phase table (low z bits, which differ across a warp) staged in
    // shared memory; the other two are nearly uniform across a warp
    extern __shared__ __align__(16) unsigned char smraw[];
    R* t0 = reinterpret_cast<R*>(smraw);
    const R* tabs = post_tabs + (long long)b * post_bstride;
    const int TT = 1 << post_tb;
    for (int i = threadIdx.x; i < 2 * TT; i += blockDim.x) t0[i] = tabs[i];
    __syncthreads();
    const long long mask = TT - 1;
    for (int i = 2 * threadIdx.x; i < CH; i += 2 * blockDim.x) {
      C e[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long z = ztrans(base + i + h, n, post_zmode);
        const C ph = cmul<R>(cmul<R>(ldc<R>(t0 + 2 * (z & mask)),
                                     ldc<R>(tabs + 2 * (TT + ((z >> post_tb) & mask)))),
                             ldc<R>(tabs + 2 * (2 * TT + ((z >> (2 * post_tb)) & mask))));
        e[h] = cmul<R>(ph, cmul<R>(Tb[(i + h) >> la], Ta[(i + h) & ma]));
      }
      store_pair<R>(out + i, e[0], e[1]);
    }
  } else {
    // pairs (i, i + 1) share Tb (n >= 1, so la >= 1)
    for (int i = 2 * threadIdx.x; i < CH; i += 2 * blockDim.x) {
      const C tb = Tb[i >> la];
      store_pair<R>(out + i, cmul<R>(tb, Ta[i & ma]), cmul<R>(tb, Ta[(i + 1) & ma]));
    }
  }
}

// ---------------------------------------------------------------------------
// Bit-marginal reduction shared by <Z>, diagonal-layer gradients
// ---------------------------------------------------------------------------

// Per thread: u_p = zt_p ? (W - accz_p) : accz_p, with accz_p the per-thread
// sums over the compile-time j bits (acc[s] holds z bit acc_lo + s).
template <int NA, class A>
__device__ __forceinline__ A marg_u(int p, long long zt, A W, const A* acc, int acc_lo) {
  A a = 0;
  const int q = p - acc_lo;
#pragma unroll
  for (int s = 0; s < NA; ++s)
    if (s == q) a = acc[s];
  return ((zt >> p) & 1) ? (W - a) : a;
}

// part[v * nblk + blk] = the block's sum of W (v = 0) and of u_p (v = 1 + p)
// for v < nvals (two: each thread's values are the sums over two sets, a
// chunk and its mirror); wred holds nvals * kWarps entries of A.
template <int NA, class A>
__device__ __forceinline__ void marg_reduce(A* wred, int nvals, double* part, long long nblk,
                                            long long blk, long long zt, A W, const A* acc,
                                            bool two, long long zt2, A W2, const A* acc2) {
  block_sums<A>(
      wred, nvals,
      [&](int v) -> A {
        if (v == 0) return two ? W + W2 : W;
        A u = marg_u<NA, A>(v - 1, zt, W, acc, 7);
        if (two) u += marg_u<NA, A>(v - 1, zt2, W2, acc2, 7);
        return u;
      },
      [&](int v, double sum) { part[(long long)v * nblk + blk] = sum; });
}

// ---------------------------------------------------------------------------
// Diagonal / complement pass
// ---------------------------------------------------------------------------
// CTA = one chunk of CH = 2^cb amplitudes (XC: a chunk and its mirror chunk);
// amplitude i of the chunk is handled by thread i % 256 at step j = i / 256.
template <class R, int NS, int ZM, int XC, int JB>
__global__ void __launch_bounds__(kThreads) k_diag(const DiagPass P, const R* __restrict__ coef,
                                                   const cx<R>* src0, cx<R>* dst0,
                                                   const cx<R>* src1, cx<R>* dst1,
                                                   double* __restrict__ part) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* scol = reinterpret_cast<R*>(smraw);  // [nvals][kWarps] warp totals
  const int n = P.n, cb = P.cb;
  const long long N = 1LL << n;
  const int CH = 1 << cb;
  const int nchb = n - cb;
  const long long nch = 1LL << nchb;
  const long long cpb = XC ? (nch > 1 ? nch / 2 : 1) : nch;  // CTAs per sample
  const int b = (int)(blockIdx.x / cpb);
  const long long ch = blockIdx.x % cpb;
  const long long base = ch << cb;
  const long long sb = (long long)b << n;
  const R* tabs = coef + P.coef + (long long)b * P.bstride;
  const int tid = threadIdx.x;
  constexpr int NJ = 1 << JB;
  const bool active = tid < CH;

  if (!XC) {
    R W = 0, acc[JB + 2];
#pragma unroll
    for (int s = 0; s < JB + 2; ++s) acc[s] = 0;
    if (active) {
      if constexpr (NS == 1) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const long long k = base + tid + (j << 8);
          const C ph = diag_phase<R>(tabs, P.tb, ztrans(k, n, ZM));
          dst0[sb + k] = cmul<R>(ph, src0[sb + k]);
        }
      } else {
        // U steps' loads (both states and the phase-table entries) before
        // their stores: 2U amplitude loads in flight per thread; the step
        // loop itself stays rolled (a fully unrolled one missed the
        // instruction cache), the marginal bits of step j are runtime tests
        constexpr int U = NJ < 4 ? NJ : 4;
#pragma unroll 1
        for (int j0 = 0; j0 < NJ; j0 += U) {
          C xs[U], ls[U], ph[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long k = base + tid + ((j0 + u) << 8);
            xs[u] = src0[sb + k];
            ls[u] = src1[sb + k];
            ph[u] = diag_phase<R>(tabs, P.tb, ztrans(k, n, ZM));
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int j = j0 + u;
            const long long k = base + tid + (j << 8);
            const C y = cmulc<R>(ph[u], xs[u]);  // conj(phase) * psi
            const C w_ = cmulc<R>(ph[u], ls[u]);  // conj(phase) * lambda
            dst0[sb + k] = y;
            dst1[sb + k] = w_;
            const R w = im_cdot<R>(w_, y);
            W += w;
            const int zb = zj_bits<ZM>(j);
#pragma unroll
            for (int s = 0; s < JB + 2; ++s) acc[s] += ((zb >> (7 + s)) & 1) ? w : (R)0;
          }
        }
      }
    }
    if (NS == 2) {
      const long long zt = ztrans(base + tid, n, ZM);
      marg_reduce<JB + 2, R>(scol, P.nvals, part, gridDim.x, blockIdx.x, active ? zt : 0, W, acc,
                             false, 0, (R)0, acc);
    }
  } else {
    // mirror chunk of `ch` is nch-1-ch; a single chunk is its own mirror
    const bool single = (nch == 1);
    const long long mbase = (nch - 1 - ch) << cb;
    const int lim = single ? CH / 2 : CH;
    R W = 0, acc[JB + 2], Wm = 0, accm[JB + 2];
#pragma unroll
    for (int s = 0; s < JB + 2; ++s) acc[s] = accm[s] = 0;
    if constexpr (NS == 1) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int i = tid + (j << 8);
        if (i < lim) {
          const long long k = base + i;
          const long long km = N - 1 - k;  // = mbase + (CH - 1 - i)
          const C xk = src0[sb + k], xm = src0[sb + km];
          if (P.has_phase) {
            dst0[sb + k] = cmul<R>(diag_phase<R>(tabs, P.tb, km), xm);
            dst0[sb + km] = cmul<R>(diag_phase<R>(tabs, P.tb, k), xk);
          } else {
            dst0[sb + k] = xm;
            dst0[sb + km] = xk;
          }
        }
      }
    } else {
      // U steps' loads (both states at k and ~k, and the phase-table entries)
      // are issued before any of their stores, so a thread has 4U amplitude
      // loads in flight instead of 4 (the step loop stays rolled: fully
      // unrolled it missed the instruction cache): a thread's elements are its own, and k
      // and ~k of different steps never coincide (k + k' = N - 1 would need
      // two indices of one chunk, or of a chunk and its mirror at the same
      // step, to add up to an odd number they cannot reach), so the reorder
      // is safe in place.
      constexpr int U = NJ < 4 ? NJ : 4;
#pragma unroll 1
      for (int j0 = 0; j0 < NJ; j0 += U) {
        C pk[U], pm[U], lk[U], lm[U], phk[U], phm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = tid + ((j0 + u) << 8);
          if (i < lim) {
            const long long k = base + i;
            const long long km = N - 1 - k;  // = mbase + (CH - 1 - i)
            pk[u] = src0[sb + k]; pm[u] = src0[sb + km];
            lk[u] = src1[sb + k]; lm[u] = src1[sb + km];
            if (P.has_phase) {
              phk[u] = diag_phase<R>(tabs, P.tb, k);
              phm[u] = diag_phase<R>(tabs, P.tb, km);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + u;
          const int i = tid + (j << 8);
          if (i < lim) {
            const long long k = base + i;
            const long long km = N - 1 - k;
            C yk, ym, uk, um;
            if (P.has_phase) {
              yk = cmulc<R>(phk[u], pm[u]); uk = cmulc<R>(phk[u], lm[u]);  // in[k] = conj(ph(k)) out[~k]
              ym = cmulc<R>(phm[u], pk[u]); um = cmulc<R>(phm[u], lk[u]);
            } else {
              yk = pm[u]; uk = lm[u]; ym = pk[u]; um = lk[u];
            }
            dst0[sb + k] = yk; dst1[sb + k] = uk;
            dst0[sb + km] = ym; dst1[sb + km] = um;
            const R wk = im_cdot<R>(uk, yk), wm = im_cdot<R>(um, ym);
            W += wk;
            Wm += wm;
#pragma unroll
            for (int s = 0; s < JB + 2; ++s) {
              // z = k: j-bit contribution (j << 8); mirror: z = km, i' = CH-1-i
              const bool on = ((j << 8) >> (7 + s)) & 1;
              acc[s] += on ? wk : (R)0;
              accm[s] += on ? wm : (R)0;
            }
          }
        }
      }
    }
    if (NS == 2) {
      // k = base ^ tid ^ (j << 8); km = (mbase + CH - 1) ^ tid ^ (j << 8), so the
      // mirror uses the same j-bit accumulators with the complemented constant.
      const bool act = tid < lim || (tid < CH && !single);
      const long long zt = base + tid;
      const long long ztm = (mbase + CH - 1) ^ tid;
      marg_reduce<JB + 2, R>(scol, P.nvals, part, gridDim.x, blockIdx.x, act ? zt : 0,
                             act ? W : (R)0, acc, true, act ? ztm : 0, act ? Wm : (R)0, accm);
    }
  }
}

// ---------------------------------------------------------------------------
// <Z> marginals of |psi|^2 and lambda = O psi
// ---------------------------------------------------------------------------
template <class R, int JB>
__global__ void __launch_bounds__(kThreads) k_expect(int n, int cb, const cx<R>* __restrict__ psi,
                                                     double* __restrict__ part) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nchb = n - cb;
  const int b = (int)(blockIdx.x >> nchb);
  const long long base = ((long long)blockIdx.x & ((1LL << nchb) - 1)) << cb;
  const C* s = psi + ((long long)b << n) + base;
  const int tid = threadIdx.x;
  const bool active = tid < (1 << cb);
  R W = 0, acc[JB + 2];
#pragma unroll
  for (int q = 0; q < JB + 2; ++q) acc[q] = 0;
  if (active) {
#pragma unroll
    for (int j = 0; j < (1 << JB); ++j) {
      const C x = s[tid + (j << 8)];
      const R w = x.x * x.x + x.y * x.y;
      W += w;
#pragma unroll
      for (int q = 0; q < JB + 2; ++q)
        if (((j << 8) >> (7 + q)) & 1) acc[q] += w;
    }
  }
  // per-CTA sums in the state's precision (the FP64 rate is a small fraction of
  // the FP32 rate); one conversion per CTA value, the sums over CTAs in FP64
  R* sr = reinterpret_cast<R*>(smraw);
  const long long zt = active ? (base + tid) : 0;
  sr[tid] = W;
  for (int p = 0; p < n; ++p) {
    R a = 0;
#pragma unroll
    for (int q = 0; q < JB + 2; ++q)
      if (q == p - 7) a = acc[q];
    sr[(1 + p) * kThreads + tid] = ((zt >> p) & 1) ? (W - a) : a;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  for (int v = warp; v < n + 1; v += kWarps) {
    R t = 0;
#pragma unroll
    for (int e = 0; e < kThreads / 32; ++e) t += sr[v * kThreads + lane + 32 * e];
    t = warp_sum_r<R>(t);
    if (lane == 0) part[(long long)v * gridDim.x + blockIdx.x] = (double)t;
  }
}

// lambda[b][k] = (sum_q g[b][q] (1 - 2 bit_{n-1-q}(k))) psi[b][k]
template <class R>
__global__ void __launch_bounds__(kThreads) k_laminit(int n, int cb, const double* __restrict__ gez,
                                                      const cx<R>* __restrict__ psi,
                                                      cx<R>* __restrict__ lam) {
  using C = cx<R>;
  __shared__ double g[kMaxQubits];
  __shared__ R Ta[64], Tb[64];
  const int nchb = n - cb;
  const int b = (int)(blockIdx.x >> nchb);
  const long long base = ((long long)blockIdx.x & ((1LL << nchb) - 1)) << cb;
  for (int q = threadIdx.x; q < n; q += blockDim.x) g[q] = gez[(long long)b * n + q];
  __syncthreads();
  const int la = cb < 6 ? cb : 6, lb = cb - la;
  // o(i) = Tb[i >> la] + Ta[i & (2^la - 1)]: Tb holds the total, the chunk's
  // fixed bits and the upper in-chunk bits, Ta the low bits, both in the
  // state's precision
  for (int e = threadIdx.x; e < 128; e += blockDim.x) {
    double acc = 0;
    if (e < 64) {
      for (int i = 0; i < la; ++i)
        if ((e >> i) & 1) acc += g[n - 1 - i];
      Ta[e] = (R)(-2.0 * acc);
    } else {
      const int f = e - 64;
      double tot = 0;
      for (int q = 0; q < n; ++q) {
        tot += g[q];
        const int p = n - 1 - q;
        if (p >= cb && ((base >> p) & 1)) acc += g[q];
      }
      for (int i = 0; i < lb; ++i)
        if ((f >> i) & 1) acc += g[n - 1 - (la + i)];
      Tb[f] = (R)(tot - 2.0 * acc);
    }
  }
  __syncthreads();
  const long long off = ((long long)b << n) + base;
  const int CH = 1 << cb, ma = (1 << la) - 1;
  // pairs (i, i + 1) share Tb (n >= 1, so la >= 1)
  for (int i = 2 * threadIdx.x; i < CH; i += 2 * blockDim.x) {
    const R tb = Tb[i >> la];
    const R o0 = tb + Ta[i & ma], o1 = tb + Ta[(i + 1) & ma];
    const C x0 = psi[off + i], x1 = psi[off + i + 1];
    store_pair<R>(lam + off + i, mk<R>(o0 * x0.x, o0 * x0.y), mk<R>(o1 * x1.x, o1 * x1.y));
  }
}

// ---------------------------------------------------------------------------
// CNOT ring permutation (closed-form GF(2) index map)
// ---------------------------------------------------------------------------
// NS = 1: out[k] = in[f^-1(k)] (forward).  NS = 2: new[y] = old[f(y)] for
// psi and lambda (backward, the inverse permutation).
// With gez != NULL (backward only) lambda is not read: lambda = O psi with
// O = sum_q g[b][q] Z_q is formed from the loaded psi (the first backward step).
template <class R, int NS>
__global__ void __launch_bounds__(kThreads) k_ring(const RingPass P, const cx<R>* src0, cx<R>* dst0,
                                                   const cx<R>* src1, cx<R>* dst1,
                                                   const double* __restrict__ gez, const R* __restrict__ coef,
                                                   double* __restrict__ part) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* S = reinterpret_cast<C*>(smraw);
  const int n = P.n;
  if constexpr (NS == 2) {
    if (P.pre && !gez) {
      // backward: undo the diagonal layer that follows the ring in the
      // forward (its phase by the tile's own index: z = k), then the ring.
      // Thread tid holds tile elements e = tid + kThreads j: index bits 0..7
      // are tid's, bits 8 .. t-2 and the top bit (n - 1) come from j, the
      // rest from the tile.  w = Im(conj(lambda) psi) is unchanged by the
      // phase, so the marginals are summed from the loaded values.
      // (a whole-state CTA is the tile t = n: no tile bits, bit n - 1 the top)
      const int t = P.whole ? n : P.t, H = 1 << (t - 1);
      const int fb = n - t;
      const int b = (int)(blockIdx.x >> fb);
      const long long f = blockIdx.x & ((1LL << fb) - 1);
      const long long sb = (long long)b << n;
      const long long tb = f << (t - 1);
      const long long ib = tb ^ (tb >> 1);
      const long long A = ib & ~(long long)(H - 1);
      const long long Bk = A ^ (3LL << (n - 2));
      const int il = (int)(ib & (H - 1));
      const long long topbit = 1LL << (n - 1);
      const R* tabs = coef + P.pre_coef + (long long)b * P.pre_bstride;
      C* S1 = S + 2 * H;
      const int nj = (2 * H) / kThreads, jb = t - 9;  // jl bits 8 .. t-2 are j bits 0 .. jb-1
      R W = 0, T = 0, Aj[4] = {0, 0, 0, 0};
      // four steps' loads (both states and the phase-table entries) before
      // their smem writes, so each thread has eight amplitude loads in flight
#pragma unroll 1
      for (int j0 = 0; j0 < nj; j0 += 4) {
        C xs[4], ls[4], ph[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = threadIdx.x + (j0 + u) * kThreads;
          if (j0 + u >= nj) break;
          const int top = e >> (t - 1), jl = e & (H - 1);
          const long long k = tb + jl + (top ? topbit : 0);
          xs[u] = src0[sb + k];
          ls[u] = src1[sb + k];
          ph[u] = diag_phase<R>(tabs, P.pre_tb, k);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          if (j >= nj) break;
          const int e = threadIdx.x + j * kThreads;
          S[e] = cmulc<R>(ph[u], xs[u]);
          S1[e] = cmulc<R>(ph[u], ls[u]);
          if (P.pre_grad) {
            const R w = im_cdot<R>(ls[u], xs[u]);
            W += w;
            if ((e >> (t - 1)) & 1) T += w;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (q < jb && ((j >> q) & 1)) Aj[q] += w;
          }
        }
      }
      __syncthreads();
      if (P.whole) {
        for (int k = threadIdx.x; k < 2 * H; k += kThreads) {
          const int y = ring_f(k, n);
          dst0[sb + k] = S[y];
          dst1[sb + k] = S1[y];
        }
      }
      for (int s2 = 0; s2 < 2 && !P.whole; ++s2) {
        const C* Ss = s2 ? S1 : S;
        C* dst = s2 ? dst1 : dst0;
        for (int e = 2 * threadIdx.x; e < 2 * H; e += 2 * kThreads) {
          const int u = e >> (t - 1), yl = e & (H - 1);
          const int jl = gray_inv(yl ^ il);
          const int top = u ^ (jl & 1);
          store_pair<R>(dst + sb + (u ? Bk : A) + yl, Ss[top * H + jl], Ss[(top ^ 1) * H + (jl ^ 1)]);
        }
      }
      if (P.pre_grad) {
        // per warp: W, the masked sums for lane bits 0..4, the j-bit sums and
        // the top-bit sum in the state's precision (each over 32 lanes);
        // across warps in FP64
        __shared__ R red[11][kWarps];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        R vals[11];
        vals[0] = warp_sum_r<R>(W);
#pragma unroll
        for (int q = 0; q < 5; ++q) vals[1 + q] = warp_sum_r<R>(((lane >> q) & 1) ? W : (R)0);
#pragma unroll
        for (int q = 0; q < 4; ++q) vals[6 + q] = q < jb ? warp_sum_r<R>(Aj[q]) : (R)0;
        vals[10] = warp_sum_r<R>(T);
        if (lane == 0)
          for (int v = 0; v < 11; ++v) red[v][warp] = vals[v];
        __syncthreads();
        const long long nblk = gridDim.x;
        for (int v = threadIdx.x; v <= n; v += kThreads) {
          // v = 0: W; v = 1 + p: M_p, the sum of w over elements with index bit p
          const int p = v - 1;
          double sum = 0;
          for (int w2 = 0; w2 < kWarps; ++w2) {
            double x;
            if (v == 0 || (p >= t - 1 && p < n - 1)) x = red[0][w2];
            else if (p < 5) x = red[1 + p][w2];
            else if (p < 8) x = ((w2 >> (p - 5)) & 1) ? red[0][w2] : 0.0;
            else if (p < t - 1) x = red[6 + (p - 8)][w2];
            else x = red[10][w2];
            sum += x;
          }
          if (p >= t - 1 && p < n - 1 && !((tb >> p) & 1)) sum = 0;
          part[(long long)v * nblk + blockIdx.x] = sum;
        }
      }
      return;
    }
  }
  if (NS == 2 && gez) {
    __shared__ double Sg[kMaxQubits];
    const int b = P.whole ? (int)blockIdx.x : (int)(blockIdx.x >> (n - P.t));
    const long long sb = (long long)b << n;
    for (int q = threadIdx.x; q < n; q += kThreads) Sg[q] = gez[(long long)b * n + q];
    __syncthreads();
    if (P.whole) {
      const int N = 1 << n;
      for (int i = threadIdx.x; i < N; i += kThreads) S[i] = src0[sb + i];
      __syncthreads();
      for (int k = threadIdx.x; k < N; k += kThreads) {
        const int y = ring_f(k, n);
        double o = 0;
        for (int q = 0; q < n; ++q) o += ((y >> (n - 1 - q)) & 1) ? -Sg[q] : Sg[q];
        const C x = S[y];
        dst0[sb + k] = x;
        dst1[sb + k] = mk<R>((R)o * x.x, (R)o * x.y);
      }
      return;
    }
    const int t = P.t, H = 1 << (t - 1);
    const long long f = blockIdx.x & ((1LL << (n - t)) - 1);
    const long long tb = f << (t - 1);
    const long long ib = tb ^ (tb >> 1);
    const long long A = ib & ~(long long)(H - 1);
    const long long Bk = A ^ (3LL << (n - 2));
    const int il = (int)(ib & (H - 1));
    const long long topbit = 1LL << (n - 1);
    // o(k) = sum_q g_q - 2 sum_{bits p of k} g_{n-1-p}, split into the low 6 bits
    // and the next 6 bits of the half-tile index (tables in the state's
    // precision) and c0[top]: the total, the tile's fixed bits and the top bit
    __shared__ R Ta[64], Tb[64], c0[2];
    for (int e = threadIdx.x; e < 128; e += kThreads) {
      R acc = 0;
      const int lo = e < 64 ? 0 : 6, v = e & 63;
      for (int i = 0; i < 6; ++i)
        if (((v >> i) & 1) && lo + i < t - 1) acc += (R)Sg[n - 1 - (lo + i)];
      if (e < 64) Ta[v] = -2 * acc; else Tb[v] = -2 * acc;
    }
    if (threadIdx.x == 128) {
      double tot = 0, hi = 0;
      for (int q = 0; q < n; ++q) tot += Sg[q];
      for (int p = t - 1; p < n - 1; ++p)
        if ((tb >> p) & 1) hi += Sg[n - 1 - p];
      c0[0] = (R)(tot - 2.0 * hi);
      c0[1] = (R)(tot - 2.0 * (hi + Sg[0]));
    }
    for (int e = threadIdx.x; e < 2 * H; e += kThreads) {
      const int top = e >> (t - 1), jl = e & (H - 1);
      S[e] = src0[sb + tb + jl + (top ? topbit : 0)];
    }
    __syncthreads();
    // element pairs (yl, yl ^ 1): gray_inv(x ^ 1) = gray_inv(x) ^ 1, so the pair
    // reads (top, jl) and (top ^ 1, jl ^ 1) and writes 16 (c64) bytes per state
    for (int e = 2 * threadIdx.x; e < 2 * H; e += 2 * kThreads) {
      const int u = e >> (t - 1), yl = e & (H - 1);
      const int jl = gray_inv(yl ^ il);
      const int top = u ^ (jl & 1);
      const C x0 = S[top * H + jl], x1 = S[(top ^ 1) * H + (jl ^ 1)];
      const R o0 = c0[top] + Ta[jl & 63] + Tb[(jl >> 6) & 63];
      const R o1 = c0[top ^ 1] + Ta[(jl ^ 1) & 63] + Tb[(jl >> 6) & 63];
      const long long d = sb + (u ? Bk : A) + yl;
      store_pair<R>(dst0 + d, x0, x1);
      store_pair<R>(dst1 + d, mk<R>(o0 * x0.x, o0 * x0.y), mk<R>(o1 * x1.x, o1 * x1.y));
    }
    return;
  }
  if (P.whole) {
    const int N = 1 << n;
    const long long sb = (long long)blockIdx.x << n;
    for (int s = 0; s < NS; ++s) {
      const C* src = s ? src1 : src0;
      C* dst = s ? dst1 : dst0;
      for (int i = threadIdx.x; i < N; i += kThreads) S[i] = src[sb + i];
      __syncthreads();
      for (int k = threadIdx.x; k < N; k += kThreads)
        dst[sb + k] = S[NS == 1 ? ring_finv(k, n) : ring_f(k, n)];
      __syncthreads();
    }
    return;
  }
  const int t = P.t;
  const int H = 1 << (t - 1);
  const int fb = n - t;
  const int b = (int)(blockIdx.x >> fb);
  const long long f = blockIdx.x & ((1LL << fb) - 1);
  const long long sb = (long long)b << n;
  const long long tb = f << (t - 1);                       // tile base (bits t-1 .. n-2)
  const long long ib = tb ^ (tb >> 1);                     // f^-1(tile base)
  const long long A = ib & ~(long long)(H - 1);            // block A, B = A ^ 3 << (n-2)
  const long long Bk = A ^ (3LL << (n - 2));
  const int il = (int)(ib & (H - 1));
  const long long topbit = 1LL << (n - 1);
  for (int s = 0; s < NS; ++s) {
    const C* src = s ? src1 : src0;
    C* dst = s ? dst1 : dst0;
    if (NS == 1) {
      // load the two input blocks, write the output tile
      for (int y = threadIdx.x; y < H; y += kThreads) {
        S[y] = src[sb + A + y];
        S[H + y] = src[sb + Bk + y];
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 2 * H; e += kThreads) {
        const int top = e >> (t - 1), jl = e & (H - 1);
        const int u = (jl & 1) ^ top;
        dst[sb + tb + jl + (top ? topbit : 0)] = S[u * H + (il ^ jl ^ (jl >> 1))];
      }
    } else {
      // load the tile (old), write the two blocks (new[y] = old[f(y)])
      for (int e = threadIdx.x; e < 2 * H; e += kThreads) {
        const int top = e >> (t - 1), jl = e & (H - 1);
        S[e] = src[sb + tb + jl + (top ? topbit : 0)];
      }
      __syncthreads();
      for (int e = 2 * threadIdx.x; e < 2 * H; e += 2 * kThreads) {
        const int u = e >> (t - 1), yl = e & (H - 1);
        const int jl = gray_inv(yl ^ il);
        const int top = u ^ (jl & 1);
        store_pair<R>(dst + sb + (u ? Bk : A) + yl, S[top * H + jl], S[(top ^ 1) * H + (jl ^ 1)]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Reductions of per-CTA partials (fixed order, float64)
// ---------------------------------------------------------------------------
// rows: job j has batch * nvals rows starting at row0[j]; V[row] = sum of the
// sample's CTAs' partials for that value.  One warp per row (a row sums at
// most a few dozen partials: one CTA per row left most of 10^5 CTAs idle on
// batches of hundreds of samples).
#if QC_INST_R != 8
static __global__ void __launch_bounds__(kThreads) k_red1(const RedJob* __restrict__ jobs,
                                                   const long long* __restrict__ row0, int njobs,
                                                   long long rowbase, long long nrows,
                                                   const double* __restrict__ part, double* __restrict__ V) {
  const long long rl = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (rl >= nrows) return;
  const int lane = threadIdx.x & 31;
  const long long row = rowbase + rl;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {  // last job with row0 <= row
    int mid = (lo + hi + 1) >> 1;
    if (row0[mid] <= row) lo = mid; else hi = mid - 1;
  }
  const RedJob J = jobs[lo];
  const long long r = row - row0[lo];
  const int bsm = (int)(r / J.nvals), v = (int)(r % J.nvals);
  const double* p = part + J.part_off + (long long)v * J.nblk + (long long)bsm * J.blk_per_sample;
  double s = 0;
  for (int i = lane; i < J.blk_per_sample; i += 32) s += p[i];
  s = warp_sum(s);
  if (lane == 0) V[row] = s;
}
#endif

// one warp per output of a job group: combine values into gradients, the
// lanes over the batch (added to d_theta / d_x, which the caller zeroes
// first; a group's outputs write distinct entries).
#if QC_INST_R != 8
static __global__ void k_finalize(const RedJob* __restrict__ jobs, const long long* __restrict__ row0,
                           const int* __restrict__ out0, int njobs, int outbase, int nout,
                           const RedOut* __restrict__ outs, int batch, int n_in,
                           const double* __restrict__ V, double* __restrict__ d_theta,
                           double* __restrict__ d_x) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= nout) return;
  const int lane = threadIdx.x & 31;
  const int o = outbase + t;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (out0[mid] <= o) lo = mid; else hi = mid - 1;
  }
  const RedJob J = jobs[lo];
  const RedOut ro = outs[o];
  const double* v = V + row0[lo];
  double tot = 0;
  for (int b = lane; b < batch; b += 32) {
    const double* vb = v + (long long)b * J.nvals;
    const double g = J.kind == RK_DIRECT ? ro.scale * vb[ro.val]
                                         : ro.scale * (vb[0] - 2.0 * vb[1 + ro.val]);
    if (J.source == QC_SRC_INPUT) {
      if (d_x) d_x[(long long)b * n_in + ro.pidx] += g;
    } else {
      tot += g;
    }
  }
  if (J.source == QC_SRC_THETA) {
    tot = warp_sum(tot);
    if (lane == 0 && d_theta) d_theta[ro.pidx] += tot;
  }
}
#endif

// <Z_q> from marginals: ez[b][q] = W - 2 M_{n-1-q}, one block per (b, q)
// summing the sample's CTA partials of W and of the qubit's bit marginal.
static __global__ void __launch_bounds__(kThreads) k_ez_from_marg(int n, int blk_per_sample, long long nblk,
                                                           const double* __restrict__ part,
                                                           double* __restrict__ ez) {
  const int b = blockIdx.x / n, q = blockIdx.x % n;
  const int p = n - 1 - q;
  const double* w = part + (long long)b * blk_per_sample;
  const double* m = part + (long long)(1 + p) * nblk + (long long)b * blk_per_sample;
  double sw = 0, sm = 0;
  for (int i = threadIdx.x; i < blk_per_sample; i += kThreads) {
    sw += w[i];
    sm += m[i];
  }
  __shared__ double red[2][kWarps];
  sw = warp_sum(sw);
  sm = warp_sum(sm);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sw;
    red[1][threadIdx.x >> 5] = sm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0;
    for (int k = 0; k < kWarps; ++k) { a += red[0][k]; c += red[1][k]; }
    ez[(long long)b * n + q] = a - 2.0 * c;
  }
}

// ---------------------------------------------------------------------------
// Whole circuit of one sample in shared memory (small n)
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void sm_1q_fwd(cx<R>* S, int n, int p, const R* m, int real) {
  using C = cx<R>;
  const int half = 1 << (n - 1);
  const C m00 = ldc<R>(m), m01 = ldc<R>(m + 2), m10 = ldc<R>(m + 4), m11 = ldc<R>(m + 6);
  for (int i = threadIdx.x; i < half; i += blockDim.x) {
    const int a = ((i >> p) << (p + 1)) | (i & ((1 << p) - 1));
    const int a1 = a | (1 << p);
    const C x0 = S[a], x1 = S[a1];
    S[a] = cfma<R>(m01, x1, cmul<R>(m00, x0));
    S[a1] = cfma<R>(m11, x1, cmul<R>(m10, x0));
  }
  (void)real;
}

// undo a single-qubit gate on psi and lambda; returns this thread's share of
// 2 Re <lambda|A|psi> (input side)
template <class R>
__device__ __forceinline__ double sm_1q_bwd(cx<R>* P, cx<R>* L, int n, int p, const R* m, int np) {
  using C = cx<R>;
  const int half = 1 << (n - 1);
  const C m00 = ldc<R>(m), m01 = ldc<R>(m + 2), m10 = ldc<R>(m + 4), m11 = ldc<R>(m + 6);
  const C a00 = ldc<R>(m + 8), a01 = ldc<R>(m + 10), a10 = ldc<R>(m + 12), a11 = ldc<R>(m + 14);
  R g = 0;
  for (int i = threadIdx.x; i < half; i += blockDim.x) {
    const int a = ((i >> p) << (p + 1)) | (i & ((1 << p) - 1));
    const int a1 = a | (1 << p);
    C x0 = P[a], x1 = P[a1], u0 = L[a], u1 = L[a1];
    C y0 = cfmac<R>(m10, x1, cfmac<R>(m00, x0, mk<R>(0, 0)));
    C y1 = cfmac<R>(m11, x1, cfmac<R>(m01, x0, mk<R>(0, 0)));
    C w0 = cfmac<R>(m10, u1, cfmac<R>(m00, u0, mk<R>(0, 0)));
    C w1 = cfmac<R>(m11, u1, cfmac<R>(m01, u0, mk<R>(0, 0)));
    P[a] = y0; P[a1] = y1; L[a] = w0; L[a1] = w1;
    if (np) {
      C t0 = cfma<R>(a01, y1, cmul<R>(a00, y0));
      C t1 = cfma<R>(a11, y1, cmul<R>(a10, y0));
      g += re_cdot<R>(w0, t0) + re_cdot<R>(w1, t1);
    }
  }
  return 2.0 * (double)g;
}

template <class R>
__device__ __forceinline__ void sm_2q_fwd(cx<R>* S, int n, int plo, const R* m) {
  using C = cx<R>;
  const int quarter = 1 << (n - 2);
  for (int i = threadIdx.x; i < quarter; i += blockDim.x) {
    // insert zeros at bits plo and plo+1
    const int a = ((i >> plo) << (plo + 2)) | (i & ((1 << plo) - 1));
    C x[4], y[4];
    for (int s = 0; s < 4; ++s) x[s] = S[a | (s << plo)];
    for (int r = 0; r < 4; ++r) {
      C t = mk<R>(0, 0);
      for (int s = 0; s < 4; ++s) t = cfma<R>(ldc<R>(m + 2 * (r * 4 + s)), x[s], t);
      y[r] = t;
    }
    for (int s = 0; s < 4; ++s) S[a | (s << plo)] = y[s];
  }
}

template <class R>
__device__ __forceinline__ void sm_2q_bwd(cx<R>* P, cx<R>* L, int n, int plo, const R* m, int np,
                                          double g[3]) {
  using C = cx<R>;
  const int quarter = 1 << (n - 2);
  R gl[3] = {0, 0, 0};
  for (int i = threadIdx.x; i < quarter; i += blockDim.x) {
    const int a = ((i >> plo) << (plo + 2)) | (i & ((1 << plo) - 1));
    C x[4], u[4], y[4], w[4];
    for (int s = 0; s < 4; ++s) { x[s] = P[a | (s << plo)]; u[s] = L[a | (s << plo)]; }
    for (int r = 0; r < 4; ++r) {
      C t = mk<R>(0, 0), z = mk<R>(0, 0);
      for (int s = 0; s < 4; ++s) {
        C ms = ldc<R>(m + 2 * (s * 4 + r));
        t = cfmac<R>(ms, x[s], t);
        z = cfmac<R>(ms, u[s], z);
      }
      y[r] = t; w[r] = z;
    }
    for (int s = 0; s < 4; ++s) { P[a | (s << plo)] = y[s]; L[a | (s << plo)] = w[s]; }
    for (int k = 0; k < np; ++k) {
      const R* A = m + kRec2qA + 32 * k;
      for (int r = 0; r < 4; ++r) {
        C t = mk<R>(0, 0);
        for (int s = 0; s < 4; ++s) t = cfma<R>(ldc<R>(A + 2 * (r * 4 + s)), y[s], t);
        gl[k] += re_cdot<R>(w[r], t);
      }
    }
  }
  for (int k = 0; k < 3; ++k) g[k] = 2.0 * (double)gl[k];
}

// block sum of `v` (all threads participate); result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < kWarps; ++w) s += red[w];
  return s;
}

template <class R, int BWD>
__global__ void __launch_bounds__(kThreads) k_smem(const SmemLayer* __restrict__ prog, int nl, int n,
                                                   int batch, const R* __restrict__ coef,
                                                   const cx<R>* psi_in, cx<R>* psi_out,
                                                   double* __restrict__ ez,
                                                   const double* __restrict__ gez,
                                                   double* __restrict__ part, int nslots) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = 1 << n;
  C* P = reinterpret_cast<C*>(smraw);
  C* L = P + N;  // BWD only
  double* red = reinterpret_cast<double*>(P + (BWD ? 2 * N : N));
  double* marg = red + kWarps;  // (n + 1) values
  const int b = blockIdx.x;
  const long long sb = (long long)b << n;
  (void)batch;

  if (!BWD) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) P[i] = mk<R>(i == 0 ? 1 : 0, 0);
  } else {
    // lambda = O psi_L
    const double* g = gez + (long long)b * n;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      double o = 0;
      for (int q = 0; q < n; ++q) o += ((i >> (n - 1 - q)) & 1) ? -g[q] : g[q];
      const C x = psi_in[sb + i];
      P[i] = x;
      L[i] = mk<R>((R)o * x.x, (R)o * x.y);
    }
  }
  __syncthreads();

  for (int li = 0; li < nl; ++li) {
    const int l = BWD ? nl - 1 - li : li;
    const SmemLayer Ly = prog[l];
    const R* cf = coef + Ly.coef + (long long)b * Ly.bstride;
    switch (Ly.cls) {
      case LC_ROT1:
        for (int q = 0; q < n; ++q) {
          const int p = n - 1 - q;
          if (!BWD) {
            sm_1q_fwd<R>(P, n, p, cf + q * kRec1q, Ly.real);
          } else {
            double g = sm_1q_bwd<R>(P, L, n, p, cf + q * kRec1q, Ly.slot >= 0);
            if (Ly.slot >= 0) {
              g = block_sum(g, red);
              if (threadIdx.x == 0) part[(long long)(Ly.slot + q) * batch + b] = g;
            }
          }
          __syncthreads();
        }
        break;
      case LC_DENSE2:
        for (int gi = 0; gi < Ly.ngates; ++gi) {
          const int q0 = Ly.parity + 2 * gi;
          const int plo = n - 2 - q0;
          const R* m = cf + gi * kRec2q;
          if (!BWD) {
            sm_2q_fwd<R>(P, n, plo, m);
          } else {
            double g[3];
            const int np = Ly.slot >= 0 ? Ly.np_per_gate : 0;
            sm_2q_bwd<R>(P, L, n, plo, m, np, g);
            for (int k = 0; k < np; ++k) {
              double s = block_sum(g[k], red);
              if (threadIdx.x == 0) part[(long long)(Ly.slot + 3 * gi + k) * batch + b] = s;
            }
          }
          __syncthreads();
        }
        break;
      case LC_DIAG: {
        if (!BWD) {
          for (int k = threadIdx.x; k < N; k += blockDim.x)
            P[k] = cmul<R>(diag_phase<R>(cf, Ly.tb, ztrans(k, n, Ly.zmode)), P[k]);
          __syncthreads();
        } else {
          double W = 0, Mp[kMaxQubits];
          for (int p = 0; p < n; ++p) Mp[p] = 0;
          for (int k = threadIdx.x; k < N; k += blockDim.x) {
            const long long z = ztrans(k, n, Ly.zmode);
            const C ph = diag_phase<R>(cf, Ly.tb, z);
            const C y = cmulc<R>(ph, P[k]), u = cmulc<R>(ph, L[k]);
            P[k] = y; L[k] = u;
            const double w = (double)im_cdot<R>(u, y);
            W += w;
            for (int p = 0; p < n; ++p)
              if ((z >> p) & 1) Mp[p] += w;
          }
          if (Ly.slot >= 0) {
            double Wt = block_sum(W, red);
            for (int p = 0; p < n; ++p) {
              double s = block_sum(Mp[p], red);
              if (threadIdx.x == 0) marg[p] = s;
            }
            __syncthreads();
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
              const int p = Ly.kind == QC_L_ISINGZZ_RING ? ((n - 2 - j) % n + n) % n : n - 1 - j;
              part[(long long)(Ly.slot + j) * batch + b] = Ly.gscale * (Wt - 2.0 * marg[p]);
            }
          }
          __syncthreads();
        }
        break;
      }
      case LC_XCOMP: {
        if (!BWD) {
          for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
            const int km = N - 1 - k;
            const C xk = P[k], xm = P[km];
            if (Ly.has_phase) {
              P[k] = cmul<R>(diag_phase<R>(cf, Ly.tb, km), xm);
              P[km] = cmul<R>(diag_phase<R>(cf, Ly.tb, k), xk);
            } else {
              P[k] = xm; P[km] = xk;
            }
          }
          __syncthreads();
        } else {
          double W = 0, Mp[kMaxQubits];
          for (int p = 0; p < n; ++p) Mp[p] = 0;
          for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
            const int km = N - 1 - k;
            const C pk = P[k], pm = P[km], lk = L[k], lm = L[km];
            C yk = pm, uk = lm, ym = pk, um = lk;
            if (Ly.has_phase) {
              const C phk = diag_phase<R>(cf, Ly.tb, k), phm = diag_phase<R>(cf, Ly.tb, km);
              yk = cmulc<R>(phk, pm); uk = cmulc<R>(phk, lm);
              ym = cmulc<R>(phm, pk); um = cmulc<R>(phm, lk);
            }
            P[k] = yk; L[k] = uk; P[km] = ym; L[km] = um;
            if (Ly.slot >= 0) {
              const double wk = (double)im_cdot<R>(uk, yk), wm = (double)im_cdot<R>(um, ym);
              W += wk + wm;
              for (int p = 0; p < n; ++p) {
                if ((k >> p) & 1) Mp[p] += wk;
                if ((km >> p) & 1) Mp[p] += wm;
              }
            }
          }
          if (Ly.slot >= 0) {
            double Wt = block_sum(W, red);
            for (int p = 0; p < n; ++p) {
              double s = block_sum(Mp[p], red);
              if (threadIdx.x == 0) marg[p] = s;
            }
            __syncthreads();
            for (int j = threadIdx.x; j < n; j += blockDim.x)
              part[(long long)(Ly.slot + j) * batch + b] = Ly.gscale * (Wt - 2.0 * marg[n - 1 - j]);
          }
          __syncthreads();
        }
        break;
      }
      case LC_RING: {
        constexpr int kMaxPer = 32;  // N <= 8192 with 256 threads
        for (int s = 0; s < (BWD ? 2 : 1); ++s) {
          C* S = s ? L : P;
          C tmp[kMaxPer];
#pragma unroll
          for (int e = 0; e < kMaxPer; ++e) {
            const int k = threadIdx.x + e * kThreads;
            if (k < N) tmp[e] = S[BWD ? ring_f(k, n) : ring_finv(k, n)];
          }
          __syncthreads();
#pragma unroll
          for (int e = 0; e < kMaxPer; ++e) {
            const int k = threadIdx.x + e * kThreads;
            if (k < N) S[k] = tmp[e];
          }
          __syncthreads();
        }
        break;
      }
    }
  }

  if (!BWD) {
    if (psi_out)
      for (int i = threadIdx.x; i < N; i += blockDim.x) psi_out[sb + i] = P[i];
    if (ez) {
      double W = 0, Mp[kMaxQubits];
      for (int p = 0; p < n; ++p) Mp[p] = 0;
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const C x = P[k];
        const double w = (double)x.x * x.x + (double)x.y * x.y;
        W += w;
        for (int p = 0; p < n; ++p)
          if ((k >> p) & 1) Mp[p] += w;
      }
      double Wt = block_sum(W, red);
      for (int p = 0; p < n; ++p) {
        double s = block_sum(Mp[p], red);
        if (threadIdx.x == 0) marg[p] = s;
      }
      __syncthreads();
      for (int q = threadIdx.x; q < n; q += blockDim.x) ez[(long long)b * n + q] = Wt - 2.0 * marg[n - 1 - q];
    }
  }
  (void)nslots;
}

// ---------------------------------------------------------------------------
// Launch wrappers (host)
// ---------------------------------------------------------------------------
template <class R>
cudaError_t launch_coef(const CoefJob* jobs, int njobs, int n, int batch, int n_in, const double* x,
                        const double* theta, void* coef, cudaStream_t st) {
  if (njobs == 0) return cudaSuccess;
  dim3 grid(njobs, batch);
  k_coef<R><<<grid, 128, 0, st>>>(jobs, njobs, n, batch, n_in, x, theta, (R*)coef);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_prodvec(const ProdVecJob& P, int n, int batch, int n_in, const double* x,
                           const double* theta, void* pv, cudaStream_t st) {
  int tot = batch * n;
  k_prodvec<R><<<(tot + 127) / 128, 128, 0, st>>>(P, n, batch, n_in, x, theta, (R*)pv);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_prodinit(int n, int cb, int batch, const void* pv, void* psi,
                           const void* post_tabs, long long post_bstride, int post_tb,
                           int post_zmode, cudaStream_t st) {
  long long grid = (long long)batch << (n - cb);
  const size_t smem = post_tabs ? ((size_t)2 * sizeof(R)) << post_tb : 0;
  if (smem > 40 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_prodinit<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_prodinit<R><<<(unsigned)grid, kThreads, smem, st>>>(n, cb, (const R*)pv, (cx<R>*)psi,
                                                     (const R*)post_tabs, post_bstride, post_tb,
                                                     post_zmode);
  return cudaGetLastError();
}

#if QC_INST_R != 8
size_t tile_smem_bytes(const TilePass& P, int ns, int rsize) { return tile_smem_layout(P, ns, rsize).end; }
#endif

template <class R>
cudaError_t launch_tile(const TilePass& P, int rb, int ns, int batch, int cps, const void* coef,
                        const void* s0, void* d0, const void* s1, void* d1, double* part,
                        cudaStream_t st) {
  if (P.xload) return cudaErrorInvalidValue;  // complemented loads: TMA variants only
  if (ns == 1) return launch_tile_fwd<R>(P, rb, batch, cps, coef, s0, d0, s1, d1, part, st);
  return launch_tile_bwd<R>(P, rb, batch, cps, coef, s0, d0, s1, d1, part, st);
}

#if QC_INST_R != 8
long long diag_grid(const DiagPass& P, int batch) {
  long long nch = 1LL << (P.n - P.cb);
  long long cpb = P.xcomp ? (nch > 1 ? nch / 2 : 1) : nch;
  return cpb * batch;
}
#endif

template <class R, int NS, int ZM, int XC, int JB>
static cudaError_t launch_diag_jb(const DiagPass& P, int batch, const void* coef, const void* s0,
                                  void* d0, const void* s1, void* d1, double* part,
                                  cudaStream_t st) {
  size_t smem = NS == 2 ? (size_t)P.nvals * kWarps * sizeof(R) : 0;
  auto kern = k_diag<R, NS, ZM, XC, JB>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<(unsigned)diag_grid(P, batch), kThreads, smem, st>>>(P, (const R*)coef, (const cx<R>*)s0,
                                                              (cx<R>*)d0, (const cx<R>*)s1,
                                                              (cx<R>*)d1, part);
  return cudaGetLastError();
}

template <class R, int NS, int ZM, int XC>
static cudaError_t launch_diag_z(const DiagPass& P, int batch, const void* coef, const void* s0,
                                 void* d0, const void* s1, void* d1, double* part, cudaStream_t st) {
  const int jb = P.cb > 8 ? P.cb - 8 : 0;
  switch (jb) {
    case 0: return launch_diag_jb<R, NS, ZM, XC, 0>(P, batch, coef, s0, d0, s1, d1, part, st);
    case 1: return launch_diag_jb<R, NS, ZM, XC, 1>(P, batch, coef, s0, d0, s1, d1, part, st);
    case 2: return launch_diag_jb<R, NS, ZM, XC, 2>(P, batch, coef, s0, d0, s1, d1, part, st);
    case 3: return launch_diag_jb<R, NS, ZM, XC, 3>(P, batch, coef, s0, d0, s1, d1, part, st);
    case 4: return launch_diag_jb<R, NS, ZM, XC, 4>(P, batch, coef, s0, d0, s1, d1, part, st);
    case 5: return launch_diag_jb<R, NS, ZM, XC, 5>(P, batch, coef, s0, d0, s1, d1, part, st);
    case 6: return launch_diag_jb<R, NS, ZM, XC, 6>(P, batch, coef, s0, d0, s1, d1, part, st);
  }
  return cudaErrorInvalidValue;
}

template <class R>
cudaError_t launch_diag(const DiagPass& P, int ns, int batch, const void* coef, const void* s0,
                        void* d0, const void* s1, void* d1, double* part, cudaStream_t st) {
  if (P.xcomp) {
    if (ns == 1) return launch_diag_z<R, 1, Z_IDENT, 1>(P, batch, coef, s0, d0, s1, d1, part, st);
    return launch_diag_z<R, 2, Z_IDENT, 1>(P, batch, coef, s0, d0, s1, d1, part, st);
  }
  if (P.zmode == Z_RINGXOR) {
    if (ns == 1) return launch_diag_z<R, 1, Z_RINGXOR, 0>(P, batch, coef, s0, d0, s1, d1, part, st);
    return launch_diag_z<R, 2, Z_RINGXOR, 0>(P, batch, coef, s0, d0, s1, d1, part, st);
  }
  if (ns == 1) return launch_diag_z<R, 1, Z_IDENT, 0>(P, batch, coef, s0, d0, s1, d1, part, st);
  return launch_diag_z<R, 2, Z_IDENT, 0>(P, batch, coef, s0, d0, s1, d1, part, st);
}

#if QC_INST_R != 8
size_t ring_smem_bytes(const RingPass& P, int rsize) {
  size_t amps = P.whole ? ((size_t)1 << P.n) : ((size_t)1 << P.t);
  return amps * 2 * rsize * (P.pre ? 2 : 1);  // both states with a fused diagonal
}
#endif

template <class R>
cudaError_t launch_ring(const RingPass& P, int ns, int batch, const void* s0, void* d0,
                        const void* s1, void* d1, const double* gez, const void* coef, double* part,
                        cudaStream_t st) {
  size_t smem = ring_smem_bytes(P, sizeof(R));
  long long grid = P.whole ? batch : ((long long)batch << (P.n - P.t));
  if (ns == 1) {
    auto kern = k_ring<R, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, kThreads, smem, st>>>(P, (const cx<R>*)s0, (cx<R>*)d0, nullptr, nullptr,
                                                 nullptr, (const R*)coef, part);
  } else {
    auto kern = k_ring<R, 2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, kThreads, smem, st>>>(P, (const cx<R>*)s0, (cx<R>*)d0, (const cx<R>*)s1,
                                                 (cx<R>*)d1, gez, (const R*)coef, part);
  }
  return cudaGetLastError();
}

template <class R, int JB>
static cudaError_t launch_expect_jb(int n, int cb, int batch, const void* psi, double* part,
                                    cudaStream_t st) {
  size_t smem = (size_t)(n + 1) * kThreads * sizeof(double);
  auto kern = k_expect<R, JB>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  long long grid = (long long)batch << (n - cb);
  kern<<<(unsigned)grid, kThreads, smem, st>>>(n, cb, (const cx<R>*)psi, part);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_expect(int n, int cb, int batch, const void* psi, double* part, double* ez,
                          cudaStream_t st) {
  const int jb = cb > 8 ? cb - 8 : 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (jb) {
    case 0: e = launch_expect_jb<R, 0>(n, cb, batch, psi, part, st); break;
    case 1: e = launch_expect_jb<R, 1>(n, cb, batch, psi, part, st); break;
    case 2: e = launch_expect_jb<R, 2>(n, cb, batch, psi, part, st); break;
    case 3: e = launch_expect_jb<R, 3>(n, cb, batch, psi, part, st); break;
    case 4: e = launch_expect_jb<R, 4>(n, cb, batch, psi, part, st); break;
    case 5: e = launch_expect_jb<R, 5>(n, cb, batch, psi, part, st); break;
    case 6: e = launch_expect_jb<R, 6>(n, cb, batch, psi, part, st); break;
  }
  if (e != cudaSuccess) return e;
  long long nblk = (long long)batch << (n - cb);
  k_ez_from_marg<<<batch * n, kThreads, 0, st>>>(n, 1 << (n - cb), nblk, part, ez);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_laminit(int n, int cb, int batch, const double* gez, const void* psi, void* lam,
                           cudaStream_t st) {
  long long grid = (long long)batch << (n - cb);
  k_laminit<R><<<(unsigned)grid, kThreads, 0, st>>>(n, cb, gez, (const cx<R>*)psi, (cx<R>*)lam);
  return cudaGetLastError();
}

#if QC_INST_R != 8
cudaError_t launch_reduce(const RedJob* jobs, const long long* row0, const int* out0, int njobs,
                          long long rowbase, long long nrows, int outbase, int nout,
                          const RedOut* outs, int batch, int n_in, const double* part, double* V,
                          double* d_theta, double* d_x, cudaStream_t st) {
  if (njobs == 0) return cudaSuccess;
  k_red1<<<(unsigned)((nrows + kWarps - 1) / kWarps), kThreads, 0, st>>>(jobs, row0, njobs, rowbase, nrows,
                                                                        part, V);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // four warps (outputs) per block
  k_finalize<<<(nout + 3) / 4, 128, 0, st>>>(jobs, row0, out0, njobs, outbase, nout, outs, batch, n_in, V,
                                             d_theta, d_x);
  return cudaGetLastError();
}
#endif

#if QC_INST_R != 8
// Plan tables are written into the caller's workspace by this kernel: the
// bytes travel in the kernel's parameter block, so the copy is ordered on the
// stream like any launch and needs neither a device allocation nor a host
// synchronisation.
static __global__ void __launch_bounds__(kThreads) k_upload(const __grid_constant__ UploadChunk U,
                                                          unsigned char* __restrict__ dst) {
  const uint4* src = reinterpret_cast<const uint4*>(U.data);
  uint4* d = reinterpret_cast<uint4*>(dst + U.off);
  for (unsigned i = threadIdx.x; i < U.n / 16; i += blockDim.x) d[i] = src[i];
}

cudaError_t launch_upload(const void* host, size_t bytes, void* dst, cudaStream_t st) {
  const unsigned char* h = static_cast<const unsigned char*>(host);
  for (size_t o = 0; o < bytes; o += kUploadBytes) {
    UploadChunk U;
    const size_t k = bytes - o < kUploadBytes ? bytes - o : kUploadBytes;
    U.off = o;
    U.n = (unsigned)((k + 15) & ~(size_t)15);
    memcpy(U.data, h + o, k);
    if (U.n > k) memset(U.data + k, 0, U.n - k);
    k_upload<<<1, kThreads, 0, st>>>(U, static_cast<unsigned char*>(dst));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
#endif

// Loads the <Z> kernels of an n-qubit circuit into the current context (with
// lazy module loading a kernel's code is otherwise loaded, which may allocate,
// at its first launch).
template <class R>
cudaError_t preload_expect(int n) {
  const int cb = n < 14 ? n : 14;
  const int jb = cb > 8 ? cb - 8 : 0;
  cudaFuncAttributes a;
  cudaError_t e = cudaErrorInvalidValue;
  switch (jb) {
    case 0: e = cudaFuncGetAttributes(&a, k_expect<R, 0>); break;
    case 1: e = cudaFuncGetAttributes(&a, k_expect<R, 1>); break;
    case 2: e = cudaFuncGetAttributes(&a, k_expect<R, 2>); break;
    case 3: e = cudaFuncGetAttributes(&a, k_expect<R, 3>); break;
    case 4: e = cudaFuncGetAttributes(&a, k_expect<R, 4>); break;
    case 5: e = cudaFuncGetAttributes(&a, k_expect<R, 5>); break;
    case 6: e = cudaFuncGetAttributes(&a, k_expect<R, 6>); break;
  }
  if (e != cudaSuccess) return e;
  return cudaFuncGetAttributes(&a, k_ez_from_marg);
}

#if QC_INST_R != 8
size_t smem_circuit_bytes(int n, int bwd, int rsize) {
  size_t amps = (size_t)1 << n;
  return amps * 2 * rsize * (bwd ? 2 : 1) + (kWarps + kMaxQubits + 1) * sizeof(double);
}
#endif

template <class R>
cudaError_t launch_smem(const SmemLayer* prog, int nl, int n, int batch, int bwd, const void* coef,
                        const void* psi_in, void* psi_out, double* ez, const double* gez,
                        double* part, int nslots, cudaStream_t st) {
  size_t smem = smem_circuit_bytes(n, bwd, sizeof(R));
  if (!bwd) {
    auto kern = k_smem<R, 0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<batch, kThreads, smem, st>>>(prog, nl, n, batch, (const R*)coef, (const cx<R>*)psi_in,
                                        (cx<R>*)psi_out, ez, gez, part, nslots);
  } else {
    auto kern = k_smem<R, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<batch, kThreads, smem, st>>>(prog, nl, n, batch, (const R*)coef, (const cx<R>*)psi_in,
                                        (cx<R>*)psi_out, ez, gez, part, nslots);
  }
  return cudaGetLastError();
}

#define QC_INST(R)                                                                                 \
  template cudaError_t launch_coef<R>(const CoefJob*, int, int, int, int, const double*,           \
                                      const double*, void*, cudaStream_t);                         \
  template cudaError_t launch_prodvec<R>(const ProdVecJob&, int, int, int, const double*,          \
                                         const double*, void*, cudaStream_t);                      \
  template cudaError_t launch_prodinit<R>(int, int, int, const void*, void*, const void*,          \
                                          long long, int, int, cudaStream_t);                      \
  template cudaError_t launch_tile<R>(const TilePass&, int, int, int, int, const void*,           \
                                      const void*, void*, const void*, void*, double*,             \
                                      cudaStream_t);                                               \
  template cudaError_t launch_diag<R>(const DiagPass&, int, int, const void*, const void*, void*,  \
                                      const void*, void*, double*, cudaStream_t);                  \
  template cudaError_t launch_ring<R>(const RingPass&, int, int, const void*, void*, const void*,  \
                                      void*, const double*, const void*, double*, cudaStream_t);   \
  template cudaError_t launch_expect<R>(int, int, int, const void*, double*, double*,              \
                                        cudaStream_t);                                             \
  template cudaError_t preload_expect<R>(int);                                                     \
  template cudaError_t launch_laminit<R>(int, int, int, const double*, const void*, void*,         \
                                         cudaStream_t);                                            \
  template cudaError_t launch_smem<R>(const SmemLayer*, int, int, int, int, const void*,           \
                                      const void*, void*, double*, const double*, double*, int,    \
                                      cudaStream_t);

#if QC_INST_R != 8
QC_INST(float)
#endif
#if QC_INST_R != 4
QC_INST(double)
#endif

}  // namespace qc
