// Gate matrices (Appendix A of arXiv 2506.04891) and their parameter
// derivatives, evaluated in float64 on the device.  Matrices are row-major;
// for two-qubit gates the first qubit of the pair is the more significant
// index of the 4x4 matrix.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "../../include/qlayer.h"

namespace qc {

struct dc {
  double x, y;
};

__device__ __forceinline__ dc dmk(double a, double b) { return dc{a, b}; }
__device__ __forceinline__ dc dmul(dc a, dc b) { return dc{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ dc dadd(dc a, dc b) { return dc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dc dconj(dc a) { return dc{a.x, -a.y}; }
__device__ __forceinline__ dc dscale(dc a, double s) { return dc{a.x * s, a.y * s}; }
// exp(i a)
__device__ __forceinline__ dc dexpi(double a) {
  double s, c;
  sincos(a, &s, &c);
  return dc{c, s};
}

constexpr double kPi = 3.14159265358979323846;
constexpr double kInvSqrt2 = 0.70710678118654752440;

// Single-qubit gate matrix M(t) of a layer kind.
__device__ inline void gate1q(int kind, double t, dc M[4]) {
  switch (kind) {
    case QC_L_RX: {
      double s, c;
      sincos(0.5 * t, &s, &c);
      M[0] = dmk(c, 0); M[1] = dmk(0, -s); M[2] = dmk(0, -s); M[3] = dmk(c, 0);
      break;
    }
    case QC_L_RY: {
      double s, c;
      sincos(0.5 * t, &s, &c);
      M[0] = dmk(c, 0); M[1] = dmk(-s, 0); M[2] = dmk(s, 0); M[3] = dmk(c, 0);
      break;
    }
    case QC_L_RZ:
      M[0] = dexpi(-0.5 * t); M[1] = dmk(0, 0); M[2] = dmk(0, 0); M[3] = dexpi(0.5 * t);
      break;
    case QC_L_SX:
      M[0] = dmk(0.5, 0.5); M[1] = dmk(0.5, -0.5); M[2] = dmk(0.5, -0.5); M[3] = dmk(0.5, 0.5);
      break;
    case QC_L_GPI:
      M[0] = dmk(0, 0); M[1] = dexpi(-2.0 * kPi * t); M[2] = dexpi(2.0 * kPi * t); M[3] = dmk(0, 0);
      break;
    case QC_L_GPI2: {
      dc em = dexpi(-2.0 * kPi * t), ep = dexpi(2.0 * kPi * t);
      // -i e = (e.y, -e.x)
      M[0] = dmk(kInvSqrt2, 0);
      M[1] = dscale(dmk(em.y, -em.x), kInvSqrt2);
      M[2] = dscale(dmk(ep.y, -ep.x), kInvSqrt2);
      M[3] = dmk(kInvSqrt2, 0);
      break;
    }
    case QC_L_X:
      M[0] = dmk(0, 0); M[1] = dmk(1, 0); M[2] = dmk(1, 0); M[3] = dmk(0, 0);
      break;
    case QC_L_Z:
      M[0] = dmk(1, 0); M[1] = dmk(0, 0); M[2] = dmk(0, 0); M[3] = dmk(-1, 0);
      break;
    case QC_L_S:
      M[0] = dmk(1, 0); M[1] = dmk(0, 0); M[2] = dmk(0, 0); M[3] = dmk(0, 1);
      break;
    case QC_L_H:
      M[0] = dmk(kInvSqrt2, 0); M[1] = dmk(kInvSqrt2, 0); M[2] = dmk(kInvSqrt2, 0); M[3] = dmk(-kInvSqrt2, 0);
      break;
    default:
      M[0] = dmk(1, 0); M[1] = dmk(0, 0); M[2] = dmk(0, 0); M[3] = dmk(1, 0);
  }
}

// dM/dt of a parametrised single-qubit gate (zero for fixed gates).
__device__ inline void dgate1q(int kind, double t, dc D[4]) {
  D[0] = D[1] = D[2] = D[3] = dmk(0, 0);
  switch (kind) {
    case QC_L_RX: {
      double s, c;
      sincos(0.5 * t, &s, &c);
      D[0] = dmk(-0.5 * s, 0); D[1] = dmk(0, -0.5 * c); D[2] = dmk(0, -0.5 * c); D[3] = dmk(-0.5 * s, 0);
      break;
    }
    case QC_L_RY: {
      double s, c;
      sincos(0.5 * t, &s, &c);
      D[0] = dmk(-0.5 * s, 0); D[1] = dmk(-0.5 * c, 0); D[2] = dmk(0.5 * c, 0); D[3] = dmk(-0.5 * s, 0);
      break;
    }
    case QC_L_RZ: {
      dc a = dexpi(-0.5 * t), b = dexpi(0.5 * t);
      D[0] = dmul(dmk(0, -0.5), a); D[3] = dmul(dmk(0, 0.5), b);
      break;
    }
    case QC_L_GPI: {
      const double w = 2.0 * kPi;
      dc em = dexpi(-w * t), ep = dexpi(w * t);
      D[1] = dmul(dmk(0, -w), em); D[2] = dmul(dmk(0, w), ep);
      break;
    }
    case QC_L_GPI2: {
      const double w = 2.0 * kPi;
      dc em = dexpi(-w * t), ep = dexpi(w * t);
      // d/dt of -i e^{-iwt} = -i (-i w) e^{-iwt} = -w e^{-iwt}; of -i e^{iwt} = w e^{iwt}
      D[1] = dscale(em, -w * kInvSqrt2);
      D[2] = dscale(ep, w * kInvSqrt2);
      break;
    }
    default:
      break;
  }
}

// A = M^dagger D (the generator whose expectation gives the gradient).
__device__ inline void mdag_mul(const dc* M, const dc* D, dc* A, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      dc s = dmk(0, 0);
      for (int k = 0; k < d; ++k) s = dadd(s, dmul(dconj(M[k * d + i]), D[k * d + j]));
      A[i * d + j] = s;
    }
}

// Molmer-Sorensen gate with the (3,0) entry conjugated (the printed matrix
// repeats the (0,3) phase there and is not unitary).
__device__ inline void gate_ms(double p0, double p1, double th, dc M[16]) {
  for (int i = 0; i < 16; ++i) M[i] = dmk(0, 0);
  double s, c;
  sincos(kPi * th, &s, &c);
  const double w = 2.0 * kPi;
  M[0] = M[5] = M[10] = M[15] = dmk(c, 0);
  dc mis = dmk(0, -s);
  M[0 * 4 + 3] = dmul(mis, dexpi(-w * (p0 + p1)));
  M[1 * 4 + 2] = dmul(mis, dexpi(-w * (p1 - p0)));
  M[2 * 4 + 1] = dmul(mis, dexpi(-w * (p0 - p1)));
  M[3 * 4 + 0] = dmul(mis, dexpi(+w * (p0 + p1)));
}

// d MS / d(which), which = 0: phi0, 1: phi1, 2: theta.
__device__ inline void dgate_ms(double p0, double p1, double th, int which, dc D[16]) {
  for (int i = 0; i < 16; ++i) D[i] = dmk(0, 0);
  double s, c;
  sincos(kPi * th, &s, &c);
  const double w = 2.0 * kPi;
  dc e03 = dexpi(-w * (p0 + p1)), e12 = dexpi(-w * (p1 - p0));
  dc e21 = dexpi(-w * (p0 - p1)), e30 = dexpi(+w * (p0 + p1));
  if (which == 2) {
    D[0] = D[5] = D[10] = D[15] = dmk(-kPi * s, 0);
    dc mic = dmk(0, -kPi * c);
    D[3] = dmul(mic, e03); D[6] = dmul(mic, e12); D[9] = dmul(mic, e21); D[12] = dmul(mic, e30);
    return;
  }
  // the phase exponent of each entry is +-w * (linear in phi); derivative = (i * dexp) * entry
  double k03 = -w, k12 = (which == 0) ? w : -w, k21 = (which == 0) ? -w : w, k30 = w;
  dc mis = dmk(0, -s);
  D[3] = dmul(dmul(mis, e03), dmk(0, k03));
  D[6] = dmul(dmul(mis, e12), dmk(0, k12));
  D[9] = dmul(dmul(mis, e21), dmk(0, k21));
  D[12] = dmul(dmul(mis, e30), dmk(0, k30));
}

// CZ = diag(1, 1, 1, -1); SWAP exchanges |01> and |10> (Appendix A).
__device__ inline void gate_cz(dc M[16]) {
  for (int i = 0; i < 16; ++i) M[i] = dmk(0, 0);
  M[0] = dmk(1, 0); M[5] = dmk(1, 0); M[10] = dmk(1, 0); M[15] = dmk(-1, 0);
}
__device__ inline void gate_swap(dc M[16]) {
  for (int i = 0; i < 16; ++i) M[i] = dmk(0, 0);
  M[0 * 4 + 0] = dmk(1, 0); M[1 * 4 + 2] = dmk(1, 0); M[2 * 4 + 1] = dmk(1, 0); M[3 * 4 + 3] = dmk(1, 0);
}

// ECR = (I (x) X - X (x) Y) / sqrt(2), first qubit the left factor.
__device__ inline void gate_ecr(dc M[16]) {
  for (int i = 0; i < 16; ++i) M[i] = dmk(0, 0);
  const double r = kInvSqrt2;
  M[0 * 4 + 1] = dmk(r, 0);  M[0 * 4 + 3] = dmk(0, r);
  M[1 * 4 + 0] = dmk(r, 0);  M[1 * 4 + 2] = dmk(0, -r);
  M[2 * 4 + 1] = dmk(0, r);  M[2 * 4 + 3] = dmk(r, 0);
  M[3 * 4 + 0] = dmk(0, -r); M[3 * 4 + 2] = dmk(r, 0);
}

}  // namespace qc
