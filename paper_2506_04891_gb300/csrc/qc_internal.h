// Internal descriptors shared by the host planner (qc_api.cu) and the kernels
// (qc_kernels.cu).  Plain structs: they are passed to kernels by value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qlayer.h"

namespace qc {

constexpr int kMaxQubits = 30;
constexpr int kThreads = 256;        // block size of every pass kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxTileOps = 48;      // gate ops in one tile pass
constexpr int kMaxRounds = 8;
constexpr int kDiagTables = 3;       // diagonal phase = T0[z0] * T1[z1] * T2[z2]

// Layer classes: how a layer is applied.
enum LayerClass {
  LC_ROT1 = 0,    // non-diagonal single-qubit gate on every qubit (RX, RY, SX, GPI2)
  LC_DIAG = 1,    // diagonal phase (RZ, ISINGZZ_RING)
  LC_RING = 2,    // CNOT ring permutation
  LC_XCOMP = 3,   // index complement k -> ~k with an optional phase (X, GPI)
  LC_DENSE2 = 4,  // two-qubit gates on a brick of qubit pairs (MS, ECR)
};

// z-transform of a diagonal layer: the phase is a product over the bits of z(k).
enum ZMode { Z_IDENT = 0, Z_RINGXOR = 1 };

// Coefficient records, in units of the state's real type R.
constexpr int kRec1q = 20;    // M (2x2 complex) + A = M^dagger dM (2x2 complex) + the real parts
                              // of M packed (m00, m01, m10, m11) at kRealOff
constexpr int kRealOff = 16;
// two-qubit record: M (4x4 complex, 32 R), then for MS the phases e_r of its
// generator K (K[r][r ^ 3] = e_r, M = cos(pi theta) I - i sin(pi theta) K;
// 4 complex, 8 R) and the three A = M^dagger dM (4x4 complex each)
constexpr int kRec2q = 136;
constexpr int kRec2qK = 32;   // offset of the generator phases
constexpr int kRec2qA = 40;   // offset of the first A

struct LayerInfo {
  int kind, source, offset, parity;
  int cls;
  int nparams;          // parameters read (0 if unparametrised)
  int ngates;           // 1q: n; dense2: pairs; diag/xcomp: n phase bits
  int diff;             // source is THETA or INPUT
  int per_sample;       // source is INPUT
  int real;             // ROT1 with a real matrix (RY)
  int zmode;            // DIAG: ZMode
  int has_phase;        // XCOMP: GPI has a phase, X none
  double gscale;        // DIAG/XCOMP gradient g_j = gscale * (W - 2 M_{zbit(j)})
  // device coefficient placement (R units, relative to the coefficient base)
  long long coef_off;
  long long coef_bstride;   // per-sample stride (0 when shared)
  int tb;                   // DIAG/XCOMP: bits per table (tables of 2^tb complex)
  int pstride;              // parameter j of the layer is offset + pstride * j (1, or 3 for
                            // the layers a Rot layer expands into)
  int rot_phase;            // RZ part of a Rot: the phase tables carry e^{i(phi+lambda)/2},
                            // lambda = parameter offset + pstride * j + 1
};

// One gate op inside a tile pass.
struct TileOp {
  int16_t l;        // local bit (1q) or lower local bit of the pair (2q)
  int8_t is2q;
  int8_t real;      // 1q with a real matrix
  int8_t gk;        // 1q generator: 0 generic A, 1 A = -i/2 X (RX), 2 A = -i/2 Y (RY)
  int8_t ck;        // companion generator (1q): 0 none, 1 X, 2 Y -- the gradient of the
                    // preceding RX / RY layer's gate on the same qubit, taken on the
                    // states between the two layers
  int16_t np;       // gradient parameters produced (0, 1 or 3)
  int16_t slot;     // first gradient slot in the pass's partial vector
  int16_t cslot;    // companion gradient slot (ck != 0)
  int16_t pat;      // 2q: nonzero pattern of the gate matrix, 0 columns r ^ {0, 3}, 1 r ^ {1, 3}
  int32_t soff;     // offset of the op's coefficients in the staged smem block (R units)
  int32_t nco;      // number of R to stage
  long long coef;   // coefficient offset (R units) for sample 0
  long long bstride;// per-sample stride (0 = shared)
};

// A tile pass: the CTA loads 2^t amplitudes whose local bit l maps to global bit
// l (l < c) or h0 + (l - c) (l >= c), applies rounds of register-blocked gate
// ops, and stores them back.
struct TilePass {
  int n, t, c, h0;
  int nrounds;
  int8_t rlo[kMaxRounds];            // round r: register bits [rlo[r], rlo[r] + RB)
  int16_t rop[kMaxRounds + 1];       // ops of round r: [rop[r], rop[r+1])
  int nops;
  int nstage;                        // shared-memory tile buffers (2 or 3)
  int nslots;                        // gradient slots (bwd)
  int ncomp;                         // companion slots: the last ncomp of the nslots
  int store;                         // 0: gradient only, no store
  int ncoef;                         // R units of staged coefficients
  // deferred gradient reduction: the per-thread FP32 sums of every slot stay
  // on the SM until the CTA's last tile and are then reduced in FP64 once.
  // 1 (single-qubit ops only, <= 4 rounds): own slots in registers, rslot /
  // rcslot give the slot of the op on register bit i of round r and of its
  // companion (-1 if none), companions in shared memory ([ncomp][kThreads] R);
  // 2 (any pass whose sums fit): every slot in shared memory
  // ([nslots][kThreads] R); 0: each round reduces its sums in FP64.
  int defer;
  int16_t rslot[4][4];
  int16_t rcslot[4][4];
  // op on register bit i of round r (lower bit for two-qubit ops), -1 if none
  int8_t rbit[kMaxRounds][5];
  int kind;                          // 0: complex 1q, 1: real 1q, 2: two-qubit (uniform per pass)
  int rb;                            // register bits per round the rounds were planned for
  int sx;                            // 1: constant SX layer without companions (TMA: additions-only variant)
  int xload;                         // 1: an X layer (k -> ~k) fused into the loads: tile element k
                                     //    is read from index ~k (not with gather or scatter)
  // fused neighbours (forward unless noted)
  int gather;        // 1: load psi[f^-1(k)] (a CNOT ring applied before this pass's gates)
  int scatter;       // 1: store to f^-1(k) (backward: inverse CNOT ring after this pass)
  int pre, post;     // 1: multiply by a diagonal phase before / after the gates
  int pre_zmode, post_zmode, pre_tb, post_tb;
  long long pre_coef, pre_bstride, post_coef, post_bstride;
  // backward pre (contiguous first pass, round 0 at register bits 0..RB-1):
  // undo a diagonal layer on psi and lambda and write its bit marginals
  // [W, M_0 .. M_{n-1}] per CTA to part[pre_moff + v * grid + block]
  int pre_grad;
  long long pre_moff;
  TileOp ops[kMaxTileOps];
};

// Forward pass whose post phase (a following diagonal layer) takes the
// compile-time element patterns: a contiguous 2^12 tile (c = t) whose last
// register round holds index bits 8 .. 11 (4 register bits), ring or
// identity z map.
__host__ __device__ inline bool fwd_post_contig(const TilePass& P) {
  return P.t == 12 && P.c == 12 && P.nrounds >= 1 && P.nrounds <= kMaxRounds &&
         P.rlo[P.nrounds - 1] == 8 && (P.post_zmode == Z_IDENT || P.post_zmode == Z_RINGXOR);
}

// Resident CTAs per SM a tile pass is compiled for (see the launch bounds of
// the tile kernel): the complex64 real-gate forward pass 3, others 2 (a
// fused-diagonal backward pass at one CTA per SM without spills measured
// slower than two with some).
inline int tile_resident(int rsize, int kind, int ns, int pre) {
  (void)pre;
  return (rsize == 4 && kind == 1 && ns == 1) ? 3 : 2;
}

// Shared-memory carve-out of a tile pass, in bytes from the dynamic base, used
// by the kernel and by the launch size alike: tile buffers, staged
// coefficients, per-warp gradient sums, per-thread deferred companion sums
// (backward, deferred), backward pre-diagonal marginals and phase-ratio table,
// end.  Every block starts on a 16-byte boundary.
struct TileSmem {
  size_t buf, sco, sred, sdef, smarg, sratio, smacc, fph, end;
};
// backward pre-diagonal: per-thread running marginal sums kept in shared
// memory (W, up to 8 element-bit sums, up to 2 tile-and-lane bits, the lane's
// tile-only bit)
constexpr int kPreAcc = 12;
// Forward pre/post phase block (one per diagonal the pass multiplies in):
// element-varying z bits, the compressed pattern of each per-thread element,
// and the product of the per-bit phase ratios for every pattern.
constexpr int kFphMaxSE = 8;
struct FwdPhaseMeta {
  int ok;      // 0: the tile has more than 16 elements per thread or 8 such bits
  int nse, semask;
  int sepos[kFphMaxSE];
  int patk[16];
};
constexpr size_t kFphBytes(int rsize) {
  return ((sizeof(FwdPhaseMeta) + 15) & ~(size_t)15) + (size_t)(1 << kFphMaxSE) * 2 * rsize;
}
__host__ __device__ inline size_t tsm_align16(size_t x) { return (x + 15) & ~(size_t)15; }
// per-thread deferred sums a backward pass keeps in shared memory
__host__ __device__ inline int tile_defer_slots(const TilePass& P) {
  return P.defer == 1 ? P.ncomp : P.defer == 2 ? P.nslots : 0;
}
__host__ __device__ inline TileSmem tile_smem_layout(const TilePass& P, int ns, int rsize) {
  TileSmem L;
  L.buf = 0;
  L.sco = tsm_align16(L.buf + (size_t)P.nstage * ns * ((size_t)1 << P.t) * 2 * rsize);
  L.sred = tsm_align16(L.sco + (size_t)P.ncoef * rsize);
  L.sdef = tsm_align16(L.sred + (size_t)kWarps * (P.nslots > 0 ? P.nslots : 1) * sizeof(double));
  L.smarg = tsm_align16(L.sdef + (ns == 2 ? (size_t)tile_defer_slots(P) * kThreads * rsize : 0));
  const bool pre = ns == 2 && P.pre;
  L.sratio = tsm_align16(L.smarg + (pre ? (size_t)kWarps * (P.n + 1) * sizeof(double) : 0));
  L.smacc = L.sratio;
  L.fph = tsm_align16(L.smacc + (pre ? (size_t)kPreAcc * kThreads * rsize : 0));
  const size_t nfph = ns == 1 ? (size_t)(P.pre ? 1 : 0) + (P.post ? 1 : 0) : (pre ? 1 : 0);
  L.end = tsm_align16(L.fph + nfph * kFphBytes(rsize));
  return L;
}

// Diagonal / complement pass (elementwise).
struct DiagPass {
  int n;
  int cb;            // chunk bits (CTA handles 2^cb contiguous amplitudes)
  int zmode;         // ZMode
  int xcomp;         // 1: out[k] = phase(~k) * in[~k]
  int has_phase;
  int tb;            // bits per table
  long long coef;    // table offset (R units)
  long long bstride; // per-sample stride of the tables
  int nvals;         // bwd: 1 + n marginal values
};

struct RingPass {
  int n;
  int t;             // CTA covers 2^t amplitudes (two halves of 2^(t-1))
  int whole;         // 1: whole state per CTA (n <= t)
  // backward, a tile (or whole state) of 2^10 .. 2^13 amplitudes: a diagonal
  // layer with the identity z map undone on psi and lambda before the
  // permutation, and
  // (pre_grad) its bit marginals [W, M_0 .. M_{n-1}] per CTA written to
  // part[v * grid + block]
  int pre, pre_grad, pre_tb;
  long long pre_coef, pre_bstride;
};

// Reduction of per-CTA partials into parameter gradients.
enum RedKind { RK_DIRECT = 0, RK_MARGINAL = 1 };
struct RedJob {
  long long part_off;  // offset (doubles) of the launch's partials, layout [nvals][nblk]
  int nblk;            // CTAs of the launch
  int nvals;
  int blk_per_sample;
  int kind;            // RedKind
  int nout;            // gradient outputs of the job
  int source;          // QC_SRC_THETA or QC_SRC_INPUT
  int out_off;         // index of output 0 in theta / x[b]
  int first;           // index of this job's first entry in the per-output map
  int per_sample_out;  // 1 when every sample's CTA set must be reduced separately
};
// Per-output map entry: RK_DIRECT: value index; RK_MARGINAL: z-bit and scale.
struct RedOut {
  int val;             // DIRECT: value index; MARGINAL: z-bit p (value 1 + p)
  int pidx;            // index in theta (THETA) or x[b] (INPUT)
  double scale;        // MARGINAL: g = scale * (V[0] - 2 V[1 + p]); DIRECT: g = scale * V[val]
};

// Whole-circuit-in-shared-memory program (one CTA per sample).
struct SmemLayer {
  int cls;
  int kind;
  int real;
  int zmode, has_phase, tb;
  int ngates, np_per_gate, parity;
  long long coef, bstride;
  int slot;          // first gradient slot (per-sample partial vector), -1 if none
  double gscale;
};

// One launch of the table-upload kernel: up to kUploadBytes bytes carried in
// the kernel's parameter block, written to dst + off (16-byte multiples).
constexpr size_t kUploadBytes = 16384;
struct UploadChunk {
  unsigned long long off;
  unsigned n;
  unsigned pad;
  alignas(16) unsigned char data[kUploadBytes];
};

// Shape of a circuit handle and the thread-local error message, for entry
// points defined outside qc_api.cu.
void circuit_shape(const qc_circuit* c, int* n, int* dtype);
qc_status set_error(qc_status s, const char* msg);
// qc_noalloc.cu: resolves the no-allocation scratch array's address and loads
// the <Z> kernels on the current device (best effort; errors are cleared)
void noalloc_prepare(int n, int dtype);
// counts a device allocation, free or device-wide synchronisation the
// library makes (diagnostics: qc_alloc_count)
void count_alloc();

}  // namespace qc
