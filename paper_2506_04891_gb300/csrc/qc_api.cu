// C ABI (include/qlayer.h): validation, per-layer planning, workspace layout
// and execution of the forward / <Z> / adjoint-backward kernel sequences.
//
// Planner (the GPU analogue of the paper's per-layer technique selection,
// Sec. 3): every layer class maps to the kernel that needs the fewest HBM
// passes for the qubit count at hand:
//   ROT1 / DENSE2 -> tile passes (2^t amplitudes staged in shared memory),
//                    ceil over the bit ranges that a tile can hold;
//   DIAG          -> one elementwise pass with factored phase tables
//                    (Diagonal Tensor Product, Sec. 2.4.2);
//   XCOMP         -> one elementwise pass over mirrored chunks (X, GPI: Sec. 2.4.1);
//   RING          -> one permutation pass with the closed-form index map (Sec. 2.3);
//   leading single-qubit layers -> one write-only product-state pass;
//   small n       -> the whole circuit of a sample in one CTA's shared memory.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "../../include/qlayer.h"
#include "qc_internal.h"
#include "qc_kernels.h"

using namespace qc;

namespace {

thread_local std::string g_last_error;

// ---- launch counting and optional per-launch event timing (diagnostics) ----
enum ProfClass {
  PC_COEF, PC_PRODINIT, PC_TILE_F, PC_TILE_B, PC_DIAG_F, PC_DIAG_B, PC_RING_F, PC_RING_B,
  PC_EXPECT, PC_LAMINIT, PC_REDUCE, PC_SMEM_F, PC_SMEM_B, PC_UPLOAD, PC_N
};
const char* kProfNames[PC_N] = {"coef", "prodinit", "tile_fwd", "tile_bwd", "diag_fwd", "diag_bwd",
                                "ring_fwd", "ring_bwd", "expect", "laminit", "reduce", "smem_fwd",
                                "smem_bwd", "upload"};
unsigned long long g_launches = 0;
bool g_prof = false;
struct ProfRec {
  int cls;
  double bytes;
  cudaEvent_t a, b;
};
std::vector<ProfRec> g_recs;
size_t g_nrec = 0;

struct ProfScope {
  ProfRec* r = nullptr;
  cudaStream_t st;
  int nl;
  ProfScope(int cls, double bytes, cudaStream_t s, int nlaunch = 1) : st(s), nl(nlaunch) {
    g_launches += nlaunch;
    if (!g_prof) return;
    if (g_nrec == g_recs.size()) {
      ProfRec x;
      x.cls = 0;
      x.bytes = 0;
      cudaEventCreate(&x.a);
      cudaEventCreate(&x.b);
      g_recs.push_back(x);
    }
    r = &g_recs[g_nrec++];
    r->cls = cls;
    r->bytes = bytes;
    cudaEventRecord(r->a, st);
  }
  ~ProfScope() {
    if (r) cudaEventRecord(r->b, st);
  }
};

qc_status fail(qc_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
qc_status cuda_fail(cudaError_t e, const char* where) {
  return fail(QC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

enum StepType { ST_PRODINIT, ST_TILE, ST_DIAG, ST_RING, ST_LAMINIT };
enum BufId { B_NONE = -1, B_PSIOUT = 0, B_RUN0 = 1, B_RUN1 = 2, B_LAM0 = 3, B_LAM1 = 4, B_CKPT = 16 };

struct Step {
  int type = ST_TILE;
  int ns = 1;
  int rb = 4;
  TilePass tp;
  DiagPass dp;
  RingPass rp;
  int cb = 12;
  int cps = 1;  // tile passes: CTAs per sample
  int s0 = B_NONE, d0 = B_NONE, s1 = B_NONE, d1 = B_NONE;
  long long part_off = 0;
  int layer = -1;
  int post_layer = -1;  // PRODINIT: diagonal layer applied to the product state
  long long post_coef = 0, post_bstride = 0;
  int post_tb = 0, post_zmode = 0;
  int laminit = 0;      // backward RING: lambda formed from psi (first backward step)
  int tma = 0;          // TILE: the TMA-staged kernel runs this pass
  int tc = 0;           // TILE: the tensor-core dense block runs this pass (experiment)
};

struct OutMap {
  int job;
  int val;
  int pidx;
  double scale;
};

struct Plan {
  int batch = 0;
  bool smem = false;
  bool unplaced = false;  // a gate found no round (invalid geometry): the plan is refused
  std::vector<Step> fwd, bwd;
  std::vector<CoefJob> coef_jobs;
  ProdVecJob pv{};
  int nlead = 0;
  int nckpt = 0;
  std::vector<int> ckpt_after;  // layer whose output each slot holds
  size_t S = 0;                 // bytes of one batch of states
  size_t coef_elems = 0;
  size_t off_coef = 0, off_pv = 0, off_run0 = 0, off_run1 = 0, off_lam0 = 0, off_lam1 = 0,
         off_ckpt = 0, off_part = 0, off_V = 0, ws_fwd = 0, ws_bwd = 0;
  size_t part_doubles = 0;
  // reductions
  std::vector<RedJob> jobs;
  std::vector<long long> row0;
  std::vector<OutMap> outs;
  long long nrows = 0;
  bool overlap = false;
  // whole-circuit program
  std::vector<SmemLayer> prog;
  int nslots = 0;
  // Device tables (coefficient jobs, reduction jobs and maps, the
  // whole-circuit program): one host blob that every call writes into the
  // first bytes of the caller's workspace (off_tables = 0) with the upload
  // kernel, so no call allocates device memory or waits on the host.
  std::vector<unsigned char> tables;
  size_t o_cj = 0, o_j = 0, o_r = 0, o_o0 = 0, o_ro = 0, o_pr = 0;
  unsigned long long last_use = 0;  // plan cache recency
  std::vector<std::vector<int>> job_groups;  // finalize groups (serial when outputs overlap)
};

// Device addresses of a plan's tables inside a workspace.
struct PlanDev {
  const CoefJob* coef_jobs;
  const RedJob* jobs;
  const long long* row0;
  const int* out0;
  const RedOut* outs;
  const SmemLayer* prog;
};
PlanDev plan_dev(const Plan& p, const char* ws) {
  PlanDev d;
  d.coef_jobs = reinterpret_cast<const CoefJob*>(ws + p.o_cj);
  d.jobs = reinterpret_cast<const RedJob*>(ws + p.o_j);
  d.row0 = reinterpret_cast<const long long*>(ws + p.o_r);
  d.out0 = reinterpret_cast<const int*>(ws + p.o_o0);
  d.outs = reinterpret_cast<const RedOut*>(ws + p.o_ro);
  d.prog = reinterpret_cast<const SmemLayer*>(ws + p.o_pr);
  return d;
}

// Device allocations, frees and device-wide synchronisations made by the
// library (diagnostics).  None is reachable from the compute calls after
// qc_create.
unsigned long long g_alloc_calls = 0;

}  // namespace

struct qc_circuit {
  int n = 0;
  qc_dtype dtype = QC_C64;
  int rsize = 4;
  qc_options opt{};
  std::vector<LayerInfo> layers;
  int n_theta = 0, n_in = 0;
  std::map<int, std::unique_ptr<Plan>> plans;  // host-only plans, at most kMaxPlans
  unsigned long long plan_clock = 0;
  // <Z> partial sums of qc_expect_z, allocated by qc_create: room for every
  // CTA of at least one sample; larger batches run in sample chunks
  void* exp_scratch = nullptr;
  size_t exp_scratch_bytes = 0;
  const void* last_ws = nullptr;
  int last_batch = -1;
};

namespace {

// Tile geometry: the circuit's options first, then the process-wide
// environment knobs QC_TMAX_FWD, QC_TMAX_BWD (tile bits), QC_RB_FWD,
// QC_RB_BWD (register bits per round), QC_TILE_STAGES (read once), then the
// defaults.  0 = unset.
int env_knob(const char* name) {
  const char* v = getenv(name);
  return v ? atoi(v) : 0;
}

// Largest tile (log2 amplitudes): two buffers of ns states must leave room
// for two CTAs per SM.
int tile_tmax(const qc_circuit* c, int ns) {
  if (ns == 1 && c->opt.tile_bits_fwd > 0) return c->opt.tile_bits_fwd;
  if (ns == 2 && c->opt.tile_bits_bwd > 0) return c->opt.tile_bits_bwd;
  // complex64 backward: 2^12 amplitudes of psi and lambda in one buffer (64 KB),
  // two CTAs per SM overlapping each other's copies (see tile_stages)
  if (c->dtype == QC_C64) return 12;
  return ns == 2 ? 10 : 11;
}

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      cached = v;
    else
      cached = 152;  // GB300; used when planning without a device
    cudaGetLastError();
  }
  return cached;
}

// CTAs per sample of a persistent tile pass.  The slots are the SMs times the
// pass's residency (its compiled CTAs per SM, fewer if its shared memory does
// not fit that many); each CTA walks its sample's tiles with a stride of the
// CTAs per sample c, so a pass takes about ceil(B c / slots) waves of
// ceil(tiles / c) tile times plus a per-CTA fixed cost (staging, the final
// reductions: about two tile times).  c minimises that: a batch that does not
// divide the slots would otherwise leave a nearly empty last wave (32
// samples: 288 CTAs, not 320 for 304 slots) or idle slots (200 samples of
// 2^24 amplitudes: three CTAs per sample in two full waves, 1.5x faster than
// one CTA per sample).
int tile_cps(int batch, int n, int t, int resident) {
  const long long tps = 1LL << (n - t);
  const long long slots = std::max<long long>(1, (long long)resident * sm_count());
  constexpr long long kCtaFixedTiles = 2;
  long long best = 1;
  long long best_cost = -1;
  const long long cmax = std::min<long long>(tps, 4096);
  for (long long c = 1; c <= cmax; ++c) {
    const long long waves = ((long long)batch * c + slots - 1) / slots;
    const long long cost = waves * ((tps + c - 1) / c + kCtaFixedTiles);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return (int)best;
}
int pass_cps(const qc_circuit* c, int batch, const TilePass& tp, int ns) {
  const int rs = (int)c->rsize;
  int res = tile_resident(rs, tp.kind, ns, ns == 2 && tp.pre);
  const size_t per_sm = 228 * 1024, per_cta_reserved = 1024;
  while (res > 1 && (size_t)res * (tile_smem_bytes(tp, ns, rs) + per_cta_reserved) > per_sm) --res;
  return tile_cps(batch, c->n, tp.t, res);
}
int contig_bits(const qc_circuit* c) { return c->dtype == QC_C64 ? 3 : 2; }
// Register bits per round: 4, except the complex128 backward (two states of
// 16-byte amplitudes) takes 3.  With 2^12-amplitude tiles every thread of a
// 256-thread CTA has work at 4 bits.
// Default register bits: 4 forward.  Backward: 4 (complex64) or 3
// (complex128), one less for the passes whose gate math needs the most
// registers per amplitude: complex-matrix single-qubit layers with gradients
// (in complex128 all of them) and, in complex128, every brick layer
// (measured faster on the IBM and IonQ native-gate circuits; real RY layers,
// constant complex layers such as SX and, in complex64, brick layers keep
// the larger count: the MS backward's two-nonzero rows and generator-phase
// gradients fit four bits, two gates per round).
int reg_bits(const qc_circuit* c, int ns, const LayerInfo* L = nullptr) {
  if (ns == 1 && c->opt.reg_bits_fwd > 0) return c->opt.reg_bits_fwd;
  if (ns == 2 && c->opt.reg_bits_bwd > 0) return c->opt.reg_bits_bwd;
  if (ns != 2) return 4;
  const int base = c->dtype == QC_C128 ? 3 : 4;
  if (L && L->cls == LC_ROT1 && !L->real && (c->dtype == QC_C128 || (L->diff && L->nparams > 0))) return base - 1;
  if (L && L->cls == LC_DENSE2 && c->dtype == QC_C128) return base - 1;
  return base;
}

// Shared-memory tile buffers of a pass.  Forward: two (one tile in flight
// while one is processed) measured faster on zz26 than three: the passes are
// bound by issue and shared-memory traffic, not by bytes in flight.  Complex64
// backward: one buffer of 2^12 amplitudes per CTA; the two CTAs of an SM
// overlap each other's copies, and the larger tile takes 7 instead of 10
// shared-memory rounds per 26-qubit layer (measured 6% faster on zz26 than
// 2^11 tiles with two buffers).  Three buffers only where two CTAs still fit.
int tile_stages(const qc_circuit* c, TilePass& P, int ns, int rsize) {
  int k = ns == 1 ? c->opt.stages_fwd : c->opt.stages_bwd;
  if (k == 0 && ns == 2 && c->dtype == QC_C64) k = 1;
  if (k == 1) return 1;
  if (k != 3) return 2;
  P.nstage = 3;
  const size_t per_sm = 228 * 1024, per_cta_reserved = 1024;
  return 2 * (tile_smem_bytes(P, ns, rsize) + per_cta_reserved) <= per_sm ? 3 : 2;
}

// set by plan_tile_layer when a gate found no round; read by build_plan
thread_local bool g_plan_unplaced = false;

// Register bits per round of a pass of tile size t: a two-qubit op needs both
// of its bits in the same round, so brick layers take at least two, and a pass
// has at most kMaxRounds rounds.
int pass_rb(const qc_circuit* c, const LayerInfo& L, int ns, int t) {
  int rb = std::max(reg_bits(c, ns, &L), L.cls == LC_DENSE2 ? 2 : 1);
  rb = std::max(rb, (t + kMaxRounds - 1) / kMaxRounds);
  return std::min(rb, t);
}

bool cuts_pair(const LayerInfo& L, int n, int e) {
  // boundary between bits e-1 and e cuts a brick pair (p_lo, p_hi) = (e-1, e)
  if (L.cls != LC_DENSE2 || e <= 0 || e >= n) return false;
  const int q = n - 1 - e;  // qubit of the pair's high bit (first qubit)
  return q >= L.parity && ((q - L.parity) % 2 == 0) && q + 1 <= n - 1;
}

struct PassOpInfo {
  int pidx;  // absolute parameter index of the op's first parameter (or -1)
};

// Builds the tile passes of a ROT1 or DENSE2 layer.  pidx_per_slot gets one
// entry {pass, slot, parameter index, companion} per gradient slot.  `comp`
// (backward, ROT1 only): the preceding RX / RY layer, whose gradients the ops
// also produce (companion slots follow the pass's own slots).
bool tma_rounds_conflict_free(const TilePass& P, int rb);
bool tma_enabled(const qc_circuit* c);
std::vector<TilePass> plan_tile_layer(const qc_circuit* c, const LayerInfo& L, int ns,
                                      std::vector<std::vector<int>>& pidx_per_slot,
                                      const LayerInfo* comp = nullptr) {
  const int n = c->n;
  const int tmax = tile_tmax(c, ns);
  const int cbits = contig_bits(c);
  std::vector<TilePass> out;
  // later passes share the bits left after the first one evenly
  const int rest = std::max(0, n - tmax);
  const int later_cap = tmax - cbits;
  // brick layers may have to end a pass one bit early so no pair is cut
  const int eff_cap = L.cls == LC_DENSE2 ? later_cap - 1 : later_cap;
  const int nlater = rest > 0 ? (rest + eff_cap - 1) / eff_cap : 0;
  const int even_cap = nlater > 0 ? (rest + nlater - 1) / nlater : later_cap;
  int s = 0;
  bool first = true;
  while (s < n) {
    int cap = first ? tmax : std::min(later_cap, std::max(even_cap, 2));
    int e = std::min(n, s + cap);
    if (e < n && cuts_pair(L, n, e)) e -= 1;
    TilePass P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    if (first) {
      // the tile keeps its full width when a brick pair ends the op range one
      // bit early (the pair goes to the next pass, which starts at e): the
      // extra bit carries no op, and the full-width tile can be staged by TMA
      const int w = std::min(n, s + cap);
      P.c = w; P.h0 = w; P.t = w;
    } else {
      // spare tile capacity widens the contiguous low segment
      P.c = std::min(s, std::max(cbits, tmax - (e - s)));
      P.h0 = s;
      P.t = P.c + (e - s);
    }
    auto local = [&](int p) { return first ? p : P.c + (p - s); };
    struct OpTmp { TileOp op; std::vector<int> pidx; int cpidx; };
    std::vector<OpTmp> ops;
    if (L.cls == LC_ROT1) {
      for (int p = s; p < e; ++p) {
        const int q = n - 1 - p;
        OpTmp o;
        memset(&o.op, 0, sizeof(o.op));
        o.op.l = (int16_t)local(p);
        o.op.is2q = 0;
        o.op.real = (int8_t)L.real;
        o.op.gk = (int8_t)(L.kind == QC_L_RX ? 1 : (L.kind == QC_L_RY ? 2 : 0));
        o.op.np = (int16_t)((ns == 2 && L.diff) ? 1 : 0);
        // real ops stage the packed real matrix; complex ones M (+ A backward)
        o.op.coef = L.coef_off + (long long)q * kRec1q + (L.real ? kRealOff : 0);
        o.op.bstride = L.coef_bstride;
        o.op.nco = L.real ? 4 : (ns == 2 ? 16 : 8);
        if (o.op.np) o.pidx.push_back(L.offset + L.pstride * q);
        o.cpidx = -1;
        if (ns == 2 && comp) {
          o.op.ck = (int8_t)(comp->kind == QC_L_RX ? 1 : 2);
          o.cpidx = comp->offset + comp->pstride * q;
        }
        ops.push_back(o);
      }
    } else {
      for (int i = 0; i < L.ngates; ++i) {
        const int q0 = L.parity + 2 * i;
        const int plo = n - 2 - q0, phi = plo + 1;
        if (plo < s || phi >= e) continue;
        OpTmp o;
        memset(&o.op, 0, sizeof(o.op));
        o.cpidx = -1;
        o.op.l = (int16_t)local(plo);
        o.op.is2q = 1;
        o.op.pat = (int16_t)(L.kind == QC_L_ECR_BRICK ? 1 : 0);
        const int np = (ns == 2 && L.diff && L.kind == QC_L_MS_BRICK) ? 3 : 0;
        o.op.np = (int16_t)np;
        o.op.coef = L.coef_off + (long long)i * kRec2q;
        o.op.bstride = L.coef_bstride;
        o.op.nco = 32 + (np ? 8 : 0);  // M, and for the MS backward its generator phases
        for (int k = 0; k < np; ++k) o.pidx.push_back(L.offset + 3 * i + k);
        ops.push_back(o);
      }
    }
    if (ops.empty()) {  // e.g. the unpaired top qubit of an odd brick
      s = e;
      first = false;
      continue;
    }
    // rounds of RB register bits
    int RB = pass_rb(c, L, ns, P.t);
    std::vector<int> assigned;
    int nass = 0, nr = 0;
    std::vector<TileOp> ordered;
    std::vector<std::vector<int>> ordered_pidx;
    std::vector<int> ordered_cpidx;
    auto place = [&](int rb) {
      assigned.assign(ops.size(), 0);
      nass = nr = 0;
      ordered.clear();
      ordered_pidx.clear();
      ordered_cpidx.clear();
      P.rop[0] = 0;
      while (nass < (int)ops.size()) {
        int lo = 1 << 30;
        for (size_t k = 0; k < ops.size(); ++k)
          if (!assigned[k]) lo = std::min(lo, (int)ops[k].op.l);
        lo = std::min(lo, P.t - rb);
        const int hi = lo + rb;
        int got = 0;
        // a round's ops in increasing bit order (the TMA pass numbers them so)
        std::vector<size_t> in_round;
        for (size_t k = 0; k < ops.size(); ++k) {
          if (assigned[k]) continue;
          const int top = ops[k].op.l + (ops[k].op.is2q ? 1 : 0);
          if (ops[k].op.l >= lo && top < hi) {
            assigned[k] = 1;
            ++nass;
            ++got;
            in_round.push_back(k);
          }
        }
        std::stable_sort(in_round.begin(), in_round.end(),
                         [&](size_t x, size_t y) { return ops[x].op.l < ops[y].op.l; });
        for (size_t k : in_round) {
          ordered.push_back(ops[k].op);
          ordered_pidx.push_back(ops[k].pidx);
          ordered_cpidx.push_back(ops[k].cpidx);
        }
        if (!got || nr >= kMaxRounds) break;  // the check below turns this into an error
        P.rlo[nr] = (int8_t)lo;
        ++nr;
        P.rop[nr] = (int16_t)ordered.size();
      }
      P.nrounds = nr;
      return nass == (int)ops.size();
    };
    place(RB);
    if (L.cls == LC_DENSE2 && RB == 4 && tma_enabled(c) && P.t == 12 && nass == (int)ops.size() &&
        !tma_rounds_conflict_free(P, 4)) {
      // pairs at odd local bits put round 0 at bit 1, where four register
      // bits leave bit 7 as a lane bit and the TMA tile's shared-memory reads
      // conflict; three register bits keep the lanes on bits 0 and 4..6, so
      // the pass can be staged by TMA
      if (place(3) && tma_rounds_conflict_free(P, 3)) RB = 3;
      else place(RB);
    }
    P.rb = RB;
    if (nass < (int)ops.size()) g_plan_unplaced = true;
    P.nrounds = nr;
    P.nops = (int)ordered.size();
    int soff = 0, slot = 0;
    for (int k = 0; k < P.nops; ++k) {
      P.ops[k] = ordered[k];
      P.ops[k].soff = soff;
      soff += P.ops[k].nco;
      P.ops[k].slot = (int16_t)slot;
      P.ops[k].cslot = -1;
      for (int q = 0; q < P.ops[k].np; ++q) pidx_per_slot.push_back({(int)out.size(), slot + q, ordered_pidx[k][q], 0});
      slot += P.ops[k].np;
    }
    for (int k = 0; k < P.nops; ++k) {
      if (!P.ops[k].ck) continue;
      P.ops[k].cslot = (int16_t)slot;
      pidx_per_slot.push_back({(int)out.size(), slot, ordered_cpidx[k], 1});
      ++slot;
      ++P.ncomp;
    }
    P.ncoef = soff;
    P.nslots = slot;
    P.store = 1;
    P.kind = L.cls == LC_DENSE2 ? 2 : (L.real ? 1 : 0);
    P.sx = (L.kind == QC_L_SX && P.ncomp == 0) ? 1 : 0;
    for (int r = 0; r < kMaxRounds; ++r)
      for (int i = 0; i < 5; ++i) P.rbit[r][i] = -1;
    for (int k = 0, r = 0; k < P.nops; ++k) {
      while (r + 1 < P.nrounds && P.rop[r + 1] <= k) ++r;
      P.rbit[r][P.ops[k].l - P.rlo[r]] = (int8_t)k;
    }
    // deferred reduction when every gradient op is single-qubit and rounds fit
    for (int r = 0; r < 4; ++r)
      for (int i = 0; i < 4; ++i) P.rslot[r][i] = P.rcslot[r][i] = -1;
    // the kernel keeps deferred sums for 4 rounds (3 at 4 register bits)
    bool defer = P.nrounds <= (RB == 4 ? 3 : 4) && slot > 0;
    for (int k = 0; k < P.nops && defer; ++k) {
      const TileOp& o = P.ops[k];
      if (o.np == 0 && !o.ck) continue;
      if (o.is2q || o.np > 1) { defer = false; break; }
      int r = 0;
      while (r + 1 < P.nrounds && P.rop[r + 1] <= k) ++r;
      const int i = o.l - P.rlo[r];
      if (i < 0 || i >= 4) { defer = false; break; }
      if (o.np) P.rslot[r][i] = o.slot;
      if (o.ck) P.rcslot[r][i] = o.cslot;
    }
    P.defer = defer ? 1 : 0;
    if (!defer)
      for (int r = 0; r < 4; ++r)
        for (int i = 0; i < 4; ++i) P.rslot[r][i] = P.rcslot[r][i] = -1;
    P.nstage = tile_stages(c, P, ns, (int)c->rsize);
    if (!defer && slot > 0 && ns == 2) {
      // otherwise every slot in shared memory, where two CTAs per SM still
      // fit (plus the TMA pass's alignment slack): the per-round FP64 warp
      // sums cost more than the pass's gate arithmetic on parametrised
      // brick layers
      P.defer = 2;
      const size_t per_sm = 228 * 1024, per_cta = tile_smem_bytes(P, ns, (int)c->rsize) + 2048;
      if (2 * per_cta > per_sm) P.defer = 0;
    }
    out.push_back(P);
    s = e;
    first = false;
  }
  return out;
}

int diag_zbit(const LayerInfo& L, int n, int j) {
  if (L.kind == QC_L_ISINGZZ_RING) return ((n - 2 - j) % n + n) % n;
  return n - 1 - j;
}

bool smem_fits(const qc_circuit* c) {
  const int lim = c->dtype == QC_C64 ? 13 : 12;
  return c->n <= lim;
}
// The automatic choice: the whole-circuit shared-memory kernel (one CTA per
// sample, one gate sweep and barrier per gate) wins only where the layer
// path is launch-bound: measured on HEA circuits, 0.8-1.0x the layer path's
// time for n <= 10 (complex64) / n <= 8 (complex128) at batch <= 64, slower
// above (n = 12, batch 256: 1.5x complex64, 1.6x complex128; n = 13, 1.8x).
bool smem_auto(const qc_circuit* c, int batch) {
  const int lim = c->dtype == QC_C64 ? 10 : 8;
  return c->n <= lim && batch <= 128;
}

void add_job(Plan& P, int kind, int source, long long part_off, long long nblk, int nvals,
             long long bps, const std::vector<OutMap>& outs) {
  RedJob J;
  memset(&J, 0, sizeof(J));
  J.part_off = part_off;
  J.nblk = (int)nblk;
  J.nvals = nvals;
  J.blk_per_sample = (int)bps;
  J.kind = kind;
  J.nout = (int)outs.size();
  J.source = source;
  J.first = (int)P.outs.size();
  const int jid = (int)P.jobs.size();
  P.jobs.push_back(J);
  P.row0.push_back(P.nrows);
  P.nrows += (long long)P.batch * nvals;
  for (auto o : outs) {
    o.job = jid;
    P.outs.push_back(o);
  }
}

// ---- TMA-staged tile passes (complex64) ----
// Whether the TMA kernel may run a pass: 2^12-amplitude tiles of >= 16
// contiguous amplitudes (one 128-byte swizzle row), a box of at most 256 rows
// per dimension, no gathered loads, the fused diagonals in the forms that
// kernel has, and every round's shared-memory accesses free of bank conflicts
// in the 128-byte swizzled layout (element i at i ^ (((i >> 4) & 7) << 1)):
// a round on bits [0, RB) reads 16-byte pairs, and the 3 lane bits of a
// quarter warp must move to 3 independent chunk bits; a higher round reads
// 8-byte elements, and the 4 lane bits of a half warp must move to 4
// independent bits of the element's position in its 128-byte row.
int gf2_rank(int* rows, int nr) {
  int rank = 0;
  for (int bit = 0; bit < 30 && rank < nr; ++bit) {
    int piv = -1;
    for (int i = rank; i < nr; ++i)
      if ((rows[i] >> bit) & 1) { piv = i; break; }
    if (piv < 0) continue;
    std::swap(rows[rank], rows[piv]);
    for (int i = 0; i < nr; ++i)
      if (i != rank && ((rows[i] >> bit) & 1)) rows[i] ^= rows[rank];
    ++rank;
  }
  return rank;
}
bool tma_rounds_conflict_free(const TilePass& P, int rb) {
  auto swz = [](int i) { return i ^ (((i >> 4) & 7) << 1); };
  for (int r = 0; r < P.nrounds; ++r) {
    const int lo = P.rlo[r];
    int lanes[5], k = 0;
    for (int p = 0; p < P.t && k < 5; ++p)
      if (p < lo || p >= lo + rb) lanes[k++] = p;
    int rows[4];
    const int nr = lo == 0 ? 3 : 4;
    if (k < nr) return false;
    for (int j = 0; j < nr; ++j) rows[j] = lo == 0 ? (swz(1 << lanes[j]) >> 1) & 7 : swz(1 << lanes[j]) & 15;
    if (gf2_rank(rows, nr) < nr) return false;
  }
  return true;
}
bool tma_enabled(const qc_circuit* c) { return c->dtype == QC_C64 && c->opt.tma == 1; }
bool tma_pass_ok(const qc_circuit* c, const Step& st) {
  if (!tma_enabled(c) || st.type != ST_TILE) return false;
  const TilePass& P = st.tp;
  if (P.t != 12 || P.c < 4 || P.t - P.c > 8 || P.gather || P.nstage < 1 || P.nstage > 2) return false;
  if (P.kind == 2) {
    if (P.pre || P.post || st.rb < 2 || st.rb > 4) return false;
  } else if (st.rb != 3 && st.rb != 4) {
    return false;
  }
  if (P.xload) {
    // the complemented-load variants (see launch_tma_ns)
    if (P.gather || P.scatter) return false;
    if (st.ns == 1 && !(P.kind == 2 && !P.pre && !P.post && (st.rb == 3 || st.rb == 4))) return false;
    if (st.ns == 2 && !(P.kind == 0 && P.sx && P.pre && st.rb == 4)) return false;
  }
  if (st.ns == 1) {
    if (P.pre || P.scatter) return false;
    if (P.post && !(st.rb == 4 && P.kind != 2 && fwd_post_contig(P))) return false;
  } else {
    if (P.post) return false;
    if (P.pre && !(st.rb == 4 && P.c == 12 && P.nrounds >= 1 && P.rlo[0] == 0)) return false;
  }
  return tma_rounds_conflict_free(P, st.rb);
}
// CTAs per sample of a TMA pass: three per SM for the real-gate forward, two
// otherwise, fewer if the shared memory does not fit
int tma_cps(const qc_circuit* c, int batch, const Step& st) {
  int res = (st.ns == 1 && st.tp.kind == 1) ? 3 : 2;
  const size_t per_sm = 228 * 1024, per_cta_reserved = 1024;
  while (res > 1 && (size_t)res * (tile_tma_smem_bytes(st.tp, st.ns) + per_cta_reserved) > per_sm) --res;
  return tile_cps(batch, c->n, st.tp.t, res);
}

// Packs the plan's device tables into one blob (layout: coef jobs | jobs |
// row0 | out0 | outs | prog, each 256-byte aligned) placed at the start of the
// workspace, and moves every other workspace region after it.
void build_tables(Plan& p) {
  std::vector<unsigned char>& host = p.tables;
  host.clear();
  auto put = [&](const void* src, size_t bytes) {
    size_t o = align256(host.size());
    host.resize(o + bytes);
    if (bytes) memcpy(host.data() + o, src, bytes);
    return o;
  };
  p.o_cj = put(p.coef_jobs.data(), p.coef_jobs.size() * sizeof(CoefJob));
  p.o_j = put(p.jobs.data(), p.jobs.size() * sizeof(RedJob));
  p.o_r = put(p.row0.data(), p.row0.size() * sizeof(long long));
  std::vector<RedOut> ro;
  for (auto& o : p.outs) {
    RedOut r;
    r.val = o.val;
    r.pidx = o.pidx;
    r.scale = o.scale;
    ro.push_back(r);
  }
  // outputs are ordered by job; k_finalize maps a flat output id to its job
  std::vector<int> out0;
  for (auto& J : p.jobs) out0.push_back(J.first);
  p.o_o0 = put(out0.data(), out0.size() * sizeof(int));
  p.o_ro = put(ro.data(), ro.size() * sizeof(RedOut));
  p.o_pr = put(p.prog.data(), p.prog.size() * sizeof(SmemLayer));
  host.resize(align256(std::max<size_t>(host.size(), 16)));
  const size_t shift = host.size();
  for (size_t* o : {&p.off_coef, &p.off_pv, &p.off_run0, &p.off_run1, &p.off_lam0, &p.off_lam1,
                    &p.off_ckpt, &p.off_part, &p.off_V, &p.ws_fwd, &p.ws_bwd})
    *o += shift;
}

std::unique_ptr<Plan> build_plan(const qc_circuit* c, int batch) {
  g_plan_unplaced = false;
  auto P = std::make_unique<Plan>();
  Plan& p = *P;
  p.batch = batch;
  const int n = c->n;
  const int L = (int)c->layers.size();
  const size_t N = (size_t)1 << n;
  p.S = (size_t)batch * N * 2 * c->rsize;

  // coefficient layout
  size_t ce = 0;
  for (int l = 0; l < L; ++l) {
    const LayerInfo& Li = c->layers[l];
    size_t sz = 0;
    if (Li.cls == LC_ROT1) sz = (size_t)n * kRec1q;
    else if (Li.cls == LC_DENSE2) sz = (size_t)Li.ngates * kRec2q;
    else if ((Li.cls == LC_DIAG || Li.cls == LC_XCOMP) && Li.has_phase) sz = (size_t)kDiagTables * 2 * ((size_t)1 << Li.tb);
    if (!sz) continue;
    CoefJob J;
    memset(&J, 0, sizeof(J));
    J.cls = Li.cls; J.kind = Li.kind; J.source = Li.source; J.offset = Li.offset;
    J.parity = Li.parity; J.ngates = Li.ngates; J.per_sample = Li.per_sample;
    J.has_phase = Li.has_phase; J.tb = Li.tb;
    J.pstride = Li.pstride; J.rot_phase = Li.rot_phase;
    J.coef_off = (long long)ce;
    J.bstride = Li.per_sample ? (long long)sz : 0;
    ce += Li.per_sample ? sz * batch : sz;
    ce = (ce + 1) & ~(size_t)1;
    p.coef_jobs.push_back(J);
  }
  p.coef_elems = ce;
  // write back offsets into a local copy of layer infos
  std::vector<LayerInfo> LI = c->layers;
  {
    size_t k = 0;
    for (int l = 0; l < L; ++l) {
      LayerInfo& Li = LI[l];
      const bool has = Li.cls == LC_ROT1 || Li.cls == LC_DENSE2 ||
                       ((Li.cls == LC_DIAG || Li.cls == LC_XCOMP) && Li.has_phase);
      if (!has) continue;
      Li.coef_off = p.coef_jobs[k].coef_off;
      Li.coef_bstride = p.coef_jobs[k].bstride;
      ++k;
    }
  }

  bool smem = false;
  if (c->opt.path == 1) smem = true;
  else if (c->opt.path == 0) smem = smem_auto(c, batch);
  p.smem = smem;

  size_t off = 0;
  p.off_coef = off;
  off = align256(off + ce * c->rsize);

  if (smem) {
    int slot = 0;
    for (int l = 0; l < L; ++l) {
      const LayerInfo& Li = LI[l];
      SmemLayer S;
      memset(&S, 0, sizeof(S));
      S.cls = Li.cls; S.kind = Li.kind; S.real = Li.real; S.zmode = Li.zmode;
      S.has_phase = Li.has_phase; S.tb = Li.tb; S.ngates = Li.ngates;
      S.np_per_gate = Li.kind == QC_L_MS_BRICK ? 3 : 1;
      S.parity = Li.parity;
      S.coef = Li.coef_off; S.bstride = Li.coef_bstride;
      S.gscale = Li.gscale;
      S.slot = -1;
      if (Li.diff && Li.nparams > 0) {
        S.slot = slot;
        std::vector<OutMap> outs;
        for (int j = 0; j < Li.nparams; ++j)
          outs.push_back(OutMap{0, j, Li.offset + (Li.cls == LC_DENSE2 ? j : Li.pstride * j), 1.0});
        add_job(p, RK_DIRECT, Li.source, (long long)slot * batch, batch, Li.nparams, 1, outs);
        slot += Li.nparams;
      }
      p.prog.push_back(S);
    }
    p.nslots = slot;
    p.part_doubles = (size_t)slot * batch;
    p.off_part = off;
    off = align256(off + p.part_doubles * 8);
    p.off_V = off;
    off = align256(off + (size_t)p.nrows * 8);
    p.ws_fwd = p.ws_bwd = std::max<size_t>(off, 256);
  } else {
    const int ck = c->opt.ckpt_every < 0 ? (p.S >= ((size_t)1 << 30) ? 4 : 0) : c->opt.ckpt_every;
    const bool fuse = c->opt.fuse != 0;
    auto is_tile = [&](int l) { return l >= 0 && l < L && (LI[l].cls == LC_ROT1 || LI[l].cls == LC_DENSE2); };
    auto is_phase = [&](int l) { return l >= 0 && l < L && LI[l].cls == LC_DIAG; };
    auto is_ring = [&](int l) { return l >= 0 && l < L && LI[l].cls == LC_RING; };
    auto tile_steps = [&](const LayerInfo& Li, int ns, std::vector<std::vector<int>>& pslots,
                          const LayerInfo* comp = nullptr) {
      std::vector<Step> v;
      for (auto& tp : plan_tile_layer(c, Li, ns, pslots, comp)) {
        Step st;
        st.type = ST_TILE; st.ns = ns; st.tp = tp; st.rb = tp.rb;
        st.cps = pass_cps(c, batch, tp, ns);
        v.push_back(st);
      }
      return v;
    };
    auto diag_step = [&](const LayerInfo& Li, int ns) {
      Step st;
      st.type = ST_DIAG; st.ns = ns;
      memset(&st.dp, 0, sizeof(st.dp));
      st.dp.n = n; st.dp.cb = std::min(n, ns == 2 ? 14 : 12); st.dp.zmode = Li.zmode;
      st.dp.xcomp = Li.cls == LC_XCOMP; st.dp.has_phase = Li.has_phase; st.dp.tb = Li.tb;
      st.dp.coef = Li.coef_off; st.dp.bstride = Li.coef_bstride; st.dp.nvals = n + 1;
      return st;
    };
    auto ring_step = [&](int ns) {
      Step st;
      st.type = ST_RING; st.ns = ns;
      memset(&st.rp, 0, sizeof(st.rp));
      st.rp.n = n;
      const size_t w = 2 * c->rsize;
      st.rp.whole = ((size_t)1 << n) * w * ns <= 96 * 1024;
      st.rp.t = std::min(tile_tmax(c, ns), n - 1);
      return st;
    };

    // need[l]: some layer <= l has gradients
    std::vector<int> need(L, 0);
    for (int l = 0; l < L; ++l) need[l] = (l > 0 ? need[l - 1] : 0) || (LI[l].diff && LI[l].nparams > 0);

    // ---------------- backward groups (reverse order) ----------------
    struct BGroup {
      int hi, lo;               // layers covered; the group's input is the state after `hi`
      std::vector<Step> steps;
      std::vector<std::vector<int>> pslots;
      int layer;                // layer whose parameters the group differentiates
      int comp = -1;            // layer whose gradients ride along as companions
      int pre_layer = -1;       // diagonal layer undone in the first pass's round 0
    };
    // tile passes of layer tl, folding a leading RX / RY layer before it
    // (companion gradients; that layer is never undone) or scattering
    // through a CNOT ring before it
    auto tile_group = [&](int tl, BGroup& g) {
      const LayerInfo& Lt = LI[tl];
      const bool fold = fuse && Lt.cls == LC_ROT1 && tl >= 1 && LI[tl - 1].cls == LC_ROT1 &&
                        (LI[tl - 1].kind == QC_L_RX || LI[tl - 1].kind == QC_L_RY) &&
                        LI[tl - 1].diff && LI[tl - 1].nparams > 0 && (tl == 1 || !need[tl - 2]);
      if (fold) {
        g.comp = tl - 1;
        g.steps = tile_steps(Lt, 2, g.pslots, &LI[tl - 1]);
        g.lo = tl - 1;
      } else {
        g.steps = tile_steps(Lt, 2, g.pslots);
        g.lo = tl;
        if (fuse && !g.steps.empty() && is_ring(tl - 1) && need[tl - 1]) {
          g.steps.back().tp.scatter = 1;  // the last (top) pass holds bit n-1
          g.lo = tl - 1;
        }
      }
    };
    std::vector<BGroup> bgroups;
    bool laminit_fused = false;
    {
      int i = L - 1;
      while (i >= 0 && need[i]) {
        BGroup g;
        g.hi = i;
        g.layer = i;
        const LayerInfo& Li = LI[i];
        if (fuse && Li.cls == LC_DIAG && i >= 1 && LI[i - 1].cls == LC_ROT1 && need[i - 1]) {
          // the diagonal layer rides in round 0 of the next layer's contiguous
          // first pass (register bits 0..RB-1), when that pass has one
          BGroup h;
          h.hi = i;
          h.layer = i - 1;
          tile_group(i - 1, h);
          if (!h.steps.empty()) {
            Step& f0 = h.steps.front();
            TilePass& tp = f0.tp;
            // a contiguous pass of 2^9 .. 2^12 amplitudes (2 .. 16 per thread);
            // the kernel's pre variant is built for 3 and 4 register bits (its
            // TMA form for 4 only; a complex64 pass at 3 bits fused with
            // per-thread copies measured as fast as a diagonal pass plus a TMA
            // tile pass)
            if (tp.c == tp.t && tp.nrounds > 0 && tp.t >= 9 && tp.t <= 12 && (f0.rb == 3 || f0.rb == 4) &&
                (Li.zmode == Z_IDENT || Li.zmode == Z_RINGXOR)) {
              tp.pre = 1;
              tp.pre_zmode = Li.zmode;
              tp.pre_tb = Li.tb;
              tp.pre_coef = Li.coef_off;
              tp.pre_bstride = Li.coef_bstride;
              tp.pre_grad = (Li.diff && Li.nparams > 0) ? 1 : 0;
              f0.cps = pass_cps(c, batch, tp, 2);
              h.pre_layer = i;
              i = h.lo - 1;
              bgroups.push_back(std::move(h));
              continue;
            }
          }
        }
        if (fuse && Li.cls == LC_DIAG && Li.zmode == Z_IDENT && i >= 1 && LI[i - 1].cls == LC_RING && need[i - 1]) {
          // the diagonal layer undone (and differentiated) in the next
          // backward ring pass, before its permutation, when its tile (the
          // whole state for a whole-state pass) has at least 2^10 amplitudes
          // (the kernel's loads come in steps of four per thread)
          Step r = ring_step(2);
          const int rt = r.rp.whole ? n : r.rp.t;
          if (rt >= 10 && rt <= 13) {
            r.rp.pre = 1;
            r.rp.pre_grad = (Li.diff && Li.nparams > 0) ? 1 : 0;
            r.rp.pre_tb = Li.tb;
            r.rp.pre_coef = Li.coef_off;
            r.rp.pre_bstride = Li.coef_bstride;
            g.steps.push_back(r);
            g.lo = i - 1;
            g.pre_layer = i;
            i = g.lo - 1;
            bgroups.push_back(std::move(g));
            continue;
          }
        }
        if (Li.cls == LC_ROT1 || Li.cls == LC_DENSE2) {
          tile_group(i, g);
        } else if (Li.cls == LC_RING) {
          g.steps.push_back(ring_step(2));
          g.lo = i;
          if (fuse && bgroups.empty()) laminit_fused = true;
        } else {
          g.steps.push_back(diag_step(Li, 2));
          g.lo = i;
        }
        i = g.lo - 1;
        bgroups.push_back(std::move(g));
      }
    }
    // an X layer (no phase) undone by complemented loads in the next group's
    // first pass, where that pass runs the TMA variant built for it (the SX
    // pass with the following diagonal undone in round 0)
    for (size_t k = 0; fuse && k + 1 < bgroups.size(); ++k) {
      BGroup& gx = bgroups[k];
      BGroup& gt = bgroups[k + 1];
      const LayerInfo& X = LI[gx.hi];
      if (gx.steps.size() != 1 || gx.steps[0].type != ST_DIAG || X.kind != QC_L_X || X.has_phase) continue;
      if (gt.steps.empty() || gt.steps.front().type != ST_TILE) continue;
      Step probe = gt.steps.front();
      probe.tp.xload = 1;
      if (!tma_pass_ok(c, probe)) continue;
      gt.steps.front().tp.xload = 1;
      gt.hi = gx.hi;
      bgroups.erase(bgroups.begin() + (long)k);
    }
    std::set<int> bstarts;
    for (auto& g : bgroups) bstarts.insert(g.hi);

    // ---------------- forward groups ----------------
    int lead = 0;
    if (fuse) {
      while (lead < L && lead < kMaxLeading) {
        const LayerInfo& Li = LI[lead];
        const bool single = Li.cls == LC_ROT1 ||
                            (Li.cls == LC_DIAG && (Li.kind == QC_L_RZ || Li.kind == QC_L_Z || Li.kind == QC_L_S)) ||
                            Li.cls == LC_XCOMP;
        if (!single) break;
        ++lead;
      }
    }
    p.nlead = lead;
    p.pv.nl = lead;
    for (int l = 0; l < lead; ++l) {
      p.pv.kind[l] = LI[l].kind;
      p.pv.source[l] = LI[l].source;
      p.pv.offset[l] = LI[l].offset;
      p.pv.pstride[l] = LI[l].pstride;
      p.pv.rot_phase[l] = LI[l].rot_phase;
    }
    struct FGroup {
      int hi;
      std::vector<Step> steps;
    };
    std::vector<FGroup> fgroups;
    {
      FGroup g;
      Step st;
      st.type = ST_PRODINIT;
      st.cb = std::min(n, 12);
      st.layer = lead - 1;
      st.post_layer = -1;
      int i = lead;
      if (fuse && lead > 0 && is_phase(i)) {  // diagonal right after the product block
        st.post_layer = i;
        st.post_coef = LI[i].coef_off;
        st.post_bstride = LI[i].coef_bstride;
        st.post_tb = LI[i].tb;
        st.post_zmode = LI[i].zmode;
        ++i;
      }
      g.hi = i - 1;
      g.steps.push_back(st);
      fgroups.push_back(std::move(g));
      int pend_ring = -1, pend_pre = -1;
      while (i < L) {
        const LayerInfo& Li = LI[i];
        if (fuse && pend_ring < 0 && pend_pre < 0 && is_ring(i) &&
            (is_tile(i + 1) || (is_phase(i + 1) && is_tile(i + 2)))) {
          pend_ring = i++;
          continue;
        }
        if (fuse && pend_pre < 0 && is_phase(i) && is_tile(i + 1)) {
          pend_pre = i++;
          continue;
        }
        FGroup h;
        std::vector<std::vector<int>> dummy;
        std::vector<Step> tsteps;
        if (is_tile(i)) tsteps = tile_steps(Li, 1, dummy);
        if (is_tile(i) && tsteps.empty()) {
          // a brick layer without pairs: nothing to apply; pending neighbours run on their own
          for (int l : {pend_ring, pend_pre}) {
            if (l < 0) continue;
            FGroup q;
            q.steps.push_back(LI[l].cls == LC_RING ? ring_step(1) : diag_step(LI[l], 1));
            q.hi = l;
            fgroups.push_back(std::move(q));
          }
          pend_ring = pend_pre = -1;
          ++i;
          continue;
        }
        if (is_tile(i)) {
          h.steps = tsteps;
          if (pend_ring >= 0) {  // top pass first: it gathers through the ring
            std::rotate(h.steps.begin(), h.steps.end() - 1, h.steps.end());
            h.steps.front().tp.gather = 1;
          }
          if (fuse && is_phase(i + 1) && c->dtype == QC_C64 && Li.cls == LC_ROT1) {
            // a following diagonal rides in the last round of the contiguous
            // pass when that pass takes the compile-time element patterns: run
            // it last (the layer's gates commute; a gathering pass stays first)
            for (size_t k = pend_ring >= 0 ? 1 : 0; k + 1 < h.steps.size(); ++k) {
              TilePass probe = h.steps[k].tp;
              probe.post_zmode = LI[i + 1].zmode;
              if (h.steps[k].rb == 4 && fwd_post_contig(probe)) {
                const Step mv = h.steps[k];
                h.steps.erase(h.steps.begin() + (long)k);
                h.steps.push_back(mv);
                break;
              }
            }
          }
          if (pend_pre >= 0) {
            const LayerInfo& D = LI[pend_pre];
            TilePass& tp = h.steps.front().tp;
            tp.pre = 1; tp.pre_zmode = D.zmode; tp.pre_tb = D.tb;
            tp.pre_coef = D.coef_off; tp.pre_bstride = D.coef_bstride;
          }
          int hi = i;
          if (fuse && is_phase(i + 1)) {
            const LayerInfo& D = LI[i + 1];
            TilePass& tp = h.steps.back().tp;
            tp.post = 1; tp.post_zmode = D.zmode; tp.post_tb = D.tb;
            tp.post_coef = D.coef_off; tp.post_bstride = D.coef_bstride;
            hi = i + 1;
          }
          pend_ring = pend_pre = -1;
          h.hi = hi;
          i = hi + 1;
        } else {
          if (Li.cls == LC_RING) h.steps.push_back(ring_step(1));
          else h.steps.push_back(diag_step(Li, 1));
          h.hi = i++;
        }
        fgroups.push_back(std::move(h));
      }
    }

    // an X layer (no phase) applied by complemented loads in the next group's
    // first pass, where that pass runs the TMA variant built for it (a brick
    // layer's first pass)
    for (size_t k = 0; fuse && k + 1 < fgroups.size(); ++k) {
      FGroup& gx = fgroups[k];
      FGroup& gt = fgroups[k + 1];
      if (gx.steps.size() != 1 || gx.steps[0].type != ST_DIAG) continue;
      const LayerInfo& X = LI[gx.hi];
      if (X.kind != QC_L_X || X.has_phase) continue;
      if (gt.steps.empty() || gt.steps.front().type != ST_TILE) continue;
      Step probe = gt.steps.front();
      probe.tp.xload = 1;
      if (!tma_pass_ok(c, probe)) continue;
      gt.steps.front().tp.xload = 1;
      fgroups.erase(fgroups.begin() + (long)k);
    }

    // checkpoints: forward group ends that are also backward group inputs
    std::map<int, int> ck_slot;
    if (ck > 0) {
      int last = -1;
      for (auto& g : fgroups) {
        const int l = g.hi;
        if (l < 0 || l >= L - 1 || !bstarts.count(l)) continue;
        if (l - last >= ck) {
          ck_slot[l] = (int)p.ckpt_after.size();
          p.ckpt_after.push_back(l);
          last = l;
        }
      }
    }
    p.nckpt = (int)p.ckpt_after.size();

    // forward buffers: symbolic A/B renamed at the end so the final state is psi_out
    {
      const int A = 1, Bb = 2;
      auto other = [&](int x) { return x == A ? Bb : A; };
      int cur = -1;
      for (auto& g : fgroups) {
        const bool to_ck = ck_slot.count(g.hi) > 0;
        for (size_t k = 0; k < g.steps.size(); ++k) {
          Step& st = g.steps[k];
          if (st.layer < 0 || st.type != ST_PRODINIT) st.layer = g.hi;
          const bool last = k + 1 == g.steps.size();
          if (st.type == ST_PRODINIT) {
            st.d0 = to_ck ? B_CKPT + ck_slot[g.hi] : A;
          } else {
            st.s0 = cur;
            const bool inplace_ok = st.type != ST_RING && !(st.type == ST_TILE && (st.tp.gather || st.tp.xload));
            if (last && to_ck) st.d0 = B_CKPT + ck_slot[g.hi];
            else if (inplace_ok && (cur == A || cur == Bb)) st.d0 = cur;
            else if (cur == A || cur == Bb) st.d0 = other(cur);
            else st.d0 = A;
          }
          cur = st.d0;
          p.fwd.push_back(st);
        }
      }
      const int fin = cur;
      for (auto& st : p.fwd) {
        auto ren = [&](int& bb) {
          if (bb == fin) bb = B_PSIOUT;
          else if (bb == A || bb == Bb) bb = B_RUN0;
        };
        ren(st.s0);
        ren(st.d0);
      }
    }

    // backward buffers and gradient bookkeeping
    if (!bgroups.empty() && !laminit_fused) {
      Step st;
      st.type = ST_LAMINIT;
      st.cb = std::min(n, 12);
      st.s0 = B_PSIOUT;
      st.d1 = B_LAM0;
      p.bwd.push_back(st);
    }
    int cp = B_PSIOUT, cl = B_LAM0;
    long long part_off = 0;
    auto isrun = [](int x) { return x == B_RUN0 || x == B_RUN1; };
    auto orun = [](int x) { return x == B_RUN0 ? B_RUN1 : B_RUN0; };
    auto olam = [](int x) { return x == B_LAM0 ? B_LAM1 : B_LAM0; };
    for (size_t gi = 0; gi < bgroups.size(); ++gi) {
      BGroup& g = bgroups[gi];
      const LayerInfo& Li = LI[g.layer];
      int sp = ck_slot.count(g.hi) ? B_CKPT + ck_slot[g.hi] : cp;
      for (size_t k = 0; k < g.steps.size(); ++k) {
        Step& st = g.steps[k];
        st.layer = g.layer;
        st.s0 = sp;
        st.s1 = cl;
        const bool lam_here = laminit_fused && gi == 0 && st.type == ST_RING;
        st.laminit = lam_here ? 1 : 0;
        const bool oop = st.type == ST_RING || (st.type == ST_TILE && (st.tp.scatter || st.tp.xload));
        st.d0 = (!oop && isrun(sp)) ? sp : (isrun(sp) ? orun(sp) : B_RUN0);
        st.d1 = lam_here ? B_LAM0 : (!oop ? cl : olam(cl));
        if (g.lo == 0 && k + 1 == g.steps.size() && st.type == ST_TILE) st.tp.store = 0;
        if (st.type == ST_TILE && st.tp.nslots > 0) {
          const long long nblk = (long long)batch * st.cps;
          st.part_off = part_off;
          std::vector<OutMap> outs, couts;
          int nown = 0;
          for (auto& e : g.pslots)
            if (e[0] == (int)k && !e[3]) ++nown;
          for (auto& e : g.pslots) {
            if (e[0] != (int)k) continue;
            if (e[3]) couts.push_back(OutMap{0, e[1] - nown, e[2], 1.0});
            else outs.push_back(OutMap{0, e[1], e[2], 1.0});
          }
          if (nown > 0) add_job(p, RK_DIRECT, Li.source, part_off, nblk, nown, st.cps, outs);
          if (!couts.empty())
            add_job(p, RK_DIRECT, LI[g.comp].source, part_off + nblk * nown, nblk,
                    st.tp.nslots - nown, st.cps, couts);
          part_off += nblk * st.tp.nslots;
        }
        if (st.type == ST_TILE && st.tp.pre && st.tp.pre_grad) {
          // the fused diagonal's marginals [W, M_0 .. M_{n-1}] per CTA
          const LayerInfo& D = LI[g.pre_layer];
          const long long nblk = (long long)batch * st.cps;
          if (st.tp.nslots == 0) st.part_off = part_off;
          st.tp.pre_moff = part_off - st.part_off;
          std::vector<OutMap> outs;
          for (int j = 0; j < D.nparams; ++j)
            outs.push_back(OutMap{0, diag_zbit(D, n, j), D.offset + D.pstride * j, D.gscale});
          add_job(p, RK_MARGINAL, D.source, part_off, nblk, n + 1, st.cps, outs);
          part_off += nblk * (n + 1);
        } else if (st.type == ST_RING && st.rp.pre && st.rp.pre_grad) {
          // the fused diagonal's marginals [W, M_0 .. M_{n-1}] per ring CTA
          const LayerInfo& D = LI[g.pre_layer];
          const long long bps = st.rp.whole ? 1 : 1LL << (n - st.rp.t), nblk = (long long)batch * bps;
          st.part_off = part_off;
          std::vector<OutMap> outs;
          for (int j = 0; j < D.nparams; ++j)
            outs.push_back(OutMap{0, diag_zbit(D, n, j), D.offset + D.pstride * j, D.gscale});
          add_job(p, RK_MARGINAL, D.source, part_off, nblk, n + 1, bps, outs);
          part_off += nblk * (n + 1);
        } else if (st.type == ST_DIAG && Li.diff && Li.nparams > 0) {
          const long long nblk = diag_grid(st.dp, batch);
          st.part_off = part_off;
          std::vector<OutMap> outs;
          for (int j = 0; j < Li.nparams; ++j)
            outs.push_back(OutMap{0, diag_zbit(Li, n, j), Li.offset + Li.pstride * j, Li.gscale});
          add_job(p, RK_MARGINAL, Li.source, part_off, nblk, n + 1, nblk / batch, outs);
          part_off += nblk * (n + 1);
        } else if (st.type == ST_DIAG) {
          st.part_off = -1;  // no gradient: marginals go to a scratch region
        }
        sp = st.d0;
        cl = st.d1;
        p.bwd.push_back(st);
      }
      cp = sp;
    }
    // diag passes without gradients still write marginals: give them a scratch region
    long long scratch_need = 0;
    for (auto& s : p.bwd)
      if (s.type == ST_DIAG && s.part_off < 0) scratch_need = std::max(scratch_need, diag_grid(s.dp, batch) * (n + 1));
    for (auto& s : p.bwd)
      if (s.type == ST_DIAG && s.part_off < 0) s.part_off = part_off;
    part_off += scratch_need;
    // <Z> partials (forward, ez requested)
    const int cbe = std::min(n, 14);
    const long long ez_need = ((long long)batch << (n - cbe)) * (n + 1);
    p.part_doubles = (size_t)std::max(part_off, ez_need);

    // workspace layout
    p.off_pv = off;
    off = align256(off + (size_t)batch * n * 4 * c->rsize);
    p.off_part = off;
    off = align256(off + p.part_doubles * 8);
    p.off_V = off;
    off = align256(off + (size_t)std::max<long long>(p.nrows, 1) * 8);
    p.off_ckpt = off;
    off = align256(off + (size_t)p.nckpt * p.S);
    p.off_run0 = off;
    off = align256(off + p.S);
    p.ws_fwd = off;
    p.off_run1 = off;
    off = align256(off + p.S);
    p.off_lam0 = off;
    off = align256(off + p.S);
    p.off_lam1 = off;
    off = align256(off + p.S);
    p.ws_bwd = off;
  }

  // finalize groups: serial when two jobs write the same output
  {
    std::map<std::pair<int, int>, int> seen;
    for (auto& o : p.outs) {
      auto key = std::make_pair(p.jobs[o.job].source, o.pidx);
      if (seen.count(key) && seen[key] != o.job) p.overlap = true;
      seen[key] = o.job;
    }
    if (!p.jobs.empty()) {
      if (p.overlap) {
        for (size_t j = 0; j < p.jobs.size(); ++j) p.job_groups.push_back({(int)j});
      } else {
        std::vector<int> all;
        for (size_t j = 0; j < p.jobs.size(); ++j) all.push_back((int)j);
        p.job_groups.push_back(all);
      }
    }
  }
  P->unplaced = g_plan_unplaced;
  for (auto* v : {&p.fwd, &p.bwd})
    for (Step& st : *v)
      if (st.type == ST_TILE && c->dtype == QC_C64 && c->opt.tc_dense == 1 && tile_tc_ok(st.tp, st.ns)) {
        st.tc = 1;  // one 192 KB CTA per SM
        st.cps = tile_cps(batch, c->n, st.tp.t, 1);
      } else if (st.type == ST_TILE && tma_pass_ok(c, st)) {
        st.tma = 1;
        st.cps = tma_cps(c, batch, st);
      }
  build_tables(p);
  return P;
}

// Writes the plan's device tables into the caller's workspace (stream order).
qc_status upload_tables(const Plan& p, char* ws, cudaStream_t st) {
  if (p.tables.empty()) return QC_OK;
  ProfScope ps(PC_UPLOAD, 0, st, (int)((p.tables.size() + kUploadBytes - 1) / kUploadBytes));
  cudaError_t e = launch_upload(p.tables.data(), p.tables.size(), ws, st);
  if (e != cudaSuccess) return cuda_fail(e, "plan table upload");
  return QC_OK;
}

constexpr size_t kMaxPlans = 16;

// Plans are host-only (their device tables travel with every call), so the
// cache is bounded: the least recently used plan is dropped beyond kMaxPlans.
qc_status get_plan(qc_circuit* c, int batch, Plan** out) {
  auto it = c->plans.find(batch);
  if (it == c->plans.end()) {
    auto P = build_plan(c, batch);
    if (P->unplaced) return fail(QC_ERR_UNSUPPORTED, "planner: a gate found no round in its tile pass");
    if (c->plans.size() >= kMaxPlans) {
      auto lru = c->plans.begin();
      for (auto j = c->plans.begin(); j != c->plans.end(); ++j)
        if (j->second->last_use < lru->second->last_use) lru = j;
      c->plans.erase(lru);
    }
    it = c->plans.emplace(batch, std::move(P)).first;
  }
  it->second->last_use = ++c->plan_clock;
  *out = it->second.get();
  return QC_OK;
}

template <class R>
qc_status run_coef(qc_circuit* c, Plan& p, int batch, const double* x, const double* theta,
                   char* ws, cudaStream_t st) {
  if (p.coef_jobs.empty()) return QC_OK;
  ProfScope ps(PC_COEF, 0, st);
  cudaError_t e = launch_coef<R>(plan_dev(p, ws).coef_jobs, (int)p.coef_jobs.size(), c->n, batch,
                                 c->n_in, x, theta, ws + p.off_coef, st);
  if (e != cudaSuccess) return cuda_fail(e, "coef kernel");
  return QC_OK;
}

struct Bufs {
  void* b[32];
};

template <class R>
qc_status run_steps(qc_circuit* c, Plan& p, const std::vector<Step>& steps, int batch,
                    const double* x, const double* theta, const double* gez, void* psi_out,
                    char* ws, cudaStream_t st) {
  Bufs B;
  memset(&B, 0, sizeof(B));
  B.b[B_PSIOUT] = psi_out;
  B.b[B_RUN0] = ws + p.off_run0;
  B.b[B_RUN1] = ws + p.off_run1;
  B.b[B_LAM0] = ws + p.off_lam0;
  B.b[B_LAM1] = ws + p.off_lam1;
  auto buf = [&](int id) -> void* {
    if (id == B_NONE) return nullptr;
    if (id >= B_CKPT) return ws + p.off_ckpt + (size_t)(id - B_CKPT) * p.S;
    return B.b[id];
  };
  const char* coef = ws + p.off_coef;
  double* part = (double*)(ws + p.off_part);
  const double S = (double)p.S;
  for (const Step& s : steps) {
    cudaError_t e = cudaSuccess;
    // algorithmic bytes of one launch: every pass reads and writes each state once
    const double passb = s.ns == 2 ? (s.type == ST_TILE && !s.tp.store ? 2 * S : 4 * S) : 2 * S;
    switch (s.type) {
      case ST_PRODINIT: {
        ProfScope ps(PC_PRODINIT, S, st, 2);
        e = launch_prodvec<R>(p.pv, c->n, batch, c->n_in, x, theta, ws + p.off_pv, st);
        if (e == cudaSuccess) {
          const bool post = s.post_layer >= 0;
          e = launch_prodinit<R>(c->n, s.cb, batch, ws + p.off_pv, buf(s.d0),
                                 post ? coef + s.post_coef * sizeof(R) : nullptr, s.post_bstride,
                                 s.post_tb, s.post_zmode, st);
        }
        break;
      }
      case ST_TILE: {
        ProfScope ps(s.ns == 2 ? PC_TILE_B : PC_TILE_F, passb, st);
        if (s.tc && sizeof(R) == 4)
          e = launch_tile_tc(s.tp, batch, s.cps, coef, buf(s.s0), buf(s.d0), st);
        else if (s.tma && sizeof(R) == 4)
          e = s.ns == 1 ? launch_tile_tma_fwd(s.tp, s.rb, batch, s.cps, coef, buf(s.s0), buf(s.d0), buf(s.s1),
                                              buf(s.d1), part + s.part_off, st)
                        : launch_tile_tma_bwd(s.tp, s.rb, batch, s.cps, coef, buf(s.s0), buf(s.d0), buf(s.s1),
                                              buf(s.d1), part + s.part_off, st);
        else
          e = launch_tile<R>(s.tp, s.rb, s.ns, batch, s.cps, coef, buf(s.s0), buf(s.d0), buf(s.s1),
                             buf(s.d1), part + s.part_off, st);
        break;
      }
      case ST_DIAG: {
        ProfScope ps(s.ns == 2 ? PC_DIAG_B : PC_DIAG_F, passb, st);
        e = launch_diag<R>(s.dp, s.ns, batch, coef, buf(s.s0), buf(s.d0), buf(s.s1), buf(s.d1),
                           part + s.part_off, st);
        break;
      }
      case ST_RING: {
        // with lambda formed from psi in the same launch only psi is read
        ProfScope ps(s.ns == 2 ? PC_RING_B : PC_RING_F, s.laminit ? 3 * S : passb, st);
        e = launch_ring<R>(s.rp, s.ns, batch, buf(s.s0), buf(s.d0), s.laminit ? nullptr : buf(s.s1),
                           buf(s.d1), s.laminit ? gez : nullptr, coef, part + s.part_off, st);
        break;
      }
      case ST_LAMINIT: {
        ProfScope ps(PC_LAMINIT, 2 * S, st);
        e = launch_laminit<R>(c->n, s.cb, batch, gez, buf(s.s0), buf(s.d1), st);
        break;
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "layer kernel launch");
  }
  return QC_OK;
}

qc_status run_reduce(qc_circuit* c, Plan& p, int batch, char* ws, double* d_theta, double* d_x,
                     cudaStream_t st) {
  if (p.jobs.empty()) return QC_OK;
  const double* part = (const double*)(ws + p.off_part);
  double* V = (double*)(ws + p.off_V);
  const PlanDev d = plan_dev(p, ws);
  for (auto& g : p.job_groups) {
    // a group is a contiguous run of jobs
    const int j0 = g.front(), nj = (int)g.size();
    long long rows = 0;
    int nout = 0;
    for (int j : g) { rows += (long long)batch * p.jobs[j].nvals; nout += p.jobs[j].nout; }
    ProfScope ps(PC_REDUCE, 0, st, 2);
    cudaError_t e = launch_reduce(d.jobs + j0, d.row0 + j0, d.out0 + j0, nj, p.row0[j0], rows,
                                  p.jobs[j0].first, nout, d.outs, batch, c->n_in, part, V,
                                  d_theta, d_x, st);
    if (e != cudaSuccess) return cuda_fail(e, "reduce kernels");
  }
  return QC_OK;
}

qc_status check_common(qc_circuit* c, int batch) {
  if (!c) return fail(QC_ERR_INVALID, "circuit handle is NULL");
  if (batch <= 0) return fail(QC_ERR_INVALID, "batch must be positive");
  if ((size_t)batch * ((size_t)1 << c->n) > ((size_t)1 << 40)) return fail(QC_ERR_INVALID, "batch * 2^n too large");
  return QC_OK;
}

template <class R>
qc_status forward_impl(qc_circuit* c, int batch, const double* x, const double* theta, void* psi_out,
                       double* ez, void* workspace, size_t wbytes, cudaStream_t st) {
  Plan* p;
  qc_status s = get_plan(c, batch, &p);
  if (s != QC_OK) return s;
  if (wbytes < p->ws_fwd) return fail(QC_ERR_OOM, "workspace smaller than qc_workspace_bytes");
  if ((uintptr_t)workspace % 256) return fail(QC_ERR_INVALID, "workspace must be 256-byte aligned");
  if ((uintptr_t)psi_out % 16) return fail(QC_ERR_INVALID, "psi_out must be 16-byte aligned");
  char* ws = (char*)workspace;
  s = upload_tables(*p, ws, st);
  if (s != QC_OK) return s;
  s = run_coef<R>(c, *p, batch, x, theta, ws, st);
  if (s != QC_OK) return s;
  if (p->smem) {
    ProfScope ps(PC_SMEM_F, (double)p->S, st);
    cudaError_t e = launch_smem<R>(plan_dev(*p, ws).prog, (int)p->prog.size(), c->n, batch, 0, ws + p->off_coef,
                                   nullptr, psi_out, ez, nullptr, nullptr, p->nslots, st);
    if (e != cudaSuccess) return cuda_fail(e, "whole-circuit forward kernel");
  } else {
    s = run_steps<R>(c, *p, p->fwd, batch, x, theta, nullptr, psi_out, ws, st);
    if (s != QC_OK) return s;
    if (ez) {
      const int cbe = std::min(c->n, 14);
      ProfScope ps(PC_EXPECT, (double)p->S, st, 2);
      cudaError_t e = launch_expect<R>(c->n, cbe, batch, psi_out, (double*)(ws + p->off_part), ez, st);
      if (e != cudaSuccess) return cuda_fail(e, "expect kernel");
    }
  }
  c->last_ws = workspace;
  c->last_batch = batch;
  return QC_OK;
}

template <class R>
qc_status backward_impl(qc_circuit* c, int batch, const double* x, const double* theta,
                        const void* psi_out, const double* gez, double* d_theta, double* d_x,
                        void* workspace, size_t wbytes, cudaStream_t st) {
  Plan* p;
  qc_status s = get_plan(c, batch, &p);
  if (s != QC_OK) return s;
  if (wbytes < p->ws_bwd) return fail(QC_ERR_OOM, "workspace smaller than qc_workspace_bytes");
  if ((uintptr_t)workspace % 256) return fail(QC_ERR_INVALID, "workspace must be 256-byte aligned");
  if (p->nckpt > 0 && (c->last_ws != workspace || c->last_batch != batch))
    return fail(QC_ERR_INVALID, "checkpointed backward needs the workspace of the preceding forward");
  char* ws = (char*)workspace;
  s = upload_tables(*p, ws, st);
  if (s != QC_OK) return s;
  cudaError_t e;
  if (d_theta && c->n_theta > 0) {
    e = cudaMemsetAsync(d_theta, 0, sizeof(double) * c->n_theta, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset d_theta");
  }
  if (d_x && c->n_in > 0) {
    e = cudaMemsetAsync(d_x, 0, sizeof(double) * c->n_in * (size_t)batch, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset d_x");
  }
  s = run_coef<R>(c, *p, batch, x, theta, ws, st);
  if (s != QC_OK) return s;
  if (p->smem) {
    ProfScope ps(PC_SMEM_B, (double)p->S, st);
    e = launch_smem<R>(plan_dev(*p, ws).prog, (int)p->prog.size(), c->n, batch, 1, ws + p->off_coef, psi_out,
                       nullptr, nullptr, gez, (double*)(ws + p->off_part), p->nslots, st);
    if (e != cudaSuccess) return cuda_fail(e, "whole-circuit backward kernel");
  } else {
    s = run_steps<R>(c, *p, p->bwd, batch, x, theta, gez, const_cast<void*>(psi_out), ws, st);
    if (s != QC_OK) return s;
  }
  return run_reduce(c, *p, batch, ws, d_theta, d_x, st);
}

int layer_class(int kind) {
  switch (kind) {
    case QC_L_RX: case QC_L_RY: case QC_L_SX: case QC_L_GPI2: case QC_L_H: return LC_ROT1;
    case QC_L_RZ: case QC_L_ISINGZZ_RING: case QC_L_Z: case QC_L_S: return LC_DIAG;
    case QC_L_CNOT_RING: return LC_RING;
    case QC_L_X: case QC_L_GPI: return LC_XCOMP;
    case QC_L_MS_BRICK: case QC_L_ECR_BRICK: case QC_L_CZ_BRICK: case QC_L_SWAP_BRICK: return LC_DENSE2;
  }
  return -1;
}

}  // namespace

namespace qc {
void count_alloc() { ++g_alloc_calls; }
void circuit_shape(const qc_circuit* c, int* n, int* dtype) {
  *n = c->n;
  *dtype = (int)c->dtype;
}
qc_status set_error(qc_status s, const char* msg) { return fail(s, msg); }
}  // namespace qc

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

QC_API int qc_version(void) { return 101; }

QC_API void qc_default_options(qc_options* opt) {
  if (!opt) return;
  opt->ckpt_every = -1;
  opt->path = 0;
  opt->fuse = 1;
  opt->tile_bits_fwd = opt->tile_bits_bwd = 0;
  opt->reg_bits_fwd = opt->reg_bits_bwd = 0;
  opt->stages_fwd = opt->stages_bwd = 0;
  opt->tma = 1;
  opt->tc_dense = 0;
}

QC_API const char* qc_last_error(void) { return g_last_error.c_str(); }

QC_API qc_status qc_create(int n, qc_dtype dtype, const qc_layer* layers, int n_layers,
                           const qc_options* opt, qc_circuit** out) {
  if (!out) return fail(QC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > kMaxQubits) return fail(QC_ERR_INVALID, "n must be in [1, 30]");
  if (dtype != QC_C64 && dtype != QC_C128) return fail(QC_ERR_INVALID, "unknown dtype");
  if (n_layers < 0 || (n_layers > 0 && !layers)) return fail(QC_ERR_INVALID, "bad layer list");
  qc_options o;
  qc_default_options(&o);
  if (opt) o = *opt;
  // geometry left at 0 takes the process environment (QC_TMAX_FWD / _BWD,
  // QC_RB_FWD / _BWD, QC_TILE_STAGES), then the same range checks
  auto from_env = [](int32_t& f, const char* name) {
    if (f == 0) f = env_knob(name);
  };
  from_env(o.tile_bits_fwd, "QC_TMAX_FWD");
  from_env(o.tile_bits_bwd, "QC_TMAX_BWD");
  from_env(o.reg_bits_fwd, "QC_RB_FWD");
  from_env(o.reg_bits_bwd, "QC_RB_BWD");
  from_env(o.stages_fwd, "QC_TILE_STAGES");
  from_env(o.stages_bwd, "QC_TILE_STAGES");
  // QC_TMA=0 turns the TMA-staged passes off for circuits left at the default
  if (o.tma == 1 && getenv("QC_TMA") && atoi(getenv("QC_TMA")) == 0) o.tma = 0;
  // QC_TC_DENSE=1 turns the tensor-core dense block on for circuits left at the default
  if (o.tc_dense == 0 && getenv("QC_TC_DENSE") && atoi(getenv("QC_TC_DENSE")) == 1) o.tc_dense = 1;
  if (o.path < 0 || o.path > 2) return fail(QC_ERR_INVALID, "options.path must be 0, 1 or 2");
  if (o.ckpt_every < -1) return fail(QC_ERR_INVALID, "options.ckpt_every must be >= -1");
  {
    const int fmax = dtype == QC_C64 ? 13 : 12, bmax = dtype == QC_C64 ? 12 : 11;
    if (o.tile_bits_fwd != 0 && (o.tile_bits_fwd < 6 || o.tile_bits_fwd > fmax))
      return fail(QC_ERR_INVALID, "options.tile_bits_fwd (or QC_TMAX_FWD) out of range");
    if (o.tile_bits_bwd != 0 && (o.tile_bits_bwd < 6 || o.tile_bits_bwd > bmax))
      return fail(QC_ERR_INVALID, "options.tile_bits_bwd (or QC_TMAX_BWD) out of range");
    if (o.reg_bits_fwd < 0 || o.reg_bits_fwd > 4 || o.reg_bits_bwd < 0 || o.reg_bits_bwd > 4)
      return fail(QC_ERR_INVALID, "options.reg_bits_* (or QC_RB_*) must be in 0 .. 4");
    if (o.stages_fwd < 0 || o.stages_fwd > 3 || o.stages_bwd < 0 || o.stages_bwd > 3)
      return fail(QC_ERR_INVALID, "options.stages_* (or QC_TILE_STAGES) must be in 0 .. 3");
    if (o.tma != 0 && o.tma != 1) return fail(QC_ERR_INVALID, "options.tma must be 0 or 1");
    if (o.tc_dense != 0 && o.tc_dense != 1) return fail(QC_ERR_INVALID, "options.tc_dense must be 0 or 1");
  }
  auto c = std::make_unique<qc_circuit>();
  c->n = n;
  c->dtype = dtype;
  c->rsize = dtype == QC_C64 ? 4 : 8;
  c->opt = o;
  if (o.path == 1 && !smem_fits(c.get()))
    return fail(QC_ERR_UNSUPPORTED, "whole-circuit shared-memory path needs n <= 13 (c64) / 12 (c128)");
  // a Rot layer runs as three layers RZ(lambda), RY(theta), RZ(phi) (the
  // last carrying the global phase e^{i(phi+lambda)/2}) on strided parameters
  struct Sub { qc_layer in; int pstride, rot_phase, user; };
  std::vector<Sub> subs;
  for (int l = 0; l < n_layers; ++l) {
    const qc_layer& in = layers[l];
    if (in.kind == QC_L_ROT) {
      if (in.source < QC_SRC_NONE || in.source > QC_SRC_INPUT)
        return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": unknown source");
      if (in.source != QC_SRC_NONE && in.offset < 0)
        return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": negative offset");
      if (in.source == QC_SRC_THETA) c->n_theta = std::max(c->n_theta, in.offset + 3 * n);
      if (in.source == QC_SRC_INPUT) c->n_in = std::max(c->n_in, in.offset + 3 * n);
      subs.push_back(Sub{qc_layer{QC_L_RZ, in.source, in.offset + 2, 0}, 3, 0, l});
      subs.push_back(Sub{qc_layer{QC_L_RY, in.source, in.offset + 0, 0}, 3, 0, l});
      subs.push_back(Sub{qc_layer{QC_L_RZ, in.source, in.offset + 1, 0}, 3, 1, l});
    } else {
      subs.push_back(Sub{in, 1, 0, l});
    }
  }
  for (const Sub& sub : subs) {
    const qc_layer& in = sub.in;
    const int l = sub.user;
    LayerInfo L;
    memset(&L, 0, sizeof(L));
    L.kind = in.kind;
    L.source = in.source;
    L.offset = in.offset;
    L.parity = in.parity;
    L.pstride = sub.pstride;
    L.rot_phase = sub.rot_phase;
    L.cls = layer_class(in.kind);
    if (L.cls < 0) return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": unknown kind");
    if (in.source < QC_SRC_NONE || in.source > QC_SRC_INPUT)
      return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": unknown source");
    if ((in.kind == QC_L_CNOT_RING || in.kind == QC_L_ISINGZZ_RING) && n < 2)
      return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": ring layers need n >= 2");
    if (L.cls == LC_DENSE2) {
      if (in.parity != 0 && in.parity != 1)
        return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": brick parity must be 0 or 1");
      L.ngates = std::max(0, (n - in.parity) / 2);
    } else if (L.cls == LC_ROT1) {
      L.ngates = n;
    } else {
      L.ngates = n;
    }
    switch (in.kind) {
      case QC_L_RX: case QC_L_RY: case QC_L_RZ: case QC_L_GPI: case QC_L_GPI2: case QC_L_ISINGZZ_RING:
        L.nparams = n; break;
      case QC_L_MS_BRICK: L.nparams = 3 * L.ngates; break;
      default: L.nparams = 0;
    }
    const bool never_param = in.kind == QC_L_CNOT_RING || in.kind == QC_L_X || in.kind == QC_L_SX ||
                             in.kind == QC_L_ECR_BRICK || in.kind == QC_L_Z || in.kind == QC_L_S ||
                             in.kind == QC_L_H || in.kind == QC_L_CZ_BRICK || in.kind == QC_L_SWAP_BRICK;
    if (never_param && in.source != QC_SRC_NONE)
      return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": unparametrised kind needs source NONE");
    if (in.source != QC_SRC_NONE && in.offset < 0)
      return fail(QC_ERR_INVALID, "layer " + std::to_string(l) + ": negative offset");
    L.diff = (in.source == QC_SRC_THETA || in.source == QC_SRC_INPUT) && L.nparams > 0;
    L.per_sample = in.source == QC_SRC_INPUT && L.nparams > 0;
    L.real = in.kind == QC_L_RY;
    L.zmode = in.kind == QC_L_ISINGZZ_RING ? Z_RINGXOR : Z_IDENT;
    L.has_phase = (L.cls == LC_DIAG) || in.kind == QC_L_GPI;
    L.gscale = in.kind == QC_L_GPI ? -4.0 * 3.14159265358979323846 : 1.0;
    L.tb = (n + kDiagTables - 1) / kDiagTables;
    if (L.tb < 1) L.tb = 1;
    if (sub.pstride == 1) {  // (Rot's bound was taken above)
      if (in.source == QC_SRC_THETA) c->n_theta = std::max(c->n_theta, in.offset + L.nparams);
      if (in.source == QC_SRC_INPUT) c->n_in = std::max(c->n_in, in.offset + L.nparams);
    }
    c->layers.push_back(L);
  }
  // the <Z> scratch of qc_expect_z: 2 MiB or one sample's partial sums,
  // whichever is larger; on a host without a usable device it stays NULL
  // (planning calls still work; qc_expect_z then reports the missing device)
  {
    const int cb = std::min(n, 14);
    const size_t per_sample = ((size_t)1 << (n - cb)) * (n + 1) * sizeof(double);
    const size_t bytes = std::max<size_t>(per_sample, (size_t)2 << 20);
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      count_alloc();
      if (cudaMalloc(&c->exp_scratch, bytes) == cudaSuccess) c->exp_scratch_bytes = bytes;
      else c->exp_scratch = nullptr;
    }
    cudaGetLastError();
    noalloc_prepare(n, (int)dtype);
  }
  *out = c.release();
  return QC_OK;
}

QC_API qc_status qc_destroy(qc_circuit* c) {
  if (!c) return QC_OK;
  if (c->exp_scratch) {
    // work in flight may still read the scratch
    count_alloc();
    cudaDeviceSynchronize();
    count_alloc();
    cudaFree(c->exp_scratch);
  }
  delete c;
  return QC_OK;
}

QC_API qc_status qc_num_params(const qc_circuit* c, int* n_theta, int* n_in) {
  if (!c) return fail(QC_ERR_INVALID, "circuit handle is NULL");
  if (n_theta) *n_theta = c->n_theta;
  if (n_in) *n_in = c->n_in;
  return QC_OK;
}

QC_API qc_status qc_workspace_bytes(const qc_circuit* cc, int batch, size_t* bytes) {
  qc_circuit* c = const_cast<qc_circuit*>(cc);
  qc_status s = check_common(c, batch);
  if (s != QC_OK) return s;
  if (!bytes) return fail(QC_ERR_INVALID, "bytes is NULL");
  Plan* p;
  s = get_plan(c, batch, &p);
  if (s != QC_OK) return s;
  *bytes = std::max(p->ws_fwd, p->ws_bwd);
  return QC_OK;
}

QC_API qc_status qc_forward(qc_circuit* c, int batch, const double* x, const double* theta,
                            void* psi_out, double* ez, void* workspace, size_t workspace_bytes,
                            void* stream) {
  qc_status s = check_common(c, batch);
  if (s != QC_OK) return s;
  if (!psi_out) return fail(QC_ERR_INVALID, "psi_out is NULL");
  if (!workspace) return fail(QC_ERR_INVALID, "workspace is NULL");
  if (c->n_in > 0 && !x) return fail(QC_ERR_INVALID, "circuit reads x but x is NULL");
  if (c->n_theta > 0 && !theta) return fail(QC_ERR_INVALID, "circuit reads theta but theta is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (c->dtype == QC_C64) return forward_impl<float>(c, batch, x, theta, psi_out, ez, workspace, workspace_bytes, st);
  return forward_impl<double>(c, batch, x, theta, psi_out, ez, workspace, workspace_bytes, st);
}

QC_API qc_status qc_expect_z(qc_circuit* c, int batch, const void* psi, double* ez, void* stream) {
  qc_status s = check_common(c, batch);
  if (s != QC_OK) return s;
  if (!psi || !ez) return fail(QC_ERR_INVALID, "psi and ez must be non-NULL");
  if (!c->exp_scratch)
    return fail(QC_ERR_CUDA, "qc_expect_z: the circuit was created without a usable CUDA device");
  const int n = c->n, cb = std::min(n, 14);
  // samples per launch: the partial sums of a chunk fit the scratch qc_create
  // allocated (launches on one stream reuse it in order)
  const size_t per_sample = ((size_t)1 << (n - cb)) * (n + 1) * sizeof(double);
  const int chunk = (int)std::max<size_t>(1, c->exp_scratch_bytes / per_sample);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t sbytes = ((size_t)1 << n) * 2 * c->rsize;
  for (int b0 = 0; b0 < batch; b0 += chunk) {
    const int nb = std::min(chunk, batch - b0);
    const char* ps_in = (const char*)psi + (size_t)b0 * sbytes;
    ProfScope ps(PC_EXPECT, (double)nb * sbytes, st, 2);
    cudaError_t e = c->dtype == QC_C64
                        ? launch_expect<float>(n, cb, nb, ps_in, (double*)c->exp_scratch, ez + (size_t)b0 * n, st)
                        : launch_expect<double>(n, cb, nb, ps_in, (double*)c->exp_scratch, ez + (size_t)b0 * n, st);
    if (e != cudaSuccess) return cuda_fail(e, "expect kernel");
  }
  return QC_OK;
}

QC_API qc_status qc_backward(qc_circuit* c, int batch, const double* x, const double* theta,
                             const void* psi_out, const double* g_ez, double* d_theta, double* d_x,
                             void* workspace, size_t workspace_bytes, void* stream) {
  qc_status s = check_common(c, batch);
  if (s != QC_OK) return s;
  if (!psi_out || !g_ez) return fail(QC_ERR_INVALID, "psi_out and g_ez must be non-NULL");
  if (!workspace) return fail(QC_ERR_INVALID, "workspace is NULL");
  if (c->n_in > 0 && !x) return fail(QC_ERR_INVALID, "circuit reads x but x is NULL");
  if (c->n_theta > 0 && !theta) return fail(QC_ERR_INVALID, "circuit reads theta but theta is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (c->dtype == QC_C64)
    return backward_impl<float>(c, batch, x, theta, psi_out, g_ez, d_theta, d_x, workspace, workspace_bytes, st);
  return backward_impl<double>(c, batch, x, theta, psi_out, g_ez, d_theta, d_x, workspace, workspace_bytes, st);
}

QC_API qc_status qc_staging_bytes(const qc_circuit* c, int batch, size_t* bytes) {
  if (!c || batch <= 0 || !bytes) return fail(QC_ERR_INVALID, "bad arguments");
  size_t b = 0;
  b += align256((size_t)batch * std::max(c->n_in, 1) * 8);  // x
  b += align256((size_t)std::max(c->n_theta, 1) * 8);       // theta
  b += align256((size_t)batch * c->n * 8);                  // g
  b += align256((size_t)batch * c->n * 8);                  // ez
  b += align256((size_t)std::max(c->n_theta, 1) * 8);       // d_theta
  b += align256((size_t)batch * std::max(c->n_in, 1) * 8);  // d_x
  *bytes = b;
  return QC_OK;
}

QC_API qc_status qc_step_host(qc_circuit* c, int batch, const double* x_h, const double* th_h,
                              const double* g_h, double* ez_h, double* dth_h, double* dx_h,
                              void* psi_out, void* workspace, size_t wbytes, void* staging,
                              void* stream) {
  qc_status s = check_common(c, batch);
  if (s != QC_OK) return s;
  if (!staging || !g_h) return fail(QC_ERR_INVALID, "staging and g_ez_host must be non-NULL");
  cudaStream_t st = (cudaStream_t)stream;
  char* sp = (char*)staging;
  size_t o = 0;
  double* x = (double*)(sp + o); o += align256((size_t)batch * std::max(c->n_in, 1) * 8);
  double* th = (double*)(sp + o); o += align256((size_t)std::max(c->n_theta, 1) * 8);
  double* g = (double*)(sp + o); o += align256((size_t)batch * c->n * 8);
  double* ez = (double*)(sp + o); o += align256((size_t)batch * c->n * 8);
  double* dth = (double*)(sp + o); o += align256((size_t)std::max(c->n_theta, 1) * 8);
  double* dx = (double*)(sp + o);
  cudaError_t e = cudaSuccess;
  if (c->n_in > 0 && x_h) e = cudaMemcpyAsync(x, x_h, (size_t)batch * c->n_in * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && c->n_theta > 0 && th_h) e = cudaMemcpyAsync(th, th_h, (size_t)c->n_theta * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g, g_h, (size_t)batch * c->n * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "host->device copy");
  s = qc_forward(c, batch, x, th, psi_out, ez, workspace, wbytes, stream);
  if (s != QC_OK) return s;
  s = qc_backward(c, batch, x, th, psi_out, g, dth, dx, workspace, wbytes, stream);
  if (s != QC_OK) return s;
  if (ez_h) e = cudaMemcpyAsync(ez_h, ez, (size_t)batch * c->n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && dth_h && c->n_theta > 0) e = cudaMemcpyAsync(dth_h, dth, (size_t)c->n_theta * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && dx_h && c->n_in > 0) e = cudaMemcpyAsync(dx_h, dx, (size_t)batch * c->n_in * 8, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "device->host copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return QC_OK;
}

QC_API qc_status qc_wait(void* stream, int timeout_ms) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  e = cudaEventRecord(ev, st);
  if (e != cudaSuccess) { cudaEventDestroy(ev); return cuda_fail(e, "cudaEventRecord"); }
  // host-side polling with a limit; the device never spins
  const long long limit_us = (long long)timeout_ms * 1000;
  long long waited = 0;
  while (true) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) { cudaEventDestroy(ev); return cuda_fail(e, "cudaEventQuery"); }
    if (waited >= limit_us) { cudaEventDestroy(ev); return fail(QC_ERR_TIMEOUT, "stream still busy after timeout"); }
    struct timespec ts = {0, 200000};
    nanosleep(&ts, nullptr);
    waited += 200;
  }
  cudaEventDestroy(ev);
  return QC_OK;
}

QC_API unsigned long long qc_launch_count(void) { return g_launches; }

QC_API unsigned long long qc_alloc_count(void) { return g_alloc_calls; }

QC_API qc_status qc_kernel_timeouts(unsigned long long* count) {
  if (!count) return fail(QC_ERR_INVALID, "count is NULL");
  count_alloc();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  *count = tma_take_timeouts_fwd() + tma_take_timeouts_bwd() + tc_take_timeouts();
  return QC_OK;
}

QC_API qc_status qc_profile_enable(int on) {
  g_prof = on != 0;
  g_nrec = 0;
  return QC_OK;
}

QC_API qc_status qc_profile_summary(char* buf, size_t len) {
  count_alloc();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  double ms[PC_N] = {0}, bytes[PC_N] = {0};
  long long cnt[PC_N] = {0};
  for (size_t i = 0; i < g_nrec; ++i) {
    float t = 0;
    if (cudaEventElapsedTime(&t, g_recs[i].a, g_recs[i].b) != cudaSuccess) continue;
    ms[g_recs[i].cls] += t;
    bytes[g_recs[i].cls] += g_recs[i].bytes;
    cnt[g_recs[i].cls] += 1;
  }
  std::string o;
  char line[256];
  for (int k = 0; k < PC_N; ++k) {
    if (!cnt[k]) continue;
    snprintf(line, sizeof line, "%s %lld %.6f %.6e\n", kProfNames[k], cnt[k], ms[k], bytes[k]);
    o += line;
  }
  if (buf && len) {
    size_t k = std::min(len - 1, o.size());
    memcpy(buf, o.data(), k);
    buf[k] = 0;
  }
  return QC_OK;
}

// Text description of the plan for `batch` (host only; for tests and tools).
QC_API qc_status qc_describe_plan(const qc_circuit* cc, int batch, char* buf, size_t len) {
  qc_circuit* c = const_cast<qc_circuit*>(cc);
  qc_status s = check_common(c, batch);
  if (s != QC_OK) return s;
  Plan* p;
  s = get_plan(c, batch, &p);
  if (s != QC_OK) return s;
  std::string o;
  char line[512];
  snprintf(line, sizeof line, "path=%s nlead=%d nckpt=%d ws_fwd=%zu ws_bwd=%zu jobs=%zu outs=%zu overlap=%d\n",
           p->smem ? "smem" : "layer", p->nlead, p->nckpt, p->ws_fwd, p->ws_bwd, p->jobs.size(),
           p->outs.size(), (int)p->overlap);
  o += line;
  auto dump = [&](const char* tag, const std::vector<Step>& v) {
    for (auto& st : v) {
      if (st.type == ST_TILE) {
        // post: 0 none, 1 a following diagonal's phase, 2 the same with the
        // contiguous pass's compile-time element patterns
        const int post = !st.tp.post ? 0
                         : (st.ns == 1 && st.rb == 4 && c->dtype == QC_C64 && fwd_post_contig(st.tp)) ? 2 : 1;
        snprintf(line, sizeof line, "%s layer=%d TILE ns=%d t=%d c=%d h0=%d rb=%d cps=%d stages=%d rounds=%d ops=%d slots=%d defer=%d store=%d pre=%d post=%d xl=%d tma=%d tc=%d src=%d dst=%d",
                 tag, st.layer, st.ns, st.tp.t, st.tp.c, st.tp.h0, st.rb, st.cps, st.tp.nstage, st.tp.nrounds, st.tp.nops, st.tp.nslots,
                 st.tp.defer,
                 st.tp.store, st.tp.pre, post, st.tp.xload, st.tma, st.tc, st.s0, st.d0);
        o += line;
        for (int k = 0; k < st.tp.nops; ++k) {
          snprintf(line, sizeof line, " [l=%d%s np=%d%s]", st.tp.ops[k].l, st.tp.ops[k].is2q ? ",2q" : "",
                   st.tp.ops[k].np, st.tp.ops[k].ck ? (st.tp.ops[k].ck == 1 ? " +X" : " +Y") : "");
          o += line;
        }
        o += "\n";
      } else if (st.type == ST_DIAG) {
        snprintf(line, sizeof line, "%s layer=%d DIAG ns=%d xcomp=%d z=%d cb=%d src=%d dst=%d\n", tag, st.layer, st.ns,
                 st.dp.xcomp, st.dp.zmode, st.dp.cb, st.s0, st.d0);
        o += line;
      } else if (st.type == ST_RING) {
        snprintf(line, sizeof line, "%s layer=%d RING ns=%d whole=%d t=%d pre=%d src=%d dst=%d\n", tag, st.layer,
                 st.ns, st.rp.whole, st.rp.t, st.rp.pre, st.s0, st.d0);
        o += line;
      } else if (st.type == ST_PRODINIT) {
        snprintf(line, sizeof line, "%s layer=%d PRODINIT dst=%d\n", tag, st.layer, st.d0);
        o += line;
      } else if (st.type == ST_LAMINIT) {
        snprintf(line, sizeof line, "%s LAMINIT\n", tag);
        o += line;
      }
    }
  };
  dump("F", p->fwd);
  dump("B", p->bwd);
  if (buf && len) {
    size_t k = std::min(len - 1, o.size());
    memcpy(buf, o.data(), k);
    buf[k] = 0;
  }
  return QC_OK;
}

}  // extern "C"
