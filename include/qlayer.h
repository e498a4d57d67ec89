/*
 * qlayer.h -- C ABI of the GB300 layered QML state-vector simulator.
 *
 * The library applies whole layers of uniformly applied gates to a batch of
 * n-qubit state vectors (Sec. 2 of arXiv 2506.04891, "Techniques for Applying
 * Layers of Gates to a State Vector"), measures single-qubit <Z> (Sec. 3,
 * circuits whose "single-qubit observables <Z> are measured and summed") and
 * differentiates the measurement with a hand-written adjoint sweep.
 *
 * Conventions shared by every call
 * --------------------------------
 * State layout: psi[b][k], b < batch, k < 2^n, interleaved complex
 *   (float2 for QC_C64, double2 for QC_C128), batch-major, 16-byte aligned.
 *   Qubit q is bit (n-1-q) of k: qubit 0 is the most significant bit, as in
 *   the binary counting matrix J printed in Sec. 2.4.1.
 * Parameters: x and theta are always float64 (device pointers).  x[b][j] is
 *   sample b's input vector (n_input_per_sample columns); theta[p] is the
 *   trainable vector shared by the batch.  A layer reads its parameters at
 *   x[b][offset + j] (QC_SRC_INPUT) or theta[offset + j] (QC_SRC_THETA);
 *   QC_SRC_NONE means every parameter of the layer is 0.
 * Parameter count of a layer: n for RX, RY, RZ, GPI, GPI2 (parameter j acts on
 *   qubit j) and ISINGZZ_RING (parameter j acts on qubits (j, j+1 mod n));
 *   3 per gate for MS_BRICK ((phi0, phi1, theta) of gate i at offset+3i);
 *   0 for CNOT_RING, X, SX, ECR_BRICK.
 * Ring layers: CNOT_RING is CNOT(q -> q+1 mod n) applied for q = 0..n-1 in
 *   that order (Sec. 2.3); ISINGZZ_RING follows the K_Rzz definition of
 *   Sec. 2.4.1 (for n = 2 the pair (0,1) appears twice).  Ring layers need n >= 2.
 * Brick layers (MS_BRICK, ECR_BRICK): gates on qubit pairs (parity + 2i,
 *   parity + 2i + 1), no wrap-around; the first qubit of a pair is the more
 *   significant index of the 4x4 matrix.
 * Gate matrices: Appendix A, with angles of GPI/GPI2/MS in turns as printed.
 *   Two printed matrices are not unitary; the library uses ECR =
 *   (I(x)X - X(x)Y)/sqrt(2) (reproduces the two printed rows) and MS with entry
 *   (3,0) = -i exp(+2 pi i (phi0+phi1)) sin(pi theta).
 *
 * Ownership: every device buffer passed in belongs to the caller.  A circuit
 *   handle owns one device buffer, the partial sums of qc_expect_z, which
 *   qc_create allocates and qc_destroy frees.  The plan tables a call needs
 *   (coefficient and reduction jobs) are written into the caller's workspace
 *   by each qc_forward / qc_backward, in stream order, so after qc_create no
 *   compute call allocates device memory, frees it or synchronises the
 *   device (qc_alloc_count counts the calls that do).
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Every
 *   compute call only enqueues work on that stream and returns; it never
 *   synchronises unless its description says so.
 * Errors: every call returns a qc_status and never aborts.  Invalid arguments
 *   are rejected on the host before anything is enqueued (QC_ERR_INVALID);
 *   a failed launch returns QC_ERR_CUDA.  qc_last_error() returns a
 *   thread-local message describing the last failure on the calling thread.
 * Thread safety: one circuit handle must not be used from two threads at once.
 */
#ifndef QLAYER_H
#define QLAYER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define QC_API __attribute__((visibility("default")))
#else
#define QC_API
#endif

typedef struct qc_circuit qc_circuit;

typedef enum {
  QC_OK = 0,
  QC_ERR_INVALID = 1,     /* bad argument, rejected on the host */
  QC_ERR_OOM = 2,         /* workspace too small / device allocation failed */
  QC_ERR_CUDA = 3,        /* a CUDA call or launch failed */
  QC_ERR_TIMEOUT = 4,     /* qc_wait: the stream did not finish in time */
  QC_ERR_UNSUPPORTED = 5  /* valid request this build does not implement */
} qc_status;

typedef enum { QC_C64 = 0, QC_C128 = 1 } qc_dtype;

typedef enum {
  QC_L_RX = 0,            /* rotation layers (Appendix A, single qubit rotation) */
  QC_L_RY = 1,
  QC_L_RZ = 2,            /* diagonal (Sec. 2.4, Eigenphase / Tensor Product) */
  QC_L_ISINGZZ_RING = 3,  /* diagonal ring of Rzz (Sec. 2.4.1, K_Rzz) */
  QC_L_CNOT_RING = 4,     /* permutation layer (Sec. 2.3) */
  QC_L_X = 5,             /* permutation layer: k -> 2^n - 1 - k */
  QC_L_SX = 6,            /* fixed single-qubit gate */
  QC_L_GPI = 7,           /* anti-diagonal (Sec. 2.4.1, GPI mapping) */
  QC_L_GPI2 = 8,          /* IonQ native single-qubit gate */
  QC_L_MS_BRICK = 9,      /* IonQ native two-qubit gate on a brick pattern */
  QC_L_ECR_BRICK = 10,    /* IBM native two-qubit gate on a brick pattern */
  QC_L_Z = 11,            /* diagonal constants on every qubit (Appendix A, (anti)diagonal) */
  QC_L_S = 12,
  QC_L_H = 13,            /* fixed gate (Appendix A, fixed gates) */
  QC_L_CZ_BRICK = 14,     /* diagonal two-qubit constant on a brick pattern */
  QC_L_SWAP_BRICK = 15,   /* permutation two-qubit constant on a brick pattern */
  QC_L_ROT = 16           /* Rot(theta, phi, lambda) as printed in Appendix A: three
                             parameters per qubit, qubit j reads offset + 3j + {0, 1, 2};
                             run as e^{i(phi+lambda)/2} RZ(phi) RY(theta) RZ(lambda) */
} qc_layer_kind;

typedef enum { QC_SRC_NONE = 0, QC_SRC_THETA = 1, QC_SRC_INPUT = 2 } qc_source;

typedef struct {
  int32_t kind;    /* qc_layer_kind */
  int32_t source;  /* qc_source */
  int32_t offset;  /* index of the layer's first parameter in theta or x[b] */
  int32_t parity;  /* brick layers: 0 or 1; ignored otherwise */
} qc_layer;

typedef struct {
  /* Adjoint re-anchoring checkpoints: keep the forward state after every
   * ckpt_every-th layer in the workspace; the backward sweep reads psi from
   * there instead of its uncomputed copy.  -1 = automatic (on for states of
   * 1 GiB or more), 0 = off. */
  int32_t ckpt_every;
  /* 0 = automatic (the shared-memory path for n <= 10 with QC_C64 and n <= 8
   * with QC_C128 at batch <= 128, where the layer path is launch-bound; the
   * layer path otherwise); 1 = whole circuit per sample in shared memory
   * (n <= 13 for QC_C64 and n <= 12 for QC_C128); 2 = layer-by-layer HBM
   * passes. */
  int32_t path;
  /* Layer path: 1 (default) fuses what the planner can fuse (leading
   * single-qubit layers into the product-state init, <Z> into the last
   * forward pass, lambda init into the first backward pass); 0 = one kernel
   * pass per layer. */
  int32_t fuse;
  /* Layer-path tile geometry (0 = the planner's default).  tile_bits_*: log2
   * amplitudes per shared-memory tile (forward default 12 for QC_C64, 11 for
   * QC_C128; backward 12 / 10; allowed 6 .. 13 / 12 forward, 6 .. 12 / 11
   * backward).  reg_bits_*: index bits held in registers per round (1 .. 4;
   * defaults 4, except in the backward: 3 for QC_C128, and one less again
   * for the passes of complex single-qubit layers (3 for QC_C64 where the
   * layer has gradients, 2 for QC_C128) and, in QC_C128, of every brick
   * layer (2); the planner raises
   * it where a pass needs more: two for brick layers, and at most eight
   * rounds per pass; a QC_C64 brick pass whose pairs start at odd bits takes
   * 3 where 4 would keep it from TMA staging).
   * stages_*: shared-memory tile buffers per CTA (1, 2 or 3; default 2, 1 for
   * the QC_C64 backward; 3 only
   * where two CTAs per SM still fit; with 1 the CTAs of an SM overlap each
   * other's copies instead of their own).  A tuner may try
   * several (paper_2506_04891_gb300.tune); results never depend on them
   * beyond rounding.  A field left at 0 takes, at qc_create, the process
   * environment variable QC_TMAX_FWD, QC_TMAX_BWD, QC_RB_FWD, QC_RB_BWD or
   * QC_TILE_STAGES (both sweeps) when set; out-of-range values, from either
   * source, make qc_create return QC_ERR_INVALID. */
  int32_t tile_bits_fwd;
  int32_t tile_bits_bwd;
  int32_t reg_bits_fwd;
  int32_t reg_bits_bwd;
  int32_t stages_fwd;
  int32_t stages_bwd;
  /* Tile copies of the QC_C64 layer path: 1 (default) = TMA
   * (cp.async.bulk.tensor, mbarrier completion) wherever the pass geometry
   * allows (2^12-amplitude tiles with at least 16 contiguous amplitudes, no
   * gathered loads; the planner also checks that every register round reads
   * shared memory without bank conflicts), per-thread cp.async copies
   * elsewhere; 0 = per-thread copies everywhere.  With the default 1, the
   * process environment variable QC_TMA=0 (read at qc_create) turns it off. */
  int32_t tma;
  /* Experiment, default 0: 1 runs every eligible forward pass of a real
   * single-qubit layer (one gate on each of the 7 high bits of a 2^12 tile
   * with 32 contiguous amplitudes, nothing fused) as one 128 x 128 dense
   * block on the tensor cores (tcgen05.mma kind::tf32, 3xTF32 split, FP32
   * accuracy).  On GB300 it is slower than the register rounds of the tile
   * pass, which stay the default.  The process environment variable
   * QC_TC_DENSE=1 (read at qc_create) turns it on when the field is 0. */
  int32_t tc_dense;
} qc_options;

/* Version of this ABI (major * 100 + minor). */
QC_API int qc_version(void);

/* Fills *opt with the defaults {-1, 0, 1, 0, 0, 0, 0, 0, 0, 1, 0}. */
QC_API void qc_default_options(qc_options* opt);

/* Validates a layer list and builds a circuit for n qubits (1 <= n <= 30).
 * `layers` (host memory, n_layers >= 0 entries) is copied.  `opt` may be
 * NULL for defaults.  On success *out receives a handle; on failure *out is
 * left NULL.  On the current device it allocates the qc_expect_z scratch
 * (max(2 MiB, 8 (n+1) 2^(n - min(n,14)) bytes)) and loads the <Z> kernels;
 * without a usable device the handle still serves the host-only calls
 * (planning, sizes, descriptions). */
QC_API qc_status qc_create(int n, qc_dtype dtype, const qc_layer* layers, int n_layers,
                           const qc_options* opt, qc_circuit** out);

/* Frees the handle and its device tables (synchronises the device first).
 * NULL is accepted. */
QC_API qc_status qc_destroy(qc_circuit* c);

/* Number of theta entries and per-sample x columns the circuit reads. */
QC_API qc_status qc_num_params(const qc_circuit* c, int* n_theta, int* n_input_per_sample);

/* Device workspace qc_forward / qc_backward need for `batch` samples
 * (host only: plans the batch, at most 16 plans are kept per handle). */
QC_API qc_status qc_workspace_bytes(const qc_circuit* c, int batch, size_t* bytes);

/* Forward pass (Sec. 2/3): psi_out[b] = U_L ... U_1 |0...0> for b < batch.
 *   x        device, [batch][n_input_per_sample] float64 (NULL if none read)
 *   theta    device, [n_theta] float64 (NULL if none read)
 *   psi_out  device, [batch][2^n] complex, written
 *   ez       device, [batch][n] float64 or NULL: if given, <Z_q> of psi_out
 *            is written too (same values as qc_expect_z)
 *   workspace device, >= qc_workspace_bytes(batch) bytes, 256-byte aligned;
 *            on return it holds the re-anchoring checkpoints that the next
 *            qc_backward of the same inputs reads. */
QC_API qc_status qc_forward(qc_circuit* c, int batch, const double* x, const double* theta,
                            void* psi_out, double* ez, void* workspace, size_t workspace_bytes,
                            void* stream);

/* <Z_q> per sample: ez[b][q] = sum_k |psi[b][k]|^2 (1 - 2 bit_{n-1-q}(k)).
 * psi: device [batch][2^n] complex; ez: device [batch][n] float64.
 * Reductions are deterministic (fixed order, float64 above the thread level).
 * Large batches run as several launches that reuse the handle's scratch in
 * stream order, so two calls on one handle must not overlap on the GPU. */
QC_API qc_status qc_expect_z(qc_circuit* c, int batch, const void* psi, double* ez, void* stream);

/* <Z_q> exactly as qc_expect_z computes it, for callers that must not
 * allocate device memory while they run.  (The paper has no counterpart:
 * this entry point exists for the library's users, not for the method.)
 * Who needs it: a caller whose device memory is wholly held by another
 * allocator (a framework's caching pool, a budget reserved at start-up), or
 * whose loop cannot afford the device-wide synchronisation that a cudaMalloc
 * or cudaFree may cause.  The per-CTA partial sums live in a fixed array that
 * is part of this library's device image (8 MiB, held by every device that
 * loads the library until the process exits); qc_create resolves its address
 * and loads the kernels on the current device, so no call here loads code or
 * allocates.  If qc_create ran before the device was usable, the first call
 * does that set-up instead; make that first call outside any stream capture.
 * Limit: batch * 2^(n - min(n, 14)) * (n + 1) <= 2^20 partial sums (n = 26:
 * batch <= 9); larger requests return QC_ERR_INVALID and enqueue nothing.
 * Every call on a device shares the one array: calls that overlap on the GPU
 * (other streams, or other threads) race and give wrong results, so order
 * them (one stream, or events).  psi, ez and the return values are as for
 * qc_expect_z. */
QC_API qc_status qc_expect_z_noalloc(qc_circuit* c, int batch, const void* psi, double* ez,
                                     void* stream);

/* Adjoint backward of L = sum_b sum_q g_ez[b][q] <Z_q>_b.
 *   psi_out  the state qc_forward wrote for the same (x, theta); read only
 *   g_ez     device [batch][n] float64 upstream gradient dL/d<Z_q>
 *   d_theta  device [n_theta] float64 (overwritten; summed over the batch) or NULL
 *   d_x      device [batch][n_input_per_sample] float64 (overwritten) or NULL
 *   workspace the buffer the preceding qc_forward of the same inputs used when
 *            checkpoints are on (checked: same pointer and batch, else
 *            QC_ERR_INVALID). */
QC_API qc_status qc_backward(qc_circuit* c, int batch, const double* x, const double* theta,
                             const void* psi_out, const double* g_ez, double* d_theta,
                             double* d_x, void* workspace, size_t workspace_bytes, void* stream);

/* One training step from HOST buffers: copies x, theta and g_ez from host to
 * the device (pinned memory recommended), runs forward, <Z> and backward,
 * copies ez, d_theta and d_x back to the host and synchronises the stream.
 * Device buffers: psi_out ([batch][2^n]) and workspace as above, plus
 * `staging`, >= qc_staging_bytes(batch) bytes of device memory. */
QC_API qc_status qc_staging_bytes(const qc_circuit* c, int batch, size_t* bytes);
QC_API qc_status qc_step_host(qc_circuit* c, int batch, const double* x_host,
                              const double* theta_host, const double* g_ez_host,
                              double* ez_host, double* d_theta_host, double* d_x_host,
                              void* psi_out, void* workspace, size_t workspace_bytes,
                              void* staging, void* stream);

/* Waits for `stream` with a host-side limit (polling, never a device spin):
 * QC_ERR_TIMEOUT if it is still busy after timeout_ms milliseconds. */
QC_API qc_status qc_wait(void* stream, int timeout_ms);

/* Message for the last failed call on this thread ("" if none). */
QC_API const char* qc_last_error(void);

/* ---- diagnostics ----
 * qc_launch_count: number of kernels this library has enqueued in the process.
 * qc_profile_enable(1): from now on, bracket every enqueued kernel (or kernel
 *   pair) with CUDA events on its stream; (0) stops; both reset the records.
 * qc_alloc_count: number of device allocations, frees and device-wide
 *   synchronisations the library has made in the process (qc_create,
 *   qc_destroy and qc_profile_summary make them; the compute calls do not).
 * qc_profile_summary: synchronises the device and writes one line per kernel
 *   class, "name launches total_ms algorithmic_bytes", where the bytes are
 *   the state traffic the method needs per launch (each state read and written
 *   once per pass), summed over launches. */
QC_API unsigned long long qc_launch_count(void);
QC_API unsigned long long qc_alloc_count(void);
/* CTAs of TMA-staged tile passes that gave up waiting (2 s) for a tile copy
 * since the last call, which clears the count; such a CTA leaves its tiles
 * unprocessed.  Synchronises the device (diagnostics). */
QC_API qc_status qc_kernel_timeouts(unsigned long long* count);
QC_API qc_status qc_profile_enable(int on);
QC_API qc_status qc_profile_summary(char* buf, size_t len);

/* Measured arithmetic ceiling of the current device (diagnostics for the
 * roofline): kind 0 = FP32 fmaf, 1 = packed FP32x2 FMA (__ffma2_rn), 2 = FP64
 * fma; *tflops receives TFLOP/s at 2 flops per FMA lane.  Runs its own
 * kernels on a private stream and waits for them; allocates nothing. */
QC_API qc_status qc_fma_peak(int kind, double* tflops);

/* Text description of the plan for `batch` (host only: no device access):
 * one line per kernel pass with its geometry and buffers. */
QC_API qc_status qc_describe_plan(const qc_circuit* c, int batch, char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* QLAYER_H */
