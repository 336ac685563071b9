/*
 * sv_api.h -- C ABI of the GB300 state-vector simulator (libsv.so).
 *
 * The library keeps the full vector of 2^n complex amplitudes resident in GPU
 * memory and applies gates to it in place.  The paper this follows describes
 * a Schroedinger simulator as exactly that: the state of an n-qubit circuit is
 * a 2^n complex vector, every circuit moment is a 2^n x 2^n matrix, and
 * simulation is matrix-vector multiplication whose cost grows linearly with
 * the number of gates (Sec. I-A "Background"; Sec. II "Methods", assumption
 * (a)).  Keeping the state on the device avoids the CPU<->GPU transfer cost
 * the paper identifies as the reason GPU simulation loses at small widths
 * (Sec. III, opening discussion); only scalars, samples and the small
 * circuit description cross the host link.
 *
 * Conventions shared by every entry point:
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - amplitudes are interleaved (re, im): SV_C64 = 2 x float (8 B per
 *     amplitude), SV_C128 = 2 x double (16 B per amplitude);
 *   - a k-qubit gate matrix is row-major 2^k x 2^k complex FP64 on the host,
 *     interleaved (re, im); bit j of its row/column index is targets[j];
 *   - a gate acts only where every control qubit is |1>.
 *
 * Ownership: the caller owns every device buffer (amplitudes, workspace) and
 * every host buffer.  A state handle borrows its buffers and must be
 * destroyed before they are freed.  The handle itself owns only host metadata
 * (plan caches, a pinned staging buffer, CUDA events).
 *
 * Streams: all work is enqueued on the stream given to sv_create.  Calls
 * returning host values (expectations, norms, samples, gradients)
 * synchronise that stream before they return; the others return as soon as
 * the work is enqueued.
 *
 * Errors: every entry point returns an sv_status; nothing throws or aborts
 * across the ABI.  Arguments are validated on the host before anything is
 * enqueued (qubits in range and distinct, controls disjoint from targets,
 * sizes, alignment).  On failure, sv_last_error() returns a thread-local
 * message describing the last error of the calling thread.  Device-side
 * waits are bounded: a wait that runs out sets a device flag and the call
 * reports SV_ETIMEOUT.
 */
#ifndef SV_API_H
#define SV_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SV_OK = 0,
  SV_EINVAL = 1,        /* bad argument (qubits, sizes, pointers, alignment) */
  SV_ENOMEM = 2,        /* workspace too small, or a host allocation failed */
  SV_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  SV_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
  SV_EUNSUPPORTED = 5   /* valid request this build does not implement */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

/* Arithmetic of fused dense blocks.  In the tensor-core modes the fusion
 * width defaults to 5 (complex64 states of >= 12 qubits).  Split-BF16 runs
 * inside 12-qubit tile passes unless sv_options.tile_m asks for another tile
 * size: every uncontrolled dense or diagonal block of up to 5 qubits goes to
 * the tensor cores, padded to 5 qubits with idle qubits of its tile, and
 * passes made only of such blocks (at most 6) take the pipelined tensor-core
 * kernel; blocks with controls stay on the CUDA cores.  Split-TF32 applies
 * dense 4- and 5-qubit blocks on the tensor cores (a 4-qubit block padded
 * with an idle qubit), as passes of their own unless tile_m is 12.
 * complex128 states always use FP64 CUDA-core arithmetic. */
typedef enum {
  SV_PREC_PLAIN = 0,       /* FP32 FMA on CUDA cores */
  SV_PREC_TC_BF16X3 = 1,   /* tensor cores, split-BF16 (3 products), FP32 accumulate */
  SV_PREC_TC_TF32X3 = 2    /* tensor cores, split-TF32 (3 products), FP32 accumulate */
} sv_prec;

/* Named gates (matrices built by the library in FP64; readings as in the
 * library documentation: U3 is OpenQASM's, SX/SY/SW are ((1+i)/2)(I - iP),
 * FSIM(theta, phi) acts on |01>,|10> with cos(theta), -i sin(theta) and
 * puts e^{-i phi} on |11>). */
typedef enum {
  SV_GATE_MATRIX = 0,   /* explicit matrix from sv_circuit.matrices */
  SV_GATE_H = 1, SV_GATE_X, SV_GATE_Y, SV_GATE_Z, SV_GATE_S, SV_GATE_SDG, SV_GATE_T,
  SV_GATE_TDG, SV_GATE_SX, SV_GATE_SY, SV_GATE_SW, SV_GATE_ID,
  SV_GATE_RX = 20, SV_GATE_RY, SV_GATE_RZ, SV_GATE_PHASE,  /* one angle */
  SV_GATE_U3 = 30,                                         /* three angles */
  SV_GATE_CZ = 40, SV_GATE_SWAP,                           /* two targets */
  SV_GATE_FSIM = 50                                        /* two targets, two angles */
} sv_gate;

typedef struct {
  int32_t gate;          /* sv_gate */
  int32_t n_targets;     /* 1..6 */
  int32_t n_controls;    /* 0..8 */
  int32_t param;         /* -1, or index into the parameter vector: angles[0] := params[param] */
  int32_t targets[6];
  int32_t controls[8];
  double angles[3];
  int64_t matrix_offset; /* SV_GATE_MATRIX: offset, in complex entries, into sv_circuit.matrices */
} sv_op;

typedef struct {
  int32_t n_qubits;
  int32_t n_ops;
  int32_t n_params;
  int32_t reserved;
  const sv_op *ops;          /* host array of n_ops */
  const double *matrices;    /* host FP64 interleaved complex pool (may be NULL if unused) */
} sv_circuit;

typedef enum {
  SV_MODE_TILED = 0,       /* fuse gates into blocks, group blocks into shared-memory tile passes */
  SV_MODE_PER_GATE = 1,    /* one global-memory pass per (fused) block */
  SV_MODE_TILED_GRAPH = 2  /* as TILED; sv_apply_circuit_batch replays its launch from a CUDA graph */
} sv_mode;

typedef struct {
  int32_t fusion_k;          /* 0 = default, 1 = no fusion, 2..6 = max qubits per fused block */
  int32_t tile_m;            /* 0 = default; else qubits held per shared-memory tile */
  int32_t prec;              /* sv_prec */
  int32_t mode;              /* sv_mode */
  uint64_t timeout_cycles;   /* 0 = default budget for bounded device waits */
} sv_options;

/* Pauli string: X on the bits of x_mask, Z on the bits of z_mask, Y where both
 * are set (P = i^{popcount(x&z)} X^x Z^z). */
typedef struct {
  uint64_t x_mask;
  uint64_t z_mask;
  double coeff;
} sv_pauli_term;

typedef struct sv_state sv_state;

/* ---------------------------------------------------------------------------
 * State handles (Sec. I-A: the state is the vector of 2^n amplitudes)
 * ------------------------------------------------------------------------- */

/* Workspace bytes a state of this size needs for reductions, sampling and
 * uploaded gate programs. */
size_t sv_workspace_bytes(int n_qubits, sv_dtype dtype);

/* Wrap caller-owned device memory as a state.
 *   amps_dev:  >= 2^n amplitudes of `dtype`, 256-byte aligned.
 *   ws_dev:    >= sv_workspace_bytes(n, dtype), 256-byte aligned.
 *   stream:    a cudaStream_t (NULL = legacy default stream).
 * The amplitudes are not initialised.  n_qubits in [1, 34].
 * Errors: SV_EINVAL (sizes, alignment, n), SV_ENOMEM (workspace), SV_ECUDA. */
sv_status sv_create(int n_qubits, sv_dtype dtype, void *amps_dev, size_t amps_bytes,
                    void *ws_dev, size_t ws_bytes, void *stream, sv_state **out);
sv_status sv_destroy(sv_state *s);

/* psi := |index>  (one write pass).  SV_EINVAL if index >= 2^n.
 * The handle then knows the state is a basis state: sv_apply_circuit
 * follows it through circuits whose every gate maps a basis state to a
 * basis state times a phase (X, CNOT, Toffoli and other multi-controlled X,
 * SWAP, Z, S, T, CZ, fSim(pi/2, phi), diagonal and monomial matrices, any
 * controls) on the host and rewrites two amplitudes, with no pass over the
 * state -- the reversible-arithmetic case of the paper's multiplier circuits
 * (Sec. III-A) and the sparsity remark of Sec. IV.  Every other library
 * call that writes the amplitudes ends this; a caller that writes the
 * amplitude buffer itself must call sv_mark_modified (or sv_set_basis /
 * sv_upload) before the next sv_apply_circuit. */
sv_status sv_set_basis(sv_state *s, uint64_t index);
/* Declare that the caller changed the amplitudes outside the library (for
 * example through the tensor that owns them): the handle forgets that the
 * state was a basis state.  Never fails for a valid handle. */
sv_status sv_mark_modified(sv_state *s);
/* Copy 2^n amplitudes host -> device / device -> host (bytes must equal the
 * state size); synchronous w.r.t. the host.  Used for checkpoints and for
 * end-to-end runs that start from a host state.  Page-locked host memory
 * (cudaHostAlloc / cudaHostRegister, e.g. a pinned torch tensor) aligned to
 * 16 bytes is moved by a copy kernel whose SMs read or write it directly
 * over the GPU's host link; other host memory goes through
 * cudaMemcpyAsync.  Errors: SV_EINVAL (null pointer, size mismatch),
 * SV_ECUDA. */
sv_status sv_upload(sv_state *s, const void *host, size_t bytes);
sv_status sv_download(sv_state *s, void *host, size_t bytes);
/* Wait for all work enqueued on the state's stream; reports device-side
 * errors raised by earlier calls: SV_ETIMEOUT when a bounded wait ran out,
 * SV_EUNSUPPORTED when a tile pass met a block its launch did not carry (an
 * internal invariant; the block was not applied).  Clears them. */
sv_status sv_synchronize(sv_state *s);

/* ---------------------------------------------------------------------------
 * Gate application (Sec. II: simulation is matrix-vector multiplication)
 * ------------------------------------------------------------------------- */

/* Apply one k-qubit gate (k = 1..6) with nctrl controls (0..8) in place.
 * matrix: host FP64 2^k x 2^k complex, row-major, interleaved.  If adjoint
 * is nonzero the conjugate transpose is applied.  The matrix is assumed
 * unitary; libraries built with SV_DEBUG, or any build run with the
 * environment variable SV_CHECK_UNITARY=1, check max |U^dagger U - I| <=
 * 1e-10 on the host for this call and for every MATRIX op of a circuit and
 * reject others with SV_EINVAL before anything is enqueued.  Errors:
 * SV_EINVAL for qubits out of range, duplicated, controls overlapping
 * targets, or a failed unitarity check. */
sv_status sv_apply_gate(sv_state *s, const int32_t *targets, int k, const int32_t *controls,
                        int nctrl, const double *matrix, int adjoint);

/* Apply a whole circuit in place: gates are fused into dense blocks of at
 * most opt->fusion_k qubits (products formed in FP64 on the host; gates only
 * move across gates on disjoint qubits), then grouped into shared-memory tile
 * passes so that each pass reads and writes the state once.
 *   params: host FP64 vector of c->n_params (may be NULL if none is used).
 *   opt:    may be NULL (defaults).
 * Fused blocks whose matrix is a 0/1 permutation (CNOT, Toffoli, C^3X and
 * their products) only move amplitudes inside the tile: a pass made only of
 * such blocks is composed on the host into one gather table per setting of
 * its global control qubits (at most 5 of them, tables within half the
 * program area) and moves each amplitude once, exactly; a state known to be
 * a basis state (see sv_set_basis) takes no pass at all when every gate
 * maps basis states to basis states.
 * Errors: SV_EINVAL (malformed op, width mismatch), SV_ENOMEM (program does
 * not fit the workspace). */
sv_status sv_apply_circuit(sv_state *s, const sv_circuit *c, const double *params,
                           const sv_options *opt);

/* Report how sv_apply_circuit would execute this circuit with these options:
 * the number of fused blocks and of tile passes (one kernel launch, one read
 * and one write of the state each).  Builds and caches the plan; launches
 * nothing.  Same errors as sv_apply_circuit. */
sv_status sv_plan_info(sv_state *s, const sv_circuit *c, const double *params, const sv_options *opt,
                       int64_t *n_blocks, int64_t *n_passes);

/* The arithmetic of that plan: real multiply-adds per state amplitude,
 * summed over its fused blocks.  A dense k-qubit block with c controls
 * costs 4 * 2^k / 2^c (each affected amplitude takes 2^k complex
 * multiply-adds of 4 real ones), a diagonal block 4 / 2^c; blocks run on
 * the tensor cores count as dense blocks of the size they run at (split-BF16
 * tile passes pad every block to 5 qubits: 128 each).  This is the work the tile passes'
 * arithmetic roofline counts (times 2^n amplitudes, 2 flops each).
 *   fma_per_amp: host pointer, receives the sum.
 * Builds and caches the plan; launches nothing.  Same errors as
 * sv_apply_circuit, and SV_EINVAL when fma_per_amp is NULL. */
sv_status sv_plan_fmas(sv_state *s, const sv_circuit *c, const double *params, const sv_options *opt,
                       double *fma_per_amp);

/* Apply circs[b] (with parameters params[b], host FP64, either may repeat)
 * to states[b] for b < B, states of any widths, in one call: every circuit
 * is fused and planned into tile passes as by sv_apply_circuit.  The narrow
 * states (passes with fewer tiles than the GPU has SMs) go through ONE
 * persistent launch: a cooperative kernel works through the queue of all
 * their (state, pass, tile) items in pass order, a tile of pass p waiting
 * until pass p-1 of its own state is complete (Sec. I motivates many
 * independent simulations: variational training evaluates many circuits).
 * The wide states, and programs with tensor-core passes, follow as ordinary
 * full-grid launches of their passes, spread over up to four library-owned
 * streams forked from the states' stream after that launch and joined back
 * into it (the call stays stream-ordered).  Waits are
 * bounded by opt->timeout_cycles polls (~128 ns each; 0 = about 1 s); a wait
 * that runs out stops the launch and the next sv_synchronize on states[0]
 * returns SV_ETIMEOUT.  With opt->mode == SV_MODE_TILED_GRAPH the counter
 * reset and the launch are captured once per batch layout and replayed as a
 * CUDA graph.  fusion_k / tile_m left at 0 take the autotuner's cached
 * choice for the circuit's shape, if any.  All states must be distinct and
 * share one stream and device; the first state's workspace holds the batch
 * tables.  Enqueues only (no synchronisation).  Errors: SV_EINVAL (arguments,
 * per-gate mode), SV_ENOMEM (batch tables exceed the first state's reduction
 * area), SV_ECUDA. */
sv_status sv_apply_circuit_batch(sv_state *const *states, int B, const sv_circuit *const *circs,
                                 const double *const *params, const sv_options *opt);

/* ---------------------------------------------------------------------------
 * Observables (Sec. I: simulated output values feed an error function)
 * ------------------------------------------------------------------------- */

/* out = sum_t coeff_t Re <psi|P_t|psi>; products in the state's precision,
 * accumulated in FP64.  Synchronises.  SV_EINVAL for masks beyond n. */
sv_status sv_expect(sv_state *s, const sv_pauli_term *terms, int n_terms, double *out_host);
/* out[q] = <Z_q> for q = 0..n-1 in one read pass.  Synchronises. */
sv_status sv_expect_z_all(sv_state *s, double *out_host);
/* Same values as sv_expect_z_all, for callers that cannot allocate device
 * memory: code running while a CUDA graph is being captured, plug-ins whose
 * host application owns the device allocator, or loops that may not pay an
 * allocation's implicit synchronisation.  The paper has no counterpart; this
 * is a service of this library.
 *   amps_dev:  2^n_qubits amplitudes of `dtype` on the current device,
 *              256-byte aligned (no state handle needed).
 *   out_dev:   device array of n_qubits doubles, written with <Z_q>.
 *   stream:    cudaStream_t the work is enqueued on; the call does not
 *              synchronise (read out_dev after the stream reaches it).
 * The call allocates nothing and uses no workspace: its block partial sums
 * go to one fixed array of 143,360 bytes inside the library, which every
 * GPU that loads the library keeps until the process exits.  The first call
 * on a device looks up that array's device address (once per device), so
 * make it before any stream capture.  All calls share the array: calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race and give wrong results; serialise them.
 * Errors: SV_EINVAL for null or misaligned pointers, pointers that are not
 * device (or managed) memory of the current device, an unknown dtype, or
 * n_qubits outside [1, 34] (the array's limit); SV_ECUDA if the runtime
 * cannot resolve the array or launch. */
sv_status sv_expect_z_all_noalloc(const void *amps_dev, int n_qubits, sv_dtype dtype, double *out_dev,
                                  void *stream);
/* norm2 = sum_x |psi_x|^2 (FP64 accumulation).  Synchronises. */
sv_status sv_norm(sv_state *s, double *norm2_out);
/* psi := psi / sqrt(sum |psi|^2); optionally returns the old norm^2. */
sv_status sv_renormalize(sv_state *s, double *norm2_out);
/* Measurement sampling: shot j returns the smallest x with
 * CDF(x) > u_j * sum|psi|^2, CDF the inclusive prefix sum of |psi_x|^2 in
 * index order (FP64), u_j = (SplitMix64(seed, j) >> 11) * 2^-53 where
 * SplitMix64(seed, j) is the j-th output of the sequential SplitMix64
 * generator seeded with `seed`.  out_host: n_shots uint64.  Synchronises. */
sv_status sv_sample(sv_state *s, int64_t n_shots, uint64_t seed, uint64_t *out_host);

/* ---------------------------------------------------------------------------
 * Differentiation (Sec. I: variational training needs the error function's
 * parameter gradient)
 * ------------------------------------------------------------------------- */

/* Adjoint-method gradient of E(theta) = <psi_out|H|psi_out>,
 * psi_out = circuit(theta) psi_in:  forward sweep on psi, lambda = H psi,
 * then a reverse sweep that un-applies each gate from both vectors and adds
 * Im<lambda|G_j|psi> for each parametric gate U_j = exp(-i theta G_j / 2)
 * (RX, RY, RZ; PHASE with G = diag(0, -2)); no tape of states is kept.
 *   psi:            in = psi_in; out = psi_out.
 *   lambda_scratch: a state of the same width and dtype (clobbered).
 *   params:         host FP64, c->n_params.
 *   expval_out:     host double; grad_out: host double[c->n_params].
 * Parametric gates must be uncontrolled single-qubit RX/RY/RZ/PHASE
 * (SV_EUNSUPPORTED otherwise).  Synchronises. */
sv_status sv_adjoint_grad(sv_state *psi, sv_state *lambda_scratch, const sv_circuit *c,
                          const double *params, const sv_pauli_term *terms, int n_terms,
                          const sv_options *opt, double *expval_out, double *grad_out);

/* Batched form: B parameter sets of one circuit, psi[b] / lam[b] as above,
 * params row-major B x n_params, expval_out[B], grad_out row-major
 * B x n_params.  All states must have the same width, dtype and stream. */
sv_status sv_adjoint_grad_batch(sv_state *const *psi, sv_state *const *lam, int B,
                                const sv_circuit *c, const double *params,
                                const sv_pauli_term *terms, int n_terms, const sv_options *opt,
                                double *expval_out, double *grad_out);

/* ---------------------------------------------------------------------------
 * Runtime services
 * ------------------------------------------------------------------------- */

/* Time candidate (fusion_k in 2..6, tile_m in 10..13, limited by n) pairs
 * for this circuit on `scratch` (its contents are clobbered; the circuit must
 * not be parametric) and write the fastest into *inout.  The choice is
 * cached per (n, dtype, op-count bucket, widest op) in memory and, if the
 * SV_TUNE_CACHE environment variable names a file, in that JSON file;
 * sv_apply_circuit and sv_apply_circuit_batch use it for options left at 0.
 * Only CUDA-core timings (inout->prec == SV_PREC_PLAIN) enter the cache, and
 * only calls in that precision mode read it: the tensor-core modes keep
 * 5-qubit blocks and 12-qubit tiles.  Synchronises. */
sv_status sv_autotune(sv_state *scratch, const sv_circuit *c, sv_options *inout);

/* Launch a one-thread kernel that waits, bounded by `polls` polls (~128 ns
 * each), on a device counter that nothing ever increments, and report the
 * outcome: SV_ETIMEOUT when the bound is reached (the expected result; the
 * context stays usable), SV_OK otherwise.  Exercises the same bounded wait
 * the persistent batch kernel uses, without any fault.  Synchronises
 * `stream`.  The paper has no counterpart. */
sv_status sv_wait_selftest(void *stream, uint64_t polls);

/* Number of kernels this library has launched in this process (all
 * devices).  Lets callers count device work without a profiler. */
uint64_t sv_kernel_launch_count(void);

/* Bound on the number of planned circuit programs the library keeps in host
 * memory (all state handles together; default 2048).  A program is cached
 * per (state, circuit, parameters, options) so repeated sv_apply_circuit
 * calls skip fusion and planning; beyond the bound the oldest entries are
 * dropped (a call that is using an entry keeps it alive until it returns).
 * max_programs <= 0 only queries.  Returns the previous bound.  Thread-safe.
 * The paper has no counterpart: this is a service of this library. */
int64_t sv_program_cache_limit(int64_t max_programs);

const char *sv_last_error(void);
const char *sv_status_string(sv_status st);

#ifdef __cplusplus
}
#endif
#endif /* SV_API_H */
