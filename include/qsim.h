/*
 * qsim.h -- C ABI of the GB300 state-vector engine for reversible wiring
 * diagrams (J. R. Burger, "New approaches to quantum computer simulation in
 * a classical supercomputer").
 *
 * The engine applies a wiring diagram of L steps -- NOT, controlled-NOT,
 * Toffoli and multi-controlled NOT -- to a state vector of 2^M complex
 * amplitudes held in GPU memory.  Each step is a symmetric permutation
 * matrix with one unit entry per row (Sec. 2a), so the engine only moves
 * amplitudes: states come back bit-exact.
 *
 * Index convention (Sec. 2b): bit b of a state index is the paper's address
 * wire a(b+1); a(1) is the least significant bit.  A step's target bit is
 * the paper's 'goto' wire minus one; its control bits are the 'from' wires.
 *
 * Memory layout: amplitude i sits at byte offset i * sizeof(amplitude),
 * interleaved (re, im): two floats for QSIM_C64, two doubles for
 * QSIM_C128.  Host buffers passed in are owned by the caller and only read
 * or written during the call.  Device buffers are owned by the library
 * unless created with qsim_create_with_buffers.
 *
 * Errors: every int-returning call returns QSIM_OK (0) or a negative code;
 * qsim_last_error() then describes the failure (thread-local string).  A
 * call that fails validation changes nothing.  Calls on one context must
 * not overlap from different host threads.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QSIM_OK 0
#define QSIM_EINVAL (-1)   /* bad argument: M, dtype, step, size or pointer */
#define QSIM_ENOMEM (-2)   /* a device or host allocation failed          */
#define QSIM_ECUDA (-3)    /* a CUDA runtime call failed                   */
#define QSIM_ETIMEOUT (-4) /* a bounded device-side wait gave up           */
#define QSIM_EBUSY (-5)    /* admission refused: over the memory budget    */
#define QSIM_ENOTFOUND (-6)/* unknown request id                           */

#define QSIM_MAX_QUBITS 34 /* 2^34 amplitudes: 128 GiB (c64), 256 GiB (c128) */

typedef enum { QSIM_C64 = 0, QSIM_C128 = 1 } qsim_dtype;

/* One wiring-diagram step (Sec. 2b-2g).  The amplitude pair (i, i ^ 2^target)
 * is exchanged for every index i with (i & ctrl_mask) == ctrl_pol:
 *   ctrl_mask == 0          NOT on a(target+1)                (Sec. 2e)
 *   one bit in ctrl_mask    controlled-NOT, 'from' above or below 'goto'
 *                           (Sec. 2b, 2c, 2f)
 *   two bits                Toffoli (Sec. 2g)
 *   more bits               multi-controlled NOT (Sec. 2g)
 * ctrl_pol bit = 1 fires on |1> of that control, 0 on |0>.  Valid steps:
 * target < M, target not in ctrl_mask, ctrl_mask < 2^M, ctrl_pol a subset
 * of ctrl_mask, reserved == 0.  24 bytes, no padding. */
typedef struct qsim_step {
    uint32_t target;
    uint32_t reserved;
    uint64_t ctrl_mask;
    uint64_t ctrl_pol;
} qsim_step;

/* Kernel strategies.  AUTO lets the planner choose per segment. */
typedef enum {
    QSIM_STRATEGY_AUTO = 0,
    QSIM_STRATEGY_SWEEP = 1,  /* one in-place pass per step over the toggled
                                 pairs only (Sec. 2b 'intelligent looping') */
    QSIM_STRATEGY_TILE = 2,   /* in-place passes, each applying a run of steps
                                 whose targets lie in one tile of address bits
                                 (Sec. 2i: sequential steps processed together) */
    QSIM_STRATEGY_GATHER = 3, /* out-of-place passes k2(i) = k1(x(i)) with x
                                 evaluated per index (Sec. 2h product, final
                                 gather); needs a scratch buffer */
    QSIM_STRATEGY_INPLACE = 4 /* AUTO restricted to in-place passes: the state
                                 never leaves its buffer, no scratch is used */
} qsim_strategy;

typedef struct qsim_ctx qsim_ctx;

/* Statistics of the most recent qsim_apply_circuit on a context. */
typedef struct qsim_plan_stats {
    uint64_t steps_in;        /* steps passed in                                 */
    uint64_t steps_cancelled; /* adjacent equal steps removed (each is an involution) */
    uint64_t passes;          /* kernel launches over the state                  */
    uint64_t sweep_passes;    /* of which pair-swap sweeps                       */
    uint64_t tile_passes;     /* of which tile passes                            */
    uint64_t gather_passes;   /* of which index-gather passes                    */
    double algorithmic_bytes; /* sum over passes of bytes read + written as the
                                 method requires (untouched tiles/pairs excluded) */
    double full_pass_equiv;   /* algorithmic_bytes / (2 * state bytes)           */
    double est_ms;            /* the planner's cost-model estimate of the plan's
                                 device time on GB300 (ms)                        */
} qsim_plan_stats;

/* ---- context lifetime --------------------------------------------------- */

/* Create a context for a 2^M-amplitude state of the given dtype on the
 * current CUDA device, allocate its state (cudaMalloc, zero-filled; no scratch
 * until a gather pass needs one) and a private stream.  M in [1, QSIM_MAX_QUBITS].
 * Returns QSIM_EINVAL for bad M/dtype, QSIM_ENOMEM when the state does not fit. */
int qsim_create(uint32_t M, int dtype, qsim_ctx **out);

/* Create a context over caller-owned device memory (e.g. tensors from the
 * PyTorch caching allocator).  d_state: 2^M amplitudes, 256-byte aligned.
 * d_scratch: NULL or a second buffer of the same size, enabling gather
 * passes.  stream: a cudaStream_t (NULL = legacy default stream) on which
 * every kernel of the context runs.  The caller keeps ownership and must
 * keep the buffers alive until qsim_destroy.  After qsim_apply_circuit the
 * current state may sit in either buffer: ask qsim_state_device(). */
int qsim_create_with_buffers(uint32_t M, int dtype, void *d_state, void *d_scratch,
                             void *stream, qsim_ctx **out);

/* Release the context and every device buffer it owns.  NULL is ignored. */
void qsim_destroy(qsim_ctx *ctx);

/* ---- state transfer (the paper's k1 in, k2 out) -------------------------- */

/* Copy 2^M amplitudes from host memory into the state (k1, Sec. 2b).
 * n_amps must equal 2^M.  Synchronous with respect to host_amps. */
int qsim_load_state(qsim_ctx *ctx, const void *host_amps, size_t n_amps);

/* Set the state to the product state of App. 1 without sending 2^M
 * amplitudes: k1(i) = product over bits b of q_b(bit b of i), where qubits
 * holds 4*M doubles (re q_b(0), im q_b(0), re q_b(1), im q_b(1)) for b = 0
 * (the paper's a(1)) to M-1.  Computed on the device as the product of the
 * factors of the bits above the lowest min(M, 10) (three partial products of
 * up to 8 bits each) times the product of the factors of those lowest bits;
 * every partial product is taken in FP64 from the most significant bit down,
 * every real product and sum rounded separately.  complex128 multiplies the
 * partial products in FP64; complex64 in float-float arithmetic (about 48
 * significant bits, within 2^-42 of |k1(i)|) and rounds once at the end.
 * Queued on the context's stream; qubits is copied during the call. */
int qsim_load_product_state(qsim_ctx *ctx, const double *qubits);

/* Apply a circuit to the product state of App. 1 (qubits as for
 * qsim_load_product_state) without writing that state out first: when the
 * plan's first pass is a tile pass, it computes every source amplitude from
 * the qubits instead of loading it -- the product over the tile's outside
 * bits once per tile, over its high bits per tile for each of their values,
 * over its low bits once per pass, all in FP64; for complex64 the per-output
 * product of the last two is taken in float-float arithmetic (about 48
 * significant bits) and rounded once, for complex128 in FP64.  Other plans
 * start from qsim_load_product_state.  With compiled kernels on, the planner
 * also weighs a plan without closed passes (a closed pass cannot generate the
 * input) and keeps the one estimated cheaper with the input's cost included.
 * The context's state is overwritten.
 * d_probs NULL: no probabilities; else as qsim_apply_circuit_probabilities.
 * Errors as qsim_apply_circuit. */
int qsim_apply_circuit_product(qsim_ctx *ctx, const double *qubits, const qsim_step *steps, size_t L,
                               double *d_probs);

/* Copy the state (k2) to host memory; n_amps must equal 2^M.  Waits for all
 * work queued on the context and reports device-side errors. */
int qsim_read_state(qsim_ctx *ctx, void *host_amps, size_t n_amps);

/* As qsim_load_state, but queued on the context's stream without waiting:
 * host_amps must stay valid and unchanged until the next qsim_synchronize
 * (pinned memory makes the copy asynchronous).  Lets a caller overlap the
 * copy-in of one state with work on another context. */
int qsim_load_state_async(qsim_ctx *ctx, const void *host_amps, size_t n_amps);

/* Device pointer of the buffer that holds the current state. */
void *qsim_state_device(qsim_ctx *ctx);

/* ---- the wiring diagram ---------------------------------------------------- */

/* Apply steps[0], steps[1], ..., steps[L-1] in that order:
 * k2 = U_L ... U_1 k1 (Sec. 2a, 2h; Summary of Method).  All steps are
 * validated first; on QSIM_EINVAL nothing is applied.  The steps are copied
 * during the call.  Work is queued on the context's stream and the call
 * returns without waiting for it; errors of queued kernels surface at the
 * next qsim_synchronize / qsim_read_state / qsim_probabilities. */
int qsim_apply_circuit(qsim_ctx *ctx, const qsim_step *steps, size_t L);

/* qsim_apply_circuit followed by the FP64 probabilities of the new state
 * (the post-processing of Sec. 2b) into device memory d_probs (2^M doubles,
 * 8-byte aligned; not NULL), with the same results as qsim_apply_circuit +
 * qsim_probabilities_device(ctx, d_probs, NULL).  When the plan's last pass
 * is a tile or gather pass, that pass writes the probabilities beside the
 * amplitudes it stores (a tile pass then visits every tile), saving one
 * read of the state; otherwise a separate pass computes them.  Queued on
 * the context's stream like qsim_apply_circuit.  QSIM_EINVAL for a NULL or
 * misaligned d_probs or an invalid circuit (nothing is queued then). */
int qsim_apply_circuit_probabilities(qsim_ctx *ctx, const qsim_step *steps, size_t L,
                                     double *d_probs);

/* One measured candidate plan of qsim_autotune. */
typedef struct qsim_tune_result {
    int strategy;       /* QSIM_STRATEGY_* */
    int tile_bits;      /* tile width k for QSIM_STRATEGY_TILE (0: default)     */
    int low_bits;       /* contiguous low tile bits l (0: default)              */
    int jit;            /* compiled gather kernels allowed                      */
    double ms;          /* fastest forward application over the repetitions;
                           negative: the planner rejected the candidate         */
    uint64_t passes;    /* passes of the plan                                   */
} qsim_tune_result;

/* Measure candidate plans for this circuit on the context's own state and
 * keep the fastest (the strategy choice and tile shape of Sec. 2i's
 * segmentation, picked by timing instead of the cost model).  Candidates:
 * the cost model's choice (also restricted to in-place passes), the gathers
 * with and without compiled kernels
 * (when a second buffer is allowed), in-place tile passes for tile widths k
 * of the default and the two below it and run lengths l = 3..6, and per-step
 * sweeps when L <= 64.  Each candidate applies the circuit and then the
 * reversed circuit (every step is its own inverse), reps + 1 times, timing
 * the forward applications with CUDA events, so the state is unchanged at
 * the end, bit for bit.  Synchronous.  out (cap entries, may be NULL with
 * cap 0) receives the candidates fastest first; *n_out (may be NULL) their
 * count.  Afterwards the context's strategy, tile shape and compiled-kernel
 * switch are those of the fastest.  QSIM_EINVAL for an invalid circuit or
 * reps outside 1..100; profiling records are not touched. */
int qsim_autotune(qsim_ctx *ctx, const qsim_step *steps, size_t L, int reps, qsim_tune_result *out,
                  size_t cap, size_t *n_out);

/* The row array of the circuit's product (Sec. 2h) -- the information about
 * the unitary matrix that the paper's conclusions propose to keep for design
 * automation: d_rows[i] = x(i) with k2(i) = k1(x(i)) for k2 = U_L ... U_1 k1,
 * for all 2^M rows, written to device memory (2^M uint64, 8-byte aligned) on
 * the context's stream.  The state is not touched.  Every step is used (no
 * cancellation); QSIM_EINVAL for an invalid step or one with more than eight
 * controls. */
int qsim_row_array(qsim_ctx *ctx, const qsim_step *steps, size_t L, uint64_t *d_rows);

/* The paper's final gather for a stored row array (Sec. 2b, k2(i) = k1(x(i)),
 * with x as qsim_row_array writes it, Sec. 2h): d_out[i] = d_in[d_rows[i] mod
 * 2^M] for all 2^M rows, and with d_probs non-NULL also d_probs[i] = the FP64
 * probability of d_out[i] (as qsim_probabilities).  No context: d_in and
 * d_out (2^M amplitudes of dtype, distinct, aligned to one amplitude), d_rows
 * (2^M uint64, 8-byte aligned) and d_probs (2^M doubles) are caller-owned
 * device memory; the work is queued on stream (cudaStream_t, NULL = legacy
 * default) and the call returns without waiting.  loads_in_flight (0 = 8, or
 * 4, 8, 16) sets how many source reads each thread keeps in flight.  Rows are
 * reduced modulo 2^M, so no read leaves d_in.  QSIM_EINVAL for M outside
 * [1, QSIM_MAX_QUBITS], an unknown dtype, NULL or misaligned pointers,
 * d_in == d_out or another loads_in_flight. */
int qsim_gather_rows(const void *d_in, void *d_out, const uint64_t *d_rows, uint32_t M, int dtype,
                     double *d_probs, int loads_in_flight, void *stream);

/* Force a strategy for subsequent qsim_apply_circuit calls (tests and
 * tuning).  tile_bits: total tile width k (0 = default), low_bits: how many
 * of them are the lowest address bits (0 = default). */
int qsim_set_strategy(qsim_ctx *ctx, int strategy, int tile_bits, int low_bits);

/* Circuit-specialised gather kernels.  With enable = 1, every out-of-place
 * gather segment of at least 32 steps that is not a plain NOT/CNOT run (those
 * use GF(2) tables) is written out as CUDA source -- one bit-plane update per
 * step, the steps last to first -- and compiled for the GPU by NVRTC on first
 * use; the compiled kernel is cached for the life of the process, keyed by
 * (M, dtype, steps), and reused by every later apply of the same segment.
 * The first apply of a new circuit pays the compile time (about a second);
 * the general bit-sliced kernel runs when enable = 0 (the default).  Returns
 * QSIM_ECUDA from qsim_apply_circuit if NVRTC is not available. */
int qsim_set_jit(qsim_ctx *ctx, int enable);

/* Compile, without a GPU, the kernels that qsim_apply_circuit with jit on
 * would compile for this circuit (strategy GATHER), so that a later apply
 * finds them cached.  canonicalize as for qsim_set_canonicalize.
 * compile_ms (may be NULL) receives the compile time spent by this call. */
int qsim_jit_precompile(uint32_t M, int dtype, const qsim_step *steps, size_t L, int canonicalize,
                        double *compile_ms);

/* Affine (NOT/CNOT-only) gather segments, x(i) = A i ^ b over GF(2) (the
 * Sec. 2h product of such steps): with enable = 1 (default) they run as
 * coset-blocked tiles, whose reads and writes are aligned runs of 2^run_bits
 * amplitudes (run_bits 0: runs of 1 KiB; at most 7), moved through a
 * pipeline whose stages hold at least stage_kib KiB of tiles (0: 32; at most
 * 96); with enable = 0 each output reads its source directly (scattered
 * reads).  Results are identical.  QSIM_EINVAL for run_bits outside [0, 7] or
 * stage_kib outside [0, 96]. */
int qsim_set_coset(qsim_ctx *ctx, int enable, int run_bits, int stage_kib);

/* Testing hook for failure handling (no counterpart in the paper).  Arms the
 * next tile pass of this context only: its producer warp leaves before
 * issuing any copy, and the consumers' pipeline waits (mbarrier polls) give
 * up after poll_limit polls instead of the default of about 2^24, so every
 * wait runs out with no bulk copy in flight.  That pass changes no amplitude
 * and sets the context's error flag; the next qsim_synchronize or
 * qsim_read_state returns QSIM_ETIMEOUT and clears the flag, and the context
 * stays usable.  poll_limit must be in [1, 2^20] (QSIM_EINVAL otherwise).  A
 * pass that is not a tile pass leaves the hook armed. */
int qsim_set_wait_test(qsim_ctx *ctx, uint32_t poll_limit);

/* Adjacent equal steps cancel in pairs (each step is its own inverse,
 * Sec. 2a).  enable = 1 (default) removes them before planning; 0 applies
 * every step as given. */
int qsim_set_canonicalize(qsim_ctx *ctx, int enable);

/* Statistics of the last qsim_apply_circuit. */
int qsim_get_plan_stats(qsim_ctx *ctx, qsim_plan_stats *out);

/* Per-pass device timing (tracing).  With enable = 1, every pass launched by
 * qsim_apply_circuit is bracketed by CUDA events on the context's stream, and
 * the records accumulate over successive applies.  qsim_get_pass_times waits
 * for queued work and writes, for each recorded pass (at most cap), the
 * device time in milliseconds, the kernel (1 sweep, 2 tile, 3 affine gather,
 * 4 bit-sliced gather, 5 compiled gather, 6 probabilities from
 * qsim_probabilities_device, 7 coset gather, 8 closed tile pass) and its
 * algorithmic bytes (any pointer may be
 * NULL); *n_out receives the number of recorded launches.  When cap covers
 * them all the record is cleared. */
int qsim_set_profiling(qsim_ctx *ctx, int enable);
int qsim_get_pass_times(qsim_ctx *ctx, double *ms, uint32_t *kinds, double *alg_bytes,
                        size_t cap, size_t *n_out);

/* Wait for queued work (kernels and probability copies); returns
 * QSIM_ETIMEOUT / QSIM_ECUDA if a kernel failed. */
int qsim_synchronize(qsim_ctx *ctx);

/* ---- post-processing ----------------------------------------------------- */

/* FP64 basis-state probabilities p(i) = re^2 + im^2 into
 * host_probs[0 .. 2^M-1]; n must be 2^M.  complex64: the squares are exact
 * in FP64 and the sum is rounded once (identical to separately rounded
 * products).  complex128: im^2 rounded, then one fused multiply-add (within
 * one unit in the last place of separately rounded products).  norm_out (may be NULL) receives sum_i p(i), reduced in FP64 on the
 * device.  Synchronous. */
int qsim_probabilities(qsim_ctx *ctx, double *host_probs, size_t n, double *norm_out);

/* As qsim_probabilities without the norm, queued without waiting: the
 * probabilities are computed on the context's stream into a device buffer of
 * the context (2^M doubles, allocated on first use; if that allocation fails,
 * in chunks through two small buffers) and copied to host_probs (2^M
 * doubles; must stay valid and unread until the next qsim_synchronize) on a
 * second stream of the context.  qsim_synchronize waits for both. */
int qsim_probabilities_async(qsim_ctx *ctx, double *host_probs, size_t n);

/* qsim_apply_circuit, then the probabilities of the result to host_probs,
 * queued without waiting: the circuit's last tile or gather pass writes them
 * into the context's device buffer beside the amplitudes (see
 * qsim_apply_circuit_probabilities), and one copy on the context's second
 * stream brings them to host_probs (2^M doubles, valid after the next
 * qsim_synchronize).  Errors as qsim_apply_circuit; QSIM_EINVAL if n != 2^M. */
int qsim_apply_circuit_probabilities_async(qsim_ctx *ctx, const qsim_step *steps, size_t L,
                                           double *host_probs, size_t n);

/* As qsim_probabilities, into device memory d_probs (2^M doubles, 8-byte
 * aligned), queued on the context's stream.  norm_out (may be NULL) is a
 * host pointer; when given the call waits for the result. */
int qsim_probabilities_device(qsim_ctx *ctx, double *d_probs, double *norm_out);

/* ---- batches of independent circuits --------------------------------------- */

/* A batch runs n independent wiring diagrams, circuit i on its own
 * 2^M[i]-amplitude state, all of one dtype.  Not in the paper, which runs one
 * circuit at a time: many small circuits each leave most of the GPU idle
 * and pay a launch per pass, so a batch plans every circuit once (out-of-place
 * gather passes: GF(2) tables for NOT/CNOT runs, bit-sliced evaluation
 * otherwise, sweeps for steps with more than eight controls), groups the
 * p-th pass of every circuit into one persistent launch (level p), captures
 * the levels of a run into a CUDA graph and replays it.  Every step is
 * applied (no cancellation). */
typedef struct qsim_batch qsim_batch;

typedef struct qsim_batch_stats {
    uint64_t circuits;
    uint64_t levels;          /* persistent launches per run                 */
    uint64_t items;           /* work items per run (16384 outputs each)     */
    uint64_t passes;          /* circuit passes per run                      */
    uint64_t amplitude_steps; /* sum over circuits of 2^M[i] * L[i]          */
    double algorithmic_bytes; /* bytes read + written per run                */
    uint64_t arena_bytes;     /* device memory of the two state arenas       */
    void *stream;             /* cudaStream_t the batch runs on              */
    uint64_t coset_passes;    /* NOT/CNOT gathers read in coset-tile order   */
    uint64_t affine_passes;   /* NOT/CNOT gathers read row by row            */
    uint64_t sliced_passes;   /* bit-sliced gathers of other segments        */
    uint64_t sweep_passes;    /* in-place sweeps (steps beyond 8 controls)   */
} qsim_batch_stats;

/* Per-batch planning choices. */
typedef struct qsim_batch_options {
    uint32_t coset_min_qubits; /* NOT/CNOT circuits with M >= this read their
                                  sources in coset-tile order (aligned runs);
                                  smaller ones row by row (their states stay
                                  in L2).  qsim_batch_create uses 18.      */
} qsim_batch_options;

/* Plan and allocate a batch.  M[i] in [1, QSIM_MAX_QUBITS]; steps[i] points to
 * L[i] steps (copied).  The states start zero-filled.  Device memory: two
 * arenas of sum_i 2^M[i] amplitudes.  QSIM_EINVAL names the first invalid
 * circuit; QSIM_ENOMEM when the arenas do not fit. */
int qsim_batch_create(size_t n, const uint32_t *M, int dtype, const qsim_step *const *steps,
                      const size_t *L, qsim_batch **out);

/* qsim_batch_create with planning options (opts NULL: the defaults). */
int qsim_batch_create_ex(size_t n, const uint32_t *M, int dtype, const qsim_step *const *steps,
                         const size_t *L, const qsim_batch_options *opts, qsim_batch **out);
void qsim_batch_destroy(qsim_batch *b);

/* Copy circuit i's state in from / out to host memory (n_amps = 2^M[i]);
 * synchronous. */
int qsim_batch_load_state(qsim_batch *b, size_t i, const void *host_amps, size_t n_amps);
int qsim_batch_read_state(qsim_batch *b, size_t i, void *host_amps, size_t n_amps);

/* Device pointer of circuit i's current state. */
void *qsim_batch_state_device(qsim_batch *b, size_t i);

/* Apply every circuit once: one graph launch (asynchronous). */
int qsim_batch_run(qsim_batch *b);

/* Apply every circuit once with one plain kernel launch per circuit pass,
 * no graph (the comparison for qsim_batch_run; same kernels' arithmetic). */
int qsim_batch_run_plain(qsim_batch *b);

int qsim_batch_synchronize(qsim_batch *b);
int qsim_batch_info(qsim_batch *b, qsim_batch_stats *out);

/* ---- serving: continuous batching of simulation requests ------------------ */

/* A server accepts simulation requests at any time and keeps the GPU busy
 * with all of them (the paper has no counterpart).  Each request -- M, an
 * input state in host memory, a wiring diagram -- is validated and planned at
 * submission, then waits in arrival order (with bounded backfill, see
 * qsim_server_set_backfill) until its device memory fits in the server's HBM
 * budget, its result fits in the server's pinned host result arena, and the
 * uploads already queued are short (under 8 GiB).  Device memory is two
 * blocks: the input state plus plan tables (amp bytes per amplitude), and a
 * second buffer of amp bytes per amplitude when the plan has more than one
 * gather pass, else of 8.  A scheduler thread uploads admitted states on a
 * copy stream and runs rounds back to back: a round launches the next pass
 * of every request whose state is on the device as one persistent launch,
 * so requests that arrive while others run join the next round.  The last
 * gather pass writes only the FP64 probabilities (the served result), into
 * the buffer it does not read; then the other block returns to the budget,
 * the probabilities are copied into the result arena on a second copy
 * stream, and their block returns after the copy.  All steps are applied (no
 * cancellation). */
typedef struct qsim_server qsim_server;

typedef struct qsim_server_stats {
    uint64_t submitted, admitted, completed;
    uint64_t rounds;            /* persistent launches of request passes       */
    uint64_t launches;          /* all kernel launches                          */
    uint64_t active, waiting;   /* requests admitted / queued right now         */
    uint64_t budget_bytes;      /* HBM budget                                   */
    uint64_t in_use_bytes;      /* of it allocated to admitted requests now     */
    uint64_t peak_in_use_bytes;
    uint64_t host_in_use_bytes; /* result arena bytes held by unreleased results */
    double amplitude_steps;     /* sum over completed requests of 2^M * L       */
    uint64_t backfilled;        /* requests admitted ahead of the queue's head  */
    uint64_t h2d_bytes;         /* states copied in                             */
    uint64_t d2h_bytes;         /* probabilities copied out                     */
    double h2d_busy_ms;         /* summed durations of the state copies in and  */
    double d2h_busy_ms;         /* of the result copies out (completed requests) */
    double compute_busy_ms;     /* summed durations of the request-pass rounds  */
    double issue_ms, issue_ms_max; /* host time spent issuing the copies (total,
                                      longest): a copy from host memory that is
                                      not pinned runs while it is issued */
    uint64_t evicted;           /* running requests swapped out to host memory  */
    uint64_t swapped_in;        /* of them brought back to the device           */
} qsim_server_stats;

/* Reserve hbm_budget_bytes of device memory (one cudaMalloc) and a pinned
 * host result arena of host_result_bytes, create the streams and start the
 * scheduler thread on the current device. */
int qsim_server_create(size_t hbm_budget_bytes, size_t host_result_bytes, int dtype,
                       qsim_server **out);

/* Queue a request.  host_amps (2^M amplitudes of the server's dtype; pinned
 * memory uploads fastest) must stay valid and unchanged until the request is
 * done; steps are copied.  QSIM_EINVAL for an invalid circuit, QSIM_EBUSY if
 * the request could never fit the budgets.  *req_id identifies it. */
int qsim_server_submit(qsim_server *s, uint32_t M, const void *host_amps, const qsim_step *steps,
                       size_t L, uint64_t *req_id);

/* *done = 1 once the probabilities are in the result arena; then
 * *latency_ms (may be NULL) is submit-to-result time and *probs (may be NULL)
 * points at the 2^M FP64 probabilities, valid until qsim_server_release.
 * A request whose uploads could not be queued at admission (a failed CUDA
 * call) holds no memory and is complete but failed: poll returns QSIM_ECUDA
 * with the reason in qsim_last_error(), and it still needs releasing. */
int qsim_server_poll(qsim_server *s, uint64_t req_id, int *done, double *latency_ms,
                     const double **probs);

/* Report finished requests in completion order, each once: up to cap ids
 * (and their submit-to-result latencies, may be NULL) into the arrays;
 * *n_out receives how many. */
int qsim_server_drain(qsim_server *s, uint64_t *ids, double *latency_ms, size_t cap, size_t *n_out);

/* Return a finished request's result memory to the arena and forget it. */
int qsim_server_release(qsim_server *s, uint64_t req_id);

/* Block until no request is waiting or running (QSIM_ETIMEOUT after timeout_s). */
int qsim_server_wait_all(qsim_server *s, double timeout_s);

/* Admission policy.  Requests are admitted in arrival order; while the
 * oldest waiting request does not fit and has waited less than
 * max_head_wait_ms, later requests that fit are admitted ahead of it
 * (backfill, default 100 ms).  After that nothing passes it, so the budget
 * drains until it fits.  A negative value disables backfill (strict FIFO). */
int qsim_server_set_backfill(qsim_server *s, double max_head_wait_ms);

/* Copies in and out on two streams that overlap (n = 2, default) or on one
 * stream (n = 1).  QSIM_EBUSY while requests are running. */
int qsim_server_set_copy_streams(qsim_server *s, int n);

/* Upload each admitted state in copies of at most bytes (0, the default: one
 * copy per state); bytes must be 0 or at least 1 MiB and a multiple of 256
 * (QSIM_EINVAL otherwise).  Applies to requests admitted afterwards. */
int qsim_server_set_upload_chunk(qsim_server *s, size_t bytes);

/* Eviction (off by default, evict_after_ms < 0): once the head of the queue
 * has waited evict_after_ms without fitting the budget, running requests --
 * the most recently admitted first, between their passes -- are copied out
 * to blocks of the host result arena and their device memory returns to the
 * budget until the head fits (Sec. 1 and Sec. 5 trade memory for
 * processing; here whole states move to host memory and back).  A
 * swapped-out request returns, ahead of everything but the head, as soon as
 * it fits, and runs on from its next pass with the same result bits.  A
 * request is evicted only if its state fits the host arena. */
int qsim_server_set_eviction(qsim_server *s, double evict_after_ms);

/* Pause (paused != 0) or resume admission.  While paused, submitted requests
 * wait and admitted ones run to completion; e.g. to submit a group of
 * requests that should be admitted together. */
int qsim_server_set_paused(qsim_server *s, int paused);

int qsim_server_get_stats(qsim_server *s, qsim_server_stats *out);

/* Timeline of one finished request, in milliseconds since tracing was
 * switched on: host clock for submit/admit/done, device events for the
 * copies (start = when the copy stream reached the copy).  A device time
 * that could not be read is -1. */
typedef struct qsim_server_trace_record {
    uint64_t id;
    uint32_t M;
    uint32_t passes;
    uint64_t L;
    double submit_ms, admit_ms;
    double upload_start_ms, upload_end_ms;     /* state and tables in  */
    double compute_start_ms, compute_end_ms;   /* rounds with its passes (-1: none) */
    double download_start_ms, download_end_ms; /* probabilities out   */
    double done_ms;                            /* seen complete       */
} qsim_server_trace_record;

/* Switch per-request tracing on (clears the record and sets the time
 * origin) or off.  At most 2^22 records are kept. */
int qsim_server_set_tracing(qsim_server *s, int enable);

/* Move up to cap trace records (completion order) into out; *n_out gets
 * how many.  Returned records are removed from the server's record. */
int qsim_server_get_trace(qsim_server *s, qsim_server_trace_record *out, size_t cap, size_t *n_out);

/* Stop the scheduler, wait for queued GPU work and free everything. */
void qsim_server_destroy(qsim_server *s);

/* ---- host-only planning (no GPU needed) ------------------------------------ */

/* Plan a circuit exactly as qsim_apply_circuit would, without touching a GPU
 * (the segmentation of Sec. 2i into passes).  Inputs as for
 * qsim_set_strategy plus scratch_available (nonzero: gather passes allowed).
 * Outputs, each optional (NULL skips it):
 *   stats      -- as qsim_get_plan_stats
 *   order      -- circuit index of every applied step, in application order
 *                 (length = steps_in - steps_cancelled, at most cap)
 *   pass_ends  -- exclusive end in 'order' of each pass (length = passes)
 *   pass_kinds -- 1 sweep, 2 tile, 3 gather for each pass
 * Returns QSIM_EINVAL for invalid steps or when an output would exceed cap. */
int qsim_plan_circuit(uint32_t M, int dtype, const qsim_step *steps, size_t L, int strategy,
                      int tile_bits, int low_bits, int scratch_available, qsim_plan_stats *stats,
                      uint64_t *order, uint64_t *pass_ends, uint32_t *pass_kinds, size_t cap);

/* Planning options for qsim_plan_circuit_ex (the switches a context holds). */
typedef struct qsim_plan_options {
    int strategy;          /* qsim_strategy                                       */
    int tile_bits;         /* as qsim_set_strategy (0: default)                   */
    int low_bits;
    int scratch_available; /* nonzero: gather passes allowed                      */
    int jit;               /* nonzero: compiled gather kernels (qsim_set_jit)     */
    int coset;             /* nonzero: coset-blocked affine gathers (default on)  */
    int coset_run_bits;    /* as qsim_set_coset                                   */
    int canonicalize;      /* nonzero: adjacent equal steps cancel (default on)   */
    int closed_known;      /* nonzero: closed_delta is given                      */
    uint64_t closed_delta; /* address bits the circuit's net row map can change
                              (OR over all rows of x(i) ^ i; a context finds it
                              on the device when compiled kernels are on): with
                              jit, a closed tile pass is weighed               */
} qsim_plan_options;

/* qsim_plan_circuit with every planning switch, reporting per pass the kernel
 * variant (as qsim_get_pass_times: 1 sweep, 2 tile, 3 affine gather, 4
 * bit-sliced gather, 5 compiled gather, 7 coset gather, 8 closed tile pass)
 * and the cost model's
 * estimated time in ms (pass_est_ms, may be NULL).  opts NULL: defaults. */
int qsim_plan_circuit_ex(uint32_t M, int dtype, const qsim_step *steps, size_t L,
                         const qsim_plan_options *opts, qsim_plan_stats *stats, uint64_t *order,
                         uint64_t *pass_ends, uint32_t *pass_variants, double *pass_est_ms,
                         size_t cap);

/* ---- allocation-free variant (the paper has no counterpart) --------------- */

/* FP64 probabilities and norm of a state held in caller-owned device memory,
 * computed without a context and without allocating anything.  It serves
 * callers that cannot allocate device memory when they need the result: a
 * process whose GPU memory is wholly reserved by another allocator (such as
 * a framework's caching pool), a plug-in that a host application confines to
 * a fixed memory budget, or a latency-critical loop that must not enter the
 * driver's allocator.  (qsim_create allocates, so they cannot use a context.)
 *   d_state  2^M amplitudes of dtype, aligned to one amplitude; read only
 *   d_probs  NULL, or 2^M doubles receiving p(i) = re^2 + im^2 (as in
 *            qsim_probabilities)
 *   d_norm   one double receiving sum_i p(i)
 *   stream   cudaStream_t (NULL = legacy default stream); the work is queued
 *            there and the call returns without waiting
 * Scratch: the norm's per-block partial sums live in a fixed device array of
 * 1024 doubles (8 KiB) compiled into the library; every GPU that loads the
 * library holds it until the process exits.  The launch never uses more
 * than 1024 blocks, so every M in [1, QSIM_MAX_QUBITS] fits; M outside that
 * range, an unknown dtype, a NULL d_state/d_norm or a misaligned pointer
 * returns QSIM_EINVAL with a message in qsim_last_error().  Every call looks
 * up the array's device address (cudaGetSymbolAddress) in the CUDA context
 * current on the calling thread, so a later context on the same device or a
 * device reset leaves no stale address.  The first call in a context may load
 * the library's device code into it (CUDA loads modules lazily), and that load
 * reserves device memory for the module: make the first call (or any other
 * launch of this library) at start-up, while memory is still free, and before
 * any stream capture.  After that, a call allocates nothing.  All calls share the one array and every call overwrites it, so
 * calls whose work overlaps on the GPU (different streams, or several host
 * threads) race: serialise them.  Calls no cudaMalloc, cudaFree or other
 * allocating routine. */
int qsim_probabilities_noalloc(const void *d_state, uint32_t M, int dtype, double *d_probs,
                               double *d_norm, void *stream);

/* ---- diagnostics ------------------------------------------------------------ */

/* Message describing the last error on this host thread ("" if none). */
const char *qsim_last_error(void);

/* Library version string. */
const char *qsim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
