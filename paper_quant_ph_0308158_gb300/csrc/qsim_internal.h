// qsim_internal.h -- types shared by the host planner and the CUDA kernels.
//
// A circuit is executed as a list of passes over the state.  Each pass is
// one kernel launch of one of three strategies:
//   SWEEP  : one step, in place, visiting only the toggled amplitude pairs
//            (Sec. 2b 'intelligent looping').
//   TILE   : a run of steps whose targets all lie in a set S of k address
//            bits; each CTA holds the 2^k amplitudes of one tile (all other
//            bits fixed) in shared memory, applies the whole run there, and
//            writes the tile back in place (Sec. 2i: sequential steps
//            processed together).
//   GATHER : out-of-place k2(i) = k1(x(i)) with x evaluated per output index
//            (Sec. 2h product, Sec. 2b final gather); x is an affine map over
//            GF(2) for CNOT/NOT-only segments, else the step list itself.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qsim {

constexpr int kMaxTileBits = 14;      // 2^14 amplitudes per tile at most
constexpr size_t kMaxTileBytes = 128 * 1024;  // and 128 KiB of shared memory
constexpr int kMaxHighBits = 10;      // tile bits above the contiguous run (tile kernel)
constexpr int kMaxHighBitsClosed = 13;  // the same for closed passes
constexpr int kMaxTileSteps = 256;    // steps per tile pass (shared-memory list)
constexpr int kMaxGatherSteps = 4096; // steps per general gather pass
constexpr uint32_t kClosedMinQubits = 12;  // circuits examined for a closed pass
constexpr size_t kClosedMinSteps = 16;

// A tile step in the tile's local coordinates.  Local bit q < l is global bit
// q; local bit l + p is global bit high[p].  cl/pl: control mask/polarity on
// local bits; tmask: 1 << local target; co/po: control mask/polarity on the
// bits outside the tile (constant over a tile).
struct TileStep {
    uint32_t cl;
    uint32_t pl;
    uint32_t tmask;
    uint32_t pad;
    uint64_t co;
    uint64_t po;
};
static_assert(sizeof(TileStep) == 32, "TileStep layout");

// A step of a bit-sliced gather pass (16 bytes).  Bit planes live in shared
// memory as [plane][thread] words; plane M is all ones and stands in for an
// absent control.  Word x: target plane | nc << 8 | neg << 16 | slow << 24,
// where neg bit q marks control q as firing on |0> and slow is set when the
// step has more than two controls or any control on |0>.  Words y and z hold
// control planes 0..3 and 4..7 (one byte each; unused bytes = plane M).
constexpr int kSlicedThreads = 256;
constexpr int kSlicedMaxControls = 8;
struct SlicedStep {
    uint32_t x;
    uint32_t y;
    uint32_t z;
    uint32_t pad;
};
static_assert(sizeof(SlicedStep) == 16, "SlicedStep layout");

struct SweepParams {
    uint64_t n_pairs;   // 2^(M-1-c)
    uint64_t pol;       // control polarity
    uint64_t half;      // 1 << target
    uint32_t nins;      // number of zero-bit insertions (controls + target), <= M
    uint32_t ins[QSIM_MAX_QUBITS];  // insertion positions, ascending
};

struct TilePass {
    uint32_t k, l, nh;  // tile width, contiguous low bits, high bits
    uint32_t high[kMaxHighBitsClosed];
    uint32_t tma;       // 1: tensor-map copies (else one bulk copy per run)
    uint32_t tma_ndims; // dimensions of the view that carry tile bits
    uint32_t tma_start[6];    // first address bit of each dimension's range
    uint64_t tma_dim[5];      // extents in 8-byte elements
    uint64_t tma_stride[5];   // byte strides (dimension 0: element size)
    uint32_t tma_box[5];      // box extents
    uint32_t box_bytes;       // bytes moved by one copy
    uint32_t nrest;           // tile bits enumerated by separate copies
    uint32_t rest_pos[kMaxHighBitsClosed];
    uint32_t nout;      // address bits outside the tile (M - k)
    uint32_t outpos[40];  // their positions, in tile-id bit order: bits that
                          // are controls of some step come last (slowest)
    uint64_t n_tiles;   // 2^(M-k)
    uint32_t step_off;  // offset of this pass's steps in the TileStep buffer
    uint32_t nsteps;
    uint32_t all_local; // 1 when no step has a control outside the tile
    uint32_t affine;    // 1 when every step has at most one control (NOT/CNOT)
    double touched;     // estimated fraction of tiles with an active step
    double rebuilds;    // estimated permutation-table builds (tiles whose
                        // active steps differ from the tile before)
    // Closed pass (qsim_jit_closed): the segment's net row map changes only
    // address bits inside the tile, so each tile holds every source of its
    // outputs; the segment's steps (Plan::jit_steps) are compiled in and
    // evaluated per output, in place.
    uint32_t closed;
    uint32_t jit_off, jit_n;
};

struct GatherPass {
    uint32_t affine;     // 1: x(i) = A i ^ b through byte tables
    uint32_t jit;        // 1: circuit-specialised compiled kernel (jit.cu)
    uint32_t jit_off;    // offset of the segment's steps in Plan::jit_steps
    uint32_t jit_n;      // number of those steps
    uint32_t nbytes;     // index bytes covered by tables (affine)
    uint32_t table_off;  // offset of 256 * nbytes entries in the table buffer
    uint32_t step_off;   // general: offset in the SlicedStep buffer
    uint32_t nsteps;     // general: number of steps (applied last to first)
    uint64_t bvec;       // affine: constant term
    // Coset-blocked affine gather (gather_coset_kernel): the output space is
    // cut into cosets T(t) + S, S = span(low r bits, A^-1 of the low r bits),
    // so a tile's 2^(r+d) outputs are 2^d aligned runs of 2^r and its
    // sources are 2^d aligned runs of 2^r too.  Tables at coset_off in
    // Plan::gather_tables: out-base [ctb][256], source-base [ctb][256] (tile
    // index bytes), dstrun [2^d], srcrun [2^d], then the local permutation
    // (2^(r+d) u16, four per word).
    uint32_t coset;      // 1: run through gather_coset_kernel
    uint32_t cr, cd, ce; // run bits r, coset bits d, log2 of tiles per stage
    uint32_t ctb;        // tile-index bytes of the base tables
    uint32_t coset_off;
    uint64_t n_tiles;    // 2^(M - r - d)
};

enum PassKind : uint32_t { kSweep = 1, kTile = 2, kGather = 3 };
// Kernel variant reported by tracing: 1 sweep, 2 tile, 3 affine gather,
// 4 bit-sliced gather, 5 compiled gather, 7 coset-blocked affine gather,
// 8 closed tile pass (6 is the probabilities pass).
uint32_t pass_variant(const struct Pass &p);

struct Pass {
    PassKind kind;
    SweepParams sweep;
    TilePass tile;
    GatherPass gather;
    double alg_bytes;   // bytes read + written as the method requires
    uint32_t nsteps;    // circuit steps this pass applies
};

struct PlanOptions {
    int strategy = QSIM_STRATEGY_AUTO;
    int tile_bits = 0;  // 0: default for the dtype
    int low_bits = 0;   // 0: default for the dtype
    int lookahead = 512;
    size_t amp_bytes = 16;
    bool scratch_available = false;
    bool cancel_adjacent = true;
    bool jit = false;        // compile non-affine gather segments (jit.cu)
    bool coset = true;       // affine segments through coset-blocked tiles
    bool closed_known = false;  // closed_delta holds the bits the circuit's net map changes
    uint64_t closed_delta = 0;
    int coset_run_bits = 0;  // r of those tiles (0: runs of 1 KiB)
    int coset_stage_kib = 0; // pipeline stage of those passes (0: 32 KiB)
    int jit_min_steps = 32;  // shorter segments use the general kernel
};

struct Plan {
    std::vector<Pass> passes;
    std::vector<TileStep> tile_steps;
    std::vector<SlicedStep> sliced_steps;
    std::vector<uint64_t> gather_tables;
    std::vector<qsim_step> jit_steps;  // steps of compiled gather segments, circuit order
    std::vector<uint64_t> order;      // circuit step index of each applied step
    std::vector<uint64_t> pass_ends;  // exclusive end in 'order' of each pass
    uint64_t steps_in = 0;
    uint64_t cancelled = 0;
};

// Host planner (planner.cpp).  Returns QSIM_OK or QSIM_EINVAL with msg set.
int validate_steps(uint32_t M, const qsim_step *steps, size_t L, std::string *msg);
int make_plan(uint32_t M, const qsim_step *steps, size_t L, const PlanOptions &opt,
              Plan *plan, std::string *msg);
// The cost model's estimated device time of a plan / one pass (planner.cpp).
double plan_estimated_ms(const Plan &plan, uint32_t M, size_t amp);
double pass_estimated_ms(const Pass &p, uint32_t M, size_t amp);
// Estimated time of writing an App. 1 product state on its own, and of a
// plan applied to such an input: generated by its first (tile) pass when
// fused, else written first by its own pass.
double product_state_estimated_ms(uint32_t M, size_t amp);
double product_plan_estimated_ms(const Plan &plan, uint32_t M, size_t amp, bool fused);

// One circuit's pass inside a batched launch (batch.cu builds them).
struct BatchPass {
    const char *in;        // gather source (unused by sweeps)
    char *out;             // gather destination (NULL: probabilities only) / sweep state
    uint32_t M;
    uint32_t kind;         // 1 sweep, 3 affine gather, 4 bit-sliced gather,
                           // 7 affine gather in coset-tile order
    uint32_t nbytes;       // affine: table bytes
    uint32_t nsteps;       // bit-sliced: steps
    uint64_t bvec;         // affine: constant term
    const uint64_t *tables;       // affine tables (device); coset: the pass's coset tables
    const SlicedStep *steps;      // bit-sliced steps (device)
    double *probs;                // gathers: non-null = also write FP64 probabilities
    uint32_t cr, cd, ctb, pad;    // coset: run bits, coset bits, tile-index bytes
    SweepParams sweep;
};
// A work item: outputs (or sweep pairs) [start, start + count) of one pass;
// bit-sliced items start on a multiple of 16384 outputs.
struct BatchItem {
    uint32_t pass;
    uint32_t pad;
    uint64_t start;
    uint64_t count;
};
constexpr uint64_t kBatchItemOutputs = 16384;  // = 256 threads x 64 outputs

// Message returned by qsim_last_error() on this host thread (qsim_api.cu).
void set_last_error(const std::string &msg);

// Kernel launchers (kernels.cu).  All return cudaError_t as int.  A non-null
// d_probs makes a tile or gather pass also write the FP64 probabilities of
// the state it leaves (2^M doubles).
int launch_sweep(void *state, int amp_bytes, const SweepParams &p, int *d_err, void *stream);
// Testing hook for the tile pipeline's bounded waits (qsim_set_wait_test):
// poll_limit polls before a wait gives up (0: the default, seconds), and a
// producer warp that leaves before issuing any copy (the hook always sets
// both, so no wait gives up while a copy is in flight).
struct WaitTest {
    uint32_t poll_limit = 0;
    bool stall_producer = false;
};
// d_prod non-null: product input (App. 1) -- the pass computes its source
// amplitudes from the table block written by product_tables() instead of
// loading them (the state's previous contents are ignored).
int launch_tile(void *state, int amp_bytes, const TilePass &p, const TileStep *d_steps,
                int *d_err, double *d_probs, void *stream, const WaitTest *wt = nullptr,
                const double *d_prod = nullptr);
// Host tables of a product-input tile pass, as FP64 complex pairs: per
// address bit b < M its factors (q_b(0), q_b(1)) at [2b], [2b+1] (the block
// reserves 2 * QSIM_MAX_QUBITS entries), then the products over the tile's
// low l bits for each of their values, then over its high bits.
std::vector<double> product_tables(uint32_t M, const double *qubits, const TilePass &t);
int launch_gather(const void *in, void *out, int amp_bytes, uint32_t M, const GatherPass &p,
                  const uint64_t *d_tables, const SlicedStep *d_steps, int *d_err, double *d_probs,
                  void *stream);
int launch_probabilities(const void *state, int amp_bytes, uint64_t n, double *d_probs,
                         double *d_partials, int n_partials, double *d_norm, void *stream);
int probabilities_partials_needed();
// k2(i) = k1(rows[i] mod 2^M) with loads_in_flight (4, 8 or 16) reads per thread.
int launch_gather_rows(const void *in, void *out, const uint64_t *rows, int amp_bytes, uint32_t M,
                       double *d_probs, int loads_in_flight, void *stream);
size_t batch_smem_bytes(uint32_t max_sliced_M);
int launch_product_state(void *state, int amp_bytes, uint32_t M, const double *d_qubits, void *stream);
int launch_row_array(uint64_t *d_rows, uint32_t M, const SlicedStep *d_steps, uint32_t nsteps,
                     void *stream);
// Bit-sliced descriptors of a step list (planner.cpp); QSIM_EINVAL for a step
// with more controls than a descriptor holds.
int sliced_steps_of(uint32_t M, const qsim_step *steps, size_t L, std::vector<SlicedStep> *out,
                    std::string *msg);
int launch_batch_level(int amp_bytes, bool wide, const BatchPass *d_passes, const BatchItem *d_items,
                       uint32_t n_items, uint32_t *d_counter, size_t smem, void *stream);
size_t tile_smem_bytes(int amp_bytes, int k);
// Whether a product-input (App. 1) tile pass with this layout fits in shared memory.
bool tile_product_fits(const TilePass &t);
// The tensor map (128 bytes) of a tile layout over a state: 0 on success, 1
// without the driver's encoder, 2 when the driver rejects the layout.
int encode_tile_map(void *state, const TilePass &t, void *map128);
// Shared memory of a coset-gather launch and its pipeline depth.
size_t coset_smem_bytes(int amp_bytes, uint32_t r, uint32_t d, uint32_t e, uint32_t *stages);

// Compiled gather (jit.cu).  Return QSIM_OK or a QSIM_* error with msg set.
int jit_compile(uint32_t M, int amp, const qsim_step *steps, size_t n, double *compile_ms,
                std::string *msg);
// Compile and load a compiled gather ahead of its launch (cached).
int jit_prepare(uint32_t M, int amp, const qsim_step *steps, size_t n, std::string *msg);
int launch_jit_gather(const void *in, void *out, int amp, uint32_t M, const qsim_step *steps,
                      size_t n, double *d_probs, void *stream, std::string *msg);
// The address bits that the row map of a step list can change: OR over every
// row i of x(i) ^ i, evaluated on the device (compiled, cached by steps).
// d_word: 8 bytes of device scratch; synchronises the stream.
int jit_delta(uint32_t M, const qsim_step *steps, size_t n, uint64_t *d_word, void *stream,
              uint64_t *delta, std::string *msg);
// Closed tile pass: compile ahead of its launch (cached), and launch.
int jit_prepare_closed(uint32_t M, int amp, const qsim_step *steps, size_t n, const TilePass &t,
                       std::string *msg);
int launch_jit_closed(void *state, int amp, uint32_t M, const qsim_step *steps, size_t n,
                      const TilePass &t, double *d_probs, int *d_err, void *stream, std::string *msg);
int num_sms();

}  // namespace qsim
