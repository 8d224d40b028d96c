// qsim_api.cu -- the C ABI (include/qsim.h): contexts, state transfer,
// circuit application and probabilities.  Host code only; kernels live in
// kernels.cu and the planner in planner.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qsim_internal.h"

using namespace qsim;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? QSIM_ENOMEM : QSIM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define QSIM_CUDA(call, what)                       \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t amp_bytes_of(int dtype) { return dtype == QSIM_C64 ? 8 : dtype == QSIM_C128 ? 16 : 0; }

constexpr size_t kProbChunk = size_t(1) << 24;  // amplitudes per host-probability chunk

}  // namespace

void qsim::set_last_error(const std::string &msg) { g_err = msg; }

struct qsim_ctx {
    uint32_t M = 0;
    int dtype = 0;
    size_t amp = 0;
    uint64_t n = 0;
    int device = 0;
    void *buf[2] = {nullptr, nullptr};
    bool own[2] = {false, false};
    int cur = 0;
    bool external = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int *d_err = nullptr;
    // plan tables: device copy and pinned host staging
    char *d_plan = nullptr;
    size_t d_plan_cap = 0;
    char *h_plan = nullptr;
    size_t h_plan_cap = 0;
    cudaEvent_t plan_ev = nullptr;
    bool plan_ev_pending = false;
    double *d_partials = nullptr;
    double *d_norms = nullptr;
    double *d_probs_chunk[2] = {nullptr, nullptr};  // double buffer for host probabilities
    double *d_probs_full = nullptr;                   // whole-state buffer for asynchronous reads
    cudaEvent_t full_copied = nullptr;                // its copy to the host is done
    cudaEvent_t full_written = nullptr;               // the context's stream wrote it
    bool full_pending = false;
    cudaStream_t copy_stream = nullptr;               // device-to-host copies of those chunks
    cudaEvent_t chunk_ready[2] = {nullptr, nullptr}, chunk_copied[2] = {nullptr, nullptr};
    PlanOptions opts;
    qsim_plan_stats stats{};
    // tracing: events around each pass of the last apply
    bool profiling = false;
    std::vector<cudaEvent_t> ev;        // 2 per pass
    std::vector<uint32_t> prof_kinds;
    std::vector<double> prof_bytes;
    // testing hook for the next tile pass (qsim_set_wait_test), then cleared
    WaitTest wait_test;
    bool wait_test_armed = false;
};

namespace {

int ctx_init_common(qsim_ctx *c)
{
    QSIM_CUDA(cudaGetDevice(&c->device), "cudaGetDevice");
    QSIM_CUDA(cudaMalloc(&c->d_err, sizeof(int)), "cudaMalloc(error flag)");
    QSIM_CUDA(cudaMemset(c->d_err, 0, sizeof(int)), "cudaMemset(error flag)");
    const int np = probabilities_partials_needed();
    QSIM_CUDA(cudaMalloc(&c->d_partials, sizeof(double) * np), "cudaMalloc(partials)");
    const size_t nchunks = (c->n + kProbChunk - 1) / kProbChunk;
    QSIM_CUDA(cudaMalloc(&c->d_norms, sizeof(double) * (nchunks + 1)), "cudaMalloc(norms)");
    QSIM_CUDA(cudaEventCreateWithFlags(&c->plan_ev, cudaEventDisableTiming), "cudaEventCreate");
    c->opts.amp_bytes = c->amp;
    return QSIM_OK;
}

void ctx_free(qsim_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 2; ++i)
        if (c->own[i] && c->buf[i]) cudaFree(c->buf[i]);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_plan) cudaFree(c->d_plan);
    if (c->h_plan) cudaFreeHost(c->h_plan);
    if (c->plan_ev) cudaEventDestroy(c->plan_ev);
    if (c->d_partials) cudaFree(c->d_partials);
    if (c->d_norms) cudaFree(c->d_norms);
    if (c->d_probs_full) cudaFree(c->d_probs_full);
    if (c->full_copied) cudaEventDestroy(c->full_copied);
    if (c->full_written) cudaEventDestroy(c->full_written);
    for (int i = 0; i < 2; ++i) {
        if (c->d_probs_chunk[i]) cudaFree(c->d_probs_chunk[i]);
        if (c->chunk_ready[i]) cudaEventDestroy(c->chunk_ready[i]);
        if (c->chunk_copied[i]) cudaEventDestroy(c->chunk_copied[i]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// Read and clear the device error flag (waits for the stream).
int check_device(qsim_ctx *c)
{
    // ordered on the context's stream only: a copy on the legacy default
    // stream would also wait for other work that runs there
    int flag = 0;
    QSIM_CUDA(cudaMemcpyAsync(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
              "read error flag");
    QSIM_CUDA(cudaStreamSynchronize(c->stream), "kernel execution");
    if (flag) {
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
        if (flag & 4)
            return fail(QSIM_ECUDA, "closed tile pass: a source row left its tile (error flag " +
                                        std::to_string(flag) + ")");
        return fail(QSIM_ETIMEOUT, "a bounded device wait gave up (error flag " +
                                       std::to_string(flag) + ")");
    }
    return QSIM_OK;
}

int ensure_scratch(qsim_ctx *c)
{
    const int other = 1 - c->cur;
    if (c->buf[other]) return QSIM_OK;
    if (c->external) return fail(QSIM_EINVAL, "no scratch buffer was given to this context");
    QSIM_CUDA(cudaMalloc(&c->buf[other], c->amp * c->n), "cudaMalloc(scratch state)");
    c->own[other] = true;
    return QSIM_OK;
}

int ensure_plan_buffers(qsim_ctx *c, size_t bytes)
{
    if (c->plan_ev_pending) {
        QSIM_CUDA(cudaEventSynchronize(c->plan_ev), "plan staging reuse");
        c->plan_ev_pending = false;
    }
    if (bytes > c->h_plan_cap) {
        if (c->h_plan) cudaFreeHost(c->h_plan);
        c->h_plan = nullptr;
        size_t cap = bytes + bytes / 2 + 4096;
        QSIM_CUDA(cudaMallocHost(&c->h_plan, cap), "cudaMallocHost(plan staging)");
        c->h_plan_cap = cap;
    }
    if (bytes > c->d_plan_cap) {
        // previous kernels on the stream may still read the old table
        QSIM_CUDA(cudaStreamSynchronize(c->stream), "plan table resize");
        if (c->d_plan) cudaFree(c->d_plan);
        c->d_plan = nullptr;
        size_t cap = bytes + bytes / 2 + 4096;
        QSIM_CUDA(cudaMalloc(&c->d_plan, cap), "cudaMalloc(plan tables)");
        c->d_plan_cap = cap;
    }
    return QSIM_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void fill_stats(const Plan &plan, uint32_t M, size_t amp, qsim_plan_stats *st)
{
    std::memset(st, 0, sizeof(*st));
    st->steps_in = plan.steps_in;
    st->steps_cancelled = plan.cancelled;
    st->passes = plan.passes.size();
    for (const Pass &p : plan.passes) {
        if (p.kind == kSweep) ++st->sweep_passes;
        if (p.kind == kTile) ++st->tile_passes;
        if (p.kind == kGather) ++st->gather_passes;
        st->algorithmic_bytes += p.alg_bytes;
    }
    st->full_pass_equiv = st->algorithmic_bytes / (2.0 * (double)amp * (double)(1ull << M));
    st->est_ms = plan_estimated_ms(plan, M, amp);
}

int plan_options(int strategy, int tile_bits, int low_bits, PlanOptions *o)
{
    if (strategy < QSIM_STRATEGY_AUTO || strategy > QSIM_STRATEGY_INPLACE)
        return fail(QSIM_EINVAL, "unknown strategy");
    if (tile_bits < 0 || tile_bits > kMaxTileBits) return fail(QSIM_EINVAL, "tile_bits out of range");
    if (low_bits < 0 || low_bits > kMaxTileBits) return fail(QSIM_EINVAL, "low_bits out of range");
    o->strategy = strategy;
    o->tile_bits = tile_bits;
    o->low_bits = low_bits;
    return QSIM_OK;
}

}  // namespace

extern "C" {

int qsim_create(uint32_t M, int dtype, qsim_ctx **out)
{
    if (!out) return fail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (M < 1 || M > QSIM_MAX_QUBITS) return fail(QSIM_EINVAL, "M out of range");
    const size_t amp = amp_bytes_of(dtype);
    if (!amp) return fail(QSIM_EINVAL, "unknown dtype");
    qsim_ctx *c = new qsim_ctx;
    c->M = M;
    c->dtype = dtype;
    c->amp = amp;
    c->n = 1ull << M;
    int rc = ctx_init_common(c);
    if (rc == QSIM_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreate");
        c->own_stream = (e == cudaSuccess);
    }
    if (rc == QSIM_OK) {
        cudaError_t e = cudaMalloc(&c->buf[0], amp * c->n);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(state)");
        else {
            c->own[0] = true;
            e = cudaMemsetAsync(c->buf[0], 0, amp * c->n, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemset(state)");
        }
    }
    if (rc != QSIM_OK) {
        ctx_free(c);
        return rc;
    }
    c->opts.scratch_available = true;  // allocated on first gather pass
    *out = c;
    return QSIM_OK;
}

int qsim_create_with_buffers(uint32_t M, int dtype, void *d_state, void *d_scratch, void *stream,
                             qsim_ctx **out)
{
    if (!out) return fail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (M < 1 || M > QSIM_MAX_QUBITS) return fail(QSIM_EINVAL, "M out of range");
    const size_t amp = amp_bytes_of(dtype);
    if (!amp) return fail(QSIM_EINVAL, "unknown dtype");
    if (!d_state) return fail(QSIM_EINVAL, "d_state is NULL");
    if ((reinterpret_cast<uintptr_t>(d_state) & 255u) ||
        (reinterpret_cast<uintptr_t>(d_scratch) & 255u))
        return fail(QSIM_EINVAL, "device buffers must be 256-byte aligned");
    if (d_scratch == d_state) return fail(QSIM_EINVAL, "scratch must differ from the state buffer");
    qsim_ctx *c = new qsim_ctx;
    c->M = M;
    c->dtype = dtype;
    c->amp = amp;
    c->n = 1ull << M;
    c->external = true;
    c->buf[0] = d_state;
    c->buf[1] = d_scratch;
    c->stream = static_cast<cudaStream_t>(stream);
    int rc = ctx_init_common(c);
    if (rc != QSIM_OK) {
        ctx_free(c);
        return rc;
    }
    c->opts.scratch_available = d_scratch != nullptr;
    *out = c;
    return QSIM_OK;
}

void qsim_destroy(qsim_ctx *ctx) { ctx_free(ctx); }

void *qsim_state_device(qsim_ctx *ctx) { return ctx ? ctx->buf[ctx->cur] : nullptr; }

int qsim_load_state(qsim_ctx *c, const void *host, size_t n_amps)
{
    if (!c || !host) return fail(QSIM_EINVAL, "NULL argument");
    if (n_amps != c->n) return fail(QSIM_EINVAL, "n_amps must equal 2^M");
    QSIM_CUDA(cudaMemcpyAsync(c->buf[c->cur], host, c->amp * c->n, cudaMemcpyHostToDevice, c->stream),
              "cudaMemcpy(load state)");
    QSIM_CUDA(cudaStreamSynchronize(c->stream), "cudaMemcpy(load state)");
    return QSIM_OK;
}

int qsim_load_state_async(qsim_ctx *c, const void *host, size_t n_amps)
{
    if (!c || !host) return fail(QSIM_EINVAL, "NULL argument");
    if (n_amps != c->n) return fail(QSIM_EINVAL, "n_amps must equal 2^M");
    QSIM_CUDA(cudaMemcpyAsync(c->buf[c->cur], host, c->amp * c->n, cudaMemcpyHostToDevice, c->stream),
              "cudaMemcpy(load state)");
    return QSIM_OK;
}

int qsim_load_product_state(qsim_ctx *c, const double *qubits)
{
    if (!c || !qubits) return fail(QSIM_EINVAL, "NULL argument");
    const size_t bytes = sizeof(double) * 4 * c->M;
    // the qubit table rides in the plan-table staging buffers
    int rc = ensure_plan_buffers(c, bytes);
    if (rc != QSIM_OK) return rc;
    std::memcpy(c->h_plan, qubits, bytes);
    QSIM_CUDA(cudaMemcpyAsync(c->d_plan, c->h_plan, bytes, cudaMemcpyHostToDevice, c->stream),
              "cudaMemcpy(qubits)");
    QSIM_CUDA(cudaEventRecord(c->plan_ev, c->stream), "cudaEventRecord");
    c->plan_ev_pending = true;
    const int e = launch_product_state(c->buf[c->cur], (int)c->amp, c->M,
                                       reinterpret_cast<const double *>(c->d_plan), c->stream);
    if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "product-state launch");
    return QSIM_OK;
}

int qsim_row_array(qsim_ctx *c, const qsim_step *steps, size_t L, uint64_t *d_rows)
{
    if (!c || !d_rows) return fail(QSIM_EINVAL, "NULL argument");
    if (reinterpret_cast<uintptr_t>(d_rows) & 7u) return fail(QSIM_EINVAL, "d_rows misaligned");
    std::vector<SlicedStep> sl;
    std::string msg;
    int rc = sliced_steps_of(c->M, steps, L, &sl, &msg);
    if (rc != QSIM_OK) return fail(rc, msg);
    const size_t bytes = std::max<size_t>(16, sl.size() * sizeof(SlicedStep));
    rc = ensure_plan_buffers(c, bytes);
    if (rc != QSIM_OK) return rc;
    if (!sl.empty()) {
        std::memcpy(c->h_plan, sl.data(), sl.size() * sizeof(SlicedStep));
        QSIM_CUDA(cudaMemcpyAsync(c->d_plan, c->h_plan, sl.size() * sizeof(SlicedStep),
                                  cudaMemcpyHostToDevice, c->stream),
                  "cudaMemcpy(steps)");
        QSIM_CUDA(cudaEventRecord(c->plan_ev, c->stream), "cudaEventRecord");
        c->plan_ev_pending = true;
    }
    const int e = launch_row_array(d_rows, c->M, reinterpret_cast<const SlicedStep *>(c->d_plan),
                                   (uint32_t)sl.size(), c->stream);
    if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "row-array launch");
    return QSIM_OK;
}

int qsim_gather_rows(const void *d_in, void *d_out, const uint64_t *d_rows, uint32_t M, int dtype,
                     double *d_probs, int loads_in_flight, void *stream)
{
    if (M < 1 || M > QSIM_MAX_QUBITS) return fail(QSIM_EINVAL, "M out of range");
    const size_t amp = amp_bytes_of(dtype);
    if (!amp) return fail(QSIM_EINVAL, "unknown dtype");
    if (!d_in || !d_out || !d_rows) return fail(QSIM_EINVAL, "NULL argument");
    if (d_in == d_out) return fail(QSIM_EINVAL, "the gather is out of place: d_out must differ from d_in");
    if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & (amp - 1) ||
        (reinterpret_cast<uintptr_t>(d_rows) & 7u) || (reinterpret_cast<uintptr_t>(d_probs) & 7u))
        return fail(QSIM_EINVAL, "misaligned device pointer");
    if (loads_in_flight == 0) loads_in_flight = 8;
    if (loads_in_flight != 4 && loads_in_flight != 8 && loads_in_flight != 16)
        return fail(QSIM_EINVAL, "loads_in_flight must be 0, 4, 8 or 16");
    const int e = launch_gather_rows(d_in, d_out, d_rows, (int)amp, M, d_probs, loads_in_flight, stream);
    if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "row gather launch");
    return QSIM_OK;
}

int qsim_read_state(qsim_ctx *c, void *host, size_t n_amps)
{
    if (!c || !host) return fail(QSIM_EINVAL, "NULL argument");
    if (n_amps != c->n) return fail(QSIM_EINVAL, "n_amps must equal 2^M");
    int rc = check_device(c);
    if (rc != QSIM_OK) return rc;
    QSIM_CUDA(cudaMemcpyAsync(host, c->buf[c->cur], c->amp * c->n, cudaMemcpyDeviceToHost, c->stream),
              "cudaMemcpy(read state)");
    QSIM_CUDA(cudaStreamSynchronize(c->stream), "cudaMemcpy(read state)");
    return QSIM_OK;
}

int qsim_set_strategy(qsim_ctx *c, int strategy, int tile_bits, int low_bits)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    return plan_options(strategy, tile_bits, low_bits, &c->opts);
}

int qsim_set_jit(qsim_ctx *c, int enable)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    c->opts.jit = enable != 0;
    return QSIM_OK;
}

int qsim_jit_precompile(uint32_t M, int dtype, const qsim_step *steps, size_t L, int canonicalize,
                        double *compile_ms)
{
    const size_t amp = amp_bytes_of(dtype);
    if (!amp) return fail(QSIM_EINVAL, "unknown dtype");
    PlanOptions o;
    o.amp_bytes = amp;
    o.scratch_available = true;
    o.strategy = QSIM_STRATEGY_GATHER;
    o.jit = true;
    o.cancel_adjacent = canonicalize != 0;
    Plan plan;
    std::string msg;
    int rc = make_plan(M, steps, L, o, &plan, &msg);
    if (rc != QSIM_OK) return fail(rc, msg);
    double total = 0;
    for (const Pass &p : plan.passes) {
        if (p.kind != kGather || !p.gather.jit) continue;
        double ms = 0;
        rc = jit_compile(M, (int)amp, plan.jit_steps.data() + p.gather.jit_off, p.gather.jit_n, &ms, &msg);
        if (rc != QSIM_OK) return fail(rc, msg);
        total += ms;
    }
    if (compile_ms) *compile_ms = total;
    return QSIM_OK;
}

int qsim_set_coset(qsim_ctx *c, int enable, int run_bits, int stage_kib)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    if (run_bits < 0 || run_bits > 7) return fail(QSIM_EINVAL, "run_bits must be in [0, 7]");
    if (stage_kib < 0 || stage_kib > 96) return fail(QSIM_EINVAL, "stage_kib must be in [0, 96]");
    c->opts.coset = enable != 0;
    c->opts.coset_run_bits = run_bits;
    c->opts.coset_stage_kib = stage_kib;
    return QSIM_OK;
}

int qsim_set_wait_test(qsim_ctx *c, uint32_t poll_limit)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    if (poll_limit == 0 || poll_limit > (1u << 20)) return fail(QSIM_EINVAL, "poll_limit must be in [1, 2^20]");
    c->wait_test.poll_limit = poll_limit;
    c->wait_test.stall_producer = true;
    c->wait_test_armed = true;
    return QSIM_OK;
}

int qsim_set_canonicalize(qsim_ctx *c, int enable)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    c->opts.cancel_adjacent = enable != 0;
    return QSIM_OK;
}

int qsim_get_plan_stats(qsim_ctx *c, qsim_plan_stats *out)
{
    if (!c || !out) return fail(QSIM_EINVAL, "NULL argument");
    *out = c->stats;
    return QSIM_OK;
}

int qsim_synchronize(qsim_ctx *c)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    if (c->copy_stream) QSIM_CUDA(cudaStreamSynchronize(c->copy_stream), "probability copies");
    return check_device(c);
}

// Record the start of a profiled launch of kernel kind 'kind' with the given
// algorithmic bytes; returns the event slot (or -1 without profiling).
static int prof_begin(qsim_ctx *c, uint32_t kind, double bytes)
{
    if (!c->profiling) return -1;
    const size_t slot = c->prof_kinds.size();
    while (c->ev.size() < 2 * (slot + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -2;
        c->ev.push_back(e);
    }
    if (cudaEventRecord(c->ev[2 * slot], c->stream) != cudaSuccess) return -2;
    c->prof_kinds.push_back(kind);
    c->prof_bytes.push_back(bytes);
    return (int)slot;
}

static int prof_end(qsim_ctx *c, int slot)
{
    if (slot == -2) return fail(QSIM_ECUDA, "profiling events");
    if (slot < 0) return QSIM_OK;
    QSIM_CUDA(cudaEventRecord(c->ev[2 * (size_t)slot + 1], c->stream), "cudaEventRecord");
    return QSIM_OK;
}

// FP64 probabilities of the current state into device memory (no norm).
static int probabilities_pass(qsim_ctx *c, double *d_probs)
{
    const int slot = prof_begin(c, 6, (double)c->n * (double)(c->amp + 8));
    const int e = launch_probabilities(c->buf[c->cur], (int)c->amp, c->n, d_probs, c->d_partials,
                                       probabilities_partials_needed(), nullptr, c->stream);
    if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "probabilities launch");
    return prof_end(c, slot);
}

// Apply a circuit; with d_probs also write the FP64 probabilities of the
// result, from the last pass when its kernel can (tile and gather passes),
// else by a probabilities pass after it.
static int apply_impl(qsim_ctx *c, const qsim_step *steps, size_t L, double *d_probs,
                      const double *qubits = nullptr)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    if (reinterpret_cast<uintptr_t>(d_probs) & 7u) return fail(QSIM_EINVAL, "d_probs misaligned");
    Plan plan;
    std::string msg;
    PlanOptions o = c->opts;
    o.amp_bytes = c->amp;
    int rc = validate_steps(c->M, steps, L, &msg);
    if (rc != QSIM_OK) return fail(rc, msg);
    // With compiled kernels, the address bits the circuit's net row map can
    // change (found once per circuit on the device, then cached) let the
    // planner weigh a closed tile pass.
    if (o.jit && (o.strategy == QSIM_STRATEGY_AUTO || o.strategy == QSIM_STRATEGY_INPLACE) &&
        c->M >= kClosedMinQubits && L >= kClosedMinSteps) {
        uint64_t delta = 0;
        std::string dmsg;
        if (jit_delta(c->M, steps, L, reinterpret_cast<uint64_t *>(c->d_partials), c->stream, &delta, &dmsg) ==
            QSIM_OK) {
            o.closed_known = true;
            o.closed_delta = delta;
        }
    }
    rc = make_plan(c->M, steps, L, o, &plan, &msg);
    if (rc != QSIM_OK) return fail(rc, msg);
    if (qubits && o.closed_known) {
        // a closed pass cannot generate the product input (App. 1), a first
        // tile pass can: weigh the plan without closed passes too, charging
        // a plan that cannot take the input its own product-state pass and
        // one that can the per-amplitude cost of generating it
        const auto takes_input = [](const Plan &p) {
            return !p.passes.empty() && p.passes[0].kind == kTile && !p.passes[0].tile.closed &&
                   tile_product_fits(p.passes[0].tile);
        };
        const auto cost = [&](const Plan &p) { return product_plan_estimated_ms(p, c->M, c->amp, takes_input(p)); };
        PlanOptions o2 = o;
        o2.closed_known = false;
        Plan alt;
        std::string amsg;
        if (make_plan(c->M, steps, L, o2, &alt, &amsg) == QSIM_OK && cost(alt) < cost(plan)) plan = std::move(alt);
    }
    fill_stats(plan, c->M, c->amp, &c->stats);
    // product input (App. 1): a first tile pass computes its sources from the
    // qubits; any other plan starts from the state written out first
    const bool fuse_input = qubits && !plan.passes.empty() && plan.passes[0].kind == kTile &&
                            !plan.passes[0].tile.closed && tile_product_fits(plan.passes[0].tile);
    if (qubits && !fuse_input) {
        rc = qsim_load_product_state(c, qubits);
        if (rc != QSIM_OK) return rc;
    }
    if (plan.passes.empty()) return d_probs ? probabilities_pass(c, d_probs) : QSIM_OK;
    std::vector<double> prod;
    if (fuse_input) prod = product_tables(c->M, qubits, plan.passes[0].tile);

    bool need_scratch = false;
    for (const Pass &p : plan.passes) need_scratch |= (p.kind == kGather);
    if (need_scratch) {
        rc = ensure_scratch(c);
        if (rc != QSIM_OK) return rc;
    }
    // compile every circuit-specialised kernel before the first launch, so a
    // compile failure leaves the state untouched
    for (const Pass &p : plan.passes) {
        std::string jmsg;
        if (p.kind == kTile && p.tile.closed)
            rc = jit_prepare_closed(c->M, (int)c->amp, plan.jit_steps.data() + p.tile.jit_off, p.tile.jit_n,
                                    p.tile, &jmsg);
        else if (p.kind == kGather && p.gather.jit)
            rc = jit_prepare(c->M, (int)c->amp, plan.jit_steps.data() + p.gather.jit_off, p.gather.jit_n, &jmsg);
        else
            continue;
        if (rc != QSIM_OK) return fail(rc, jmsg);
    }
    // one contiguous table: tile steps | sliced steps | gather tables
    const size_t off_tile = 0;
    const size_t sz_tile = plan.tile_steps.size() * sizeof(TileStep);
    const size_t off_sliced = align_up(off_tile + sz_tile, 256);
    const size_t sz_sliced = plan.sliced_steps.size() * sizeof(SlicedStep);
    const size_t off_tab = align_up(off_sliced + sz_sliced, 256);
    const size_t sz_tab = plan.gather_tables.size() * sizeof(uint64_t);
    const size_t off_prod = align_up(off_tab + sz_tab, 256);
    const size_t sz_prod = prod.size() * sizeof(double);
    const size_t total = off_prod + sz_prod;
    if (total > 0) {
        rc = ensure_plan_buffers(c, total);
        if (rc != QSIM_OK) return rc;
        if (sz_tile) std::memcpy(c->h_plan + off_tile, plan.tile_steps.data(), sz_tile);
        if (sz_sliced) std::memcpy(c->h_plan + off_sliced, plan.sliced_steps.data(), sz_sliced);
        if (sz_tab) std::memcpy(c->h_plan + off_tab, plan.gather_tables.data(), sz_tab);
        if (sz_prod) std::memcpy(c->h_plan + off_prod, prod.data(), sz_prod);
        QSIM_CUDA(cudaMemcpyAsync(c->d_plan, c->h_plan, total, cudaMemcpyHostToDevice, c->stream),
                  "cudaMemcpy(plan tables)");
        QSIM_CUDA(cudaEventRecord(c->plan_ev, c->stream), "cudaEventRecord");
        c->plan_ev_pending = true;
    }
    const TileStep *d_tile = reinterpret_cast<const TileStep *>(c->d_plan + off_tile);
    const SlicedStep *d_sliced = reinterpret_cast<const SlicedStep *>(c->d_plan + off_sliced);
    const uint64_t *d_tab = reinterpret_cast<const uint64_t *>(c->d_plan + off_tab);
    const double n = (double)c->n;
    bool fused = false;
    for (size_t pi = 0; pi < plan.passes.size(); ++pi) {
        const Pass &p = plan.passes[pi];
        // the last pass writes the probabilities when its kernel can (every
        // kind but a sweep; on the M = 32 adder the closed pass writing them
        // took 18.5 ms against 11.8 + 11.7 ms for a separate pass)
        double *pp = (d_probs && pi + 1 == plan.passes.size() && p.kind != kSweep) ? d_probs : nullptr;
        double bytes = (pi == 0 && fuse_input) ? n * c->amp : p.alg_bytes;  // product input: writes only
        if (pp) {
            // every tile is read; touched tiles are written; plus the probabilities
            bytes = (pi == 0 && fuse_input ? n * c->amp
                     : p.kind == kTile && !p.tile.closed ? n * c->amp + 0.5 * p.alg_bytes
                                                         : p.alg_bytes) + 8.0 * n;
            fused = true;
        }
        const int slot = prof_begin(c, pass_variant(p), bytes);
        int e = cudaSuccess;
        if (p.kind == kSweep) {
            e = launch_sweep(c->buf[c->cur], (int)c->amp, p.sweep, c->d_err, c->stream);
        } else if (p.kind == kTile && p.tile.closed) {
            std::string jmsg;
            const int jrc = launch_jit_closed(c->buf[c->cur], (int)c->amp, c->M,
                                              plan.jit_steps.data() + p.tile.jit_off, p.tile.jit_n, p.tile,
                                              pp, c->d_err, c->stream, &jmsg);
            if (jrc != QSIM_OK) return fail(jrc, jmsg);
        } else if (p.kind == kTile) {
            e = launch_tile(c->buf[c->cur], (int)c->amp, p.tile, d_tile, c->d_err, pp, c->stream,
                            c->wait_test_armed ? &c->wait_test : nullptr,
                            (pi == 0 && fuse_input) ? reinterpret_cast<const double *>(c->d_plan + off_prod)
                                                    : nullptr);
            c->wait_test_armed = false;
        } else if (p.gather.jit) {
            std::string jmsg;
            const int jrc = launch_jit_gather(c->buf[c->cur], c->buf[1 - c->cur], (int)c->amp, c->M,
                                              plan.jit_steps.data() + p.gather.jit_off,
                                              p.gather.jit_n, pp, c->stream, &jmsg);
            if (jrc != QSIM_OK) return fail(jrc, jmsg);
            c->cur = 1 - c->cur;
        } else {
            e = launch_gather(c->buf[c->cur], c->buf[1 - c->cur], (int)c->amp, c->M, p.gather,
                              d_tab, d_sliced, c->d_err, pp, c->stream);
            if (e == cudaSuccess) c->cur = 1 - c->cur;
        }
        if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "kernel launch");
        const int prc = prof_end(c, slot);
        if (prc != QSIM_OK) return prc;
    }
    if (d_probs && !fused) return probabilities_pass(c, d_probs);
    return QSIM_OK;
}

int qsim_apply_circuit(qsim_ctx *c, const qsim_step *steps, size_t L)
{
    return apply_impl(c, steps, L, nullptr);
}

int qsim_apply_circuit_product(qsim_ctx *c, const double *qubits, const qsim_step *steps, size_t L,
                               double *d_probs)
{
    if (!c || !qubits) return fail(QSIM_EINVAL, "NULL argument");
    return apply_impl(c, steps, L, d_probs, qubits);
}

int qsim_apply_circuit_probabilities(qsim_ctx *c, const qsim_step *steps, size_t L, double *d_probs)
{
    if (!d_probs) return fail(QSIM_EINVAL, "d_probs is NULL");
    return apply_impl(c, steps, L, d_probs);
}

int qsim_autotune(qsim_ctx *c, const qsim_step *steps, size_t L, int reps, qsim_tune_result *out,
                  size_t cap, size_t *n_out)
{
    if (!c || (L && !steps)) return fail(QSIM_EINVAL, "NULL argument");
    if (reps < 1 || reps > 100) return fail(QSIM_EINVAL, "reps must be in 1..100");
    if (cap && !out) return fail(QSIM_EINVAL, "out is NULL");
    std::string msg;
    int rc = validate_steps(c->M, steps, L, &msg);
    if (rc != QSIM_OK) return fail(rc, msg);
    rc = check_device(c);
    if (rc != QSIM_OK) return rc;
    // candidate plans: the cost model's choice, the gathers (when a second
    // buffer is allowed), in-place tile passes over a range of tile widths k
    // and run lengths l, and per-step sweeps for short circuits
    std::vector<qsim_tune_result> cand;
    auto add = [&](int strategy, int k, int l, int jit) {
        qsim_tune_result r{};
        r.strategy = strategy;
        r.tile_bits = k;
        r.low_bits = l;
        r.jit = jit;
        r.ms = -1.0;
        cand.push_back(r);
    };
    add(QSIM_STRATEGY_AUTO, 0, 0, c->opts.jit ? 1 : 0);
    add(QSIM_STRATEGY_INPLACE, 0, 0, 0);
    if (c->opts.scratch_available) {
        add(QSIM_STRATEGY_GATHER, 0, 0, 0);
        if (c->M >= 10) add(QSIM_STRATEGY_GATHER, 0, 0, 1);
    }
    const int kdef = c->amp == 16 ? 13 : 14;
    for (int k = kdef; k >= kdef - 2; --k) {
        if (k > (int)c->M || k < 4) continue;
        for (int l = 3; l <= 6 && l < k; ++l) add(QSIM_STRATEGY_TILE, k, l, 0);
    }
    if (L <= 64) add(QSIM_STRATEGY_SWEEP, 0, 0, 0);

    const PlanOptions saved = c->opts;
    const bool saved_prof = c->profiling;
    c->profiling = false;
    std::vector<qsim_step> rev(steps, steps + L);
    std::reverse(rev.begin(), rev.end());  // each step is its own inverse (Sec. 2a)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QSIM_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    QSIM_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    int err = QSIM_OK;
    for (auto &cd : cand) {
        c->opts = saved;
        c->opts.strategy = cd.strategy;
        c->opts.tile_bits = cd.tile_bits;
        c->opts.low_bits = cd.low_bits;
        c->opts.jit = cd.jit != 0;
        // forward then backward leaves the state as it was, bit for bit; the
        // first pair compiles and warms up, then the forward passes are timed
        if (apply_impl(c, steps, L, nullptr) != QSIM_OK || apply_impl(c, rev.data(), L, nullptr) != QSIM_OK) {
            err = check_device(c);
            if (err != QSIM_OK) break;
            continue;  // the planner rejects this candidate (e.g. a tile wider than allowed)
        }
        cd.passes = c->stats.passes;
        double best = 1e300;
        for (int r = 0; r < reps && err == QSIM_OK; ++r) {
            cudaEventRecord(e0, c->stream);
            if (apply_impl(c, steps, L, nullptr) != QSIM_OK) err = QSIM_ECUDA;
            cudaEventRecord(e1, c->stream);
            if (err == QSIM_OK && apply_impl(c, rev.data(), L, nullptr) != QSIM_OK) err = QSIM_ECUDA;
            if (err == QSIM_OK) err = check_device(c);
            float ms = 0.f;
            if (err == QSIM_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, (double)ms);
        }
        if (err != QSIM_OK) break;
        cd.ms = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->profiling = saved_prof;
    c->opts = saved;
    if (err != QSIM_OK) return err;
    std::stable_sort(cand.begin(), cand.end(), [](const qsim_tune_result &a, const qsim_tune_result &b) {
        if ((a.ms < 0) != (b.ms < 0)) return b.ms < 0;
        return a.ms < b.ms;
    });
    if (cand.empty() || cand[0].ms < 0) return fail(QSIM_EINVAL, "no candidate plan ran");
    // the context keeps the fastest plan
    c->opts.strategy = cand[0].strategy;
    c->opts.tile_bits = cand[0].tile_bits;
    c->opts.low_bits = cand[0].low_bits;
    c->opts.jit = cand[0].jit != 0;
    if (n_out) *n_out = cand.size();
    for (size_t i = 0; i < cand.size() && i < cap; ++i) out[i] = cand[i];
    return QSIM_OK;
}

int qsim_set_profiling(qsim_ctx *c, int enable)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    c->profiling = enable != 0;
    c->prof_kinds.clear();
    c->prof_bytes.clear();
    return QSIM_OK;
}

int qsim_get_pass_times(qsim_ctx *c, double *ms, uint32_t *kinds, double *alg_bytes, size_t cap,
                        size_t *n_out)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    const size_t n = c->prof_kinds.size();
    if (n_out) *n_out = n;
    int rc = check_device(c);
    if (rc != QSIM_OK) return rc;
    for (size_t i = 0; i < n && i < cap; ++i) {
        if (ms) {
            float t = 0.f;
            QSIM_CUDA(cudaEventElapsedTime(&t, c->ev[2 * i], c->ev[2 * i + 1]), "cudaEventElapsedTime");
            ms[i] = t;
        }
        if (kinds) kinds[i] = c->prof_kinds[i];
        if (alg_bytes) alg_bytes[i] = c->prof_bytes[i];
    }
    if (cap >= n) {  // everything was read: start a new record
        c->prof_kinds.clear();
        c->prof_bytes.clear();
    }
    return QSIM_OK;
}

int qsim_probabilities_device(qsim_ctx *c, double *d_probs, double *norm_out)
{
    if (!c) return fail(QSIM_EINVAL, "ctx is NULL");
    if (reinterpret_cast<uintptr_t>(d_probs) & 7u) return fail(QSIM_EINVAL, "d_probs misaligned");
    const int slot = prof_begin(c, 6, (double)c->n * (double)(c->amp + (d_probs ? 8 : 0)));
    int e = launch_probabilities(c->buf[c->cur], (int)c->amp, c->n, d_probs, c->d_partials,
                                 probabilities_partials_needed(), norm_out ? c->d_norms : nullptr,
                                 c->stream);
    if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "probabilities launch");
    int prc = prof_end(c, slot);
    if (prc != QSIM_OK) return prc;
    if (norm_out) {
        int rc = check_device(c);
        if (rc != QSIM_OK) return rc;
        QSIM_CUDA(cudaMemcpyAsync(norm_out, c->d_norms, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                  "read norm");
        QSIM_CUDA(cudaStreamSynchronize(c->stream), "read norm");
    }
    return QSIM_OK;
}

namespace {

// Queue the probabilities of the current state and their copy into host
// memory (chunks double-buffered between the context's stream and its copy
// stream); with norms, also the per-chunk norms.  Returns without waiting.
int queue_host_probabilities(qsim_ctx *c, double *host_probs, bool norms, size_t *nchunks_out);

// The whole-state probability buffer for asynchronous reads, allocated on
// first use (nullptr and no error if it cannot be: callers fall back to the
// chunked path).  The context's stream waits until the previous copy out of
// it is done, so a new write never races the copy.
double *full_probs_buffer(qsim_ctx *c)
{
    if (!c->d_probs_full) {
        if (cudaMalloc(&c->d_probs_full, sizeof(double) * c->n) != cudaSuccess) {
            cudaGetLastError();
            c->d_probs_full = nullptr;
            return nullptr;
        }
        if (cudaEventCreateWithFlags(&c->full_copied, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->full_written, cudaEventDisableTiming) != cudaSuccess)
            return nullptr;
    }
    if (c->full_pending) {
        if (cudaStreamWaitEvent(c->stream, c->full_copied, 0) != cudaSuccess) return nullptr;
        c->full_pending = false;
    }
    return c->d_probs_full;
}

// After the context's stream has written the whole-state buffer: one copy of
// it to the host on the copy stream.
int copy_full_probabilities(qsim_ctx *c, double *host_probs)
{
    if (!c->copy_stream) {
        QSIM_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    }
    QSIM_CUDA(cudaEventRecord(c->full_written, c->stream), "cudaEventRecord");
    QSIM_CUDA(cudaStreamWaitEvent(c->copy_stream, c->full_written, 0), "cudaStreamWaitEvent");
    QSIM_CUDA(cudaMemcpyAsync(host_probs, c->d_probs_full, sizeof(double) * c->n, cudaMemcpyDeviceToHost,
                              c->copy_stream),
              "cudaMemcpy(probabilities)");
    QSIM_CUDA(cudaEventRecord(c->full_copied, c->copy_stream), "cudaEventRecord");
    c->full_pending = true;
    return QSIM_OK;
}

}  // namespace

int qsim_probabilities_async(qsim_ctx *c, double *host_probs, size_t n)
{
    if (!c || !host_probs) return fail(QSIM_EINVAL, "NULL argument");
    if (n != c->n) return fail(QSIM_EINVAL, "n must equal 2^M");
    if (double *d = full_probs_buffer(c)) {  // one kernel, one copy out
        const int e = launch_probabilities(c->buf[c->cur], (int)c->amp, c->n, d, c->d_partials,
                                           probabilities_partials_needed(), nullptr, c->stream);
        if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "probabilities launch");
        return copy_full_probabilities(c, host_probs);
    }
    size_t nchunks = 0;
    return queue_host_probabilities(c, host_probs, false, &nchunks);
}

int qsim_apply_circuit_probabilities_async(qsim_ctx *c, const qsim_step *steps, size_t L,
                                           double *host_probs, size_t n)
{
    if (!c || !host_probs) return fail(QSIM_EINVAL, "NULL argument");
    if (n != c->n) return fail(QSIM_EINVAL, "n must equal 2^M");
    double *d = full_probs_buffer(c);
    if (!d) {  // no room for the whole buffer: apply, then chunked probabilities
        int rc = qsim_apply_circuit(c, steps, L);
        if (rc != QSIM_OK) return rc;
        size_t nchunks = 0;
        return queue_host_probabilities(c, host_probs, false, &nchunks);
    }
    int rc = apply_impl(c, steps, L, d);
    if (rc != QSIM_OK) return rc;
    return copy_full_probabilities(c, host_probs);
}

int qsim_probabilities(qsim_ctx *c, double *host_probs, size_t n, double *norm_out)
{
    if (!c || !host_probs) return fail(QSIM_EINVAL, "NULL argument");
    if (n != c->n) return fail(QSIM_EINVAL, "n must equal 2^M");
    int rc = check_device(c);
    if (rc != QSIM_OK) return rc;
    size_t nchunks = 0;
    rc = queue_host_probabilities(c, host_probs, norm_out != nullptr, &nchunks);
    if (rc != QSIM_OK) return rc;
    QSIM_CUDA(cudaStreamSynchronize(c->copy_stream), "cudaMemcpy(probabilities)");
    rc = check_device(c);
    if (rc != QSIM_OK) return rc;
    if (norm_out) {
        std::vector<double> norms(nchunks);
        QSIM_CUDA(cudaMemcpyAsync(norms.data(), c->d_norms, sizeof(double) * nchunks, cudaMemcpyDeviceToHost,
                                  c->stream),
                  "read norms");
        QSIM_CUDA(cudaStreamSynchronize(c->stream), "read norms");
        // pairwise over chunk sums
        while (norms.size() > 1) {
            std::vector<double> nx((norms.size() + 1) / 2);
            for (size_t i = 0; i < nx.size(); ++i)
                nx[i] = norms[2 * i] + (2 * i + 1 < norms.size() ? norms[2 * i + 1] : 0.0);
            norms.swap(nx);
        }
        *norm_out = norms[0];
    }
    return QSIM_OK;
}

namespace {

int queue_host_probabilities(qsim_ctx *c, double *host_probs, bool want_norms, size_t *nchunks_out)
{
    // Chunks of probabilities alternate between two device buffers: the kernel
    // for chunk k+1 runs on the context's stream while chunk k is copied out
    // on a second stream.
    const size_t chunk = c->n < kProbChunk ? c->n : kProbChunk;
    if (!c->copy_stream) {
        QSIM_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        for (int i = 0; i < 2; ++i) {
            QSIM_CUDA(cudaMalloc(&c->d_probs_chunk[i], sizeof(double) * chunk), "cudaMalloc(probabilities)");
            QSIM_CUDA(cudaEventCreateWithFlags(&c->chunk_ready[i], cudaEventDisableTiming), "cudaEventCreate");
            QSIM_CUDA(cudaEventCreateWithFlags(&c->chunk_copied[i], cudaEventDisableTiming), "cudaEventCreate");
        }
    }
    const size_t nchunks = (c->n + chunk - 1) / chunk;
    *nchunks_out = nchunks;
    const char *state = static_cast<const char *>(c->buf[c->cur]);
    for (size_t k = 0; k < nchunks; ++k) {
        const int b = (int)(k & 1);
        // the buffer's previous chunk must be out before it is overwritten
        // (also across calls: the events persist on the context)
        QSIM_CUDA(cudaStreamWaitEvent(c->stream, c->chunk_copied[b], 0), "cudaStreamWaitEvent");
        int e = launch_probabilities(state + k * chunk * c->amp, (int)c->amp, chunk, c->d_probs_chunk[b],
                                     c->d_partials, probabilities_partials_needed(),
                                     want_norms ? c->d_norms + k : nullptr, c->stream);
        if (e != cudaSuccess) return cuda_fail((cudaError_t)e, "probabilities launch");
        QSIM_CUDA(cudaEventRecord(c->chunk_ready[b], c->stream), "cudaEventRecord");
        QSIM_CUDA(cudaStreamWaitEvent(c->copy_stream, c->chunk_ready[b], 0), "cudaStreamWaitEvent");
        QSIM_CUDA(cudaMemcpyAsync(host_probs + k * chunk, c->d_probs_chunk[b], sizeof(double) * chunk,
                                  cudaMemcpyDeviceToHost, c->copy_stream),
                  "cudaMemcpy(probabilities)");
        QSIM_CUDA(cudaEventRecord(c->chunk_copied[b], c->copy_stream), "cudaEventRecord");
    }
    return QSIM_OK;
}

}  // namespace

int qsim_plan_circuit(uint32_t M, int dtype, const qsim_step *steps, size_t L, int strategy,
                      int tile_bits, int low_bits, int scratch_available, qsim_plan_stats *stats,
                      uint64_t *order, uint64_t *pass_ends, uint32_t *pass_kinds, size_t cap)
{
    const size_t amp = amp_bytes_of(dtype);
    if (!amp) return fail(QSIM_EINVAL, "unknown dtype");
    PlanOptions o;
    int rc = plan_options(strategy, tile_bits, low_bits, &o);
    if (rc != QSIM_OK) return rc;
    o.amp_bytes = amp;
    o.scratch_available = scratch_available != 0;
    Plan plan;
    std::string msg;
    rc = make_plan(M, steps, L, o, &plan, &msg);
    if (rc != QSIM_OK) return fail(rc, msg);
    if (stats) fill_stats(plan, M, amp, stats);
    if ((order && plan.order.size() > cap) || ((pass_ends || pass_kinds) && plan.passes.size() > cap))
        return fail(QSIM_EINVAL, "output capacity too small");
    if (order) std::memcpy(order, plan.order.data(), plan.order.size() * sizeof(uint64_t));
    if (pass_ends) std::memcpy(pass_ends, plan.pass_ends.data(), plan.pass_ends.size() * sizeof(uint64_t));
    if (pass_kinds)
        for (size_t i = 0; i < plan.passes.size(); ++i) pass_kinds[i] = (uint32_t)plan.passes[i].kind;
    return QSIM_OK;
}

int qsim_plan_circuit_ex(uint32_t M, int dtype, const qsim_step *steps, size_t L,
                         const qsim_plan_options *opts, qsim_plan_stats *stats, uint64_t *order,
                         uint64_t *pass_ends, uint32_t *pass_variants, double *pass_est_ms, size_t cap)
{
    const size_t amp = amp_bytes_of(dtype);
    if (!amp) return fail(QSIM_EINVAL, "unknown dtype");
    qsim_plan_options d{};
    d.strategy = QSIM_STRATEGY_AUTO;
    d.scratch_available = 1;
    d.coset = 1;
    d.canonicalize = 1;
    const qsim_plan_options &q = opts ? *opts : d;
    PlanOptions o;
    int rc = plan_options(q.strategy, q.tile_bits, q.low_bits, &o);
    if (rc != QSIM_OK) return rc;
    if (q.coset_run_bits < 0 || q.coset_run_bits > 7) return fail(QSIM_EINVAL, "coset_run_bits must be in [0, 7]");
    o.amp_bytes = amp;
    o.scratch_available = q.scratch_available != 0;
    o.jit = q.jit != 0;
    o.coset = q.coset != 0;
    o.coset_run_bits = q.coset_run_bits;
    o.cancel_adjacent = q.canonicalize != 0;
    o.closed_known = q.closed_known != 0;
    o.closed_delta = q.closed_delta;
    Plan plan;
    std::string msg;
    rc = make_plan(M, steps, L, o, &plan, &msg);
    if (rc != QSIM_OK) return fail(rc, msg);
    if (stats) fill_stats(plan, M, amp, stats);
    if ((order && plan.order.size() > cap) ||
        ((pass_ends || pass_variants || pass_est_ms) && plan.passes.size() > cap))
        return fail(QSIM_EINVAL, "output capacity too small");
    if (order) std::memcpy(order, plan.order.data(), plan.order.size() * sizeof(uint64_t));
    if (pass_ends) std::memcpy(pass_ends, plan.pass_ends.data(), plan.pass_ends.size() * sizeof(uint64_t));
    for (size_t i = 0; i < plan.passes.size(); ++i) {
        if (pass_variants) pass_variants[i] = pass_variant(plan.passes[i]);
        if (pass_est_ms) pass_est_ms[i] = pass_estimated_ms(plan.passes[i], M, amp);
    }
    return QSIM_OK;
}

const char *qsim_last_error(void) { return g_err.c_str(); }

const char *qsim_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }

}  // extern "C"
