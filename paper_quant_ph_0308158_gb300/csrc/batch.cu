// batch.cu -- many independent wiring diagrams in one persistent launch per
// pass level, replayed from a captured CUDA graph.
//
// Every circuit of a batch owns a 2^M[i]-amplitude state inside one device
// arena (plus a scratch arena of the same size for out-of-place gathers).
// All circuits are planned once, at creation, with out-of-place gather
// passes (GF(2) tables for NOT/CNOT runs -- read in coset-tile order for
// states of at least coset_min_qubits, so that every DRAM burst is used in
// full -- bit-sliced evaluation otherwise; steps with more than eight
// controls as in-place sweeps).  Level p holds the
// p-th pass of every circuit that has one; a level is one launch of
// batch_kernel whose CTAs pull work items (16384 outputs of one pass) from a
// counter.  The levels of a run are captured once into a CUDA graph and
// replayed by qsim_batch_run.  qsim_batch_run_plain launches the very same
// passes one kernel per circuit pass, for comparison.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "qsim_internal.h"

using namespace qsim;

namespace {

size_t amp_of(int dtype) { return dtype == QSIM_C64 ? 8 : dtype == QSIM_C128 ? 16 : 0; }

int bfail(int code, const std::string &msg)
{
    set_last_error(msg);
    return code;
}

#define QB_CUDA(call, what)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return bfail(e_ == cudaErrorMemoryAllocation ? QSIM_ENOMEM : QSIM_ECUDA,         \
                         std::string(what) + ": " + cudaGetErrorString(e_));                \
    } while (0)

}  // namespace

struct qsim_batch {
    int dtype = 0;
    size_t amp = 0;
    size_t n = 0;
    bool wide = false;
    std::vector<uint32_t> M;
    std::vector<uint64_t> off;    // amplitude offset of circuit i in each arena
    std::vector<uint32_t> gpass;  // gather passes of circuit i (state moves arena each)
    std::vector<Plan> plans;
    char *arena[2] = {nullptr, nullptr};
    size_t arena_bytes = 0;
    char *d_tab = nullptr;        // affine tables + bit-sliced steps of every plan
    std::vector<size_t> tab_off, sl_off;  // per circuit, bytes into d_tab
    // per run parity: per level, device pass and item arrays
    struct Level {
        BatchPass *d_passes = nullptr;
        BatchItem *d_items = nullptr;
        uint32_t n_items = 0;
        size_t smem = 0;
    };
    std::vector<Level> levels[2];
    uint32_t *d_counters = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    uint64_t runs = 0;
    uint32_t coset_min_qubits = 18;  // affine passes of larger states in coset-tile order
    int *d_err = nullptr;            // error flag of the plain per-circuit launches
    uint64_t coset_passes = 0, affine_passes = 0, sliced_passes = 0, sweep_passes = 0;
    double alg_bytes = 0;
    uint64_t steps_total = 0;
    uint64_t amp_steps = 0;
};

namespace {

void batch_free(qsim_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int r = 0; r < 2; ++r) {
        if (b->graph[r]) cudaGraphExecDestroy(b->graph[r]);
        for (auto &lv : b->levels[r]) {
            if (lv.d_passes) cudaFree(lv.d_passes);
            if (lv.d_items) cudaFree(lv.d_items);
        }
    }
    for (int a = 0; a < 2; ++a)
        if (b->arena[a]) cudaFree(b->arena[a]);
    if (b->d_tab) cudaFree(b->d_tab);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->d_err) cudaFree(b->d_err);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Arena holding circuit i's state at the start of a run of parity r.
int start_arena(const qsim_batch *b, size_t i, uint64_t runs)
{
    return (int)((runs * b->gpass[i]) & 1u);
}

// Build the device pass/item lists of every level for runs of parity r.
int build_levels(qsim_batch *b, int r)
{
    size_t nlev = 0;
    for (const Plan &p : b->plans) nlev = std::max(nlev, p.passes.size());
    b->levels[r].assign(nlev, {});
    std::vector<int> cur(b->n);
    for (size_t i = 0; i < b->n; ++i) cur[i] = start_arena(b, i, (uint64_t)r);
    for (size_t lv = 0; lv < nlev; ++lv) {
        std::vector<BatchPass> passes;
        std::vector<BatchItem> items;
        uint32_t max_sliced_M = 0;
        // larger work first, so the tail of the level is short
        std::vector<size_t> order;
        for (size_t i = 0; i < b->n; ++i)
            if (lv < b->plans[i].passes.size()) order.push_back(i);
        std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
            const Pass &px = b->plans[x].passes[lv], &py = b->plans[y].passes[lv];
            const double cx = (double)(1ull << b->M[x]) * (px.kind == kGather && !px.gather.affine ? px.nsteps : 1);
            const double cy = (double)(1ull << b->M[y]) * (py.kind == kGather && !py.gather.affine ? py.nsteps : 1);
            return cx > cy;
        });
        for (size_t i : order) {
            const Pass &p = b->plans[i].passes[lv];
            BatchPass bp{};
            char *a_in = b->arena[cur[i]] + b->off[i] * b->amp;
            char *a_out = b->arena[1 - cur[i]] + b->off[i] * b->amp;
            bp.M = b->M[i];
            const uint64_t n = 1ull << b->M[i];
            uint64_t units = n;
            if (p.kind == kSweep) {
                bp.kind = 1;
                bp.out = a_in;  // in place
                bp.sweep = p.sweep;
                units = p.sweep.n_pairs;
            } else if (p.gather.affine && p.gather.coset && b->M[i] >= b->coset_min_qubits) {
                bp.kind = 7;
                bp.in = a_in;
                bp.out = a_out;
                bp.bvec = p.gather.bvec;
                bp.cr = p.gather.cr;
                bp.cd = p.gather.cd;
                bp.ctb = p.gather.ctb;
                bp.tables = reinterpret_cast<const uint64_t *>(b->d_tab + b->tab_off[i]) + p.gather.coset_off;
                cur[i] = 1 - cur[i];
            } else if (p.gather.affine) {
                bp.kind = 3;
                bp.in = a_in;
                bp.out = a_out;
                bp.nbytes = p.gather.nbytes;
                bp.bvec = p.gather.bvec;
                bp.tables = reinterpret_cast<const uint64_t *>(b->d_tab + b->tab_off[i]) + p.gather.table_off;
                cur[i] = 1 - cur[i];
            } else {
                bp.kind = 4;
                bp.in = a_in;
                bp.out = a_out;
                bp.nsteps = p.gather.nsteps;
                bp.steps = reinterpret_cast<const SlicedStep *>(b->d_tab + b->sl_off[i]) + p.gather.step_off;
                max_sliced_M = std::max(max_sliced_M, b->M[i]);
                cur[i] = 1 - cur[i];
            }
            const uint32_t pid = (uint32_t)passes.size();
            passes.push_back(bp);
            for (uint64_t s0 = 0; s0 < units; s0 += kBatchItemOutputs) {
                BatchItem it{};
                it.pass = pid;
                it.start = s0;
                it.count = std::min<uint64_t>(kBatchItemOutputs, units - s0);
                items.push_back(it);
            }
        }
        qsim_batch::Level &L = b->levels[r][lv];
        L.n_items = (uint32_t)items.size();
        L.smem = batch_smem_bytes(max_sliced_M);
        QB_CUDA(cudaMalloc(&L.d_passes, sizeof(BatchPass) * std::max<size_t>(1, passes.size())), "cudaMalloc(batch passes)");
        QB_CUDA(cudaMalloc(&L.d_items, sizeof(BatchItem) * std::max<size_t>(1, items.size())), "cudaMalloc(batch items)");
        QB_CUDA(cudaMemcpy(L.d_passes, passes.data(), sizeof(BatchPass) * passes.size(), cudaMemcpyHostToDevice), "upload batch passes");
        QB_CUDA(cudaMemcpy(L.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice), "upload batch items");
    }
    return QSIM_OK;
}

int capture(qsim_batch *b, int r)
{
    const size_t nlev = b->levels[r].size();
    QB_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(uint32_t) * std::max<size_t>(1, nlev), b->stream);
    for (size_t lv = 0; lv < nlev && e == cudaSuccess; ++lv) {
        const auto &L = b->levels[r][lv];
        e = (cudaError_t)launch_batch_level((int)b->amp, b->wide, L.d_passes, L.d_items, L.n_items,
                                            b->d_counters + lv, L.smem, b->stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(QSIM_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    }
    QB_CUDA(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph[r], g, 0);
    cudaGraphDestroy(g);
    QB_CUDA(e, "cudaGraphInstantiate");
    return QSIM_OK;
}

}  // namespace

extern "C" {

int qsim_batch_create(size_t n, const uint32_t *M, int dtype, const qsim_step *const *steps,
                      const size_t *L, qsim_batch **out)
{
    return qsim_batch_create_ex(n, M, dtype, steps, L, nullptr, out);
}

int qsim_batch_create_ex(size_t n, const uint32_t *M, int dtype, const qsim_step *const *steps,
                         const size_t *L, const qsim_batch_options *opts, qsim_batch **out)
{
    if (!out) return bfail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    const size_t amp = amp_of(dtype);
    if (!amp) return bfail(QSIM_EINVAL, "unknown dtype");
    if (n == 0 || !M || !L || !steps) return bfail(QSIM_EINVAL, "empty batch or NULL arrays");
    qsim_batch *b = new qsim_batch;
    b->dtype = dtype;
    b->amp = amp;
    b->n = n;
    b->M.assign(M, M + n);
    b->off.resize(n);
    b->gpass.resize(n);
    b->plans.resize(n);
    b->tab_off.resize(n);
    b->sl_off.resize(n);
    if (opts) b->coset_min_qubits = opts->coset_min_qubits;
    uint64_t total = 0;
    size_t tab_bytes = 0;
    PlanOptions o;
    o.amp_bytes = amp;
    o.scratch_available = true;
    o.strategy = QSIM_STRATEGY_GATHER;
    o.cancel_adjacent = false;
    for (size_t i = 0; i < n; ++i) {
        std::string msg;
        int rc = make_plan(M[i], steps[i], L[i], o, &b->plans[i], &msg);
        if (rc != QSIM_OK) {
            batch_free(b);
            return bfail(rc, "circuit " + std::to_string(i) + ": " + msg);
        }
        if (M[i] > 32) b->wide = true;
        b->off[i] = total;
        total += 1ull << M[i];
        uint32_t g = 0;
        for (const Pass &p : b->plans[i].passes) {
            if (p.kind == kGather) ++g;
            b->alg_bytes += p.alg_bytes;
            if (p.kind == kSweep) ++b->sweep_passes;
            else if (!p.gather.affine) ++b->sliced_passes;
            else if (p.gather.coset && M[i] >= b->coset_min_qubits) ++b->coset_passes;
            else ++b->affine_passes;
        }
        b->gpass[i] = g;
        b->steps_total += L[i];
        b->amp_steps += (1ull << M[i]) * (uint64_t)L[i];
        b->tab_off[i] = tab_bytes;
        tab_bytes += ((b->plans[i].gather_tables.size() * sizeof(uint64_t) + 255) / 256) * 256;
        b->sl_off[i] = tab_bytes;
        tab_bytes += ((b->plans[i].sliced_steps.size() * sizeof(SlicedStep) + 255) / 256) * 256;
    }
    b->arena_bytes = total * amp;
    int rc = QSIM_OK;
    auto fail_free = [&](int code) {
        batch_free(b);
        return code;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_free(bfail(QSIM_ECUDA, "cudaStreamCreate"));
    for (int a = 0; a < 2; ++a) {
        e = cudaMalloc(&b->arena[a], b->arena_bytes);
        if (e != cudaSuccess)
            return fail_free(bfail(QSIM_ENOMEM, "cudaMalloc(batch arena of " +
                                                    std::to_string(b->arena_bytes) + " bytes)"));
    }
    e = cudaMemset(b->arena[0], 0, b->arena_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tab, std::max<size_t>(256, tab_bytes));
    if (e != cudaSuccess) return fail_free(bfail(QSIM_ENOMEM, "batch tables"));
    std::vector<char> h(tab_bytes);
    for (size_t i = 0; i < n; ++i) {
        const Plan &p = b->plans[i];
        if (!p.gather_tables.empty())
            std::memcpy(h.data() + b->tab_off[i], p.gather_tables.data(), p.gather_tables.size() * sizeof(uint64_t));
        if (!p.sliced_steps.empty())
            std::memcpy(h.data() + b->sl_off[i], p.sliced_steps.data(), p.sliced_steps.size() * sizeof(SlicedStep));
    }
    if (tab_bytes) e = cudaMemcpy(b->d_tab, h.data(), tab_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_free(bfail(QSIM_ECUDA, "upload batch tables"));
    size_t nlev = 0;
    for (const Plan &p : b->plans) nlev = std::max(nlev, p.passes.size());
    e = cudaMalloc(&b->d_counters, sizeof(uint32_t) * std::max<size_t>(1, nlev));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return fail_free(bfail(QSIM_ENOMEM, "batch counters"));
    for (int r = 0; r < 2 && rc == QSIM_OK; ++r) rc = build_levels(b, r);
    for (int r = 0; r < 2 && rc == QSIM_OK; ++r) rc = capture(b, r);
    if (rc != QSIM_OK) return fail_free(rc);
    *out = b;
    return QSIM_OK;
}

void qsim_batch_destroy(qsim_batch *b) { batch_free(b); }

int qsim_batch_load_state(qsim_batch *b, size_t i, const void *host, size_t n_amps)
{
    if (!b || !host || i >= b->n) return bfail(QSIM_EINVAL, "bad batch, index or pointer");
    if (n_amps != (1ull << b->M[i])) return bfail(QSIM_EINVAL, "n_amps must equal 2^M[i]");
    char *dst = b->arena[start_arena(b, i, b->runs)] + b->off[i] * b->amp;
    QB_CUDA(cudaMemcpyAsync(dst, host, n_amps * b->amp, cudaMemcpyHostToDevice, b->stream), "load batch state");
    QB_CUDA(cudaStreamSynchronize(b->stream), "load batch state");
    return QSIM_OK;
}

int qsim_batch_read_state(qsim_batch *b, size_t i, void *host, size_t n_amps)
{
    if (!b || !host || i >= b->n) return bfail(QSIM_EINVAL, "bad batch, index or pointer");
    if (n_amps != (1ull << b->M[i])) return bfail(QSIM_EINVAL, "n_amps must equal 2^M[i]");
    QB_CUDA(cudaStreamSynchronize(b->stream), "batch execution");
    const char *src = b->arena[start_arena(b, i, b->runs)] + b->off[i] * b->amp;
    QB_CUDA(cudaMemcpyAsync(host, src, n_amps * b->amp, cudaMemcpyDeviceToHost, b->stream), "read batch state");
    QB_CUDA(cudaStreamSynchronize(b->stream), "read batch state");
    return QSIM_OK;
}

void *qsim_batch_state_device(qsim_batch *b, size_t i)
{
    if (!b || i >= b->n) return nullptr;
    return b->arena[start_arena(b, i, b->runs)] + b->off[i] * b->amp;
}

int qsim_batch_run(qsim_batch *b)
{
    if (!b) return bfail(QSIM_EINVAL, "batch is NULL");
    QB_CUDA(cudaGraphLaunch(b->graph[b->runs & 1u], b->stream), "cudaGraphLaunch");
    ++b->runs;
    return QSIM_OK;
}

int qsim_batch_run_plain(qsim_batch *b)
{
    if (!b) return bfail(QSIM_EINVAL, "batch is NULL");
    for (size_t i = 0; i < b->n; ++i) {
        int cur = start_arena(b, i, b->runs);
        const Plan &p = b->plans[i];
        const uint64_t *tab = reinterpret_cast<const uint64_t *>(b->d_tab + b->tab_off[i]);
        const SlicedStep *sl = reinterpret_cast<const SlicedStep *>(b->d_tab + b->sl_off[i]);
        for (const Pass &ps : p.passes) {
            char *a_in = b->arena[cur] + b->off[i] * b->amp;
            char *a_out = b->arena[1 - cur] + b->off[i] * b->amp;
            int e;
            if (ps.kind == kSweep) {
                e = launch_sweep(a_in, (int)b->amp, ps.sweep, nullptr, b->stream);
            } else {
                GatherPass g = ps.gather;
                if (b->M[i] < b->coset_min_qubits) g.coset = 0;  // as in the batched plan
                e = launch_gather(a_in, a_out, (int)b->amp, b->M[i], g, tab, sl, b->d_err, nullptr, b->stream);
                cur = 1 - cur;
            }
            if (e != cudaSuccess)
                return bfail(QSIM_ECUDA, std::string("plain launch: ") + cudaGetErrorString((cudaError_t)e));
        }
    }
    ++b->runs;
    return QSIM_OK;
}

int qsim_batch_synchronize(qsim_batch *b)
{
    if (!b) return bfail(QSIM_EINVAL, "batch is NULL");
    QB_CUDA(cudaStreamSynchronize(b->stream), "batch execution");
    return QSIM_OK;
}

int qsim_batch_info(qsim_batch *b, qsim_batch_stats *out)
{
    if (!b || !out) return bfail(QSIM_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->circuits = b->n;
    out->levels = b->levels[0].size();
    for (const auto &lv : b->levels[0]) out->items += lv.n_items;
    for (const Plan &p : b->plans) out->passes += p.passes.size();
    out->amplitude_steps = b->amp_steps;
    out->algorithmic_bytes = b->alg_bytes;
    out->arena_bytes = 2 * b->arena_bytes;
    out->stream = b->stream;
    out->coset_passes = b->coset_passes;
    out->affine_passes = b->affine_passes;
    out->sliced_passes = b->sliced_passes;
    out->sweep_passes = b->sweep_passes;
    return QSIM_OK;
}

}  // extern "C"
