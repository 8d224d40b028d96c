// server.cu -- a request loop that serves circuit simulations continuously.
//
// Requests (M, input state, wiring diagram) are validated and planned when
// they are submitted, then wait in FIFO order for admission.  A request is
// admitted when its device memory (state + scratch + FP64 probabilities +
// plan tables) fits in the server's HBM budget -- one cudaMalloc made at
// creation and managed by a first-fit allocator -- and its result fits in the
// pinned host result arena.  Admitted requests upload their state on a copy
// stream.  A scheduler thread runs rounds back to back: each round takes the
// next pass of every request whose state is on the device and launches them
// all as one persistent batch_kernel level (the kernel of qsim_batch), so
// requests that arrive while others run join at the next round and their
// work overlaps on the device.  After its last pass a request's probabilities
// are computed, copied to the host arena on a second copy stream, and its
// device memory is returned to the budget.  The paper has no counterpart: it
// runs one circuit at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qsim_internal.h"

using namespace qsim;

namespace {

using Clock = std::chrono::steady_clock;

int sfail(int code, const std::string &msg)
{
    set_last_error(msg);
    return code;
}

// First-fit allocator over [0, size) with 256-byte granularity; coalesces on free.
class Arena {
  public:
    void init(size_t size) { free_[0] = size; size_ = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                sizes_[*off] = bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off)
    {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t bytes = s->second;
        sizes_.erase(s);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            free_.erase(next);
        }
        auto nx = free_.lower_bound(off);
        if (nx != free_.begin()) {
            auto prev = std::prev(nx);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> sizes_;  // allocated offset -> length
    size_t used_ = 0, peak_ = 0, size_ = 0;
};

struct Request {
    uint64_t id = 0;
    uint32_t M = 0;
    const void *host_in = nullptr;
    Plan plan;
    uint64_t L = 0;
    // device layout inside the arena
    size_t dev_off = 0, host_off = 0;
    char *buf[2] = {nullptr, nullptr};
    double *d_probs = nullptr;
    char *d_tab = nullptr;   // affine tables then sliced steps
    size_t sl_off = 0;       // byte offset of the sliced steps in d_tab
    int cur = 0;
    size_t next_pass = 0;
    enum State { kWaiting, kUploading, kRunning, kFinishing, kDone } state = kWaiting;
    cudaEvent_t uploaded = nullptr, finished = nullptr;
    Clock::time_point t_submit, t_admit, t_done;
    size_t dev_bytes = 0, host_bytes = 0;
};

}  // namespace

struct qsim_server {
    int dtype = 0;
    size_t amp = 0;
    uint32_t max_M = 0;
    char *d_arena = nullptr;
    char *h_arena = nullptr;
    Arena dev, host;
    cudaStream_t compute = nullptr, h2d = nullptr, d2h = nullptr;
    double *d_partials = nullptr, *d_norms = nullptr;
    cudaEvent_t probs_ready = nullptr;
    int device = 0;
    // per-round device descriptors: a ring of slots
    static constexpr int kSlots = 4;
    struct Slot {
        BatchPass *d_passes = nullptr;
        BatchItem *d_items = nullptr;
        BatchPass *h_passes = nullptr;
        BatchItem *h_items = nullptr;
        size_t cap_passes = 0, cap_items = 0;
        uint32_t *d_counter = nullptr;
        cudaEvent_t done = nullptr;
        bool busy = false;
    } slots[kSlots];
    int slot_next = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> waiting;
    std::vector<std::shared_ptr<Request>> active;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    std::deque<uint64_t> completions;  // finished ids not yet drained
    uint64_t next_id = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::string worker_error;
    qsim_server_stats st{};
};

namespace {

size_t amp_of(int dtype) { return dtype == QSIM_C64 ? 8 : dtype == QSIM_C128 ? 16 : 0; }

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t tables_bytes(const Plan &p, size_t *sl_off)
{
    const size_t t = align256(p.gather_tables.size() * sizeof(uint64_t));
    *sl_off = t;
    return t + align256(p.sliced_steps.size() * sizeof(SlicedStep));
}

// Try to admit the head of the queue; called with the lock held.
bool admit_one(qsim_server *s)
{
    if (s->waiting.empty()) return false;
    auto r = s->waiting.front();
    const size_t n = 1ull << r->M;
    size_t sl_off = 0;
    const size_t tb = tables_bytes(r->plan, &sl_off);
    r->dev_bytes = align256(n * s->amp) * 2 + align256(n * 8) + tb;
    r->host_bytes = align256(n * 8);
    size_t doff = 0, hoff = 0;
    if (!s->dev.alloc(r->dev_bytes, &doff)) return false;
    if (!s->host.alloc(r->host_bytes, &hoff)) {
        s->dev.release(doff);
        return false;
    }
    s->waiting.pop_front();
    r->dev_off = doff;
    r->host_off = hoff;
    char *base = s->d_arena + doff;
    r->buf[0] = base;
    r->buf[1] = base + align256(n * s->amp);
    r->d_probs = reinterpret_cast<double *>(base + 2 * align256(n * s->amp));
    r->d_tab = base + 2 * align256(n * s->amp) + align256(n * 8);
    r->sl_off = sl_off;
    r->t_admit = Clock::now();
    // upload state and tables on the copy stream
    cudaMemcpyAsync(r->buf[0], r->host_in, n * s->amp, cudaMemcpyHostToDevice, s->h2d);
    if (!r->plan.gather_tables.empty())
        cudaMemcpyAsync(r->d_tab, r->plan.gather_tables.data(),
                        r->plan.gather_tables.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s->h2d);
    if (!r->plan.sliced_steps.empty())
        cudaMemcpyAsync(r->d_tab + sl_off, r->plan.sliced_steps.data(),
                        r->plan.sliced_steps.size() * sizeof(SlicedStep), cudaMemcpyHostToDevice, s->h2d);
    cudaEventRecord(r->uploaded, s->h2d);
    r->state = Request::kUploading;
    s->active.push_back(r);
    ++s->st.admitted;
    return true;
}

// Queue the FP64 probabilities of a request whose passes are all queued, and
// their copy into the host result arena.
void finish_request(qsim_server *s, const std::shared_ptr<Request> &r)
{
    const uint64_t n = 1ull << r->M;
    launch_probabilities(r->buf[r->cur], (int)s->amp, n, r->d_probs, s->d_partials,
                         probabilities_partials_needed(), nullptr, s->compute);
    s->st.launches += 1;
    cudaEventRecord(s->probs_ready, s->compute);
    cudaStreamWaitEvent(s->d2h, s->probs_ready, 0);
    cudaMemcpyAsync(s->h_arena + r->host_off, r->d_probs, n * 8, cudaMemcpyDeviceToHost, s->d2h);
    cudaEventRecord(r->finished, s->d2h);
    r->state = Request::kFinishing;
}

int ensure_slot(qsim_server::Slot &sl, size_t np, size_t ni)
{
    if (np > sl.cap_passes) {
        if (sl.d_passes) cudaFree(sl.d_passes);
        if (sl.h_passes) cudaFreeHost(sl.h_passes);
        sl.cap_passes = np * 2;
        if (cudaMalloc(&sl.d_passes, sizeof(BatchPass) * sl.cap_passes) != cudaSuccess ||
            cudaMallocHost(&sl.h_passes, sizeof(BatchPass) * sl.cap_passes) != cudaSuccess)
            return QSIM_ENOMEM;
    }
    if (ni > sl.cap_items) {
        if (sl.d_items) cudaFree(sl.d_items);
        if (sl.h_items) cudaFreeHost(sl.h_items);
        sl.cap_items = ni * 2;
        if (cudaMalloc(&sl.d_items, sizeof(BatchItem) * sl.cap_items) != cudaSuccess ||
            cudaMallocHost(&sl.h_items, sizeof(BatchItem) * sl.cap_items) != cudaSuccess)
            return QSIM_ENOMEM;
    }
    return QSIM_OK;
}

// One scheduling round: the next pass of every ready request in one launch.
// Returns true if work was launched.
bool run_round(qsim_server *s, std::vector<std::shared_ptr<Request>> &ready)
{
    qsim_server::Slot &sl = s->slots[s->slot_next];
    if (sl.busy) {
        if (cudaEventQuery(sl.done) != cudaSuccess) return false;  // ring full: wait
        sl.busy = false;
    }
    std::vector<BatchPass> passes;
    std::vector<BatchItem> items;
    uint32_t max_sliced_M = 0;
    bool wide = false;
    for (auto &r : ready) {
        const Pass &p = r->plan.passes[r->next_pass];
        BatchPass bp{};
        bp.M = r->M;
        if (r->M > 32) wide = true;
        uint64_t units = 1ull << r->M;
        if (p.kind == kSweep) {
            bp.kind = 1;
            bp.out = r->buf[r->cur];
            bp.sweep = p.sweep;
            units = p.sweep.n_pairs;
        } else if (p.gather.affine) {
            bp.kind = 3;
            bp.in = r->buf[r->cur];
            bp.out = r->buf[1 - r->cur];
            bp.nbytes = p.gather.nbytes;
            bp.bvec = p.gather.bvec;
            bp.tables = reinterpret_cast<const uint64_t *>(r->d_tab) + p.gather.table_off;
            r->cur = 1 - r->cur;
        } else {
            bp.kind = 4;
            bp.in = r->buf[r->cur];
            bp.out = r->buf[1 - r->cur];
            bp.nsteps = p.gather.nsteps;
            bp.steps = reinterpret_cast<const SlicedStep *>(r->d_tab + r->sl_off) + p.gather.step_off;
            max_sliced_M = std::max(max_sliced_M, r->M);
            r->cur = 1 - r->cur;
        }
        const uint32_t pid = (uint32_t)passes.size();
        passes.push_back(bp);
        for (uint64_t s0 = 0; s0 < units; s0 += kBatchItemOutputs)
            items.push_back(BatchItem{pid, 0, s0, std::min<uint64_t>(kBatchItemOutputs, units - s0)});
        ++r->next_pass;
    }
    if (ensure_slot(sl, passes.size(), items.size()) != QSIM_OK) {
        s->worker_error = "out of memory for round descriptors";
        return false;
    }
    std::memcpy(sl.h_passes, passes.data(), passes.size() * sizeof(BatchPass));
    std::memcpy(sl.h_items, items.data(), items.size() * sizeof(BatchItem));
    cudaMemcpyAsync(sl.d_passes, sl.h_passes, passes.size() * sizeof(BatchPass), cudaMemcpyHostToDevice, s->compute);
    cudaMemcpyAsync(sl.d_items, sl.h_items, items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, s->compute);
    cudaMemsetAsync(sl.d_counter, 0, sizeof(uint32_t), s->compute);
    int e = launch_batch_level((int)s->amp, wide, sl.d_passes, sl.d_items, (uint32_t)items.size(),
                               sl.d_counter, batch_smem_bytes(max_sliced_M), s->compute);
    if (e != cudaSuccess) s->worker_error = std::string("round launch: ") + cudaGetErrorString((cudaError_t)e);
    cudaEventRecord(sl.done, s->compute);
    sl.busy = true;
    s->slot_next = (s->slot_next + 1) % qsim_server::kSlots;
    ++s->st.rounds;
    ++s->st.launches;
    // requests whose last pass was just queued: probabilities, then copy out
    for (auto &r : ready)
        if (r->next_pass == r->plan.passes.size()) finish_request(s, r);
    return true;
}

void worker_loop(qsim_server *s)
{
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        std::vector<std::shared_ptr<Request>> ready;
        bool launched = false, idle = true;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // completions free memory first
            for (auto it = s->active.begin(); it != s->active.end();) {
                auto &r = *it;
                if (r->state == Request::kFinishing && cudaEventQuery(r->finished) == cudaSuccess) {
                    r->t_done = Clock::now();
                    r->state = Request::kDone;
                    s->completions.push_back(r->id);
                    s->dev.release(r->dev_off);
                    ++s->st.completed;
                    s->st.amplitude_steps += (double)(1ull << r->M) * (double)r->L;
                    it = s->active.erase(it);
                    s->cv.notify_all();
                } else {
                    ++it;
                }
            }
            while (admit_one(s)) {
            }
            for (auto &r : s->active) {
                if (r->state == Request::kUploading && cudaEventQuery(r->uploaded) == cudaSuccess) {
                    r->state = Request::kRunning;
                    if (r->plan.passes.empty()) finish_request(s, r);  // nothing to apply
                }
                if (r->state == Request::kRunning && r->next_pass < r->plan.passes.size())
                    ready.push_back(r);
            }
            if (!ready.empty()) launched = run_round(s, ready);
            idle = ready.empty() && s->waiting.empty() && s->active.empty();
            s->st.active = s->active.size();
            s->st.waiting = s->waiting.size();
            s->st.in_use_bytes = s->dev.used();
            s->st.peak_in_use_bytes = s->dev.peak();
            if (idle) s->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
        if (!launched && !idle) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

int qsim_server_create(size_t hbm_budget_bytes, size_t host_result_bytes, int dtype, qsim_server **out)
{
    if (!out) return sfail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    const size_t amp = amp_of(dtype);
    if (!amp) return sfail(QSIM_EINVAL, "unknown dtype");
    if (hbm_budget_bytes < (1u << 20) || host_result_bytes < (1u << 20))
        return sfail(QSIM_EINVAL, "budgets must be at least 1 MiB");
    auto *s = new qsim_server;
    s->dtype = dtype;
    s->amp = amp;
    cudaError_t e = cudaMalloc(&s->d_arena, hbm_budget_bytes);
    if (e != cudaSuccess) {
        delete s;
        return sfail(QSIM_ENOMEM, "cudaMalloc(" + std::to_string(hbm_budget_bytes) + " byte HBM budget)");
    }
    e = cudaMallocHost(&s->h_arena, host_result_bytes);
    if (e != cudaSuccess) {
        cudaFree(s->d_arena);
        delete s;
        return sfail(QSIM_ENOMEM, "cudaMallocHost(result arena)");
    }
    s->dev.init(hbm_budget_bytes);
    s->host.init(host_result_bytes);
    cudaGetDevice(&s->device);
    cudaEventCreateWithFlags(&s->probs_ready, cudaEventDisableTiming);
    cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
    cudaMalloc(&s->d_partials, sizeof(double) * probabilities_partials_needed());
    cudaMalloc(&s->d_norms, sizeof(double));
    for (auto &sl : s->slots) {
        cudaMalloc(&sl.d_counter, sizeof(uint32_t));
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    s->st.budget_bytes = hbm_budget_bytes;
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return QSIM_OK;
}

int qsim_server_submit(qsim_server *s, uint32_t M, const void *host_amps, const qsim_step *steps,
                       size_t L, uint64_t *req_id)
{
    if (!s || !host_amps || !req_id) return sfail(QSIM_EINVAL, "NULL argument");
    auto r = std::make_shared<Request>();
    PlanOptions o;
    o.amp_bytes = s->amp;
    o.scratch_available = true;
    o.strategy = QSIM_STRATEGY_GATHER;
    o.cancel_adjacent = false;
    std::string msg;
    int rc = make_plan(M, steps, L, o, &r->plan, &msg);
    if (rc != QSIM_OK) return sfail(rc, msg);
    const size_t n = 1ull << M;
    size_t sl_off = 0;
    const size_t need = align256(n * s->amp) * 2 + align256(n * 8) + tables_bytes(r->plan, &sl_off);
    if (need > s->dev.size() || align256(n * 8) > s->host.size())
        return sfail(QSIM_EBUSY, "request needs " + std::to_string(need) + " bytes, more than the budget");
    r->M = M;
    r->L = L;
    r->host_in = host_amps;
    r->t_submit = Clock::now();
    cudaEventCreateWithFlags(&r->uploaded, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&r->finished, cudaEventDisableTiming);
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->waiting.push_back(r);
    s->all[r->id] = r;
    ++s->st.submitted;
    *req_id = r->id;
    s->cv.notify_all();
    return QSIM_OK;
}

int qsim_server_poll(qsim_server *s, uint64_t id, int *done, double *latency_ms, const double **probs)
{
    if (!s || !done) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return sfail(QSIM_ENOTFOUND, "unknown request id");
    const auto &r = it->second;
    *done = r->state == Request::kDone;
    if (*done) {
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        if (probs) *probs = reinterpret_cast<const double *>(s->h_arena + r->host_off);
    }
    return QSIM_OK;
}

int qsim_server_drain(qsim_server *s, uint64_t *ids, double *latency_ms, size_t cap, size_t *n_out)
{
    if (!s || !n_out || (cap && !ids)) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    size_t n = 0;
    while (n < cap && !s->completions.empty()) {
        const uint64_t id = s->completions.front();
        s->completions.pop_front();
        auto it = s->all.find(id);
        if (it == s->all.end()) continue;
        ids[n] = id;
        if (latency_ms)
            latency_ms[n] = std::chrono::duration<double, std::milli>(it->second->t_done - it->second->t_submit).count();
        ++n;
    }
    *n_out = n;
    return QSIM_OK;
}

int qsim_server_release(qsim_server *s, uint64_t id)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return sfail(QSIM_ENOTFOUND, "unknown request id");
    if (it->second->state != Request::kDone) return sfail(QSIM_EBUSY, "request still running");
    s->host.release(it->second->host_off);
    cudaEventDestroy(it->second->uploaded);
    cudaEventDestroy(it->second->finished);
    s->all.erase(it);
    s->cv.notify_all();
    return QSIM_OK;
}

int qsim_server_wait_all(qsim_server *s, double timeout_s)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (!(s->waiting.empty() && s->active.empty())) {
        if (!s->worker_error.empty()) return sfail(QSIM_ECUDA, s->worker_error);
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout &&
            !(s->waiting.empty() && s->active.empty()))
            return sfail(QSIM_ETIMEOUT, "requests still pending");
    }
    return QSIM_OK;
}

int qsim_server_get_stats(qsim_server *s, qsim_server_stats *out)
{
    if (!s || !out) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->host_in_use_bytes = s->host.used();
    return QSIM_OK;
}

void qsim_server_destroy(qsim_server *s)
{
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->compute);
    cudaStreamSynchronize(s->h2d);
    cudaStreamSynchronize(s->d2h);
    for (auto &kv : s->all) {
        cudaEventDestroy(kv.second->uploaded);
        cudaEventDestroy(kv.second->finished);
    }
    for (auto &sl : s->slots) {
        if (sl.d_passes) cudaFree(sl.d_passes);
        if (sl.d_items) cudaFree(sl.d_items);
        if (sl.h_passes) cudaFreeHost(sl.h_passes);
        if (sl.h_items) cudaFreeHost(sl.h_items);
        if (sl.d_counter) cudaFree(sl.d_counter);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    cudaFree(s->d_partials);
    cudaFree(s->d_norms);
    cudaEventDestroy(s->probs_ready);
    cudaFree(s->d_arena);
    cudaFreeHost(s->h_arena);
    cudaStreamDestroy(s->compute);
    cudaStreamDestroy(s->h2d);
    cudaStreamDestroy(s->d2h);
    delete s;
}

}  // extern "C"
