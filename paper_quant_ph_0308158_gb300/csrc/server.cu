// server.cu -- a request loop that serves circuit simulations continuously.
//
// Requests (M, input state, wiring diagram) are validated and planned when
// they are submitted, then wait in FIFO order for admission (with bounded
// backfill, see admit()).  A request is admitted when its two device blocks
// (input state + plan tables; a second buffer sized for what the plan writes
// there) fit in the server's HBM budget -- one cudaMalloc made at creation
// and managed by a first-fit allocator -- its result fits in the pinned host
// result arena, and the uploads already queued are short.  Admitted requests
// upload their state on a copy stream.  A scheduler thread runs rounds back
// to back: each round takes the next pass of every request whose state is
// on the device and launches them all as one persistent batch_kernel level
// (the kernel of qsim_batch), so requests that arrive while others run join
// at the next round and their work overlaps on the device.  A request's last
// gather pass writes only the FP64 probabilities of its result (the served
// output), into the buffer it does not read; the other block then returns to
// the budget, the probabilities are copied to the host arena on a second
// copy stream, and their block returns after the copy.  The paper has no
// counterpart: it runs one circuit at a time.
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

#include "arena.h"
#include "qsim_internal.h"

using namespace qsim;

namespace {

using Clock = std::chrono::steady_clock;

int sfail(int code, const std::string &msg)
{
    set_last_error(msg);
    return code;
}

struct Request {
    uint64_t id = 0;
    uint32_t M = 0;
    const void *host_in = nullptr;
    Plan plan;
    uint64_t L = 0;
    // device memory: two arena blocks.  Block 0 holds the input state buf[0]
    // and the plan tables, block 1 the second buffer buf[1], sized for what
    // the plan writes there (a state for a gather pass that is not the last,
    // else only the probabilities).  The probabilities go to the buffer the
    // last pass does not read; once they are written the other block is
    // returned to the budget, and the probabilities' block after the copy out.
    size_t off[2] = {0, 0}, bytes[2] = {0, 0};
    bool held[2] = {false, false};
    size_t host_off = 0;
    char *buf[2] = {nullptr, nullptr};
    char *d_tab = nullptr;   // affine tables then sliced steps
    size_t sl_off = 0;       // byte offset of the sliced steps in d_tab
    int cur = 0;
    size_t next_pass = 0;
    bool probs_fused = false;  // the last pass writes the probabilities (and no state)
    int probs_buf = -1;        // buffer holding the probabilities
    double compute_start_ms = -1, compute_end_ms = -1;  // rounds that ran its passes (trace)
    enum State { kWaiting, kUploading, kRunning, kComputing, kFinishing, kDone, kDraining, kSwappingOut,
                 kSwappedOut }
        state = kWaiting;
    int last_slot = -1;        // round slot of the last round that ran one of its passes
    size_t swap_off = 0;       // host block holding its state while swapped out
    bool swap_held = false;
    cudaEvent_t swapped = nullptr;  // the state's copy out (eviction) is done
    cudaEvent_t uploaded = nullptr, computed = nullptr, finished = nullptr;
    cudaEvent_t up0 = nullptr, down0 = nullptr;  // timing: starts of the two copies
    Clock::time_point t_submit, t_admit, t_done;
    size_t host_bytes = 0;
    bool failed = false;     // admission failed: no memory held, 'error' says why
    std::string error;
};

}  // namespace

struct qsim_server {
    int dtype = 0;
    size_t amp = 0;
    char *d_arena = nullptr;
    char *h_arena = nullptr;
    Arena dev, host;
    cudaStream_t compute = nullptr, h2d = nullptr, d2h = nullptr;
    double *d_partials = nullptr, *d_norms = nullptr;
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
        cudaEvent_t start = nullptr, done = nullptr;  // timing events around the round
        bool busy = false;
        std::vector<std::shared_ptr<Request>> members;  // requests with a pass in the round
    } slots[kSlots];
    double max_head_wait_ms = 100.0;  // backfill admission while the head waited less
    size_t pending_upload_bytes = 0;  // admitted states not yet on the device
    int copy_streams = 2;             // 2: copies in and out overlap; 1: one copy stream
    size_t upload_chunk = 0;          // state uploads in copies of at most this many bytes (0: one)
    double evict_after_ms = -1.0;     // evict running requests for a head that waited this long
    uint64_t evicting_for = 0;        // head request id that evictions are making room for
    std::deque<std::shared_ptr<Request>> swapped;  // evicted requests, in eviction order
    cudaEvent_t t0_event = nullptr;   // device-time origin of the trace
    Clock::time_point t0;             // host-time origin of the trace
    bool tracing = false;
    std::vector<qsim_server_trace_record> trace;
    bool paused = false;              // admission paused (running requests continue)
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

// Bytes of the two device blocks of a request (see Request): follow the
// plan's ping-pong and record the largest write into each buffer.
void block_sizes(const Plan &p, uint32_t M, size_t amp, size_t out[2])
{
    const size_t n = 1ull << M;
    size_t need[2] = {n * amp, n * 8};
    int cur = 0;
    for (size_t i = 0; i < p.passes.size(); ++i) {
        if (p.passes[i].kind == kSweep) continue;  // in place
        if (i + 1 < p.passes.size()) need[1 - cur] = std::max(need[1 - cur], n * amp);
        cur = 1 - cur;
    }
    size_t sl = 0;
    out[0] = align256(need[0]) + tables_bytes(p, &sl);
    out[1] = align256(need[1]);
}

// Admitted states whose upload has not finished, in bytes, above which no
// further request is admitted (about 40 ms of the host link).
constexpr size_t kMaxPendingUpload = 8ull << 30;

// Try to admit waiting request r; called with the lock held.
// Outcome of one admission attempt.
enum Admit { kNotAdmitted, kAdmitted, kAdmitFailed };

// An admitted request whose uploads could not be queued: give back both
// device blocks and the host block and complete it as failed, so that it
// never runs on memory it did not fill.  Called with the lock held.
Admit fail_admission(qsim_server *s, const std::shared_ptr<Request> &r, const char *what,
                     cudaError_t e)
{
    for (int b = 0; b < 2; ++b)
        if (r->held[b]) {
            s->dev.release(r->off[b]);
            r->held[b] = false;
        }
    s->host.release(r->host_off);
    r->failed = true;
    r->error = std::string(what) + ": " + cudaGetErrorString(e);
    r->state = Request::kDone;
    r->t_done = Clock::now();
    s->completions.push_back(r->id);
    return kAdmitFailed;
}

Admit try_admit(qsim_server *s, const std::shared_ptr<Request> &r)
{
    const size_t n = 1ull << r->M;
    // a request is admitted when the uploads already queued are short, so
    // that its memory is not held while it waits for the copy stream
    if (s->pending_upload_bytes >= kMaxPendingUpload) return kNotAdmitted;
    size_t sl_off = 0;
    const size_t tb = tables_bytes(r->plan, &sl_off);
    block_sizes(r->plan, r->M, s->amp, r->bytes);
    // result probabilities, then a pinned copy of the plan tables: a copy
    // from pageable memory would hold this thread until the copy stream
    // reached it
    r->host_bytes = align256(n * 8) + tb;
    size_t hoff = 0;
    if (!s->dev.alloc(r->bytes[0], &r->off[0])) return kNotAdmitted;
    if (!s->dev.alloc(r->bytes[1], &r->off[1])) {
        s->dev.release(r->off[0]);
        return kNotAdmitted;
    }
    if (!s->host.alloc(r->host_bytes, &hoff)) {
        s->dev.release(r->off[0]);
        s->dev.release(r->off[1]);
        return kNotAdmitted;
    }
    r->held[0] = r->held[1] = true;
    r->host_off = hoff;
    r->buf[0] = s->d_arena + r->off[0];
    r->buf[1] = s->d_arena + r->off[1];
    r->d_tab = r->buf[0] + align256(n * s->amp);
    r->sl_off = sl_off;
    r->t_admit = Clock::now();
    // upload state and tables on the copy stream
    char *h_tab = s->h_arena + hoff + align256(n * 8);
    if (!r->plan.gather_tables.empty())
        std::memcpy(h_tab, r->plan.gather_tables.data(), r->plan.gather_tables.size() * sizeof(uint64_t));
    if (!r->plan.sliced_steps.empty())
        std::memcpy(h_tab + sl_off, r->plan.sliced_steps.data(),
                    r->plan.sliced_steps.size() * sizeof(SlicedStep));
    cudaError_t e = cudaEventRecord(r->up0, s->h2d);
    if (e != cudaSuccess) return fail_admission(s, r, "cudaEventRecord(upload start)", e);
    const auto e0 = Clock::now();
    {
        const size_t total = n * s->amp;
        const size_t chunk = s->upload_chunk ? s->upload_chunk : total;
        for (size_t off = 0; off < total && e == cudaSuccess; off += chunk)
            e = cudaMemcpyAsync(r->buf[0] + off, static_cast<const char *>(r->host_in) + off,
                                std::min(chunk, total - off), cudaMemcpyHostToDevice, s->h2d);
    }
    if (e != cudaSuccess) return fail_admission(s, r, "cudaMemcpyAsync(state upload)", e);
    if (tb) {
        e = cudaMemcpyAsync(r->d_tab, h_tab, tb, cudaMemcpyHostToDevice, s->h2d);
        if (e != cudaSuccess) return fail_admission(s, r, "cudaMemcpyAsync(plan tables)", e);
    }
    // a copy from memory the driver does not see as pinned runs on this
    // thread (and stalls the scheduler): record how long issuing took
    const double enq = std::chrono::duration<double, std::milli>(Clock::now() - e0).count();
    s->st.issue_ms += enq;
    s->st.issue_ms_max = std::max(s->st.issue_ms_max, enq);
    e = cudaEventRecord(r->uploaded, s->h2d);
    if (e != cudaSuccess) return fail_admission(s, r, "cudaEventRecord(uploaded)", e);
    s->st.h2d_bytes += n * s->amp;
    s->pending_upload_bytes += n * s->amp;
    r->state = Request::kUploading;
    s->active.push_back(r);
    ++s->st.admitted;
    return kAdmitted;
}

// A swapped-out request comes back: its blocks are allocated again, its state
// is copied into the buffer that held it (so the plan's ping-pong and block
// sizes stay as at admission) and its tables are copied again; it then runs
// on from its next pass.  Called with the lock held.
bool try_swap_in(qsim_server *s, const std::shared_ptr<Request> &r)
{
    const size_t n = 1ull << r->M;
    if (s->pending_upload_bytes >= kMaxPendingUpload) return false;
    size_t sl_off = 0;
    const size_t tb = tables_bytes(r->plan, &sl_off);
    if (!s->dev.alloc(r->bytes[0], &r->off[0])) return false;
    if (!s->dev.alloc(r->bytes[1], &r->off[1])) {
        s->dev.release(r->off[0]);
        return false;
    }
    r->held[0] = r->held[1] = true;
    r->buf[0] = s->d_arena + r->off[0];
    r->buf[1] = s->d_arena + r->off[1];
    r->d_tab = r->buf[0] + align256(n * s->amp);
    const char *h_tab = s->h_arena + r->host_off + align256(n * 8);
    cudaError_t e = cudaEventRecord(r->up0, s->h2d);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->buf[r->cur], s->h_arena + r->swap_off, n * s->amp, cudaMemcpyHostToDevice, s->h2d);
    if (e == cudaSuccess && tb) e = cudaMemcpyAsync(r->d_tab, h_tab, tb, cudaMemcpyHostToDevice, s->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(r->uploaded, s->h2d);
    if (e != cudaSuccess) {
        if (!s->worker_error.size()) s->worker_error = std::string("swap-in copy: ") + cudaGetErrorString(e);
        return false;
    }
    s->st.h2d_bytes += n * s->amp;
    s->pending_upload_bytes += n * s->amp;
    r->state = Request::kUploading;
    s->active.push_back(r);
    ++s->st.swapped_in;
    return true;
}

// Copy an evicted request's state out to a host block once its last round
// has finished; its device blocks return to the budget when the copy is done.
// Returns false if it must wait (round still running, or no host block yet).
bool start_swap_out(qsim_server *s, const std::shared_ptr<Request> &r)
{
    if (r->last_slot >= 0 && cudaEventQuery(s->slots[r->last_slot].done) != cudaSuccess) return false;
    const size_t n = 1ull << r->M;
    size_t off = 0;
    if (!s->host.alloc(n * s->amp, &off)) return false;
    cudaStream_t st = s->copy_streams == 1 ? s->h2d : s->d2h;
    cudaError_t e = cudaMemcpyAsync(s->h_arena + off, r->buf[r->cur], n * s->amp, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(r->swapped, st);
    if (e != cudaSuccess) {
        s->host.release(off);
        if (s->worker_error.empty()) s->worker_error = std::string("eviction copy: ") + cudaGetErrorString(e);
        return false;
    }
    r->swap_off = off;
    r->swap_held = true;
    r->state = Request::kSwappingOut;
    s->st.d2h_bytes += n * s->amp;
    return true;
}

// Make room for the head of the queue, which has waited evict_after_ms: the
// running requests admitted most recently leave the rounds (they drain), and
// once their last round has finished their states are copied out to host
// blocks (start_swap_out) -- the paper's trade of memory for processing
// (Sec. 1, Sec. 5) applied to whole states.  Called with the lock held.
void evict_for(qsim_server *s, const std::shared_ptr<Request> &head)
{
    for (const auto &r : s->active)
        if (r->state == Request::kDraining || r->state == Request::kSwappingOut) return;  // under way
    size_t hb[2];
    block_sizes(head->plan, head->M, s->amp, hb);
    const size_t need = hb[0] + hb[1];
    size_t freed = s->dev.capacity() - s->dev.used();
    const size_t host_free = s->host.capacity() - s->host.used();
    size_t host_need = 0;
    for (auto it = s->active.rbegin(); it != s->active.rend() && freed < need; ++it) {
        const auto &r = *it;
        if (r->state != Request::kRunning || r->next_pass >= r->plan.passes.size()) continue;
        const size_t n = 1ull << r->M;
        if (host_need + n * s->amp > host_free) continue;
        host_need += n * s->amp;
        r->state = Request::kDraining;
        ++s->st.evicted;
        freed += r->bytes[0] + r->bytes[1];
        s->evicting_for = head->id;
    }
}

// Admission: FIFO, except that while the head of the queue does not fit and
// has waited less than max_head_wait_ms, later requests that fit are admitted
// ahead of it (backfill); after that nothing passes the head, so the budget
// drains until it fits -- or, with eviction on, running requests are swapped
// out to host memory for it once it has waited evict_after_ms.  Swapped-out
// requests come back as soon as they fit, ahead of everything but the head.
// Called with the lock held.
void admit(qsim_server *s)
{
    constexpr size_t kWindow = 256;  // requests looked at behind the head
    if (s->paused) return;
    while (!s->waiting.empty() && try_admit(s, s->waiting.front()) != kNotAdmitted) {
        if (s->waiting.front()->id == s->evicting_for) s->evicting_for = 0;
        s->waiting.pop_front();
    }
    if (s->waiting.empty()) s->evicting_for = 0;
    if (!s->evicting_for)  // the memory freed for a head is the head's first
        for (auto it = s->swapped.begin(); it != s->swapped.end();) {
            if (try_swap_in(s, *it)) it = s->swapped.erase(it);
            else ++it;
        }
    if (s->waiting.empty()) return;
    const double head_wait =
        std::chrono::duration<double, std::milli>(Clock::now() - s->waiting.front()->t_submit).count();
    if (s->evict_after_ms >= 0 && head_wait >= s->evict_after_ms) evict_for(s, s->waiting.front());
    if (s->max_head_wait_ms < 0 || head_wait >= s->max_head_wait_ms || s->evicting_for) return;
    size_t looked = 0;
    for (auto it = std::next(s->waiting.begin()); it != s->waiting.end() && looked < kWindow; ++looked) {
        const Admit a = try_admit(s, *it);
        if (a != kNotAdmitted) {
            if (a == kAdmitted) ++s->st.backfilled;
            it = s->waiting.erase(it);
        } else {
            ++it;
        }
    }
}

// Queue the FP64 probabilities of a request whose passes are all queued (the
// copy out is queued once they are written, see start_download).
void finish_request(qsim_server *s, const std::shared_ptr<Request> &r)
{
    const uint64_t n = 1ull << r->M;
    if (!r->probs_fused) {  // the final state is in buf[cur]; the other buffer is free
        r->probs_buf = 1 - r->cur;
        launch_probabilities(r->buf[r->cur], (int)s->amp, n,
                             reinterpret_cast<double *>(r->buf[r->probs_buf]), s->d_partials,
                             probabilities_partials_needed(), nullptr, s->compute);
        s->st.launches += 1;
    }
    cudaEventRecord(r->computed, s->compute);
    r->state = Request::kComputing;
}

// The probabilities are written: return the other block to the budget and
// queue their copy into the host result arena.  Queued only now, so that a
// copy stream shared with the uploads never waits on the compute stream.
void start_download(qsim_server *s, const std::shared_ptr<Request> &r)
{
    const uint64_t n = 1ull << r->M;
    const int other = 1 - r->probs_buf;
    s->dev.release(r->off[other]);
    r->held[other] = false;
    cudaStream_t st = s->copy_streams == 1 ? s->h2d : s->d2h;
    cudaEventRecord(r->down0, st);
    const auto e0 = Clock::now();
    cudaMemcpyAsync(s->h_arena + r->host_off, r->buf[r->probs_buf], n * 8, cudaMemcpyDeviceToHost, st);
    const double enq = std::chrono::duration<double, std::milli>(Clock::now() - e0).count();
    s->st.issue_ms += enq;
    s->st.issue_ms_max = std::max(s->st.issue_ms_max, enq);
    s->st.d2h_bytes += n * 8;
    cudaEventRecord(r->finished, st);
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
    if (sl.busy) return false;  // ring full: wait for the oldest round
    std::vector<BatchPass> passes;
    std::vector<BatchItem> items;
    uint32_t max_sliced_M = 0;
    bool wide = false;
    for (auto &r : ready) {
        const Pass &p = r->plan.passes[r->next_pass];
        const bool last = r->next_pass + 1 == r->plan.passes.size();
        BatchPass bp{};
        bp.M = r->M;
        if (r->M > 32) wide = true;
        uint64_t units = 1ull << r->M;
        if (p.kind == kSweep) {
            bp.kind = 1;
            bp.out = r->buf[r->cur];
            bp.sweep = p.sweep;
            units = p.sweep.n_pairs;
        } else {
            bp.in = r->buf[r->cur];
            bp.out = r->buf[1 - r->cur];
            if (p.gather.affine) {
                bp.kind = 3;
                bp.nbytes = p.gather.nbytes;
                bp.bvec = p.gather.bvec;
                bp.tables = reinterpret_cast<const uint64_t *>(r->d_tab) + p.gather.table_off;
            } else {
                bp.kind = 4;
                bp.nsteps = p.gather.nsteps;
                bp.steps = reinterpret_cast<const SlicedStep *>(r->d_tab + r->sl_off) + p.gather.step_off;
                max_sliced_M = std::max(max_sliced_M, r->M);
            }
            if (last) {  // only the probabilities of the result are served: no state is stored
                bp.probs = reinterpret_cast<double *>(bp.out);
                bp.out = nullptr;
                r->probs_buf = 1 - r->cur;
                r->probs_fused = true;
            }
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
    cudaEventRecord(sl.start, s->compute);
    int e = launch_batch_level((int)s->amp, wide, sl.d_passes, sl.d_items, (uint32_t)items.size(),
                               sl.d_counter, batch_smem_bytes(max_sliced_M), s->compute);
    if (e != cudaSuccess) s->worker_error = std::string("round launch: ") + cudaGetErrorString((cudaError_t)e);
    cudaEventRecord(sl.done, s->compute);
    sl.busy = true;
    if (s->tracing) sl.members = ready;
    s->slot_next = (s->slot_next + 1) % qsim_server::kSlots;
    ++s->st.rounds;
    ++s->st.launches;
    // requests whose last pass was just queued: probabilities, then copy out
    for (auto &r : ready) {
        r->last_slot = (int)(&sl - s->slots);
        if (r->next_pass == r->plan.passes.size()) finish_request(s, r);
    }
    return true;
}

constexpr size_t kMaxTrace = 1u << 22;

double host_ms(const qsim_server *s, Clock::time_point t)
{
    return std::chrono::duration<double, std::milli>(t - s->t0).count();
}

double dev_ms(const qsim_server *s, cudaEvent_t e)
{
    float ms = 0.f;
    return cudaEventElapsedTime(&ms, s->t0_event, e) == cudaSuccess ? (double)ms : -1.0;
}

// One finished request's timeline (host and device clocks share the origin
// taken when tracing was switched on).  Called with the lock held.
void record_trace(qsim_server *s, const Request &r)
{
    qsim_server_trace_record t{};
    t.id = r.id;
    t.M = r.M;
    t.passes = (uint32_t)r.plan.passes.size();
    t.L = r.L;
    t.submit_ms = host_ms(s, r.t_submit);
    t.admit_ms = host_ms(s, r.t_admit);
    t.upload_start_ms = dev_ms(s, r.up0);
    t.upload_end_ms = dev_ms(s, r.uploaded);
    t.compute_start_ms = r.compute_start_ms;
    t.compute_end_ms = r.compute_end_ms;
    t.download_start_ms = dev_ms(s, r.down0);
    t.download_end_ms = dev_ms(s, r.finished);
    t.done_ms = host_ms(s, r.t_done);
    s->trace.push_back(t);
}

// Retire finished rounds: their descriptor slots become free and their
// durations are added to the compute time.  Called with the lock held.
void retire_rounds(qsim_server *s)
{
    for (auto &sl : s->slots) {
        if (!sl.busy || cudaEventQuery(sl.done) != cudaSuccess) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sl.start, sl.done) == cudaSuccess) s->st.compute_busy_ms += ms;
        if (s->tracing) {
            const double a = dev_ms(s, sl.start), b = dev_ms(s, sl.done);
            for (auto &r : sl.members) {
                if (r->compute_start_ms < 0) r->compute_start_ms = a;
                r->compute_end_ms = b;
            }
        }
        sl.members.clear();
        sl.busy = false;
    }
}

void worker_loop(qsim_server *s)
{
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        std::vector<std::shared_ptr<Request>> ready;
        bool launched = false, idle = true;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            retire_rounds(s);
            // completions free memory first: the block without the
            // probabilities once they are written, the rest after the copy out
            for (auto it = s->active.begin(); it != s->active.end();) {
                auto &r = *it;
                if (r->state == Request::kComputing && cudaEventQuery(r->computed) == cudaSuccess)
                    start_download(s, r);
                if (r->state == Request::kFinishing && cudaEventQuery(r->finished) == cudaSuccess) {
                    r->t_done = Clock::now();
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, r->up0, r->uploaded) == cudaSuccess) s->st.h2d_busy_ms += ms;
                    if (cudaEventElapsedTime(&ms, r->down0, r->finished) == cudaSuccess) s->st.d2h_busy_ms += ms;
                    if (s->tracing && s->trace.size() < kMaxTrace) record_trace(s, *r);
                    r->state = Request::kDone;
                    s->completions.push_back(r->id);
                    for (int b = 0; b < 2; ++b)
                        if (r->held[b]) s->dev.release(r->off[b]);
                    r->held[0] = r->held[1] = false;
                    ++s->st.completed;
                    s->st.amplitude_steps += (double)(1ull << r->M) * (double)r->L;
                    it = s->active.erase(it);
                    s->cv.notify_all();
                } else {
                    ++it;
                }
            }
            retire_rounds(s);  // after the completions: their rounds are done
            // evicted states copied out: their device blocks return to the budget
            for (auto it = s->active.begin(); it != s->active.end();) {
                auto &r = *it;
                if (r->state == Request::kDraining) start_swap_out(s, r);
                if (r->state == Request::kSwappingOut && cudaEventQuery(r->swapped) == cudaSuccess) {
                    for (int b = 0; b < 2; ++b)
                        if (r->held[b]) s->dev.release(r->off[b]);
                    r->held[0] = r->held[1] = false;
                    r->state = Request::kSwappedOut;
                    s->swapped.push_back(r);
                    it = s->active.erase(it);
                } else {
                    ++it;
                }
            }
            admit(s);
            for (auto &r : s->active) {
                if (r->state == Request::kUploading && cudaEventQuery(r->uploaded) == cudaSuccess) {
                    r->state = Request::kRunning;
                    s->pending_upload_bytes -= (1ull << r->M) * s->amp;
                    if (r->swap_held) {  // back from host memory
                        s->host.release(r->swap_off);
                        r->swap_held = false;
                    }
                    if (r->plan.passes.empty()) finish_request(s, r);  // nothing to apply
                }
                if (r->state == Request::kRunning && r->next_pass < r->plan.passes.size())
                    ready.push_back(r);
            }
            if (!ready.empty()) launched = run_round(s, ready);
            idle = ready.empty() && s->waiting.empty() && s->active.empty() && s->swapped.empty();
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
    cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
    cudaMalloc(&s->d_partials, sizeof(double) * probabilities_partials_needed());
    cudaMalloc(&s->d_norms, sizeof(double));
    for (auto &sl : s->slots) {
        cudaMalloc(&sl.d_counter, sizeof(uint32_t));
        cudaEventCreate(&sl.start);
        cudaEventCreate(&sl.done);
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
    o.coset = false;  // affine passes run inside batch_kernel work items
    std::string msg;
    int rc = make_plan(M, steps, L, o, &r->plan, &msg);
    if (rc != QSIM_OK) return sfail(rc, msg);
    const size_t n = 1ull << M;
    size_t sl_off = 0, blocks[2];
    block_sizes(r->plan, M, s->amp, blocks);
    const size_t need = blocks[0] + blocks[1];
    if (need > s->dev.size() || align256(n * 8) + tables_bytes(r->plan, &sl_off) > s->host.size())
        return sfail(QSIM_EBUSY, "request needs " + std::to_string(need) + " bytes, more than the budget");
    r->M = M;
    r->L = L;
    r->host_in = host_amps;
    r->t_submit = Clock::now();
    cudaEventCreate(&r->uploaded);
    cudaEventCreateWithFlags(&r->computed, cudaEventDisableTiming);
    cudaEventCreate(&r->finished);
    cudaEventCreate(&r->up0);
    cudaEventCreate(&r->down0);
    cudaEventCreateWithFlags(&r->swapped, cudaEventDisableTiming);
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
    if (r->failed) return sfail(QSIM_ECUDA, "request " + std::to_string(id) + " failed: " + r->error);
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
    if (!it->second->failed) s->host.release(it->second->host_off);  // a failed one gave it back
    cudaEventDestroy(it->second->uploaded);
    cudaEventDestroy(it->second->computed);
    cudaEventDestroy(it->second->finished);
    cudaEventDestroy(it->second->up0);
    cudaEventDestroy(it->second->down0);
    cudaEventDestroy(it->second->swapped);
    s->all.erase(it);
    s->cv.notify_all();
    return QSIM_OK;
}

int qsim_server_wait_all(qsim_server *s, double timeout_s)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (!(s->waiting.empty() && s->active.empty() && s->swapped.empty())) {
        if (!s->worker_error.empty()) return sfail(QSIM_ECUDA, s->worker_error);
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout &&
            !(s->waiting.empty() && s->active.empty() && s->swapped.empty()))
            return sfail(QSIM_ETIMEOUT, "requests still pending");
    }
    return QSIM_OK;
}

int qsim_server_set_backfill(qsim_server *s, double max_head_wait_ms)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_head_wait_ms = max_head_wait_ms;
    return QSIM_OK;
}

int qsim_server_set_paused(qsim_server *s, int paused)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
    s->cv.notify_all();
    return QSIM_OK;
}

int qsim_server_set_tracing(qsim_server *s, int enable)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (enable && !s->tracing) {
        s->trace.clear();
        if (!s->t0_event && cudaEventCreate(&s->t0_event) != cudaSuccess)
            return sfail(QSIM_ECUDA, "cudaEventCreate(trace origin)");
        cudaEventRecord(s->t0_event, s->h2d);
        cudaEventSynchronize(s->t0_event);
        s->t0 = Clock::now();
    }
    s->tracing = enable != 0;
    return QSIM_OK;
}

int qsim_server_get_trace(qsim_server *s, qsim_server_trace_record *out, size_t cap, size_t *n_out)
{
    if (!s || !n_out || (cap && !out)) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t n = std::min(cap, s->trace.size());
    if (n) std::memcpy(out, s->trace.data(), n * sizeof(qsim_server_trace_record));
    s->trace.erase(s->trace.begin(), s->trace.begin() + (std::ptrdiff_t)n);
    *n_out = n;
    return QSIM_OK;
}

int qsim_server_set_eviction(qsim_server *s, double evict_after_ms)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->evict_after_ms = evict_after_ms;
    s->cv.notify_all();
    return QSIM_OK;
}

int qsim_server_set_upload_chunk(qsim_server *s, size_t bytes)
{
    if (!s) return sfail(QSIM_EINVAL, "NULL argument");
    if (bytes && (bytes < (1u << 20) || bytes % 256)) return sfail(QSIM_EINVAL, "chunk must be 0 or >= 1 MiB, a multiple of 256");
    std::lock_guard<std::mutex> lk(s->mu);
    s->upload_chunk = bytes;
    return QSIM_OK;
}

int qsim_server_set_copy_streams(qsim_server *s, int n)
{
    if (!s || (n != 1 && n != 2)) return sfail(QSIM_EINVAL, "copy streams must be 1 or 2");
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->active.empty()) return sfail(QSIM_EBUSY, "requests are running");
    s->copy_streams = n;
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
        cudaEventDestroy(kv.second->computed);
        cudaEventDestroy(kv.second->finished);
        cudaEventDestroy(kv.second->up0);
        cudaEventDestroy(kv.second->down0);
    }
    for (auto &sl : s->slots) {
        if (sl.d_passes) cudaFree(sl.d_passes);
        if (sl.d_items) cudaFree(sl.d_items);
        if (sl.h_passes) cudaFreeHost(sl.h_passes);
        if (sl.h_items) cudaFreeHost(sl.h_items);
        if (sl.d_counter) cudaFree(sl.d_counter);
        if (sl.start) cudaEventDestroy(sl.start);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    cudaFree(s->d_partials);
    cudaFree(s->d_norms);
    if (s->t0_event) cudaEventDestroy(s->t0_event);
    cudaFree(s->d_arena);
    cudaFreeHost(s->h_arena);
    cudaStreamDestroy(s->compute);
    cudaStreamDestroy(s->h2d);
    cudaStreamDestroy(s->d2h);
    delete s;
}

}  // extern "C"
