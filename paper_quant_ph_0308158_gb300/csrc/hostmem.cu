// Page-locked host memory placed for fast host<->device copies.
//
// The state goes in and the FP64 probabilities come out over the host link
// (NVLink-C2C on a Grace host), so the end-to-end rate of a circuit is set by
// those copies once the kernels are fast.  A copy runs at the link rate only
// from host pages the link reaches at full speed, and on a virtualised host
// that is not true of every page: measured 1 GiB chunks of one process's
// page-locked memory copied at 211 GB/s in and 193 GB/s out, except a few
// chunks at 90-150 GB/s (1-7 GB/s on their first copy).  Nothing the process
// can read (its NUMA nodes, its page sizes) tells them apart, so this
// allocator measures: it fills the request with 1 GiB huge-page chunks, each
// page-locked and timed with one copy in each direction, keeps the chunks
// within 15 % of the fastest seen, moves them (mremap keeps their physical
// pages) into one contiguous range and locks that range as one registration.
// Rejected chunks are held until the end, so that the kernel does not hand
// their pages back, and then freed.  Host memory left for the rest of the
// system is checked before every chunk is populated.
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "qsim_internal.h"

namespace {

constexpr size_t kChunk = 1ull << 30;          // one probed unit of a large request
constexpr size_t kSmallAlign = 2ull << 20;     // small requests: one chunk, 2 MiB granules
constexpr size_t kProbeBytes = 32ull << 20;    // per copy direction and probe position
constexpr size_t kHostReserve = 8ull << 30;    // host memory always left to the system
constexpr double kKeepFrac = 0.85;             // a chunk within 15 % of the fastest is kept

std::mutex g_mu;
std::map<uintptr_t, size_t> g_regions;  // base -> bytes of every live allocation

int hfail(int code, const std::string &msg)
{
    qsim::set_last_error(msg);
    return code;
}

size_t avail_bytes()
{
    const long pages = sysconf(_SC_AVPHYS_PAGES), psz = sysconf(_SC_PAGE_SIZE);
    return (pages > 0 && psz > 0) ? (size_t)pages * (size_t)psz : 0;
}

// Anonymous read/write (or reserved, PROT_NONE) mapping of 'bytes' whose start
// is a multiple of 'align' (a power of two), or nullptr.
void *map_aligned(size_t bytes, size_t align, bool reserve_only)
{
    const size_t len = bytes + align;
    void *p = mmap(nullptr, len, reserve_only ? PROT_NONE : (PROT_READ | PROT_WRITE),
                   MAP_PRIVATE | MAP_ANONYMOUS | MAP_NORESERVE, -1, 0);
    if (p == MAP_FAILED) return nullptr;
    const uintptr_t b = reinterpret_cast<uintptr_t>(p);
    const uintptr_t a = (b + align - 1) & ~(uintptr_t)(align - 1);
    if (a > b) munmap(p, a - b);
    const uintptr_t end = b + len, used = a + bytes;
    if (end > used) munmap(reinterpret_cast<void *>(used), end - used);
    return reinterpret_cast<void *>(a);
}

struct Candidate {
    void *p = nullptr;
    double h2d = 0, d2h = 0;  // GB/s, the slower of the probed positions
};

// Times copies between page-locked host chunks and one device buffer.
struct Prober {
    void *dev = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ok = false;
    Prober()
    {
        ok = cudaMalloc(&dev, kProbeBytes) == cudaSuccess &&
             cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    }
    ~Prober()
    {
        if (s) cudaStreamSynchronize(s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        if (dev) cudaFree(dev);
    }
    // GB/s of one copy of n bytes, or 0 on a CUDA error
    double rate(char *host, size_t n, bool d2h)
    {
        if (cudaEventRecord(e0, s) != cudaSuccess) return 0;
        const cudaError_t e = d2h ? cudaMemcpyAsync(host, dev, n, cudaMemcpyDeviceToHost, s)
                                  : cudaMemcpyAsync(dev, host, n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
            return 0;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0) return 0;
        return (double)n / (ms * 1e-3) / 1e9;
    }
    // both directions at the start and the middle of a chunk: the slower
    void probe(Candidate &c, size_t chunk)
    {
        const size_t n = std::min(kProbeBytes, chunk / 2);
        c.h2d = c.d2h = 1e30;
        for (size_t off : {(size_t)0, chunk / 2}) {
            char *h = static_cast<char *>(c.p) + off;
            c.h2d = std::min(c.h2d, rate(h, n, false));
            c.d2h = std::min(c.d2h, rate(h, n, true));
        }
    }
};

void release(Candidate &c, size_t chunk, bool registered)
{
    if (!c.p) return;
    if (registered) cudaHostUnregister(c.p);
    munmap(c.p, chunk);
    c.p = nullptr;
}

}  // namespace

extern "C" {

int qsim_host_alloc(size_t bytes, void **out)
{
    if (!out) return hfail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (bytes == 0) return hfail(QSIM_EINVAL, "bytes is 0");
    const size_t chunk = bytes >= kChunk ? kChunk : (bytes + kSmallAlign - 1) / kSmallAlign * kSmallAlign;
    const size_t nch = (bytes + chunk - 1) / chunk;
    const size_t total = nch * chunk;
    if (total + kHostReserve > avail_bytes())
        return hfail(QSIM_ENOMEM, "host memory: " + std::to_string(total) + " bytes requested, " +
                                      std::to_string(avail_bytes()) + " available");
    // 512 MiB (the largest transparent huge page in use) for 1 GiB chunks
    const size_t align = chunk == kChunk ? (kSmallAlign << 8) : kSmallAlign;
    char *base = static_cast<char *>(map_aligned(total, align, true));
    if (!base) return hfail(QSIM_ENOMEM, "mmap(reserve " + std::to_string(total) + " bytes)");
    Prober pr;
    if (!pr.ok) {
        munmap(base, total);
        return hfail(QSIM_ECUDA, "host allocation probe: device buffer or stream");
    }
    std::vector<Candidate> cands;
    double best_h2d = 0, best_d2h = 0;
    auto kept = [&](const Candidate &c) { return c.h2d >= kKeepFrac * best_h2d && c.d2h >= kKeepFrac * best_d2h; };
    auto n_kept = [&]() { return (size_t)std::count_if(cands.begin(), cands.end(), kept); };
    const size_t max_cands = nch + std::max<size_t>(8, nch / 4);
    int rc = QSIM_OK;
    std::string msg;
    while (n_kept() < nch && cands.size() < max_cands) {
        // rejected chunks stay populated: stop taking more when the host runs low
        if (cands.size() >= nch && chunk + kHostReserve > avail_bytes()) break;
        if (cands.size() < nch && (nch - cands.size()) * chunk + kHostReserve > avail_bytes()) {
            rc = QSIM_ENOMEM;
            msg = "host memory ran short while populating chunks";
            break;
        }
        Candidate c;
        c.p = map_aligned(chunk, align, false);
        if (!c.p) {
            rc = QSIM_ENOMEM;
            msg = "mmap(" + std::to_string(chunk) + " bytes)";
            break;
        }
        madvise(c.p, chunk, MADV_HUGEPAGE);
        std::memset(c.p, 0, chunk);  // populate (the kernel picks the physical pages here)
        if (cudaHostRegister(c.p, chunk, cudaHostRegisterDefault) != cudaSuccess) {
            cudaGetLastError();
            munmap(c.p, chunk);
            rc = QSIM_ECUDA;
            msg = "cudaHostRegister(" + std::to_string(chunk) + " bytes)";
            break;
        }
        pr.probe(c, chunk);
        best_h2d = std::max(best_h2d, c.h2d);
        best_d2h = std::max(best_d2h, c.d2h);
        cands.push_back(c);
    }
    if (rc == QSIM_OK && cands.size() < nch) {
        rc = QSIM_ENOMEM;
        msg = "host memory ran short while populating chunks";
    }
    if (rc != QSIM_OK) {
        for (Candidate &c : cands) release(c, chunk, true);
        munmap(base, total);
        return hfail(rc, msg);
    }
    // the nch fastest (by their slower direction relative to the best) fill the range
    std::stable_sort(cands.begin(), cands.end(), [&](const Candidate &a, const Candidate &b) {
        return std::min(a.h2d / best_h2d, a.d2h / best_d2h) > std::min(b.h2d / best_h2d, b.d2h / best_d2h);
    });
    for (size_t i = 0; i < cands.size(); ++i) {
        if (i >= nch) {
            release(cands[i], chunk, true);
            continue;
        }
        cudaHostUnregister(cands[i].p);
        void *to = base + i * chunk;
        void *r = mremap(cands[i].p, chunk, chunk, MREMAP_MAYMOVE | MREMAP_FIXED, to);
        if (r != to) {
            munmap(cands[i].p, chunk);  // it cannot move: give it up, and the request fails below
            rc = QSIM_ENOMEM;
            msg = "mremap of a host chunk";
        }
        cands[i].p = nullptr;
    }
    if (rc == QSIM_OK && cudaHostRegister(base, total, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        rc = QSIM_ECUDA;
        msg = "cudaHostRegister(" + std::to_string(total) + " bytes)";
    }
    if (rc != QSIM_OK) {
        munmap(base, total);
        return hfail(rc, msg);
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_regions[reinterpret_cast<uintptr_t>(base)] = total;
    }
    *out = base;
    return QSIM_OK;
}

int qsim_host_free(void *p)
{
    if (!p) return QSIM_OK;
    size_t total = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_regions.find(reinterpret_cast<uintptr_t>(p));
        if (it == g_regions.end()) return hfail(QSIM_EINVAL, "not an allocation of qsim_host_alloc");
        total = it->second;
        g_regions.erase(it);
    }
    cudaHostUnregister(p);
    munmap(p, total);
    return QSIM_OK;
}

}  // extern "C"
