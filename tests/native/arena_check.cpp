// Host check of the serving budget's first-fit allocator (built and run by
// tests/test_native_checks.py, no GPU): random allocation and release sequences
// against the invariants -- blocks are 256-byte multiples inside the arena,
// allocated and free blocks never overlap and together cover it exactly,
// adjacent free blocks are always merged, the used and peak counters agree,
// an allocation fails only when no free block is large enough, and freeing
// everything leaves one free block of the whole size.
#include <cstdio>
#include <random>
#include <vector>

#include "../../paper_quant_ph_0308158_gb300/csrc/arena.h"

namespace {

int check(const qsim::Arena &a, size_t peak_seen, const char *when)
{
    size_t pos = 0, used = 0;
    auto f = a.free_blocks().begin();
    auto u = a.allocated().begin();
    bool prev_free = false;
    while (f != a.free_blocks().end() || u != a.allocated().end()) {
        const bool take_free = u == a.allocated().end() ||
                               (f != a.free_blocks().end() && f->first < u->first);
        const size_t off = take_free ? f->first : u->first, len = take_free ? f->second : u->second;
        if (off != pos || len == 0 || len % 256 || off % 256) {
            std::printf("violation after %s: block at %zu (expected %zu), length %zu\n", when, off, pos, len);
            return 1;
        }
        if (take_free && prev_free) {
            std::printf("violation after %s: adjacent free blocks at %zu not merged\n", when, off);
            return 1;
        }
        prev_free = take_free;
        if (!take_free) used += len;
        pos += len;
        if (take_free) ++f; else ++u;
    }
    if (pos != a.size() || used != a.used() || a.peak() != peak_seen) {
        std::printf("violation after %s: cover %zu of %zu, used %zu vs %zu, peak %zu vs %zu\n", when, pos,
                    a.size(), used, a.used(), a.peak(), peak_seen);
        return 1;
    }
    return 0;
}

}  // namespace

int main()
{
    std::mt19937_64 rng(256);
    long ops = 0;
    for (int trial = 0; trial < 200; ++trial) {
        qsim::Arena a;
        const size_t size = 256 * (1 + rng() % 20000);
        a.init(size);
        std::vector<size_t> live;
        size_t peak = 0;
        for (int k = 0; k < 2000; ++k) {
            if (live.empty() || rng() % 3) {
                const size_t want = 1 + rng() % (size / 8 + 1);
                const size_t need = (want + 255) / 256 * 256;
                size_t largest = 0;
                for (const auto &fb : a.free_blocks()) largest = std::max(largest, fb.second);
                size_t off = 0;
                const bool ok = a.alloc(want, &off);
                if (ok != (largest >= need)) {
                    std::printf("violation: allocation of %zu %s with largest free block %zu\n", want,
                                ok ? "succeeded" : "failed", largest);
                    return 1;
                }
                if (ok) {
                    live.push_back(off);
                    peak = std::max(peak, a.used());
                }
                if (check(a, peak, "alloc")) return 1;
            } else {
                const size_t i = rng() % live.size();
                a.release(live[i]);
                live.erase(live.begin() + (long)i);
                if (check(a, peak, "release")) return 1;
            }
            ++ops;
        }
        for (size_t off : live) a.release(off);
        a.release(12345);  // unknown offsets are ignored
        if (check(a, peak, "releasing everything")) return 1;
        if (a.free_blocks().size() != 1 || a.free_blocks().begin()->second != size || a.used() != 0) {
            std::printf("violation: arena not whole after releasing everything\n");
            return 1;
        }
    }
    std::printf("ok: %ld operations\n", ops);
    return 0;
}
