// Host check of the tile planner (built and run by tests/test_native_checks.py,
// no GPU).  It includes the planner's source and verifies, for random tile
// geometries and for the plans of random circuits:
//   1. the local bit order covers the tile's address bits exactly once, and
//      the bits outside the tile are exactly the tile-id bits;
//   2. every tensor-map copy stays inside the tensor's extents, starts on a
//      16-byte boundary (x times the 8-byte element), lands on a 128-byte
//      aligned shared-memory offset, and each of its elements is the
//      amplitude whose global index the local order names;
//   3. the per-tile step encoding (local control/polarity/target masks,
//      out-of-tile control/polarity) maps every sampled output row to the
//      same source row as the circuit's own steps applied last to first.
// Prints "ok ..." and exits 0, or prints the first violation and exits 1.
#include <cstdio>
#include <random>
#include <vector>

#include "../../paper_quant_ph_0308158_gb300/csrc/planner.cpp"

using namespace qsim;

namespace {

int fail_at(const char *what, uint32_t M, size_t amp)
{
    std::printf("violation: %s (M=%u, amplitude %zu bytes)\n", what, M, amp);
    return 1;
}

uint64_t tile_mask_of(const TilePass &t)
{
    uint64_t m = (t.l >= 64) ? ~0ull : ((1ull << t.l) - 1ull);
    for (uint32_t q = 0; q < t.nh; ++q) m |= 1ull << t.high[q];
    return m;
}

// Global index of local index j of the tile at base (local order: the l low
// bits, then high[0..nh)).
uint64_t global_of(const TilePass &t, uint64_t base, uint64_t j)
{
    uint64_t g = base | (j & ((1ull << t.l) - 1ull));
    for (uint32_t q = 0; q < t.nh; ++q)
        if ((j >> (t.l + q)) & 1ull) g |= 1ull << t.high[q];
    return g;
}

uint64_t local_of(const TilePass &t, uint64_t g)
{
    uint64_t j = g & ((1ull << t.l) - 1ull);
    for (uint32_t q = 0; q < t.nh; ++q)
        if ((g >> t.high[q]) & 1ull) j |= 1ull << (t.l + q);
    return j;
}

// Properties 1 and 2 for one laid-out tile pass; samples elements of copies
// issued for random tiles.
int check_layout(uint32_t M, size_t amp, const TilePass &t, std::mt19937_64 &rng, long *elems)
{
    const uint64_t tmask = tile_mask_of(t);
    uint64_t seen = (1ull << t.l) - 1ull;
    for (uint32_t q = 0; q < t.nh; ++q) {
        if (t.high[q] >= M || ((seen >> t.high[q]) & 1ull)) return fail_at("tile bit repeated or out of range", M, amp);
        seen |= 1ull << t.high[q];
    }
    if (t.k != t.l + t.nh) return fail_at("tile width", M, amp);
    if (t.nout != M - t.k) return fail_at("tile-id bit count", M, amp);
    uint64_t out = 0;
    for (uint32_t q = 0; q < t.nout; ++q) {
        if (t.outpos[q] >= M || ((tmask >> t.outpos[q]) & 1ull) || ((out >> t.outpos[q]) & 1ull))
            return fail_at("tile-id bits", M, amp);
        out |= 1ull << t.outpos[q];
    }
    const uint64_t all = M >= 64 ? ~0ull : ((1ull << M) - 1ull);
    if ((out | tmask) != all) return fail_at("tile and tile-id bits do not cover the index", M, amp);
    if (!t.tma) return 0;
    const uint32_t epa = amp == 16 ? 2 : 1;
    uint64_t boxel = 1;
    for (int d = 0; d < 5; ++d) boxel *= t.tma_box[d];
    if (boxel * 8 != t.box_bytes) return fail_at("box bytes", M, amp);
    if (t.box_bytes % 128) return fail_at("box not a multiple of 128 bytes", M, amp);
    if ((boxel / epa) << t.nrest != (1ull << t.k)) return fail_at("copies do not add up to the tile", M, amp);
    for (int trial = 0; trial < 8; ++trial) {
        uint64_t tile = t.nout ? rng() & ((1ull << t.nout) - 1ull) : 0;
        uint64_t base = 0;
        for (uint32_t q = 0; q < t.nout; ++q)
            if ((tile >> q) & 1ull) base |= 1ull << t.outpos[q];
        const uint32_t r = t.nrest ? (uint32_t)(rng() % (1u << t.nrest)) : 0u;
        uint64_t g = base;
        for (uint32_t q = 0; q < t.nrest; ++q)
            if ((r >> q) & 1u) g |= 1ull << t.rest_pos[q];
        uint64_t c[5];
        for (int d = 0; d < 5; ++d) {
            const uint32_t w = t.tma_start[d + 1] - t.tma_start[d];
            const uint64_t v = w ? ((g >> t.tma_start[d]) & ((1ull << w) - 1ull)) : 0ull;
            c[d] = d == 0 ? v * epa : v;
            if (c[d] > 0x7fffffffull) return fail_at("coordinate overflow", M, amp);
            if (c[d] + t.tma_box[d] > t.tma_dim[d]) return fail_at("box outside the tensor", M, amp);
        }
        if ((c[0] * 8) % 16) return fail_at("x not on a 16-byte boundary", M, amp);
        if (((uint64_t)r * t.box_bytes) % 128) return fail_at("shared-memory offset not 128-byte aligned", M, amp);
        for (int smp = 0; smp < 32; ++smp) {
            const uint64_t e = rng() % boxel;
            uint64_t rem = e, byte = 0;
            for (int d = 0; d < 5; ++d) {
                const uint64_t i = rem % t.tma_box[d];
                rem /= t.tma_box[d];
                byte += d == 0 ? (c[d] + i) * 8 : (c[d] + i) * t.tma_stride[d];
            }
            const uint64_t local = (uint64_t)r * (boxel / epa) + e / epa;
            if (byte / amp != global_of(t, base, local)) return fail_at("copy element at the wrong index", M, amp);
            ++*elems;
        }
    }
    return 0;
}

// Property 3 for one tile pass of a plan.
int check_steps(uint32_t M, size_t amp, const Plan &plan, size_t pi, const qsim_step *steps,
                std::mt19937_64 &rng, long *rows)
{
    const Pass &p = plan.passes[pi];
    const TilePass &t = p.tile;
    const uint64_t tmask = tile_mask_of(t);
    const uint64_t first = pi ? plan.pass_ends[pi - 1] : 0, last = plan.pass_ends[pi];
    if (last - first != t.nsteps) return fail_at("pass step count", M, amp);
    for (uint32_t q = 0; q < t.nsteps; ++q) {
        const TileStep &ts = plan.tile_steps[t.step_off + q];
        const qsim_step &s = steps[plan.order[first + q]];
        if (!((tmask >> s.target) & 1ull)) return fail_at("step target outside its tile", M, amp);
        if (__builtin_popcount(ts.tmask) != 1) return fail_at("local target mask", M, amp);
        if ((ts.pl & ~ts.cl) || (ts.po & ~ts.co) || (ts.co & tmask)) return fail_at("step encoding", M, amp);
    }
    const uint64_t all = M >= 64 ? ~0ull : ((1ull << M) - 1ull);
    for (int smp = 0; smp < 64; ++smp) {
        const uint64_t g = rng() & all;
        // reference: the circuit's steps of this pass, last to first, on the row
        uint64_t x = g;
        for (uint64_t k = last; k-- > first;) {
            const qsim_step &s = steps[plan.order[k]];
            if ((x & s.ctrl_mask) == s.ctrl_pol) x ^= 1ull << s.target;
        }
        // the kernel's way: tile base constant, local index permuted
        const uint64_t base = g & ~tmask;
        uint64_t j = local_of(t, g);
        for (int q = (int)t.nsteps - 1; q >= 0; --q) {
            const TileStep &ts = plan.tile_steps[t.step_off + q];
            if ((base & ts.co) != ts.po) continue;  // inactive on this tile
            if ((j & ts.cl) == ts.pl) j ^= ts.tmask;
        }
        if (global_of(t, base, j) != x) return fail_at("tile step encoding maps a row wrongly", M, amp);
        ++*rows;
    }
    return 0;
}

}  // namespace

int main()
{
    std::mt19937_64 rng(20260);
    long elems = 0, rows = 0, layouts = 0, passes = 0;
    // random geometries straight into the layout routine
    for (int trial = 0; trial < 20000; ++trial) {
        const uint32_t M = 6 + (uint32_t)(rng() % 29);  // 6..34
        const size_t amp = (rng() & 1) ? 16 : 8;
        uint32_t l = 1 + (uint32_t)(rng() % 8);
        if (l > M) l = M;
        uint32_t nh = (uint32_t)(rng() % 11);
        if (l + nh > M) nh = M - l;
        if (l + nh > 14) nh = 14 - l;
        uint64_t hm = 0;
        for (uint32_t cnt = 0; cnt < nh;) {
            const uint32_t b = l + (uint32_t)(rng() % (M - l));
            if (!((hm >> b) & 1ull)) {
                hm |= 1ull << b;
                ++cnt;
            }
        }
        TilePass t{};
        layout_tile(M, l, hm, amp, &t);
        // tile-id bits as the planner would order them (any order will do here)
        t.nout = 0;
        for (uint32_t b = 0; b < M; ++b)
            if (!((tile_mask_of(t) >> b) & 1ull)) t.outpos[t.nout++] = b;
        if (check_layout(M, amp, t, rng, &elems)) return 1;
        layouts += t.tma ? 1 : 0;
    }
    // plans of random circuits (in place: tile passes and sweeps)
    for (int trial = 0; trial < 400; ++trial) {
        const uint32_t M = 6 + (uint32_t)(rng() % 29);
        const size_t amp = (rng() & 1) ? 16 : 8;
        const size_t L = 1 + rng() % 300;
        std::vector<qsim_step> st(L);
        for (auto &s : st) {
            s.target = (uint32_t)(rng() % M);
            s.reserved = 0;
            const int nc = (int)(rng() % std::min<uint32_t>(4, M));
            uint64_t cm = 0;
            for (int c = 0; c < nc;) {
                const uint32_t b = (uint32_t)(rng() % M);
                if (b != s.target && !((cm >> b) & 1ull)) {
                    cm |= 1ull << b;
                    ++c;
                }
            }
            s.ctrl_mask = cm;
            s.ctrl_pol = cm & rng();
        }
        PlanOptions o;
        o.amp_bytes = amp;
        o.strategy = (trial & 1) ? QSIM_STRATEGY_TILE : QSIM_STRATEGY_INPLACE;
        if (trial % 3 == 0) {
            o.tile_bits = 6 + (int)(rng() % 9);
            o.low_bits = 1 + (int)(rng() % 6);
        }
        Plan plan;
        std::string msg;
        if (make_plan(M, st.data(), L, o, &plan, &msg) != QSIM_OK) {
            std::printf("violation: plan rejected a valid circuit: %s\n", msg.c_str());
            return 1;
        }
        for (size_t pi = 0; pi < plan.passes.size(); ++pi) {
            if (plan.passes[pi].kind != kTile) continue;
            if (check_layout(M, amp, plan.passes[pi].tile, rng, &elems)) return 1;
            if (check_steps(M, amp, plan, pi, st.data(), rng, &rows)) return 1;
            ++passes;
        }
    }
    std::printf("ok: %ld copy elements, %ld tensor-map layouts, %ld tile passes, %ld rows\n", elems,
                layouts, passes, rows);
    return 0;
}
