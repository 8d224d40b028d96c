// Host check of the gather and sweep planning (built and run by
// tests/test_native_checks.py, no GPU).  It includes the planner's source and,
// for the plans of random circuits, evaluates every pass's encoding on
// sampled rows the way its kernel does, against the circuit's own steps:
//   - affine passes: x(i) = b ^ XOR over index bytes of the per-byte tables;
//   - coset tiles of affine passes: every (tile, run, offset) names an output
//     row once (all rows are covered for M <= 16), the row's source is where
//     the coset kernel reads it (source run base, run, offset), and every run
//     is aligned;
//   - bit-sliced passes: the step descriptors (target, control planes, the
//     all-ones plane for absent controls, negated controls, fast/slow path)
//     applied last to first to a single row;
//   - compiled passes: the kept step list is the pass's steps in order;
//   - sweeps: pair bases enumerated by inserting zero bits into a counter
//     are exactly the rows the step toggles, each once.
// Prints "ok ..." and exits 0, or prints the first violation and exits 1.
#include <cstdio>
#include <random>
#include <vector>

#include "../../paper_quant_ph_0308158_gb300/csrc/planner.cpp"

using namespace qsim;

namespace {

int fail(const char *what, uint32_t M)
{
    std::printf("violation: %s (M=%u)\n", what, M);
    return 1;
}

// The pass's steps applied to a row last to first (the gather's inverse map).
uint64_t source_row(const qsim_step *steps, const Plan &plan, uint64_t first, uint64_t last, uint64_t i)
{
    for (uint64_t k = last; k-- > first;) {
        const qsim_step &s = steps[plan.order[k]];
        if ((i & s.ctrl_mask) == s.ctrl_pol) i ^= 1ull << s.target;
    }
    return i;
}

// One bit-sliced descriptor applied to one row (bit b of row = plane b;
// plane M is all ones).
uint64_t sliced_apply(const SlicedStep &d, uint32_t M, uint64_t row)
{
    auto plane = [&](uint32_t p) -> uint64_t { return p == M ? 1ull : ((row >> p) & 1ull); };
    const uint32_t t = d.x & 0xffu;
    uint64_t m;
    if (!(d.x >> 24)) {
        m = plane(d.y & 0xffu) & plane((d.y >> 8) & 0xffu);
    } else {
        const uint32_t nc = (d.x >> 8) & 0xffu, neg = (d.x >> 16) & 0xffu;
        m = 1;
        for (uint32_t c = 0; c < nc; ++c) {
            const uint32_t cp = ((c < 4 ? d.y : d.z) >> (8 * (c & 3))) & 0xffu;
            const uint64_t v = plane(cp);
            m &= ((neg >> c) & 1u) ? (v ^ 1ull) : v;
        }
    }
    return row ^ (m << t);
}

// Where the coset kernel writes local output j of tile t and where it reads
// its source, from the pass's tables alone.
struct CosetRow {
    uint64_t out, src;
};
CosetRow coset_row(const Plan &plan, const GatherPass &g, uint64_t t, uint32_t j)
{
    const uint64_t *tab = plan.gather_tables.data() + g.coset_off;
    const uint64_t low = (1ull << g.cr) - 1ull;
    uint64_t ob = 0, sb = g.bvec;
    for (uint32_t k = 0; k < g.ctb; ++k) {
        ob ^= tab[256 * k + ((t >> (8 * k)) & 255u)];
        sb ^= tab[256 * g.ctb + 256 * k + ((t >> (8 * k)) & 255u)];
    }
    const uint64_t *dstrun = tab + 512 * g.ctb;
    const uint64_t *srcrun = dstrun + (1u << g.cd);
    const uint64_t *perm = srcrun + (1u << g.cd);
    const uint32_t loc = (uint32_t)((perm[j / 4] >> (16 * (j % 4))) & 0xffffu);
    CosetRow r;
    r.out = (ob ^ dstrun[j >> g.cr]) | (j & low);
    r.src = ((sb & ~low) ^ srcrun[loc >> g.cr]) | ((loc & low) ^ (sb & low));
    return r;
}

uint64_t insert_zero(uint64_t x, uint32_t pos)
{
    const uint64_t lo = x & ((1ull << pos) - 1ull);
    return ((x >> pos) << (pos + 1)) | lo;
}

}  // namespace

int main()
{
    std::mt19937_64 rng(7741);
    long rows = 0, affine = 0, sliced = 0, compiled = 0, sweeps = 0, cosets = 0;
    for (int trial = 0; trial < 1500; ++trial) {
        const uint32_t M = 2 + (uint32_t)(rng() % 33);  // 2..34
        const size_t L = 1 + rng() % 600;
        const int kind = trial % 3;  // 0: CNOT/NOT only, 1: up to 8 controls, 2: up to 11
        std::vector<qsim_step> st(L);
        for (auto &s : st) {
            s.target = (uint32_t)(rng() % M);
            s.reserved = 0;
            const uint32_t maxc = std::min<uint32_t>(kind == 0 ? 1 : (kind == 1 ? 8 : 11), M - 1);
            const int nc = (int)(rng() % (maxc + 1));
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
        o.amp_bytes = (rng() & 1) ? 16 : 8;
        o.strategy = QSIM_STRATEGY_GATHER;
        o.scratch_available = true;
        o.cancel_adjacent = (trial & 4) != 0;
        o.jit = (trial & 8) != 0;
        o.coset_run_bits = (int)(rng() % 8);  // 0: default
        Plan plan;
        std::string msg;
        if (make_plan(M, st.data(), L, o, &plan, &msg) != QSIM_OK) {
            std::printf("violation: plan rejected a valid circuit: %s\n", msg.c_str());
            return 1;
        }
        if (plan.order.size() + plan.cancelled != L) return fail("steps lost by the plan", M);
        const uint64_t all = M >= 64 ? ~0ull : ((1ull << M) - 1ull);
        for (size_t pi = 0; pi < plan.passes.size(); ++pi) {
            const Pass &p = plan.passes[pi];
            const uint64_t first = pi ? plan.pass_ends[pi - 1] : 0, last = plan.pass_ends[pi];
            if (p.kind == kSweep) {
                if (last - first != 1) return fail("sweep with more than one step", M);
                const qsim_step &s = st[plan.order[first]];
                const SweepParams &w = p.sweep;
                if (w.n_pairs != (1ull << (M - 1 - __builtin_popcountll(s.ctrl_mask))))
                    return fail("sweep pair count", M);
                for (int smp = 0; smp < 64; ++smp) {
                    const uint64_t q = rng() % w.n_pairs;
                    uint64_t j = q;
                    for (uint32_t k = 0; k < w.nins; ++k) j = insert_zero(j, w.ins[k]);
                    j |= w.pol;
                    if ((j & s.ctrl_mask) != s.ctrl_pol || (j & w.half) || j > all)
                        return fail("sweep pair base is not a toggled row", M);
                    // distinct counters give distinct bases: the counter comes back
                    // from the free bits of the base
                    uint64_t back = 0, nb = 0;
                    for (uint32_t b = 0; b < M; ++b) {
                        if (((s.ctrl_mask | w.half) >> b) & 1ull) continue;
                        back |= ((j >> b) & 1ull) << nb++;
                    }
                    if (back != q) return fail("sweep pair enumeration is not one to one", M);
                    ++rows;
                }
                ++sweeps;
                continue;
            }
            if (p.kind != kGather) return fail("non-gather pass in a gather plan", M);
            const GatherPass &g = p.gather;
            if (g.jit) {
                if (g.jit_n != last - first) return fail("compiled pass step count", M);
                for (uint64_t k = 0; k < g.jit_n; ++k) {
                    const qsim_step &a = plan.jit_steps[g.jit_off + k], &b = st[plan.order[first + k]];
                    if (a.target != b.target || a.ctrl_mask != b.ctrl_mask || a.ctrl_pol != b.ctrl_pol)
                        return fail("compiled pass keeps different steps", M);
                }
                ++compiled;
                continue;
            }
            for (int smp = 0; smp < 64; ++smp) {
                const uint64_t i = rng() & all;
                const uint64_t want = source_row(st.data(), plan, first, last, i);
                uint64_t got;
                if (g.affine) {
                    got = g.bvec;
                    for (uint32_t b = 0; b < g.nbytes; ++b)
                        got ^= plan.gather_tables[g.table_off + 256 * b + ((i >> (8 * b)) & 255u)];
                } else {
                    if (g.nsteps != last - first) return fail("bit-sliced pass step count", M);
                    got = i;
                    for (uint32_t q = g.nsteps; q-- > 0;)
                        got = sliced_apply(plan.sliced_steps[g.step_off + q], M, got);
                }
                if (got != want) return fail(g.affine ? "affine tables map a row wrongly"
                                                      : "bit-sliced descriptors map a row wrongly", M);
                ++rows;
            }
            if (g.affine && g.coset) {
                const uint64_t low = (1ull << g.cr) - 1ull;
                if (((uint64_t)o.amp_bytes << (g.cr + g.cd)) > 64 * 1024) return fail("coset tile above 64 KiB", M);
                if (g.cr + g.cd + __builtin_ctzll(g.n_tiles) != M) return fail("coset tile count", M);
                const uint32_t nloc = 1u << (g.cr + g.cd);
                const uint64_t *tab = plan.gather_tables.data() + g.coset_off;
                for (uint32_t b = 0; b < (2u << g.cd); ++b)
                    if (tab[512 * g.ctb + b] & low) return fail("coset run base not aligned", M);
                if (M <= 16) {  // the tiles cover every row exactly once
                    std::vector<char> seen(1ull << M, 0);
                    for (uint64_t t = 0; t < g.n_tiles; ++t)
                        for (uint32_t j = 0; j < nloc; ++j) {
                            const CosetRow cr = coset_row(plan, g, t, j);
                            if (cr.out > all || seen[cr.out]) return fail("coset tiles overlap", M);
                            seen[cr.out] = 1;
                            if (cr.src != source_row(st.data(), plan, first, last, cr.out))
                                return fail("coset tile reads the wrong source", M);
                        }
                } else {
                    for (int smp = 0; smp < 256; ++smp) {
                        const uint64_t t = rng() % g.n_tiles;
                        const uint32_t j = (uint32_t)(rng() % nloc);
                        const CosetRow cr = coset_row(plan, g, t, j);
                        if (cr.out > all || cr.src != source_row(st.data(), plan, first, last, cr.out))
                            return fail("coset tile reads the wrong source", M);
                    }
                }
                ++cosets;
            }
            if (g.affine) ++affine; else ++sliced;
        }
    }
    std::printf("ok: %ld affine (%ld coset-tiled), %ld bit-sliced, %ld compiled, %ld sweep passes; %ld rows\n",
                affine, cosets, sliced, compiled, sweeps, rows);
    if (cosets == 0) return fail("no coset-tiled pass was checked", 0);
    return 0;
}
