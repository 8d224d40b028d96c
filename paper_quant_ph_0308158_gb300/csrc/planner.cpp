// planner.cpp -- host side of the engine: step validation, canonicalisation,
// segmentation of the wiring diagram into passes, and the per-pass tables the
// kernels read.
//
// Passes (see qsim_internal.h):
//   * TILE passes apply runs of steps whose targets lie in one tile of k
//     address bits (the lowest l bits, which give contiguous runs of 2^l
//     amplitudes, plus up to k-l chosen higher bits).  Segments are grown
//     greedily in circuit order; a later step may join an earlier segment when
//     it commutes with every step it overtakes (Sec. 2i notes that steps can
//     be grouped; two steps commute when neither's target is a control of the
//     other, since each then leaves the other's control bits unchanged).
//   * SWEEP passes apply one step over its toggled pairs only (Sec. 2b).
//   * GATHER passes evaluate the inverse wiring diagram on every output index
//     (Sec. 2h product, then the gather k2(i) = k1(x(i))): as a GF(2) affine
//     map when the segment has only NOT/CNOT steps, otherwise step by step in
//     bit-sliced form.
#include <algorithm>
#include <cstring>
#include <string>

#include "qsim_internal.h"

namespace qsim {

namespace {

inline int popcount64(uint64_t x) { return __builtin_popcountll(x); }

inline uint64_t full_mask(uint32_t M) { return M >= 64 ? ~0ull : ((1ull << M) - 1ull); }

bool same_step(const qsim_step &a, const qsim_step &b)
{
    return a.target == b.target && a.ctrl_mask == b.ctrl_mask && a.ctrl_pol == b.ctrl_pol;
}

// splitmix64: deterministic sampling of tile ids for the touched-fraction estimate.
uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

int validate_steps(uint32_t M, const qsim_step *steps, size_t L, std::string *msg)
{
    if (M < 1 || M > QSIM_MAX_QUBITS) {
        if (msg) *msg = "M must be in [1, " + std::to_string(QSIM_MAX_QUBITS) + "]";
        return QSIM_EINVAL;
    }
    if (L > 0 && steps == nullptr) {
        if (msg) *msg = "steps is NULL";
        return QSIM_EINVAL;
    }
    const uint64_t all = full_mask(M);
    for (size_t i = 0; i < L; ++i) {
        const qsim_step &s = steps[i];
        const char *why = nullptr;
        if (s.target >= M)
            why = "target bit >= M";
        else if (s.reserved != 0)
            why = "reserved field is not zero";
        else if (s.ctrl_mask & ~all)
            why = "control bit >= M";
        else if ((s.ctrl_mask >> s.target) & 1ull)
            why = "target bit is also a control";
        else if (s.ctrl_pol & ~s.ctrl_mask)
            why = "polarity bit outside the control mask";
        if (why) {
            if (msg) *msg = "step " + std::to_string(i) + ": " + why;
            return QSIM_EINVAL;
        }
    }
    return QSIM_OK;
}

namespace {

// Adjacent equal steps cancel (each step matrix is its own inverse, Sec. 2a).
// A stack removes nested pairs too (A B B A -> nothing).
std::vector<uint64_t> canonical_order(const qsim_step *steps, size_t L, bool cancel,
                                      uint64_t *cancelled)
{
    std::vector<uint64_t> st;
    st.reserve(L);
    for (size_t i = 0; i < L; ++i) {
        if (cancel && !st.empty() && same_step(steps[st.back()], steps[i]))
            st.pop_back();
        else
            st.push_back(i);
    }
    *cancelled = L - st.size();
    return st;
}

double state_bytes(uint32_t M, size_t amp) { return (double)amp * (double)(1ull << M); }

Pass make_sweep(uint32_t M, const qsim_step &s, size_t amp)
{
    Pass p{};
    p.kind = kSweep;
    p.nsteps = 1;
    const int c = popcount64(s.ctrl_mask);
    p.sweep.n_pairs = 1ull << (M - 1 - c);
    p.sweep.pol = s.ctrl_pol;
    p.sweep.half = 1ull << s.target;
    uint64_t ins = s.ctrl_mask | (1ull << s.target);
    uint32_t n = 0;
    while (ins) {
        p.sweep.ins[n++] = (uint32_t)__builtin_ctzll(ins);
        ins &= ins - 1;
    }
    p.sweep.nins = n;
    p.alg_bytes = 2.0 * (double)amp * (double)(1ull << (M - c));
    return p;
}

struct TileGeom {
    uint32_t k, l, nh_max;
};

TileGeom tile_geometry(uint32_t M, const PlanOptions &o)
{
    TileGeom g;
    // 128 KiB tiles (one shared-memory stage: more target bits per pass beat
    // deeper pipelining) whose lowest l bits give runs of 256 bytes for
    // full-sector, coalesced stores; tiles move in tensor-map boxes, so short
    // runs do not multiply the number of copies
    const uint32_t kdef = o.amp_bytes == 16 ? 13 : 14;
    const uint32_t ldef = o.amp_bytes == 16 ? 4 : 5;
    uint32_t k = o.tile_bits > 0 ? (uint32_t)o.tile_bits : kdef;
    uint32_t l = o.low_bits > 0 ? (uint32_t)o.low_bits : ldef;
    k = std::min<uint32_t>(std::min<uint32_t>(k, kMaxTileBits), M);
    while (k > 1 && (o.amp_bytes << k) > kMaxTileBytes) --k;  // one tile fits shared memory
    l = std::min(l, k);
    if (o.amp_bytes == 8 && l < 1) l = 1;  // bulk copies move >= 16 bytes
    if (k < l) k = l;
    g.k = k;
    g.l = l;
    g.nh_max = std::min<uint32_t>(k - l, kMaxHighBits);
    g.k = g.l + g.nh_max;
    return g;
}

// Local bit order of a tile and its tensor-map copy layout.  The tile's bits
// are the lowest l address bits, extended upwards while the next bit is also
// a tile bit (one contiguous run, at most 256 copy elements), then up to four
// further runs of tile bits ("groups", at most 8 bits each, the largest
// first), then the remaining tile bits.  One tensor copy moves the run and the
// four groups as a box of a 5-dimensional view of the state (dimension d
// spans the address bits from the start of group d to the start of group
// d+1); the remaining bits are enumerated by issuing one copy per value.  The
// local index of an amplitude in shared memory lists the bits in that order.
void layout_tile(uint32_t M, uint32_t l, uint64_t high_mask, size_t amp, TilePass *t)
{
    const uint32_t epa = amp == 16 ? 2 : 1;          // 8-byte copy elements per amplitude
    const uint32_t lmax = amp == 16 ? 7 : 8;         // box dimension 0 <= 256 elements
    uint32_t a0 = l;
    while (a0 < lmax && a0 < M && ((high_mask >> a0) & 1ull)) ++a0;
    uint64_t rest = high_mask & ~((1ull << a0) - 1ull);
    // runs of consecutive tile bits above the low run, split at 8 bits
    struct Grp { uint32_t start, width; };
    std::vector<Grp> runs;
    for (uint64_t h = rest; h;) {
        const uint32_t b = (uint32_t)__builtin_ctzll(h);
        uint32_t w = 0;
        while (w < 8 && ((h >> (b + w)) & 1ull)) ++w;
        runs.push_back({b, w});
        h &= ~(((1ull << w) - 1ull) << b);
    }
    std::vector<Grp> chosen = runs;
    std::stable_sort(chosen.begin(), chosen.end(),
                     [](const Grp &x, const Grp &y) { return x.width > y.width; });
    if (chosen.size() > 4) chosen.resize(4);
    std::sort(chosen.begin(), chosen.end(), [](const Grp &x, const Grp &y) { return x.start < y.start; });
    uint64_t chosen_mask = 0;
    for (const Grp &c : chosen) chosen_mask |= ((1ull << c.width) - 1ull) << c.start;
    t->l = a0;
    t->nh = 0;
    for (const Grp &c : chosen)
        for (uint32_t q = 0; q < c.width; ++q) t->high[t->nh++] = c.start + q;
    t->nrest = 0;
    for (uint64_t h = rest & ~chosen_mask; h; h &= h - 1) {
        const uint32_t b = (uint32_t)__builtin_ctzll(h);
        t->rest_pos[t->nrest++] = b;
        t->high[t->nh++] = b;
    }
    t->k = t->l + t->nh;
    // tensor-map view: ranges [start[d], start[d+1]) of address bits; a
    // range wider than 30 bits is split by a dimension with box extent 1
    // (coordinates are 32-bit signed)
    std::vector<Grp> dimgrp;  // per dimension >= 1: group start and box width
    for (const Grp &c : chosen) dimgrp.push_back(c);
    for (;;) {
        uint32_t st[6];
        uint32_t nd = 0;
        st[nd++] = 0;
        for (const Grp &c : dimgrp) st[nd++] = c.start;
        st[nd] = M;
        int wide = -1;
        for (uint32_t d = 0; d < nd; ++d)
            if (st[d + 1] - st[d] + (d == 0 && epa == 2 ? 1 : 0) > 30) wide = (int)d;
        if (wide < 0 || nd >= 5) break;
        const uint32_t at = st[wide] + 28;  // the new range starts 28 bits in
        dimgrp.insert(dimgrp.begin() + wide, Grp{at, 0});
        std::sort(dimgrp.begin(), dimgrp.end(), [](const Grp &x, const Grp &y) { return x.start < y.start; });
    }
    uint32_t start[6];
    uint32_t nd = 0;
    start[nd++] = 0;
    for (const Grp &c : dimgrp) start[nd++] = c.start;
    const uint32_t ndims = nd;
    start[nd] = M;
    bool fits = true;
    for (uint32_t d = 0; d < ndims; ++d) {
        const uint32_t width = start[d + 1] - start[d] + (d == 0 && epa == 2 ? 1 : 0);
        if (width > 30) fits = false;
    }
    t->tma = fits ? 1u : 0u;
    const uint64_t total_bytes = (uint64_t)amp << M;
    for (uint32_t d = 0; d < 5; ++d) {
        if (d < ndims) {
            t->tma_start[d] = start[d];
            t->tma_dim[d] = (1ull << (start[d + 1] - start[d])) * (d == 0 ? epa : 1);
            t->tma_stride[d] = d == 0 ? amp : (uint64_t)amp << start[d];
            t->tma_box[d] = d == 0 ? (epa << a0) : (1u << dimgrp[d - 1].width);
        } else {  // unused dimensions: extent 1
            t->tma_start[d] = M;
            t->tma_dim[d] = 1;
            t->tma_stride[d] = total_bytes;
            t->tma_box[d] = 1;
        }
    }
    t->tma_start[5] = M;
    t->tma_ndims = ndims;
    t->box_bytes = (uint32_t)(amp << (t->k - t->nrest));
    // Copy-engine rules, checked here so that no copy can break them: every
    // box lands on a 128-byte boundary of shared memory (stage buffers are
    // whole tiles), box extents are at most 256 elements, the first
    // coordinate is a multiple of 16 bytes (the low a0 >= 1 bits of a box
    // origin are zero), and each box lies inside its dimension.
    const uint64_t tile_bytes = (uint64_t)amp << t->k;
    bool ok = t->tma && t->box_bytes % 128 == 0 && tile_bytes % 128 == 0 && a0 >= 1;
    for (uint32_t d = 0; d < 5 && ok; ++d) {
        ok = t->tma_box[d] >= 1 && t->tma_box[d] <= 256 && t->tma_box[d] <= t->tma_dim[d] &&
             t->tma_dim[d] % t->tma_box[d] == 0 && t->tma_stride[d] % (d == 0 ? 8 : 16) == 0;
    }
    if (ok && ((uint64_t)t->tma_box[0] * 8) % 16 != 0) ok = false;
    t->tma = ok ? 1u : 0u;
}

// Build one tile pass for the given step indices and high-bit set.
void emit_tile(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &seg,
               uint64_t high_mask, const TileGeom &g, const PlanOptions &o, Plan *plan)
{
    Pass p{};
    p.kind = kTile;
    TilePass &t = p.tile;
    // pad the high set with unused bits so the tile always has k bits when M allows
    uint32_t want = std::min<uint32_t>(g.nh_max, M - g.l);
    for (uint32_t b = g.l; b < M && (uint32_t)popcount64(high_mask) < want; ++b)
        high_mask |= 1ull << b;
    layout_tile(M, g.l, high_mask, o.amp_bytes, &t);
    int8_t g2l[64];
    for (int b = 0; b < 64; ++b) g2l[b] = -1;
    for (uint32_t b = 0; b < t.l; ++b) g2l[b] = (int8_t)b;
    for (uint32_t q = 0; q < t.nh; ++q) g2l[t.high[q]] = (int8_t)(t.l + q);
    t.n_tiles = 1ull << (M - t.k);
    t.step_off = (uint32_t)plan->tile_steps.size();
    t.nsteps = (uint32_t)seg.size();
    const uint64_t tile_mask = ((1ull << g.l) - 1ull) | high_mask;
    bool all_local = true;
    for (uint64_t idx : seg) {
        const qsim_step &s = steps[idx];
        TileStep ts{};
        for (uint64_t c = s.ctrl_mask & tile_mask; c; c &= c - 1) {
            const uint32_t b = (uint32_t)__builtin_ctzll(c);
            ts.cl |= 1u << g2l[b];
            if ((s.ctrl_pol >> b) & 1ull) ts.pl |= 1u << g2l[b];
        }
        ts.tmask = 1u << g2l[s.target];
        ts.co = s.ctrl_mask & ~tile_mask;
        ts.po = s.ctrl_pol & ~tile_mask;
        if (ts.co) all_local = false;
        plan->tile_steps.push_back(ts);
    }
    t.all_local = all_local ? 1u : 0u;
    bool affine = true;
    for (uint64_t idx : seg) affine = affine && popcount64(steps[idx].ctrl_mask) <= 1;
    t.affine = affine ? 1u : 0u;
    // tile-id bit order: out-of-tile bits that no step controls vary fastest,
    // control bits slowest (runs of tiles with the same active steps)
    uint64_t ctl_out = 0;
    for (uint32_t j = 0; j < t.nsteps; ++j) ctl_out |= plan->tile_steps[t.step_off + j].co;
    t.nout = 0;
    for (int pass2 = 0; pass2 < 2; ++pass2)
        for (uint32_t b = 0; b < M; ++b) {
            if ((tile_mask >> b) & 1ull) continue;
            const bool is_ctl = (ctl_out >> b) & 1ull;
            if (is_ctl == (pass2 == 1)) t.outpos[t.nout++] = b;
        }
    // fraction of tiles that have at least one active step
    double touched = 1.0;
    if (!all_local) {
        const int samples = 512;
        int hit = 0;
        uint64_t seed = 0x5eed0000ull + plan->passes.size();
        for (int i = 0; i < samples; ++i) {
            const uint64_t tile = splitmix64(seed) & (t.n_tiles - 1);
            uint64_t base = 0;
            for (uint32_t q = 0; q < t.nout; ++q)
                if ((tile >> q) & 1ull) base |= 1ull << t.outpos[q];
            for (uint32_t j = 0; j < t.nsteps; ++j) {
                const TileStep &ts = plan->tile_steps[t.step_off + j];
                if ((base & ts.co) == ts.po) {
                    ++hit;
                    break;
                }
            }
        }
        touched = (double)hit / samples;
    }
    t.touched = touched;
    // Tiles are dealt in tile-id order with the out-of-tile control bits
    // slowest, so the active set changes at most once per value of those
    // bits (and per CTA range); an affine pass reuses one table throughout.
    {
        const int nctl = popcount64(ctl_out);
        const double changes = nctl >= 40 ? 1e12 : (double)(1ull << nctl);
        t.rebuilds = t.affine ? 152.0 : std::min((double)t.n_tiles * touched, changes) + 152.0;
    }
    p.nsteps = t.nsteps;
    p.alg_bytes = 2.0 * state_bytes(M, o.amp_bytes) * touched;
    plan->passes.push_back(p);
}

// Greedy, commutation-aware tile segmentation of 'order' (circuit indices).
void plan_tiles(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &order,
                const PlanOptions &o, bool sweep_singles, Plan *plan)
{
    const TileGeom g = tile_geometry(M, o);
    const uint64_t low_mask = (1ull << g.l) - 1ull;
    const size_t n = order.size();
    std::vector<char> done(n, 0);
    size_t first = 0;
    while (first < n) {
        std::vector<uint64_t> seg;
        std::vector<size_t> seg_pos;
        uint64_t high = 0;
        uint64_t def_targets = 0, def_controls = 0;  // unions over overtaken steps
        int scanned = 0, deferred = 0;
        for (size_t j = first; j < n && scanned < o.lookahead; ++j) {
            if (done[j]) continue;
            ++scanned;
            const qsim_step &s = steps[order[j]];
            const uint64_t tb = 1ull << s.target;
            const bool commutes = !(def_controls & tb) && !(def_targets & s.ctrl_mask);
            bool take = false;
            if (commutes) {
                if ((tb & low_mask) || (tb & high)) {
                    take = true;
                } else if ((uint32_t)popcount64(high) < g.nh_max) {
                    high |= tb;
                    take = true;
                }
            }
            if (take) {
                seg.push_back(order[j]);
                seg_pos.push_back(j);
                if ((int)seg.size() >= kMaxTileSteps) break;
            } else {
                def_targets |= tb;
                def_controls |= s.ctrl_mask;
                if (++deferred > 96 || (def_targets | def_controls) == full_mask(M)) break;
            }
        }
        if (seg.empty()) {
            // the first pending step fits no tile (a geometry with no free
            // high bit and a target above the low bits): it becomes a sweep
            seg.push_back(order[first]);
            seg_pos.push_back(first);
            done[first] = 1;
            plan->passes.push_back(make_sweep(M, steps[order[first]], o.amp_bytes));
            plan->order.push_back(order[first]);
            plan->pass_ends.push_back(plan->order.size());
            while (first < n && done[first]) ++first;
            continue;
        }
        for (size_t j : seg_pos) done[j] = 1;
        if (seg.size() == 1 && sweep_singles) {
            plan->passes.push_back(make_sweep(M, steps[seg[0]], o.amp_bytes));
        } else {
            emit_tile(M, steps, seg, high, g, o, plan);
        }
        for (uint64_t idx : seg) plan->order.push_back(idx);
        plan->pass_ends.push_back(plan->order.size());
        while (first < n && done[first]) ++first;
    }
}

bool is_affine_step(const qsim_step &s) { return popcount64(s.ctrl_mask) <= 1; }

// Vectors over GF(2) (bit b = coordinate b) in reduced echelon form: every
// kept vector has a pivot (its highest set bit) that no other kept vector has.
struct Echelon {
    uint64_t v[64];
    bool has[64] = {false};
    int rank = 0;
    // Insert x; returns false when x is already in the span.
    bool add(uint64_t x)
    {
        for (int b = 63; b >= 0; --b)
            if (has[b] && ((x >> b) & 1ull)) x ^= v[b];
        if (!x) return false;
        const int p = 63 - __builtin_clzll(x);
        for (int b = 0; b < 64; ++b)
            if (has[b] && ((v[b] >> p) & 1ull)) v[b] ^= x;
        v[p] = x;
        has[p] = true;
        ++rank;
        return true;
    }
};

uint64_t apply_cols(const uint64_t *col, uint64_t i)
{
    uint64_t x = 0;
    for (; i; i &= i - 1) x ^= col[__builtin_ctzll(i)];
    return x;
}

// Coset tiles of the affine map x(i) = A i ^ b, A given by its columns
// col[j] = A e_j (invertible).  Returns false if A is singular (never for a
// product of NOT/CNOT steps).
//
// S = span(e_0..e_{r-1}) + A^-1 span(e_0..e_{r-1}) has a basis of the r low
// unit vectors and d vectors w_k without low bits, in reduced echelon form
// with pivots p_k; the other high bits ("complement" bits) number a tile.
// Output i = T(t) ^ dstrun[beta] ^ l (l < 2^r) for tile t, where T deposits
// t into the complement bits: a bijection, and each (t, beta) is an aligned
// run of 2^r outputs.  A S contains the low source bits, so its high parts
// have a basis u_k (pivots q_k) of the same size d, and the sources of tile t
// are the aligned runs (A T(t) ^ b) & ~low ^ srcrun[gamma].  The source of
// local output (beta, l) is y = A(dstrun[beta] ^ l): run gamma (bits q_k of
// y), offset (y ^ A T(t) ^ b) & low.
bool emit_coset_r(uint32_t M, const uint64_t *col, uint32_t r, const PlanOptions &o, GatherPass *gp,
                  Plan *plan);

// Largest run length r (at most the requested one) whose tiles of 2^(r+d)
// amplitudes stay within 64 KiB, so that the pipeline holds two stages.
bool emit_coset(uint32_t M, const uint64_t *col, uint64_t bvec, const PlanOptions &o, GatherPass *gp,
                Plan *plan)
{
    (void)bvec;
    const uint32_t amp = (uint32_t)o.amp_bytes;
    uint32_t r = o.coset_run_bits > 0 ? (uint32_t)o.coset_run_bits : (amp == 16 ? 6u : 7u);  // 1 KiB runs
    r = std::min(std::min(r, 7u), M);  // local indices (r + d <= 14 bits) fit 16 bits
    const size_t keep = plan->gather_tables.size();
    for (; r >= 1; --r) {
        if (!emit_coset_r(M, col, r, o, gp, plan)) return false;
        if (((uint64_t)amp << (gp->cr + gp->cd)) <= 64 * 1024) return true;
        plan->gather_tables.resize(keep);
    }
    return false;
}

bool emit_coset_r(uint32_t M, const uint64_t *col, uint32_t r, const PlanOptions &o, GatherPass *gp,
                  Plan *plan)
{
    const uint32_t amp = (uint32_t)o.amp_bytes;
    if (amp == 8 && r < 1) return false;  // bulk copies move >= 16 bytes
    const uint64_t low = (1ull << r) - 1ull;
    // A^-1 by elimination on the columns, remembering which columns combine
    uint64_t piv_v[64], piv_c[64];
    bool has[64] = {false};
    for (uint32_t j = 0; j < M; ++j) {
        uint64_t v = col[j], c = 1ull << j;
        for (int b = (int)M - 1; b >= 0 && v; --b) {
            if (!((v >> b) & 1ull)) continue;
            if (has[b]) {
                v ^= piv_v[b];
                c ^= piv_c[b];
            } else {
                piv_v[b] = v;
                piv_c[b] = c;
                has[b] = true;
                v = 0;
                c = 0;
                break;
            }
        }
        if (v || c) return false;  // a dependent column
    }
    auto solve = [&](uint64_t target) {  // w with A w = target
        uint64_t w = 0;
        for (int b = (int)M - 1; b >= 0; --b)
            if ((target >> b) & 1ull) {
                target ^= piv_v[b];
                w ^= piv_c[b];
            }
        return w;
    };
    Echelon W;
    for (uint32_t j = 0; j < r; ++j) W.add(solve(1ull << j) & ~low);
    const uint32_t d = (uint32_t)W.rank;
    std::vector<uint64_t> wv, pos;  // w_k by ascending pivot; complement bits
    for (uint32_t b = r; b < M; ++b) {
        if (W.has[b]) wv.push_back(W.v[b]);
        else pos.push_back(b);
    }
    Echelon U;
    for (uint32_t j = 0; j < r; ++j) U.add(col[j] & ~low);
    for (uint64_t w : wv) U.add(apply_cols(col, w) & ~low);
    if ((uint32_t)U.rank != d) return false;
    std::vector<uint64_t> uv;
    std::vector<uint32_t> q;
    for (uint32_t b = r; b < M; ++b)
        if (U.has[b]) {
            uv.push_back(U.v[b]);
            q.push_back(b);
        }
    gp->coset = 1;
    gp->cr = r;
    gp->cd = d;
    const uint32_t nc = (uint32_t)pos.size();  // M - r - d
    gp->n_tiles = 1ull << nc;
    gp->ctb = (nc + 7) / 8;
    // tiles per pipeline stage: stages of at least stage_kib KiB (default
    // 32), at most 64 tiles
    const uint64_t stage = (uint64_t)(o.coset_stage_kib > 0 ? o.coset_stage_kib : 32) * 1024;
    uint32_t e = 0;
    while (e < nc && e < 6 && ((uint64_t)amp << (r + d + e)) < stage && ((uint64_t)amp << (r + d + e + 1)) <= 96 * 1024)
        ++e;
    gp->ce = e;
    gp->coset_off = (uint32_t)plan->gather_tables.size();
    std::vector<uint64_t> &tab = plan->gather_tables;
    for (uint32_t k = 0; k < gp->ctb; ++k)  // out bases
        for (uint32_t v = 0; v < 256; ++v) {
            uint64_t t = 0;
            for (uint32_t j = 0; j < 8; ++j)
                if (((v >> j) & 1u) && 8 * k + j < nc) t |= 1ull << pos[8 * k + j];
            tab.push_back(t);
        }
    for (uint32_t k = 0; k < gp->ctb; ++k)  // source bases (without b)
        for (uint32_t v = 0; v < 256; ++v) tab.push_back(apply_cols(col, tab[gp->coset_off + 256 * k + v]));
    for (uint32_t beta = 0; beta < (1u << d); ++beta) {
        uint64_t x = 0;
        for (uint32_t k = 0; k < d; ++k)
            if ((beta >> k) & 1u) x ^= wv[k];
        tab.push_back(x);
    }
    const size_t src_off = tab.size();
    for (uint32_t g = 0; g < (1u << d); ++g) {
        uint64_t x = 0;
        for (uint32_t k = 0; k < d; ++k)
            if ((g >> k) & 1u) x ^= uv[k];
        tab.push_back(x);
    }
    const uint32_t nloc = 1u << (r + d);
    const size_t perm_off = tab.size();
    tab.resize(perm_off + (nloc + 3) / 4, 0);
    for (uint32_t j = 0; j < nloc; ++j) {
        const uint64_t beta = j >> r, l = j & low;
        const uint64_t y = apply_cols(col, tab[gp->coset_off + 2 * 256 * gp->ctb + beta] ^ l);
        uint32_t g = 0;
        for (uint32_t k = 0; k < d; ++k) g |= (uint32_t)((y >> q[k]) & 1ull) << k;
        if ((y & ~low) != tab[src_off + g]) return false;  // not in A S: cannot happen
        const uint64_t loc = ((uint64_t)g << r) | (y & low);
        tab[perm_off + j / 4] |= loc << (16 * (j % 4));
    }
    return true;
}

// GF(2) affine map x(i) = A i ^ b of the inverse of a NOT/CNOT segment:
// x = g_1(g_2(... g_n(i))), built by composing each step onto the outputs of
// the map so far, last step first.  Stored as per-byte XOR tables.
void emit_affine(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &seg,
                 const PlanOptions &o, Plan *plan)
{
    uint64_t row[64];  // row[t]: input bits that XOR into output bit t
    uint64_t bvec = 0;
    for (uint32_t t = 0; t < M; ++t) row[t] = 1ull << t;
    for (size_t q = seg.size(); q-- > 0;) {
        const qsim_step &s = steps[seg[q]];
        const uint32_t t = s.target;
        if (s.ctrl_mask == 0) {
            bvec ^= 1ull << t;
        } else {
            const uint32_t c = (uint32_t)__builtin_ctzll(s.ctrl_mask);
            row[t] ^= row[c];
            const uint64_t bc = (bvec >> c) & 1ull;
            const uint64_t flip = bc ^ (((s.ctrl_pol >> c) & 1ull) ? 0ull : 1ull);
            bvec ^= flip << t;
        }
    }
    uint64_t col[64];
    for (uint32_t j = 0; j < M; ++j) {
        uint64_t c = 0;
        for (uint32_t t = 0; t < M; ++t) c |= ((row[t] >> j) & 1ull) << t;
        col[j] = c;
    }
    Pass p{};
    p.kind = kGather;
    GatherPass &gp = p.gather;
    gp.affine = 1;
    gp.nbytes = (M + 7) / 8;
    gp.table_off = (uint32_t)plan->gather_tables.size();
    gp.bvec = bvec;
    for (uint32_t b = 0; b < gp.nbytes; ++b) {
        for (uint32_t v = 0; v < 256; ++v) {
            uint64_t x = 0;
            for (uint32_t j = 0; j < 8; ++j)
                if (((v >> j) & 1u) && 8 * b + j < M) x ^= col[8 * b + j];
            plan->gather_tables.push_back(x);
        }
    }
    p.nsteps = (uint32_t)seg.size();
    p.alg_bytes = 2.0 * state_bytes(M, o.amp_bytes);
    if (o.coset) {
        const size_t keep = plan->gather_tables.size();
        if (!emit_coset(M, col, bvec, o, &gp, plan)) {
            plan->gather_tables.resize(keep);
            gp.coset = 0;
        }
    }
    plan->passes.push_back(p);
}

void emit_sliced(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &seg,
                 const PlanOptions &o, Plan *plan)
{
    Pass p{};
    p.kind = kGather;
    GatherPass &gp = p.gather;
    gp.affine = 0;
    gp.step_off = (uint32_t)plan->sliced_steps.size();
    gp.nsteps = (uint32_t)seg.size();
    for (size_t q = 0; q < seg.size(); ++q) {
        const qsim_step &s = steps[seg[q]];
        SlicedStep h{};
        uint32_t cp[kSlicedMaxControls];
        for (int c = 0; c < kSlicedMaxControls; ++c) cp[c] = M;  // the all-ones plane
        uint32_t nc = 0, neg = 0;
        for (uint64_t m = s.ctrl_mask; m; m &= m - 1) {
            const uint32_t b = (uint32_t)__builtin_ctzll(m);
            if (!((s.ctrl_pol >> b) & 1ull)) neg |= 1u << nc;
            cp[nc++] = b;
        }
        const uint32_t slow = (nc > 2 || neg) ? 1u : 0u;
        h.x = s.target | (nc << 8) | (neg << 16) | (slow << 24);
        h.y = cp[0] | (cp[1] << 8) | (cp[2] << 16) | (cp[3] << 24);
        h.z = cp[4] | (cp[5] << 8) | (cp[6] << 16) | (cp[7] << 24);
        plan->sliced_steps.push_back(h);
    }
    p.nsteps = (uint32_t)seg.size();
    p.alg_bytes = 2.0 * state_bytes(M, o.amp_bytes);
    plan->passes.push_back(p);
}

// A gather segment compiled into its own kernel (jit.cu): the plan keeps the
// steps in circuit order; the kernel applies them last to first.
void emit_compiled(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &seg,
                   const PlanOptions &o, Plan *plan)
{
    Pass p{};
    p.kind = kGather;
    GatherPass &gp = p.gather;
    gp.jit = 1;
    gp.jit_off = (uint32_t)plan->jit_steps.size();
    gp.jit_n = (uint32_t)seg.size();
    for (uint64_t idx : seg) plan->jit_steps.push_back(steps[idx]);
    p.nsteps = (uint32_t)seg.size();
    p.alg_bytes = 2.0 * state_bytes(M, o.amp_bytes);
    plan->passes.push_back(p);
}

// Gather segmentation: maximal runs; affine runs use tables, others bit-sliced.
// Steps with more controls than the sliced descriptor holds run as sweeps.
void plan_gather(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &order,
                 const PlanOptions &o, Plan *plan)
{
    size_t i = 0;
    const size_t n = order.size();
    while (i < n) {
        const qsim_step &s0 = steps[order[i]];
        if (popcount64(s0.ctrl_mask) > kSlicedMaxControls) {
            plan->passes.push_back(make_sweep(M, s0, o.amp_bytes));
            plan->order.push_back(order[i]);
            plan->pass_ends.push_back(plan->order.size());
            ++i;
            continue;
        }
        size_t j = i;
        bool affine = true;
        while (j < n && (j - i) < (size_t)kMaxGatherSteps &&
               popcount64(steps[order[j]].ctrl_mask) <= kSlicedMaxControls) {
            affine = affine && is_affine_step(steps[order[j]]);
            ++j;
        }
        std::vector<uint64_t> seg(order.begin() + i, order.begin() + j);
        if (affine)
            emit_affine(M, steps, seg, o, plan);
        else if (o.jit && M >= 10 && (int)seg.size() >= o.jit_min_steps)
            emit_compiled(M, steps, seg, o, plan);
        else
            emit_sliced(M, steps, seg, o, plan);
        for (uint64_t idx : seg) plan->order.push_back(idx);
        plan->pass_ends.push_back(plan->order.size());
        i = j;
    }
}

// ---- cost model ---------------------------------------------------------------
//
// Estimated device time of a pass on GB300, from measured rates (6.78 TB/s
// copy bandwidth): tile and sweep passes stream their bytes at about 90 %
// and 87 % of it; a coset gather streams aligned runs; a gather that reads
// single amplitudes at scattered rows pays a 64-byte DRAM access per read and
// runs those at about half the copy rate; evaluating a non-affine segment
// costs integer work per step and output (bit-sliced interpreter or compiled
// kernel); every launch costs a few microseconds.
constexpr double kPeakBytesPerS = 6.78e12;
constexpr double kEffTile = 0.90;
constexpr double kEffSweep = 0.87;
constexpr double kEffCoset = 0.80;
constexpr double kRandomReadBytes = 64.0;
constexpr double kEffRandom = 0.50;
constexpr double kSlicedStepS = 2.8e-14;  // per step and output, interpreter
constexpr double kCompiledStepS = 2.2e-15; // per step and output, compiled kernel
constexpr double kLaunchS = 4e-6;
constexpr double kEffClosed = 0.92;        // closed pass: tiles dealt cyclically, 64-byte runs
constexpr double kTableStepS = 2.1e-11;    // tile table build, per local index and step, one SM
constexpr double kSms = 152.0;
constexpr double kClosedStepS = 1.2e-15;   // per step and output, planes in registers

double gather_cost_s(uint32_t M, size_t amp, bool affine, bool coset, bool compiled, size_t nsteps)
{
    const double n = (double)(1ull << M);
    if (affine && coset) return kLaunchS + 2.0 * n * (double)amp / (kEffCoset * kPeakBytesPerS);
    double t = kLaunchS + n * (kRandomReadBytes + (double)amp) / (kEffRandom * kPeakBytesPerS);
    if (!affine) t += (double)nsteps * n * (compiled ? kCompiledStepS : kSlicedStepS);
    return t;
}

double pass_cost_s(const Pass &p, uint32_t M, size_t amp)
{
    if (p.kind == kSweep) return kLaunchS + p.alg_bytes / (kEffSweep * kPeakBytesPerS);
    if (p.kind == kTile && p.tile.closed) {
        // streaming and per-output evaluation overlap (the next tile's
        // sources are found while it loads)
        const double mem = p.alg_bytes / (kEffClosed * kPeakBytesPerS);
        const double alu = (double)p.tile.jit_n * (double)(1ull << M) * kClosedStepS;
        return kLaunchS + std::max(mem, alu) + 0.1 * std::min(mem, alu);
    }
    if (p.kind == kTile) {
        // table builds: every local index through every step, by the SMs
        const double build = p.tile.rebuilds * (double)(1u << p.tile.k) * (double)p.tile.nsteps *
                             kTableStepS / kSms;
        return kLaunchS + p.alg_bytes / (kEffTile * kPeakBytesPerS) + build;
    }
    const GatherPass &g = p.gather;
    return gather_cost_s(M, amp, g.affine != 0, g.coset != 0, g.jit != 0,
                         g.jit ? g.jit_n : g.nsteps);
}

double plan_cost_s(const Plan &plan, uint32_t M, size_t amp)
{
    double t = 0;
    for (const Pass &p : plan.passes) t += pass_cost_s(p, M, amp);
    return t;
}

// Estimated cost of one gather pass (or several, beyond the step limit) over
// order[i, j), as plan_gather would cut it.
double gather_range_cost_s(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &order,
                           size_t i, size_t j, const PlanOptions &o)
{
    double t = 0;
    while (i < j) {
        const size_t e = std::min(j, i + (size_t)kMaxGatherSteps);
        bool affine = true, wide = false;
        for (size_t q = i; q < e; ++q) {
            affine = affine && is_affine_step(steps[order[q]]);
            wide = wide || popcount64(steps[order[q]].ctrl_mask) > kSlicedMaxControls;
        }
        if (wide) return 1e30;  // left to the pure plans
        const bool compiled = !affine && o.jit && M >= 10 && (int)(e - i) >= o.jit_min_steps;
        t += gather_cost_s(M, o.amp_bytes, affine, o.coset, compiled, e - i);
        i = e;
    }
    return t;
}

// With compiled kernels, a tile pass whose permutation table would be
// rebuilt for many tiles (steps controlled by bits outside the tile) runs
// instead as a closed pass over the same tile: its steps only change tile
// bits, so each output's source is evaluated from the compiled steps with
// the outside bits constant per tile.  Converted where the cost model
// expects it to be faster.
void close_tile_passes(uint32_t M, const qsim_step *steps, const PlanOptions &o, Plan *plan)
{
    if (!o.jit) return;
    for (size_t pi = 0; pi < plan->passes.size(); ++pi) {
        Pass &p = plan->passes[pi];
        if (p.kind != kTile || p.tile.closed || p.tile.k < 10 || p.tile.l < 1 || !p.tile.tma) continue;
        Pass c = p;
        TilePass &t = c.tile;
        t.closed = 1;
        const uint64_t first = pi ? plan->pass_ends[pi - 1] : 0, last = plan->pass_ends[pi];
        t.jit_n = (uint32_t)(last - first);
        c.alg_bytes = 2.0 * state_bytes(M, o.amp_bytes);
        if (pass_cost_s(c, M, o.amp_bytes) >= pass_cost_s(p, M, o.amp_bytes)) continue;
        t.jit_off = (uint32_t)plan->jit_steps.size();
        for (uint64_t q = first; q < last; ++q) plan->jit_steps.push_back(steps[plan->order[q]]);
        t.nsteps = 0;
        t.all_local = 1;
        t.touched = 1.0;
        p = c;
    }
}

// Append the passes of src (planned on its own) to dst, rebasing the
// offsets of their tables and step lists.
void append_plan(const Plan &src, Plan *dst)
{
    const uint32_t tile0 = (uint32_t)dst->tile_steps.size(), sl0 = (uint32_t)dst->sliced_steps.size();
    const uint32_t tab0 = (uint32_t)dst->gather_tables.size(), jit0 = (uint32_t)dst->jit_steps.size();
    const uint64_t ord0 = dst->order.size();
    for (Pass p : src.passes) {
        if (p.kind == kTile) {
            p.tile.step_off += tile0;
            p.tile.jit_off += jit0;
        } else if (p.kind == kGather) {
            p.gather.table_off += tab0;
            p.gather.coset_off += tab0;
            p.gather.step_off += sl0;
            p.gather.jit_off += jit0;
        }
        dst->passes.push_back(p);
    }
    dst->tile_steps.insert(dst->tile_steps.end(), src.tile_steps.begin(), src.tile_steps.end());
    dst->sliced_steps.insert(dst->sliced_steps.end(), src.sliced_steps.begin(), src.sliced_steps.end());
    dst->gather_tables.insert(dst->gather_tables.end(), src.gather_tables.begin(), src.gather_tables.end());
    dst->jit_steps.insert(dst->jit_steps.end(), src.jit_steps.begin(), src.jit_steps.end());
    dst->order.insert(dst->order.end(), src.order.begin(), src.order.end());
    for (uint64_t e : src.pass_ends) dst->pass_ends.push_back(e + ord0);
}

// Per-segment choice (Sec. 2i groups sequential steps; each group may take
// its own strategy).  The applied order is cut at long NOT/CNOT runs, which a
// coset gather moves in one streaming pass; each run of blocks between cuts
// becomes either one gather (its steps merged) or the tile passes of its
// blocks, whichever the cost model prefers, by dynamic programming over the
// blocks.  Returns false when there is nothing to cut.
constexpr size_t kMinAffineRun = 24;
constexpr size_t kMaxBlocks = 48;

bool plan_hybrid(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &order,
                 const PlanOptions &o, Plan *plan)
{
    // blocks: [start, end) of order; affine runs of >= kMinAffineRun steps
    // stand alone, everything between them forms one block
    std::vector<std::pair<size_t, size_t>> blocks;
    const size_t n = order.size();
    size_t cur = 0, i = 0;
    while (i < n) {
        if (!is_affine_step(steps[order[i]])) {
            ++i;
            continue;
        }
        size_t j = i;
        while (j < n && is_affine_step(steps[order[j]])) ++j;
        if (j - i >= kMinAffineRun) {
            if (cur < i) blocks.push_back({cur, i});
            blocks.push_back({i, j});
            cur = j;
        }
        i = j;
    }
    if (cur < n) blocks.push_back({cur, n});
    if (blocks.size() < 2 || blocks.size() > kMaxBlocks) return false;
    const size_t B = blocks.size();
    // tile cost of each block alone (its own greedy segmentation)
    std::vector<double> tcost(B);
    for (size_t b = 0; b < B; ++b) {
        Plan tmp;
        std::vector<uint64_t> sub(order.begin() + blocks[b].first, order.begin() + blocks[b].second);
        plan_tiles(M, steps, sub, o, true, &tmp);
        close_tile_passes(M, steps, o, &tmp);
        tcost[b] = plan_cost_s(tmp, M, o.amp_bytes);
    }
    // best[j]: cheapest cover of blocks [0, j); choice: start block and kind
    std::vector<double> best(B + 1, 1e300);
    std::vector<size_t> from(B + 1, 0);
    std::vector<char> as_gather(B + 1, 0);
    best[0] = 0;
    for (size_t j = 1; j <= B; ++j) {
        double tiles = 0;
        for (size_t a = j; a-- > 0;) {
            tiles += tcost[a];
            const double g = gather_range_cost_s(M, steps, order, blocks[a].first, blocks[j - 1].second, o);
            const double c = std::min(tiles, g);
            if (best[a] + c < best[j]) {
                best[j] = best[a] + c;
                from[j] = a;
                as_gather[j] = g < tiles;
            }
        }
    }
    std::vector<std::pair<size_t, size_t>> segs;  // (block range end j, start a)
    for (size_t j = B; j > 0; j = from[j]) segs.push_back({j, from[j]});
    std::reverse(segs.begin(), segs.end());
    for (const auto &sg : segs) {
        const size_t a = sg.second, j = sg.first;
        if (as_gather[j]) {
            std::vector<uint64_t> sub(order.begin() + blocks[a].first, order.begin() + blocks[j - 1].second);
            plan_gather(M, steps, sub, o, plan);
        } else {
            for (size_t b = a; b < j; ++b) {
                std::vector<uint64_t> sub(order.begin() + blocks[b].first, order.begin() + blocks[b].second);
                Plan tmp;
                plan_tiles(M, steps, sub, o, true, &tmp);
                close_tile_passes(M, steps, o, &tmp);
                append_plan(tmp, plan);
            }
        }
    }
    return true;
}

// Closed tile pass: when the circuit's net row map changes only the address
// bits in delta (the OR over all rows of x(i) ^ i, found on the device), every
// output's source lies in the same coset of those bits.  A tile over delta,
// filled up from bit 0 to the widest tile shared memory holds (so that the
// low address bits give contiguous runs), then holds every source of its
// outputs, and one in-place pass applies the whole circuit: Sec. 2i's
// grouping of sequential steps taken to a whole circuit, with the Sec. 2h
// product evaluated per output.  Needs compiled kernels.
bool plan_closed(uint32_t M, const qsim_step *steps, const std::vector<uint64_t> &order,
                 const PlanOptions &o, Plan *plan)
{
    if (!o.jit || !o.closed_known || order.empty()) return false;
    uint32_t kmax = std::min<uint32_t>(o.amp_bytes == 16 ? 13 : 14, M);
    if (o.tile_bits > 0) kmax = std::min<uint32_t>(kmax, (uint32_t)o.tile_bits);
    uint64_t T = o.closed_delta & full_mask(M);
    if ((uint32_t)popcount64(T) > kmax) return false;
    for (uint32_t b = 0; b < M && (uint32_t)popcount64(T) < kmax; ++b) T |= 1ull << b;
    uint32_t l = 0;
    while (l < M && ((T >> l) & 1ull)) ++l;
    l = std::min<uint32_t>(l, o.amp_bytes == 16 ? 7 : 8);  // a tensor-map box row is <= 256 words
    const uint32_t k = (uint32_t)popcount64(T);
    if (l < 1 || k < 10 || k - l > (uint32_t)kMaxHighBitsClosed) return false;
    Pass p{};
    p.kind = kTile;
    TilePass &t = p.tile;
    layout_tile(M, l, T & ~((1ull << l) - 1ull), o.amp_bytes, &t);
    if (!t.tma || t.k != k) return false;
    t.closed = 1;
    t.n_tiles = 1ull << (M - k);
    t.nout = 0;
    for (uint32_t b = 0; b < M; ++b)
        if (!((T >> b) & 1ull)) t.outpos[t.nout++] = b;
    t.step_off = (uint32_t)plan->tile_steps.size();
    t.nsteps = 0;
    t.all_local = 1;
    t.touched = 1.0;
    t.jit_off = (uint32_t)plan->jit_steps.size();
    t.jit_n = (uint32_t)order.size();
    for (uint64_t idx : order) plan->jit_steps.push_back(steps[idx]);
    p.nsteps = t.jit_n;
    p.alg_bytes = 2.0 * state_bytes(M, o.amp_bytes);
    plan->passes.push_back(p);
    for (uint64_t idx : order) plan->order.push_back(idx);
    plan->pass_ends.push_back(plan->order.size());
    return true;
}

}  // namespace

int make_plan(uint32_t M, const qsim_step *steps, size_t L, const PlanOptions &o, Plan *plan,
              std::string *msg)
{
    int rc = validate_steps(M, steps, L, msg);
    if (rc != QSIM_OK) return rc;
    if (o.amp_bytes != 8 && o.amp_bytes != 16) {
        if (msg) *msg = "amplitude size must be 8 or 16 bytes";
        return QSIM_EINVAL;
    }
    *plan = Plan{};
    plan->steps_in = L;
    std::vector<uint64_t> order = canonical_order(steps, L, o.cancel_adjacent, &plan->cancelled);
    if (order.empty()) return QSIM_OK;

    int strategy = o.strategy;
    PlanOptions oo = o;
    if (strategy == QSIM_STRATEGY_INPLACE) {
        strategy = QSIM_STRATEGY_AUTO;
        oo.scratch_available = false;
    }
    if (strategy == QSIM_STRATEGY_GATHER && !o.scratch_available) {
        if (msg) *msg = "gather strategy needs a scratch buffer";
        return QSIM_EINVAL;
    }
    if (strategy == QSIM_STRATEGY_SWEEP) {
        for (uint64_t idx : order) {
            plan->passes.push_back(make_sweep(M, steps[idx], oo.amp_bytes));
            plan->order.push_back(idx);
            plan->pass_ends.push_back(plan->order.size());
        }
        return QSIM_OK;
    }
    if (strategy == QSIM_STRATEGY_TILE) {
        plan_tiles(M, steps, order, oo, false, plan);
        return QSIM_OK;
    }
    if (strategy == QSIM_STRATEGY_GATHER) {
        plan_gather(M, steps, order, oo, plan);
        return QSIM_OK;
    }
    // AUTO: the in-place tile/sweep plan, or -- when a scratch buffer is
    // allowed -- the gather plan or a per-segment mix of both, whichever the
    // cost model expects to run fastest.
    Plan tp;
    tp.steps_in = plan->steps_in;
    tp.cancelled = plan->cancelled;
    plan_tiles(M, steps, order, oo, true, &tp);
    close_tile_passes(M, steps, oo, &tp);
    double tcost = plan_cost_s(tp, M, oo.amp_bytes);
    {
        Plan cp;
        cp.steps_in = plan->steps_in;
        cp.cancelled = plan->cancelled;
        if (plan_closed(M, steps, order, oo, &cp)) {
            const double ccost = plan_cost_s(cp, M, oo.amp_bytes);
            if (ccost < tcost) {
                tp = std::move(cp);
                tcost = ccost;
            }
        }
    }
    if (oo.scratch_available) {
        Plan gp;
        gp.steps_in = plan->steps_in;
        gp.cancelled = plan->cancelled;
        plan_gather(M, steps, order, oo, &gp);
        const double gcost = plan_cost_s(gp, M, oo.amp_bytes);
        Plan hp;
        hp.steps_in = plan->steps_in;
        hp.cancelled = plan->cancelled;
        const double hcost = plan_hybrid(M, steps, order, oo, &hp) ? plan_cost_s(hp, M, oo.amp_bytes) : 1e300;
        if (hcost < gcost && hcost < tcost) {
            *plan = std::move(hp);
            return QSIM_OK;
        }
        if (gcost < tcost) {
            *plan = std::move(gp);
            return QSIM_OK;
        }
    }
    *plan = std::move(tp);
    return QSIM_OK;
}

double plan_estimated_ms(const Plan &plan, uint32_t M, size_t amp) { return 1e3 * plan_cost_s(plan, M, amp); }

double pass_estimated_ms(const Pass &p, uint32_t M, size_t amp) { return 1e3 * pass_cost_s(p, M, amp); }

// App. 1 input, per amplitude: the product-state kernel (complex64: one
// float-float complex product; complex128: one FP64 complex product), and a
// first tile pass that generates its sources (a product from two tables) and
// writes the probabilities, which is bound by instruction issue, not HBM.
constexpr double kProductOutS[2] = {1.3e-12, 1.1e-11};       // complex64, complex128
constexpr double kProductFusedOutS[2] = {5.5e-12, 1.4e-11};

double product_state_estimated_ms(uint32_t M, size_t amp)
{
    const double n = (double)(1ull << M);
    const double write = n * (double)amp / (kEffTile * kPeakBytesPerS);
    return 1e3 * (kLaunchS + std::max(write, n * kProductOutS[amp == 16]));
}

double product_plan_estimated_ms(const Plan &plan, uint32_t M, size_t amp, bool fused)
{
    if (!fused || plan.passes.empty()) return plan_estimated_ms(plan, M, amp) + product_state_estimated_ms(M, amp);
    const double first = pass_cost_s(plan.passes[0], M, amp);
    const double gen = kLaunchS + (double)(1ull << M) * kProductFusedOutS[amp == 16];
    return 1e3 * (plan_cost_s(plan, M, amp) - first + std::max(first, gen));
}

std::vector<double> product_tables(uint32_t M, const double *qubits, const TilePass &t)
{
    // complex products with each real product and sum rounded separately
    struct C {
        double re, im;
    };
    auto mul = [](C a, C b) {
        volatile double p1 = a.re * b.re, p2 = a.im * b.im, p3 = a.re * b.im, p4 = a.im * b.re;
        return C{p1 - p2, p3 + p4};
    };
    auto q = [&](uint32_t b, uint32_t v) { return C{qubits[4 * b + 2 * v], qubits[4 * b + 2 * v + 1]}; };
    std::vector<double> out(2 * (2 * QSIM_MAX_QUBITS + (1u << t.l) + (1u << t.nh)), 0.0);
    for (uint32_t b = 0; b < M; ++b)
        for (uint32_t v = 0; v < 2; ++v) {
            out[2 * (2 * b + v)] = qubits[4 * b + 2 * v];
            out[2 * (2 * b + v) + 1] = qubits[4 * b + 2 * v + 1];
        }
    size_t at = 2 * QSIM_MAX_QUBITS;
    for (uint32_t u = 0; u < (1u << t.l); ++u, ++at) {
        C c{1.0, 0.0};
        for (uint32_t b = t.l; b-- > 0;) c = mul(c, q(b, (u >> b) & 1u));
        out[2 * at] = c.re;
        out[2 * at + 1] = c.im;
    }
    for (uint32_t h = 0; h < (1u << t.nh); ++h, ++at) {
        C c{1.0, 0.0};
        for (uint32_t k = t.nh; k-- > 0;) c = mul(c, q(t.high[k], (h >> k) & 1u));
        out[2 * at] = c.re;
        out[2 * at + 1] = c.im;
    }
    return out;
}

int sliced_steps_of(uint32_t M, const qsim_step *steps, size_t L, std::vector<SlicedStep> *out,
                    std::string *msg)
{
    int rc = validate_steps(M, steps, L, msg);
    if (rc != QSIM_OK) return rc;
    for (size_t i = 0; i < L; ++i)
        if (popcount64(steps[i].ctrl_mask) > kSlicedMaxControls) {
            if (msg) *msg = "step " + std::to_string(i) + " has more than " +
                            std::to_string(kSlicedMaxControls) + " controls";
            return QSIM_EINVAL;
        }
    Plan tmp;
    std::vector<uint64_t> seg(L);
    for (size_t i = 0; i < L; ++i) seg[i] = i;
    PlanOptions o;
    emit_sliced(M, steps, seg, o, &tmp);
    *out = std::move(tmp.sliced_steps);
    return QSIM_OK;
}

uint32_t pass_variant(const Pass &p)
{
    if (p.kind == kTile && p.tile.closed) return 8;
    if (p.kind != kGather) return (uint32_t)p.kind;
    if (p.gather.affine) return p.gather.coset ? 7 : 3;
    return p.gather.jit ? 5 : 4;
}

}  // namespace qsim
