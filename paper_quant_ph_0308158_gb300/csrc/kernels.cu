// kernels.cu -- sm_103a kernels of the reversible wiring-diagram engine.
//
// The circuit kernels only move amplitudes (8-byte complex64 or 16-byte
// complex128 words); index arithmetic is integer.  Floating point appears in
// the FP64 probabilities (and their norm) and in the App. 1 product-state
// input, which is computed, not moved.
//
//   sweep_kernel          one step in place over the toggled pairs only
//                         (Sec. 2b 'intelligent looping'), 16-byte vectors.
//   tile_kernel           a run of steps on 2^k-amplitude tiles staged in
//                         shared memory by bulk-async (TMA) copies, in place
//                         (Sec. 2i: sequential steps processed together);
//                         optionally generating its sources from the qubits
//                         of a product state (App. 1).
//   gather_affine_kernel  k2(i) = k1(A i ^ b) for CNOT/NOT segments
//                         (Sec. 2h product of the steps, Sec. 2b gather).
//   gather_coset_kernel   the same map over coset tiles of the output space,
//                         so that reads and writes are aligned runs.
//   gather_sliced_kernel  k2(i) = k1(x(i)) with x(i) evaluated for 64 output
//                         indices at once in bit-sliced form, steps applied
//                         last to first (Sec. 2h product, Sec. 2b gather).
//   row_array_kernel      x(i) for every output (the Sec. 2h row array).
//   gather_rows_kernel    k2(i) = k1(x(i)) from a stored row array.
//   batch_kernel          one pass level of many circuits (persistent CTAs
//                         pulling work items).
//   product_state_kernel  k1(i) = product over qubits of q_b(bit b of i).
//   probs_kernel          p(i) = re^2 + im^2 in FP64 and a norm partial sum;
//   probs_pairs_kernel    the same without the norm, two complex64
//                         amplitudes per 16-byte load.
// The closed pass and the compiled gather are generated per circuit (jit.cu).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "prob_math.cuh"
#include "qsim_internal.h"

namespace qsim {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kWaitLimit = 1u << 24;  // bounded mbarrier polls (seconds)

template <int B> struct AmpOf;
template <> struct AmpOf<8> { using T = uint2; };
template <> struct AmpOf<16> { using T = uint4; };

// FP64 probability of one amplitude held as raw words (prob_math.cuh)
QSIM_PROB_MATH(__device__ __forceinline__, __device__ __noinline__)
__device__ __forceinline__ double amp_prob(const uint2 &v) { return qsim_prob_bits(v.x, v.y); }
__device__ __forceinline__ double amp_prob(const uint4 &v) { return qsim_prob_bits(v.x, v.y, v.z, v.w); }

// One amplitude at a data-dependent row (the gather's read).  FILL64: the
// read-only path with a 64-byte L2 fill instead of the default larger one,
// which cuts the DRAM bytes fetched per random 16-byte read of a large state;
// otherwise the plain read-only load (better when the state sits in L2, as
// the small states of a batch do).
__device__ __forceinline__ uint2 ld_row64(const uint2 *p)
{
    uint2 v;
    asm("ld.global.nc.L2::64B.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_row64(const uint4 *p)
{
    uint4 v;
    asm("ld.global.nc.L2::64B.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

template <bool FILL64, typename A>
__device__ __forceinline__ A ld_row(const A *p)
{
    if (FILL64) return ld_row64(p);
    return __ldg(p);
}

// Insert a zero bit at position pos of x (bits >= pos move up by one).
__device__ __forceinline__ uint64_t insert_zero(uint64_t x, uint32_t pos)
{
    const uint64_t lo = x & ((1ull << pos) - 1ull);
    return ((x >> pos) << (pos + 1)) | lo;
}

// ---- mbarrier / bulk-async copy (TMA) wrappers ------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// One box of a 5-dimensional tensor map into shared memory.
__device__ __forceinline__ void tensor_g2s(void *dst_smem, const CUtensorMap *map, int c0, int c1,
                                           int c2, int c3, int c4, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ============================================================================
// (a) per-step sweep over toggled pairs
// ============================================================================

// The first index of pair q: a zero inserted at every listed bit (target,
// controls and, for the paired complex64 form, bit 0), then the polarity.
__device__ __forceinline__ uint64_t sweep_index(uint64_t q, const SweepParams &p, uint32_t first)
{
    uint64_t j = first ? insert_zero(q, 0) : q;
#pragma unroll 1
    for (uint32_t s = 0; s < p.nins; ++s) j = insert_zero(j, p.ins[s]);
    return j | p.pol;
}

// One step in place, every access 16 bytes wide (uint4), two units per
// thread in flight.  MODE 0: complex128, a unit is one pair.  complex64 (two
// amplitudes per vector): MODE 1, target bit 0: a unit is one vector whose
// halves swap; MODE 2, bit 0 free: a unit is two neighbouring pairs, two
// whole vectors swap (a high target moves contiguous blocks); MODE 3, bit 0 a
// control: a unit is one pair, the active half of each of its two vectors
// swaps and the inactive half is written back unchanged (no other unit of
// the step touches either vector).
template <int MODE>
__global__ void __launch_bounds__(kThreads) sweep_kernel(uint4 *__restrict__ st, SweepParams p, uint64_t units)
{
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    const uint64_t hv = MODE == 0 ? p.half : p.half >> 1;  // partner offset in vectors
    for (uint64_t q = (uint64_t)blockIdx.x * kThreads + threadIdx.x; q < units; q += 2 * stride) {
        uint64_t v[2];
        bool on[2];
        uint4 a[2], b[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t qq = q + (uint64_t)u * stride;
            on[u] = qq < units;
            if (!on[u]) continue;
            const uint64_t j = sweep_index(qq, p, MODE == 2);
            v[u] = MODE == 0 ? j : j >> 1;
            a[u] = st[v[u]];
            if (MODE != 1) b[u] = st[v[u] + hv];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!on[u]) continue;
            if (MODE == 1) {
                st[v[u]] = make_uint4(a[u].z, a[u].w, a[u].x, a[u].y);
            } else if (MODE == 3) {
                uint4 x = a[u], y = b[u];
                if (p.pol & 1ull) {  // the odd halves are the active ones
                    x.z = b[u].z; x.w = b[u].w; y.z = a[u].z; y.w = a[u].w;
                } else {
                    x.x = b[u].x; x.y = b[u].y; y.x = a[u].x; y.y = a[u].y;
                }
                st[v[u]] = x;
                st[v[u] + hv] = y;
            } else {
                st[v[u]] = b[u];
                st[v[u] + hv] = a[u];
            }
        }
    }
}

// ============================================================================
// (b) tile pass: TMA bulk loads into shared memory, in-tile permutation,
//     in-place stores
// ============================================================================

// Per tile, the permutation of its 2^k local indices depends only on which
// steps are active there (their controls outside the tile are constant over
// a tile).  It is kept as a table perm[j] = source of local output j and is
// recomputed only when the set of active steps changes from one tile to the
// next.  Tiles are dealt to CTAs in contiguous ranges of the tile id, whose
// highest bits are the out-of-tile control bits, so a CTA sees long runs of
// tiles with the same active set.
constexpr int kTileThreads = 512;
constexpr int kMaxOutBits = 40;
constexpr uint32_t kProductStages = 4;            // stages of a product-input tile pass
constexpr size_t kMaxTileSmem = 227 * 1024;       // dynamic shared memory of one CTA
constexpr int kMaskWords = kMaxTileSteps / 32;

struct TileKParams {
    char *state;
    double *probs;                 // non-null: also write FP64 probabilities (every tile)
    const TileStep *steps;
    int *err;
    uint64_t n_tiles;
    uint32_t k, l, nh, nsteps, all_local, stages, nout;
    uint32_t buf_bytes;            // stage region: tiles, or the product tables
    uint32_t high[kMaxHighBits];
    uint32_t outpos[kMaxOutBits];  // global bit of tile-id bit q
    uint32_t tma, nrest, epa, box_bytes;
    uint32_t affine;               // every step has at most one control
    uint32_t start[6];             // tensor view: first address bit of each dimension
    uint32_t rest_pos[kMaxHighBits];
    uint32_t wait_limit;           // polls before a pipeline wait gives up
    uint32_t stall_producer;       // testing: the producer leaves without loading a tile
    // App. 1 input (product-input pass): source amplitudes are computed, not
    // loaded.  qtab: per address bit b, (q_b(0), q_b(1)) as FP64 complex;
    // plow: the product over the tile's low l bits for each of their 2^l
    // values; phigh: over its high bits for each of their 2^nh values.
    // The stage region then holds those two tables and, per stage, the
    // tile's products over its high bits (written by the producer warp).
    const double2 *qtab, *plow, *phigh;
};

struct TileStageMeta {
    uint64_t base;                 // global index of local index 0; ~0 = no tile
    uint32_t mask[kMaskWords];     // active steps
    uint32_t same;                 // active set equals the previous tile's
    uint32_t pad;
};

constexpr uint64_t kNoTile = ~0ull;

__device__ __forceinline__ uint64_t tile_base(uint64_t tile, const uint32_t *outpos)
{
    uint64_t b = 0;
    for (uint32_t q = 0; tile; ++q, tile >>= 1)
        if (tile & 1ull) b |= 1ull << outpos[q];
    return b;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait on an mbarrier phase; false if the limit was reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (unsigned w = 0; w < limit; ++w)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"r"(kTileThreads) : "memory");
}

// Warp-specialised pipeline: warps 0..15 consume tiles, warp 16 produces.
// Stage s has a 'full' barrier (one producer arrival + the bytes of the
// bulk copies) and an 'empty' barrier (one arrival per consumer warp).  The
// producer finds the CTA's next tile with an active step, publishes its
// base and active-step mask in the stage's metadata, and issues one bulk
// copy per contiguous run of 2^l amplitudes; an empty tile marks the end.
// Float-float complex products of the product-input pass (FP32 work, not
// FP64 issue), written so that no multiply-add contraction can break their
// error-free parts.
#include "ff_math.cuh"

__device__ __forceinline__ double2 dcmul(double2 a, double2 b)
{
    return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                        __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}

// Partial products of the product-input pass kept per tile: float-float for
// complex64 output, FP64 for complex128.
template <int B> struct ProdT;
template <> struct ProdT<8> {
    using T = FFc;
    static __device__ __forceinline__ T of(double2 v) { return ffc_of(v); }
    static __device__ __forceinline__ T scale(const T &c, const T &h) { return ffc_mul(c, h); }
    static __device__ __forceinline__ uint2 mul(const T &a, const T &b)
    {
        const float re = ff_dot2_round(a.rh, a.rl, b.rh, b.rl, a.ih, a.il, b.ih, b.il, -1.0f);
        const float im = ff_dot2_round(a.rh, a.rl, b.ih, b.il, a.ih, a.il, b.rh, b.rl, 1.0f);
        return make_uint2(__float_as_uint(re), __float_as_uint(im));
    }
};
template <> struct ProdT<16> {
    using T = double2;
    static __device__ __forceinline__ T of(double2 v) { return v; }
    static __device__ __forceinline__ T scale(const T &c, const T &h) { return dcmul(c, h); }
    static __device__ __forceinline__ uint4 mul(const T &a, const T &b)
    {
        const double2 v = dcmul(a, b);
        const unsigned long long x = (unsigned long long)__double_as_longlong(v.x);
        const unsigned long long y = (unsigned long long)__double_as_longlong(v.y);
        return make_uint4((uint32_t)x, (uint32_t)(x >> 32), (uint32_t)y, (uint32_t)(y >> 32));
    }
};

template <int B, bool PROBS, bool PRODUCT>
__global__ void __launch_bounds__(kTileThreads + 32, 1)
    tile_kernel(TileKParams p, const __grid_constant__ CUtensorMap tmap)
{
    using A = typename AmpOf<B>::T;
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t tile_amps = 1u << p.k;
    const size_t tile_bytes = (size_t)B * tile_amps;
    char *bufs = reinterpret_cast<char *>(smem);
    uint64_t *depo = reinterpret_cast<uint64_t *>(smem + p.buf_bytes);
    TileStageMeta *meta = reinterpret_cast<TileStageMeta *>(depo + (1u << p.nh));
    uint64_t *full = reinterpret_cast<uint64_t *>(meta + p.stages);
    uint64_t *empty = full + p.stages;
    TileStep *steps_sm = reinterpret_cast<TileStep *>(empty + p.stages);
    uint32_t *outpos = reinterpret_cast<uint32_t *>(steps_sm + p.nsteps);
    uint16_t *perm = reinterpret_cast<uint16_t *>(outpos + kMaxOutBits);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nthreads = kTileThreads + 32;
    for (uint32_t r = tid; r < (1u << p.nh); r += nthreads) {
        uint64_t d = 0;
        for (uint32_t q = 0; q < p.nh; ++q) d |= (uint64_t)((r >> q) & 1u) << p.high[q];
        depo[r] = d;
    }
    for (uint32_t i = tid; i < p.nsteps; i += nthreads) steps_sm[i] = p.steps[i];
    for (uint32_t i = tid; i < kMaxOutBits; i += nthreads) outpos[i] = p.outpos[i];
    // product input: the stage region holds the products over the low bits,
    // over the high bits, and per stage the tile's scaled high products
    using PT = typename ProdT<B>::T;
    PT *tlow = reinterpret_cast<PT *>(bufs);
    PT *phigh = tlow + (1u << p.l);
    PT *thigh = phigh + (1u << p.nh);  // + stage * 2^nh
    if (PRODUCT) {
        for (uint32_t u = tid; u < (1u << p.l); u += nthreads) tlow[u] = ProdT<B>::of(p.plow[u]);
        for (uint32_t h = tid; h < (1u << p.nh); h += nthreads) phigh[h] = ProdT<B>::of(p.phigh[h]);
    }
    if (tid == 0) {
        for (uint32_t s = 0; s < p.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kTileThreads / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // contiguous range of tile ids for this CTA
    const uint64_t per = (p.n_tiles + gridDim.x - 1) / gridDim.x;
    const uint64_t begin = (uint64_t)blockIdx.x * per;
    const uint64_t end = begin + per < p.n_tiles ? begin + per : p.n_tiles;

    if (warp == kTileThreads / 32) {
        // ---------------- producer warp ----------------
        // testing hook: leave before any copy is issued, so that every
        // consumer's first wait runs out with nothing in flight
        if (p.stall_producer) return;
        uint64_t next = begin;
        uint32_t last[kMaskWords];
        bool have_last = false;
        const uint32_t run_bytes = (uint32_t)B << p.l;
        for (uint32_t it = 0;; ++it) {
            const uint32_t s = it % p.stages;
            if (it >= p.stages && !mbar_wait_bounded(&empty[s], ((it / p.stages) - 1) & 1u, p.wait_limit)) {
                if (lane == 0) atomicOr(p.err, 2);
                return;
            }
            uint64_t base = kNoTile;
            uint32_t mask[kMaskWords];
            while (next < end) {
                base = tile_base(next, outpos);
                ++next;
                bool any = false;
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w) {
                    const uint32_t i = w * 32 + lane;
                    bool act = false;
                    if (i < p.nsteps) act = p.all_local || (base & steps_sm[i].co) == steps_sm[i].po;
                    mask[w] = __ballot_sync(0xffffffffu, act);
                    any |= mask[w] != 0;
                }
                if (any || PROBS || PRODUCT) break;  // these passes write every tile
                base = kNoTile;
            }
            bool same = have_last && base != kNoTile;
            if (base != kNoTile) {
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w) same = same && (mask[w] == last[w]);
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w) last[w] = mask[w];
                have_last = true;
            }
            if (lane == 0) {
                meta[s].base = base;
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w) meta[s].mask[w] = base != kNoTile ? mask[w] : 0u;
                meta[s].same = same ? 1u : 0u;
            }
            __syncwarp();
            if (base == kNoTile) {
                if (lane == 0) mbar_arrive(&full[s]);  // end marker, no bytes
                return;
            }
            if (PRODUCT) {
                // nothing to load: the tile's factor over the bits outside it
                // (FP64, a butterfly product over the lanes, which leaves the
                // same value in every lane since each complex product is
                // commutative bit for bit), then its products over the high
                // tile bits (complex64: in float-float) for the consumers
                double2 f = make_double2(1.0, 0.0);
                if ((uint32_t)lane < p.nout) {
                    const uint32_t b = outpos[lane];
                    f = p.qtab[2 * b + (uint32_t)((base >> b) & 1ull)];
                }
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    double2 g;
                    g.x = __shfl_xor_sync(0xffffffffu, f.x, off);
                    g.y = __shfl_xor_sync(0xffffffffu, f.y, off);
                    f = dcmul(f, g);
                }
                const PT c = ProdT<B>::of(f);
                PT *th = thigh + ((size_t)s << p.nh);
                for (uint32_t h = lane; h < (1u << p.nh); h += 32) th[h] = ProdT<B>::scale(c, phigh[h]);
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[s]);
                continue;
            }
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(&full[s], run_bytes << p.nh);
            __syncwarp();
            char *buf = bufs + tile_bytes * s;
            if (p.tma) {
                // one tensor copy per value of the enumerated tile bits
                for (uint32_t r = lane; r < (1u << p.nrest); r += 32) {
                    uint64_t g = base;
                    for (uint32_t q = 0; q < p.nrest; ++q)
                        if ((r >> q) & 1u) g |= 1ull << p.rest_pos[q];
                    int c[5];
#pragma unroll
                    for (int d = 0; d < 5; ++d) {
                        const uint32_t w = p.start[d + 1] - p.start[d];
                        const uint64_t v = w ? ((g >> p.start[d]) & ((1ull << w) - 1ull)) : 0ull;
                        c[d] = (int)(d == 0 ? v * p.epa : v);
                    }
                    tensor_g2s(buf + (size_t)r * p.box_bytes, &tmap, c[0], c[1], c[2], c[3], c[4],
                               &full[s]);
                }
            } else {
                for (uint32_t r = lane; r < (1u << p.nh); r += 32)
                    bulk_g2s(buf + (size_t)r * run_bytes, p.state + (base + depo[r]) * B, run_bytes,
                             &full[s]);
            }
        }
    }

    // ---------------- consumer warps ----------------
    const uint32_t lmask = (1u << p.l) - 1u;
    bool have_perm = false;  // perm holds the table of an earlier tile
    uint32_t c0 = 0, delta = 0;  // affine passes: image of 0 in that table, shift now
    A *st = reinterpret_cast<A *>(p.state);
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % p.stages;
        if (!mbar_wait_bounded(&full[s], (it / p.stages) & 1u, p.wait_limit)) {
            if (tid == 0) atomicOr(p.err, 1);
            return;
        }
        const uint64_t base = meta[s].base;
        if (base == kNoTile) break;
        // no active step: only a pass writing probabilities or product input
        // sends such a tile
        bool idle = PROBS || PRODUCT;
#pragma unroll
        for (int w = 0; w < kMaskWords; ++w) idle = idle && meta[s].mask[w] == 0u;
        if (PROBS && !PRODUCT && idle) {
            const A *buf = reinterpret_cast<const A *>(bufs + tile_bytes * s);
            for (uint32_t j = tid; j < tile_amps; j += kTileThreads)
                p.probs[base + depo[j >> p.l] + (j & lmask)] = amp_prob(buf[j]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            continue;
        }
        if (idle) {
            // product input, no active step: every output is its own source
        } else if (!meta[s].same && p.affine && have_perm) {
            // NOT/CNOT segment: every tile's map is A j ^ c(tile) with the same
            // A, so the table of the first tile is reused with c(tile) ^ c(first)
            uint32_t c = 0;
            for (int q = (int)p.nsteps - 1; q >= 0; --q) {
                if (!((meta[s].mask[q >> 5] >> (q & 31)) & 1u)) continue;
                if ((c & steps_sm[q].cl) == steps_sm[q].pl) c ^= steps_sm[q].tmask;
            }
            delta = c ^ c0;
        } else if (!meta[s].same) {
            consumer_sync();  // every consumer is done with the previous table
            for (uint32_t j0 = 0; j0 < tile_amps; j0 += kTileThreads * 8) {
                uint32_t src[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) src[e] = j0 + tid + e * kTileThreads;
                for (int q = (int)p.nsteps - 1; q >= 0; --q) {
                    if (!((meta[s].mask[q >> 5] >> (q & 31)) & 1u)) continue;
                    const uint32_t cl = steps_sm[q].cl, pl = steps_sm[q].pl, tm = steps_sm[q].tmask;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if ((src[e] & cl) == pl) src[e] ^= tm;
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t j = j0 + tid + e * kTileThreads;
                    if (j < tile_amps) perm[j] = (uint16_t)src[e];
                }
            }
            // the table's own image of local index 0 (every thread evaluates it)
            c0 = 0;
            for (int q = (int)p.nsteps - 1; q >= 0; --q) {
                if (!((meta[s].mask[q >> 5] >> (q & 31)) & 1u)) continue;
                if ((c0 & steps_sm[q].cl) == steps_sm[q].pl) c0 ^= steps_sm[q].tmask;
            }
            delta = 0;
            have_perm = true;
            consumer_sync();  // the new table is complete
        }
        const A *buf = reinterpret_cast<const A *>(bufs + tile_bytes * s);
        const PT *th = thigh + ((size_t)s << p.nh);
        for (uint32_t j0 = 0; j0 < tile_amps; j0 += kTileThreads * 4) {
            A v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t j = j0 + tid + e * kTileThreads;
                if (j < tile_amps) {
                    if (PRODUCT) {
                        const uint32_t src = idle ? j : ((uint32_t)perm[j] ^ delta);
                        v[e] = ProdT<B>::mul(th[src >> p.l], tlow[src & lmask]);
                    } else {
                        v[e] = buf[perm[j] ^ delta];
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t j = j0 + tid + e * kTileThreads;
                if (j < tile_amps) {
                    const uint64_t g = base + depo[j >> p.l] + (j & lmask);
                    st[g] = v[e];
                    if (PROBS) p.probs[g] = amp_prob(v[e]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
    }
}

// ============================================================================
// (c) gather passes
// ============================================================================

// Affine gather of outputs [o0, o1): x(i) = b ^ XOR over index bytes of
// per-byte tables (already in shared memory).
template <int B, bool WIDE, typename I, bool FILL64>
__device__ __forceinline__ void affine_range(const char *__restrict__ in, char *__restrict__ out,
                                             uint64_t o0, uint64_t o1, uint64_t step,
                                             const I *tab, uint32_t nbytes, uint64_t bvec,
                                             double *__restrict__ probs)
{
    using A = typename AmpOf<B>::T;
    const A *src = reinterpret_cast<const A *>(in);
    A *dst = reinterpret_cast<A *>(out);
    for (uint64_t i0 = o0; i0 < o1; i0 += 4 * step) {
        A v[4];
        uint64_t idx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = i0 + u * step;
            idx[u] = i;
            if (i < o1) {
                I x = (I)bvec;
                for (uint32_t b = 0; b < nbytes; ++b) x ^= tab[b * 256 + ((i >> (8 * b)) & 255u)];
                v[u] = ld_row<FILL64>(&src[x]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (idx[u] < o1) {
                if (dst) dst[idx[u]] = v[u];  // no destination: probabilities only
                if (probs) probs[idx[u]] = amp_prob(v[u]);
            }
    }
}

template <int B, bool WIDE>
__global__ void __launch_bounds__(kThreads) gather_affine_kernel(const char *__restrict__ in,
                                                                 char *__restrict__ out, uint64_t n,
                                                                 const uint64_t *__restrict__ tables,
                                                                 uint32_t nbytes, uint64_t bvec,
                                                                 double *__restrict__ probs)
{
    using I = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    __shared__ I tab[5 * 256];
    for (uint32_t i = threadIdx.x; i < nbytes * 256; i += kThreads) tab[i] = (I)tables[i];
    __syncthreads();
    affine_range<B, WIDE, I, true>(in, out, (uint64_t)blockIdx.x * kThreads + threadIdx.x, n,
                             (uint64_t)gridDim.x * kThreads, tab, nbytes, bvec, probs);
}

// Bit-sliced gather.  Each thread owns 64 consecutive output indices
// my + j (j = 0..63) as bit planes: plane b is a 64-bit word whose bit j is
// bit b of index my + j.  Steps run last to first on the planes (target
// plane ^= AND of the control planes, a control on |0> complemented); two
// 32x32 bit transposes turn the planes back into 64 source indices, which
// the warp exchanges through shared memory so that every store instruction
// writes 32 consecutive amplitudes.  Planes live in shared memory as
// [plane][thread] words; plane M is all ones and stands in for absent
// controls, so the common steps (<= 2 controls, all on |1>) run without
// branches.
constexpr int kSlicedChunk = 256;            // steps staged in shared memory at a time
constexpr uint64_t kSlicedOutputs = kThreads * 64;  // outputs per CTA iteration

__device__ __forceinline__ void transpose32(uint32_t (&a)[32])
{
    // Bit-matrix transpose by five rounds of masked block swaps
    // (textbook recursive transpose; row r, bit c <-> row c, bit r).
    uint32_t m = 0x0000ffffu;
#pragma unroll
    for (int j = 16; j != 0; j >>= 1, m ^= (m << j)) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (k & j) continue;
            const uint32_t t = ((a[k] >> j) ^ a[k | j]) & m;
            a[k | j] ^= t;
            a[k] ^= t << j;
        }
    }
}

__device__ __forceinline__ uint64_t lds64(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void sts64(uint32_t addr, uint64_t v)
{
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

constexpr uint32_t kPlaneStride = kThreads * 8;  // bytes between planes of one thread

__host__ __device__ constexpr size_t sliced_smem_for(uint32_t M)
{
    return sizeof(uint64_t) * (size_t)(M + 1) * kThreads + sizeof(uint32_t) * 8 * 32 * 33 +
           sizeof(SlicedStep) * kSlicedChunk + 8 * 32 * 33;
}

// One CTA: outputs [cbase, cbase + kSlicedOutputs) of a bit-sliced pass.
// Every thread of the CTA must call it (it synchronises the CTA).  With MAP
// the source rows x(i) themselves are written to out (64-bit integers, the
// row array of the product, Sec. 2h) instead of gathering amplitudes.
template <int B, bool WIDE, bool MAP = false, bool FILL64 = true>
__device__ void sliced_chunk(const char *__restrict__ in, char *__restrict__ out, uint32_t M,
                             uint64_t n, const SlicedStep *__restrict__ steps, uint32_t nsteps,
                             uint64_t cbase, unsigned char *smem, double *__restrict__ probs)
{
    using A = typename AmpOf<B>::T;
    // planes: [M + 1][kThreads] u64 ; table: [8 warps][32][33] u32 ;
    // step chunk: kSlicedChunk SlicedStep ; hi: [8][32][33] u8 (WIDE)
    static_assert(kSlicedThreads == kThreads, "plane offsets assume kThreads threads");
    uint64_t *planes = reinterpret_cast<uint64_t *>(smem);
    uint32_t *tabs = reinterpret_cast<uint32_t *>(planes + (size_t)(M + 1) * kThreads);
    SlicedStep *chunk = reinterpret_cast<SlicedStep *>(tabs + 8 * 32 * 33);
    uint8_t *his = reinterpret_cast<uint8_t *>(chunk + kSlicedChunk);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *tab = tabs + warp * 32 * 33;
    uint8_t *hi = his + warp * 32 * 33;
    const A *src = reinterpret_cast<const A *>(in);
    A *dst = reinterpret_cast<A *>(out);
    const uint32_t pbase = smem_addr(planes) + tid * 8;  // this thread's plane 0

    const uint64_t my = cbase + (uint64_t)tid * 64;
    // bits 0..5 enumerate j; higher bits are those of 'my'
    const uint64_t pat[6] = {0xaaaaaaaaaaaaaaaaull, 0xccccccccccccccccull,
                             0xf0f0f0f0f0f0f0f0ull, 0xff00ff00ff00ff00ull,
                             0xffff0000ffff0000ull, 0xffffffff00000000ull};
    __syncthreads();  // the previous user of this shared memory is done
#pragma unroll
    for (uint32_t b = 0; b < 6; ++b)
        if (b < M) sts64(pbase + b * kPlaneStride, pat[b]);
    for (uint32_t b = 6; b < M; ++b)
        sts64(pbase + b * kPlaneStride, ((my >> b) & 1ull) ? ~0ull : 0ull);
    sts64(pbase + M * kPlaneStride, ~0ull);  // the all-ones plane
    for (int64_t s_end = (int64_t)nsteps; s_end > 0; s_end -= kSlicedChunk) {
        const int64_t s_beg = s_end > kSlicedChunk ? s_end - kSlicedChunk : 0;
        const int cn = (int)(s_end - s_beg);
        __syncthreads();
        for (int i = tid; i < cn; i += kThreads) chunk[i] = steps[s_beg + i];
        __syncthreads();
#pragma unroll 2
        for (int q = cn - 1; q >= 0; --q) {
            const uint4 d = *reinterpret_cast<const uint4 *>(&chunk[q]);
            // d.x: target | nc << 8 | neg << 16 | slow << 24 ; d.y, d.z: control planes
            const uint32_t ta = pbase + (d.x & 0xffu) * kPlaneStride;
            uint64_t m;
            if (!(d.x >> 24)) {
                m = lds64(pbase + (d.y & 0xffu) * kPlaneStride) &
                    lds64(pbase + ((d.y >> 8) & 0xffu) * kPlaneStride);
            } else {
                const uint32_t nc = (d.x >> 8) & 0xffu, neg = (d.x >> 16) & 0xffu;
                m = ~0ull;
                for (uint32_t c = 0; c < nc; ++c) {
                    const uint32_t cp = ((c < 4 ? d.y : d.z) >> (8 * (c & 3))) & 0xffu;
                    const uint64_t v = lds64(pbase + cp * kPlaneStride);
                    m &= ((neg >> c) & 1u) ? ~v : v;
                }
            }
            sts64(ta, lds64(ta) ^ m);
        }
    }
    // planes -> 64 source indices, 32 at a time, exchanged for coalesced stores
    const uint64_t wbase = cbase + (uint64_t)warp * 32 * 64;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        uint32_t r[32];
#pragma unroll
        for (int b = 0; b < 32; ++b)
            r[b] = (b < (int)M) ? (uint32_t)(lds64(pbase + b * kPlaneStride) >> (32 * half)) : 0u;
        transpose32(r);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; ++j) tab[lane * 33 + j] = r[j];
        if (WIDE) {
            const uint32_t w32 = (M > 32) ? (uint32_t)(lds64(pbase + 32 * kPlaneStride) >> (32 * half)) : 0u;
            const uint32_t w33 = (M > 33) ? (uint32_t)(lds64(pbase + 33 * kPlaneStride) >> (32 * half)) : 0u;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                hi[lane * 33 + j] = (uint8_t)(((w32 >> j) & 1u) | (((w33 >> j) & 1u) << 1));
        }
        __syncwarp();
        // row e of the table holds lane e's indices my_e + 32 half + (0..31)
#pragma unroll 1
        for (int e0 = 0; e0 < 32; e0 += 8) {
            A v[8];
            uint64_t o[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u;
                o[u] = wbase + (uint64_t)e * 64 + 32 * half + lane;
                uint64_t x = tab[e * 33 + lane];
                if (WIDE) x |= (uint64_t)hi[e * 33 + lane] << 32;
                if (MAP) {
                    if (o[u] < n) reinterpret_cast<uint64_t *>(out)[o[u]] = x;
                } else if (o[u] < n) {
                    v[u] = ld_row<FILL64>(&src[x]);
                }
            }
            if (!MAP) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (o[u] < n) {
                        if (dst) dst[o[u]] = v[u];  // no destination: probabilities only
                        if (probs) probs[o[u]] = amp_prob(v[u]);
                    }
            }
        }
    }
    __syncwarp();
}

template <int B, bool WIDE>
__global__ void __launch_bounds__(kThreads, 2) gather_sliced_kernel(
    const char *__restrict__ in, char *__restrict__ out, uint32_t M, uint64_t n,
    const SlicedStep *__restrict__ steps, uint32_t nsteps, double *__restrict__ probs)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint64_t per_iter = (uint64_t)gridDim.x * kSlicedOutputs;
    // the loop bound is uniform over the CTA, so the barriers inside are safe
    for (uint64_t cbase = (uint64_t)blockIdx.x * kSlicedOutputs; cbase < n; cbase += per_iter)
        sliced_chunk<B, WIDE>(in, out, M, n, steps, nsteps, cbase, smem, probs);
}

// Row array of the product of a step list: rows[i] = x(i) for every output
// row i (the array the paper keeps, Sec. 2h), evaluated bit-sliced.
template <bool WIDE>
__global__ void __launch_bounds__(kThreads, 2) row_array_kernel(uint64_t *__restrict__ rows,
                                                                 uint32_t M, uint64_t n,
                                                                 const SlicedStep *__restrict__ steps,
                                                                 uint32_t nsteps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint64_t per_iter = (uint64_t)gridDim.x * kSlicedOutputs;
    for (uint64_t cbase = (uint64_t)blockIdx.x * kSlicedOutputs; cbase < n; cbase += per_iter)
        sliced_chunk<8, WIDE, true>(nullptr, reinterpret_cast<char *>(rows), M, n, steps, nsteps,
                                    cbase, smem, nullptr);
}

// ============================================================================
// (c) coset-blocked affine gather: coalesced reads and writes
// ============================================================================

// A CTA owns groups of 2^e coset tiles (see GatherPass): a producer warp
// loads each tile's 2^d source runs of 2^r amplitudes with bulk-async copies
// into one pipeline stage; 16 consumer warps write the tile's 2^d output runs,
// each output taking its source from the stage through the pass's local
// permutation (plus the tile's low-bit offset).  Every global access is part
// of an aligned run of 2^r amplitudes.
constexpr int kCosetMaxGroup = 64;  // tiles per stage

struct CosetKParams {
    const char *in;
    char *out;
    double *probs;                 // non-null: also write FP64 probabilities
    int *err;
    const uint64_t *tabs;          // out-base [ctb][256], source-base [ctb][256], dstrun, srcrun, perm
    uint64_t n_groups;             // tiles / 2^e
    uint64_t bvec;
    uint32_t r, d, e, ctb, stages, wait_limit;
};

struct CosetStageMeta {
    uint64_t ob[kCosetMaxGroup];   // output base of each tile
    uint64_t sb[kCosetMaxGroup];   // source base of each tile (with its low bits)
    uint32_t end;                  // no more groups
    uint32_t pad;
};

template <int B, bool PROBS>
__global__ void __launch_bounds__(kTileThreads + 32, 1) gather_coset_kernel(CosetKParams p)
{
    using A = typename AmpOf<B>::T;
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t rd = p.r + p.d;
    const uint32_t G = 1u << p.e;
    const size_t stage_bytes = (size_t)B << (rd + p.e);
    const uint32_t nd = 1u << p.d;
    char *bufs = reinterpret_cast<char *>(smem);
    CosetStageMeta *meta = reinterpret_cast<CosetStageMeta *>(smem + stage_bytes * p.stages);
    uint64_t *full = reinterpret_cast<uint64_t *>(meta + p.stages);
    uint64_t *empty = full + p.stages;
    uint64_t *dstrun = empty + p.stages;
    uint64_t *srcrun = dstrun + nd;
    uint16_t *perm = reinterpret_cast<uint16_t *>(srcrun + nd);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nthreads = kTileThreads + 32;
    const uint64_t *g_dst = p.tabs + 512 * p.ctb;
    for (uint32_t i = tid; i < 2 * nd; i += nthreads) dstrun[i] = g_dst[i];  // dstrun, srcrun
    const uint16_t *g_perm = reinterpret_cast<const uint16_t *>(g_dst + 2 * nd);
    for (uint32_t i = tid; i < (1u << rd); i += nthreads) perm[i] = g_perm[i];
    if (tid == 0) {
        for (uint32_t s = 0; s < p.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kTileThreads / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const uint64_t per = (p.n_groups + gridDim.x - 1) / gridDim.x;
    const uint64_t begin = (uint64_t)blockIdx.x * per;
    const uint64_t end = begin + per < p.n_groups ? begin + per : p.n_groups;
    const uint64_t low = (1ull << p.r) - 1ull;

    if (warp == kTileThreads / 32) {
        // ---------------- producer warp ----------------
        const uint32_t run_bytes = (uint32_t)B << p.r;
        const uint64_t *tout = p.tabs, *tsrc = p.tabs + 256 * p.ctb;
        for (uint32_t it = 0;; ++it) {
            const uint32_t s = it % p.stages;
            if (it >= p.stages && !mbar_wait_bounded(&empty[s], ((it / p.stages) - 1) & 1u, p.wait_limit)) {
                if (lane == 0) atomicOr(p.err, 2);
                return;
            }
            const uint64_t g = begin + it;
            if (g >= end) {
                if (lane == 0) {
                    meta[s].end = 1;
                    mbar_arrive(&full[s]);  // end marker, no bytes
                }
                return;
            }
            for (uint32_t q = lane; q < G; q += 32) {
                const uint64_t t = (g << p.e) | q;
                uint64_t ob = 0, sb = p.bvec;
                for (uint32_t k = 0; k < p.ctb; ++k) {
                    const uint32_t v = (uint32_t)((t >> (8 * k)) & 255u);
                    ob ^= __ldg(tout + 256 * k + v);
                    sb ^= __ldg(tsrc + 256 * k + v);
                }
                meta[s].ob[q] = ob;
                meta[s].sb[q] = sb;
            }
            if (lane == 0) meta[s].end = 0;
            __syncwarp();
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)stage_bytes);
            __syncwarp();
            char *buf = bufs + stage_bytes * s;
            for (uint32_t idx = lane; idx < (G << p.d); idx += 32) {
                const uint32_t q = idx >> p.d, gam = idx & (nd - 1);
                const uint64_t run = (meta[s].sb[q] & ~low) ^ srcrun[gam];
                bulk_g2s(buf + (size_t)idx * run_bytes, p.in + run * B, run_bytes, &full[s]);
            }
        }
    }

    // ---------------- consumer warps ----------------
    A *dst = reinterpret_cast<A *>(p.out);
    const uint32_t nloc = 1u << rd;
    const uint32_t total = G << rd;
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % p.stages;
        if (!mbar_wait_bounded(&full[s], (it / p.stages) & 1u, p.wait_limit)) {
            if (tid == 0) atomicOr(p.err, 1);
            return;
        }
        if (meta[s].end) break;
        const A *buf = reinterpret_cast<const A *>(bufs + stage_bytes * s);
        for (uint32_t j0 = 0; j0 < total; j0 += kTileThreads * 4) {
            A v[4];
            uint64_t o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t j = j0 + tid + u * kTileThreads;
                if (j < total) {
                    const uint32_t q = j >> rd, jj = j & (nloc - 1);
                    const uint64_t sb = meta[s].sb[q];
                    v[u] = buf[((uint32_t)q << rd) | (perm[jj] ^ (uint32_t)(sb & low))];
                    o[u] = (meta[s].ob[q] ^ dstrun[jj >> p.r]) | (jj & low);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t j = j0 + tid + u * kTileThreads;
                if (j < total) {
                    dst[o[u]] = v[u];
                    if (PROBS) p.probs[o[u]] = amp_prob(v[u]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
    }
}

// ============================================================================
// gather by a stored row array: k2(i) = k1(x(i)) (Sec. 2b), x given
// ============================================================================

// Each thread keeps U source reads in flight: U coalesced row-array reads,
// then U reads of single amplitudes at those rows, then U coalesced stores.
// Rows are taken modulo 2^M.  With the row array of a circuit this is the
// same random-read pattern as that circuit's gather pass, with no index
// arithmetic.
template <int B, int U>
__global__ void __launch_bounds__(kThreads) gather_rows_kernel(const char *__restrict__ in,
                                                               char *__restrict__ out,
                                                               const uint64_t *__restrict__ rows,
                                                               uint64_t n, double *__restrict__ probs)
{
    using A = typename AmpOf<B>::T;
    const A *src = reinterpret_cast<const A *>(in);
    A *dst = reinterpret_cast<A *>(out);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i0 < n; i0 += U * stride) {
        uint64_t x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = i0 + u * stride;
            x[u] = i < n ? (__ldcs(rows + i) & (n - 1)) : 0;
        }
        A v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * stride < n) v[u] = ld_row<true>(&src[x[u]]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = i0 + u * stride;
            if (i < n) {
                dst[i] = v[u];
                if (probs) probs[i] = amp_prob(v[u]);
            }
        }
    }
}

// Sweep of pair indices [q0, q1) of one step (in place).
template <int B>
__device__ __forceinline__ void sweep_range(char *__restrict__ state, const SweepParams &p,
                                            uint64_t q0, uint64_t q1, uint64_t step)
{
    using A = typename AmpOf<B>::T;
    A *st = reinterpret_cast<A *>(state);
    for (uint64_t q = q0; q < q1; q += step) {
        uint64_t j = q;
        for (uint32_t s = 0; s < p.nins; ++s) j = insert_zero(j, p.ins[s]);
        j |= p.pol;
        const A a = st[j];
        const A b = st[j + p.half];
        st[j] = b;
        st[j + p.half] = a;
    }
}

// ============================================================================
// batched execution: one persistent launch over the passes of many circuits
// ============================================================================

// Affine gather in coset-tile order: position p of the pass names local
// output p mod 2^(r+d) of coset tile p >> (r+d) (see GatherPass).  A work
// item covers whole tiles, so all reads of a tile's aligned source runs come
// from one CTA within microseconds and every DRAM burst fetched is used in
// full from L2, with no staging.
template <int B>
__device__ __forceinline__ void coset_order_range(const BatchPass &P, uint64_t p0, uint64_t p1,
                                                  uint64_t step)
{
    using A = typename AmpOf<B>::T;
    const A *src = reinterpret_cast<const A *>(P.in);
    A *dst = reinterpret_cast<A *>(P.out);
    const uint32_t rd = P.cr + P.cd;
    const uint64_t low = (1ull << P.cr) - 1ull;
    const uint64_t *tout = P.tables, *tsrc = P.tables + 256 * P.ctb;
    const uint64_t *dstrun = P.tables + 512 * P.ctb, *srcrun = dstrun + (1u << P.cd);
    const uint16_t *perm = reinterpret_cast<const uint16_t *>(srcrun + (1u << P.cd));
    for (uint64_t q0 = p0; q0 < p1; q0 += 4 * step) {
        A v[4];
        uint64_t o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t q = q0 + u * step;
            if (q < p1) {
                const uint64_t t = q >> rd;
                const uint32_t jj = (uint32_t)(q & ((1ull << rd) - 1ull));
                uint64_t ob = 0, sb = P.bvec;
                for (uint32_t k = 0; k < P.ctb; ++k) {
                    const uint32_t b = (uint32_t)((t >> (8 * k)) & 255u);
                    ob ^= __ldg(tout + 256 * k + b);
                    sb ^= __ldg(tsrc + 256 * k + b);
                }
                const uint32_t loc = __ldg(perm + jj);
                const uint64_t s = ((sb & ~low) ^ __ldg(srcrun + (loc >> P.cr))) | ((loc & low) ^ (sb & low));
                o[u] = (ob ^ __ldg(dstrun + (jj >> P.cr))) | (jj & low);
                v[u] = __ldg(src + s);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q0 + u * step < p1) {
                if (dst) dst[o[u]] = v[u];
                if (P.probs) P.probs[o[u]] = amp_prob(v[u]);
            }
    }
}

// CTAs take work items (a range of outputs of one circuit's pass) from a
// global counter until the level's list is exhausted; the affine tables of
// the last circuit served stay in shared memory.
template <int B, bool WIDE>
__global__ void __launch_bounds__(kThreads) batch_kernel(const BatchPass *__restrict__ passes,
                                                         const BatchItem *__restrict__ items,
                                                         uint32_t n_items, uint32_t *counter)
{
    using I = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ int32_t s_tables;  // pass whose affine tables are loaded, -1 none
    I *tab = reinterpret_cast<I *>(smem);
    if (threadIdx.x == 0) s_tables = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= n_items) break;
        const BatchItem item = items[it];
        const BatchPass &P = passes[item.pass];
        const uint64_t o1 = item.start + item.count;
        if (P.kind == 3) {
            if (s_tables != (int32_t)item.pass) {
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < P.nbytes * 256; i += kThreads) tab[i] = (I)P.tables[i];
                __syncthreads();
                if (threadIdx.x == 0) s_tables = (int32_t)item.pass;
            }
            affine_range<B, WIDE, I, false>(P.in, P.out, item.start + threadIdx.x, o1, kThreads, tab,
                                     P.nbytes, P.bvec, P.probs);
        } else if (P.kind == 4) {
            if (threadIdx.x == 0) s_tables = -1;
            sliced_chunk<B, WIDE, false, false>(P.in, P.out, P.M, o1, P.steps, P.nsteps, item.start, smem,
                                                P.probs);
        } else if (P.kind == 7) {
            coset_order_range<B>(P, item.start + threadIdx.x, o1, kThreads);
        } else {
            sweep_range<B>(P.out, P.sweep, item.start + threadIdx.x, o1, kThreads);
        }
    }
}

// ============================================================================
// FP64 probabilities and norm
// ============================================================================

// ============================================================================
// product-state input (App. 1): k1(i) = product over qubits of q_b(bit b of i)
// ============================================================================

// Complex product with each real product and sum rounded separately.
__device__ __forceinline__ double2 cmul_rn(double2 a, double2 b)
{
    return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                        __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}

// Product of the factors of bits [lo, hi) of index i, most significant
// first; q holds (q_b(0), q_b(1)) for each bit b.
__device__ __forceinline__ double2 partial_product(const double2 *q, uint64_t i, int lo, int hi)
{
    double2 acc = q[2 * (hi - 1) + ((i >> (hi - 1)) & 1ull)];
    for (int b = hi - 2; b >= lo; --b) acc = cmul_rn(acc, q[2 * b + ((i >> b) & 1ull)]);
    return acc;
}

constexpr int kProductLowBits = 10;   // low-bit partial products: one table per CTA
constexpr int kProductGroupBits = 8;  // high bits in three groups of up to 8: three tables

// k1(i) = (product over the high bits) x (product over the low h bits).  Each
// CTA tabulates the low-bit partial products (2^h) and the partial products
// of three groups of high bits (2^8 each) in FP64, kept as ProdT (complex64:
// float-float, so the per-amplitude work is FP32; complex128: FP64).  Each
// warp takes runs of 2^h consecutive amplitudes: the run's high product is
// two table products, then every amplitude one product with the low table.
template <int B>
__global__ void __launch_bounds__(kThreads) product_state_kernel(char *__restrict__ state,
                                                                 const double *__restrict__ qubits,
                                                                 uint32_t M, uint64_t n)
{
    using PT = typename ProdT<B>::T;
    __shared__ double2 q[2 * QSIM_MAX_QUBITS];
    __shared__ PT lo_tab[1 << kProductLowBits];
    __shared__ PT grp[3][1 << kProductGroupBits];
    const int h = M < (uint32_t)kProductLowBits ? (int)M : kProductLowBits;
    for (uint32_t j = threadIdx.x; j < 2 * M; j += kThreads)
        q[j] = make_double2(qubits[2 * j], qubits[2 * j + 1]);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < (1u << h); j += kThreads) lo_tab[j] = ProdT<B>::of(partial_product(q, j, 0, h));
    for (uint32_t e = threadIdx.x; e < 3u << kProductGroupBits; e += kThreads) {
        const int g = (int)(e >> kProductGroupBits);
        const uint32_t j = e & ((1u << kProductGroupBits) - 1u);
        const int lo = h + kProductGroupBits * g;
        const int hi = lo + kProductGroupBits < (int)M ? lo + kProductGroupBits : (int)M;
        grp[g][j] = ProdT<B>::of(lo < hi ? partial_product(q, (uint64_t)j << lo, lo, hi) : make_double2(1.0, 0.0));
    }
    __syncthreads();
    const uint32_t warps = kThreads / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint64_t runs = n >> h;
    const uint32_t gm = (1u << kProductGroupBits) - 1u;
    for (uint64_t r = (uint64_t)blockIdx.x * warps + warp; r < runs; r += (uint64_t)gridDim.x * warps) {
        PT hv = ProdT<B>::scale(grp[0][r & gm], grp[1][(r >> kProductGroupBits) & gm]);
        hv = ProdT<B>::scale(hv, grp[2][(r >> (2 * kProductGroupBits)) & gm]);
        for (uint32_t j = lane; j < (1u << h); j += 32) {
            auto v = ProdT<B>::mul(hv, lo_tab[j]);
            reinterpret_cast<decltype(v) *>(state)[(r << h) | j] = v;
        }
    }
}

constexpr int kProbBlocks = 1024;

template <int B>
__device__ __forceinline__ double prob_of(const char *__restrict__ state, uint64_t i)
{
    using A = typename AmpOf<B>::T;
    return amp_prob(__ldcs(reinterpret_cast<const A *>(state) + i));
}

template <int B, bool NORM>
__global__ void __launch_bounds__(kThreads) probs_kernel(const char *__restrict__ state,
                                                         double *__restrict__ probs, uint64_t n,
                                                         double *__restrict__ partials)
{
    __shared__ double red[kThreads];
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {  // four independent loads in flight
        double p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = prob_of<B>(state, i + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (probs) __stcs(probs + i + u * stride, p[u]);
            if (NORM) acc += p[u];
        }
    }
    for (; i < n; i += stride) {
        const double p = prob_of<B>(state, i);
        if (probs) __stcs(probs + i, p);
        if (NORM) acc += p;
    }
    if (!NORM) return;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// complex64 probabilities without the norm: two amplitudes per 16-byte load
// and two probabilities per 16-byte store, eight amplitudes in flight per
// thread (the same arithmetic as probs_kernel, amplitude by amplitude).
__global__ void __launch_bounds__(kThreads) probs_pairs_kernel(const uint4 *__restrict__ state,
                                                               double2 *__restrict__ probs, uint64_t npairs)
{
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    for (; i + 3 * stride < npairs; i += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(state + i + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            __stcs(probs + i + u * stride, make_double2(qsim_prob_bits(v[u].x, v[u].y), qsim_prob_bits(v[u].z, v[u].w)));
    }
    for (; i < npairs; i += stride) {
        const uint4 v = __ldcs(state + i);
        __stcs(probs + i, make_double2(qsim_prob_bits(v.x, v.y), qsim_prob_bits(v.z, v.w)));
    }
}

__global__ void __launch_bounds__(kThreads) reduce_kernel(const double *__restrict__ partials,
                                                          int n, double *__restrict__ out)
{
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) acc += partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

int g_num_sms = 0;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace

int num_sms()
{
    if (g_num_sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_num_sms = v > 0 ? v : 1;
    }
    return g_num_sms;
}

// ---- launchers --------------------------------------------------------------

int launch_sweep(void *state, int amp_bytes, const SweepParams &p, int * /*d_err*/, void *stream)
{
    if (p.n_pairs == 0) return cudaSuccess;
    // complex64: bit 0 is the target, a control, or free (the lowest
    // insertion is bit 0 exactly when it is the target or a control)
    const bool bit0_listed = p.nins > 0 && p.ins[0] == 0;
    const int mode = amp_bytes == 16 ? 0 : p.half == 1 ? 1 : bit0_listed ? 3 : 2;
    const uint64_t units = mode == 2 ? p.n_pairs / 2 : p.n_pairs;
    const uint64_t want = (units + 2 * kThreads - 1) / (2 * kThreads);
    const uint64_t cap = (uint64_t)num_sms() * 8;
    const int grid = (int)(want < cap ? (want ? want : 1) : cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint4 *st = static_cast<uint4 *>(state);
    switch (mode) {
    case 0: sweep_kernel<0><<<grid, kThreads, 0, s>>>(st, p, units); break;
    case 1: sweep_kernel<1><<<grid, kThreads, 0, s>>>(st, p, units); break;
    case 2: sweep_kernel<2><<<grid, kThreads, 0, s>>>(st, p, units); break;
    default: sweep_kernel<3><<<grid, kThreads, 0, s>>>(st, p, units); break;
    }
    return cudaGetLastError();
}

static uint32_t tile_stages(int amp_bytes, int k)
{
    const size_t tb = (size_t)amp_bytes << k;
    if (tb <= 64 * 1024) return 3;
    return 1;
}

// Stage region of a product-input pass: the products over the low bits and
// over the high bits, and the tile's scaled high products per stage (16 bytes
// an entry for both amplitude types), rounded to 128 bytes.
static size_t product_region_bytes(uint32_t l, uint32_t nh)
{
    const size_t b = 16 * (((size_t)1 << l) + ((size_t)1 << nh) * (1 + kProductStages));
    return (b + 127) / 128 * 128;
}

static size_t tile_smem_for(size_t region, uint32_t st, int k)
{
    return region + sizeof(uint64_t) * (1u << kMaxHighBits) + sizeof(TileStageMeta) * st +
           2 * sizeof(uint64_t) * st + sizeof(TileStep) * kMaxTileSteps + sizeof(uint32_t) * kMaxOutBits +
           sizeof(uint16_t) * ((size_t)1 << k);
}

size_t tile_smem_bytes(int amp_bytes, int k)
{
    const uint32_t st = tile_stages(amp_bytes, k);
    return tile_smem_for(((size_t)amp_bytes << k) * st, st, k);
}

bool tile_product_fits(const TilePass &t)
{
    return tile_smem_for(product_region_bytes(t.l, t.nh), kProductStages, (int)t.k) <= kMaxTileSmem;
}

int encode_tile_map(void *state, const TilePass &t, void *map128)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return 1;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    for (int d = 0; d < 5; ++d) {
        dims[d] = t.tma_dim[d];
        box[d] = t.tma_box[d];
    }
    for (int d = 1; d < 5; ++d) strides[d - 1] = t.tma_stride[d];
    CUresult r = enc(static_cast<CUtensorMap *>(map128), CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, state, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 2;
}

int launch_tile(void *state, int amp_bytes, const TilePass &t, const TileStep *d_steps,
                int *d_err, double *d_probs, void *stream, const WaitTest *wt, const double *d_prod)
{
    TileKParams p;
    const double2 *prod = reinterpret_cast<const double2 *>(d_prod);
    p.qtab = prod;
    p.plow = prod ? prod + 2 * QSIM_MAX_QUBITS : nullptr;
    p.phigh = prod ? p.plow + (1u << t.l) : nullptr;
    p.wait_limit = (wt && wt->poll_limit) ? wt->poll_limit : kWaitLimit;
    p.stall_producer = (wt && wt->stall_producer) ? 1u : 0u;
    p.state = static_cast<char *>(state);
    p.probs = d_probs;
    p.steps = d_steps + t.step_off;
    p.err = d_err;
    p.n_tiles = t.n_tiles;
    p.k = t.k;
    p.l = t.l;
    p.nh = t.nh;
    p.nsteps = t.nsteps;
    p.all_local = t.all_local;
    // a product-input pass loads nothing: its stages hold small tables only
    p.stages = prod ? kProductStages : tile_stages(amp_bytes, (int)t.k);
    p.buf_bytes = (uint32_t)(prod ? product_region_bytes(t.l, t.nh) : ((size_t)amp_bytes << t.k) * p.stages);
    p.nout = t.nout;
    for (int i = 0; i < kMaxHighBits; ++i) p.high[i] = t.high[i];
    for (int i = 0; i < kMaxOutBits; ++i) p.outpos[i] = i < (int)t.nout ? t.outpos[i] : 0u;
    p.tma = t.tma;
    p.affine = t.affine;
    p.nrest = t.nrest;
    p.epa = amp_bytes == 16 ? 2 : 1;
    p.box_bytes = t.box_bytes;
    for (int i = 0; i < 6; ++i) p.start[i] = t.tma_start[i];
    for (int i = 0; i < kMaxHighBits; ++i) p.rest_pos[i] = t.rest_pos[i];
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof(tmap));
    if (t.tma) {
        const int te = encode_tile_map(state, t, &tmap);
        if (te == 1) p.tma = 0;  // no driver entry point: one bulk copy per run
        else if (te != 0) return cudaErrorInvalidValue;
    }
    if (prod && !tile_product_fits(t)) return cudaErrorInvalidValue;
    const size_t smem = prod ? tile_smem_for(p.buf_bytes, p.stages, (int)t.k) : tile_smem_bytes(amp_bytes, (int)t.k);
    const uint64_t cap = (uint64_t)num_sms();
    const int grid = (int)(t.n_tiles < cap ? t.n_tiles : cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    // the pass that writes probabilities is its own instantiation, so the
    // other passes carry no per-amplitude test
    auto run = [&](auto kernel) -> cudaError_t {
        cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        kernel<<<grid, kTileThreads + 32, smem, s>>>(p, tmap);
        return cudaGetLastError();
    };
    if (prod) {
        if (amp_bytes == 8) e = d_probs ? run(tile_kernel<8, true, true>) : run(tile_kernel<8, false, true>);
        else e = d_probs ? run(tile_kernel<16, true, true>) : run(tile_kernel<16, false, true>);
    } else {
        if (amp_bytes == 8) e = d_probs ? run(tile_kernel<8, true, false>) : run(tile_kernel<8, false, false>);
        else e = d_probs ? run(tile_kernel<16, true, false>) : run(tile_kernel<16, false, false>);
    }
    return e;
}

static size_t sliced_smem_bytes(uint32_t M) { return sliced_smem_for(M); }

template <int B, bool W>
static cudaError_t launch_sliced(const void *in, void *out, uint32_t M, uint64_t n,
                                 const SlicedStep *steps, uint32_t nsteps, double *probs,
                                 cudaStream_t s)
{
    const size_t smem = sliced_smem_bytes(M);
    cudaError_t e = cudaFuncSetAttribute(gather_sliced_kernel<B, W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_sliced_kernel<B, W>, kThreads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    const uint64_t chunks = (n + kSlicedOutputs - 1) / kSlicedOutputs;
    const uint64_t cap = (uint64_t)num_sms() * per_sm;
    const int grid = (int)(chunks < cap ? chunks : cap);
    gather_sliced_kernel<B, W><<<grid, kThreads, smem, s>>>(
        static_cast<const char *>(in), static_cast<char *>(out), M, n, steps, nsteps, probs);
    return cudaGetLastError();
}

size_t coset_smem_bytes(int amp_bytes, uint32_t r, uint32_t d, uint32_t e, uint32_t *stages)
{
    const size_t stage = (size_t)amp_bytes << (r + d + e);
    const size_t fixed = 2 * sizeof(uint64_t) * ((size_t)1 << d) + sizeof(uint16_t) * ((size_t)1 << (r + d));
    const size_t per = stage + sizeof(CosetStageMeta) + 2 * sizeof(uint64_t);
    const size_t budget = 200 * 1024;
    uint32_t st = (uint32_t)((budget - fixed) / per);
    st = st > 8 ? 8 : st;
    if (st < 1) st = 1;
    if (stages) *stages = st;
    return per * st + fixed;
}

static int launch_coset(const void *in, void *out, int amp_bytes, const GatherPass &g,
                        const uint64_t *d_tables, int *d_err, double *d_probs, cudaStream_t s,
                        uint32_t wait_limit)
{
    CosetKParams p;
    p.in = static_cast<const char *>(in);
    p.out = static_cast<char *>(out);
    p.probs = d_probs;
    p.err = d_err;
    p.tabs = d_tables + g.coset_off;
    p.n_groups = g.n_tiles >> g.ce;
    p.bvec = g.bvec;
    p.r = g.cr;
    p.d = g.cd;
    p.e = g.ce;
    p.ctb = g.ctb;
    p.wait_limit = wait_limit ? wait_limit : kWaitLimit;
    const size_t smem = coset_smem_bytes(amp_bytes, g.cr, g.cd, g.ce, &p.stages);
    const uint64_t cap = (uint64_t)num_sms();
    const int grid = (int)(p.n_groups < cap ? p.n_groups : cap);
    auto run = [&](auto kernel) -> cudaError_t {
        cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        kernel<<<grid, kTileThreads + 32, smem, s>>>(p);
        return cudaGetLastError();
    };
    if (amp_bytes == 8) return d_probs ? run(gather_coset_kernel<8, true>) : run(gather_coset_kernel<8, false>);
    return d_probs ? run(gather_coset_kernel<16, true>) : run(gather_coset_kernel<16, false>);
}

int launch_gather(const void *in, void *out, int amp_bytes, uint32_t M, const GatherPass &g,
                  const uint64_t *d_tables, const SlicedStep *d_steps, int *d_err,
                  double *d_probs, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t n = 1ull << M;
    if (g.affine && g.coset) return launch_coset(in, out, amp_bytes, g, d_tables, d_err, d_probs, s, 0);
    if (g.affine) {
        const uint64_t want = (n + kThreads * 4 - 1) / (kThreads * 4);
        const uint64_t cap = (uint64_t)num_sms() * 8;
        const int grid = (int)(want < cap ? want : cap);
        const uint64_t *tab = d_tables + g.table_off;
        const char *i = static_cast<const char *>(in);
        char *o = static_cast<char *>(out);
        if (amp_bytes == 8) {
            if (M > 32)
                gather_affine_kernel<8, true><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec, d_probs);
            else
                gather_affine_kernel<8, false><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec, d_probs);
        } else {
            if (M > 32)
                gather_affine_kernel<16, true><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec, d_probs);
            else
                gather_affine_kernel<16, false><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec, d_probs);
        }
        return cudaGetLastError();
    }
    const SlicedStep *st = d_steps + g.step_off;
    if (amp_bytes == 8)
        return M > 32 ? launch_sliced<8, true>(in, out, M, n, st, g.nsteps, d_probs, s)
                      : launch_sliced<8, false>(in, out, M, n, st, g.nsteps, d_probs, s);
    return M > 32 ? launch_sliced<16, true>(in, out, M, n, st, g.nsteps, d_probs, s)
                  : launch_sliced<16, false>(in, out, M, n, st, g.nsteps, d_probs, s);
}

int launch_gather_rows(const void *in, void *out, const uint64_t *rows, int amp_bytes, uint32_t M,
                       double *d_probs, int loads_in_flight, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t n = 1ull << M;
    const int U = loads_in_flight;
    const uint64_t want = (n + (uint64_t)kThreads * U - 1) / ((uint64_t)kThreads * U);
    const uint64_t cap = (uint64_t)num_sms() * 8;
    const int grid = (int)(want < cap ? (want ? want : 1) : cap);
    const char *i = static_cast<const char *>(in);
    char *o = static_cast<char *>(out);
#define QSIM_ROWS(BB, UU) gather_rows_kernel<BB, UU><<<grid, kThreads, 0, s>>>(i, o, rows, n, d_probs)
    if (amp_bytes == 8) {
        if (U == 4) QSIM_ROWS(8, 4); else if (U == 8) QSIM_ROWS(8, 8); else QSIM_ROWS(8, 16);
    } else {
        if (U == 4) QSIM_ROWS(16, 4); else if (U == 8) QSIM_ROWS(16, 8); else QSIM_ROWS(16, 16);
    }
#undef QSIM_ROWS
    return cudaGetLastError();
}

int probabilities_partials_needed() { return kProbBlocks; }

int launch_probabilities(const void *state, int amp_bytes, uint64_t n, double *d_probs,
                         double *d_partials, int n_partials, double *d_norm, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char *st = static_cast<const char *>(state);
    // complex64, probabilities only, both buffers on 16-byte boundaries (a
    // caller's d_probs need only be 8-byte aligned)
    if (!d_norm && amp_bytes == 8 && n >= 2 && n % 2 == 0 && d_probs &&
        (reinterpret_cast<uintptr_t>(st) & 15u) == 0 && (reinterpret_cast<uintptr_t>(d_probs) & 15u) == 0) {
        const uint64_t np = n / 2;
        const uint64_t want = (np + kThreads * 4 - 1) / (kThreads * 4);
        const uint64_t cap = (uint64_t)num_sms() * 16;
        const int grid = (int)(want < cap ? (want ? want : 1) : cap);
        probs_pairs_kernel<<<grid, kThreads, 0, s>>>(reinterpret_cast<const uint4 *>(st),
                                                     reinterpret_cast<double2 *>(d_probs), np);
        return cudaGetLastError();
    }
    if (!d_norm) {  // probabilities only: no accumulation, no reduction
        const uint64_t want = (n + kThreads * 4 - 1) / (kThreads * 4);
        const uint64_t cap = (uint64_t)num_sms() * 16;
        const int grid = (int)(want < cap ? (want ? want : 1) : cap);
        if (amp_bytes == 8)
            probs_kernel<8, false><<<grid, kThreads, 0, s>>>(st, d_probs, n, nullptr);
        else
            probs_kernel<16, false><<<grid, kThreads, 0, s>>>(st, d_probs, n, nullptr);
        return cudaGetLastError();
    }
    const uint64_t want = (n + kThreads - 1) / kThreads;
    uint64_t grid = want < (uint64_t)n_partials ? want : (uint64_t)n_partials;
    if (grid < 1) grid = 1;
    if (amp_bytes == 8)
        probs_kernel<8, true><<<(int)grid, kThreads, 0, s>>>(st, d_probs, n, d_partials);
    else
        probs_kernel<16, true><<<(int)grid, kThreads, 0, s>>>(st, d_probs, n, d_partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_kernel<<<1, kThreads, 0, s>>>(d_partials, (int)grid, d_norm);
    return cudaGetLastError();
}

size_t batch_smem_bytes(uint32_t max_sliced_M)
{
    const size_t tabs = 5 * 256 * sizeof(uint64_t);
    const size_t sl = max_sliced_M ? sliced_smem_for(max_sliced_M) : 0;
    return tabs > sl ? tabs : sl;
}

template <int B, bool W>
static cudaError_t launch_batch_t(const BatchPass *passes, const BatchItem *items, uint32_t n_items,
                                  uint32_t *counter, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<B, W>, kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const uint64_t cap = (uint64_t)num_sms() * per_sm;
    const int grid = (int)(n_items < cap ? n_items : cap);
    if (grid < 1) return cudaSuccess;
    batch_kernel<B, W><<<grid, kThreads, smem, s>>>(passes, items, n_items, counter);
    return cudaGetLastError();
}

int launch_batch_level(int amp_bytes, bool wide, const BatchPass *d_passes, const BatchItem *d_items,
                       uint32_t n_items, uint32_t *d_counter, size_t smem, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (amp_bytes == 8)
        return wide ? launch_batch_t<8, true>(d_passes, d_items, n_items, d_counter, smem, s)
                    : launch_batch_t<8, false>(d_passes, d_items, n_items, d_counter, smem, s);
    return wide ? launch_batch_t<16, true>(d_passes, d_items, n_items, d_counter, smem, s)
                : launch_batch_t<16, false>(d_passes, d_items, n_items, d_counter, smem, s);
}

int launch_product_state(void *state, int amp_bytes, uint32_t M, const double *d_qubits, void *stream)
{
    const uint64_t n = 1ull << M;
    const int h = M < (uint32_t)kProductLowBits ? (int)M : kProductLowBits;
    if ((int)M > h + 3 * kProductGroupBits) return cudaErrorInvalidValue;
    const uint64_t runs = n >> h;
    const uint64_t warps = (runs + kThreads / 32 - 1) / (kThreads / 32);
    const uint64_t cap = (uint64_t)num_sms() * 8;
    const int grid = (int)(warps < cap ? warps : cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (amp_bytes == 8)
        product_state_kernel<8><<<grid, kThreads, 0, s>>>(static_cast<char *>(state), d_qubits, M, n);
    else
        product_state_kernel<16><<<grid, kThreads, 0, s>>>(static_cast<char *>(state), d_qubits, M, n);
    return cudaGetLastError();
}

int launch_row_array(uint64_t *d_rows, uint32_t M, const SlicedStep *d_steps, uint32_t nsteps,
                     void *stream)
{
    const uint64_t n = 1ull << M;
    const size_t smem = sliced_smem_for(M);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t chunks = (n + kSlicedOutputs - 1) / kSlicedOutputs;
    const uint64_t cap = (uint64_t)num_sms() * 2;
    const int grid = (int)(chunks < cap ? chunks : cap);
    cudaError_t e;
    if (M > 32) {
        e = cudaFuncSetAttribute(row_array_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) row_array_kernel<true><<<grid, kThreads, smem, s>>>(d_rows, M, n, d_steps, nsteps);
    } else {
        e = cudaFuncSetAttribute(row_array_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) row_array_kernel<false><<<grid, kThreads, smem, s>>>(d_rows, M, n, d_steps, nsteps);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace qsim
