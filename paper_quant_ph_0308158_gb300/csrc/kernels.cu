// kernels.cu -- sm_103a kernels of the reversible wiring-diagram engine.
//
// Every kernel only moves amplitudes (8-byte complex64 or 16-byte
// complex128 words); index arithmetic is integer.  The one floating-point
// kernel is the FP64 probability / norm reduction.
//
//   sweep_kernel          one step in place over the toggled pairs only
//                         (Sec. 2b 'intelligent looping').
//   tile_kernel           a run of steps on 2^k-amplitude tiles staged in
//                         shared memory by bulk-async (TMA) copies, in place
//                         (Sec. 2i: sequential steps processed together).
//   gather_affine_kernel  k2(i) = k1(A i ^ b) for CNOT/NOT segments
//                         (Sec. 2h product of the steps, Sec. 2b gather).
//   gather_sliced_kernel  k2(i) = k1(x(i)) with x(i) evaluated for 32 output
//                         indices at once in bit-sliced form, steps applied
//                         last to first (Sec. 2h product, Sec. 2b gather).
//   probs_kernel          p(i) = re^2 + im^2 in FP64 and a norm partial sum.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "qsim_internal.h"

namespace qsim {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kWaitLimit = 1u << 24;  // bounded mbarrier polls (seconds)

template <int B> struct AmpOf;
template <> struct AmpOf<8> { using T = uint2; };
template <> struct AmpOf<16> { using T = uint4; };

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

template <int B>
__global__ void __launch_bounds__(kThreads) sweep_kernel(char *__restrict__ state, SweepParams p)
{
    using A = typename AmpOf<B>::T;
    A *st = reinterpret_cast<A *>(state);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t q = (uint64_t)blockIdx.x * kThreads + threadIdx.x; q < p.n_pairs; q += stride) {
        uint64_t j = q;
#pragma unroll 1
        for (uint32_t s = 0; s < p.nins; ++s) j = insert_zero(j, p.ins[s]);
        j |= p.pol;
        const A a = st[j];
        const A b = st[j + p.half];
        st[j] = b;
        st[j + p.half] = a;
    }
}

// ============================================================================
// (b) tile pass: TMA bulk loads into shared memory, in-tile permutation,
//     in-place stores
// ============================================================================

struct TileKParams {
    char *state;
    const TileStep *steps;
    int *err;
    uint64_t n_tiles;
    uint32_t k, l, nh, nsteps, all_local, stages;
    uint32_t high[kMaxHighBits];
};

struct TileStageMeta {
    uint64_t base;  // global index of local index 0; ~0 = no tile
    int32_t cnt;    // active steps
    int32_t pad;
};

constexpr uint64_t kNoTile = ~0ull;

__device__ __forceinline__ uint64_t tile_base(uint64_t tile, const TileKParams &p)
{
    uint64_t b = tile << p.l;
    for (uint32_t q = 0; q < p.nh; ++q) b = insert_zero(b, p.high[q]);
    return b;
}

// Warp 0: pick this CTA's next tile that has an active step, record its
// active steps (in order), arm the stage barrier and issue one bulk copy per
// contiguous run of 2^l amplitudes.
template <int B>
__device__ uint64_t tile_produce(const TileKParams &p, int s, uint64_t next, char *buf,
                                 const uint64_t *depo, TileStageMeta *meta, uint2 *list,
                                 const TileStep *steps_sm, uint64_t *bar)
{
    const int lane = threadIdx.x & 31;
    uint64_t base = kNoTile;
    int cnt = 0;
    while (next < p.n_tiles) {
        base = tile_base(next, p);
        next += gridDim.x;
        if (p.all_local) {
            cnt = (int)p.nsteps;
            break;
        }
        cnt = 0;
        for (uint32_t s0 = 0; s0 < p.nsteps; s0 += 32) {
            const uint32_t i = s0 + lane;
            bool act = false;
            TileStep st;
            if (i < p.nsteps) {
                st = steps_sm[i];
                act = (base & st.co) == st.po;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (act) {
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                list[pos] = make_uint2(st.cl | (st.pl << 16), st.tmask);
            }
            cnt += __popc(bal);
        }
        if (cnt > 0) break;
        base = kNoTile;
    }
    if (lane == 0) {
        meta[s].base = base;
        meta[s].cnt = cnt;
    }
    if (base == kNoTile) return next;
    fence_proxy_async_smem();
    const uint32_t run_bytes = (uint32_t)B << p.l;
    if (lane == 0) mbar_arrive_expect_tx(bar, run_bytes << p.nh);
    __syncwarp();
    const char *g = p.state;
    for (uint32_t r = lane; r < (1u << p.nh); r += 32) {
        const uint64_t gi = base + depo[r];
        bulk_g2s(buf + (size_t)r * run_bytes, g + gi * B, run_bytes, bar);
    }
    return next;
}

template <int B>
__global__ void __launch_bounds__(kThreads, 1) tile_kernel(TileKParams p)
{
    using A = typename AmpOf<B>::T;
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t tile_amps = 1u << p.k;
    const size_t tile_bytes = (size_t)B * tile_amps;
    char *bufs = reinterpret_cast<char *>(smem);
    uint64_t *depo = reinterpret_cast<uint64_t *>(smem + tile_bytes * p.stages);
    TileStageMeta *meta = reinterpret_cast<TileStageMeta *>(depo + (1u << p.nh));
    uint64_t *bars = reinterpret_cast<uint64_t *>(meta + p.stages);
    TileStep *steps_sm = reinterpret_cast<TileStep *>(bars + p.stages);
    uint2 *lists = reinterpret_cast<uint2 *>(steps_sm + p.nsteps);  // stages (+1) lists

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    for (uint32_t r = tid; r < (1u << p.nh); r += kThreads) {
        uint64_t d = 0;
        for (uint32_t q = 0; q < p.nh; ++q) d |= (uint64_t)((r >> q) & 1u) << p.high[q];
        depo[r] = d;
    }
    for (uint32_t i = tid; i < p.nsteps; i += kThreads) steps_sm[i] = p.steps[i];
    if (tid == 0) {
        for (uint32_t s = 0; s < p.stages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint2 *shared_list = lists + (size_t)p.stages * kMaxTileSteps;
    if (p.all_local) {
        for (uint32_t i = tid; i < p.nsteps; i += kThreads)
            shared_list[i] = make_uint2(steps_sm[i].cl | (steps_sm[i].pl << 16), steps_sm[i].tmask);
    }
    uint64_t next = blockIdx.x;
    if (warp == 0) {
        for (uint32_t s = 0; s < p.stages; ++s)
            next = tile_produce<B>(p, (int)s, next, bufs + tile_bytes * s, depo, meta,
                                   lists + (size_t)s * kMaxTileSteps, steps_sm, &bars[s]);
    }
    __syncthreads();

    const uint32_t lmask = (1u << p.l) - 1u;
    uint32_t parity = 0;  // bit s: phase of stage s
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % p.stages;
        const uint64_t base = meta[s].base;
        if (base == kNoTile) break;
        bool ok = false;
        for (unsigned w = 0; w < kWaitLimit && !ok; ++w) ok = mbar_try_wait(&bars[s], (parity >> s) & 1u);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(p.err, 1);
            return;
        }
        parity ^= 1u << s;
        const A *buf = reinterpret_cast<const A *>(bufs + tile_bytes * s);
        const uint2 *list = p.all_local ? shared_list : lists + (size_t)s * kMaxTileSteps;
        const int cnt = meta[s].cnt;
        A *st = reinterpret_cast<A *>(p.state);
        for (uint32_t j0 = 0; j0 < tile_amps; j0 += kThreads * 8) {
            uint32_t src[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) src[e] = j0 + tid + e * kThreads;
            for (int q = cnt - 1; q >= 0; --q) {
                const uint2 d = list[q];
                const uint32_t cl = d.x & 0xffffu, pl = d.x >> 16, tm = d.y;
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if ((src[e] & cl) == pl) src[e] ^= tm;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t j = j0 + tid + e * kThreads;
                if (j < tile_amps) {
                    const A v = buf[src[e]];
                    st[base + depo[j >> p.l] + (j & lmask)] = v;
                }
            }
        }
        __syncthreads();
        if (warp == 0)
            next = tile_produce<B>(p, (int)s, next, bufs + tile_bytes * s, depo, meta,
                                   lists + (size_t)s * kMaxTileSteps, steps_sm, &bars[s]);
        __syncthreads();
    }
}

// ============================================================================
// (c) gather passes
// ============================================================================

template <int B, bool WIDE>
__global__ void __launch_bounds__(kThreads) gather_affine_kernel(const char *__restrict__ in,
                                                                 char *__restrict__ out, uint64_t n,
                                                                 const uint64_t *__restrict__ tables,
                                                                 uint32_t nbytes, uint64_t bvec)
{
    using A = typename AmpOf<B>::T;
    using I = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    __shared__ I tab[5 * 256];
    for (uint32_t i = threadIdx.x; i < nbytes * 256; i += kThreads) tab[i] = (I)tables[i];
    __syncthreads();
    const A *src = reinterpret_cast<const A *>(in);
    A *dst = reinterpret_cast<A *>(out);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i0 < n; i0 += 4 * stride) {
        A v[4];
        uint64_t idx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = i0 + u * stride;
            idx[u] = i;
            if (i < n) {
                I x = (I)bvec;
                for (uint32_t b = 0; b < nbytes; ++b) x ^= tab[b * 256 + ((i >> (8 * b)) & 255u)];
                v[u] = __ldg(&src[x]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (idx[u] < n) dst[idx[u]] = v[u];
    }
}

// Bit-sliced gather.  A warp owns 1024 consecutive output indices per
// iteration; lane l holds indices base + 32 l + j (j = 0..31) as bit planes:
// plane b is a 32-bit word whose bit j is bit b of index base + 32 l + j.
// Steps run last to first on the planes (target plane ^= AND of control
// planes, each complemented for polarity 0); a 32x32 bit transpose turns the
// planes back into 32 source indices, which the warp then gathers with
// coalesced stores.  Planes live in shared memory, indexed by bit.
constexpr int kSlicedChunk = 256;  // steps staged in shared memory at a time

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

template <int B, bool WIDE>
__global__ void __launch_bounds__(kThreads) gather_sliced_kernel(
    const char *__restrict__ in, char *__restrict__ out, uint32_t M, uint64_t n,
    const SlicedStep *__restrict__ steps, uint32_t nsteps)
{
    using A = typename AmpOf<B>::T;
    extern __shared__ __align__(128) unsigned char smem[];
    // planes: [M][kThreads] u32 ; table: [8 warps][32][33] u32 ; hi: [8][32][33] u8 ;
    // step chunk: kSlicedChunk SlicedStep
    static_assert(kSlicedThreads == kThreads, "plane offsets assume kThreads threads");
    uint32_t *planes = reinterpret_cast<uint32_t *>(smem);
    uint32_t *tabs = planes + (size_t)M * kThreads;
    SlicedStep *chunk = reinterpret_cast<SlicedStep *>(tabs + 8 * 32 * 33);
    uint8_t *his = reinterpret_cast<uint8_t *>(chunk + kSlicedChunk);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *tab = tabs + warp * 32 * 33;
    uint8_t *hi = his + warp * 32 * 33;
    const A *src = reinterpret_cast<const A *>(in);
    A *dst = reinterpret_cast<A *>(out);
    unsigned char *pl = reinterpret_cast<unsigned char *>(planes) + tid * 4;
    const uint64_t per_iter = (uint64_t)gridDim.x * kThreads * 32;

    for (uint64_t cbase = (uint64_t)blockIdx.x * kThreads * 32; cbase < n; cbase += per_iter) {
        // every thread of the CTA iterates the same number of times (uniform
        // loop bound) so the step-chunk barriers below are safe.
        const uint64_t my = cbase + (uint64_t)tid * 32;  // first index of this lane
        // initial planes: bits 0..4 enumerate j, higher bits copy 'my'
        const uint32_t pat[5] = {0xaaaaaaaau, 0xccccccccu, 0xf0f0f0f0u, 0xff00ff00u, 0xffff0000u};
        for (uint32_t b = 0; b < M; ++b) {
            const uint32_t w = (b < 5) ? pat[b] : (((my >> b) & 1ull) ? 0xffffffffu : 0u);
            planes[b * kThreads + tid] = w;
        }
        // steps, last to first, staged in chunks
        for (int64_t s_end = (int64_t)nsteps; s_end > 0; s_end -= kSlicedChunk) {
            const int64_t s_beg = s_end > kSlicedChunk ? s_end - kSlicedChunk : 0;
            const int cn = (int)(s_end - s_beg);
            __syncthreads();
            for (int i = tid; i < cn; i += kThreads) chunk[i] = steps[s_beg + i];
            __syncthreads();
            for (int q = cn - 1; q >= 0; --q) {
                const SlicedStep d = chunk[q];
                uint32_t m = 0xffffffffu;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    if (c >= d.nc) break;
                    const uint32_t v = *reinterpret_cast<const uint32_t *>(pl + d.c_off[c]);
                    m &= ((d.neg >> c) & 1) ? ~v : v;
                }
                *reinterpret_cast<uint32_t *>(pl + d.t_off) ^= m;
            }
        }
        // planes -> 32 source indices of this lane
        uint32_t r[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) r[b] = (b < (int)M) ? planes[b * kThreads + tid] : 0u;
        transpose32(r);
#pragma unroll
        for (int j = 0; j < 32; ++j) tab[lane * 33 + j] = r[j];
        if (WIDE) {
            const uint32_t w32 = (M > 32) ? planes[32 * kThreads + tid] : 0u;
            const uint32_t w33 = (M > 33) ? planes[33 * kThreads + tid] : 0u;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                hi[lane * 33 + j] = (uint8_t)(((w32 >> j) & 1u) | (((w33 >> j) & 1u) << 1));
        }
        __syncwarp();
        // coalesced gather: entry e of every lane's row -> outputs
        const uint64_t wbase = cbase + (uint64_t)warp * 1024;
#pragma unroll 4
        for (int e0 = 0; e0 < 32; e0 += 8) {
            A v[8];
            uint64_t o[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u;
                o[u] = wbase + (uint64_t)e * 32 + lane;
                uint64_t x = tab[e * 33 + lane];
                if (WIDE) x |= (uint64_t)hi[e * 33 + lane] << 32;
                if (o[u] < n) v[u] = __ldg(&src[x]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (o[u] < n) dst[o[u]] = v[u];
        }
        __syncwarp();
    }
}

// ============================================================================
// FP64 probabilities and norm
// ============================================================================

constexpr int kProbBlocks = 1024;

template <int B>
__global__ void __launch_bounds__(kThreads) probs_kernel(const char *__restrict__ state,
                                                         double *__restrict__ probs, uint64_t n,
                                                         double *__restrict__ partials)
{
    __shared__ double red[kThreads];
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        double re, im;
        if (B == 8) {
            const float2 v = reinterpret_cast<const float2 *>(state)[i];
            re = (double)v.x;
            im = (double)v.y;
        } else {
            const double2 v = reinterpret_cast<const double2 *>(state)[i];
            re = v.x;
            im = v.y;
        }
        const double p = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
        if (probs) probs[i] = p;
        acc += p;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
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
    const uint64_t want = (p.n_pairs + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    const int grid = (int)(want < cap ? want : cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (amp_bytes == 8)
        sweep_kernel<8><<<grid, kThreads, 0, s>>>(static_cast<char *>(state), p);
    else
        sweep_kernel<16><<<grid, kThreads, 0, s>>>(static_cast<char *>(state), p);
    return cudaGetLastError();
}

static uint32_t tile_stages(int amp_bytes, int k)
{
    const size_t tb = (size_t)amp_bytes << k;
    if (tb <= 64 * 1024) return 3;
    return 1;
}

size_t tile_smem_bytes(int amp_bytes, int k)
{
    const uint32_t st = tile_stages(amp_bytes, k);
    return ((size_t)amp_bytes << k) * st + sizeof(uint64_t) * (1u << kMaxHighBits) +
           sizeof(TileStageMeta) * st + sizeof(uint64_t) * st + sizeof(TileStep) * kMaxTileSteps +
           sizeof(uint2) * kMaxTileSteps * (st + 1);
}

int launch_tile(void *state, int amp_bytes, const TilePass &t, const TileStep *d_steps,
                int *d_err, void *stream)
{
    TileKParams p;
    p.state = static_cast<char *>(state);
    p.steps = d_steps + t.step_off;
    p.err = d_err;
    p.n_tiles = t.n_tiles;
    p.k = t.k;
    p.l = t.l;
    p.nh = t.nh;
    p.nsteps = t.nsteps;
    p.all_local = t.all_local;
    p.stages = tile_stages(amp_bytes, (int)t.k);
    for (int i = 0; i < kMaxHighBits; ++i) p.high[i] = t.high[i];
    const size_t smem = tile_smem_bytes(amp_bytes, (int)t.k);
    const uint64_t cap = (uint64_t)num_sms();
    const int grid = (int)(t.n_tiles < cap ? t.n_tiles : cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (amp_bytes == 8) {
        e = cudaFuncSetAttribute(tile_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        tile_kernel<8><<<grid, kThreads, smem, s>>>(p);
    } else {
        e = cudaFuncSetAttribute(tile_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        tile_kernel<16><<<grid, kThreads, smem, s>>>(p);
    }
    return cudaGetLastError();
}

static size_t sliced_smem_bytes(uint32_t M)
{
    return sizeof(uint32_t) * ((size_t)M * kThreads + 8 * 32 * 33) +
           sizeof(SlicedStep) * kSlicedChunk + 8 * 32 * 33;
}

template <int B, bool W>
static cudaError_t launch_sliced(const void *in, void *out, uint32_t M, uint64_t n,
                                 const SlicedStep *steps, uint32_t nsteps, cudaStream_t s)
{
    const size_t smem = sliced_smem_bytes(M);
    cudaError_t e = cudaFuncSetAttribute(gather_sliced_kernel<B, W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_sliced_kernel<B, W>, kThreads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    const uint64_t chunks = (n + kThreads * 32 - 1) / (kThreads * 32);
    const uint64_t cap = (uint64_t)num_sms() * per_sm;
    const int grid = (int)(chunks < cap ? chunks : cap);
    gather_sliced_kernel<B, W><<<grid, kThreads, smem, s>>>(
        static_cast<const char *>(in), static_cast<char *>(out), M, n, steps, nsteps);
    return cudaGetLastError();
}

int launch_gather(const void *in, void *out, int amp_bytes, uint32_t M, const GatherPass &g,
                  const uint64_t *d_tables, const SlicedStep *d_steps, int * /*d_err*/,
                  void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t n = 1ull << M;
    if (g.affine) {
        const uint64_t want = (n + kThreads * 4 - 1) / (kThreads * 4);
        const uint64_t cap = (uint64_t)num_sms() * 8;
        const int grid = (int)(want < cap ? want : cap);
        const uint64_t *tab = d_tables + g.table_off;
        const char *i = static_cast<const char *>(in);
        char *o = static_cast<char *>(out);
        if (amp_bytes == 8) {
            if (M > 32)
                gather_affine_kernel<8, true><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec);
            else
                gather_affine_kernel<8, false><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec);
        } else {
            if (M > 32)
                gather_affine_kernel<16, true><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec);
            else
                gather_affine_kernel<16, false><<<grid, kThreads, 0, s>>>(i, o, n, tab, g.nbytes, g.bvec);
        }
        return cudaGetLastError();
    }
    const SlicedStep *st = d_steps + g.step_off;
    if (amp_bytes == 8)
        return M > 32 ? launch_sliced<8, true>(in, out, M, n, st, g.nsteps, s)
                      : launch_sliced<8, false>(in, out, M, n, st, g.nsteps, s);
    return M > 32 ? launch_sliced<16, true>(in, out, M, n, st, g.nsteps, s)
                  : launch_sliced<16, false>(in, out, M, n, st, g.nsteps, s);
}

int probabilities_partials_needed() { return kProbBlocks; }

int launch_probabilities(const void *state, int amp_bytes, uint64_t n, double *d_probs,
                         double *d_partials, int n_partials, double *d_norm, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t want = (n + kThreads - 1) / kThreads;
    uint64_t grid = want < (uint64_t)n_partials ? want : (uint64_t)n_partials;
    if (grid < 1) grid = 1;
    if (amp_bytes == 8)
        probs_kernel<8><<<(int)grid, kThreads, 0, s>>>(static_cast<const char *>(state), d_probs, n,
                                                       d_partials);
    else
        probs_kernel<16><<<(int)grid, kThreads, 0, s>>>(static_cast<const char *>(state), d_probs, n,
                                                        d_partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_kernel<<<1, kThreads, 0, s>>>(d_partials, (int)grid, d_norm);
    return cudaGetLastError();
}

}  // namespace qsim
