// jit.cu -- circuit-specialised gather kernels compiled at run time.
//
// The bit-sliced gather evaluates the inverse wiring diagram on 32 output
// indices at once: plane[target] ^= AND of control planes, for every step,
// last to first (Sec. 2h product evaluated per row, Sec. 2b gather).  The
// general kernel reads step descriptors and keeps the planes in shared
// memory, because a register cannot be selected by a run-time bit number.
// Here the generator writes the step list out as straight-line CUDA source
// (one `pT ^= pA & pB;` per step), so every plane lives in a register and a
// Toffoli costs one 3-input logic instruction.  NVRTC compiles the source for
// sm_103a; the cubin is loaded with cudaLibraryLoadData and cached by a hash
// of (M, amplitude size, steps).  NVRTC is opened with dlopen on first use,
// so the library loads without it.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <chrono>
#include <cstring>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "prob_math.cuh"
#include "qsim_internal.h"

namespace qsim {

namespace {

struct Nvrtc {
    bool ok = false;
    std::string err;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) errstr = nullptr;
};

Nvrtc &nvrtc()
{
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            n.err = "NVRTC (libnvrtc.so) could not be loaded";
            return;
        }
#define QSIM_SYM(field, name)                                            \
    n.field = reinterpret_cast<decltype(n.field)>(dlsym(h, #name));      \
    if (!n.field) {                                                      \
        n.err = "NVRTC symbol missing: " #name;                          \
        return;                                                          \
    }
        QSIM_SYM(create, nvrtcCreateProgram)
        QSIM_SYM(compile, nvrtcCompileProgram)
        QSIM_SYM(log_size, nvrtcGetProgramLogSize)
        QSIM_SYM(log, nvrtcGetProgramLog)
        QSIM_SYM(cubin_size, nvrtcGetCUBINSize)
        QSIM_SYM(cubin, nvrtcGetCUBIN)
        QSIM_SYM(destroy, nvrtcDestroyProgram)
        QSIM_SYM(errstr, nvrtcGetErrorString)
#undef QSIM_SYM
        n.ok = true;
    });
    return n;
}

struct JitEntry {
    std::vector<uint64_t> key;  // full key, checked on every hit
    std::vector<char> cubin;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    double compile_ms = 0;
};

std::mutex g_jit_mu;
std::unordered_map<uint64_t, std::unique_ptr<JitEntry>> g_jit_cache;

std::vector<uint64_t> make_key(uint32_t M, int amp, const qsim_step *steps, size_t n)
{
    std::vector<uint64_t> k;
    k.reserve(2 + 3 * n);
    k.push_back(M);
    k.push_back((uint64_t)amp);
    for (size_t i = 0; i < n; ++i) {
        k.push_back(steps[i].target);
        k.push_back(steps[i].ctrl_mask);
        k.push_back(steps[i].ctrl_pol);
    }
    return k;
}

uint64_t fnv1a(const std::vector<uint64_t> &k)
{
    uint64_t h = 0xcbf29ce484222325ull;
    for (uint64_t w : k)
        for (int b = 0; b < 8; ++b) {
            h ^= (w >> (8 * b)) & 0xffu;
            h *= 0x100000001b3ull;
        }
    return h;
}

// The steps as bit-plane updates on planes p0..p{M-1}, last step first (the
// inverse circuit evaluated on output indices): a NOT complements its target
// plane, a controlled step XORs the AND of its control planes (a control on
// |0> complemented) into the target plane.
void step_lines(std::ostringstream &s, const qsim_step *steps, size_t n)
{
    for (size_t q = n; q-- > 0;) {
        const qsim_step &st = steps[q];
        s << "    p" << st.target;
        if (st.ctrl_mask == 0) {
            s << " = ~p" << st.target << ";\n";
            continue;
        }
        s << " ^= ";
        bool first = true;
        for (uint64_t m = st.ctrl_mask; m; m &= m - 1) {
            const uint32_t b = (uint32_t)__builtin_ctzll(m);
            if (!first) s << " & ";
            first = false;
            s << (((st.ctrl_pol >> b) & 1ull) ? "p" : "~p") << b;
        }
        s << ";\n";
    }
}

const char *kLanePattern[5] = {"0xaaaaaaaau", "0xccccccccu", "0xf0f0f0f0u", "0xff00ff00u", "0xffff0000u"};

// Source of the kernel that finds which address bits a step list can change:
// every output row's source x(i) is evaluated (32 rows per thread, bit
// planes) and the OR over all rows of x(i) ^ i is accumulated into *out.
std::string generate_delta_source(uint32_t M, const qsim_step *steps, size_t n)
{
    std::ostringstream s;
    s << "typedef unsigned int u32;\ntypedef unsigned long long u64;\n"
         "extern \"C\" __global__ void __launch_bounds__(256) qsim_jit_delta(u64 n, u64* out) {\n"
         "  u64 acc = 0;\n"
         "  const u32 valid = n >= 32ull ? 0xffffffffu : (u32)((1ull << n) - 1ull);\n"
         "  for (u64 my = ((u64)blockIdx.x * 256ull + threadIdx.x) * 32ull; my < n;"
         " my += (u64)gridDim.x * 256ull * 32ull) {\n";
    for (uint32_t b = 0; b < M; ++b) {
        if (b < 5)
            s << "    u32 p" << b << " = " << kLanePattern[b] << ";\n";
        else
            s << "    u32 p" << b << " = 0u - (u32)((my >> " << b << ") & 1ull);\n";
    }
    step_lines(s, steps, n);
    for (uint32_t b = 0; b < M; ++b) {
        s << "    acc |= (u64)(((p" << b << " ^ ";
        if (b < 5) s << kLanePattern[b];
        else s << "(0u - (u32)((my >> " << b << ") & 1ull))";
        s << ") & valid) != 0u) << " << b << ";\n";
    }
    s << "  }\n"
         "  u32 lo = (u32)acc, hi = (u32)(acc >> 32);\n"
         "  lo = __reduce_or_sync(0xffffffffu, lo);\n"
         "  hi = __reduce_or_sync(0xffffffffu, hi);\n"
         "  if ((threadIdx.x & 31) == 0 && (lo | hi)) atomicOr(out, ((u64)hi << 32) | lo);\n"
         "}\n";
    return s.str();
}

// CUDA source of one circuit-specialised gather kernel.  Output index
// my + j (j = 0..31) of a thread is held as 32-bit planes p0..p{M-1};
// the steps are emitted last to first.
std::string generate_source(uint32_t M, int amp, const qsim_step *steps, size_t n)
{
    const bool wide = M > 32;
    std::ostringstream s;
    s << "typedef unsigned int u32;\ntypedef unsigned long long u64;\n";
    // random reads: read-only path with a 64-byte L2 fill (fewer DRAM bytes
    // per 16-byte read than the default fill)
    if (amp == 16)
        s << "struct __align__(16) Amp { u32 a, b, c, d; };\n"
             "__device__ __forceinline__ Amp ldnc(const Amp* p) { Amp v; asm volatile("
             "\"ld.global.nc.L2::64B.v4.u32 {%0,%1,%2,%3}, [%4];\" : \"=r\"(v.a), \"=r\"(v.b), \"=r\"(v.c), "
             "\"=r\"(v.d) : \"l\"(p)); return v; }\n";
    else
        s << "struct __align__(8) Amp { u32 a, b; };\n"
             "__device__ __forceinline__ Amp ldnc(const Amp* p) { Amp v; asm volatile("
             "\"ld.global.nc.L2::64B.v2.u32 {%0,%1}, [%2];\" : \"=r\"(v.a), \"=r\"(v.b) : \"l\"(p)); "
             "return v; }\n";
    // 32x32 bit transpose: five rounds of masked block swaps
    s << "__device__ __forceinline__ void tr32(u32 (&a)[32]) {\n"
         "  u32 m = 0x0000ffffu;\n"
         "#pragma unroll\n"
         "  for (int j = 16; j != 0; j >>= 1, m ^= (m << j)) {\n"
         "#pragma unroll\n"
         "    for (int k = 0; k < 32; ++k) { if (k & j) continue;\n"
         "      const u32 t = ((a[k] >> j) ^ a[k | j]) & m; a[k | j] ^= t; a[k] ^= t << j; }\n"
         "  }\n}\n";
    // FP64 probabilities of the gathered amplitudes (same functions as the
    // library's own kernels)
    s << "#define QSIM_Q __device__ __forceinline__\n#define QSIM_QN __device__ __noinline__\n"
      << kProbMathSource << "\n";
    s << "extern \"C\" __global__ void __launch_bounds__(256) qsim_jit_gather("
         "const Amp* __restrict__ in, Amp* __restrict__ out, u64 n, double* __restrict__ probs) {\n"
         "  __shared__ u32 tabs[8 * 32 * 33];\n";
    if (wide) s << "  __shared__ unsigned char his[8 * 32 * 33];\n";
    s << "  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;\n"
         "  u32* tab = tabs + warp * 32 * 33;\n";
    if (wide) s << "  unsigned char* hi = his + warp * 32 * 33;\n";
    s << "  for (u64 cbase = (u64)blockIdx.x * 8192ull; cbase < n; cbase += (u64)gridDim.x * 8192ull) {\n"
         "    const u64 my = cbase + (u64)tid * 32ull;\n";
    const char *pat[5] = {"0xaaaaaaaau", "0xccccccccu", "0xf0f0f0f0u", "0xff00ff00u", "0xffff0000u"};
    for (uint32_t b = 0; b < M; ++b) {
        if (b < 5)
            s << "    u32 p" << b << " = " << pat[b] << ";\n";
        else
            s << "    u32 p" << b << " = 0u - (u32)((my >> " << b << ") & 1ull);\n";
    }
    step_lines(s, steps, n);
    s << "    u32 r[32];\n";
    for (uint32_t b = 0; b < 32; ++b) {
        if (b < M)
            s << "    r[" << b << "] = p" << b << ";\n";
        else
            s << "    r[" << b << "] = 0u;\n";
    }
    s << "    tr32(r);\n    __syncwarp();\n"
         "#pragma unroll\n    for (int j = 0; j < 32; ++j) tab[lane * 33 + j] = r[j];\n";
    if (wide) {
        s << "    {\n      const u32 w32 = p32;\n      const u32 w33 = " << (M > 33 ? "p33" : "0u")
          << ";\n"
             "#pragma unroll\n      for (int j = 0; j < 32; ++j) hi[lane * 33 + j] = (unsigned char)"
             "(((w32 >> j) & 1u) | (((w33 >> j) & 1u) << 1));\n    }\n";
    }
    s << "    __syncwarp();\n"
         "    const u64 wbase = cbase + (u64)warp * 1024ull;\n"
         "#pragma unroll 1\n"
         "    for (int e0 = 0; e0 < 32; e0 += 8) {\n"
         "      Amp v[8]; u64 o[8];\n"
         "#pragma unroll\n"
         "      for (int u = 0; u < 8; ++u) {\n"
         "        o[u] = wbase + (u64)(e0 + u) * 32ull + lane;\n"
         "        u64 x = tab[(e0 + u) * 33 + lane];\n";
    if (wide) s << "        x |= (u64)hi[(e0 + u) * 33 + lane] << 32;\n";
    // probabilities beside the stores (a uniform test: one kernel serves both)
    s << "        if (o[u] < n) v[u] = ldnc(in + x);\n"
         "      }\n"
         "#pragma unroll\n"
         "      for (int u = 0; u < 8; ++u) if (o[u] < n) {\n"
         "        out[o[u]] = v[u];\n"
         "        if (probs) probs[o[u]] = "
      << (amp == 16 ? "qsim_prob_bits(v[u].a, v[u].b, v[u].c, v[u].d)"
                    : "qsim_prob_bits(v[u].a, v[u].b)")
      << ";\n"
         "      }\n"
         "    }\n"
         "    __syncwarp();\n"
         "  }\n}\n";
    return s.str();
}

// Closed tile pass of one circuit: every output row's source lies in its own
// tile (the circuit's net map changes only tile bits), so a tile is loaded
// into shared memory by tensor-map copies, each output's source is found by
// evaluating the circuit on bit planes, and the tile is written back in place.
const char *kClosedTemplate = R"QSIMSRC(
typedef unsigned int u32;
typedef unsigned long long u64;
typedef unsigned short u16;
struct __align__(64) TMap { u64 v[16]; };
struct Params { char *state; double *probs; int *err; u64 n_tiles; u32 wait_limit; u32 pad; };
#define QSIM_Q __device__ __forceinline__
#define QSIM_QN __device__ __noinline__
@PROBMATH@
@AMPDEF@
__device__ __forceinline__ u32 sa(const void *p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64 *b, u32 c)
{ asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sa(b)), "r"(c) : "memory"); }
__device__ __forceinline__ void mbar_expect(u64 *b, u32 bytes)
{ asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" :: "r"(sa(b)), "r"(bytes) : "memory"); }
__device__ __forceinline__ void mbar_arrive(u64 *b)
{ asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" :: "r"(sa(b)) : "memory"); }
__device__ __forceinline__ bool mbar_wait(u64 *b, u32 parity, u32 limit)
{
  for (u32 w = 0; w < limit; ++w) {
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(sa(b)), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma5(void *dst, const TMap *m, int c0, int c1, int c2, int c3, int c4, u64 *bar)
{
  asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
               :: "r"(sa(dst)), "l"((u64)m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(sa(bar)) : "memory");
}
__device__ __forceinline__ void tr32(u32 (&a)[32])
{
  u32 m = 0x0000ffffu;
#pragma unroll
  for (int j = 16; j != 0; j >>= 1, m ^= (m << j)) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & j) continue;
      const u32 t = ((a[k] >> j) ^ a[k | j]) & m;
      a[k | j] ^= t;
      a[k] ^= t << j;
    }
  }
}
#define K @K@
#define L @L@
#define NH @NH@
#define NREST @NREST@
#define NT @NT@
#define AB @B@
#define BOX_BYTES @BOX@
#define TABN ((NT * 33 + 7) / 8 * 8)  /* exchange-table entries, rounded to 16 bytes */
#define STAGES @STAGES@
__device__ __forceinline__ u64 tile_base(u64 t) { u64 b = 0; @TILEBASE@ return b; }
__device__ __forceinline__ u64 deposit_high(u32 r) { u64 d = 0; @DEPHIGH@ return d; }
__device__ __forceinline__ u64 deposit_rest(u32 r) { u64 d = 0; @DEPREST@ return d; }
extern "C" __global__ void __launch_bounds__(NT + 32, 1)
qsim_jit_closed(const __grid_constant__ Params p, const __grid_constant__ TMap tmap)
{
  extern __shared__ __align__(128) unsigned char smem[];
  Amp *bufs = reinterpret_cast<Amp *>(smem);
  u64 *depo = reinterpret_cast<u64 *>(smem + ((size_t)AB << K) * STAGES);
  u16 *tabs = reinterpret_cast<u16 *>(depo + (1u << NH));
  u64 *full = reinterpret_cast<u64 *>(tabs + TABN);
  u64 *empty = full + STAGES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (u32 r = tid; r < (1u << NH); r += NT + 32) depo[r] = deposit_high(r);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NT / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // tiles are dealt out cyclically: CTA b takes tiles b, b + grid, ...  At any
  // moment the CTAs then work on consecutive tiles, whose short runs share
  // DRAM pages.
  const u64 cnt = blockIdx.x < p.n_tiles ? (p.n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (warp == NT / 32) {
    // producer warp: tile it goes to stage it % STAGES once that stage's
    // previous tile has been consumed
    for (u64 i = 0; i < cnt; ++i) {
      const u64 t = blockIdx.x + i * gridDim.x;
      const u32 it = (u32)i, s = it % STAGES;
      if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) - 1) & 1u, p.wait_limit)) {
        if (lane == 0) atomicOr(p.err, 2);
        return;
      }
      const u64 base = tile_base(t);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (lane == 0) mbar_expect(&full[s], (u32)((size_t)AB << K));
      __syncwarp();
      char *buf = reinterpret_cast<char *>(bufs) + ((size_t)AB << K) * s;
      for (u32 r = lane; r < (1u << NREST); r += 32) {
        const u64 g = base | deposit_rest(r);
        @COORDS@
        tma5(buf + (size_t)r * BOX_BYTES, &tmap, c0, c1, c2, c3, c4, &full[s]);
      }
    }
    return;
  }
  // consumer warps: sources of the next tile's outputs while it loads, then
  // shared memory to global memory in coalesced runs
  u16 *tab = tabs + warp * 32 * 33;
  for (u64 i = 0; i < cnt; ++i) {
    const u64 t = blockIdx.x + i * gridDim.x;
    const u32 it = (u32)i, s = it % STAGES;
    const u64 base = tile_base(t);
    {
      const u32 j0 = (u32)tid * 32u;
@PLANES@
@STEPS@
@CHECK@
      u32 r[32];
@RLOCAL@
      tr32(r);
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 32; ++u) tab[lane * 33 + u] = (u16)r[u];
      __syncwarp();
    }
    if (!mbar_wait(&full[s], (it / STAGES) & 1u, p.wait_limit)) {
      if (tid == 0) atomicOr(p.err, 1);
      return;
    }
    const Amp *buf = bufs + ((size_t)1 << K) * s;
#pragma unroll 1
    for (int e0 = 0; e0 < 32; e0 += 8) {
      Amp v[8];
      u64 g[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const u32 j = ((u32)warp * 32u + (u32)(e0 + u)) * 32u + (u32)lane;
        v[u] = buf[tab[(e0 + u) * 33 + lane]];
        g[u] = base + depo[j >> L] + (j & ((1u << L) - 1u));
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        reinterpret_cast<Amp *>(p.state)[g[u]] = v[u];
        if (p.probs) p.probs[g[u]] = AMP_PROB(v[u]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}
)QSIMSRC";



void replace_all(std::string &s, const std::string &from, const std::string &to)
{
    for (size_t pos = 0; (pos = s.find(from, pos)) != std::string::npos; pos += to.size())
        s.replace(pos, from.size(), to);
}

// Local bit q of a tile -> address bit (low run first, then the high bits in
// the layout's order: the order of the amplitudes in shared memory).
std::vector<uint32_t> tile_local_bits(const TilePass &t)
{
    std::vector<uint32_t> lb;
    for (uint32_t q = 0; q < t.l; ++q) lb.push_back(q);
    for (uint32_t q = 0; q < t.nh; ++q) lb.push_back(t.high[q]);
    return lb;
}

// Pipeline stages of a closed pass: as many tiles as fit next to the
// exchange tables and the deposit table in 220 KiB of shared memory, at most 4.
uint32_t closed_stages(int amp, const TilePass &t)
{
    const size_t nt = ((size_t)1 << t.k) / 32;
    const size_t fixed = 2 * ((nt * 33 + 7) / 8 * 8) + sizeof(uint64_t) * ((size_t)1 << t.nh) + 64;
    const size_t tile = (size_t)amp << t.k;
    size_t st = (220 * 1024 - fixed) / (tile + 16);
    if (st > 4) st = 4;
    return st < 1 ? 1 : (uint32_t)st;
}

std::string generate_closed_source(uint32_t M, int amp, const qsim_step *steps, size_t n, const TilePass &t)
{
    std::string src = kClosedTemplate;
    const std::vector<uint32_t> lb = tile_local_bits(t);
    const uint32_t K = t.k;
    std::vector<int> local_of(64, -1);
    for (uint32_t q = 0; q < K; ++q) local_of[lb[q]] = (int)q;
    std::ostringstream planes, check, rl, tb, dh, dr, co;
    for (uint32_t b = 0; b < M; ++b) {
        const int q = local_of[b];
        planes << "      u32 p" << b << " = ";
        if (q >= 0 && q < 5) planes << kLanePattern[q] << ";\n";
        else if (q >= 5) planes << "0u - ((j0 >> " << q << ") & 1u);\n";
        else planes << "0u - (u32)((base >> " << b << ") & 1ull);\n";
    }
    check << "      u32 viol = 0u;\n";
    for (uint32_t b = 0; b < M; ++b)
        if (local_of[b] < 0) check << "      viol |= p" << b << " ^ (0u - (u32)((base >> " << b << ") & 1ull));\n";
    check << "      if (viol) atomicOr(p.err, 4);\n";
    for (uint32_t q = 0; q < 32; ++q) {
        rl << "      r[" << q << "] = ";
        if (q < K) rl << "p" << lb[q] << ";\n";
        else rl << "0u;\n";
    }
    for (uint32_t q = 0; q < t.nout; ++q) tb << "if ((t >> " << q << ") & 1ull) b |= 1ull << " << t.outpos[q] << "; ";
    for (uint32_t q = 0; q < t.nh; ++q) dh << "if ((r >> " << q << ") & 1u) d |= 1ull << " << t.high[q] << "; ";
    for (uint32_t q = 0; q < t.nrest; ++q) dr << "if ((r >> " << q << ") & 1u) d |= 1ull << " << t.rest_pos[q] << "; ";
    const uint32_t epa = amp == 16 ? 2 : 1;
    for (int d = 0; d < 5; ++d) {
        const uint32_t w = t.tma_start[d + 1] - t.tma_start[d];
        co << "        const int c" << d << " = ";
        if (w == 0) co << "0;\n";
        else co << "(int)(((g >> " << t.tma_start[d] << ") & " << ((1ull << w) - 1ull) << "ull)"
                << (d == 0 && epa == 2 ? " * 2ull" : "") << ");\n";
    }
    std::ostringstream st;
    step_lines(st, steps, n);
    replace_all(src, "@PROBMATH@", kProbMathSource);
    replace_all(src, "@AMPDEF@", amp == 16
                ? "struct __align__(16) Amp { u32 a, b, c, d; };\n#define AMP_PROB(v) qsim_prob_bits((v).a, (v).b, (v).c, (v).d)"
                : "struct __align__(8) Amp { u32 a, b; };\n#define AMP_PROB(v) qsim_prob_bits((v).a, (v).b)");
    replace_all(src, "@K@", std::to_string(K));
    replace_all(src, "@L@", std::to_string(t.l));
    replace_all(src, "@NH@", std::to_string(t.nh));
    replace_all(src, "@NREST@", std::to_string(t.nrest));
    replace_all(src, "@NT@", std::to_string((1u << K) / 32));
    replace_all(src, "@B@", std::to_string(amp));
    replace_all(src, "@BOX@", std::to_string(t.box_bytes));
    replace_all(src, "@STAGES@", std::to_string(closed_stages(amp, t)));
    replace_all(src, "@TILEBASE@", tb.str());
    replace_all(src, "@DEPHIGH@", dh.str());
    replace_all(src, "@DEPREST@", dr.str());
    replace_all(src, "@COORDS@", co.str());
    replace_all(src, "@PLANES@", planes.str());
    replace_all(src, "@STEPS@", st.str());
    replace_all(src, "@CHECK@", check.str());
    replace_all(src, "@RLOCAL@", rl.str());
    return src;
}

std::vector<uint64_t> closed_key(uint32_t M, int amp, const qsim_step *steps, size_t n, const TilePass &t)
{
    std::vector<uint64_t> k = {0xC105EDull, M, (uint64_t)amp, t.k, t.l, t.nh, t.nrest, t.box_bytes, t.nout};
    for (uint32_t q = 0; q < t.nh; ++q) k.push_back(t.high[q]);
    for (uint32_t q = 0; q < t.nrest; ++q) k.push_back(t.rest_pos[q]);
    for (uint32_t q = 0; q < 6; ++q) k.push_back(t.tma_start[q]);
    for (uint32_t q = 0; q < t.nout; ++q) k.push_back(t.outpos[q]);
    const std::vector<uint64_t> sk = make_key(M, amp, steps, n);
    k.insert(k.end(), sk.begin() + 2, sk.end());
    return k;
}

// Changed-bit sets already found, keyed by (M, steps).
std::mutex g_delta_mu;
std::unordered_map<uint64_t, std::pair<std::vector<uint64_t>, uint64_t>> g_delta_cache;

// Compile (or find) a generated kernel; with load = true also load it on the
// device.  key identifies the source completely (kind, sizes, layout, steps);
// gen writes the source on a miss.
template <typename Gen>
int jit_get_kernel(std::vector<uint64_t> key, const char *kernel_name, Gen gen, bool load,
                   JitEntry **out, std::string *msg)
{
    const uint64_t h = fnv1a(key);
    std::lock_guard<std::mutex> lk(g_jit_mu);
    auto it = g_jit_cache.find(h);
    JitEntry *e = nullptr;
    if (it != g_jit_cache.end() && it->second->key == key) {
        e = it->second.get();
    } else {
        Nvrtc &nv = nvrtc();
        if (!nv.ok) {
            *msg = nv.err;
            return QSIM_ECUDA;
        }
        const auto t0 = std::chrono::steady_clock::now();
        const std::string src = gen();
        nvrtcProgram prog;
        nvrtcResult r = nv.create(&prog, src.c_str(), "qsim_jit.cu", 0, nullptr, nullptr);
        if (r != NVRTC_SUCCESS) {
            *msg = std::string("nvrtcCreateProgram: ") + nv.errstr(r);
            return QSIM_ECUDA;
        }
        const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
        r = nv.compile(prog, 3, opts);
        if (r != NVRTC_SUCCESS) {
            size_t ls = 0;
            nv.log_size(prog, &ls);
            std::string lg(ls, '\0');
            if (ls) nv.log(prog, &lg[0]);
            nv.destroy(&prog);
            *msg = std::string("NVRTC compile failed: ") + nv.errstr(r) + "\n" + lg.substr(0, 2000);
            return QSIM_ECUDA;
        }
        size_t cs = 0;
        nv.cubin_size(prog, &cs);
        auto ent = std::make_unique<JitEntry>();
        ent->cubin.resize(cs);
        nv.cubin(prog, ent->cubin.data());
        nv.destroy(&prog);
        ent->key = std::move(key);
        ent->compile_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        e = ent.get();
        g_jit_cache[h] = std::move(ent);
    }
    if (load && !e->kern) {
        cudaError_t ce = cudaLibraryLoadData(&e->lib, e->cubin.data(), nullptr, nullptr, 0, nullptr,
                                             nullptr, 0);
        if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&e->kern, e->lib, kernel_name);
        if (ce != cudaSuccess) {
            e->kern = nullptr;
            *msg = std::string("loading a compiled kernel: ") + cudaGetErrorString(ce);
            return QSIM_ECUDA;
        }
    }
    *out = e;
    return QSIM_OK;
}

// The compiled gather of one segment.
int jit_get(uint32_t M, int amp, const qsim_step *steps, size_t n, bool load, JitEntry **out,
            std::string *msg)
{
    return jit_get_kernel(make_key(M, amp, steps, n), "qsim_jit_gather",
                          [&] { return generate_source(M, amp, steps, n); }, load, out, msg);
}

}  // namespace

int jit_compile(uint32_t M, int amp, const qsim_step *steps, size_t n, double *compile_ms,
                std::string *msg)
{
    JitEntry *e = nullptr;
    int rc = jit_get(M, amp, steps, n, false, &e, msg);
    if (rc == QSIM_OK && compile_ms) *compile_ms = e->compile_ms;
    return rc;
}

int jit_prepare(uint32_t M, int amp, const qsim_step *steps, size_t n, std::string *msg)
{
    JitEntry *e = nullptr;
    return jit_get(M, amp, steps, n, true, &e, msg);
}

int launch_jit_gather(const void *in, void *out, int amp, uint32_t M, const qsim_step *steps,
                      size_t n, double *d_probs, void *stream, std::string *msg)
{
    JitEntry *e = nullptr;
    int rc = jit_get(M, amp, steps, n, true, &e, msg);
    if (rc != QSIM_OK) return rc;
    const uint64_t total = 1ull << M;
    const uint64_t chunks = (total + 8191) / 8192;
    const uint64_t cap = (uint64_t)num_sms() * 4;
    const unsigned grid = (unsigned)(chunks < cap ? chunks : cap);
    const void *a0 = in;
    void *a1 = out;
    uint64_t a2 = total;
    double *a3 = d_probs;
    void *args[] = {(void *)&a0, (void *)&a1, (void *)&a2, (void *)&a3};
    cudaError_t ce = cudaLaunchKernel(reinterpret_cast<const void *>(e->kern), dim3(grid), dim3(256),
                                      args, 0, static_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) {
        *msg = std::string("compiled gather launch: ") + cudaGetErrorString(ce);
        return QSIM_ECUDA;
    }
    return QSIM_OK;
}

int jit_delta(uint32_t M, const qsim_step *steps, size_t n, uint64_t *d_word, void *stream,
              uint64_t *delta, std::string *msg)
{
    std::vector<uint64_t> key = make_key(M, 0, steps, n);
    key[1] = 0xDE17Aull;  // a kernel kind of its own
    const uint64_t h = fnv1a(key);
    {
        std::lock_guard<std::mutex> lk(g_delta_mu);
        auto it = g_delta_cache.find(h);
        if (it != g_delta_cache.end() && it->second.first == key) {
            *delta = it->second.second;
            return QSIM_OK;
        }
    }
    JitEntry *e = nullptr;
    int rc = jit_get_kernel(key, "qsim_jit_delta", [&] { return generate_delta_source(M, steps, n); },
                            true, &e, msg);
    if (rc != QSIM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaMemsetAsync(d_word, 0, sizeof(uint64_t), s);
    const uint64_t total = 1ull << M;
    const uint64_t groups = (total + 256ull * 32 - 1) / (256ull * 32);
    const uint64_t cap = (uint64_t)num_sms() * 8;
    const unsigned grid = (unsigned)(groups < cap ? groups : cap);
    uint64_t a0 = total;
    uint64_t *a1 = d_word;
    void *args[] = {(void *)&a0, (void *)&a1};
    if (ce == cudaSuccess)
        ce = cudaLaunchKernel(reinterpret_cast<const void *>(e->kern), dim3(grid), dim3(256), args, 0, s);
    uint64_t out = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&out, d_word, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        *msg = std::string("changed-bit kernel: ") + cudaGetErrorString(ce);
        return QSIM_ECUDA;
    }
    *delta = out;
    std::lock_guard<std::mutex> lk(g_delta_mu);
    g_delta_cache[h] = {std::move(key), out};
    return QSIM_OK;
}

namespace {

struct ClosedParams {
    char *state;
    double *probs;
    int *err;
    uint64_t n_tiles;
    uint32_t wait_limit;
    uint32_t pad;
};

size_t closed_smem_bytes(int amp, const TilePass &t)
{
    const size_t nt = ((size_t)1 << t.k) / 32;
    const size_t tabn = (nt * 33 + 7) / 8 * 8;
    const size_t st = closed_stages(amp, t);
    return ((size_t)amp << t.k) * st + sizeof(uint64_t) * ((size_t)1 << t.nh) + 2 * tabn +
           2 * sizeof(uint64_t) * st;
}

int closed_get(uint32_t M, int amp, const qsim_step *steps, size_t n, const TilePass &t, JitEntry **e,
               std::string *msg)
{
    // at least one consumer warp (32 threads x 32 outputs) besides the producer
    if (t.k < 10 || t.k > (uint32_t)kMaxTileBits || t.nh > (uint32_t)kMaxHighBitsClosed ||
        t.nrest > t.nh || t.l < 1) {
        *msg = "closed tile pass: tile width outside [10, 14]";
        return QSIM_EINVAL;
    }
    return jit_get_kernel(closed_key(M, amp, steps, n, t), "qsim_jit_closed",
                          [&] { return generate_closed_source(M, amp, steps, n, t); }, true, e, msg);
}

}  // namespace

int jit_prepare_closed(uint32_t M, int amp, const qsim_step *steps, size_t n, const TilePass &t,
                       std::string *msg)
{
    JitEntry *e = nullptr;
    return closed_get(M, amp, steps, n, t, &e, msg);
}

int launch_jit_closed(void *state, int amp, uint32_t M, const qsim_step *steps, size_t n,
                      const TilePass &t, double *d_probs, int *d_err, void *stream, std::string *msg)
{
    JitEntry *e = nullptr;
    int rc = closed_get(M, amp, steps, n, t, &e, msg);
    if (rc != QSIM_OK) return rc;
    alignas(64) unsigned char tmap[128];
    std::memset(tmap, 0, sizeof(tmap));
    if (!t.tma || encode_tile_map(state, t, tmap) != 0) {
        *msg = "closed tile pass: the tile layout has no tensor map";
        return QSIM_ECUDA;
    }
    const size_t smem = closed_smem_bytes(amp, t);
    cudaError_t ce = cudaFuncSetAttribute(reinterpret_cast<const void *>(e->kern),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ClosedParams p{static_cast<char *>(state), d_probs, d_err, t.n_tiles, 1u << 24, 0u};
    void *args[] = {(void *)&p, (void *)tmap};
    const uint64_t cap = (uint64_t)num_sms();
    const unsigned grid = (unsigned)(t.n_tiles < cap ? t.n_tiles : cap);
    const unsigned block = (unsigned)((1u << t.k) / 32 + 32);
    if (ce == cudaSuccess)
        ce = cudaLaunchKernel(reinterpret_cast<const void *>(e->kern), dim3(grid), dim3(block), args, smem,
                              static_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) {
        *msg = std::string("closed tile pass launch: ") + cudaGetErrorString(ce);
        return QSIM_ECUDA;
    }
    return QSIM_OK;
}

}  // namespace qsim
