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

// Compile (or find) the kernel; with load = true also load it on the device.
int jit_get(uint32_t M, int amp, const qsim_step *steps, size_t n, bool load, JitEntry **out,
            std::string *msg)
{
    std::vector<uint64_t> key = make_key(M, amp, steps, n);
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
        const std::string src = generate_source(M, amp, steps, n);
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
        if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&e->kern, e->lib, "qsim_jit_gather");
        if (ce != cudaSuccess) {
            e->kern = nullptr;
            *msg = std::string("loading the compiled gather: ") + cudaGetErrorString(ce);
            return QSIM_ECUDA;
        }
    }
    *out = e;
    return QSIM_OK;
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

}  // namespace qsim
