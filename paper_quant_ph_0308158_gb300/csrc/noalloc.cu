// noalloc.cu -- probabilities and norm of a caller-owned device state without
// any allocation and without a qsim_ctx.
//
// Some callers cannot allocate device memory at the moment they need a
// result: a process whose GPU memory is wholly reserved by another allocator
// (a framework's caching pool), a plug-in that a host application confines to
// a fixed memory budget, or a latency-critical loop that must not enter the
// driver's allocator.  Creating a qsim_ctx allocates (error flag, plan tables,
// partial sums), so those callers use qsim_probabilities_noalloc instead.  The
// only scratch memory it needs -- the per-block partial sums of the norm
// reduction -- lives in the fixed array below, which every GPU that loads this
// library holds until the process exits.  Every call resolves the array's
// device address afresh in the CUDA context that is current (after the first
// resolution in a context this is a lookup that allocates nothing), so a
// context created later on the same device, or a device reset, never leaves a
// stale address behind.  The first call in a context may load this library's
// device code into it (CUDA loads modules lazily by default), and that load
// reserves the module's device memory: make that first call, or any other
// launch of this library, while memory is still available -- at start-up, and
// before any stream capture.  Calls whose work overlaps on the GPU share the
// array and race.
#include <cuda_runtime.h>

#include <string>

#include "qsim_internal.h"

namespace {

// 1024 FP64 partial sums (8 KiB): the probability kernel launches at most this
// many blocks, whatever the state size.
constexpr int kNoAllocPartials = 1024;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

int noalloc_fail(int code, const std::string &msg)
{
    qsim::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int qsim_probabilities_noalloc(const void *d_state, uint32_t M, int dtype,
                                          double *d_probs, double *d_norm, void *stream)
{
    if (M < 1 || M > QSIM_MAX_QUBITS)
        return noalloc_fail(QSIM_EINVAL, "M must be in [1, " + std::to_string(QSIM_MAX_QUBITS) +
                                             "] (2^M amplitudes)");
    const int amp = dtype == QSIM_C64 ? 8 : dtype == QSIM_C128 ? 16 : 0;
    if (!amp) return noalloc_fail(QSIM_EINVAL, "unknown dtype");
    if (!d_state || !d_norm) return noalloc_fail(QSIM_EINVAL, "d_state and d_norm are required");
    if ((reinterpret_cast<uintptr_t>(d_state) & (uintptr_t)(amp - 1)) ||
        (reinterpret_cast<uintptr_t>(d_probs) & 7u) || (reinterpret_cast<uintptr_t>(d_norm) & 7u))
        return noalloc_fail(QSIM_EINVAL, "misaligned device pointer");
    if (qsim::probabilities_partials_needed() > kNoAllocPartials)
        return noalloc_fail(QSIM_EINVAL, "reduction needs more partial sums than the fixed scratch");

    // Resolve the array's device address in the current context.  The
    // host-side name g_noalloc_partials is only a stand-in and must never
    // reach a kernel.
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess)
        return noalloc_fail(QSIM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    double *partials = static_cast<double *>(p);
    // Every block writes its partial before the final reduction reads it, so
    // nothing left over from an earlier call is ever read.
    const int rc = qsim::launch_probabilities(d_state, amp, 1ull << M, d_probs, partials,
                                              kNoAllocPartials, d_norm, stream);
    if (rc != cudaSuccess)
        return noalloc_fail(QSIM_ECUDA, std::string("launch: ") + cudaGetErrorString((cudaError_t)rc));
    return QSIM_OK;
}
