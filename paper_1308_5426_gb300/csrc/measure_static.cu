// Allocation-free energy and magnetisation measurement.
//
// potts_lr_create allocates device memory, and so does every handle-based call
// path before it can run.  Some callers cannot allocate: code that runs inside
// a host framework that owns all device memory and forbids cudaMalloc, code
// in a latency-critical loop that must not pay for the device-wide
// synchronisation a cudaMalloc/cudaFree can bring, or code that has already
// reserved exactly the memory it may use.  potts_lr_measure_static serves
// them: the caller passes its own device buffers for the inputs (packed spins,
// the J* table) and the outputs (E, M), and the measure kernel's scratch --
// the per-configuration results it writes before they are copied out -- lives
// in the fixed array below instead of memory allocated per call or per handle.
//
// The array is a file-scope __device__ object: every GPU that loads this
// library holds it (kStaticMeasureMaxR * 2 doubles = 64 KB) until the process
// exits.  In host code its name is only a host-side stand-in, not a device
// address, so the entry point asks the runtime for the device address once
// per device (cudaGetSymbolAddress, with that device current) and hands that
// pointer to the kernel.  The address is cached together with the device's
// current context: after a cudaDeviceReset the runtime loads the module into
// a new context, and the first call there looks the address up again.
#include <mutex>

#include <cuda.h>

#include "../../include/potts_lr.h"
#include "measure_body.cuh"
#include "potts_internal.h"

namespace plr {
namespace {

constexpr int kStaticMeasureMaxR = 4096;
constexpr int kMaxDevices = 64;

// scratch: E of configuration r at [r], M at [kStaticMeasureMaxR + r]
static __device__ __align__(256) double g_measure_scratch[2 * kStaticMeasureMaxR];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// the calling thread's current context (driver entry point found through the
// runtime, so the library needs no link-time dependency on the driver)
CUcontext current_context()
{
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (Fn)p;
    });
    CUcontext c = nullptr;
    if (fn) fn(&c);
    return c;
}

__global__ void __launch_bounds__(kAuxThreads) measure_static_kernel(const uint32_t* __restrict__ spins, int L,
                                                                     int q, int W, int c,
                                                                     const double* __restrict__ J,
                                                                     double* __restrict__ scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int r = blockIdx.x;
    double E, M;
    measure_body(spins + (size_t)r * W, L, q, c, J, smem, &E, &M);
    if (threadIdx.x == 0) {
        scratch[r] = E;
        scratch[kStaticMeasureMaxR + r] = M;
    }
}

}  // namespace
}  // namespace plr

using namespace plr;

extern "C" int potts_lr_measure_static(const uint32_t* spins, int L, int q, int R, const double* jstar,
                                       int pair_factor, double* E, double* M, void* cuda_stream)
{
    if (!spins || !jstar || !E || !M) return POTTS_LR_EINVAL;
    if (L < 2 || L > kMaxL || q < 2 || q > kMaxQ || R < 1 || R > kStaticMeasureMaxR ||
        (pair_factor != 1 && pair_factor != 2))
        return POTTS_LR_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return POTTS_LR_ECUDA;
    const CUcontext ctx = current_context();  // null before the runtime first used the device
    double* scratch = nullptr;
    {
        // once per device (and context), with that device current: the
        // device address of the array
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_measure_scratch) != cudaSuccess || !p) return POTTS_LR_ECUDA;
            g_scratch_ptr[dev] = (double*)p;
            g_scratch_ctx[dev] = current_context();  // the context the lookup ran in
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int W = (L + 7) / 8;
    const size_t smem = measure_smem_bytes(L, q);  // at most 32 KB for L <= 65536 (one tile's window)
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(measure_static_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return POTTS_LR_ECUDA;
    measure_static_kernel<<<R, kAuxThreads, smem, st>>>(spins, L, q, W, pair_factor, jstar, scratch);
    if (cudaGetLastError() != cudaSuccess) return POTTS_LR_ECUDA;
    const size_t bytes = (size_t)R * sizeof(double);
    if (cudaMemcpyAsync(E, scratch, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return POTTS_LR_ECUDA;
    if (cudaMemcpyAsync(M, scratch + kStaticMeasureMaxR, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return POTTS_LR_ECUDA;
    return POTTS_LR_OK;
}
