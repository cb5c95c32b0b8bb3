// Throughput probes for roofline denominators: FP64 add, FP32 add, shared-
// memory and L2 bandwidth of this GPU, measured with CUDA events on a private
// stream.  Each probe kernel runs long independent dependency chains at full
// occupancy so that the pipe (not latency) is the limit.
#include <cstring>

#include "../../include/potts_lr.h"
#include "potts_internal.h"

namespace plr {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeIters = 4096;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) add_probe(T* out, T seed)
{
    // 8 independent accumulator chains per thread, 2 adds each per iteration
    T a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed * (T)(threadIdx.x + c);
    const T d0 = seed * (T)1e-3, d1 = seed * (T)-1e-3;
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            a[c] += d0;
            a[c] += d1;
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == (T)123456.789) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(kProbeThreads) smem_probe(float* out, int iters)
{
    // each warp streams float loads and stores over its own 4 KB of shared memory
    __shared__ float buf[kProbeThreads * 4];
    const int tid = threadIdx.x;
    for (int i = tid; i < kProbeThreads * 4; i += kProbeThreads) buf[i] = (float)i;
    __syncthreads();
    const int w = tid >> 5, lane = tid & 31;
    volatile float* base = buf + w * 128;  // every access goes to shared memory
    float acc = 0.0f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float v = base[r * 32 + lane];
            acc += v;
            base[((r + 1) & 3) * 32 + lane] = v + 1.0f;
        }
    }
    if (acc == 123456.0f) out[0] = acc;
}

// 64-bit integer adds (the FX64 field update): 8 independent chains per
// thread, two adds each per iteration, written as PTX adds so that the
// compiler cannot fold the (associative) integer chains into one multiply
__global__ void __launch_bounds__(kProbeThreads) i64_probe(long long* out, long long seed)
{
    long long a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed * (long long)(threadIdx.x + c);
    const long long d0 = seed * 3, d1 = seed * -5;
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            asm volatile("add.s64 %0, %0, %1;" : "+l"(a[c]) : "l"(d0));
            asm volatile("add.s64 %0, %0, %1;" : "+l"(a[c]) : "l"(d1));
        }
    }
    long long s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 123456789ll) out[0] = s;  // keeps the chains alive
}

// L2 bandwidth: each CTA reads and rewrites its own slice of a buffer that
// stays resident in L2 (far below its 129 MB), 16 bytes per thread access
__global__ void __launch_bounds__(kProbeThreads) l2_probe(float4* buf, size_t per_cta, int iters)
{
    float4* p = buf + (size_t)blockIdx.x * per_cta;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = 0; it < iters; ++it) {
        for (size_t i = threadIdx.x; i < per_cta; i += kProbeThreads) {
            float4 v = __ldcg(p + i);
            acc.x += v.x;
            v.x += 1.0f;
            __stcg(p + i, v);
        }
    }
    if (acc.x == 123456.0f) buf[0] = acc;
}

}  // namespace
}  // namespace plr

using namespace plr;

extern "C" int potts_lr_probe(int what, double* value)
{
    if (!value || what < 0 || what > 4) return POTTS_LR_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return POTTS_LR_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return POTTS_LR_ECUDA;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return POTTS_LR_ECUDA;
    void* out = nullptr;
    cudaEvent_t e0, e1;
    int rc = POTTS_LR_OK;
    const int blocks = sms * 8;  // 2048 threads per SM
    const size_t l2_per_cta = ((size_t)32 << 20) / 16 / (size_t)blocks;  // float4s per CTA of a 32 MB buffer
    if (cudaMalloc(&out, what == 3 ? l2_per_cta * blocks * 16 : 16) != cudaSuccess) {
        cudaStreamDestroy(st);
        return POTTS_LR_ENOMEM;
    }
    bool ok = cudaEventCreate(&e0) == cudaSuccess;
    if (ok && cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        ok = false;
    }
    if (!ok) {
        cudaFree(out);
        cudaStreamDestroy(st);
        return POTTS_LR_ECUDA;
    }
    const int smem_iters = 1 << 16;
    const int l2_iters = 256;
    if (what == 3 && cudaMemsetAsync(out, 0, l2_per_cta * blocks * 16, st) != cudaSuccess) ok = false;
    double work = 0.0;
    for (int rep = 0; rep < 2 && ok; ++rep) {  // first pass warms up
        ok = cudaEventRecord(e0, st) == cudaSuccess;
        if (what == 0) add_probe<double><<<blocks, kProbeThreads, 0, st>>>((double*)out, 1.0);
        else if (what == 1) add_probe<float><<<blocks, kProbeThreads, 0, st>>>((float*)out, 1.0f);
        else if (what == 2) smem_probe<<<blocks, kProbeThreads, 0, st>>>((float*)out, smem_iters);
        else if (what == 4) i64_probe<<<blocks, kProbeThreads, 0, st>>>((long long*)out, 1ll);
        else l2_probe<<<blocks, kProbeThreads, 0, st>>>((float4*)out, l2_per_cta, l2_iters);
        ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess;
    }
    ok = cudaStreamSynchronize(st) == cudaSuccess && ok;
    float ms = 0.0f;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f;
    if (what <= 1 || what == 4) work = (double)blocks * kProbeThreads * kProbeIters * 16.0;  // adds
    else if (what == 2) work = (double)blocks * kProbeThreads * smem_iters * 4.0 * 2.0 * 4.0;  // bytes (load + store)
    else work = (double)blocks * (double)l2_per_cta * l2_iters * 16.0 * 2.0;                 // bytes (load + store)
    if (ok) *value = work / (ms * 1e-3);  // left untouched on any failure
    else rc = POTTS_LR_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaStreamDestroy(st);
    return rc;
}
