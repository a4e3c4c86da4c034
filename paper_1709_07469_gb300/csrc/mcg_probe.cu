// mcg_probe.cu -- measured instruction-issue peaks of the GPU, the
// denominators of the walks' rooflines.  The mixed walk is bound by plain
// 32-bit lane arithmetic (integer multiplies and xors of the generator, float
// arithmetic of the transform and the step), so its roofline is the rate at
// which the SMs issue lane instructions; the plain double-precision walk is
// bound by the FP64 pipe, so its roofline is the DFMA rate.  These kernels
// issue long runs of independent instructions of one kind and time them with
// CUDA events.
#include <cstdint>

#include <cuda_runtime.h>

#include "mcg_internal.h"
#include "mcgrav.h"

namespace mcg {
namespace {

constexpr int kChains = 8;        // independent dependency chains per thread
constexpr int kProbeThreads = 256;

// kind 0: FFMA on every chain; kind 1: FFMA on even chains, three-input xor
// on odd chains (the two pipes the walk mostly uses, issued side by side).
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) issue_probe_kernel(int iters, float* sink)
{
    float f[kChains];
    uint32_t u[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        f[c] = 1.0f + 1e-7f * (float)(threadIdx.x + c);
        u[c] = threadIdx.x * 2654435761u + c;
    }
    const float a = 0.999999f, b = 1e-7f;
    const uint32_t k1 = 0x9E3779B9u, k2 = 0xBB67AE85u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == 0 || (c & 1) == 0) {
                    f[c] = fmaf(f[c], a, b);
                } else {
                    uint32_t v;
                    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(v) : "r"(u[c]), "r"(k1 + r), "r"(k2));
                    u[c] = v;
                }
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += f[c] + (float)(u[c] & 1u);
    if (s == 12345.0f) *sink = s;  // keeps the chains alive; never true in practice
}

// kind 2: DFMA on every chain (the double-precision pipe).
__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(int iters, float* sink)
{
    double f[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) f[c] = 1.0 + 1e-9 * (double)(threadIdx.x + c);
    const double a = 0.9999999999, b = 1e-12;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) f[c] = fma(f[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += f[c];
    if (s == 12345.0) *sink = (float)s;  // keeps the chains alive; never true in practice
}

const void* probe_fn(int kind)
{
    return kind == 0 ? (const void*)issue_probe_kernel<0>
                     : (kind == 1 ? (const void*)issue_probe_kernel<1> : (const void*)dfma_probe_kernel);
}

}  // namespace
}  // namespace mcg

using namespace mcg;

extern "C" int mcg_issue_probe(int32_t kind, int32_t iters, double* lane_ops_per_s, double* seconds)
{
    if (kind < 0 || kind > 2)
        return set_error(MCG_ERR_ARG, "kind must be 0 (FFMA), 1 (FFMA + LOP3) or 2 (DFMA)");
    if (iters <= 0) return set_error(MCG_ERR_ARG, "iters must be positive");
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_fn(kind), kProbeThreads, 0);
    if (e) return set_error(MCG_ERR_CUDA, "probe set-up: %s", cudaGetErrorString(e));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    float* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float))) || (e = cudaEventCreate(&a)) || (e = cudaEventCreate(&b))) {
        if (sink) cudaFree(sink);
        if (a) cudaEventDestroy(a);
        return set_error(MCG_ERR_CUDA, "probe set-up: %s", cudaGetErrorString(e));
    }
    float ms = 0.f;
    for (int rep = 0; rep < 2 && !e; ++rep) {  // the first launch warms up
        if ((e = cudaEventRecord(a, 0))) break;
        if (kind == 0) issue_probe_kernel<0><<<blocks, kProbeThreads>>>(iters, sink);
        else if (kind == 1) issue_probe_kernel<1><<<blocks, kProbeThreads>>>(iters, sink);
        else dfma_probe_kernel<<<blocks, kProbeThreads>>>(iters, sink);
        if ((e = cudaGetLastError()) || (e = cudaEventRecord(b, 0)) || (e = cudaEventSynchronize(b))) break;
        e = cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e) return set_error(MCG_ERR_CUDA, "probe launch: %s", cudaGetErrorString(e));
    const double ops = (double)blocks * kProbeThreads * (double)iters * 16.0 * kChains;
    if (seconds) *seconds = ms * 1e-3;
    if (lane_ops_per_s) *lane_ops_per_s = ops / (ms * 1e-3);
    return MCG_OK;
}
