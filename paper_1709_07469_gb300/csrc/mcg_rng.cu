// mcg_rng.cu -- the walk's random numbers exposed for verification: raw
// Philox4x32-10 blocks and the normals of given step blocks, computed by the
// same device functions the walk kernels inline.
#include <cuda_runtime.h>

#include "mcg_device.cuh"
#include "mcg_internal.h"

namespace mcg {

namespace {

__global__ void philox_kernel(const uint4* __restrict__ ctr, const uint2* __restrict__ key, int64_t n,
                              uint4* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 k = key[i];
    out[i] = philox4x32_10(ctr[i], k.x, k.y);
}

__global__ void normals_f64_kernel(uint32_t k0, uint32_t k1, uint32_t s, uint32_t p, uint32_t b0, int64_t nb,
                                   double* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double z[12];
    normals12_f64(s, p, b0 + (uint32_t)i, k0, k1, z);
    for (int j = 0; j < 12; ++j) out[12 * i + j] = z[j];
}

__global__ void normals_f32_kernel(uint32_t k0, uint32_t k1, uint32_t s, uint32_t p, uint32_t b0, int64_t nb,
                                   float* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    float z[12];
    // unit step scale: lnscale = -2 ln 2
    normals12_f32(s, p, b0 + (uint32_t)i, k0, k1, -1.3862943611198906f, z);
    for (int j = 0; j < 12; ++j) out[12 * i + j] = z[j];
}

}  // namespace

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t g = (n + 255) / 256;
    philox_kernel<<<(unsigned)g, 256, 0, st>>>((const uint4*)ctr, (const uint2*)key, n, (uint4*)out);
    return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t s, uint32_t p, uint32_t b0, int64_t nblocks, int precision,
                           void* out, cudaStream_t st)
{
    if (nblocks <= 0) return cudaSuccess;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int64_t g = (nblocks + 127) / 128;
    if (precision == MCG_FP64)
        normals_f64_kernel<<<(unsigned)g, 128, 0, st>>>(k0, k1, s, p, b0, nblocks, (double*)out);
    else
        normals_f32_kernel<<<(unsigned)g, 128, 0, st>>>(k0, k1, s, p, b0, nblocks, (float*)out);
    return cudaGetLastError();
}

}  // namespace mcg
