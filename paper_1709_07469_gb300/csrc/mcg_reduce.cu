// mcg_reduce.cu -- per-station statistics (the Monte Carlo mean of Eq. 7,
// the sample variance and the standard error).
//
// One block per station reads the batch's per-path values twice: pass 1 the
// mean, pass 2 the sum of squared deviations about it.  Each thread sums a
// fixed strided subset with Neumaier compensation; the block then combines
// the partials with warp shuffles (a butterfly over each warp's lanes, then
// the same over the warps' sums), always in the same order, so the result
// does not depend on scheduling.  The batch statistics are merged into the
// running state with Chan's formula, batch after batch in the order the host
// issues them.
#include <cuda_runtime.h>

#include "mcg_internal.h"

namespace mcg {

namespace {

constexpr int kReduceThreads = 256;

struct Neumaier {
    double s = 0.0, c = 0.0;
    __device__ void add(double x)
    {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ double value() const { return s + c; }
};

// Block sum of one value per thread in a fixed order: a butterfly over the
// lanes of each warp (__shfl_xor_sync: lanes i and i ^ o add the same two
// numbers, so every lane ends with the same warp sum), then the same over the
// warps' sums; every thread returns the block's sum.
template <typename T>
__device__ T block_sum(T v, T* sh)
{
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __syncthreads();  // the previous call's readers are done with sh
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T r = lane < kReduceThreads / 32 ? sh[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
    return r;
}

__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const double* __restrict__ pp_u,
                                                                const double* __restrict__ pp_d,
                                                                const int64_t* __restrict__ pp_steps, int64_t N,
                                                                mcg_station_state* __restrict__ states)
{
    __shared__ double sh[kReduceThreads / 32];
    __shared__ unsigned long long shs[kReduceThreads / 32];
    const int64_t s = blockIdx.x;
    const double* u = pp_u + s * N;
    const double* d = pp_d + s * N;
    const int64_t* st = pp_steps + s * N;
    const int t = threadIdx.x;

    Neumaier su, sd;
    unsigned long long steps = 0ull;
    for (int64_t i = t; i < N; i += kReduceThreads) {
        su.add(u[i]);
        sd.add(d[i]);
        steps += (unsigned long long)st[i];
    }
    const double nb = (double)N;
    const double mean_u = block_sum(su.value(), sh) / nb;
    const double mean_d = block_sum(sd.value(), sh) / nb;

    Neumaier qu, qd;
    for (int64_t i = t; i < N; i += kReduceThreads) {
        const double a = u[i] - mean_u, b = d[i] - mean_d;
        qu.add(a * a);
        qd.add(b * b);
    }
    const double m2_u = block_sum(qu.value(), sh);
    const double m2_d = block_sum(qd.value(), sh);

    const unsigned long long steps_all = block_sum(steps, shs);

    if (t == 0) {
        mcg_station_state a = states[s];
        const double na = a.n;
        if (na == 0.0) {
            a.mean_u = mean_u;
            a.m2_u = m2_u;
            a.mean_d = mean_d;
            a.m2_d = m2_d;
        } else {
            const double n = na + nb;
            const double du = mean_u - a.mean_u, dd = mean_d - a.mean_d;
            a.mean_u = a.mean_u + du * (nb / n);
            a.m2_u = a.m2_u + m2_u + du * du * (na * nb / n);
            a.mean_d = a.mean_d + dd * (nb / n);
            a.m2_d = a.m2_d + m2_d + dd * dd * (na * nb / n);
        }
        a.n = na + nb;
        a.steps = a.steps + (double)steps_all;
        states[s] = a;
    }
}

__global__ void finalize_kernel(const mcg_station_state* __restrict__ states, int64_t S, double* u, double* gz,
                                double* se_u, double* se_gz, int64_t* n_paths, int64_t* path_steps)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const mcg_station_state a = states[s];
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (u) u[s] = a.mean_u;
    if (gz) gz[s] = a.mean_d;
    if (se_u) se_u[s] = a.n > 1.0 ? sqrt(a.m2_u / (a.n - 1.0) / a.n) : nan;
    if (se_gz) se_gz[s] = a.n > 1.0 ? sqrt(a.m2_d / (a.n - 1.0) / a.n) : nan;
    if (n_paths) n_paths[s] = (int64_t)a.n;
    if (path_steps) path_steps[s] = (int64_t)a.steps;
}

}  // namespace

void preload_reduce_kernels()
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, (const void*)reduce_kernel) != cudaSuccess) cudaGetLastError();
    if (cudaFuncGetAttributes(&a, (const void*)finalize_kernel) != cudaSuccess) cudaGetLastError();
}

cudaError_t launch_reduce(const double* pp_u, const double* pp_d, const int64_t* pp_steps, int64_t S, int64_t N,
                          mcg_station_state* states, cudaStream_t st)
{
    if (S <= 0 || N <= 0) return cudaSuccess;
    reduce_kernel<<<(unsigned)S, kReduceThreads, 0, st>>>(pp_u, pp_d, pp_steps, N, states);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const mcg_station_state* states, int64_t S, double* u, double* gz, double* se_u,
                            double* se_gz, int64_t* n_paths, int64_t* path_steps, cudaStream_t st)
{
    if (S <= 0) return cudaSuccess;
    finalize_kernel<<<(unsigned)((S + 127) / 128), 128, 0, st>>>(states, S, u, gz, se_u, se_gz, n_paths,
                                                                 path_steps);
    return cudaGetLastError();
}

}  // namespace mcg
