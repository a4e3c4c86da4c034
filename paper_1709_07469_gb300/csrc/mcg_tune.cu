// mcg_tune.cu -- launch autotuning and the moving-average smoothing of a
// station line (host code).
#include <cstring>

#include <cuda_runtime.h>

#include "mcg_internal.h"
#include "mcgrav.h"

using namespace mcg;

extern "C" {

int mcg_autotune(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
                 const double* stations_dev, int64_t S, double dt, uint64_t seed, mcg_options* opts)
{
    if (!opts || !stations_dev || S <= 0) return set_error(MCG_ERR_ARG, "autotune needs options and stations");
    WalkParams P;
    mcg_options o = *opts;
    o.max_steps = 2048;  // every path runs exactly 2048 RNG-steps: no exit tail in the timing
    o.block = 128;
    o.refill_min = 1;
    int rc = make_params(domain, density, boundary, dt, seed, &o, P);
    if (rc) return rc;
    // about 2.6e5 timed walks in all (a few per lane of the persistent grid),
    // at most 2048 per station: enough to fill the GPU without a large scratch
    int64_t N = (262144 + S - 1) / S;
    if (N > 2048) N = 2048;
    const size_t n = (size_t)S * (size_t)N;
    const size_t work = mcg_walk_work_bytes(S, N, o.precision);
    const size_t bytes = 3 * align256(n * sizeof(double)) + align256(work) + 256;
    char* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MCG_ERR_OOM, "autotune scratch: %s", cudaGetErrorString(e));
    }
    P.stations = stations_dev;
    P.S = S;
    P.N = N;
    P.p0 = 0;
    P.total = (unsigned long long)n;
    P.pp_u = (double*)buf;
    P.pp_d = (double*)(buf + align256(n * sizeof(double)));
    P.pp_steps = (int64_t*)(buf + 2 * align256(n * sizeof(double)));
    char* w = buf + 3 * align256(n * sizeof(double));
    if (o.precision == MCG_MIXED) {
        P.frec = (float*)w;
        P.drec = (double*)(w + align256(n * 3 * 8 * sizeof(float)));
    }
    P.status = (int32_t*)(w + align256(work));
    P.counter = (unsigned long long*)(w + align256(work) + 128);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks[3] = {64, 96, 128};
    const int refills[3] = {1, 4, 16};
    float best = 1e30f;
    int best_block = 128, best_refill = 1;
    rc = MCG_OK;
    for (int rep = 0; rep < 2 && rc == MCG_OK; ++rep) {  // the first pass warms up
        for (int bi = 0; bi < 3 && rc == MCG_OK; ++bi)
            for (int ri = 0; ri < 3 && rc == MCG_OK; ++ri) {
                P.refill_min = refills[ri];
                if ((e = cudaMemset(P.counter, 0, sizeof(unsigned long long))) || (e = cudaEventRecord(a)) ||
                    (e = launch_walk(P, o.precision, blocks[bi], 0)) || (e = cudaEventRecord(b)) ||
                    (e = cudaEventSynchronize(b))) {
                    rc = set_error(MCG_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(e));
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep == 1 && ms < best) {
                    best = ms;
                    best_block = blocks[bi];
                    best_refill = refills[ri];
                }
            }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    if (rc) return rc;
    opts->block = best_block;
    opts->refill_min = best_refill;
    return MCG_OK;
}

int mcg_smooth_moving_average(const double* y, int64_t n, int32_t span, double* out)
{
    if (n < 0 || span < 1) return set_error(MCG_ERR_ARG, "need n >= 0 and span >= 1");
    if (n == 0) return MCG_OK;
    if (!y || !out || y == out) return set_error(MCG_ERR_ARG, "y and out must be distinct host arrays");
    if (span % 2 == 0) span -= 1;
    const int64_t half = span / 2;
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = half;
        if (i < k) k = i;
        if (n - 1 - i < k) k = n - 1 - i;
        double s = 0.0;
        for (int64_t j = i - k; j <= i + k; ++j) s += y[j];
        out[i] = s / (double)(2 * k + 1);
    }
    return MCG_OK;
}

}  // extern "C"
