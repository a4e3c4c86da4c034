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
    o.max_steps = 2048;  // stage 1: every path runs exactly 2048 RNG-steps, no exit tail in the timing
    o.block = 128;
    o.refill_min = 1;
    int rc = make_params(domain, density, boundary, dt, seed, &o, P);
    if (rc) return rc;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Stage 1 (stepping rate): about 2.6e5 capped walks (a few per lane of the
    // persistent grid), at most 2048 per station.  Stage 2 (exit-time tail):
    // uncapped walks, two per resident lane, so the launch ends in the tail
    // that migration shortens.
    int64_t N1 = (262144 + S - 1) / S;
    if (N1 > 2048) N1 = 2048;
    const int kind = (P.rho_kind == MCG_RHO_VOXEL && P.zq) ? kRhoVoxelPacked : P.rho_kind;
    const int64_t lanes = (int64_t)sms * walk_blocks_per_sm(o.precision, kind, 128) * 128;
    int64_t N2 = (2 * lanes + S - 1) / S;
    if ((double)N2 * (double)S > 1048576.0) N2 = (1048576 + S - 1) / S;
    if (N2 < 1) N2 = 1;
    const bool stage2 = o.precision == MCG_MIXED;
    const int64_t Nmax = (stage2 && N2 > N1) ? N2 : N1;
    const size_t n = (size_t)S * (size_t)Nmax;
    const size_t work = mcg_walk_work_bytes(S, Nmax, o.precision);
    const size_t bytes = 3 * align256(n * sizeof(double)) + align256(work) + 256;
    char* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MCG_ERR_OOM, "autotune scratch: %s", cudaGetErrorString(e));
    }
    char* w = buf + 3 * align256(n * sizeof(double));
    P.stations = stations_dev;
    P.S = S;
    P.p0 = 0;
    P.pp_u = (double*)buf;
    P.pp_d = (double*)(buf + align256(n * sizeof(double)));
    P.pp_steps = (int64_t*)(buf + 2 * align256(n * sizeof(double)));
    P.status = (int32_t*)(w + align256(work));
    P.counter = (unsigned long long*)(w + align256(work) + 128);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // times one launch of the current P (block threads) in ms, or < 0 on error
    auto timed = [&](int block) -> float {
        float ms = -1.0f;
        if ((e = reset_walk(P, 0)) || (e = cudaEventRecord(a)) || (e = launch_walk(P, o.precision, block, 0)) ||
            (e = cudaEventRecord(b)) || (e = cudaEventSynchronize(b)))
            return -1.0f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    };
    // median of three timings
    auto med3 = [](const float* t) {
        const float a = t[0], b = t[1], c = t[2];
        return a > b ? (b > c ? b : (a > c ? c : a)) : (a > c ? a : (b > c ? c : b));
    };
    // Stage 1: block size, on capped walks (every walk of a warp ends at the
    // cap together, so the refill policy plays no part here); one warm-up
    // launch, then the median of three launches per candidate.
    const int blocks[3] = {64, 96, 128};
    int best_block = 128, best_refill = 1, best_spill = P.spill_max;
    rc = MCG_OK;
    P.N = N1;
    P.total = (unsigned long long)S * (unsigned long long)N1;
    if (o.precision == MCG_MIXED) bind_work(P, w, false);
    {
        float t1[3][3];
        if (timed(128) < 0.0f) rc = set_error(MCG_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(e));
        for (int rep = 0; rep < 3 && rc == MCG_OK; ++rep)
            for (int bi = 0; bi < 3 && rc == MCG_OK; ++bi) {
                t1[bi][rep] = timed(blocks[bi]);
                if (t1[bi][rep] < 0.0f) rc = set_error(MCG_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(e));
            }
        float best = 1e30f;
        for (int bi = 0; bi < 3 && rc == MCG_OK; ++bi)
            if (med3(t1[bi]) < best) {
                best = med3(t1[bi]);
                best_block = blocks[bi];
            }
    }
    // Stage 2 (mixed walk): refill threshold x spill threshold, on uncapped
    // walks whose launch ends in the exit-time tail (refills happen as walks
    // exit at random steps, and migration shortens the tail).  One timing per
    // candidate is noisy there: the median of three decides, and the default
    // (refill 1, the options' spill threshold) stays unless another pair is
    // faster by more than 1 %.
    if (rc == MCG_OK && o.precision == MCG_MIXED) {
        P.max_steps = opts->max_steps;
        P.N = N2;
        P.total = (unsigned long long)S * (unsigned long long)N2;
        bind_work(P, w, o.migrate != 0);
        const int refills[3] = {1, 4, 16};
        const int spills_m[4] = {8, 16, 24, 32};
        const int dflt_spill = P.spill_max;
        const int* spills = o.migrate ? spills_m : &dflt_spill;
        const int ns = o.migrate ? 4 : 1;
        float t2[3][4][3];
        P.refill_min = 1;
        const float warm = timed(best_block);
        if (warm < 0.0f) rc = set_error(MCG_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(e));
        const bool too_long = warm > 2000.0f;  // very long walks: keep the defaults
        for (int rep = 0; rep < 3 && rc == MCG_OK && !too_long; ++rep)
            for (int ri = 0; ri < 3 && rc == MCG_OK; ++ri)
                for (int si = 0; si < ns && rc == MCG_OK; ++si) {
                    P.refill_min = refills[ri];
                    P.spill_max = spills[si];
                    t2[ri][si][rep] = timed(best_block);
                    if (t2[ri][si][rep] < 0.0f)
                        rc = set_error(MCG_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(e));
                }
        best_spill = dflt_spill;
        if (rc == MCG_OK && !too_long) {
            float med_dflt = -1.0f;
            for (int si = 0; si < ns; ++si)
                if (spills[si] == dflt_spill) med_dflt = med3(t2[0][si]);
            float best2 = med_dflt > 0.0f ? med_dflt / 1.01f : 1e30f;
            for (int ri = 0; ri < 3; ++ri)
                for (int si = 0; si < ns; ++si)
                    if (med3(t2[ri][si]) < best2) {
                        best2 = med3(t2[ri][si]);
                        best_refill = refills[ri];
                        best_spill = spills[si];
                    }
        }
        if (too_long) best_spill = opts->spill_max > 0 ? opts->spill_max : 24;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    if (rc) return rc;
    opts->block = best_block;
    opts->refill_min = best_refill;
    opts->spill_max = best_spill;
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
