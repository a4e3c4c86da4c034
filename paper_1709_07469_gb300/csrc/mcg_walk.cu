// mcg_walk.cu -- the walk kernels (Sec. 2.3 of the paper, steps 1-4).
//
// Both kernels are persistent: every warp keeps 32 walks in flight and, as
// walks exit, refills the free lanes from a global work counter with one
// warp-aggregated atomic (__ballot_sync / __shfl_sync), so lanes do not idle
// behind the long exit-time tail.  A lane owns one path (station s, path p)
// and its common-random-number copies x0, x0 + h e_z, x0 - h e_z, which share
// every Gaussian increment.  Random numbers come four steps at a time: three
// Philox4x32-10 calls -> twelve normals -> four Euler-Maruyama steps.
//
//  * walk_fp64_kernel : the plain double-precision walk; its arithmetic
//    follows the problem statement operation by operation (no contraction)
//    so that a path agrees with a plain double-precision evaluation to
//    rounding of the transcendental functions.
//  * walk_mixed_kernel: single-precision stepping, random-number transform
//    and density lookup; the source integral keeps single-precision partial
//    sums over at most 64 steps which are flushed into a double accumulator;
//    the exit-segment clip, the boundary value and the per-path estimate are
//    double precision and run in exit_mixed_kernel.  Once the work list is
//    used up, walks migrate from sparse warps to warps with free lanes.
//
// Launch shape: 128 threads, at least MCG_MIXED_MINB blocks per SM (the
// register bound that gave the best rate; the grid is sized from the
// occupancy the compiled kernel actually gets).
#include <type_traits>

#include <cuda_runtime.h>

#include "mcg_device.cuh"
#include "mcg_internal.h"

namespace mcg {

namespace {

#ifndef MCG_MIXED_MINB
#define MCG_MIXED_MINB 5
#endif

constexpr unsigned kFull = 0xffffffffu;
constexpr double kNaN = __builtin_nan("");


// Claims new items for the lanes of this warp that are free.  Returns the
// claimed item in `item`; lanes beyond the end of the work list become
// `exhausted`.
__device__ __forceinline__ bool refill(const WalkParams& P, bool busy, bool& exhausted,
                                       unsigned long long& item)
{
    const unsigned want = __ballot_sync(kFull, !busy && !exhausted);
    if (want == 0u) return false;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(want) - 1;
    unsigned long long base = 0ull;
    if (lane == leader) base = atomicAdd(P.counter, (unsigned long long)__popc(want));
    base = __shfl_sync(kFull, base, leader);
    if (busy || exhausted) return false;
    item = base + (unsigned long long)__popc(want & ((1u << lane) - 1u));
    if (item >= P.total) {
        exhausted = true;
        return false;
    }
    return true;
}

// A station whose walk copies are not all strictly inside Omega gets NaN
// and the MCG_ERR_ARG bit (mcgrav_solve rejects such stations up front).
__device__ __forceinline__ bool station_ok(const WalkParams& P, const double* stations, int32_t* status, uint32_t s,
                                           unsigned long long item)
{
    const double x = stations[3 * s], y = stations[3 * s + 1], z = stations[3 * s + 2];
    bool ok;
    if (P.ball) {
        const double dx = x - P.cen[0], dy = y - P.cen[1], dz = z - P.cen[2];
        const double q = dx * dx + dy * dy;
        ok = q + dz * dz < P.R2 && q + (dz + P.h) * (dz + P.h) < P.R2 && q + (dz - P.h) * (dz - P.h) < P.R2;
    } else {
        ok = x > P.lo[0] && x < P.hi[0] && y > P.lo[1] && y < P.hi[1] && z - P.h > P.lo[2] && z + P.h < P.hi[2] &&
             z > P.lo[2] && z < P.hi[2];
    }
    if (!ok) {
        P.pp_u[item] = kNaN;
        P.pp_d[item] = kNaN;
        P.pp_steps[item] = 0;  // no completion flag: the mixed walk's exit kernel writes NaN too
        atomicOr(status, 1 << MCG_ERR_ARG);
    }
    return ok;
}

__device__ __forceinline__ int64_t nstep_of(uint32_t blk, int m) { return 4 * (int64_t)blk + m + 1; }

// The cancel flag may live in host-mapped or device memory and is written
// by the host while the kernel runs: read it with a system-scope relaxed
// load so the write is observed whatever caches the line.
__device__ __forceinline__ bool cancelled(const WalkParams& P)
{
    int c = 0;
    if ((threadIdx.x & 31) == 0 && P.cancel != nullptr)
        asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(c) : "l"((const void*)P.cancel) : "memory");
    return __shfl_sync(kFull, c, 0) != 0;
}

// ---------------------------------------------------------------------------
// Migration of walks between warps (mixed walk).  Once the work list is used
// up, a warp's lanes empty one by one as its walks exit, and a warp with a
// few long walks left would keep issuing instructions for 32 lanes to the
// end.  Such a warp (at most P.spill_max walks live, migration on) writes its
// walks to the pool and leaves; warps with free lanes claim pooled walks.
// A walk's state is all of it: the random streams are keyed by (station,
// path, step), so where a walk continues does not change its numbers.
//   reserve: CAS on pool_ctr[0] below pool_cap; entries written, then the
//            slot's ready flag set with release semantics;
//   claim  : CAS on pool_ctr[1] below pool_ctr[0]; acquire on the ready flag
//            (a bounded wait: the producer is a running warp between its
//            reservation and its store, so the flag comes);
//   leave  : a warp with no walks adds 1 to pool_ctr[2]; the last warp to
//            leave (count = all warps of the grid) sees every earlier spill
//            and, if the pool still holds walks, takes them over.
// Each warp spills at most once, so slots are never reused.
// ---------------------------------------------------------------------------
#ifndef MCG_SPILL_BACKLOG
#define MCG_SPILL_BACKLOG 64
#endif
constexpr unsigned long long kSpillBacklog = MCG_SPILL_BACKLOG;  // ... while fewer pooled walks wait
constexpr int kReadySpin = 1 << 20;                   // bounded wait for a ready flag (~0.1 s)

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* a)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* a)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* a, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Leader: claims up to `want` pooled walks; returns the count, first slot in base.
__device__ __forceinline__ unsigned pool_take(const WalkParams& P, unsigned want, unsigned long long& base)
{
    for (int t = 0; t < 32; ++t) {
        const unsigned long long r = ld_acquire_u64(P.pool_ctr);
        const unsigned long long c = ld_acquire_u64(P.pool_ctr + 1);
        if (c >= r) return 0u;
        const unsigned long long k = (r - c) < want ? (r - c) : want;
        if (atomicCAS(P.pool_ctr + 1, c, c + k) == c) {
            base = c;
            return (unsigned)k;
        }
    }
    return 0u;
}

// Leader: reserves n slots if the pool has room and few walks wait there.
__device__ __forceinline__ bool pool_reserve(const WalkParams& P, unsigned n, unsigned long long& base)
{
    for (int t = 0; t < 32; ++t) {
        const unsigned long long r = ld_acquire_u64(P.pool_ctr);
        const unsigned long long c = ld_acquire_u64(P.pool_ctr + 1);
        if (r - c >= kSpillBacklog || r + n > P.pool_cap) return false;
        if (atomicCAS(P.pool_ctr, r, r + n) == r) {
            base = r;
            return true;
        }
    }
    return false;
}

// Leader: records that this warp has no walks.  Returns false when it was
// the last warp of the grid to leave and walks are still pooled: it must
// take them over.
__device__ __forceinline__ bool pool_leave(const WalkParams& P, bool stop)
{
    __threadfence();
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long prev = atomicAdd(P.pool_ctr + 2, 1ull);
    if (stop || prev + 1ull != warps) return true;
    __threadfence();
    if (ld_acquire_u64(P.pool_ctr + 1) < ld_acquire_u64(P.pool_ctr)) {
        atomicAdd(P.pool_ctr + 2, ~0ull);  // -1: still here
        return false;
    }
    return true;
}

// Fraction theta in [0, 1] of the step X -> X + dW (coordinates relative to
// the ball centre) at which the segment leaves the ball of radius R: the
// positive root of |X + theta dW|^2 = R^2 in the form without cancellation.
__device__ __forceinline__ double ball_theta(const double* q, const double* dW, double R2)
{
    double a = 0.0, b = 0.0, c = -R2;
    for (int k = 0; k < 3; ++k) {
        a = __dadd_rn(a, __dmul_rn(dW[k], dW[k]));
        b = __dadd_rn(b, __dmul_rn(__dmul_rn(2.0, q[k]), dW[k]));
        c = __dadd_rn(c, __dmul_rn(q[k], q[k]));
    }
    const double D = __dadd_rn(__dmul_rn(b, b), -__dmul_rn(__dmul_rn(4.0, a), c));
    const double t = (b >= 0.0) ? __ddiv_rn(__dmul_rn(-2.0, c), __dadd_rn(b, __dsqrt_rn(D)))
                                : __ddiv_rn(__dadd_rn(-b, __dsqrt_rn(D)), __dmul_rn(2.0, a));
    return fmin(fmax(t, 0.0), 1.0);
}

// ---------------------------------------------------------------------------
// Exit handling (double precision).  X: last inside point, Y: first point
// not strictly inside, both as the walk computed them.  Clips the segment at
// its first boundary crossing (lowest axis on ties), closes the trapezoid
// over the clipped part and returns g(x*) - 2 pi G I.
// ---------------------------------------------------------------------------
__device__ __noinline__ double exit_fp64(const WalkParams& P, const ModelRef& M, const double* X, const double* dW,
                                         const double* Y, double I, double rp)
{
    double xs[3];
    double theta = 1.0;
    int face = -1;
    if (P.clip && P.ball) {
        const double q[3] = {__dadd_rn(X[0], -P.cen[0]), __dadd_rn(X[1], -P.cen[1]), __dadd_rn(X[2], -P.cen[2])};
        theta = ball_theta(q, dW, P.R2);
        for (int k = 0; k < 3; ++k) xs[k] = __dadd_rn(X[k], __dmul_rn(theta, dW[k]));
    } else if (P.clip) {
        int kstar = -1;
        double tmin = __longlong_as_double(0x7ff0000000000000LL), bstar = 0.0;
        for (int k = 0; k < 3; ++k) {
            double b;
            if (Y[k] <= P.lo[k]) b = P.lo[k];
            else if (Y[k] >= P.hi[k]) b = P.hi[k];
            else continue;
            const double t = __ddiv_rn(__dadd_rn(b, -X[k]), dW[k]);
            if (t < tmin) {
                tmin = t;
                kstar = k;
                bstar = b;
            }
        }
        if (kstar < 0) return kNaN;
        theta = fmin(fmax(tmin, 0.0), 1.0);
        for (int k = 0; k < 3; ++k) xs[k] = __dadd_rn(X[k], __dmul_rn(theta, dW[k]));
        xs[kstar] = bstar;
        face = 2 * kstar + (bstar == P.hi[kstar] ? 1 : 0);
    } else {
        xs[0] = Y[0];
        xs[1] = Y[1];
        xs[2] = Y[2];
    }
    const double r = rho_f64(P, M, xs);
    I = __dadd_rn(I, __dmul_rn(__dmul_rn(__dmul_rn(0.5, __dadd_rn(rp, r)), theta), P.dt));
    return __dadd_rn(boundary_value(P, M, face, xs), -__dmul_rn(P.two_pi_G, I));
}

// Mixed walk exit (run by exit_mixed_kernel, one thread per path, so the
// double-precision work is convergent): X, Y relative to the box centre in
// single precision as the walk computed them; the walk's sum acc (flushed +
// partial) is S = rho_0 / 2 + sum_{n=1}^{N-1} rho_n, so the trapezoid integral
// over the inside steps is dt (S - rho_{N-1} / 2).
__device__ __forceinline__ double exit_mixed(const WalkParams& P, const ModelRef& M, const float* Xf, const float* Yf,
                                             double acc, float rp)
{
    double X[3], dW[3], xs[3];
    for (int k = 0; k < 3; ++k) {
        X[k] = (double)Xf[k];
        dW[k] = (double)Yf[k] - (double)Xf[k];
    }
    double theta = 1.0;
    int face = -1;
    if (P.clip && P.ball) {
        theta = ball_theta(X, dW, P.R2);
        for (int k = 0; k < 3; ++k) xs[k] = P.cen[k] + (X[k] + theta * dW[k]);
    } else if (P.clip) {
        int kstar = -1;
        double tmin = __longlong_as_double(0x7ff0000000000000LL);
        for (int k = 0; k < 3; ++k) {
            if (!(fabsf(Yf[k]) >= P.half_f[k])) continue;  // the test that ended the walk
            const double b = (Yf[k] > 0.f ? P.hi[k] : P.lo[k]) - P.cen[k];
            const double t = (b - X[k]) / dW[k];
            if (t < tmin) {
                tmin = t;
                kstar = k;
            }
        }
        if (kstar < 0) return kNaN;
        theta = fmin(fmax(tmin, 0.0), 1.0);
        for (int k = 0; k < 3; ++k) xs[k] = P.cen[k] + (X[k] + theta * dW[k]);
        const bool upper = Yf[kstar] > 0.f;
        xs[kstar] = upper ? P.hi[kstar] : P.lo[kstar];
        face = 2 * kstar + (upper ? 1 : 0);
    } else {
        for (int k = 0; k < 3; ++k) xs[k] = P.cen[k] + (double)Yf[k];
    }
    const double r = rho_f64(P, M, xs);
    const double rpd = (double)rp;
    const double I = P.dt * (acc - 0.5 * rpd) + 0.5 * theta * P.dt * (rpd + r);
    return boundary_value<true>(P, M, face, xs) - P.two_pi_G * I;
}

// Exit record of copy c of item `item` (record c * total + item of frec):
// 32 bytes, written as two 16-byte stores that fill one sector -- X (the walk
// position before the exit step, copy 0's coordinates; copy c adds its z
// offset), Y (the copy's first point not strictly inside Omega) and the
// source sum flushed + partial in double.  rho at X is not stored:
// exit_mixed_kernel evaluates the same single-precision density function at
// the same X, which gives the walk's value bit for bit.  The record is valid
// once the item's step count carries kDoneFlag.
__device__ __forceinline__ void put_exit(const WalkParams& P, int c, unsigned long long item, float x0, float x1,
                                         float x2, float y0, float y1, float y2, float partial, double flushed)
{
    const double acc = flushed + (double)partial;
    float4* r = (float4*)P.frec + 2 * ((size_t)c * P.total + item);
    r[0] = make_float4(x0, x1, x2, y0);
    r[1] = make_float4(y1, y2, __int_as_float(__double2loint(acc)), __int_as_float(__double2hiint(acc)));
}

__device__ __forceinline__ void write_path(const WalkParams& P, int32_t* status, unsigned long long item, double u0,
                                           double up, double um, int64_t steps)
{
    const double d = P.crn ? (up - um) / (2.0 * P.h) : kNaN;
    P.pp_u[item] = u0;
    P.pp_d[item] = d;
    P.pp_steps[item] = steps;
    const bool bad = !isfinite(u0) || (P.crn && !isfinite(d));
    if (bad) atomicOr(status, 1 << MCG_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Brownian-bridge exit test of an inside step X -> Y (the paper's Remark on
// exit-time estimation, after Gobet): the bridge crosses the plane of a face
// at distances d_X, d_Y with probability exp(-2 d_X d_Y / sd^2); with the
// faces taken as independent the step exits with probability
// 1 - prod (1 - p_face).  One uniform per RNG-step n: Philox counter
// (n / 4, p, s, 2), word n % 4, shared by the copies.  Returns the face with
// the largest p (2k lower, 2k+1 upper) if the step exits, else -1.
// ---------------------------------------------------------------------------
__device__ __noinline__ int bridge_face_f64(const WalkParams& P, const double* X, const double* Y, uint32_t s,
                                            uint32_t p, uint32_t n)
{
    double q = 1.0, pmax = -1.0;
    int kmax = -1;
    for (int f = 0; f < 6; ++f) {
        const int k = f >> 1;
        const double dX = (f & 1) ? __dadd_rn(P.hi[k], -X[k]) : __dadd_rn(X[k], -P.lo[k]);
        const double dY = (f & 1) ? __dadd_rn(P.hi[k], -Y[k]) : __dadd_rn(Y[k], -P.lo[k]);
        const double pk = exp(__ddiv_rn(__dmul_rn(__dmul_rn(-2.0, dX), dY), __dmul_rn(P.sd, P.sd)));
        q = __dmul_rn(q, __dadd_rn(1.0, -pk));
        if (pk > pmax) {
            pmax = pk;
            kmax = f;
        }
    }
    const uint4 w = philox4x32_10(make_uint4(n >> 2, p, s, 2u), P.key0, P.key1);
    const uint32_t word = (n & 3u) == 0u ? w.x : (n & 3u) == 1u ? w.y : (n & 3u) == 2u ? w.z : w.w;
    return (u01_f64(word) < 1.0 - q) ? kmax : -1;
}

// Single-precision bridge test of the copies `cand` for step m of block blk
// (walk position (wx, wy, wz) -> (nx, ny, nz), box-centre coordinates, copy c
// shifted by +h, -h in z).  Returns the mask of copies that exit and, 3 bits
// per copy, their faces.
__device__ __noinline__ unsigned bridge_exits_f32(const WalkParams& P, unsigned cand, float wx, float wy, float wz,
                                                  float nx, float ny, float nz, float hf, uint32_t s, uint32_t p,
                                                  uint32_t blk, int m, unsigned* faces)
{
    const uint4 w = philox4x32_10(make_uint4(blk, p, s, 2u), P.key0, P.key1);
    const uint32_t word = m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
    const float U = u01_f32(word);
    const float hx = P.half_f[0], hy = P.half_f[1], hz = P.half_f[2], K = P.bridge_k_f;
    const float pxy[4] = {__expf(K * (wx + hx) * (nx + hx)), __expf(K * (hx - wx) * (hx - nx)),
                          __expf(K * (wy + hy) * (ny + hy)), __expf(K * (hy - wy) * (hy - ny))};
    float qxy = 1.0f, pbest = -1.0f;
    int fbest = -1;
    for (int f = 0; f < 4; ++f) {
        qxy *= 1.0f - pxy[f];
        if (pxy[f] > pbest) {
            pbest = pxy[f];
            fbest = f;
        }
    }
    unsigned out = 0u, fb = 0u;
    for (int c = 0; c < 3; ++c) {
        if (!(cand & (1u << c))) continue;
        const float off = c == 0 ? 0.0f : (c == 1 ? hf : -hf);
        const float zX = wz + off, zY = nz + off;
        const float plo = __expf(K * (zX + hz) * (zY + hz)), phi = __expf(K * (hz - zX) * (hz - zY));
        const float q = qxy * (1.0f - plo) * (1.0f - phi);
        if (U < 1.0f - q) {
            int f = fbest;
            float pb = pbest;
            if (plo > pb) {
                pb = plo;
                f = 4;
            }
            if (phi > pb) f = 5;
            out |= 1u << c;
            fb |= (unsigned)f << (3 * c);
        }
    }
    *faces = fb;
    return out;
}

// ---------------------------------------------------------------------------
// Plain double-precision walk.
// ---------------------------------------------------------------------------
template <bool CRN, bool SEG>
__global__ void __launch_bounds__(128) walk_fp64_kernel(const WalkParams P)
{
    constexpr int NC = CRN ? 3 : 1;
    bool busy = false, exhausted = false;
    unsigned long long item = 0ull;
    uint32_t s = 0u, p = 0u;
    int64_t n = 0;
    double W[3], I[NC], rp[NC], u[3];
    unsigned alive = 0u;
    int64_t steps = 0;
    const double off[3] = {0.0, P.h, -P.h};
    unsigned iter = 0u;
    // the walk's request (its own in a multi-request launch)
    uint32_t k0 = P.key0, k1 = P.key1;
    int32_t* status = P.status;
    ModelRef M = model_of(P);

    for (;;) {
        if ((++iter & 255u) == 0u && cancelled(P)) {
            if ((threadIdx.x & 31) == 0) atomicOr(P.status, 1 << MCG_ERR_CANCELLED);
            if (busy) {  // this walk gives no result
                P.pp_u[item] = kNaN;
                P.pp_d[item] = kNaN;
                P.pp_steps[item] = steps;
            }
            busy = false;
            exhausted = true;
        }
        if (refill(P, busy, exhausted, item)) {
            const double* st = P.stations;
            unsigned long long local = item, N = (unsigned long long)P.N, p0 = (unsigned long long)P.p0;
            if constexpr (SEG) {
                const WalkSeg& g = P.seg[find_seg(P, item)];
                local = item - g.begin;
                N = (unsigned long long)g.N;
                p0 = (unsigned long long)g.p0;
                st = g.stations;
                status = g.status;
                k0 = g.key0;
                k1 = g.key1;
                M = model_of(g);
            }
            s = (uint32_t)(local / N);
            if (station_ok(P, st, status, s, item)) {
                p = (uint32_t)(p0 + local % N);
                for (int k = 0; k < 3; ++k) W[k] = st[3 * s + k];
                for (int c = 0; c < NC; ++c) {
                    const double X[3] = {W[0], W[1], __dadd_rn(W[2], off[c])};
                    rp[c] = rho_f64(P, M, X);
                    I[c] = 0.0;
                }
                u[0] = u[1] = u[2] = kNaN;
                alive = (1u << NC) - 1u;
                n = 0;
                steps = 0;
                busy = true;
            }
        }
        if (!__any_sync(kFull, busy)) break;
        if (!busy) continue;

        double z[12];
        normals12_f64(s, p, (uint32_t)(n >> 2), k0, k1, z);
#pragma unroll 1
        for (int m = 0; m < 4 && alive; ++m) {
            const double dW[3] = {__dmul_rn(P.sd, z[3 * m]), __dmul_rn(P.sd, z[3 * m + 1]),
                                  __dmul_rn(P.sd, z[3 * m + 2])};
            const double Wn[3] = {__dadd_rn(W[0], dW[0]), __dadd_rn(W[1], dW[1]), __dadd_rn(W[2], dW[2])};
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (!(alive & (1u << c))) continue;
                const double X[3] = {W[0], W[1], __dadd_rn(W[2], off[c])};
                const double Y[3] = {Wn[0], Wn[1], __dadd_rn(Wn[2], off[c])};
                steps += 1;
                bool inside;
                if (P.ball) {
                    const double dx = __dadd_rn(Y[0], -P.cen[0]), dy = __dadd_rn(Y[1], -P.cen[1]),
                                 dz = __dadd_rn(Y[2], -P.cen[2]);
                    inside = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) < P.R2;
                } else {
                    inside = Y[0] > P.lo[0] && Y[0] < P.hi[0] && Y[1] > P.lo[1] && Y[1] < P.hi[1] && Y[2] > P.lo[2] &&
                             Y[2] < P.hi[2];
                }
                // (multi-request launches run without the bridge test)
                const int kb = (!SEG && inside && P.bridge) ? bridge_face_f64(P, X, Y, s, p, (uint32_t)n) : -1;
                if (inside && kb < 0) {
                    const double r = rho_f64(P, M, Y);
                    I[c] = __dadd_rn(I[c], __dmul_rn(__dmul_rn(0.5, __dadd_rn(rp[c], r)), P.dt));
                    rp[c] = r;
                } else if (inside) {
                    // the bridge left Omega: end on face kb below Y after a full step
                    double xs[3] = {Y[0], Y[1], Y[2]};
                    xs[kb >> 1] = (kb & 1) ? P.hi[kb >> 1] : P.lo[kb >> 1];
                    const double r = rho_f64(P, M, xs);
                    const double Ic = __dadd_rn(I[c], __dmul_rn(__dmul_rn(0.5, __dadd_rn(rp[c], r)), P.dt));
                    u[c] = __dadd_rn(boundary_value(P, M, kb, xs), -__dmul_rn(P.two_pi_G, Ic));
                    alive &= ~(1u << c);
                } else {
                    u[c] = exit_fp64(P, M, X, dW, Y, I[c], rp[c]);
                    alive &= ~(1u << c);
                }
            }
            W[0] = Wn[0];
            W[1] = Wn[1];
            W[2] = Wn[2];
            ++n;
        }
        if (!alive) {
            write_path(P, status, item, u[0], u[1], u[2], steps);
            busy = false;
        } else if (n >= P.max_steps) {
            atomicOr(status, 1 << MCG_ERR_STEP_CAP);
            P.pp_u[item] = kNaN;
            P.pp_d[item] = kNaN;
            P.pp_steps[item] = steps;
            busy = false;
        }
    }
}

// ---------------------------------------------------------------------------
// Mixed-precision walk: single-precision stepping and no double-precision
// arithmetic in the step loop.  The three common-random-number copies are
// updated branch-free; exits (rare) take a side branch that writes an exit
// record, which exit_mixed_kernel turns into per-path values.  A warp runs up
// to 16 blocks (64 steps) between refills, two blocks per loop iteration;
// after them it flushes the single-precision partial sums into the double
// sums (a real, warp-uniform branch, so the slow double-precision unit sees
// one instruction per copy per 64 steps).  With a prism or sphere density in
// the box, a warp whose walks all stay, by the block's radius bound, inside
// Omega and away from the density for the next four steps only moves them
// (one test per block instead of one per step); otherwise every step tests
// the exit and samples the density.
// ---------------------------------------------------------------------------
//
// SEG: a multi-request launch (the segment table maps each item to its
// request); each lane then carries its walk's generator key and model array,
// and keeps the segment index with the walk's other cold state.
template <int RHO, bool CRN, bool BRIDGE, bool BALL, bool SEG>
__global__ void __launch_bounds__(128, MCG_MIXED_MINB) walk_mixed_kernel(const WalkParams P)
{
    static_assert(!(SEG && (BRIDGE || BALL)), "multi-request launches use the box without the bridge test");
    // Per-walk state touched only at refills, exits and flushes lives in
    // shared memory (one slot per thread); the step loop keeps the position,
    // the partial sums, the path indices and the live-copy mask in registers.
    __shared__ double sh_D[3][128];              // flushed sums per copy
    __shared__ unsigned long long sh_item[128];  // work item of the walk
    __shared__ long long sh_steps[128];          // EM steps of the copies that have exited
    __shared__ int sh_seg[SEG ? 128 : 1];        // segment of the walk (multi-request launch)
    const int t = threadIdx.x;
    bool busy = false, exhausted = false;
    uint32_t s = 0u, p = 0u, blk = 0u;
    float wx = 0.f, wy = 0.f, wz = 0.f;
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;  // single-precision partial sums
    unsigned alive = 0u;
    const float hx = P.half_f[0], hy = P.half_f[1], hz = P.half_f[2];
    const float hf = CRN ? P.h_f : 0.0f;
    unsigned round = 0u;
    const int lane = t & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    const bool migrate = P.pool != nullptr;
    bool stop = false;     // cancelled: take no more work of any kind
    bool spilled = false;  // this warp has spilled its walks once
    uint32_t k0 = P.key0, k1 = P.key1;  // generator key of the lane's walk
    ModelRef M = model_of(P);           // model arrays of the lane's walk
    // the lane's walk now belongs to the request of launch item `it`
    auto adopt = [&](unsigned long long it) {
        if constexpr (SEG) {
            const int gi = find_seg(P, it);
            const WalkSeg& g = P.seg[gi];
            k0 = g.key0;
            k1 = g.key1;
            M = model_of(g);
            sh_seg[t] = gi;
        }
    };

    for (;;) {
        if ((++round & 15u) == 0u && cancelled(P)) {
            // walks in flight, pooled walks and unclaimed items give no result
            if (lane == 0) atomicOr(P.status, 1 << MCG_ERR_CANCELLED);
            if (busy) {
                const unsigned long long it = sh_item[t];  // (no completion flag: NaN)
                P.pp_steps[it] = sh_steps[t] + (long long)__popc(alive) * 4 * (long long)blk;
            }
            busy = false;
            exhausted = true;
            stop = true;
        }
        unsigned long long item = 0ull;
        bool start = refill(P, busy, exhausted, item);
        const double* st = P.stations;
        if (start) {
            unsigned long long local = item, N = (unsigned long long)P.N, p0 = (unsigned long long)P.p0;
            int32_t* status = P.status;
            if constexpr (SEG) {
                adopt(item);
                const WalkSeg& g = P.seg[sh_seg[t]];
                local = item - g.begin;
                N = (unsigned long long)g.N;
                p0 = (unsigned long long)g.p0;
                st = g.stations;
                status = g.status;
            }
            s = (uint32_t)(local / N);
            p = (uint32_t)(p0 + local % N);
            start = station_ok(P, st, status, s, item);
        }
        if (start) {
            wx = (float)(st[3 * s + 0] - P.cen[0]);
            wy = (float)(st[3 * s + 1] - P.cen[1]);
            wz = (float)(st[3 * s + 2] - P.cen[2]);
            float r0, r1, r2;
            rho3_f32<RHO>(P, SEG ? M : model_of(P), wx, wy, wz, hf, r0, r1, r2);
            S0 = 0.5f * r0;
            S1 = 0.5f * r1;
            S2 = 0.5f * r2;
            sh_D[0][t] = sh_D[1][t] = sh_D[2][t] = 0.0;
            sh_item[t] = item;
            sh_steps[t] = 0;
            alive = CRN ? 7u : 1u;
            blk = 0u;
            busy = true;
        }
        if (migrate && !stop) {
            // the work list is used up: fill free lanes with pooled walks
            const unsigned freem = __ballot_sync(kFull, !busy);
            if (freem && __any_sync(kFull, exhausted)) {
                unsigned long long base = 0ull;
                unsigned got = 0u;
                if (lane == 0) got = pool_take(P, (unsigned)__popc(freem), base);
                got = __shfl_sync(kFull, got, 0);
                base = __shfl_sync(kFull, base, 0);
                const unsigned rank = (unsigned)__popc(freem & lanes_below);
                if (!busy && rank < got) {
                    const unsigned long long slot = base + rank;
                    uint32_t ready = 0u;
                    for (int i = 0; i < kReadySpin && !ready; ++i) {
                        ready = ld_acquire_u32(P.pool_ready + slot);
                        if (!ready) __nanosleep(64);
                    }
                    if (ready) {
                        const uint4* e = (const uint4*)(P.pool + slot * kPoolEntryBytes);
                        const uint4 e0 = e[0], e1 = e[1], e2 = e[2], e3 = e[3], e4 = e[4];
                        sh_item[t] = ((unsigned long long)e0.y << 32) | e0.x;
                        adopt(sh_item[t]);
                        blk = e0.z;
                        alive = e0.w;
                        wx = __uint_as_float(e1.x);
                        wy = __uint_as_float(e1.y);
                        wz = __uint_as_float(e1.z);
                        s = e1.w;
                        p = e2.x;
                        sh_steps[t] = (long long)(((unsigned long long)e2.w << 32) | e2.z);
                        sh_D[0][t] = __hiloint2double((int)e3.y, (int)e3.x);
                        sh_D[1][t] = __hiloint2double((int)e3.w, (int)e3.z);
                        sh_D[2][t] = __hiloint2double((int)e4.y, (int)e4.x);
                        S0 = S1 = S2 = 0.f;
                        busy = true;
                    } else {
                        atomicOr(P.status, 1 << MCG_ERR_TIMEOUT);
                    }
                }
            }
        }
        unsigned livem = __ballot_sync(kFull, busy);
        if (migrate && !stop && !spilled && livem != 0u && __popc(livem) <= P.spill_max &&
            __any_sync(kFull, exhausted)) {
            // few walks left here and nothing new to start: hand them over
            unsigned long long base = 0ull;
            int ok = 0;
            if (lane == 0) ok = pool_reserve(P, (unsigned)__popc(livem), base) ? 1 : 0;
            if (__shfl_sync(kFull, ok, 0)) {
                base = __shfl_sync(kFull, base, 0);
                if (busy) {
                    const unsigned long long slot = base + (unsigned)__popc(livem & lanes_below);
                    const unsigned long long it = sh_item[t];
                    const unsigned long long st = (unsigned long long)sh_steps[t];
                    const double D0 = sh_D[0][t] + (double)S0, D1 = sh_D[1][t] + (double)S1,
                                 D2 = sh_D[2][t] + (double)S2;
                    uint4* e = (uint4*)(P.pool + slot * kPoolEntryBytes);
                    e[0] = make_uint4((uint32_t)it, (uint32_t)(it >> 32), blk, alive);
                    e[1] = make_uint4(__float_as_uint(wx), __float_as_uint(wy), __float_as_uint(wz), s);
                    e[2] = make_uint4(p, 0u, (uint32_t)st, (uint32_t)(st >> 32));
                    e[3] = make_uint4((uint32_t)__double2loint(D0), (uint32_t)__double2hiint(D0),
                                      (uint32_t)__double2loint(D1), (uint32_t)__double2hiint(D1));
                    e[4] = make_uint4((uint32_t)__double2loint(D2), (uint32_t)__double2hiint(D2), 0u, 0u);
                    st_release_u32(P.pool_ready + slot, 1u);
                    busy = false;
                }
                spilled = true;
                livem = 0u;
            }
        }
        if (livem == 0u) {
            if (!migrate) break;
            int leave = 1;
            if (lane == 0) leave = pool_leave(P, stop) ? 1 : 0;
            if (__shfl_sync(kFull, leave, 0)) break;
            continue;  // the last warp: take over the pooled walks
        }

        // two four-step blocks per iteration for the analytic densities; one
        // for the voxel grid, whose larger step body (prefetched lookups)
        // otherwise strains the instruction cache
        constexpr int kBlocksUnrolled = (RHO == MCG_RHO_VOXEL || RHO == kRhoVoxelPacked) ? 1 : 2;
#pragma unroll (kBlocksUnrolled)
        for (int k = 0; k < 16; ++k) {
            if (busy) {
                // the block's twelve normals in polar form: coordinate j of
                // the moves is nr[j / 2] cs[j]; (a single-request launch reads
                // its key straight from the launch parameters: uniform across
                // the warp)
                float nr[6], cs[12];
                polar12_f32(s, p, blk, SEG ? k0 : P.key0, SEG ? k1 : P.key1, P.lnscale_f, nr, cs);
                // one fused multiply-add per coordinate and step
                auto mv = [&](float x, int j) -> float { return fmaf(nr[j >> 1], cs[j], x); };
                // Voxel grid: the block's four positions are known once its
                // normals are, so all twelve density loads are issued here
                // and their latency overlaps the steps (same positions, same
                // summation order: results are unchanged).
                constexpr bool kPrefetch = RHO == MCG_RHO_VOXEL || RHO == kRhoVoxelPacked;
                // Quiet block (box domain, prism or sphere density): no
                // coordinate moves by more than -(nr[0] + ... + nr[5]) over
                // the block, so if that bound keeps every copy inside the
                // conservative box and outside the density's support box for
                // the whole block, the four steps only move (the boxes' margin,
                // 1e-5 of the domain, is some twenty times the single-precision
                // rounding of the bound and of the four moves).  The decision is
                // taken for the warp (all live lanes quiet), so a warp never
                // runs both the quiet moves and the full steps.
                constexpr bool kBlockTest = !BALL && !kPrefetch &&
                                            (RHO == MCG_RHO_PRISM || RHO == MCG_RHO_SPHERE);
                // The same bound with the domain alone: a warp whose copies all
                // stay surely inside Omega for the block runs its steps without
                // exit tests.  (Not for the voxel grid: the second copy of the
                // step body costs its kernel six registers and a sixth of its
                // resident warps.)
                constexpr bool kBlockInside = !BALL && !kPrefetch;
                bool all_quiet = false, all_inside = false;
                if constexpr (kBlockTest || kBlockInside) {
                    const float rs = ((nr[0] + nr[1]) + (nr[2] + nr[3])) + (nr[4] + nr[5]);  // <= 0
                    const bool inside =
                        fabsf(wx) - rs < P.in_f[0] && fabsf(wy) - rs < P.in_f[1] && fabsf(wz) - rs < P.in_f[2];
                    const unsigned am = __activemask();
                    if constexpr (kBlockTest) {
                        const bool far = fabsf(wx - P.far_c[0]) + rs > P.far_h[0] ||
                                         fabsf(wy - P.far_c[1]) + rs > P.far_h[1] ||
                                         fabsf(wz - P.far_c[2]) + rs > P.far_h[2];
                        all_quiet = __all_sync(am, inside && far);
                    }
                    if constexpr (kBlockInside) all_inside = __all_sync(am, inside);
                }
                // common step: every copy surely inside Omega and surely
                // outside the density's support -> nothing to do but move
                // (ki: the block test already showed every copy inside)
                auto common = [&](auto ki, float nx, float ny, float nz, bool& inside_all, float& qxy) -> bool {
                    qxy = BALL ? nx * nx + ny * ny : 0.0f;
                    if constexpr (decltype(ki)::value)
                        inside_all = true;
                    else
                        inside_all = BALL ? qxy + nz * nz < P.in_r2_f
                                          : fabsf(nx) < P.in_f[0] && fabsf(ny) < P.in_f[1] && fabsf(nz) < P.in_f[2];
                    if constexpr (kBlockTest) return false;  // the block test decided: full step
                    bool no_rho = true;
                    if constexpr (RHO == MCG_RHO_PRISM) {
                        no_rho = !(fabsf(nx - P.far_c[0]) <= P.far_h[0] && fabsf(ny - P.far_c[1]) <= P.far_h[1] &&
                                   fabsf(nz - P.far_c[2]) <= P.far_h[2]);
                    } else if constexpr (RHO == MCG_RHO_SPHERE) {
                        const float dx = nx - P.sc_f[0], dy = ny - P.sc_f[1], dz = nz - P.sc_f[2];
                        no_rho = dx * dx + dy * dy + dz * dz > P.far_r2;
                    } else if constexpr (RHO == MCG_RHO_VOXEL || RHO == kRhoVoxelPacked) {
                        no_rho = false;
                    }
                    return inside_all && no_rho;
                };
                float px[4], py[4], pz[4], rv[4][3];
                if constexpr (kPrefetch) {
                    float x = wx, y = wy, zz = wz;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        x = mv(x, 3 * m);
                        y = mv(y, 3 * m + 1);
                        zz = mv(zz, 3 * m + 2);
                        px[m] = x;
                        py[m] = y;
                        pz[m] = zz;
                        rho3_f32<RHO>(P, SEG ? M : model_of(P), x, y, zz, hf, rv[m][0], rv[m][1], rv[m][2]);
                    }
                }
                if (all_quiet) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        wx = mv(wx, 3 * m);
                        wy = mv(wy, 3 * m + 1);
                        wz = mv(wz, 3 * m + 2);
                    }
                } else {
                    auto full_steps = [&](auto ki) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float nx = kPrefetch ? px[m] : mv(wx, 3 * m);
                        const float ny = kPrefetch ? py[m] : mv(wy, 3 * m + 1);
                        const float nz = kPrefetch ? pz[m] : mv(wz, 3 * m + 2);
                        bool inside_all;
                        float qxy;
                        if (!common(ki, nx, ny, nz, inside_all, qxy)) {  // otherwise rho = 0 at every copy: sums unchanged
                            if (!inside_all) {
                                unsigned ins;
                                if (BALL) {
                                    const float za = nz, zb = nz + hf, zc = nz - hf;
                                    ins = (qxy + za * za < P.R2_f) ? 1u : 0u;
                                    if (CRN) {
                                        ins |= (qxy + zb * zb < P.R2_f) ? 2u : 0u;
                                        ins |= (qxy + zc * zc < P.R2_f) ? 4u : 0u;
                                    }
                                } else {
                                    const bool inxy = fabsf(nx) < hx && fabsf(ny) < hy;
                                    ins = (inxy && fabsf(nz) < hz) ? 1u : 0u;
                                    if (CRN) {
                                        ins |= (inxy && fabsf(nz + hf) < hz) ? 2u : 0u;
                                        ins |= (inxy && fabsf(nz - hf) < hz) ? 4u : 0u;
                                    }
                                }
                                const unsigned out = alive & ~ins;
                                if (out) {  // some copy left Omega on this step
                                    const unsigned long long it = sh_item[t];
                                    if (out & 1u) put_exit(P, 0, it, wx, wy, wz, nx, ny, nz, S0, sh_D[0][t]);
                                    if (CRN && (out & 2u)) put_exit(P, 1, it, wx, wy, wz, nx, ny, nz + hf, S1, sh_D[1][t]);
                                    if (CRN && (out & 4u)) put_exit(P, 2, it, wx, wy, wz, nx, ny, nz - hf, S2, sh_D[2][t]);
                                    sh_steps[t] += nstep_of(blk, m) * (long long)__popc(out);
                                    alive &= ins;
                                }
                                if (BRIDGE && alive) {  // within the bridge band of a face
                                    unsigned faces = 0u;
                                    const unsigned bx = bridge_exits_f32(P, alive, wx, wy, wz, nx, ny, nz, hf, s, p, blk, m,
                                                                         &faces);
                                    if (bx) {
                                        const unsigned long long it = sh_item[t];
                                        const float yb[3] = {nx, ny, nz};
                                        for (int c = 0; c < 3; ++c) {
                                            if (!(bx & (1u << c))) continue;
                                            const float off = c == 0 ? 0.0f : (c == 1 ? hf : -hf);
                                            float y3[3] = {yb[0], yb[1], yb[2] + off};
                                            const int f = (int)((faces >> (3 * c)) & 7u);
                                            y3[f >> 1] = (f & 1) ? P.half_f[f >> 1] : -P.half_f[f >> 1];
                                            const float part = c == 0 ? S0 : (c == 1 ? S1 : S2);
                                            put_exit(P, c, it, wx, wy, wz, y3[0], y3[1], y3[2], part, sh_D[c][t]);
                                        }
                                        sh_steps[t] += nstep_of(blk, m) * (long long)__popc(bx);
                                        alive &= ~bx;
                                    }
                                }
                            }
                            if constexpr (RHO == MCG_RHO_PRISM) {
                                // the prism's density is rho0 or 0: add rho0 where a
                                // copy is inside (the tests of rho3_f32<PRISM>)
                                const bool inxy = nx >= P.plo_f[0] && nx < P.phi_f[0] && ny >= P.plo_f[1] &&
                                                  ny < P.phi_f[1];
                                const float zb = __fadd_rn(nz, hf), zc = __fsub_rn(nz, hf);
                                if (inxy && nz >= P.plo_f[2] && nz < P.phi_f[2]) S0 += P.rho0_f;
                                if (CRN) {
                                    if (inxy && zb >= P.plo_f[2] && zb < P.phi_f[2]) S1 += P.rho0_f;
                                    if (inxy && zc >= P.plo_f[2] && zc < P.phi_f[2]) S2 += P.rho0_f;
                                }
                            } else {
                                float ra, rb, rc;
                                if constexpr (kPrefetch) {
                                    ra = rv[m][0];
                                    rb = rv[m][1];
                                    rc = rv[m][2];
                                } else {
                                    rho3_f32<RHO>(P, SEG ? M : model_of(P), nx, ny, nz, hf, ra, rb, rc);
                                }
                                S0 += ra;
                                if (CRN) {
                                    S1 += rb;
                                    S2 += rc;
                                }
                            }
                        }
                        wx = nx;
                        wy = ny;
                        wz = nz;
                        // no early exit when the last copy leaves: the remaining
                        // steps of the block write nothing (no live copy), and a
                        // branch-free four-step body schedules better
                    }
                    };
                    if (kBlockInside && all_inside)
                        full_steps(std::true_type{});
                    else
                        full_steps(std::false_type{});
                }
                ++blk;
                if (!alive) {  // every copy has its exit record: mark the item complete
                    P.pp_steps[sh_item[t]] = sh_steps[t] | kDoneFlag;
                    busy = false;
                } else if (4 * (int64_t)blk >= P.max_steps) {
                    const unsigned long long it = sh_item[t];
                    atomicOr(SEG ? P.seg[sh_seg[t]].status : P.status, 1 << MCG_ERR_STEP_CAP);
                    // (no completion flag: the exit kernel writes NaN)
                    P.pp_steps[it] = sh_steps[t] + (long long)__popc(alive) * 4 * (long long)blk;
                    busy = false;
                }
            }
            // enough lanes want new work: leave the block loop to refill them
            if (__popc(__ballot_sync(kFull, !busy && !exhausted)) >= P.refill_min) break;
        }
        // warp-uniform flush of the partial sums (at most 16 blocks = 64 steps each)
        sh_D[0][t] += (double)S0;
        S0 = 0.f;
        if (CRN) {
            sh_D[1][t] += (double)S1;
            sh_D[2][t] += (double)S2;
            S1 = S2 = 0.f;
        }
    }
}

// Per-path values of one item from its exit records (double precision).  The
// density at the last inside point is re-evaluated from X by the walk's own
// single-precision function.
template <int RHO, bool SEG>
__device__ __forceinline__ void exit_item(const WalkParams& P, unsigned long long item, float hf)
{
    ModelRef M = model_of(P);
    int32_t* status = P.status;
    if constexpr (SEG) {  // the item's request: its model arrays and status word
        const WalkSeg& g = P.seg[find_seg(P, item)];
        M = model_of(g);
        status = g.status;
    }
    double u[3] = {kNaN, kNaN, kNaN};
    const int nc = P.crn ? 3 : 1;
    const size_t T = P.total;
    for (int c = 0; c < nc; ++c) {
        const float4* rec = (const float4*)P.frec + 2 * ((size_t)c * T + item);
        const float4 a = rec[0], b = rec[1];
        float r[3];
        rho3_f32<RHO>(P, M, a.x, a.y, a.z, hf, r[0], r[1], r[2]);
        const float X[3] = {a.x, a.y, c == 0 ? a.z : (c == 1 ? a.z + hf : a.z - hf)};
        const float Y[3] = {a.w, b.x, b.y};
        const double acc = __hiloint2double(__float_as_int(b.w), __float_as_int(b.z));
        u[c] = exit_mixed(P, M, X, Y, acc, r[c]);
    }
    const double d = P.crn ? (u[1] - u[2]) / (2.0 * P.h) : kNaN;
    P.pp_u[item] = u[0];
    P.pp_d[item] = d;
    if (!isfinite(u[0]) || (P.crn && !isfinite(d))) atomicOr(status, 1 << MCG_ERR_NONFINITE);
}

// Exit evaluation, convergent: each warp scans its items 32 at a time, writes
// NaN for the ones without a result (no completion flag: capped, cancelled,
// never started, lost, outside Omega), clears the flag of the others and
// queues them in
// shared memory, evaluating them 32 at a time, so the slow double-precision
// pipe never runs a warp whose lanes are mostly idle.
template <int RHO, bool SEG>
__global__ void __launch_bounds__(128) exit_mixed_kernel(const WalkParams P)
{
    __shared__ unsigned long long queue[4][64];
    const float hf = P.crn ? P.h_f : 0.0f;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long* q = queue[w];
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long first = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + w) * 32ull;
    int qn = 0;  // queued items (warp-uniform)
    for (unsigned long long base = first; base < P.total; base += warps * 32ull) {
        const unsigned long long item = base + (unsigned long long)lane;
        const bool in = item < P.total;
        const long long steps = in ? (long long)P.pp_steps[item] : 0ll;
        const bool valid = (steps & kDoneFlag) != 0;
        if (valid) P.pp_steps[item] = steps & ~kDoneFlag;
        if (in && !valid) {
            P.pp_u[item] = kNaN;
            P.pp_d[item] = kNaN;
        }
        const unsigned vm = __ballot_sync(kFull, valid);
        if (valid) q[qn + __popc(vm & ((1u << lane) - 1u))] = item;
        qn += __popc(vm);
        __syncwarp();
        if (qn >= 32) {
            exit_item<RHO, SEG>(P, q[lane], hf);
            const int rest = qn - 32;
            unsigned long long v = 0ull;
            if (lane < rest) v = q[32 + lane];
            __syncwarp();
            if (lane < rest) q[lane] = v;
            __syncwarp();
            qn = rest;
        }
    }
    if (lane < qn) exit_item<RHO, SEG>(P, q[lane], hf);
}

template <int RHO, bool CRN, bool BRIDGE, bool BALL, bool SEG>
cudaError_t launch_mixed(const WalkParams& P, int block, int grid, cudaStream_t st)
{
    walk_mixed_kernel<RHO, CRN, BRIDGE, BALL, SEG><<<grid, block, 0, st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long need = (P.total + 127ull) / 128ull;
    const unsigned long long cap = (unsigned long long)sms * 16ull;
    exit_mixed_kernel<RHO, SEG><<<(unsigned)(need < cap ? need : cap), 128, 0, st>>>(P);
    return cudaGetLastError();
}

template <int RHO>
cudaError_t launch_mixed_rho(const WalkParams& P, int block, int grid, cudaStream_t st)
{
    if (P.seg) return P.crn ? launch_mixed<RHO, true, false, false, true>(P, block, grid, st)
                            : launch_mixed<RHO, false, false, false, true>(P, block, grid, st);
    if (P.ball) return P.crn ? launch_mixed<RHO, true, false, true, false>(P, block, grid, st)
                             : launch_mixed<RHO, false, false, true, false>(P, block, grid, st);
    if (P.crn) return P.bridge ? launch_mixed<RHO, true, true, false, false>(P, block, grid, st)
                               : launch_mixed<RHO, true, false, false, false>(P, block, grid, st);
    return P.bridge ? launch_mixed<RHO, false, true, false, false>(P, block, grid, st)
                    : launch_mixed<RHO, false, false, false, false>(P, block, grid, st);
}

template <int RHO>
const void* mixed_fn(bool crn, bool seg)
{
    if (seg)
        return crn ? (const void*)walk_mixed_kernel<RHO, true, false, false, true>
                   : (const void*)walk_mixed_kernel<RHO, false, false, false, true>;
    return crn ? (const void*)walk_mixed_kernel<RHO, true, false, false, false>
               : (const void*)walk_mixed_kernel<RHO, false, false, false, false>;
}

const void* kernel_fn(int precision, int rho_kind, bool crn, bool seg)
{
    if (precision == MCG_FP64) {
        if (seg) return crn ? (const void*)walk_fp64_kernel<true, true> : (const void*)walk_fp64_kernel<false, true>;
        return crn ? (const void*)walk_fp64_kernel<true, false> : (const void*)walk_fp64_kernel<false, false>;
    }
    switch (rho_kind) {
    case kRhoVoxelPacked: return mixed_fn<kRhoVoxelPacked>(crn, seg);
    case MCG_RHO_SPHERE: return mixed_fn<MCG_RHO_SPHERE>(crn, seg);
    case MCG_RHO_PRISM: return mixed_fn<MCG_RHO_PRISM>(crn, seg);
    case MCG_RHO_VOXEL: return mixed_fn<MCG_RHO_VOXEL>(crn, seg);
    default: return mixed_fn<MCG_RHO_NONE>(crn, seg);
    }
}

}  // namespace

namespace {

template <typename K>
void touch(K kernel)
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, (const void*)kernel) != cudaSuccess) cudaGetLastError();
}

template <int RHO>
void touch_mixed()
{
    touch(walk_mixed_kernel<RHO, true, false, true, false>);
    touch(walk_mixed_kernel<RHO, false, false, true, false>);
    touch(walk_mixed_kernel<RHO, true, true, false, false>);
    touch(walk_mixed_kernel<RHO, true, false, false, false>);
    touch(walk_mixed_kernel<RHO, false, true, false, false>);
    touch(walk_mixed_kernel<RHO, false, false, false, false>);
    touch(walk_mixed_kernel<RHO, true, false, false, true>);
    touch(walk_mixed_kernel<RHO, false, false, false, true>);
    touch(exit_mixed_kernel<RHO, false>);
    touch(exit_mixed_kernel<RHO, true>);
}

}  // namespace

void preload_walk_kernels()
{
    touch(walk_fp64_kernel<true, false>);
    touch(walk_fp64_kernel<false, false>);
    touch(walk_fp64_kernel<true, true>);
    touch(walk_fp64_kernel<false, true>);
    touch_mixed<MCG_RHO_NONE>();
    touch_mixed<MCG_RHO_SPHERE>();
    touch_mixed<MCG_RHO_PRISM>();
    touch_mixed<MCG_RHO_VOXEL>();
    touch_mixed<kRhoVoxelPacked>();
}

int walk_blocks_per_sm(int precision, int rho_kind, int block, bool seg)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_fn(precision, rho_kind, true, seg), block, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_walk(const WalkParams& P, int precision, int block, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // a multi-request launch runs in the box without the bridge test
    if (P.seg && (P.ball || P.bridge || P.nseg <= 0)) return cudaErrorInvalidValue;
    const int kind = (P.rho_kind == MCG_RHO_VOXEL && P.zq) ? kRhoVoxelPacked : P.rho_kind;
    const int per_sm = walk_blocks_per_sm(precision, kind, block, P.seg != nullptr);
    long long grid = (long long)sms * per_sm;
    const long long need = (long long)((P.total + (unsigned long long)block - 1ull) / (unsigned long long)block);
    if (grid > need) grid = need > 0 ? need : 1;
    const bool crn = P.crn != 0;
    if (precision == MCG_FP64) {
        if (P.seg) {
            if (crn) walk_fp64_kernel<true, true><<<(int)grid, block, 0, st>>>(P);
            else walk_fp64_kernel<false, true><<<(int)grid, block, 0, st>>>(P);
        } else {
            if (crn) walk_fp64_kernel<true, false><<<(int)grid, block, 0, st>>>(P);
            else walk_fp64_kernel<false, false><<<(int)grid, block, 0, st>>>(P);
        }
        return cudaGetLastError();
    }
    switch (kind) {
    case kRhoVoxelPacked: return launch_mixed_rho<kRhoVoxelPacked>(P, block, (int)grid, st);
    case MCG_RHO_SPHERE: return launch_mixed_rho<MCG_RHO_SPHERE>(P, block, (int)grid, st);
    case MCG_RHO_PRISM: return launch_mixed_rho<MCG_RHO_PRISM>(P, block, (int)grid, st);
    case MCG_RHO_VOXEL: return launch_mixed_rho<MCG_RHO_VOXEL>(P, block, (int)grid, st);
    default: return launch_mixed_rho<MCG_RHO_NONE>(P, block, (int)grid, st);
    }
}

}  // namespace mcg
