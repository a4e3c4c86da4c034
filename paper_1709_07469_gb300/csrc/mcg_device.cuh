// mcg_device.cuh -- device functions of the walk: Philox4x32-10, Box-Muller
// in double and single precision, density samplers, boundary data.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mcg_internal.h"

namespace mcg {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies of counter words 0 and 2; the high halves are xor-ed
// with words 1 / 3 and the round key, which advances by the Weyl constants.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32->64 multiply gives both halves of each product
        const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Double precision normals (the plain FP64 walk): u = (w + 1/2) 2^-32,
// r = sqrt(-2 ln u1), angle 2 pi u2, cosine first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double u01_f64(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }

__device__ __forceinline__ void box_muller_f64(uint32_t w1, uint32_t w2, double& z0, double& z1)
{
    const double r = sqrt(-2.0 * log(u01_f64(w1)));
    const double a = 2.0 * 3.14159265358979323846 * u01_f64(w2);
    double sn, cs;
    sincos(a, &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
}

__device__ __forceinline__ void normals12_f64(uint32_t s, uint32_t p, uint32_t b, uint32_t k0, uint32_t k1,
                                              double z[12])
{
#pragma unroll
    for (uint32_t i = 0; i < 3; ++i) {
        const uint4 w = philox4x32_10(make_uint4(3u * b + i, p, s, 0u), k0, k1);
        box_muller_f64(w.x, w.y, z[4 * i], z[4 * i + 1]);
        box_muller_f64(w.z, w.w, z[4 * i + 2], z[4 * i + 3]);
    }
}

// ---------------------------------------------------------------------------
// Single precision normals (the mixed walk).  u = ((w >> 9) + 1/2) 2^-23 is
// built exactly from the mantissa bits: 1 + (w >> 9) 2^-23 minus the float
// just below 1.  The radius uses the hardware base-2 logarithm and square
// root; the angle 2 pi u2 is taken as pi + 2 pi (u2 - 1/2) so the sine and
// cosine approximations see (-pi, pi): cos(2 pi u2) = -cos(a), sin(2 pi u2)
// = -sin(a).  `lnscale` = -2 ln 2 sd^2 folds the step scale into r.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1 + (w >> 9) 2^-23 in [1, 2): exponent bits 0x7F funnel-shifted in above
// the top 23 bits of w.
__device__ __forceinline__ float one_plus_mantissa(uint32_t w)
{
    return __uint_as_float(__funnelshift_r(w, 0x7Fu, 9));
}
__device__ __forceinline__ float u01_f32(uint32_t w) { return one_plus_mantissa(w) - 0.99999994f; }
// u - 1/2, exact: (1 + m 2^-23) - 1.5 is exact, + 2^-24 lands on the grid.
__device__ __forceinline__ float u01m_f32(uint32_t w) { return (one_plus_mantissa(w) - 1.5f) + 0x1p-24f; }

// The angle 2 pi (u2 - 1/2) = 2 pi v - 2 pi (1.5 - 2^-24), v = 1 + m 2^-23,
// as one fused multiply-add (within one rounding of the exact angle).
constexpr float kTwoPi = 6.28318530717958648f;
constexpr float kAngleOffset = (float)(-6.283185307179586476925 * (1.5 - 0x1p-24));

__device__ __forceinline__ void box_muller_f32(uint32_t w1, uint32_t w2, float lnscale, float& z0, float& z1)
{
    const float nr = -sqrt_approx(lnscale * lg2_approx(u01_f32(w1)));  // -sd sqrt(-2 ln u1)
    const float a = fmaf(one_plus_mantissa(w2), kTwoPi, kAngleOffset);
    z0 = nr * cos_approx(a);
    z1 = nr * sin_approx(a);
}

__device__ __forceinline__ void normals12_f32(uint32_t s, uint32_t p, uint32_t b, uint32_t k0, uint32_t k1,
                                              float lnscale, float z[12])
{
#pragma unroll
    for (uint32_t i = 0; i < 3; ++i) {
        const uint4 w = philox4x32_10(make_uint4(3u * b + i, p, s, 0u), k0, k1);
        box_muller_f32(w.x, w.y, lnscale, z[4 * i], z[4 * i + 1]);
        box_muller_f32(w.z, w.w, lnscale, z[4 * i + 2], z[4 * i + 3]);
    }
}

// The same twelve normals in polar form, as the walk consumes them: normal j
// is nr[j / 2] * cs[j] with cs[j] the cosine (j even) or sine (j odd) of the
// pair's angle and nr <= 0 the scaled radius with its sign.  Every normal's
// magnitude is at most -nr[j / 2], which bounds a block's excursion.
__device__ __forceinline__ void polar_pair_f32(uint32_t w1, uint32_t w2, float lnscale, float& nr, float& c,
                                               float& sn)
{
    nr = -sqrt_approx(lnscale * lg2_approx(u01_f32(w1)));
    const float a = fmaf(one_plus_mantissa(w2), kTwoPi, kAngleOffset);
    c = cos_approx(a);
    sn = sin_approx(a);
}

__device__ __forceinline__ void polar12_f32(uint32_t s, uint32_t p, uint32_t b, uint32_t k0, uint32_t k1,
                                            float lnscale, float nr[6], float cs[12])
{
#pragma unroll
    for (uint32_t i = 0; i < 3; ++i) {
        const uint4 w = philox4x32_10(make_uint4(3u * b + i, p, s, 0u), k0, k1);
        polar_pair_f32(w.x, w.y, lnscale, nr[2 * i], cs[4 * i], cs[4 * i + 1]);
        polar_pair_f32(w.z, w.w, lnscale, nr[2 * i + 1], cs[4 * i + 2], cs[4 * i + 3]);
    }
}

// ---------------------------------------------------------------------------
// The model arrays a walk reads: the launch's own, or (multi-request launch)
// those of the walk's request.
// ---------------------------------------------------------------------------
struct ModelRef {
    const float* grid;
    const float4* zq;
    const float* faces;
    const float4* tq;
};

__device__ __forceinline__ ModelRef model_of(const WalkParams& P) { return ModelRef{P.grid, P.zq, P.faces, P.tq}; }

__device__ __forceinline__ ModelRef model_of(const WalkSeg& g)
{
    return ModelRef{g.grid, g.zq, g.faces, g.tq};
}

// Segment of launch item `item` (binary search over the sorted begins).
__device__ __forceinline__ int find_seg(const WalkParams& P, unsigned long long item)
{
    int lo = 0, hi = P.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&P.seg[mid].begin) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Density samplers.
// ---------------------------------------------------------------------------
// floor(t) as an integer without a conversion instruction: adding
// 1.5 * 2^23 rounded toward -infinity leaves floor(t) + 1.5 * 2^23 exactly
// for |t| < 2^22 (the float spacing there is 1), so its bit pattern minus
// that of 1.5 * 2^23 is floor(t).  Beyond |t| >= 2^22 the result is far
// outside any grid (below -2^22 or at least 2^22), which the callers' range
// tests reject.
constexpr float kFloorMagic = 12582912.0f;   // 1.5 * 2^23
constexpr uint32_t kFloorMagicBits = 0x4B400000u;

__device__ __forceinline__ int floor_int(float t)
{
    return (int)(__float_as_uint(__fadd_rd(t, kFloorMagic)) - kFloorMagicBits);
}

// Cell of a point of the voxel grid: t_k = (x_k - origin_k) / spacing_k in
// single precision (difference, then product with the reciprocal spacing),
// cell index floor(t_k); for z also the position within the layer,
// fr = t_z - floor(t_z) (exact: Sterbenz, or t_z itself below 1), which
// places the copies at z +- h.
__device__ __forceinline__ void voxel_cell(const WalkParams& P, float x, float y, float z, int& ix, int& iy, int& iz,
                                           float& fr)
{
    ix = floor_int(__fmul_rn(__fsub_rn(x, P.org_f[0]), P.inv_sp_f[0]));
    iy = floor_int(__fmul_rn(__fsub_rn(y, P.org_f[1]), P.inv_sp_f[1]));
    const float tz = __fmul_rn(__fsub_rn(z, P.org_f[2]), P.inv_sp_f[2]);
    const float vz = __fadd_rd(tz, kFloorMagic);
    iz = (int)(__float_as_uint(vz) - kFloorMagicBits);
    fr = __fsub_rn(tz, __fsub_rn(vz, kFloorMagic));
}

// Density at the three common-random-number copies (x, y, z), (x, y, z+h),
// (x, y, z-h): the x / y part is computed once.  Every rounding step is
// explicit (no contraction left to the compiler), so the walk kernel and the
// exit kernel, which re-evaluates rho at the last inside point, agree bit for
// bit.
template <int RHO>
__device__ __forceinline__ void rho3_f32(const WalkParams& P, const ModelRef& M, float x, float y, float z, float h,
                                         float& ra, float& rb, float& rc)
{
    if constexpr (RHO == MCG_RHO_SPHERE) {
        const float dx = __fsub_rn(x, P.sc_f[0]), dy = __fsub_rn(y, P.sc_f[1]), dz = __fsub_rn(z, P.sc_f[2]);
        const float q = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        const float za = dz, zb = __fadd_rn(dz, h), zc = __fsub_rn(dz, h);
        ra = (__fmaf_rn(za, za, q) < P.srad2_f) ? P.rho0_f : 0.0f;
        rb = (__fmaf_rn(zb, zb, q) < P.srad2_f) ? P.rho0_f : 0.0f;
        rc = (__fmaf_rn(zc, zc, q) < P.srad2_f) ? P.rho0_f : 0.0f;
    } else if constexpr (RHO == MCG_RHO_PRISM) {
        const bool inxy = x >= P.plo_f[0] && x < P.phi_f[0] && y >= P.plo_f[1] && y < P.phi_f[1];
        const float zb = __fadd_rn(z, h), zc = __fsub_rn(z, h);
        ra = (inxy && z >= P.plo_f[2] && z < P.phi_f[2]) ? P.rho0_f : 0.0f;
        rb = (inxy && zb >= P.plo_f[2] && zb < P.phi_f[2]) ? P.rho0_f : 0.0f;
        rc = (inxy && zc >= P.plo_f[2] && zc < P.phi_f[2]) ? P.rho0_f : 0.0f;
    } else if constexpr (RHO == MCG_RHO_VOXEL) {
        int ix, iy, iz;
        float fr;
        voxel_cell(P, x, y, z, ix, iy, iz, fr);
        // unsigned index arithmetic: out-of-range cells wrap to large values
        // that the range tests reject (no signed overflow)
        const unsigned nx = (unsigned)P.nx, ny = (unsigned)P.ny, nz = (unsigned)P.nz;
        const bool inxy = (unsigned)ix < nx && (unsigned)iy < ny;
        const unsigned base = (unsigned)ix + nx * (unsigned)iy, plane = nx * ny;
        // the copies' layers: iz + floor(fr + h / dz), iz + floor(fr - h / dz)
        const unsigned ka = (unsigned)iz;
        const unsigned kb = ka + (unsigned)floor_int(__fadd_rn(fr, P.hz_f));
        const unsigned kc = ka + (unsigned)floor_int(__fsub_rn(fr, P.hz_f));
        ra = (inxy && ka < nz) ? __ldg(M.grid + (base + plane * ka)) : 0.0f;
        rb = (inxy && kb < nz) ? __ldg(M.grid + (base + plane * kb)) : 0.0f;
        rc = (inxy && kc < nz) ? __ldg(M.grid + (base + plane * kc)) : 0.0f;
    } else if constexpr (RHO == kRhoVoxelPacked) {
        // The same cells as above, read through the packed grid: with
        // h <= half a cell the copies' layers differ from iz by at most one
        // (floor(fr + h/dz) is 1 exactly when the rounded sum reaches 1, and
        // floor(fr - h/dz) is -1 exactly when fr < h/dz), and the 16-byte
        // entry of layer iz holds layers iz-1, iz, iz+1 (0 outside the grid),
        // so one load serves all three copies.
        int ix, iy, iz;
        float fr;
        voxel_cell(P, x, y, z, ix, iy, iz, fr);
        const unsigned nx = (unsigned)P.nx, ny = (unsigned)P.ny, kz = (unsigned)iz + 1u;
        const bool in = (unsigned)ix < nx && (unsigned)iy < ny && kz < (unsigned)P.nz + 2u;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) q = __ldg(M.zq + ((kz * ny + (unsigned)iy) * nx + (unsigned)ix));
        ra = q.y;
        rb = __fadd_rn(fr, P.hz_f) >= 1.0f ? q.z : q.y;
        rc = fr < P.hz_f ? q.x : q.y;
    } else {
        ra = rb = rc = 0.0f;
    }
}

// Double precision density at an absolute point (same cells as above).
__device__ __forceinline__ double rho_f64(const WalkParams& P, const ModelRef& M, const double x[3])
{
    switch (P.rho_kind) {
    case MCG_RHO_SPHERE: {
        const double dx = __dadd_rn(x[0], -P.sc[0]), dy = __dadd_rn(x[1], -P.sc[1]),
                     dz = __dadd_rn(x[2], -P.sc[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        return r2 < P.srad2 ? P.rho0 : 0.0;
    }
    case MCG_RHO_PRISM:
        for (int k = 0; k < 3; ++k)
            if (!(x[k] >= P.plo[k] && x[k] < P.phi[k])) return 0.0;
        return P.rho0;
    case MCG_RHO_VOXEL: {
        int idx[3];
        const int n[3] = {P.nx, P.ny, P.nz};
        for (int k = 0; k < 3; ++k) {
            const double t = floor(__ddiv_rn(__dadd_rn(x[k], -P.org[k]), P.sp[k]));
            if (!(t >= 0.0 && t < (double)n[k])) return 0.0;
            idx[k] = (int)t;
        }
        return (double)__ldg(M.grid + idx[0] + P.nx * (idx[1] + P.ny * idx[2]));
    }
    default:
        return 0.0;
    }
}

// ---------------------------------------------------------------------------
// Boundary data (double precision, evaluated once per copy at its exit).
// ---------------------------------------------------------------------------
// log(t + r), r = |(t, p, q)|, stable for t < 0 via (p^2 + q^2) / (r - t).
__device__ __forceinline__ double log_tr(double t, double p, double q, double r)
{
    return t >= 0.0 ? log(t + r) : log(p * p + q * q) - log(r - t);
}

// Nagy's corner function of the prism potential; terms with a vanishing
// polynomial prefactor are their limit 0.
static __device__ __noinline__ double prism_corner(double x, double y, double z)
{
    const double r = sqrt(x * x + y * y + z * z);
    if (r == 0.0) return 0.0;
    double f = 0.0;
    if (x * y != 0.0) f += x * y * log_tr(z, x, y, r);
    if (y * z != 0.0) f += y * z * log_tr(x, y, z, r);
    if (z * x != 0.0) f += z * x * log_tr(y, z, x, r);
    if (x != 0.0) f -= 0.5 * x * x * atan(y * z / (x * r));
    if (y != 0.0) f -= 0.5 * y * y * atan(z * x / (y * r));
    if (z != 0.0) f -= 0.5 * z * z * atan(x * y / (z * r));
    return f;
}

// Phi of a homogeneous prism [lo, hi) at x: -G rho times the alternating
// corner sum (+ at the all-upper corner).
__device__ __forceinline__ double prism_potential(double G, double rho, const double lo[3], const double hi[3],
                                                  const double x[3])
{
    double s = 0.0;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        const int i = c & 1, j = (c >> 1) & 1, k = (c >> 2) & 1;
        const double f = prism_corner((i ? hi[0] : lo[0]) - x[0], (j ? hi[1] : lo[1]) - x[1],
                                      (k ? hi[2] : lo[2]) - x[2]);
        s += ((3 - i - j - k) & 1) ? -f : f;
    }
    return -G * rho * s;
}

// The same prism sum with the corners taken in pairs along one axis: the
// two logarithms of a pair become one of a ratio, ln((t1 + r1)/(t0 + r0))
// with each t + r formed without cancellation, and the two arctangents one
// angle, atan(t1) - atan(t0) = arg((1 + i t1)(1 - i t0)).  Half the
// transcendental functions of the direct sum, and closer to the exact value
// (a 40-digit reference: 4e-13 relative at points of the domain boundary
// against 5e-12 for the direct sum).  The exit evaluation of the mixed walk
// uses it; the plain FP64 walk keeps the direct sum, operation by operation
// as the problem states it.
__device__ __forceinline__ double log_pair(double t0, double r0, double t1, double r1, double p2)
{
    const double v0 = t0 >= 0.0 ? t0 + r0 : p2 / (r0 - t0);
    const double v1 = t1 >= 0.0 ? t1 + r1 : p2 / (r1 - t1);
    return log(v1 / v0);
}

__device__ __forceinline__ double atan_pair(double t0, double t1) { return atan2(t1 - t0, 1.0 + t1 * t0); }

// [[[F]]] for corner offsets a[i], b[j], c[k] (index 1: upper limit); every
// term whose polynomial prefactor vanishes is its limit 0, as in prism_corner.
static __device__ __noinline__ double prism_sum_paired(const double a[2], const double b[2], const double c[2])
{
    double r[2][2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 2; ++k) r[i][j][k] = sqrt(a[i] * a[i] + b[j] * b[j] + c[k] * c[k]);
    double T = 0.0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double sg = (i == j) ? 1.0 : -1.0;  // sign of the pair's upper corner
            const double ab = a[i] * b[j], bc = b[i] * c[j], ca = c[i] * a[j];
            // x y ln(z + r) paired over z; y z ln(x + r) over x; z x ln(y + r) over y
            if (ab != 0.0) T += sg * ab * log_pair(c[0], r[i][j][0], c[1], r[i][j][1], a[i] * a[i] + b[j] * b[j]);
            if (bc != 0.0) T += sg * bc * log_pair(a[0], r[0][i][j], a[1], r[1][i][j], b[i] * b[i] + c[j] * c[j]);
            if (ca != 0.0) T += sg * ca * log_pair(b[0], r[j][0][i], b[1], r[j][1][i], c[i] * c[i] + a[j] * a[j]);
            // x^2/2 atan(yz/(xr)) and y^2/2 atan(zx/(yr)) paired over z;
            // z^2/2 atan(xy/(zr)) paired over x
            if (a[i] != 0.0) {
                const double t0 = b[j] * c[0] / (a[i] * r[i][j][0]), t1 = b[j] * c[1] / (a[i] * r[i][j][1]);
                T -= 0.5 * sg * a[i] * a[i] * atan_pair(t0, t1);
            }
            if (b[j] != 0.0) {
                const double t0 = c[0] * a[i] / (b[j] * r[i][j][0]), t1 = c[1] * a[i] / (b[j] * r[i][j][1]);
                T -= 0.5 * sg * b[j] * b[j] * atan_pair(t0, t1);
            }
            if (c[j] != 0.0) {
                const double t0 = a[0] * b[i] / (c[j] * r[0][i][j]), t1 = a[1] * b[i] / (c[j] * r[1][i][j]);
                T -= 0.5 * sg * c[j] * c[j] * atan_pair(t0, t1);
            }
        }
    return T;
}

__device__ __forceinline__ double prism_potential_paired(double G, double rho, const double lo[3],
                                                         const double hi[3], const double x[3])
{
    const double a[2] = {lo[0] - x[0], hi[0] - x[0]}, b[2] = {lo[1] - x[1], hi[1] - x[1]},
                 c[2] = {lo[2] - x[2], hi[2] - x[2]};
    return -G * rho * prism_sum_paired(a, b, c);
}

__device__ __forceinline__ double sphere_potential(const WalkParams& P, const double x[3])
{
    const double dx = x[0] - P.sc[0], dy = x[1] - P.sc[1], dz = x[2] - P.sc[2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double a = P.srad, a2 = a * a;
    const double M = 4.0 / 3.0 * 3.14159265358979323846 * a * a * a * P.rho0;
    if (r >= a) return -P.G * M / r;
    return -P.G * M * (3.0 * a2 - r * r) / (2.0 * a2 * a);
}

// Bilinear read of face `face` (0..5) at the absolute boundary point x.
__device__ __forceinline__ double table_value(const WalkParams& P, const ModelRef& M, int face, const double x[3])
{
    const int k = face >> 1;
    const int a = (k == 0) ? 1 : 0, b = (k == 2) ? 1 : 2;
    const float* t = M.faces + (int64_t)face * P.nu * P.nv;
    const double tu = (x[a] - P.lo[a]) / (P.hi[a] - P.lo[a]) * (double)(P.nu - 1);
    const double tv = (x[b] - P.lo[b]) / (P.hi[b] - P.lo[b]) * (double)(P.nv - 1);
    const double fu = fmin(fmax(floor(tu), 0.0), (double)(P.nu - 2));
    const double fv = fmin(fmax(floor(tv), 0.0), (double)(P.nv - 2));
    const int iu = (int)fu, iv = (int)fv;
    const double au = tu - fu, av = tv - fv;
    double f00, f10, f01, f11;
    if (M.tq) {  // the cell's four corners in one 16-byte load
        const float4 c = __ldg(M.tq + ((int64_t)face * (P.nv - 1) + iv) * (P.nu - 1) + iu);
        f00 = c.x;
        f10 = c.y;
        f01 = c.z;
        f11 = c.w;
    } else {
        const float* r0 = t + (int64_t)P.nu * iv + iu;
        f00 = __ldg(r0);
        f10 = __ldg(r0 + 1);
        f01 = __ldg(r0 + P.nu);
        f11 = __ldg(r0 + P.nu + 1);
    }
    return (1.0 - au) * (1.0 - av) * f00 + au * (1.0 - av) * f10 + (1.0 - au) * av * f01 + au * av * f11;
}

// g at the absolute exit point x on face `face` (-1 if not on a face).
// PAIRED: the prism closed form by the paired corner sum (the mixed walk's
// exit evaluation) instead of the direct one (the plain FP64 walk).
template <bool PAIRED = false>
static __device__ __noinline__ double boundary_value(const WalkParams& P, const ModelRef& M, int face, const double* x)
{
    switch (P.g_kind) {
    case MCG_G_SPHERE:
        return sphere_potential(P, x);
    case MCG_G_PRISM:
        return PAIRED ? prism_potential_paired(P.G, P.rho0, P.plo, P.phi, x)
                      : prism_potential(P.G, P.rho0, P.plo, P.phi, x);
    case MCG_G_TABLE:
        return face < 0 ? __longlong_as_double(0x7ff8000000000000LL) : table_value(P, M, face, x);
    case MCG_G_POLY: {
        const double* c = P.poly;
        const double X = x[0], Y = x[1], Z = x[2];
        return c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * X + c[5] * Y * Y + c[6] * Z * Z +
               c[7] * X * Y + c[8] * Y * Z + c[9] * Z * X + c[10] * X * Y * Z;
    }
    default:
        return 0.0;
    }
}

}  // namespace mcg
