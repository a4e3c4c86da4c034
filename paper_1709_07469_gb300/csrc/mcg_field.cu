// mcg_field.cu -- the exact potential Phi and vertical gravity dPhi/dz of the
// density models at arbitrary points: the closed forms the walk's estimates
// are checked against (the paper compares its stochastic solution with the
// analytic prism field, Sec. 4.2, and with a finite-element solution).
//
//  * sphere: -G M / r outside, -G M (3 a^2 - r^2) / (2 a^3) inside;
//  * prism : Nagy's corner function F summed over the eight corners,
//            Phi = -G rho [[[F]]], dPhi/dz = G rho [[[dF/dz]]];
//  * voxel : the direct sum of the voxels' prism potentials regrouped by grid
//            node: every node is a corner of up to eight cells, each adding
//            its density with the corner's sign, so
//              Phi(x) = -G sum_nodes w_n F(n - x),  w_n = sum_cells s rho,
//            one corner-function evaluation per node instead of eight per
//            cell (the node-summation form of the prism sum).  Double
//            precision throughout, with compensated sums in a fixed order.
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "mcg_device.cuh"
#include "mcg_internal.h"

namespace mcg {

namespace {

struct FieldParams {
    int32_t kind;
    double G, rho0;
    double c[3], a;           // sphere
    double lo[3], hi[3];      // prism
    const float* grid;        // voxel grid, x fastest
    int32_t nx, ny, nz;
    double org[3], sp[3];
    const double* x;          // points, n x 3
    int64_t n;
    double* phi;
    double* gz;
};

__device__ __forceinline__ void neumaier(double& s, double& c, double v)
{
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

// F(x, y, z) and dF/dz of the prism corner function (Nagy):
//   F     = xy ln(z+r) + yz ln(x+r) + zx ln(y+r)
//           - x^2/2 atan(yz/(xr)) - y^2/2 atan(zx/(yr)) - z^2/2 atan(xy/(zr)),
//   dF/dz = x ln(y+r) + y ln(x+r) - z atan(xy/(zr)),
// a term whose polynomial prefactor is 0 taken as its limit 0; the two share
// their logarithms and the z arctangent.
__device__ __forceinline__ void corner_f_dfdz(double x, double y, double z, double& F, double& D)
{
    F = 0.0;
    D = 0.0;
    const double r = sqrt(x * x + y * y + z * z);
    if (r == 0.0) return;
    const double lx = (y != 0.0) ? log_tr(x, y, z, r) : 0.0;   // ln(x + r)
    const double ly = (x != 0.0) ? log_tr(y, z, x, r) : 0.0;   // ln(y + r)
    if (x * y != 0.0) F += x * y * log_tr(z, x, y, r);
    if (y * z != 0.0) F += y * z * lx;
    if (z * x != 0.0) F += z * x * ly;
    if (x != 0.0) F -= 0.5 * x * x * atan(y * z / (x * r));
    if (y != 0.0) F -= 0.5 * y * y * atan(z * x / (y * r));
    if (x != 0.0) D += x * ly;
    if (y != 0.0) D += y * lx;
    if (z != 0.0) {
        const double az = atan(x * y / (z * r));
        F -= 0.5 * z * z * az;
        D -= z * az;
    }
}

// Closed forms of the sphere and the prism, one thread per point.
__global__ void field_closed_kernel(const FieldParams P)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const double* x = P.x + 3 * i;
    double phi = 0.0, gz = 0.0;   // no density: no field
    if (P.kind == MCG_RHO_SPHERE) {
        const double dx = x[0] - P.c[0], dy = x[1] - P.c[1], dz = x[2] - P.c[2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double M = 4.0 / 3.0 * 3.14159265358979323846 * P.a * P.a * P.a * P.rho0;
        if (r >= P.a) {
            phi = -P.G * M / r;
            gz = P.G * M * dz / (r * r * r);
        } else {
            phi = -P.G * M * (3.0 * P.a * P.a - r * r) / (2.0 * P.a * P.a * P.a);
            gz = P.G * M * dz / (P.a * P.a * P.a);
        }
    } else if (P.kind == MCG_RHO_PRISM) {
        double sf = 0.0, sd = 0.0;
        for (int c = 0; c < 8; ++c) {
            const int ci = c & 1, cj = (c >> 1) & 1, ck = (c >> 2) & 1;
            double F, D;
            corner_f_dfdz((ci ? P.hi[0] : P.lo[0]) - x[0], (cj ? P.hi[1] : P.lo[1]) - x[1],
                          (ck ? P.hi[2] : P.lo[2]) - x[2], F, D);
            const bool neg = ((3 - ci - cj - ck) & 1) != 0;   // sign flips with every lower limit
            sf += neg ? -F : F;
            sd += neg ? -D : D;
        }
        phi = -P.G * P.rho0 * sf;
        gz = P.G * P.rho0 * sd;
    }
    if (P.phi) P.phi[i] = phi;
    if (P.gz) P.gz[i] = gz;
}

__device__ __forceinline__ double cell(const FieldParams& P, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= P.nx || j >= P.ny || k >= P.nz) return 0.0;
    return (double)__ldg(P.grid + i + (int64_t)P.nx * (j + (int64_t)P.ny * k));
}

// Voxel model by node summation: one block per point, threads stride over
// the (nx+1)(ny+1)(nz+1) nodes with compensated partial sums, then one thread
// adds the partials in thread order (deterministic).
constexpr int kFieldThreads = 256;

__global__ void __launch_bounds__(kFieldThreads) field_voxel_kernel(const FieldParams P)
{
    __shared__ double sh[2][kFieldThreads];
    const int64_t i = blockIdx.x;
    const double x0 = P.x[3 * i], x1 = P.x[3 * i + 1], x2 = P.x[3 * i + 2];
    const int64_t Nx = P.nx + 1, Ny = P.ny + 1, Nn = Nx * Ny * (int64_t)(P.nz + 1);
    double sf = 0.0, cf = 0.0, sd = 0.0, cd = 0.0;
    for (int64_t q = threadIdx.x; q < Nn; q += kFieldThreads) {
        const int a = (int)(q % Nx), b = (int)((q / Nx) % Ny), c = (int)(q / (Nx * Ny));
        // node (a, b, c) is the upper corner (sign +) of cell a-1 and the
        // lower corner (sign -) of cell a along each axis
        double w = 0.0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int di = m & 1, dj = (m >> 1) & 1, dk = (m >> 2) & 1;
            const double v = cell(P, a - 1 + di, b - 1 + dj, c - 1 + dk);
            w += ((di + dj + dk) & 1) ? -v : v;
        }
        if (w == 0.0) continue;
        double F, D;
        corner_f_dfdz(P.org[0] + a * P.sp[0] - x0, P.org[1] + b * P.sp[1] - x1, P.org[2] + c * P.sp[2] - x2, F,
                      D);
        neumaier(sf, cf, w * F);
        neumaier(sd, cd, w * D);
    }
    sh[0][threadIdx.x] = sf + cf;
    sh[1][threadIdx.x] = sd + cd;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, c0 = 0.0, s1 = 0.0, c1 = 0.0;
        for (int t = 0; t < kFieldThreads; ++t) {
            neumaier(s0, c0, sh[0][t]);
            neumaier(s1, c1, sh[1][t]);
        }
        if (P.phi) P.phi[i] = -P.G * (s0 + c0);
        if (P.gz) P.gz[i] = P.G * (s1 + c1);
    }
}

// The walks' own density samplers at given points and their two copies
// (x, y, z + h), (x, y, z - h), out[3 i + c]: the mixed walk's single-
// precision sampler on the point taken relative to the domain centre (the
// walk's frame), or the plain walk's double-precision sampler.
template <int RHO>
__global__ void density_f32_kernel(const WalkParams P, const double* __restrict__ x, int64_t n,
                                   double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float wx = (float)(x[3 * i] - P.cen[0]), wy = (float)(x[3 * i + 1] - P.cen[1]),
                wz = (float)(x[3 * i + 2] - P.cen[2]);
    float a, b, c;
    rho3_f32<RHO>(P, model_of(P), wx, wy, wz, P.h_f, a, b, c);
    out[3 * i] = a;
    out[3 * i + 1] = b;
    out[3 * i + 2] = c;
}

__global__ void density_f64_kernel(const WalkParams P, const double* __restrict__ x, int64_t n,
                                   double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double off[3] = {0.0, P.h, -P.h};
    for (int c = 0; c < 3; ++c) {
        const double X[3] = {x[3 * i], x[3 * i + 1], __dadd_rn(x[3 * i + 2], off[c])};
        out[3 * i + c] = rho_f64(P, model_of(P), X);
    }
}

}  // namespace

void preload_field_kernels()
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, (const void*)field_closed_kernel) != cudaSuccess) cudaGetLastError();
    if (cudaFuncGetAttributes(&a, (const void*)field_voxel_kernel) != cudaSuccess) cudaGetLastError();
    const void* fns[6] = {(const void*)density_f64_kernel,           (const void*)density_f32_kernel<MCG_RHO_NONE>,
                          (const void*)density_f32_kernel<MCG_RHO_SPHERE>, (const void*)density_f32_kernel<MCG_RHO_PRISM>,
                          (const void*)density_f32_kernel<MCG_RHO_VOXEL>,  (const void*)density_f32_kernel<kRhoVoxelPacked>};
    for (const void* f : fns)
        if (cudaFuncGetAttributes(&a, f) != cudaSuccess) cudaGetLastError();
}

}  // namespace mcg

using namespace mcg;

extern "C" int mcg_field(const mcg_density* density, const double* points_dev, int64_t n, double* phi_dev,
                         double* gz_dev, void* stream)
{
    if (!density) return set_error(MCG_ERR_ARG, "null density");
    if (n < 0) return set_error(MCG_ERR_ARG, "n must be non-negative");
    if (n == 0 || (!phi_dev && !gz_dev)) return MCG_OK;
    if (!points_dev) return set_error(MCG_ERR_ARG, "null points");
    if (!std::isfinite(density->G)) return set_error(MCG_ERR_ARG, "G must be finite");
    preload_kernels();
    FieldParams P;
    std::memset(&P, 0, sizeof(P));
    P.kind = density->kind;
    P.G = density->G;
    P.rho0 = density->rho0;
    P.x = points_dev;
    P.n = n;
    P.phi = phi_dev;
    P.gz = gz_dev;
    cudaStream_t st = (cudaStream_t)stream;
    switch (density->kind) {
    case MCG_RHO_NONE:
    case MCG_RHO_SPHERE:
    case MCG_RHO_PRISM: {
        for (int k = 0; k < 3; ++k) {
            P.c[k] = density->center[k];
            P.lo[k] = density->lo[k];
            P.hi[k] = density->hi[k];
        }
        P.a = density->radius;
        if (density->kind == MCG_RHO_SPHERE && !(density->radius > 0.0))
            return set_error(MCG_ERR_ARG, "sphere radius must be positive");
        const int64_t blocks = (n + 127) / 128;
        if (blocks > 2147483647LL) return set_error(MCG_ERR_ARG, "too many points");
        field_closed_kernel<<<(unsigned)blocks, 128, 0, st>>>(P);
        break;
    }
    case MCG_RHO_VOXEL: {
        if (!density->grid) return set_error(MCG_ERR_ARG, "voxel grid pointer is null");
        if (density->nx <= 0 || density->ny <= 0 || density->nz <= 0 || density->nx >= 65535 ||
            density->ny >= 65535 || density->nz >= 65535)
            return set_error(MCG_ERR_ARG, "voxel dims must be in [1, 65534]");
        if (n > 2147483647LL) return set_error(MCG_ERR_ARG, "too many points");
        P.grid = density->grid;
        P.nx = (int32_t)density->nx;
        P.ny = (int32_t)density->ny;
        P.nz = (int32_t)density->nz;
        for (int k = 0; k < 3; ++k) {
            if (!(density->spacing[k] > 0.0)) return set_error(MCG_ERR_ARG, "voxel spacing must be positive");
            P.org[k] = density->origin[k];
            P.sp[k] = density->spacing[k];
        }
        field_voxel_kernel<<<(unsigned)n, kFieldThreads, 0, st>>>(P);
        break;
    }
    default:
        return set_error(MCG_ERR_ARG, "unknown density kind %d", density->kind);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MCG_OK : set_error(MCG_ERR_CUDA, "field kernel launch: %s", cudaGetErrorString(e));
}

extern "C" int mcg_density_at(const mcg_domain* domain, const mcg_density* density, double h, int32_t precision,
                              const double* points_dev, int64_t n, double* out_dev, void* stream)
{
    if (!domain || !density) return set_error(MCG_ERR_ARG, "null domain or density");
    if (precision != MCG_FP64 && precision != MCG_MIXED) return set_error(MCG_ERR_ARG, "bad precision");
    if (!(h >= 0.0) || !std::isfinite(h)) return set_error(MCG_ERR_ARG, "h must be finite and non-negative");
    if (n < 0) return set_error(MCG_ERR_ARG, "n must be non-negative");
    mcg_boundary zero;
    std::memset(&zero, 0, sizeof(zero));
    zero.kind = MCG_G_ZERO;
    mcg_options o;
    mcg_options_default(&o);
    o.h = h;
    o.crn_gz = 1;
    o.precision = precision;
    WalkParams P;
    const int rc = make_params(domain, density, &zero, 1.0, 0, &o, P);
    if (rc) return rc;
    if (n == 0) return MCG_OK;
    if (!points_dev || !out_dev) return set_error(MCG_ERR_ARG, "null device buffer");
    if (n > 2147483647LL * 128LL) return set_error(MCG_ERR_ARG, "too many points");
    preload_kernels();
    const unsigned blocks = (unsigned)((n + 127) / 128);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == MCG_FP64) {
        density_f64_kernel<<<blocks, 128, 0, st>>>(P, points_dev, n, out_dev);
    } else {
        const int kind = (P.rho_kind == MCG_RHO_VOXEL && P.zq) ? kRhoVoxelPacked : P.rho_kind;
        switch (kind) {
        case MCG_RHO_SPHERE: density_f32_kernel<MCG_RHO_SPHERE><<<blocks, 128, 0, st>>>(P, points_dev, n, out_dev); break;
        case MCG_RHO_PRISM: density_f32_kernel<MCG_RHO_PRISM><<<blocks, 128, 0, st>>>(P, points_dev, n, out_dev); break;
        case MCG_RHO_VOXEL: density_f32_kernel<MCG_RHO_VOXEL><<<blocks, 128, 0, st>>>(P, points_dev, n, out_dev); break;
        case kRhoVoxelPacked:
            density_f32_kernel<kRhoVoxelPacked><<<blocks, 128, 0, st>>>(P, points_dev, n, out_dev);
            break;
        default: density_f32_kernel<MCG_RHO_NONE><<<blocks, 128, 0, st>>>(P, points_dev, n, out_dev); break;
        }
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MCG_OK : set_error(MCG_ERR_CUDA, "density kernel launch: %s", cudaGetErrorString(e));
}
