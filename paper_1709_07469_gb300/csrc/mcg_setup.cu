// mcg_setup.cu -- set-up of the heterogeneous model, run once per model
// outside the walk: the Gaussian-random-field density grid and the boundary
// tables of the Dirichlet data (the potential of the voxel model on the six
// faces of the box, by prism summation).
#include <cmath>

#include <cuda_runtime.h>

#include "mcg_device.cuh"
#include "mcg_internal.h"

namespace mcg {

namespace {

constexpr int kMaxTaps = 63;

struct Taps {
    double w[kMaxTaps];
    int R;
};

// White noise: voxels 4q..4q+3 take the two Box-Muller pairs of Philox
// counter (q, 0, 0, 1).
__global__ void grf_noise_kernel(uint32_t k0, uint32_t k1, int64_t n, double* __restrict__ a)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * q >= n) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)q, 0u, 0u, 1u), k0, k1);
    double z[4];
    box_muller_f64(w.x, w.y, z[0], z[1]);
    box_muller_f64(w.z, w.w, z[2], z[3]);
    for (int j = 0; j < 4; ++j)
        if (4 * q + j < n) a[4 * q + j] = z[j];
}

// One separable pass of the Gaussian filter along an axis of length L and
// stride st, zero outside the grid, taps summed from -R to R.
__global__ void grf_smooth_kernel(const double* __restrict__ a, double* __restrict__ b, int64_t n, int64_t L,
                                  int64_t st, const Taps T)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int64_t coord = (v / st) % L;
    double acc = 0.0;
    for (int m = -T.R; m <= T.R; ++m) {
        const int64_t c2 = coord + m;
        if (c2 < 0 || c2 >= L) continue;
        acc = __dadd_rn(acc, __dmul_rn(T.w[m + T.R], a[v + m * st]));
    }
    b[v] = acc;
}

// Mean and population standard deviation of a (one block, fixed order:
// strided Neumaier partial sums, then a pairwise tree).  out[0] = mean,
// out[1] = std.
__device__ void neumaier_add(double& s, double& c, double x)
{
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

__global__ void __launch_bounds__(1024) grf_moments_kernel(const double* __restrict__ a, int64_t n,
                                                           double* __restrict__ out)
{
    __shared__ double sh[1024];
    const int t = threadIdx.x;
    double s = 0.0, c = 0.0;
    for (int64_t i = t; i < n; i += 1024) neumaier_add(s, c, a[i]);
    sh[t] = s + c;
    __syncthreads();
    for (int k = 512; k > 0; k >>= 1) {
        if (t < k) sh[t] += sh[t + k];
        __syncthreads();
    }
    const double mean = sh[0] / (double)n;
    __syncthreads();
    s = 0.0;
    c = 0.0;
    for (int64_t i = t; i < n; i += 1024) {
        const double d = a[i] - mean;
        neumaier_add(s, c, d * d);
    }
    sh[t] = s + c;
    __syncthreads();
    for (int k = 512; k > 0; k >>= 1) {
        if (t < k) sh[t] += sh[t + k];
        __syncthreads();
    }
    if (t == 0) {
        out[0] = mean;
        out[1] = sqrt(sh[0] / (double)n);
    }
}

__global__ void grf_transform_kernel(const double* __restrict__ a, int64_t n, const double* __restrict__ mom,
                                     double amp, float* __restrict__ grid)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const double Z = (a[v] - mom[0]) / mom[1];
    grid[v] = (float)(amp * (exp(Z) - 1.0));
}

// ---------------------------------------------------------------------------
// Boundary tables.
// ---------------------------------------------------------------------------
struct TableParams {
    double lo[3], hi[3];
    int32_t nu, nv;
    const float* grid;
    int32_t nx, ny, nz;
    double org[3], sp[3];
    double vol;              // cell volume
    double near2;            // squared radius of the exact (near) zone
    double G;
    float* out;
};

constexpr int kTableThreads = 256;
constexpr int kRowsPerTile = 8;

__device__ __forceinline__ void node_position(const TableParams& T, int64_t node, double x[3])
{
    const int64_t per_face = (int64_t)T.nu * T.nv;
    const int f = (int)(node / per_face);
    const int64_t r = node % per_face;
    const int iu = (int)(r % T.nu), iv = (int)(r / T.nu);
    const int k = f >> 1;
    const int a = (k == 0) ? 1 : 0, b = (k == 2) ? 1 : 2;
    x[k] = (f & 1) ? T.hi[k] : T.lo[k];
    x[a] = T.lo[a] + (T.hi[a] - T.lo[a]) * (double)iu / (double)(T.nu - 1);
    x[b] = T.lo[b] + (T.hi[b] - T.lo[b]) * (double)iv / (double)(T.nv - 1);
}

// Point-mass far field for every voxel (single-precision terms, summed per
// row in single precision and per row into double), then the exact prism
// potential in place of the point mass for voxels whose centre lies within
// the near radius.  Writes Phi = -G sum.
__global__ void __launch_bounds__(kTableThreads) tables_kernel(const TableParams T)
{
    __shared__ float rho_s[kRowsPerTile][128];
    __shared__ float cx_s[128];  // voxel-centre x offsets, (float)ix * sx
    const int64_t nodes = 6ll * T.nu * T.nv;
    const int64_t node = (int64_t)blockIdx.x * kTableThreads + threadIdx.x;
    double x[3] = {0.0, 0.0, 0.0};
    if (node < nodes) node_position(T, node, x);
    // node relative to the first voxel centre, single precision
    const float px = (float)(x[0] - (T.org[0] + 0.5 * T.sp[0]));
    const float py = (float)(x[1] - (T.org[1] + 0.5 * T.sp[1]));
    const float pz = (float)(x[2] - (T.org[2] + 0.5 * T.sp[2]));
    const float sx = (float)T.sp[0], sy = (float)T.sp[1], sz = (float)T.sp[2];
    for (int i = threadIdx.x; i < 128; i += kTableThreads) cx_s[i] = (float)i * sx;
    double acc = 0.0;
    const int rows = T.ny * T.nz;
    for (int r0 = 0; r0 < rows; r0 += kRowsPerTile) {
        __syncthreads();
        for (int i = threadIdx.x; i < kRowsPerTile * 128; i += kTableThreads) {
            const int rr = i / 128, ix = i % 128;
            const int row = r0 + rr;
            rho_s[rr][ix] = (row < rows && ix < T.nx) ? __ldg(T.grid + (int64_t)row * T.nx + ix) : 0.0f;
        }
        __syncthreads();
        for (int rr = 0; rr < kRowsPerTile && r0 + rr < rows; ++rr) {
            const int row = r0 + rr;
            const float dy = (float)(row % T.ny) * sy - py;
            const float dz = (float)(row / T.ny) * sz - pz;
            const float dyz2 = fmaf(dy, dy, dz * dz);
            float part = 0.0f;
            for (int ix = 0; ix < T.nx; ++ix) {
                const float dx = cx_s[ix] - px;
                part = fmaf(rho_s[rr][ix], rsqrtf(fmaf(dx, dx, dyz2)), part);
            }
            acc += (double)part;
        }
    }
    if (node >= nodes) return;
    acc *= T.vol;
    // near zone: exact prism minus the point mass already counted
    const double R = sqrt(T.near2);
    int ilo[3], ihi[3];
    const int n[3] = {T.nx, T.ny, T.nz};
    for (int k = 0; k < 3; ++k) {
        const double a = fmin(fmax(floor((x[k] - R - T.org[k]) / T.sp[k]), 0.0), (double)n[k]);
        const double b = fmin(fmax(floor((x[k] + R - T.org[k]) / T.sp[k]), -1.0), (double)(n[k] - 1));
        ilo[k] = (int)a;
        ihi[k] = (int)b;
    }
    for (int iz = ilo[2]; iz <= ihi[2]; ++iz)
        for (int iy = ilo[1]; iy <= ihi[1]; ++iy)
            for (int ix = ilo[0]; ix <= ihi[0]; ++ix) {
                const double cx = T.org[0] + (ix + 0.5) * T.sp[0] - x[0];
                const double cy = T.org[1] + (iy + 0.5) * T.sp[1] - x[1];
                const double cz = T.org[2] + (iz + 0.5) * T.sp[2] - x[2];
                if (cx * cx + cy * cy + cz * cz >= T.near2) continue;
                const float rho = __ldg(T.grid + ((int64_t)iz * T.ny + iy) * T.nx + ix);
                if (rho == 0.0f) continue;
                const double lo[3] = {T.org[0] + ix * T.sp[0], T.org[1] + iy * T.sp[1], T.org[2] + iz * T.sp[2]};
                const double hi[3] = {lo[0] + T.sp[0], lo[1] + T.sp[1], lo[2] + T.sp[2]};
                // prism_potential returns -G rho [[[F]]]; with G = -1 it gives +rho [[[F]]]
                const double exact = prism_potential(-1.0, (double)rho, lo, hi, x);
                const float dx = cx_s[ix] - px, dy = (float)iy * sy - py, dz = (float)iz * sz - pz;
                const double pm = T.vol * (double)(rho * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))));
                acc += exact - pm;
            }
    T.out[node] = (float)(-T.G * acc);
}

// Packed voxel grid: entry (iz + 1, iy, ix) = layers iz-1, iz, iz+1 of
// column (ix, iy), 0 outside the grid, for iz = -1 .. nz.
__global__ void voxel_pack_kernel(const float* __restrict__ g, int nx, int ny, int nz, float4* __restrict__ out)
{
    const int64_t n = (int64_t)nx * ny * (nz + 2);
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)(e / ((int64_t)nx * ny)) - 1;
    const int64_t col = (int64_t)iy * nx + ix, plane = (int64_t)nx * ny;
    float v[3];
    for (int d = 0; d < 3; ++d) {
        const int k = iz - 1 + d;
        v[d] = (k >= 0 && k < nz) ? g[col + plane * k] : 0.0f;
    }
    out[e] = make_float4(v[0], v[1], v[2], 0.0f);
}

// Packed tables: entry (f, iv, iu) = the corners (iu, iv), (iu+1, iv),
// (iu, iv+1), (iu+1, iv+1) of cell (iu, iv) of face f.
__global__ void table_pack_kernel(const float* __restrict__ t, int nu, int nv, float4* __restrict__ out)
{
    const int64_t cells = (int64_t)(nu - 1) * (nv - 1);
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 6 * cells) return;
    const int f = (int)(e / cells);
    const int64_t r = e % cells;
    const int iu = (int)(r % (nu - 1)), iv = (int)(r / (nu - 1));
    const float* row = t + (int64_t)f * nu * nv + (int64_t)iv * nu + iu;
    out[e] = make_float4(row[0], row[1], row[nu], row[nu + 1]);
}

}  // namespace

int voxel_pack(const mcg_density* rho, float* out, cudaStream_t st)
{
    if (!rho || !out) return set_error(MCG_ERR_ARG, "null argument");
    if (rho->kind != MCG_RHO_VOXEL || !rho->grid) return set_error(MCG_ERR_ARG, "voxel_pack needs a voxel density");
    if (rho->nx <= 0 || rho->ny <= 0 || rho->nz <= 0) return set_error(MCG_ERR_ARG, "voxel dims must be positive");
    if ((double)rho->nx * (double)rho->ny * (double)(rho->nz + 2) >= 2147483647.0)
        return set_error(MCG_ERR_ARG, "voxel grid too large to pack");
    if ((uintptr_t)out % 16 != 0) return set_error(MCG_ERR_ARG, "packed grid must be 16-byte aligned");
    const int64_t n = rho->nx * rho->ny * (rho->nz + 2);
    voxel_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rho->grid, (int)rho->nx, (int)rho->ny,
                                                                      (int)rho->nz, (float4*)out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MCG_OK : set_error(MCG_ERR_CUDA, "voxel pack kernel: %s", cudaGetErrorString(e));
}

int table_pack(const mcg_boundary* b, float* out, cudaStream_t st)
{
    if (!b || !out) return set_error(MCG_ERR_ARG, "null argument");
    if (b->kind != MCG_G_TABLE || !b->faces || b->nu < 2 || b->nv < 2)
        return set_error(MCG_ERR_ARG, "table_pack needs tables with nu, nv >= 2");
    if ((uintptr_t)out % 16 != 0) return set_error(MCG_ERR_ARG, "packed tables must be 16-byte aligned");
    const int64_t n = 6ll * (b->nu - 1) * (b->nv - 1);
    if (n >= 2147483647LL) return set_error(MCG_ERR_ARG, "tables too large to pack");
    table_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b->faces, b->nu, b->nv, (float4*)out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MCG_OK : set_error(MCG_ERR_CUDA, "table pack kernel: %s", cudaGetErrorString(e));
}

int grf_density(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, double sigma_vox, double amp, float* grid_out,
                double* work, cudaStream_t st)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return set_error(MCG_ERR_ARG, "grid dims must be positive");
    if (!(sigma_vox > 0.0) || !std::isfinite(sigma_vox)) return set_error(MCG_ERR_ARG, "sigma_vox must be positive");
    const int R = (int)std::ceil(3.0 * sigma_vox);
    if (2 * R + 1 > kMaxTaps) return set_error(MCG_ERR_ARG, "sigma_vox too large (at most %d taps)", kMaxTaps);
    if (!grid_out || !work) return set_error(MCG_ERR_ARG, "null device buffer");
    const int64_t n = nx * ny * nz;
    Taps T;
    T.R = R;
    double wsum = 0.0;
    for (int m = -R; m <= R; ++m) {
        T.w[m + R] = std::exp(-(double)m * (double)m / (2.0 * sigma_vox * sigma_vox));
        wsum += T.w[m + R];
    }
    for (int m = 0; m <= 2 * R; ++m) T.w[m] /= wsum;
    double* a = work;
    double* b = work + n;
    double* mom = work + 2 * n;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int64_t q = (n + 3) / 4;
    grf_noise_kernel<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(k0, k1, n, a);
    const int64_t dims[3] = {nx, ny, nz}, strides[3] = {1, nx, nx * ny};
    for (int axis = 0; axis < 3; ++axis) {
        grf_smooth_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n, dims[axis], strides[axis], T);
        double* t = a;
        a = b;
        b = t;
    }
    grf_moments_kernel<<<1, 1024, 0, st>>>(a, n, mom);
    grf_transform_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, mom, amp, grid_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MCG_OK : set_error(MCG_ERR_CUDA, "grf kernels: %s", cudaGetErrorString(e));
}

int boundary_tables(const mcg_domain* d, const mcg_density* rho, int32_t nu, int32_t nv, double near_cells,
                    float* faces_out, cudaStream_t st)
{
    if (!d || !rho || !faces_out) return set_error(MCG_ERR_ARG, "null argument");
    if (rho->kind != MCG_RHO_VOXEL || !rho->grid) return set_error(MCG_ERR_ARG, "tables need a voxel density");
    if (nu < 2 || nv < 2) return set_error(MCG_ERR_ARG, "tables need nu, nv >= 2");
    if (rho->nx <= 0 || rho->nx > 128 || rho->ny <= 0 || rho->nz <= 0)
        return set_error(MCG_ERR_ARG, "table generation supports 1 <= nx <= 128 cells along x");
    if (!(near_cells >= 0.0)) return set_error(MCG_ERR_ARG, "near_cells must be >= 0");
    TableParams T;
    for (int k = 0; k < 3; ++k) {
        if (!(d->lo[k] < d->hi[k])) return set_error(MCG_ERR_ARG, "domain lo >= hi");
        if (!(rho->spacing[k] > 0.0)) return set_error(MCG_ERR_ARG, "voxel spacing must be positive");
        T.lo[k] = d->lo[k];
        T.hi[k] = d->hi[k];
        T.org[k] = rho->origin[k];
        T.sp[k] = rho->spacing[k];
    }
    T.nu = nu;
    T.nv = nv;
    T.grid = rho->grid;
    T.nx = (int32_t)rho->nx;
    T.ny = (int32_t)rho->ny;
    T.nz = (int32_t)rho->nz;
    T.vol = T.sp[0] * T.sp[1] * T.sp[2];
    const double diag = std::sqrt(T.sp[0] * T.sp[0] + T.sp[1] * T.sp[1] + T.sp[2] * T.sp[2]);
    T.near2 = (near_cells * diag) * (near_cells * diag);
    T.G = rho->G;
    T.out = faces_out;
    const int64_t nodes = 6ll * nu * nv;
    tables_kernel<<<(unsigned)((nodes + kTableThreads - 1) / kTableThreads), kTableThreads, 0, st>>>(T);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MCG_OK : set_error(MCG_ERR_CUDA, "tables kernel: %s", cudaGetErrorString(e));
}

}  // namespace mcg
