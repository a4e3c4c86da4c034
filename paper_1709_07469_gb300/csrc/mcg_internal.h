// mcg_internal.h -- launch parameters shared by the translation units of
// libmcgrav (host side of the C ABI and the kernels).  Not part of the ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mcgrav.h"

namespace mcg {

// Everything one walk launch needs, passed by value as a kernel parameter.
// Coordinates of the mixed-precision walk are relative to the box centre
// (`cen`), so the exit test is |x_k| < half_k; the FP64 walk uses absolute
// coordinates exactly as the problem states them.
struct WalkParams {
    // domain: the box (lo, hi), or the ball |x - cen| < R (ball = 1)
    int32_t ball;
    double R, R2;
    float R2_f, in_r2_f;           // ball radius^2; all copies surely inside below in_r2_f
    double lo[3], hi[3], cen[3];
    float half_f[3];
    float in_f[3];                 // all three copies surely inside: |x_k| < in_f[k]
    float far_c[3], far_h[3];      // density surely 0 at all copies outside this box
    float far_r2;                  // ... or (sphere) beyond this squared radius
    // density
    int32_t rho_kind;
    double G, rho0;
    float rho0_f;
    double sc[3], srad, srad2;     // sphere centre, radius, radius^2 (absolute)
    float sc_f[3], srad2_f;        // sphere centre relative to cen
    double plo[3], phi[3];         // prism (absolute)
    float plo_f[3], phi_f[3];      // prism relative to cen
    const float* grid;
    int32_t nx, ny, nz;
    double org[3], sp[3];          // voxel origin / spacing (absolute)
    float org_f[3], inv_sp_f[3];   // origin relative to cen, 1/spacing
    float hz_f;                    // h / spacing[2]: the copies' z offset in cells
    const float4* zq;              // packed voxel grid (layers iz-1, iz, iz+1 per cell), or null
    // boundary data
    int32_t g_kind;
    const float* faces;
    const float4* tq;              // packed table cells (four corners), or null
    int32_t nu, nv;
    double poly[11];
    // walk
    double dt, sd, h, two_pi_G;
    float sd_f, h_f, lnscale_f;    // lnscale_f = -2 ln 2 sd^2
    int32_t crn, clip, bridge, refill_min;
    int32_t spill_max;             // a warp with at most this many live walks hands them over
    float bridge_k_f;              // -2 / (sigma^2 dt), single precision
    double bridge_k;               // -2 / (sigma^2 dt)
    int64_t max_steps;
    uint32_t key0, key1;
    // work list: item i -> station i / N, path p0 + i % N
    const double* stations;
    int64_t S, N, p0;
    unsigned long long total;
    double* pp_u;
    double* pp_d;
    int64_t* pp_steps;
    int32_t* status;
    unsigned long long* counter;
    float* frec;                   // mixed walk: exit records (32 bytes per copy per item), or null
    volatile int32_t* cancel;
    // mixed walk, migration of walks between warps once the work list is used
    // up (null pool: off).  pool: kPoolEntryBytes per slot; pool_ready: one
    // flag per slot; pool_ctr: [0] slots reserved, [1] slots claimed, [2]
    // warps gone.
    unsigned char* pool;
    uint32_t* pool_ready;
    unsigned long long* pool_ctr;
    unsigned long long pool_cap;
    uint32_t fault_unpublished;    // host side: pool slots reserved and never published
    // multi-request launch: segment table (device) sorted by begin, or null
    const struct WalkSeg* seg;
    int32_t nseg;
};

// One request's part of a multi-request walk launch (the server's batched
// rounds): items begin .. begin + S N - 1 of the launch are paths p0 .. p0 +
// N - 1 of each of the request's S stations, item begin + s N + (p - p0).
// The requests of one launch share every scalar of the problem (domain,
// density and boundary kinds, grid geometry, step, h) but have their own
// stations, generator key, status word and model arrays.
struct WalkSeg {
    unsigned long long begin;
    const double* stations;
    int64_t N, p0;
    int32_t* status;
    const float* grid;
    const float4* zq;
    const float* faces;
    const float4* tq;
    uint32_t key0, key1;
};

// Completion flag of a mixed-walk item, kept in its step count: set when every
// copy has left Omega and written its exit record.  The exit kernel evaluates
// flagged items only and clears the flag; an item without it (never started,
// cancelled, capped, lost, station outside Omega) gets NaN.  Step counts stay
// far below 2^62.
constexpr long long kDoneFlag = 1LL << 62;

// Kernel-template tag of the voxel density read through the packed grid
// (WalkParams::zq); not a public density kind.
constexpr int kRhoVoxelPacked = 4;

constexpr size_t kPoolEntryBytes = 80;
constexpr unsigned long long kPoolMaxSlots = 1ull << 19;

// Offsets inside the mixed walk's scratch of n = S * N items (mcg_api.cu):
// exit records, migration pool, ready flags, pool counters.
constexpr size_t kExitRecordBytes = 32;
struct WorkLayout {
    size_t frec, pool, ready, ctr, total;
    unsigned long long cap;
};
WorkLayout work_layout(size_t n);
// Points P's mixed-walk buffers into `work` (layout above); migration on/off.
void bind_work(WalkParams& P, void* work, bool migrate);
// mcgrav_solve's workspace parts (mcg_api.cu).
size_t solve_shared_bytes(int64_t S);
size_t solve_set_bytes(int64_t S, int64_t batch);
// Zeroes the work counter, marks every item "no result" (exit records of the
// mixed walk, per-path values of the FP64 walk, steps 0) and, with migration,
// zeroes the pool's flags and counters.
cudaError_t reset_walk(const WalkParams& P, cudaStream_t st);

// Kernel launchers (mcg_walk.cu).
cudaError_t launch_walk(const WalkParams& P, int precision, int block, cudaStream_t st);
int walk_blocks_per_sm(int precision, int rho_kind, int block, bool seg = false);

// Reduction launchers (mcg_reduce.cu).
cudaError_t launch_reduce(const double* pp_u, const double* pp_d, const int64_t* pp_steps, int64_t S,
                          int64_t N, mcg_station_state* states, cudaStream_t st);
cudaError_t launch_finalize(const mcg_station_state* states, int64_t S, double* u, double* gz, double* se_u,
                            double* se_gz, int64_t* n_paths, int64_t* path_steps, cudaStream_t st);

// RNG launchers (mcg_rng.cu).
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, uint32_t s, uint32_t p, uint32_t b0, int64_t nblocks, int precision,
                           void* out, cudaStream_t st);

// Packed model arrays (mcg_setup.cu).
int voxel_pack(const mcg_density* rho, float* out, cudaStream_t st);
int table_pack(const mcg_boundary* b, float* out, cudaStream_t st);

// Set-up launchers (mcg_setup.cu).
int grf_density(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, double sigma_vox, double amp, float* grid_out,
                double* work, cudaStream_t st);
int boundary_tables(const mcg_domain* d, const mcg_density* rho, int32_t nu, int32_t nv, double near_cells,
                    float* faces_out, cudaStream_t st);

// Loads every walk and reduction kernel of the library into the current
// context (cudaFuncGetAttributes).  With CUDA's lazy module loading the first
// launch of a kernel otherwise loads it on the spot, and that load waits for
// the kernels already running on the device: a host thread that queues the
// exit kernel behind a running walk would block until the walk ends.
// preload_kernels() does it once per device (mcg_api.cu).
void preload_walk_kernels();    // mcg_walk.cu
void preload_reduce_kernels();  // mcg_reduce.cu
void preload_field_kernels();   // mcg_field.cu
void preload_kernels();

// Thread-local error message (mcg_api.cu).
int set_error(int code, const char* fmt, ...);

// Argument checks shared by the entry points (mcg_api.cu).
int make_params(const mcg_domain* D, const mcg_density* R, const mcg_boundary* B, double dt, uint64_t seed,
                const mcg_options* o, WalkParams& P);
int check_station(const WalkParams& P, const double* x, int64_t s);
int status_from_bits(int bits);
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace mcg
