// mcg_api.cu -- the C ABI declared in include/mcgrav.h: argument checks, the
// walk's launch parameters, and the one-call solver that runs walk ->
// reduce batch by batch and copies the station results back.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include <cuda_runtime.h>

#include "mcg_internal.h"
#include "mcgrav.h"

namespace mcg {

namespace {
thread_local char g_err[512] = "";

constexpr double kPi = 3.14159265358979323846;

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int cuda_fail(cudaError_t e, const char* what)
{
    return set_error(MCG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

int set_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

// True when p is host memory (pageable or pinned): mcgrav_solve then stages
// the array in its workspace instead of letting kernels read it.
bool host_memory(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

// mcgrav_solve's workspace: a shared part (stations, station states, status
// word, finalized results) and one or two per-launch sets (per-path values,
// work counter, walk scratch) -- two when the solve has several batches, so
// consecutive batches alternate between them on two streams.
size_t solve_shared_bytes(int64_t S)
{
    const size_t s = (size_t)S;
    return align256(s * 3 * sizeof(double)) + align256(s * sizeof(mcg_station_state)) + 256 +
           align256(s * 6 * sizeof(double));
}

size_t solve_set_bytes(int64_t S, int64_t batch)
{
    const size_t n = (size_t)S * (size_t)batch;
    return 2 * align256(n * sizeof(double)) + align256(n * sizeof(int64_t)) + 256 +
           mcg_walk_work_bytes(S, batch, MCG_MIXED);
}

void preload_kernels()
{
    static std::atomic<unsigned long long> loaded{0};  // one bit per device ordinal < 64
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (loaded.load(std::memory_order_acquire) & bit)) return;
    std::lock_guard<std::mutex> lock(mu);
    if (bit && (loaded.load(std::memory_order_relaxed) & bit)) return;
    preload_walk_kernels();
    preload_reduce_kernels();
    preload_field_kernels();
    loaded.fetch_or(bit, std::memory_order_release);
}

WorkLayout work_layout(size_t n)
{
    WorkLayout L;
    L.cap = n < kPoolMaxSlots ? (unsigned long long)n : kPoolMaxSlots;
    size_t o = 0;
    L.frec = o;
    o += align256(n * 3 * kExitRecordBytes);
    L.pool = o;
    o += align256((size_t)L.cap * kPoolEntryBytes);
    L.ready = o;
    o += align256((size_t)L.cap * sizeof(uint32_t));
    L.ctr = o;
    o += 256;
    L.total = o;
    return L;
}

void bind_work(WalkParams& P, void* work, bool migrate)
{
    const WorkLayout L = work_layout((size_t)P.total);
    unsigned char* w = (unsigned char*)work;
    P.frec = (float*)(w + L.frec);
    if (migrate && L.cap > 0) {
        P.pool = w + L.pool;
        P.pool_ready = (uint32_t*)(w + L.ready);
        P.pool_ctr = (unsigned long long*)(w + L.ctr);
        P.pool_cap = L.cap;
    } else {
        P.pool = nullptr;
        P.pool_ready = nullptr;
        P.pool_ctr = nullptr;
        P.pool_cap = 0;
    }
}

cudaError_t reset_walk(const WalkParams& P, cudaStream_t st)
{
    const size_t T = (size_t)P.total;
    cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), st);
    // Items that never finish (cancel, a lost walk) must not read an earlier
    // launch's values: steps 0, which also clears the mixed walk's completion
    // flags (its exit kernel writes NaN for items without one), or NaN
    // per-path values (FP64 walk, which writes them directly).
    if (e == cudaSuccess) e = cudaMemsetAsync(P.pp_steps, 0, T * sizeof(int64_t), st);
    if (e == cudaSuccess && !P.frec) e = cudaMemsetAsync(P.pp_u, 0xFF, T * sizeof(double), st);
    if (e == cudaSuccess && !P.frec) e = cudaMemsetAsync(P.pp_d, 0xFF, T * sizeof(double), st);
    if (e == cudaSuccess && P.pool) {
        // flags and counters are adjacent: one memset covers both
        const size_t bytes = (size_t)((unsigned char*)P.pool_ctr - (unsigned char*)P.pool_ready) + 256;
        e = cudaMemsetAsync(P.pool_ready, 0, bytes, st);
        // test hook: slots counted as reserved whose ready flag nobody sets
        // (the low byte of the little-endian reservation counter)
        if (e == cudaSuccess && P.fault_unpublished)
            e = cudaMemsetAsync(P.pool_ctr, (int)P.fault_unpublished, 1, st);
    }
    return e;
}

// Checks the problem description and fills the launch parameters (without
// the work list, which the caller adds).
int make_params(const mcg_domain* D, const mcg_density* R, const mcg_boundary* B, double dt, uint64_t seed,
                const mcg_options* o, WalkParams& P)
{
    if (!D || !R || !B || !o) return set_error(MCG_ERR_ARG, "null domain/density/boundary/options");
    preload_kernels();
    std::memset(&P, 0, sizeof(P));
    if (D->kind == MCG_DOMAIN_BALL) {
        if (!finite3(D->center) || !(D->radius > 0.0) || !std::isfinite(D->radius))
            return set_error(MCG_ERR_ARG, "ball domain needs a finite centre and radius > 0");
        P.ball = 1;
        P.R = D->radius;
        P.R2 = D->radius * D->radius;
        P.R2_f = (float)P.R2;
        for (int k = 0; k < 3; ++k) {
            P.cen[k] = D->center[k];
            P.lo[k] = D->center[k] - D->radius;  // bounding box
            P.hi[k] = D->center[k] + D->radius;
            P.half_f[k] = (float)D->radius;
        }
    } else if (D->kind == MCG_DOMAIN_BOX) {
        if (!finite3(D->lo) || !finite3(D->hi)) return set_error(MCG_ERR_ARG, "domain bounds must be finite");
        for (int k = 0; k < 3; ++k) {
            if (!(D->lo[k] < D->hi[k])) return set_error(MCG_ERR_ARG, "domain lo[%d] >= hi[%d]", k, k);
            P.lo[k] = D->lo[k];
            P.hi[k] = D->hi[k];
            P.cen[k] = 0.5 * (D->lo[k] + D->hi[k]);
            P.half_f[k] = (float)(0.5 * (D->hi[k] - D->lo[k]));
        }
    } else {
        return set_error(MCG_ERR_ARG, "unknown domain kind %d", D->kind);
    }
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(MCG_ERR_ARG, "dt must be positive and finite");
    if (!(o->sigma > 0.0) || !std::isfinite(o->sigma)) return set_error(MCG_ERR_ARG, "sigma must be positive");
    if (o->crn_gz && !(o->h > 0.0)) return set_error(MCG_ERR_ARG, "h must be positive when crn_gz = 1");
    if (o->precision != MCG_FP64 && o->precision != MCG_MIXED)
        return set_error(MCG_ERR_ARG, "precision must be MCG_FP64 or MCG_MIXED");
    if (o->max_steps <= 0) return set_error(MCG_ERR_ARG, "max_steps must be positive");
    if (o->block != 0 && (o->block < 32 || o->block > 128 || o->block % 32 != 0))
        return set_error(MCG_ERR_ARG, "block must be 0 or a multiple of 32 in [32, 128]");

    P.rho_kind = R->kind;
    P.G = R->G;
    P.rho0 = R->rho0;
    P.rho0_f = (float)R->rho0;
    if (!std::isfinite(R->G)) return set_error(MCG_ERR_ARG, "G must be finite");
    switch (R->kind) {
    case MCG_RHO_NONE:
        break;
    case MCG_RHO_SPHERE:
        if (!(R->radius > 0.0) || !finite3(R->center)) return set_error(MCG_ERR_ARG, "sphere radius/centre");
        for (int k = 0; k < 3; ++k) {
            P.sc[k] = R->center[k];
            P.sc_f[k] = (float)(R->center[k] - P.cen[k]);
        }
        P.srad = R->radius;
        P.srad2 = R->radius * R->radius;
        P.srad2_f = (float)P.srad2;
        break;
    case MCG_RHO_PRISM:
        for (int k = 0; k < 3; ++k) {
            if (!(R->lo[k] < R->hi[k])) return set_error(MCG_ERR_ARG, "prism lo[%d] >= hi[%d]", k, k);
            P.plo[k] = R->lo[k];
            P.phi[k] = R->hi[k];
            P.plo_f[k] = (float)(R->lo[k] - P.cen[k]);
            P.phi_f[k] = (float)(R->hi[k] - P.cen[k]);
        }
        break;
    case MCG_RHO_VOXEL: {
        if (!R->grid) return set_error(MCG_ERR_ARG, "voxel grid pointer is null");
        if (R->nx <= 0 || R->ny <= 0 || R->nz <= 0) return set_error(MCG_ERR_ARG, "voxel dims must be positive");
        if ((double)R->nx * (double)R->ny * (double)R->nz >= 2147483647.0)
            return set_error(MCG_ERR_ARG, "voxel grid too large (>= 2^31 cells)");
        P.grid = R->grid;
        P.nx = (int32_t)R->nx;
        P.ny = (int32_t)R->ny;
        P.nz = (int32_t)R->nz;
        for (int k = 0; k < 3; ++k) {
            if (!(R->spacing[k] > 0.0)) return set_error(MCG_ERR_ARG, "voxel spacing must be positive");
            P.org[k] = R->origin[k];
            P.sp[k] = R->spacing[k];
            P.org_f[k] = (float)(R->origin[k] - P.cen[k]);
            P.inv_sp_f[k] = (float)(1.0 / R->spacing[k]);
        }
        break;
    }
    default:
        return set_error(MCG_ERR_ARG, "unknown density kind %d", R->kind);
    }

    P.g_kind = B->kind;
    switch (B->kind) {
    case MCG_G_ZERO:
    case MCG_G_POLY:
        break;
    case MCG_G_SPHERE:
        if (R->kind != MCG_RHO_SPHERE) return set_error(MCG_ERR_ARG, "MCG_G_SPHERE needs a sphere density");
        break;
    case MCG_G_PRISM:
        if (R->kind != MCG_RHO_PRISM) return set_error(MCG_ERR_ARG, "MCG_G_PRISM needs a prism density");
        break;
    case MCG_G_TABLE:
        if (!B->faces || B->nu < 2 || B->nv < 2) return set_error(MCG_ERR_ARG, "tables need faces and nu, nv >= 2");
        if (!o->clip) return set_error(MCG_ERR_ARG, "tabulated boundary data needs clip = 1");
        if (P.ball) return set_error(MCG_ERR_ARG, "tabulated boundary data needs the box domain");
        break;
    default:
        return set_error(MCG_ERR_ARG, "unknown boundary kind %d", B->kind);
    }
    P.faces = B->faces;
    P.nu = B->nu;
    P.nv = B->nv;
    if (B->kind == MCG_G_TABLE && B->quads) {
        if ((uintptr_t)B->quads % 16 != 0) return set_error(MCG_ERR_ARG, "boundary quads must be 16-byte aligned");
        P.tq = (const float4*)B->quads;
    }
    for (int i = 0; i < 11; ++i) P.poly[i] = B->poly[i];

    P.dt = dt;
    P.sd = o->sigma * std::sqrt(dt);
    P.h = o->crn_gz ? o->h : 0.0;
    P.two_pi_G = 2.0 * kPi * R->G;
    P.sd_f = (float)P.sd;
    P.h_f = (float)P.h;
    if (R->kind == MCG_RHO_VOXEL) P.hz_f = (float)(P.h / R->spacing[2]);
    if (R->kind == MCG_RHO_VOXEL && R->zpack) {
        if ((uintptr_t)R->zpack % 16 != 0) return set_error(MCG_ERR_ARG, "voxel zpack must be 16-byte aligned");
        // one packed entry covers the copies' layers only while h <= half a cell
        if (!(P.hz_f <= 0.5f)) return set_error(MCG_ERR_ARG, "zpack needs h <= spacing[2] / 2");
        P.zq = (const float4*)R->zpack;
    }
    P.lnscale_f = (float)(-2.0 * std::log(2.0) * P.sd * P.sd);
    P.crn = o->crn_gz ? 1 : 0;
    P.clip = o->clip ? 1 : 0;
    P.bridge = o->bridge ? 1 : 0;
    if (P.bridge && P.ball) return set_error(MCG_ERR_ARG, "the Brownian-bridge test needs the box domain");
    if (o->refill_min < 0 || o->refill_min > 32) return set_error(MCG_ERR_ARG, "refill_min must be in [0, 32]");
    P.refill_min = o->refill_min > 0 ? o->refill_min : 1;
    if (o->spill_max < 0 || o->spill_max > 32) return set_error(MCG_ERR_ARG, "spill_max must be in [0, 32]");
    P.spill_max = o->spill_max > 0 ? o->spill_max : 24;
    P.bridge_k = -2.0 / (P.sd * P.sd);
    P.bridge_k_f = (float)P.bridge_k;
    // Conservative boxes for the walk's common step (all copies inside, no
    // density at any copy): a margin of 1e-5 of the largest half-width
    // covers the single-precision rounding of the tests several times over.
    {
        const double hmax = std::fmax(std::fmax(P.half_f[0], P.half_f[1]), P.half_f[2]);
        // with the bridge test, steps within 6 sd of a face take the exact
        // path: beyond that exp(-2 d_X d_Y / sd^2) < exp(-72) is below any
        // uniform the generator can produce
        const double margin = 1e-5 * hmax + (P.bridge ? 6.0 * P.sd : 0.0);
        P.in_f[0] = (float)(P.half_f[0] - margin);
        P.in_f[1] = (float)(P.half_f[1] - margin);
        P.in_f[2] = (float)(P.half_f[2] - P.h - margin);
        if (P.ball) {
            const double rin = P.R - P.h - margin;
            P.in_r2_f = rin > 0.0 ? (float)(rin * rin) : -1.0f;
        }
        if (R->kind == MCG_RHO_PRISM) {
            for (int k = 0; k < 3; ++k) {
                P.far_c[k] = (float)(0.5 * ((double)P.plo_f[k] + (double)P.phi_f[k]));
                P.far_h[k] = (float)(0.5 * ((double)P.phi_f[k] - (double)P.plo_f[k]) + margin + (k == 2 ? P.h : 0.0));
            }
        } else if (R->kind == MCG_RHO_SPHERE) {
            const double rf = R->radius + P.h + margin;
            P.far_r2 = (float)(rf * rf);
            // the cube around that ball, for tests of a whole step block
            for (int k = 0; k < 3; ++k) {
                P.far_c[k] = P.sc_f[k];
                P.far_h[k] = (float)rf;
            }
        }
    }
    P.max_steps = o->max_steps;
    if (o->fault_unpublished < 0 || o->fault_unpublished > 255)
        return set_error(MCG_ERR_ARG, "fault_unpublished must be in [0, 255]");
    P.fault_unpublished = (uint32_t)o->fault_unpublished;
    P.key0 = (uint32_t)seed;
    P.key1 = (uint32_t)(seed >> 32);
    P.cancel = o->cancel;
    return MCG_OK;
}

int check_station(const WalkParams& P, const double* x, int64_t s)
{
    if (!finite3(x)) return set_error(MCG_ERR_ARG, "station %lld is not finite", (long long)s);
    const double off[3] = {0.0, P.h, -P.h};
    for (int c = 0; c < (P.crn ? 3 : 1); ++c) {
        const double y[3] = {x[0], x[1], x[2] + off[c]};
        bool in = true;
        if (P.ball) {
            const double dx = y[0] - P.cen[0], dy = y[1] - P.cen[1], dz = y[2] - P.cen[2];
            in = dx * dx + dy * dy + dz * dz < P.R2;
        } else {
            for (int k = 0; k < 3; ++k) in = in && y[k] > P.lo[k] && y[k] < P.hi[k];
        }
        if (!in)
            return set_error(MCG_ERR_ARG, "station %lld (copy %d) is not strictly inside the domain", (long long)s,
                             c);
    }
    return MCG_OK;
}

// Status of a walk from its device status word.  Every nonzero word is an
// error: an unknown bit maps to MCG_ERR_CUDA rather than to success.
int status_from_bits(int bits)
{
    if (bits == 0) return MCG_OK;
    if (bits & (1 << MCG_ERR_ARG)) return set_error(MCG_ERR_ARG, "a station lies on or outside the domain");
    if (bits & (1 << MCG_ERR_TIMEOUT))
        return set_error(MCG_ERR_TIMEOUT, "a bounded wait on a migrated walk gave up (that walk reads NaN)");
    if (bits & (1 << MCG_ERR_CANCELLED)) return set_error(MCG_ERR_CANCELLED, "cancelled");
    if (bits & (1 << MCG_ERR_STEP_CAP)) return set_error(MCG_ERR_STEP_CAP, "a path exceeded max_steps");
    if (bits & (1 << MCG_ERR_NONFINITE)) return set_error(MCG_ERR_NONFINITE, "a per-path value was not finite");
    return set_error(MCG_ERR_CUDA, "unknown walk status bits 0x%x", (unsigned)bits);
}

}  // namespace mcg

// ---------------------------------------------------------------------------
// Fixed scratch for mcg_walk_static: a file-scope device array that every GPU
// loading this library holds until the process exits.  Layout: the walk's
// work counter (first 256 bytes), then the mixed walk's exit records.
// ---------------------------------------------------------------------------
#define MCG_STATIC_SCRATCH_BYTES (64u << 20)
static __device__ __align__(256) unsigned char mcg_static_scratch[MCG_STATIC_SCRATCH_BYTES];

namespace mcg {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_base[kMaxDevices] = {};

// Device address of mcg_static_scratch on `dev` (the current device).  The
// host-side symbol is only a stand-in for the array, so the address is
// looked up once per device with that device current.
int static_scratch(int dev, unsigned char** base)
{
    if (dev < 0 || dev >= kMaxDevices) return set_error(MCG_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_base[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, mcg_static_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return set_error(MCG_ERR_CUDA, "cudaGetSymbolAddress(mcg_static_scratch) on device %d: %s", dev,
                             cudaGetErrorString(e));
        }
        g_static_base[dev] = ptr;
    }
    *base = (unsigned char*)g_static_base[dev];
    return MCG_OK;
}

// Largest S * N whose exit records fit behind the 256-byte counter slot.
int64_t static_max_items()
{
    const size_t avail = (size_t)MCG_STATIC_SCRATCH_BYTES - 256;
    int64_t n = (int64_t)(avail / (3 * kExitRecordBytes));
    while (n > 0 && align256((size_t)n * 3 * kExitRecordBytes) > avail) --n;
    return n;
}

}  // namespace
}  // namespace mcg

using namespace mcg;

extern "C" {

void mcg_options_default(mcg_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->h = 1e-2;
    o->sigma = 1.0;
    o->precision = MCG_MIXED;
    o->clip = 1;
    o->crn_gz = 1;
    o->block = 0;
    o->max_steps = (int64_t)1 << 31;
    o->batch_paths = 0;
    o->stream = nullptr;
    o->cancel = nullptr;
    o->bridge = 0;
    o->refill_min = 1;
    o->graph = 1;
    o->migrate = 1;
    o->fault_unpublished = 0;
    o->spill_max = 24;
}

const char* mcg_last_error(void) { return g_err; }

const char* mcg_version(void) { return "mcgrav 0.1 sm_103a"; }

size_t mcg_workspace_bytes(int64_t S, int64_t batch)
{
    if (S <= 0 || batch <= 0) return 0;
    return solve_shared_bytes(S) + 2 * solve_set_bytes(S, batch);
}

size_t mcg_walk_work_bytes(int64_t S, int64_t N, int32_t precision)
{
    if (S <= 0 || N <= 0 || precision != MCG_MIXED) return 0;
    return work_layout((size_t)S * (size_t)N).total;
}

int mcg_walk(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
             const double* stations_dev, int64_t S, int64_t p0, int64_t N, double dt, uint64_t seed,
             const mcg_options* opts, double* pp_u, double* pp_d, int64_t* pp_steps, void* work_dev,
             int32_t* status_dev, unsigned long long* counter_dev)
{
    WalkParams P;
    int rc = make_params(domain, density, boundary, dt, seed, opts, P);
    if (rc) return rc;
    if (S < 0 || N < 0 || p0 < 0) return set_error(MCG_ERR_ARG, "S, N and p0 must be non-negative");
    if (p0 + N > (int64_t)1 << 32) return set_error(MCG_ERR_ARG, "path indices must fit in 32 bits");
    if (S > (int64_t)1 << 32) return set_error(MCG_ERR_ARG, "station indices must fit in 32 bits");
    if (S == 0 || N == 0) return MCG_OK;
    if (!stations_dev || !pp_u || !pp_d || !pp_steps || !status_dev || !counter_dev)
        return set_error(MCG_ERR_ARG, "null device buffer");
    P.stations = stations_dev;
    P.S = S;
    P.N = N;
    P.p0 = p0;
    P.total = (unsigned long long)S * (unsigned long long)N;
    P.pp_u = pp_u;
    P.pp_d = pp_d;
    P.pp_steps = pp_steps;
    P.status = status_dev;
    P.counter = counter_dev;
    if (opts->precision == MCG_MIXED) {
        if (!work_dev) return set_error(MCG_ERR_ARG, "the mixed walk needs work_dev (mcg_walk_work_bytes)");
        if ((uintptr_t)work_dev % 256 != 0) return set_error(MCG_ERR_ARG, "work_dev must be 256-byte aligned");
        bind_work(P, work_dev, opts->migrate != 0);
    }
    cudaStream_t st = (cudaStream_t)opts->stream;
    cudaError_t e = reset_walk(P, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
    e = launch_walk(P, opts->precision, opts->block ? opts->block : 128, st);
    if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    return MCG_OK;
}

int mcg_reduce(const double* pp_u, const double* pp_d, const int64_t* pp_steps, int64_t S, int64_t N,
               mcg_station_state* states_dev, void* stream)
{
    if (S < 0 || N < 0) return set_error(MCG_ERR_ARG, "S and N must be non-negative");
    if (S == 0 || N == 0) return MCG_OK;
    if (!pp_u || !pp_d || !pp_steps || !states_dev) return set_error(MCG_ERR_ARG, "null device buffer");
    if (S > 2147483647LL) return set_error(MCG_ERR_ARG, "too many stations for one reduction");
    preload_kernels();
    cudaError_t e = launch_reduce(pp_u, pp_d, pp_steps, S, N, states_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? MCG_OK : cuda_fail(e, "reduce kernel launch");
}

int mcg_finalize(const mcg_station_state* states_dev, int64_t S, double* u, double* gz, double* se_u,
                 double* se_gz, int64_t* n_paths, int64_t* path_steps, void* stream)
{
    if (S < 0) return set_error(MCG_ERR_ARG, "S must be non-negative");
    if (S == 0) return MCG_OK;
    if (!states_dev) return set_error(MCG_ERR_ARG, "null states");
    preload_kernels();
    cudaError_t e = launch_finalize(states_dev, S, u, gz, se_u, se_gz, n_paths, path_steps, (cudaStream_t)stream);
    return e == cudaSuccess ? MCG_OK : cuda_fail(e, "finalize kernel launch");
}

int mcgrav_solve(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
                 const double* stations, int64_t S, int64_t paths, double dt, uint64_t seed,
                 const mcg_options* opts_in, mcg_result* out)
{
    mcg_options opts;
    if (opts_in) opts = *opts_in;
    else mcg_options_default(&opts);
    WalkParams P;
    int rc = make_params(domain, density, boundary, dt, seed, &opts, P);
    if (rc) return rc;
    if (S < 0 || paths <= 0) return set_error(MCG_ERR_ARG, "need S >= 0 and paths >= 1");
    if (paths > (int64_t)1 << 32) return set_error(MCG_ERR_ARG, "paths must fit in 32 bits");
    if (S > 0 && (!stations || !out)) return set_error(MCG_ERR_ARG, "null stations or result");
    for (int64_t s = 0; s < S; ++s)
        if ((rc = check_station(P, stations + 3 * s, s))) return rc;
    if (S == 0) return MCG_OK;

    int64_t batch = opts.batch_paths;
    if (batch <= 0) {
        // per-path buffers, exit records and migration pool of at most ~4 GiB per launch
        const double per_path = (double)mcg_workspace_bytes(S, 4096) / (4096.0 * (double)S);
        const int64_t cap = (int64_t)((double)(4ull << 30) / (per_path * (double)S));
        batch = paths < cap ? paths : (cap > 0 ? cap : 1);
    }
    if (batch > paths) batch = paths;
    const int64_t nbatch = (paths + batch - 1) / batch;
    const int nsets = nbatch >= 2 ? 2 : 1;
    const size_t set_bytes = solve_set_bytes(S, batch);
    // a voxel grid or boundary tables in host memory are staged in the workspace
    mcg_density den = *density;
    mcg_boundary bnd = *boundary;
    size_t grid_bytes = 0, faces_bytes = 0, zpack_bytes = 0, quad_bytes = 0;
    if (den.kind == MCG_RHO_VOXEL && den.grid && host_memory(den.grid))
        grid_bytes = (size_t)den.nx * (size_t)den.ny * (size_t)den.nz * sizeof(float);
    if (bnd.kind == MCG_G_TABLE && bnd.faces && host_memory(bnd.faces))
        faces_bytes = 6 * (size_t)bnd.nu * (size_t)bnd.nv * sizeof(float);
    // packed copies for the walk's 16-byte loads, unless the caller brought them
    if (den.kind == MCG_RHO_VOXEL && !den.zpack && P.hz_f <= 0.5f)
        zpack_bytes = mcg_voxel_pack_bytes(den.nx, den.ny, den.nz);
    if (bnd.kind == MCG_G_TABLE && !bnd.quads) quad_bytes = mcg_table_pack_bytes(bnd.nu, bnd.nv);
    const size_t bytes = solve_shared_bytes(S) + (size_t)nsets * set_bytes + align256(grid_bytes) +
                         align256(faces_bytes) + align256(zpack_bytes) + align256(quad_bytes);
    char* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MCG_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    cudaStream_t st = (cudaStream_t)opts.stream;
    const size_t s_ = (size_t)S, n_ = (size_t)S * (size_t)batch;
    char* q = ws;
    double* d_st = (double*)q;
    q += align256(s_ * 3 * sizeof(double));
    mcg_station_state* d_state = (mcg_station_state*)q;
    q += align256(s_ * sizeof(mcg_station_state));
    int32_t* d_status = (int32_t*)q;
    q += 256;
    double* d_res = (double*)q;
    q += align256(s_ * 6 * sizeof(double));
    struct BatchSet {
        double* u;
        double* d;
        int64_t* steps;
        unsigned long long* counter;
        void* work;
    } set[2] = {};
    for (int k = 0; k < nsets; ++k) {
        set[k].u = (double*)q;
        q += align256(n_ * sizeof(double));
        set[k].d = (double*)q;
        q += align256(n_ * sizeof(double));
        set[k].steps = (int64_t*)q;
        q += align256(n_ * sizeof(int64_t));
        set[k].counter = (unsigned long long*)q;
        q += 256;
        set[k].work = (void*)q;
        q += mcg_walk_work_bytes(S, batch, MCG_MIXED);
    }
    float* d_grid = grid_bytes ? (float*)q : nullptr;
    q += align256(grid_bytes);
    float* d_faces = faces_bytes ? (float*)q : nullptr;
    q += align256(faces_bytes);
    float* d_zpack = zpack_bytes ? (float*)q : nullptr;
    q += align256(zpack_bytes);
    float* d_quads = quad_bytes ? (float*)q : nullptr;

    double* h_res = new double[6 * s_];
    int32_t h_status = 0;
    rc = MCG_OK;
    do {
        if ((e = cudaMemcpyAsync(d_st, stations, s_ * 3 * sizeof(double), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemsetAsync(d_state, 0, s_ * sizeof(mcg_station_state), st)) ||
            (e = cudaMemsetAsync(d_status, 0, 256, st)) ||
            (grid_bytes && (e = cudaMemcpyAsync(d_grid, den.grid, grid_bytes, cudaMemcpyHostToDevice, st))) ||
            (faces_bytes && (e = cudaMemcpyAsync(d_faces, bnd.faces, faces_bytes, cudaMemcpyHostToDevice, st)))) {
            rc = cuda_fail(e, "workspace initialisation");
            break;
        }
        if (grid_bytes) den.grid = d_grid;
        if (faces_bytes) bnd.faces = d_faces;
        if (d_zpack) {
            if ((rc = voxel_pack(&den, d_zpack, st))) break;
            den.zpack = d_zpack;
        }
        if (d_quads) {
            if ((rc = table_pack(&bnd, d_quads, st))) break;
            bnd.quads = d_quads;
        }
        // The batches (counter and pool reset, walk, exit evaluation,
        // reduction), then the finalize.  With several batches, batch j runs
        // on stream j % 2 with buffer set j % 2, so one batch's exit-time
        // tail overlaps the next batch; each reduction waits for the one
        // before it, so the statistics merge in batch order.  With opts.graph
        // the whole sequence is captured once into a CUDA graph and launched
        // as one unit.
        const bool use_graph = opts.graph && nbatch >= 2;
        cudaStream_t run = st, run2 = nullptr;
        cudaEvent_t ev_fork = nullptr, ev_red = nullptr, ev_join = nullptr;
        if ((use_graph && (e = cudaStreamCreateWithFlags(&run, cudaStreamNonBlocking))) ||
            (nsets == 2 && (e = cudaStreamCreateWithFlags(&run2, cudaStreamNonBlocking))) ||
            (e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&ev_red, cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming)) ||
            (use_graph && (e = cudaStreamBeginCapture(run, cudaStreamCaptureModeThreadLocal)))) {
            rc = cuda_fail(e, "stream / event / capture set-up");
        }
        const bool capturing = use_graph && rc == MCG_OK;
        if (rc == MCG_OK && nsets == 2) {
            if ((e = cudaEventRecord(ev_fork, run)) || (e = cudaStreamWaitEvent(run2, ev_fork, 0)))
                rc = cuda_fail(e, "stream fork");
        }
        cudaStream_t qs[2] = {run, run2};
        mcg_options ro = opts;
        int64_t j = 0;
        for (int64_t p0 = 0; p0 < paths && rc == MCG_OK; p0 += batch, ++j) {
            const int64_t nb = (paths - p0) < batch ? (paths - p0) : batch;
            const int k = (int)(j % nsets);
            ro.stream = qs[k];
            rc = mcg_walk(domain, &den, &bnd, d_st, S, p0, nb, dt, seed, &ro, set[k].u, set[k].d,
                          set[k].steps, set[k].work, d_status, set[k].counter);
            if (rc == MCG_OK && j > 0 && (e = cudaStreamWaitEvent(qs[k], ev_red, 0)))
                rc = cuda_fail(e, "reduction order");
            if (rc == MCG_OK) rc = mcg_reduce(set[k].u, set[k].d, set[k].steps, S, nb, d_state, qs[k]);
            if (rc == MCG_OK && (e = cudaEventRecord(ev_red, qs[k]))) rc = cuda_fail(e, "reduction order");
        }
        if (nsets == 2 && (capturing || rc == MCG_OK)) {
            // join the second stream back (also required to end a capture)
            if ((e = cudaEventRecord(ev_join, run2)) || (e = cudaStreamWaitEvent(run, ev_join, 0)))
                if (rc == MCG_OK) rc = cuda_fail(e, "stream join");
        }
        if (rc == MCG_OK)
            rc = mcg_finalize(d_state, S, d_res, d_res + s_, d_res + 2 * s_, d_res + 3 * s_,
                              (int64_t*)(d_res + 4 * s_), (int64_t*)(d_res + 5 * s_), run);
        if (capturing) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t ge = cudaStreamEndCapture(run, &graph);
            if (rc == MCG_OK && ge == cudaSuccess) ge = cudaGraphInstantiate(&exec, graph, 0);
            if (rc == MCG_OK && ge == cudaSuccess) {
                // the graph runs after the initialisation already queued on st
                cudaEvent_t ready;
                ge = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
                if (ge == cudaSuccess) {
                    cudaEventRecord(ready, st);
                    cudaStreamWaitEvent(run, ready, 0);
                    ge = cudaGraphLaunch(exec, run);
                    cudaEventRecord(ready, run);
                    cudaStreamWaitEvent(st, ready, 0);
                    cudaEventDestroy(ready);
                }
            }
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (rc == MCG_OK && ge != cudaSuccess) rc = cuda_fail(ge, "graph launch");
        }
        // the call's own streams and events: their work is waited for below
        // (the result copy on st follows the join / the graph launch)
        if (use_graph && run != st) {
            cudaStreamSynchronize(run);
            cudaStreamDestroy(run);
        }
        if (run2) {
            cudaStreamSynchronize(run2);
            cudaStreamDestroy(run2);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_red) cudaEventDestroy(ev_red);
        if (ev_join) cudaEventDestroy(ev_join);
        if (rc) break;
        if ((e = cudaMemcpyAsync(h_res, d_res, 6 * s_ * sizeof(double), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(&h_status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            rc = cuda_fail(e, "result copy");
            break;
        }
        for (int64_t s = 0; s < S; ++s) {
            if (out->u) out->u[s] = h_res[s];
            if (out->gz) out->gz[s] = opts.crn_gz ? h_res[s_ + s] : NAN;
            if (out->se_u) out->se_u[s] = h_res[2 * s_ + s];
            if (out->se_gz) out->se_gz[s] = opts.crn_gz ? h_res[3 * s_ + s] : NAN;
            if (out->n_paths) std::memcpy(&out->n_paths[s], &h_res[4 * s_ + s], sizeof(int64_t));
            if (out->path_steps) std::memcpy(&out->path_steps[s], &h_res[5 * s_ + s], sizeof(int64_t));
        }
        rc = status_from_bits(h_status);
    } while (0);
    if (rc == MCG_ERR_CUDA) cudaStreamSynchronize(st);
    delete[] h_res;
    cudaFree(ws);
    return rc;
}

int mcg_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out, void* stream)
{
    if (n < 0) return set_error(MCG_ERR_ARG, "n must be non-negative");
    if (n == 0) return MCG_OK;
    if (!ctr || !key || !out) return set_error(MCG_ERR_ARG, "null device buffer");
    cudaError_t e = launch_philox(ctr, key, n, out, (cudaStream_t)stream);
    return e == cudaSuccess ? MCG_OK : cuda_fail(e, "philox kernel launch");
}

int mcg_normals(uint64_t seed, uint32_t s, uint32_t p, uint32_t b0, int64_t nblocks, int32_t precision, void* out,
                void* stream)
{
    if (nblocks < 0) return set_error(MCG_ERR_ARG, "nblocks must be non-negative");
    if (precision != MCG_FP64 && precision != MCG_MIXED) return set_error(MCG_ERR_ARG, "bad precision");
    if (nblocks == 0) return MCG_OK;
    if (!out) return set_error(MCG_ERR_ARG, "null output");
    cudaError_t e = launch_normals(seed, s, p, b0, nblocks, precision, out, (cudaStream_t)stream);
    return e == cudaSuccess ? MCG_OK : cuda_fail(e, "normals kernel launch");
}

int mcg_states_merge(const mcg_station_state* parts, int64_t R, int64_t S, mcg_station_state* out)
{
    if (R < 0 || S < 0) return set_error(MCG_ERR_ARG, "R and S must be non-negative");
    if (R == 0 || S == 0) return MCG_OK;
    if (!parts || !out) return set_error(MCG_ERR_ARG, "null states");
    for (int64_t s = 0; s < S; ++s) {
        mcg_station_state a;
        std::memset(&a, 0, sizeof(a));
        for (int64_t r = 0; r < R; ++r) {
            const mcg_station_state& b = parts[r * S + s];
            if (!(b.n > 0.0)) continue;
            if (a.n == 0.0) {
                a = b;
                continue;
            }
            const double n = a.n + b.n;
            const double du = b.mean_u - a.mean_u, dd = b.mean_d - a.mean_d;
            a.mean_u = a.mean_u + du * (b.n / n);
            a.m2_u = a.m2_u + b.m2_u + du * du * (a.n * b.n / n);
            a.mean_d = a.mean_d + dd * (b.n / n);
            a.m2_d = a.m2_d + b.m2_d + dd * dd * (a.n * b.n / n);
            a.steps = a.steps + b.steps;
            a.n = n;
        }
        out[s] = a;
    }
    return MCG_OK;
}

size_t mcg_grf_work_bytes(int64_t nx, int64_t ny, int64_t nz)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
    return (size_t)2 * (size_t)nx * (size_t)ny * (size_t)nz * sizeof(double) + 256;
}

int mcg_grf_density(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, double sigma_vox, double amp,
                    float* grid_out, void* work, void* stream)
{
    return grf_density(seed, nx, ny, nz, sigma_vox, amp, grid_out, (double*)work, (cudaStream_t)stream);
}

int mcg_boundary_tables(const mcg_domain* domain, const mcg_density* density, int32_t nu, int32_t nv,
                        double near_cells, float* faces_out, void* stream)
{
    return boundary_tables(domain, density, nu, nv, near_cells, faces_out, (cudaStream_t)stream);
}

size_t mcg_voxel_pack_bytes(int64_t nx, int64_t ny, int64_t nz)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
    return (size_t)16 * (size_t)nx * (size_t)ny * (size_t)(nz + 2);
}

int mcg_voxel_pack(const mcg_density* density, float* out, void* stream)
{
    return voxel_pack(density, out, (cudaStream_t)stream);
}

size_t mcg_table_pack_bytes(int32_t nu, int32_t nv)
{
    if (nu < 2 || nv < 2) return 0;
    return (size_t)16 * 6 * (size_t)(nu - 1) * (size_t)(nv - 1);
}

int mcg_table_pack(const mcg_boundary* boundary, float* out, void* stream)
{
    return table_pack(boundary, out, (cudaStream_t)stream);
}

int64_t mcg_walk_static_max_items(void) { return static_max_items(); }

int mcg_walk_static(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
                    const double* stations_dev, int64_t S, int64_t p0, int64_t N, double dt, uint64_t seed,
                    const mcg_options* opts, double* pp_u, double* pp_d, int64_t* pp_steps, int32_t* status_dev)
{
    WalkParams P;
    int rc = make_params(domain, density, boundary, dt, seed, opts, P);
    if (rc) return rc;
    if (S < 0 || N < 0 || p0 < 0) return set_error(MCG_ERR_ARG, "S, N and p0 must be non-negative");
    if (p0 + N > (int64_t)1 << 32) return set_error(MCG_ERR_ARG, "path indices must fit in 32 bits");
    if (S > (int64_t)1 << 32) return set_error(MCG_ERR_ARG, "station indices must fit in 32 bits");
    if (S == 0 || N == 0) return MCG_OK;
    const int64_t max_items = static_max_items();
    if (S > max_items / N)
        return set_error(MCG_ERR_ARG, "mcg_walk_static: S * N = %lld exceeds the fixed scratch limit of %lld paths",
                         (long long)S * (long long)N, (long long)max_items);
    if (!stations_dev || !pp_u || !pp_d || !pp_steps || !status_dev)
        return set_error(MCG_ERR_ARG, "null device buffer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char* base = nullptr;
    if ((rc = static_scratch(dev, &base))) return rc;
    const size_t n = (size_t)S * (size_t)N;
    P.stations = stations_dev;
    P.S = S;
    P.N = N;
    P.p0 = p0;
    P.total = (unsigned long long)n;
    P.pp_u = pp_u;
    P.pp_d = pp_d;
    P.pp_steps = pp_steps;
    P.status = status_dev;
    P.counter = (unsigned long long*)base;
    if (opts->precision == MCG_MIXED) {
        P.frec = (float*)(base + 256);
    }
    cudaStream_t st = (cudaStream_t)opts->stream;
    // the counter starts at zero and every item without its completion flag
    // (the step counts are cleared), so that an item that does not finish
    // (cancel) never reads the last call's records left in the shared array;
    // there is no migration pool here
    e = reset_walk(P, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(static scratch)");
    e = launch_walk(P, opts->precision, opts->block ? opts->block : 128, st);
    if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    return MCG_OK;
}

}  // extern "C"
