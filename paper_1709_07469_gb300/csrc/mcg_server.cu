// mcg_server.cu -- continuous batching of solve requests (host runtime).
//
// A scheduler thread admits queued requests while their device buffers fit
// the HBM budget, and advances every admitted request round by round: each
// round walks whole chunks of `chunk_paths` more paths of each of the
// request's stations (path indices continue where the last round stopped),
// reduces them into the request's station statistics, finalizes and copies
// u, g_z, standard errors and path counts into pinned host memory.
//
// Rounds are launched in batches on a pool of stream slots, one batch in
// flight per slot: the ready rounds of requests whose problems share every
// scalar (domain, density and boundary kinds, grid geometry, step, h) go
// into one walk launch -- a segment table gives each launch item its
// request's stations, path range, generator key, status word and model
// arrays -- followed by each request's own reduction.  The ready rounds are
// spread over the free slots, so several launches are in flight and one
// launch's exit-time tail runs beside the others.  When a batch has
// completed the thread decides on the host, request by request, whether the
// target is reached; if not, the request's next round joins a later batch.
// A request's numbers depend only on its own seed, stations and target:
// which batch a round runs in changes nothing.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "mcg_internal.h"
#include "mcgrav.h"

using namespace mcg;
using Clock = std::chrono::steady_clock;

namespace {

// Pinned host blocks reused across requests.  Allocating or freeing pinned
// memory is not stream-ordered (and a pageable host->device copy waits for
// its stream to drain), so a request never does either while others run:
// its host side (station staging, results, status word) comes from this
// pool, which grows on demand and frees its blocks when the last owner (the
// server or a request still held by the caller) lets go of it.
struct PinnedPool {
    std::mutex mu;
    std::multimap<size_t, void*> free_blocks;  // capacity -> block
    std::vector<void*> all;
    ~PinnedPool()
    {
        for (void* b : all) cudaFreeHost(b);
    }
    // A block of at least `bytes`; its capacity in *cap.  nullptr on failure.
    void* take(size_t bytes, size_t* cap)
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = free_blocks.lower_bound(bytes);
        if (it != free_blocks.end() && it->first <= 4 * bytes + 4096) {
            void* b = it->second;
            *cap = it->first;
            free_blocks.erase(it);
            return b;
        }
        size_t c = 4096;
        while (c < bytes) c *= 2;
        void* b = nullptr;
        if (cudaMallocHost(&b, c) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        all.push_back(b);
        *cap = c;
        return b;
    }
    void give(void* b, size_t cap)
    {
        std::lock_guard<std::mutex> lk(mu);
        free_blocks.emplace(cap, b);
    }
};

}  // namespace

struct mcg_model {
    mcg_domain dom;
    mcg_density den;
    mcg_boundary bnd;
    double dt = 0.0;
    double h = 0.0;
    float* grid = nullptr;   // owned device copy
    float* faces = nullptr;  // owned device copy
    float* zpack = nullptr;  // owned packed grid (mcg_voxel_pack)
    float* quads = nullptr;  // owned packed tables (mcg_table_pack)
};

struct mcg_request {
    mcg_server* server = nullptr;
    const mcg_model* model = nullptr;
    int64_t S = 0;
    double target = 0.0;
    uint64_t seed = 0;
    // scheduler-thread state
    WalkParams P;
    std::vector<unsigned char> compat;  // requests with equal keys may share a walk launch
    bool segable = false;               // its walk can run as a segment of a shared launch
    char* dev = nullptr;                // stations | states | status word | results
    size_t bytes = 0;
    int slot = -1;                      // slot of the last batch the request ran in
    int64_t round = 0;
    int64_t done_paths = 0;   // paths per station merged so far
    int64_t round_paths = 0;  // paths per station of the round planned / in flight
    bool in_flight = false;
    cudaEvent_t ev = nullptr;           // admission copies done
    double* h_res = nullptr;  // pinned: 6 S doubles + status word + 3 S station coordinates
    size_t h_cap = 0;         // capacity of the pinned block behind h_res
    std::shared_ptr<PinnedPool> pinned;
    // published state
    std::mutex mu;
    std::condition_variable cv;
    bool done = false;
    int status = MCG_OK;
    std::string message;
    std::vector<double> res;  // 6 S: u, gz, se_u, se_gz, n (int64 bits), steps (int64 bits)
    std::atomic<int64_t> paths{0};
    std::atomic<int64_t> rounds{0};
    std::atomic<bool> cancel{false};
    Clock::time_point t_submit, t_done;
};

// One stream with at most one batch of rounds in flight.
struct ServerSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    mcg::WalkSeg* h_seg = nullptr;  // pinned: the batch's segment table, then its status word
    std::vector<mcg_request*> reqs;
    char* dev = nullptr;            // the batch's per-path buffers, walk scratch, table
    size_t bytes = 0;
    bool busy = false;
    // instantiated graphs of this slot's batches, by the batch's request count
    // (the topology: one walk, then per request reduce, finalize, copies)
    std::map<size_t, cudaGraphExec_t> exec;
};

struct mcg_server {
    mcg_server_config cfg;
    int device = 0;
    std::vector<ServerSlot> slots;
    cudaStream_t admit_st = nullptr;  // admission copies
    std::mutex mu;
    std::condition_variable cv;
    std::deque<mcg_request*> pending;
    bool stopping = false;
    std::vector<mcg_request*> active;
    size_t used = 0;
    std::shared_ptr<PinnedPool> pinned = std::make_shared<PinnedPool>();
    cudaMemPool_t pool = nullptr;  // the server's own stream-ordered device pool
    std::thread th;
    std::atomic<int64_t> n_launches{0}, n_rounds{0};  // walk launches, request rounds in them
};

namespace {

constexpr int kMaxSeg = 64;                         // requests in one walk launch at most
constexpr unsigned long long kMinBatchItems = 1ull << 18;  // smaller batches do not fill the GPU

// Device layout of a request: stations | states | status word | results.
struct ReqLayout {
    size_t st, states, status, res, total;
};

ReqLayout req_layout(int64_t S)
{
    ReqLayout L;
    const size_t s = (size_t)S;
    size_t o = 0;
    L.st = o;
    o += align256(s * 3 * sizeof(double));
    L.states = o;
    o += align256(s * sizeof(mcg_station_state));
    L.status = o;
    o += 256;
    L.res = o;
    o += align256(s * 6 * sizeof(double));
    L.total = o;
    return L;
}

// Device layout of a batch of n items: per-path u, d, steps | work counter +
// batch status word | segment table | walk scratch.
struct BatchLayout {
    size_t u, d, steps, ctr, seg, work, total;
};

BatchLayout batch_layout(size_t n, int precision)
{
    BatchLayout L;
    size_t o = 0;
    L.u = o;
    o += align256(n * sizeof(double));
    L.d = o;
    o += align256(n * sizeof(double));
    L.steps = o;
    o += align256(n * sizeof(int64_t));
    L.ctr = o;
    o += 256;
    L.seg = o;
    o += align256(kMaxSeg * sizeof(WalkSeg));
    L.work = o;
    o += mcg_walk_work_bytes(1, (int64_t)n, precision);
    L.total = o;
    return L;
}

// The problem scalars of a request with its own data (stations, key, model
// arrays, status) masked out: requests with equal keys can share a walk
// launch (the launch takes its scalars from any of them).
std::vector<unsigned char> compat_key(const WalkParams& P0)
{
    WalkParams P = P0;  // make_params zeroed every byte first, padding included
    P.key0 = P.key1 = 0;
    P.grid = nullptr;
    P.zq = P.zq ? (const float4*)16 : nullptr;  // packed or not selects the kernel
    P.faces = nullptr;
    P.tq = P.tq ? (const float4*)16 : nullptr;
    const unsigned char* b = (const unsigned char*)&P;
    return std::vector<unsigned char>(b, b + sizeof(P));
}

void finish(mcg_request* r, int status, const char* msg)
{
    std::lock_guard<std::mutex> lk(r->mu);
    if (r->h_res) r->res.assign(r->h_res, r->h_res + 6 * r->S);
    r->status = status;
    if (msg) r->message = msg;
    r->t_done = Clock::now();
    r->done = true;
    r->cv.notify_all();
}

// Paths per station of the request's next round: min_paths (in whole
// chunks) first, then the chunks the request's own spread says it still needs
// (90 % of the estimate, at least one chunk, at most max_round_paths), never
// past max_paths.  Depends only on the request's own results.
int64_t next_round_paths(const mcg_server* sv, const mcg_request* r)
{
    const int64_t chunk = sv->cfg.chunk_paths;
    int64_t m = 1;
    if (r->done_paths < sv->cfg.min_paths) {
        // the first round takes the request straight to min_paths
        m = (sv->cfg.min_paths - r->done_paths + chunk - 1) / chunk;
        const int64_t mmax = sv->cfg.max_round_paths / chunk;
        if (m > mmax) m = mmax;
    } else {
        double need = 0.0;
        for (int64_t s = 0; s < r->S; ++s) {
            const double u = r->h_res[s], se = r->h_res[2 * r->S + s];
            const double sd = se * std::sqrt((double)r->done_paths);
            const double n_s = (sd / (r->target * std::fabs(u))) * (sd / (r->target * std::fabs(u)));
            if (std::isfinite(n_s) && n_s > need) need = n_s;
        }
        const double rest = 0.9 * (need - (double)r->done_paths);
        if (rest > (double)chunk) m = (int64_t)std::ceil(rest / (double)chunk);
        const int64_t mmax = sv->cfg.max_round_paths / chunk;
        if (m > mmax) m = mmax;
    }
    int64_t n = m * chunk;
    if (r->done_paths + n > sv->cfg.max_paths) n = sv->cfg.max_paths - r->done_paths;
    return n > 0 ? n : chunk;
}

// Launches a captured batch through the slot's instantiated graph for that
// request count: updated in place when the topology matches (the usual case),
// instantiated afresh otherwise.
cudaError_t launch_slot_graph(ServerSlot& sl, size_t nreq, cudaGraph_t g, cudaStream_t st)
{
    auto it = sl.exec.find(nreq);
    if (it != sl.exec.end()) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(it->second, g, &info) == cudaSuccess) return cudaGraphLaunch(it->second, st);
        cudaGetLastError();
        cudaGraphExecDestroy(it->second);
        sl.exec.erase(it);
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) return e;
    sl.exec[nreq] = ex;
    return cudaGraphLaunch(ex, st);
}

// Launches one batch of rounds (each request's round_paths already planned)
// on slot `k`: one walk over all their items, then per request its reduction,
// finalize and result copies, then the slot's event.  A batch of one request
// is a plain launch of that request's problem.  Returns MCG_ERR_OOM when the
// batch's buffers do not fit now (nothing launched).
int launch_batch(mcg_server* sv, int k, const std::vector<mcg_request*>& reqs)
{
    ServerSlot& sl = sv->slots[k];
    cudaStream_t st = sl.st;
    const int prec = sv->cfg.walk.precision;
    std::vector<unsigned long long> begin(reqs.size());
    unsigned long long T = 0;
    for (size_t i = 0; i < reqs.size(); ++i) {
        begin[i] = T;
        T += (unsigned long long)reqs[i]->S * (unsigned long long)reqs[i]->round_paths;
    }
    const BatchLayout L = batch_layout((size_t)T, prec);
    cudaError_t e = cudaMallocFromPoolAsync((void**)&sl.dev, L.total, sv->pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sl.dev = nullptr;
        return MCG_ERR_OOM;
    }
    sl.bytes = L.total;
    WalkParams P = reqs[0]->P;
    P.total = T;
    P.pp_u = (double*)(sl.dev + L.u);
    P.pp_d = (double*)(sl.dev + L.d);
    P.pp_steps = (int64_t*)(sl.dev + L.steps);
    P.counter = (unsigned long long*)(sl.dev + L.ctr);
    int32_t* bstatus = (int32_t*)(sl.dev + L.ctr + 128);
    if (prec == MCG_MIXED) bind_work(P, sl.dev + L.work, sv->cfg.walk.migrate != 0);
    int32_t* h_bstatus = (int32_t*)(sl.h_seg + kMaxSeg);
    *h_bstatus = 0;
    const ReqLayout R0 = req_layout(reqs[0]->S);
    if (reqs.size() == 1) {  // the request's own problem, as a plain launch
        mcg_request* r = reqs[0];
        P.stations = (const double*)(r->dev + R0.st);
        P.S = r->S;
        P.N = r->round_paths;
        P.p0 = r->done_paths;
        P.status = (int32_t*)(r->dev + R0.status);
    } else {
        for (size_t i = 0; i < reqs.size(); ++i) {
            const mcg_request* r = reqs[i];
            const ReqLayout RL = req_layout(r->S);
            WalkSeg& g = sl.h_seg[i];
            g.begin = begin[i];
            g.stations = (const double*)(r->dev + RL.st);
            g.N = r->round_paths;
            g.p0 = r->done_paths;
            g.status = (int32_t*)(r->dev + RL.status);
            g.grid = r->P.grid;
            g.zq = r->P.zq;
            g.faces = r->P.faces;
            g.tq = r->P.tq;
            g.key0 = r->P.key0;
            g.key1 = r->P.key1;
        }
        P.stations = nullptr;
        P.S = 0;
        P.N = 1;
        P.p0 = 0;
        P.status = bstatus;  // what no single request can be blamed for (a lost walk)
        P.seg = (const WalkSeg*)(sl.dev + L.seg);
        P.nseg = (int32_t)reqs.size();
    }
    for (mcg_request* r : reqs)  // the first round waits for the admission copies
        if (r->round == 0 && (e = cudaStreamWaitEvent(st, r->ev, 0)))
            return set_error(MCG_ERR_CUDA, "admission order: %s", cudaGetErrorString(e));
    // The batch's work on the slot's stream: segment table, walk, then per
    // request its reduction, finalize and result copies.  With walk.graph the
    // sequence is captured and launched as one CUDA graph (the slot keeps one
    // instantiated graph per request count and updates it in place).
    auto issue = [&]() -> int {
        if (P.seg &&
            (e = cudaMemcpyAsync(sl.dev + L.seg, sl.h_seg, reqs.size() * sizeof(WalkSeg), cudaMemcpyHostToDevice, st)))
            return set_error(MCG_ERR_CUDA, "segment table: %s", cudaGetErrorString(e));
        if ((e = cudaMemsetAsync(bstatus, 0, sizeof(int32_t), st)) || (e = reset_walk(P, st)) ||
            (e = launch_walk(P, prec, sv->cfg.walk.block ? sv->cfg.walk.block : 128, st)))
            return set_error(MCG_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
        for (size_t i = 0; i < reqs.size(); ++i) {
            mcg_request* r = reqs[i];
            const ReqLayout RL = req_layout(r->S);
            mcg_station_state* states = (mcg_station_state*)(r->dev + RL.states);
            double* res = (double*)(r->dev + RL.res);
            if ((e = launch_reduce(P.pp_u + begin[i], P.pp_d + begin[i], P.pp_steps + begin[i], r->S,
                                   r->round_paths, states, st)) ||
                (e = launch_finalize(states, r->S, res, res + r->S, res + 2 * r->S, res + 3 * r->S,
                                     (int64_t*)(res + 4 * r->S), (int64_t*)(res + 5 * r->S), st)) ||
                (e = cudaMemcpyAsync(r->h_res, res, 6 * r->S * sizeof(double), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaMemcpyAsync(r->h_res + 6 * r->S, r->dev + RL.status, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, st)))
                return set_error(MCG_ERR_CUDA, "round reduction: %s", cudaGetErrorString(e));
        }
        if ((e = cudaMemcpyAsync(h_bstatus, bstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, st)))
            return set_error(MCG_ERR_CUDA, "batch status: %s", cudaGetErrorString(e));
        return MCG_OK;
    };
    int rc = MCG_OK;
    if (sv->cfg.walk.graph) {
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)))
            return set_error(MCG_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
        rc = issue();
        cudaGraph_t g = nullptr;
        cudaError_t ge = cudaStreamEndCapture(st, &g);
        if (rc == MCG_OK && ge == cudaSuccess) ge = launch_slot_graph(sl, reqs.size(), g, st);
        if (g) cudaGraphDestroy(g);
        if (rc == MCG_OK && ge != cudaSuccess) rc = set_error(MCG_ERR_CUDA, "batch graph: %s", cudaGetErrorString(ge));
    } else {
        rc = issue();
    }
    if (rc != MCG_OK) return rc;
    if ((e = cudaEventRecord(sl.ev, st)))
        return set_error(MCG_ERR_CUDA, "batch event: %s", cudaGetErrorString(e));
    for (mcg_request* r : reqs) {
        r->in_flight = true;
        r->slot = k;
    }
    sl.reqs = reqs;
    sl.busy = true;
    sv->used += sl.bytes;
    sv->n_launches.fetch_add(1);
    sv->n_rounds.fetch_add((int64_t)reqs.size());
    return MCG_OK;
}

int admit(mcg_server* sv, mcg_request* r)
{
    cudaStream_t st = sv->admit_st;
    const ReqLayout L = req_layout(r->S);
    cudaError_t e = cudaMallocFromPoolAsync((void**)&r->dev, L.total, sv->pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        r->dev = nullptr;
        return MCG_ERR_OOM;
    }
    r->bytes = L.total;
    // from the pinned staging copy: a pageable source would make this call
    // wait until the stream has drained
    if ((e = cudaMemcpyAsync(r->dev + L.st, r->h_res + 6 * r->S + 1, r->S * 3 * sizeof(double),
                             cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemsetAsync(r->dev + L.states, 0, r->S * sizeof(mcg_station_state), st)) ||
        (e = cudaMemsetAsync(r->dev + L.status, 0, 256, st)) || (e = cudaEventRecord(r->ev, st))) {
        cudaFreeAsync(r->dev, st);
        r->dev = nullptr;
        return MCG_ERR_CUDA;
    }
    sv->used += L.total;
    return MCG_OK;
}

void release(mcg_server* sv, mcg_request* r)
{
    if (r->dev) {
        // after the last batch that used it (or the admission copies)
        cudaFreeAsync(r->dev, r->slot >= 0 ? sv->slots[r->slot].st : sv->admit_st);
        r->dev = nullptr;
        sv->used -= r->bytes;
    }
}

// The request reached its end after the round whose results are in h_res?
bool reached(const mcg_server* sv, const mcg_request* r, int64_t n)
{
    if (n >= sv->cfg.max_paths) return true;
    if (n < sv->cfg.min_paths) return false;
    for (int64_t s = 0; s < r->S; ++s) {
        const double u = r->h_res[s], se = r->h_res[2 * r->S + s];
        if (!(se <= r->target * std::fabs(u))) return false;
    }
    return true;
}

void retire(mcg_server* sv, mcg_request* r)
{
    std::lock_guard<std::mutex> lk(sv->mu);
    for (size_t i = 0; i < sv->active.size(); ++i)
        if (sv->active[i] == r) {
            sv->active.erase(sv->active.begin() + i);
            break;
        }
}

// A batch has completed (q: its event's status): every request in it either
// ends (target, cap, cancel, error) or becomes ready for its next round.
// After finish() the caller may free a request at any moment: nothing here
// touches it again once it has been finished.
void complete_batch(mcg_server* sv, ServerSlot& sl, cudaError_t q)
{
    const int32_t bbits = *(const int32_t*)(sl.h_seg + kMaxSeg);
    for (mcg_request* r : sl.reqs) {
        r->in_flight = false;
        int end = -1;  // status that ends the request, -1: continue
        const char* msg = nullptr;
        if (q != cudaSuccess) {
            end = MCG_ERR_CUDA;
            msg = cudaGetErrorString(q);
        } else {
            r->round++;
            r->rounds.store(r->round);
            r->done_paths += r->round_paths;
            int64_t n = 0;
            std::memcpy(&n, r->h_res + 4 * r->S, sizeof(int64_t));
            r->paths.store(n);
            int32_t bits = 0;
            std::memcpy(&bits, r->h_res + 6 * r->S, sizeof(int32_t));
            bits |= bbits;
            if (bits) {
                end = status_from_bits(bits);  // never MCG_OK for a nonzero word
                msg = "walk status";
            } else if (r->cancel.load()) {
                end = MCG_ERR_CANCELLED;
                msg = "cancelled";
            } else if (reached(sv, r, n)) {
                end = MCG_OK;
            }
        }
        if (end >= 0) {
            release(sv, r);
            retire(sv, r);
            finish(r, end, msg);
        }
    }
    cudaFreeAsync(sl.dev, sl.st);
    sl.dev = nullptr;
    sv->used -= sl.bytes;
    sl.bytes = 0;
    sl.reqs.clear();
    sl.busy = false;
}

// Forms batches of the ready rounds for the free slots: the planned items of
// all ready rounds are spread evenly over the free slots (at least
// kMinBatchItems, at most cfg.batch_items per batch, one request at least),
// each batch holding requests of one compatibility key in admission order.
bool form_batches(mcg_server* sv, std::vector<mcg_request*>& ready)
{
    std::vector<int> free_slots;
    for (int k = 0; k < (int)sv->slots.size(); ++k)
        if (!sv->slots[k].busy) free_slots.push_back(k);
    if (ready.empty() || free_slots.empty()) return false;
    unsigned long long total = 0;
    for (mcg_request* r : ready) {
        r->round_paths = next_round_paths(sv, r);
        total += (unsigned long long)r->S * (unsigned long long)r->round_paths;
    }
    unsigned long long per = (total + free_slots.size() - 1) / free_slots.size();
    const unsigned long long cap = sv->cfg.batch ? (unsigned long long)sv->cfg.batch_items : 0ull;
    if (per < kMinBatchItems) per = kMinBatchItems;
    if (per > cap) per = cap;
    bool progressed = false;
    size_t f = 0;
    while (!ready.empty() && f < free_slots.size()) {
        mcg_request* r0 = ready.front();
        std::vector<mcg_request*> batch{r0};
        unsigned long long items = (unsigned long long)r0->S * (unsigned long long)r0->round_paths;
        std::vector<mcg_request*> rest;
        for (size_t i = 1; i < ready.size(); ++i) {
            mcg_request* r = ready[i];
            const unsigned long long n = (unsigned long long)r->S * (unsigned long long)r->round_paths;
            if (sv->cfg.batch && r0->segable && r->segable && batch.size() < (size_t)kMaxSeg && items < per &&
                items + n <= cap && r->compat == r0->compat) {
                batch.push_back(r);
                items += n;
            } else {
                rest.push_back(r);
            }
        }
        // the batch's buffers must fit the budget unless nothing else is in flight
        bool any_busy = false;
        for (const ServerSlot& sl : sv->slots) any_busy = any_busy || sl.busy;
        if (any_busy && sv->used + batch_layout((size_t)items, sv->cfg.walk.precision).total >
                            (size_t)sv->cfg.hbm_budget)
            break;
        const int rc = launch_batch(sv, free_slots[f], batch);
        if (rc == MCG_ERR_OOM && any_busy) break;  // retry when a batch frees its buffers
        if (rc != MCG_OK) {
            for (mcg_request* r : batch) {
                release(sv, r);
                retire(sv, r);
                finish(r, rc == MCG_ERR_OOM ? MCG_ERR_OOM : MCG_ERR_CUDA, "round launch failed");
            }
        } else {
            ++f;
        }
        progressed = true;
        ready.swap(rest);
    }
    return progressed;
}

void scheduler(mcg_server* sv)
{
    cudaSetDevice(sv->device);
    for (;;) {
        bool progressed = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->stopping && sv->pending.empty() && sv->active.empty()) break;
            // admission: FIFO, while the budget and the slot count allow
            while (!sv->pending.empty() && (int)sv->active.size() < sv->cfg.max_active) {
                mcg_request* r = sv->pending.front();
                const size_t need = req_layout(r->S).total;
                if (!sv->active.empty() && sv->used + need > (size_t)sv->cfg.hbm_budget) break;
                sv->pending.pop_front();
                lk.unlock();
                const int rc = admit(sv, r);
                lk.lock();
                if (rc == MCG_OK) {
                    sv->active.push_back(r);
                } else if (rc == MCG_ERR_OOM && !sv->active.empty()) {
                    sv->pending.push_front(r);  // retry when memory frees up
                    break;
                } else {
                    finish(r, rc, "admission failed");
                }
                progressed = true;
            }
        }
        // completed batches
        for (ServerSlot& sl : sv->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            complete_batch(sv, sl, q);
            progressed = true;
        }
        // the ready rounds: admitted requests not in flight; a cancelled one
        // ends here once it has results of at least one round
        std::vector<mcg_request*> act, ready;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            act = sv->active;
        }
        for (mcg_request* r : act) {
            if (r->in_flight) continue;
            if (r->cancel.load() && r->round > 0) {
                release(sv, r);
                retire(sv, r);
                finish(r, MCG_ERR_CANCELLED, "cancelled");
                progressed = true;
                continue;
            }
            ready.push_back(r);
        }
        if (form_batches(sv, ready)) progressed = true;
        if (!progressed) {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace

extern "C" {

void mcg_server_config_default(mcg_server_config* c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->streams = 8;
    c->max_active = 64;
    c->hbm_budget = (int64_t)8 << 30;
    c->chunk_paths = 4096;
    c->min_paths = 2 * 4096;
    c->max_paths = 10000000;
    c->max_round_paths = 16 * 4096;
    mcg_options_default(&c->walk);
    c->batch = 1;
    c->batch_items = (int64_t)1 << 22;
}

int mcg_model_create(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary, double dt,
                     double h, mcg_model** out)
{
    if (!out) return set_error(MCG_ERR_ARG, "null output");
    *out = nullptr;
    mcg_options o;
    mcg_options_default(&o);
    o.h = h;
    WalkParams P;
    int rc = make_params(domain, density, boundary, dt, 0, &o, P);
    if (rc) return rc;
    mcg_model* m = new mcg_model();
    m->dom = *domain;
    m->den = *density;
    m->bnd = *boundary;
    m->dt = dt;
    m->h = h;
    m->den.zpack = nullptr;  // the model never keeps a caller's array: it packs its own copy
    m->bnd.quads = nullptr;
    cudaError_t e = cudaSuccess;
    if (density->kind == MCG_RHO_VOXEL) {
        const size_t n = (size_t)density->nx * density->ny * density->nz;
        if ((e = cudaMalloc(&m->grid, n * sizeof(float))) ||
            (e = cudaMemcpy(m->grid, density->grid, n * sizeof(float), cudaMemcpyDefault))) {
            mcg_model_destroy(m);
            return set_error(e == cudaErrorMemoryAllocation ? MCG_ERR_OOM : MCG_ERR_CUDA, "model grid: %s",
                             cudaGetErrorString(e));
        }
        m->den.grid = m->grid;
    }
    if (boundary->kind == MCG_G_TABLE) {
        const size_t n = (size_t)6 * boundary->nu * boundary->nv;
        if ((e = cudaMalloc(&m->faces, n * sizeof(float))) ||
            (e = cudaMemcpy(m->faces, boundary->faces, n * sizeof(float), cudaMemcpyDefault))) {
            mcg_model_destroy(m);
            return set_error(e == cudaErrorMemoryAllocation ? MCG_ERR_OOM : MCG_ERR_CUDA, "model faces: %s",
                             cudaGetErrorString(e));
        }
        m->bnd.faces = m->faces;
    }
    // packed copies for the walk's 16-byte loads (the grid one only while the
    // copies' layers stay within one cell of each other: h <= spacing_z / 2)
    if (density->kind == MCG_RHO_VOXEL && P.hz_f <= 0.5f) {
        const size_t b = mcg_voxel_pack_bytes(density->nx, density->ny, density->nz);
        if ((e = cudaMalloc(&m->zpack, b))) {
            mcg_model_destroy(m);
            return set_error(e == cudaErrorMemoryAllocation ? MCG_ERR_OOM : MCG_ERR_CUDA, "model zpack: %s",
                             cudaGetErrorString(e));
        }
        if ((rc = voxel_pack(&m->den, m->zpack, 0))) {
            mcg_model_destroy(m);
            return rc;
        }
        m->den.zpack = m->zpack;
    }
    if (boundary->kind == MCG_G_TABLE) {
        const size_t b = mcg_table_pack_bytes(boundary->nu, boundary->nv);
        if ((e = cudaMalloc(&m->quads, b))) {
            mcg_model_destroy(m);
            return set_error(e == cudaErrorMemoryAllocation ? MCG_ERR_OOM : MCG_ERR_CUDA, "model quads: %s",
                             cudaGetErrorString(e));
        }
        if ((rc = table_pack(&m->bnd, m->quads, 0))) {
            mcg_model_destroy(m);
            return rc;
        }
        m->bnd.quads = m->quads;
    }
    if ((e = cudaStreamSynchronize(0))) {
        mcg_model_destroy(m);
        return set_error(MCG_ERR_CUDA, "model set-up: %s", cudaGetErrorString(e));
    }
    *out = m;
    return MCG_OK;
}

int mcg_model_destroy(mcg_model* m)
{
    if (!m) return MCG_OK;
    if (m->grid) cudaFree(m->grid);
    if (m->faces) cudaFree(m->faces);
    if (m->zpack) cudaFree(m->zpack);
    if (m->quads) cudaFree(m->quads);
    delete m;
    return MCG_OK;
}

int mcg_server_create(const mcg_server_config* cfg_in, mcg_server** out)
{
    if (!out) return set_error(MCG_ERR_ARG, "null output");
    *out = nullptr;
    mcg_server_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else mcg_server_config_default(&cfg);
    if (cfg.streams <= 0 || cfg.streams > 64) return set_error(MCG_ERR_ARG, "streams must be in [1, 64]");
    if (cfg.max_active <= 0) return set_error(MCG_ERR_ARG, "max_active must be positive");
    if (cfg.chunk_paths <= 0 || cfg.max_paths < cfg.chunk_paths || cfg.hbm_budget <= 0)
        return set_error(MCG_ERR_ARG, "need chunk_paths > 0, max_paths >= chunk_paths, hbm_budget > 0");
    if (cfg.max_round_paths < cfg.chunk_paths) cfg.max_round_paths = cfg.chunk_paths;
    cfg.max_round_paths -= cfg.max_round_paths % cfg.chunk_paths;
    if (cfg.walk.precision != MCG_FP64 && cfg.walk.precision != MCG_MIXED)
        return set_error(MCG_ERR_ARG, "walk.precision must be MCG_FP64 or MCG_MIXED");
    if (cfg.batch != 0 && cfg.batch != 1) return set_error(MCG_ERR_ARG, "batch must be 0 or 1");
    if (cfg.batch && cfg.batch_items <= 0) return set_error(MCG_ERR_ARG, "batch_items must be positive");
    mcg_server* sv = new mcg_server();
    sv->cfg = cfg;
    cudaGetDevice(&sv->device);
    // Request buffers come from a device pool of the server's own: freed
    // buffers stay cached (up to the budget) instead of going back to the
    // driver after every request, and a buffer freed on one stream is reused
    // on another only once that free has completed -- the pool never makes
    // one stream wait for another (no internal dependencies).  The process's
    // default pool is left as it was.
    {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = sv->device;
        const cudaError_t e = cudaMemPoolCreate(&sv->pool, &props);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete sv;
            return set_error(MCG_ERR_CUDA, "cudaMemPoolCreate: %s", cudaGetErrorString(e));
        }
        uint64_t thr = (uint64_t)cfg.hbm_budget;
        cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &thr);
        int off = 0;
        cudaMemPoolSetAttribute(sv->pool, cudaMemPoolReuseAllowInternalDependencies, &off);
    }
    // the stream slots (each with its pinned segment table and status word)
    // and the admission stream
    cudaError_t e = cudaStreamCreateWithFlags(&sv->admit_st, cudaStreamNonBlocking);
    sv->slots.resize(cfg.streams);
    for (int i = 0; i < cfg.streams && e == cudaSuccess; ++i) {
        ServerSlot& sl = sv->slots[i];
        if ((e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking)) ||
            (e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) ||
            (e = cudaMallocHost((void**)&sl.h_seg, kMaxSeg * sizeof(WalkSeg) + 256)))
            break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (ServerSlot& sl : sv->slots) {
            if (sl.st) cudaStreamDestroy(sl.st);
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.h_seg) cudaFreeHost(sl.h_seg);
        }
        if (sv->admit_st) cudaStreamDestroy(sv->admit_st);
        cudaMemPoolDestroy(sv->pool);
        delete sv;
        return set_error(MCG_ERR_CUDA, "server streams: %s", cudaGetErrorString(e));
    }
    sv->th = std::thread(scheduler, sv);
    *out = sv;
    return MCG_OK;
}

int mcg_server_destroy(mcg_server* sv)
{
    if (!sv) return MCG_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv.notify_all();
    sv->th.join();
    for (ServerSlot& sl : sv->slots) {
        cudaStreamSynchronize(sl.st);
        for (auto& x : sl.exec) cudaGraphExecDestroy(x.second);
        cudaStreamDestroy(sl.st);
        cudaEventDestroy(sl.ev);
        cudaFreeHost(sl.h_seg);
    }
    cudaStreamSynchronize(sv->admit_st);
    cudaStreamDestroy(sv->admit_st);
    cudaMemPoolDestroy(sv->pool);
    delete sv;
    return MCG_OK;
}

int mcg_submit(mcg_server* sv, const mcg_model* m, const double* stations, int64_t S, double target_rel_se,
               uint64_t seed, mcg_request** out)
{
    if (!sv || !m || !out) return set_error(MCG_ERR_ARG, "null server/model/output");
    *out = nullptr;
    if (S <= 0 || !stations) return set_error(MCG_ERR_ARG, "need S >= 1 stations");
    if (S > (int64_t)1 << 32) return set_error(MCG_ERR_ARG, "too many stations");
    if (!(target_rel_se > 0.0)) return set_error(MCG_ERR_ARG, "target_rel_se must be positive");
    mcg_request* r = new mcg_request();
    mcg_options o = sv->cfg.walk;
    o.h = m->h;
    int rc = make_params(&m->dom, &m->den, &m->bnd, m->dt, seed, &o, r->P);
    for (int64_t s = 0; rc == MCG_OK && s < S; ++s) rc = check_station(r->P, stations + 3 * s, s);
    if (rc) {
        delete r;
        return rc;
    }
    r->compat = compat_key(r->P);
    r->segable = !r->P.ball && !r->P.bridge;
    r->server = sv;
    r->model = m;
    r->S = S;
    r->target = target_rel_se;
    r->seed = seed;
    cudaError_t e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
    const size_t hbytes = (9 * (size_t)S + 1) * sizeof(double);
    if (e == cudaSuccess) {
        r->pinned = sv->pinned;
        r->h_res = (double*)r->pinned->take(hbytes, &r->h_cap);
        if (!r->h_res) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        if (r->ev) cudaEventDestroy(r->ev);
        delete r;
        return set_error(MCG_ERR_CUDA, "request set-up: %s", cudaGetErrorString(e));
    }
    std::memset(r->h_res, 0, (6 * S + 1) * sizeof(double));
    std::memcpy(r->h_res + 6 * S + 1, stations, 3 * (size_t)S * sizeof(double));
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) {
            r->pinned->give(r->h_res, r->h_cap);
            cudaEventDestroy(r->ev);
            delete r;
            return set_error(MCG_ERR_ARG, "server is stopping");
        }
        sv->pending.push_back(r);
    }
    sv->cv.notify_all();
    *out = r;
    return MCG_OK;
}

static void copy_result(const mcg_request* r, mcg_result* out)
{
    if (!out) return;
    const int64_t S = r->S;
    for (int64_t s = 0; s < S; ++s) {
        if (out->u) out->u[s] = r->res[s];
        if (out->gz) out->gz[s] = r->res[S + s];
        if (out->se_u) out->se_u[s] = r->res[2 * S + s];
        if (out->se_gz) out->se_gz[s] = r->res[3 * S + s];
        if (out->n_paths) std::memcpy(&out->n_paths[s], &r->res[4 * S + s], sizeof(int64_t));
        if (out->path_steps) std::memcpy(&out->path_steps[s], &r->res[5 * S + s], sizeof(int64_t));
    }
}

int mcg_poll(mcg_request* r, mcg_result* out, int* done)
{
    if (!r || !done) return set_error(MCG_ERR_ARG, "null request/done");
    std::lock_guard<std::mutex> lk(r->mu);
    *done = r->done ? 1 : 0;
    if (!r->done) return MCG_OK;
    copy_result(r, out);
    if (r->status) set_error(r->status, "%s", r->message.c_str());
    return r->status;
}

int mcg_wait(mcg_request* r, mcg_result* out, int64_t timeout_ms)
{
    if (!r) return set_error(MCG_ERR_ARG, "null request");
    std::unique_lock<std::mutex> lk(r->mu);
    if (timeout_ms < 0) r->cv.wait(lk, [&] { return r->done; });
    else if (!r->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
        return set_error(MCG_ERR_TIMEOUT, "request not finished within %lld ms", (long long)timeout_ms);
    copy_result(r, out);
    if (r->status) set_error(r->status, "%s", r->message.c_str());
    return r->status;
}

int mcg_cancel(mcg_request* r)
{
    if (!r) return set_error(MCG_ERR_ARG, "null request");
    r->cancel.store(true);
    if (r->server) r->server->cv.notify_all();
    return MCG_OK;
}

int mcg_request_info(const mcg_request* r, int64_t* paths, int64_t* rounds, double* seconds)
{
    if (!r) return set_error(MCG_ERR_ARG, "null request");
    if (paths) *paths = r->paths.load();
    if (rounds) *rounds = r->rounds.load();
    if (seconds) {
        mcg_request* rr = const_cast<mcg_request*>(r);
        std::lock_guard<std::mutex> lk(rr->mu);
        const Clock::time_point t = r->done ? r->t_done : Clock::now();
        *seconds = std::chrono::duration<double>(t - r->t_submit).count();
    }
    return MCG_OK;
}

int mcg_server_stats(const mcg_server* s, int64_t* launches, int64_t* rounds)
{
    if (!s) return set_error(MCG_ERR_ARG, "null server");
    if (launches) *launches = s->n_launches.load();
    if (rounds) *rounds = s->n_rounds.load();
    return MCG_OK;
}

int mcg_request_free(mcg_request* r)
{
    if (!r) return MCG_OK;
    {
        std::unique_lock<std::mutex> lk(r->mu);
        if (!r->done) return set_error(MCG_ERR_ARG, "request still running (cancel and wait first)");
    }
    if (r->h_res) r->pinned->give(r->h_res, r->h_cap);
    if (r->ev) cudaEventDestroy(r->ev);
    delete r;
    return MCG_OK;
}

}  // extern "C"
