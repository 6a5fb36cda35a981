// Request server: continuous batching of whole reconstructions on one GPU.
//
// The host runtime around the reconstruction. Requests of any geometry, view count and
// storage type are queued by cbct_server_submit; one worker thread admits them in
// submission order whenever a stream slot is free and the device bytes of the admitted
// requests stay within the budget, enqueues each admitted request's whole pipeline on its
// slot's stream (copy in, the multigrid iteration as one CUDA graph, copy out) and
// retires requests when their completion event fires. Admission does not wait for other
// requests to finish their work: new requests join while earlier ones are mid-iteration,
// and the GPU runs the kernels of all active streams side by side.
//
// Priorities. Under size priority a request's whole pipeline goes to a stream of its
// size class, smallest first. Under age priority the oldest admitted request runs on the
// highest-priority streams, the next oldest one level lower, and so on: the request at
// the head of the line keeps the GPU almost as if it ran alone (its thread blocks are
// scheduled first), and the others fill what it leaves idle (kernel tails, small
// launches, the gaps between dependent launches). Requests move up as older ones finish,
// so their work is enqueued step by step (one A2 iteration per step, at most three steps
// in flight), each step on the stream of the request's current rank and ordered after
// the previous step by an event.
//
// Device memory: every request takes one block from a stream-ordered pool
// (cudaMallocFromPoolAsync on its stream) and gives it back with cudaFreeAsync after its
// last copy, so blocks are reused across requests without device-wide synchronisation.
// Each block holds the request's geometry tables, y, the reconstruction workspace and
// the output volume; nothing is shared between requests, and every kernel of the
// iteration is deterministic, so a request's result does not depend on its neighbours.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cbct_internal.cuh"

namespace cbct {
namespace {

constexpr size_t DEFAULT_BUDGET = 150ull << 30; // 150 GB
constexpr int DEFAULT_SLOTS = 16;
constexpr int MAX_SLOTS = 64;
constexpr double DEFAULT_BYPASS_S = 2.0;
constexpr int N_CLASSES = 3; // stream priority classes: small, medium, large requests
constexpr int MAX_AGE_LEVELS = 8; // priority levels used under age priority (capped by the device's range)
constexpr int STEPS_AHEAD = 3;    // age priority: steps of one request in flight at once

enum RequestState { RQ_QUEUED = 0, RQ_ACTIVE = 1, RQ_DONE = 2 };

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Request {
    long long id = 0;
    cbct_geometry geom{};        // host fields; device tables point into `block`
    std::vector<double> angles;
    std::vector<float2> cs;      // host (cos, sin) table, kept until the request is done
    const float *y_host = nullptr;
    float *f_host = nullptr;
    float mu = 0.0f;
    int levels = 1;
    std::vector<int> iters;
    cbct_recon_opts opts{};
    // byte offsets inside the block
    size_t off_cs = 0, off_ray4 = 0, off_ray2 = 0, off_y = 0, off_f = 0, off_ws = 0, ws_bytes = 0, bytes = 0;
    size_t wset = 0;             // bytes of the finest volume: what its projector keeps in L2
    int cls = 0;                 // priority class (0 = highest)
    int slot = -1;
    char *block = nullptr;
    cudaEvent_t done_ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    // age priority: the reconstruction enqueued step by step
    ReconCursor *cursor = nullptr;
    cudaEvent_t step_ev[STEPS_AHEAD] = {};        // the last steps issued (ring)
    long long steps_issued = 0, steps_done = 0;  // the set-up copies count as step 0
    int cur_stream = -1;                         // stream index of the last step
    bool tail_enqueued = false;                  // the copy-out and release are enqueued
    RequestState state = RQ_QUEUED;
    cbct_status status = CBCT_OK;
    std::string message;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

} // namespace
} // namespace cbct

using namespace cbct;

struct cbct_server {
    cbct_server_opts opts{};
    int device = 0;
    size_t budget = 0;
    cudaMemPool_t pool = nullptr;
    size_t l2_budget = 0;               // bound on the summed wset of admitted requests
    double max_bypass_s = DEFAULT_BYPASS_S;
    int nclass = N_CLASSES;             // priority levels (stream classes)
    std::vector<cudaStream_t> streams;  // nclass x max_active, class-major
    std::vector<int> free_slots[N_CLASSES]; // size/none: stream indices per class; age: slots in [0]
    unsigned int *flags_host = nullptr; // one pinned status word per stream (64-byte stride)
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::list<Request *> queue;         // stable iterators: submit appends while the worker scans
    std::vector<Request *> active;
    std::unordered_map<long long, std::unique_ptr<Request>> requests;
    long long next_id = 1, submitted = 0, completed = 0, failed = 0;
    int max_active_seen = 0;
    size_t bytes_in_use = 0, max_bytes_seen = 0, wset_in_use = 0;
    long long bypassed = 0;
    bool stopping = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
    unsigned int *slot_flags(int slot) { return flags_host + 16 * slot; }
    bool age() const { return opts.size_priority == CBCT_PRIORITY_AGE; }
    cudaStream_t stream_of(int cls, int slot) const { return streams[(size_t)cls * opts.max_active + slot]; }
};

namespace {

// Lays out a request's block: geometry tables, y, output volume, workspace.
void plan_block(Request *r)
{
    const cbct_geometry_desc &d = r->geom.desc;
    const size_t K = (size_t)d.n_views, rays = K * d.nu;
    const size_t M = rays * d.nv, N = (size_t)d.nx * d.ny * d.nz;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    r->off_cs = take(sizeof(float2) * K);
    r->off_ray4 = take(sizeof(float4) * rays);
    r->off_ray2 = take(sizeof(float2) * rays);
    r->off_y = take(sizeof(float) * M);
    r->off_f = take(sizeof(float) * N);
    r->ws_bytes = reconstruct_ws_bytes(&r->geom); // depends on the sizes only
    r->off_ws = take(r->ws_bytes);
    r->bytes = off;
}

bool is_pinned(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

#define SRV_TRY(expr)                                                                              \
    do {                                                                                           \
        cbct_status _s = (expr);                                                                   \
        if (_s != CBCT_OK) return _s;                                                              \
    } while (0)

// The set-up of a request on stream st: its device block, the view and ray tables and
// the projections. Runs on the worker thread.
cbct_status enqueue_prologue(cbct_server *srv, Request *r, cudaStream_t st)
{
    void *blk = nullptr;
    SRV_TRY(check_cuda(cudaMallocFromPoolAsync(&blk, r->bytes, srv->pool, st), "server: device block"));
    r->block = (char *)blk;
    cbct_geometry &g = r->geom;
    g.d_cs = reinterpret_cast<float2 *>(r->block + r->off_cs);
    g.d_ray4 = reinterpret_cast<float4 *>(r->block + r->off_ray4);
    g.d_ray2 = reinterpret_cast<float2 *>(r->block + r->off_ray2);
    const cbct_geometry_desc &d = g.desc;
    const size_t M = (size_t)d.n_views * d.nv * d.nu;
    SRV_TRY(check_cuda(cudaMemcpyAsync(g.d_cs, r->cs.data(), sizeof(float2) * d.n_views, cudaMemcpyHostToDevice, st),
                       "server: view table"));
    SRV_TRY(launch_ray_table(&g, st));
    return check_cuda(cudaMemcpyAsync(r->block + r->off_y, r->y_host, sizeof(float) * M, cudaMemcpyHostToDevice, st),
                      "server: projections in");
}

// The end of a request on stream st: the volume and the status word out, the block back
// to the pool once the copies have run, then the completion event (so a retired
// request's bytes are free in the pool as well as in the budget).
cbct_status enqueue_tail(cbct_server *srv, Request *r, cudaStream_t st)
{
    const cbct_geometry_desc &d = r->geom.desc;
    const size_t N = (size_t)d.nx * d.ny * d.nz;
    SRV_TRY(check_cuda(cudaMemcpyAsync(r->f_host, r->block + r->off_f, sizeof(float) * N, cudaMemcpyDeviceToHost, st),
                       "server: volume out"));
    SRV_TRY(check_cuda(cudaMemcpyAsync(srv->slot_flags(r->slot), reconstruct_flags_address(&r->geom, r->block + r->off_ws),
                                       sizeof(unsigned int), cudaMemcpyDeviceToHost, st),
                       "server: status out"));
    cudaError_t e = cudaFreeAsync(r->block, st);
    if (e != cudaSuccess) return check_cuda(e, "server: block release");
    r->block = nullptr;
    SRV_TRY(check_cuda(cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming), "server: event"));
    return check_cuda(cudaEventRecord(r->done_ev, st), "server: event");
}

// Enqueues everything a request does on its slot's stream (size or no priority). Runs on
// the worker thread.
cbct_status enqueue_request(cbct_server *srv, Request *r)
{
    cudaStream_t st = srv->streams[r->slot];
    SRV_TRY(enqueue_prologue(srv, r, st));
    cbct_geometry &g = r->geom;
    const float *y_dev = reinterpret_cast<const float *>(r->block + r->off_y);
    float *f_dev = reinterpret_cast<float *>(r->block + r->off_f);
    void *ws = r->block + r->off_ws;
    if (srv->opts.use_graphs) {
        SRV_TRY(check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "server: capture"));
        cbct_status s = reconstruct_enqueue(y_dev, &g, r->mu, r->levels, r->iters.data(), r->opts, ws, r->ws_bytes,
                                            f_dev, st);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (s != CBCT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return check_cuda(e, "server: capture");
        e = cudaGraphInstantiate(&r->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            r->exec = nullptr;
            return check_cuda(e, "server: graph instantiation");
        }
        SRV_TRY(check_cuda(cudaGraphLaunch(r->exec, st), "server: graph launch"));
    } else {
        SRV_TRY(reconstruct_enqueue(y_dev, &g, r->mu, r->levels, r->iters.data(), r->opts, ws, r->ws_bytes, f_dev, st));
    }
    return enqueue_tail(srv, r, st);
}

// Age priority: the set-up of a newly admitted request on the streams of priority level
// cls; its steps follow from issue_steps.
cbct_status enqueue_request_stepped(cbct_server *srv, Request *r, int cls)
{
    const int idx = cls * srv->opts.max_active + r->slot;
    cudaStream_t st = srv->streams[idx];
    for (cudaEvent_t &ev : r->step_ev)
        SRV_TRY(check_cuda(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "server: event"));
    SRV_TRY(enqueue_prologue(srv, r, st));
    SRV_TRY(reconstruct_cursor_create(reinterpret_cast<const float *>(r->block + r->off_y), &r->geom, r->mu, r->levels,
                                      r->iters.data(), r->opts, r->block + r->off_ws, r->ws_bytes,
                                      reinterpret_cast<float *>(r->block + r->off_f), &r->cursor));
    SRV_TRY(check_cuda(cudaEventRecord(r->step_ev[0], st), "server: event"));
    r->steps_issued = 1;
    r->cur_stream = idx;
    return CBCT_OK;
}

// Age priority: notes the request's finished steps and keeps STEPS_AHEAD in flight, the new ones
// on the streams of priority level cls (ordered after the previous step by its event);
// after the last step, the tail. Runs on the worker thread without the lock.
cbct_status issue_steps(cbct_server *srv, Request *r, int cls, bool &progressed)
{
    while (r->steps_done < r->steps_issued) {
        const cudaError_t e = cudaEventQuery(r->step_ev[r->steps_done % STEPS_AHEAD]);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return check_cuda(e, "server: request work");
        r->steps_done++;
    }
    const int idx = cls * srv->opts.max_active + r->slot;
    while (!r->tail_enqueued && r->steps_issued - r->steps_done < STEPS_AHEAD) {
        cudaStream_t st = srv->streams[idx];
        if (idx != r->cur_stream)
            SRV_TRY(check_cuda(cudaStreamWaitEvent(st, r->step_ev[(r->steps_issued - 1) % STEPS_AHEAD], 0),
                               "server: step order"));
        r->cur_stream = idx;
        SRV_TRY(reconstruct_cursor_step(r->cursor, st));
        progressed = true;
        if (reconstruct_cursor_finished(r->cursor)) {
            SRV_TRY(enqueue_tail(srv, r, st));
            r->tail_enqueued = true;
        } else {
            // step steps_issued - STEPS_AHEAD, the previous user of this event, has completed
            SRV_TRY(check_cuda(cudaEventRecord(r->step_ev[r->steps_issued % STEPS_AHEAD], st), "server: event"));
            r->steps_issued++;
        }
    }
    return CBCT_OK;
}

// Leaves a failed request's streams idle and its block back in the pool. Runs without
// the lock.
void abort_request(cbct_server *srv, Request *r)
{
    const int ncls = srv->age() ? srv->nclass : 1;
    for (int c = 0; c < ncls; ++c)
        cudaStreamSynchronize(srv->age() ? srv->stream_of(c, r->slot) : srv->streams[r->slot]);
    if (r->block) {
        cudaStream_t st = srv->age() ? srv->stream_of(0, r->slot) : srv->streams[r->slot];
        cudaFreeAsync(r->block, st);
        cudaStreamSynchronize(st);
        r->block = nullptr;
    }
    cudaGetLastError();
}

// Returns a request's slot and bytes. Caller holds the lock.
void retire(cbct_server *srv, Request *r, cbct_status status, const std::string &msg)
{
    if (r->exec) {
        cudaGraphExecDestroy(r->exec);
        r->exec = nullptr;
    }
    if (r->done_ev) {
        cudaEventDestroy(r->done_ev);
        r->done_ev = nullptr;
    }
    for (cudaEvent_t &ev : r->step_ev)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    if (r->cursor) {
        reconstruct_cursor_destroy(r->cursor);
        r->cursor = nullptr;
    }
    r->status = status;
    r->message = msg;
    r->state = RQ_DONE;
    r->t_done = srv->now();
    srv->free_slots[r->cls].push_back(r->slot);
    srv->bytes_in_use -= r->bytes;
    srv->wset_in_use -= r->wset;
    if (status == CBCT_OK) srv->completed++;
    else srv->failed++;
    srv->cv_done.notify_all();
}

void worker_main(cbct_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        bool progressed = false;
        // 1. retire requests whose work has completed
        for (size_t i = 0; i < srv->active.size();) {
            Request *r = srv->active[i];
            if (!r->done_ev) { // age priority: still being enqueued step by step
                ++i;
                continue;
            }
            cudaError_t e = cudaEventQuery(r->done_ev);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            cbct_status status = CBCT_OK;
            std::string msg;
            if (e != cudaSuccess) {
                status = check_cuda(e, "server: request work");
                msg = cbct_last_error();
            } else if (*srv->slot_flags(r->slot) & 2u) {
                status = CBCT_ERR_TIMEOUT;
                msg = "a projector block timed out waiting for its trace record";
            } else if (*srv->slot_flags(r->slot) & 1u) {
                status = CBCT_ERR_NONFINITE;
                msg = "an inner product of the iteration was not finite";
            }
            retire(srv, r, status, msg);
            srv->active[i] = srv->active.back();
            srv->active.pop_back();
            progressed = true;
        }
        // 1b. age priority: steps of the admitted requests, oldest first, each on the
        //     streams of its rank (the oldest on the highest priority)
        if (srv->age() && !srv->active.empty()) {
            std::vector<Request *> order(srv->active);
            std::sort(order.begin(), order.end(), [](const Request *a, const Request *b) { return a->id < b->id; });
            std::vector<std::pair<Request *, cbct_status>> failed;
            std::vector<std::string> messages;
            lk.unlock(); // only this thread changes the admitted requests
            for (size_t rank = 0; rank < order.size(); ++rank) {
                Request *r = order[rank];
                if (r->tail_enqueued) continue;
                const int cls = (int)std::min<size_t>(rank, (size_t)srv->nclass - 1);
                const cbct_status st = issue_steps(srv, r, cls, progressed);
                if (st != CBCT_OK) {
                    failed.emplace_back(r, st);
                    messages.emplace_back(cbct_last_error());
                    abort_request(srv, r);
                }
            }
            lk.lock();
            for (size_t f = 0; f < failed.size(); ++f) {
                Request *r = failed[f].first;
                srv->active.erase(std::find(srv->active.begin(), srv->active.end(), r));
                retire(srv, r, failed[f].second, messages[f]);
                progressed = true;
            }
        }
        // 2. admission. Scan the queue in submission order while a slot is free. Device
        //    memory is granted strictly in order (the scan stops at the first request the
        //    budget cannot hold). A request whose volume would not fit in L2 beside the
        //    volumes already admitted is passed over, so that smaller requests behind it can
        //    start, until it has waited max_bypass_s; from then on nothing overtakes it. A
        //    request is always admitted onto an idle device.
        for (auto it = srv->queue.begin(); it != srv->queue.end() && (int)srv->active.size() < srv->opts.max_active;) {
            Request *r = *it;
            if (srv->bytes_in_use + r->bytes > srv->budget) break;
            const bool fits_l2 = srv->active.empty() || srv->wset_in_use + r->wset <= srv->l2_budget;
            if (!fits_l2) {
                if (srv->now() - r->t_submit > srv->max_bypass_s) break;
                ++it;
                continue;
            }
            if (it != srv->queue.begin()) srv->bypassed++;
            it = srv->queue.erase(it);
            if (srv->age()) r->cls = 0; // one list of slots; the priority level follows the rank
            r->slot = srv->free_slots[r->cls].back();
            srv->free_slots[r->cls].pop_back();
            r->state = RQ_ACTIVE;
            r->t_admit = srv->now();
            srv->bytes_in_use += r->bytes;
            srv->wset_in_use += r->wset;
            if (srv->bytes_in_use > srv->max_bytes_seen) srv->max_bytes_seen = srv->bytes_in_use;
            srv->active.push_back(r); // listed before the unlock: retire() runs only under the lock
            if ((int)srv->active.size() > srv->max_active_seen) srv->max_active_seen = (int)srv->active.size();
            // the newest admitted request is the youngest: the lowest rank so far
            const int cls_age = std::min((int)srv->active.size() - 1, srv->nclass - 1);
            lk.unlock();
            cbct_status s = srv->age() ? enqueue_request_stepped(srv, r, cls_age) : enqueue_request(srv, r);
            std::string msg = s == CBCT_OK ? std::string() : std::string(cbct_last_error());
            // leave the streams idle and the block back in the pool before the slot is reused
            if (s != CBCT_OK) abort_request(srv, r);
            lk.lock();
            if (s != CBCT_OK) {
                for (size_t i = 0; i < srv->active.size(); ++i)
                    if (srv->active[i] == r) {
                        srv->active[i] = srv->active.back();
                        srv->active.pop_back();
                        break;
                    }
                retire(srv, r, s, msg);
            }
            progressed = true;
        }
        if (srv->stopping && srv->queue.empty() && srv->active.empty()) break;
        if (!progressed) {
            if (srv->active.empty())
                srv->cv_work.wait(lk, [&] { return srv->stopping || !srv->queue.empty(); });
            else
                srv->cv_work.wait_for(lk, std::chrono::microseconds(50)); // poll completion events
        }
    }
}

} // namespace

extern "C" cbct_status cbct_server_create(const cbct_server_opts *opts, cbct_server **out)
{
    if (!out) return set_error(CBCT_ERR_INVALID_ARG, "server_create: null argument");
    *out = nullptr;
    cbct_server_opts o{0, DEFAULT_SLOTS, 1, 0, 1, 0.0};
    if (opts) o = *opts;
    if (o.max_active < 1 || o.max_active > MAX_SLOTS)
        return set_error(CBCT_ERR_INVALID_ARG, "server_create: max_active must be in 1..%d", MAX_SLOTS);
    if (!(o.max_bypass_s >= 0.0) || !std::isfinite(o.max_bypass_s))
        return set_error(CBCT_ERR_INVALID_ARG, "server_create: max_bypass_s must be finite and >= 0");
    std::unique_ptr<cbct_server> srv(new cbct_server());
    srv->opts = o;
    srv->t0 = std::chrono::steady_clock::now();
    SRV_TRY(check_cuda(cudaGetDevice(&srv->device), "server_create"));
    size_t free_b = 0, total_b = 0;
    SRV_TRY(check_cuda(cudaMemGetInfo(&free_b, &total_b), "server_create"));
    size_t budget = o.hbm_budget_bytes ? o.hbm_budget_bytes : DEFAULT_BUDGET;
    const size_t cap = (size_t)(0.9 * (double)free_b);
    srv->budget = budget < cap ? budget : cap;
    int l2 = 0;
    SRV_TRY(check_cuda(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, srv->device), "server_create"));
    srv->l2_budget = o.l2_budget_bytes ? o.l2_budget_bytes : (size_t)l2;
    srv->max_bypass_s = o.max_bypass_s > 0.0 ? o.max_bypass_s : DEFAULT_BYPASS_S;
    if (o.size_priority < CBCT_PRIORITY_NONE || o.size_priority > CBCT_PRIORITY_AGE)
        return set_error(CBCT_ERR_INVALID_ARG, "server_create: size_priority must be 0 (none), 1 (size) or 2 (age)");
    int least = 0, greatest = 0;
    SRV_TRY(check_cuda(cudaDeviceGetStreamPriorityRange(&least, &greatest), "server_create"));
    // age priority: one level per rank, as many as the device offers (up to MAX_AGE_LEVELS)
    srv->nclass = o.size_priority == CBCT_PRIORITY_AGE ? std::max(1, std::min(MAX_AGE_LEVELS, least - greatest + 1))
                                                       : N_CLASSES;
    // kernels' shared-memory opt-ins, so that nothing is set while a stream is captured
    SRV_TRY(project_prepare());
    SRV_TRY(tf_prepare());
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = srv->device;
    SRV_TRY(check_cuda(cudaMemPoolCreate(&srv->pool, &props), "server_create: memory pool"));
    unsigned long long keep = ~0ull; // keep freed blocks in the pool for the next requests
    cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    const int nstreams = srv->nclass * o.max_active;
    cudaError_t e = cudaHostAlloc(&srv->flags_host, sizeof(unsigned int) * 16 * nstreams, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(srv->pool);
        return check_cuda(e, "server_create: status words");
    }
    for (int c = 0; c < srv->nclass; ++c) {
        // size: class 0 (small requests) gets the greatest priority, the last class the
        // least; age: level c (rank c, 0 = oldest) gets the c-th greatest
        const int prio = o.size_priority == CBCT_PRIORITY_AGE ? greatest + c
                         : o.size_priority == CBCT_PRIORITY_SIZE
                             ? (c == 0 ? greatest : c == N_CLASSES - 1 ? least : (greatest + least) / 2)
                             : 0;
        for (int s = 0; s < o.max_active; ++s) {
            cudaStream_t st;
            e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio);
            if (e != cudaSuccess) {
                for (cudaStream_t x : srv->streams) cudaStreamDestroy(x);
                cudaFreeHost(srv->flags_host);
                cudaMemPoolDestroy(srv->pool);
                return check_cuda(e, "server_create: streams");
            }
            if (o.size_priority != CBCT_PRIORITY_AGE) srv->free_slots[c].push_back((int)srv->streams.size());
            else if (c == 0) srv->free_slots[0].push_back(s);
            srv->streams.push_back(st);
        }
    }
    srv->worker = std::thread(worker_main, srv.get());
    *out = srv.release();
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_submit(cbct_server *srv, const cbct_geometry_desc *desc, const float *y_host,
                                          float mu, float lambda, int levels, const int *iters,
                                          const cbct_recon_opts *opts, float *f_host, long long *id)
{
    if (!srv || !desc || !y_host || !f_host || !iters || !id)
        return set_error(CBCT_ERR_INVALID_ARG, "server_submit: null argument");
    SRV_TRY(validate_geometry_desc(*desc));
    SRV_TRY(check_projector_fits(*desc));
    cbct_recon_opts o{3, 1, 1, CBCT_F32};
    if (opts) o = *opts;
    SRV_TRY(validate_recon_args(mu, lambda, levels, iters, o));
    if (!is_pinned(y_host) || !is_pinned(f_host))
        return set_error(CBCT_ERR_INVALID_ARG, "server_submit: y_host and f_host must be page-locked host memory");
    std::unique_ptr<Request> r(new Request());
    r->geom.desc = *desc;
    r->angles.resize(desc->n_views);
    r->cs.resize(desc->n_views);
    view_table(*desc, r->angles.data(), r->cs.data());
    r->geom.desc.angles = r->angles.data();
    r->geom.angles = r->angles.data();
    r->geom.device = srv->device;
    r->y_host = y_host;
    r->f_host = f_host;
    r->mu = mu;
    r->levels = levels;
    r->iters.assign(iters, iters + levels);
    r->opts = o;
    plan_block(r.get());
    r->wset = sizeof(float) * (size_t)desc->nx * desc->ny * desc->nz;
    r->cls = r->wset * 8 <= srv->l2_budget ? 0 : r->wset * 2 <= srv->l2_budget ? 1 : 2;
    if (r->bytes > srv->budget)
        return set_error(CBCT_ERR_INVALID_ARG, "server_submit: the request needs %zu device bytes, the budget is %zu",
                         r->bytes, srv->budget);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return set_error(CBCT_ERR_INVALID_ARG, "server_submit: the server is shutting down");
    r->id = srv->next_id++;
    r->t_submit = srv->now();
    *id = r->id;
    srv->queue.push_back(r.get());
    srv->requests[r->id] = std::move(r);
    srv->submitted++;
    srv->cv_work.notify_one();
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_wait(cbct_server *srv, long long id, double timeout_s, cbct_request_info *info)
{
    if (!srv) return set_error(CBCT_ERR_INVALID_ARG, "server_wait: null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->requests.find(id);
    if (it == srv->requests.end()) return set_error(CBCT_ERR_INVALID_ARG, "server_wait: unknown request %lld", id);
    Request *r = it->second.get();
    auto done = [&] { return r->state == RQ_DONE; };
    if (timeout_s < 0.0) srv->cv_done.wait(lk, done);
    else srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
    if (info) {
        info->status = r->state == RQ_DONE ? (int)r->status : (int)CBCT_ERR_TIMEOUT;
        info->done = r->state == RQ_DONE && r->status == CBCT_OK;
        info->t_submit = r->t_submit;
        info->t_admit = r->t_admit;
        info->t_done = r->t_done;
        info->device_bytes = r->bytes;
    }
    if (r->state != RQ_DONE) return set_error(CBCT_ERR_TIMEOUT, "server_wait: request %lld not finished", id);
    if (r->status != CBCT_OK) return set_error(r->status, "%s", r->message.c_str());
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_stats_get(cbct_server *srv, cbct_server_stats *s)
{
    if (!srv || !s) return set_error(CBCT_ERR_INVALID_ARG, "server_stats: null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    s->submitted = srv->submitted;
    s->completed = srv->completed;
    s->failed = srv->failed;
    s->queued = (int)srv->queue.size();
    s->active = (int)srv->active.size();
    s->max_active_seen = srv->max_active_seen;
    s->bytes_in_use = srv->bytes_in_use;
    s->max_bytes_seen = srv->max_bytes_seen;
    s->budget_bytes = srv->budget;
    s->l2_budget_bytes = srv->l2_budget;
    s->bypassed = srv->bypassed;
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_destroy(cbct_server *srv)
{
    if (!srv) return CBCT_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    cudaError_t e = cudaSuccess;
    for (cudaStream_t st : srv->streams) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(st);
    }
    cudaFreeHost(srv->flags_host);
    cudaMemPoolDestroy(srv->pool);
    delete srv;
    return check_cuda(e, "server_destroy");
}
