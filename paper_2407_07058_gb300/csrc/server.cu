// server.cu -- the serving entry points of include/appd.h: continuous batching.
//
// Admission: a request for an n-vertex graph needs 8 n^2 bytes of device
// memory (its W and M slots).  It is admitted while the admitted total stays
// within the budget (minus the server's fixed workspaces) and the in-flight
// count below its limit; otherwise submit returns APPD_ERR_BUSY and the caller
// retries after releasing finished requests.  Slots come from a stream-ordered
// memory pool of the server's own whose release threshold is the budget, so
// memory freed by one request is kept mapped for the next instead of being
// returned to the driver at every synchronization (re-mapping hundreds of MB
// costs milliseconds and shows up as latency spikes).
//
// Dispatch: a server thread owns NSLOT stream slots, each with its own
// batched-kernel runtime (workspace slices) and single-solve workspace, so
// slots never share scratch.  Whenever a slot is free and requests are
// committed, it takes every committed request as one batch: graphs up to the
// size cut-over go through one persistent batched launch, larger ones through
// the multi-CTA single-solve pipeline, all on that slot's stream, followed by
// an event.  Requests committed while a batch runs wait for the next free
// slot, so new work is admitted and launched while earlier work is still on
// the GPU (the two slots' kernels overlap as SMs free up).  poll() retires
// completed batches without blocking.
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/appd.h"
#include "internal.h"

using namespace appd;

namespace {

constexpr int NSLOT = 2;

struct Req {
    uint64_t id = 0;
    int64_t n = 0;
    appd_dtype dt = APPD_F32;
    void* W = nullptr;
    void* M = nullptr;
    size_t bytes = 0;
    cudaEvent_t ready = nullptr;   // recorded on the caller's stream at commit
    bool committed = false;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    BatchRuntime* rt = nullptr;
    Workspace* ws = nullptr;
    bool busy = false;        // a batch is in flight and its event is recorded
    bool launching = false;   // a batch is being enqueued (event not recorded yet)
    std::vector<uint64_t> ids;
};

}  // namespace

struct appd_server {
    std::mutex mu;
    std::condition_variable cv;
    size_t budget = 0;
    size_t reserved = 0;   // fixed workspaces
    size_t used = 0;
    int32_t max_inflight = 0;
    uint64_t next_id = 1;
    int device = 0;
    cudaStream_t alloc_stream = nullptr;
    cudaMemPool_t pool = nullptr;                 // the slots' memory pool
    cudaEvent_t alloc_done = nullptr;             // the latest slot allocation
    cudaEvent_t release_ready = nullptr;          // caller's stream at release
    std::vector<cudaEvent_t> event_pool;          // commit events, reused
    Slot slots[NSLOT];
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<uint64_t> pending;    // committed, not yet launched
    std::deque<uint64_t> finished;   // completed, not yet reported by poll
    std::thread dispatcher;
    bool stop = false;
    u32* status = nullptr;
    BatchTuning tune;
    appd_status error = APPD_OK;     // first dispatch error, reported by poll
};

namespace {

// Moves requests of completed slots to `finished`.  Caller holds sv->mu.
void retire(appd_server* sv)
{
    for (Slot& sl : sv->slots) {
        if (!sl.busy || sl.launching)
            continue;
        cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady)
            continue;
        if (q != cudaSuccess && sv->error == APPD_OK)
            sv->error = APPD_ERR_CUDA;
        for (uint64_t id : sl.ids) {
            auto it = sv->reqs.find(id);
            if (it != sv->reqs.end()) {
                it->second.done = true;
                sv->finished.push_back(id);
            }
        }
        sl.ids.clear();
        sl.busy = false;
    }
}

void dispatch_loop(appd_server* sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        retire(sv);
        Slot* free_slot = nullptr;
        bool any_busy = false;
        for (Slot& sl : sv->slots) {
            if (!sl.busy && !sl.launching && !free_slot)
                free_slot = &sl;
            any_busy |= sl.busy || sl.launching;
        }
        if (sv->stop && sv->pending.empty() && !any_busy)
            return;
        if (free_slot && !sv->pending.empty()) {
            BatchDesc d;
            std::vector<uint64_t> big;
            std::vector<uint64_t> ids(sv->pending.begin(), sv->pending.end());
            sv->pending.clear();
            for (uint64_t id : ids) {
                const Req& r = sv->reqs[id];
                if (r.n <= sv->tune.n_split) {
                    d.w.push_back(r.W);
                    d.m.push_back(r.M);
                    d.n.push_back((u32)r.n);
                    d.dt.push_back((uint8_t)r.dt);
                } else {
                    big.push_back(id);
                }
            }
            std::vector<Req> bigreq;
            for (uint64_t id : big)
                bigreq.push_back(sv->reqs[id]);
            std::vector<cudaEvent_t> ready;
            for (uint64_t id : ids) {
                Req& r = sv->reqs[id];
                if (r.ready) {
                    ready.push_back(r.ready);
                    r.ready = nullptr;
                }
            }
            free_slot->launching = true;
            free_slot->ids = ids;
            lk.unlock();
            // the batch starts after every request's W is complete
            cudaError_t e = cudaSuccess;
            for (cudaEvent_t ev : ready)
                if (e == cudaSuccess)
                    e = cudaStreamWaitEvent(free_slot->stream, ev, 0);
            if (e == cudaSuccess)
                e = batch_launch(*free_slot->rt, d, sv->status, free_slot->stream, false);
            int st = APPD_OK;
            for (const Req& r : bigreq) {
                if (st != APPD_OK)
                    break;
                st = solve_on(*free_slot->ws, sv->status, r.W, r.n, (int)r.dt, r.M,
                              free_slot->stream, false);
            }
            cudaError_t e2 = cudaEventRecord(free_slot->done, free_slot->stream);
            lk.lock();
            // the waits are enqueued: the events may be recorded again
            sv->event_pool.insert(sv->event_pool.end(), ready.begin(), ready.end());
            // only now may retire() look at the event: it belongs to this batch
            free_slot->launching = false;
            free_slot->busy = true;
            if ((e != cudaSuccess || st != APPD_OK || e2 != cudaSuccess) && sv->error == APPD_OK)
                sv->error = (st != APPD_OK) ? (appd_status)st : APPD_ERR_CUDA;
            continue;
        }
        // nothing to launch: wait for a commit, or poll the busy slots
        sv->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 2000));
    }
}

}  // namespace

extern "C" {

appd_status appd_server_create(size_t budget_bytes, int32_t max_inflight, appd_server** out)
{
    if (!out || max_inflight <= 0 || budget_bytes == 0)
        return APPD_ERR_INVALID;
    appd_server* sv = new appd_server();
    sv->budget = budget_bytes;
    sv->max_inflight = max_inflight;
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return APPD_ERR_CUDA;
    }
    sv->status = device_status_word();
    // the batched path's parameters as they are set for this process
    // (appd_batched_tuning, appd_batched_prim_max or appd_batched_autotune)
    sv->tune = current_batch_tuning();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&sv->alloc_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&sv->alloc_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&sv->release_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = sv->device;
        e = cudaMemPoolCreate(&sv->pool, &props);
    }
    if (e == cudaSuccess) {
        uint64_t keep = (uint64_t)budget_bytes;   // the attribute is a 64-bit unsigned value
        e = cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    // load every kernel module now, so that no request pays a first load
    if (e == cudaSuccess)
        e = preload_kernels();
    for (Slot& sl : sv->slots) {
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = batch_runtime_create(sv->tune.n_split, sv->tune, &sl.rt);
        if (e == cudaSuccess)
            e = workspace_create(65536, &sl.ws);
    }
    if (e != cudaSuccess || !sv->status) {
        appd_server_destroy(sv);
        return e == cudaErrorMemoryAllocation ? APPD_ERR_NOMEM : APPD_ERR_CUDA;
    }
    size_t reserved = 0;
    for (Slot& sl : sv->slots)
        reserved += sl.ws->bytes + (size_t)batch_runtime_cap(sl.rt) * 4096;
    sv->reserved = reserved;
    sv->dispatcher = std::thread(dispatch_loop, sv);
    *out = sv;
    return APPD_OK;
}

appd_status appd_server_submit(appd_server* sv, int64_t n, appd_dtype dt, appd_stream_t s,
                               uint64_t* req_id, void** W_slot)
{
    if (!sv || !req_id || !W_slot || n <= 0 || !dtype_ok((int)dt))
        return APPD_ERR_INVALID;
    if (n > 65536)
        return APPD_ERR_TOO_LARGE;
    const size_t bytes = (size_t)n * (size_t)n * 4;
    Req r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if ((int32_t)sv->reqs.size() >= sv->max_inflight ||
            sv->reserved + sv->used + 2 * bytes > sv->budget)
            return APPD_ERR_BUSY;
        r.id = sv->next_id++;
        sv->used += 2 * bytes;   // reserve before allocating
    }
    r.n = n;
    r.dt = dt;
    r.bytes = bytes;
    std::lock_guard<std::mutex> lk(sv->mu);
    cudaError_t e = cudaMallocFromPoolAsync(&r.W, bytes, sv->pool, sv->alloc_stream);
    if (e == cudaSuccess)
        e = cudaMallocFromPoolAsync(&r.M, bytes, sv->pool, sv->alloc_stream);
    // the caller fills W on s: s waits for the allocation (no host wait)
    if (e == cudaSuccess)
        e = cudaEventRecord(sv->alloc_done, sv->alloc_stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent((cudaStream_t)s, sv->alloc_done, 0);
    if (e != cudaSuccess) {
        if (r.W)
            cudaFreeAsync(r.W, sv->alloc_stream);
        if (r.M)
            cudaFreeAsync(r.M, sv->alloc_stream);
        sv->used -= 2 * bytes;
        return e == cudaErrorMemoryAllocation ? APPD_ERR_NOMEM : APPD_ERR_CUDA;
    }
    *req_id = r.id;
    *W_slot = r.W;
    sv->reqs.emplace(r.id, r);
    return APPD_OK;
}

appd_status appd_server_submit_many(appd_server* sv, int32_t count, const int64_t* ns,
                                    const uint8_t* dts, appd_stream_t s, uint64_t* req_ids,
                                    void** W_slots, int32_t* admitted)
{
    if (!sv || count < 0 || !admitted || (count > 0 && (!ns || !dts || !req_ids || !W_slots)))
        return APPD_ERR_INVALID;
    *admitted = 0;
    for (int32_t k = 0; k < count; ++k) {
        if (ns[k] <= 0 || !dtype_ok((int)dts[k]))
            return APPD_ERR_INVALID;
        if (ns[k] > 65536)
            return APPD_ERR_TOO_LARGE;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    cudaError_t e = cudaSuccess;
    int32_t k = 0;
    for (; k < count; ++k) {
        const size_t bytes = (size_t)ns[k] * (size_t)ns[k] * 4;
        if ((int32_t)sv->reqs.size() >= sv->max_inflight ||
            sv->reserved + sv->used + 2 * bytes > sv->budget)
            break;
        Req r;
        r.id = sv->next_id++;
        r.n = ns[k];
        r.dt = (appd_dtype)dts[k];
        r.bytes = bytes;
        e = cudaMallocFromPoolAsync(&r.W, bytes, sv->pool, sv->alloc_stream);
        if (e == cudaSuccess)
            e = cudaMallocFromPoolAsync(&r.M, bytes, sv->pool, sv->alloc_stream);
        if (e != cudaSuccess) {
            if (r.W)
                cudaFreeAsync(r.W, sv->alloc_stream);
            break;
        }
        sv->used += 2 * bytes;
        req_ids[k] = r.id;
        W_slots[k] = r.W;
        sv->reqs.emplace(r.id, r);
    }
    *admitted = k;
    if (k > 0) {
        // s waits (on the device) for every allocation made so far
        cudaError_t e2 = cudaEventRecord(sv->alloc_done, sv->alloc_stream);
        if (e2 == cudaSuccess)
            e2 = cudaStreamWaitEvent((cudaStream_t)s, sv->alloc_done, 0);
        if (e2 != cudaSuccess)
            return APPD_ERR_CUDA;
    }
    if (e != cudaSuccess && k == 0)
        return e == cudaErrorMemoryAllocation ? APPD_ERR_NOMEM : APPD_ERR_CUDA;
    return (k == 0 && count > 0) ? APPD_ERR_BUSY : APPD_OK;
}

appd_status appd_server_commit(appd_server* sv, uint64_t req_id, appd_stream_t s)
{
    return appd_server_commit_many(sv, 1, &req_id, s);
}

appd_status appd_server_commit_many(appd_server* sv, int32_t count, const uint64_t* req_ids,
                                    appd_stream_t s)
{
    if (!sv || count < 0 || (count > 0 && !req_ids))
        return APPD_ERR_INVALID;
    if (count == 0)
        return APPD_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int32_t k = 0; k < count; ++k) {
            auto it = sv->reqs.find(req_ids[k]);
            if (it == sv->reqs.end())
                return APPD_ERR_NOT_FOUND;
            if (it->second.committed)
                return APPD_ERR_INVALID;
        }
        // one event for the group: the requests' W are complete together
        cudaEvent_t ev = nullptr;
        if (!sv->event_pool.empty()) {
            ev = sv->event_pool.back();
            sv->event_pool.pop_back();
        } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            return APPD_ERR_CUDA;
        }
        if (cudaEventRecord(ev, (cudaStream_t)s) != cudaSuccess) {
            sv->event_pool.push_back(ev);
            return APPD_ERR_CUDA;
        }
        for (int32_t k = 0; k < count; ++k) {
            Req& r = sv->reqs[req_ids[k]];
            r.ready = (k == 0) ? ev : nullptr;   // the first request carries the event
            r.committed = true;
            sv->pending.push_back(req_ids[k]);
        }
    }
    sv->cv.notify_one();
    return APPD_OK;
}

appd_status appd_server_poll(appd_server* sv, uint64_t* done_ids, const void** M_ptrs, int32_t cap,
                             int32_t* n_done)
{
    if (!sv || !n_done || cap < 0 || (cap > 0 && (!done_ids || !M_ptrs)))
        return APPD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    retire(sv);
    int32_t k = 0;
    while (k < cap && !sv->finished.empty()) {
        const uint64_t id = sv->finished.front();
        sv->finished.pop_front();
        done_ids[k] = id;
        M_ptrs[k] = sv->reqs[id].M;
        ++k;
    }
    *n_done = k;
    if (sv->error != APPD_OK) {
        appd_status e = sv->error;
        sv->error = APPD_OK;
        return e;
    }
    return APPD_OK;
}

appd_status appd_server_release(appd_server* sv, uint64_t req_id, appd_stream_t s)
{
    return appd_server_release_many(sv, 1, &req_id, s);
}

appd_status appd_server_release_many(appd_server* sv, int32_t count, const uint64_t* req_ids,
                                     appd_stream_t s)
{
    if (!sv || count < 0 || (count > 0 && !req_ids))
        return APPD_ERR_INVALID;
    if (count == 0)
        return APPD_OK;
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int32_t k = 0; k < count; ++k) {
        auto it = sv->reqs.find(req_ids[k]);
        if (it == sv->reqs.end())
            return APPD_ERR_NOT_FOUND;
        if (it->second.committed && !it->second.done)
            return APPD_ERR_BUSY;
    }
    // the slots are freed in stream order after the work the caller enqueued
    // on s so far (its reads of M, or its writes of an uncommitted W), so the
    // pool cannot hand the memory to a later request while that work runs
    cudaError_t e = cudaEventRecord(sv->release_ready, (cudaStream_t)s);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(sv->alloc_stream, sv->release_ready, 0);
    if (e != cudaSuccess)
        return APPD_ERR_CUDA;
    for (int32_t k = 0; k < count; ++k) {
        auto it = sv->reqs.find(req_ids[k]);
        Req& r = it->second;
        if (r.ready) {   // committed but never launched: its event returns to the pool
            sv->event_pool.push_back(r.ready);
            r.ready = nullptr;
        }
        cudaFreeAsync(r.W, sv->alloc_stream);
        cudaFreeAsync(r.M, sv->alloc_stream);
        sv->used -= 2 * r.bytes;
        sv->reqs.erase(it);
    }
    return APPD_OK;
}

appd_status appd_server_destroy(appd_server* sv)
{
    if (!sv)
        return APPD_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->pending.clear();   // committed but not launched: dropped
    }
    sv->cv.notify_all();
    if (sv->dispatcher.joinable())
        sv->dispatcher.join();
    for (Slot& sl : sv->slots)
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
    for (auto& kv : sv->reqs) {
        cudaFreeAsync(kv.second.W, sv->alloc_stream);
        cudaFreeAsync(kv.second.M, sv->alloc_stream);
        if (kv.second.ready)
            cudaEventDestroy(kv.second.ready);
    }
    for (cudaEvent_t ev : sv->event_pool)
        cudaEventDestroy(ev);
    if (sv->alloc_done)
        cudaEventDestroy(sv->alloc_done);
    if (sv->release_ready)
        cudaEventDestroy(sv->release_ready);
    if (sv->alloc_stream) {
        cudaStreamSynchronize(sv->alloc_stream);
        cudaStreamDestroy(sv->alloc_stream);
    }
    if (sv->pool)
        cudaMemPoolDestroy(sv->pool);
    for (Slot& sl : sv->slots) {
        batch_runtime_destroy(sl.rt);
        workspace_destroy(sl.ws);
        if (sl.done)
            cudaEventDestroy(sl.done);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
    }
    delete sv;
    return APPD_OK;
}

}  // extern "C"
