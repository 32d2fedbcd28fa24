// server.cu -- the serving entry points of include/appd.h.
//
// Admission: a request for an n-vertex graph needs 8 n^2 bytes on the device
// (its W and M slots).  It is admitted while the admitted total stays within
// the budget (minus the solver workspace) and the in-flight count below the
// limit; otherwise submit returns APPD_ERR_BUSY and the caller retries after
// releasing finished requests.  Slots come from the stream-ordered allocator
// on the server's stream, so admission and release never synchronize the
// device.  Committed requests are handed to the solver in arrival order and
// complete asynchronously; poll reports finished ones without blocking.
#include <cstdint>
#include <deque>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/appd.h"
#include "internal.h"

namespace {

struct Req {
    uint64_t id = 0;
    int64_t n = 0;
    appd_dtype dt = APPD_F32;
    void* W = nullptr;
    void* M = nullptr;
    size_t bytes = 0;
    bool committed = false;
    bool done = false;
    cudaEvent_t ev = nullptr;
};

}  // namespace

struct appd_server {
    std::mutex mu;
    size_t budget = 0;
    size_t used = 0;
    int32_t max_inflight = 0;
    uint64_t next_id = 1;
    cudaStream_t stream = nullptr;
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<uint64_t> pending;   // committed, not yet reported done
};

extern "C" {

appd_status appd_server_create(size_t budget_bytes, int32_t max_inflight, appd_server** out)
{
    if (!out || max_inflight <= 0 || budget_bytes == 0)
        return APPD_ERR_INVALID;
    appd_server* sv = new appd_server();
    sv->budget = budget_bytes;
    sv->max_inflight = max_inflight;
    if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete sv;
        return APPD_ERR_CUDA;
    }
    *out = sv;
    return APPD_OK;
}

appd_status appd_server_submit(appd_server* sv, int64_t n, appd_dtype dt, uint64_t* req_id,
                               void** W_slot)
{
    if (!sv || !req_id || !W_slot || n <= 0 || ((int)dt != APPD_F32 && (int)dt != APPD_U32))
        return APPD_ERR_INVALID;
    if (n > 65536)
        return APPD_ERR_TOO_LARGE;
    std::lock_guard<std::mutex> lk(sv->mu);
    const size_t bytes = (size_t)n * (size_t)n * 4;
    if ((int32_t)sv->reqs.size() >= sv->max_inflight || sv->used + 2 * bytes > sv->budget)
        return APPD_ERR_BUSY;
    Req r;
    r.id = sv->next_id++;
    r.n = n;
    r.dt = dt;
    r.bytes = bytes;
    if (cudaMallocAsync(&r.W, bytes, sv->stream) != cudaSuccess)
        return APPD_ERR_NOMEM;
    if (cudaMallocAsync(&r.M, bytes, sv->stream) != cudaSuccess) {
        cudaFreeAsync(r.W, sv->stream);
        return APPD_ERR_NOMEM;
    }
    // the caller may fill W from another stream: make the slot valid first
    if (cudaStreamSynchronize(sv->stream) != cudaSuccess)
        return APPD_ERR_CUDA;
    if (cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess)
        return APPD_ERR_CUDA;
    sv->used += 2 * bytes;
    *req_id = r.id;
    *W_slot = r.W;
    sv->reqs.emplace(r.id, r);
    return APPD_OK;
}

appd_status appd_server_commit(appd_server* sv, uint64_t req_id)
{
    if (!sv)
        return APPD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(req_id);
    if (it == sv->reqs.end())
        return APPD_ERR_NOT_FOUND;
    Req& r = it->second;
    if (r.committed)
        return APPD_ERR_INVALID;
    appd_status st = appd_solve(r.W, r.n, r.dt, r.M, (appd_stream_t)sv->stream);
    if (st != APPD_OK)
        return st;
    if (cudaEventRecord(r.ev, sv->stream) != cudaSuccess)
        return APPD_ERR_CUDA;
    r.committed = true;
    sv->pending.push_back(req_id);
    return APPD_OK;
}

appd_status appd_server_poll(appd_server* sv, uint64_t* done_ids, const void** M_ptrs, int32_t cap,
                             int32_t* n_done)
{
    if (!sv || !n_done || cap < 0 || (cap > 0 && (!done_ids || !M_ptrs)))
        return APPD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    int32_t k = 0;
    while (k < cap && !sv->pending.empty()) {
        uint64_t id = sv->pending.front();
        Req& r = sv->reqs[id];
        cudaError_t q = cudaEventQuery(r.ev);
        if (q == cudaErrorNotReady)
            break;
        if (q != cudaSuccess)
            return APPD_ERR_CUDA;
        r.done = true;
        done_ids[k] = id;
        M_ptrs[k] = r.M;
        ++k;
        sv->pending.pop_front();
    }
    *n_done = k;
    return APPD_OK;
}

appd_status appd_server_release(appd_server* sv, uint64_t req_id)
{
    if (!sv)
        return APPD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(req_id);
    if (it == sv->reqs.end())
        return APPD_ERR_NOT_FOUND;
    Req& r = it->second;
    if (r.committed && !r.done)
        return APPD_ERR_BUSY;
    cudaFreeAsync(r.W, sv->stream);
    cudaFreeAsync(r.M, sv->stream);
    cudaEventDestroy(r.ev);
    sv->used -= 2 * r.bytes;
    sv->reqs.erase(it);
    return APPD_OK;
}

appd_status appd_server_destroy(appd_server* sv)
{
    if (!sv)
        return APPD_ERR_INVALID;
    cudaStreamSynchronize(sv->stream);
    for (auto& kv : sv->reqs) {
        cudaFreeAsync(kv.second.W, sv->stream);
        cudaFreeAsync(kv.second.M, sv->stream);
        cudaEventDestroy(kv.second.ev);
    }
    cudaStreamSynchronize(sv->stream);
    cudaStreamDestroy(sv->stream);
    delete sv;
    return APPD_OK;
}

}  // extern "C"
