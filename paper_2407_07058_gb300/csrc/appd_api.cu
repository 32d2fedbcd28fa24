// appd_api.cu -- the C ABI (include/appd.h): argument checks, the per-device
// workspace, the device status word, and the launch sequence of a solve.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/appd.h"
#include "internal.h"

using namespace appd;

namespace {

constexpr int MAX_DEV = 64;
std::mutex g_mu;
Workspace* g_ws[MAX_DEV] = {};
u32* g_status[MAX_DEV] = {};
BatchTuning g_tune;
BatchRuntime* g_brt[MAX_DEV] = {};
BatchTuning g_brt_tune[MAX_DEV];

// ------------------------------------------------------------- profiling
struct ProfMark {
    int phase;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfMark> g_marks;
std::vector<cudaEvent_t> g_event_pool;
size_t g_pool_used = 0;
long long g_launches = 0;
Counters* g_last_ctr = nullptr;

cudaEvent_t pool_event()
{
    if (g_pool_used == g_event_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        g_event_pool.push_back(e);
    }
    return g_event_pool[g_pool_used++];
}


size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

appd_status cuda_fail(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation)
        return APPD_ERR_NOMEM;
    return APPD_ERR_CUDA;
}

}  // namespace

size_t appd::workspace_layout(Workspace& w, char* base, int64_t cap)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = align_up(off, 256);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t N = (size_t)cap;
    const int lv = ceil_log2(cap) + 1;
    const size_t ntiles = (N + 2047) / 2048 + 1;
    w.ctr = (Counters*)take(sizeof(Counters));
    w.part = (u32*)take(4096 * sizeof(u32));
    w.best[0] = (u64*)take(N * 8);
    w.best[1] = (u64*)take(N * 8);
    u32** u32s[] = {&w.comp, &w.hook, &w.par, &w.flag, &w.rootid, &w.label, &w.cnt, &w.fillc,
                    &w.members, &w.nchunk, &w.item_group, &w.deg, &w.afill, &w.parent, &w.pe_key,
                    &w.nha, &w.first_child, &w.next_sib, &w.pos, &w.order, &w.nsize, &w.gap};
    for (u32** p : u32s)
        *p = (u32*)take((N + 4) * sizeof(u32));
    w.gstart = (u32*)take((N + 4) * sizeof(u32));
    w.chunk_start = (u32*)take((N + 4) * sizeof(u32));
    w.adj_off = (u32*)take((N + 4) * sizeof(u32));
    w.a4_start = (u32*)take((N + 4) * sizeof(u32));
    w.label16 = (unsigned short*)take((N + 8) * sizeof(unsigned short));
    w.mst = (u64*)take((N + 1) * 8);
    w.adj = (u32*)take(2 * N * sizeof(u32));
    w.aslot = (u32*)take(2 * N * sizeof(u32));
    for (int i = 0; i < 2; ++i) {
        w.lr_d[i] = (u32*)take(2 * N * sizeof(u32) + 16);
        w.lr_nx[i] = (u32*)take(2 * N * sizeof(u32) + 16);
        w.skey[i] = (u64*)take((N + 1) * 8);
        w.sval[i] = (u32*)take((N + 1) * sizeof(u32));
    }
    w.ord = (u64*)take(N * 8);
    w.jump = (u32*)take((size_t)lv * N * sizeof(u32));
    w.mxo = (u64*)take((size_t)lv * N * 8);
    w.hist = (u32*)take(256 * ntiles * sizeof(u32));
    w.st = (u32*)take((size_t)lv * N * sizeof(u32));
    return align_up(off, 256);
}

cudaError_t appd::workspace_create(int64_t n, Workspace** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    int64_t cap = 1024;
    while (cap < n)
        cap *= 2;
    Workspace* nw = new Workspace();
    nw->device = dev;
    nw->cap = cap;
    nw->n = 0;
    const size_t bytes = workspace_layout(*nw, nullptr, cap);
    void* base = nullptr;
    e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
        delete nw;
        return e;
    }
    workspace_layout(*nw, (char*)base, cap);
    nw->base = base;
    nw->bytes = bytes;
    cudaDeviceGetAttribute(&nw->sms, cudaDevAttrMultiProcessorCount, dev);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    nw->coop_blocks = nw->sms;
    nw->coop_threads = 512;
    nw->contract_blocks = nw->sms;
    nw->bin_cap = (u32)((smem_optin - 2048) / 8);
    nw->bin_cap2 = (u32)((smem_optin / 2 - 2048) / 8);
    nw->bin_cap_t = contract_tma_bin_cap(smem_optin);
    *out = nw;
    return cudaSuccess;
}

void appd::workspace_destroy(Workspace* w)
{
    if (!w)
        return;
    cudaDeviceSynchronize();
    cudaFree(w->base);
    cudaFree(w->cscratch);
    cudaFree(w->pscratch);
    cudaFree(w->hostW);
    cudaFree(w->hostM);
    delete w;
}

namespace {

// The device's workspace with capacity >= n (grown if needed).
appd_status get_ws(int64_t n, Workspace** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return APPD_ERR_CUDA;
    Workspace*& w = g_ws[dev];
    if (w && w->cap >= n) {
        *out = w;
        return APPD_OK;
    }
    if (w) {
        workspace_destroy(w);
        w = nullptr;
    }
    e = workspace_create(n, &w);
    if (e != cudaSuccess)
        return cuda_fail(e);
    *out = w;
    return APPD_OK;
}

appd_status get_status(u32** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return APPD_ERR_CUDA;
    if (!g_status[dev]) {
        cudaError_t e = cudaMalloc(&g_status[dev], 256);
        if (e != cudaSuccess)
            return cuda_fail(e);
        e = cudaMemset(g_status[dev], 0, 256);
        if (e != cudaSuccess)
            return cuda_fail(e);
    }
    *out = g_status[dev];
    return APPD_OK;
}

// Per-solve sizes on the shared workspace.
void set_sizes(Workspace& w, int64_t n)
{
    w.n = n;
    w.levels = n > 1 ? ceil_log2(n) : 1;
    if (w.levels < 1)
        w.levels = 1;
    int stl = 1;
    while (((int64_t)1 << stl) <= n - 1)
        ++stl;
    w.st_levels = stl;
    w.ntiles = (u32)((n - 1 + 2047) / 2048);
    if (w.ntiles == 0)
        w.ntiles = 1;
}

appd_status check_args(const void* W, int64_t n, int dt, const void* M)
{
    if (n < 0 || !W || !M || !dtype_ok(dt))
        return APPD_ERR_INVALID;
    if (n > (int64_t)MAX_N)
        return APPD_ERR_TOO_LARGE;
    if (M != W) {
        const char* a = (const char*)W;
        const char* b = (const char*)M;
        size_t bytes = (size_t)n * (size_t)n * 4;
        if (a < b + bytes && b < a + bytes)
            return APPD_ERR_ALIAS;
    }
    return APPD_OK;
}

// Holds the workspace of one solve; n is recorded in the workspace's size
// fields for the launch functions.
struct SolveCtx {
    Workspace* ws = nullptr;
    u32* status = nullptr;
    int64_t cap = 0;
};

appd_status prepare(int64_t n, SolveCtx& c)
{
    appd_status st = get_ws(n, &c.ws);
    if (st != APPD_OK)
        return st;
    st = get_status(&c.status);
    if (st != APPD_OK)
        return st;
    c.cap = c.ws->cap;
    return APPD_OK;
}

// Runs MST + leaf order for a graph of size n on the workspace (whose arrays
// have capacity c.cap).  cbuf must hold contraction_scratch_bytes(n).
appd_status mst_and_order(SolveCtx& c, const void* W, int64_t n, int dt, void* cbuf, bool order,
                          cudaStream_t s)
{
    Workspace& w = *c.ws;
    set_sizes(w, n);
    g_last_ctr = w.ctr;
    cudaError_t e = run_mst(w, W, dt, cbuf, contraction_scratch_bytes(n), c.status, s);
    if (e == cudaSuccess && order) {
        prof_begin(PH_LEAF, s);
        e = run_leaf_order(w, c.status, s);
        prof_end(PH_LEAF, s);
        prof_launches(1);
    }
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status ensure_cscratch(Workspace& w, int64_t n)
{
    size_t need = contraction_scratch_bytes(n);
    if (w.cscratch_bytes >= need)
        return APPD_OK;
    cudaDeviceSynchronize();
    cudaFree(w.cscratch);
    w.cscratch = nullptr;
    w.cscratch_bytes = 0;
    cudaError_t e = cudaMalloc(&w.cscratch, need);
    if (e != cudaSuccess)
        return cuda_fail(e);
    w.cscratch_bytes = need;
    return APPD_OK;
}

appd_status solve_with(Workspace& w, u32* status, const void* W, int64_t n, int dt, void* M,
                       cudaStream_t s, bool alg4)
{
    SolveCtx c;
    c.ws = &w;
    c.status = status;
    c.cap = w.cap;
    appd_status st;
    void* cbuf = M;
    if (M == W) {
        if ((st = ensure_cscratch(w, n)) != APPD_OK)
            return st;
        cbuf = w.cscratch;
    }
    if ((st = mst_and_order(c, W, n, dt, cbuf, true, s)) != APPD_OK)
        return st;
    set_sizes(w, n);
    prof_begin(PH_FILL, s);
    cudaError_t e = alg4 ? run_fill_alg4(w, dt, M, c.status, s) : run_fill(w, dt, M, s);
    prof_end(PH_FILL, s);
    prof_launches(alg4 ? 4 : 1);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status solve_impl(const void* W, int64_t n, int dt, void* M, cudaStream_t s, bool alg4)
{
    appd_status st = check_args(W, n, dt, M);
    if (st != APPD_OK || n == 0)
        return st;
    std::lock_guard<std::mutex> lk(g_mu);
    SolveCtx c;
    if ((st = prepare(n, c)) != APPD_OK)
        return st;
    return solve_with(*c.ws, c.status, W, n, dt, M, s, alg4);
}

// Probe of the bounded grid barrier: CTA 1 never arrives, so CTA 0's wait
// runs out after limit_ns and records DEV_TIMEOUT; both CTAs then return.
__global__ void k_wait_probe(GridBar* bar, u32* status, u64 limit_ns)
{
    if (blockIdx.x != 0)
        return;
    grid_sync(bar, status, limit_ns);
}

__global__ void k_check_sym(const u32* __restrict__ W, u32 n, u32* __restrict__ bad)
{
    u64 total = (u64)n * n;
    for (u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (u64)gridDim.x * blockDim.x) {
        u32 i = (u32)(idx / n), j = (u32)(idx - (u64)i * n);
        if (i < j && W[idx] != W[(size_t)j * n + i])
            *bad = 1u;
    }
}

}  // namespace

namespace appd {

void prof_begin(int phase, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on)
        return;
    ProfMark m{phase, pool_event(), nullptr};
    cudaEventRecord(m.a, s);
    g_marks.push_back(m);
}

void prof_end(int phase, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on)
        return;
    for (auto it = g_marks.rbegin(); it != g_marks.rend(); ++it) {
        if (it->phase == phase && it->b == nullptr) {
            it->b = pool_event();
            cudaEventRecord(it->b, s);
            return;
        }
    }
}

void prof_launches(int k)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_on)
        g_launches += k;
}

}  // namespace appd

int appd::solve_on(Workspace& ws, u32* status, const void* W, int64_t n, int dt, void* M,
                   cudaStream_t s, bool alg4)
{
    if (n == 0)
        return APPD_OK;
    return (int)solve_with(ws, status, W, n, dt, M, s, alg4);
}

BatchTuning appd::current_batch_tuning()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_tune;
}

u32* appd::device_status_word()
{
    std::lock_guard<std::mutex> lk(g_mu);
    u32* st = nullptr;
    return get_status(&st) == APPD_OK ? st : nullptr;
}

extern "C" {

int32_t appd_profile_begin(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_marks.clear();
    g_pool_used = 0;
    g_launches = 0;
    g_prof_on = true;
    return 0;
}

int32_t appd_profile_end(double* out, int32_t cap)
{
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    double acc[PH_COUNT + 2] = {0};
    for (const ProfMark& m : g_marks) {
        if (!m.b)
            continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess)
            acc[m.phase] += ms;
    }
    acc[PH_COUNT] = (double)g_launches;
    if (g_last_ctr) {
        u32 c[2] = {0, 0};
        if (cudaMemcpy(c, g_last_ctr->c, sizeof(c), cudaMemcpyDeviceToHost) == cudaSuccess)
            acc[PH_COUNT + 1] = c[1];
    }
    int32_t k = 0;
    for (; k < cap && k < PH_COUNT + 2; ++k)
        out[k] = acc[k];
    return k;
}

const char* appd_status_str(appd_status st)
{
    switch (st) {
    case APPD_OK: return "APPD_OK";
    case APPD_ERR_INVALID: return "APPD_ERR_INVALID";
    case APPD_ERR_TOO_LARGE: return "APPD_ERR_TOO_LARGE";
    case APPD_ERR_NOMEM: return "APPD_ERR_NOMEM";
    case APPD_ERR_CUDA: return "APPD_ERR_CUDA";
    case APPD_ERR_ASYMMETRIC: return "APPD_ERR_ASYMMETRIC";
    case APPD_ERR_TIMEOUT: return "APPD_ERR_TIMEOUT";
    case APPD_ERR_BUSY: return "APPD_ERR_BUSY";
    case APPD_ERR_ALIAS: return "APPD_ERR_ALIAS";
    case APPD_ERR_NOT_FOUND: return "APPD_ERR_NOT_FOUND";
    case APPD_ERR_INTERNAL: return "APPD_ERR_INTERNAL";
    }
    return "APPD_ERR_UNKNOWN";
}

appd_status appd_solve(const void* W, int64_t n, appd_dtype dt, void* M, appd_stream_t s)
{
    return solve_impl(W, n, (int)dt, M, (cudaStream_t)s, false);
}

appd_status appd_solve_points(const float* X, int64_t n, int32_t d, appd_dtype dt, void* M,
                              appd_stream_t s)
{
    if (n < 0 || !X || !M || (dt != APPD_F32 && dt != APPD_F32_WIDEST) || points_dim(d) == 0)
        return APPD_ERR_INVALID;
    if (n > (int64_t)MAX_N)
        return APPD_ERR_TOO_LARGE;
    {
        const char* a = (const char*)X;
        const char* b = (const char*)M;
        const size_t xb = (size_t)n * (size_t)d * 4, mb = (size_t)n * (size_t)n * 4;
        if (a < b + mb && b < a + xb)
            return APPD_ERR_ALIAS;
    }
    if (n == 0)
        return APPD_OK;
    cudaStream_t cs = (cudaStream_t)s;
    std::lock_guard<std::mutex> lk(g_mu);
    SolveCtx c;
    appd_status st;
    if ((st = prepare(n, c)) != APPD_OK)
        return st;
    Workspace& w = *c.ws;
    const int D = points_dim(d);
    // two coordinate arrays (vertex order, component order) and two u32 per row
    auto bytes_for = [](size_t rows, int dim) { return rows * dim * sizeof(float) * 2 + rows * 8; };
    const size_t need = bytes_for(points_rows_padded((u32)n), D);
    if (w.pscratch_bytes < need) {
        cudaDeviceSynchronize();
        cudaFree(w.pscratch);
        w.pscratch = nullptr;
        w.pscratch_bytes = 0;
        // sized for the workspace's capacity at 32 dimensions, so that it is
        // allocated once
        const size_t full = bytes_for(points_rows_padded((u32)w.cap), 32);
        cudaError_t e = cudaMalloc(&w.pscratch, full);
        if (e != cudaSuccess)
            return cuda_fail(e);
        w.pscratch_bytes = full;
    }
    cudaError_t e = launch_pts_pad(X, (u32)n, d, w.pscratch, cs);
    prof_launches(1);
    if (e != cudaSuccess)
        return cuda_fail(e);
    set_sizes(w, n);
    g_last_ctr = w.ctr;
    const size_t rows = points_rows_padded((u32)n);
    PointsSrc ps;
    ps.P = w.pscratch;
    ps.D = D;
    ps.Ps = w.pscratch + rows * D;
    ps.pvid = (u32*)(w.pscratch + 2 * rows * D);
    ps.pcomp = ps.pvid + rows;
    e = run_mst(w, nullptr, (int)dt, M, contraction_scratch_bytes(n), c.status, cs, &ps);
    if (e == cudaSuccess) {
        prof_begin(PH_LEAF, cs);
        e = run_leaf_order(w, c.status, cs);
        prof_end(PH_LEAF, cs);
        prof_launches(1);
    }
    if (e == cudaSuccess) {
        prof_begin(PH_FILL, cs);
        e = run_fill(w, (int)dt, M, cs);
        prof_end(PH_FILL, cs);
        prof_launches(1);
    }
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_solve_alg4(const void* W, int64_t n, appd_dtype dt, void* M, appd_stream_t s)
{
    return solve_impl(W, n, (int)dt, M, (cudaStream_t)s, true);
}

appd_status appd_solve_host(const void* W_host, int64_t n, appd_dtype dt, void* M_host,
                            appd_stream_t s)
{
    appd_status st = check_args(W_host, n, (int)dt, M_host);
    if (st != APPD_OK || n == 0)
        return st;
    cudaStream_t cs = (cudaStream_t)s;
    const size_t bytes = (size_t)n * (size_t)n * 4;
    void *dW = nullptr, *dM = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        Workspace* w = nullptr;
        if ((st = get_ws(n, &w)) != APPD_OK)
            return st;
        if (w->host_bytes < bytes) {
            cudaStreamSynchronize(cs);
            cudaFree(w->hostW);
            cudaFree(w->hostM);
            w->hostW = w->hostM = nullptr;
            w->host_bytes = 0;
            cudaError_t e = cudaMalloc(&w->hostW, bytes);
            if (e != cudaSuccess)
                return cuda_fail(e);
            e = cudaMalloc(&w->hostM, bytes);
            if (e != cudaSuccess) {
                cudaFree(w->hostW);
                w->hostW = nullptr;
                return cuda_fail(e);
            }
            w->host_bytes = bytes;
        }
        dW = w->hostW;
        dM = w->hostM;
    }
    cudaError_t e = cudaMemcpyAsync(dW, W_host, bytes, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess)
        return cuda_fail(e);
    st = solve_impl(dW, n, (int)dt, dM, cs, false);
    if (st != APPD_OK)
        return st;
    e = cudaMemcpyAsync(M_host, dM, bytes, cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess)
        return cuda_fail(e);
    e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

// Pipelined host entry: per device, two copy streams (in, out) and two
// device buffer pairs; the solve runs on the caller's stream.  One call's
// copy in and solve overlap the previous call's copy out (the host link
// carries both directions at once).
namespace {
// Each direction's copy is split into PIPE_LANES pieces on as many streams:
// host-to-device and device-to-host copies running at the same time move
// about 15% more bytes per second that way than as one copy each (measured
// on GB300: 343 vs 293 GB/s for both directions together).
constexpr int PIPE_LANES = 4;
struct HostPipe {
    cudaStream_t in[PIPE_LANES] = {}, out[PIPE_LANES] = {};
    cudaEvent_t ev_in[2][PIPE_LANES] = {}, ev_comp[2] = {}, ev_out[2][PIPE_LANES] = {};
    void* dW[2] = {};
    void* dM[2] = {};
    size_t bytes = 0;
    uint64_t k = 0;
};
HostPipe* g_pipe[MAX_DEV] = {};
std::mutex g_pipe_mu;

void pipe_destroy(HostPipe* p)
{
    if (!p)
        return;
    // the buffers are in use until the last solve on each pair (on a caller's
    // stream) and the copies on the internal streams have finished
    for (int i = 0; i < 2; ++i)
        if (p->ev_comp[i])
            cudaEventSynchronize(p->ev_comp[i]);
    for (int l = 0; l < PIPE_LANES; ++l)
        for (cudaStream_t st : {p->in[l], p->out[l]})
            if (st)
                cudaStreamSynchronize(st);
    for (int i = 0; i < 2; ++i) {
        cudaFree(p->dW[i]);
        cudaFree(p->dM[i]);
        cudaEventDestroy(p->ev_comp[i]);
        for (int l = 0; l < PIPE_LANES; ++l) {
            cudaEventDestroy(p->ev_in[i][l]);
            cudaEventDestroy(p->ev_out[i][l]);
        }
    }
    for (int l = 0; l < PIPE_LANES; ++l)
        for (cudaStream_t st : {p->in[l], p->out[l]})
            if (st)
                cudaStreamDestroy(st);
    delete p;
}

cudaError_t pipe_get(int dev, size_t bytes, HostPipe** out)
{
    HostPipe*& p = g_pipe[dev];
    if (p && p->bytes >= bytes) {
        *out = p;
        return cudaSuccess;
    }
    pipe_destroy(p);
    p = new HostPipe();
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < PIPE_LANES; ++l)
        for (cudaStream_t* st : {&p->in[l], &p->out[l]})
            if (e == cudaSuccess)
                e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&p->ev_comp[i], cudaEventDisableTiming);
        for (int l = 0; l < PIPE_LANES; ++l)
            for (cudaEvent_t* ev : {&p->ev_in[i][l], &p->ev_out[i][l]})
                if (e == cudaSuccess)
                    e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaMalloc(&p->dW[i], bytes);
        if (e == cudaSuccess)
            e = cudaMalloc(&p->dM[i], bytes);
    }
    if (e != cudaSuccess) {
        pipe_destroy(p);
        p = nullptr;
        return e;
    }
    p->bytes = bytes;
    *out = p;
    return cudaSuccess;
}
}  // namespace

appd_status appd_solve_host_async(const void* W_host, int64_t n, appd_dtype dt, void* M_host,
                                  appd_stream_t s)
{
    appd_status st = check_args(W_host, n, (int)dt, M_host);
    if (st != APPD_OK || n == 0)
        return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return APPD_ERR_CUDA;
    const size_t bytes = (size_t)n * (size_t)n * 4;
    cudaStream_t cs = (cudaStream_t)s;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe* p = nullptr;
    cudaError_t e = pipe_get(dev, bytes, &p);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? APPD_ERR_NOMEM : cuda_fail(e);
    const int b = (int)(p->k++ & 1);
    // piece l of the buffers: [l * piece, min(bytes, (l + 1) * piece)), 16-byte aligned
    const size_t piece = ((bytes + PIPE_LANES - 1) / PIPE_LANES + 15) & ~(size_t)15;
    auto span = [&](int l, size_t* off) -> size_t {
        *off = (size_t)l * piece;
        return *off >= bytes ? 0 : (bytes - *off < piece ? bytes - *off : piece);
    };
    // copy in once this pair's previous solve, the only reader of dW[b], is
    // done (the pair's previous copy out may still be running)
    for (int l = 0; l < PIPE_LANES; ++l) {
        size_t off;
        const size_t len = span(l, &off);
        e = cudaStreamWaitEvent(p->in[l], p->ev_comp[b], 0);
        if (e == cudaSuccess && len)
            e = cudaMemcpyAsync((char*)p->dW[b] + off, (const char*)W_host + off, len, cudaMemcpyHostToDevice,
                                p->in[l]);
        if (e == cudaSuccess)
            e = cudaEventRecord(p->ev_in[b][l], p->in[l]);
        if (e != cudaSuccess)
            return cuda_fail(e);
    }
    // the solve, on s: after the copy in and after the pair's M was copied out
    for (int l = 0; l < PIPE_LANES && e == cudaSuccess; ++l)
        if ((e = cudaStreamWaitEvent(cs, p->ev_in[b][l], 0)) == cudaSuccess)
            e = cudaStreamWaitEvent(cs, p->ev_out[b][l], 0);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if ((st = solve_impl(p->dW[b], n, (int)dt, p->dM[b], cs, false)) != APPD_OK)
        return st;
    if ((e = cudaEventRecord(p->ev_comp[b], cs)) != cudaSuccess)
        return cuda_fail(e);
    for (int l = 0; l < PIPE_LANES; ++l) {
        size_t off;
        const size_t len = span(l, &off);
        e = cudaStreamWaitEvent(p->out[l], p->ev_comp[b], 0);
        if (e == cudaSuccess && len)
            e = cudaMemcpyAsync((char*)M_host + off, (const char*)p->dM[b] + off, len, cudaMemcpyDeviceToHost,
                                p->out[l]);
        if (e == cudaSuccess)
            e = cudaEventRecord(p->ev_out[b][l], p->out[l]);
        if (e != cudaSuccess)
            return cuda_fail(e);
    }
    return APPD_OK;
}

appd_status appd_solve_host_wait(appd_stream_t s)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return APPD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe* p = g_pipe[dev];
    if (!p)
        return APPD_OK;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        for (int l = 0; l < PIPE_LANES && e == cudaSuccess; ++l)
            e = cudaStreamWaitEvent((cudaStream_t)s, p->ev_out[b][l], 0);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_insert_vertex(const void* M, int64_t n, appd_dtype dt, const void* w, void* M_out,
                               appd_stream_t s)
{
    if (n < 0 || (n > 0 && (!M || !w)) || !M_out || !dtype_ok((int)dt))
        return APPD_ERR_INVALID;
    if (n + 1 > (int64_t)MAX_N)
        return APPD_ERR_TOO_LARGE;
    const char* o = (const char*)M_out;
    const size_t ob = (size_t)(n + 1) * (size_t)(n + 1) * 4;
    auto overlaps = [&](const void* p, size_t bytes) {
        const char* a = (const char*)p;
        return a < o + ob && o < a + bytes;
    };
    if (overlaps(M, (size_t)n * (size_t)n * 4) || overlaps(w, (size_t)n * 4))
        return APPD_ERR_ALIAS;
    std::lock_guard<std::mutex> lk(g_mu);
    SolveCtx c;
    appd_status st = prepare(n > 0 ? n : 1, c);
    if (st != APPD_OK)
        return st;
    cudaError_t e = run_insert(M, n, (int)dt, w, M_out, c.ws->hook, c.ws->sms, (cudaStream_t)s);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_insert_vertex_tree(const uint32_t* keys, const uint32_t* lo, const uint32_t* hi,
                                    int64_t n, appd_dtype dt, const void* w, void* M_out,
                                    uint32_t* keys_out, uint32_t* lo_out, uint32_t* hi_out,
                                    appd_stream_t s)
{
    const bool outs = keys_out || lo_out || hi_out;
    if (n < 0 || !M_out || !dtype_ok((int)dt) || (n > 0 && !w) || (n > 1 && (!keys || !lo || !hi)) ||
        (outs && n > 0 && (!keys_out || !lo_out || !hi_out)))
        return APPD_ERR_INVALID;
    if (n + 1 > (int64_t)MAX_N)
        return APPD_ERR_TOO_LARGE;
    {
        const char* o = (const char*)M_out;
        const size_t ob = (size_t)(n + 1) * (size_t)(n + 1) * 4;
        auto overlaps = [&](const void* p, size_t bytes) {
            const char* a = (const char*)p;
            return p && a < o + ob && o < a + bytes;
        };
        const size_t eb = (size_t)(n > 0 ? n - 1 : 0) * 4;
        if (overlaps(w, (size_t)n * 4) || overlaps(keys, eb) || overlaps(lo, eb) || overlaps(hi, eb) ||
            overlaps(keys_out, (size_t)n * 4) || overlaps(lo_out, (size_t)n * 4) || overlaps(hi_out, (size_t)n * 4))
            return APPD_ERR_ALIAS;
    }
    cudaStream_t cs = (cudaStream_t)s;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(M_out, 0, 4, cs);
        return e == cudaSuccess ? APPD_OK : cuda_fail(e);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    SolveCtx c;
    appd_status st;
    if ((st = prepare(n + 1, c)) != APPD_OK)
        return st;
    Workspace& ws = *c.ws;
    cudaError_t e = run_insert_tree(ws, keys, lo, hi, (const u32*)w, (u32)n, (int)dt, c.status, cs);
    set_sizes(ws, n + 1);
    g_last_ctr = ws.ctr;
    if (e == cudaSuccess) {
        prof_begin(PH_LEAF, cs);
        e = run_leaf_order(ws, c.status, cs);
        prof_end(PH_LEAF, cs);
        prof_launches(1);
    }
    if (e == cudaSuccess) {
        prof_begin(PH_FILL, cs);
        e = run_fill(ws, (int)dt, M_out, cs);
        prof_end(PH_FILL, cs);
        prof_launches(1);
    }
    if (e == cudaSuccess && outs)
        e = launch_mst_split(ws.mst, (u32)(n + 1), keys_out, lo_out, hi_out, cs);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_mst(const void* W, int64_t n, appd_dtype dt, uint64_t* edges_out, appd_stream_t s)
{
    appd_status st = check_args(W, n, (int)dt, edges_out);
    if (st == APPD_ERR_ALIAS)
        st = APPD_OK;
    if (st == APPD_OK && n > (int64_t)SHORT_N)
        st = APPD_ERR_TOO_LARGE;   // the endpoints of this format have 16 bits
    if (st != APPD_OK || n <= 1)
        return st;
    std::lock_guard<std::mutex> lk(g_mu);
    SolveCtx c;
    if ((st = prepare(n, c)) != APPD_OK)
        return st;
    if ((st = ensure_cscratch(*c.ws, n)) != APPD_OK)
        return st;
    if ((st = mst_and_order(c, W, n, (int)dt, c.ws->cscratch, false, (cudaStream_t)s)) != APPD_OK)
        return st;
    // up to SHORT_N vertices the packed edges already are key << 32 | lo << 16 | hi
    cudaError_t e = cudaMemcpyAsync(edges_out, c.ws->mst, (size_t)(n - 1) * 8,
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)s);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_mst_edges(const void* W, int64_t n, appd_dtype dt, uint32_t* keys, uint32_t* lo,
                           uint32_t* hi, appd_stream_t s)
{
    if (n < 0 || !W || !dtype_ok((int)dt) || (n > 1 && (!keys || !lo || !hi)))
        return APPD_ERR_INVALID;
    if (n > (int64_t)MAX_N)
        return APPD_ERR_TOO_LARGE;
    if (n <= 1)
        return APPD_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    SolveCtx c;
    appd_status st;
    if ((st = prepare(n, c)) != APPD_OK)
        return st;
    if ((st = ensure_cscratch(*c.ws, n)) != APPD_OK)
        return st;
    if ((st = mst_and_order(c, W, n, (int)dt, c.ws->cscratch, false, (cudaStream_t)s)) != APPD_OK)
        return st;
    cudaError_t e = launch_mst_split(c.ws->mst, (u32)n, keys, lo, hi, (cudaStream_t)s);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_leaf_order(const void* W, int64_t n, appd_dtype dt, uint32_t* pos_out,
                            uint32_t* gap_out, appd_stream_t s)
{
    if (n < 0 || !W || !pos_out || (n > 1 && !gap_out) || !dtype_ok((int)dt))
        return APPD_ERR_INVALID;
    if (n > (int64_t)MAX_N)
        return APPD_ERR_TOO_LARGE;
    if (n == 0)
        return APPD_OK;
    cudaStream_t cs = (cudaStream_t)s;
    if (n == 1) {
        cudaError_t e = cudaMemsetAsync(pos_out, 0, 4, cs);
        return e == cudaSuccess ? APPD_OK : cuda_fail(e);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    SolveCtx c;
    appd_status st;
    if ((st = prepare(n, c)) != APPD_OK)
        return st;
    if ((st = ensure_cscratch(*c.ws, n)) != APPD_OK)
        return st;
    if ((st = mst_and_order(c, W, n, (int)dt, c.ws->cscratch, true, cs)) != APPD_OK)
        return st;
    cudaError_t e = cudaMemcpyAsync(pos_out, c.ws->pos, (size_t)n * 4, cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(gap_out, c.ws->gap, (size_t)(n - 1) * 4, cudaMemcpyDeviceToDevice, cs);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_solve_batched(const int64_t* offsets, const void* Ws, const int64_t* ns,
                               const uint8_t* dts, void* Ms, int32_t count, appd_stream_t s)
{
    if (count < 0 || (count > 0 && (!offsets || !ns || !Ws || !Ms)))
        return APPD_ERR_INVALID;
    for (int32_t g = 0; g < count; ++g) {
        if (ns[g] < 0 || offsets[g] < 0)
            return APPD_ERR_INVALID;
        if (ns[g] > (int64_t)MAX_N)
            return APPD_ERR_TOO_LARGE;
        if (dts && !dtype_ok(dts[g]))
            return APPD_ERR_INVALID;
    }
    if (Ws != Ms) {
        for (int32_t g = 0; g < count; ++g) {
            const u32* W = (const u32*)Ws + offsets[g];
            const u32* M = (const u32*)Ms + offsets[g];
            const size_t bytes = (size_t)ns[g] * (size_t)ns[g] * 4;
            if ((const char*)W < (const char*)M + bytes && (const char*)M < (const char*)W + bytes)
                return APPD_ERR_ALIAS;
        }
    }
    BatchTuning tune;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        tune = g_tune;
    }
    BatchDesc d;
    for (int32_t g = 0; g < count; ++g) {
        if (ns[g] == 0)
            continue;
        const u32* W = (const u32*)Ws + offsets[g];
        u32* M = (u32*)Ms + offsets[g];
        const uint8_t dt = dts ? dts[g] : (uint8_t)APPD_F32;
        if (ns[g] <= tune.n_split) {
            d.w.push_back(W);
            d.m.push_back(M);
            d.n.push_back((u32)ns[g]);
            d.dt.push_back(dt);
        } else {
            appd_status st = appd_solve(W, ns[g], (appd_dtype)dt, M, s);
            if (st != APPD_OK)
                return st;
        }
    }
    if (d.n.empty())
        return APPD_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    u32* status = nullptr;
    appd_status st;
    if ((st = get_status(&status)) != APPD_OK)
        return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return APPD_ERR_CUDA;
    const int64_t nmax = *std::max_element(d.n.begin(), d.n.end());
    BatchRuntime*& rt = g_brt[dev];
    if (!rt || batch_runtime_cap(rt) < nmax || !(g_brt_tune[dev] == tune)) {
        batch_runtime_destroy(rt);
        rt = nullptr;
        cudaError_t e = batch_runtime_create(nmax, tune, &rt);
        if (e != cudaSuccess)
            return cuda_fail(e);
        g_brt_tune[dev] = tune;
    }
    cudaError_t e = batch_launch(*rt, d, status, (cudaStream_t)s, true);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_batched_tuning(int32_t ctas_per_sm, int32_t fill_rows, int64_t n_split)
{
    if (ctas_per_sm < 1 || ctas_per_sm > 2 || fill_rows < 64 || fill_rows > 2048 ||
        (fill_rows & (fill_rows - 1)) != 0 ||
        n_split < 1 || n_split > 65536)
        return APPD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune.ctas_per_sm = ctas_per_sm;
    g_tune.fill_rows = fill_rows;
    g_tune.n_split = n_split;
    return APPD_OK;
}

appd_status appd_batched_prim_max(int32_t prim_max)
{
    if (prim_max < 0 || prim_max > 512)
        return APPD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune.prim_max = (u32)prim_max;
    return APPD_OK;
}

appd_status appd_batched_get_prim_max(int32_t* prim_max)
{
    if (!prim_max)
        return APPD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    *prim_max = (int32_t)g_tune.prim_max;
    return APPD_OK;
}

appd_status appd_check_symmetric(const void* W, int64_t n, appd_dtype dt, appd_stream_t s)
{
    if (n < 0 || !W || !dtype_ok((int)dt))
        return APPD_ERR_INVALID;
    if (n > (int64_t)MAX_N)
        return APPD_ERR_TOO_LARGE;
    if (n <= 1)
        return APPD_OK;
    u32* status = nullptr;
    appd_status st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if ((st = get_status(&status)) != APPD_OK)
            return st;
    }
    cudaStream_t cs = (cudaStream_t)s;
    u32* flag = status + 16;   // scratch word next to the status word
    cudaError_t e = cudaMemsetAsync(flag, 0, 4, cs);
    if (e != cudaSuccess)
        return cuda_fail(e);
    k_check_sym<<<1024, 256, 0, cs>>>((const u32*)W, (u32)n, flag);
    u32 h = 0;
    e = cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess)
        return cuda_fail(e);
    return h ? APPD_ERR_ASYMMETRIC : APPD_OK;
}

appd_status appd_probe_bounded_wait(int32_t limit_ms, appd_stream_t s)
{
    if (limit_ms < 1 || limit_ms > 10000)
        return APPD_ERR_INVALID;
    u32* status = nullptr;
    appd_status st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if ((st = get_status(&status)) != APPD_OK)
            return st;
    }
    cudaStream_t cs = (cudaStream_t)s;
    GridBar* bar = reinterpret_cast<GridBar*>(status + 32);   // scratch words of the status block
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), cs);
    if (e != cudaSuccess)
        return cuda_fail(e);
    void* args[] = {&bar, &status, nullptr};
    u64 lim = (u64)limit_ms * 1000000ull;
    args[2] = &lim;
    e = cudaLaunchCooperativeKernel((const void*)k_wait_probe, dim3(2), dim3(32), args, 0, cs);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_last_device_status(appd_stream_t s)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    u32* status = nullptr;
    appd_status st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if ((st = get_status(&status)) != APPD_OK)
            return st;
    }
    u32 h = 0;
    // the library's status word, and the one that appd_solve_noalloc keeps
    // in its static array (it allocates nothing, so it cannot share ours)
    int dev = 0;
    cudaGetDevice(&dev);
    u32* words[2] = {status, noalloc_status_word(dev)};
    for (u32* wp : words) {
        if (!wp)
            continue;
        u32 x = 0;
        e = cudaMemcpy(&x, wp, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return cuda_fail(e);
        if (x) {
            e = cudaMemset(wp, 0, 4);
            if (e != cudaSuccess)
                return cuda_fail(e);
        }
        h |= x;
    }
    if (h & DEV_TIMEOUT)
        return APPD_ERR_TIMEOUT;
    if (h & DEV_INTERNAL)
        return APPD_ERR_INTERNAL;
    return APPD_OK;
}

appd_status appd_debug_mark_failed(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return APPD_ERR_CUDA;
    cudaError_t e = cudaDeviceSynchronize();
    const u32 one = 1u;
    if (e == cudaSuccess && g_ws[dev])
        e = cudaMemcpy(&g_ws[dev]->ctr->bar.failed, &one, sizeof(u32), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = batch_runtime_mark_failed(g_brt[dev]);
    if (e == cudaSuccess)
        e = noalloc_mark_failed(dev);
    return e == cudaSuccess ? APPD_OK : cuda_fail(e);
}

appd_status appd_release_workspaces(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return APPD_ERR_CUDA;
    cudaDeviceSynchronize();
    if (g_ws[dev]) {
        workspace_destroy(g_ws[dev]);
        g_ws[dev] = nullptr;
    }
    batch_runtime_destroy(g_brt[dev]);
    g_brt[dev] = nullptr;
    {
        std::lock_guard<std::mutex> lp(g_pipe_mu);
        pipe_destroy(g_pipe[dev]);
        g_pipe[dev] = nullptr;
    }
    return APPD_OK;
}

}  // extern "C"
