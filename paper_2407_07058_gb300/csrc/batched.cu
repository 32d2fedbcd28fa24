// batched.cu -- many independent graphs through one persistent launch.
//
// Graphs up to a size cut-over are solved one per CTA: a persistent grid
// (a few CTAs per SM) pops graph indices from an atomic work queue, largest
// first, and runs the whole pipeline of a single solve inside the CTA --
// round-1 row minima, the Boruvka rounds (the same component bookkeeping and
// contraction items as the single-solve kernels, with block-wide barriers
// instead of grid barriers), the leaf order, and the tiled fill.  Each CTA
// owns a workspace slice; each graph's M buffer is its contraction scratch.
// Larger graphs in a batch go through the multi-CTA single-solve pipeline.
// A batch's launch sequence (queue reset + kernel) is captured once into a
// CUDA graph and replayed for repeated batches with the same layout.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "fill_device.cuh"
#include "leaf_device.cuh"
#include "mst_device.cuh"

namespace appd {

// Device view of one CTA's workspace slice.
struct SliceWs {
    Counters* ctr;
    u32* part;
    u64 *best0, *best1;
    u32 *comp, *hook, *par, *flag, *rootid, *label, *cnt, *fillc, *gstart, *members, *nchunk,
        *chunk_start, *item_group;
    u64* mst;
    u32 *deg, *adj_off, *afill, *adj, *aslot, *lr_d0, *lr_d1, *lr_nx0, *lr_nx1, *parent, *pe_key;
    u64* ord;
    u32* jump;
    u64* mxo;
    u32* nha;
    u64 *skey0, *skey1;
    u32 *hist, *first_child, *next_sib, *pos, *order, *nsize, *gap, *st;
    u64* cscratch;   // contraction matrices for in-place graphs (M == W), or null
};

struct BatchArgs {
    const u32* const* wp;   // per-graph W (device pointers)
    u32* const* mp;         // per-graph M
    const u32* ns;          // per-graph n
    const uint8_t* dts;     // per-graph dtype
    const u32* queue;       // graph indices, largest first
    u32 count;
    u32* next;              // work-queue head
    SliceWs* slices;
    u32* status;
    u32 bin_cap;          // u64 bins that fit the dynamic shared memory
    u32 fill_rows;        // rows per fill tile
};

constexpr int BATCH_THREADS = 512;

// Round-1 row minima of one graph by one CTA (each warp a row).
template <int DT>
__device__ void rowmin_cta(const u32* __restrict__ W, u32 n, u64* __restrict__ best)
{
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (u32 i = w; i < n; i += nw) {
        const u32* r = W + (size_t)i * n;
        u64 m = EDGE_INF;
        u32 j = lane;
        for (; j + 96 < n; j += 128) {
            const u32 b0 = ld_stream_u32(r + j), b1 = ld_stream_u32(r + j + 32);
            const u32 b2 = ld_stream_u32(r + j + 64), b3 = ld_stream_u32(r + j + 96);
            const u64 c0 = ((u64)key_of(b0, DT) << 32) | j, c1 = ((u64)key_of(b1, DT) << 32) | (j + 32);
            const u64 c2 = ((u64)key_of(b2, DT) << 32) | (j + 64), c3 = ((u64)key_of(b3, DT) << 32) | (j + 96);
            if (j != i && c0 < m) m = c0;
            if (j + 32 != i && c1 < m) m = c1;
            if (j + 64 != i && c2 < m) m = c2;
            if (j + 96 != i && c3 < m) m = c3;
        }
        for (; j < n; j += 32) {
            const u64 c = ((u64)key_of(ld_stream_u32(r + j), DT) << 32) | j;
            if (j != i && c < m)
                m = c;
        }
        m = warp_min_u64(m);
        if (lane == 0)
            best[i] = pack_edge((u32)(m >> 32), i, (u32)m & 0xFFFFu);
    }
}

template <int DT>
__device__ void solve_one(const SliceWs& w, const u32* W, u32* M, u32 n, const BatchArgs& b,
                          unsigned char* smem, u32* s_rows, u64* s_red)
{
    BlockTeam t;
    const u32 tid = threadIdx.x;
    if (n == 1) {
        if (tid == 0)
            M[0] = 0u;
        __syncthreads();
        return;
    }
    Counters* ctr = w.ctr;
    for (u32 v = tid; v < n; v += blockDim.x)
        w.comp[v] = v;
    if (tid == 0) {
        for (int i = 0; i < MAX_LEVELS + 2; ++i)
            ctr->c[i] = 0;
        ctr->c[0] = n;
        ctr->done = 0;
        ctr->mst_count = 0;
        ctr->jump_flag[0] = ctr->jump_flag[1] = ctr->jump_flag[2] = 0;
    }
    rowmin_cta<DT>(W, n, w.best0);
    __syncthreads();

    // contraction scratch: M (16-byte aligned start) unless solving in place
    const u32 h = n / 2;
    u64* cb0 = (M == W) ? w.cscratch : (u64*)(((uintptr_t)M + 15) & ~(uintptr_t)15);
    u64* cb1 = (u64*)((char*)cb0 + (((size_t)h * h * sizeof(u64) + 15) & ~(size_t)15));
    const bool vec = (n % 4 == 0) && (((uintptr_t)W & 15u) == 0);
    const int levels = ceil_log2_dev(n);
    for (int r = 0; r < levels; ++r) {
        StepArgs sa;
        sa.level = r;
        sa.n = n;
        sa.best_in = (r & 1) ? w.best1 : w.best0;
        sa.best_out = (r & 1) ? w.best0 : w.best1;
        sa.comp = w.comp;
        sa.hook = w.hook;
        sa.par = w.par;
        sa.flag = w.flag;
        sa.rootid = w.rootid;
        sa.label = w.label;
        sa.cnt = w.cnt;
        sa.fillc = w.fillc;
        sa.gstart = w.gstart;
        sa.members = w.members;
        sa.nchunk = w.nchunk;
        sa.chunk_start = w.chunk_start;
        sa.item_group = w.item_group;
        sa.mst = w.mst;
        sa.cnext = (r & 1) ? cb1 : cb0;
        sa.part = w.part;
        sa.ctr = ctr;
        sa.status = b.status;
        sa.bin_cap = b.bin_cap;
        step_body(t, sa);
        __syncthreads();
        if (*(volatile u32*)&ctr->done)
            break;
        ContractArgs ca;
        ca.level = r;
        ca.cin = (r == 0) ? (const void*)W : (const void*)((r & 1) ? cb0 : cb1);
        ca.cout = (r & 1) ? cb1 : cb0;
        ca.best_out = sa.best_out;
        ca.label = w.label;
        ca.members = w.members;
        ca.gstart = w.gstart;
        ca.nchunk = w.nchunk;
        ca.chunk_start = w.chunk_start;
        ca.item_group = w.item_group;
        ca.ctr = ctr;
        ca.bin_cap = b.bin_cap;
        const u32 cr = ((volatile u32*)ctr->c)[r], cn = ((volatile u32*)ctr->c)[r + 1];
        const u32 tc = *(volatile u32*)&ctr->total_chunks;
        const u32 total = tc * *(volatile u32*)&ctr->nbr;
        u64* bins = reinterpret_cast<u64*>(smem);
        for (u32 item = 0; item < total; ++item) {
            if (r == 0) {
                if (vec)
                    contract_item<DT, 1, true>(ca, item, cr, cn, tc, bins, s_rows, s_red);
                else
                    contract_item<DT, 1, false>(ca, item, cr, cn, tc, bins, s_rows, s_red);
            } else {
                contract_item<DT, 0, false>(ca, item, cr, cn, tc, bins, s_rows, s_red);
            }
        }
        __syncthreads();
    }

    LeafArgs la;
    la.n = n;
    la.levels = levels;
    int stl = 1;
    while ((1u << stl) <= n - 1)
        ++stl;
    la.st_levels = stl;
    la.mst = w.mst;
    la.deg = w.deg;
    la.adj_off = w.adj_off;
    la.afill = w.afill;
    la.adj = w.adj;
    la.aslot = w.aslot;
    la.lr_d0 = w.lr_d0;
    la.lr_d1 = w.lr_d1;
    la.lr_nx0 = w.lr_nx0;
    la.lr_nx1 = w.lr_nx1;
    la.parent = w.parent;
    la.pe_key = w.pe_key;
    la.ord = w.ord;
    la.jump = w.jump;
    la.mxo = w.mxo;
    la.nha = w.nha;
    la.skey0 = w.skey0;
    la.skey1 = w.skey1;
    la.hist = w.hist;
    la.ntiles = (n - 1 + 2047) / 2048;
    la.first_child = w.first_child;
    la.next_sib = w.next_sib;
    la.pos = w.pos;
    la.order = w.order;
    la.nsize = w.nsize;
    la.gap = w.gap;
    la.st = w.st;
    la.part = w.part;
    la.ctr = ctr;
    la.status = b.status;
    leaf_body(t, la);
    __syncthreads();

    const u32 fr = b.fill_rows;
    for (u32 j0 = 0; j0 < n; j0 += FC)
        for (u32 r0 = 0; r0 < n; r0 += fr)
            fill_tile<DT>(w.pos, w.st, n, j0, r0, min(fr, n - r0), fr, M, smem);
}

__global__ void __launch_bounds__(BATCH_THREADS, 1) k_batched(BatchArgs b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u32 s_q;
    __shared__ u32 s_rows[CONTRACT_ROWS];
    __shared__ u64 s_red[32];
    const SliceWs& w = b.slices[blockIdx.x];   // fields are read on use (cached)
    for (;;) {
        if (threadIdx.x == 0)
            s_q = atomicAdd(b.next, 1u);
        __syncthreads();
        const u32 q = s_q;
        __syncthreads();
        if (q >= b.count)
            break;
        const u32 g = b.queue[q];
        const u32 n = b.ns[g];
        const u32* W = b.wp[g];
        u32* M = b.mp[g];
        if (n == 0)
            continue;
        if (b.dts[g] == 1)
            solve_one<1>(w, W, M, n, b, smem, s_rows, s_red);
        else
            solve_one<0>(w, W, M, n, b, smem, s_rows, s_red);
    }
}

// ------------------------------------------------------------------ host
struct BatchRuntime {
    int device = -1;
    int sms = 0;
    int nslices = 0;
    int64_t cap = 0;
    BatchTuning tune;
    void* slice_mem = nullptr;
    SliceWs* d_slices = nullptr;
    void* scratch_mem = nullptr;   // per-slice contraction scratch for in-place graphs
    u32* d_next = nullptr;
    void* d_desc = nullptr;        // descriptors of the uncached launch path
    size_t desc_bytes = 0;
    size_t smem = 0;
    u32 bin_cap = 0;
    struct Plan {
        void* dev = nullptr;
        cudaGraphExec_t exec = nullptr;
    };
    std::map<std::vector<int64_t>, Plan> plans;
};

namespace {

SliceWs to_slice(const Workspace& w)
{
    SliceWs s;
    s.ctr = w.ctr;
    s.part = w.part;
    s.best0 = w.best[0];
    s.best1 = w.best[1];
    s.comp = w.comp;
    s.hook = w.hook;
    s.par = w.par;
    s.flag = w.flag;
    s.rootid = w.rootid;
    s.label = w.label;
    s.cnt = w.cnt;
    s.fillc = w.fillc;
    s.gstart = w.gstart;
    s.members = w.members;
    s.nchunk = w.nchunk;
    s.chunk_start = w.chunk_start;
    s.item_group = w.item_group;
    s.mst = w.mst;
    s.deg = w.deg;
    s.adj_off = w.adj_off;
    s.afill = w.afill;
    s.adj = w.adj;
    s.aslot = w.aslot;
    s.lr_d0 = w.lr_d[0];
    s.lr_d1 = w.lr_d[1];
    s.lr_nx0 = w.lr_nx[0];
    s.lr_nx1 = w.lr_nx[1];
    s.parent = w.parent;
    s.pe_key = w.pe_key;
    s.ord = w.ord;
    s.jump = w.jump;
    s.mxo = w.mxo;
    s.nha = w.nha;
    s.skey0 = w.skey[0];
    s.skey1 = w.skey[1];
    s.hist = w.hist;
    s.first_child = w.first_child;
    s.next_sib = w.next_sib;
    s.pos = w.pos;
    s.order = w.order;
    s.nsize = w.nsize;
    s.gap = w.gap;
    s.st = w.st;
    s.cscratch = nullptr;
    return s;
}

cudaError_t ensure_scratch(BatchRuntime& rt)
{
    if (rt.scratch_mem)
        return cudaSuccess;
    const size_t per = (contraction_scratch_bytes(rt.cap) + 255) & ~(size_t)255;
    cudaError_t e = cudaMalloc(&rt.scratch_mem, per * rt.nslices);
    if (e != cudaSuccess)
        return e;
    std::vector<SliceWs> hs(rt.nslices);
    e = cudaMemcpy(hs.data(), rt.d_slices, sizeof(SliceWs) * rt.nslices, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return e;
    for (int i = 0; i < rt.nslices; ++i)
        hs[i].cscratch = (u64*)((char*)rt.scratch_mem + per * i);
    return cudaMemcpy(rt.d_slices, hs.data(), sizeof(SliceWs) * rt.nslices, cudaMemcpyHostToDevice);
}

// descriptor block layout: wp | mp | ns | queue | dts
size_t desc_layout(u32 cnt, size_t off[5])
{
    off[0] = 0;
    off[1] = off[0] + 8 * (size_t)cnt;
    off[2] = off[1] + 8 * (size_t)cnt;
    off[3] = off[2] + 4 * (size_t)cnt;
    off[4] = off[3] + 4 * (size_t)cnt;
    return (off[4] + cnt + 255) & ~(size_t)255;
}

void fill_desc(const BatchDesc& d, std::vector<unsigned char>& host, const size_t off[5])
{
    const u32 cnt = (u32)d.n.size();
    std::vector<u32> q(cnt);
    std::iota(q.begin(), q.end(), 0u);
    std::stable_sort(q.begin(), q.end(), [&](u32 a, u32 b) { return d.n[a] > d.n[b]; });
    memcpy(host.data() + off[0], d.w.data(), 8 * cnt);
    memcpy(host.data() + off[1], d.m.data(), 8 * cnt);
    memcpy(host.data() + off[2], d.n.data(), 4 * cnt);
    memcpy(host.data() + off[3], q.data(), 4 * cnt);
    memcpy(host.data() + off[4], d.dt.data(), cnt);
}

BatchArgs make_args(const BatchRuntime& rt, void* dev, const size_t off[5], u32 cnt, u32* status)
{
    BatchArgs a;
    a.wp = (const u32* const*)((char*)dev + off[0]);
    a.mp = (u32* const*)((char*)dev + off[1]);
    a.ns = (const u32*)((char*)dev + off[2]);
    a.queue = (const u32*)((char*)dev + off[3]);
    a.dts = (const uint8_t*)((char*)dev + off[4]);
    a.count = cnt;
    a.next = rt.d_next;
    a.slices = rt.d_slices;
    a.status = status;
    a.bin_cap = rt.bin_cap;
    a.fill_rows = (u32)rt.tune.fill_rows;
    return a;
}

}  // namespace

cudaError_t batch_runtime_create(int64_t cap, const BatchTuning& tune, BatchRuntime** out)
{
    BatchRuntime* nr = new BatchRuntime();
    cudaError_t e = cudaGetDevice(&nr->device);
    if (e != cudaSuccess) {
        delete nr;
        return e;
    }
    cudaDeviceGetAttribute(&nr->sms, cudaDevAttrMultiProcessorCount, nr->device);
    int64_t c = 1024;
    while (c < cap)
        c *= 2;
    nr->cap = c;
    nr->tune = tune;
    nr->nslices = nr->sms * tune.ctas_per_sm;
    Workspace tmp;
    const size_t per = (workspace_layout(tmp, nullptr, c) + 255) & ~(size_t)255;
    if ((e = cudaMalloc(&nr->slice_mem, per * nr->nslices)) != cudaSuccess) {
        delete nr;
        return e;
    }
    std::vector<SliceWs> hs(nr->nslices);
    for (int i = 0; i < nr->nslices; ++i) {
        Workspace w;
        workspace_layout(w, (char*)nr->slice_mem + per * i, c);
        hs[i] = to_slice(w);
    }
    if ((e = cudaMalloc(&nr->d_slices, sizeof(SliceWs) * nr->nslices)) == cudaSuccess)
        e = cudaMemcpy(nr->d_slices, hs.data(), sizeof(SliceWs) * nr->nslices, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&nr->d_next, 256);
    // dynamic shared memory: the fill tile (the contraction bins fit inside it)
    nr->smem = fill_smem_bytes((u32)tune.fill_rows);
    nr->bin_cap = (u32)(nr->smem / sizeof(u64));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nr->smem);
    if (e != cudaSuccess) {
        batch_runtime_destroy(nr);
        return e;
    }
    *out = nr;
    return cudaSuccess;
}

void batch_runtime_destroy(BatchRuntime* rt)
{
    if (!rt)
        return;
    cudaDeviceSynchronize();
    for (auto& kv : rt->plans) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaFree(kv.second.dev);
    }
    cudaFree(rt->slice_mem);
    cudaFree(rt->d_slices);
    cudaFree(rt->scratch_mem);
    cudaFree(rt->d_next);
    cudaFree(rt->d_desc);
    delete rt;
}

int64_t batch_runtime_cap(const BatchRuntime* rt) { return rt->cap; }

cudaError_t batch_launch(BatchRuntime& rt, const BatchDesc& d, u32* status, cudaStream_t s,
                         bool cache_graph)
{
    const u32 cnt = (u32)d.n.size();
    if (cnt == 0)
        return cudaSuccess;
    cudaError_t e;
    bool inplace = false;
    for (u32 i = 0; i < cnt; ++i)
        inplace |= (d.w[i] == (const void*)d.m[i]);
    if (inplace && (e = ensure_scratch(rt)) != cudaSuccess)
        return e;
    size_t off[5];
    const size_t bytes = desc_layout(cnt, off);
    std::vector<unsigned char> host(bytes);
    if (!cache_graph) {
        // one descriptor block per runtime: launches on the runtime are
        // ordered on its stream, so the next upload follows the last kernel
        if (rt.desc_bytes < bytes) {
            cudaFree(rt.d_desc);
            rt.d_desc = nullptr;
            rt.desc_bytes = 0;
            if ((e = cudaMalloc(&rt.d_desc, bytes)) != cudaSuccess)
                return e;
            rt.desc_bytes = bytes;
        }
        fill_desc(d, host, off);
        // pageable source: the copy is staged before the call returns
        if ((e = cudaMemcpyAsync(rt.d_desc, host.data(), bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(rt.d_next, 0, sizeof(u32), s)) != cudaSuccess)
            return e;
        BatchArgs a = make_args(rt, rt.d_desc, off, cnt, status);
        prof_launches(1);
        prof_begin(PH_BATCHED, s);
        k_batched<<<rt.nslices, BATCH_THREADS, rt.smem, s>>>(a);
        prof_end(PH_BATCHED, s);
        return cudaGetLastError();
    }
    std::vector<int64_t> key;
    key.reserve(4 * cnt + 1);
    key.push_back((int64_t)(uintptr_t)s);
    for (u32 i = 0; i < cnt; ++i) {
        key.push_back((int64_t)(uintptr_t)d.w[i]);
        key.push_back((int64_t)(uintptr_t)d.m[i]);
        key.push_back(d.n[i]);
        key.push_back(d.dt[i]);
    }
    auto it = rt.plans.find(key);
    if (it == rt.plans.end()) {
        BatchRuntime::Plan p;
        if ((e = cudaMalloc(&p.dev, bytes)) != cudaSuccess)
            return e;
        fill_desc(d, host, off);
        if ((e = cudaMemcpy(p.dev, host.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        BatchArgs a = make_args(rt, p.dev, off, cnt, status);
        cudaStream_t cap_s;
        if ((e = cudaStreamCreateWithFlags(&cap_s, cudaStreamNonBlocking)) != cudaSuccess)
            return e;
        cudaGraph_t graph;
        e = cudaStreamBeginCapture(cap_s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(rt.d_next, 0, sizeof(u32), cap_s);
            k_batched<<<rt.nslices, BATCH_THREADS, rt.smem, cap_s>>>(a);
            e = cudaStreamEndCapture(cap_s, &graph);
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&p.exec, graph, 0);
            cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cap_s);
        if (e != cudaSuccess) {
            cudaFree(p.dev);
            return e;
        }
        it = rt.plans.emplace(key, p).first;
    }
    prof_launches(1);
    prof_begin(PH_BATCHED, s);
    e = cudaGraphLaunch(it->second.exec, s);
    prof_end(PH_BATCHED, s);
    return e;
}

}  // namespace appd
