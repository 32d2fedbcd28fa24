// noalloc.cu -- a solve entry point that never allocates device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory
// budget enforced by someone else (a pre-sized pool, an arena owned by a
// framework), or an embedding that forbids the driver's allocator once it has
// started.  appd_solve_noalloc serves them for graphs up to NOALLOC_MAX_N
// vertices: it runs the one-CTA-per-graph solve of the batched kernel on a
// single CTA, with every scratch array (the workspace of the MST, leaf order
// and fill, the contraction matrices, a status word) carved from one
// file-scope device array that the library image carries.  The caller still
// passes W and M.
//
// Shared state, and what that means for callers:
//  - The array is one per device and shared by every call on that device;
//    it keeps the previous call's contents.  The kernel initialises every
//    field it reads before reading it (component labels, counters, degree and
//    bin arrays); nothing needs to be zero beforehand.
//  - Calls whose kernels overlap on the GPU (different streams without
//    ordering, or several host threads) race on the array.  Order them.
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and sets the kernel's
//    shared-memory limit; make that first call before any stream capture.
#include <mutex>

#include "../../include/appd.h"
#include "fill_device.cuh"
#include "leaf_device.cuh"
#include "mst_device.cuh"

namespace appd {

constexpr int64_t NOALLOC_MAX_N = 1024;
constexpr size_t NOALLOC_BYTES = (size_t)4 << 20;   // 4 MiB per device
constexpr int NOALLOC_THREADS = 512;
constexpr u32 NOALLOC_FILL_ROWS = 128;

// The scratch: a host-side name for a device array.  Host code must not pass
// `noalloc_scratch` itself to a kernel (it is not a device address); it uses
// the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char noalloc_scratch[NOALLOC_BYTES];

struct NoallocWs {
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
    u32 *sval0, *sval1;
    u32 *hist, *first_child, *next_sib, *pos, *order, *nsize, *gap, *st;
    u64* cscratch;   // contraction matrices (used when M == W)
    u32* status;     // device-detected errors of this entry point (sticky until
                     // appd_last_device_status reads and clears them)
};

// Round-1 row minima by one CTA (each warp a row); same result as the other
// round-1 kernels.
template <int DT>
__device__ void noalloc_rowmin(const u32* __restrict__ W, u32 n, u64* __restrict__ best)
{
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (u32 i = w; i < n; i += nw) {
        const u32* r = W + (size_t)i * n;
        u64 m = EDGE_INF;
        for (u32 j = lane; j < n; j += 32) {
            const u64 c = ((u64)key_of(r[j], DT) << 32) | j;
            if (j != i && c < m)
                m = c;
        }
        m = warp_min_u64(m);
        if (lane == 0)
            best[i] = pack_edge((u32)(m >> 32), i, (u32)m, n);
    }
}

template <int DT>
__device__ void noalloc_solve(const NoallocWs& w, const u32* W, u32* M, u32 n, unsigned char* smem,
                              u32 bin_cap, u32* s_rows, u64* s_red)
{
    BlockTeam t;
    const u32 tid = threadIdx.x;
    if (n == 1) {
        if (tid == 0)
            M[0] = 0u;
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
        // the control block lives in the shared array: a failure recorded by
        // an earlier call must not stop this one
        ctr->bar.count = 0;
        ctr->bar.abort = 0;
        ctr->bar.failed = 0;
    }
    noalloc_rowmin<DT>(W, n, w.best0);
    __syncthreads();
    const u32 h = n / 2;
    u64* cb0 = (M == W) ? w.cscratch : (u64*)(((uintptr_t)M + 15) & ~(uintptr_t)15);
    u64* cb1 = (u64*)((char*)cb0 + (((size_t)h * h * sizeof(u64) + 15) & ~(size_t)15));
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
        sa.status = w.status;
        sa.bin_cap = bin_cap;
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
        ca.bin_cap = bin_cap;
        const u32 cr = ((volatile u32*)ctr->c)[r], cn = ((volatile u32*)ctr->c)[r + 1];
        const u32 tc = *(volatile u32*)&ctr->total_chunks;
        const u32 total = tc * *(volatile u32*)&ctr->nbr;
        u64* bins = reinterpret_cast<u64*>(smem);
        for (u32 item = 0; item < total; ++item) {
            if (r == 0)
                contract_item<DT, 1, false>(ca, item, cr, cn, tc, bins, s_rows, s_red);
            else
                contract_item<DT, 0, false>(ca, item, cr, cn, tc, bins, s_rows, s_red);
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
    la.sval0 = w.sval0;
    la.sval1 = w.sval1;
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
    la.status = w.status;
    leaf_body(t, la);
    __syncthreads();
    if (solve_failed(&ctr->bar))   // no valid leaf order: leave M unwritten
        return;
    for (u32 j0 = 0; j0 < n; j0 += FC)
        for (u32 r0 = 0; r0 < n; r0 += NOALLOC_FILL_ROWS)
            fill_tile<DT>(w.pos, w.st, n, j0, r0, min(NOALLOC_FILL_ROWS, n - r0), NOALLOC_FILL_ROWS, M,
                          smem);
}

__global__ void __launch_bounds__(NOALLOC_THREADS, 1) k_solve_noalloc(NoallocWs w, const u32* W, u32* M,
                                                                     u32 n, int dt, u32 bin_cap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u32 s_rows[CONTRACT_ROWS];
    __shared__ u64 s_red[32];
    switch (dt) {
    case 1: noalloc_solve<1>(w, W, M, n, smem, bin_cap, s_rows, s_red); break;
    case 2: noalloc_solve<2>(w, W, M, n, smem, bin_cap, s_rows, s_red); break;
    case 3: noalloc_solve<3>(w, W, M, n, smem, bin_cap, s_rows, s_red); break;
    default: noalloc_solve<0>(w, W, M, n, smem, bin_cap, s_rows, s_red); break;
    }
}

namespace {

struct NoallocDev {
    bool ready = false;
    NoallocWs ws;
    size_t smem = 0;
};

std::mutex g_na_mu;
NoallocDev g_na[64];

// Once per device, with that device current: find the array's device
// address and lay the workspace out inside it.  No allocation.
cudaError_t noalloc_setup(int dev, NoallocDev& d)
{
    void* base = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base, noalloc_scratch);
    if (e != cudaSuccess)
        return e;
    Workspace w;
    const size_t ws_bytes = (workspace_layout(w, nullptr, NOALLOC_MAX_N) + 255) & ~(size_t)255;
    const size_t cs_bytes = (contraction_scratch_bytes(NOALLOC_MAX_N) + 255) & ~(size_t)255;
    if (ws_bytes + cs_bytes + 256 > NOALLOC_BYTES)
        return cudaErrorInvalidValue;   // layout does not fit the array (a build error)
    workspace_layout(w, (char*)base, NOALLOC_MAX_N);
    NoallocWs& s = d.ws;
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
    s.sval0 = w.sval[0];
    s.sval1 = w.sval[1];
    s.hist = w.hist;
    s.first_child = w.first_child;
    s.next_sib = w.next_sib;
    s.pos = w.pos;
    s.order = w.order;
    s.nsize = w.nsize;
    s.gap = w.gap;
    s.st = w.st;
    s.cscratch = (u64*)((char*)base + ws_bytes);
    s.status = (u32*)((char*)base + ws_bytes + cs_bytes);
    d.smem = fill_smem_bytes(NOALLOC_FILL_ROWS);
    e = cudaFuncSetAttribute(k_solve_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.smem);
    if (e != cudaSuccess)
        return e;
    (void)dev;
    d.ready = true;
    return cudaSuccess;
}

}  // namespace

cudaError_t noalloc_mark_failed(int dev)
{
    if (dev < 0 || dev >= 64)
        return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na[dev].ready)
        return cudaSuccess;
    const u32 one = 1u;
    return cudaMemcpy(&g_na[dev].ws.ctr->bar.failed, &one, sizeof(u32), cudaMemcpyHostToDevice);
}

// The status word of this device's no-allocation array, or null before the
// first appd_solve_noalloc on the device (nothing has been recorded then).
u32* noalloc_status_word(int dev)
{
    if (dev < 0 || dev >= 64)
        return nullptr;
    std::lock_guard<std::mutex> lk(g_na_mu);
    return g_na[dev].ready ? g_na[dev].ws.status : nullptr;
}

}  // namespace appd

using namespace appd;

extern "C" appd_status appd_solve_noalloc(const void* W, int64_t n, appd_dtype dt, void* M,
                                          appd_stream_t s)
{
    if (n < 0 || !W || !M || !dtype_ok((int)dt))
        return APPD_ERR_INVALID;
    if (n > NOALLOC_MAX_N)
        return APPD_ERR_TOO_LARGE;   // the static scratch is sized for NOALLOC_MAX_N vertices
    if (M != W) {
        const char* a = (const char*)W;
        const char* b = (const char*)M;
        const size_t bytes = (size_t)n * (size_t)n * 4;
        if (a < b + bytes && b < a + bytes)
            return APPD_ERR_ALIAS;
    }
    if (n == 0)
        return APPD_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return APPD_ERR_CUDA;
    NoallocDev* d = &g_na[dev];
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!d->ready && noalloc_setup(dev, *d) != cudaSuccess)
            return APPD_ERR_CUDA;
    }
    const u32 bin_cap = (u32)(d->smem / sizeof(u64));
    k_solve_noalloc<<<1, NOALLOC_THREADS, d->smem, (cudaStream_t)s>>>(d->ws, (const u32*)W, (u32*)M,
                                                                      (u32)n, (int)dt, bin_cap);
    return cudaGetLastError() == cudaSuccess ? APPD_OK : APPD_ERR_CUDA;
}
