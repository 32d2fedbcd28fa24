// mst_kernels.cu -- dense Boruvka minimum spanning tree of the complete graph.
//
// The paper builds the MST with Prim's algorithm in O(n^2) (Section 3).  Prim
// is n sequential steps; on the GPU we use Boruvka instead, which reaches the
// same tree (the MST is unique under the packed-edge order):
//   round 1  (k_rowmin)   best[i] = min over j != i of packed(i, j)
//   each round (k_step)   hook every component to the other end of its best
//                         edge, break mutual pairs, pointer-jump to roots,
//                         relabel, record the new MST edges, group the rows
//                         of the current matrix by new component
//   contraction (k_contract_*)  C_{r+1}(A,B) = min over rows a in A and
//                         columns b in B (b's component != A) of C_r(a,b);
//                         C_0 is W itself.  The same pass gives the next
//                         round's best[A] = min over B of C_{r+1}(A,B).
// The round count is data dependent (<= ceil(log2 n)); the host enqueues the
// maximum number of rounds and finished rounds exit at once, so a solve is a
// fixed launch sequence with no host synchronisation.
#include <cooperative_groups.h>

#include "mst_device.cuh"

namespace appd {

int ceil_log2(int64_t x)
{
    int l = 0;
    while ((int64_t(1) << l) < x)
        ++l;
    return l;
}

// ------------------------------------------------------------ round 1 (K1)
// One CTA per row (grid-stride).  The tie-break inside one row is "smaller
// column wins", which equals the packed order for a fixed row.
template <int DT, bool VEC>
__global__ void __launch_bounds__(256) k_rowmin(const u32* __restrict__ W, u32 n,
                                                u64* __restrict__ best)
{
    __shared__ u64 sh[32];
    for (u32 row = blockIdx.x; row < n; row += gridDim.x) {
        const u32* r = W + (size_t)row * n;
        u64 m = EDGE_INF;
        auto take = [&](u32 bits, u32 j) {
            u64 c = ((u64)key_of(bits, DT) << 32) | j;
            if (j != row && c < m)
                m = c;
        };
        if (VEC) {
            const u32 n4 = n >> 2;
            u32 g = threadIdx.x;
            for (; g + 3 * 256 < n4; g += 4 * 256) {
                uint4 v0 = ld_stream_v4(r + 4 * g);
                uint4 v1 = ld_stream_v4(r + 4 * (g + 256));
                uint4 v2 = ld_stream_v4(r + 4 * (g + 512));
                uint4 v3 = ld_stream_v4(r + 4 * (g + 768));
                take(v0.x, 4 * g), take(v0.y, 4 * g + 1), take(v0.z, 4 * g + 2), take(v0.w, 4 * g + 3);
                u32 b1 = 4 * (g + 256);
                take(v1.x, b1), take(v1.y, b1 + 1), take(v1.z, b1 + 2), take(v1.w, b1 + 3);
                u32 b2 = 4 * (g + 512);
                take(v2.x, b2), take(v2.y, b2 + 1), take(v2.z, b2 + 2), take(v2.w, b2 + 3);
                u32 b3 = 4 * (g + 768);
                take(v3.x, b3), take(v3.y, b3 + 1), take(v3.z, b3 + 2), take(v3.w, b3 + 3);
            }
            for (; g < n4; g += 256) {
                uint4 v = ld_stream_v4(r + 4 * g);
                take(v.x, 4 * g), take(v.y, 4 * g + 1), take(v.z, 4 * g + 2), take(v.w, 4 * g + 3);
            }
            for (u32 j = 4 * n4 + threadIdx.x; j < n; j += 256)
                take(r[j], j);
        } else {
            for (u32 j = threadIdx.x; j < n; j += 256)
                take(ld_stream_u32(r + j), j);
        }
        m = block_min_u64(m, sh);
        if (threadIdx.x == 0)
            best[row] = pack_edge((u32)(m >> 32), row, (u32)m & 0xFFFFu);
    }
}

// Round 1 over the upper triangle only (K1, symmetric form).  W is
// symmetric, so element (i, j), i < j, is both a candidate for row i and for
// row j.  A CTA owns 128 rows x 1024 columns; each warp a 128-column slab.
// Lanes own 4 columns: their column minima over the CTA's rows give row j's
// candidates from rows i < j; per-row minima are warp reductions
// (redux.sync) merged across warps in shared memory.  Both go to best[] with 64-bit atomic minima on packed edges, so
// every unordered pair is read once (half of W).  best[] starts at +inf.
constexpr u32 RS_ROWS = 128, RS_COLS = 1024;

template <int DT>
__global__ void __launch_bounds__(256) k_rowmin_sym(const u32* __restrict__ W, u32 n,
                                                    u64* __restrict__ best)
{
    __shared__ u64 s_row[RS_ROWS];
    const u32 i0 = blockIdx.y * RS_ROWS, c0 = blockIdx.x * RS_COLS;
    if (c0 + RS_COLS - 1 <= i0 || i0 >= n || c0 >= n)   // no pair i < j in this tile
        return;
    const u32 w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (u32 r = threadIdx.x; r < RS_ROWS; r += blockDim.x)
        s_row[r] = EDGE_INF;
    __syncthreads();
    const u32 j = c0 + 128 * w + 4 * lane;   // this lane's first column (n % 4 == 0)
    const bool live = j < n;
    const u32 imax = min(n, i0 + RS_ROWS);
    // does any of this warp's columns need the j > i mask?
    const bool mask = (c0 + 128 * w) <= (imax - 1);
    u64 cm0 = EDGE_INF, cm1 = EDGE_INF, cm2 = EDGE_INF, cm3 = EDGE_INF;
    for (u32 pass = 0; pass < RS_ROWS / 32; ++pass) {
        const u32 ib = i0 + 32 * pass;
        if (ib >= imax)
            break;
        for (u32 r8 = 0; r8 < 32; r8 += 8) {
            // issue eight rows' loads before consuming any (memory-level parallelism)
            uint4 v[8];
#pragma unroll
            for (u32 q = 0; q < 8; ++q) {
                const u32 i = ib + r8 + q;
                if (live && i < imax)
                    v[q] = ld_stream_v4(W + (size_t)i * n + j);
            }
#pragma unroll
            for (u32 q = 0; q < 8; ++q) {
                const u32 r = r8 + q, i = ib + r;
                u64 rp = EDGE_INF;
                if (live && i < imax) {
                    const u32 k0 = key_of(v[q].x, DT), k1 = key_of(v[q].y, DT);
                    const u32 k2 = key_of(v[q].z, DT), k3 = key_of(v[q].w, DT);
                    const u64 e0 = ((u64)k0 << 32) | j, e1 = ((u64)k1 << 32) | (j + 1);
                    const u64 e2 = ((u64)k2 << 32) | (j + 2), e3 = ((u64)k3 << 32) | (j + 3);
                    const u64 f0 = ((u64)k0 << 32) | i, f1 = ((u64)k1 << 32) | i;
                    const u64 f2 = ((u64)k2 << 32) | i, f3 = ((u64)k3 << 32) | i;
                    const bool ok0 = !mask || j > i, ok1 = !mask || j + 1 > i;
                    const bool ok2 = !mask || j + 2 > i, ok3 = !mask || j + 3 > i;
                    if (ok0) { rp = e0 < rp ? e0 : rp; cm0 = f0 < cm0 ? f0 : cm0; }
                    if (ok1) { rp = e1 < rp ? e1 : rp; cm1 = f1 < cm1 ? f1 : cm1; }
                    if (ok2) { rp = e2 < rp ? e2 : rp; cm2 = f2 < cm2 ? f2 : cm2; }
                    if (ok3) { rp = e3 < rp ? e3 : rp; cm3 = f3 < cm3 ? f3 : cm3; }
                }
                // warp minimum of (key, column) for row i: smallest key, then the
                // smallest column among the lanes holding it
                const u32 rk = (u32)(rp >> 32);
                const u32 kmin = __reduce_min_sync(0xFFFFFFFFu, rk);
                const u32 jmin = __reduce_min_sync(0xFFFFFFFFu, rk == kmin ? (u32)rp : 0xFFFFFFFFu);
                if (lane == r && jmin != 0xFFFFFFFFu)
                    atomicMin(&s_row[32 * pass + r], ((u64)kmin << 32) | jmin);
            }
        }
    }
    // column candidates: edge (i, j) with i the smallest-key row (ties: lower i)
    if (live) {
        if (cm0 != EDGE_INF) atomicMin(&best[j], pack_edge((u32)(cm0 >> 32), (u32)cm0, j));
        if (cm1 != EDGE_INF) atomicMin(&best[j + 1], pack_edge((u32)(cm1 >> 32), (u32)cm1, j + 1));
        if (cm2 != EDGE_INF) atomicMin(&best[j + 2], pack_edge((u32)(cm2 >> 32), (u32)cm2, j + 2));
        if (cm3 != EDGE_INF) atomicMin(&best[j + 3], pack_edge((u32)(cm3 >> 32), (u32)cm3, j + 3));
    }
    __syncthreads();
    for (u32 r = threadIdx.x; r < RS_ROWS && i0 + r < n; r += blockDim.x) {
        u64 x = s_row[r];
        if (x != EDGE_INF)
            atomicMin(&best[i0 + r], pack_edge((u32)(x >> 32), i0 + r, (u32)x));
    }
}

__global__ void k_step(StepArgs a)
{
    GridTeam t{&a.ctr->bar, a.status};
    step_body(t, a);
}

// Work loop of the contraction: each CTA takes items (a group A, a chunk of
// at most CONTRACT_ROWS of its rows, a range of bins), reduces every column
// of those rows into shared-memory bins indexed by the column's new
// component, and writes the bins as row A of C_{r+1} (plain stores when one
// item covers the group, atomic minima otherwise) together with the row's
// minimum, the next round's best edge of A.
template <int DT, int LEVEL0, bool VEC>
__global__ void __launch_bounds__(CONTRACT_THREADS, 1) k_contract(ContractArgs a)
{
    extern __shared__ __align__(16) u64 bins[];
    __shared__ u32 s_item, s_rows[CONTRACT_ROWS];
    __shared__ u64 s_red[32];
    Counters* ctr = a.ctr;
    if (*(volatile u32*)&ctr->done)
        return;
    const int r = a.level;
    const u32 cr = ((volatile u32*)ctr->c)[r];       // columns of C_r (and rows)
    const u32 cn = ((volatile u32*)ctr->c)[r + 1];   // size of C_{r+1}
    const u32 total_chunks = *(volatile u32*)&ctr->total_chunks;
    const u32 nbr = *(volatile u32*)&ctr->nbr;
    const u32 total = total_chunks * nbr;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&ctr->item_next, 1u);
        __syncthreads();
        const u32 item = s_item;
        if (item >= total)
            break;
        contract_item<DT, LEVEL0, VEC>(a, item, cr, cn, total_chunks, bins, s_rows, s_red);
    }
}

// ------------------------------------------------------------------ host
namespace {

__global__ void k_mst_init(Counters* ctr, u32* comp, u32 n, u32 bar_reset)
{
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        comp[v] = v;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i < MAX_LEVELS + 2; ++i)
            ctr->c[i] = 0;
        ctr->c[0] = n;
        ctr->done = (n <= 1) ? 1u : 0u;
        ctr->mst_count = 0;
        ctr->item_next = 0;
        ctr->total_chunks = 0;
        ctr->nbr = 0;
        ctr->jump_flag[0] = ctr->jump_flag[1] = ctr->jump_flag[2] = 0;
        if (bar_reset) {
            ctr->bar.count = 0;
            ctr->bar.abort = 0;
        }
    }
}

template <class K>
cudaError_t set_smem(K kern, size_t bytes)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t contraction_scratch_bytes(int64_t n)
{
    size_t h = (size_t)(n / 2), q = (size_t)(n / 4);
    return (h * h + q * q) * sizeof(u64) + 64;
}

cudaError_t run_mst(Workspace& ws, const void* W, int dt, void* cbuf, size_t cbuf_bytes,
                    u32* status, cudaStream_t s)
{
    const u32 n = (u32)ws.n;
    cudaError_t err;
    k_mst_init<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(ws.ctr, ws.comp, n, 1);
    prof_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess)
        return err;
    if (n <= 1)
        return cudaSuccess;
    const bool vec = (n % 4 == 0) && ((uintptr_t)W % 16 == 0);
    prof_launches(1);
    prof_begin(PH_ROWMIN, s);
    if (vec) {
        // upper-triangle tiles; best[] is reduced with atomic minima from +inf
        if ((err = cudaMemsetAsync(ws.best[0], 0xFF, (size_t)n * sizeof(u64), s)) != cudaSuccess)
            return err;
        dim3 grid((n + RS_COLS - 1) / RS_COLS, (n + RS_ROWS - 1) / RS_ROWS);
        if (dt == 0)
            k_rowmin_sym<0><<<grid, 256, 0, s>>>((const u32*)W, n, ws.best[0]);
        else
            k_rowmin_sym<1><<<grid, 256, 0, s>>>((const u32*)W, n, ws.best[0]);
        if ((err = cudaGetLastError()) != cudaSuccess)
            return err;
    } else {
        int grid = ws.sms * 8;
        if (grid > (int)n)
            grid = (int)n;
        if (dt == 0)
            k_rowmin<0, false><<<grid, 256, 0, s>>>((const u32*)W, n, ws.best[0]);
        else
            k_rowmin<1, false><<<grid, 256, 0, s>>>((const u32*)W, n, ws.best[0]);
        if ((err = cudaGetLastError()) != cudaSuccess)
            return err;
    }
    prof_end(PH_ROWMIN, s);
    // contraction matrices: C_1, C_3, ... in the first half, C_2, C_4, ... after it
    const size_t h = (size_t)(n / 2);
    // the u64 matrices need 16-byte alignment; a caller's M may start anywhere
    // 4-byte aligned (batched layouts), so round up (the buffer has slack)
    u64* cb[2];
    cb[0] = (u64*)(((uintptr_t)cbuf + 15) & ~(uintptr_t)15);
    cb[1] = (u64*)((char*)cb[0] + ((h * h * sizeof(u64) + 15) & ~(size_t)15));
    (void)cbuf_bytes;
    const size_t smem = (size_t)ws.bin_cap * sizeof(u64);
    auto k0 = (dt == 0) ? (vec ? k_contract<0, 1, true> : k_contract<0, 1, false>)
                        : (vec ? k_contract<1, 1, true> : k_contract<1, 1, false>);

    auto k1 = k_contract<0, 0, false>;
    if ((err = set_smem(k0, smem)) != cudaSuccess)
        return err;
    if ((err = set_smem(k1, smem)) != cudaSuccess)
        return err;
    for (int r = 0; r < ws.levels; ++r) {
        StepArgs sa;
        sa.level = r;
        sa.n = n;
        sa.best_in = ws.best[r & 1];
        sa.best_out = ws.best[(r + 1) & 1];
        sa.comp = ws.comp;
        sa.hook = ws.hook;
        sa.par = ws.par;
        sa.flag = ws.flag;
        sa.rootid = ws.rootid;
        sa.label = ws.label;
        sa.cnt = ws.cnt;
        sa.fillc = ws.fillc;
        sa.gstart = ws.gstart;
        sa.members = ws.members;
        sa.nchunk = ws.nchunk;
        sa.chunk_start = ws.chunk_start;
        sa.item_group = ws.item_group;
        sa.mst = ws.mst;
        sa.cnext = cb[r & 1];
        sa.part = ws.part;
        sa.ctr = ws.ctr;
        sa.status = status;
        sa.bin_cap = ws.bin_cap;
        err = cudaMemsetAsync(&ws.ctr->bar, 0, 2 * sizeof(u32), s);
        if (err != cudaSuccess)
            return err;
        void* args[] = {&sa};
        prof_begin(PH_STEP, s);
        err = cudaLaunchCooperativeKernel((const void*)k_step, dim3(ws.coop_blocks),
                                          dim3(ws.coop_threads), args, 0, s);
        prof_end(PH_STEP, s);
        prof_launches(2);
        if (err != cudaSuccess)
            return err;

        ContractArgs ca;
        ca.level = r;
        ca.cin = (r == 0) ? W : (const void*)cb[(r - 1) & 1];
        ca.cout = cb[r & 1];
        ca.best_out = ws.best[(r + 1) & 1];
        ca.label = ws.label;
        ca.members = ws.members;
        ca.gstart = ws.gstart;
        ca.nchunk = ws.nchunk;
        ca.chunk_start = ws.chunk_start;
        ca.item_group = ws.item_group;
        ca.ctr = ws.ctr;
        ca.bin_cap = ws.bin_cap;
        dim3 grid(ws.contract_blocks), block(CONTRACT_THREADS);
        const int ph = (r == 0) ? PH_CONTRACT0 : PH_CONTRACT;
        prof_begin(ph, s);
        if (r == 0)
            k0<<<grid, block, smem, s>>>(ca);
        else
            k1<<<grid, block, smem, s>>>(ca);
        prof_end(ph, s);
        if ((err = cudaGetLastError()) != cudaSuccess)
            return err;
    }
    return cudaSuccess;
}

}  // namespace appd
