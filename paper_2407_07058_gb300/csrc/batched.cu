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
    u32 warp_bins;        // u64 bins per warp when each warp owns a group
    u32 fill_rows;        // rows per fill tile
};

constexpr int BATCH_THREADS = 512;

// Column groups of a row that starts at any 4-byte boundary.
//
// out[u] = columns [4g, 4g + 4) of the row for g = g0 + 32u, where g0 is the
// calling lane's first group (the warp covers 32 * U consecutive groups).
// Every group costs one aligned 16-byte load: when the row is not 16-byte
// aligned, a group's upper columns sit in the next aligned block, which the
// neighbouring lane loaded (lane 31 takes lane 0's next block, or loads one
// extra block past the warp's range).  Blocks not wholly inside [lo, hi) --
// only at the two ends of the matrix -- are read element by element, so no
// load leaves the matrix.  Columns >= n hold other rows' values (or 0): the
// caller masks them.  All 32 lanes must call it together.
template <int U>
__device__ __forceinline__ void load_groups(const u32* row, u32 n, const u32* lo, const u32* hi, u32 g0,
                                            uint4 (&out)[U])
{
    const u32 lane = threadIdx.x & 31;
    const u32 s = (u32)(((uintptr_t)row >> 2) & 3u);
    const u32* base = row - s;            // 16-byte aligned
    const u32 nb = (n + s + 3) >> 2;      // aligned blocks that hold the row
    auto blk = [&](u32 bi) -> uint4 {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (bi < nb) {
            const u32* p = base + 4 * (size_t)bi;
            if (p >= lo && p + 4 <= hi) {
                v = ld_stream_v4(p);
            } else {
                v.x = (p >= lo && p < hi) ? ld_stream_u32(p) : 0u;
                v.y = (p + 1 >= lo && p + 1 < hi) ? ld_stream_u32(p + 1) : 0u;
                v.z = (p + 2 >= lo && p + 2 < hi) ? ld_stream_u32(p + 2) : 0u;
                v.w = (p + 3 >= lo && p + 3 < hi) ? ld_stream_u32(p + 3) : 0u;
            }
        }
        return v;
    };
    uint4 bk[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
        bk[u] = blk(g0 + 32 * u);
    if (s == 0) {
#pragma unroll
        for (int u = 0; u < U; ++u)
            out[u] = bk[u];
        return;
    }
    const uint4 extra = (lane == 31) ? blk(g0 + 32 * (U - 1) + 1) : make_uint4(0u, 0u, 0u, 0u);
    const int src = (lane + 1) & 31;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        uint4 nx;
        nx.x = __shfl_sync(0xFFFFFFFFu, bk[u].x, src);
        nx.y = __shfl_sync(0xFFFFFFFFu, bk[u].y, src);
        nx.z = __shfl_sync(0xFFFFFFFFu, bk[u].z, src);
        uint4 nl = extra;
        if (u + 1 < U) {
            nl.x = __shfl_sync(0xFFFFFFFFu, bk[u + 1 < U ? u + 1 : u].x, 0);
            nl.y = __shfl_sync(0xFFFFFFFFu, bk[u + 1 < U ? u + 1 : u].y, 0);
            nl.z = __shfl_sync(0xFFFFFFFFu, bk[u + 1 < U ? u + 1 : u].z, 0);
        }
        if (lane == 31)
            nx = nl;
        const uint4 c = bk[u];
        out[u] = (s == 1) ? make_uint4(c.y, c.z, c.w, nx.x)
                          : (s == 2) ? make_uint4(c.z, c.w, nx.x, nx.y) : make_uint4(c.w, nx.x, nx.y, nx.z);
    }
}

// Round-1 row minima of one graph by one CTA: each warp takes a row and
// keeps eight 16-byte loads per lane in flight (64 KB per CTA).
template <int DT>
__device__ void rowmin_cta(const u32* __restrict__ W, u32 n, u64* __restrict__ best)
{
    constexpr int U = 8;
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const u32* hi = W + (size_t)n * n;
    const u32 ng = (n + 3) >> 2;
    for (u32 i = w; i < n; i += nw) {
        const u32* r = W + (size_t)i * n;
        u64 m = EDGE_INF;
        for (u32 c0 = 0; c0 < ng; c0 += 32 * U) {
            uint4 v[U];
            load_groups<U>(r, n, W, hi, c0 + lane, v);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const u32 j = 4 * (c0 + lane + 32 * u);
                const u32 x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const u64 c = ((u64)key_of(x[t], DT) << 32) | (j + t);
                    if (j + t < n && j + t != i && c < m)
                        m = c;
                }
            }
        }
        m = warp_min_u64(m);
        if (lane == 0)
            best[i] = pack_edge((u32)(m >> 32), i, (u32)m & 0xFFFFu);
    }
}

// Sorts up to four uniform row ids ascending; slots past np repeat the
// smallest row (same key, same row: such a slot never changes a minimum).
__device__ __forceinline__ void sort_rows4(u32* rid, u32 np)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if ((u32)q >= np)
            rid[q] = 0xFFFFFFFFu;
    auto cs = [&](int a, int c) {
        const u32 lo = min(rid[a], rid[c]), hi = max(rid[a], rid[c]);
        rid[a] = lo;
        rid[c] = hi;
    };
    cs(0, 1);
    cs(2, 3);
    cs(0, 2);
    cs(1, 3);
    cs(1, 2);
#pragma unroll
    for (int q = 1; q < 4; ++q)
        if ((u32)q >= np)
            rid[q] = rid[0];
}

// One contraction level with one warp per group: warp w folds every row of
// group A (A = w, w + warps, ...) into its own cn bins in shared memory, then
// writes row A of C_{r+1} (row stride sout) and A's row minimum.  Groups
// proceed concurrently and independently (no block barrier between groups),
// so 16 groups' loads are in flight instead of one item's.  Level 0 reads W
// rows at any alignment (load_groups); later levels read C_r with row stride
// sin.  Needs cn <= the per-warp capacity.
template <int DT, int LEVEL0>
__device__ void contract_level_warps(const ContractArgs& a, u32 cr, u32 cn, u32 sin, u32 sout,
                                     const u32* wlo, const u32* whi, u64* wbins, u32 wcap)
{
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64* bins = wbins + (size_t)wid * wcap;
    for (u32 A = wid; A < cn; A += nw) {
        for (u32 b = lane; b < cn; b += 32)
            bins[b] = EDGE_INF;
        __syncwarp();
        const u32 m0 = a.gstart[A], m1 = a.gstart[A + 1];
        for (u32 p = m0; p < m1; p += 4) {
            const u32 np = min(4u, m1 - p);
            u32 rid[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                rid[q] = a.members[p + ((u32)q < np ? q : 0)];
            if (LEVEL0) {
                constexpr int U = 2;
                sort_rows4(rid, np);
                const u32* W = (const u32*)a.cin;
                const u32 ng = (cr + 3) >> 2;
                for (u32 c0 = 0; c0 < ng; c0 += 32 * U) {
                    uint4 v[4][U];
                    load_groups<U>(W + (size_t)rid[0] * cr, cr, wlo, whi, c0 + lane, v[0]);
#pragma unroll
                    for (int q = 1; q < 4; ++q) {
                        if ((u32)q < np) {
                            load_groups<U>(W + (size_t)rid[q] * cr, cr, wlo, whi, c0 + lane, v[q]);
                        } else {
#pragma unroll
                            for (int u = 0; u < U; ++u)
                                v[q][u] = v[0][u];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const u32 g = c0 + lane + 32 * u;
                        uint4 lab = make_uint4(A, A, A, A);
                        if (g < ng) {
                            lab = *reinterpret_cast<const uint4*>(a.label + 4 * g);
                            if (4 * g + 1 >= cr)
                                lab.y = A;
                            if (4 * g + 2 >= cr)
                                lab.z = A;
                            if (4 * g + 3 >= cr)
                                lab.w = A;
                        }
                        const uint4 x[4] = {v[0][u], v[1][u], v[2][u], v[3][u]};
                        fold_group<DT, 4, true>(x, rid, 4 * g, lab, A, 0, cn, bins);
                    }
                }
            } else {
                const u64* C = (const u64*)a.cin;
                const u64* rp[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    rp[q] = C + (size_t)rid[q] * sin;
                auto update = [&](u32 L, u64 e) {
                    if (L != A && e < bins[L])
                        atomicMin(&bins[L], e);
                };
                u32 jt = 0;
                if (((sin & 1u) == 0) && (((uintptr_t)C & 15u) == 0)) {
                    const u32 n2 = cr >> 1;
                    for (u32 g0 = lane; g0 < n2; g0 += 64) {
                        uint4 v[2][4];
                        uint2 lab[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const u32 g = g0 + 32 * u;
                            const bool ok = g < n2;
                            v[u][0] = ok ? ld_stream_v4(rp[0] + 2 * g) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                            for (int q = 1; q < 4; ++q)
                                v[u][q] = (ok && (u32)q < np) ? ld_stream_v4(rp[q] + 2 * g) : v[u][0];
                            lab[u] = ok ? *reinterpret_cast<const uint2*>(a.label + 2 * g) : make_uint2(A, A);
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            u64 e0 = EDGE_INF, e1 = EDGE_INF;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const u64 x0 = ((u64)v[u][q].y << 32) | v[u][q].x;
                                const u64 x1 = ((u64)v[u][q].w << 32) | v[u][q].z;
                                e0 = x0 < e0 ? x0 : e0;
                                e1 = x1 < e1 ? x1 : e1;
                            }
                            update(lab[u].x, e0);
                            update(lab[u].y, e1);
                        }
                    }
                    jt = 2 * n2;
                }
                for (u32 j = jt + lane; j < cr; j += 32) {
                    u64 e = rp[0][j];
#pragma unroll
                    for (int q = 1; q < 4; ++q)
                        if ((u32)q < np) {
                            const u64 x = rp[q][j];
                            e = x < e ? x : e;
                        }
                    update(a.label[j], e);
                }
            }
        }
        __syncwarp();
        u64 m = EDGE_INF;
        u64* dst = a.cout + (size_t)A * sout;
        for (u32 b = lane; b < cn; b += 32) {
            const u64 v = bins[b];
            dst[b] = v;
            m = v < m ? v : m;
        }
        m = warp_min_u64(m);
        if (lane == 0 && m != EDGE_INF)
            atomicMin(&a.best_out[A], m);
        __syncwarp();
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
    const bool vec = (n % 4 == 0) && (((uintptr_t)W & 15u) == 0);

    // contraction scratch: M (16-byte aligned start) unless solving in place
    const u32 h = n / 2;
    u64* cb0 = (M == W) ? w.cscratch : (u64*)(((uintptr_t)M + 15) & ~(uintptr_t)15);
    u64* cb1 = (u64*)((char*)cb0 + (((size_t)h * h * sizeof(u64) + 15) & ~(size_t)15));
    const int levels = ceil_log2_dev(n);
    // row stride of C_r: the warp-per-group contraction pads odd widths to
    // even (16-byte aligned rows) where the scratch half has room
    u32 stride = n;
    const size_t cap_half[2] = {(size_t)h * h, (size_t)(n / 4) * (n / 4)};
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
        u64* bins = reinterpret_cast<u64*>(smem);
        if (cn <= b.warp_bins) {
            const u32 sout = ((cn & 1u) && (size_t)cn * (cn + 1) <= cap_half[r & 1]) ? cn + 1 : cn;
            if (r == 0)
                contract_level_warps<DT, 1>(ca, cr, cn, stride, sout, W, W + (size_t)n * n, bins, b.warp_bins);
            else
                contract_level_warps<DT, 0>(ca, cr, cn, stride, sout, W, W, bins, b.warp_bins);
            stride = sout;
            __syncthreads();
            continue;
        }
        stride = cn;
        const u32 tc = *(volatile u32*)&ctr->total_chunks;
        const u32 total = tc * *(volatile u32*)&ctr->nbr;
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

    // one column block at a time, all rows (in batches of fill_rows): the
    // block's sort and table are built once
    for (u32 j0 = 0; j0 < n; j0 += FC)
        fill_tile<DT>(w.pos, w.st, n, j0, 0, n, b.fill_rows, M, smem);
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
        switch (b.dts[g]) {
        case 1: solve_one<1>(w, W, M, n, b, smem, s_rows, s_red); break;
        case 2: solve_one<2>(w, W, M, n, b, smem, s_rows, s_red); break;
        case 3: solve_one<3>(w, W, M, n, b, smem, s_rows, s_red); break;
        default: solve_one<0>(w, W, M, n, b, smem, s_rows, s_red); break;
        }
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
    u32 warp_bins = 0;
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
    a.warp_bins = rt.warp_bins;
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
    // dynamic shared memory: the fill tile, or per-warp contraction bins for
    // up to 1024 groups, whichever is larger (the phases reuse it in turn)
    nr->smem = std::max(fill_smem_bytes((u32)tune.fill_rows),
                        (size_t)(BATCH_THREADS / 32) * 1024 * sizeof(u64));
    nr->bin_cap = (u32)(nr->smem / sizeof(u64));
    nr->warp_bins = (u32)(nr->bin_cap / (BATCH_THREADS / 32));
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
