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
    u32 *sval0, *sval1;
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
    u32 fill_rows;        // rows per fill batch (shared memory of a fill tile)
    u32* posst;           // leaf positions and sparse tables of all graphs
    const u64* pst_off;   // graph g's pos at posst + pst_off[g], its table after n entries
    u64* best0;           // round-1 minima of all graphs (k_rowmin_batched)
    const u64* row_off;   // graph g's minima at best0 + row_off[g]
    u32* gfail;           // per graph: 1 when its solve failed (the fill skips it)
    u32 prim_max;         // graphs up to this size are solved by one warp with Prim
};

constexpr int BATCH_THREADS = 512;
// largest graph a warp solves by Prim (a lane keeps n / 32 distances)
constexpr u32 PRIM_WARP_MAX = 512;

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

// Round-1 minimum of row i of an n-vertex graph by one warp.  A minimum
// does not care which lane sees which column, so the warp walks the 16-byte
// aligned blocks that cover the row (any row alignment, no realignment) and
// maps each element back to its column; blocks not wholly inside the matrix
// (only at its two ends) are read element by element.  Minima are kept as
// (key, column) pairs of 32-bit words: a lane visits its columns in
// increasing order and keeps the first strictly smaller key (the first
// valid column always enters), and the warp reduces (key, column).
template <int DT>
__device__ void row_best_warp(const u32* __restrict__ W, u32 n, u32 i, u64* __restrict__ best)
{
    constexpr int U = 4;
    const u32 lane = threadIdx.x & 31;
    const u32* hi = W + (size_t)n * n;
    const u32* r = W + (size_t)i * n;
    const u32 s = (u32)(((uintptr_t)r >> 2) & 3u);
    const u32* base = r - s;
    const u32 nb = (n + s + 3) >> 2;
    u32 bk = 0xFFFFFFFFu, bj = 0xFFFFFFFFu;
    for (u32 b0 = 0; b0 < nb; b0 += 32 * U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u32 bi = b0 + lane + 32 * u;
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (bi < nb) {
                const u32* p = base + 4 * (size_t)bi;
                if (p >= W && p + 4 <= hi) {
                    v[u] = ld_stream_v4(p);
                } else {
                    v[u].x = (p >= W && p < hi) ? ld_stream_u32(p) : 0u;
                    v[u].y = (p + 1 >= W && p + 1 < hi) ? ld_stream_u32(p + 1) : 0u;
                    v[u].z = (p + 2 >= W && p + 2 < hi) ? ld_stream_u32(p + 2) : 0u;
                    v[u].w = (p + 3 >= W && p + 3 < hi) ? ld_stream_u32(p + 3) : 0u;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u32 j0 = 4 * (b0 + lane + 32 * u) - s;   // column of the block's first word (wraps below 0)
            const u32 x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const u32 j = j0 + t, k = key_of(x[t], DT);
                if (j < n && j != i && (k < bk || bj == 0xFFFFFFFFu)) {
                    bk = k;
                    bj = j;
                }
            }
        }
    }
    const u32 kmin = __reduce_min_sync(0xFFFFFFFFu, bj == 0xFFFFFFFFu ? 0xFFFFFFFFu : bk);
    const u32 jmin = __reduce_min_sync(0xFFFFFFFFu, (bj != 0xFFFFFFFFu && bk == kmin) ? bj : 0xFFFFFFFFu);
    if (lane == 0)
        best[i] = pack_edge(kmin, i, jmin, n);
}

// Round-1 minima of every graph of a batch before k_batched: one CTA per
// task of ROWB_ROWS rows of one graph, a warp per row, at full occupancy.
constexpr int ROWB_THREADS = 256;
constexpr u32 ROWB_ROWS = 32;

__global__ void __launch_bounds__(ROWB_THREADS) k_rowmin_batched(BatchArgs b, const uint2* __restrict__ tasks)
{
    const uint2 tk = tasks[blockIdx.x];   // graph, first row
    const u32 g = tk.x, n = b.ns[g];
    const u32* W = b.wp[g];
    u64* best = b.best0 + b.row_off[g];
    const u32 w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const u32 r1 = min(n, tk.y + ROWB_ROWS);
    for (u32 i = tk.y + w; i < r1; i += nw) {
        switch (b.dts[g]) {
        case 1: row_best_warp<1>(W, n, i, best); break;
        case 2: row_best_warp<2>(W, n, i, best); break;
        case 3: row_best_warp<3>(W, n, i, best); break;
        default: row_best_warp<0>(W, n, i, best); break;
        }
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

// One contraction level with one warp per group: a warp claims a group A,
// folds every row of A into its own cn bins in shared memory, writes row A
// of C_{r+1} (row stride sout) and A's row minimum, and claims the next.
// Groups proceed concurrently and independently (no block barrier between
// groups), so 16 groups' loads are in flight instead of one item's.  Level 0
// reads W rows at any alignment (load_groups); later levels read C_r with
// row stride sin.  Needs cn <= the per-warp capacity.
template <int DT, int LEVEL0>
__device__ void contract_level_warps(const ContractArgs& a, u32 cr, u32 cn, u32 sin, u32 sout,
                                     const u32* wlo, const u32* whi, u64* wbins, u32 wcap, u32* gnext)
{
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u64* bins = wbins + (size_t)wid * wcap;
    // bins start empty once per level; each group's write-out empties them
    // again for the warp's next group
    for (u32 b = lane; b < cn; b += 32)
        bins[b] = EDGE_INF;
    __syncwarp();
    // groups are claimed one at a time (sizes vary), so no warp idles behind
    // a statically assigned share; *gnext starts at 0 (the caller resets it)
    for (;;) {
        u32 A = 0;
        if (lane == 0)
            A = atomicAdd(gnext, 1u);
        A = __shfl_sync(0xFFFFFFFFu, A, 0);
        if (A >= cn)
            break;
        const u32 m0 = a.gstart[A], m1 = a.gstart[A + 1];
        for (u32 p = m0; p < m1; p += 4) {
            const u32 np = min(4u, m1 - p);
            u32 rid[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                rid[q] = a.members[p + ((u32)q < np ? q : 0)];
            if (LEVEL0) {
                constexpr int U = 3;
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
                        fold_group<DT, 4, true>(x, rid, 4 * g, lab, A, 0, cn, bins, cr);
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
            bins[b] = EDGE_INF;
            m = v < m ? v : m;
        }
        m = warp_min_u64(m);
        if (lane == 0 && m != EDGE_INF)
            atomicMin(&a.best_out[A], m);
        __syncwarp();
    }
}

template <int DT>
__device__ void solve_one(const SliceWs& w, const u32* W, u32* M, u32 n, u32* pos_g, u64* best0,
                          u32* fail_g, const BatchArgs& b, unsigned char* smem, u32* s_rows,
                          u64* s_red)
{
    BlockTeam t;
    const u32 tid = threadIdx.x;
    if (n == 1) {
        if (tid == 0) {
            M[0] = 0u;
            *fail_g = 0u;
        }
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
        // the slice's control block outlives the graph: a failure recorded
        // by an earlier graph (or a stale allocation) must not stop this one
        ctr->bar.count = 0;
        ctr->bar.abort = 0;
        ctr->bar.failed = 0;
    }
    // round-1 minima come from k_rowmin_batched (best0)
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
        sa.best_in = (r & 1) ? w.best1 : best0;
        sa.best_out = (r & 1) ? best0 : w.best1;
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
            __shared__ u32 s_gnext;   // next group to claim
            if (threadIdx.x == 0)
                s_gnext = 0;
            __syncthreads();
            const u32 sout = ((cn & 1u) && (size_t)cn * (cn + 1) <= cap_half[r & 1]) ? cn + 1 : cn;
            if (r == 0)
                contract_level_warps<DT, 1>(ca, cr, cn, stride, sout, W, W + (size_t)n * n, bins, b.warp_bins,
                                            &s_gnext);
            else
                contract_level_warps<DT, 0>(ca, cr, cn, stride, sout, W, W, bins, b.warp_bins, &s_gnext);
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
    la.sval0 = w.sval0;
    la.sval1 = w.sval1;
    la.hist = w.hist;
    la.ntiles = (n - 1 + 2047) / 2048;
    la.first_child = w.first_child;
    la.next_sib = w.next_sib;
    la.pos = pos_g;
    la.order = w.order;
    la.nsize = w.nsize;
    la.gap = w.gap;
    la.st = pos_g + n;
    la.part = w.part;
    la.ctr = ctr;
    la.status = b.status;
    leaf_body(t, la);
    __syncthreads();
    // the fill runs afterwards for every graph of the batch at once
    // (k_fill_batched), reading pos and the sparse table from posst; a graph
    // whose solve failed has no valid leaf order and is skipped there
    if (tid == 0)
        *fail_g = solve_failed(&ctr->bar) ? 1u : 0u;
    __syncthreads();
}

// A small graph on one warp, by Prim's algorithm from vertex 0 (Section 3's
// MST step, as the paper does it): each lane keeps the packed distance of
// its vertices v = lane + 32 t to the tree, the warp takes the smallest
// (the strict order (key, lo, hi), so the tree is the minimum spanning tree
// the other paths find), records the vertex's position and the edge that
// added it, and relaxes with the new vertex's row.  Prim's visiting order is
// a leaf order for the fill: M(v_a, v_b) is the largest of the edges that
// added v_{a+1} .. v_b (the tree path argument of the leaf order), so the
// positions and the sparse table over those gaps go to the arena exactly as
// the one-CTA leaf order leaves them, and the grid-wide fill follows.
template <int DT>
__device__ void prim_warp(const u32* __restrict__ W, u32* M, u32 n, u32* pos, u32* fail_g)
{
    constexpr int T = PRIM_WARP_MAX / 32;
    const u32 lane = threadIdx.x & 31;
    if (n == 1) {
        if (lane == 0) {
            M[0] = 0u;
            pos[0] = 0u;
            *fail_g = 0u;
        }
        __syncwarp();
        return;
    }
    u32* st = pos + n;
    u64 dist[T];
    u32 out = 0;   // bit t: vertex lane + 32 t is in the tree (or past n)
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const u32 v = lane + 32 * t;
        dist[t] = EDGE_INF;
        if (v >= n || v == 0)
            out |= 1u << t;
        else
            dist[t] = pack_edge(key_of(W[v], DT), 0, v, n);
    }
    if (lane == 0)
        pos[0] = 0u;
    for (u32 k = 1; k < n; ++k) {
        u64 m = EDGE_INF;
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (!((out >> t) & 1u) && dist[t] < m)
                m = dist[t];
        const u64 e = warp_min_u64(m);
        // the unique slot that holds e: the vertex that joins
        u32 b = 0xFFFFFFFFu;
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (!((out >> t) & 1u) && dist[t] == e) {
                b = lane + 32 * t;
                out |= 1u << t;
            }
        b = __reduce_min_sync(0xFFFFFFFFu, b);
        if (lane == 0) {
            pos[b] = k;
            st[k - 1] = edge_key(e);
        }
        const u32* row = W + (size_t)b * n;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const u32 v = lane + 32 * t;
            if (!((out >> t) & 1u)) {
                const u64 c = pack_edge(key_of(row[v], DT), b, v, n);
                dist[t] = c < dist[t] ? c : dist[t];
            }
        }
    }
    __syncwarp();
    // the sparse table over the n - 1 gaps, one level at a time
    const u32 m = n - 1;
    for (u32 k = 1; (1u << k) <= m; ++k) {
        const u32 h = 1u << (k - 1);
        const u32* sp = st + (size_t)(k - 1) * n;
        u32* sc = st + (size_t)k * n;
        for (u32 x = lane; x + 2 * h <= m; x += 32) {
            const u32 p = sp[x], q = sp[x + h];
            sc[x] = p > q ? p : q;
        }
        __syncwarp();
    }
    if (lane == 0)
        *fail_g = 0u;
    __syncwarp();
}

template <int DT>
__device__ __forceinline__ void prim_graph(const BatchArgs& b, u32 g)
{
    prim_warp<DT>(b.wp[g], b.mp[g], b.ns[g], b.posst + b.pst_off[g], b.gfail + g);
}

// Graphs of at most prim_max vertices, one per warp, claimed warp by warp.
__device__ void prim_warps(const BatchArgs& b, u32 first_q)
{
    const u32 lane = threadIdx.x & 31;
    u32 q = first_q;
    for (;;) {
        if (q >= b.count)
            break;
        const u32 g = b.queue[q];
        if (b.ns[g] > 0) {
            switch (b.dts[g]) {
            case 1: prim_graph<1>(b, g); break;
            case 2: prim_graph<2>(b, g); break;
            case 3: prim_graph<3>(b, g); break;
            default: prim_graph<0>(b, g); break;
            }
        }
        u32 nq = 0;
        if (lane == 0)
            nq = atomicAdd(b.next, 1u);
        q = __shfl_sync(0xFFFFFFFFu, nq, 0);
    }
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
        if (n <= b.prim_max) {
            // the queue is sorted by size: every graph from here on is small;
            // warp 0 takes this one, the other warps claim their own
            u32 q0 = q;
            if ((threadIdx.x >> 5) != 0) {
                u32 nq = 0;
                if ((threadIdx.x & 31) == 0)
                    nq = atomicAdd(b.next, 1u);
                q0 = __shfl_sync(0xFFFFFFFFu, nq, 0);
            }
            prim_warps(b, q0);
            break;
        }
        if (n == 0)
            continue;
        u32* pos_g = b.posst + b.pst_off[g];
        u64* best_g = b.best0 + b.row_off[g];
        u32* fail_g = b.gfail + g;
        switch (b.dts[g]) {
        case 1: solve_one<1>(w, W, M, n, pos_g, best_g, fail_g, b, smem, s_rows, s_red); break;
        case 2: solve_one<2>(w, W, M, n, pos_g, best_g, fail_g, b, smem, s_rows, s_red); break;
        case 3: solve_one<3>(w, W, M, n, pos_g, best_g, fail_g, b, smem, s_rows, s_red); break;
        default: solve_one<0>(w, W, M, n, pos_g, best_g, fail_g, b, smem, s_rows, s_red); break;
        }
    }
}

// The fill of every graph of a batch: one CTA per tile (graph, 128 columns,
// all rows in batches of fill_rows), from the tile list built with the batch
// layout.
// All CTAs of the GPU share the work, at the occupancy of the single-solve
// fill, instead of one CTA filling a whole graph.
constexpr int FILLB_THREADS = 256;

__global__ void __launch_bounds__(FILLB_THREADS) k_fill_batched(BatchArgs b, const uint4* __restrict__ tiles)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const uint4 tl = tiles[blockIdx.x];   // graph, first column, first row, rows
    const u32 g = tl.x, n = b.ns[g];
    if (*(volatile const u32*)(b.gfail + g))   // no valid leaf order: leave M unwritten
        return;
    const u32* pos = b.posst + b.pst_off[g];
    switch (b.dts[g]) {
    case 1: fill_tile<1>(pos, pos + n, n, tl.y, tl.z, tl.w, b.fill_rows, b.mp[g], smem); break;
    case 2: fill_tile<2>(pos, pos + n, n, tl.y, tl.z, tl.w, b.fill_rows, b.mp[g], smem); break;
    case 3: fill_tile<3>(pos, pos + n, n, tl.y, tl.z, tl.w, b.fill_rows, b.mp[g], smem); break;
    default: fill_tile<0>(pos, pos + n, n, tl.y, tl.z, tl.w, b.fill_rows, b.mp[g], smem); break;
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
    size_t fill_smem = 0;
    u32 bin_cap = 0;
    u32 warp_bins = 0;
    void* arena = nullptr;         // minima / leaf-order arena of the uncached launch path
    size_t arena_bytes = 0;
    struct Plan {
        void* dev = nullptr;
        void* arena = nullptr;
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

// descriptor block layout: wp | mp | ns | queue | dts | pst_off | row_off |
// fill tiles | row tasks
struct DescLayout {
    size_t off[9];
    size_t bytes;
    u32 ntiles, ntasks;
    size_t posst_words;   // leaf positions + sparse tables of every graph
    size_t rows;          // vertices of every graph (round-1 minima)
    size_t arena_bytes;   // posst, then the minima (8-byte aligned), then a failure flag per graph
    size_t gfail_off;     // byte offset of the failure flags in the arena
};

// sparse-table levels of an n-vertex graph (as the leaf order builds it)
inline u32 st_levels_of(u32 n)
{
    u32 l = 1;
    while (n > 1 && (1u << l) <= n - 1)
        ++l;
    return l;
}

DescLayout desc_layout(const BatchDesc& d, u32 fill_rows, u32 prim_max)
{
    DescLayout L;
    const size_t cnt = d.n.size();
    L.ntiles = L.ntasks = 0;
    L.posst_words = L.rows = 0;
    for (u32 n : d.n) {
        if (n >= 2) {
            L.ntiles += (n + FC - 1) / FC;
            if (n > prim_max)   // round-1 minima only for the graphs Boruvka solves
                L.ntasks += (n + ROWB_ROWS - 1) / ROWB_ROWS;
        }
        L.posst_words += (size_t)n * (1 + st_levels_of(n));
        L.rows += n;
    }
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    L.off[0] = 0;
    L.off[1] = L.off[0] + 8 * cnt;
    L.off[2] = L.off[1] + 8 * cnt;
    L.off[3] = L.off[2] + 4 * cnt;
    L.off[4] = L.off[3] + 4 * cnt;
    L.off[5] = a16(L.off[4] + cnt);
    L.off[6] = a16(L.off[5] + 8 * cnt);
    L.off[7] = a16(L.off[6] + 8 * cnt);
    L.off[8] = a16(L.off[7] + 16 * (size_t)L.ntiles);
    L.bytes = (L.off[8] + 8 * (size_t)L.ntasks + 255) & ~(size_t)255;
    L.gfail_off = ((L.posst_words * 4 + 7) & ~(size_t)7) + 8 * L.rows;
    L.arena_bytes = L.gfail_off + 4 * cnt + 256;
    return L;
}

void fill_desc(const BatchDesc& d, u32 fill_rows, u32 prim_max, const DescLayout& L,
               std::vector<unsigned char>& host)
{
    const u32 cnt = (u32)d.n.size();
    std::vector<u32> q(cnt);
    std::iota(q.begin(), q.end(), 0u);
    std::stable_sort(q.begin(), q.end(), [&](u32 a, u32 b) { return d.n[a] > d.n[b]; });
    std::vector<u64> pst(cnt), roff(cnt);
    std::vector<uint4> tiles;
    std::vector<uint2> tasks;
    tiles.reserve(L.ntiles);
    tasks.reserve(L.ntasks);
    u64 acc = 0, racc = 0;
    // largest graphs first, so the row tasks and fill tiles of the long
    // graphs start early
    for (u32 k = 0; k < cnt; ++k) {
        const u32 g = q[k];
        const u32 n = d.n[g];
        if (n < 2)
            continue;
        if (n > prim_max)
            for (u32 r0 = 0; r0 < n; r0 += ROWB_ROWS)
                tasks.push_back(make_uint2(g, r0));
        // a tile is a whole column block: its sort and table are built once,
        // the rows follow in batches of fill_rows
        for (u32 j0 = 0; j0 < n; j0 += FC)
            tiles.push_back(make_uint4(g, j0, 0u, n));
    }
    for (u32 g = 0; g < cnt; ++g) {
        pst[g] = acc;
        acc += (u64)d.n[g] * (1 + st_levels_of(d.n[g]));
        roff[g] = racc;
        racc += d.n[g];
    }
    memcpy(host.data() + L.off[0], d.w.data(), 8 * cnt);
    memcpy(host.data() + L.off[1], d.m.data(), 8 * cnt);
    memcpy(host.data() + L.off[2], d.n.data(), 4 * cnt);
    memcpy(host.data() + L.off[3], q.data(), 4 * cnt);
    memcpy(host.data() + L.off[4], d.dt.data(), cnt);
    memcpy(host.data() + L.off[5], pst.data(), 8 * cnt);
    memcpy(host.data() + L.off[6], roff.data(), 8 * cnt);
    memcpy(host.data() + L.off[7], tiles.data(), 16 * tiles.size());
    memcpy(host.data() + L.off[8], tasks.data(), 8 * tasks.size());
}

BatchArgs make_args(const BatchRuntime& rt, void* dev, const DescLayout& L, u32 cnt, void* arena,
                    u32* status)
{
    BatchArgs a;
    a.wp = (const u32* const*)((char*)dev + L.off[0]);
    a.mp = (u32* const*)((char*)dev + L.off[1]);
    a.ns = (const u32*)((char*)dev + L.off[2]);
    a.queue = (const u32*)((char*)dev + L.off[3]);
    a.dts = (const uint8_t*)((char*)dev + L.off[4]);
    a.pst_off = (const u64*)((char*)dev + L.off[5]);
    a.row_off = (const u64*)((char*)dev + L.off[6]);
    a.posst = (u32*)arena;
    a.best0 = (u64*)((char*)arena + ((L.posst_words * 4 + 7) & ~(size_t)7));
    a.gfail = (u32*)((char*)arena + L.gfail_off);
    a.count = cnt;
    a.next = rt.d_next;
    a.slices = rt.d_slices;
    a.status = status;
    a.bin_cap = rt.bin_cap;
    a.warp_bins = rt.warp_bins;
    a.fill_rows = (u32)rt.tune.fill_rows;
    a.prim_max = rt.tune.prim_max < PRIM_WARP_MAX ? rt.tune.prim_max : PRIM_WARP_MAX;
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
    // dynamic shared memory of k_batched: per-warp contraction bins for up to
    // 1024 groups (the item path uses the same space as one bin array); the
    // fill kernel's tile
    nr->smem = (size_t)(BATCH_THREADS / 32) * 1024 * sizeof(u64);
    nr->bin_cap = (u32)(nr->smem / sizeof(u64));
    nr->warp_bins = (u32)(nr->bin_cap / (BATCH_THREADS / 32));
    nr->fill_smem = fill_smem_bytes((u32)tune.fill_rows);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nr->smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fill_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)nr->fill_smem);
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
        cudaFree(kv.second.arena);
    }
    cudaFree(rt->arena);
    cudaFree(rt->slice_mem);
    cudaFree(rt->d_slices);
    cudaFree(rt->scratch_mem);
    cudaFree(rt->d_next);
    cudaFree(rt->d_desc);
    delete rt;
}

int64_t batch_runtime_cap(const BatchRuntime* rt) { return rt->cap; }

cudaError_t batch_runtime_mark_failed(BatchRuntime* rt)
{
    if (!rt)
        return cudaSuccess;
    Workspace tmp;
    const size_t per = (workspace_layout(tmp, nullptr, rt->cap) + 255) & ~(size_t)255;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < rt->nslices && e == cudaSuccess; ++i) {
        Workspace w;
        workspace_layout(w, (char*)rt->slice_mem + per * i, rt->cap);
        const u32 one = 1u;
        e = cudaMemcpy(&w.ctr->bar.failed, &one, sizeof(u32), cudaMemcpyHostToDevice);
    }
    return e;
}

cudaError_t preload_batched()
{
    return touch_kernels(k_batched, k_fill_batched, k_rowmin_batched);
}

// Enqueues the batch's kernels on s: round-1 minima of every graph, queue
// reset, the per-graph MST and leaf order, the fill of every graph.
static void enqueue_batch(const BatchRuntime& rt, const BatchArgs& a, const void* dev, const DescLayout& L,
                          cudaStream_t s)
{
    if (L.ntasks)
        k_rowmin_batched<<<L.ntasks, ROWB_THREADS, 0, s>>>(a, (const uint2*)((const char*)dev + L.off[8]));
    cudaMemsetAsync(rt.d_next, 0, sizeof(u32), s);
    k_batched<<<rt.nslices, BATCH_THREADS, rt.smem, s>>>(a);
    if (L.ntiles)
        k_fill_batched<<<L.ntiles, FILLB_THREADS, rt.fill_smem, s>>>(a, (const uint4*)((const char*)dev + L.off[7]));
}

static u32 batch_launches(const DescLayout& L) { return 1u + (L.ntasks ? 1u : 0u) + (L.ntiles ? 1u : 0u); }

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
    const u32 fr = (u32)rt.tune.fill_rows;
    const u32 pm = rt.tune.prim_max < PRIM_WARP_MAX ? rt.tune.prim_max : PRIM_WARP_MAX;
    const DescLayout L = desc_layout(d, fr, pm);
    std::vector<unsigned char> host(L.bytes);
    if (!cache_graph) {
        // one descriptor block and one arena per runtime: launches on the
        // runtime are ordered on its stream, so the next upload follows the
        // last kernel
        // both grow to the next power of two (at least 4 MB): a growth
        // frees the old buffer, which waits for the whole device, so it must
        // stay rare when batches of changing size follow each other
        auto grow = [](size_t need) {
            size_t b = (size_t)4 << 20;
            while (b < need)
                b *= 2;
            return b;
        };
        if (rt.desc_bytes < L.bytes) {
            cudaFree(rt.d_desc);
            rt.d_desc = nullptr;
            rt.desc_bytes = 0;
            const size_t b = grow(L.bytes);
            if ((e = cudaMalloc(&rt.d_desc, b)) != cudaSuccess)
                return e;
            rt.desc_bytes = b;
        }
        if (rt.arena_bytes < L.arena_bytes) {
            cudaFree(rt.arena);
            rt.arena = nullptr;
            rt.arena_bytes = 0;
            const size_t b = grow(L.arena_bytes);
            if ((e = cudaMalloc(&rt.arena, b)) != cudaSuccess)
                return e;
            rt.arena_bytes = b;
        }
        fill_desc(d, fr, pm, L, host);
        // pageable source: the copy is staged before the call returns
        if ((e = cudaMemcpyAsync(rt.d_desc, host.data(), L.bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return e;
        BatchArgs a = make_args(rt, rt.d_desc, L, cnt, rt.arena, status);
        prof_launches(batch_launches(L));
        prof_begin(PH_BATCHED, s);
        enqueue_batch(rt, a, rt.d_desc, L, s);
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
        auto drop = [&]() {
            cudaFree(p.dev);
            cudaFree(p.arena);
        };
        if ((e = cudaMalloc(&p.dev, L.bytes)) != cudaSuccess)
            return e;
        if ((e = cudaMalloc(&p.arena, L.arena_bytes)) != cudaSuccess) {
            drop();
            return e;
        }
        fill_desc(d, fr, pm, L, host);
        if ((e = cudaMemcpy(p.dev, host.data(), L.bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
            drop();
            return e;
        }
        BatchArgs a = make_args(rt, p.dev, L, cnt, p.arena, status);
        cudaStream_t cap_s;
        if ((e = cudaStreamCreateWithFlags(&cap_s, cudaStreamNonBlocking)) != cudaSuccess) {
            drop();
            return e;
        }
        cudaGraph_t graph;
        e = cudaStreamBeginCapture(cap_s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_batch(rt, a, p.dev, L, cap_s);
            e = cudaStreamEndCapture(cap_s, &graph);
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&p.exec, graph, 0);
            cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cap_s);
        if (e != cudaSuccess) {
            drop();
            return e;
        }
        it = rt.plans.emplace(key, p).first;
    }
    prof_launches(batch_launches(L));
    prof_begin(PH_BATCHED, s);
    e = cudaGraphLaunch(it->second.exec, s);
    prof_end(PH_BATCHED, s);
    return e;
}

}  // namespace appd
