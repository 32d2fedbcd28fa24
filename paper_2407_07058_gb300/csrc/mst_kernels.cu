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

#include "internal.h"

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

// --------------------------------------------------- Boruvka step (K2)
struct StepArgs {
    int level;
    u32 n;
    const u64* best_in;
    u64* best_out;
    u32 *comp, *hook, *par, *flag, *rootid, *label, *cnt, *fillc, *gstart, *members, *nchunk,
        *chunk_start, *item_group;
    u64* mst;
    u64* cnext;
    u32* part;
    Counters* ctr;
    u32* status;
    u32 bin_cap;
};

__global__ void k_step(StepArgs a)
{
    GridTeam t{&a.ctr->bar, a.status};
    Counters* ctr = a.ctr;
    if (*(volatile u32*)&ctr->done)
        return;
    const int r = a.level;
    const u32 c = ((volatile u32*)ctr->c)[r];
    const u32 me = t.rank(), ts = t.size();
    const u32 mst_base = *(volatile u32*)&ctr->mst_count;

    // hook: the other end of each component's best edge
    for (u32 x = me; x < c; x += ts) {
        u64 e = a.best_in[x];
        u32 h = x;
        if (e != EDGE_INF && edge_lo(e) < a.n && edge_hi(e) < a.n) {
            u32 ca = a.comp[edge_lo(e)], cb = a.comp[edge_hi(e)];
            if (ca != x && cb != x)
                atomicOr(a.status, DEV_INTERNAL);
            h = (ca == x) ? cb : ca;
        } else {
            atomicOr(a.status, DEV_INTERNAL);
        }
        a.hook[x] = h < c ? h : x;
        a.cnt[x] = 0;
        a.fillc[x] = 0;
    }
    if (!t.sync())
        return;
    // mutual pairs share their best edge; the smaller id becomes the root
    for (u32 x = me; x < c; x += ts) {
        u32 b = a.hook[x];
        bool root = (b < c && a.hook[b] == x && x < b);
        a.par[x] = root ? x : (b < c ? b : x);
    }
    if (!t.sync())
        return;
    // pointer jumping to the roots; three rotating flags so that resetting
    // the next round's flag never races with a late reader of this one
    for (int it = 0; it < 64; ++it) {
        volatile u32* fl = (volatile u32*)ctr->jump_flag;
        if (me == 0)
            fl[(it + 1) % 3] = 0;
        bool changed = false;
        for (u32 x = me; x < c; x += ts) {
            u32 p = a.par[x], pp = a.par[p];
            if (p != pp) {
                a.par[x] = pp;
                changed = true;
            }
        }
        if (changed)
            fl[it % 3] = 1;
        if (!t.sync())
            return;
        if (fl[it % 3] == 0)
            break;
        if (it == 63 && me == 0)
            atomicOr(a.status, DEV_INTERNAL);
    }
    for (u32 x = me; x < c; x += ts)
        a.flag[x] = (a.par[x] == x) ? 1u : 0u;
    if (!t.sync())
        return;
    u32 cn = 0;
    if (!team_excl_scan(t, a.flag, a.rootid, c, a.part, &cn))
        return;
    if (!t.sync())
        return;
    // relabel, record MST edges of hooked components, group sizes
    for (u32 x = me; x < c; x += ts) {
        u32 p = a.par[x];
        u32 A = a.rootid[p];
        a.label[x] = A;
        if (p != x)
            a.mst[mst_base + x - a.rootid[x]] = a.best_in[x];
        atomicAdd(&a.cnt[A], 1u);
    }
    if (!t.sync())
        return;
    for (u32 v = me; v < a.n; v += ts)
        a.comp[v] = a.label[a.comp[v]];
    for (u32 A = me; A < cn; A += ts) {
        a.nchunk[A] = (a.cnt[A] + CONTRACT_ROWS - 1) / CONTRACT_ROWS;
        a.best_out[A] = EDGE_INF;
    }
    if (!t.sync())
        return;
    u32 csum = 0, total_chunks = 0;
    if (!team_excl_scan(t, a.cnt, a.gstart, cn, a.part, &csum))
        return;
    if (!t.sync())
        return;
    if (!team_excl_scan(t, a.nchunk, a.chunk_start, cn, a.part, &total_chunks))
        return;
    if (!t.sync())
        return;
    // scatter component members; map chunks to groups; init multi-chunk rows
    for (u32 x = me; x < c; x += ts) {
        u32 A = a.label[x];
        u32 s = atomicAdd(&a.fillc[A], 1u);
        a.members[a.gstart[A] + s] = x;
    }
    for (u32 A = me; A < cn; A += ts) {
        u32 s0 = a.chunk_start[A], k = a.nchunk[A];
        for (u32 q = 0; q < k; ++q)
            a.item_group[s0 + q] = A;
    }
    if (cn > 1) {
        for (u32 A = t.block(); A < cn; A += t.nblocks()) {
            if (a.nchunk[A] > 1) {
                u64* row = a.cnext + (size_t)A * cn;
                for (u32 b = threadIdx.x; b < cn; b += blockDim.x)
                    row[b] = EDGE_INF;
            }
        }
    }
    if (me == 0) {
        a.gstart[cn] = c;
        a.chunk_start[cn] = total_chunks;
        ctr->c[r + 1] = cn;
        ctr->total_chunks = total_chunks;
        ctr->nbr = (cn + a.bin_cap - 1) / a.bin_cap;
        ctr->item_next = 0;
        ctr->mst_count = mst_base + (c - cn);
        if (cn <= 1)
            ctr->done = 1;
    }
}

// ------------------------------------------------------ contraction (K3)
struct ContractArgs {
    int level;
    const void* cin;     // W (level 0) or C_r
    u64* cout;           // C_{r+1}
    u64* best_out;
    const u32 *label, *members, *gstart, *nchunk, *chunk_start, *item_group;
    Counters* ctr;
    u32 bin_cap;
};

// Column work of one contraction item with NR rows of W (level 0).  rows[]
// holds the item's rows in ascending order, so within a column "first
// strictly smaller key" is the packed-edge order.  U column groups are loaded
// before any is consumed, so that few-row items still keep enough 16-byte
// loads in flight.
template <int C>
__device__ __forceinline__ u32 lane_of(const uint4& v)
{
    return C == 0 ? v.x : (C == 1 ? v.y : (C == 2 ? v.z : v.w));
}

// one column: the smallest key over the item's rows (first strictly smaller
// wins, rows ascending), packed with its endpoints, folded into bin L
template <int DT, int NR, int C>
__device__ __forceinline__ void column_w(const uint4* v, const u32* rid, u32 j, u32 L, u32 A, u32 b0,
                                         u32 nb, u64* bins)
{
    const u32 rel = L - b0;
    if (L == A || rel >= nb)
        return;
    u32 bk = key_of(lane_of<C>(v[0]), DT), bi = rid[0];
#pragma unroll
    for (int q = 1; q < NR; ++q) {
        const u32 k = key_of(lane_of<C>(v[q]), DT);
        if (k < bk) {
            bk = k;
            bi = rid[q];
        }
    }
    const u64 e = pack_edge(bk, bi, j);
    u64* slot = &bins[rel];
    if (e < *slot)
        atomicMin(slot, e);
}

// Folds the 4 columns of one group (columns j..j+3, labels lab) into the
// bins.  All four bins are read before any atomic: a stale read can only
// cause a redundant atomicMin, never a lost update, and the four shared
// loads then overlap instead of forming one dependent chain.
template <int DT, int NP, bool ONE>
__device__ __forceinline__ void fold_group(const uint4* x, const u32* rid, u32 j, uint4 lab, u32 A,
                                           u32 b0, u32 nb, u64* bins)
{
    u32 L[4] = {lab.x, lab.y, lab.z, lab.w};
    u64 e[4];
    u32 rel[4];
    bool ok[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        rel[c] = ONE ? L[c] : L[c] - b0;
        ok[c] = (L[c] != A) && (ONE || rel[c] < nb);
        u32 v0 = c == 0 ? x[0].x : (c == 1 ? x[0].y : (c == 2 ? x[0].z : x[0].w));
        u32 bk = key_of(v0, DT), bi = rid[0];
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            u32 vq = c == 0 ? x[q].x : (c == 1 ? x[q].y : (c == 2 ? x[q].z : x[q].w));
            const u32 k = key_of(vq, DT);
            if (k < bk) {
                bk = k;
                bi = rid[q];
            }
        }
        e[c] = pack_edge(bk, bi, j + c);
    }
    u64 cur[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        cur[c] = ok[c] ? bins[rel[c]] : 0ull;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (ok[c] && e[c] < cur[c])
            atomicMin(&bins[rel[c]], e[c]);
}

template <int DT, bool VEC>
__device__ __forceinline__ void contract_cols_w(const u32* __restrict__ Wp, u32 cr,
                                                const u32* __restrict__ label,
                                                const u32* __restrict__ srows, u32 np, u32 A, u32 b0,
                                                u32 nb, u64* bins)
{
    // up to 4 rows per pass; rows past np repeat row 0 (same key and row, so
    // they never change a column's minimum) without being loaded again
    constexpr int NR = 4, U = 1;
    const u32 tid = threadIdx.x, bd = blockDim.x;
    u32 rid[NR];
    const u32* rp[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        rid[q] = srows[(u32)q < np ? q : 0];
        rp[q] = Wp + (size_t)rid[q] * cr;
    }
    u32 jt = 0;
    if (VEC) {
        const u32 n4 = cr >> 2;
        for (u32 g0 = tid; g0 < n4; g0 += U * bd) {
            uint4 v[U][NR];
            uint4 lab[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const u32 g = g0 + u * bd;
                if (g < n4) {
                    v[u][0] = ld_stream_v4(rp[0] + 4 * g);
#pragma unroll
                    for (int q = 1; q < NR; ++q)
                        v[u][q] = ((u32)q < np) ? ld_stream_v4(rp[q] + 4 * g) : v[u][0];
                    lab[u] = *reinterpret_cast<const uint4*>(label + 4 * g);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const u32 g = g0 + u * bd;
                if (g < n4)
                    fold_group<DT, NR, false>(v[u], rid, 4 * g, lab[u], A, b0, nb, bins);
            }
        }
        jt = 4 * n4;
    }
    for (u32 j = jt + tid; j < cr; j += bd) {
        uint4 x[NR];
        x[0].x = ld_stream_u32(rp[0] + j);
#pragma unroll
        for (int q = 1; q < NR; ++q)
            x[q].x = ((u32)q < np) ? ld_stream_u32(rp[q] + j) : x[0].x;
        column_w<DT, NR, 0>(x, rid, j, label[j], A, b0, nb, bins);
    }
}

// Column work of one item pass of up to 4 rows of C_r (levels >= 1):
// entries are packed edges already, so a column reduces by a plain minimum.
__device__ __forceinline__ void contract_cols_c(const u64* __restrict__ Cp, u32 cr,
                                                const u32* __restrict__ label,
                                                const u32* __restrict__ srows, u32 np, u32 A, u32 b0,
                                                u32 nb, u64* bins)
{
    constexpr int NR = 4;
    const u32 tid = threadIdx.x, bd = blockDim.x;
    const u64* rp[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q)
        rp[q] = Cp + (size_t)srows[(u32)q < np ? q : 0] * cr;
    auto update = [&](u32 L, u64 e) {
        u32 rel = L - b0;
        if (L != A && rel < nb) {
            u64* slot = &bins[rel];
            if (e < *slot)
                atomicMin(slot, e);
        }
    };
    u32 jt = 0;
    if (((cr & 1u) == 0) && (((uintptr_t)Cp & 15u) == 0)) {
        const u32 n2 = cr >> 1;
        for (u32 g = tid; g < n2; g += bd) {
            uint4 v[NR];
            v[0] = ld_stream_v4(rp[0] + 2 * g);
#pragma unroll
            for (int q = 1; q < NR; ++q)
                v[q] = ((u32)q < np) ? ld_stream_v4(rp[q] + 2 * g) : v[0];
            const uint2 lab = *reinterpret_cast<const uint2*>(label + 2 * g);
            u64 e0 = EDGE_INF, e1 = EDGE_INF;
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                u64 x0 = ((u64)v[q].y << 32) | v[q].x;
                u64 x1 = ((u64)v[q].w << 32) | v[q].z;
                e0 = x0 < e0 ? x0 : e0;
                e1 = x1 < e1 ? x1 : e1;
            }
            update(lab.x, e0);
            update(lab.y, e1);
        }
        jt = 2 * n2;
    }
    for (u32 j = jt + tid; j < cr; j += bd) {
        u64 e = rp[0][j];
#pragma unroll
        for (int q = 1; q < NR; ++q) {
            if ((u32)q < np) {
                u64 x = rp[q][j];
                e = x < e ? x : e;
            }
        }
        update(label[j], e);
    }
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
    const u32 tid = threadIdx.x, bd = blockDim.x;

    for (;;) {
        if (tid == 0)
            s_item = atomicAdd(&ctr->item_next, 1u);
        __syncthreads();
        const u32 item = s_item;
        if (item >= total)
            break;
        const u32 br = item / total_chunks, ch = item - br * total_chunks;
        const u32 A = a.item_group[ch];
        const u32 k = ch - a.chunk_start[A];
        const u32 m0 = a.gstart[A] + k * CONTRACT_ROWS;
        const u32 m1 = min(a.gstart[A + 1], m0 + CONTRACT_ROWS);
        const u32 nrows = m1 - m0;
        const bool single = a.nchunk[A] == 1;
        const u32 b0 = br * a.bin_cap;
        const u32 nb = min(cn - b0, a.bin_cap);
        if (tid < nrows)
            s_rows[tid] = a.members[m0 + tid];
        for (u32 b = tid; b < nb; b += bd)
            bins[b] = EDGE_INF;
        __syncthreads();
        if (LEVEL0 && tid == 0) {
            for (u32 i = 1; i < nrows; ++i) {
                u32 v = s_rows[i], j = i;
                while (j > 0 && s_rows[j - 1] > v) {
                    s_rows[j] = s_rows[j - 1];
                    --j;
                }
                s_rows[j] = v;
            }
        }
        __syncthreads();
        // rows in passes of at most 4 (register budget); bins merge passes
        for (u32 p0 = 0; p0 < nrows; p0 += 4) {
            const u32 np = min(4u, nrows - p0);
            if (LEVEL0)
                contract_cols_w<DT, VEC>((const u32*)a.cin, cr, a.label, s_rows + p0, np, A, b0, nb,
                                         bins);
            else
                contract_cols_c((const u64*)a.cin, cr, a.label, s_rows + p0, np, A, b0, nb, bins);
        }
        __syncthreads();
        // write row A of C_{r+1} (this bin range) and fold the row minimum
        u64 m = EDGE_INF;
        u64* dst = a.cout + (size_t)A * cn + b0;
        for (u32 b = tid; b < nb; b += bd) {
            u64 v = bins[b];
            if (single)
                dst[b] = v;
            else if (v != EDGE_INF)
                atomicMin(dst + b, v);
            m = v < m ? v : m;
        }
        m = block_min_u64(m, s_red);
        if (tid == 0 && m != EDGE_INF)
            atomicMin(&a.best_out[A], m);
        __syncthreads();
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
        err = cudaMemsetAsync(&ws.ctr->bar.count, 0, sizeof(u32), s);
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
