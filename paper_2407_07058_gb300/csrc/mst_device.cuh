// mst_device.cuh -- device code of the Boruvka MST shared by the single-solve
// kernels (mst_kernels.cu) and the batched kernel (batched.cu).
#pragma once

#include "internal.h"

namespace appd {

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
    u32 update_comp = 1;   // 0: the caller maps comp[] through label[] later
    unsigned short* label16 = nullptr;   // 16-bit copy of label[] (level 0 only)
};

// One Boruvka round's component bookkeeping, written once for a team (the
// grid of a cooperative launch, or one CTA of the batched kernel).
template <class Team>
__device__ void step_body(const Team& t, const StepArgs& a)
{
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
        u32 h = x, lo = 0, hi = 0;
        if (e != EDGE_INF)
            edge_ends(e, a.n, &lo, &hi);
        if (e != EDGE_INF && lo < a.n && hi < a.n) {
            u32 ca = a.comp[lo], cb = a.comp[hi];
            if (ca != x && cb != x)
                record_failure(a.status, &ctr->bar.failed, DEV_INTERNAL);
            h = (ca == x) ? cb : ca;
        } else {
            record_failure(a.status, &ctr->bar.failed, DEV_INTERNAL);
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
            record_failure(a.status, &ctr->bar.failed, DEV_INTERNAL);
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
        if (a.label16)
            a.label16[x] = (unsigned short)A;
        if (p != x)
            a.mst[mst_base + x - a.rootid[x]] = a.best_in[x];
        atomicAdd(&a.cnt[A], 1u);
    }
    if (!t.sync())
        return;
    if (a.update_comp)
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
    u32* comp = nullptr;   // vertex -> component, mapped through label[] here when
    u32 n = 0;             // this round's step left it (|C_r| <= comp_max_c)
    u32 comp_max_c = 0;
    const unsigned short* label16 = nullptr;   // level-0 labels as 16 bits (bulk-copy form)
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

// the same with an index that is a compile-time constant after unrolling
__device__ __forceinline__ u32 lane_of_dyn(const uint4& v, int c)
{
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// one column: the smallest key over the item's rows (first strictly smaller
// wins, rows ascending), packed with its endpoints, folded into bin L
template <int DT, int NR, int C>
__device__ __forceinline__ void column_w(const uint4* v, const u32* rid, u32 j, u32 L, u32 A, u32 b0,
                                         u32 nb, u64* bins, u32 n)
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
    const u64 e = pack_edge(bk, bi, j, n);
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
                                           u32 b0, u32 nb, u64* bins, u32 n)
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
        e[c] = pack_edge(bk, bi, j + c, n);
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
                    fold_group<DT, NR, false>(v[u], rid, 4 * g, lab[u], A, b0, nb, bins, cr);
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
        column_w<DT, NR, 0>(x, rid, j, label[j], A, b0, nb, bins, cr);
    }
}

// One column group (4 columns from j) of an upper-triangle pass: each
// column's smallest key over the pass's rows (rows ascending, first strictly
// smaller wins), packed with its endpoints and folded into bin L.  MASK:
// some row of the pass reaches column j + 3, so each row counts only right
// of its diagonal; otherwise every row counts at every column.  The chosen
// row is always left of the column, so (row, column) is already (lo, hi).
template <int DT, bool MASK>
__device__ __forceinline__ void fold_upper(const uint4* v, const u32* rid, u32 j, uint4 lab, u32 A,
                                           u32 b0, u32 nb, u64* bins, u32 n)
{
    constexpr int NR = 4;
    const u32 L[4] = {lab.x, lab.y, lab.z, lab.w};
    u64 e[4];
    u32 rel[4];
    bool ok[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const u32 col = j + c;
        rel[c] = L[c] - b0;
        ok[c] = (L[c] != A) && (rel[c] < nb) && (!MASK || col > rid[0]);
        u32 bk = key_of(lane_of_dyn(v[0], c), DT), bi = rid[0];
#pragma unroll
        for (int q = 1; q < NR; ++q) {
            const u32 k = key_of(lane_of_dyn(v[q], c), DT);
            if ((!MASK || col > rid[q]) && k < bk) {
                bk = k;
                bi = rid[q];
            }
        }
        e[c] = ((u64)bk << 32) | pair_code(bi, col, n);
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

// Column work of one item pass over the upper triangle of W only (level 0,
// W symmetric, 16-byte aligned rows): row q contributes its columns j >
// rows[q].  rows[] is ascending, so columns j <= rows[0] are skipped, row 0
// is valid wherever any row is (it seeds each column's minimum), and a
// row's column groups that lie wholly at or left of its diagonal are not
// loaded.  The result P(A, B) covers pairs a < b only, so
// C_1(A, B) = min(P(A, B), P(B, A)): C_1's row minima are P's row minima
// (this epilogue) folded with P's column minima (k_colmin_p), and level 1
// contracts P itself and symmetrizes its much smaller result (k_sym).
template <int DT>
__device__ __forceinline__ void contract_cols_w_upper(const u32* __restrict__ Wp, u32 cr,
                                                      const u32* __restrict__ label,
                                                      const u32* __restrict__ srows, u32 np, u32 A,
                                                      u32 b0, u32 nb, u64* bins)
{
    constexpr int NR = 4;
    const u32 tid = threadIdx.x, bd = blockDim.x;
    u32 rid[NR];
    const u32* rp[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        rid[q] = srows[(u32)q < np ? q : 0];
        rp[q] = Wp + (size_t)rid[q] * cr;
    }
    const u32 n4 = cr >> 2;
    const u32 rmax = rid[np - 1];   // the pass's largest row
    for (u32 g = ((rid[0] + 1) >> 2) + tid; g < n4; g += bd) {
        const u32 j = 4 * g;
        uint4 v[NR];
        v[0] = ld_stream_v4(rp[0] + j);
#pragma unroll
        for (int q = 1; q < NR; ++q)
            v[q] = ((u32)q < np && j + 3 > rid[q]) ? ld_stream_v4(rp[q] + j) : v[0];
        const uint4 lab = *reinterpret_cast<const uint4*>(label + j);
        if (j > rmax)
            fold_upper<DT, false>(v, rid, j, lab, A, b0, nb, bins, cr);
        else
            fold_upper<DT, true>(v, rid, j, lab, A, b0, nb, bins, cr);
    }
}

// Column work of one item pass of up to 8 rows of C_r (levels >= 1):
// entries are packed edges already, so a column reduces by a plain minimum;
// eight rows' loads are in flight before any is used.
__device__ __forceinline__ void contract_cols_c(const u64* __restrict__ Cp, u32 cr,
                                                const u32* __restrict__ label,
                                                const u32* __restrict__ srows, u32 np, u32 A, u32 b0,
                                                u32 nb, u64* bins)
{
    constexpr int NR = 8;
    const u32 tid = threadIdx.x, bd = blockDim.x;
    u32 rr[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q)
        rr[q] = srows[(u32)q < np ? q : 0];
    auto rowp = [&](int q) { return Cp + (size_t)rr[q] * cr; };
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
            v[0] = ld_stream_v4(rowp(0) + 2 * g);
#pragma unroll
            for (int q = 1; q < NR; ++q)
                v[q] = ((u32)q < np) ? ld_stream_v4(rowp(q) + 2 * g) : v[0];
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
        u64 e = rowp(0)[j];
#pragma unroll
        for (int q = 1; q < NR; ++q) {
            if ((u32)q < np) {
                u64 x = rowp(q)[j];
                e = x < e ? x : e;
            }
        }
        update(label[j], e);
    }
}

// One contraction work item: rows of group A (a chunk of at most
// CONTRACT_ROWS), one bin range.  Every thread of the CTA calls it; bins is
// the CTA's shared memory (>= min(cn, bin_cap) u64).  UPPER (level 0, VEC):
// upper-triangle pass; the row minima come from the symmetrization.
template <int DT, int LEVEL0, bool VEC, bool UPPER = false>
__device__ __forceinline__ void contract_item(const ContractArgs& a, u32 item, u32 cr, u32 cn,
                                              u32 total_chunks, u64* bins, u32* s_rows, u64* s_red)
{
    const u32 tid = threadIdx.x, bd = blockDim.x;
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
    // rows in passes of at most 4 (W) or 8 (C_r, cheaper per entry) for the
    // register budget; bins merge passes
    for (u32 p0 = 0; p0 < nrows; p0 += (LEVEL0 ? 4u : 8u)) {
        const u32 np = min(LEVEL0 ? 4u : 8u, nrows - p0);
        if (LEVEL0 && UPPER)
            contract_cols_w_upper<DT>((const u32*)a.cin, cr, a.label, s_rows + p0, np, A, b0, nb, bins);
        else if (LEVEL0)
            contract_cols_w<DT, VEC>((const u32*)a.cin, cr, a.label, s_rows + p0, np, A, b0, nb, bins);
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

}  // namespace appd
