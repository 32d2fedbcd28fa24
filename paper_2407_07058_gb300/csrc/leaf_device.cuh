// leaf_device.cuh -- device code of the leaf order shared by the single-solve
// kernel (leaf_order.cu) and the batched kernel (batched.cu).
#pragma once

#include "internal.h"

namespace appd {

struct LeafArgs {
    u32 n;
    int levels;      // binary-lifting levels (>= 1)
    int st_levels;   // sparse-table levels over n-1 gaps
    const u64* mst;  // n-1 packed edges
    u32 *deg, *adj_off, *afill, *adj, *aslot;
    u32 *lr_d0, *lr_d1, *lr_nx0, *lr_nx1;
    u32 *parent, *pe_key;
    u64* ord;
    u32* jump;
    u64* mxo;
    u32* nha;
    u64 *skey0, *skey1;
    u32 *sval0, *sval1;   // the child vertex carried beside each sort key
    u32* hist;
    u32 ntiles;
    u32 *first_child, *next_sib;
    u32 *pos, *order, *nsize, *gap, *st;
    u32* part;
    Counters* ctr;
    u32* status;
};

constexpr u32 LR_END = 0xFFFFFFFFu;
constexpr int SORT_TILE = 2048;
constexpr int SORT_NW = 16;   // warps of a 512-thread CTA

// Wyllie list ranking: d[a] becomes the sum of weights from a to the end of
// its list (inclusive).  Returns the buffer index that holds the result.
template <class Team>
__device__ int list_rank(const Team& t, u32 na, u32* d0, u32* d1, u32* x0, u32* x1, int rounds,
                         bool* ok)
{
    u32 *dc = d0, *dn = d1, *xc = x0, *xn = x1;
    int cur = 0;
    for (int it = 0; it < rounds; ++it) {
        for (u32 a = t.rank(); a < na; a += t.size()) {
            u32 nx = xc[a];
            if (nx != LR_END) {
                dn[a] = dc[a] + dc[nx];
                xn[a] = xc[nx];
            } else {
                dn[a] = dc[a];
                xn[a] = LR_END;
            }
        }
        if (!t.sync()) {
            *ok = false;
            return cur;
        }
        u32* tmp = dc;
        dc = dn;
        dn = tmp;
        tmp = xc;
        xc = xn;
        xn = tmp;
        cur ^= 1;
    }
    *ok = true;
    return cur;
}

// All phases of the leaf order for one team (the grid of a cooperative
// launch, or one 512-thread CTA of the batched kernel).
template <class Team>
__device__ void leaf_body(const Team& t, const LeafArgs& a)
{
    const u32 n = a.n, m = n - 1, na = 2 * m;
    const u32 me = t.rank(), ts = t.size();
    // an earlier phase of this solve failed: the tree may be incomplete
    if (solve_failed(&a.ctr->bar))
        return;
    __shared__ u32 s_cnt[256];
    __shared__ u32 s_off[256];
    __shared__ u32 s_wc[SORT_NW][256];

    // ---- adjacency of the MST
    for (u32 v = me; v < n; v += ts) {
        a.deg[v] = 0;
        a.afill[v] = 0;
        a.first_child[v] = NONE32;
    }
    if (!t.sync())
        return;
    for (u32 e = me; e < m; e += ts) {
        u32 lo, hi;
        edge_ends(a.mst[e], n, &lo, &hi);
        atomicAdd(&a.deg[lo], 1u);
        atomicAdd(&a.deg[hi], 1u);
    }
    if (!t.sync())
        return;
    u32 tot = 0;
    if (!team_excl_scan(t, a.deg, a.adj_off, n, a.part, &tot))
        return;
    if (!t.sync())
        return;
    for (u32 e = me; e < m; e += ts) {
        u32 lo, hi;
        edge_ends(a.mst[e], n, &lo, &hi);
        u32 s0 = atomicAdd(&a.afill[lo], 1u);
        a.adj[a.adj_off[lo] + s0] = 2 * e;       // arc lo -> hi
        a.aslot[2 * e] = s0;
        u32 s1 = atomicAdd(&a.afill[hi], 1u);
        a.adj[a.adj_off[hi] + s1] = 2 * e + 1;   // arc hi -> lo
        a.aslot[2 * e + 1] = s1;
    }
    if (!t.sync())
        return;
    // ---- Euler tour successor of every arc; the tour starts at vertex 0
    const u32 first = a.adj[a.adj_off[0]];
    for (u32 x = me; x < na; x += ts) {
        u32 elo, ehi;
        edge_ends(a.mst[x >> 1], n, &elo, &ehi);
        u32 dst = (x & 1) ? elo : ehi;
        u32 sl = a.aslot[x ^ 1u] + 1;
        if (sl == a.deg[dst])
            sl = 0;
        u32 nx = a.adj[a.adj_off[dst] + sl];
        if (nx == first)
            nx = LR_END;
        a.lr_nx0[x] = nx;
        a.lr_d0[x] = (nx == LR_END) ? 0u : 1u;
    }
    if (!t.sync())
        return;
    bool ok = true;
    int rounds = ceil_log2_dev(na) + 1;
    int which = list_rank(t, na, a.lr_d0, a.lr_d1, a.lr_nx0, a.lr_nx1, rounds, &ok);
    if (!ok)
        return;
    const u32* dist = which ? a.lr_d1 : a.lr_d0;   // arcs after this one
    // ---- orientation: the earlier arc of an edge goes down the tree
    for (u32 e = me; e < m; e += ts) {
        u64 x = a.mst[e];
        u32 lo, hi;
        edge_ends(x, n, &lo, &hi);
        const u32 key = edge_key(x);
        bool down_lo_hi = dist[2 * e] > dist[2 * e + 1];   // more arcs after it == earlier
        u32 child = down_lo_hi ? hi : lo, par = down_lo_hi ? lo : hi;
        a.parent[child] = par;
        a.pe_key[child] = key;
        a.ord[child] = ((u64)key << 32) | child;
    }
    if (me == 0) {
        a.parent[0] = 0;
        a.pe_key[0] = 0;
        a.ord[0] = EDGE_INF;
    }
    if (!t.sync())
        return;
    // ---- binary lifting: jump[k][v] = 2^k-th ancestor, mxo[k][v] = max ord
    // over v and its next 2^k - 1 ancestors (the root's ord is infinite)
    for (u32 v = me; v < n; v += ts) {
        a.jump[v] = a.parent[v];
        a.mxo[v] = a.ord[v];
    }
    if (!t.sync())
        return;
    // two levels per phase from the last complete one: level k is jump^2 of
    // level k-1 and level k+1 its jump^4, with the maxima over the same hops
    for (int k = 1; k < a.levels; k += 2) {
        const u32* jp = a.jump + (size_t)(k - 1) * n;
        const u64* mp = a.mxo + (size_t)(k - 1) * n;
        u32* jc = a.jump + (size_t)k * n;
        u64* mc = a.mxo + (size_t)k * n;
        const bool two = k + 1 < a.levels;
        for (u32 v = me; v < n; v += ts) {
            const u32 j1 = jp[v], j2 = jp[j1];
            const u64 m01 = mp[v] > mp[j1] ? mp[v] : mp[j1];
            jc[v] = j2;
            mc[v] = m01;
            if (two) {
                const u32 j3 = jp[j2];
                const u64 m23 = mp[j2] > mp[j3] ? mp[j2] : mp[j3];
                jc[(size_t)n + v] = jp[j3];
                mc[(size_t)n + v] = m01 > m23 ? m01 : m23;
            }
        }
        if (!t.sync())
            return;
    }
    // ---- nearest heavier ancestor, and the sort keys (nha, key of y's
    // parent edge) with y carried beside them
    for (u32 y = me + 1; y < n; y += ts) {
        u32 z = a.parent[y];
        const u64 tg = a.ord[y];
        for (int k = a.levels - 1; k >= 0; --k) {
            if (a.mxo[(size_t)k * n + z] < tg)
                z = a.jump[(size_t)k * n + z];
        }
        a.nha[y] = z;
        a.skey0[y - 1] = ((u64)z << 32) | a.pe_key[y];
        a.sval0[y - 1] = y;
    }
    if (!t.sync())
        return;
    // ---- stable LSD radix sort of the keys, 8 bits per pass over the key
    // and the bits that nha needs; the input is in increasing y, so equal
    // keys keep y ascending and the order is (nha, ord)
    const int passes = (32 + ceil_log2_dev(n) + 7) / 8;
    {
        u64* in = a.skey0;
        u64* out = a.skey1;
        u32* vin = a.sval0;
        u32* vout = a.sval1;
        const u32 ntiles = a.ntiles;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int pass = 0; pass < passes; ++pass) {
            const int shift = 8 * pass;
            for (u32 tile = t.block(); tile < ntiles; tile += t.nblocks()) {
                for (u32 d = threadIdx.x; d < 256; d += blockDim.x)
                    s_cnt[d] = 0;
                __syncthreads();
                const u32 b0 = tile * SORT_TILE, b1 = min(m, b0 + SORT_TILE);
                for (u32 i = b0 + threadIdx.x; i < b1; i += blockDim.x)
                    atomicAdd(&s_cnt[(u32)(in[i] >> shift) & 255u], 1u);
                __syncthreads();
                for (u32 d = threadIdx.x; d < 256; d += blockDim.x)
                    a.hist[d * ntiles + tile] = s_cnt[d];
                __syncthreads();
            }
            if (!t.sync())
                return;
            u32 htot = 0;
            if (!team_excl_scan(t, a.hist, a.hist, 256 * ntiles, a.part, &htot))
                return;
            if (!t.sync())
                return;
            for (u32 tile = t.block(); tile < ntiles; tile += t.nblocks()) {
                for (u32 d = threadIdx.x; d < 256; d += blockDim.x) {
                    s_off[d] = a.hist[d * ntiles + tile];
                    s_cnt[d] = 0;   // running count of this tile
                }
                const u32 b0 = tile * SORT_TILE, b1 = min(m, b0 + SORT_TILE);
                for (u32 base = b0; base < b1; base += blockDim.x) {
                    const u32 i = base + threadIdx.x;
                    const bool valid = i < b1;
                    const u64 key = valid ? in[i] : 0ull;
                    const u32 val = valid ? vin[i] : 0u;
                    const u32 d = valid ? ((u32)(key >> shift) & 255u) : (256u + lane);
                    const u32 peers = __match_any_sync(0xFFFFFFFFu, d);
                    const u32 rank_w = __popc(peers & ((1u << lane) - 1u));
                    for (u32 x = threadIdx.x; x < SORT_NW * 256; x += blockDim.x)
                        (&s_wc[0][0])[x] = 0;
                    __syncthreads();
                    if (valid && rank_w == 0)
                        s_wc[w][d] = __popc(peers);
                    __syncthreads();
                    for (u32 dd = threadIdx.x; dd < 256; dd += blockDim.x) {
                        u32 run = s_cnt[dd];
                        for (int ww = 0; ww < SORT_NW; ++ww) {
                            u32 c = s_wc[ww][dd];
                            s_wc[ww][dd] = run;
                            run += c;
                        }
                        s_cnt[dd] = run;
                    }
                    __syncthreads();
                    if (valid) {
                        const u32 dst = s_off[d] + s_wc[w][d] + rank_w;
                        out[dst] = key;
                        vout[dst] = val;
                    }
                    __syncthreads();
                }
            }
            if (!t.sync())
                return;
            u64* tmp = in;
            in = out;
            out = tmp;
            u32* vt = vin;
            vin = vout;
            vout = vt;
        }
    }
    // the sorted keys are in skey0 after an even number of passes
    const u64* sk = (passes & 1) ? a.skey1 : a.skey0;
    const u32* sv = (passes & 1) ? a.sval1 : a.sval0;
    // ---- first child / next sibling of the nearest-heavier-ancestor tree
    for (u32 i = me; i < m; i += ts) {
        const u32 p = (u32)(sk[i] >> 32), y = sv[i];
        if (i == 0 || (u32)(sk[i - 1] >> 32) != p)
            a.first_child[p] = y;
        a.next_sib[y] = (i + 1 < m && (u32)(sk[i + 1] >> 32) == p) ? sv[i + 1] : NONE32;
    }
    if (!t.sync())
        return;
    // ---- preorder by an Euler tour of that tree: arc 2v goes down into v,
    // 2v+1 comes back up; down arcs weigh 1
    for (u32 x = me; x < 2 * n; x += ts) {
        u32 v = x >> 1, nx, wgt;
        if (v == 0) {
            nx = LR_END;
            wgt = 0;
        } else if ((x & 1) == 0) {
            u32 fc = a.first_child[v];
            nx = fc != NONE32 ? 2 * fc : 2 * v + 1;
            wgt = 1;
        } else {
            u32 ns = a.next_sib[v];
            u32 p = a.nha[v];
            nx = ns != NONE32 ? 2 * ns : (p == 0 ? LR_END : 2 * p + 1);
            wgt = 0;
        }
        a.lr_nx0[x] = nx;
        a.lr_d0[x] = wgt;
    }
    if (!t.sync())
        return;
    rounds = ceil_log2_dev(2 * n) + 1;
    which = list_rank(t, 2 * n, a.lr_d0, a.lr_d1, a.lr_nx0, a.lr_nx1, rounds, &ok);
    if (!ok)
        return;
    const u32* suf = which ? a.lr_d1 : a.lr_d0;   // down arcs from here to the end
    for (u32 v = me; v < n; v += ts) {
        if (v == 0) {
            a.pos[0] = 0;
            a.order[0] = 0;
            a.nsize[0] = n;
        } else {
            u32 sd = suf[2 * v];
            if (sd < 1 || sd > n - 1) {   // not a tree: report, never write out of range
                record_failure(a.status, &a.ctr->bar.failed, DEV_INTERNAL);
                continue;
            }
            u32 p = n - sd;
            a.pos[v] = p;
            a.order[p] = v;
            a.gap[p - 1] = a.pe_key[v];
            a.nsize[v] = sd - suf[2 * v + 1];
        }
    }
    if (!t.sync())
        return;
    // ---- sparse table over gap[0..m)
    for (u32 x = me; x < m; x += ts)
        a.st[x] = a.gap[x];
    if (!t.sync())
        return;
    // two levels per phase from the last complete one (level k - 1):
    // level k from two of its entries, level k + 1 from four
    for (int k = 1; k < a.st_levels; k += 2) {
        const u32* sp = a.st + (size_t)(k - 1) * n;
        u32* sc = a.st + (size_t)k * n;
        const u32 h = 1u << (k - 1);
        const bool two = k + 1 < a.st_levels;
        for (u32 x = me; x + 2 * h <= m; x += ts) {
            const u32 p = sp[x], q = sp[x + h];
            const u32 m01 = p > q ? p : q;
            sc[x] = m01;
            if (two && x + 4 * h <= m) {
                const u32 r = sp[x + 2 * h], s = sp[x + 3 * h];
                const u32 m23 = r > s ? r : s;
                sc[(size_t)n + x] = m01 > m23 ? m01 : m23;
            }
        }
        if (!t.sync())
            return;
    }
}

}  // namespace appd
