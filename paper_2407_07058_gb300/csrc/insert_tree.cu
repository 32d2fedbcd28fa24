// insert_tree.cu -- warm start by a tree update (Section 6.1's warm start,
// done through the minimum spanning tree).
//
// A minimum spanning tree T of G and the weights w(k) of a new vertex p's
// edges determine the tree of G + p: every edge of G outside T is the largest
// on a cycle of G's edges, which stays a cycle in G + p, so the minimum
// spanning tree of G + p uses only T's n - 1 edges and p's n edges.  The new
// tree is found by Boruvka's algorithm on those 2n - 1 edges, O(n log n)
// work; the leaf order and the fill of the (n + 1) x (n + 1) matrix then run
// as in a solve.  M of G is not read at all: the cost is one write of the
// new matrix, plus work linear in n up to a logarithm.
//
// Each Boruvka round, for the current components (each named by a
// representative vertex): every edge whose ends lie in different components
// offers itself to both by a 64-bit atomic minimum on the packed edge (the
// strict order (key, lo, hi), so the choice is unique); every component hooks
// to the other end of its best edge; of a mutual pair the smaller
// representative stays a root and the other records the shared edge; pointer
// jumping brings every component to its root.  The graph is connected, so
// every round at least halves the components.
#include "leaf_device.cuh"

namespace appd {

struct TreeInsArgs {
    const u32 *keys, *lo, *hi;   // T: n - 1 edges (order keys, endpoints lo < hi)
    const u32* w;                // p's n weights
    u32 n;                       // vertices of G; p is vertex n
    int dt;
    u32 *comp, *par, *root;      // n + 1 each
    u64* best;                   // n + 1
    u64* mst;                    // n: the new tree, packed for n + 1 vertices
    Counters* ctr;
    u32* status;
};

// packed edge e of T + star(p), numbered T's edges first
__device__ __forceinline__ u64 ins_edge(const TreeInsArgs& a, u32 e, u32 N)
{
    if (e + 1 < a.n)
        return ((u64)a.keys[e] << 32) | pair_code(a.lo[e], a.hi[e], N);
    const u32 k = e - (a.n - 1);
    return ((u64)key_of(a.w[k], a.dt) << 32) | pair_code(k, a.n, N);
}

constexpr int INS_MAX_ROUNDS = 40;

template <class Team>
__device__ void tree_insert_body(const Team& t, const TreeInsArgs& a)
{
    Counters* ctr = a.ctr;
    const u32 N = a.n + 1, E = 2 * a.n - 1;
    const u32 me = t.rank(), ts = t.size();
    for (u32 v = me; v < N; v += ts)
        a.comp[v] = v;
    if (me == 0) {
        ctr->mst_count = 0;
        ctr->jump_flag[0] = ctr->jump_flag[1] = ctr->jump_flag[2] = 0;
    }
    if (!t.sync())
        return;
    bool complete = false;
    for (int round = 0; round < INS_MAX_ROUNDS; ++round) {
        if (*(volatile u32*)&ctr->mst_count >= a.n) {
            complete = true;
            break;
        }
        for (u32 v = me; v < N; v += ts)
            if (a.comp[v] == v)
                a.best[v] = EDGE_INF;
        if (!t.sync())
            return;
        for (u32 e = me; e < E; e += ts) {
            const u64 x = ins_edge(a, e, N);
            u32 u, v;
            edge_ends(x, N, &u, &v);
            const u32 cu = a.comp[u], cv = a.comp[v];
            if (cu != cv) {
                if (x < a.best[cu])
                    atomicMin(&a.best[cu], x);
                if (x < a.best[cv])
                    atomicMin(&a.best[cv], x);
            }
        }
        if (!t.sync())
            return;
        // hook to the other end's component
        for (u32 c = me; c < N; c += ts) {
            if (a.comp[c] != c)
                continue;
            const u64 x = a.best[c];
            u32 h = c;
            if (x != EDGE_INF) {
                u32 u, v;
                edge_ends(x, N, &u, &v);
                const u32 cu = a.comp[u], cv = a.comp[v];
                if (cu != c && cv != c)
                    record_failure(a.status, &ctr->bar.failed, DEV_INTERNAL);
                h = (cu == c) ? cv : cu;
            }
            a.par[c] = h;
        }
        if (!t.sync())
            return;
        // of a mutual pair the smaller representative stays a root; every
        // other hooked component records its edge
        for (u32 c = me; c < N; c += ts) {
            if (a.comp[c] != c)
                continue;
            const u32 h = a.par[c];
            const bool keep_root = (h == c) || (a.par[h] == c && c < h);
            a.root[c] = keep_root ? 1u : 0u;
            if (!keep_root) {
                const u32 slot = atomicAdd(&ctr->mst_count, 1u);
                if (slot < a.n)
                    a.mst[slot] = a.best[c];
                else
                    record_failure(a.status, &ctr->bar.failed, DEV_INTERNAL);
            }
        }
        if (!t.sync())
            return;
        for (u32 c = me; c < N; c += ts)
            if (a.comp[c] == c && a.root[c])
                a.par[c] = c;
        if (!t.sync())
            return;
        // pointer jumping over the representatives (three rotating flags, so
        // resetting the next one never races with a late reader)
        for (int it = 0; it < 64; ++it) {
            volatile u32* fl = (volatile u32*)ctr->jump_flag;
            if (me == 0)
                fl[(it + 1) % 3] = 0;
            bool changed = false;
            for (u32 c = me; c < N; c += ts) {
                if (a.comp[c] != c)
                    continue;
                const u32 p = a.par[c], pp = a.par[p];
                if (p != pp) {
                    a.par[c] = pp;
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
        for (u32 v = me; v < N; v += ts)
            a.comp[v] = a.par[a.comp[v]];
        if (!t.sync())
            return;
    }
    if (!complete && *(volatile u32*)&ctr->mst_count < a.n && me == 0)
        record_failure(a.status, &ctr->bar.failed, DEV_INTERNAL);
}

__global__ void __launch_bounds__(512) k_insert_tree(TreeInsArgs a)
{
    GridTeam t{&a.ctr->bar, a.status};
    tree_insert_body(t, a);
}

constexpr u32 INS_BLOCK_MAX_N = 8192;

__global__ void __launch_bounds__(1024) k_insert_tree_block(TreeInsArgs a)
{
    BlockTeam t;
    tree_insert_body(t, a);
}

cudaError_t preload_insert_tree() { return touch_kernels(k_insert_tree, k_insert_tree_block); }

// The new tree of G + p into ws.mst (n edges, packed for n + 1 vertices).
cudaError_t run_insert_tree(Workspace& ws, const u32* keys, const u32* lo, const u32* hi, const u32* w,
                            u32 n, int dt, u32* status, cudaStream_t s)
{
    TreeInsArgs a;
    a.keys = keys;
    a.lo = lo;
    a.hi = hi;
    a.w = w;
    a.n = n;
    a.dt = dt;
    a.comp = ws.comp;
    a.par = ws.par;
    a.root = ws.flag;
    a.best = ws.best[0];
    a.mst = ws.mst;
    a.ctr = ws.ctr;
    a.status = status;
    // the control block starts clean: barrier words and the failure flag
    cudaError_t e = cudaMemsetAsync(&ws.ctr->bar, 0, sizeof(GridBar), s);
    if (e != cudaSuccess)
        return e;
    prof_launches(1);
    if (n + 1 <= INS_BLOCK_MAX_N) {
        k_insert_tree_block<<<1, 1024, 0, s>>>(a);
        return cudaGetLastError();
    }
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_insert_tree, dim3(ws.coop_blocks), dim3(512), args, 0, s);
}

}  // namespace appd
