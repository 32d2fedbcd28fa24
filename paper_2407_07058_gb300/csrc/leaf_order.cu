// leaf_order.cu -- single-linkage leaf order and merge heights from the MST.
//
// Section 3 notes that the APPD matrix can also be produced by adding the MST
// edges from small to large (a single-linkage dendrogram), and Section 7
// notes that the distances follow from the dendrogram.  We need, for the
// fill, a leaf order pos[] and gaps gap[k] (merge height between the leaves
// at positions k and k+1) such that
//     key(M(i,j)) = max gap[min(pos_i,pos_j) .. max(pos_i,pos_j) - 1].
// Prim's visiting order on the MST is such an order (its gap before vertex v
// is the weight that added v).  Prim itself is sequential; we obtain the same
// kind of order in O(log n) parallel phases:
//   1. root the MST at vertex 0 with an Euler tour and list ranking;
//   2. for every non-root y, ord(y) = (key of y's parent edge, y); its
//      nearest heavier ancestor nha(y) is the first vertex z above y's parent
//      edge (z's own parent edge) with ord(z) > ord(y), found by binary
//      lifting over ancestor maxima (the root counts as infinitely heavy);
//   3. the tree y -> nha(y) visited in preorder, children in increasing
//      ord, starts at the root, and the gap before each y is its parent
//      edge's key.  Children are ordered by an LSD radix sort of
//      (nha, ord); the preorder comes from a second Euler tour.
//   4. a sparse table over the gaps for O(1) range maxima.
// All phases run in one cooperative kernel separated by bounded grid
// barriers; up to LEAF_BLOCK_MAX_N vertices they run on one CTA instead,
// whose block barriers cost a fraction of a grid barrier's (the phases are
// short at that size, so the barriers dominate).
#include "leaf_device.cuh"

namespace appd {

__global__ void __launch_bounds__(512) k_leaf_order(LeafArgs a)
{
    GridTeam t{&a.ctr->bar, a.status};
    leaf_body(t, a);
}

constexpr u32 LEAF_BLOCK_MAX_N = 2048;

// 512 threads: the radix sort's per-warp counts are sized for 16 warps
__global__ void __launch_bounds__(512) k_leaf_order_block(LeafArgs a)
{
    BlockTeam t;
    leaf_body(t, a);
}

cudaError_t preload_leaf() { return touch_kernels(k_leaf_order, k_leaf_order_block); }

cudaError_t run_leaf_order(Workspace& ws, u32* status, cudaStream_t s)
{
    if (ws.n < 2)
        return cudaSuccess;
    LeafArgs a;
    a.n = (u32)ws.n;
    a.levels = ws.levels;
    a.st_levels = ws.st_levels;
    a.mst = ws.mst;
    a.deg = ws.deg;
    a.adj_off = ws.adj_off;
    a.afill = ws.afill;
    a.adj = ws.adj;
    a.aslot = ws.aslot;
    a.lr_d0 = ws.lr_d[0];
    a.lr_d1 = ws.lr_d[1];
    a.lr_nx0 = ws.lr_nx[0];
    a.lr_nx1 = ws.lr_nx[1];
    a.parent = ws.parent;
    a.pe_key = ws.pe_key;
    a.ord = ws.ord;
    a.jump = ws.jump;
    a.mxo = ws.mxo;
    a.nha = ws.nha;
    a.skey0 = ws.skey[0];
    a.skey1 = ws.skey[1];
    a.sval0 = ws.sval[0];
    a.sval1 = ws.sval[1];
    a.hist = ws.hist;
    a.ntiles = ws.ntiles;
    a.first_child = ws.first_child;
    a.next_sib = ws.next_sib;
    a.pos = ws.pos;
    a.order = ws.order;
    a.nsize = ws.nsize;
    a.gap = ws.gap;
    a.st = ws.st;
    a.part = ws.part;
    a.ctr = ws.ctr;
    a.status = status;
    if (a.n <= LEAF_BLOCK_MAX_N) {
        k_leaf_order_block<<<1, 512, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaError_t err = cudaMemsetAsync(&ws.ctr->bar, 0, 2 * sizeof(u32), s);
    if (err != cudaSuccess)
        return err;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_leaf_order, dim3(ws.coop_blocks), dim3(512),
                                       args, 0, s);
}

}  // namespace appd
