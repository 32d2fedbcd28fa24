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
#include <type_traits>

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
// General form (rows not 16-byte aligned): one CTA per row (grid-stride).
// The tie-break inside one row is "smaller column wins", which equals the
// packed order for a fixed row.
template <int DT>
__global__ void __launch_bounds__(256) k_rowmin(const u32* __restrict__ W, u32 n, u64* __restrict__ best)
{
    __shared__ u64 sh[32];
    for (u32 row = blockIdx.x; row < n; row += gridDim.x) {
        const u32* r = W + (size_t)row * n;
        u64 m = EDGE_INF;
        for (u32 j = threadIdx.x; j < n; j += 256) {
            const u64 c = ((u64)key_of(ld_stream_u32(r + j), DT) << 32) | j;
            if (j != row && c < m)
                m = c;
        }
        m = block_min_u64(m, sh);
        if (threadIdx.x == 0)
            best[row] = pack_edge((u32)(m >> 32), row, (u32)m, n);
    }
}

// Round 1 over the upper triangle only (K1, symmetric form).  W is
// symmetric, so element (i, j), i < j, is both a candidate for row i and for
// row j.  A CTA owns 256 rows x 1024 columns; each warp a 128-column slab.
// Lanes own 4 columns: their column minima over the CTA's rows give row j's
// candidates from rows i < j; per-row minima are warp reductions
// (redux.sync) merged across warps in shared memory.  Both go to best[] with 64-bit atomic minima on packed edges, so
// every unordered pair is read once (half of W).  best[] starts at +inf.
constexpr u32 RS_ROWS = 256, RS_COLS = 1024;

// FP32 inputs: the pass also records in *signs whether any element it uses
// has its sign bit set, so that the level-0 contraction knows whether every
// weight of the upper triangle is a non-negative float (or a NaN with the
// sign bit clear), whose raw bits already compare in the order of their
// keys.  Minimax: a warp off the diagonal compares raw bits itself while
// every batch of eight rows it loads has no sign bit (one OR per element
// instead of the two-instruction key); the first batch with one switches
// the warp to keys for the rest of its slab (its column minima, raw bits
// of non-negative floats, become keys by setting the top bit).  Warps on
// the diagonal use keys throughout and report a sign bit through their
// smallest row minimum (a key below 2^31).  Widest keys are complemented;
// an OR of the raw bits reports it there.
template <int DT>
__global__ void __launch_bounds__(256, 4) k_rowmin_sym(const u32* __restrict__ W, u32 n,
                                                    u64* __restrict__ best, u32* __restrict__ signs)
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
    // Column minima as (key, row) pairs.  Rows are visited in descending
    // order and a key replaces the minimum when <= it, so the survivor is the
    // smallest key with the smallest row (the packed-edge order for a fixed
    // column); starting from key 0xFFFFFFFF the first valid row always enters.
    u32 ck[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    u32 ci[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    u32 sg = 0;              // widest FP32: OR of the raw bits
    u32 smin = 0xFFFFFFFFu;  // minimax FP32, keyed warps: smallest row minimum key
    bool keyed = DT != 0 || mask;   // warp-uniform
    // one batch of eight loaded rows (descending), compared under CDT; raw
    // minimax minima (CDT != DT) become keys by setting the top bit
    auto consume = [&](const uint4 (&v)[8], u32 ib, int pass, int r8, auto cdt_tag) {
        constexpr int CDT = decltype(cdt_tag)::value;
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            const u32 r = r8 + q, i = ib + r;
            // row i's minimum over this lane's columns, same rule over
            // descending columns: the smallest key at the smallest column
            u32 rk = 0xFFFFFFFFu, rj = 0xFFFFFFFFu;
            if (live && i < imax) {
                const u32 k[4] = {key_of(v[q].x, CDT), key_of(v[q].y, CDT), key_of(v[q].z, CDT),
                                  key_of(v[q].w, CDT)};
                if (!mask) {
                    if constexpr (DT == 2)
                        sg |= v[q].x | v[q].y | v[q].z | v[q].w;
#pragma unroll
                    for (int c = 3; c >= 0; --c)
                        if (k[c] <= rk) {
                            rk = k[c];
                            rj = j + c;
                        }
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (k[c] <= ck[c]) {
                            ck[c] = k[c];
                            ci[c] = i;
                        }
                } else {
                    if constexpr (DT == 2) {
                        const u32 e[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            sg |= j + c > i ? e[c] : 0u;
                    }
#pragma unroll
                    for (int c = 3; c >= 0; --c)
                        if (j + c > i && k[c] <= rk) {
                            rk = k[c];
                            rj = j + c;
                        }
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (j + c > i && k[c] <= ck[c]) {
                            ck[c] = k[c];
                            ci[c] = i;
                        }
                }
            }
            // warp minimum of (key, column) for row i: smallest key, then the
            // smallest column among the lanes holding it
            const u32 kmin = __reduce_min_sync(0xFFFFFFFFu, rk);
            const u32 jmin = __reduce_min_sync(0xFFFFFFFFu, rk == kmin ? rj : 0xFFFFFFFFu);
            const u32 kkey = CDT == DT ? kmin : (kmin | 0x80000000u);
            if (lane == r && jmin != 0xFFFFFFFFu)
                atomicMin(&s_row[32 * pass + r], ((u64)kkey << 32) | jmin);
            if constexpr (DT == 0 && CDT == DT)
                smin = min(smin, kmin);
        }
    };
    for (int pass = RS_ROWS / 32 - 1; pass >= 0; --pass) {
        const u32 ib = i0 + 32 * pass;
        if (ib >= imax)
            continue;
        for (int r8 = 24; r8 >= 0; r8 -= 8) {
            // issue eight rows' loads before consuming any (memory-level parallelism)
            uint4 v[8];
#pragma unroll
            for (u32 q = 0; q < 8; ++q) {
                const u32 i = ib + r8 + q;
                if (live && i < imax)
                    v[q] = ld_stream_v4(W + (size_t)i * n + j);
            }
            if constexpr (DT == 0) {
                if (!keyed) {
                    u32 o = 0;
#pragma unroll
                    for (u32 q = 0; q < 8; ++q)
                        if (live && ib + r8 + q < imax)
                            o |= v[q].x | v[q].y | v[q].z | v[q].w;
                    if (__any_sync(0xFFFFFFFFu, o >> 31)) {
                        keyed = true;
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            ck[c] |= 0x80000000u;
                        if (lane == 0)
                            atomicOr(signs, 1u);
                    }
                }
                if (!keyed) {
                    consume(v, ib, pass, r8, std::integral_constant<int, 1>{});
                    continue;
                }
            }
            consume(v, ib, pass, r8, std::integral_constant<int, DT>{});
        }
    }
    if constexpr (DT == 0) {
        if (!keyed)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                ck[c] |= 0x80000000u;
        if (lane == 0 && smin < 0x80000000u)
            atomicOr(signs, 1u);
    }
    if constexpr (DT == 2)
        if (__any_sync(0xFFFFFFFFu, sg >> 31) && lane == 0)
            atomicOr(signs, 1u);
    // column candidates: edge (i, j) with i the smallest-key row (ties: lower i)
    if (live) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (ci[c] != 0xFFFFFFFFu)
                atomicMin(&best[j + c], pack_edge(ck[c], ci[c], j + c, n));
    }
    __syncthreads();
    for (u32 r = threadIdx.x; r < RS_ROWS && i0 + r < n; r += blockDim.x) {
        u64 x = s_row[r];
        if (x != EDGE_INF)
            atomicMin(&best[i0 + r], pack_edge((u32)(x >> 32), i0 + r, (u32)x, n));
    }
}

// A round's step runs on the cooperative grid while the current matrix has
// more than STEP_BLOCK_MAX_C rows, else on one CTA, whose barriers cost a
// fraction of a grid barrier's; the host enqueues both and each form checks
// the size on the device.  The one-CTA form leaves the O(n) vertex-to-
// component update to the round's contraction, which runs on the full grid.
constexpr u32 STEP_BLOCK_MAX_C = 4096, STEP_BLOCK_THREADS = 1024;

__global__ void k_step(StepArgs a)
{
    if (((volatile u32*)a.ctr->c)[a.level] <= STEP_BLOCK_MAX_C)
        return;
    GridTeam t{&a.ctr->bar, a.status};
    step_body(t, a);
}

__global__ void __launch_bounds__(STEP_BLOCK_THREADS) k_step_block(StepArgs a)
{
    if (((volatile u32*)a.ctr->c)[a.level] > STEP_BLOCK_MAX_C)
        return;
    a.update_comp = 0;
    BlockTeam t;
    step_body(t, a);
}

// Work loop of the contraction: each CTA takes items (a group A, a chunk of
// at most CONTRACT_ROWS of its rows, a range of a.bin_cap bins), reduces
// every column of those rows into shared-memory bins indexed by the column's
// new component, and writes the bins as row A of C_{r+1} (plain stores when
// one item covers the group, atomic minima otherwise) together with the
// row's minimum, the next round's best edge of A.  TWO: 512 threads, two
// CTAs per SM, so one CTA's barriers and bin traffic overlap the other's
// loads.  The kernel runs only when run_min <= |C_{r+1}| <= run_max (the
// host enqueues both forms and the device picks by size).
template <int DT, int LEVEL0, bool VEC, bool UPPER, bool TWO>
__global__ void __launch_bounds__(TWO ? CONTRACT_THREADS2 : CONTRACT_THREADS, TWO ? 2 : 1)
    k_contract(ContractArgs a, u32 run_min, u32 run_max)
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
    if (cn < run_min || cn > run_max)
        return;
    if (cr <= a.comp_max_c)
        for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x)
            a.comp[v] = a.label[a.comp[v]];
    const u32 total_chunks = *(volatile u32*)&ctr->total_chunks;
    const u32 nbr = (cn + a.bin_cap - 1) / a.bin_cap;
    const u32 total = total_chunks * nbr;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&ctr->item_next, 1u);
        __syncthreads();
        const u32 item = s_item;
        if (item >= total)
            break;
        contract_item<DT, LEVEL0, VEC, UPPER>(a, item, cr, cn, total_chunks, bins, s_rows, s_red);
    }
}

// Every level from the third on, in one cooperative launch (the first two
// keep their own kernels: the passes over W or the points, the column minima
// of P and the symmetrization of C_2).  Per level: the step, on the whole
// grid while the matrix has more than STEP_BLOCK_MAX_C rows and on CTA 0
// alone below that (the other CTAs wait at the grid barrier, whose bounded
// wait covers it), then the contraction with every CTA taking items, then a
// grid barrier.  The loop ends at the level that leaves one component, so no
// launch is spent on rounds with nothing to do.
constexpr u32 LEVELS_THREADS = 512;

struct LevelsArgs {
    StepArgs sa;       // fields shared by the levels; level, best_in/out, cnext set per level
    ContractArgs ca;   // likewise; level, cin, cout, best_out set per level
    u64* cb[2];        // C_1, C_3, ... and C_2, C_4, ...
    u64* best[2];
    int first, last;   // the levels [first, last)
};

__global__ void __launch_bounds__(LEVELS_THREADS, 1) k_levels(LevelsArgs a)
{
    extern __shared__ __align__(16) u64 bins[];
    __shared__ u32 s_item, s_rows[CONTRACT_ROWS];
    __shared__ u64 s_red[32];
    Counters* ctr = a.sa.ctr;
    GridTeam grid{&ctr->bar, a.sa.status};
    for (int r = a.first; r < a.last; ++r) {
        if (*(volatile u32*)&ctr->done)   // read after a grid barrier: the same in every CTA
            break;
        StepArgs sa = a.sa;
        sa.level = r;
        sa.best_in = a.best[r & 1];
        sa.best_out = a.best[(r + 1) & 1];
        sa.cnext = a.cb[r & 1];
        const u32 cr = ((volatile u32*)ctr->c)[r];
        if (cr > STEP_BLOCK_MAX_C) {
            step_body(grid, sa);
        } else if (blockIdx.x == 0) {
            sa.update_comp = 0;   // the contraction below maps comp[] on the whole grid
            BlockTeam bt;
            step_body(bt, sa);
        }
        if (!grid.sync())
            return;
        if (*(volatile u32*)&ctr->done)
            break;
        ContractArgs ca = a.ca;
        ca.level = r;
        ca.cin = a.cb[(r - 1) & 1];
        ca.cout = a.cb[r & 1];
        ca.best_out = a.best[(r + 1) & 1];
        const u32 cn = ((volatile u32*)ctr->c)[r + 1];
        if (cr <= ca.comp_max_c)
            for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < ca.n; v += gridDim.x * blockDim.x)
                ca.comp[v] = ca.label[ca.comp[v]];
        const u32 total_chunks = *(volatile u32*)&ctr->total_chunks;
        const u32 total = total_chunks * ((cn + ca.bin_cap - 1) / ca.bin_cap);
        for (;;) {
            if (threadIdx.x == 0)
                s_item = atomicAdd(&ctr->item_next, 1u);
            __syncthreads();
            const u32 item = s_item;
            if (item >= total)
                break;
            contract_item<0, 0, false>(ca, item, cr, cn, total_chunks, bins, s_rows, s_red);
        }
        if (!grid.sync())
            return;
    }
}

// The level-0 contraction over the upper triangle leaves P with P(A, B) =
// min over pairs a in A, b in B with a < b, so C_1(A, B) = min(P(A, B),
// P(B, A)).  C_1 is never formed: its row minima (the round-1 best edges)
// are P's row minima (the contraction's epilogue) folded with P's column
// minima (k_colmin_p); level 1 contracts P itself into Q, with
// Q(X, Y) = min over A in X, B in Y of P(A, B), so C_2(X, Y) =
// min(Q(X, Y), Q(Y, X)), which k_sym forms in place (C_2 is small) together
// with C_2's row minima.
constexpr u32 CMIN_ROWS = 256, CMIN_THREADS = 256;

__global__ void __launch_bounds__(CMIN_THREADS) k_colmin_p(const u64* __restrict__ P, Counters* ctr,
                                                           u64* __restrict__ best_out)
{
    if (*(volatile u32*)&ctr->done)
        return;
    const u32 cn = ((volatile u32*)ctr->c)[1];
    const u32 j = blockIdx.x * CMIN_THREADS + threadIdx.x;
    const u32 r0 = blockIdx.y * CMIN_ROWS;
    if (j >= cn || r0 >= cn)
        return;
    const u32 r1 = min(cn, r0 + CMIN_ROWS);
    u64 m = EDGE_INF;
    u32 r = r0;
    for (; r + 8 <= r1; r += 8) {
        u64 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            v[q] = P[(size_t)(r + q) * cn + j];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            m = v[q] < m ? v[q] : m;
    }
    for (; r < r1; ++r) {
        const u64 v = P[(size_t)r * cn + j];
        m = v < m ? v : m;
    }
    if (m != EDGE_INF)
        atomicMin(&best_out[j], m);
}

// In-place symmetrization of C_{level+1} (row stride |C_{level+1}|): each CTA
// takes tile pairs (ti <= tj) of SYM_T x SYM_T, writes the minimum to both
// tiles (no other CTA touches them), and folds the row minima into best_out
// with atomic minima.
constexpr u32 SYM_T = 64, SYM_THREADS = 512;

__global__ void __launch_bounds__(SYM_THREADS) k_sym(u64* __restrict__ C, Counters* ctr, int level,
                                                     u64* __restrict__ best_out)
{
    extern __shared__ __align__(16) u64 s_sym[];
    u64(*s_a)[SYM_T + 1] = reinterpret_cast<u64(*)[SYM_T + 1]>(s_sym);
    u64(*s_b)[SYM_T + 1] = reinterpret_cast<u64(*)[SYM_T + 1]>(s_sym + SYM_T * (SYM_T + 1));
    if (*(volatile u32*)&ctr->done)
        return;
    const u32 cn = ((volatile u32*)ctr->c)[level + 1];
    const u32 T = (cn + SYM_T - 1) / SYM_T;
    constexpr u32 RY = SYM_THREADS / SYM_T;   // rows per sweep
    const u32 x = threadIdx.x % SYM_T, y0 = threadIdx.x / SYM_T;
    for (u32 p = blockIdx.x; p < T * T; p += gridDim.x) {
        const u32 ti = p / T, tj = p - ti * T;
        if (ti > tj)
            continue;
        const u32 ra = ti * SYM_T, rb = tj * SYM_T;
        // all sixteen loads of a thread are issued before any is used
        u64 va[SYM_T / RY], vb[SYM_T / RY];
#pragma unroll
        for (u32 k = 0; k < SYM_T / RY; ++k) {
            const u32 y = y0 + RY * k;
            va[k] = (ra + y < cn && rb + x < cn) ? C[(size_t)(ra + y) * cn + rb + x] : EDGE_INF;
            vb[k] = (rb + y < cn && ra + x < cn) ? C[(size_t)(rb + y) * cn + ra + x] : EDGE_INF;
        }
#pragma unroll
        for (u32 k = 0; k < SYM_T / RY; ++k) {
            s_a[y0 + RY * k][x] = va[k];
            s_b[y0 + RY * k][x] = vb[k];
        }
        __syncthreads();
#pragma unroll
        for (u32 k = 0; k < SYM_T / RY; ++k) {
            const u32 y = y0 + RY * k;
            // C_1(ra + y, rb + x) and C_1(rb + y, ra + x)
            const u64 ma = min(s_a[y][x], s_b[x][y]);
            const u64 mb = min(s_b[y][x], s_a[x][y]);
            if (ra + y < cn && rb + x < cn)
                C[(size_t)(ra + y) * cn + rb + x] = ma;
            if (rb + y < cn && ra + x < cn)
                C[(size_t)(rb + y) * cn + ra + x] = mb;
            const u64 wa = warp_min_u64(ma);
            if ((threadIdx.x & 31) == 0 && ra + y < cn && wa != EDGE_INF)
                atomicMin(&best_out[ra + y], wa);
            if (ti != tj) {
                const u64 wb = warp_min_u64(mb);
                if ((threadIdx.x & 31) == 0 && rb + y < cn && wb != EDGE_INF)
                    atomicMin(&best_out[rb + y], wb);
            }
        }
        __syncthreads();
    }
}

inline size_t sym_smem_bytes() { return 2 * SYM_T * (SYM_T + 1) * sizeof(u64); }

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
        ctr->signs = 0;
        if (bar_reset) {
            ctr->bar.count = 0;
            ctr->bar.abort = 0;
        }
        ctr->bar.failed = 0;
    }
}

template <class K>
cudaError_t set_smem(K kern, size_t bytes)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

__global__ void k_mst_split(const u64* __restrict__ mst, u32 n, u32* __restrict__ keys, u32* __restrict__ lo,
                            u32* __restrict__ hi)
{
    for (u32 e = blockIdx.x * blockDim.x + threadIdx.x; e + 1 < n; e += gridDim.x * blockDim.x) {
        const u64 x = mst[e];
        keys[e] = edge_key(x);
        edge_ends(x, n, lo + e, hi + e);
    }
}

cudaError_t launch_mst_split(const u64* mst, u32 n, u32* keys, u32* lo, u32* hi, cudaStream_t s)
{
    const u32 m = n - 1, grid = (m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024;
    k_mst_split<<<grid, 256, 0, s>>>(mst, n, keys, lo, hi);
    return cudaGetLastError();
}

cudaError_t preload_mst()
{
    return touch_kernels(k_rowmin<0>, k_rowmin<1>, k_rowmin<2>, k_rowmin<3>, k_rowmin_sym<0>, k_rowmin_sym<1>,
                         k_rowmin_sym<2>, k_rowmin_sym<3>, k_step, k_step_block, k_mst_init, k_colmin_p, k_sym,
                         k_contract<0, 1, true, true, true>, k_contract<1, 1, true, true, true>,
                         k_contract<2, 1, true, true, true>, k_contract<3, 1, true, true, true>,
                         k_contract<0, 1, true, true, false>, k_contract<1, 1, true, true, false>,
                         k_contract<2, 1, true, true, false>, k_contract<3, 1, true, true, false>,
                         k_contract<0, 1, false, false, true>, k_contract<1, 1, false, false, true>,
                         k_contract<2, 1, false, false, true>, k_contract<3, 1, false, false, true>,
                         k_contract<0, 1, false, false, false>, k_contract<1, 1, false, false, false>,
                         k_contract<2, 1, false, false, false>, k_contract<3, 1, false, false, false>,
                         k_contract<0, 0, false, false, true>, k_mst_split, k_levels);
}

cudaError_t preload_kernels()
{
    cudaError_t e = preload_mst();
    if (e == cudaSuccess)
        e = preload_contract_tma();
    if (e == cudaSuccess)
        e = preload_leaf();
    if (e == cudaSuccess)
        e = preload_fill();
    if (e == cudaSuccess)
        e = preload_batched();
    if (e == cudaSuccess)
        e = preload_points();
    if (e == cudaSuccess)
        e = preload_insert_tree();
    return e;
}

size_t contraction_scratch_bytes(int64_t n)
{
    size_t h = (size_t)(n / 2), q = (size_t)(n / 4);
    return (h * h + q * q) * sizeof(u64) + 64;
}

cudaError_t run_mst(Workspace& ws, const void* W, int dt, void* cbuf, size_t cbuf_bytes,
                    u32* status, cudaStream_t s, const PointsSrc* ps)
{
    const u32 n = (u32)ws.n;
    cudaError_t err;
    k_mst_init<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(ws.ctr, ws.comp, n, 1);
    prof_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess)
        return err;
    if (n <= 1)
        return cudaSuccess;
    // vec: rows of W 16-byte aligned (upper-triangle passes over W);
    // upper: level 0 leaves the unsymmetrized P (stored W with vec, or points)
    const bool vec = !ps && (n % 4 == 0) && ((uintptr_t)W % 16 == 0);
    const bool upper = vec || ps;
    prof_launches(1);
    prof_begin(PH_ROWMIN, s);
    if (ps) {
        if ((err = cudaMemsetAsync(ws.best[0], 0xFF, (size_t)n * sizeof(u64), s)) != cudaSuccess)
            return err;
        if ((err = launch_rowmin_pts(ps->P, ps->D, n, dt, ws.best[0], s)) != cudaSuccess)
            return err;
    } else if (vec) {
        // upper-triangle tiles; best[] is reduced with atomic minima from +inf
        if ((err = cudaMemsetAsync(ws.best[0], 0xFF, (size_t)n * sizeof(u64), s)) != cudaSuccess)
            return err;
        dim3 grid((n + RS_COLS - 1) / RS_COLS, (n + RS_ROWS - 1) / RS_ROWS);
        auto kr = dt == 0 ? k_rowmin_sym<0> : dt == 1 ? k_rowmin_sym<1> : dt == 2 ? k_rowmin_sym<2>
                                                                                : k_rowmin_sym<3>;
        kr<<<grid, 256, 0, s>>>((const u32*)W, n, ws.best[0], &ws.ctr->signs);
        if ((err = cudaGetLastError()) != cudaSuccess)
            return err;
    } else {
        int grid = ws.sms * 8;
        if (grid > (int)n)
            grid = (int)n;
        auto kr = dt == 0 ? k_rowmin<0> : dt == 1 ? k_rowmin<1> : dt == 2 ? k_rowmin<2> : k_rowmin<3>;
        kr<<<grid, 256, 0, s>>>((const u32*)W, n, ws.best[0]);
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
    const size_t smem = (size_t)ws.bin_cap * sizeof(u64), smem2 = (size_t)ws.bin_cap2 * sizeof(u64);
    // level 0 reads the upper triangle of W when rows are 16-byte aligned;
    // two CTAs per SM when C_1's row fits their bins, else one with all bins
    auto pick0 = [&](auto two) {
        constexpr bool T = decltype(two)::value;
        switch (dt) {
        case 0: return vec ? k_contract<0, 1, true, true, T> : k_contract<0, 1, false, false, T>;
        case 1: return vec ? k_contract<1, 1, true, true, T> : k_contract<1, 1, false, false, T>;
        case 2: return vec ? k_contract<2, 1, true, true, T> : k_contract<2, 1, false, false, T>;
        default: return vec ? k_contract<3, 1, true, true, T> : k_contract<3, 1, false, false, T>;
        }
    };
    auto k0a = pick0(std::true_type{});
    auto k0b = pick0(std::false_type{});
    auto k1 = k_contract<0, 0, false, false, true>;
    if ((err = set_smem(k0a, smem2)) != cudaSuccess || (err = set_smem(k0b, smem)) != cudaSuccess ||
        (err = set_smem(k1, smem2)) != cudaSuccess || (err = set_smem(k_sym, sym_smem_bytes())) != cudaSuccess)
        return err;
    // levels 0 and 1 here; every later level in one persistent launch below
    const int direct_levels = ws.levels < 2 ? ws.levels : 2;
    for (int r = 0; r < direct_levels; ++r) {
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
        // level 0 of the upper-triangle path also keeps 16-bit labels (every
        // component of round 1 has two or more vertices: ids < 32768)
        sa.label16 = (r == 0 && vec && ws.bin_cap_t > 0) ? ws.label16 : nullptr;
        // every round at least halves the components, so round r has at most
        // n >> r rows: rounds that cannot exceed the one-CTA limit skip the
        // grid form (and its barrier reset)
        const bool grid_step = (n >> r) > STEP_BLOCK_MAX_C;
        if (grid_step && (err = cudaMemsetAsync(&ws.ctr->bar, 0, 2 * sizeof(u32), s)) != cudaSuccess)
            return err;
        void* args[] = {&sa};
        prof_begin(PH_STEP, s);
        err = grid_step ? cudaLaunchCooperativeKernel((const void*)k_step, dim3(ws.coop_blocks),
                                                      dim3(ws.coop_threads), args, 0, s)
                        : cudaSuccess;
        if (err == cudaSuccess) {
            k_step_block<<<1, STEP_BLOCK_THREADS, 0, s>>>(sa);
            err = cudaGetLastError();
        }
        prof_end(PH_STEP, s);
        prof_launches(grid_step ? 3 : 2);
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
        ca.comp = ws.comp;
        ca.n = n;
        ca.comp_max_c = STEP_BLOCK_MAX_C;
        const int ph = (r == 0) ? PH_CONTRACT0 : PH_CONTRACT;
        prof_begin(ph, s);
        ContractArgs ca1 = ca;
        ca.bin_cap = ws.bin_cap2;
        if (r == 0 && ps) {
            // the point set's level 0: coordinates in component order, then
            // each group against every later group's contiguous columns
            if ((err = launch_pts_gather(ps->P, ps->D, ws.members, ws.label, n, ps->Ps, ps->pvid, ps->pcomp,
                                         s)) != cudaSuccess)
                return err;
            if ((err = launch_contract_pts_sorted(ca, ps->Ps, ps->pvid, ps->pcomp, ps->D, dt, 3 * ws.contract_blocks,
                                                  s)) != cudaSuccess)
                return err;
            prof_launches(2);
        } else if (r == 0 && vec && ws.bin_cap_t > 0) {
            // upper triangle streamed by bulk copies while |C_1| fits beside
            // the copy ring, else one CTA per SM with all bins
            ContractArgs cat = ca;
            cat.bin_cap = ws.bin_cap_t;
            cat.label16 = ws.label16;
            err = launch_contract0_tma(cat, dt, ws.contract_blocks, ws.bin_cap_t, status, &ws.ctr->signs, s);
            if (err != cudaSuccess)
                return err;
            k0b<<<ws.contract_blocks, CONTRACT_THREADS, smem, s>>>(ca1, ws.bin_cap_t + 1, 0xFFFFFFFFu);
            prof_launches(1);
        } else if (r == 0) {
            k0a<<<2 * ws.contract_blocks, CONTRACT_THREADS2, smem2, s>>>(ca, 0u, ws.bin_cap2);
            k0b<<<ws.contract_blocks, CONTRACT_THREADS, smem, s>>>(ca1, ws.bin_cap2 + 1, 0xFFFFFFFFu);
            prof_launches(1);
        } else {
            k1<<<2 * ws.contract_blocks, CONTRACT_THREADS2, smem2, s>>>(ca, 0u, 0xFFFFFFFFu);
        }
        if (upper && r == 0) {
            // C_1's row minima also take P's column minima
            prof_launches(1);
            const u32 g = (u32)((h + CMIN_THREADS - 1) / CMIN_THREADS);
            const u32 gy = (u32)((h + CMIN_ROWS - 1) / CMIN_ROWS);
            k_colmin_p<<<dim3(g, gy), CMIN_THREADS, 0, s>>>(cb[0], ws.ctr, ws.best[1]);
        }
        if (upper && r == 1) {
            // level 1 contracted the unsymmetrized P: symmetrize C_2
            prof_launches(1);
            k_sym<<<ws.sms * 3, SYM_THREADS, sym_smem_bytes(), s>>>(cb[1], ws.ctr, 1, ws.best[0]);
        }
        prof_end(ph, s);
        if ((err = cudaGetLastError()) != cudaSuccess)
            return err;
    }
    if (ws.levels > 2) {
        LevelsArgs la;
        StepArgs& sa = la.sa;
        sa.level = 2;
        sa.n = n;
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
        sa.part = ws.part;
        sa.ctr = ws.ctr;
        sa.status = status;
        sa.bin_cap = ws.bin_cap2;
        sa.label16 = nullptr;
        ContractArgs& ca = la.ca;
        ca.level = 2;
        ca.label = ws.label;
        ca.members = ws.members;
        ca.gstart = ws.gstart;
        ca.nchunk = ws.nchunk;
        ca.chunk_start = ws.chunk_start;
        ca.item_group = ws.item_group;
        ca.ctr = ws.ctr;
        ca.bin_cap = ws.bin_cap2;
        ca.comp = ws.comp;
        ca.n = n;
        ca.comp_max_c = STEP_BLOCK_MAX_C;
        la.cb[0] = cb[0];
        la.cb[1] = cb[1];
        la.best[0] = ws.best[0];
        la.best[1] = ws.best[1];
        la.first = 2;
        la.last = ws.levels;
        if ((err = set_smem(k_levels, smem2)) != cudaSuccess)
            return err;
        if ((err = cudaMemsetAsync(&ws.ctr->bar, 0, 2 * sizeof(u32), s)) != cudaSuccess)
            return err;
        void* args[] = {&la};
        prof_begin(PH_CONTRACT, s);
        err = cudaLaunchCooperativeKernel((const void*)k_levels, dim3(ws.coop_blocks), dim3(LEVELS_THREADS), args,
                                          smem2, s);
        prof_end(PH_CONTRACT, s);
        prof_launches(1);
        if (err != cudaSuccess)
            return err;
    }
    // the point set's tree carries keys of squared distances: convert them
    if (ps)
        return launch_mst_sqrt(ws.mst, n - 1, dt, s);
    return cudaSuccess;
}

}  // namespace appd
