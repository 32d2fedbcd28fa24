// points.cu -- the solve of a point set's complete graph without storing W.
//
// A dataset becomes a complete graph whose edge weights are the distances
// between its points (Section 1; the experiments of Section 4 run on point
// datasets).  appd_solve_points takes the points instead of W and computes
// the edge weights where they are consumed, so W is never written or read:
//
//   W(i,j) = sqrt(s),  s = 0, then for k = 0 .. d-1:
//            t = x(i,k) - x(j,k) (FP32),  s = fma(t, t, s) (one rounding),
//   with a correctly rounded square root; W(i,i) = +0.
//
// Only the two passes that read W in the stored-matrix solve change: the
// round-1 minima (k_rowmin_pts) and the level-0 contraction
// (k_contract_pts), both over the upper triangle i < j.  They compare s
// instead of sqrt(s): the square root is monotone, so ordering edges by
// (key(s), lo, hi) refines the order by W, and the spanning tree found is a
// minimum spanning tree for W as well; the n - 1 tree edges' keys are then
// converted to key(sqrt(s)) (k_mst_sqrt), and the leaf order and the fill
// run unchanged.  Every output is still the weight of one edge, bit for bit.
//
// Coordinates are first copied into a zero-padded n_pad x D array (D a power
// of two >= d, at most 32): a padded coordinate adds t = 0 and fma(0, 0, s)
// = s exactly, so s does not change.  Both passes are bound by FP32
// arithmetic (2 D operations per pair), not by memory.
#include "mst_device.cuh"

namespace appd {

namespace {

template <int D>
__device__ __forceinline__ float sq_dist(const float (&a)[D], const float (&b)[D])
{
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float t = __fsub_rn(a[k], b[k]);
        s = __fmaf_rn(t, t, s);
    }
    return s;
}

template <int D>
__device__ __forceinline__ void load_pt(const float* __restrict__ p, float (&x)[D])
{
    if constexpr (D % 4 == 0) {
#pragma unroll
        for (int k = 0; k < D; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + k);
            x[k] = v.x;
            x[k + 1] = v.y;
            x[k + 2] = v.z;
            x[k + 3] = v.w;
        }
    } else {
        static_assert(D == 2, "padded dimensions are 2 or a multiple of 4");
        const float2 v = *reinterpret_cast<const float2*>(p);
        x[0] = v.x;
        x[1] = v.y;
    }
}

// A squared distance is +0 or positive (finite coordinates), so its bits
// order it; the widest order reverses that.  sbits_order gives a value whose
// unsigned order is the key order, and order_to_key the key itself:
// key_of(bits, DT) is bits | 0x80000000 for DT = 0 and ~(bits | 0x80000000)
// = ~bits & 0x7FFFFFFF for DT = 2, both monotone in the value below.
template <int DT>
__device__ __forceinline__ u32 sbits_order(float s)
{
    return (DT & 2) ? ~__float_as_uint(s) : __float_as_uint(s);
}

template <int DT>
__device__ __forceinline__ u32 order_to_key(u32 u)
{
    return (DT & 2) ? (u & 0x7FFFFFFFu) : (u | 0x80000000u);
}

// columns per thread of the contraction (512 threads, up to 128 registers):
// the columns' coordinates take 16..32 registers
template <int D>
constexpr int cols_per_thread()
{
    return D <= 4 ? 8 : (D == 8 ? 4 : (D == 16 ? 2 : 1));
}

// columns per lane of the round-1 tile (two 256-thread CTAs per SM, up to
// 128 registers): the columns' coordinates take 16..64 registers
template <int D>
constexpr int cols_per_lane()
{
    return D <= 4 ? 8 : (D <= 16 ? 4 : 2);
}

}  // namespace

__global__ void k_pts_pad(const float* __restrict__ X, u32 n, int d, int D, u32 npad, float* __restrict__ P)
{
    const u64 total = (u64)npad * D;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        const u32 i = (u32)(e / D);
        const int k = (int)(e - (u64)i * D);
        P[e] = (i < n && k < d) ? X[(u64)i * d + k] : 0.0f;
    }
}

// Round 1 over the upper triangle, as k_rowmin_sym does for a stored W: a
// CTA owns 256 rows x (8 warps x 32 lanes x CPL) columns; a lane keeps its
// CPL columns' coordinates in registers and walks the rows (coordinates in
// shared memory, read as broadcasts) in descending order.  Each pair (i, j),
// i < j, is a candidate for row i (warp minimum per row, merged across
// warps in shared memory) and for row j (running column minimum); both go to
// best[] by 64-bit atomic minima.  Rows descending with "<=" leave the
// smallest key at the smallest row (and, per row, the smallest column).
constexpr u32 RP_ROWS = 256, RP_THREADS = 256;

template <int DT, int D>
__global__ void __launch_bounds__(RP_THREADS, 2)
    k_rowmin_pts(const float* __restrict__ P, u32 n, u64* __restrict__ best)
{
    constexpr int CPL = cols_per_lane<D>();
    constexpr u32 TCOLS = 8 * 32 * CPL;
    __shared__ __align__(16) float s_pts[RP_ROWS * D];
    __shared__ u64 s_row[RP_ROWS];
    const u32 i0 = blockIdx.y * RP_ROWS, c0 = blockIdx.x * TCOLS;
    if (c0 + TCOLS - 1 <= i0 || i0 >= n || c0 >= n)   // no pair i < j in this tile
        return;
    const u32 w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const u32 imax = min(n, i0 + RP_ROWS);
    for (u32 r = threadIdx.x; r < RP_ROWS; r += blockDim.x)
        s_row[r] = EDGE_INF;
    for (u32 e = threadIdx.x; e < RP_ROWS * D; e += blockDim.x)
        s_pts[e] = P[(size_t)i0 * D + e];   // P has npad >= i0 + RP_ROWS rows
    __syncthreads();
    const u32 j = c0 + (32 * w + lane) * CPL;   // this lane's first column
    float cx[CPL][D];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        if (j + c < n) {
            load_pt<D>(P + (size_t)(j + c) * D, cx[c]);
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k)
                cx[c][k] = 0.0f;
        }
    }
    u32 ck[CPL], ci[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
        ck[c] = ci[c] = 0xFFFFFFFFu;
    const bool any = j < n;
    // no mask where every column of the tile lies right of every row and below n
    const bool clear = c0 >= imax && c0 + TCOLS <= n;
    // (the order values below are the keys' order; see sbits_order)
    for (u32 i = imax; i-- > i0;) {
        float rx[D];
#pragma unroll
        for (int k = 0; k < D; ++k)
            rx[k] = s_pts[(i - i0) * D + k];
        u32 rk = 0xFFFFFFFFu, rj = 0xFFFFFFFFu;
        if (clear) {
#pragma unroll
            for (int c = CPL - 1; c >= 0; --c) {
                const u32 u = sbits_order<DT>(sq_dist<D>(rx, cx[c]));
                if (u <= rk) {
                    rk = u;
                    rj = j + c;
                }
                if (u <= ck[c]) {
                    ck[c] = u;
                    ci[c] = i;
                }
            }
        } else if (any && j + CPL - 1 > i) {
#pragma unroll
            for (int c = CPL - 1; c >= 0; --c) {
                const u32 col = j + c;
                const u32 u = sbits_order<DT>(sq_dist<D>(rx, cx[c]));
                const bool ok = col > i && col < n;
                if (ok && u <= rk) {
                    rk = u;
                    rj = col;
                }
                if (ok && u <= ck[c]) {
                    ck[c] = u;
                    ci[c] = i;
                }
            }
        }
        const u32 kmin = __reduce_min_sync(0xFFFFFFFFu, rk);
        const u32 jmin = __reduce_min_sync(0xFFFFFFFFu, rk == kmin ? rj : 0xFFFFFFFFu);
        if (lane == 0 && jmin != 0xFFFFFFFFu)
            atomicMin(&s_row[i - i0], ((u64)order_to_key<DT>(kmin) << 32) | jmin);
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c)
        if (ci[c] != 0xFFFFFFFFu)
            atomicMin(&best[j + c], pack_edge(order_to_key<DT>(ck[c]), ci[c], j + c, n));
    __syncthreads();
    for (u32 r = threadIdx.x; r < RP_ROWS && i0 + r < n; r += blockDim.x) {
        const u64 x = s_row[r];
        if (x != EDGE_INF)
            atomicMin(&best[i0 + r], pack_edge((u32)(x >> 32), i0 + r, (u32)x, n));
    }
}

// The level-0 contraction of the points' graph over the upper triangle: the
// same work items as k_contract (group A, at most CONTRACT_ROWS of its rows,
// one bin range), the rows' coordinates in shared memory, every column j
// right of the item's smallest row swept once per item with its coordinates
// in registers.  For each column, the smallest key over the item's rows left
// of it (rows ascending, first strictly smaller wins: the packed order) is
// folded into the bin of j's component; the bins become row A of P, whose
// symmetrization and column minima follow as for a stored W.
constexpr u32 CP_THREADS = 512;

template <int DT, int D>
__global__ void __launch_bounds__(CP_THREADS, 1) k_contract_pts(ContractArgs a, const float* __restrict__ P)
{
    constexpr int CPC = cols_per_thread<D>();
    extern __shared__ __align__(16) u64 bins[];
    __shared__ __align__(16) float s_rp[CONTRACT_ROWS * D];
    __shared__ u32 s_item, s_rows[CONTRACT_ROWS];
    __shared__ u64 s_red[32];
    Counters* ctr = a.ctr;
    if (*(volatile u32*)&ctr->done)
        return;
    const u32 cr = ((volatile u32*)ctr->c)[0];   // level 0: n
    const u32 cn = ((volatile u32*)ctr->c)[1];
    const u32 tid = threadIdx.x, bd = blockDim.x;
    if (cr <= a.comp_max_c)
        for (u32 v = blockIdx.x * bd + tid; v < a.n; v += gridDim.x * bd)
            a.comp[v] = a.label[a.comp[v]];
    const u32 total_chunks = *(volatile u32*)&ctr->total_chunks;
    const u32 nbr = (cn + a.bin_cap - 1) / a.bin_cap;
    const u32 total = total_chunks * nbr;
    for (;;) {
        if (tid == 0)
            s_item = atomicAdd(&ctr->item_next, 1u);
        __syncthreads();
        const u32 item = s_item;
        if (item >= total)
            break;
        const u32 br = item / total_chunks, ch = item - br * total_chunks;
        const u32 A = a.item_group[ch];
        const u32 kq = ch - a.chunk_start[A];
        const u32 m0 = a.gstart[A] + kq * CONTRACT_ROWS;
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
        if (tid == 0) {   // rows ascending (at most CONTRACT_ROWS)
            for (u32 q = 1; q < nrows; ++q) {
                const u32 v = s_rows[q];
                u32 p = q;
                while (p > 0 && s_rows[p - 1] > v) {
                    s_rows[p] = s_rows[p - 1];
                    --p;
                }
                s_rows[p] = v;
            }
        }
        __syncthreads();
        for (u32 e = tid; e < nrows * D; e += bd)
            s_rp[e] = P[(size_t)s_rows[e / D] * D + (e % D)];
        __syncthreads();
        const u32 r0 = s_rows[0];
        for (u32 g = (r0 + 1) / CPC + tid; g * CPC < cr; g += bd) {
            const u32 j = g * CPC;
            float cx[CPC][D];
#pragma unroll
            for (int c = 0; c < CPC; ++c)
                load_pt<D>(P + (size_t)(j + c) * D, cx[c]);
            u32 bk[CPC], bi[CPC];
#pragma unroll
            for (int c = 0; c < CPC; ++c)
                bk[c] = bi[c] = 0xFFFFFFFFu;
            for (u32 q = 0; q < nrows; ++q) {
                const u32 row = s_rows[q];
                if (row >= j + CPC - 1)   // rows ascending: none of the rest reach these columns
                    break;
                float rx[D];
#pragma unroll
                for (int k = 0; k < D; ++k)
                    rx[k] = s_rp[q * D + k];
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    const u32 k = key_of(__float_as_uint(sq_dist<D>(rx, cx[c])), DT);
                    if (j + c > row && (bi[c] == 0xFFFFFFFFu || k < bk[c])) {
                        bk[c] = k;
                        bi[c] = row;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < CPC; ++c) {
                const u32 col = j + c;
                if (bi[c] == 0xFFFFFFFFu || col >= cr)
                    continue;
                const u32 L = a.label[col];
                const u32 rel = L - b0;
                if (L == A || rel >= nb)
                    continue;
                const u64 e = ((u64)bk[c] << 32) | pair_code(bi[c], col, cr);
                if (e < bins[rel])
                    atomicMin(&bins[rel], e);
            }
        }
        __syncthreads();
        // row A of P (this bin range) and its minimum
        u64 m = EDGE_INF;
        u64* dst = a.cout + (size_t)A * cn + b0;
        for (u32 b = tid; b < nb; b += bd) {
            const u64 v = bins[b];
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

// ------------------------------------------------ level 0, sorted columns
// After the level-0 step the members list holds the vertices grouped by
// component (group A at positions gstart[A] .. gstart[A+1]).  k_pts_gather
// copies the coordinates into that order (Ps), with each position's vertex
// (pvid) and component (pcomp).  k_contract_pts_sorted then takes group A's
// rows against every later position: those columns belong to groups B > A,
// each group's columns contiguous, so P'(A, B) = min over the run of B's
// columns of the column minima -- a run reduction instead of a bin array.
// Row A of P' holds INF for B <= A, so C_1(A, B) = min(P'(A, B), P'(B, A))
// as for the upper-triangle P of a stored W, and the same column minima and
// level-1 symmetrization follow.
__global__ void k_pts_gather(const float* __restrict__ P, int D, const u32* __restrict__ members,
                             const u32* __restrict__ label, u32 n, float* __restrict__ Ps,
                             u32* __restrict__ pvid, u32* __restrict__ pcomp)
{
    for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const u32 v = members[q];
        pvid[q] = v;
        pcomp[q] = label[v];
        for (int k = 0; k < D; ++k)
            Ps[(size_t)q * D + k] = P[(size_t)v * D + k];
    }
}

constexpr u32 CS_THREADS = 256;
constexpr u32 CS_ROWCAP = 256;   // rows of a group kept in shared memory

template <int D>
constexpr int cols_sorted()
{
    return D <= 4 ? 8 : (D == 8 ? 4 : (D == 16 ? 2 : 1));
}

template <int DT, int D>
__global__ void __launch_bounds__(CS_THREADS, 3)
    k_contract_pts_sorted(ContractArgs a, const float* __restrict__ Ps, const u32* __restrict__ pvid,
                          const u32* __restrict__ pcomp)
{
    constexpr int CPC = cols_sorted<D>();
    constexpr u32 CH = CS_THREADS * CPC;   // columns per chunk
    __shared__ __align__(16) float s_rp[CS_ROWCAP * D];
    __shared__ u32 s_rv[CS_ROWCAP];
    __shared__ u64 s_e[CH];
    __shared__ u32 s_b[CH];
    __shared__ u32 s_item;
    __shared__ u64 s_carry_e[2];
    __shared__ u32 s_carry_b[2];
    __shared__ u64 s_red[32];
    Counters* ctr = a.ctr;
    if (*(volatile u32*)&ctr->done)
        return;
    const u32 n = ((volatile u32*)ctr->c)[0];
    const u32 cn = ((volatile u32*)ctr->c)[1];
    const u32 tid = threadIdx.x;
    if (n <= a.comp_max_c)
        for (u32 v = blockIdx.x * blockDim.x + tid; v < a.n; v += gridDim.x * blockDim.x)
            a.comp[v] = a.label[a.comp[v]];
    for (;;) {
        if (tid == 0)
            s_item = atomicAdd(&ctr->item_next, 1u);
        __syncthreads();
        const u32 A = s_item;
        if (A >= cn)
            break;
        const u32 g0 = a.gstart[A], g1 = a.gstart[A + 1];
        const u32 nrows = g1 - g0;
        const bool rows_in_smem = nrows <= CS_ROWCAP;
        if (rows_in_smem) {
            for (u32 e = tid; e < nrows * D; e += CS_THREADS)
                s_rp[e] = Ps[(size_t)g0 * D + e];
            for (u32 r = tid; r < nrows; r += CS_THREADS)
                s_rv[r] = pvid[g0 + r];
        }
        u64* row = a.cout + (size_t)A * cn;
        for (u32 b = tid; b <= A; b += CS_THREADS)   // no pairs with groups B <= A
            row[b] = EDGE_INF;
        if (tid == 0) {
            s_carry_b[0] = 0xFFFFFFFFu;
            s_carry_e[0] = EDGE_INF;
        }
        u64 mrow = EDGE_INF;   // this thread's part of row A's minimum
        __syncthreads();
        int cur = 0;
        for (u32 q0 = g1; q0 < n; q0 += CH) {
            // 1. each column's smallest (key, row vertex) over the group's rows
            const u32 qt = q0 + tid * CPC;
            float cx[CPC][D];
            u32 bk[CPC], bv[CPC], vq[CPC];
#pragma unroll
            for (int c = 0; c < CPC; ++c) {
                const u32 q = qt + c;
                if (q < n) {
                    load_pt<D>(Ps + (size_t)q * D, cx[c]);
                    vq[c] = pvid[q];
                } else {
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        cx[c][k] = 0.0f;
                    vq[c] = 0u;
                }
                bk[c] = bv[c] = 0xFFFFFFFFu;
            }
            for (u32 r = 0; r < nrows; ++r) {
                float rx[D];
                u32 vr;
                if (rows_in_smem) {
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        rx[k] = s_rp[r * D + k];
                    vr = s_rv[r];
                } else {
                    load_pt<D>(Ps + (size_t)(g0 + r) * D, rx);
                    vr = pvid[g0 + r];
                }
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    const u32 u = sbits_order<DT>(sq_dist<D>(rx, cx[c]));
                    if (u < bk[c] || (u == bk[c] && vr < bv[c])) {
                        bk[c] = u;
                        bv[c] = vr;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < CPC; ++c) {
                const u32 q = qt + c;
                const u32 i = tid * CPC + c;
                if (q < n && bv[c] != 0xFFFFFFFFu) {
                    s_e[i] = ((u64)order_to_key<DT>(bk[c]) << 32) |
                             pair_code(min(bv[c], vq[c]), max(bv[c], vq[c]), n);
                    s_b[i] = pcomp[q];
                } else {
                    s_e[i] = EDGE_INF;
                    s_b[i] = q < n ? pcomp[q] : 0xFFFFFFFFu;
                }
            }
            __syncthreads();
            // 2. one thread per run of equal B in the chunk reduces it; the
            // run that reaches the chunk's end is carried into the next chunk
            const u32 ncol = min(CH, n - q0);
            const u32 cb = s_carry_b[cur];
            const u64 ce = s_carry_e[cur];
            for (u32 i = tid; i < ncol; i += CS_THREADS) {
                const u32 B = s_b[i];
                if (i > 0 && s_b[i - 1] == B)
                    continue;   // not a run start
                u64 v = EDGE_INF;
                u32 j = i;
                for (; j < ncol && s_b[j] == B; ++j)
                    v = s_e[j] < v ? s_e[j] : v;
                if (i == 0) {
                    if (cb == B) {
                        v = ce < v ? ce : v;
                    } else if (cb != 0xFFFFFFFFu) {
                        row[cb] = ce;   // the carried run ended with the last chunk
                        mrow = ce < mrow ? ce : mrow;
                    }
                }
                if (j < ncol) {
                    row[B] = v;
                    mrow = v < mrow ? v : mrow;
                } else {
                    s_carry_b[cur ^ 1] = B;
                    s_carry_e[cur ^ 1] = v;
                }
            }
            cur ^= 1;
            __syncthreads();
        }
        // the last run of the item
        if (tid == 0 && s_carry_b[cur] != 0xFFFFFFFFu) {
            const u64 v = s_carry_e[cur];
            row[s_carry_b[cur]] = v;
            mrow = v < mrow ? v : mrow;
        }
        mrow = block_min_u64(mrow, s_red);
        if (tid == 0 && mrow != EDGE_INF)
            atomicMin(&a.best_out[A], mrow);
        __syncthreads();
    }
}

// The tree's edges carry key(s); the leaf order and the fill need the key of
// the weight itself, key(sqrt(s)).  The square root is monotone, so the tree
// stays a minimum spanning tree under the weights' order.
template <int DT>
__global__ void k_mst_sqrt(u64* __restrict__ mst, u32 m)
{
    for (u32 e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        const u64 x = mst[e];
        const float s = __uint_as_float(bits_of(edge_key(x), DT));
        const u32 k = key_of(__float_as_uint(__fsqrt_rn(s)), DT);
        mst[e] = ((u64)k << 32) | (x & 0xFFFFFFFFull);
    }
}

// ------------------------------------------------------------------ host
int points_dim(int d)
{
    if (d < 1 || d > 32)
        return 0;
    int D = 2;
    while (D < d)
        D *= 2;
    return D;
}

u32 points_rows_padded(u32 n) { return (n + 255u) / 256u * 256u; }

template <class K>
static cudaError_t set_smem_pts(K kern, size_t bytes)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_pts_pad(const float* X, u32 n, int d, float* P, cudaStream_t s)
{
    const int D = points_dim(d);
    const u32 npad = points_rows_padded(n);
    const u64 total = (u64)npad * D;
    u32 grid = (u32)((total + 255) / 256);
    if (grid > 4096)
        grid = 4096;
    k_pts_pad<<<grid, 256, 0, s>>>(X, n, d, D, npad, P);
    return cudaGetLastError();
}

template <int DT, int D>
static cudaError_t rowmin_pts_d(const float* P, u32 n, u64* best, cudaStream_t s)
{
    constexpr int CPL = cols_per_lane<D>();
    constexpr u32 TCOLS = 8 * 32 * CPL;
    dim3 grid((n + TCOLS - 1) / TCOLS, (n + RP_ROWS - 1) / RP_ROWS);
    k_rowmin_pts<DT, D><<<grid, RP_THREADS, 0, s>>>(P, n, best);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t rowmin_pts_dt(const float* P, int D, u32 n, u64* best, cudaStream_t s)
{
    switch (D) {
    case 2: return rowmin_pts_d<DT, 2>(P, n, best, s);
    case 4: return rowmin_pts_d<DT, 4>(P, n, best, s);
    case 8: return rowmin_pts_d<DT, 8>(P, n, best, s);
    case 16: return rowmin_pts_d<DT, 16>(P, n, best, s);
    default: return rowmin_pts_d<DT, 32>(P, n, best, s);
    }
}

cudaError_t launch_rowmin_pts(const float* P, int D, u32 n, int dt, u64* best, cudaStream_t s)
{
    return (dt & 2) ? rowmin_pts_dt<2>(P, D, n, best, s) : rowmin_pts_dt<0>(P, D, n, best, s);
}

template <int DT, int D>
static cudaError_t contract_pts_d(const ContractArgs& ca, const float* P, int blocks, size_t smem,
                                  cudaStream_t s)
{
    auto k = k_contract_pts<DT, D>;
    cudaError_t e = set_smem_pts(k, smem);
    if (e != cudaSuccess)
        return e;
    k<<<blocks, CP_THREADS, smem, s>>>(ca, P);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t contract_pts_dt(const ContractArgs& ca, const float* P, int D, int blocks, size_t smem,
                                   cudaStream_t s)
{
    switch (D) {
    case 2: return contract_pts_d<DT, 2>(ca, P, blocks, smem, s);
    case 4: return contract_pts_d<DT, 4>(ca, P, blocks, smem, s);
    case 8: return contract_pts_d<DT, 8>(ca, P, blocks, smem, s);
    case 16: return contract_pts_d<DT, 16>(ca, P, blocks, smem, s);
    default: return contract_pts_d<DT, 32>(ca, P, blocks, smem, s);
    }
}

// one CTA per SM with every bin the shared memory holds (a second bin range
// would compute every distance again)
u32 contract_pts_bin_cap(int smem_optin)
{
    return (u32)((smem_optin - 4096) / 8);
}

cudaError_t launch_contract_pts(const ContractArgs& ca, const float* P, int D, int dt, int blocks,
                                cudaStream_t s)
{
    const size_t smem = (size_t)ca.bin_cap * sizeof(u64);
    return (dt & 2) ? contract_pts_dt<2>(ca, P, D, blocks, smem, s) : contract_pts_dt<0>(ca, P, D, blocks, smem, s);
}

cudaError_t launch_pts_gather(const float* P, int D, const u32* members, const u32* label, u32 n, float* Ps,
                              u32* pvid, u32* pcomp, cudaStream_t s)
{
    const u32 grid = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_pts_gather<<<grid, 256, 0, s>>>(P, D, members, label, n, Ps, pvid, pcomp);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t contract_sorted_dt(const ContractArgs& ca, const float* Ps, const u32* pvid, const u32* pcomp,
                                      int D, int blocks, cudaStream_t s)
{
    switch (D) {
    case 2: k_contract_pts_sorted<DT, 2><<<blocks, CS_THREADS, 0, s>>>(ca, Ps, pvid, pcomp); break;
    case 4: k_contract_pts_sorted<DT, 4><<<blocks, CS_THREADS, 0, s>>>(ca, Ps, pvid, pcomp); break;
    case 8: k_contract_pts_sorted<DT, 8><<<blocks, CS_THREADS, 0, s>>>(ca, Ps, pvid, pcomp); break;
    case 16: k_contract_pts_sorted<DT, 16><<<blocks, CS_THREADS, 0, s>>>(ca, Ps, pvid, pcomp); break;
    default: k_contract_pts_sorted<DT, 32><<<blocks, CS_THREADS, 0, s>>>(ca, Ps, pvid, pcomp); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_contract_pts_sorted(const ContractArgs& ca, const float* Ps, const u32* pvid,
                                       const u32* pcomp, int D, int dt, int blocks, cudaStream_t s)
{
    return (dt & 2) ? contract_sorted_dt<2>(ca, Ps, pvid, pcomp, D, blocks, s)
                    : contract_sorted_dt<0>(ca, Ps, pvid, pcomp, D, blocks, s);
}

cudaError_t launch_mst_sqrt(u64* mst, u32 m, int dt, cudaStream_t s)
{
    if (m == 0)
        return cudaSuccess;
    const u32 grid = (m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024;
    if (dt & 2)
        k_mst_sqrt<2><<<grid, 256, 0, s>>>(mst, m);
    else
        k_mst_sqrt<0><<<grid, 256, 0, s>>>(mst, m);
    return cudaGetLastError();
}

cudaError_t preload_points()
{
    return touch_kernels(k_pts_pad, k_rowmin_pts<0, 2>, k_rowmin_pts<0, 4>, k_rowmin_pts<0, 8>,
                         k_rowmin_pts<0, 16>, k_rowmin_pts<0, 32>, k_rowmin_pts<2, 2>, k_rowmin_pts<2, 4>,
                         k_rowmin_pts<2, 8>, k_rowmin_pts<2, 16>, k_rowmin_pts<2, 32>, k_contract_pts<0, 2>,
                         k_contract_pts<0, 4>, k_contract_pts<0, 8>, k_contract_pts<0, 16>,
                         k_contract_pts<0, 32>, k_contract_pts<2, 2>, k_contract_pts<2, 4>,
                         k_contract_pts<2, 8>, k_contract_pts<2, 16>, k_contract_pts<2, 32>, k_mst_sqrt<0>,
                         k_mst_sqrt<2>, k_pts_gather, k_contract_pts_sorted<0, 2>, k_contract_pts_sorted<0, 4>,
                         k_contract_pts_sorted<0, 8>, k_contract_pts_sorted<0, 16>,
                         k_contract_pts_sorted<0, 32>, k_contract_pts_sorted<2, 2>,
                         k_contract_pts_sorted<2, 4>, k_contract_pts_sorted<2, 8>,
                         k_contract_pts_sorted<2, 16>, k_contract_pts_sorted<2, 32>);
}

}  // namespace appd
