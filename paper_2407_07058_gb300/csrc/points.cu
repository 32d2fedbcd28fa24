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
// (k_pts_gather + k_contract_pts_sorted), both over the pairs i < j.  They compare s
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

// Two columns' squared distances to one row at once with the packed FP32
// instructions (sub.rn.f32x2, fma.rn.f32x2: each half rounded exactly as the
// scalar __fsub_rn / __fmaf_rn, so the sums are bit-identical to sq_dist):
// rr[k] holds the row's coordinate k in both halves, c2[k] the two columns'
// coordinates k (low half: the first column).  Half the issue slots of two
// scalar sums; the FMA pipe's throughput is the same.
template <int D>
__device__ __forceinline__ u64 sq_dist2(const u64* rr, const u64 (&c2)[D])
{
    u64 s = 0ull;   // +0.0f in both halves
#pragma unroll
    for (int k = 0; k < D; ++k) {
        u64 t;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(rr[k]), "l"(c2[k]));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(s) : "l"(t));
    }
    return s;
}

__device__ __forceinline__ u64 pack_f2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack_f2(u64 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
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

// For D <= 16 the columns are taken in pairs with the packed FP32
// instructions (sq_dist2), the rows' coordinates stored twice per word in
// shared memory; D = 32 keeps scalar sums (its doubled rows would not fit
// the static shared memory).
template <int DT, int D>
__global__ void __launch_bounds__(RP_THREADS, 2)
    k_rowmin_pts(const float* __restrict__ P, u32 n, u64* __restrict__ best)
{
    constexpr int CPL = cols_per_lane<D>();
    constexpr bool PACKED = D <= 16;
    constexpr u32 TCOLS = 8 * 32 * CPL;
    constexpr int SW = PACKED ? RP_ROWS * D : 1;   // packed row words
    constexpr int SF = PACKED ? 1 : RP_ROWS * D;   // scalar row words
    __shared__ __align__(16) u64 s_pts2[SW];
    __shared__ __align__(16) float s_pts[SF];
    __shared__ u64 s_row[RP_ROWS];
    const u32 i0 = blockIdx.y * RP_ROWS, c0 = blockIdx.x * TCOLS;
    if (c0 + TCOLS - 1 <= i0 || i0 >= n || c0 >= n)   // no pair i < j in this tile
        return;
    const u32 w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const u32 imax = min(n, i0 + RP_ROWS);
    for (u32 r = threadIdx.x; r < RP_ROWS; r += blockDim.x)
        s_row[r] = EDGE_INF;
    for (u32 e = threadIdx.x; e < RP_ROWS * D; e += blockDim.x) {
        const float x = P[(size_t)i0 * D + e];   // P has npad >= i0 + RP_ROWS rows
        if constexpr (PACKED)
            s_pts2[e] = pack_f2(x, x);
        else
            s_pts[e] = x;
    }
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
    u64 cx2[CPL / 2][PACKED ? D : 1];
    if constexpr (PACKED) {
#pragma unroll
        for (int p2 = 0; p2 < CPL / 2; ++p2)
#pragma unroll
            for (int k = 0; k < D; ++k)
                cx2[p2][k] = pack_f2(cx[2 * p2][k], cx[2 * p2 + 1][k]);
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
        // the row's squared distances to this lane's columns
        float sd[CPL];
        if constexpr (PACKED) {
            const u64* rr = s_pts2 + (size_t)(i - i0) * D;
#pragma unroll
            for (int p2 = 0; p2 < CPL / 2; ++p2)
                unpack_f2(sq_dist2<D>(rr, cx2[p2]), sd[2 * p2], sd[2 * p2 + 1]);
        } else {
            float rx[D];
#pragma unroll
            for (int k = 0; k < D; ++k)
                rx[k] = s_pts[(i - i0) * D + k];
#pragma unroll
            for (int c = 0; c < CPL; ++c)
                sd[c] = sq_dist<D>(rx, cx[c]);
        }
        u32 rk = 0xFFFFFFFFu, rj = 0xFFFFFFFFu;
        if (clear) {
#pragma unroll
            for (int c = CPL - 1; c >= 0; --c) {
                const u32 u = sbits_order<DT>(sd[c]);
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
                const u32 u = sbits_order<DT>(sd[c]);
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

// ------------------------------------------------ level 0, sorted columns
// After the level-0 step the members list holds the vertices grouped by
// component (group A at positions gstart[A] .. gstart[A+1]).  k_pts_gather
// copies the coordinates into that order (Ps), with each position's vertex
// (pvid) and component (pcomp).  k_contract_pts_sorted then takes a chunk of
// at most CONTRACT_ROWS rows of a group A (the step's work items, so a large
// group is shared by several CTAs) against every later position: those
// columns belong to groups B > A, each group's columns contiguous, so
// P'(A, B) = min over the run of B's columns of the column minima -- a run
// reduction instead of a bin array.  Row A of P' holds INF for B <= A (the
// step leaves a group of several chunks an all-INF row, and its chunks merge
// by atomic minima), so C_1(A, B) = min(P'(A, B), P'(B, A)) as for the
// upper-triangle P of a stored W, and the same column minima and level-1
// symmetrization follow.
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
    constexpr int CPC = cols_sorted<D>();       // columns per thread and pass
    constexpr int PASSES = 8 / CPC;             // passes per chunk between barriers
    constexpr u32 CH = CS_THREADS * CPC * PASSES;   // columns per chunk (2048)
    __shared__ __align__(16) float s_rp[CONTRACT_ROWS * D];
    __shared__ u32 s_rv[CONTRACT_ROWS];
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
    const u32 total_chunks = *(volatile u32*)&ctr->total_chunks;
    const u32 tid = threadIdx.x;
    if (n <= a.comp_max_c)
        for (u32 v = blockIdx.x * blockDim.x + tid; v < a.n; v += gridDim.x * blockDim.x)
            a.comp[v] = a.label[a.comp[v]];
    for (;;) {
        if (tid == 0)
            s_item = atomicAdd(&ctr->item_next, 1u);
        __syncthreads();
        const u32 ch = s_item;
        if (ch >= total_chunks)
            break;
        const u32 A = a.item_group[ch];
        const u32 g0 = a.gstart[A] + (ch - a.chunk_start[A]) * CONTRACT_ROWS;
        const u32 nrows = min(a.gstart[A + 1], g0 + CONTRACT_ROWS) - g0;
        const bool single = a.nchunk[A] == 1;
        const u32 qbeg = a.gstart[A + 1];   // the first position of a later group
        for (u32 e = tid; e < nrows * D; e += CS_THREADS)
            s_rp[e] = Ps[(size_t)g0 * D + e];
        if (tid < nrows)
            s_rv[tid] = pvid[g0 + tid];
        u64* row = a.cout + (size_t)A * cn;
        if (single)   // no pairs with groups B <= A (a multi-chunk row is all INF already)
            for (u32 b = tid; b <= A; b += CS_THREADS)
                row[b] = EDGE_INF;
        if (tid == 0) {
            s_carry_b[0] = 0xFFFFFFFFu;
            s_carry_e[0] = EDGE_INF;
        }
        u64 mrow = EDGE_INF;   // this thread's part of the chunk's row minimum
        auto put = [&](u32 B, u64 v) {
            if (single)
                row[B] = v;
            else if (v < row[B])
                atomicMin(row + B, v);
            mrow = v < mrow ? v : mrow;
        };
        __syncthreads();
        int cur = 0;
        for (u32 q0 = qbeg; q0 < n; q0 += CH) {
            // 1. each column's smallest (order, row vertex) over the chunk's
            // rows; in pass p thread t takes the columns
            // q0 + t + (p * CPC + c) * CS_THREADS, so the coordinate loads and
            // the shared-memory stores run contiguously across a warp
#pragma unroll 1
            for (int pass = 0; pass < PASSES; ++pass) {
                float cx[CPC][D];
                u32 bk[CPC], bv[CPC], vq[CPC];
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    const u32 q = q0 + tid + (pass * CPC + c) * CS_THREADS;
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
                    float rx[D], sd[CPC];
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        rx[k] = s_rp[r * D + k];
#pragma unroll
                    for (int c = 0; c < CPC; ++c)
                        sd[c] = sq_dist<D>(rx, cx[c]);
                    const u32 vr = s_rv[r];
#pragma unroll
                    for (int c = 0; c < CPC; ++c) {
                        const u32 u = sbits_order<DT>(sd[c]);
                        if (u < bk[c] || (u == bk[c] && vr < bv[c])) {
                            bk[c] = u;
                            bv[c] = vr;
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    const u32 i = tid + (pass * CPC + c) * CS_THREADS;
                    const u32 q = q0 + i;
                    if (q < n && bv[c] != 0xFFFFFFFFu) {
                        s_e[i] = ((u64)order_to_key<DT>(bk[c]) << 32) |
                                 pair_code(min(bv[c], vq[c]), max(bv[c], vq[c]), n);
                        s_b[i] = pcomp[q];
                    } else {
                        s_e[i] = EDGE_INF;
                        s_b[i] = q < n ? pcomp[q] : 0xFFFFFFFFu;
                    }
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
                    if (cb == B)
                        v = ce < v ? ce : v;
                    else if (cb != 0xFFFFFFFFu)
                        put(cb, ce);   // the carried run ended with the last chunk
                }
                if (j < ncol) {
                    put(B, v);
                } else {
                    s_carry_b[cur ^ 1] = B;
                    s_carry_e[cur ^ 1] = v;
                }
            }
            cur ^= 1;
            __syncthreads();
        }
        // the last run of the chunk's columns
        if (tid == 0 && s_carry_b[cur] != 0xFFFFFFFFu)
            put(s_carry_b[cur], s_carry_e[cur]);
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
                         k_rowmin_pts<2, 8>, k_rowmin_pts<2, 16>, k_rowmin_pts<2, 32>, k_mst_sqrt<0>,
                         k_mst_sqrt<2>, k_pts_gather, k_contract_pts_sorted<0, 2>, k_contract_pts_sorted<0, 4>,
                         k_contract_pts_sorted<0, 8>, k_contract_pts_sorted<0, 16>,
                         k_contract_pts_sorted<0, 32>, k_contract_pts_sorted<2, 2>,
                         k_contract_pts_sorted<2, 4>, k_contract_pts_sorted<2, 8>,
                         k_contract_pts_sorted<2, 16>, k_contract_pts_sorted<2, 32>);
}

}  // namespace appd
