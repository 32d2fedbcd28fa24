// fill_device.cuh -- the fill tile shared by the single-solve kernel
// (fill.cu) and the batched kernel (batched.cu).
#pragma once

#include "internal.h"

namespace appd {

constexpr int FC = 128;   // columns per CTA
constexpr int FT = 512;   // threads per CTA (32 warps per SM at two CTAs: more stores in flight)

__device__ __forceinline__ u32 rmq_gap(const u32* __restrict__ st, u32 stride, u32 a, u32 b)
{
    // max gap[a..b]; an empty range (only on an invalid order) gives 0
    if (b < a)
        return 0u;
    u32 l = 31 - __clz(b - a + 1);
    u32 x = __ldg(st + (size_t)l * stride + a);
    u32 y = __ldg(st + (size_t)l * stride + b - (1u << l) + 1);
    return x > y ? x : y;
}

// dynamic shared memory layout of k_fill
struct FillSmem {
    u32 T[FC + 1][FC];   // T[t][col]: running max of A outward from split t
    u32 q[FC];           // sorted column positions
    u32 col[FC];         // sorted index -> column offset
    u32 rank[FC];        // column offset -> sorted index
    u32 A[FC];           // A[k] = max gap between q[k] and q[k+1]
};

inline size_t fill_smem_bytes(u32 rows_per_cta) { return sizeof(FillSmem) + (size_t)rows_per_cta * 12; }

// For a row with leaf position p, let t = #{sorted columns with q < p}.  Its
// value at the column with sorted index k is max(R_p, A[t..k-1]) for k >= t
// and max(L_p, A[k..t-2]) for k < t, where R_p / L_p are the largest gaps
// from p to the nearest column on each side.  The A-parts depend only on
// (t, k): they form the table T, built once per tile, so each output element
// costs one shared load, one max and the key-to-bits transform.
// One tile: columns [j0, j0+FC) x rows [r0, r0+nr), the rows in batches of
// rows_cap.  smem_raw holds a FillSmem followed by 3 * rows_cap u32; every
// thread of the CTA (>= FC + 1 threads) calls it.
template <int DT>
__device__ __forceinline__ void fill_tile(const u32* __restrict__ pos, const u32* __restrict__ st,
                                          u32 n, u32 j0, u32 r0, u32 nr, u32 rows_cap,
                                          u32* __restrict__ M, unsigned char* smem_raw)
{
    FillSmem& S = *reinterpret_cast<FillSmem*>(smem_raw);
    u32* s_t = reinterpret_cast<u32*>(smem_raw + sizeof(FillSmem));
    u32* s_L = s_t + rows_cap;
    u32* s_R = s_L + rows_cap;
    const u32 tid = threadIdx.x, nthr = blockDim.x;
    const u32 nc = min((u32)FC, n - j0);

    // 1. sort the tile's column positions: positions are distinct, so a
    //    column's sorted index is the number of smaller positions
    if (tid < FC)
        S.q[tid] = tid < nc ? __ldg(pos + j0 + tid) : 0xFFFFFFFFu;
    __syncthreads();
    if (tid < nc) {
        const u32 p = S.q[tid];
        u32 k = 0;
#pragma unroll 8
        for (u32 c = 0; c < nc; ++c)
            k += S.q[c] < p;
        S.rank[tid] = k;
        S.A[k] = p;       // A holds the sorted positions until step 2
    }
    __syncthreads();
    if (tid < nc) {
        S.col[S.rank[tid]] = tid;
        S.q[tid] = S.A[tid];
    }
    __syncthreads();
    // 2. gaps between consecutive sorted columns
    u32 gap = 0;
    if (tid + 1 < nc)
        gap = rmq_gap(st, n, S.q[tid], S.q[tid + 1] - 1);
    __syncthreads();
    if (tid + 1 < nc)
        S.A[tid] = gap;
    __syncthreads();
    // 3. the table, one sorted column per thread: T[t][col k] is the max of
    //    A[t..k-1] for t <= k and of A[k..t-2] for t > k (0 when empty).
    //    The 32 columns a warp writes at once are distinct, so the stores
    //    spread over the banks.
    if (tid < nc) {
        const u32 k = tid, ck = S.col[k];
        u32 cur = 0;
        for (u32 t = k + 1; t-- > 0;) {
            if (t < k)
                cur = max(cur, S.A[t]);
            S.T[t][ck] = cur;
        }
        cur = 0;
        for (u32 t = k + 1; t <= nc; ++t) {
            if (t >= k + 2)
                cur = max(cur, S.A[t - 2]);
            S.T[t][ck] = cur;
        }
    }
    const u32 lane = tid & 31, w = tid >> 5;
    const bool vec = (nc == FC) && (n % 4u) == 0 && (((uintptr_t)M & 15u) == 0);
    for (u32 rb = 0; rb < nr; rb += rows_cap) {
        const u32 nb = min(rows_cap, nr - rb);
        // row split points and sides
        for (u32 r = tid; r < nb; r += nthr) {
            const u32 p = __ldg(pos + r0 + rb + r);
            u32 lo = 0, hi = nc;
            while (lo < hi) {
                const u32 mid = (lo + hi) >> 1;
                if (S.q[mid] < p)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            s_t[r] = lo;
            s_L[r] = lo > 0 ? rmq_gap(st, n, S.q[lo - 1], p - 1) : 0u;
            s_R[r] = (lo < nc && S.q[lo] != p) ? rmq_gap(st, n, p, S.q[lo] - 1) : 0u;
        }
        __syncthreads();
        // 4. rows: one warp per row, each lane four consecutive columns
        if (vec) {
            const u32 jj = 4 * lane;
            const uint4 rk = *reinterpret_cast<const uint4*>(&S.rank[jj]);
            for (u32 r = w; r < nb; r += nthr / 32) {
                const u32 t = s_t[r], L = s_L[r], R = s_R[r];
                const uint4 tv = *reinterpret_cast<const uint4*>(&S.T[t][jj]);
                u32 v0 = max(tv.x, rk.x >= t ? R : L);
                u32 v1 = max(tv.y, rk.y >= t ? R : L);
                u32 v2 = max(tv.z, rk.z >= t ? R : L);
                u32 v3 = max(tv.w, rk.w >= t ? R : L);
                uint4 o = make_uint4(bits_of(v0, DT), bits_of(v1, DT), bits_of(v2, DT), bits_of(v3, DT));
                const u32 i = r0 + rb + r;
                const u32 dc = i - j0 - jj;     // the diagonal cell is all-zero bits
                if (dc < 4u) {
                    if (dc == 0) o.x = 0u;
                    if (dc == 1) o.y = 0u;
                    if (dc == 2) o.z = 0u;
                    if (dc == 3) o.w = 0u;
                }
                __stcs(reinterpret_cast<uint4*>(M + (size_t)i * n + j0 + jj), o);
            }
        } else {
            // rows not 16-byte aligned (or a narrow tile): 4-byte stores, the
            // lane's four column ranks kept in registers
            u32 rk[FC / 32];
#pragma unroll
            for (int k = 0; k < FC / 32; ++k)
                rk[k] = (lane + 32 * k < nc) ? S.rank[lane + 32 * k] : 0u;
            for (u32 r = w; r < nb; r += nthr / 32) {
                const u32 t = s_t[r], L = s_L[r], R = s_R[r];
                const u32 i = r0 + rb + r;
                u32* row = M + (size_t)i * n + j0;
                const u32 dcol = i - j0;   // the diagonal's column in this tile (if < nc)
#pragma unroll
                for (int k = 0; k < FC / 32; ++k) {
                    const u32 c = lane + 32 * k;
                    if (c < nc) {
                        const u32 v = max(S.T[t][c], rk[k] >= t ? R : L);
                        __stcs(row + c, c == dcol ? 0u : bits_of(v, DT));
                    }
                }
            }
        }
        __syncthreads();   // the next batch (or tile) reuses the shared memory
    }
}

}  // namespace appd
