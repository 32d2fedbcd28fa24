// fill.cu -- writing M from the leaf order.
//
// k_fill (the product path): M(i,j) = largest gap between pos(i) and pos(j),
// i.e. the height of the single-linkage merge that first joins i and j
// (reading the distances off the dendrogram, Section 7).  Each CTA owns a
// tile of 256 columns and a range of rows:
//   - the columns' positions are sorted once per CTA (bitonic in smem);
//   - A[k] = largest gap between consecutive sorted column positions (one
//     sparse-table query each);
//   - every row with position p splits the sorted columns at t; its values
//     are running maxima of A outward from t, combined with the largest gap
//     from p to the nearest column on each side.  The running maxima for all
//     t form a (FC+1) x FC table built once per CTA;
//   - each warp writes whole row segments with 16-byte streaming stores,
//     each output element once.  The kernel is bound by HBM write bandwidth.
// k_a4_fill (comparison): Algorithm 4's calculation-and-copy (Sections 3, 5,
// and the per-edge parallel variant of Section 6.2): one work item per MST
// edge e fills the cross block tree1 x tree2 and its transpose with w(e).
// In the leaf order tree1 is [pos(nha(y)), pos(y)) and tree2 is
// [pos(y), pos(y) + nsize(y)) for the edge above vertex y; the target cells
// are scattered in M, which is what this form costs.
#include "internal.h"

namespace appd {

constexpr int FC = 128;   // columns per CTA
constexpr int FT = 256;   // threads per CTA

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
    u64 sort[FC];
    u32 q[FC];           // sorted column positions
    u32 col[FC];         // sorted index -> column offset
    u32 rank[FC];        // column offset -> sorted index
    u32 A[FC];           // A[k] = max gap between q[k] and q[k+1]
};

size_t fill_smem_bytes(u32 rows_per_cta) { return sizeof(FillSmem) + (size_t)rows_per_cta * 12; }

// For a row with leaf position p, let t = #{sorted columns with q < p}.  Its
// value at the column with sorted index k is max(R_p, A[t..k-1]) for k >= t
// and max(L_p, A[k..t-2]) for k < t, where R_p / L_p are the largest gaps
// from p to the nearest column on each side.  The A-parts depend only on
// (t, k): they form the table T, built once per CTA, so each output element
// costs one shared load, one max and the key-to-bits transform.
template <int DT>
__global__ void __launch_bounds__(FT, 2) k_fill(const u32* __restrict__ pos, const u32* __restrict__ st,
                                                u32 n, u32 rows_per_cta, u32* __restrict__ M)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FillSmem& S = *reinterpret_cast<FillSmem*>(smem_raw);
    u32* s_t = reinterpret_cast<u32*>(smem_raw + sizeof(FillSmem));
    u32* s_L = s_t + rows_per_cta;
    u32* s_R = s_L + rows_per_cta;

    const u32 tid = threadIdx.x;
    const u32 j0 = blockIdx.x * FC;
    const u32 nc = min((u32)FC, n - j0);
    const u32 r0 = blockIdx.y * rows_per_cta;
    const u32 nr = min(rows_per_cta, n - r0);

    // 1. sort the tile's column positions (bitonic, FC elements)
    if (tid < FC)
        S.sort[tid] = ((u64)(tid < nc ? __ldg(pos + j0 + tid) : 0xFFFFFFFFu) << 32) | tid;
    __syncthreads();
    for (u32 k = 2; k <= FC; k <<= 1) {
        for (u32 j = k >> 1; j > 0; j >>= 1) {
            if (tid < FC) {
                u32 ixj = tid ^ j;
                if (ixj > tid) {
                    bool up = (tid & k) == 0;
                    u64 x = S.sort[tid], y = S.sort[ixj];
                    if ((x > y) == up) {
                        S.sort[tid] = y;
                        S.sort[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (tid < FC) {
        u64 e = S.sort[tid];
        S.q[tid] = (u32)(e >> 32);
        S.col[tid] = (u32)e;
        if (tid < nc)
            S.rank[(u32)e] = tid;
    }
    __syncthreads();
    // 2. gaps between consecutive sorted columns; row split points and sides
    if (tid + 1 < nc)
        S.A[tid] = rmq_gap(st, n, S.q[tid], S.q[tid + 1] - 1);
    for (u32 r = tid; r < nr; r += FT) {
        u32 p = __ldg(pos + r0 + r);
        u32 lo = 0, hi = nc;
        while (lo < hi) {
            u32 mid = (lo + hi) >> 1;
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
    // 3. the table: row t holds the running maxima outward from split t
    if (tid <= nc) {
        const u32 t = tid;
        u32 cur = 0;
        for (u32 k = t; k < nc; ++k) {
            if (k > t) {
                u32 a = S.A[k - 1];
                cur = cur > a ? cur : a;
            }
            S.T[t][S.col[k]] = cur;
        }
        cur = 0;
        for (u32 k = t; k-- > 0;) {
            if (k + 1 < t) {
                u32 a = S.A[k];
                cur = cur > a ? cur : a;
            }
            S.T[t][S.col[k]] = cur;
        }
    }
    __syncthreads();
    // 4. rows: one warp per row, each lane four consecutive columns
    const u32 lane = tid & 31, w = tid >> 5;
    const bool vec = (nc == FC) && (n % 4u) == 0 && (((uintptr_t)M & 15u) == 0);
    if (vec) {
        const u32 jj = 4 * lane;
        const uint4 rk = *reinterpret_cast<const uint4*>(&S.rank[jj]);
        for (u32 r = w; r < nr; r += FT / 32) {
            const u32 t = s_t[r], L = s_L[r], R = s_R[r];
            const uint4 tv = *reinterpret_cast<const uint4*>(&S.T[t][jj]);
            u32 v0 = max(tv.x, rk.x >= t ? R : L);
            u32 v1 = max(tv.y, rk.y >= t ? R : L);
            u32 v2 = max(tv.z, rk.z >= t ? R : L);
            u32 v3 = max(tv.w, rk.w >= t ? R : L);
            uint4 o = make_uint4(bits_of(v0, DT), bits_of(v1, DT), bits_of(v2, DT), bits_of(v3, DT));
            const u32 i = r0 + r;
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
        for (u32 r = w; r < nr; r += FT / 32) {
            const u32 t = s_t[r], L = s_L[r], R = s_R[r];
            const u32 i = r0 + r;
            for (u32 c = lane; c < nc; c += 32) {
                u32 v = max(S.T[t][c], S.rank[c] >= t ? R : L);
                M[(size_t)i * n + j0 + c] = (j0 + c == i) ? 0u : bits_of(v, DT);
            }
        }
    }
}

// ----------------------------------------------------- Algorithm 4 form
constexpr int A4_TR = 8;     // tree1 positions per tile
constexpr int A4_TC = 256;   // tree2 positions per tile

__global__ void k_a4_count(const u32* __restrict__ pos, const u32* __restrict__ nha,
                           const u32* __restrict__ nsize, u32 n, u32* __restrict__ tiles)
{
    for (u32 y = blockIdx.x * blockDim.x + threadIdx.x + 1; y < n; y += gridDim.x * blockDim.x) {
        u32 rows = pos[y] - pos[nha[y]];
        u32 cols = nsize[y];
        tiles[y - 1] = ((rows + A4_TR - 1) / A4_TR) * ((cols + A4_TC - 1) / A4_TC);
    }
}

__global__ void k_a4_scan(u32* __restrict__ tiles, u32 m, Counters* ctr)
{
    BlockTeam t;
    u32 total = 0;
    team_excl_scan(t, tiles, tiles, m, nullptr, &total);
    if (threadIdx.x == 0) {
        tiles[m] = total;
        ctr->fill_total = total;
        ctr->fill_next = 0;
    }
}

template <int DT>
__global__ void __launch_bounds__(256) k_a4_fill(const u32* __restrict__ pos, const u32* __restrict__ order,
                                                 const u32* __restrict__ nha, const u32* __restrict__ nsize,
                                                 const u32* __restrict__ pe_key, const u32* __restrict__ start,
                                                 u32 n, const Counters* __restrict__ ctr,
                                                 u32* __restrict__ M)
{
    __shared__ u32 s_e;
    const u32 total = ctr->fill_total, m = n - 1;
    for (u32 tile = blockIdx.x; tile < total; tile += gridDim.x) {
        if (threadIdx.x == 0) {
            u32 lo = 0, hi = m - 1;   // last edge with start <= tile
            while (lo < hi) {
                u32 mid = (lo + hi + 1) >> 1;
                if (start[mid] <= tile)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            s_e = lo;
        }
        __syncthreads();
        const u32 e = s_e, y = e + 1;
        __syncthreads();
        const u32 py = pos[y], pp = pos[nha[y]];
        if (pp >= py || py + nsize[y] > n)   // invalid order: nothing in range to write
            continue;
        const u32 rows = py - pp, cols = nsize[y];
        const u32 tcols = (cols + A4_TC - 1) / A4_TC;
        const u32 local = tile - start[e];
        const u32 tr = local / tcols, tc = local - tr * tcols;
        const u32 val = bits_of(pe_key[y], DT);
        const u32 z = tc * A4_TC + threadIdx.x;
        if (z < cols) {
            const u32 j = order[py + z];
            const u32 x0 = tr * A4_TR, x1 = min(rows, x0 + A4_TR);
            for (u32 x = x0; x < x1; ++x) {
                const u32 i = order[pp + x];
                M[(size_t)i * n + j] = val;
                M[(size_t)j * n + i] = val;
            }
        }
    }
}

__global__ void k_diag_zero(u32* __restrict__ M, u32 n)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        M[(size_t)i * n + i] = 0u;
}

cudaError_t run_fill(Workspace& ws, int dt, void* M, cudaStream_t s)
{
    const u32 n = (u32)ws.n;
    if (n == 1)
        return cudaMemsetAsync(M, 0, sizeof(u32), s);
    const u32 gx = (n + FC - 1) / FC;
    // rows per CTA: enough CTAs for several waves, at most 1024 rows
    u64 target = (u64)ws.sms * 2 * 4;
    u32 rows = (u32)(((u64)n * gx + target - 1) / target);
    if (rows < 32)
        rows = 32;
    if (rows > 1024)
        rows = 1024;
    dim3 grid(gx, (n + rows - 1) / rows);
    const size_t smem = fill_smem_bytes(rows);
    cudaError_t e;
    if (dt == 0) {
        if ((e = cudaFuncSetAttribute(k_fill<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)fill_smem_bytes(1024))) != cudaSuccess)
            return e;
        k_fill<0><<<grid, FT, smem, s>>>(ws.pos, ws.st, n, rows, (u32*)M);
    } else {
        if ((e = cudaFuncSetAttribute(k_fill<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)fill_smem_bytes(1024))) != cudaSuccess)
            return e;
        k_fill<1><<<grid, FT, smem, s>>>(ws.pos, ws.st, n, rows, (u32*)M);
    }
    return cudaGetLastError();
}

cudaError_t run_fill_alg4(Workspace& ws, int dt, void* M, u32* status, cudaStream_t s)
{
    (void)status;
    const u32 n = (u32)ws.n;
    if (n == 1)
        return cudaMemsetAsync(M, 0, sizeof(u32), s);
    const u32 m = n - 1;
    k_a4_count<<<(m + 255) / 256, 256, 0, s>>>(ws.pos, ws.nha, ws.nsize, n, ws.a4_start);
    k_a4_scan<<<1, 1024, 0, s>>>(ws.a4_start, m, ws.ctr);
    k_diag_zero<<<(n + 255) / 256, 256, 0, s>>>((u32*)M, n);
    const int grid = ws.sms * 8;
    if (dt == 0)
        k_a4_fill<0><<<grid, 256, 0, s>>>(ws.pos, ws.order, ws.nha, ws.nsize, ws.pe_key, ws.a4_start,
                                         n, ws.ctr, (u32*)M);
    else
        k_a4_fill<1><<<grid, 256, 0, s>>>(ws.pos, ws.order, ws.nha, ws.nsize, ws.pe_key, ws.a4_start,
                                         n, ws.ctr, (u32*)M);
    return cudaGetLastError();
}

}  // namespace appd
