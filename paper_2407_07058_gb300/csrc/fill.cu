// fill.cu -- writing M from the leaf order.
//
// k_fill (the product path): M(i,j) = largest gap between pos(i) and pos(j),
// i.e. the height of the single-linkage merge that first joins i and j
// (reading the distances off the dendrogram, Section 7).  Each CTA owns a
// tile of 256 columns and a range of rows:
//   - the columns' positions are sorted once per CTA (bitonic in smem);
//   - A[k] = largest gap between consecutive sorted column positions (one
//     sparse-table query each), with a small sparse table over A in smem;
//   - per chunk of 32 rows, every row r with position p splits the sorted
//     columns at t (columns left / right of p); the values for the sorted
//     columns are running maxima of A outward from t, written into smem;
//   - rows are stored coalesced (16-byte streaming stores), each output
//     element once.  The kernel is bound by HBM write bandwidth.
// k_a4_fill (comparison): Algorithm 4's calculation-and-copy (Sections 3, 5,
// and the per-edge parallel variant of Section 6.2): one work item per MST
// edge e fills the cross block tree1 x tree2 and its transpose with w(e).
// In the leaf order tree1 is [pos(nha(y)), pos(y)) and tree2 is
// [pos(y), pos(y) + nsize(y)) for the edge above vertex y; the target cells
// are scattered in M, which is what this form costs.
#include "internal.h"

namespace appd {

constexpr int FC = 256;   // columns per CTA
constexpr int FR = 32;    // rows per chunk
constexpr int FA_LEVELS = 8;

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

template <int DT>
__global__ void __launch_bounds__(256) k_fill(const u32* __restrict__ pos, const u32* __restrict__ st,
                                              u32 n, u32 rows_per_cta, u32* __restrict__ M)
{
    __shared__ u64 s_sort[FC];
    __shared__ u32 s_q[FC];
    __shared__ u32 s_rank[FC];
    __shared__ u32 s_A[FA_LEVELS][FC];
    __shared__ u32 s_V[FR][FC + 1];
    __shared__ u32 s_p[FR], s_t[FR], s_L[FR], s_R[FR];

    const u32 tid = threadIdx.x;
    const u32 j0 = blockIdx.x * FC;
    const u32 nc = min((u32)FC, n - j0);

    u32 q = (tid < nc) ? __ldg(pos + j0 + tid) : 0xFFFFFFFFu;
    s_sort[tid] = ((u64)q << 32) | tid;
    __syncthreads();
    for (u32 k = 2; k <= FC; k <<= 1) {
        for (u32 j = k >> 1; j > 0; j >>= 1) {
            u32 ixj = tid ^ j;
            if (ixj > tid) {
                bool up = (tid & k) == 0;
                u64 x = s_sort[tid], y = s_sort[ixj];
                if ((x > y) == up) {
                    s_sort[tid] = y;
                    s_sort[ixj] = x;
                }
            }
            __syncthreads();
        }
    }
    {
        u64 e = s_sort[tid];
        s_q[tid] = (u32)(e >> 32);
        if (tid < nc)
            s_rank[(u32)e] = tid;
    }
    __syncthreads();
    if (tid + 1 < nc)
        s_A[0][tid] = rmq_gap(st, n, s_q[tid], s_q[tid + 1] - 1);
    __syncthreads();
    for (int l = 1; l < FA_LEVELS; ++l) {
        u32 h = 1u << (l - 1);
        if (tid + 2 * h <= nc - 1) {
            u32 x = s_A[l - 1][tid], y = s_A[l - 1][tid + h];
            s_A[l][tid] = x > y ? x : y;
        }
        __syncthreads();
    }
    auto rangeA = [&](u32 a, u32 b) -> u32 {   // max A[a..b], 0 if empty
        if ((int)b < (int)a)
            return 0u;
        u32 l = 31 - __clz(b - a + 1);
        u32 x = s_A[l][a], y = s_A[l][b - (1u << l) + 1];
        return x > y ? x : y;
    };

    const u32 r_begin = blockIdx.y * rows_per_cta;
    const u32 r_end = min(n, r_begin + rows_per_cta);
    const u32 lane = tid & 31, w = tid >> 5;
    const bool vec = (n % 4u) == 0 && (((uintptr_t)M & 15u) == 0);
    for (u32 i0 = r_begin; i0 < r_end; i0 += FR) {
        const u32 nr = min((u32)FR, r_end - i0);
        if (tid < nr) {
            u32 p = __ldg(pos + i0 + tid);
            u32 lo = 0, hi = nc;
            while (lo < hi) {
                u32 mid = (lo + hi) >> 1;
                if (s_q[mid] < p)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            u32 Lv = 0, Rv = 0;
            if (lo > 0)
                Lv = rmq_gap(st, n, s_q[lo - 1], p - 1);
            if (lo < nc && s_q[lo] != p)
                Rv = rmq_gap(st, n, p, s_q[lo] - 1);
            s_p[tid] = p;
            s_t[tid] = lo;
            s_L[tid] = Lv;
            s_R[tid] = Rv;
        }
        __syncthreads();
        if (lane < nr) {
            const u32 t = s_t[lane], p = s_p[lane];
            const u32 ks = 32 * w, ke = min(ks + 32, nc);
            // right of the row's position: running max upward from t
            u32 k = max(ks, t);
            if (k < ke) {
                u32 cur = s_R[lane];
                u32 pre = rangeA(t, k - 1);
                cur = cur > pre ? cur : pre;
                for (;;) {
                    bool diag = (k == t) && (s_q[t] == p);
                    s_V[lane][k] = diag ? 0u : bits_of(cur, DT);
                    if (++k >= ke)
                        break;
                    u32 a = s_A[0][k - 1];
                    cur = cur > a ? cur : a;
                }
            }
            // left of it: running max downward from t-1
            const u32 kt = min(ke, t);
            if (kt > ks) {
                k = kt - 1;
                u32 cur = s_L[lane];
                u32 pre = rangeA(k, t - 2);
                cur = cur > pre ? cur : pre;
                for (;;) {
                    s_V[lane][k] = bits_of(cur, DT);
                    if (k == ks)
                        break;
                    --k;
                    u32 a = s_A[0][k];
                    cur = cur > a ? cur : a;
                }
            }
        }
        __syncthreads();
        if (vec) {
            const u32 g4 = nc >> 2;
            for (u32 g = tid; g < nr * g4; g += 256) {
                const u32 rr = g / g4, c4 = g - rr * g4, jj = 4 * c4;
                uint4 o;
                o.x = s_V[rr][s_rank[jj]];
                o.y = s_V[rr][s_rank[jj + 1]];
                o.z = s_V[rr][s_rank[jj + 2]];
                o.w = s_V[rr][s_rank[jj + 3]];
                __stcs(reinterpret_cast<uint4*>(M + (size_t)(i0 + rr) * n + j0 + jj), o);
            }
        } else {
            for (u32 g = tid; g < nr * nc; g += 256) {
                const u32 rr = g / nc, jj = g - rr * nc;
                M[(size_t)(i0 + rr) * n + j0 + jj] = s_V[rr][s_rank[jj]];
            }
        }
        __syncthreads();
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
    // enough CTAs to fill the GPU, but at least 32 rows per CTA
    u64 target = (u64)ws.sms * 8;
    u32 rows = (u32)(((u64)n * gx + target - 1) / target);
    rows = (rows + FR - 1) / FR * FR;
    if (rows < FR)
        rows = FR;
    if (rows > 1024)
        rows = 1024;
    dim3 grid(gx, (n + rows - 1) / rows);
    if (dt == 0)
        k_fill<0><<<grid, 256, 0, s>>>(ws.pos, ws.st, n, rows, (u32*)M);
    else
        k_fill<1><<<grid, 256, 0, s>>>(ws.pos, ws.st, n, rows, (u32*)M);
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
