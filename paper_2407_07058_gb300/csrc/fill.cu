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
#include "fill_device.cuh"

namespace appd {

// rows_per_cta rows of one column block per CTA, in batches of rows_cap
// (the column block's sort and table are built once per CTA)
constexpr u32 FILL_ROWS_MAX = 8192;

template <int DT>
__global__ void __launch_bounds__(FT, 2) k_fill(const u32* __restrict__ pos, const u32* __restrict__ st,
                                                u32 n, u32 rows_per_cta, u32 rows_cap, u32* __restrict__ M,
                                                const Counters* __restrict__ ctr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (solve_failed(&ctr->bar))   // no valid leaf order: leave M unwritten
        return;
    const u32 r0 = blockIdx.y * rows_per_cta;
    fill_tile<DT>(pos, st, n, blockIdx.x * FC, r0, min(rows_per_cta, n - r0), rows_cap, M, smem_raw);
}

// ----------------------------------------------------- Algorithm 4 form
constexpr int A4_TR = 8;     // tree1 positions per tile
constexpr int A4_TC = 256;   // tree2 positions per tile

__global__ void k_a4_count(const u32* __restrict__ pos, const u32* __restrict__ nha,
                           const u32* __restrict__ nsize, u32 n, u32* __restrict__ tiles,
                           const Counters* __restrict__ ctr)
{
    if (solve_failed(&ctr->bar))   // no valid leaf order: leave M unwritten
        return;
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
    if (solve_failed(&ctr->bar))
        return;
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

cudaError_t preload_fill()
{
    return touch_kernels(k_fill<0>, k_fill<1>, k_fill<2>, k_fill<3>, k_a4_count, k_a4_scan, k_diag_zero,
                         k_a4_fill<0>, k_a4_fill<1>, k_a4_fill<2>, k_a4_fill<3>);
}

cudaError_t run_fill(Workspace& ws, int dt, void* M, cudaStream_t s)
{
    const u32 n = (u32)ws.n;
    if (n == 1)
        return cudaMemsetAsync(M, 0, sizeof(u32), s);
    const u32 gx = (n + FC - 1) / FC;
    // rows per CTA: enough CTAs for several waves, at most FILL_ROWS_MAX rows
    // (handled in batches of at most 1024, so the shared memory stays small)
    u64 target = (u64)ws.sms * 2 * 4;
    u32 rows = (u32)(((u64)n * gx + target - 1) / target);
    if (rows < 32)
        rows = 32;
    if (rows > FILL_ROWS_MAX)
        rows = FILL_ROWS_MAX;
    const u32 cap = rows < 1024 ? rows : 1024;
    dim3 grid(gx, (n + rows - 1) / rows);
    const size_t smem = fill_smem_bytes(cap);
    cudaError_t e;
    auto kf = dt == 0 ? k_fill<0> : dt == 1 ? k_fill<1> : dt == 2 ? k_fill<2> : k_fill<3>;
    if ((e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fill_smem_bytes(1024))) != cudaSuccess)
        return e;
    kf<<<grid, FT, smem, s>>>(ws.pos, ws.st, n, rows, cap, (u32*)M, ws.ctr);
    return cudaGetLastError();
}

cudaError_t run_fill_alg4(Workspace& ws, int dt, void* M, u32* status, cudaStream_t s)
{
    (void)status;
    const u32 n = (u32)ws.n;
    if (n == 1)
        return cudaMemsetAsync(M, 0, sizeof(u32), s);
    const u32 m = n - 1;
    k_a4_count<<<(m + 255) / 256, 256, 0, s>>>(ws.pos, ws.nha, ws.nsize, n, ws.a4_start, ws.ctr);
    k_a4_scan<<<1, 1024, 0, s>>>(ws.a4_start, m, ws.ctr);
    k_diag_zero<<<(n + 255) / 256, 256, 0, s>>>((u32*)M, n);
    const int grid = ws.sms * 8;
    auto ka = dt == 0 ? k_a4_fill<0> : dt == 1 ? k_a4_fill<1> : dt == 2 ? k_a4_fill<2> : k_a4_fill<3>;
    ka<<<grid, 256, 0, s>>>(ws.pos, ws.order, ws.nha, ws.nsize, ws.pe_key, ws.a4_start, n, ws.ctr,
                            (u32*)M);
    return cudaGetLastError();
}

}  // namespace appd
