// insert.cu -- warm start (Section 6.1): the matrix of G + p from G's.
//
// Given M, the solved n x n matrix of a graph G, and the weights w(k) of a
// new vertex p's edges, the matrix of G + p follows without a new tree.  A
// path from i to p ends with one edge k-p, so p's distance to i is
//     d(i) = min over k of max(M(i,k), w(k)),
// where M(i,i) stands for the empty path (the k = i term is w(i)).  A path
// between old vertices either avoids p (best: M(i,j)) or passes through p
// once (best: max(d(i), d(j))), so
//     M'(i,j) = min(M(i,j), max(d(i), d(j))),   M'(i,p) = M'(p,i) = d(i),
// with p as index n and an all-zero diagonal.  Comparisons use the order key
// of the dtype (reversed for the widest dtypes); cells keep the selected
// weight's bits.  Two streaming passes over M: column minima give d (M is
// symmetric), then every row of M' is written.
#include "internal.h"

namespace appd {
namespace {

constexpr int INS_THREADS = 256;

// d as order keys, column by column: M is symmetric, so d(j) = min over
// rows k != j of max(M(k,j), w(k)) (and w(j) for k = j).  A CTA takes a
// block of INS_ROWS rows and INS_COLS columns; a thread owns four columns,
// keeps their minima over the block's rows in registers (w(k) is one value
// per row), and folds them into dkey[] with atomic minima.  dkey starts at
// the keys of w (k_ins_init).
constexpr u32 INS_ROWS = 128, INS_COLS = 4 * INS_THREADS;

template <int DT>
__global__ void k_ins_init(const u32* __restrict__ w, u32 n, u32* __restrict__ dkey)
{
    for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        dkey[j] = key_of(w[j], DT);
}

template <int DT, bool VEC>
__global__ void __launch_bounds__(INS_THREADS) k_ins_dist(const u32* __restrict__ M, const u32* __restrict__ w,
                                                          u32 n, u32* __restrict__ dkey)
{
    const u32 c0 = blockIdx.x * INS_COLS, r0 = blockIdx.y * INS_ROWS;
    const u32 r1 = min(n, r0 + INS_ROWS);
    const u32 j = c0 + 4 * threadIdx.x;       // this thread's first column
    u32 mk[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    if (VEC) {
        if (j < n) {
            for (u32 k0 = r0; k0 < r1; k0 += 4) {
                uint4 v[4];
                u32 kw[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const u32 k = k0 + q;
                    v[q] = k < r1 ? ld_stream_v4(M + (size_t)k * n + j) : make_uint4(0u, 0u, 0u, 0u);
                    kw[q] = k < r1 ? key_of(__ldg(w + k), DT) : 0xFFFFFFFFu;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const u32 k = k0 + q;
                    if (k >= r1)
                        continue;
                    const u32 x[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const u32 km = key_of(x[c], DT);
                        const u32 t = km > kw[q] ? km : kw[q];
                        if (k != j + c && t < mk[c])
                            mk[c] = t;
                    }
                }
            }
        }
    } else {
        for (u32 k = r0; k < r1; ++k) {
            const u32 kw = key_of(__ldg(w + k), DT);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const u32 jj = c0 + threadIdx.x + c * INS_THREADS;   // coalesced columns
                if (jj < n && jj != k) {
                    const u32 km = key_of(ld_stream_u32(M + (size_t)k * n + jj), DT);
                    const u32 t = km > kw ? km : kw;
                    if (t < mk[c])
                        mk[c] = t;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const u32 jj = VEC ? j + c : c0 + threadIdx.x + c * INS_THREADS;
        if (jj < n && mk[c] != 0xFFFFFFFFu)
            atomicMin(dkey + jj, mk[c]);
    }
}

// Rows of M' (n + 1 wide): one CTA per row (grid-stride).  Warps access
// consecutive words (rows of M' start at any 4-byte boundary), each thread
// with four columns in flight, blockDim apart.
template <int DT>
__global__ void __launch_bounds__(INS_THREADS) k_ins_fill(const u32* __restrict__ M, const u32* __restrict__ dkey,
                                                          u32 n, u32* __restrict__ Mo)
{
    constexpr int U = 4;
    const u32 m = n + 1;
    for (u32 i = blockIdx.x; i <= n; i += gridDim.x) {
        u32* out = Mo + (size_t)i * m;
        if (i == n) {
            for (u32 j = threadIdx.x; j < n; j += blockDim.x)
                __stcs(out + j, bits_of(__ldg(dkey + j), DT));
            if (threadIdx.x == 0)
                __stcs(out + n, 0u);
            continue;
        }
        const u32* row = M + (size_t)i * n;
        const u32 ki = dkey[i], di = bits_of(ki, DT);
        for (u32 j0 = threadIdx.x; j0 < n; j0 += U * blockDim.x) {
            u32 mv[U], dv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const u32 j = j0 + u * blockDim.x;
                mv[u] = j < n ? ld_stream_u32(row + j) : 0u;
                dv[u] = j < n ? __ldg(dkey + j) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const u32 j = j0 + u * blockDim.x;
                if (j < n) {
                    const u32 kv = ki > dv[u] ? ki : dv[u];
                    __stcs(out + j, (j == i) ? 0u : (key_of(mv[u], DT) <= kv ? mv[u] : bits_of(kv, DT)));
                }
            }
        }
        if (threadIdx.x == 0)
            __stcs(out + n, di);
    }
}

template <int DT>
cudaError_t launch_insert(const u32* M, u32 n, const u32* w, u32* Mo, u32* dkey, int sms, cudaStream_t s)
{
    k_ins_init<DT><<<sms * 2, INS_THREADS, 0, s>>>(w, n, dkey);
    const dim3 grid((n + INS_COLS - 1) / INS_COLS, (n + INS_ROWS - 1) / INS_ROWS);
    if (n % 4 == 0 && ((uintptr_t)M & 15u) == 0)
        k_ins_dist<DT, true><<<grid, INS_THREADS, 0, s>>>(M, w, n, dkey);
    else
        k_ins_dist<DT, false><<<grid, INS_THREADS, 0, s>>>(M, w, n, dkey);
    k_ins_fill<DT><<<sms * 8, INS_THREADS, 0, s>>>(M, dkey, n, Mo);
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_insert(const void* M, int64_t n, int dt, const void* w, void* Mo, u32* d, int sms,
                       cudaStream_t s)
{
    if (n == 0)
        return cudaMemsetAsync(Mo, 0, sizeof(u32), s);
    prof_launches(3);
    switch (dt) {
    case 1: return launch_insert<1>((const u32*)M, (u32)n, (const u32*)w, (u32*)Mo, d, sms, s);
    case 2: return launch_insert<2>((const u32*)M, (u32)n, (const u32*)w, (u32*)Mo, d, sms, s);
    case 3: return launch_insert<3>((const u32*)M, (u32)n, (const u32*)w, (u32*)Mo, d, sms, s);
    default: return launch_insert<0>((const u32*)M, (u32)n, (const u32*)w, (u32*)Mo, d, sms, s);
    }
}

}  // namespace appd
