// contract_tma.cu -- the level-0 contraction over the upper triangle of W,
// fed by bulk asynchronous copies (cp.async.bulk) into a shared-memory ring.
//
// It computes exactly what the upper-triangle form of k_contract computes
// (Section 5's contraction of the first Boruvka round, the work split of
// mst_kernels.cu): for every work item (group A, a chunk of at most
// CONTRACT_ROWS of its rows, one bin range) and every column j right of the
// item's smallest row, the smallest packed edge (key, row, j) over the
// item's rows left of j, folded into the bin of j's new component; the bins
// become row A of P and their minimum the row's candidate best edge.
//
// One CTA per SM with two roles:
//   * a producer warp claims items and, for every chunk of TC_CH columns and
//     every row of the item that reaches the chunk (rows ascending), issues
//     one bulk copy of that row's segment right of its diagonal into the
//     next free ring stage, completing on the stage's "full" mbarrier;
//   * TC_CONS consumer threads own TC_G interleaved 4-column groups of every
//     chunk, keep the running minimum of their columns over the chunk's rows
//     in registers and fold them into the bins once per chunk (the chunk's
//     16-bit labels are read from L2, requested before the last row's work),
//     then release the stage on its "empty" mbarrier.
// One row per stage keeps the stages full (a component's rows are spread
// over the matrix, so few of them reach the left part of a row range) and
// gives each consumer 12 columns per stage to amortize the stage's fixed
// work.  The ring holds rows only, so the bins leave room for 24 consumer
// warps (the consumers are latency-bound: more warps per SM, more speed).
// At the end of an item the consumers write the bins out and reset them
// while the producer already streams the next item.
//
// Every wait is bounded (BARRIER_TIMEOUT_NS): a wait that runs out sets the
// CTA's abort flag, records DEV_TIMEOUT for the solve, every role leaves its
// loop, and the producer waits (again bounded) for the copies it issued
// before the CTA exits.
#include "internal.h"
#include "mst_device.cuh"

#include <type_traits>

namespace appd {

namespace {

constexpr int TC_CONS_WARPS = 24;
constexpr u32 TC_CONS = TC_CONS_WARPS * 32;     // consumer threads
constexpr u32 TC_THREADS = TC_CONS + 32;        // plus one producer warp
constexpr u32 TC_G = 3;                         // 4-column groups per consumer and chunk
constexpr u32 TC_CH = 4 * TC_CONS * TC_G;       // columns per chunk
constexpr u32 TC_STAGES = 4;
constexpr u32 TC_ROW_BYTES = TC_CH * 4;
constexpr u32 TC_STAGE_BYTES = TC_ROW_BYTES;
constexpr u32 TC_RING_BYTES = TC_STAGES * TC_STAGE_BYTES;
static_assert(TC_STAGE_BYTES % 16 == 0, "stages start 16-byte aligned");

enum : u32 { TF_FIRST = 1, TF_LAST = 2, TF_END_ITEM = 4, TF_END = 8 };

// what the producer tells the consumers about one stage (three 16-byte words)
struct __align__(16) TcMeta {
    u32 c0, c1, row, flags;        // columns [c0, c1) of the chunk; the stage's row; TF_* bits
    u32 A, b0, nb, single;         // the item: group, bin range, one-chunk group
    u32 r0, pad0, pad1, pad2;      // the item's smallest row
};

__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64* bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(u64* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(u64* bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(u64* bar, u32 parity)
{
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) completing on bar's transaction count
__device__ __forceinline__ void bulk_load(void* dst, const void* src, u32 bytes, u64* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Bounded wait for the phase of the given parity.  Gives up when the CTA's
// abort flag is set (if honour_abort) or after BARRIER_TIMEOUT_NS, which sets
// the flag and records DEV_TIMEOUT for the solve.
__device__ __forceinline__ bool tc_wait(u64* bar, u32 parity, volatile u32* abort, u32* status,
                                        u32* failed, bool honour_abort = true)
{
    if (mbar_test(bar, parity))
        return true;
    const u64 t0 = globaltimer_ns();
    for (;;) {
        if (mbar_test(bar, parity))
            return true;
        if (honour_abort && *abort)
            return false;
        if (globaltimer_ns() - t0 > BARRIER_TIMEOUT_NS) {
            *abort = 1u;
            record_failure(status, failed, DEV_TIMEOUT);
            return false;
        }
    }
}

// 8-byte read-only load (four 16-bit labels)
__device__ __forceinline__ uint2 ld_nc_u2(const void* p)
{
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// first column group a row reaches: columns j with j + 3 > row, rounded to 4
__device__ __forceinline__ u32 first_group_col(u32 row) { return ((row + 1u) >> 2) << 2; }

}  // namespace

template <int DT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_contract_tma(ContractArgs a, u32 run_min, u32 run_max, u32* status, const u32* signs)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ TcMeta s_meta[TC_STAGES];
    __shared__ __align__(8) u64 s_full[TC_STAGES], s_empty[TC_STAGES], s_cbar;
    __shared__ u64 s_red[TC_CONS_WARPS];
    __shared__ u32 s_prow[CONTRACT_ROWS];
    __shared__ volatile u32 s_abort;

    Counters* ctr = a.ctr;
    if (*(volatile u32*)&ctr->done)
        return;
    const u32 cr = ((volatile u32*)ctr->c)[0];   // n: level 0 only
    const u32 cn = ((volatile u32*)ctr->c)[1];
    if (cn < run_min || cn > run_max)
        return;
    unsigned char* ring = smem;
    u64* bins = reinterpret_cast<u64*>(smem + TC_RING_BYTES);
    const u32 tid = threadIdx.x;
    if (cr <= a.comp_max_c)
        for (u32 v = blockIdx.x * blockDim.x + tid; v < a.n; v += gridDim.x * blockDim.x)
            a.comp[v] = a.label[a.comp[v]];
    if (tid == 0) {
        for (u32 s = 0; s < TC_STAGES; ++s) {
            mbar_init(&s_full[s], 1u);
            mbar_init(&s_empty[s], TC_CONS_WARPS);
        }
        mbar_init(&s_cbar, TC_CONS_WARPS);
        s_abort = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const u32 nb_all = min(cn, a.bin_cap);
    for (u32 b = tid; b < nb_all; b += blockDim.x)
        bins[b] = EDGE_INF;
    __syncthreads();

    const u32 total_chunks = *(volatile u32*)&ctr->total_chunks;
    const u32 nbr = (cn + a.bin_cap - 1) / a.bin_cap;
    const u32 total = total_chunks * nbr;
    const u32* W = (const u32*)a.cin;
    const u32 lane = tid & 31, warp = tid >> 5;
    u32* failed = &ctr->bar.failed;

    if (warp == TC_CONS_WARPS) {
        // ------------------------------------------------- producer warp
        // Lane q holds the item's row of rank q; lane 0 publishes every
        // stage and issues its copies.
        constexpr u32 FULL = 0xFFFFFFFFu;
        u32 it = 0;
        bool ok = true;
        // every lane waits for stage slot it % TC_STAGES to be free
        auto take_slot = [&](u32& slot) -> bool {
            slot = it % TC_STAGES;
            return __all_sync(FULL, tc_wait(&s_empty[slot], ((it / TC_STAGES) & 1u) ^ 1u, &s_abort, status, failed));
        };
        for (;;) {
            u32 item = 0;
            if (lane == 0)
                item = atomicAdd(&ctr->item_next, 1u);
            item = __shfl_sync(FULL, item, 0);
            if (item >= total)
                break;
            const u32 br = item / total_chunks, ch = item - br * total_chunks;
            const u32 A = a.item_group[ch];
            const u32 k = ch - a.chunk_start[A];
            const u32 m0 = a.gstart[A] + k * CONTRACT_ROWS;
            const u32 m1 = min(a.gstart[A + 1], m0 + CONTRACT_ROWS);
            const u32 nrows = m1 - m0;
            const u32 single = a.nchunk[A] == 1 ? 1u : 0u;
            const u32 b0 = br * a.bin_cap;
            const u32 nb = min(cn - b0, a.bin_cap);
            // rows ascending: each row's rank is the number of smaller rows
            // (the rows of a group are distinct vertices)
            const u32 v = lane < nrows ? a.members[m0 + lane] : NONE32;
            u32 rank = 0;
#pragma unroll
            for (int q = 0; q < CONTRACT_ROWS; ++q)
                rank += __shfl_sync(FULL, v, q) < v ? 1u : 0u;
            if (lane < nrows)
                s_prow[rank] = v;
            __syncwarp();
            const u32 myrow = lane < nrows ? s_prow[lane] : 0u;
            __syncwarp();
            const u32 mycol = first_group_col(myrow);
            const u32 r0 = __shfl_sync(FULL, myrow, 0);
            const u32 d0 = first_group_col(r0);
            // an item whose rows reach no column still writes its (empty) bins
            const u32 cstart = d0 < cr ? d0 : cr;
            for (u32 c0 = cstart;;) {
                const u32 c1 = min(cr, c0 + TC_CH);
                for (u32 q = 0;; ++q) {
                    // row q reaches this chunk (q == 0 always does)
                    const u32 row = __shfl_sync(FULL, myrow, q & 31u);
                    const u32 dq = __shfl_sync(FULL, mycol, q & 31u);
                    const u32 next_col = __shfl_sync(FULL, mycol, (q + 1) & 31u);
                    const bool more = q + 1 < nrows && next_col < c1;
                    const u32 flags = (q == 0 ? TF_FIRST : 0u) | (more ? 0u : TF_LAST) |
                                      (!more && c1 == cr ? TF_END_ITEM : 0u);
                    const u32 s0 = max(c0, dq);
                    const u32 rbytes = s0 < c1 ? (c1 - s0) * 4u : 0u;
                    u32 slot;
                    if (!(ok = take_slot(slot)))
                        break;
                    if (lane == 0) {
                        unsigned char* st = ring + slot * TC_STAGE_BYTES;
                        uint4* mw = reinterpret_cast<uint4*>(&s_meta[slot]);
                        mw[0] = make_uint4(c0, c1, row, flags);
                        mw[1] = make_uint4(A, b0, nb, single);
                        mw[2] = make_uint4(r0, 0u, 0u, 0u);
                        if (rbytes == 0) {
                            mbar_arrive(&s_full[slot]);
                        } else {
                            mbar_arrive_tx(&s_full[slot], rbytes);
                            bulk_load(st + (s0 - c0) * 4u, W + (size_t)row * cr + s0, rbytes, &s_full[slot]);
                        }
                    }
                    __syncwarp();
                    ++it;
                    if (!more)
                        break;
                }
                if (!ok || c1 >= cr)
                    break;
                c0 = c1;
            }
            if (!ok)
                break;
        }
        bool end_sent = false;
        if (ok) {
            u32 slot;
            if (take_slot(slot)) {
                if (lane == 0) {
                    s_meta[slot].flags = TF_END;
                    mbar_arrive(&s_full[slot]);
                }
                end_sent = true;
            }
        }
        if (lane != 0 || (end_sent && !s_abort))
            return;   // the consumers wait for every stage's copies themselves
        // the consumers left early: the copies of the stages issued last may
        // still be in flight; wait, bounded, until they have landed.  The end
        // marker reused the slot of stage it - TC_STAGES, whose copies had
        // landed before the slot was released.
        const u32 lo = end_sent ? (it + 1 > TC_STAGES ? it + 1 - TC_STAGES : 0u)
                                : (it > TC_STAGES ? it - TC_STAGES : 0u);
        for (u32 i = lo; i < it; ++i)
            tc_wait(&s_full[i % TC_STAGES], (i / TC_STAGES) & 1u, &s_abort, status, failed, false);
        return;
    }

    // ----------------------------------------------------------- consumers
    // FP32 weights with no sign bit anywhere in the upper triangle (round 1
    // checked every element this pass reads right of a row's diagonal)
    // compare as raw bits, the unsigned order of their keys (CDT = DT | 1:
    // the identity, complemented for the widest path); a column minimum is
    // turned into its key once, at the fold.  Columns left of the item's
    // smallest row may hold other values, but they never reach a bin.
    const bool raw = (DT & 1) == 0 && signs != nullptr && *(volatile u32*)signs == 0u;
    // SH: n <= SHORT_N, the pair code is lo << 16 | hi (decided once per CTA)
    auto consumers = [&](auto cdt_tag, auto short_tag) {
    constexpr int CDT = decltype(cdt_tag)::value;
    constexpr bool SH = decltype(short_tag)::value;
    // key of DT from a minimum compared under CDT
    auto fix = [](u32 k) -> u32 {
        if constexpr (CDT == DT)
            return k;
        else if constexpr (DT == 0)
            return k | 0x80000000u;
        else
            return k & 0x7FFFFFFFu;
    };
    // group t of this thread: columns c0 + 4 * ctid + 4 * TC_CONS * t .. +3
    // (interleaved, so a warp's 16-byte shared loads are contiguous)
    const u32 ctid = tid;   // 0 .. TC_CONS-1
    u32 it = 0, cph = 0;
    u32 bk[4 * TC_G], bi[4 * TC_G];
#pragma unroll
    for (u32 i = 0; i < 4 * TC_G; ++i)
        bk[i] = bi[i] = 0u;
    // all consumer warps meet (bounded); false once any wait ran out
    auto cons_sync = [&]() -> bool {
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&s_cbar);
        const bool okw = tc_wait(&s_cbar, cph, &s_abort, status, failed);
        cph ^= 1u;
        return __all_sync(0xFFFFFFFFu, okw);
    };
    for (;;) {
        const u32 slot = it % TC_STAGES;
        if (!__all_sync(0xFFFFFFFFu, tc_wait(&s_full[slot], (it / TC_STAGES) & 1u, &s_abort, status, failed)))
            break;
        const uint4* mr = reinterpret_cast<const uint4*>(&s_meta[slot]);
        const uint4 w0 = mr[0];
        const u32 flags = w0.w;
        if (flags & TF_END)
            break;
        // the item's fields are read only at a chunk's last row (the fold and
        // the item's end)
        uint4 w1 = make_uint4(0u, 0u, 0u, 0u), w2 = w1;
        if (flags & TF_LAST) {
            w1 = mr[1];
            w2 = mr[2];
        }
        const u32 c0 = w0.x, c1 = w0.y, row = w0.z;
        const u32 A = w1.x, b0 = w1.y, nb = w1.z, single = w1.w, r0 = w2.x;
        const unsigned char* st = ring + slot * TC_STAGE_BYTES;
        const uint4* rows = reinterpret_cast<const uint4*>(st);
        // the chunk's labels at its last row, requested before the row work
        // so that their latency overlaps it
        uint2 labg[TC_G];
#pragma unroll
        for (u32 t = 0; t < TC_G; ++t) {
            const u32 j = c0 + 4u * (ctid + TC_CONS * t);
            labg[t] = ((flags & TF_LAST) && j < c1) ? ld_nc_u2(a.label16 + j) : make_uint2(0u, 0u);
        }
        // all groups' 16 bytes at once; groups left of the row's segment
        // hold stale data and are not used
        uint4 v[TC_G];
#pragma unroll
        for (u32 t = 0; t < TC_G; ++t)
            v[t] = rows[ctid + TC_CONS * t];
        const bool first = (flags & TF_FIRST) != 0;
        const u32 jf = c0 + 4u * ctid, jl = jf + 4u * TC_CONS * (TC_G - 1);
        if (!first && jf > row && jl < c1) {
            // every group of this thread lies right of the row's diagonal
#pragma unroll
            for (u32 t = 0; t < TC_G; ++t)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const u32 kk = key_of(lane_of_dyn(v[t], c), CDT);
                    if (kk < bk[4 * t + c]) {
                        bk[4 * t + c] = kk;
                        bi[4 * t + c] = row;
                    }
                }
        } else
#pragma unroll
        for (u32 t = 0; t < TC_G; ++t) {
            const u32 j = c0 + 4u * (ctid + TC_CONS * t);
            if (j >= c1)
                continue;
            if (first) {
                // the item's smallest row reaches every group of the chunk
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    bk[4 * t + c] = key_of(lane_of_dyn(v[t], c), CDT);
                    bi[4 * t + c] = row;
                }
            } else if (j > row) {
                // all four columns right of the row's diagonal
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const u32 kk = key_of(lane_of_dyn(v[t], c), CDT);
                    if (kk < bk[4 * t + c]) {
                        bk[4 * t + c] = kk;
                        bi[4 * t + c] = row;
                    }
                }
            } else if (j + 3u > row) {
                // the group that holds the row's diagonal
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const u32 kk = key_of(lane_of_dyn(v[t], c), CDT);
                    if (j + (u32)c > row && kk < bk[4 * t + c]) {
                        bk[4 * t + c] = kk;
                        bi[4 * t + c] = row;
                    }
                }
            }
        }
        if (flags & TF_LAST) {
            // fold the chunk's column minima into the bins

#pragma unroll
            for (u32 t = 0; t < TC_G; ++t) {
                const u32 j = c0 + 4u * (ctid + TC_CONS * t);
                if (j >= c1)
                    continue;
                const uint2 lab = labg[t];
                const u32 L[4] = {lab.x & 0xFFFFu, lab.x >> 16, lab.y & 0xFFFFu, lab.y >> 16};
                // columns j + c >= cmin lie right of the item's smallest row
                const u32 cmin = j > r0 ? 0u : r0 + 1u - j;
                u64 e[4];
                u32 rel[4];
                bool okc[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    rel[c] = L[c] - b0;
                    okc[c] = (L[c] != A) && (rel[c] < nb) && ((u32)c >= cmin);
                    const u32 code = SH ? ((bi[4 * t + c] << 16) | (j + (u32)c))
                                       : pair_code(bi[4 * t + c], j + (u32)c, cr);
                    e[c] = ((u64)fix(bk[4 * t + c]) << 32) | code;
                }
                u64 cur[4];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    cur[c] = okc[c] ? bins[rel[c]] : 0ull;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (okc[c] && e[c] < cur[c])
                        atomicMin(&bins[rel[c]], e[c]);
            }
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&s_empty[slot]);
        ++it;
        if (flags & TF_END_ITEM) {
            // row A of P (this bin range) and its minimum; the bins are
            // reset for the next item on the way
            if (!cons_sync())
                break;
            u64 mn = EDGE_INF;
            u64* dst = a.cout + (size_t)A * cn + b0;
            for (u32 b = ctid; b < nb; b += TC_CONS) {
                const u64 x = bins[b];
                bins[b] = EDGE_INF;
                if (single)
                    dst[b] = x;
                else if (x != EDGE_INF)
                    atomicMin(dst + b, x);
                mn = x < mn ? x : mn;
            }
            mn = warp_min_u64(mn);
            if (lane == 0)
                s_red[warp] = mn;
            if (!cons_sync())
                break;
            if (ctid == 0) {
                u64 r = EDGE_INF;
                for (int w = 0; w < TC_CONS_WARPS; ++w)
                    r = s_red[w] < r ? s_red[w] : r;
                if (r != EDGE_INF)
                    atomicMin(&a.best_out[A], r);
            }
        }
    }
    };
    using sh_yes = std::true_type;
    using sh_no = std::false_type;
    const bool sh = cr <= SHORT_N;
    if (raw) {
        if (sh)
            consumers(std::integral_constant<int, DT | 1>{}, sh_yes{});
        else
            consumers(std::integral_constant<int, DT | 1>{}, sh_no{});
    } else {
        if (sh)
            consumers(std::integral_constant<int, DT>{}, sh_yes{});
        else
            consumers(std::integral_constant<int, DT>{}, sh_no{});
    }
}

cudaError_t preload_contract_tma()
{
    return touch_kernels(k_contract_tma<0>, k_contract_tma<1>, k_contract_tma<2>, k_contract_tma<3>);
}

u32 contract_tma_bin_cap(int smem_optin)
{
    const long cap = ((long)smem_optin - (long)TC_RING_BYTES - 1024) / 8;
    return cap > 0 ? (u32)cap : 0u;
}

cudaError_t launch_contract0_tma(const ContractArgs& ca, int dt, int blocks, u32 run_max, u32* status,
                                 const u32* signs, cudaStream_t s)
{
    const size_t smem = TC_RING_BYTES + (size_t)ca.bin_cap * sizeof(u64);
    auto k = dt == 0 ? k_contract_tma<0> : dt == 1 ? k_contract_tma<1> : dt == 2 ? k_contract_tma<2>
                                                                             : k_contract_tma<3>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return err;
    k<<<blocks, TC_THREADS, smem, s>>>(ca, 0u, run_max, status, signs);
    return cudaGetLastError();
}

}  // namespace appd
