// common.cuh -- device helpers shared by the APPD kernels (sm_103a).
//
// Order keys: a 32-bit key whose unsigned order is the weight order.  For
// uint32 weights the key is the value; for FP32 it is IEEE-754 totalOrder
// (non-negative: bits | 0x80000000, negative: ~bits).  The transform is a
// bijection, so outputs are recovered bit-exactly from keys.
//
// Packed edges: key << 32 | pair(lo, hi), lo < hi.  The 32-bit pair code is
// increasing in (lo, hi) taken lexicographically, so unsigned comparison of
// packed edges is the strict total order (key, lo, hi): it refines the weight
// order, which makes the MST unique and Boruvka's hooking cycle-free.  For
// n <= 65536 the code is lo << 16 | hi; above that it is the pair's index in
// the row-major upper triangle, lo * n - lo (lo + 1) / 2 + hi - lo - 1, which
// fits 32 bits while n (n - 1) / 2 <= 2^32, i.e. n <= MAX_N.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace appd {

using u64 = unsigned long long;
using u32 = unsigned int;

constexpr u64 EDGE_INF = ~0ull;
constexpr u32 NONE32 = 0xFFFFFFFFu;

// device status bits (per device, read by appd_last_device_status)
constexpr u32 DEV_TIMEOUT = 1u;
constexpr u32 DEV_INTERNAL = 2u;

// A bounded grid barrier gives up after this long (ns) and reports a timeout.
constexpr u64 BARRIER_TIMEOUT_NS = 2000000000ull;

// dtype codes: bit 0 = uint32 (else FP32), bit 1 = widest paths (the order
// is reversed by complementing the key, Section 4.2)
__host__ __device__ __forceinline__ u32 key_of(u32 bits, int dt)
{
    const u32 m = (u32)((int)bits >> 31) | 0x80000000u;
    const u32 k = (dt & 1) ? bits : (bits ^ m);
    return (dt & 2) ? ~k : k;
}

__host__ __device__ __forceinline__ u32 bits_of(u32 key, int dt)
{
    const u32 k = (dt & 2) ? ~key : key;
    return (dt & 1) ? k : (k ^ ((k >> 31) ? 0x80000000u : 0xFFFFFFFFu));
}

// a valid dtype code (APPD_F32, APPD_U32, either with the widest flag)
__host__ __device__ __forceinline__ bool dtype_ok(int dt) { return dt >= 0 && dt <= 3; }

// the largest n the packed edges support
constexpr u32 MAX_N = 92682;
// up to this n the pair code is lo << 16 | hi
constexpr u32 SHORT_N = 65536;

// tri index of (lo, hi) minus hi: lo * n - lo (lo + 1) / 2 - lo - 1, evaluated
// modulo 2^32 (the true value of the full index lies in [0, 2^32), so the
// wrapped terms cancel); lo (lo + 1) / 2 is formed without losing the bit a
// 32-bit product of lo and lo + 1 would drop
__host__ __device__ __forceinline__ u32 tri_row_base(u32 lo, u32 n)
{
    const u32 half = (lo & 1u) ? lo * ((lo + 1u) >> 1) : (lo >> 1) * (lo + 1u);
    return lo * n - half - lo - 1u;
}

// 32-bit code of the pair lo < hi of an n-vertex graph
__host__ __device__ __forceinline__ u32 pair_code(u32 lo, u32 hi, u32 n)
{
    return n <= SHORT_N ? ((lo << 16) | hi) : tri_row_base(lo, n) + hi;
}

__host__ __device__ __forceinline__ u64 pack_edge(u32 key, u32 a, u32 b, u32 n)
{
    const u32 lo = a < b ? a : b, hi = a < b ? b : a;
    return ((u64)key << 32) | pair_code(lo, hi, n);
}

// (lo, hi) from a pair code.  For the triangular code, lo is the largest l
// whose first pair l * n - l (l + 1) / 2 does not exceed the code: a root of
// that quadratic in double precision, corrected by at most a step or two.
__host__ __device__ __forceinline__ void pair_decode(u32 t, u32 n, u32* lo, u32* hi)
{
    if (n <= SHORT_N) {
        *lo = t >> 16;
        *hi = t & 0xFFFFu;
        return;
    }
    const double b = 2.0 * (double)n - 1.0;
    double disc = b * b - 8.0 * (double)t;
    if (disc < 0.0)
        disc = 0.0;
    long long l = (long long)((b - sqrt(disc)) * 0.5);
    if (l < 0)
        l = 0;
    if (l > (long long)n - 2)
        l = (long long)n - 2;
    auto first = [n](long long x) -> u64 { return (u64)x * n - (u64)x * (u64)(x + 1) / 2; };
    while (l > 0 && first(l) > t)
        --l;
    while (l + 1 <= (long long)n - 2 && first(l + 1) <= t)
        ++l;
    *lo = (u32)l;
    *hi = (u32)((u64)t - first(l) + (u64)l + 1);
}

__host__ __device__ __forceinline__ u32 edge_key(u64 e) { return (u32)(e >> 32); }
__host__ __device__ __forceinline__ void edge_ends(u64 e, u32 n, u32* lo, u32* hi)
{
    pair_decode((u32)e, n, lo, hi);
}

__device__ __forceinline__ int ceil_log2_dev(u32 x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

__device__ __forceinline__ u64 globaltimer_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u32 ld_acquire(const u32* p)
{
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// streaming 16-byte load that does not allocate in L1
__device__ __forceinline__ uint4 ld_stream_v4(const void* p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ u32 ld_stream_u32(const void* p)
{
    u32 v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ u64 warp_min_u64(u64 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        u64 w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// min over the block; every thread gets the result.  sh: >= 32 u64 of smem.
__device__ __forceinline__ u64 block_min_u64(u64 v, u64* sh)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_min_u64(v);
    __syncthreads();
    if (lane == 0)
        sh[w] = v;
    __syncthreads();
    u64 r = EDGE_INF;
    for (int i = 0; i < nw; ++i)
        r = sh[i] < r ? sh[i] : r;
    __syncthreads();
    return r;
}

// exclusive scan over the block of one u32 per thread; *total gets the sum.
// sh: >= 33 u32 of smem.
__device__ __forceinline__ u32 block_excl_scan(u32 v, u32* total, u32* sh)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o)
            x += y;
    }
    __syncthreads();
    if (lane == 31)
        sh[w] = x;
    __syncthreads();
    if (w == 0) {
        u32 s = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u32 y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o)
                s += y;
        }
        if (lane < nw)
            sh[lane] = s;
    }
    __syncthreads();
    u32 pre = (w ? sh[w - 1] : 0u) + x - v;
    if (total)
        *total = sh[nw - 1];
    __syncthreads();
    return pre;
}

// ------------------------------------------------------------ grid barrier
// Counting barrier for cooperative launches (all CTAs co-resident).  Thread 0
// of each CTA adds one to `count`; the k-th barrier of a launch completes when
// count reaches k * gridDim.x, so one atomic per CTA and a poll suffice (no
// reset, no generation word).  The wait is bounded: after BARRIER_TIMEOUT_NS a
// CTA records DEV_TIMEOUT, sets `abort` and returns false; callers then leave
// the kernel, and a CTA waiting at any later barrier of the launch sees
// `abort` and gives up at once.  count and abort must be zero when the kernel
// starts (the host clears them before each launch).
struct GridBar {
    u32 count;
    u32 abort;
    u32 failed;  // set when a wait of the current solve ran out or its state
                 // was found inconsistent; cleared at the start of each solve
                 // (the host's memset before a launch clears count + abort only)
};

// Records a failure of the current solve: in the device status word (read
// and cleared by the host) and in the solve's own flag, which the later
// phases of the same solve test before they follow any index derived from
// the spanning tree.
__device__ __forceinline__ void record_failure(u32* status, u32* failed, u32 code)
{
    if (status)
        atomicOr(status, code);
    if (failed)
        atomicExch(failed, 1u);
}

__device__ __forceinline__ bool solve_failed(const GridBar* bar)
{
    return *(const volatile u32*)&bar->failed != 0u;
}

__device__ __forceinline__ u32 atom_add_release(u32* p, u32 v)
{
    u32 old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ bool grid_sync(GridBar* bar, u32* status,
                                          u64 limit_ns = BARRIER_TIMEOUT_NS)
{
    __shared__ u32 s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 ok = 1;
        __threadfence();
        const u32 nb = gridDim.x;
        const u32 old = atom_add_release(&bar->count, 1u);
        const u32 target = (old / nb + 1) * nb;
        if ((int)(ld_acquire(&bar->count) - target) < 0) {
            const u64 t0 = globaltimer_ns();
            while ((int)(ld_acquire(&bar->count) - target) < 0) {
                if (ld_acquire(&bar->abort)) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicExch(&bar->abort, 1u);
                    record_failure(status, &bar->failed, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// A "team" is the set of threads that cooperates on one phase: the whole
// grid of a cooperative launch, or one CTA.  Phases are written once for both.
struct GridTeam {
    GridBar* bar;
    u32* status;
    __device__ __forceinline__ u32 rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ u32 size() const { return gridDim.x * blockDim.x; }
    __device__ __forceinline__ u32 block() const { return blockIdx.x; }
    __device__ __forceinline__ u32 nblocks() const { return gridDim.x; }
    __device__ __forceinline__ bool sync() const { return grid_sync(bar, status); }
};

struct BlockTeam {
    __device__ __forceinline__ u32 rank() const { return threadIdx.x; }
    __device__ __forceinline__ u32 size() const { return blockDim.x; }
    __device__ __forceinline__ u32 block() const { return 0; }
    __device__ __forceinline__ u32 nblocks() const { return 1; }
    __device__ __forceinline__ bool sync() const
    {
        __syncthreads();
        return true;
    }
};

// Exclusive scan of in[0..L) into out[0..L) by a team; returns the total to
// every thread.  part: >= nblocks()+1 u32 of global scratch (grid team).
// Costs two team syncs (the caller's next phase may read out[] directly).
template <class Team>
__device__ bool team_excl_scan(const Team& t, const u32* in, u32* out, u32 L, u32* part,
                               u32* total_out)
{
    __shared__ u32 sh_scan[40];
    const u32 nb = t.nblocks(), b = t.block(), bd = blockDim.x;
    const u32 chunk = (L + nb - 1) / nb;
    const u32 beg = min(L, b * chunk), end = min(L, beg + chunk);
    // phase 1: per-block sums
    u32 local = 0;
    for (u32 i = beg + threadIdx.x; i < end; i += bd)
        local += in[i];
    u32 bsum = 0;
    block_excl_scan(local, &bsum, sh_scan);
    if (nb > 1) {
        if (threadIdx.x == 0)
            part[b] = bsum;
        if (!t.sync())
            return false;
    }
    // phase 2: offset of this block, then a blocked scan of the chunk
    u32 off = 0, tot = 0;
    if (nb > 1) {
        for (u32 i = threadIdx.x; i < nb; i += bd) {
            u32 v = part[i];
            if (i < b)
                off += v;
            tot += v;
        }
        // reduce off and tot over the block
        u32 o2 = 0, t2 = 0;
        block_excl_scan(off, &o2, sh_scan);
        block_excl_scan(tot, &t2, sh_scan);
        off = o2;
        tot = t2;
    } else {
        tot = bsum;
    }
    u32 carry = off;
    for (u32 base = beg; base < end; base += bd) {
        u32 i = base + threadIdx.x;
        u32 v = i < end ? in[i] : 0u;
        u32 s = 0;
        u32 p = block_excl_scan(v, &s, sh_scan);
        if (i < end)
            out[i] = carry + p;
        carry += s;
    }
    *total_out = tot;
    return true;
}

}  // namespace appd
