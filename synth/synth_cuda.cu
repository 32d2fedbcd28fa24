// synth/synth_cuda.cu -- device twin of synth.c (input generation only).
//
// Same definitions as synth.c, evaluated with explicitly rounded FP64
// intrinsics so that no multiply-add is fused (__dsub_rn, __dmul_rn,
// __dadd_rn, __dsqrt_rn are each correctly rounded), then rounded to FP32
// with __double2float_rn.  The result is bit-identical to the host generator.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t hash3(uint64_t seed, uint64_t lo, uint64_t hi)
{
    return mix64(mix64(seed) ^ ((lo << 32) | hi));
}

__global__ void euclid_kernel(const float* __restrict__ pts, int64_t n, int d, float* __restrict__ W)
{
    int64_t total = n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / n, j = idx - i * n;
        if (i == j) {
            W[idx] = 0.0f;
            continue;
        }
        int64_t lo = i < j ? i : j, hi = i < j ? j : i;
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = __dsub_rn((double)pts[lo * d + k], (double)pts[hi * d + k]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        W[idx] = __double2float_rn(__dsqrt_rn(s));
    }
}

__global__ void hash_kernel(uint64_t seed, int64_t n, uint32_t* __restrict__ W, int kind)
{
    int64_t total = n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / n, j = idx - i * n;
        if (i == j) {
            W[idx] = 0u;
            continue;
        }
        uint64_t lo = (uint64_t)(i < j ? i : j), hi = (uint64_t)(i < j ? j : i);
        uint64_t h = hash3(seed, lo, hi);
        if (kind == 1) {
            W[idx] = (uint32_t)(h & 0xFFFFu);
        } else {
            double v = __dmul_rn(__dadd_rn((double)(h >> 40), 0.5), 1.0 / 16777216.0);
            W[idx] = __float_as_uint(__double2float_rn(v));
        }
    }
}

// FP32-arithmetic Euclidean distance (the serving mix's point requests):
// fixed order, one rounding per step, correctly rounded square root
__device__ __forceinline__ float euclid32_pair(const float* __restrict__ pts, int d, int64_t lo, int64_t hi)
{
    float s = 0.0f;
    for (int k = 0; k < d; ++k) {
        const float t = __fsub_rn(pts[lo * d + k], pts[hi * d + k]);
        s = __fmaf_rn(t, t, s);
    }
    return __fsqrt_rn(s);
}

__global__ void euclid32_kernel(const float* __restrict__ pts, int64_t n, int d, float* __restrict__ W)
{
    int64_t total = n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / n, j = idx - i * n;
        W[idx] = (i == j) ? 0.0f : euclid32_pair(pts, d, i < j ? i : j, i < j ? j : i);
    }
}

// One serving request's input: W of an n-vertex graph written into its slot.
// kind 0: FP32-arithmetic Euclidean distances of the n x d points at pts;
// kind 1: hashed uint32 weights h(seed, lo, hi) & 0xFFFF.  tile0: the first
// of the request's ceil(n^2 / REQ_TILE) tiles in the launch.
struct ReqDesc {
    uint64_t slot;
    uint64_t pts;
    uint64_t tile0;
    uint64_t seed;
    uint32_t n;
    uint32_t kind;
    uint32_t d;
    uint32_t pad;
};
constexpr int REQ_TILE = 1024;

__global__ void __launch_bounds__(256) requests_kernel(const ReqDesc* __restrict__ desc, int count)
{
    __shared__ int s_r;
    const uint64_t tile = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = count - 1;   // last request with tile0 <= tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (desc[mid].tile0 <= tile)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_r = lo;
    }
    __syncthreads();
    const ReqDesc r = desc[s_r];
    const int64_t n = r.n, total = n * n;
    const int64_t base = (int64_t)(tile - r.tile0) * REQ_TILE;
    for (int q = threadIdx.x; q < REQ_TILE; q += blockDim.x) {
        const int64_t idx = base + q;
        if (idx >= total)
            break;
        const int64_t i = idx / n, j = idx - i * n;
        const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
        if (r.kind == 0) {
            float* W = reinterpret_cast<float*>(r.slot);
            W[idx] = (i == j) ? 0.0f : euclid32_pair(reinterpret_cast<const float*>(r.pts), (int)r.d, lo, hi);
        } else {
            uint32_t* W = reinterpret_cast<uint32_t*>(r.slot);
            W[idx] = (i == j) ? 0u : (uint32_t)(hash3(r.seed, (uint64_t)lo, (uint64_t)hi) & 0xFFFFu);
        }
    }
}

int grid_for(int64_t total)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (total + 255) / 256;
    int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 32;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

extern "C" int synth_cuda_euclid_f32(const float* pts, int64_t n, int d, float* W, cudaStream_t s)
{
    if (n <= 0)
        return 0;
    euclid_kernel<<<grid_for(n * n), 256, 0, s>>>(pts, n, d, W);
    return (int)cudaGetLastError();
}

extern "C" int synth_cuda_hash_u32(uint64_t seed, int64_t n, uint32_t* W, cudaStream_t s)
{
    if (n <= 0)
        return 0;
    hash_kernel<<<grid_for(n * n), 256, 0, s>>>(seed, n, W, 1);
    return (int)cudaGetLastError();
}

extern "C" int synth_cuda_uniform01_f32(uint64_t seed, int64_t n, float* W, cudaStream_t s)
{
    if (n <= 0)
        return 0;
    hash_kernel<<<grid_for(n * n), 256, 0, s>>>(seed, n, reinterpret_cast<uint32_t*>(W), 2);
    return (int)cudaGetLastError();
}

extern "C" int synth_cuda_euclid32_f32(const float* pts, int64_t n, int d, float* W, cudaStream_t s)
{
    if (n <= 0)
        return 0;
    euclid32_kernel<<<grid_for(n * n), 256, 0, s>>>(pts, n, d, W);
    return (int)cudaGetLastError();
}

// count request descriptors (device memory, 48 bytes each, tile0 ascending)
// covering total_tiles tiles of 1024 entries: one launch writes every
// request's W into its slot.
extern "C" int synth_cuda_requests(const void* desc_dev, int count, int64_t total_tiles, cudaStream_t s)
{
    if (count <= 0 || total_tiles <= 0)
        return 0;
    requests_kernel<<<(unsigned)total_tiles, 256, 0, s>>>(reinterpret_cast<const ReqDesc*>(desc_dev), count);
    return (int)cudaGetLastError();
}
