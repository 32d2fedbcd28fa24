// tune.cu -- autotuner of the batched path.
//
// The batched path has three shape parameters that depend on the GPU: the
// rows per fill batch inside a CTA (shared memory per CTA vs. the number of
// row batches per column block), the size cut-over between one-CTA-per-graph
// solving and the multi-CTA pipeline, and the largest graph one warp solves
// by Prim.  appd_batched_autotune times every (fill rows, cut-over) pair, then
// every warp limit with the best pair, on a seeded synthetic batch (graph sizes
// log-uniform in [32, 4096], uniform(0,1) weights written by a hash kernel
// below), keeps the fastest, installs it for this process, and caches it in a
// small JSON file keyed by the GPU name and driver version so later processes
// skip the search.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/appd.h"
#include "internal.h"

namespace appd {
namespace {

__device__ __forceinline__ uint64_t tune_mix(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// symmetric uniform(0,1) weights with zero diagonal (tuning data only)
__global__ void k_tune_fill(float* W, u32 n, uint64_t seed)
{
    const uint64_t total = (uint64_t)n * n;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const u32 i = (u32)(idx / n), j = (u32)(idx - (uint64_t)i * n);
        if (i == j) {
            W[idx] = 0.0f;
            continue;
        }
        const uint64_t lo = i < j ? i : j, hi = i < j ? j : i;
        const uint64_t h = tune_mix(tune_mix(seed) ^ ((lo << 32) | hi));
        W[idx] = (float)(((double)(h >> 40) + 0.5) * (1.0 / 16777216.0));
    }
}

// "<GPU name> / driver <version>"; false when no device answers
bool cache_key(std::string* key)
{
    int dev = 0, drv = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess ||
        cudaDriverGetVersion(&drv) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::string name(p.name);
    for (char& c : name)
        if (c == '"' || c == '\\')
            c = '_';
    *key = name + " / driver " + std::to_string(drv);
    return true;
}

// The cache file holds one line per key:
//   {"key": "...", "fill_rows": R, "n_split": S, "prim_max": P}
bool cache_lookup(const char* path, const std::string& key, BatchTuning* out)
{
    FILE* f = fopen(path, "r");
    if (!f)
        return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        const std::string l(line);
        if (l.find("\"key\": \"" + key + "\"") == std::string::npos)
            continue;
        int fr = 0;
        long long ns = 0;
        const size_t a = l.find("\"fill_rows\": "), b = l.find("\"n_split\": ");
        if (a == std::string::npos || b == std::string::npos)
            continue;
        const size_t c = l.find("\"prim_max\": ");
        int pm = 0;
        if (c == std::string::npos || sscanf(l.c_str() + c + 12, "%d", &pm) != 1)
            continue;   // an entry written before the warp limit was searched
        if (sscanf(l.c_str() + a + 13, "%d", &fr) == 1 && sscanf(l.c_str() + b + 11, "%lld", &ns) == 1) {
            out->fill_rows = fr;
            out->n_split = ns;
            out->ctas_per_sm = 1;
            out->prim_max = (u32)pm;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, const BatchTuning& t, double ms)
{
    FILE* f = fopen(path, "a");
    if (!f)
        return;
    fprintf(f, "{\"key\": \"%s\", \"fill_rows\": %d, \"n_split\": %lld, \"prim_max\": %u, \"ms\": %.4f}\n",
            key.c_str(), t.fill_rows, (long long)t.n_split, t.prim_max, ms);
    fclose(f);
}

}  // namespace
}  // namespace appd

using namespace appd;

extern "C" appd_status appd_batched_autotune(const char* cache_path, appd_stream_t s)
{
    std::string key;
    if (!cache_key(&key))
        return APPD_ERR_CUDA;
    BatchTuning best;
    if (cache_path && cache_lookup(cache_path, key, &best)) {
        appd_status st = appd_batched_tuning(best.ctas_per_sm, best.fill_rows, best.n_split);
        return st == APPD_OK ? appd_batched_prim_max((int32_t)best.prim_max) : st;
    }
    cudaStream_t cs = (cudaStream_t)s;
    // synthetic batch: 192 graphs, n = floor(32 * 128^u), u from a fixed sequence
    const int G = 192;
    std::vector<int64_t> ns(G), offs(G);
    int64_t total = 0;
    uint64_t state = 0x5eed;
    for (int g = 0; g < G; ++g) {
        state = state * 6364136223846793005ull + 1442695040888963407ull;
        const double u = (double)(state >> 11) / 9007199254740992.0;
        int64_t n = (int64_t)(32.0 * pow(128.0, u));
        n = n < 32 ? 32 : (n > 4096 ? 4096 : n);
        ns[g] = n;
        offs[g] = total;
        total += n * n;
    }
    void *W = nullptr, *M = nullptr;
    if (cudaMalloc(&W, (size_t)total * 4) != cudaSuccess)
        return APPD_ERR_NOMEM;
    if (cudaMalloc(&M, (size_t)total * 4) != cudaSuccess) {
        cudaFree(W);
        return APPD_ERR_NOMEM;
    }
    for (int g = 0; g < G; ++g)
        k_tune_fill<<<256, 256, 0, cs>>>((float*)W + offs[g], (u32)ns[g], 7000 + g);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int rows[] = {256, 512, 1024, 2048};
    const int64_t splits[] = {512, 1024, 2048, 4096};
    const int prims[] = {0, 64, 128, 256, 512};
    double best_ms = 1e30;
    appd_status st = APPD_OK;
    // times the current parameters: a warm-up call (builds the runtime and
    // the captured launch), then one timed call
    auto time_batch = [&](float* ms) -> appd_status {
        appd_status r = appd_solve_batched(offs.data(), W, ns.data(), nullptr, M, G, s);
        if (r != APPD_OK)
            return r;
        cudaEventRecord(e0, cs);
        r = appd_solve_batched(offs.data(), W, ns.data(), nullptr, M, G, s);
        cudaEventRecord(e1, cs);
        if (r != APPD_OK || cudaEventSynchronize(e1) != cudaSuccess)
            return r != APPD_OK ? r : APPD_ERR_CUDA;
        cudaEventElapsedTime(ms, e0, e1);
        return APPD_OK;
    };
    best.prim_max = current_batch_tuning().prim_max;
    for (int r : rows) {
        for (int64_t sp : splits) {
            float ms = 0.f;
            if ((st = appd_batched_tuning(1, r, sp)) != APPD_OK || (st = time_batch(&ms)) != APPD_OK)
                break;
            if (ms < best_ms) {
                best_ms = ms;
                best.ctas_per_sm = 1;
                best.fill_rows = r;
                best.n_split = sp;
            }
        }
        if (st != APPD_OK)
            break;
    }
    if (st == APPD_OK && (st = appd_batched_tuning(1, best.fill_rows, best.n_split)) == APPD_OK) {
        for (int pm : prims) {
            float ms = 0.f;
            if ((st = appd_batched_prim_max(pm)) != APPD_OK || (st = time_batch(&ms)) != APPD_OK)
                break;
            if (ms < best_ms) {
                best_ms = ms;
                best.prim_max = (u32)pm;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(cs);
    cudaFree(W);
    cudaFree(M);
    if (st != APPD_OK)
        return st;
    if (cache_path)
        cache_store(cache_path, key, best, best_ms);
    st = appd_batched_tuning(best.ctas_per_sm, best.fill_rows, best.n_split);
    return st == APPD_OK ? appd_batched_prim_max((int32_t)best.prim_max) : st;
}

extern "C" appd_status appd_batched_get_tuning(int32_t* ctas_per_sm, int32_t* fill_rows, int64_t* n_split)
{
    if (!ctas_per_sm || !fill_rows || !n_split)
        return APPD_ERR_INVALID;
    BatchTuning t = current_batch_tuning();
    *ctas_per_sm = t.ctas_per_sm;
    *fill_rows = t.fill_rows;
    *n_split = t.n_split;
    return APPD_OK;
}
