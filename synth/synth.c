/*
 * synth/synth.c -- seeded synthetic inputs (host side).
 *
 * Input generation only: nothing here computes minimax distances.  Both the
 * CUDA library's tests/benchmarks and the CPU oracle take their weight
 * matrices from this module (or from its device twin synth_cuda.cu, which
 * follows the same definitions bit for bit).
 *
 * Definitions
 *  - Euclidean FP32 weights: d(i,j) = sqrt(sum_k (x_ik - x_jk)^2), evaluated in
 *    FP64 in ascending k, each subtraction, square and sum rounded separately
 *    (no fused multiply-add), a correctly rounded square root, then rounded to
 *    FP32.  Only i<j is computed; (j,i) is a copy; the diagonal is +0.0.
 *  - FP32-arithmetic Euclidean weights (the serving mix's point requests):
 *    s = 0, then for k ascending t = x_lo,k - x_hi,k and s = fma(t, t, s),
 *    every step rounded to FP32, and d = sqrt(s) correctly rounded in FP32.
 *  - Hashed weights: h(seed,lo,hi) = mix(mix(seed) ^ (lo<<32 | hi)), where mix
 *    is the SplitMix64 finaliser (Steele, Lea, Flood 2014).  uint32 weights
 *    are h & 0xFFFF; uniform(0,1) FP32 weights are ((h>>40)+0.5)*2^-24
 *    rounded to FP32 from FP64.  Diagonal 0.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

uint64_t synth_mix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

uint64_t synth_hash(uint64_t seed, uint64_t lo, uint64_t hi)
{
    return synth_mix64(synth_mix64(seed) ^ ((lo << 32) | hi));
}

static float euclid_pair(const float *pts, int d, int64_t i, int64_t j)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double a = (double)pts[i * d + k];
        double b = (double)pts[j * d + k];
        double t = a - b;
        double q = t * t;
        s = s + q;
    }
    return (float)sqrt(s);
}

static float euclid32_pair(const float *pts, int d, int64_t i, int64_t j)
{
    float s = 0.0f;
    for (int k = 0; k < d; ++k) {
        const float t = pts[i * d + k] - pts[j * d + k];
        s = fmaf(t, t, s);
    }
    return sqrtf(s);
}

typedef struct {
    const float *pts;
    int64_t n;
    int d;
    float *W;
    int64_t r0, r1;
    int kind;       /* 0 euclid, 1 hash-u32, 2 uniform01, 3 euclid in FP32 arithmetic */
    uint64_t seed;
} job;

static void fill_rows(const job *jb)
{
    int64_t n = jb->n;
    for (int64_t i = jb->r0; i < jb->r1; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (i == j) {
                if (jb->kind == 1)
                    ((uint32_t *)jb->W)[i * n + j] = 0u;
                else
                    jb->W[i * n + j] = 0.0f;
                continue;
            }
            int64_t lo = i < j ? i : j, hi = i < j ? j : i;
            if (jb->kind == 0) {
                jb->W[i * n + j] = euclid_pair(jb->pts, jb->d, lo, hi);
            } else if (jb->kind == 3) {
                jb->W[i * n + j] = euclid32_pair(jb->pts, jb->d, lo, hi);
            } else {
                uint64_t h = synth_hash(jb->seed, (uint64_t)lo, (uint64_t)hi);
                if (jb->kind == 1)
                    ((uint32_t *)jb->W)[i * n + j] = (uint32_t)(h & 0xFFFFu);
                else
                    jb->W[i * n + j] = (float)(((double)(h >> 40) + 0.5) * (1.0 / 16777216.0));
            }
        }
    }
}

static void *thread_main(void *p)
{
    fill_rows((const job *)p);
    return NULL;
}

static int run(const float *pts, int64_t n, int d, float *W, int kind, uint64_t seed, int nthreads)
{
    if (n <= 0)
        return 0;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    if (nthreads > n)
        nthreads = (int)n;
    pthread_t th[256];
    job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].pts = pts;
        jobs[t].n = n;
        jobs[t].d = d;
        jobs[t].W = W;
        jobs[t].r0 = n * t / nthreads;
        jobs[t].r1 = n * (t + 1) / nthreads;
        jobs[t].kind = kind;
        jobs[t].seed = seed;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, thread_main, &jobs[t]) != 0)
            return -1;
    fill_rows(&jobs[0]);
    for (int t = 1; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    return 0;
}

int synth_euclid_f32(const float *pts, int64_t n, int d, float *W, int nthreads)
{
    return run(pts, n, d, W, 0, 0, nthreads);
}

int synth_euclid32_f32(const float *pts, int64_t n, int d, float *W, int nthreads)
{
    return run(pts, n, d, W, 3, 0, nthreads);
}

int synth_hash_u32(uint64_t seed, int64_t n, uint32_t *W, int nthreads)
{
    return run(NULL, n, 0, (float *)W, 1, seed, nthreads);
}

int synth_uniform01_f32(uint64_t seed, int64_t n, float *W, int nthreads)
{
    return run(NULL, n, 0, W, 2, seed, nthreads);
}

/* one row of the Euclidean matrix (for sampled checks at large n) */
int synth_euclid_row(const float *pts, int64_t n, int d, int64_t i, float *row)
{
    for (int64_t j = 0; j < n; ++j)
        row[j] = (i == j) ? 0.0f : euclid_pair(pts, d, i < j ? i : j, i < j ? j : i);
    return 0;
}
