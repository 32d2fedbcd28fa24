// internal.h -- workspace layout and launch functions shared by the library's
// translation units.  Not part of the public ABI (see include/appd.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "common.cuh"

namespace appd {

constexpr int MAX_LEVELS = 20;     // Boruvka levels: ceil(log2 MAX_N) = 17, plus slack
constexpr int CONTRACT_ROWS = 16;  // rows of the current matrix per contraction work item
constexpr int CONTRACT_THREADS = 1024;   // one contraction CTA per SM
constexpr int CONTRACT_THREADS2 = 512;   // two per SM (half the bins each)

// Device-resident control block of one solve.
struct Counters {
    u32 c[MAX_LEVELS + 2];   // components per level; c[0] = n
    u32 done;                // set when one component is left
    u32 mst_count;           // MST edges recorded so far
    u32 item_next;           // contraction work-queue head
    u32 total_chunks;        // contraction chunks at the current level
    u32 nbr;                 // bin ranges at the current level
    u32 jump_flag[3];        // pointer-jumping convergence flags (rotating)
    u32 fill_next;           // work-queue head of the Algorithm 4 fill
    u32 fill_total;
    u32 signs;               // OR of the sign bits of W's upper triangle (FP32 round 1)
    u32 pad;
    GridBar bar;             // grid barrier of the cooperative kernels
};

// One workspace per (device, n); everything a solve needs besides W and M.
struct Workspace {
    int device = -1;
    int64_t cap = 0;         // allocated capacity (vertices)
    int64_t n = 0;           // vertices of the solve being enqueued
    int levels = 0;          // ceil(log2 n), >= 1
    int st_levels = 0;       // sparse-table levels over n-1 gaps
    int sms = 0;
    int coop_blocks = 0;     // CTAs of the cooperative kernels
    int coop_threads = 0;
    int contract_blocks = 0;
    u32 bin_cap = 0;         // u64 bins per contraction CTA (one CTA per SM)
    u32 bin_cap2 = 0;        // u64 bins per contraction CTA (two CTAs per SM)
    u32 bin_cap_t = 0;       // u64 bins beside the copy ring of the bulk-copy contraction
    void* base = nullptr;
    size_t bytes = 0;

    Counters* ctr = nullptr;
    u32* part = nullptr;     // scan partials (coop_blocks + 1)
    // Boruvka
    u64* best[2] = {nullptr, nullptr};
    u32 *comp = nullptr, *hook = nullptr, *par = nullptr, *flag = nullptr, *rootid = nullptr,
        *label = nullptr, *cnt = nullptr, *fillc = nullptr, *gstart = nullptr, *members = nullptr,
        *nchunk = nullptr, *chunk_start = nullptr, *item_group = nullptr;
    u64* mst = nullptr;
    // dendrogram / leaf order
    u32 *deg = nullptr, *adj_off = nullptr, *afill = nullptr, *adj = nullptr, *aslot = nullptr;
    u32 *lr_d[2] = {nullptr, nullptr}, *lr_nx[2] = {nullptr, nullptr};
    u32 *parent = nullptr, *pe_key = nullptr;
    u64* ord = nullptr;
    u32* jump = nullptr;
    u64* mxo = nullptr;
    u32* nha = nullptr;
    u64* skey[2] = {nullptr, nullptr};
    u32* sval[2] = {nullptr, nullptr};
    u32* hist = nullptr;
    u32 ntiles = 0;
    u32 *first_child = nullptr, *next_sib = nullptr;
    u32 *pos = nullptr, *order = nullptr, *nsize = nullptr, *gap = nullptr, *st = nullptr;
    u32* a4_start = nullptr;   // Algorithm 4 fill: tile prefix per edge
    unsigned short* label16 = nullptr;   // level-0 labels as 16 bits (n + 8 entries)
    // contraction matrices when M cannot serve as scratch (M == W)
    void* cscratch = nullptr;
    size_t cscratch_bytes = 0;
    // zero-padded coordinates of a point-set solve (appd_solve_points)
    float* pscratch = nullptr;
    size_t pscratch_bytes = 0;
    // staging for appd_solve_host
    void* hostW = nullptr;
    void* hostM = nullptr;
    size_t host_bytes = 0;
};

// A point set in place of W (points.cu): P holds n_pad x D zero-padded FP32
// coordinates; the edge weights are computed where they are used.
struct PointsSrc {
    const float* P;   // n_pad x D, in vertex order
    int D;
    float* Ps;        // n_pad x D, the same coordinates in component order (level 0)
    u32* pvid;        // vertex at each position of that order
    u32* pcomp;       // its level-0 component
};
// padded dimension (2, 4, 8, 16 or 32) of a d-dimensional set, 0 if d is out of range
int points_dim(int d);
u32 points_rows_padded(u32 n);
cudaError_t launch_pts_pad(const float* X, u32 n, int d, float* P, cudaStream_t s);
cudaError_t launch_rowmin_pts(const float* P, int D, u32 n, int dt, u64* best, cudaStream_t s);
struct ContractArgs;
cudaError_t launch_mst_sqrt(u64* mst, u32 m, int dt, cudaStream_t s);
cudaError_t launch_pts_gather(const float* P, int D, const u32* members, const u32* label, u32 n, float* Ps,
                              u32* pvid, u32* pcomp, cudaStream_t s);
cudaError_t launch_contract_pts_sorted(const ContractArgs& ca, const float* Ps, const u32* pvid,
                                       const u32* pcomp, int D, int dt, int blocks, cudaStream_t s);
// the n - 1 packed tree edges as three arrays: key, lo, hi
cudaError_t launch_mst_split(const u64* mst, u32 n, u32* keys, u32* lo, u32* hi, cudaStream_t s);
cudaError_t preload_points();

// launch sequence pieces (all asynchronous on the stream); with ps, the
// graph is the point set's and W is not read
cudaError_t run_mst(Workspace& ws, const void* W, int dt, void* cbuf, size_t cbuf_bytes,
                    u32* status, cudaStream_t s, const PointsSrc* ps = nullptr);
cudaError_t run_leaf_order(Workspace& ws, u32* status, cudaStream_t s);
cudaError_t run_fill(Workspace& ws, int dt, void* M, cudaStream_t s);
cudaError_t run_fill_alg4(Workspace& ws, int dt, void* M, u32* status, cudaStream_t s);
// warm start (insert.cu): M' ((n+1) x (n+1)) from M (n x n) and w (n); d: n u32 scratch
cudaError_t run_insert(const void* M, int64_t n, int dt, const void* w, void* Mo, u32* d, int sms,
                       cudaStream_t s);
cudaError_t run_fill_trivial(int64_t n, void* M, cudaStream_t s);   // n == 1
// warm start by a tree update (insert_tree.cu): the minimum spanning tree of
// G + p from G's tree (n - 1 edges) and p's n weights, into ws.mst (packed
// for n + 1 vertices)
cudaError_t run_insert_tree(Workspace& ws, const u32* keys, const u32* lo, const u32* hi, const u32* w,
                            u32 n, int dt, u32* status, cudaStream_t s);
cudaError_t preload_insert_tree();
// level-0 contraction over the upper triangle fed by bulk copies
// (contract_tma.cu); runs when |C_1| <= run_max, needs n % 4 == 0, W 16-byte
// aligned, ca.label16 8-byte aligned (n + 8 entries, written by the level-0
// step) and ca.bin_cap <= contract_tma_bin_cap(smem_optin); signs: the sign
// word k_rowmin_sym filled for this W (FP32), or null when it did not run
struct ContractArgs;
u32 contract_tma_bin_cap(int smem_optin);
cudaError_t launch_contract0_tma(const ContractArgs& ca, int dt, int blocks, u32 run_max, u32* status,
                                 const u32* signs, cudaStream_t s);

// profiling (appd_profile_begin/end): phases of a solve
enum Phase { PH_ROWMIN = 0, PH_STEP, PH_CONTRACT0, PH_CONTRACT, PH_LEAF, PH_FILL, PH_BATCHED, PH_COUNT };
void prof_begin(int phase, cudaStream_t s);
void prof_end(int phase, cudaStream_t s);
void prof_launches(int k);

// Carves the workspace arrays for capacity cap out of base (or only
// measures when base is null); returns the bytes needed.
size_t workspace_layout(Workspace& w, char* base, int64_t cap);

// batched solves (batched.cu): graphs listed in `small` run one per CTA in
// the persistent kernel
struct BatchTuning {
    int ctas_per_sm = 1;     // persistent CTAs per SM (one workspace slice each)
    int fill_rows = 256;     // rows per fill tile inside a CTA
    int64_t n_split = 2048;  // larger graphs use the single-solve pipeline
    u32 prim_max = 256;      // graphs up to this size: one warp each, by Prim (<= 512)
    bool operator==(const BatchTuning& o) const
    {
        return ctas_per_sm == o.ctas_per_sm && fill_rows == o.fill_rows && n_split == o.n_split &&
               prim_max == o.prim_max;
    }
};
// the batched path's current parameters (appd_batched_tuning)
BatchTuning current_batch_tuning();

// host description of one batch of small graphs
struct BatchDesc {
    std::vector<const void*> w;
    std::vector<void*> m;
    std::vector<u32> n;
    std::vector<uint8_t> dt;
};
struct BatchRuntime;   // workspace slices + cached launch plans (batched.cu)
// sets the failure flag of every workspace slice's control block (test hook)
cudaError_t batch_runtime_mark_failed(BatchRuntime* rt);
// the same for the no-allocation array on device dev (if set up there)
cudaError_t noalloc_mark_failed(int dev);
cudaError_t batch_runtime_create(int64_t cap, const BatchTuning& tune, BatchRuntime** out);
void batch_runtime_destroy(BatchRuntime* rt);
int64_t batch_runtime_cap(const BatchRuntime* rt);
// Launches one batch on stream s (cache_graph: capture the launch once per
// layout and replay it; otherwise upload descriptors and launch directly).
// Launches on one runtime must be ordered (one stream).
cudaError_t batch_launch(BatchRuntime& rt, const BatchDesc& d, u32* status, cudaStream_t s,
                         bool cache_graph);

// single solve on an explicit workspace; returns an appd_status code
int solve_on(Workspace& ws, u32* status, const void* W, int64_t n, int dt, void* M,
             cudaStream_t s, bool alg4);
// the current device's status word
u32* device_status_word();
// the status word inside the no-allocation entry point's static array on
// device dev (null before that entry point's first call there)
u32* noalloc_status_word(int dev);
cudaError_t workspace_create(int64_t cap, Workspace** out);
void workspace_destroy(Workspace* w);

// Loads kernels now (their attributes are queried), so that a later launch
// does not pay the module's first load under lazy loading.
template <class... K>
cudaError_t touch_kernels(K... kern)
{
    cudaError_t e = cudaSuccess;
    cudaFuncAttributes at;
    ((e = (e == cudaSuccess) ? cudaFuncGetAttributes(&at, (const void*)kern) : e), ...);
    return e;
}
// every kernel of a translation unit (mst_kernels.cu, contract_tma.cu,
// leaf_order.cu, fill.cu, batched.cu)
cudaError_t preload_mst();
cudaError_t preload_contract_tma();
cudaError_t preload_leaf();
cudaError_t preload_fill();
cudaError_t preload_batched();
// all of the above
cudaError_t preload_kernels();

// sizes
size_t contraction_scratch_bytes(int64_t n);
int ceil_log2(int64_t x);

}  // namespace appd
