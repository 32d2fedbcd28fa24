/*
 * appd.h -- C ABI of the GB300 all-pairs minimax-path (APPD) library.
 *
 * Problem (arxiv 2407.07058, Section 1, Eq. 1-2): for a dense undirected
 * complete graph with symmetric n x n weight matrix W, compute the n x n
 * matrix M with M(i,j) = min over all i-j paths p of the largest edge weight
 * on p (the minimax / longest-leg / MMJ distance; the matrix is the "all
 * points path distance", APPD).  The paper computes it with Prim's MST and
 * Algorithm 4 (Sections 3 and 5); this library computes the same matrix on
 * one GPU with a dense Boruvka MST, a single-linkage leaf order and a tiled
 * range-maximum fill.
 *
 * Conventions shared by every entry point
 *  - Matrices are dense, row-major, n*n elements of 4 bytes.  dtype APPD_F32:
 *    IEEE-754 binary32; APPD_U32: unsigned 32-bit integers.
 *  - Ordering: U32 weights compare as unsigned integers; F32 weights compare
 *    by IEEE-754 totalOrder (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN).
 *    Ties are broken by the edge's endpoint pair, so results never depend on
 *    tie-breaking (Section 5 notes that the tie order is irrelevant).
 *  - Output: every off-diagonal M(i,j) is the bit pattern of one input weight
 *    (the largest edge on a minimax path); the diagonal M(i,i) is all-zero
 *    bits.  W(i,i) is never read.  Results are exact (bit-identical to the
 *    definition), so there is no tolerance.
 *  - Widest paths (Section 4.2): the dtypes APPD_F32_WIDEST / APPD_U32_WIDEST
 *    (the base dtype with the APPD_WIDEST bit set) compute instead the
 *    widest-path matrix, M(i,j) = max over all i-j paths p of the smallest
 *    edge weight on p (maximum capacity / bottleneck paths).  Every
 *    comparison runs in the reversed order, so the MST becomes the maximum
 *    spanning tree; the same conventions hold otherwise (original bits out,
 *    all-zero diagonal).  Every entry point that takes a dtype accepts them.
 *  - W must be symmetric (undirected graph, Section 1).  Only the upper
 *    triangle is relied on by the specification; results for an asymmetric W
 *    are unspecified.  appd_check_symmetric validates.
 *  - 1 <= n <= 92682 (an edge is packed with its endpoints' pair number in
 *    32 bits, and n (n - 1) / 2 <= 2^32 there); n == 0 is a no-op that
 *    returns APPD_OK; larger n returns APPD_ERR_TOO_LARGE.  A solve at the
 *    limit holds W and M, 2 x 34.4 GB, or M alone in place.
 *  - Device pointers are owned by the caller.  Calls are asynchronous on the
 *    given CUDA stream (cudaStream_t, passed as appd_stream_t; NULL is the
 *    legacy default stream).  Argument errors are returned synchronously
 *    before anything is enqueued.  Errors detected on the device (a bounded
 *    wait that ran out, an internal consistency check) are recorded in a
 *    per-device status word that appd_last_device_status returns after the
 *    caller synchronizes the stream.
 *  - The library keeps a workspace per (device, n) that it allocates on first
 *    use and reuses; calls that share a workspace must be ordered (one stream,
 *    or synchronized).  appd_release_workspaces frees them.
 *  - M is also used as scratch space during a solve (its contents before the
 *    call are ignored).  M == W (in place) is allowed; a partial overlap of
 *    M and W returns APPD_ERR_ALIAS.
 */
#ifndef APPD_H
#define APPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (cudaStream_t); declared opaquely so that this header
 * does not require the CUDA headers. */
typedef struct CUstream_st *appd_stream_t;

typedef enum {
    APPD_F32 = 0,
    APPD_U32 = 1,
    APPD_F32_WIDEST = 2,   /* APPD_F32 | APPD_WIDEST */
    APPD_U32_WIDEST = 3    /* APPD_U32 | APPD_WIDEST */
} appd_dtype;

/* dtype bit that selects the widest-path matrix (Section 4.2) */
#define APPD_WIDEST 2

typedef enum {
    APPD_OK = 0,
    APPD_ERR_INVALID = 1,    /* null pointer, n < 0, bad dtype, bad batch layout */
    APPD_ERR_TOO_LARGE = 2,  /* n above the entry point's limit */
    APPD_ERR_NOMEM = 3,      /* device or host allocation failed */
    APPD_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    APPD_ERR_ASYMMETRIC = 5, /* appd_check_symmetric found W(i,j) != W(j,i) */
    APPD_ERR_TIMEOUT = 6,    /* a bounded device wait ran out */
    APPD_ERR_BUSY = 7,       /* server: admission refused (budget or slots) */
    APPD_ERR_ALIAS = 8,      /* M partially overlaps W */
    APPD_ERR_NOT_FOUND = 9,  /* server: unknown request id */
    APPD_ERR_INTERNAL = 10   /* an internal consistency check failed on the device */
} appd_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *appd_status_str(appd_status st);

/*
 * appd_solve -- the APPD matrix of one graph (Eq. 1-2).
 *   W   device pointer, n*n elements of dtype dt, row-major, symmetric.
 *   n   number of vertices.
 *   dt  APPD_F32 or APPD_U32.
 *   M   device pointer, n*n elements of dtype dt, receives the result.
 *   s   CUDA stream.
 * Pipeline (all on the GPU, no host synchronisation): dense Boruvka MST by
 * row minima and block-min contraction of W (the MST step of Section 3, which
 * the paper does with Prim), a single-linkage leaf order of the MST with the
 * merge heights between neighbours (the ascending form of Section 3), and a
 * tiled fill M(i,j) = largest merge height between the two leaves.
 */
appd_status appd_solve(const void *W, int64_t n, appd_dtype dt, void *M, appd_stream_t s);

/*
 * appd_solve_points -- the APPD matrix of a point set's complete graph
 * (Section 1 turns a dataset into a complete graph; Section 4's experiments
 * use point datasets) without forming W: the edge weights are computed where
 * the MST reads them, so device memory holds only the points and M.
 *   X   device pointer, n x d FP32 coordinates, row-major (4-byte aligned).
 *   n   number of points; d dimensions, 1 <= d <= 32.
 *   dt  APPD_F32 (minimax) or APPD_F32_WIDEST (widest paths, Section 4.2).
 *   M   device pointer, n x n FP32, receives the result; must not overlap X
 *       (APPD_ERR_ALIAS).
 * The edge weight is the Euclidean distance evaluated in FP32 in a fixed
 * order: s = 0, then for k = 0 .. d-1, t = X(i,k) - X(j,k) rounded to FP32
 * and s = fma(t, t, s) with one rounding; W(i,j) = sqrt(s), correctly
 * rounded; W(i,i) = +0.  The result is bit-identical to appd_solve on the
 * matrix W so defined.  Coordinates must be finite.  The library keeps a
 * padded copy of the coordinates in its workspace (n x 32 floats at most).
 * 0 <= n <= 92682; other conventions as appd_solve.
 */
appd_status appd_solve_points(const float *X, int64_t n, int32_t d, appd_dtype dt, void *M,
                              appd_stream_t s);

/*
 * appd_solve_alg4 -- same result as appd_solve, but M is written by a GPU
 * form of Algorithm 4's calculation-and-copy step (Sections 3, 5 and the
 * parallel variant of Section 6.2): one work item per MST edge e fills the
 * cross block tree1 x tree2 (and its transpose) with w(e).  Kept to compare
 * the paper's fill pattern with the tiled fill.  Arguments as appd_solve.
 */
appd_status appd_solve_alg4(const void *W, int64_t n, appd_dtype dt, void *M, appd_stream_t s);

/*
 * appd_solve_host -- appd_solve on host memory: copies W (host, n*n) to the
 * device, solves, and copies M back to host memory M_host, all on stream s.
 * Host buffers may be pageable or pinned; the call returns after M_host holds
 * the result (it synchronizes s).  Device staging buffers are kept with the
 * workspace.
 */
appd_status appd_solve_host(const void *W_host, int64_t n, appd_dtype dt, void *M_host,
                            appd_stream_t s);

/*
 * appd_solve_host_async -- appd_solve_host without the wait, pipelined for a
 * stream of problems: enqueues the copy of W_host to the device, the solve
 * (on s) and the copy of M back to M_host, and returns.  Consecutive calls
 * overlap one call's copy back with the next calls' copies in and solves
 * (the host link carries both directions at once; a copy in waits only for
 * the previous solve on its buffer pair).  The library keeps, per device,
 * two device buffer pairs (4 x 4 n^2 bytes, until appd_release_workspaces)
 * and eight internal copy streams (each direction's copy is split into four
 * pieces, which moves more bytes per second over the link).  The solve is
 * ordered on s like appd_solve; the copy back is not: call
 * appd_solve_host_wait(s) and then synchronize s before reading M_host or
 * changing W_host.  Pinned host buffers (cudaHostAlloc) reach the link's
 * bandwidth.  Errors as appd_solve_host.  (Scheduling of this library; no
 * counterpart in the paper.)
 */
appd_status appd_solve_host_async(const void *W_host, int64_t n, appd_dtype dt, void *M_host,
                                  appd_stream_t s);

/* Makes s wait for the copies back of every appd_solve_host_async call made
 * so far on this device (enqueues the wait and returns). */
appd_status appd_solve_host_wait(appd_stream_t s);

/*
 * appd_solve_noalloc -- appd_solve for callers that cannot allocate device
 * memory (a framework that owns a fixed pool or arena, an embedding that does
 * not allow the driver's allocator once it is running).  No counterpart in
 * the paper: it is the same result as appd_solve, for 0 <= n <= 1024, computed
 * by one CTA with all scratch in a 4 MiB file-scope device array that the
 * library carries on every device that loads it.
 *   W, n, dt, M, s  as appd_solve; M == W is allowed.
 * Returns APPD_ERR_TOO_LARGE for n > 1024 (the array's limit).  The call
 * never allocates or frees memory.  The array is shared by all calls on a
 * device and keeps the last call's contents (the kernel initialises what it
 * reads); calls whose kernels overlap on the GPU race on it, so order them.
 * The first call on a device looks up the array's address and sets a kernel
 * attribute; make it before any stream capture.  Errors it detects on the
 * device (an internal consistency check) are kept in a status word inside the
 * array and reported, like every other entry point's, by
 * appd_last_device_status; a failed solve leaves M unwritten.
 */
appd_status appd_solve_noalloc(const void *W, int64_t n, appd_dtype dt, void *M, appd_stream_t s);

/*
 * appd_insert_vertex -- warm start (Section 6.1): the matrix of G + p from
 * the matrix of G and the new vertex's edge weights, without a new tree.
 *   M      device, n x n: the result of appd_solve (same dtype) for G.
 *   w      device, n weights: w[k] = weight of the edge between vertex k and p.
 *   M_out  device, (n+1) x (n+1), row-major: the matrix of G + p, where p is
 *          vertex n.  Must not overlap M or w (APPD_ERR_ALIAS).
 * With d(i) = min over k of max(M(i,k), w[k]) (the k = i term is w[i]),
 * M_out(i,j) = min(M(i,j), max(d(i), d(j))), M_out(i,n) = M_out(n,i) = d(i),
 * all-zero diagonal; comparisons and the widest dtypes as appd_solve.  The
 * result equals appd_solve on the (n+1)-vertex graph, bit for bit.  Two
 * streaming passes over M.  0 <= n < 92682 (n == 0: M and w may be NULL,
 * M_out becomes the 1 x 1 zero matrix); larger n returns APPD_ERR_TOO_LARGE.
 */
appd_status appd_insert_vertex(const void *M, int64_t n, appd_dtype dt, const void *w, void *M_out,
                               appd_stream_t s);

/*
 * appd_insert_vertex_tree -- warm start (Section 6.1) through the minimum
 * spanning tree: the matrix of G + p from G's tree and the new vertex's
 * weights, without reading G's matrix.
 *   keys, lo, hi  device arrays of n-1 uint32: G's minimum spanning tree as
 *                 appd_mst_edges returns it (same dtype; order keys).
 *   w             device, n weights: w[k] = weight of the edge between k and p.
 *   M_out         device, (n+1) x (n+1): the matrix of G + p, p = vertex n.
 *   keys_out, lo_out, hi_out  device arrays of n uint32 receiving the tree of
 *                 G + p (same format), or all three NULL; pass them to the
 *                 next call to insert vertices one after another.
 * Every edge of G outside its tree is the largest on a cycle of G, so the
 * tree of G + p takes only the n-1 tree edges and p's n edges: it is found by
 * Boruvka's algorithm on those 2n-1 edges (O(n log n) work), followed by the
 * leaf order and one fill of M_out, the only O(n^2) traffic.  The result
 * equals appd_solve on the (n+1)-vertex graph, bit for bit, when the tree is
 * G's minimum spanning tree.  None of the arrays may overlap M_out or the
 * tree outputs (APPD_ERR_ALIAS).  0 <= n < 92682 (n == 0: M_out becomes the
 * 1 x 1 zero matrix); dtypes and comparisons as appd_solve.
 */
appd_status appd_insert_vertex_tree(const uint32_t *keys, const uint32_t *lo, const uint32_t *hi,
                                    int64_t n, appd_dtype dt, const void *w, void *M_out,
                                    uint32_t *keys_out, uint32_t *lo_out, uint32_t *hi_out,
                                    appd_stream_t s);

/*
 * appd_mst -- the minimum spanning tree computed by the solve's MST stage.
 *   edges_out  device pointer to n-1 uint64 values; each is
 *              key << 32 | lo << 16 | hi, where lo < hi are the endpoints and
 *              key is the order key of W(lo,hi) (the weight's bits for U32;
 *              for F32, bits | 0x80000000 if the sign bit is clear, else ~bits;
 *              complemented for the widest dtypes, whose tree is the maximum
 *              spanning tree).  Edge order in the array is unspecified.
 * Under the strict order (key, lo, hi) the MST is unique, so the edge set can
 * be compared exactly with any correct MST algorithm (Section 3 uses Prim).
 * 16-bit endpoints: n <= 65536 (APPD_ERR_TOO_LARGE above; see appd_mst_edges).
 */
appd_status appd_mst(const void *W, int64_t n, appd_dtype dt, uint64_t *edges_out,
                     appd_stream_t s);

/*
 * appd_mst_edges -- the same tree for any n the library takes, as three
 * device arrays of n-1 uint32 values: keys[k] (the order key, as appd_mst),
 * lo[k] < hi[k] (the endpoints).  Edge order unspecified.
 */
appd_status appd_mst_edges(const void *W, int64_t n, appd_dtype dt, uint32_t *keys,
                           uint32_t *lo, uint32_t *hi, appd_stream_t s);

/*
 * appd_leaf_order -- the single-linkage leaf order used by the fill.
 *   pos_out  device, n uint32: position of vertex v in the order.
 *   gap_out  device, n-1 uint32: gap_out[k] = order key of the largest edge
 *            on the MST path between the vertices at positions k and k+1.
 * For all i != j: key(M(i,j)) = max(gap_out[min(p_i,p_j) .. max(p_i,p_j)-1]).
 * (Reading off distances from the dendrogram, Section 7.)
 */
appd_status appd_leaf_order(const void *W, int64_t n, appd_dtype dt, uint32_t *pos_out,
                            uint32_t *gap_out, appd_stream_t s);

/*
 * appd_solve_batched -- many independent graphs in one launch sequence.
 *   offsets  host array, count entries: element offset of graph g in Ws and Ms.
 *   Ws       device base pointer; graph g's W starts at (elem*)Ws + offsets[g].
 *   ns       host array, count entries: n of each graph (1..92682).
 *   dts      host array of count bytes (APPD_F32 / APPD_U32) or NULL (all F32).
 *   Ms       device base pointer; graph g's M starts at (elem*)Ms + offsets[g].
 *   count    number of graphs.
 * The ranges [offsets[g], offsets[g] + ns[g]^2) must not overlap between
 * graphs and M ranges must not overlap W ranges except exactly (in place).
 * Graphs up to a size cut-over run one per CTA inside a persistent kernel
 * with a work queue; larger graphs use the single-solve pipeline.
 */
appd_status appd_solve_batched(const int64_t *offsets, const void *Ws, const int64_t *ns,
                               const uint8_t *dts, void *Ms, int32_t count, appd_stream_t s);

/*
 * appd_batched_tuning -- sets the batched path's parameters for this process:
 *   ctas_per_sm  persistent CTAs per SM (1 or 2), each with its own workspace;
 *   fill_rows    rows per fill batch inside a CTA (a power of two, 64..2048);
 *   n_split      graphs with n > n_split go through the single-solve pipeline.
 * Defaults: 1, 256, 2048.  Returns APPD_ERR_INVALID for values out of range.
 * (No counterpart in the paper: scheduling parameters of this library.)
 */
appd_status appd_batched_tuning(int32_t ctas_per_sm, int32_t fill_rows, int64_t n_split);

/*
 * appd_batched_autotune -- picks the batched path's fill rows and size
 * cut-over for this GPU by timing every candidate pair (fill rows 256..2048,
 * cut-over 512..4096), then the warp-Prim limit (0..512, see
 * appd_batched_prim_max) with the best pair, on a seeded synthetic batch of
 * 192 graphs, installs the fastest for this process, and appends it to the
 * JSON-lines file cache_path
 * (keyed by GPU name and driver version; NULL: no cache).  If cache_path
 * already holds an entry for this GPU, it is installed without a search.
 * Synchronizes s; allocates 2.4 GB of device memory for the search and frees
 * it before returning.  APPD_ERR_CUDA when no device answers.  (Scheduling parameters of
 * this library; no counterpart in the paper.)
 */
appd_status appd_batched_autotune(const char *cache_path, appd_stream_t s);

/* Reads the batched path's current parameters (see appd_batched_tuning);
 * APPD_ERR_INVALID on a null pointer.  Needs no GPU. */
appd_status appd_batched_get_tuning(int32_t *ctas_per_sm, int32_t *fill_rows, int64_t *n_split);

/*
 * appd_batched_prim_max -- graphs of the batched path with at most prim_max
 * vertices (0..512) are solved one per warp by Prim's algorithm (Section 3's
 * MST step; its visiting order is the leaf order the fill reads), 16 graphs
 * at once per CTA; larger ones by the one-CTA Boruvka solve.  Default 256;
 * appd_batched_autotune searches it.  APPD_ERR_INVALID out of range.
 * appd_batched_get_prim_max reads it.  (Scheduling of this library.)
 */
appd_status appd_batched_prim_max(int32_t prim_max);
appd_status appd_batched_get_prim_max(int32_t *prim_max);

/*
 * appd_check_symmetric -- returns APPD_OK if W(i,j) and W(j,i) have identical
 * bits for all i < j, APPD_ERR_ASYMMETRIC otherwise.  Synchronizes s.
 */
appd_status appd_check_symmetric(const void *W, int64_t n, appd_dtype dt, appd_stream_t s);

/*
 * appd_last_device_status -- synchronizes s, then returns and clears the
 * device-detected error status of the current device (APPD_OK,
 * APPD_ERR_TIMEOUT or APPD_ERR_INTERNAL).
 */
appd_status appd_last_device_status(appd_stream_t s);

/*
 * appd_probe_bounded_wait -- failure-detection probe (no counterpart in the
 * paper).  Launches a two-CTA cooperative kernel in which one CTA never
 * reaches the grid barrier, so the other CTA's bounded wait runs out after
 * limit_ms (1..10000) milliseconds and records APPD_ERR_TIMEOUT in the device
 * status word; both CTAs then return and the context stays usable.  Nothing
 * faults or hangs.  Returns APPD_OK once enqueued; appd_last_device_status
 * then reports and clears the timeout.
 */
appd_status appd_probe_bounded_wait(int32_t limit_ms, appd_stream_t s);

/* Frees every cached workspace on the current device (synchronizes it). */
appd_status appd_release_workspaces(void);

/*
 * appd_debug_mark_failed -- failure injection on the host, for tests (no
 * counterpart in the paper).  Sets the per-solve failure flag in every
 * control block the library keeps on the current device (the single-solve
 * workspace, every workspace slice of the batched path, the array of
 * appd_solve_noalloc), as a solve whose bounded wait ran out would leave it.
 * The next solve on each must start clean and give the exact result.
 * Synchronizes the device.  Touches no GPU state besides those flags.
 */
appd_status appd_debug_mark_failed(void);

/* ----------------------------------------------------------- profiling */
/*
 * appd_profile_begin -- from now on the library records a CUDA event pair on
 * the caller's stream around each group of its kernel launches and counts
 * the kernels it launches.  Returns 0.
 * appd_profile_end -- synchronizes the device, stops recording, and writes
 * up to cap doubles to out: summed device milliseconds per phase
 *   [0] round-1 row minima   [1] Boruvka steps       [2] contraction of W
 *   [3] later contractions   [4] leaf order          [5] fill of M
 *   [6] batched persistent kernel
 * then [7] kernels launched, [8] components after round 1 of the last solve.
 * Returns the number of values written.
 */
int32_t appd_profile_begin(void);
int32_t appd_profile_end(double *out, int32_t cap);

/* ------------------------------------------------------------- serving */
/*
 * A continuous-batching solve server on one GPU.  Requests of different n
 * are admitted while the sum of their device footprints stays within an HBM
 * budget; each admitted request owns a slot holding its W and M on the
 * device.  Committed requests are batched into the persistent batched kernel
 * as they arrive, so new work starts while earlier work is still running.
 */
typedef struct appd_server appd_server;

/* budget_bytes: device bytes the server may hold (slots + workspace).
 * max_inflight: upper bound on admitted, unreleased requests.
 * The server takes the batched path's parameters set for the process at
 * creation (appd_batched_tuning / appd_batched_prim_max / autotune). */
appd_status appd_server_create(size_t budget_bytes, int32_t max_inflight, appd_server **out);

/* Admit a request for an n-vertex graph of dtype dt.  On APPD_OK, *req_id is
 * its id and *W_slot a device pointer to n*n elements that the caller fills
 * on stream s (s is made to wait for the slot's allocation; no host wait)
 * and must not touch after commit.  Returns APPD_ERR_BUSY if the budget or
 * slot count is exhausted. */
appd_status appd_server_submit(appd_server *sv, int64_t n, appd_dtype dt, appd_stream_t s,
                               uint64_t *req_id, void **W_slot);

/* Admit up to count requests at once (ns[k] vertices, dtype dts[k]): the
 * longest prefix of the list that fits the budget and the in-flight limit is
 * admitted, *admitted receives its length, and req_ids[k] / W_slots[k] are
 * filled for k < *admitted as appd_server_submit does; s waits (on the device)
 * for all their allocations.  Returns APPD_ERR_BUSY when count > 0 and none
 * fits, APPD_OK otherwise (including a partial admission). */
appd_status appd_server_submit_many(appd_server *sv, int32_t count, const int64_t *ns,
                                    const uint8_t *dts, appd_stream_t s, uint64_t *req_ids,
                                    void **W_slots, int32_t *admitted);

/* Queue an admitted request for solving: its W is complete once the work
 * enqueued on s before this call has run (the solve waits for that on the
 * device; the caller need not synchronize). */
appd_status appd_server_commit(appd_server *sv, uint64_t req_id, appd_stream_t s);

/* appd_server_commit for count requests at once (one device event for the
 * group).  Either all are queued or, on an unknown or already committed id,
 * none (APPD_ERR_NOT_FOUND / APPD_ERR_INVALID). */
appd_status appd_server_commit_many(appd_server *sv, int32_t count, const uint64_t *req_ids,
                                    appd_stream_t s);

/* Collect finished requests: up to cap ids in done_ids and their device M
 * pointers in M_ptrs (valid until release); *n_done receives the count.
 * Never blocks. */
appd_status appd_server_poll(appd_server *sv, uint64_t *done_ids, const void **M_ptrs,
                             int32_t cap, int32_t *n_done);

/* Free a request's slots (its M pointer becomes invalid): a finished
 * request, or one admitted but never committed.  The memory is freed in
 * stream order after the work enqueued on s so far, so the caller's reads of
 * M (or writes of an uncommitted W) enqueued on s complete before a later
 * request can reuse it; work on other streams must be ordered before s.
 * APPD_ERR_BUSY for a committed request that has not finished. */
appd_status appd_server_release(appd_server *sv, uint64_t req_id, appd_stream_t s);

/* appd_server_release for count requests; all ids are checked first, so
 * either all are released or none. */
appd_status appd_server_release_many(appd_server *sv, int32_t count, const uint64_t *req_ids,
                                     appd_stream_t s);

/* Wait for in-flight work, free all slots and the server. */
appd_status appd_server_destroy(appd_server *sv);

#ifdef __cplusplus
}
#endif

#endif /* APPD_H */
