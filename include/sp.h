/*
 * sp.h -- C ABI of libsp: dynamic single-source shortest paths on one GPU.
 *
 * The library keeps a weighted directed graph resident on the device as a
 * forward and a reverse CSR with slack in every row, together with the
 * distance and parent of every vertex from one source.  A batch of edge
 * deletions and insertions is merged into both CSRs and the distances are
 * repaired incrementally, as the DynSSSP driver of the paper does (Section 3.2
 * "Language Overview with a Motivating Example: Dynamic SSSP"; Appendix,
 * DynSSSP/Incremental/Decremental listings): deletions first, then
 * insertions.  All arithmetic is exact integer.
 *
 * Conventions shared by every entry point:
 *   - Status codes: every function returns an sp_status; no C++ exception
 *     crosses the ABI.  sp_status_str() names a code.
 *   - Ownership: the library copies every input array during the call; the
 *     caller keeps its buffers and may reuse them as soon as the call returns.
 *     The sp_graph handle and all device memory it holds belong to the
 *     library until sp_graph_destroy().
 *   - Host or device pointers: a flag on each call says whether the arrays
 *     are host memory (pageable or pinned) or device memory of the graph's
 *     device.  Device arrays must stay valid until the call returns.  Batch
 *     arrays and distance outputs in page-locked host memory that is mapped
 *     into the device's address space are read and written by kernels across
 *     the host link; other host arrays go through the copy engine.
 *   - Streams: every call is ordered on the CUDA stream given at creation and
 *     returns only after its work on that stream is complete (the status it
 *     returns is the device's).  A handle is not thread-safe; distinct
 *     handles may be used concurrently from different threads and streams.
 *   - Validation happens before any change: a batch that fails validation
 *     (SP_EINVAL) leaves the graph exactly as it was.
 *   - A device-side bound being hit (SP_ETIMEOUT) or a distance that does not
 *     fit (SP_ERANGE) during a repair leaves distances unspecified: the graph
 *     is then in SP_ESTATE until sp_sssp_init() is called again.  The edge set
 *     includes every batch that returned SP_OK or SP_ERANGE, and a batch that
 *     returned SP_ETIMEOUT from its repair (sp_loop_counters site 1-3: the
 *     CSR merge completes before any repair starts); a batch stopped in its
 *     sort or count pass (site 4 or 5) did not change the edge set.
 *   - SP_ENOMEM from a batch (a buffer or the spare pool could not grow)
 *     leaves the edge set and the distances as they were: distances that the
 *     invalidation had already changed are recomputed from the last init's
 *     sources before the call returns (without allocating).
 */
#ifndef SP_H
#define SP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sp_graph sp_graph;   /* opaque, owned by the library */

typedef enum {
    SP_OK = 0,
    SP_EINVAL = -1,        /* bad argument or batch (ids, weights, sizes)   */
    SP_ENOMEM = -2,        /* a device or host allocation failed            */
    SP_ERANGE = -3,        /* a finite distance reached SP_INF              */
    SP_ESTATE = -4,        /* call not valid in this state (e.g. no source) */
    SP_ECUDA = -5,         /* a CUDA runtime call failed                    */
    SP_ETIMEOUT = -6,      /* a device-side round cap or wait bound was hit */
    SP_ENOMEM_BUDGET = -7  /* refused: the graph would exceed a memory budget */
} sp_status;

/* Distance of an unreachable vertex: INT_MAX/2, the value the appendix's
 * OnDelete and Decremental listings store (so SP_INF + w cannot overflow). */
#define SP_INF 1073741823
/* Largest accepted edge weight; weights must be 1 <= w <= SP_WMAX. */
#define SP_WMAX (1 << 20)
/* Number of per-phase slots in sp_batch_stats. */
#define SP_NPHASE 8

/* Phases of one batch, in launch order (indexes of ms_phase / alg_bytes). */
enum {
    SP_PH_SORT = 0,      /* validate + sort the batch by (row, col)           */
    SP_PH_COUNT = 1,     /* per touched row: applied/absent/present, new size */
    SP_PH_MERGE = 2,     /* OnDelete mark + merge into forward/reverse CSR    */
    SP_PH_INVAL = 3,     /* invalidate shortest-path subtrees (Decremental 1) */
    SP_PH_PULL = 4,      /* pull repair of invalidated vertices (Decremental 2)*/
    SP_PH_ADD = 5,       /* relax inserted edges (OnAdd)                      */
    SP_PH_PUSH = 6,      /* push fixedPoint (Incremental)                     */
    SP_PH_FINISH = 7     /* status + counters back to the host                */
};

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc()
 * returns device memory of at least `bytes` bytes, 256-byte aligned, or NULL;
 * free() releases it.  `stream` is the graph's cudaStream_t.  With a NULL
 * allocator the library uses cudaMallocAsync/cudaFreeAsync on that stream. */
typedef struct {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
} sp_allocator;

/* Counters and timings of one sp_apply_batch (or sp_sssp_init) call.  The
 * applied/absent/present counts, the affected count and the round counts
 * report the batch; the per-phase arrays (alg_bytes, ms_phase) and the split
 * round counts are an extension for measurement, beyond the paper's
 * interface. */
typedef struct {
    int64_t n_del_applied;   /* deletions of present edges                  */
    int64_t n_del_absent;    /* deletions of absent edges (no-ops)          */
    int64_t n_add_applied;   /* insertions of new edges                     */
    int64_t n_add_present;   /* insertions of present edges (no-ops)        */
    int64_t affected;        /* vertices invalidated by deletions           */
    int64_t seeds;           /* vertices in the first push frontier         */
    int64_t relaxed_edges;   /* edges scanned by the push loop              */
    int64_t improved;        /* successful distance decreases in the loop   */
    int64_t rows_touched;    /* forward + reverse rows rewritten            */
    int64_t rows_relocated;  /* rows moved to the spare pool                */
    int32_t rounds_inval;    /* rounds of the subtree invalidation          */
    int32_t rounds_push;     /* rounds of the push fixedPoint               */
    int32_t n_launches;      /* kernels launched by this call               */
    int32_t regrows;         /* times the call grew a buffer and re-ran     */
    int64_t alg_bytes[SP_NPHASE]; /* algorithmic bytes moved per phase      */
    float ms_phase[SP_NPHASE];    /* device time per phase (CUDA events)    */
    float ms_total;               /* device time of the whole call          */
} sp_batch_stats;

/* Read-only facts about a graph. */
typedef struct {
    int32_t n;
    int32_t source;          /* -1 before sp_sssp_init                      */
    int64_t m;               /* current number of edges                     */
    int64_t cap_fwd;         /* edge slots of the forward store (all rows + pool) */
    int64_t cap_rev;
    int64_t pool_used_fwd;   /* spare-pool slots taken by relocated rows    */
    int64_t pool_used_rev;
    int64_t device_bytes;    /* device memory held by the handle            */
    int32_t state;           /* 0 = no distances, 1 = valid, 2 = SP_ESTATE  */
    int32_t num_sms;
    int32_t pool_step;       /* edges a lane relaxes per step in the pool
                                schedule: 5 once at least 1/64 of the
                                vertices have 5..8 out-edges, else 4 (an
                                extension: speed only, never a distance) */
    int32_t reserved;
} sp_graph_info;

/*
 * Create a graph from a CSR: row_off[n+1] (int64, row_off[0] = 0,
 * non-decreasing, row_off[n] = m), col[m] (destinations, 0 <= col < n) and
 * w[m] (1 <= w <= SP_WMAX).  Rows need not be sorted; duplicate edges are
 * rejected with SP_EINVAL.  `slack` (>= 0, e.g. 0.25) is the fraction of
 * spare slots reserved per row.  `alloc` may be NULL.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  On success *out receives the
 * handle.  The graph lives on the device that is current at the call.
 * Graph storage: the CSR of Section 3.5 ("Modified Graph Representation"),
 * with per-row slack in place of the paper's diff-CSR.
 */
sp_status sp_graph_create(int32_t n, int64_t m, const int64_t *row_off,
                          const int32_t *col, const int32_t *w,
                          int inputs_on_device, float slack,
                          const sp_allocator *alloc, void *cuda_stream,
                          sp_graph **out);

/* Release every resource of g (NULL is accepted). */
sp_status sp_graph_destroy(sp_graph *g);

/*
 * Compute distances and parents from `source` from scratch (the appendix's
 * staticSSSP: dist = INF and parent = -1 everywhere, then a fixedPoint of
 * Min relaxations seeded by the source).  Also the from-scratch comparator.
 * stats may be NULL (an extension of the boundary: per-phase timings and
 * algorithmic bytes for the benchmark; the paper's calls have none).
 * SP_EINVAL if source is out of range.
 */
sp_status sp_sssp_init(sp_graph *g, int32_t source, sp_batch_stats *stats);

/*
 * Apply one batch: deletions (del_src[i] -> del_dst[i]) then insertions
 * (add_src[i] -> add_dst[i] with weight add_w[i]), and repair distances and
 * parents (DynSSSP driver, Section 3.2 and Appendix).  Either count may be 0
 * (the matching pointers may then be NULL).  Semantics of cases the paper
 * leaves open:
 *   - deleting an absent edge, or deleting one edge twice, is a counted no-op;
 *   - inserting an edge present after the deletions is a counted no-op and
 *     keeps the old weight; among repeated insertions of one edge the smallest
 *     weight wins;
 *   - an edge deleted and inserted in one batch ends up with the new weight.
 * Requires a prior successful sp_sssp_init (else SP_ESTATE).  SP_EINVAL (ids
 * out of range, w outside [1, SP_WMAX], negative counts) leaves the graph
 * unchanged.  stats may be NULL; with stats the call also records per-phase
 * CUDA events.  inputs_on_device = 0: host arrays, moved to device staging
 * buffers first: page-locked arrays that are mapped into the device's
 * address space (cudaHostAlloc, pinned tensors) by one kernel that reads
 * them across the host link, any other host array by the copy engine.  The
 * call is synchronous, so the arrays may be reused once it returns.
 */
sp_status sp_apply_batch(sp_graph *g,
                         int64_t n_del, const int32_t *del_src, const int32_t *del_dst,
                         int64_t n_add, const int32_t *add_src, const int32_t *add_dst,
                         const int32_t *add_w,
                         int inputs_on_device, sp_batch_stats *stats);

/*
 * sp_apply_batch followed by sp_get_dist in one call: after the repair a
 * kernel enqueued behind the batch writes the distances (dist[n]) and, if
 * parent != NULL, the parents (parent[n]), and the call synchronises once.
 * This is one round of the DynSSSP driver of Section 3.2 as a server runs
 * it: apply the update batch, then hand out the node properties dist and
 * parent that the repair maintains.  Inputs as for sp_apply_batch; outputs
 * as for sp_get_dist (out_on_device: device arrays of the graph's device;
 * else host arrays, page-locked mapped ones written in place, others through
 * a device buffer and a copy).  On any status other than SP_OK the contents
 * of dist and parent are unspecified.
 */
sp_status sp_apply_batch_get(sp_graph *g,
                             int64_t n_del, const int32_t *del_src, const int32_t *del_dst,
                             int64_t n_add, const int32_t *add_src, const int32_t *add_dst,
                             const int32_t *add_w, int inputs_on_device,
                             int32_t *dist, int32_t *parent, int out_on_device,
                             sp_batch_stats *stats);

/*
 * Copy distances (dist[n]; SP_INF = unreachable) and, if parent != NULL,
 * parents (parent[n]; -1 for the source and unreachable vertices) out:
 * the node properties dist and parent that the problem statement of Section
 * 3.2 maintains (propNode<int> dist, propNode<node> parent of the DynSSSP
 * program).  out_on_device: dist/parent are device arrays of the graph's
 * device, else SP_EINVAL before anything runs (out_on_device = 0: host
 * memory; page-locked, mapped host arrays are written in place by the
 * kernel, others through a device buffer and a copy).  The call is
 * synchronous.  SP_ESTATE if no valid distances exist.
 */
sp_status sp_get_dist(sp_graph *g, int32_t *dist, int32_t *parent,
                      int out_on_device);

/* Number of edges now in the graph. */
sp_status sp_graph_num_edges(const sp_graph *g, int64_t *m);

/*
 * Install distances and parents exported earlier by sp_get_dist (host
 * arrays if in_on_device == 0, else device arrays of the graph's device;
 * n entries each), for `source`, without a recompute -- a checkpoint of the
 * node properties dist and parent of the problem statement (Section 3.2),
 * restored after the graph was rebuilt from its edge set.  The pair is
 * checked on the device first: dist[source] = 0 with parent -1, every other
 * finite distance realised by a tight parent edge, SP_INF with parent -1
 * elsewhere, and no edge offering a shorter distance.  Those conditions hold
 * exactly for the shortest-path distances of the current edge set, so the
 * restored state equals what sp_sssp_init would compute (parents may differ
 * where ties allow).  SP_EINVAL (and nothing changed) if any check fails.
 * The inputs are copied.  On success the graph is in the valid state.
 */
sp_status sp_set_dist(sp_graph *g, int32_t source, const int32_t *dist,
                      const int32_t *parent, int in_on_device);

/*
 * An upper bound of the device bytes (sp_graph_info.device_bytes) a handle
 * holds once created from a graph of n vertices and m edges with the given
 * slack and sized by sp_reserve(max_updates) for batches of up to
 * max_updates updates given in host memory.  It stays an upper bound until
 * the graph outgrows its spare pools (rows relocated by insertions) or its
 * edge count grows far past m.  Computed for the current device.  The
 * serving runtime admits graphs by it.  SP_EINVAL on out-of-range
 * arguments.  (No counterpart in the paper: memory accounting for the
 * resident-graph budget.)
 */
sp_status sp_footprint_bound(int32_t n, int64_t m, float slack, int64_t max_updates,
                             int64_t *bytes);

/*
 * Export the current edge set as a row-sorted CSR: row_off[n+1], col[m],
 * w[m] with m from sp_graph_num_edges.  `reverse` = 1 exports the reverse
 * (transpose) store instead: row v lists the sources u of edges u -> v with
 * their weights.  Used for checkpoints and for store tests.  out_on_device:
 * device arrays of the graph's device, else SP_EINVAL before anything runs.
 */
sp_status sp_export_csr(sp_graph *g, int reverse, int64_t *row_off,
                        int32_t *col, int32_t *w, int out_on_device);

/*
 * Allocation-free form of sp_export_csr(g, reverse, row_off, col, w, 1): the
 * same device-side export, for callers that must not allocate device memory
 * during the call (a serving process snapshotting a live graph into buffers
 * it reserved up front, or code held to a fixed memory footprint, where an
 * allocation could fail or stall).  The paper has no counterpart; it is a
 * property of this library's API.
 *   row_off[n+1], col[m], w[m]: device arrays of the graph's device, owned
 *   by the caller (m from sp_graph_num_edges); row_off doubles as the degree
 *   buffer before the in-place prefix sum, so it must not alias col or w.
 *   The graph's device must be current (else SP_EINVAL).
 *   Graphs with more than 2^26 vertices are rejected with SP_EINVAL: the
 *   scan's partial sums live in a fixed 512 KiB device array that every GPU
 *   loading the library holds until exit.
 *   The first call on each device looks that array's address up
 *   (cudaGetSymbolAddress); make it before any stream capture.  The address
 *   is kept for the life of the process, so it does not survive a reset of
 *   the device's primary context (cudaDeviceReset): do not call this again
 *   on a device after such a reset.  All calls share the array, so calls
 *   whose work overlaps on the GPU race; nothing in it needs to start at
 *   zero.  Like sp_export_csr, the call is synchronous: it returns after its
 *   work on the graph's stream has completed.
 */
sp_status sp_export_csr_noalloc(sp_graph *g, int reverse, int64_t *row_off,
                                int32_t *col, int32_t *w);

/* Fill *info. */
sp_status sp_graph_info_get(const sp_graph *g, sp_graph_info *info);

/*
 * Device-side bounds of the repair loops: max_rounds caps the rounds of each
 * fixedPoint loop (0 = the Bellman-Ford bound n + 1); wait_ns bounds every
 * grid-barrier wait in nanoseconds (0 = 2 s).  Hitting either returns
 * SP_ETIMEOUT.  Meant for tests of the timeout path and for latency limits.
 */
sp_status sp_set_limits(sp_graph *g, int32_t max_rounds, int64_t wait_ns);

/*
 * Near-far ordering of the push fixedPoint: with delta > 0 a round relaxes
 * only vertices whose distance is below a threshold; improved vertices at or
 * above it wait in a far pile, and the threshold rises by delta (from the
 * pile's smallest distance) whenever the near frontier runs dry.  Distances
 * are the same for every delta; delta trades rounds for redundant
 * relaxations (large delta suits low-diameter graphs, a delta near a few
 * edge weights suits high-diameter ones).  0 (the default) turns it off:
 * plain frontier rounds, as in the paper's Incremental fixedPoint.
 */
sp_status sp_set_push_delta(sp_graph *g, int32_t delta);

/*
 * Decremental invalidation strategy (the subtree walk that follows OnDelete,
 * Section 3.2).  The walk first runs frontier rounds down the
 * shortest-path tree, one tree level per round.  After `rounds` rounds with
 * vertices still to visit it switches to pointer jumping over all vertices:
 * every vertex follows its ancestors, doubling the distance per pass, until
 * it meets a cut ancestor or the root, so the remaining levels cost
 * log2(depth) passes instead of one round each.  Both strategies invalidate
 * exactly the descendants of the cut vertices.  rounds < 0: never switch;
 * 0 (the default): jump right after OnDelete.  A pass costs about one
 * frontier round on a graph of a few million vertices, so frontier rounds
 * pay only for shallow cuts on much larger graphs.
 */
sp_status sp_set_inval_switch(sp_graph *g, int32_t rounds);

/*
 * Single-block rounds of the push fixedPoint.  A round whose frontier has at
 * most max_edges out-edges is run by one thread block with the frontier in
 * shared memory and a block barrier instead of a grid barrier; the other
 * blocks wait until the frontier grows past the bound or empties.  On
 * high-diameter graphs most rounds are this small.  0 turns it off; the
 * bound is clamped to 4096 (the default).  Results do not depend on it.
 */
sp_status sp_set_local_rounds(sp_graph *g, int32_t max_edges);

/*
 * Work schedule of the push fixedPoint (the Incremental `fixedPoint` with
 * `Min` of Section 3.2, whose generated CUDA code runs one thread per vertex
 * and one launch per iteration).  Results do not depend on it.
 *   small_deg (0..64, default 8): a frontier vertex with at most small_deg
 *     out-edges is expanded by one thread; a larger one is cut into 256-edge
 *     chunks, one warp each, spread over the whole grid (a hub's edges reach
 *     every SM).  0 chunks every vertex.
 *   pool_rounds (0..16384, default 0 = off): block-local relaxation.  Every
 *     thread block keeps the vertices it improved below the near-far
 *     threshold (those with at most 16 out-edges) in a pool in shared memory
 *     and expands them itself, in up to pool_rounds sub-rounds ended by block
 *     barriers, before the round's grid barrier; a shortest-path wave then
 *     crosses many edges per grid round.  Meant for high-diameter graphs,
 *     where grid rounds, not relaxations, bound the time.
 * SP_EINVAL outside these ranges.
 */
sp_status sp_set_schedule(sp_graph *g, int32_t small_deg, int32_t pool_rounds);

/*
 * Multi-source form of sp_sssp_init: dist[v] is the shortest distance from
 * the nearest of sources[0..k) (each source has dist 0 and parent -1).  On
 * a graph made of k disjoint components with one source each -- the batched
 * form, many independent graphs packed into one handle with offset vertex
 * ids -- every component gets exactly its own single-source distances, and
 * one batch call then repairs all of them in the same launches.  `sources`
 * is host or device memory (sources_on_device).  SP_EINVAL if k < 1 or a
 * source is out of range.
 */
sp_status sp_sssp_init_multi(sp_graph *g, const int32_t *sources, int32_t k,
                             int sources_on_device, sp_batch_stats *stats);

/*
 * Capturable batch path.  sp_reserve sizes every per-batch buffer for
 * batches of up to max_updates deletions + insertions, so that
 * sp_apply_batch_async never allocates.  sp_apply_batch_async enqueues the
 * whole batch (same kernels and semantics as sp_apply_batch, device inputs
 * only) on the graph's stream without any host synchronisation and copies a
 * result record into `result` (device or pinned host memory,
 * sp_async_result_bytes() bytes) at the end; it can therefore be recorded
 * into a CUDA graph (sp_capture_apply) and replayed with new contents in the
 * same input buffers.  After the stream work completes, sp_apply_batch_finish
 * reads the record, updates the handle's host-side state (edge count,
 * validity) and fills stats; it returns the batch's status.  A batch that
 * would need a larger spare pool is not applied and finishes with
 * SP_ENOMEM: apply it with sp_apply_batch, which grows the pool.
 * Returns SP_ENOMEM from sp_apply_batch_async if the reservation is too
 * small, SP_ESTATE without valid distances.
 */
sp_status sp_reserve(sp_graph *g, int64_t max_updates);
size_t sp_async_result_bytes(void);
sp_status sp_apply_batch_async(sp_graph *g,
                               int64_t n_del, const int32_t *del_src, const int32_t *del_dst,
                               int64_t n_add, const int32_t *add_src, const int32_t *add_dst,
                               const int32_t *add_w, void *result);
sp_status sp_apply_batch_finish(sp_graph *g, const void *result_host, sp_batch_stats *stats);

/* A CUDA graph holding one recorded sp_apply_batch_async call. */
typedef struct sp_exec sp_exec;

/*
 * Record sp_apply_batch_async(g, ...) into a CUDA graph (stream capture on
 * the graph's stream) and instantiate it.  The pointers and counts are fixed
 * in the recording: to apply another batch of the same sizes, write it into
 * the same device buffers and call sp_exec_launch.
 */
sp_status sp_capture_apply(sp_graph *g,
                           int64_t n_del, const int32_t *del_src, const int32_t *del_dst,
                           int64_t n_add, const int32_t *add_src, const int32_t *add_dst,
                           const int32_t *add_w, void *result, sp_exec **out);
/* Launch a recorded batch on the graph's stream (asynchronous). */
sp_status sp_exec_launch(sp_exec *e);
/* Release a recording (NULL is accepted). */
sp_status sp_exec_destroy(sp_exec *e);
/* Wait for all work queued on the graph's stream. */
sp_status sp_sync(sp_graph *g);

/*
 * Distances of k chosen vertices: dist_out[i] = dist[vertices[i]] (SP_INF if
 * unreachable).  Both arrays are host or device memory (on_device).  One
 * gather kernel; the call returns when the values are in dist_out.
 */
sp_status sp_query(sp_graph *g, int32_t k, const int32_t *vertices, int32_t *dist_out,
                   int on_device);

/*
 * Blocks of the persistent repair loops (one per SM at most; 0 = one per
 * SM).  A server running several graphs at once gives each a share of the
 * SMs so their loops can be resident together.
 */
sp_status sp_set_loop_blocks(sp_graph *g, int32_t blocks);

/* ------------------------------------------------------------------------
 * Serving runtime: a request loop over several resident graphs.
 *
 * Update batches and distance queries are submitted per graph and answered
 * asynchronously.  Requests of one graph run in submission order; requests
 * of different graphs run concurrently on n_slots worker slots (one CUDA
 * stream each), so their work overlaps on the device and a request that
 * arrives while others are running starts as soon as a slot is free
 * (continuous batching).  Graphs are admitted by an HBM budget, counting
 * each graph at the upper bound of its footprint (sp_footprint_bound, with
 * batch buffers reserved for max_batch_updates) or at its measured size if
 * that is larger (its spare pool grew): when a request needs a graph that
 * is not resident, idle resident graphs are evicted least-recently-used
 * (their edge set, distances and parents are checkpointed to host memory)
 * until the graph fits, and the graph is rebuilt from its checkpoint with
 * its distances restored by sp_set_dist (checked exact; recomputed from the
 * source if the check fails).  No request starts while the resident graphs
 * are over the budget; a request that can fit by no eviction fails with
 * SP_ENOMEM_BUDGET.  Each graph's cooperative kernels use a share of
 * SMs/n_slots blocks, each block an SM of its own, so the grids of all slots
 * are resident at once.  Distances are unique, so a query's answer does not
 * depend on the mix it ran in.
 * ---------------------------------------------------------------------- */
typedef struct sp_server sp_server;

typedef struct {
    int64_t hbm_budget_bytes;  /* device bytes all resident graphs may hold  */
    int32_t n_slots;           /* requests in flight on the GPU at once      */
    int32_t loop_blocks;       /* persistent-loop blocks per graph (0: SMs/n_slots) */
    float slack;               /* per-row slack of every graph               */
    int32_t delta;             /* near-far width of every graph (0 = off)    */
    int64_t max_batch_updates; /* largest batch a request may carry; batch
                                  buffers are reserved for it (0: 1,048,576) */
} sp_server_config;

typedef struct {
    int32_t status;            /* sp_status of the request                   */
    int32_t kind;              /* 0 = batch, 1 = query                       */
    int32_t graph;
    int32_t slot;
    int64_t updates;           /* deletions + insertions of a batch          */
    double submit_ms, start_ms, done_ms;   /* server clock                   */
    int32_t loaded;            /* 1 if the graph was (re)loaded for it       */
    double gpu_start_ms, gpu_done_ms;   /* the request's work on the device:
                                  CUDA events on its graph's stream, ms since
                                  the server was created (-1: none ran)      */
} sp_request_info;

typedef struct {
    int64_t resident_bytes, max_resident_bytes;
    int64_t loads, evictions, batches, queries, updates;
    int32_t resident_graphs, registered_graphs;
    int64_t recoveries;        /* batches whose repair hit a device bound and
                                  whose distances were recomputed from the source */
    int64_t restores;          /* reloads whose distances came from the
                                  checkpoint (sp_set_dist), not a recompute   */
    double load_ms, evict_ms;  /* host time spent loading / evicting graphs  */
} sp_server_stats;

sp_status sp_server_create(const sp_server_config *cfg, sp_server **out);
sp_status sp_server_destroy(sp_server *s);
/* Register a graph (host CSR, copied) with its source; it is loaded on
 * demand.  SP_ENOMEM_BUDGET if it alone would not fit the budget. */
sp_status sp_server_add_graph(sp_server *s, int32_t n, int64_t m, const int64_t *row_off,
                              const int32_t *col, const int32_t *w, int32_t source,
                              int32_t *graph_id);
/* Submit a batch (host arrays, copied); *request_id identifies it.
 * SP_EINVAL if it carries more than max_batch_updates updates. */
sp_status sp_server_submit_batch(sp_server *s, int32_t graph_id,
                                 int64_t n_del, const int32_t *del_src, const int32_t *del_dst,
                                 int64_t n_add, const int32_t *add_src, const int32_t *add_dst,
                                 const int32_t *add_w, int64_t *request_id);
/* Submit a query for k vertices (host array, copied). */
sp_status sp_server_submit_query(sp_server *s, int32_t graph_id, int32_t k,
                                 const int32_t *vertices, int64_t *request_id);
/* Wait up to timeout_ms (< 0: no limit) for a request; fills *info and, for
 * a query, dist_out[k].  SP_ETIMEOUT if it is not done in time. */
sp_status sp_server_wait(sp_server *s, int64_t request_id, sp_request_info *info,
                         int32_t *dist_out, int32_t timeout_ms);
/* Wait for every submitted request. */
sp_status sp_server_drain(sp_server *s);
sp_status sp_server_stats_get(sp_server *s, sp_server_stats *out);
/* Current distances of a graph (loads it if needed), host array of n. */
sp_status sp_server_get_dist(sp_server *s, int32_t graph_id, int32_t *dist);

/* ------------------------------------------------------------------------
 * Dynamic PageRank (paper, appendix listing "Dynamic PR coded in StarPlat
 * DSL": staticPR, DynPR with Decremental / Incremental; Section 7 reports it
 * beside SSSP).  Single precision, as the listing's propNode<float>.
 *
 * A Jacobi step over a vertex set S sets, for every v in S,
 *     pr[v] = (1 - damping) / n + damping * sum_{u -> v} pr[u] / outdeg(u)
 * (vertices without out-edges pass no rank on); steps repeat until
 * sum_{v in S} |pr'[v] - pr[v]| <= beta or max_iter steps have run.
 * ---------------------------------------------------------------------- */

/* staticPR: all ranks start at 1/n and S is every vertex.  Sets the PageRank
 * settings used by later batches.  SP_EINVAL for damping outside [0, 1],
 * beta < 0 or max_iter < 1.  stats (nullable): rounds_push = Jacobi steps,
 * relaxed_edges = in-edges pulled. */
sp_status sp_pr_init(sp_graph *g, float damping, float beta, int32_t max_iter,
                     sp_batch_stats *stats);

/*
 * DynPR for one batch, same arguments and batch semantics as
 * sp_apply_batch.  First the deletions: their destinations are flagged, the
 * flags spread along out-edges to every reachable vertex of the current
 * graph (propagateNodeFlags), the deletions are merged into both stores,
 * and Jacobi steps run over the flagged vertices from their current ranks.
 * Then the same for the insertions on the graph after the deletions.
 * Unflagged vertices keep their ranks.  The whole batch is validated before
 * either phase (SP_EINVAL leaves the graph and the ranks unchanged).
 * Requires sp_pr_init (else SP_ESTATE).  SSSP distances stop being valid
 * once edges change (sp_sssp_init restores them), and an SSSP batch that
 * changes edges ends the ranks' validity (sp_pr_init restores them).
 * stats (nullable): affected = vertices flagged over both phases,
 * rounds_inval = flag-propagation rounds, rounds_push = Jacobi steps,
 * relaxed_edges = in-edges pulled; the batch counters as sp_apply_batch.
 */
sp_status sp_pr_apply_batch(sp_graph *g, int64_t n_del, const int32_t *del_src,
                            const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                            const int32_t *add_dst, const int32_t *add_w,
                            int inputs_on_device, sp_batch_stats *stats);

/* Current ranks (n floats) into host or device memory; SP_ESTATE without
 * valid ranks. */
sp_status sp_pr_get(const sp_graph *g, float *pr, int out_on_device);

/* ------------------------------------------------------------------------
 * Dynamic triangle count (paper, appendix listing "Dynamic TC coded in
 * StarPlat DSL": staticTC, Decremental, Incremental, DynTC).  The graph is
 * read as undirected and must store every edge in both directions; every
 * batch must list every updated pair in both directions.
 * ---------------------------------------------------------------------- */

/* staticTC: for every vertex v, the pairs of neighbours u < v < w with u -> w
 * an edge (every triangle once).  SP_EINVAL if some edge lacks its reverse
 * (the count is then not kept). */
sp_status sp_tc_init(sp_graph *g, int64_t *count);

/*
 * DynTC for one batch (arguments and batch semantics as sp_apply_batch):
 * the applied deletions' corrections are counted on the graph before the
 * merge and subtracted, the applied insertions' on the graph after it and
 * added; *count receives the triangle count of the new graph.  SP_EINVAL
 * (nothing changes) if an update's reverse is missing from the batch;
 * SP_ESTATE without sp_tc_init.  Changing edges ends the validity of SSSP
 * distances and PageRank ranks, and SSSP or PageRank batches that change
 * edges end the count's (sp_tc_init restores it).  stats: the batch
 * counters as sp_apply_batch; affected = triangle sightings counted.
 */
sp_status sp_tc_apply_batch(sp_graph *g, int64_t n_del, const int32_t *del_src,
                            const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                            const int32_t *add_dst, const int32_t *add_w,
                            int inputs_on_device, int64_t *count, sp_batch_stats *stats);

/*
 * sp_apply_batch runs its kernels (eight per batch) as a cached CUDA graph
 * when a batch has the same shape (deletion and insertion counts, stats or
 * not) as the one before it: one graph launch replaces the kernel launches.
 * Device inputs are read where they are (the three kernels that read them
 * are pointed at this call's arrays before the launch); host inputs are
 * first moved to internal buffers.  The graph is rebuilt when a buffer or a
 * setting changes.  on = 0 turns it off (every call launches kernels one by
 * one); the default is 1.  Results do not depend on it.  Requires a
 * non-default stream (graphs are never used on the legacy stream).
 */
sp_status sp_set_batch_graphs(sp_graph *g, int32_t on);

/*
 * Loop counters of the last call, for tuning: out[0] push rounds, [1] of
 * them run by a single block, [2] single-block episodes, [3] near-far
 * splits, [4] far-pile entries moved back, [5] invalidation rounds, [6] of
 * them pointer-jumping passes, [7] ns spent in single-block rounds, [8] ns
 * spent in the push loop, [9] the bound that ended the last call early (0
 * none, 1 a round or pass cap, 2 a barrier wait), [10] where it was hit (1
 * a loop's round cap, 2 a loop's grid barrier, 3 the wait for a
 * single-block episode, 4 the batch sort's grid barrier, 5 the count pass's
 * grid barrier), [11] the round, barrier index or episode there, [12]
 * block-local sub-rounds of the pool schedule (summed over blocks), [13]
 * entries appended to the block pools, [14] ns block 0 spent in block-local
 * sub-rounds, [15] block 0's block-local sub-rounds.  k (<= 16) entries
 * are written; the figures are those of the last synchronous call.
 */
sp_status sp_loop_counters(const sp_graph *g, int64_t *out, int32_t k);

/*
 * Test hook of the bounded waits (the failure detection of the repair
 * loops' termination bound, Section 3.2's fixedPoint run on the device):
 * from now on thread block 0 does not arrive at the grid barriers of one
 * wait site -- 2 the repair loops' barrier, 4 the batch sort's, 5 the count
 * pass's -- so every wait of that barrier runs out after the wait bound of
 * sp_set_limits and the call returns SP_ETIMEOUT with that site in
 * sp_loop_counters.  Nothing faults or hangs: each wait is bounded.  0
 * turns it off.  SP_EINVAL for any other site.
 */
sp_status sp_inject_missed_arrival(sp_graph *g, int32_t site);

/* Name of the CUDA error behind the handle's last SP_ECUDA from a failed
 * launch ("cudaSuccess" if none); static storage. */
const char *sp_last_cuda_error(const sp_graph *g);

/* Static name of a status code. */
const char *sp_status_str(sp_status s);

/* Library version as "major.minor.patch". */
const char *sp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SP_H */
