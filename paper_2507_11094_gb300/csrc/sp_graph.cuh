// sp_graph.cuh -- host-side graph handle and the launch wrappers each
// translation unit provides to sp_api.cu.
#pragma once

#include "sp_internal.cuh"

namespace sp {

// Frontier expansion: every queued vertex reserves a range of the round's
// edge space when it is enqueued; the round is then processed in chunks of
// kChunk edges, one warp per chunk, 8 consecutive edges per lane.
constexpr int kChunk = 256;
constexpr int kEdgesPerLane = kChunk / 32;
// Vertices with at most kSmallDeg edges go to a frontier's small list and
// are expanded one lane per vertex; larger ones get edge ranges and chunks.
constexpr int kSmallDeg = 8;
constexpr int kLocalRoundCap = 4096;   // frontier edges of a single-block round
constexpr int kLoopThreads = 1024;      // one-pass frontier kernels (pull, add)
constexpr int kPersistThreads = 768;    // persistent fixedPoint loops: 80 registers a thread
// the push loop with block-local relaxation: a sub-round expands about a
// hundred pool entries per block, so fewer threads with more registers each
// (128) serve it better than 768 that spill
constexpr int kPoolThreads = 512;
// Co-residency of cooperative launches from several handles at once (the
// serving runtime's slots): a handle with a block share (sp_set_loop_blocks)
// launches every cooperative kernel with at most that many blocks, each with
// at least this much dynamic shared memory.  Two such blocks do not fit in
// one SM's 228 KB, so every cooperative block holds an SM to itself and the
// shares of all slots, summed, never ask for more SMs than the GPU has: each
// grid is resident in full whatever the others do, and no grid barrier can
// wait for a block that has no SM.
constexpr size_t kExclusiveSmem = 116 * 1024;

// Per-block staging area (shared memory) for appends to a queue or a far
// pile: warps append here with shared-memory atomics and the block publishes
// everything with one global atomic when it flushes, instead of one global
// atomic per warp on a single counter (those serialize at one L2 slice).
struct Stage {
  u32 n;        // entries staged
  u32 cap;
  u32 vmin;     // far piles: smallest distance staged
  u32 *v;       // [cap] vertices
  u32 *d;       // [cap] degrees (queues with edge ranges)
};

// A frontier queue: entries (v, first edge) in slot order, and for every
// chunk the slot of the entry holding the chunk's first edge.
struct Queue {
  int2 *ent = nullptr;
  u32 *owner = nullptr;
  unsigned long long *cnt = nullptr;   // count << 32 | edges (in Ctl)
  Stage *st = nullptr;                 // block staging, or direct appends
  u32 *sv = nullptr;                   // small list
  u32 *scnt = nullptr;
  Stage *sst = nullptr;
  u32 small = kSmallDeg;               // largest out-degree kept in the small list
};

// Block-local relaxation of the push loop: two lists of entries in shared
// memory, each entry (vertex, distance it was improved to, row start / 4,
// out-degree) for vertices with at most kPoolDeg out-edges.  A sub-round
// expands one list into the other; the block runs sub-rounds on its own
// (block barriers only) before it meets the others at the grid barrier.
constexpr int kPoolDeg = 16;            // largest out-degree a pool entry may have
constexpr u32 kPoolCap = 2048;          // entries per list
struct Pool {
  uint4 *e[2];
  u32 n[2];                             // appended so far (may pass kPoolCap)
};

// One touched (store, row) pair of a batch, after sorting.
struct Seg {
  u32 first, end;        // item range in the sorted batch
  int row;
  int dir;               // 0 = forward store, 1 = reverse store
  long long old_start;   // the row's active region before the merge
  long long dest;        // region the merged row is written to
  long long new_alt;     // the row's alternate region after the merge
  unsigned long long prefix;     // key bits of (store, row)
  unsigned long long base_pref;  // item_pref[first]
  int old_deg;
  int new_deg;
  int new_cap;
  int pad;
};

// Per-call buffers that grow on demand.
struct BatchBufs {
  long long cap_items = 0;
  u64 *keys = nullptr, *keys_alt = nullptr;
  u32 *vals = nullptr, *vals_alt = nullptr;
  unsigned char *flags = nullptr;   // per item: bit0 = applied, bit1 = edge was present
  u64 *item_pref = nullptr;         // exclusive prefix of the applied updates per item
  u32 *opos = nullptr;              // per item: old entries of its row with a smaller col
  // per item in the batch's own numbering (the sort carries that number as
  // its value): weight << 32 | edge present << 31 | position in the old row
  u64 *srch = nullptr;
  Seg *seg = nullptr;
  int2 *strips = nullptr;           // merge strips: (segment, first old entry)
  long long strips_cap = 0;
  void *tmp = nullptr;
  size_t tmp_bytes = 0;
  long long cap_in = 0;             // staging for host inputs
  int *in_del_src = nullptr, *in_del_dst = nullptr;
  int *in_add_src = nullptr, *in_add_dst = nullptr, *in_add_w = nullptr;
};

// Arguments of the frontier kernels.
struct LoopArgs {
  Ctl *ctl;
  Limits lim;
  Store fwd, rev;
  u64 *s;
  u32 *qflag;
  int2 *qent[3];         // frontier buffers (rotating)
  u32 *qown[3];
  u32 *qsv[3];           // their small lists
  u32 *asv;              // small list of A
  int2 *aent;            // affected list A (entries carry reverse edges)
  u32 *aown;
  u32 *fq[3];            // far piles of the near-far push (rotating)
  u32 *ftag;             // far dedupe tags
  u32 *jmp;              // pointer-jumping words of the invalidation (flag | ancestor)
  int n;
  // fused OnDelete mark (invalidation loop only); the flag loop takes its
  // seeds from del_dst
  const int *del_src, *del_dst;
  long long n_del;
  // PageRank flags: prflag[v] == ptag marks v for the current phase
  u32 *prflag;
  u32 ptag;
  // the invalidation's cut vertices; concurrent != 0: the invalidation runs
  // beside the store update, so it reads neither store (no frontier rounds)
  u32 *cut;
  int concurrent;
  // first stage of the push loop of a batch (before its first barrier): the
  // pull over the affected list A, and OnAdd over the sorted batch items
  int seed_pull;
  const u64 *keys;
  const u32 *vals;
  const unsigned char *flags;
  long long n_items;
  int bits;
};

}  // namespace sp

struct sp_graph {
  int n = 0;
  int bits = 1;                // id bits
  int device = 0;
  int num_sms = 0;
  float slack = 0.25f;
  cudaStream_t stream = nullptr;
  sp::Alloc al;
  sp::Store fwd, rev;
  long long m = 0;
  sp::u64 *s = nullptr;
  sp::u32 *qflag = nullptr;
  int2 *qent[3] = {nullptr, nullptr, nullptr};
  sp::u32 *qown[3] = {nullptr, nullptr, nullptr};
  sp::u32 *qsv[3] = {nullptr, nullptr, nullptr};
  sp::u32 *asv = nullptr;
  int2 *aent = nullptr;
  sp::u32 *aown = nullptr;
  sp::u32 *fq[3] = {nullptr, nullptr, nullptr};
  sp::u32 *ftag = nullptr;
  sp::u32 *jmp = nullptr;
  sp::u32 *cut = nullptr;       // cut vertices of the invalidation
  // side stream of the invalidation, which runs beside the store update
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaEvent_t fork0_ev = nullptr, search_ev = nullptr;   // the search beside the sort
  cudaEvent_t ev_inval[2] = {nullptr, nullptr};
  bool last_beside = false;     // the last timed call ran the invalidation beside
  // PageRank state (allocated by sp_pr_init): ranks in two buffers that
  // agree between calls, the pull accumulators, phase flags and settings
  float *pr[2] = {nullptr, nullptr};
  float *prc[2] = {nullptr, nullptr};   // pr / outdeg (Jacobi work buffers)
  float *pracc = nullptr;
  sp::u32 *prflag = nullptr;
  sp::u32 prtag = 0;
  int pr_state = 0;            // 0 = no ranks, 1 = valid
  float pr_damping = 0.85f, pr_beta = 1e-6f;
  int pr_max_iter = 100;
  // triangle count (sp_tc_init): the current count
  long long tc_count = 0;
  int tc_state = 0;            // 0 = no count, 1 = valid
  int32_t delta_user = 0;
  int32_t jump_round_user = 0;
  // cached CUDA graph of the batch pipeline (sp_apply_batch): replayed when
  // the same batch shape repeats; `gen` changes whenever a buffer moves or a
  // setting changes, which invalidates the cache
  unsigned long long gen = 1;
  int last_err = 0;                      // cudaError_t of the last failed launch
  int batch_graphs = 1;                  // 0 = never capture
  // one graph per batch shape; the phase timing events are nodes inside it
  cudaGraph_t bg_graph = nullptr;
  cudaGraphExec_t bg_exec = nullptr;
  cudaGraphNode_t bg_sort = nullptr, bg_inval = nullptr,   // nodes that read the inputs
                  bg_search = nullptr;
  bool bg_ready = false;
  int capturing = -1;                    // >= 0 while the pipeline is captured
  unsigned long long bg_gen = 0;
  long long bg_nd = -1, bg_na = -1;
  int bg_timed = -1, bg_launches = 0;
  long long last_nd = -1, last_na = -1;
  int last_timed = -1;
  int32_t local_edges_user = 4096;
  int32_t small_deg_user = sp::kSmallDeg;   // push frontiers' small-list bound
  int32_t pool_rounds_user = 0;             // block-local sub-rounds per push round
  int32_t miss_site_user = 0;               // test hook of the bounded waits
  // the sources of the last init (one, or the batched form's list on the
  // device), kept so that a batch that fails after the invalidation can
  // restore the distances without allocating
  int *src_dev = nullptr;
  int32_t n_src = 0;
  long long own_cap = 0;        // entries of each chunk-owner table
  sp::Ctl *ctl = nullptr;       // device
  sp::Ctl *ctl_host = nullptr;  // pinned
  int *out_dist = nullptr, *out_parent = nullptr;
  sp::BatchBufs bb;
  int source = -1;
  int state = 0;                // 0 none, 1 valid, 2 needs re-init
  sp::Limits lim{};
  int32_t max_rounds_user = 0;
  long long wait_ns_user = 0;
  int loop_blocks_push = 0, loop_blocks_inval = 0, loop_blocks_pool = 0;
  bool pool_wide = false;   // the pool schedule runs five-edge steps (launch_deg_mid)
  int sort_blocks = 0;          // co-resident blocks of the batch sort
  int count_blocks = 0;         // co-resident blocks of the count pass
  int loop_blocks_user = 0;
  cudaEvent_t ev[SP_NPHASE + 1] = {};
  long long async_ni = 0;       // items of the last enqueued async batch
  int async_launches = 0;
};

namespace sp {

// sp_store.cu
sp_status store_build(sp_graph *g, sp::Store *st, const long long *row_off_d,
                      const int *col_d, const int *w_d, long long m, int reverse,
                      int *launches);
sp_status store_export(sp_graph *g, const sp::Store *st, long long *row_off_d,
                       int *col_d, int *w_d, int *launches);
sp_status store_grow_pool(sp_graph *g, sp::Store *st, long long min_pool_slots);
sp_status ensure_owner_tables(sp_graph *g);
void launch_ctl_reset(sp_graph *g, int full, int *launches);
int count_blocks(int num_sms);
// the count pass; avoid_sms: SMs held by a cooperative grid running beside
// it, which its grid must leave free to be resident in full
void launch_count(sp_graph *g, long long n_items, int *launches, int avoid_sms = 0);
void launch_merge(sp_graph *g, long long n_items, int *launches);
void launch_finish(sp_graph *g, int *launches);
// sp_sort.cu: items, sort and segments of a batch in one cooperative launch
int batch_sort_blocks(int num_sms);
size_t batch_sort_tmp_bytes(int max_blocks);
cudaError_t launch_batch_sort(sp_graph *g, const int *ds, const int *dd, long long nd,
                              const int *as, const int *ad, const int *aw, long long na,
                              int *launches);
// the captured batch-sort / invalidation node of an instantiated graph,
// pointed at another batch of the same shape
const void *batch_sort_fn();
// The old-row searches of a batch's items (their positions, whether the
// edge is there, and their weights into bb.srch), for the count pass; they
// read only the old stores, so they may run beside the batch sort.
cudaError_t launch_search(sp_graph *g, const int *ds, const int *dd, long long nd,
                          const int *as, const int *ad, const int *aw, long long na,
                          int *launches, cudaStream_t stream);
const void *search_fn();
cudaError_t retarget_search(sp_graph *g, cudaGraphExec_t ex, cudaGraphNode_t node,
                            const int *ds, const int *dd, long long nd, const int *as,
                            const int *ad, const int *aw, long long na);
cudaError_t retarget_batch_sort(sp_graph *g, cudaGraphExec_t ex, cudaGraphNode_t node,
                                const int *ds, const int *dd, long long nd, const int *as,
                                const int *ad, const int *aw, long long na);
const void *inval_fn();
cudaError_t retarget_inval(sp_graph *g, cudaGraphExec_t ex, cudaGraphNode_t node, const int *ds,
                           const int *dd, long long nd, int concurrent);
void launch_check_batch(sp_graph *g, const int *ds, const int *dd, long long nd, const int *as,
                        const int *ad, const int *aw, long long na, int *launches);

// sp_frontier.cu
int loop_blocks(int which, int num_sms);
void launch_init(sp_graph *g, int source, int *launches);
void launch_init_multi(sp_graph *g, const int *src_d, int k, int *launches);
cudaError_t launch_inval(sp_graph *g, const int *ds, const int *dd, long long nd,
                         int *launches, int concurrent = 0, cudaStream_t stream = nullptr);
// push fixedPoint; for a batch (pull != 0 or n_items > 0) its first stage
// pulls over A and relaxes the applied insertions
cudaError_t launch_push(sp_graph *g, int *launches, int pull = 0, long long n_items = 0);
// blocks (one per SM) of an invalidation beside the store update
int inval_beside_blocks(const sp_graph *g);
void launch_unpack(sp_graph *g, int *dist_d, int *parent_d, int *launches);
// The pool kernel with five-edge steps once at least 1/64 of the vertices
// have 5..8 out-edges (counted by launch_deg_mid into ctl->deg_mid).
void launch_deg_mid(sp_graph *g, int *launches);
bool pool_wide_for(long long deg_mid, int n);
void launch_stage_inputs(sp_graph *g, const int *const src[5], int *const dst[5],
                         const long long cnt[5], int *launches);
// restore of exported distances: the exactness checks (status SP_EINVAL on a
// violation), then the packed state
void launch_state_check(sp_graph *g, const int *dist_d, const int *parent_d, int src,
                        int *launches);
void launch_state_pack(sp_graph *g, const int *dist_d, const int *parent_d, int *launches);
// sp_tc.cu
void launch_tc_sym_check(sp_graph *g, int *launches);
void launch_tc_static(sp_graph *g, int *launches);
void launch_tc_batch_sym(sp_graph *g, long long nb, int *launches);
void launch_tc_delta(sp_graph *g, long long nb, int kind, int *launches);
// PageRank
cudaError_t launch_flag(sp_graph *g, const int *dst, long long n, int *launches);
void launch_pr_fill(sp_graph *g, float value, int *launches);
void launch_pr_select(sp_graph *g, int all, int *launches);
cudaError_t launch_pr(sp_graph *g, int *launches);
void launch_gather(sp_graph *g, const int *vs_d, int k, int *out_d, int *launches);

}  // namespace sp
