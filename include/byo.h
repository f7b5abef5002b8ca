/*
 * byo.h -- C ABI of libbyo.so, a GB300 (sm_103a) implementation of the graph
 * container API and the driving graph algorithms of BYO (Wheatman et al.,
 * "BYO: A Unified Framework for Benchmarking Large-Scale Graph Containers",
 * arXiv 2405.11671).
 *
 * Conventions for every call
 *   - Pointers are DEVICE pointers owned by the caller, unless the parameter
 *     name starts with host_.  The library owns only what a byo_graph holds
 *     (the container and its scratch) and frees it in byo_graph_destroy.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it; calls that return a host value or a
 *     device-side status synchronise that stream before returning.
 *   - Every call returns a byo_status; BYO_OK is 0.  byo_last_error() gives a
 *     message for the last failure on the calling host thread.  Nothing is
 *     thrown across the ABI and the library never exits the process.
 *   - Vertex ids are uint32 in [0, n); "INF" is 0xFFFFFFFF.
 *   - A byo_graph may be read by several calls at once only if they run on
 *     the same stream: its scratch is shared.
 */
#ifndef BYO_H
#define BYO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum byo_status {
  BYO_OK = 0,
  BYO_ERR_INVALID_ARG = 1,   /* bad pointer, size, id >= n, or flag combination */
  BYO_ERR_OUT_OF_MEMORY = 2, /* a device allocation failed; nothing was changed */
  BYO_ERR_CUDA = 3,          /* a CUDA runtime call or a kernel launch failed */
  BYO_ERR_TIMEOUT = 4,       /* a device-side wait gave up (BYO_TIMEOUT_MS, default 10000) */
  BYO_ERR_UNSUPPORTED = 5,   /* e.g. a batch update on a static CSR */
  BYO_ERR_NOT_SYMMETRIC = 6  /* BYO_SYMMETRIZE not given and some (u,v) lacks (v,u) */
} byo_status;

#define BYO_INF 0xFFFFFFFFu

/* byo_graph_build flags */
#define BYO_CSR 0x1u        /* static compressed sparse row container */
#define BYO_DYNAMIC 0x2u    /* dynamic blocked-adjacency container (batch updates) */
#define BYO_SYMMETRIZE 0x4u /* store every input pair (u,v) also as (v,u) */
#define BYO_OFFSETS64 0x8u  /* CSR offsets as uint64 even when m < 2^32 */
#define BYO_DYN_NO_INLINE 0x10u /* BYO_DYNAMIC without the inline head: every list in pool blocks */
#define BYO_COMPRESSED 0x20u    /* BYO_CSR with difference-encoded, byte-coded lists (BFS, degree, export) */
#define BYO_DYN_HASH 0x40u      /* BYO_DYNAMIC with unsorted lists, per-run hash indexes and semisorted batches */

typedef struct byo_graph byo_graph;

/* Message for the last failed call on this host thread ("" if none). */
const char* byo_last_error(void);

/*
 * Build a graph container from k raw pairs src[i] -> dst[i] (device arrays).
 * BYO_CSR builds the static CSR; BYO_DYNAMIC the blocked adjacency (a 64-byte
 * record per vertex with up to 12 neighbours inline -- the inline optimisation
 * of Section 4.1 -- else a run of 128-byte blocks from a device pool), which
 * accepts byo_insert_batch / byo_delete_batch.  BYO_DYN_NO_INLINE (with
 * BYO_DYNAMIC only) keeps every non-empty list in pool blocks, for the
 * inline-head ablation.  BYO_DYN_HASH (with BYO_DYNAMIC only) is the
 * hashed-blocks design of DHB (Section 5.2) with the semisort-only batch form
 * of Section 4.1: the same records, inline head and runs, but each list kept
 * in insertion order, a list in a run of C ids indexed by an open-addressing
 * table of 2C slots (id and position), and each batch grouped by source with
 * a counting semisort instead of being sorted; every algorithm runs on it
 * unchanged (levels, labels and counts are order-free; PageRank sums in list
 * order, within its tolerance).  BYO_COMPRESSED (with BYO_CSR only) keeps the CSR
 * offsets and stores each list as the paper's compressed graphs do (Section 2,
 * Section 6.5): the first neighbour relative to the vertex (2|u0 - v| +
 * (u0 < v)), then the gaps, each in 7-bit groups least significant first with
 * the 0x80 bit on all but a value's last byte.  A compressed container
 * supports byo_bfs, byo_degree, byo_graph_export_csr and byo_space; the other
 * algorithms return BYO_ERR_UNSUPPORTED.
 * Follows the graph model of Section 3 (vertices 0..n-1, a neighbour SET per
 * vertex, Section 3.1) and the CSR layout named in Section 4.2: duplicate
 * pairs collapse, self-loops are dropped, neighbours are stored ascending.
 * With BYO_SYMMETRIZE each pair is stored in both directions; without it the
 * input must already be symmetric (BYO_ERR_NOT_SYMMETRIC otherwise), since
 * every algorithm here is for undirected graphs (Section 6.2).
 * Offsets are uint64 when BYO_OFFSETS64 is set or m >= 2^32, else uint32.
 * The input arrays are only read; *out receives a new handle.
 * Synchronises the stream (to learn m).  Errors: INVALID_ARG (NULL pointers
 * with k > 0, id >= n, no container flag), OUT_OF_MEMORY, CUDA.
 */
byo_status byo_graph_build(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k, uint32_t flags,
                           void* stream, byo_graph** out);

/* Bytes the container itself occupies (the space measure of the paper's
 * container comparison, Section 6.5): for the CSR, the offsets and the
 * neighbour ids ((n+1) x 4 or 8 + 4m); for the dynamic container, the 64-byte
 * vertex records and the 128-byte blocks of the runs its lists hold (free pool
 * capacity is not counted), plus 512 bytes of index slots per block with
 * BYO_DYN_HASH; for the compressed container, the offsets, the
 * byte offsets ((n+1) x 8), the code bytes and, for lists of more than 4,096
 * values, a 16-byte checkpoint every 4,096 values (where the value's code
 * starts and the id before it, so that several warps can decode one long
 * list) plus 12 bytes per such list.  Library scratch is not included.  Synchronises
 * the stream.  Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
byo_status byo_space(const byo_graph* g, uint64_t* host_bytes, void* stream);

/* The byte codes of a BYO_COMPRESSED container: byte offsets boff[n+1] (device,
 * uint64) and, when bytes is non-NULL, the boff[n] code bytes (device);
 * *host_nbytes receives boff[n].  Synchronises the stream.  Errors:
 * INVALID_ARG, UNSUPPORTED (not a compressed container), CUDA. */
byo_status byo_export_codes(const byo_graph* g, uint64_t* boff, uint8_t* bytes, uint64_t* host_nbytes, void* stream);

/* Free a handle and everything it owns (NULL is accepted).  Synchronises the device. */
byo_status byo_graph_destroy(byo_graph* g);

/* num_vertices() of the GraphContainer API (Section 4.2). */
byo_status byo_num_vertices(const byo_graph* g, uint32_t* host_n);

/* num_edges() of the GraphContainer API (Section 4.2): stored directed entries m
 * (2x the undirected edge count).  Kept as graph metadata (Section 4.3). */
byo_status byo_num_edges(const byo_graph* g, uint64_t* host_m);

/* degree(i) of the GraphContainer API (Section 4.2) for k vertex ids vs[]
 * (device), written to out[k]; vs == NULL means all n vertices (out[n]).
 * Ids >= n give BYO_ERR_INVALID_ARG (checked on the device; synchronises). */
byo_status byo_degree(const byo_graph* g, const uint32_t* vs, uint64_t k, uint32_t* out, void* stream);

/*
 * Batch updates of a BYO_DYNAMIC container: insert_sorted_batch and
 * delete_sorted_batch of the GraphContainer API (Section 4.2).  The batch is k
 * raw device pairs in any order; as BYO does, the library sorts it first (with
 * BYO_DYN_HASH it only groups it by source, Section 4.1's semisort form).  Set
 * semantics (Section 3.1): each pair is applied in both directions, self-loops
 * are ignored, duplicates collapse, inserting a present edge or deleting an
 * absent one changes nothing.  num_edges() and degree() reflect the batch when
 * the call returns.  Synchronises the stream.  Errors: UNSUPPORTED (static
 * CSR), INVALID_ARG (NULL arrays with k > 0, id >= n), OUT_OF_MEMORY, CUDA.
 */
byo_status byo_insert_batch(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k, void* stream);
byo_status byo_delete_batch(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k, void* stream);

/* Copy the container out as a CSR: offsets[n+1] (uint64) and col[m], neighbours
 * ascending (a BYO_DYN_HASH container's lists are sorted on the way out).  For
 * a dynamic container this is the snapshot used to compare its contents after
 * each batch. */
byo_status byo_graph_export_csr(const byo_graph* g, uint64_t* offsets, uint32_t* col, void* stream);

/* ------------------------------------------------------------------------ */
/* Schedules: which edgeMap direction (Section 3.2, sparse/push vs           */
/* dense/pull, chosen from degree and num_edges as Section 6.3 describes)   */
/* and which degree bins a push iteration uses.                             */
typedef enum byo_sched_mode {
  BYO_SCHED_HEURISTIC = 0, /* Beamer-style direction switch with alpha/beta below */
  BYO_SCHED_LEARNED = 1,   /* the schedule network picks each iteration (needs mlp) */
  BYO_SCHED_PUSH = 2,      /* sparse edgeMap every iteration */
  BYO_SCHED_PULL = 3,      /* dense edgeMap every iteration */
  BYO_SCHED_FIXED = 4      /* the action below at every iteration */
} byo_sched_mode;

/* Schedule actions: 0 dense (pull); 1 sparse (push) with the thr_thread /
 * thr_warp bins below; 2 push with bins 4 / 128; 3 push with bins 64 / 4096;
 * 4 push run by a single CTA for as many consecutive levels as the schedule
 * keeps choosing it (no grid-wide barrier between those levels). */
#define BYO_NUM_ACTIONS 5

typedef struct byo_mlp byo_mlp;

typedef struct byo_sched {
  uint32_t mode;       /* byo_sched_mode */
  uint32_t thr_thread; /* push: degree < thr_thread -> one thread per vertex (power of two, >= 1) */
  uint32_t thr_warp;   /* push: degree < thr_warp -> one warp per vertex, else CTA chunks (power of two) */
  float alpha;         /* heuristic: push -> pull when frontier edges > unvisited edges / alpha */
  float beta;          /* heuristic: pull -> push when frontier vertices < n / beta */
  const byo_mlp* mlp;  /* LEARNED only */
  uint32_t action;     /* FIXED only: 0 .. BYO_NUM_ACTIONS-1 */
  uint32_t flags;      /* BYO_SCHED_NO_EARLY_EXIT | BYO_SCHED_SEQUENTIAL_MAPS (API ablations) */
} byo_sched;

/* API ablations (Section 6.3 measures BYO without the early-exit map and
 * without the parallel map): results are the same, only the work changes.
 *   BYO_SCHED_NO_EARLY_EXIT    dense (pull) iterations read every neighbour of
 *                              an unvisited vertex instead of stopping at the
 *                              first one in the frontier (the parent is still
 *                              that first one);
 *   BYO_SCHED_SEQUENTIAL_MAPS  a vertex's neighbour list is only ever walked
 *                              by one thread (no warp- or CTA-wide map of one
 *                              list, no single-CTA push levels). */
#define BYO_SCHED_NO_EARLY_EXIT 0x1u
#define BYO_SCHED_SEQUENTIAL_MAPS 0x2u

/* ------------------------------------------------------------------------ */
/* Schedule network (not in the paper: it only picks among equivalent       */
/* execution paths, so results never depend on it).  A 12 -> 32 -> 32 -> 5  */
/* ReLU MLP over the frontier features of one BFS iteration (the fields of   */
/* byo_bfs_iter), outputs = scores of the BYO_NUM_ACTIONS schedule actions.   */
/* Parameters are FP32, packed W1[32][12], b1[32], W2[32][32], b2[32],        */
/* W3[5][32], b3[5].                                                         */

/* Number of FP32 parameters (1,637). */
uint32_t byo_mlp_num_params(void);

/* New network with He-uniform weights drawn from `seed` (biases zero). */
byo_status byo_mlp_create(uint64_t seed, byo_mlp** out);
byo_status byo_mlp_destroy(byo_mlp* m);

/* Copy the parameters to / from a HOST array of byo_mlp_num_params() floats
 * (save / load).  Setting parameters resets the optimiser state. */
byo_status byo_mlp_get_params(const byo_mlp* m, float* host_params);
byo_status byo_mlp_set_params(byo_mlp* m, const float* host_params);

/* Loss and gradient on a batch: X[B][12] features, y[B] action labels, w[B]
 * sample weights (nullable = 1), all device arrays.  L = sum_i w_i *
 * CE(softmax(z_i), y_i) / sum_i w_i.  grad (nullable, device, num_params
 * floats) receives dL/dparams; *host_loss (nullable) the loss (synchronises). */
byo_status byo_mlp_loss_grad(byo_mlp* m, const float* X, const int32_t* y, const float* w, uint32_t B,
                             float* grad, float* host_loss, void* stream);

/* `epochs` full-batch Adam steps (lr, betas 0.9/0.999) on the same loss;
 * *host_loss (nullable) receives the final loss (synchronises). */
byo_status byo_mlp_train(byo_mlp* m, const float* X, const int32_t* y, const float* w, uint32_t B,
                         uint32_t epochs, float lr, float* host_loss, void* stream);

/* actions[i] = argmax of the network output for X[i] (device arrays). */
byo_status byo_mlp_predict(const byo_mlp* m, const float* X, uint32_t B, int32_t* actions, void* stream);

/* Defaults: HEURISTIC, thr_thread 16, thr_warp 1024, alpha 15, beta 18, action 1, flags 0. */
byo_sched byo_sched_default(void);

/*
 * Breadth-first search (the paper's BFS, Section 6.2, expressed with edgeMap
 * over a vertexSubset, Section 3.2) from each of num_sources sources, one after
 * another.  levels[i*n + v] = hop distance of v from sources[i], INF if
 * unreached.  parents (nullable) [i*n + v] = a neighbour of v one level closer
 * (sources[i] for the source itself, INF if unreached); push iterations may
 * pick any such neighbour, pull iterations pick the first one in ascending id
 * order.  sources is a HOST array.  sched NULL = byo_sched_default().
 * The whole traversal of one source runs in one persistent cooperative launch:
 * no host round trip per iteration.  Synchronises the stream.
 * Errors: INVALID_ARG (source >= n, NULL levels), TIMEOUT (a device-side wait
 * or the traversal itself exceeded BYO_TIMEOUT_MS), CUDA.  The status is the
 * one the first failing source's kernel wrote; the sources after it are not
 * traversed and their rows of levels/parents are unspecified.  The graph's
 * BFS state is reset before the call returns, so the next call runs normally.
 */
byo_status byo_bfs(const byo_graph* g, const uint32_t* host_sources, uint32_t num_sources, uint32_t* levels,
                   uint32_t* parents, const byo_sched* sched, void* stream);

/* Per-iteration record of the last byo_bfs source on this graph.  These are
 * the schedule features (and, with t_ns, the training data of the schedule
 * network). */
typedef struct byo_bfs_iter {
  uint32_t level;           /* frontier level processed */
  uint32_t direction;       /* 0 = pull, 1 = push */
  uint32_t action;          /* schedule action (0 .. BYO_NUM_ACTIONS-1) */
  uint32_t frontier;        /* |F| */
  uint64_t frontier_edges;  /* sum of degrees over F */
  uint64_t edges_examined;  /* neighbour ids read in this iteration */
  uint64_t unvisited_edges; /* sum of degrees over vertices not yet visited (F excluded) */
  uint32_t unvisited;       /* vertices not yet visited (F excluded) */
  uint32_t hist[4];         /* |F| split by degree: < 4, < 32, < 256, >= 256 */
  uint32_t reserved;
  uint64_t t_ns;            /* device time of the iteration (globaltimer) */
} byo_bfs_iter;

/* Copy up to cap records (host array) of the last BFS source; *host_count gets
 * the number of iterations.  Synchronises the stream. */
byo_status byo_bfs_trace(const byo_graph* g, byo_bfs_iter* host_records, uint32_t cap, uint32_t* host_count,
                         void* stream);

/*
 * Connected components (the paper's connectivity algorithm, Section 6.2):
 * labels[v] = the minimum vertex id of v's component.  Concurrent union-find,
 * hooking the larger root under the smaller, with the edges taken in Afforest
 * order (each vertex's first two neighbours, then every neighbour of the
 * vertices outside the largest sampled component), then full path
 * compression.  labels is caller-owned device memory of n entries and doubles
 * as the union-find parent array.  Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA.
 */
byo_status byo_cc(const byo_graph* g, uint32_t* labels, void* stream);

/*
 * PageRank (named in Section 6.2).  ranks[v] after `iters` iterations of
 *   p_0 = 1/n,  p_{t+1}(v) = (1-d)/n + d*( sum_{u in N(v)} p_t(u)/deg(u) + D_t/n ),
 * D_t = sum of p_t over degree-0 vertices.  Contributions p/deg are FP32 and
 * summed per vertex with compensated (Neumaier) FP32 arithmetic; the dangling
 * mass D_t and the L1 residual are reduced in FP64.  The iterations run on a
 * copy of the graph relabelled by degree order that the call builds (library
 * scratch of 4m + 16n bytes, kept with the graph); each vertex's sum keeps its
 * neighbour order.  host_residual (nullable) receives
 * sum_v |p_iters(v) - p_{iters-1}(v)|; if non-NULL the call synchronises.
 * Errors: INVALID_ARG (d outside [0,1], NULL ranks), OUT_OF_MEMORY, CUDA.
 */
byo_status byo_pagerank(const byo_graph* g, float damping, uint32_t iters, float* ranks, double* host_residual,
                        void* stream);

/*
 * Triangle count (Section 4.4: filter to a DAG, then intersect).  Each edge is
 * kept in the direction of increasing (degree, id); the count is the sum over
 * DAG edges u->v of |N+(u) intersect N+(v)|.  The DAG is stored with vertices
 * relabelled by that order; each DAG edge is intersected from the side with
 * the shorter out-list, the other side's N+ held in shared memory (staged by
 * TMA bulk copies and hashed, or a bitmap of the ranks above a high-degree
 * vertex); out-lists of 32..16384 ids are sorted by rank first, so that a
 * walked out-list of a lower-ranked endpoint starts after the other endpoint.
 * *host_count receives the number of triangles; synchronises.  The
 * environment variables BYO_TC_LIGHT_MAX, BYO_TC_WINDOW, BYO_TC_BITMAP_BITS,
 * BYO_TC_WARP_SORT_MAX and BYO_TC_SORT_MAX can only lower internal limits (so
 * that tests reach every code path on small graphs); the count is the same.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, TIMEOUT, CUDA.
 */
byo_status byo_tc(const byo_graph* g, uint64_t* host_count, void* stream);

/* Runs byo_tc and reports its intersection work (host_work3, host array of 3):
 * [0] sum_c d+(c)^2 and [1] sum_c d-(c) d+(c) -- together the out-list ids a
 * merge of both lists of every DAG edge reads -- and [2] the ids this library
 * walks (sum over DAG edges of the shorter out-list, only its ids ranked above
 * the other endpoint when that list is sorted).  Synchronises. */
byo_status byo_tc_work(const byo_graph* g, uint64_t* host_work3, void* stream);

/*
 * Single-source betweenness centrality (BC in the table of algorithms of
 * Section 6.2), by Brandes' accumulation: the BFS of byo_bfs from `source`
 * gives the levels; sigma[v] = number of shortest source-v paths (sigma of the
 * source = 1, summed over the neighbours one level closer, level by level);
 * delta[v] = sum over the neighbours w one level deeper of
 * sigma[v] / sigma[w] * (1 + delta[w]), from the deepest level up: the
 * dependency of the source on v.  delta[source] = 0; unreached vertices get
 * sigma = delta = 0 and level INF.  sigma, delta: device FP64 arrays of n
 * entries; levels: device uint32[n] (nullable: then library scratch).  Both
 * sweeps gather over each vertex's own list (no floating-point atomics), so
 * the results do not depend on scheduling; path counts are exact while below
 * 2^53.  Synchronises the stream.
 * Errors: INVALID_ARG (source >= n, NULL sigma/delta), OUT_OF_MEMORY,
 * TIMEOUT, CUDA.
 */
byo_status byo_bc(const byo_graph* g, uint32_t source, uint32_t* levels, double* sigma, double* delta, void* stream);

/* ------------------------------------------------------------------------ */
/* Many graphs at once.  byo_batch_build stores num_graphs graphs as one      */
/* container over their disjoint union: member i owns the global ids          */
/* [base_i, base_i + n_i), base_i = n_0 + ... + n_{i-1} (byo_batch_member_base */
/* returns it).  Every call of this header then works on all members at once  */
/* (e.g. byo_cc labels every member's components by their minimum global id). */
/*   host_n[i], host_k[i]  vertices and raw pairs of member i (host arrays)    */
/*   src, dst              the members' pairs concatenated, LOCAL ids (device) */
/*   flags                 as for byo_graph_build                             */
/* Errors: INVALID_ARG (a local id >= n_i, total vertices >= 2^32 - 1), OOM,  */
/* CUDA.  Synchronises the stream.                                           */
byo_status byo_batch_build(uint32_t num_graphs, const uint32_t* host_n, const uint64_t* host_k, const uint32_t* src,
                           const uint32_t* dst, uint32_t flags, void* stream, byo_graph** out);
byo_status byo_batch_member_base(const byo_graph* g, uint32_t i, uint32_t* host_base);

/*
 * Multi-source BFS: num_sources (1..64) sources in EVERY member, traversed
 * together with one bit per source (edgeMap over 64 frontiers at once, Section
 * 3.2), top-down or bottom-up per level, in one persistent launch for the whole
 * batch.  host_sources[i * num_sources + j] is source j of member i as a LOCAL
 * id (a plain graph is a batch of one).  levels[j * n + v] (device, n = total
 * vertices) = hop distance of global vertex v from source j of v's member, INF
 * if unreached.  sched (nullable): only alpha is used -- a level runs
 * top-down while its frontier's edges * alpha < the edges not yet visited.
 * Synchronises the stream.  Errors: INVALID_ARG, TIMEOUT, CUDA.
 */
byo_status byo_msbfs(const byo_graph* g, const uint32_t* host_sources, uint32_t num_sources, uint32_t* levels,
                     const byo_sched* sched, void* stream);

/* ------------------------------------------------------------------------ */
/* BFS that allocates nothing (the paper has no counterpart; this is a       */
/* deployment variant of byo_bfs).  Some callers cannot allocate device      */
/* memory: code whose device memory belongs to another allocator (a          */
/* framework's caching allocator or a fixed arena handed out by the host     */
/* application), code under a hard memory budget that must not grow, and    */
/* latency-critical loops where cudaMalloc / cudaFree would synchronise the  */
/* device.  They cannot create a byo_graph either, since building one        */
/* allocates, so this call takes the CSR itself.                            */
/*                                                                          */
/* It runs the same persistent BFS kernel as byo_bfs for ONE source.  All    */
/* scratch lives in a fixed file-scope device array of 9,324,800 bytes,    */
/* sized for n <= BYO_NOALLOC_MAX_VERTICES; every GPU that loads the       */
/* library holds it until the process exits.  The call makes no cudaMalloc, */
/* cudaFree or other allocating call.                                       */
/*   n, m     vertices (1 <= n <= BYO_NOALLOC_MAX_VERTICES, else             */
/*            BYO_ERR_INVALID_ARG) and stored entries                        */
/*   offsets  device uint64[n+1]; col device uint32 ids, neighbours of each */
/*            vertex ascending, the graph symmetric without self-loops (as  */
/*            byo_graph_export_csr returns it); col must start on a 16-byte */
/*            boundary and be readable up to index m+3 (vector reads)       */
/*   levels   device uint32[n] out; parents device uint32[n] out or NULL;   */
/*            same meaning as byo_bfs                                        */
/*   sched    as for byo_bfs (NULL = default)                               */
/* The first call on a device looks up the array's device address (with     */
/* that device current) and caches it.  cudaDeviceReset discards the       */
/* array, so the cached address is stale afterwards: do not call this      */
/* entry point on a device after resetting it.  Every call shares the one  */
/* array: calls that overlap on the GPU (other streams, other host threads) */
/* race and must not be issued.  Every call ends by reading the kernel's    */
/* status word back to the host, so it synchronises the stream.            */
/* Errors: INVALID_ARG, TIMEOUT, CUDA (the status the kernel reported).     */
#define BYO_NOALLOC_MAX_VERTICES (1u << 20)
byo_status byo_bfs_noalloc(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* col, uint32_t source,
                           uint32_t* levels, uint32_t* parents, const byo_sched* sched, void* stream);

/* ------------------------------------------------------------------------ */
/* Tracing.  Every kernel launch of the library increments a process-wide    */
/* counter.  With profiling on, the main kernels of each call are bracketed  */
/* by CUDA events on the caller's stream; byo_profile_read resolves them     */
/* (synchronising) into per-kernel launch counts and device milliseconds.    */
typedef struct byo_kernel_stat {
  char name[48];
  uint64_t launches;
  double total_ms;
} byo_kernel_stat;

/* Kernels launched by this library in this process so far. */
uint64_t byo_kernel_launches(void);
byo_status byo_profile_enable(int on);
/* Drop every recorded timing. */
byo_status byo_profile_reset(void);
/* Up to cap per-kernel records (host array) accumulated since the last reset;
 * *host_count gets the number of distinct kernels. */
byo_status byo_profile_read(byo_kernel_stat* host_stats, uint32_t cap, uint32_t* host_count);

#ifdef __cplusplus
}
#endif

#endif /* BYO_H */
