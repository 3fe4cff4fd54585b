/*
 * gbbfs.h -- C ABI of the GB300 (sm_103a) breadth-first-search library.
 *
 * The method is the level-synchronous top-down BFS of Paredes, Riley and
 * Lujan, "Breadth First Search Vectorization on the Intel Xeon Phi":
 *   - problem statement (Sec. 3): given a graph G and a source s, explore the
 *     edges of G to reach every vertex reachable from s; the result is a BFS
 *     spanning tree given as a predecessor array P with P[s] = s (Alg. 1);
 *   - layers (Sec. 3): layer L_k holds the vertices at distance k from s;
 *     L_k is fully processed before L_{k+1}, in any order inside a layer;
 *   - one layer step (Alg. 2): for every u in the frontier and every v in
 *     Adj[u], if v is not yet visited, mark it, put it on the next frontier
 *     and set P[v] = u;
 *   - the visited set is a bitmap, vertex v at word v/32, bit v%32
 *     (Sec. 3.3.1, Listing 1).  Where two threads race on one word the paper
 *     restores the bitmap afterwards (Alg. 3); by default this library sets
 *     bits with a 32-bit atomic OR instead, and BFS_OPT_MODE 2 runs the
 *     paper's racy bitmap with its restoration pass.
 *
 * Graph layout: CSR with int32 row_offsets[n+1] ("colstarts" in Sec. 3.3.1)
 * and int32 col_idx[m] ("rows"): Adj[u] = col_idx[row_offsets[u] ..
 * row_offsets[u+1]-1].  Rows are read as directed out-edges; self-loops and
 * repeated entries are allowed and change nothing.
 *
 * Output conventions (readings of the paper, which writes "infinity" for an
 * unset predecessor, Sec. 3.1):
 *   level[v]  = number of edges on a shortest path s -> v, -1 if unreached;
 *   parent[v] = a neighbour u with (u,v) in the CSR and level[u] = level[v]-1
 *               (any one of them: the race of Sec. 3.2 is benign), parent[s]
 *               = s, -1 if unreached.
 * Levels are unique and exact; parents are valid but not unique.
 *
 * Errors: functions return a bfs_status (0 = success, negative = error);
 * functions that return a pointer return NULL on error.  bfs_last_error()
 * and bfs_last_status() describe the most recent failure on the calling host
 * thread.  No call aborts the process or traps the GPU: device-side failures
 * (a bounded wait that ran out, a queue overflow) are recorded in a per-graph
 * status word read by bfs_graph_status().
 *
 * Threading: a bfs_graph may be used from several host threads, but its BFS
 * workspace is shared, so runs on one graph are serialised on the device
 * (a run on a new stream first waits for the previous run's event).
 */
#ifndef GBBFS_H
#define GBBFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bfs_graph bfs_graph;   /* opaque, owned by the library */
typedef struct bfs_server bfs_server; /* opaque, owned by the library */

typedef enum {
    BFS_OK = 0,
    BFS_NOT_READY = 1,          /* bfs_poll: the query is still running   */
    BFS_ERR_INVALID_ARG = -1,   /* bad pointer, size, root or option       */
    BFS_ERR_INVALID_GRAPH = -2, /* CSR failed validation                   */
    BFS_ERR_OOM = -3,           /* device or host allocation failed        */
    BFS_ERR_CUDA = -4,          /* a CUDA runtime call failed              */
    BFS_ERR_DEPTH = -5,         /* a level does not fit the uint8 output   */
    BFS_ERR_TIMEOUT = -6,       /* a bounded device wait ran out           */
    BFS_ERR_BUSY = -7           /* no free slot / HBM budget exhausted     */
} bfs_status;

/* Tunables of a graph (bfs_graph_set_option).  The defaults are the values
 * measured fastest on GB300; a caller may override them per graph. */
typedef enum {
    BFS_OPT_BLOCK = 1,          /* threads per CTA: 256, 512 or 1024                  */
    BFS_OPT_CTAS_PER_SM = 2,    /* resident CTAs per SM of the persistent grid (>=1)  */
    BFS_OPT_WARP_DEGREE = 3,    /* a frontier vertex with degree >= this is expanded
                                   by one warp, below it by one thread (>= 1)          */
    BFS_OPT_CTA_DEGREE = 4,     /* degree >= this: expanded by a whole CTA (>= 64)     */
    BFS_OPT_SEGMENT = 5,        /* high-degree adjacency is cut into pieces of at most
                                   this many edges, each expanded by one CTA (>= 256)  */
    BFS_OPT_TIMEOUT_NS = 6,     /* limit of every device-side wait, in ns (>= 0)        */
    BFS_OPT_LAYER_STATS = 7,    /* 1: record per-layer counters (Table 1 columns)      */
    BFS_OPT_MAX_CTAS = 8,       /* cap on the persistent grid size (0 = no cap)        */
    BFS_OPT_BATCH_WIDTH = 9,    /* sources per bit-parallel batch: 8..64, multiple of 8 */
    BFS_OPT_BATCH_BLOCK = 10,   /* threads per CTA of the batched kernels: 256 or 512   */
    BFS_OPT_MODE = 11,          /* expansion of bfs_run: 0 = work items bounded in edges
                                   (short lists packed into units, hubs cut into slices)
                                   run by independent warps, BLOCK 256 or 512 (default);
                                   1 = one item per frontier vertex, binned by degree
                                   and expanded by a thread, a warp or a whole CTA;
                                   2 = as 0 without atomics: the output bitmap is set
                                   by plain read-modify-writes and P[v] = u - n, then
                                   a restoration pass per layer repairs both bitmaps
                                   and P (Sec. 3.3.2, Alg. 3); BLOCK 256 or 512.  Its
                                   workspace (4n bytes + two bitmaps) is allocated on
                                   the first run in this mode;
                                   3 = direction-optimising: layers run as in mode 0
                                   or bottom-up (every unvisited vertex looks for a
                                   parent among its in-neighbours in the frontier
                                   bitmap), chosen per layer by ALPHA and BETA; on a
                                   graph where some edge (u, v) lacks its reverse
                                   (checked at creation) the in-edges come from a
                                   transposed CSR built on the first run in this mode
                                   (4(n+m) bytes); BLOCK 256 or 512; 2 bitmaps of
                                   workspace, allocated on first use;
                                   4 = as 0 with more, lighter warps (256-thread CTAs,
                                   BLOCK ignored) that read each item's adjacency
                                   straight from memory and claim at once             */
    BFS_OPT_ALPHA = 12,         /* mode 3: a layer runs bottom-up once the frontier's
                                   summed degree exceeds (edges of unreached vertices)
                                   / ALPHA (0 .. 2^30, default 14; 0 = never)          */
    BFS_OPT_BETA = 13,          /* mode 3: back to top-down once the frontier has fewer
                                   than n / BETA vertices (1 .. 2^30, default 24)       */
    BFS_OPT_BATCH_STREAMS = 14  /* bfs_run_batch: batches run this many at a time, each
                                   on its own stream and workspace with an equal share
                                   of the GPU's CTAs (1..8, default 4); while one batch
                                   waits at a grid barrier the others run.  Each extra
                                   stream allocates one more batch workspace          */
} bfs_option;

/* ---- library ------------------------------------------------------------ */

/* ABI version of this header (library plumbing, not in the paper;
 * increments on an incompatible change). */
int bfs_abi_version(void);

/* Message and code of the most recent failure on this host thread (library
 * plumbing, not in the paper).  The message stays valid until the thread's
 * next library call. */
const char *bfs_last_error(void);
int bfs_last_status(void);

/* ---- graph -------------------------------------------------------------- */

/*
 * Upload a CSR graph (Sec. 3.3.1) to the current CUDA device.
 *   row_offsets : n+1 int32 entries; host or device memory (detected)
 *   col_idx     : m int32 entries; host or device memory; may be NULL if m == 0
 *   n, m        : 1 <= n <= 2^31 - 2^24, 0 <= m <= 2^31 - 2^24 (indices are
 *                 32-bit on the device; the margin keeps every grid-stride
 *                 loop's last step from overflowing), else BFS_ERR_INVALID_ARG
 * The library copies both arrays into device memory it owns; the caller
 * keeps ownership of its arrays.  The copy is validated on the device:
 * row_offsets[0] == 0, non-decreasing, row_offsets[n] == m, and every
 * column in [0, n).  Internally the vertices are renumbered by decreasing
 * degree class (hubs first) so that the visited-bit tests of most edges hit
 * a small, cache-resident part of the bitmap; every result is returned in
 * the caller's numbering.  On any failure returns NULL and sets bfs_last_status()
 * to BFS_ERR_INVALID_GRAPH, BFS_ERR_INVALID_ARG, BFS_ERR_OOM or
 * BFS_ERR_CUDA.  Synchronous (returns once the graph is resident).
 */
bfs_graph *bfs_graph_create(const int32_t *row_offsets, const int32_t *col_idx,
                            int64_t n, int64_t m);

/* Free the graph of bfs_graph_create (the CSR of Sec. 3.3.1) and its
 * workspaces, after waiting for its last run.  NULL is accepted.  Returns
 * BFS_OK or BFS_ERR_CUDA; BFS_ERR_BUSY (nothing freed) while the graph is
 * registered with a server that has not been destroyed, whose worker may
 * still search it. */
int bfs_graph_destroy(bfs_graph *g);

/* n and m of the graph as given to bfs_graph_create (Sec. 3.3.1: the
 * vertices and the CSR entries), or -1 for NULL. */
int64_t bfs_graph_num_vertices(const bfs_graph *g);
int64_t bfs_graph_num_edges(const bfs_graph *g);

/* Set / read a tunable (bfs_option; not in the paper, whose tunables are
 * Xeon Phi thread counts and affinities, Sec. 5).  Options change the time
 * of a search, never its result.  Invalid values give BFS_ERR_INVALID_ARG
 * and leave the option unchanged; get returns the value, or a negative
 * bfs_status for a NULL graph or an unknown option. */
int bfs_graph_set_option(bfs_graph *g, int option, int64_t value);
int64_t bfs_graph_get_option(const bfs_graph *g, int option);

/*
 * Single-source BFS from `root`, expanded as BFS_OPT_MODE selects (default:
 * top-down, Alg. 2 with atomic bitmap updates; see BFS_OPT_MODE).
 *   root       : 0 <= root < n, else BFS_ERR_INVALID_ARG
 *   level_out  : int32[n], device memory or host memory (detected)
 *   parent_out : int32[n], device or host memory, or NULL to skip parents
 *   stream     : a cudaStream_t (NULL = the legacy default stream)
 * Stream-ordered and asynchronous when both outputs are device memory: the
 * whole search (initialisation, every layer, termination) runs as one
 * persistent cooperative kernel with no host round trip per layer.  With
 * host outputs the library searches into its own device buffers and copies
 * the results back on `stream` (pinned host memory keeps this asynchronous;
 * pageable memory makes the copy synchronous).  Caller-owned outputs must
 * stay valid until the stream reaches the end of the run.
 * Returns enqueue-time errors only; device-side errors (BFS_ERR_TIMEOUT, a
 * queue overflow reported as BFS_ERR_CUDA) are read with bfs_graph_status.
 */
int bfs_run(bfs_graph *g, int32_t root, int32_t *level_out, int32_t *parent_out,
            void *stream);

/*
 * Single-source search that allocates nothing (not in the paper: a
 * deployment variant of bfs_run).  For callers that cannot
 * allocate GPU memory at the moment they search -- a process whose device
 * memory is owned by another allocator or fixed budget, a latency-critical
 * path that must not block in cudaMalloc/cudaFree, or code running where
 * the CUDA runtime forbids allocation.  The search runs the same top-down
 * kernel as bfs_run (BFS_OPT_MODE 0, BLOCK 512) directly on the caller's
 * device CSR, with all scratch state in one fixed-size __device__ array
 * built into the library (about 7 MB, held by every GPU that loads the
 * library until the process exits).  No cudaMalloc, cudaFree or allocating
 * library call is made.
 *   row_offsets, col_idx : the caller's CSR in DEVICE memory (checked as in
 *                          bfs_graph_create; no renumbering is done)
 *   n, m                 : 1 <= n <= BFS_NOALLOC_MAX_VERTICES,
 *                          0 <= m <= BFS_NOALLOC_MAX_EDGES, else
 *                          BFS_ERR_INVALID_ARG
 *   root, level_out, parent_out, stream : as bfs_run, outputs in DEVICE memory
 * Blocks until the search has finished and returns its status (including
 * BFS_ERR_TIMEOUT from the device).  The first call on a device also sets up
 * the array on that device; make it before any stream capture.  Every call
 * shares the one array: calls from several host threads are serialised, and
 * searches that overlap on the GPU through other means would race on it.
 * The set-up is kept for the life of the process: after cudaDeviceReset on
 * a device, this entry point must not be called on that device again until
 * the library is reloaded (its cached address would belong to the destroyed
 * context).
 */
#define BFS_NOALLOC_MAX_VERTICES 131072
#define BFS_NOALLOC_MAX_EDGES 4194304
int bfs_run_noalloc(const int32_t *row_offsets, const int32_t *col_idx, int64_t n, int64_t m,
                    int32_t root, int32_t *level_out, int32_t *parent_out, void *stream);

/* Wait for the graph's last run (any bfs_run of Alg. 1-3) and return its
 * device-side status (BFS_OK, BFS_ERR_TIMEOUT or BFS_ERR_CUDA); clears the
 * status word.
 * Bounds-checking build: the same sources compiled with -DBFS_BOUNDS_CHECK
 * give a library (libgbbfs_check.so) with this same ABI whose kernels check
 * the index of every main array access (adjacency, row offsets, visited
 * bitmap, level, parent, id maps, frontier queues; for the batched search
 * and the serving loop its frontier, seen words and level rows; modes 0, 2,
 * 3 and 4).  The first index out of range is recorded with its array and
 * replaced by 0, so that the access stays inside the array; the call that
 * reads the status (this one, bfs_run_batch, bfs_run_noalloc, the server's
 * queries) returns BFS_ERR_CUDA and bfs_last_error() names the array and the
 * index.  No trap or device assert is used. */
int bfs_graph_status(bfs_graph *g);

/*
 * Per-layer counters of the last bfs_run, the columns of Table 1: for layer
 * d, vertices[d] = frontier vertices, edges[d] = adjacency entries scanned
 * (in a bottom-up layer of mode 3: entries examined by the unvisited
 * vertices), traversed[d] = vertices first reached.  Recorded only while
 * BFS_OPT_LAYER_STATS is 1.  Arrays are host int64[max_layers].  Returns the
 * number of layers (<= max_layers are written) or a negative bfs_status.
 * Synchronous.
 */
int bfs_graph_layer_stats(bfs_graph *g, int64_t *vertices, int64_t *edges,
                          int64_t *traversed, int32_t max_layers);

/* Device time at the end of each layer (Sec. 3: layer L_d) of the last
 * bfs_run, ns since the kernel started (recorded with BFS_OPT_LAYER_STATS =
 * 1).  t_end_ns: host int64[max_layers].  Returns the number of layers or a
 * negative bfs_status.  Synchronous. */
int bfs_graph_layer_times(bfs_graph *g, int64_t *t_end_ns, int32_t max_layers);

/*
 * Autotuner (not in the paper): times candidate values of the graph's own
 * tunables on `samples` sample searches of this graph (0 = 8; roots spread
 * over the vertices with edges) and leaves the fastest values set.  Options
 * are tuned one at a time, each keeping its best value before the next is
 * tried.  `what` combines:
 *   BFS_TUNE_SINGLE : the current BFS_OPT_MODE's tunables -- BLOCK; in mode 1
 *                     also WARP_DEGREE, CTA_DEGREE and SEGMENT; in mode 3
 *                     also ALPHA and BETA
 *   BFS_TUNE_BATCH  : BATCH_WIDTH, BATCH_BLOCK and BATCH_STREAMS, timed on
 *                     bfs_run_batch over 512 sources
 *   BFS_TUNE_MODE   : BFS_OPT_MODE 0 or 3, whichever is faster (applied
 *                     before BFS_TUNE_SINGLE)
 * Results never depend on the options, only the time does.  Synchronous;
 * allocates its own scratch (two int32[n] and, for BFS_TUNE_BATCH, uint8
 * [512][n]) and frees it.  On an error the options are restored and the
 * status returned.
 */
#define BFS_TUNE_SINGLE 1
#define BFS_TUNE_BATCH 2
#define BFS_TUNE_MODE 4
int bfs_graph_autotune(bfs_graph *g, int what, int32_t samples);

/* Copy the visited bitmap of the last bfs_run (uint32 words, vertex v at
 * word v>>5, bit v&31; Sec. 3.3.1, Listing 1) to host memory `words_out` of
 * `nwords` >= ceil(n/32) entries.  Synchronous. */
int bfs_graph_visited_bitmap(bfs_graph *g, uint32_t *words_out, int64_t nwords);

/*
 * Batched BFS: k sources searched together, bit-parallel, `BATCH_WIDTH`
 * (default 64) sources per uint64 visit/frontier word per vertex.  Not in
 * the paper; it reuses the layer step of Alg. 2 with one bit per source.
 *   roots     : host int32[k], each in [0, n)
 *   k         : >= 0
 *   level_out : uint8[k][n] source-major, device or host memory; level of
 *               vertex v from roots[i] at level_out[i*n + v], 0xFF = unreached
 * Synchronous.  Returns BFS_ERR_DEPTH if some level exceeds 254.
 */
int bfs_run_batch(bfs_graph *g, const int32_t *roots, int32_t k, uint8_t *level_out);

/* ---- serving ------------------------------------------------------------ */

/*
 * Serving (not in the paper; each query is the search of Sec. 3, run by the
 * batched layer step of bfs_run_batch).
 * A request loop over resident graphs with continuous batching: queries on
 * one graph are packed into the lanes of bit-parallel batches as they
 * arrive; a lane freed by a finished query is given to the next waiting one
 * while the batch keeps running.  Work is admitted while the device memory
 * it needs fits `hbm_budget_bytes` (0 = a default fraction of free memory).
 * Each registered graph gets its own host worker thread and CUDA stream.
 * While a batch is in its heavy (pull) phase, new queries on that graph wait
 * a few iterations and then join together, so that young lanes do not keep
 * the batch in its slower push form.
 * A query waits at most 60 s for room for its graph's workspace; past that
 * it fails with BFS_ERR_BUSY.  If the device itself cannot hold the
 * workspace (no other graph holds one that it could give back), the graph's
 * waiting queries fail with BFS_ERR_OOM.  Either way the server and its
 * other graphs keep running.
 * The graphs' streams should not share CUDA hardware work queues: with the
 * default of 8 queues, a small graph's result extraction can wait behind a
 * large graph's round of several milliseconds that sits on the same queue.
 * Set CUDA_DEVICE_MAX_CONNECTIONS=32 in the environment before the process's
 * first CUDA call (the Python binding sets this default when it is imported
 * first).
 */
bfs_server *bfs_server_create(int64_t hbm_budget_bytes);

/* Serving, not in the paper.  Stop the workers (each finishes its current
 * round), free the workspaces
 * and the server.  Queries still queued are dropped: drain first to keep
 * them.  NULL is accepted.  Returns BFS_OK. */
int bfs_server_destroy(bfs_server *s);

/* Serving, not in the paper.  Register a graph (not owned: keep it alive
 * until bfs_server_destroy).
 * From then on the server owns the graph's batch workspace: do not call
 * bfs_run_batch on it while it is registered (bfs_run stays available).
 * Returns a graph id >= 0 or a negative bfs_status. */
int bfs_server_add_graph(bfs_server *s, bfs_graph *g);

/* Queue one BFS query: the search of Sec. 3 from `root` on graph graph_id,
 * levels only.  level_out: host uint8[n] of that graph (caller-owned),
 * written as in bfs_run_batch (0xFF = unreached); it must stay valid until
 * bfs_poll reports completion or failure.  Into page-locked (pinned) memory
 * the row is stored by a kernel over the host link; into pageable memory it
 * is copied, which is slower under load.  *ticket receives the query's id
 * (>= 1).  Returns BFS_ERR_INVALID_ARG (NULL pointer, unknown graph, root
 * outside [0, n)), BFS_ERR_BUSY if the graph's workspace can never fit the
 * HBM budget, or the server's error once it has stopped after one. */
int bfs_submit(bfs_server *s, int graph_id, int32_t root, uint8_t *level_out,
               uint64_t *ticket);

/* Serving, not in the paper.  BFS_OK when the query is complete (level_out
 * filled), BFS_NOT_READY while
 * it waits or runs, or the negative bfs_status it failed with
 * (BFS_ERR_INVALID_ARG for an unknown ticket).  Never blocks. */
int bfs_poll(bfs_server *s, uint64_t ticket);

/* Serving, not in the paper.  Block until every submitted query has
 * completed or failed.  Returns
 * BFS_OK, or the error that stopped the server (queries that failed alone,
 * e.g. with BFS_ERR_BUSY, are reported by bfs_poll only). */
int bfs_server_drain(bfs_server *s);

/* Monitoring counters (not in the paper) of one graph of the server,
 * written to out[0..6]:
 *   out[0] queries waiting for a lane     out[1] lanes running
 *   out[2] rounds its worker has run      out[3] the batch's iteration after
 *                                                the last round (-1 = none)
 *   out[4] 1 while it holds its workspace
 *   out[5] ns since its worker last finished a round (-1 = never)
 *   out[6] what its worker is doing: 0 waiting for work, 1 admitting
 *          queries, 2 putting sources on the device, 3 launching iterations,
 *          4 reading the control block (waits for those iterations),
 *          5 delivering results, 6 waiting for workspace room, 7 stopped
 * A snapshot taken without stopping the worker.  Returns BFS_OK or
 * BFS_ERR_INVALID_ARG (NULL pointer, unknown graph id). */
int bfs_server_graph_stats(bfs_server *s, int graph_id, int64_t *out);

/* Serving, not in the paper.  Submission and completion times of a query,
 * ns on a monotonic clock
 * (latency = t_done - t_submit; t_done is 0 while it runs).  Returns BFS_OK
 * or BFS_ERR_INVALID_ARG. */
int bfs_ticket_times(bfs_server *s, uint64_t ticket, int64_t *t_submit_ns,
                     int64_t *t_done_ns);

/* Serving, not in the paper.  The path of one query through the server:
 *   t_submit_ns, t_admit_ns, t_done_ns : submission, admission into a lane
 *       of the graph's running bit-parallel search, completion (ns on the
 *       monotonic clock of bfs_ticket_times; 0 while not reached).  Queue
 *       wait = t_admit - t_submit; time in the search (iterations plus the
 *       result copy) = t_done - t_admit.
 *   join_iter, done_iter : the search's iteration counter when the lane was
 *       filled and at the end of the round that found the query finished
 *       (-1 while not reached); a query whose lanes_busy_at_join > 0 joined
 *       a search already running for other queries (continuous batching).
 *   graph_id, lane : where it ran (lane -1 until admitted).
 * `out` is caller-owned.  Returns BFS_OK or BFS_ERR_INVALID_ARG (NULL
 * argument, unknown ticket). */
typedef struct bfs_ticket_record {
    int64_t t_submit_ns, t_admit_ns, t_done_ns;
    int64_t join_iter, done_iter;
    int32_t graph_id, lane, lanes_busy_at_join, reserved;
} bfs_ticket_record;
int bfs_ticket_info(bfs_server *s, uint64_t ticket, bfs_ticket_record *out);

#ifdef __cplusplus
}
#endif

#endif /* GBBFS_H */
