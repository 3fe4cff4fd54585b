// internal.cuh -- shared declarations of the BFS library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <string>

#include "../../include/gbbfs.h"

namespace gbbfs {

// ---- error reporting -------------------------------------------------------
int set_error(int status, const std::string &msg);  // records, returns status
int cuda_error(cudaError_t e, const char *what);      // records BFS_ERR_CUDA
void clear_error();

#define GB_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);  \
    } while (0)

// ---- device status bits (sticky until bfs_graph_status reads them) --------
enum : unsigned {
    ST_TIMEOUT = 1u,   // a bounded wait gave up
    ST_OVERFLOW = 2u,  // a queue append would have run past its capacity
    ST_DEPTH = 4u,     // a level did not fit the uint8 batch encoding
    ST_BOUNDS = 8u,    // bounds-checking build: an index left its array (first one in `bounds`)
};

// Where an out-of-range index was caught (bounds-checking build).
enum : int { BS_COL = 1, BS_ROW = 2, BS_VISITED = 3, BS_LEVEL = 4, BS_PARENT = 5, BS_ORIG = 6, BS_QUEUE = 7,
             BS_FRONTIER = 8, BS_LANE_ROW = 9 };

// Text of a recorded violation word: (site << 48) | index.
inline const char *bounds_site_name(unsigned long long w)
{
    switch ((int)(w >> 48)) {
        case BS_COL: return "col_idx";
        case BS_ROW: return "row_offsets";
        case BS_VISITED: return "visited bitmap";
        case BS_LEVEL: return "level";
        case BS_PARENT: return "parent";
        case BS_ORIG: return "internal-to-caller id map";
        case BS_QUEUE: return "frontier queue";
        case BS_FRONTIER: return "frontier / seen words";
        case BS_LANE_ROW: return "level rows";
        default: return "unknown array";
    }
}

// ---- control block of the persistent single-source kernels ----------------
// Counters rotate over three sets: layer d reads set d%3, appends to set
// (d+1)%3 and clears set (d+2)%3, which nobody touches during layer d.
// The last CTA to leave a search returns every counter to zero.
struct Ctrl {
    unsigned long long eu_count[3];  // warp mode: (units << 32) | entries
    unsigned long long nf[3];        // hybrid mode: frontier vertices of a layer
    unsigned long long mf[3];        // hybrid mode: their summed degrees
    unsigned hub_count[3];           // warp mode: hub slices
    unsigned work[3];                // work-item dispenser (both modes)
    unsigned count[3];               // binned mode: small-item queue size
    unsigned big_count[3];           // binned mode: large-item queue size
    unsigned big_work[3];            // binned mode: large-item dispenser
    unsigned bar_count;              // grid barrier arrivals
    unsigned bar_gen;                // grid barrier generation
    unsigned exit_count;             // CTAs that left the kernel
    unsigned status;                 // ST_* bits
    unsigned layers;                 // layers of the last search
    unsigned long long bounds;       // bounds-checking build: first violation, (site << 48) | index
};

enum { MODE_WARP = 0, MODE_BINNED = 1, MODE_RESTORE = 2, MODE_HYBRID = 3, MODE_THIN = 4 };

struct Options {
    int block = 512;
    int ctas_per_sm = 0;      // 0 = as many as fit
    int warp_degree = 16;
    int cta_degree = 1024;
    int segment = 4096;
    int64_t timeout_ns = 4000000000LL;
    int layer_stats = 0;
    int max_ctas = 0;
    int batch_width = 64;
    int batch_block = 256;  // 8-warp CTAs: the server's grid shares are counted in them
    int batch_streams = 4;  // bfs_run_batch: batches in flight at once (1 = one after another)
    int mode = MODE_WARP;
    int alpha = 14;  // hybrid: go bottom-up when frontier edges > unexplored edges / alpha
    int beta = 24;   // hybrid: back to top-down when frontier vertices < n / beta
};

constexpr int kMaxStatLayers = 256;

struct Graph {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0, m = 0;
    // CSR in the library's internal numbering (degree-ordered, relabel.cu)
    int32_t *d_row_offsets = nullptr;
    int32_t *d_col_idx = nullptr;  // padded: m rounded up to 4, plus 4 entries
    int32_t *d_perm = nullptr;     // caller id -> internal id
    int32_t *d_orig = nullptr;     // internal id -> caller id
    int64_t split32 = 0;           // internal ids [0, split32) have degree >= 32
    int64_t n_nonzero = 0;         // internal ids [0, n_nonzero) have degree >= 1
    bool symmetric = false;        // every (u, v) has (v, u): in-edges = out-edges

    // single-source workspace
    uint32_t *d_bitmap = nullptr;  // words rounded up to a multiple of 4
    int64_t bitmap_words = 0;
    int32_t *d_eq[2][3] = {};      // warp mode: [buffer][u, beg, len] entries
    int32_t *d_uq[2][2] = {};      // warp mode: [buffer][first entry, count]
    int32_t *d_hq[2][3] = {};      // warp mode: [buffer][u, beg, len] hub slices
    int64_t hcap = 0;
    int32_t *d_q[2][3] = {};       // binned mode (lazy): small-item queue
    int32_t *d_bq[2][3] = {};      // binned mode (lazy): large-item queue
    int64_t qcap = 0, bqcap = 0;
    uint2 *d_vo = nullptr;         // restoration mode (lazy): (visited, output) word pairs
    uint32_t *d_front[2] = {};     // hybrid mode (lazy): frontier bitmaps of bottom-up layers
    int32_t *d_tro = nullptr;      // hybrid mode on a non-symmetric graph (lazy): in-edge CSR
    int32_t *d_tcol = nullptr;
    int32_t *d_pint = nullptr;     // restoration mode (lazy): internal predecessors
    Ctrl *d_ctrl = nullptr;
    int64_t *d_stats = nullptr;    // [kMaxStatLayers][4]: vertices, edges, new, t_end_ns
    int last_grid = 0;
    int32_t *d_level_tmp = nullptr;   // used when outputs are host memory
    int32_t *d_parent_tmp = nullptr;

    cudaEvent_t ws_event = nullptr;  // end of the last run on the workspace
    cudaStream_t last_stream = nullptr;
    bool ran = false;

    // batched (bit-parallel) workspace, allocated on first use
    void *batch_ws = nullptr;
    int stream_priority = 0;  // of the batched workspace's stream (set by a server)

    Options opt;
    std::mutex mu;
    std::atomic<int> servers{0};  // live servers this graph is registered with
};

// A named host-side range for profilers (NVTX, header-only; costs nothing
// when no tool is attached).  The searches are persistent kernels, so a
// range covers one launch; per-layer times come from the device counters.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// A graph registered with a live server is still in use by the server's
// worker thread: bfs_graph_destroy refuses it until the server is destroyed.
inline int graph_release_check(const Graph *g)
{
    if (g->servers.load() > 0)
        return set_error(BFS_ERR_BUSY, "bfs_graph_destroy: the graph is registered with a live server; "
                                       "destroy the server first");
    return BFS_OK;
}

// implemented in topdown.cu (degree-binned mode; its queues are allocated
// on first use by graph.cu)
int td_launch(Graph *g, int32_t root, int32_t *level, int32_t *parent, cudaStream_t s);

// implemented in topdown_warp.cu (warp-private pipelines, the default;
// MODE_RESTORE is the atomic-free variant of Alg. 3 and MODE_HYBRID the
// direction-optimising search, whose workspaces graph.cu allocates on first use)
int td_warp_launch(Graph *g, int32_t root, int32_t *level, int32_t *parent, cudaStream_t s,
                   int mode = MODE_WARP);
int64_t td_hub_capacity(int64_t m);

// implemented in msbfs.cu
int ms_run_batch(Graph *g, const int32_t *roots, int32_t k, uint8_t *level_out);
void ms_free(Graph *g);

// implemented in relabel.cu
int relabel_graph(Graph *g, const int32_t *d_ro, const int32_t *d_col);
int transpose_graph(Graph *g);  // d_tro / d_tcol from the internal CSR
int bitmap_to_caller(Graph *g, uint32_t *d_out);

bool is_device_pointer(const void *p);

// implemented in graph.cu: CSR checks (flags: 1 offsets, 2 columns, 4 ends)
__global__ void validate_csr_kernel(const int32_t *__restrict__ ro, const int32_t *__restrict__ col, int64_t n,
                                    int64_t m, unsigned *flags);

}  // namespace gbbfs
