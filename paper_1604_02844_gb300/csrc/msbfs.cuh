// msbfs.cuh -- workspace and host entry points of the bit-parallel
// multi-source search (msbfs.cu), shared with the serving loop (server.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace gbbfs {

// Control block.  Counters of iteration parity p are used by iteration
// iter (p = iter & 1) and cleared during the iteration of the other parity.
struct MsCtrl {
    unsigned fcount[2];           // frontier entries in buffer p
    unsigned long long fedges[2]; // adjacency entries of frontier buffer p
    unsigned pulls;               // iterations run as pull steps (diagnostic)
    unsigned long long seen_pairs;  // (vertex, lane) pairs set in seen
    unsigned work[2];             // EXPAND dispenser
    unsigned tcount[2];           // touched vertices
    unsigned bar_count, bar_gen, exit_count;
    unsigned status;              // ST_* bits
    unsigned iter;                // global iteration number (persists across launches)
    unsigned pad;
    unsigned long long alive[2];  // lanes present in frontier buffer p
    unsigned long long bounds;    // bounds-checking build: first violation, (site << 48) | index
};

constexpr int kMaxBatchStreams = 8;  // BFS_OPT_BATCH_STREAMS upper bound

struct MsWs {
    unsigned long long *seen = nullptr, *next = nullptr, *front[2] = {};
    uint8_t *lvl = nullptr;       // [n][64] levels, caller numbering, 0xFF = unreached
    int32_t *fq[2][3] = {};       // frontier entries (u, beg, len) per parity
    int32_t *touched = nullptr;
    MsCtrl *ctrl = nullptr;
    int32_t *start = nullptr;     // [64] iteration each lane joined
    int32_t *lane_src = nullptr;  // [64] staging for inject
    int32_t *lane_row = nullptr;  // [64] staging for extract
    MsCtrl *h_ctrl = nullptr;     // pinned
    MsCtrl *d_ctrl_mirror = nullptr;  // h_ctrl as the device addresses it (null: read by a copy)
    int32_t *h_lanes = nullptr;   // pinned, 128 entries
    int64_t fcap = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;     // bfs_run_batch: fork (first workspace) / join (the others)
    MsWs *peer[kMaxBatchStreams - 1] = {};  // bfs_run_batch: the workspaces of the other streams
    // bfs_run_batch: buffers and the captured launch sequence of the last call shape
    int32_t *b_lanes = nullptr;   // [3][b_cap] roots, internal sources, output rows
    int32_t *h_roots = nullptr;   // pinned staging of the roots
    int64_t b_cap = 0;
    uint8_t *b_tmp = nullptr;     // [b_tmp_width][n] level rows for host outputs
    int b_tmp_width = 0;
    cudaGraphExec_t b_exec = nullptr;
    struct Key {
        int32_t k = -1;
        uint8_t *out = nullptr;
        int out_dev = 0, width = 0, block = 0, max_ctas = 0, streams = 0;
        int64_t timeout_ns = 0;
        bool operator==(const Key &o) const
        {
            return k == o.k && out == o.out && out_dev == o.out_dev && width == o.width && block == o.block &&
                   max_ctas == o.max_ctas && streams == o.streams && timeout_ns == o.timeout_ns;
        }
    } b_key;
};

int ms_alloc(Graph *g, MsWs **out);
int ms_reset(Graph *g);
int ms_reset_ws(Graph *g, MsWs *w);
// sources in the caller's numbering, one per lane of `mask`
int ms_inject(Graph *g, const int32_t *lane_src_caller, unsigned long long mask);
// up to max_iters iterations, stopping when no lane has a frontier
int ms_step(Graph *g, uint32_t max_iters);
int ms_step_capped(Graph *g, uint32_t max_iters, int max_ctas);
int ms_read_ctrl(Graph *g, MsCtrl *out);
int ms_extract(Graph *g, unsigned long long mask, const int32_t *lane_row_host, uint8_t *out, int64_t out_stride,
               bool recycle);
__global__ void map_ids_kernel(int32_t *ids, const int32_t *__restrict__ perm, int k);

// Rows of a staging buffer (row r at stage + r * n) stored by a kernel into
// host buffers that the device can address (pinned memory under unified
// addressing): dst[i] receives row rows[i], for i < count.  Asynchronous on
// `stream`.  Returns false (nothing enqueued) when a destination is not
// device-addressable, so that the caller copies instead.
struct RowsToHost {
    uint8_t *dst[64];
    int32_t rows[64];
    int count;
};
bool ms_host_addressable(const void *p, uint8_t **dev_ptr);
int ms_rows_to_host(const uint8_t *stage, int64_t n, const RowsToHost &job, cudaStream_t stream);

}  // namespace gbbfs
