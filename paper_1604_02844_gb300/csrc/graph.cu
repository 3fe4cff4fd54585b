// graph.cu -- graph object, CSR upload and validation, options, status and
// the single-source entry point of the C ABI.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "internal.cuh"

namespace gbbfs {

static thread_local int t_status = BFS_OK;
static thread_local std::string t_msg;

int set_error(int status, const std::string &msg)
{
    t_status = status;
    t_msg = msg;
    return status;
}

int cuda_error(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    // consume the runtime's record of a non-sticky error (a failed
    // allocation), so that the next launch check of this thread does not
    // report it again
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA, m);
}

void clear_error()
{
    t_status = BFS_OK;
    t_msg.clear();
}

bool is_device_pointer(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // unregistered host memory on old runtimes
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// CSR validation on the device.  flags bit 0: offsets not monotone or out of
// [0, m]; bit 1: a column outside [0, n); bit 2: row_offsets[0] != 0 or
// row_offsets[n] != m.
__global__ void validate_csr_kernel(const int32_t *__restrict__ ro, const int32_t *__restrict__ col,
                                    int64_t n, int64_t m, unsigned *flags)
{
    unsigned f = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int32_t a = ro[i], b = ro[i + 1];
        if (a > b || a < 0 || (int64_t)b > m) f |= 1u;
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int32_t v = col[e];
        if (v < 0 || (int64_t)v >= n) f |= 2u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        if (ro[0] != 0 || (int64_t)ro[n] != m) f |= 4u;
    f = __reduce_or_sync(0xffffffffu, f);
    if (f && (threadIdx.x & 31) == 0) atomicOr(flags, f);
}

static void free_graph(Graph *g)
{
    if (!g) return;
    ms_free(g);
    cudaFree(g->d_row_offsets);
    cudaFree(g->d_col_idx);
    cudaFree(g->d_perm);
    cudaFree(g->d_orig);
    cudaFree(g->d_bitmap);
    for (int b = 0; b < 2; ++b) {
        for (int j = 0; j < 3; ++j) {
            cudaFree(g->d_q[b][j]);
            cudaFree(g->d_bq[b][j]);
            cudaFree(g->d_eq[b][j]);
            cudaFree(g->d_hq[b][j]);
        }
        for (int j = 0; j < 2; ++j) cudaFree(g->d_uq[b][j]);
    }
    cudaFree(g->d_vo);
    cudaFree(g->d_front[0]);
    cudaFree(g->d_front[1]);
    cudaFree(g->d_tro);
    cudaFree(g->d_tcol);
    cudaFree(g->d_pint);
    cudaFree(g->d_ctrl);
    cudaFree(g->d_stats);
    cudaFree(g->d_level_tmp);
    cudaFree(g->d_parent_tmp);
    if (g->ws_event) cudaEventDestroy(g->ws_event);
    delete g;
}

// Large-item queue capacity (binned mode): a vertex of degree d >=
// cta_degree becomes ceil(d / segment) items, so the items of one layer are
// at most m / segment + m / cta_degree (+1).  Options keep segment >= 256
// and cta_degree >= 64, the bounds used here.
static int64_t big_queue_capacity(int64_t m) { return m / 256 + m / 64 + 2; }

// Binned-mode queues, allocated the first time that mode runs.
static int alloc_binned(Graph *g)
{
    if (g->d_q[0][0]) return BFS_OK;
    g->qcap = g->n;
    g->bqcap = big_queue_capacity(g->m);
    for (int b = 0; b < 2; ++b)
        for (int j = 0; j < 3; ++j) {
            GB_CUDA(cudaMalloc(&g->d_q[b][j], (size_t)g->qcap * 4));
            GB_CUDA(cudaMalloc(&g->d_bq[b][j], (size_t)g->bqcap * 4));
        }
    return BFS_OK;
}

// Restoration-mode workspace (Alg. 3 visited and output bitmaps as word
// pairs, and `P` in the internal numbering), allocated the first time that
// mode runs.
static int alloc_restore(Graph *g)
{
    if (g->d_vo) return BFS_OK;
    GB_CUDA(cudaMalloc(&g->d_pint, (size_t)g->n * 4));
    GB_CUDA(cudaMalloc(&g->d_vo, (size_t)g->bitmap_words * 8));
    return BFS_OK;
}

// Hybrid-mode frontier bitmaps (bottom-up layers) and, on a graph that is
// not symmetric, the in-edge CSR they scan, built the first time that mode runs.
static int alloc_hybrid(Graph *g)
{
    if (!g->d_front[0])
        for (int b = 0; b < 2; ++b) GB_CUDA(cudaMalloc(&g->d_front[b], (size_t)g->bitmap_words * 4));
    if (!g->symmetric && !g->d_tro) return transpose_graph(g);
    return BFS_OK;
}

}  // namespace gbbfs

using namespace gbbfs;

extern "C" {

int bfs_abi_version(void) { return 1; }
const char *bfs_last_error(void) { return t_msg.c_str(); }
int bfs_last_status(void) { return t_status; }

bfs_graph *bfs_graph_create(const int32_t *row_offsets, const int32_t *col_idx, int64_t n, int64_t m)
{
    clear_error();
    // Vertex and edge indices are 32-bit in the kernels, whose grid-stride
    // loops step up to about 2^18 past the last index: keep 2^24 of headroom.
    constexpr int64_t kMaxIndex = (int64_t(1) << 31) - (int64_t(1) << 24);
    if (!row_offsets || n < 1 || n > kMaxIndex || m < 0 || m > kMaxIndex || (m > 0 && !col_idx)) {
        set_error(BFS_ERR_INVALID_ARG, "bfs_graph_create: need row_offsets, 1 <= n <= 2^31 - 2^24, "
                                       "0 <= m <= 2^31 - 2^24, col_idx when m > 0");
        return nullptr;
    }
    Graph *g = new (std::nothrow) Graph();
    if (!g) {
        set_error(BFS_ERR_OOM, "bfs_graph_create: host allocation");
        return nullptr;
    }
    g->n = n;
    g->m = m;
    auto fail = [&](cudaError_t e, const char *what) -> bfs_graph * {
        cuda_error(e, what);
        free_graph(g);
        return nullptr;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&g->device)) != cudaSuccess) return fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess)
        return fail(e, "cudaDeviceGetAttribute");

    // the caller's CSR, copied to temporary device arrays and validated there
    int32_t *t_ro = nullptr, *t_col = nullptr;
    auto fail_tmp = [&](cudaError_t e2, const char *what) -> bfs_graph * {
        cudaFree(t_ro);
        cudaFree(t_col);
        return fail(e2, what);
    };
    if ((e = cudaMalloc(&t_ro, (size_t)(n + 1) * 4)) != cudaSuccess) return fail_tmp(e, "cudaMalloc(row_offsets copy)");
    if ((e = cudaMalloc(&t_col, (size_t)std::max<int64_t>(m, 1) * 4)) != cudaSuccess) return fail_tmp(e, "cudaMalloc(col_idx copy)");
    if ((e = cudaMemcpy(t_ro, row_offsets, (size_t)(n + 1) * 4, cudaMemcpyDefault)) != cudaSuccess)
        return fail_tmp(e, "cudaMemcpy(row_offsets)");
    if (m > 0 && (e = cudaMemcpy(t_col, col_idx, (size_t)m * 4, cudaMemcpyDefault)) != cudaSuccess)
        return fail_tmp(e, "cudaMemcpy(col_idx)");

    // validation
    unsigned *d_flags = nullptr;
    if ((e = cudaMalloc(&d_flags, sizeof(unsigned))) != cudaSuccess) return fail_tmp(e, "cudaMalloc(flags)");
    cudaMemset(d_flags, 0, sizeof(unsigned));
    validate_csr_kernel<<<g->num_sms * 4, 256>>>(t_ro, t_col, n, m, d_flags);
    unsigned flags = 0;
    e = cudaMemcpy(&flags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d_flags);
    if (e != cudaSuccess) return fail_tmp(e, "validate_csr_kernel");
    if (flags) {
        std::string why;
        if (flags & 4u) why += " row_offsets[0] != 0 or row_offsets[n] != m;";
        if (flags & 1u) why += " row_offsets not non-decreasing within [0, m];";
        if (flags & 2u) why += " a column index outside [0, n);";
        set_error(BFS_ERR_INVALID_GRAPH, "bfs_graph_create: invalid CSR:" + why);
        cudaFree(t_ro);
        cudaFree(t_col);
        free_graph(g);
        return nullptr;
    }
    // internal degree-ordered numbering (relabel.cu)
    {
        const int rc = relabel_graph(g, t_ro, t_col);
        cudaFree(t_ro);
        cudaFree(t_col);
        if (rc != BFS_OK) {
            free_graph(g);
            return nullptr;
        }
    }

    // single-source workspace (warp mode; the binned-mode queues are lazy)
    g->bitmap_words = ((n + 31) / 32 + 3) / 4 * 4;
    g->hcap = td_hub_capacity(m);
    if ((e = cudaMalloc(&g->d_bitmap, (size_t)g->bitmap_words * 4)) != cudaSuccess) return fail(e, "cudaMalloc(bitmap)");
    for (int b = 0; b < 2; ++b) {
        for (int j = 0; j < 3; ++j) {
            if ((e = cudaMalloc(&g->d_eq[b][j], (size_t)n * 4)) != cudaSuccess) return fail(e, "cudaMalloc(entry queue)");
            if ((e = cudaMalloc(&g->d_hq[b][j], (size_t)g->hcap * 4)) != cudaSuccess) return fail(e, "cudaMalloc(hub queue)");
        }
        for (int j = 0; j < 2; ++j)
            if ((e = cudaMalloc(&g->d_uq[b][j], (size_t)n * 4)) != cudaSuccess) return fail(e, "cudaMalloc(unit queue)");
    }
    if ((e = cudaMalloc(&g->d_ctrl, sizeof(Ctrl))) != cudaSuccess) return fail(e, "cudaMalloc(ctrl)");
    if ((e = cudaMemset(g->d_ctrl, 0, sizeof(Ctrl))) != cudaSuccess) return fail(e, "cudaMemset(ctrl)");
    if ((e = cudaMemset(g->d_bitmap, 0, (size_t)g->bitmap_words * 4)) != cudaSuccess) return fail(e, "cudaMemset(bitmap)");
    if ((e = cudaMalloc(&g->d_stats, sizeof(int64_t) * 4 * kMaxStatLayers)) != cudaSuccess) return fail(e, "cudaMalloc(stats)");
    if ((e = cudaMemset(g->d_stats, 0, sizeof(int64_t) * 4 * kMaxStatLayers)) != cudaSuccess) return fail(e, "cudaMemset(stats)");
    if ((e = cudaEventCreateWithFlags(&g->ws_event, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "cudaEventCreate");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "cudaDeviceSynchronize");
    return reinterpret_cast<bfs_graph *>(g);
}

int bfs_graph_destroy(bfs_graph *gh)
{
    if (!gh) return BFS_OK;
    Graph *g = reinterpret_cast<Graph *>(gh);
    if (const int busy = graph_release_check(g)) return busy;
    cudaError_t e = cudaSuccess;
    if (g->ran) e = cudaEventSynchronize(g->ws_event);
    free_graph(g);
    if (e != cudaSuccess) return cuda_error(e, "bfs_graph_destroy");
    return BFS_OK;
}

int64_t bfs_graph_num_vertices(const bfs_graph *gh) { return gh ? reinterpret_cast<const Graph *>(gh)->n : -1; }
int64_t bfs_graph_num_edges(const bfs_graph *gh) { return gh ? reinterpret_cast<const Graph *>(gh)->m : -1; }

int bfs_graph_set_option(bfs_graph *gh, int option, int64_t v)
{
    if (!gh) return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_set_option: NULL graph");
    Graph *g = reinterpret_cast<Graph *>(gh);
    std::lock_guard<std::mutex> lk(g->mu);
    Options &o = g->opt;
    auto bad = [&](const char *why) { return set_error(BFS_ERR_INVALID_ARG, std::string("bfs_graph_set_option: ") + why); };
    switch (option) {
    case BFS_OPT_BLOCK:
        if (v != 256 && v != 512 && v != 1024) return bad("BLOCK must be 256, 512 or 1024");
        o.block = (int)v;
        break;
    case BFS_OPT_CTAS_PER_SM:
        if (v < 0 || v > 32) return bad("CTAS_PER_SM must be in [0, 32]");
        o.ctas_per_sm = (int)v;
        break;
    case BFS_OPT_WARP_DEGREE:
        if (v < 1 || v > (1 << 20)) return bad("WARP_DEGREE must be in [1, 2^20]");
        o.warp_degree = (int)v;
        break;
    case BFS_OPT_CTA_DEGREE:
        if (v < 64 || v > (1 << 30)) return bad("CTA_DEGREE must be in [64, 2^30]");
        o.cta_degree = (int)v;
        break;
    case BFS_OPT_SEGMENT:
        if (v < 256 || v > (1 << 30)) return bad("SEGMENT must be in [256, 2^30]");
        o.segment = (int)v;
        break;
    case BFS_OPT_TIMEOUT_NS:
        if (v < 0) return bad("TIMEOUT_NS must be >= 0");
        o.timeout_ns = v;
        break;
    case BFS_OPT_LAYER_STATS:
        if (v != 0 && v != 1) return bad("LAYER_STATS must be 0 or 1");
        o.layer_stats = (int)v;
        break;
    case BFS_OPT_MAX_CTAS:
        if (v < 0 || v > (1 << 20)) return bad("MAX_CTAS must be in [0, 2^20]");
        o.max_ctas = (int)v;
        break;
    case BFS_OPT_BATCH_WIDTH:
        if (v < 8 || v > 64 || v % 8) return bad("BATCH_WIDTH must be 8..64, a multiple of 8");
        o.batch_width = (int)v;
        break;
    case BFS_OPT_BATCH_BLOCK:
        if (v != 256 && v != 512) return bad("BATCH_BLOCK must be 256 or 512");
        o.batch_block = (int)v;
        break;
    case BFS_OPT_MODE:
        if (v != MODE_WARP && v != MODE_BINNED && v != MODE_RESTORE && v != MODE_HYBRID && v != MODE_THIN)
            return bad("MODE must be 0 (warp units), 1 (degree-binned), 2 (restoration, no atomics), "
                       "3 (direction-optimising) or 4 (thin warps)");
        o.mode = (int)v;
        break;
    case BFS_OPT_ALPHA:
        if (v < 0 || v > (1 << 30)) return bad("ALPHA must be in [0, 2^30] (0: top-down only)");
        o.alpha = (int)v;
        break;
    case BFS_OPT_BETA:
        if (v < 1 || v > (1 << 30)) return bad("BETA must be in [1, 2^30]");
        o.beta = (int)v;
        break;
    case BFS_OPT_BATCH_STREAMS:
        if (v < 1 || v > 8) return bad("BATCH_STREAMS must be in [1, 8]");
        o.batch_streams = (int)v;
        break;
    default:
        return bad("unknown option");
    }
    return BFS_OK;
}

int64_t bfs_graph_get_option(const bfs_graph *gh, int option)
{
    if (!gh) return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_get_option: NULL graph");
    const Options &o = reinterpret_cast<const Graph *>(gh)->opt;
    switch (option) {
    case BFS_OPT_BLOCK: return o.block;
    case BFS_OPT_CTAS_PER_SM: return o.ctas_per_sm;
    case BFS_OPT_WARP_DEGREE: return o.warp_degree;
    case BFS_OPT_CTA_DEGREE: return o.cta_degree;
    case BFS_OPT_SEGMENT: return o.segment;
    case BFS_OPT_TIMEOUT_NS: return o.timeout_ns;
    case BFS_OPT_LAYER_STATS: return o.layer_stats;
    case BFS_OPT_MAX_CTAS: return o.max_ctas;
    case BFS_OPT_BATCH_WIDTH: return o.batch_width;
    case BFS_OPT_BATCH_BLOCK: return o.batch_block;
    case BFS_OPT_MODE: return o.mode;
    case BFS_OPT_ALPHA: return o.alpha;
    case BFS_OPT_BETA: return o.beta;
    case BFS_OPT_BATCH_STREAMS: return o.batch_streams;
    default: return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_get_option: unknown option");
    }
}

int bfs_run(bfs_graph *gh, int32_t root, int32_t *level_out, int32_t *parent_out, void *stream)
{
    const NvtxRange nvtx("bfs_run");
    clear_error();
    if (!gh) return set_error(BFS_ERR_INVALID_ARG, "bfs_run: NULL graph");
    Graph *g = reinterpret_cast<Graph *>(gh);
    if (root < 0 || (int64_t)root >= g->n) return set_error(BFS_ERR_INVALID_ARG, "bfs_run: root outside [0, n)");
    if (!level_out) return set_error(BFS_ERR_INVALID_ARG, "bfs_run: level_out is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g->mu);

    const bool lvl_dev = is_device_pointer(level_out);
    const bool par_dev = parent_out == nullptr || is_device_pointer(parent_out);
    int32_t *d_level = level_out, *d_parent = parent_out;
    if (!lvl_dev) {
        if (!g->d_level_tmp) GB_CUDA(cudaMalloc(&g->d_level_tmp, (size_t)g->n * 4));
        d_level = g->d_level_tmp;
    }
    if (!par_dev) {
        if (!g->d_parent_tmp) GB_CUDA(cudaMalloc(&g->d_parent_tmp, (size_t)g->n * 4));
        d_parent = g->d_parent_tmp;
    }
    // one workspace: a run on another stream waits for the previous run
    if (g->ran && s != g->last_stream) GB_CUDA(cudaStreamWaitEvent(s, g->ws_event, 0));
    if (g->opt.mode != MODE_BINNED && g->opt.block == 1024)
        return set_error(BFS_ERR_INVALID_ARG, "bfs_run: modes 0, 2 and 3 take BLOCK 256 or 512");
    int rc;
    if (g->opt.mode == MODE_BINNED) {
        rc = alloc_binned(g);
        if (rc != BFS_OK) return rc;
        rc = td_launch(g, root, d_level, d_parent, s);
    } else if (g->opt.mode == MODE_RESTORE) {
        rc = alloc_restore(g);
        if (rc != BFS_OK) return rc;
        rc = td_warp_launch(g, root, d_level, d_parent, s, MODE_RESTORE);
    } else if (g->opt.mode == MODE_HYBRID) {
        rc = alloc_hybrid(g);
        if (rc != BFS_OK) return rc;
        rc = td_warp_launch(g, root, d_level, d_parent, s, MODE_HYBRID);
    } else if (g->opt.mode == MODE_THIN) {
        rc = td_warp_launch(g, root, d_level, d_parent, s, MODE_THIN);
    } else {
        rc = td_warp_launch(g, root, d_level, d_parent, s);
    }
    if (rc != BFS_OK) return rc;
    if (!lvl_dev) GB_CUDA(cudaMemcpyAsync(level_out, d_level, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
    if (!par_dev) GB_CUDA(cudaMemcpyAsync(parent_out, d_parent, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaEventRecord(g->ws_event, s));
    g->last_stream = s;
    g->ran = true;
    return BFS_OK;
}

int bfs_graph_status(bfs_graph *gh)
{
    clear_error();
    if (!gh) return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_status: NULL graph");
    Graph *g = reinterpret_cast<Graph *>(gh);
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->ran) GB_CUDA(cudaEventSynchronize(g->ws_event));
    unsigned st = 0;
    GB_CUDA(cudaMemcpy(&st, &g->d_ctrl->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st) GB_CUDA(cudaMemset(&g->d_ctrl->status, 0, sizeof(unsigned)));
    if (st & ST_BOUNDS) {
        unsigned long long w = 0;
        GB_CUDA(cudaMemcpy(&w, &g->d_ctrl->bounds, sizeof(w), cudaMemcpyDeviceToHost));
        GB_CUDA(cudaMemset(&g->d_ctrl->bounds, 0, sizeof(w)));
        return set_error(BFS_ERR_CUDA, std::string("bfs_run: index out of range in ") + bounds_site_name(w) +
                                           " (index " + std::to_string((long long)(w & 0xFFFFFFFFFFFFull)) + ")");
    }
    if (st & ST_TIMEOUT) return set_error(BFS_ERR_TIMEOUT, "bfs_run: a device-side wait ran out (BFS_OPT_TIMEOUT_NS)");
    if (st & ST_OVERFLOW) return set_error(BFS_ERR_CUDA, "bfs_run: a frontier queue append ran past its capacity");
    return BFS_OK;
}

int bfs_graph_layer_stats(bfs_graph *gh, int64_t *vertices, int64_t *edges, int64_t *traversed, int32_t max_layers)
{
    clear_error();
    if (!gh || max_layers < 0 || (max_layers > 0 && (!vertices || !edges || !traversed)))
        return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_layer_stats: bad argument");
    Graph *g = reinterpret_cast<Graph *>(gh);
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->ran) GB_CUDA(cudaEventSynchronize(g->ws_event));
    unsigned layers = 0;
    GB_CUDA(cudaMemcpy(&layers, &g->d_ctrl->layers, sizeof(unsigned), cudaMemcpyDeviceToHost));
    int64_t buf[4 * kMaxStatLayers];
    GB_CUDA(cudaMemcpy(buf, g->d_stats, sizeof(buf), cudaMemcpyDeviceToHost));
    int L = (int)std::min<unsigned>(layers, kMaxStatLayers);
    for (int d = 0; d < L && d < max_layers; ++d) {
        vertices[d] = buf[4 * d + 0];
        edges[d] = buf[4 * d + 1];
        traversed[d] = buf[4 * d + 2];
    }
    return L;
}

int bfs_graph_layer_times(bfs_graph *gh, int64_t *t_end_ns, int32_t max_layers)
{
    clear_error();
    if (!gh || max_layers < 0 || (max_layers > 0 && !t_end_ns))
        return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_layer_times: bad argument");
    Graph *g = reinterpret_cast<Graph *>(gh);
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->ran) GB_CUDA(cudaEventSynchronize(g->ws_event));
    unsigned layers = 0;
    GB_CUDA(cudaMemcpy(&layers, &g->d_ctrl->layers, sizeof(unsigned), cudaMemcpyDeviceToHost));
    int64_t buf[4 * kMaxStatLayers];
    GB_CUDA(cudaMemcpy(buf, g->d_stats, sizeof(buf), cudaMemcpyDeviceToHost));
    int L = (int)std::min<unsigned>(layers, kMaxStatLayers);
    for (int d = 0; d < L && d < max_layers; ++d) t_end_ns[d] = buf[4 * d + 3];
    return L;
}

int bfs_graph_visited_bitmap(bfs_graph *gh, uint32_t *words_out, int64_t nwords)
{
    clear_error();
    if (!gh || !words_out) return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_visited_bitmap: bad argument");
    Graph *g = reinterpret_cast<Graph *>(gh);
    const int64_t need = (g->n + 31) / 32;
    if (nwords < need) return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_visited_bitmap: nwords < ceil(n/32)");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->ran) GB_CUDA(cudaEventSynchronize(g->ws_event));
    uint32_t *d_out = nullptr;
    GB_CUDA(cudaMalloc(&d_out, (size_t)need * 4));
    int rc = bitmap_to_caller(g, d_out);
    if (rc == BFS_OK) {
        cudaError_t e = cudaMemcpy(words_out, d_out, (size_t)need * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpy(bitmap)");
    }
    cudaFree(d_out);
    return rc;
}

int bfs_run_batch(bfs_graph *gh, const int32_t *roots, int32_t k, uint8_t *level_out)
{
    const NvtxRange nvtx("bfs_run_batch");
    clear_error();
    if (!gh) return set_error(BFS_ERR_INVALID_ARG, "bfs_run_batch: NULL graph");
    if (k < 0 || (k > 0 && (!roots || !level_out))) return set_error(BFS_ERR_INVALID_ARG, "bfs_run_batch: bad argument");
    Graph *g = reinterpret_cast<Graph *>(gh);
    for (int32_t i = 0; i < k; ++i)
        if (roots[i] < 0 || (int64_t)roots[i] >= g->n) return set_error(BFS_ERR_INVALID_ARG, "bfs_run_batch: a root is outside [0, n)");
    if (k == 0) return BFS_OK;
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->ran) GB_CUDA(cudaEventSynchronize(g->ws_event));
    return ms_run_batch(g, roots, k, level_out);
}

}  // extern "C"
