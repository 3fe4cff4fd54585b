// fake_runtime.cpp -- a host-only stand-in for what autotune.cu calls: the
// CUDA runtime (events, streams, allocation, one copy), the option setters
// and the search entry points.  A search "costs" a time that a scenario's
// cost model derives from the graph's options; events read a clock that
// each bfs_run advances by that cost, and bfs_run_batch sleeps for its cost,
// so the autotuner's choices can be checked against a known optimum.
#include "fake_runtime.h"

#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <thread>

namespace fake {

int cost_model = 0;
int fail_block = -1;
bool fail_all = false;
bool fail_batch = false;
int reject_warp_degree = -1;
std::vector<int32_t> roots_run;
int batch_calls = 0;

static double clock_ms = 0.0;  // advanced by every bfs_run
static std::map<cudaEvent_t, double> events;
static int next_handle = 1;

static double l2(double x) { return std::log2(x); }

double single_cost(const gbbfs::Options &o)
{
    double t = 0.0;
    switch (o.mode) {
    case 0: t = 10.0; break;
    case 1: t = 20.0 + std::fabs(l2(o.warp_degree) - 3) + std::fabs(l2(o.cta_degree) - 12) +
                std::fabs(l2(o.segment) - 10);
        break;
    case 3: t = (cost_model == 1 ? 6.0 : 12.0) + 0.5 * std::fabs(l2(o.alpha) - 3) + 0.3 * std::fabs(l2(o.beta) - 6);
        break;
    case 4: t = cost_model == 2 ? 7.0 : 13.0; break;
    default: t = 30.0;
    }
    return t + (o.block == 512 ? 1.0 : 0.0);
}

double batch_cost(const gbbfs::Options &o)
{
    const double w = o.batch_width == 64 ? 4.0 : o.batch_width == 32 ? 8.0 : 12.0;
    // batches in flight at once help up to four, then the shares get small
    const double streams = o.batch_streams == 4 ? 0.0 : o.batch_streams == 2 ? 0.5 : 1.0;
    return w - (o.batch_block == 512 ? 2.0 : 0.0) + streams;
}

}  // namespace fake

extern "C" {

cudaError_t cudaMalloc(void **p, size_t size)
{
    *p = malloc(size ? size : 1);
    return cudaSuccess;
}
cudaError_t cudaFree(void *p)
{
    free(p);
    return cudaSuccess;
}
cudaError_t cudaMemcpy(void *dst, const void *src, size_t count, cudaMemcpyKind)
{
    memcpy(dst, src, count);
    return cudaSuccess;
}
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned int)
{
    *s = reinterpret_cast<cudaStream_t>((intptr_t)fake::next_handle++);
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t *e)
{
    *e = reinterpret_cast<cudaEvent_t>((intptr_t)fake::next_handle++);
    return cudaSuccess;
}
cudaError_t cudaEventDestroy(cudaEvent_t e)
{
    fake::events.erase(e);
    return cudaSuccess;
}
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t)
{
    fake::events[e] = fake::clock_ms;
    return cudaSuccess;
}
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t a, cudaEvent_t b)
{
    *ms = (float)(fake::events[b] - fake::events[a]);
    return cudaSuccess;
}

}  // extern "C"

namespace gbbfs {

static thread_local int t_status = BFS_OK;

int set_error(int status, const std::string &)
{
    t_status = status;
    return status;
}
int cuda_error(cudaError_t, const char *what) { return set_error(BFS_ERR_CUDA, what); }
void clear_error() { t_status = BFS_OK; }

}  // namespace gbbfs

using gbbfs::Graph;

extern "C" {

int bfs_last_status(void) { return gbbfs::t_status; }

int bfs_graph_set_option(bfs_graph *gh, int option, int64_t v)
{
    Graph *g = reinterpret_cast<Graph *>(gh);
    gbbfs::Options &o = g->opt;
    switch (option) {
    case BFS_OPT_MODE: o.mode = (int)v; break;
    case BFS_OPT_BLOCK: o.block = (int)v; break;
    case BFS_OPT_WARP_DEGREE:
        if (v == fake::reject_warp_degree) return gbbfs::set_error(BFS_ERR_INVALID_ARG, "rejected");
        o.warp_degree = (int)v;
        break;
    case BFS_OPT_CTA_DEGREE: o.cta_degree = (int)v; break;
    case BFS_OPT_SEGMENT: o.segment = (int)v; break;
    case BFS_OPT_ALPHA: o.alpha = (int)v; break;
    case BFS_OPT_BETA: o.beta = (int)v; break;
    case BFS_OPT_BATCH_WIDTH: o.batch_width = (int)v; break;
    case BFS_OPT_BATCH_BLOCK: o.batch_block = (int)v; break;
    case BFS_OPT_BATCH_STREAMS: o.batch_streams = (int)v; break;
    default: return gbbfs::set_error(BFS_ERR_INVALID_ARG, "unknown option");
    }
    return BFS_OK;
}

int64_t bfs_graph_get_option(const bfs_graph *gh, int option)
{
    const gbbfs::Options &o = reinterpret_cast<const Graph *>(gh)->opt;
    switch (option) {
    case BFS_OPT_MODE: return o.mode;
    case BFS_OPT_BLOCK: return o.block;
    case BFS_OPT_WARP_DEGREE: return o.warp_degree;
    case BFS_OPT_CTA_DEGREE: return o.cta_degree;
    case BFS_OPT_SEGMENT: return o.segment;
    case BFS_OPT_ALPHA: return o.alpha;
    case BFS_OPT_BETA: return o.beta;
    case BFS_OPT_BATCH_WIDTH: return o.batch_width;
    case BFS_OPT_BATCH_BLOCK: return o.batch_block;
    case BFS_OPT_BATCH_STREAMS: return o.batch_streams;
    default: return -1;
    }
}

int bfs_run(bfs_graph *gh, int32_t root, int32_t *, int32_t *, void *)
{
    Graph *g = reinterpret_cast<Graph *>(gh);
    if (fake::fail_all || g->opt.block == fake::fail_block) return gbbfs::set_error(BFS_ERR_CUDA, "fake failure");
    fake::roots_run.push_back(root);
    fake::clock_ms += fake::single_cost(g->opt);
    return BFS_OK;
}

int bfs_run_batch(bfs_graph *gh, const int32_t *, int32_t, uint8_t *)
{
    Graph *g = reinterpret_cast<Graph *>(gh);
    if (fake::fail_all || fake::fail_batch) return gbbfs::set_error(BFS_ERR_CUDA, "fake failure");
    ++fake::batch_calls;
    std::this_thread::sleep_for(std::chrono::microseconds((int)(1000 * fake::batch_cost(g->opt))));
    return BFS_OK;
}

int bfs_graph_status(bfs_graph *) { return BFS_OK; }

}  // extern "C"
