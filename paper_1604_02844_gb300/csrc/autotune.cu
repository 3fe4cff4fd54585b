// autotune.cu -- per-graph choice of the tunables by measurement.
//
// Not in the paper, whose Sec. 4.1 picks the expansion of each layer by a
// fixed rule.  bfs_graph_autotune times candidate values of one option at a
// time (coordinate descent: each option's best value is kept before the next
// option is tried) on a few sample searches of the graph itself, and leaves
// the fastest values set.  Results never depend on the options, only the
// time does.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <limits>
#include <vector>

#include "internal.cuh"

namespace gbbfs {
namespace {

struct Knob {
    int option;
    std::vector<int64_t> values;
};

// Sample roots: vertices that have edges, spread evenly over the degree
// order (hubs and low-degree vertices alike), in the caller's numbering.
int sample_roots(Graph *g, int k, std::vector<int32_t> &out)
{
    out.clear();
    const int64_t span = std::max<int64_t>(g->n_nonzero, 1);
    for (int i = 0; i < k; ++i) {
        const int64_t internal = std::min<int64_t>(g->n - 1, (int64_t)i * span / k);
        int32_t r = 0;
        GB_CUDA(cudaMemcpy(&r, g->d_orig + internal, sizeof(int32_t), cudaMemcpyDeviceToHost));
        out.push_back(r);
    }
    return BFS_OK;
}

constexpr double kFailed = std::numeric_limits<double>::infinity();

// Device time (ms) of one bfs_run per root after one warm-up run; +inf if a
// run fails.
double time_single(bfs_graph *gh, const std::vector<int32_t> &roots, int32_t *d_level, int32_t *d_parent,
                   cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    if (bfs_run(gh, roots[0], d_level, d_parent, s) != BFS_OK) return kFailed;
    if (cudaEventRecord(e0, s) != cudaSuccess) return kFailed;
    for (int32_t r : roots)
        if (bfs_run(gh, r, d_level, d_parent, s) != BFS_OK) return kFailed;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return kFailed;
    if (bfs_graph_status(gh) != BFS_OK) return kFailed;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return kFailed;
    return ms;
}

// Host time (ms) of one synchronous bfs_run_batch over all roots, after one
// warm-up call; +inf if it fails.
double time_batch(bfs_graph *gh, const std::vector<int32_t> &roots, uint8_t *d_out)
{
    const int32_t k = (int32_t)roots.size();
    if (bfs_run_batch(gh, roots.data(), k, d_out) != BFS_OK) return kFailed;
    const auto t0 = std::chrono::steady_clock::now();
    if (bfs_run_batch(gh, roots.data(), k, d_out) != BFS_OK) return kFailed;
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace gbbfs

using namespace gbbfs;

extern "C" int bfs_graph_autotune(bfs_graph *gh, int what, int32_t samples)
{
    clear_error();
    if (!gh) return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_autotune: NULL graph");
    if (what <= 0 || (what & ~(BFS_TUNE_SINGLE | BFS_TUNE_BATCH | BFS_TUNE_MODE)))
        return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_autotune: `what` must combine BFS_TUNE_* bits");
    if (samples < 0 || samples > 4096) return set_error(BFS_ERR_INVALID_ARG, "bfs_graph_autotune: samples in [0, 4096]");
    if (samples == 0) samples = 8;
    Graph *g = reinterpret_cast<Graph *>(gh);
    const Options saved = g->opt;
    std::vector<int32_t> roots;
    int rc = sample_roots(g, samples, roots);
    if (rc != BFS_OK) return rc;

    int32_t *d_level = nullptr, *d_parent = nullptr;
    uint8_t *d_batch = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&](int code) {
        cudaFree(d_level);
        cudaFree(d_parent);
        cudaFree(d_batch);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        if (code != BFS_OK) g->opt = saved;
        return code;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return cleanup(cuda_error(e, "bfs_graph_autotune: stream/events"));

    // one option at a time: keep the best value before trying the next option
    auto descend = [&](const std::vector<Knob> &knobs, auto &&measure) -> int {
        for (const Knob &kb : knobs) {
            const int64_t start = bfs_graph_get_option(gh, kb.option);
            int64_t best = start;
            double best_t = measure();
            if (best_t == kFailed) return bfs_last_status() < 0 ? bfs_last_status() : BFS_ERR_CUDA;
            for (int64_t v : kb.values) {
                if (v == start) continue;
                if (bfs_graph_set_option(gh, kb.option, v) != BFS_OK) continue;
                const double t = measure();
                if (t < best_t) {
                    best_t = t;
                    best = v;
                }
            }
            bfs_graph_set_option(gh, kb.option, best);
            clear_error();
        }
        return BFS_OK;
    };

    if (what & (BFS_TUNE_SINGLE | BFS_TUNE_MODE)) {
        if ((e = cudaMalloc(&d_level, (size_t)g->n * 4)) != cudaSuccess ||
            (e = cudaMalloc(&d_parent, (size_t)g->n * 4)) != cudaSuccess)
            return cleanup(cuda_error(e, "bfs_graph_autotune: output buffers"));
        auto single = [&] { return time_single(gh, roots, d_level, d_parent, s, e0, e1); };
        if (what & BFS_TUNE_MODE) {
            // the fastest expansion whose results equal every other's: top-down
            // with staged items (mode 0) or thin warps (mode 4, faster on
            // graphs without hubs), or direction-optimising (mode 3); the
            // atomic-free and the degree-binned modes are kept for comparison
            if ((rc = descend({{BFS_OPT_MODE, {MODE_WARP, MODE_HYBRID, MODE_THIN}}}, single)) != BFS_OK)
                return cleanup(rc);
        }
        if (what & BFS_TUNE_SINGLE) {
            std::vector<Knob> knobs;
            switch (g->opt.mode) {
            case MODE_BINNED:
                knobs = {{BFS_OPT_BLOCK, {256, 512, 1024}},
                         {BFS_OPT_WARP_DEGREE, {4, 8, 16, 32}},
                         {BFS_OPT_CTA_DEGREE, {256, 1024, 4096}},
                         {BFS_OPT_SEGMENT, {1024, 4096, 16384}}};
                break;
            case MODE_HYBRID:
                knobs = {{BFS_OPT_ALPHA, {2, 4, 8, 14, 32, 64}}, {BFS_OPT_BETA, {4, 8, 24, 64, 256}},
                         {BFS_OPT_BLOCK, {256, 512}}};
                break;
            case MODE_THIN:  // its CTA size is fixed
                break;
            default:
                knobs = {{BFS_OPT_BLOCK, {256, 512}}};
                break;
            }
            if ((rc = descend(knobs, single)) != BFS_OK) return cleanup(rc);
        }
    }
    if (what & BFS_TUNE_BATCH) {
        // the same sources for every width, so that the times compare; 512
        // of them, so that several batches can be in flight (BATCH_STREAMS)
        std::vector<int32_t> broots;
        for (int i = 0; i < 512; ++i) broots.push_back(roots[i % roots.size()]);
        if ((e = cudaMalloc(&d_batch, (size_t)broots.size() * (size_t)g->n)) != cudaSuccess)
            return cleanup(cuda_error(e, "bfs_graph_autotune: batch output"));
        auto batch = [&] { return time_batch(gh, broots, d_batch); };
        if ((rc = descend({{BFS_OPT_BATCH_WIDTH, {16, 32, 64}},
                           {BFS_OPT_BATCH_BLOCK, {256, 512}},
                           {BFS_OPT_BATCH_STREAMS, {1, 2, 4, 8}}},
                          batch)) != BFS_OK)
            return cleanup(rc);
    }
    return cleanup(BFS_OK);
}
