// scenarios.cpp -- drives bfs_graph_autotune (autotune.cu), built for the
// host against fake_runtime.cpp, whose cost model has a known optimum.
//   autotune_host <scenario>    prints "ok" and exits 0, or names the failed
//                               check and exits 1.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "fake_runtime.h"

using gbbfs::Graph;

#define CHECK(cond)                                                             \
    do {                                                                        \
        if (!(cond)) {                                                          \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            exit(1);                                                            \
        }                                                                       \
    } while (0)

namespace {

constexpr int64_t kN = 1000, kNonzero = 900;
std::vector<int32_t> orig((size_t)kN);  // internal id -> caller id

std::vector<std::unique_ptr<Graph>> owned;  // freed at exit

Graph *make_graph()
{
    for (int64_t i = 0; i < kN; ++i) orig[(size_t)i] = (int32_t)((i * 7919) % kN);
    owned.push_back(std::make_unique<Graph>());
    Graph *g = owned.back().get();
    g->n = kN;
    g->m = 16 * kN;
    g->n_nonzero = kNonzero;
    g->d_orig = orig.data();
    return g;
}

bfs_graph *H(Graph *g) { return reinterpret_cast<bfs_graph *>(g); }

// Mode 0 starts at BLOCK 512; the model makes 256 faster.
void single_mode0()
{
    Graph *g = make_graph();
    const gbbfs::Options before = g->opt;
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE, 0) == BFS_OK);
    CHECK(g->opt.mode == 0 && g->opt.block == 256);
    CHECK(g->opt.alpha == before.alpha && g->opt.batch_width == before.batch_width);
    CHECK(fake::batch_calls == 0);
}

// The faster mode is chosen first, then that mode's options: mode 3 with
// alpha 8 and beta 64, the model's optimum.
void mode_then_single()
{
    fake::cost_model = 1;
    Graph *g = make_graph();
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_MODE | BFS_TUNE_SINGLE, 4) == BFS_OK);
    CHECK(g->opt.mode == 3);
    CHECK(g->opt.alpha == 8 && g->opt.beta == 64 && g->opt.block == 256);
}

// Mode 3 slower: the search stays top-down.
void mode_stays()
{
    Graph *g = make_graph();
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_MODE | BFS_TUNE_SINGLE, 4) == BFS_OK);
    CHECK(g->opt.mode == 0 && g->opt.block == 256);
}

// On a graph where the thin-warp expansion is fastest it is chosen, and
// its options are left as they were.
void mode_thin()
{
    fake::cost_model = 2;
    Graph *g = make_graph();
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_MODE | BFS_TUNE_SINGLE, 4) == BFS_OK);
    CHECK(g->opt.mode == 4 && g->opt.block == 512);
}

// The degree-binned mode tunes its three thresholds.
void binned()
{
    Graph *g = make_graph();
    g->opt.mode = 1;
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE, 4) == BFS_OK);
    CHECK(g->opt.warp_degree == 8 && g->opt.cta_degree == 4096 && g->opt.segment == 1024);
    CHECK(g->opt.block == 256);
}

// A candidate that the option setter refuses is skipped without error.
void rejected_value()
{
    fake::reject_warp_degree = 8;
    Graph *g = make_graph();
    g->opt.mode = 1;
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE, 4) == BFS_OK);
    CHECK(g->opt.warp_degree == 4 || g->opt.warp_degree == 16);
    CHECK(bfs_last_status() == BFS_OK);
}

// A candidate whose searches fail is never chosen; the call still succeeds.
void failing_value()
{
    fake::fail_block = 256;
    Graph *g = make_graph();
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE, 4) == BFS_OK);
    CHECK(g->opt.block == 512);
}

// When even the starting values fail, the call fails and leaves every
// option as it found it.
void all_fail()
{
    fake::fail_all = true;
    Graph *g = make_graph();
    g->opt.block = 256;
    g->opt.alpha = 32;
    const gbbfs::Options before = g->opt;
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_MODE | BFS_TUNE_SINGLE | BFS_TUNE_BATCH, 4) == BFS_ERR_CUDA);
    CHECK(g->opt.block == before.block && g->opt.alpha == before.alpha && g->opt.mode == before.mode);
    CHECK(g->opt.batch_width == before.batch_width && g->opt.batch_block == before.batch_block);
}

// A failure in a later stage (the batched path) undoes what the earlier
// stages had already set.
void late_failure()
{
    fake::fail_batch = true;
    Graph *g = make_graph();
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE | BFS_TUNE_BATCH, 4) == BFS_ERR_CUDA);
    CHECK(!fake::roots_run.empty());  // the single-source stage ran (and chose 256)
    CHECK(g->opt.block == 512);
}

// The batched path: width 64, 512-thread CTAs and four batches in flight,
// timed on the host clock.
void batch()
{
    Graph *g = make_graph();
    g->opt.batch_streams = 1;  // the descent has to find the four
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_BATCH, 4) == BFS_OK);
    CHECK(g->opt.batch_width == 64 && g->opt.batch_block == 512 && g->opt.batch_streams == 4);
    CHECK(fake::batch_calls > 0 && fake::roots_run.empty());
}

void args()
{
    Graph *g = make_graph();
    CHECK(bfs_graph_autotune(nullptr, BFS_TUNE_SINGLE, 0) == BFS_ERR_INVALID_ARG);
    CHECK(bfs_graph_autotune(H(g), 0, 0) == BFS_ERR_INVALID_ARG);
    CHECK(bfs_graph_autotune(H(g), 8, 0) == BFS_ERR_INVALID_ARG);
    CHECK(bfs_graph_autotune(H(g), -1, 0) == BFS_ERR_INVALID_ARG);
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE, -1) == BFS_ERR_INVALID_ARG);
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE, 4097) == BFS_ERR_INVALID_ARG);
    CHECK(fake::roots_run.empty());
}

// Sample roots: k vertices with edges, evenly spread over the degree order,
// given to the searches in the caller's numbering.
void samples()
{
    Graph *g = make_graph();
    const int k = 5;
    CHECK(bfs_graph_autotune(H(g), BFS_TUNE_SINGLE, k) == BFS_OK);
    std::set<int32_t> expect;
    for (int i = 0; i < k; ++i) expect.insert(orig[(size_t)((int64_t)i * kNonzero / k)]);
    CHECK(!fake::roots_run.empty());
    for (int32_t r : fake::roots_run) CHECK(expect.count(r) == 1);
    CHECK(std::set<int32_t>(fake::roots_run.begin(), fake::roots_run.end()) == expect);
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc != 2) {
        fprintf(stderr, "usage: autotune_host <scenario>\n");
        return 2;
    }
    const std::string s = argv[1];
    if (s == "single_mode0") single_mode0();
    else if (s == "mode_then_single") mode_then_single();
    else if (s == "mode_thin") mode_thin();
    else if (s == "mode_stays") mode_stays();
    else if (s == "binned") binned();
    else if (s == "rejected_value") rejected_value();
    else if (s == "failing_value") failing_value();
    else if (s == "all_fail") all_fail();
    else if (s == "late_failure") late_failure();
    else if (s == "batch") batch();
    else if (s == "args") args();
    else if (s == "samples") samples();
    else {
        fprintf(stderr, "unknown scenario %s\n", s.c_str());
        return 2;
    }
    printf("ok\n");
    return 0;
}
