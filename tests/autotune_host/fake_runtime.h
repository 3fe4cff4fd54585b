// fake_runtime.h -- knobs of the host-only stand-in for the runtime under
// the autotuner (fake_runtime.cpp).
#pragma once

#include <stdint.h>

#include <vector>

#include "internal.cuh"

namespace fake {

extern int cost_model;             // 1: the direction-optimising mode is the faster one
extern int fail_block;             // bfs_run fails while BLOCK has this value
extern bool fail_all;              // every search fails
extern bool fail_batch;            // every batched search fails
extern int reject_warp_degree;     // bfs_graph_set_option refuses this WARP_DEGREE
extern std::vector<int32_t> roots_run;  // roots of every bfs_run, in order
extern int batch_calls;

double single_cost(const gbbfs::Options &o);  // ms of one bfs_run
double batch_cost(const gbbfs::Options &o);   // ms of one bfs_run_batch

}  // namespace fake
