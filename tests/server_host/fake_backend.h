// fake_backend.h -- knobs of the host-only stand-in for the device side of
// the serving loop (fake_backend.cpp).
#pragma once

#include <stdint.h>

#include <atomic>

#include "internal.cuh"
#include "msbfs.cuh"

namespace fake {

extern std::atomic<int64_t> device_free;      // bytes cudaMalloc may still hand out
extern std::atomic<int> pull_mode;            // batches with all lanes >= 2 iterations old look heavy
extern std::atomic<int> timeout_graph_n;      // steps of the graph with this n report ST_TIMEOUT
extern std::atomic<int> never_finish_root;    // a lane on this root never ends, and reports nothing
extern std::atomic<int> stuck_root;           // a lane on this root stays alive while steps run no iteration
extern std::atomic<int> deep_root;            // a lane on this root runs deep_depth iterations
extern std::atomic<int> deep_depth;
extern std::atomic<int> slow_graph_n;         // steps of the graph with this n sleep slow_step_us
extern std::atomic<int> slow_step_us;
extern std::atomic<int> injections_during_pull;  // queries put into a batch in its heavy phase
extern std::atomic<int> pull_seen;                // rounds that ended with a batch in its heavy phase
extern std::atomic<int> steps;
extern std::atomic<int> min_share;            // smallest grid share seen by a step
extern std::atomic<int> jitter_us;            // each step sleeps a pseudo-random time below this

int depth(int32_t root);                      // iterations a query on `root` runs
uint8_t level_of(int64_t n, int32_t root, int64_t v);  // its level row

}  // namespace fake
