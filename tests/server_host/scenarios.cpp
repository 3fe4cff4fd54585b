// scenarios.cpp -- drives the serving loop of server.cu, built for the host
// against fake_backend.cpp, through its C ABI.  One scenario per run:
//   server_host <scenario>      prints "ok" and exits 0, or names the
//                               failed check and exits 1.
#include <stdio.h>
#include <stdlib.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "fake_backend.h"

using gbbfs::Graph;

#define CHECK(cond)                                                             \
    do {                                                                        \
        if (!(cond)) {                                                          \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            exit(1);                                                            \
        }                                                                       \
    } while (0)

namespace {

Graph *make_graph(int64_t n, int64_t m)
{
    Graph *g = new Graph();
    g->n = n;
    g->m = m;
    g->num_sms = 4;
    g->symmetric = true;
    g->n_nonzero = n;
    return g;
}

// The server's admission size of one graph's workspace (restated here so
// that a budget can be chosen to hold exactly one of them).
int64_t ws_bytes(const Graph *g)
{
    const int64_t n = g->n, fcap = n + 2 * (g->m / 256) + 2;
    return n * (8 * 4 + 64 + 4) + fcap * 4 * 6 + 64 * n + (1 << 20);
}

constexpr int64_t kOneWorkspace = -1;

struct Query {
    int gi = 0;
    int32_t root = 0;
    std::vector<uint8_t> buf;
    uint64_t ticket = 0;
};

struct Bench {
    std::vector<Graph *> graphs;
    std::vector<int> ids;
    bfs_server *s = nullptr;

    // budget: bytes, 0 = the server's default, kOneWorkspace = room for the
    // largest graph's workspace only
    Bench(std::vector<int64_t> ns, int64_t budget)
    {
        for (int64_t n : ns) graphs.push_back(make_graph(n, 16 * n));
        if (budget == kOneWorkspace) {
            budget = 0;
            for (Graph *g : graphs) budget = std::max(budget, ws_bytes(g) + 1000);
        }
        s = bfs_server_create(budget);
        CHECK(s);
        for (Graph *g : graphs) {
            ids.push_back(bfs_server_add_graph(s, reinterpret_cast<bfs_graph *>(g)));
            CHECK(ids.back() == (int)ids.size() - 1);
        }
    }
    ~Bench()
    {
        if (s) bfs_server_destroy(s);
        for (Graph *g : graphs) delete g;
    }
    int submit(Query &q)
    {
        q.buf.assign((size_t)graphs[q.gi]->n, 0xAB);
        return bfs_submit(s, ids[q.gi], q.root, q.buf.data(), &q.ticket);
    }
    bool result_ok(const Query &q) const
    {
        const int64_t n = graphs[q.gi]->n;
        for (int64_t v = 0; v < n; ++v)
            if (q.buf[(size_t)v] != fake::level_of(n, q.root, v)) return false;
        return true;
    }
    // poll until the ticket is no longer running, at most limit_s seconds
    int wait(const Query &q, double limit_s = 20.0) const
    {
        const auto t0 = std::chrono::steady_clock::now();
        while (true) {
            const int st = bfs_poll(s, q.ticket);
            if (st != BFS_NOT_READY) return st;
            if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit_s) return 99;
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
    }
};

std::vector<Query> random_queries(const Bench &b, int k, unsigned seed)
{
    std::mt19937 rng(seed);
    std::vector<Query> qs((size_t)k);
    for (auto &q : qs) {
        q.gi = (int)(rng() % b.graphs.size());
        q.root = (int32_t)(rng() % (uint32_t)b.graphs[q.gi]->n);
    }
    return qs;
}

// Submit from a producer thread with occasional pauses, then drain.
int submit_mixed(Bench &b, std::vector<Query> &qs, unsigned seed)
{
    std::thread producer([&] {
        std::mt19937 rng(seed);
        for (auto &q : qs) {
            CHECK(b.submit(q) == BFS_OK);
            if (rng() % 8 == 0) std::this_thread::sleep_for(std::chrono::microseconds(rng() % 300));
        }
    });
    producer.join();
    return bfs_server_drain(b.s);
}

// ---- scenarios ---------------------------------------------------------------

// Queries on three graphs arriving while others run: every result lands in
// its own buffer, lanes are recycled (far more queries than 64 lanes), and
// the ticket times are ordered.
void mixed()
{
    Bench b({1000, 3000, 700}, 0);
    auto qs = random_queries(b, 3000, 1);
    CHECK(submit_mixed(b, qs, 2) == BFS_OK);
    for (auto &q : qs) {
        CHECK(bfs_poll(b.s, q.ticket) == BFS_OK);
        CHECK(b.result_ok(q));
        int64_t t0 = 0, t1 = 0;
        CHECK(bfs_ticket_times(b.s, q.ticket, &t0, &t1) == BFS_OK);
        CHECK(t1 >= t0 && t0 > 0);
    }
    CHECK(fake::min_share.load() >= 1);
    // the monitoring counters of an idle server
    for (int gi = 0; gi < 3; ++gi) {
        int64_t st[7];
        CHECK(bfs_server_graph_stats(b.s, gi, st) == BFS_OK);
        CHECK(st[0] == 0 && st[1] == 0 && st[2] > 0 && st[3] > 0 && st[4] == 1 && st[5] >= 0 && st[6] == 0);
    }
    int64_t st[7];
    CHECK(bfs_server_graph_stats(b.s, 3, st) == BFS_ERR_INVALID_ARG);
    CHECK(bfs_server_graph_stats(b.s, 0, nullptr) == BFS_ERR_INVALID_ARG);
}

// An HBM budget that holds one workspace at a time: graphs take turns, every
// query completes, and all device memory comes back at shutdown.
void tight_budget()
{
    const int64_t free0 = fake::device_free.load();
    {
        Bench b({1000, 3000, 2000}, kOneWorkspace);
        auto qs = random_queries(b, 600, 3);
        CHECK(submit_mixed(b, qs, 4) == BFS_OK);
        for (auto &q : qs) {
            CHECK(bfs_poll(b.s, q.ticket) == BFS_OK);
            CHECK(b.result_ok(q));
        }
    }
    CHECK(fake::device_free.load() == free0);
}

// The device has room for one workspace only, although the budget allows
// more: a graph whose allocation fails waits while another holds one, and
// gets it once that graph is idle.
void device_oom_wait()
{
    fake::device_free = 600'000;  // 164 B per vertex: n = 2000 or 3000 fits, not both
    Bench b({2000, 3000}, int64_t(1) << 40);
    auto qs = random_queries(b, 400, 5);
    CHECK(submit_mixed(b, qs, 6) == BFS_OK);
    for (auto &q : qs) {
        CHECK(bfs_poll(b.s, q.ticket) == BFS_OK);
        CHECK(b.result_ok(q));
    }
}

// A graph whose workspace the device can never hold: its queries fail with
// BFS_ERR_OOM, the other graph's queries complete, and the server keeps
// serving.
void device_oom_fail()
{
    fake::device_free = 400'000;  // n = 1000 fits (164 KB), n = 3000 (492 KB) never does
    Bench b({1000, 3000}, int64_t(1) << 40);
    auto qs = random_queries(b, 300, 7);
    CHECK(submit_mixed(b, qs, 8) == BFS_OK);
    int failed = 0;
    for (auto &q : qs) {
        const int st = bfs_poll(b.s, q.ticket);
        if (q.gi == 1) {
            CHECK(st == BFS_ERR_OOM);
            ++failed;
        } else {
            CHECK(st == BFS_OK);
            CHECK(b.result_ok(q));
        }
    }
    CHECK(failed > 0);
    Query again;
    again.gi = 0;
    again.root = 17;
    CHECK(b.submit(again) == BFS_OK);
    CHECK(b.wait(again) == BFS_OK);
    CHECK(b.result_ok(again));
}

// Poll the monitoring counters of graph gi until pred holds (at most 10 s).
template <class Pred>
bool await_stats(const Bench &b, int gi, Pred pred)
{
    const auto t0 = std::chrono::steady_clock::now();
    int64_t st[7];
    while (std::chrono::steady_clock::now() - t0 < std::chrono::seconds(10)) {
        CHECK(bfs_server_graph_stats(b.s, gi, st) == BFS_OK);
        if (pred(st)) return true;
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    return false;
}

// A query that waits longer than the room limit (1.5 s in this build) for
// its graph's workspace fails with BFS_ERR_BUSY; later queries are served.
void room_limit()
{
    Bench b({3000, 2000}, kOneWorkspace);
    fake::deep_root = 11;
    fake::deep_depth = 240;      // 60 rounds of 4 iterations
    fake::slow_graph_n = 3000;
    fake::slow_step_us = 40000;  // about 2.4 s in all, longer than the room limit
    Query deep;
    deep.gi = 0;
    deep.root = 11;
    CHECK(b.submit(deep) == BFS_OK);
    // the deep query holds the one workspace the budget allows
    CHECK(await_stats(b, 0, [](const int64_t *st) { return st[1] == 1 && st[4] == 1; }));
    Query starved;
    starved.gi = 1;
    starved.root = 5;
    CHECK(b.submit(starved) == BFS_OK);
    // its graph's worker waits for room, the query queued
    CHECK(await_stats(b, 1, [](const int64_t *st) { return st[6] == 6; }));
    {
        int64_t st[7];
        CHECK(bfs_server_graph_stats(b.s, 1, st) == BFS_OK);
        CHECK(st[0] == 1 && st[1] == 0 && st[4] == 0);
    }
    CHECK(b.wait(starved) == BFS_ERR_BUSY);
    int64_t t0 = 0, t1 = 0;
    CHECK(bfs_ticket_times(b.s, starved.ticket, &t0, &t1) == BFS_OK);
    CHECK(t1 - t0 >= 1'450'000'000);
    CHECK(b.wait(deep) == BFS_OK);
    CHECK(b.result_ok(deep));
    Query later;
    later.gi = 1;
    later.root = 6;
    CHECK(b.submit(later) == BFS_OK);
    CHECK(b.wait(later) == BFS_OK);
    CHECK(b.result_ok(later));
}

// A device-side timeout fails every outstanding query with BFS_ERR_TIMEOUT,
// drain reports it, new queries are refused, and shutdown does not hang.
void timeout()
{
    fake::timeout_graph_n = 1000;
    Bench b({1000, 700}, 0);
    auto qs = random_queries(b, 200, 9);
    // the failure may come while queries are still being submitted: those
    // are refused with the server's error
    std::vector<Query *> taken;
    for (auto &q : qs) {
        const int rc = b.submit(q);
        CHECK(rc == BFS_OK || rc == BFS_ERR_TIMEOUT);
        if (rc == BFS_OK) taken.push_back(&q);
    }
    CHECK(bfs_server_drain(b.s) == BFS_ERR_TIMEOUT);
    for (Query *qp : taken) {
        const Query &q = *qp;
        const int st = bfs_poll(b.s, q.ticket);
        CHECK(st == BFS_OK || st == BFS_ERR_TIMEOUT);
        if (q.gi == 0) CHECK(st == BFS_ERR_TIMEOUT);
        if (st == BFS_OK) CHECK(b.result_ok(q));
    }
    Query q;
    q.gi = 1;
    CHECK(b.submit(q) == BFS_ERR_TIMEOUT);
}

// A lane whose search never ends and never reports a depth overflow (a
// broken kernel): the host backstop ends it with BFS_ERR_DEPTH.
void depth_backstop()
{
    fake::never_finish_root = 5;
    Bench b({1000}, 0);
    Query q;
    q.root = 5;
    CHECK(b.submit(q) == BFS_OK);
    CHECK(bfs_server_drain(b.s) == BFS_ERR_DEPTH);
    CHECK(bfs_poll(b.s, q.ticket) == BFS_ERR_DEPTH);
}

// A query deeper than 254 levels: the device's own ST_DEPTH report ends it.
void kernel_depth()
{
    fake::deep_root = 7;
    fake::deep_depth = 300;
    Bench b({1000}, 0);
    Query q;
    q.root = 7;
    CHECK(b.submit(q) == BFS_OK);
    CHECK(bfs_server_drain(b.s) == BFS_ERR_DEPTH);
    CHECK(bfs_poll(b.s, q.ticket) == BFS_ERR_DEPTH);
}

// While a batch is in its heavy (pull) phase, waiting queries are not put
// into it; they join once it ends, and every query completes.
void pull_hold()
{
    fake::pull_mode = 1;
    Bench b({1000, 2000}, 0);
    auto qs = random_queries(b, 2000, 11);
    CHECK(submit_mixed(b, qs, 12) == BFS_OK);
    for (auto &q : qs) {
        CHECK(bfs_poll(b.s, q.ticket) == BFS_OK);
        CHECK(b.result_ok(q));
    }
    CHECK(fake::pull_seen.load() > 0);
    CHECK(fake::injections_during_pull.load() == 0);
}

// Eight graphs, Poisson-like arrivals in bursts with buffers recycled as
// queries finish (the serving measurement's pattern), steps of random
// length, the pull-phase hold active, and a budget that holds only some of
// the workspaces at once: every query completes, with its own result.
void stress()
{
    fake::pull_mode = 1;
    fake::jitter_us = 300;
    std::vector<int64_t> ns = {300, 700, 1000, 1500, 2000, 2500, 3000, 4000};
    int64_t budget = 0;
    {
        std::vector<int64_t> w;
        for (int64_t n : ns) {
            Graph *g = make_graph(n, 16 * n);
            w.push_back(ws_bytes(g));
            delete g;
        }
        std::sort(w.begin(), w.end());
        budget = w[7] + w[6] + w[5] + 1000;  // the three largest at once
    }
    Bench b(ns, budget);
    std::mt19937 rng(21);
    for (int run = 0; run < 3; ++run) {
        auto qs = random_queries(b, 4000, 100 + run);
        for (size_t i = 0; i < qs.size(); ++i) {
            CHECK(b.submit(qs[i]) == BFS_OK);
            if (rng() % 16 == 0) std::this_thread::sleep_for(std::chrono::microseconds(rng() % 2000));
        }
        for (auto &q : qs) {
            CHECK(b.wait(q, 30.0) == BFS_OK);
            CHECK(b.result_ok(q));
        }
    }
    CHECK(fake::injections_during_pull.load() == 0);
}

// A query submitted while another query's search runs joins that search
// (continuous batching): its record shows the lanes already busy and the
// iteration at which it joined; times and iterations are ordered.
void join_record()
{
    fake::deep_root = 7;
    fake::deep_depth = 200;
    fake::slow_graph_n = 1000;  // 2 ms per round: the long search runs about 0.1 s
    fake::slow_step_us = 2000;
    Bench b({1000}, 0);
    Query lq, q;
    lq.root = 7;
    q.root = 3;
    CHECK(b.submit(lq) == BFS_OK);
    int64_t st[7] = {};
    for (int i = 0; i < 20000; ++i) {  // until the long search has run a few rounds
        CHECK(bfs_server_graph_stats(b.s, 0, st) == BFS_OK);
        if (st[3] >= 8) break;
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    CHECK(st[3] >= 8);
    CHECK(b.submit(q) == BFS_OK);
    CHECK(b.wait(q) == BFS_OK);
    CHECK(b.result_ok(q));
    bfs_ticket_record r{}, l{};
    CHECK(bfs_ticket_info(b.s, q.ticket, &r) == BFS_OK);
    CHECK(r.lanes_busy_at_join == 1 && r.join_iter >= 8 && r.done_iter > r.join_iter);
    CHECK(r.t_submit_ns > 0 && r.t_admit_ns >= r.t_submit_ns && r.t_done_ns >= r.t_admit_ns);
    CHECK(bfs_server_drain(b.s) == BFS_OK);
    CHECK(b.result_ok(lq));
    CHECK(bfs_ticket_info(b.s, lq.ticket, &l) == BFS_OK);
    CHECK(l.lanes_busy_at_join == 0 && l.join_iter == 0 && l.lane != r.lane && l.done_iter >= 200);
    CHECK(bfs_ticket_info(b.s, 0, &l) == BFS_ERR_INVALID_ARG);
}

// A search that keeps a lane alive while its steps run no iteration (a
// lost frontier) makes the worker fail the queries instead of relaunching
// empty searches forever.
void no_progress()
{
    fake::stuck_root = 5;
    Bench b({1000}, 0);
    Query q;
    q.root = 5;
    CHECK(b.submit(q) == BFS_OK);
    CHECK(bfs_server_drain(b.s) == BFS_ERR_CUDA);
    CHECK(bfs_poll(b.s, q.ticket) == BFS_ERR_CUDA);
}

// A graph registered with a live server may not be released (its worker may
// still search it): graph_release_check, the guard of bfs_graph_destroy,
// refuses it with BFS_ERR_BUSY until every server holding it is destroyed.
void registration()
{
    Graph *g = make_graph(1000, 16000);
    CHECK(gbbfs::graph_release_check(g) == BFS_OK);
    bfs_server *a = bfs_server_create(0), *b = bfs_server_create(0);
    CHECK(a && b);
    CHECK(bfs_server_add_graph(a, reinterpret_cast<bfs_graph *>(g)) == 0);
    CHECK(bfs_server_add_graph(b, reinterpret_cast<bfs_graph *>(g)) == 0);
    CHECK(bfs_server_add_graph(a, reinterpret_cast<bfs_graph *>(g)) == BFS_ERR_INVALID_ARG);  // twice
    CHECK(gbbfs::graph_release_check(g) == BFS_ERR_BUSY);
    Query q;
    std::vector<uint8_t> buf((size_t)g->n, 0xAB);
    CHECK(bfs_submit(a, 0, 5, buf.data(), &q.ticket) == BFS_OK);
    CHECK(bfs_server_destroy(a) == BFS_OK);
    CHECK(gbbfs::graph_release_check(g) == BFS_ERR_BUSY);  // still held by b
    CHECK(bfs_server_destroy(b) == BFS_OK);
    CHECK(gbbfs::graph_release_check(g) == BFS_OK);
    delete g;
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc != 2) {
        fprintf(stderr, "usage: server_host <scenario>\n");
        return 2;
    }
    alarm(60);  // a hung scenario ends the process
    const std::string s = argv[1];
    if (s == "mixed") mixed();
    else if (s == "tight_budget") tight_budget();
    else if (s == "device_oom_wait") device_oom_wait();
    else if (s == "device_oom_fail") device_oom_fail();
    else if (s == "room_limit") room_limit();
    else if (s == "timeout") timeout();
    else if (s == "depth_backstop") depth_backstop();
    else if (s == "kernel_depth") kernel_depth();
    else if (s == "pull_hold") pull_hold();
    else if (s == "stress") stress();
    else if (s == "registration") registration();
    else if (s == "join_record") join_record();
    else if (s == "no_progress") no_progress();
    else {
        fprintf(stderr, "unknown scenario %s\n", s.c_str());
        return 2;
    }
    printf("ok\n");
    return 0;
}
