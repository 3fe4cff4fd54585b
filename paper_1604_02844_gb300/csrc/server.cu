// server.cu -- continuous-batching BFS request loop over resident graphs.
//
// Not in the paper.  Queries (graph, root) are served by the bit-parallel
// search of msbfs.cu.  Each graph with work owns a 64-lane workspace and a
// worker thread with its own CUDA stream, which repeats:
//   1. put waiting queries into free lanes of the running search (a lane
//      that joins at iteration t reports levels iter + 1 - t) -- unless the
//      search is in its heavy pull phase, which young lanes would keep from
//      pulling: then they wait one round and join together;
//   2. advance the search 4 iterations (one cooperative launch on the
//      graph's own stream, its grid capped to a share of the GPU so that
//      several graphs' searches run on the device at the same time);
//   3. read which lanes still have a frontier; the others are finished:
//      their level columns are extracted into staging rows and the lanes
//      reset, free for the next queries at once; on a second stream, while
//      the next round runs, the rows reach the callers' buffers (stored by
//      one kernel into pinned buffers, copied into pageable ones), and the
//      queries complete once they have landed.
// A workspace is created only while the device memory it needs fits the
// server's budget; a graph with no running or waiting query gives its
// workspace back when another graph needs the room.  Queries wait at most
// kRoomWaitNs for room; past that, or when the device itself cannot hold the
// workspace, the graph's waiting queries fail (the server keeps running).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "msbfs.cuh"

namespace gbbfs {
namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    int graph = 0;
    int32_t root = 0;
    uint8_t *out = nullptr;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    int lane = -1;
    int lanes_busy = 0;                 // lanes of the running search when this one joined
    int64_t join_iter = -1, done_iter = -1;  // search iterations at joining and at the round that finished it
    std::atomic<int> status{BFS_NOT_READY};
};

// What a graph's worker is doing (bfs_server_graph_stats).
enum Phase : int {
    PH_IDLE = 0,       // waiting for work
    PH_ADMIT = 1,      // admitting queries into lanes
    PH_INJECT = 2,     // putting the new lanes' sources on the device
    PH_STEP = 3,       // launching iterations
    PH_READ = 4,       // reading the control block (waits for the iterations)
    PH_FINISH = 5,     // delivering finished lanes' results
    PH_ROOM_WAIT = 6,  // waiting for workspace room
    PH_STOPPED = 7,
};

struct GraphState {
    Graph *g = nullptr;
    std::deque<uint64_t> waiting;     // tickets (under Server::mu)
    uint64_t lane_ticket[64] = {};
    unsigned lane_iter0[64] = {};     // search iteration at which each lane joined (worker thread only)
    unsigned long long running = 0;   // occupied lanes (under Server::mu)
    bool has_ws = false;              // (under Server::mu)
    int64_t ws_bytes = 0;
    uint8_t *d_stage = nullptr;       // [64][n] extraction rows
    cudaStream_t copy_stream = nullptr;  // delivery of finished lanes' rows (kernel stores, copies)
    cudaEvent_t ev_rows = nullptr, ev_copied = nullptr;  // rows extracted; rows copied out
    unsigned long long pending = 0;   // lanes whose rows are being copied out (under Server::mu)
    uint64_t pending_ticket[64] = {};
    int64_t pending_iter = -1;
    MsCtrl last{};                    // counters after the previous round (worker thread only)
    bool have_last = false;
    int64_t room_wait_since = 0;      // start of the current wait for room, 0 = none (under Server::mu)
    // monitoring (read by other threads without the lock)
    std::atomic<int> phase{PH_IDLE};
    std::atomic<int64_t> rounds{0}, last_iter{-1}, t_round_end{0};
    std::thread worker;
    std::condition_variable cv;
};

// Device bytes of one graph's serving workspace (msbfs workspace + rows).
int64_t workspace_bytes(const Graph *g)
{
    const int64_t n = g->n, fcap = n + 2 * (g->m / 256) + 2;
    return n * (8 * 4 + 64 + 4) + fcap * 4 * 6 + 64 * n + (1 << 20);
}

// Longest wait of a query for workspace room; a build may shorten it (the
// host-only tests of this loop do).
#ifndef GBBFS_ROOM_WAIT_NS
#define GBBFS_ROOM_WAIT_NS 60000000000LL
#endif
constexpr int64_t kRoomWaitNs = GBBFS_ROOM_WAIT_NS;

}  // namespace

struct Server {
    int64_t budget = 0, used = 0;
    int device = 0;
    int total_ctas = 0;
    uint32_t iters_per_step = 4;  // iterations per round (1, 2, 4, 8, 16 measured: 4 best)
    std::vector<std::unique_ptr<GraphState>> graphs;
    std::vector<std::unique_ptr<Request>> reqs;  // ticket = index + 1
    std::mutex mu;
    std::condition_variable done_cv;
    bool stop = false;
    int64_t outstanding = 0;
    int error = BFS_OK;

    void run(GraphState &gs);
    int round(GraphState &gs);
    int finish(GraphState &gs, unsigned long long mask);
    int deliver(GraphState &gs);
    static void free_ws(GraphState &gs);
    int ensure_ws(GraphState &gs);                 // with mu held
    void evict_idle(GraphState &gs, int64_t need);  // with mu held
    int alloc_ws(GraphState &gs);
    void fail_waiting(GraphState &gs, int rc);     // with mu held
    void fail_all(int rc);
};

// With mu held.  Drops the workspaces of graphs other than gs that have
// nothing running or waiting (their workers are idle and their streams are
// drained) until `need` more bytes fit the budget; need < 0 drops them all.
void Server::evict_idle(GraphState &gs, int64_t need)
{
    for (auto &o : graphs) {
        if (need >= 0 && used + need <= budget) break;
        if (o.get() != &gs && o->has_ws && o->running == 0 && o->waiting.empty() && o->pending == 0) {
            free_ws(*o);
            used -= o->ws_bytes;
        }
    }
}

// A graph's workspace, staging rows, copy stream and events, given back.
void Server::free_ws(GraphState &gs)
{
    if (gs.copy_stream) {
        cudaStreamSynchronize(gs.copy_stream);
        cudaStreamDestroy(gs.copy_stream);
    }
    if (gs.ev_rows) cudaEventDestroy(gs.ev_rows);
    if (gs.ev_copied) cudaEventDestroy(gs.ev_copied);
    gs.copy_stream = nullptr;
    gs.ev_rows = gs.ev_copied = nullptr;
    ms_free(gs.g);
    cudaFree(gs.d_stage);
    gs.d_stage = nullptr;
    gs.has_ws = false;
}

// The batched-search workspace and the extraction rows of one graph.
int Server::alloc_ws(GraphState &gs)
{
    MsWs *w = nullptr;
    int rc = ms_alloc(gs.g, &w);
    if (rc != BFS_OK) {
        ms_free(gs.g);  // a workspace left without its reset is not reused
        return rc;
    }
    cudaError_t e = cudaMalloc(&gs.d_stage, (size_t)64 * gs.g->n);
    if (e != cudaSuccess) {
        rc = cuda_error(e, "server: extraction rows");
        gs.d_stage = nullptr;
        ms_free(gs.g);
        return rc;
    }
    if ((e = cudaStreamCreateWithPriority(&gs.copy_stream, cudaStreamNonBlocking, gs.g->stream_priority)) !=
            cudaSuccess ||
        (e = cudaEventCreateWithFlags(&gs.ev_rows, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&gs.ev_copied, cudaEventDisableTiming)) != cudaSuccess) {
        rc = cuda_error(e, "server: copy stream");
        free_ws(gs);
        return rc;
    }
    return BFS_OK;
}

// With mu held.  BFS_OK once gs has its workspace; BFS_NOT_READY while it
// has to wait for room (over the budget, or the device short of memory while
// other graphs hold workspaces that they give back when idle); another
// status when the device cannot hold it.
int Server::ensure_ws(GraphState &gs)
{
    if (gs.has_ws) return BFS_OK;
    const int64_t need = workspace_bytes(gs.g);
    // smaller graphs (shorter searches) get higher stream priorities, so
    // that their few CTAs are scheduled ahead of the large searches' ones
    {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        int rank = 0, count = 0;
        for (auto &o : graphs) {
            ++count;
            if (o->g->m < gs.g->m || (o->g->m == gs.g->m && o.get() < &gs)) ++rank;
        }
        gs.g->stream_priority = count > 1 ? greatest + (least - greatest) * rank / (count - 1) : least;
    }
    if (used + need > budget) {
        evict_idle(gs, need);
        if (used + need > budget) return BFS_NOT_READY;
    }
    int rc = alloc_ws(gs);
    if (rc == BFS_ERR_OOM) {  // less free device memory than the budget assumed
        evict_idle(gs, -1);
        rc = alloc_ws(gs);
    }
    if (rc == BFS_ERR_OOM)
        for (auto &o : graphs)
            if (o.get() != &gs && o->has_ws) return BFS_NOT_READY;
    if (rc != BFS_OK) return rc;
    gs.has_ws = true;
    gs.ws_bytes = need;
    used += need;
    gs.running = 0;
    gs.have_last = false;  // a new workspace starts at iteration 0
    return BFS_OK;
}

// With mu held.  The graph's waiting queries fail with rc; the server and
// the other graphs carry on.
void Server::fail_waiting(GraphState &gs, int rc)
{
    const int64_t t = now_ns();
    for (uint64_t tk : gs.waiting) {
        Request &r = *reqs[tk - 1];
        r.t_done = t;
        r.status.store(rc);
        --outstanding;
    }
    gs.waiting.clear();
    done_cv.notify_all();
}

// Finished lanes: their rows go to the staging buffer and the lanes are
// reset (free for new queries at once); the rows then reach the callers'
// buffers on the copy stream (kernel stores into pinned buffers, copies into
// pageable ones), which overlaps the graph's next round.
// The staging rows of an earlier delivery are released first.
int Server::finish(GraphState &gs, unsigned long long mask)
{
    if (!mask) return BFS_OK;
    int rc = deliver(gs);
    if (rc != BFS_OK) return rc;
    int32_t rows[64];
    for (int i = 0; i < 64; ++i) rows[i] = ((mask >> i) & 1ull) ? i : -1;
    rc = ms_extract(gs.g, mask, rows, gs.d_stage, gs.g->n, true);
    if (rc != BFS_OK) return rc;
    MsWs *w = reinterpret_cast<MsWs *>(gs.g->batch_ws);
    cudaError_t e = cudaEventRecord(gs.ev_rows, w->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(gs.copy_stream, gs.ev_rows, 0);
    if (e != cudaSuccess) return cuda_error(e, "server: result copy");
    // rows for pinned (device-addressable) buffers are stored by one kernel,
    // the others copied
    RowsToHost job;
    job.count = 0;
    for (int i = 0; i < 64; ++i) {
        if (!((mask >> i) & 1ull)) continue;
        uint8_t *out;
        {
            std::lock_guard<std::mutex> lk(mu);
            out = reqs[gs.lane_ticket[i] - 1]->out;
        }
        uint8_t *dev = nullptr;
        if (ms_host_addressable(out, &dev)) {
            job.dst[job.count] = dev;
            job.rows[job.count] = i;
            ++job.count;
            continue;
        }
        e = cudaMemcpyAsync(out, gs.d_stage + (size_t)i * gs.g->n, (size_t)gs.g->n, cudaMemcpyDeviceToHost,
                            gs.copy_stream);
        if (e != cudaSuccess) return cuda_error(e, "server: result copy");
    }
    rc = ms_rows_to_host(gs.d_stage, gs.g->n, job, gs.copy_stream);
    if (rc != BFS_OK) return rc;
    e = cudaEventRecord(gs.ev_copied, gs.copy_stream);
    if (e != cudaSuccess) return cuda_error(e, "server: result copy");
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < 64; ++i) {
        if (!((mask >> i) & 1ull)) continue;
        gs.pending_ticket[i] = gs.lane_ticket[i];
        gs.lane_ticket[i] = 0;
    }
    gs.pending_iter = gs.have_last ? (int64_t)gs.last.iter : -1;
    gs.pending = mask;
    gs.running &= ~mask;
    return BFS_OK;
}

// Wait for the rows being copied out, then complete their queries.
int Server::deliver(GraphState &gs)
{
    if (!gs.pending) return BFS_OK;  // written by this worker only
    const cudaError_t e = cudaEventSynchronize(gs.ev_copied);
    if (e != cudaSuccess) return cuda_error(e, "server: result copy");
    const int64_t t = now_ns();
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < 64; ++i) {
        if (!((gs.pending >> i) & 1ull)) continue;
        Request &r = *reqs[gs.pending_ticket[i] - 1];
        r.t_done = t;
        r.done_iter = gs.pending_iter;
        r.status.store(BFS_OK);
        gs.pending_ticket[i] = 0;
        --outstanding;
    }
    gs.pending = 0;
    done_cv.notify_all();
    return BFS_OK;
}

// Would the next iteration of this batch be a pull step, were no lane
// younger than two iterations?  (The kernel's test in msbfs.cu.)  While it
// would, new queries wait a round: joining now would keep the batch pushing.
static bool pull_phase(const Graph *g, const MsCtrl &st, unsigned long long running)
{
    const int par = (int)(st.iter & 1);
    const unsigned long long live = st.alive[par] & running;
    return g->symmetric && live && (long long)st.fedges[par] * 16 > g->m &&
           (double)st.seen_pairs >= 0.3 * (double)__builtin_popcountll(live) * (double)g->n_nonzero;
}

// One round for one graph: waiting queries into free lanes (unless the
// batch is in its pull phase), a few iterations, finished lanes out.
int Server::round(GraphState &gs)
{
    const NvtxRange nvtx("bfs_server round");
    unsigned long long add = 0, running;
    int32_t src[64] = {0};
    int active = 1;
    gs.phase = PH_ADMIT;
    {
        std::lock_guard<std::mutex> lk(mu);
        int ws = ensure_ws(gs);
        if (ws != BFS_OK) {
            if (ws == BFS_NOT_READY) {  // no room yet: the queries wait, for a while
                const int64_t t = now_ns();
                if (!gs.room_wait_since) gs.room_wait_since = t;
                if (t - gs.room_wait_since <= kRoomWaitNs) return BFS_NOT_READY;
                ws = set_error(BFS_ERR_BUSY, "server: no room for the graph's workspace");
            }
            fail_waiting(gs, ws);
            gs.room_wait_since = 0;
            return BFS_OK;
        }
        gs.room_wait_since = 0;
        const bool hold = gs.running && gs.have_last && pull_phase(gs.g, gs.last, gs.running);
        const int busy = __builtin_popcountll(gs.running);
        const int64_t t_admit = now_ns();
        while (!hold && !gs.waiting.empty() && (gs.running | add) != ~0ull) {
            const int lane = __builtin_ctzll(~(gs.running | add));
            const uint64_t t = gs.waiting.front();
            gs.waiting.pop_front();
            gs.lane_ticket[lane] = t;
            gs.lane_iter0[lane] = gs.have_last ? gs.last.iter : 0u;
            Request &r = *reqs[t - 1];
            src[lane] = r.root;
            r.t_admit = t_admit;
            r.lane = lane;
            r.lanes_busy = busy;
            r.join_iter = (int64_t)gs.lane_iter0[lane];
            add |= 1ull << lane;
        }
        gs.running |= add;
        running = gs.running;
        active = 0;
        for (auto &o : graphs)
            if (o->running) ++active;
    }
    if (add) {
        gs.phase = PH_INJECT;
        const int rc = ms_inject(gs.g, src, add);
        if (rc != BFS_OK) return rc;
    }
    if (!running) return deliver(gs);
    // the GPU's CTAs (of 256 threads) shared among the graphs with work, but
    // no more than the graph's size calls for (one CTA per 2^16 adjacency
    // entries), so that small graphs leave room for the large ones; a graph
    // set to 512-thread CTAs gets half as many
    const int per_cta = gs.g->opt.batch_block == 512 ? 2 : 1;
    const int needed = (int)std::min<int64_t>(std::max<int64_t>(1, (gs.g->m + 65535) / 65536), total_ctas);
    const int share = std::max(1, std::min(needed, std::max(gs.g->num_sms, total_ctas / std::max(1, active))) / per_cta);
    gs.phase = PH_STEP;
    const bool had_last = gs.have_last;
    const unsigned iter_before = gs.last.iter;
    int rc = ms_step_capped(gs.g, iters_per_step, share);
    if (rc != BFS_OK) return rc;
    // the previous round's results land while these iterations run
    gs.phase = PH_FINISH;
    rc = deliver(gs);
    if (rc != BFS_OK) return rc;
    MsCtrl &st = gs.last;
    gs.phase = PH_READ;
    rc = ms_read_ctrl(gs.g, &st);
    if (rc != BFS_OK) return rc;
    gs.have_last = true;
    // Backstop: a step with live lanes always advances the iteration counter
    // unless the search has no frontier left; lanes still marked alive then
    // can never finish, so their queries end with an error instead of the
    // worker relaunching empty searches forever.
    if (had_last && !add && st.iter == iter_before && (running & st.alive[st.iter & 1]) &&
        !(st.status & (ST_TIMEOUT | ST_OVERFLOW | ST_DEPTH | ST_BOUNDS)))
        return set_error(BFS_ERR_CUDA, "server: a batched search made no progress with queries still running");
    gs.last_iter = (int64_t)st.iter;
    if (st.status & (ST_TIMEOUT | ST_OVERFLOW | ST_DEPTH | ST_BOUNDS))
        return set_error(st.status & ST_DEPTH ? BFS_ERR_DEPTH : (st.status & ST_TIMEOUT ? BFS_ERR_TIMEOUT : BFS_ERR_CUDA),
                         "server: device-side error in a batched search");
    // Backstop: a lane still searching 300 iterations after it joined would
    // have levels past 254, which the kernel itself reports (ST_DEPTH); should
    // that ever fail, the query ends with an error instead of running forever.
    for (unsigned long long a = running & st.alive[st.iter & 1]; a; a &= a - 1) {
        const int lane = __builtin_ctzll(a);
        if (st.iter - gs.lane_iter0[lane] > 300u)
            return set_error(BFS_ERR_DEPTH, "server: a query kept searching past 254 levels");
    }
    gs.phase = PH_FINISH;
    return finish(gs, running & ~st.alive[st.iter & 1]);
}

void Server::fail_all(int rc)
{
    std::lock_guard<std::mutex> lk(mu);
    if (error == BFS_OK) error = rc;
    // queries whose rows are being copied out end when their copy has landed
    // (their workers see to it as they stop): the buffers are in use till then
    std::vector<char> copying(reqs.size(), 0);
    int64_t in_copy = 0;
    for (auto &gs : graphs)
        for (int i = 0; i < 64; ++i)
            if ((gs->pending >> i) & 1ull) {
                copying[gs->pending_ticket[i] - 1] = 1;
                ++in_copy;
            }
    for (size_t k = 0; k < reqs.size(); ++k) {
        Request &r = *reqs[k];
        if (!copying[k] && r.status.load() == BFS_NOT_READY) {
            r.status.store(rc);
            r.t_done = now_ns();
        }
    }
    for (auto &gs : graphs) {
        gs->waiting.clear();
        gs->running = 0;
    }
    outstanding = in_copy;
    done_cv.notify_all();
    for (auto &gs : graphs) gs->cv.notify_all();
}

void Server::run(GraphState &gs)
{
    cudaSetDevice(device);
    while (true) {
        gs.phase = PH_IDLE;
        {
            std::unique_lock<std::mutex> lk(mu);
            gs.cv.wait(lk, [&] { return stop || error != BFS_OK || !gs.waiting.empty() || gs.running || gs.pending; });
            if (stop || error != BFS_OK) break;
        }
        const int rc = round(gs);
        ++gs.rounds;
        gs.t_round_end = now_ns();
        if (rc == BFS_NOT_READY) {  // waiting for HBM budget
            gs.phase = PH_ROOM_WAIT;
            std::this_thread::sleep_for(std::chrono::microseconds(200));
            continue;
        }
        if (rc != BFS_OK) {
            fail_all(rc);
            break;
        }
    }
    // rows still being copied out: their queries end once the copy has landed
    if (gs.pending && deliver(gs) != BFS_OK) {
        std::lock_guard<std::mutex> lk(mu);
        for (int i = 0; i < 64; ++i) {
            if (!((gs.pending >> i) & 1ull)) continue;
            Request &r = *reqs[gs.pending_ticket[i] - 1];
            r.t_done = now_ns();
            r.status.store(BFS_ERR_CUDA);
            gs.pending_ticket[i] = 0;
            --outstanding;
        }
        gs.pending = 0;
        done_cv.notify_all();
    }
    gs.phase = PH_STOPPED;
}

}  // namespace gbbfs

using namespace gbbfs;

extern "C" {

bfs_server *bfs_server_create(int64_t hbm_budget_bytes)
{
    clear_error();
    if (hbm_budget_bytes < 0) {
        set_error(BFS_ERR_INVALID_ARG, "bfs_server_create: negative budget");
        return nullptr;
    }
    nvtxInitialize(nullptr);  // once, before any worker thread names a range
    Server *s = new (std::nothrow) Server();
    if (!s) {
        set_error(BFS_ERR_OOM, "bfs_server_create: host allocation");
        return nullptr;
    }
    cudaGetDevice(&s->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    s->total_ctas = 4 * sms;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->budget = hbm_budget_bytes > 0 ? hbm_budget_bytes : (int64_t)(0.8 * (double)free_b);
    return reinterpret_cast<bfs_server *>(s);
}

int bfs_server_destroy(bfs_server *sh)
{
    if (!sh) return BFS_OK;
    Server *s = reinterpret_cast<Server *>(sh);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto &gs : s->graphs) gs->cv.notify_all();
    }
    for (auto &gs : s->graphs)
        if (gs->worker.joinable()) gs->worker.join();
    for (auto &gs : s->graphs) {
        if (gs->has_ws) Server::free_ws(*gs);
        gs->g->stream_priority = 0;
        gs->g->servers.fetch_sub(1);  // the graph may be destroyed again
    }
    delete s;
    return BFS_OK;
}

int bfs_server_add_graph(bfs_server *sh, bfs_graph *gh)
{
    clear_error();
    if (!sh || !gh) return set_error(BFS_ERR_INVALID_ARG, "bfs_server_add_graph: NULL argument");
    Server *s = reinterpret_cast<Server *>(sh);
    Graph *g = reinterpret_cast<Graph *>(gh);
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &gs : s->graphs)
        if (gs->g == g) return set_error(BFS_ERR_INVALID_ARG, "bfs_server_add_graph: graph already added");
    {
        // the server manages the graph's batch workspace from now on
        std::lock_guard<std::mutex> glk(g->mu);
        ms_free(g);
    }
    auto gs = std::make_unique<GraphState>();
    gs->g = g;
    g->servers.fetch_add(1);  // bfs_graph_destroy refuses it until this server is destroyed
    GraphState *raw = gs.get();
    s->graphs.push_back(std::move(gs));
    raw->worker = std::thread([s, raw] { s->run(*raw); });
    return (int)s->graphs.size() - 1;
}

int bfs_submit(bfs_server *sh, int graph_id, int32_t root, uint8_t *level_out, uint64_t *ticket)
{
    clear_error();
    if (!sh || !level_out || !ticket) return set_error(BFS_ERR_INVALID_ARG, "bfs_submit: NULL argument");
    Server *s = reinterpret_cast<Server *>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error != BFS_OK) return set_error(s->error, "bfs_submit: the server stopped after an error");
    if (graph_id < 0 || graph_id >= (int)s->graphs.size()) return set_error(BFS_ERR_INVALID_ARG, "bfs_submit: unknown graph id");
    GraphState &gs = *s->graphs[graph_id];
    if (root < 0 || (int64_t)root >= gs.g->n) return set_error(BFS_ERR_INVALID_ARG, "bfs_submit: root outside [0, n)");
    if (workspace_bytes(gs.g) > s->budget)
        return set_error(BFS_ERR_BUSY, "bfs_submit: the graph's workspace exceeds the server's HBM budget");
    auto r = std::make_unique<Request>();
    r->graph = graph_id;
    r->root = root;
    r->out = level_out;
    r->t_submit = now_ns();
    s->reqs.push_back(std::move(r));
    const uint64_t t = s->reqs.size();
    gs.waiting.push_back(t);
    ++s->outstanding;
    *ticket = t;
    gs.cv.notify_one();
    return BFS_OK;
}

int bfs_poll(bfs_server *sh, uint64_t ticket)
{
    if (!sh) return set_error(BFS_ERR_INVALID_ARG, "bfs_poll: NULL server");
    Server *s = reinterpret_cast<Server *>(sh);
    Request *r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (ticket == 0 || ticket > s->reqs.size()) return set_error(BFS_ERR_INVALID_ARG, "bfs_poll: unknown ticket");
        r = s->reqs[ticket - 1].get();
    }
    const int st = r->status.load();
    if (st < 0) set_error(st, "bfs_poll: the query failed");
    return st;
}

int bfs_server_drain(bfs_server *sh)
{
    if (!sh) return set_error(BFS_ERR_INVALID_ARG, "bfs_server_drain: NULL server");
    Server *s = reinterpret_cast<Server *>(sh);
    std::unique_lock<std::mutex> lk(s->mu);
    s->done_cv.wait(lk, [&] { return s->outstanding == 0 || s->error != BFS_OK; });
    return s->error;
}

int bfs_server_graph_stats(bfs_server *sh, int graph_id, int64_t *out)
{
    if (!sh || !out) return set_error(BFS_ERR_INVALID_ARG, "bfs_server_graph_stats: NULL argument");
    Server *s = reinterpret_cast<Server *>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    if (graph_id < 0 || graph_id >= (int)s->graphs.size())
        return set_error(BFS_ERR_INVALID_ARG, "bfs_server_graph_stats: unknown graph id");
    const GraphState &gs = *s->graphs[graph_id];
    out[0] = (int64_t)gs.waiting.size();
    out[1] = __builtin_popcountll(gs.running);
    out[2] = gs.rounds.load();
    out[3] = gs.last_iter.load();
    out[4] = gs.has_ws ? 1 : 0;
    const int64_t t = gs.t_round_end.load();
    out[5] = t ? now_ns() - t : -1;
    out[6] = gs.phase.load();
    return BFS_OK;
}

int bfs_ticket_times(bfs_server *sh, uint64_t ticket, int64_t *t_submit_ns, int64_t *t_done_ns)
{
    if (!sh || !t_submit_ns || !t_done_ns) return set_error(BFS_ERR_INVALID_ARG, "bfs_ticket_times: NULL argument");
    Server *s = reinterpret_cast<Server *>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket > s->reqs.size()) return set_error(BFS_ERR_INVALID_ARG, "bfs_ticket_times: unknown ticket");
    Request &r = *s->reqs[ticket - 1];
    *t_submit_ns = r.t_submit;
    *t_done_ns = r.t_done;
    return BFS_OK;
}

int bfs_ticket_info(bfs_server *sh, uint64_t ticket, bfs_ticket_record *out)
{
    if (!sh || !out) return set_error(BFS_ERR_INVALID_ARG, "bfs_ticket_info: NULL argument");
    Server *s = reinterpret_cast<Server *>(sh);
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket > s->reqs.size()) return set_error(BFS_ERR_INVALID_ARG, "bfs_ticket_info: unknown ticket");
    const Request &r = *s->reqs[ticket - 1];
    out->t_submit_ns = r.t_submit;
    out->t_admit_ns = r.t_admit;
    out->t_done_ns = r.t_done;
    out->join_iter = r.join_iter;
    out->done_iter = r.done_iter;
    out->graph_id = r.graph;
    out->lane = r.lane;
    out->lanes_busy_at_join = r.lanes_busy;
    out->reserved = 0;
    return BFS_OK;
}

}  // extern "C"
