// fake_backend.cpp -- a host-only stand-in for the CUDA runtime calls and
// the batched-search entry points that server.cu uses, so that the serving
// loop's scheduling (admission, eviction, lane recycling, the pull-phase
// hold, error paths) can be exercised on a machine without a GPU.
//
// "Device" memory is host memory counted against a settable capacity.  A
// lane's search is a countdown: a query on root r runs depth(r) iterations
// and its level row is level_of(g, r, v), a value that depends only on the
// graph, the root and the vertex, so a result delivered to the wrong buffer
// or from the wrong lane is visible.
#include "fake_backend.h"

#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

namespace fake {

std::atomic<int64_t> device_free{int64_t(1) << 40};
std::atomic<int> pull_mode{0};
std::atomic<int> timeout_graph_n{-1};
std::atomic<int> never_finish_root{-1};
std::atomic<int> stuck_root{-1};
std::atomic<int> deep_root{-1};
std::atomic<int> deep_depth{0};
std::atomic<int> slow_graph_n{-1};
std::atomic<int> slow_step_us{0};
std::atomic<int> injections_during_pull{0};
std::atomic<int> pull_seen{0};
std::atomic<int> steps{0};
std::atomic<int> min_share{1 << 30};
std::atomic<int> jitter_us{0};

static std::mutex alloc_mu;
static std::map<void *, size_t> allocs;

// Streams that the server creates itself defer their copies until an event
// recorded after them, or the stream, is synchronised: a copy then reads its
// source as it is at that moment, so a source overwritten before the wait
// delivers wrong rows.  The workspace streams (null here) run at once.
struct Stream {
    std::mutex mu;
    std::vector<std::function<void()>> ops;
    size_t done = 0;
};
struct Event {
    Stream *s = nullptr;
    size_t upto = 0;
};
static std::mutex streams_mu;
static std::set<const void *> streams;

static Stream *as_stream(cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(streams_mu);
    return streams.count((const void *)st) ? reinterpret_cast<Stream *>(st) : nullptr;
}

static void run_until(Stream *s, size_t upto)
{
    std::lock_guard<std::mutex> lk(s->mu);
    while (s->done < upto && s->done < s->ops.size()) s->ops[s->done++]();
}

int depth(int32_t root) { return root == deep_root.load() ? deep_depth.load() : 1 + (int)(root % 9); }

uint8_t level_of(int64_t n, int32_t root, int64_t v)
{
    return (uint8_t)((root * 7 + v * 13 + n) % 251);
}

}  // namespace fake

// ---- CUDA runtime stand-ins (the declarations come from cuda_runtime_api.h)
extern "C" {

cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaGetDevice(int *d)
{
    *d = 0;
    return cudaSuccess;
}
cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr a, int)
{
    *v = a == cudaDevAttrMultiProcessorCount ? 4 : 0;
    return cudaSuccess;
}
cudaError_t cudaDeviceGetStreamPriorityRange(int *least, int *greatest)
{
    *least = 0;
    *greatest = -5;
    return cudaSuccess;
}
cudaError_t cudaMemGetInfo(size_t *free_b, size_t *total_b)
{
    *free_b = (size_t)fake::device_free.load();
    *total_b = *free_b;
    return cudaSuccess;
}
cudaError_t cudaMalloc(void **p, size_t size)
{
    std::lock_guard<std::mutex> lk(fake::alloc_mu);
    if ((int64_t)size > fake::device_free.load()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    *p = malloc(size ? size : 1);
    fake::allocs[*p] = size;
    fake::device_free -= (int64_t)size;
    return cudaSuccess;
}
cudaError_t cudaFree(void *p)
{
    if (!p) return cudaSuccess;
    std::lock_guard<std::mutex> lk(fake::alloc_mu);
    auto it = fake::allocs.find(p);
    if (it == fake::allocs.end()) return cudaErrorInvalidValue;
    fake::device_free += (int64_t)it->second;
    fake::allocs.erase(it);
    free(p);
    return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t count, cudaMemcpyKind, cudaStream_t st)
{
    if (fake::Stream *s = fake::as_stream(st)) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->ops.push_back([dst, src, count] { memcpy(dst, src, count); });
        return cudaSuccess;
    }
    memcpy(dst, src, count);
    return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t st)
{
    if (fake::Stream *s = fake::as_stream(st)) fake::run_until(s, SIZE_MAX);
    return cudaSuccess;
}
cudaError_t cudaStreamCreateWithPriority(cudaStream_t *st, unsigned int, int)
{
    fake::Stream *s = new fake::Stream();
    std::lock_guard<std::mutex> lk(fake::streams_mu);
    fake::streams.insert(s);
    *st = reinterpret_cast<cudaStream_t>(s);
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t st)
{
    fake::Stream *s = fake::as_stream(st);
    if (!s) return cudaErrorInvalidValue;
    fake::run_until(s, SIZE_MAX);
    {
        std::lock_guard<std::mutex> lk(fake::streams_mu);
        fake::streams.erase(s);
    }
    delete s;
    return cudaSuccess;
}
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *ev, unsigned int)
{
    *ev = reinterpret_cast<cudaEvent_t>(new fake::Event());
    return cudaSuccess;
}
cudaError_t cudaEventDestroy(cudaEvent_t ev)
{
    delete reinterpret_cast<fake::Event *>(ev);
    return cudaSuccess;
}
cudaError_t cudaEventRecord(cudaEvent_t ev, cudaStream_t st)
{
    fake::Event *e = reinterpret_cast<fake::Event *>(ev);
    e->s = fake::as_stream(st);
    if (e->s) {
        std::lock_guard<std::mutex> lk(e->s->mu);
        e->upto = e->s->ops.size();
    }
    return cudaSuccess;
}
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned int) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t ev)
{
    fake::Event *e = reinterpret_cast<fake::Event *>(ev);
    if (e->s) fake::run_until(e->s, e->upto);
    return cudaSuccess;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char *cudaGetErrorName(cudaError_t) { return "fake"; }
const char *cudaGetErrorString(cudaError_t) { return "fake"; }

}  // extern "C"

// ---- library internals that server.cu calls ------------------------------
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
    return set_error(e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA, what);
}
void clear_error()
{
    t_status = BFS_OK;
    t_msg.clear();
}

namespace {

struct Lane {
    bool on = false;
    int32_t root = 0;
    int left = 0;
    unsigned start = 0;
};

// MsWs first, so that the server's cast of batch_ws to MsWs reads it.
struct FakeWs {
    MsWs ws;
    MsCtrl ctrl{};
    Lane lanes[64];
    void *mem = nullptr;  // the workspace's share of "device" memory
};
static_assert(offsetof(FakeWs, ws) == 0, "MsWs must come first");

FakeWs *fws(Graph *g) { return reinterpret_cast<FakeWs *>(g->batch_ws); }

}  // namespace

int ms_alloc(Graph *g, MsWs **out)
{
    if (g->batch_ws) {
        *out = &fws(g)->ws;
        return BFS_OK;
    }
    FakeWs *f = new FakeWs();
    const cudaError_t e = cudaMalloc(&f->mem, (size_t)g->n * 100);
    if (e != cudaSuccess) {
        delete f;
        return cuda_error(e, "fake ms_alloc");
    }
    g->batch_ws = f;
    *out = &f->ws;
    return BFS_OK;
}

void ms_free(Graph *g)
{
    FakeWs *f = fws(g);
    if (!f) return;
    cudaFree(f->mem);
    delete f;
    g->batch_ws = nullptr;
}

int ms_reset(Graph *) { return BFS_OK; }

// The server's pull test, restated for the fake's own counters.
static bool in_pull(const Graph *g, const MsCtrl &c)
{
    const int par = (int)(c.iter & 1);
    return g->symmetric && c.alive[par] && (long long)c.fedges[par] * 16 > g->m &&
           (double)c.seen_pairs >= 0.3 * (double)__builtin_popcountll(c.alive[par]) * (double)g->n_nonzero;
}

int ms_inject(Graph *g, const int32_t *src, unsigned long long mask)
{
    FakeWs *f = fws(g);
    if (fake::pull_mode.load() && in_pull(g, f->ctrl)) ++fake::injections_during_pull;
    const int par = (int)(f->ctrl.iter & 1);
    for (int i = 0; i < 64; ++i) {
        if (!((mask >> i) & 1ull)) continue;
        if (f->lanes[i].on) return set_error(BFS_ERR_CUDA, "fake: lane injected twice");
        f->lanes[i] = Lane{true, src[i], fake::depth(src[i]), f->ctrl.iter};
        f->ctrl.alive[par] |= 1ull << i;
    }
    return BFS_OK;
}

int ms_step_capped(Graph *g, uint32_t max_iters, int max_ctas)
{
    FakeWs *f = fws(g);
    MsCtrl &c = f->ctrl;
    ++fake::steps;
    if (max_ctas < fake::min_share.load()) fake::min_share = max_ctas;
    if (g->n == fake::slow_graph_n.load())
        std::this_thread::sleep_for(std::chrono::microseconds(fake::slow_step_us.load()));
    if (fake::jitter_us.load() > 0) {
        thread_local unsigned x = 12345u + (unsigned)(uintptr_t)g;
        x = x * 1664525u + 1013904223u;
        std::this_thread::sleep_for(std::chrono::microseconds((x >> 8) % (unsigned)fake::jitter_us.load()));
    }
    if (g->n == fake::timeout_graph_n.load()) {
        c.status |= ST_TIMEOUT;
        return BFS_OK;
    }
    // a faulty search: a lane on stuck_root stays alive while no iteration runs
    for (int i = 0; i < 64; ++i)
        if (((c.alive[c.iter & 1] >> i) & 1ull) && f->lanes[i].root == fake::stuck_root.load()) return BFS_OK;
    for (uint32_t it = 0; it < max_iters; ++it) {
        const int par = (int)(c.iter & 1);
        if (!c.alive[par]) break;
        unsigned long long next = 0;
        for (int i = 0; i < 64; ++i) {
            if (!((c.alive[par] >> i) & 1ull)) continue;
            Lane &l = f->lanes[i];
            const bool forever = l.root == fake::never_finish_root.load();
            if (!forever && (int)(c.iter + 1 - l.start) > 254) c.status |= ST_DEPTH;
            if (forever || --l.left > 0) next |= 1ull << i;
        }
        c.alive[par] = 0;
        c.alive[par ^ 1] = next;
        ++c.iter;
        // in pull mode, a batch whose lanes are all at least two iterations
        // old looks like one in its heavy phase
        bool old = next != 0;
        for (int i = 0; i < 64; ++i)
            if (((next >> i) & 1ull) && c.iter - f->lanes[i].start < 2) old = false;
        const int np = (int)(c.iter & 1);
        c.fedges[np] = (fake::pull_mode.load() && old) ? (unsigned long long)g->m : 0ull;
        c.seen_pairs = (fake::pull_mode.load() && old) ? (unsigned long long)(64 * g->n) : 0ull;
    }
    return BFS_OK;
}

int ms_step(Graph *g, uint32_t max_iters) { return ms_step_capped(g, max_iters, 0); }

int ms_read_ctrl(Graph *g, MsCtrl *out)
{
    if (fake::pull_mode.load() && in_pull(g, fws(g)->ctrl)) ++fake::pull_seen;
    *out = fws(g)->ctrl;
    return BFS_OK;
}

// Half of the callers' buffers (by address) count as device-addressable, so
// that every scenario runs both delivery paths: rows stored by the kernel
// (deferred on the copy stream like a copy) and rows copied.
bool ms_host_addressable(const void *p, uint8_t **dev_ptr)
{
    if (!((reinterpret_cast<uintptr_t>(p) >> 4) & 1u)) return false;
    *dev_ptr = static_cast<uint8_t *>(const_cast<void *>(p));
    return true;
}

int ms_rows_to_host(const uint8_t *stage, int64_t n, const RowsToHost &job, cudaStream_t stream)
{
    for (int i = 0; i < job.count; ++i) {
        const cudaError_t e = cudaMemcpyAsync(job.dst[i], stage + (size_t)job.rows[i] * n, (size_t)n,
                                              cudaMemcpyDeviceToHost, stream);
        if (e != cudaSuccess) return set_error(BFS_ERR_CUDA, "fake: row store");
    }
    return BFS_OK;
}

int ms_extract(Graph *g, unsigned long long mask, const int32_t *row, uint8_t *out, int64_t stride, bool recycle)
{
    FakeWs *f = fws(g);
    for (int i = 0; i < 64; ++i) {
        if (!((mask >> i) & 1ull)) continue;
        Lane &l = f->lanes[i];
        if (!l.on) return set_error(BFS_ERR_CUDA, "fake: extracting a free lane");
        if (row && row[i] >= 0)
            for (int64_t v = 0; v < g->n; ++v) out[(size_t)row[i] * stride + v] = fake::level_of(g->n, l.root, v);
        if (recycle) l.on = false;
    }
    return BFS_OK;
}

}  // namespace gbbfs
