// topdown.cu -- single-source level-synchronous top-down BFS on sm_103a.
//
// The whole search is one persistent cooperative kernel:
//   init (Alg. 1/2 initialisation: P[u] = "infinity" (-1) for u != s,
//         P[s] = s, the visited bitmap holds s only, the frontier holds s)
//   for each layer d (Sec. 3: layer L_d is finished before L_{d+1} starts):
//     expand every frontier item: for each v in its slice of Adj[u]
//       (Alg. 2 inner loop), test the visited bit (word v>>5, bit v&31,
//       Listing 1), claim it with a 32-bit atomicOr (replacing the paper's
//       restoration pass, Alg. 3), and the winner writes level[v] = d+1,
//       parent[v] = u and appends v to the next frontier (Alg. 1 "out.add");
//     grid barrier, swap frontiers (Alg. 1 "swap(in, out)")
//   until the next frontier is empty.
//
// Work split by degree.  A frontier item is (u, beg, len): a slice of Adj[u].
// Vertices of degree >= cta_degree are cut into slices of <= segment edges
// at discovery time and go to a "large" queue; each large slice is expanded
// by a whole CTA.  Other vertices go to the "small" queue, consumed in chunks
// of BLOCK items: items with len >= warp_degree are expanded by one warp,
// the rest are flattened over the CTA with a block prefix sum (each thread
// takes one edge of the concatenated short lists).  Every expansion loop is
// warp-uniform so the claim/append step can use ballot + popc.
//
// Next-frontier compaction: winners of a warp reserve slots in a CTA-local
// shared-memory buffer with one shared atomic per warp (ballot/popc ranks);
// the buffer is flushed to the global queue with one global atomicAdd per
// flush and coalesced stores.
//
// Every wait is bounded: the grid barrier gives up after timeout_ns, sets
// ST_TIMEOUT, and every CTA then leaves the kernel through the normal exit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"

namespace gbbfs {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int OB = 2048;  // CTA out-buffer capacity (small items)

struct TdParams {
    const int32_t *__restrict__ ro;
    const int32_t *__restrict__ col;
    int32_t *level;
    int32_t *parent;  // may be null
    const int32_t *__restrict__ perm;  // caller id -> internal id
    const int32_t *__restrict__ orig;  // internal id -> caller id
    uint32_t *bitmap;
    int32_t *qu[2], *qb[2], *ql[2];  // small-item queue [buffer]
    int32_t *bu[2], *bb[2], *bl[2];  // large-item queue [buffer]
    Ctrl *ctrl;
    int64_t *stats;  // [kMaxStatLayers][4] or null
    int32_t n;
    int32_t root;
    int32_t warp_degree, cta_degree, segment;
    uint32_t qcap, bqcap;
    int32_t bitmap_words;
    uint64_t timeout_ns;
};

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Bounded grid barrier (all CTAs are co-resident: cooperative launch).
// Returns false if this or another CTA gave up waiting.
__device__ bool grid_sync(Ctrl *c, unsigned nblocks, uint64_t timeout_ns, int *s_ok)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(&c->bar_gen);
        const unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            st_release(&c->bar_gen, gen + 1);
        } else {
            const uint64_t t0 = globaltimer();
            unsigned spins = 0;
            while (ld_acquire(&c->bar_gen) == gen) {
                if ((++spins & 31) == 0) {
                    if (ld_relaxed(&c->status) & ST_TIMEOUT) break;
                    if (globaltimer() - t0 > timeout_ns || spins > (1u << 30)) {
                        atomicOr(&c->status, ST_TIMEOUT);
                        break;
                    }
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        *s_ok = !(ld_relaxed(&c->status) & ST_TIMEOUT);
    }
    __syncthreads();
    return *s_ok != 0;
}

// Exclusive prefix sum over the CTA; s_warp holds >= 33 ints.
template <int BLOCK>
__device__ __forceinline__ int block_exclusive_scan(int x, int *s_warp, int &total)
{
    constexpr int WARPS = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < WARPS ? s_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    total = s_warp[32];
    return inc - x + s_warp[warp];
}

struct OutBuf {
    int32_t *u, *b, *l;
    int *cnt;
    int *gbase;
};

// Claim v for the next layer and append it.  Called by all 32 lanes of a
// warp (warp-uniform); lanes with valid == false take part in the votes only.
__device__ __forceinline__ void visit(bool valid, int v, int u, int next_level, const TdParams &p,
                                      int set_out, int qo, const OutBuf &ob, unsigned &my_new)
{
    const int lane = threadIdx.x & 31;
    bool win = false;
    if (valid) {
        const unsigned w = (unsigned)v >> 5, bit = 1u << (v & 31);
        if (!(__ldcg(p.bitmap + w) & bit)) win = !(atomicOr(p.bitmap + w, bit) & bit);
    }
    int rb = 0, len = 0;
    if (win) {
        const int ov = __ldg(p.orig + v);  // results leave in the caller's numbering
        p.level[ov] = next_level;
        if (p.parent) p.parent[ov] = __ldg(p.orig + u);
        rb = __ldg(p.ro + v);
        len = __ldg(p.ro + v + 1) - rb;
        ++my_new;
    }
    const bool small = win && len > 0 && len < p.cta_degree;
    const bool big = win && len >= p.cta_degree;
    const unsigned ms = __ballot_sync(FULL, small);
    if (ms) {
        const int cnt = __popc(ms);
        const int leader = __ffs(ms) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(ob.cnt, cnt);
        base = __shfl_sync(FULL, base, leader);
        const int over = min(cnt, max(0, base + cnt - OB));
        unsigned gbase = 0;
        if (over) {
            if (lane == leader) gbase = atomicAdd(&p.ctrl->count[set_out], (unsigned)over);
            gbase = __shfl_sync(FULL, gbase, leader);
        }
        if (small) {
            const int idx = base + __popc(ms & lanemask_lt());
            if (idx < OB) {
                ob.u[idx] = v;
                ob.b[idx] = rb;
                ob.l[idx] = len;
            } else {
                const unsigned gi = gbase + (unsigned)(idx - max(base, OB));
                if (gi < p.qcap) {
                    p.qu[qo][gi] = v;
                    p.qb[qo][gi] = rb;
                    p.ql[qo][gi] = len;
                } else {
                    atomicOr(&p.ctrl->status, ST_OVERFLOW);
                }
            }
        }
    }
    if (__any_sync(FULL, big) && big) {
        const int nseg = (len + p.segment - 1) / p.segment;
        unsigned gi = atomicAdd(&p.ctrl->big_count[set_out], (unsigned)nseg);
        for (int s = 0; s < nseg; ++s, ++gi) {
            if (gi < p.bqcap) {
                p.bu[qo][gi] = v;
                p.bb[qo][gi] = rb + s * p.segment;
                p.bl[qo][gi] = min(p.segment, len - s * p.segment);
            } else {
                atomicOr(&p.ctrl->status, ST_OVERFLOW);
            }
        }
    }
}

// Move the CTA buffer to the global small queue when it is half full (or
// always, with force).  Called by the whole CTA.
template <int BLOCK>
__device__ __forceinline__ void flush(bool force, const TdParams &p, int set_out, int qo, const OutBuf &ob)
{
    __syncthreads();
    const int c = min(*ob.cnt, OB);
    if (c > 0 && (force || c >= OB / 2)) {
        if (threadIdx.x == 0) *ob.gbase = (int)atomicAdd(&p.ctrl->count[set_out], (unsigned)c);
        __syncthreads();
        const unsigned gb = (unsigned)*ob.gbase;
        for (int i = threadIdx.x; i < c; i += BLOCK) {
            const unsigned gi = gb + (unsigned)i;
            if (gi < p.qcap) {
                p.qu[qo][gi] = ob.u[i];
                p.qb[qo][gi] = ob.b[i];
                p.ql[qo][gi] = ob.l[i];
            } else {
                atomicOr(&p.ctrl->status, ST_OVERFLOW);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) *ob.cnt = 0;
        __syncthreads();
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) td_kernel(TdParams p)
{
    __shared__ int32_t s_ou[OB], s_ob[OB], s_ol[OB];
    __shared__ int32_t s_off[BLOCK], s_beg[BLOCK], s_u[BLOCK];
    __shared__ int s_warp[33];
    __shared__ int s_ocnt, s_gbase, s_ok;
    __shared__ unsigned s_item, s_chunk, s_f, s_bf;
    __shared__ unsigned long long s_stat[3];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned G = gridDim.x;
    Ctrl *c = p.ctrl;
    const OutBuf ob{s_ou, s_ob, s_ol, &s_ocnt, &s_gbase};
    const uint64_t t_start = globaltimer();

    // ---- initialisation (a1) ------------------------------------------------
    {
        const int64_t stride = (int64_t)G * BLOCK;
        for (int64_t i = (int64_t)blockIdx.x * BLOCK + tid; i < p.n; i += stride) {
            const bool is_root = (i == p.root);
            p.level[i] = is_root ? 0 : -1;
            if (p.parent) p.parent[i] = is_root ? p.root : -1;
        }
        const int rint = __ldg(p.perm + p.root);  // the root in internal numbering
        const int rw = rint >> 5;
        for (int64_t w = (int64_t)blockIdx.x * BLOCK + tid; w < p.bitmap_words; w += stride)
            p.bitmap[w] = (w == rw) ? (1u << (rint & 31)) : 0u;
        if (blockIdx.x == 0) {
            if (p.stats)
                for (int i = tid; i < 4 * kMaxStatLayers; i += BLOCK) p.stats[i] = 0;
            if (tid == 0) {
                const int rb = p.ro[rint], len = p.ro[rint + 1] - rb;
                unsigned cnt = 0, bcnt = 0;
                if (len > 0 && len < p.cta_degree) {
                    p.qu[0][0] = rint;
                    p.qb[0][0] = rb;
                    p.ql[0][0] = len;
                    cnt = 1;
                } else if (len >= p.cta_degree) {
                    const int nseg = (len + p.segment - 1) / p.segment;
                    for (int s = 0; s < nseg && (unsigned)s < p.bqcap; ++s) {
                        p.bu[0][s] = rint;
                        p.bb[0][s] = rb + s * p.segment;
                        p.bl[0][s] = min(p.segment, len - s * p.segment);
                    }
                    bcnt = (unsigned)nseg;
                }
                c->count[0] = cnt;
                c->big_count[0] = bcnt;
            }
        }
    }
    bool ok = grid_sync(c, G, p.timeout_ns, &s_ok);

    // ---- layers ---------------------------------------------------------------
    for (int d = 0; ok; ++d) {
        if (tid == 0) {
            s_f = ld_relaxed(&c->count[d % 3]);
            s_bf = ld_relaxed(&c->big_count[d % 3]);
            s_ocnt = 0;
            if (p.stats) s_stat[0] = s_stat[1] = s_stat[2] = 0;
        }
        __syncthreads();
        const unsigned f = min(s_f, p.qcap), bf = min(s_bf, p.bqcap);
        if (f == 0 && bf == 0) {
            if (blockIdx.x == 0 && tid == 0) c->layers = (unsigned)d;
            break;
        }
        const int set_in = d % 3, set_out = (d + 1) % 3, set_rst = (d + 2) % 3;
        if (blockIdx.x == 0 && tid == 0) {
            c->count[set_rst] = 0;
            c->work[set_rst] = 0;
            c->big_count[set_rst] = 0;
            c->big_work[set_rst] = 0;
        }
        const int qi = d & 1, qo = qi ^ 1;
        const int next_level = d + 1;
        unsigned my_new = 0;
        unsigned long long my_edges = 0, my_vertices = 0;

        // (1) large items: one slice of <= segment edges per CTA at a time
        for (;;) {
            if (tid == 0) s_item = atomicAdd(&c->big_work[set_in], 1u);
            __syncthreads();
            const unsigned it = s_item;
            if (it >= bf) break;
            const int u = __ldcg(p.bu[qi] + it), b = __ldcg(p.bb[qi] + it), l = __ldcg(p.bl[qi] + it);
            for (int k0 = warp * 32; k0 < l; k0 += BLOCK) {
                const int k = k0 + lane;
                const bool valid = k < l;
                const int v = valid ? __ldg(p.col + b + k) : 0;
                visit(valid, v, u, next_level, p, set_out, qo, ob, my_new);
            }
            if (tid == 0) {
                my_edges += (unsigned long long)l;
                my_vertices += (b == __ldg(p.ro + u)) ? 1ull : 0ull;
            }
            flush<BLOCK>(false, p, set_out, qo, ob);
        }

        // (2) small items, BLOCK per chunk
        for (;;) {
            if (tid == 0) s_chunk = atomicAdd(&c->work[set_in], (unsigned)BLOCK);
            __syncthreads();
            const unsigned base = s_chunk;
            if (base >= f) break;
            const unsigned i = base + tid;
            int u = 0, b = 0, l = 0;
            if (i < f) {
                u = __ldcg(p.qu[qi] + i);
                b = __ldcg(p.qb[qi] + i);
                l = __ldcg(p.ql[qi] + i);
                my_edges += (unsigned long long)l;
                my_vertices += 1;
            }
            const bool wbin = l >= p.warp_degree;
            int total;
            const int off = block_exclusive_scan<BLOCK>(wbin ? 0 : l, s_warp, total);
            s_off[tid] = off;
            s_beg[tid] = b;
            s_u[tid] = u;
            __syncthreads();

            // warp bin: each warp expands its own lanes' items one at a time
            unsigned wm = __ballot_sync(FULL, wbin);
            while (wm) {
                const int src = __ffs(wm) - 1;
                wm &= wm - 1;
                const int wu = __shfl_sync(FULL, u, src);
                const int wb = __shfl_sync(FULL, b, src);
                const int wl = __shfl_sync(FULL, l, src);
                for (int k0 = 0; k0 < wl; k0 += 32) {
                    const int k = k0 + lane;
                    const bool valid = k < wl;
                    const int v = valid ? __ldg(p.col + wb + k) : 0;
                    visit(valid, v, wu, next_level, p, set_out, qo, ob, my_new);
                }
            }

            // thread bin: the short lists flattened over the CTA
            for (int e0 = warp * 32; e0 < total; e0 += BLOCK) {
                const int e = e0 + lane;
                const bool valid = e < total;
                int v = 0, su = 0;
                if (valid) {
                    int lo = 0, hi = BLOCK;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s_off[mid] <= e) lo = mid;
                        else hi = mid;
                    }
                    su = s_u[lo];
                    v = __ldg(p.col + s_beg[lo] + (e - s_off[lo]));
                }
                visit(valid, v, su, next_level, p, set_out, qo, ob, my_new);
            }
            flush<BLOCK>(false, p, set_out, qo, ob);
        }
        flush<BLOCK>(true, p, set_out, qo, ob);

        if (p.stats && d < kMaxStatLayers) {
            unsigned long long a = my_vertices, e = my_edges, t = my_new;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(FULL, a, o);
                e += __shfl_down_sync(FULL, e, o);
                t += __shfl_down_sync(FULL, t, o);
            }
            if (lane == 0) {
                atomicAdd(&s_stat[0], a);
                atomicAdd(&s_stat[1], e);
                atomicAdd(&s_stat[2], t);
            }
            __syncthreads();
            if (tid == 0) {
                atomicAdd((unsigned long long *)&p.stats[4 * d + 0], s_stat[0]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 1], s_stat[1]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 2], s_stat[2]);
            }
        }
        ok = grid_sync(c, G, p.timeout_ns, &s_ok);
        if (p.stats && d < kMaxStatLayers && blockIdx.x == 0 && tid == 0)
            p.stats[4 * d + 3] = (int64_t)(globaltimer() - t_start);
    }

    // ---- exit: the last CTA out returns the control block to zero ----------
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned old = atomicAdd(&c->exit_count, 1u);
        if (old == G - 1) {
            for (int j = 0; j < 3; ++j) {
                c->count[j] = 0;
                c->work[j] = 0;
                c->big_count[j] = 0;
                c->big_work[j] = 0;
            }
            c->bar_count = 0;
            c->exit_count = 0;
            __threadfence();
        }
    }
}

template <int BLOCK>
int launch_block(Graph *g, const TdParams &prm, cudaStream_t s)
{
    auto kern = td_kernel<BLOCK>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, 0);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(td_kernel)");
    if (per_sm < 1) return set_error(BFS_ERR_CUDA, "td_kernel: no CTA fits on an SM");
    if (g->opt.ctas_per_sm > 0) per_sm = std::min(per_sm, g->opt.ctas_per_sm);
    int grid = per_sm * g->num_sms;
    if (g->opt.max_ctas > 0) grid = std::min(grid, g->opt.max_ctas);
    TdParams p = prm;
    void *args[] = {&p};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(BLOCK), args, 0, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(td_kernel)");
    g->last_grid = grid;
    return BFS_OK;
}

}  // namespace

int td_launch(Graph *g, int32_t root, int32_t *level, int32_t *parent, cudaStream_t s)
{
    TdParams p;
    p.ro = g->d_row_offsets;
    p.col = g->d_col_idx;
    p.level = level;
    p.parent = parent;
    p.perm = g->d_perm;
    p.orig = g->d_orig;
    p.bitmap = g->d_bitmap;
    for (int b = 0; b < 2; ++b) {
        p.qu[b] = g->d_q[b][0];
        p.qb[b] = g->d_q[b][1];
        p.ql[b] = g->d_q[b][2];
        p.bu[b] = g->d_bq[b][0];
        p.bb[b] = g->d_bq[b][1];
        p.bl[b] = g->d_bq[b][2];
    }
    p.ctrl = g->d_ctrl;
    p.stats = g->opt.layer_stats ? g->d_stats : nullptr;
    p.n = (int32_t)g->n;
    p.root = root;
    p.warp_degree = g->opt.warp_degree;
    p.cta_degree = g->opt.cta_degree;
    p.segment = g->opt.segment;
    p.qcap = (uint32_t)g->qcap;
    p.bqcap = (uint32_t)std::min<int64_t>(g->bqcap, 0xFFFFFFFFLL);
    p.bitmap_words = (int32_t)g->bitmap_words;
    p.timeout_ns = (uint64_t)g->opt.timeout_ns;
    switch (g->opt.block) {
    case 256: return launch_block<256>(g, p, s);
    case 512: return launch_block<512>(g, p, s);
    case 1024: return launch_block<1024>(g, p, s);
    default: return set_error(BFS_ERR_INVALID_ARG, "td_launch: unsupported block size");
    }
}

}  // namespace gbbfs
