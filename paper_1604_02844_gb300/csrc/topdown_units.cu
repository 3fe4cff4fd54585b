// topdown_units.cu -- single-source level-synchronous top-down BFS,
// edge-balanced work units (the default expansion mode).
//
// Same method as topdown.cu (Alg. 2 with an atomic visited bitmap, word
// v>>5 bit v&31 as in Listing 1, P[s] = s, layer L_d finished before
// L_{d+1}, Sec. 3), one persistent cooperative kernel per search, but the
// frontier is organised so that every piece of work a CTA picks up is
// bounded in edges rather than in vertices:
//
//  * A frontier entry is (u, beg, len) with 1 <= len <= T (T = 2*BLOCK).
//    Vertices of degree > T are "hubs": they are cut into slices of T edges
//    at discovery time and each slice is its own work item.
//  * When a CTA flushes its shared-memory buffer of newly reached vertices
//    it writes the entries contiguously and cuts them into units: a new unit
//    starts where the running edge count crosses a multiple of T, or every
//    BLOCK entries.  A unit therefore holds <= BLOCK entries and < 2T edges.
//    The flush reserves entries and units with one 64-bit atomicAdd.
//  * The next layer hands out hub slices, then units, one per atomicAdd.
//
// Per work item: the CTA loads its entries, prefix-sums their lengths and
// copies the item's adjacency into shared memory with cp.async (4-byte,
// no register staging) -- issued for the NEXT item while the current one is
// processed, so the col_idx stream overlaps the bitmap work.  Processing
// is filter-then-claim: pass A reads the visited word of every staged edge
// (all loads of a thread in flight together) and compacts the unvisited
// ones into a candidate list with warp ballots; pass B claims candidates
// with atomicOr, and each winner writes level/parent, reads its row_offsets
// pair and reserves a slot in the CTA's out buffer (warp-aggregated).
//
// All waits are bounded (grid barrier timeout -> ST_TIMEOUT, clean exit).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.cuh"

namespace gbbfs {
namespace {

using namespace dev;

struct UParams {
    const int32_t *__restrict__ ro;
    const int32_t *__restrict__ col;
    int32_t *level;
    int32_t *parent;  // may be null
    const int32_t *__restrict__ perm;  // caller id -> internal id
    const int32_t *__restrict__ orig;  // internal id -> caller id
    uint32_t *bitmap;
    int32_t *eu[2], *eb[2], *el[2];  // entry queue [buffer]: vertex, adjacency begin, length
    int32_t *us[2], *uc[2];          // unit queue [buffer]: first entry, entry count
    int32_t *hu[2], *hb[2], *hl[2];  // hub-slice queue [buffer]
    UnitCtrl *ctrl;
    int64_t *stats;  // [kMaxStatLayers][4] or null
    int32_t n;
    int32_t root;
    uint32_t ecap, ucap, hcap;
    int32_t bitmap_words;
    uint64_t timeout_ns;
};

template <int BLOCK>
struct Cfg {
    static constexpr int T = 2 * BLOCK;     // unit edge target, hub slice length
    static constexpr int MAXE = 2 * T;      // edges of one item are < MAXE
    static constexpr int OB = 2 * MAXE;     // out-buffer entries
    static constexpr int PER = OB / BLOCK;  // out-buffer entries per thread in a flush
    static constexpr int EPT = MAXE / BLOCK;  // staged edges per thread
};

template <int BLOCK>
struct Smem {
    int32_t col[2][Cfg<BLOCK>::MAXE];  // staged adjacency (double buffer)
    int32_t src[2][Cfg<BLOCK>::MAXE];  // source vertex of each staged edge
    int32_t off[BLOCK + 1];            // item entries: prefix of lengths
    int32_t iu[BLOCK];                 // item entries: vertex
    int32_t ib[BLOCK];                 // item entries: adjacency begin
    int32_t ou[Cfg<BLOCK>::OB];        // out buffer: vertex
    int32_t ob[Cfg<BLOCK>::OB];        // out buffer: adjacency begin
    int32_t ol[Cfg<BLOCK>::OB];        // out buffer: length
    int32_t cand[2 * Cfg<BLOCK>::MAXE];  // candidates (v, u) pairs; unit starts in a flush
    int warp[33];
    int ocnt, ccnt, ok, items;
    unsigned nitem;
    int et[2];
    unsigned long long ebase_ubase;
    unsigned long long st[3];
};

template <int BLOCK>
__device__ __forceinline__ int search_entry(const int32_t *off, int cnt, int e)
{
    // largest j in [0, cnt) with off[j] <= e (lengths are >= 1)
    int lo = 0, hi = cnt;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Load the entries of work item `item` and start copying its adjacency into
// staging buffer `buf`.  Whole CTA.  Returns nothing; the edge count goes to
// sm.et[buf].
template <int BLOCK>
__device__ void load_and_stage(Smem<BLOCK> &sm, const UParams &p, int qi, unsigned nH, unsigned item, int buf,
                               unsigned long long &my_vertices)
{
    const int tid = threadIdx.x;
    int cnt;
    if (item < nH) {
        cnt = 1;
        if (tid == 0) {
            const int u = __ldcg(p.hu[qi] + item), b = __ldcg(p.hb[qi] + item), l = __ldcg(p.hl[qi] + item);
            sm.iu[0] = u;
            sm.ib[0] = b;
            sm.off[0] = 0;
            sm.off[1] = l;
            if (p.stats) my_vertices += (b == __ldg(p.ro + u)) ? 1ull : 0ull;
        }
        __syncthreads();
    } else {
        const unsigned k = item - nH;
        const int start = __ldcg(p.us[qi] + k);
        cnt = __ldcg(p.uc[qi] + k);
        if (cnt < 0 || cnt > BLOCK) {  // cannot happen for units cut by flush_units
            if (tid == 0) atomicOr(&p.ctrl->status, ST_OVERFLOW);
            cnt = 0;
        }
        int u = 0, b = 0, l = 0;
        if (tid < cnt) {
            u = __ldcg(p.eu[qi] + start + tid);
            b = __ldcg(p.eb[qi] + start + tid);
            l = __ldcg(p.el[qi] + start + tid);
        }
        int total;
        const int o = block_exclusive_scan<BLOCK>(l, sm.warp, total);
        if (tid < cnt) {
            sm.off[tid] = o;
            sm.iu[tid] = u;
            sm.ib[tid] = b;
        }
        if (tid == 0) {
            sm.off[cnt] = total;
            my_vertices += (unsigned long long)cnt;
        }
        __syncthreads();
    }
    int et = sm.off[cnt];
    if (et >= Cfg<BLOCK>::MAXE) {  // cannot happen: units hold < 2T edges, slices T
        if (tid == 0) atomicOr(&p.ctrl->status, ST_OVERFLOW);
        et = 0;
    }
    for (int e = tid; e < et; e += BLOCK) {
        const int j = search_entry<BLOCK>(sm.off, cnt, e);
        cp_async4(&sm.col[buf][e], p.col + sm.ib[j] + (e - sm.off[j]));
        sm.src[buf][e] = sm.iu[j];
    }
    cp_async_commit();
    if (tid == 0) sm.et[buf] = et;
}

// Write the out buffer to the global entry queue and cut it into units.
template <int BLOCK>
__device__ void flush_units(Smem<BLOCK> &sm, const UParams &p, int set_out, int qo)
{
    constexpr int T = Cfg<BLOCK>::T, PER = Cfg<BLOCK>::PER;
    const int tid = threadIdx.x;
    const int c = sm.ocnt;  // stable: callers synchronise first
    const int i0 = min(tid * PER, c), i1 = min(i0 + PER, c);
    int sum = 0;
    for (int i = i0; i < i1; ++i) sum += sm.ol[i];
    int tot;
    const int toff = block_exclusive_scan<BLOCK>(sum, sm.warp, tot);
    int nu = 0;
    {
        int off = toff;
        for (int i = i0; i < i1; ++i) {
            const bool start = (i == 0) || (i % BLOCK == 0) || (off / T != (off - sm.ol[i - 1]) / T);
            nu += start;
            off += sm.ol[i];
        }
    }
    int tot_units;
    const int uoff = block_exclusive_scan<BLOCK>(nu, sm.warp, tot_units);
    if (tid == 0) {
        const unsigned long long add = ((unsigned long long)tot_units << 32) | (unsigned long long)c;
        sm.ebase_ubase = atomicAdd(&p.ctrl->eu_count[set_out], add);
    }
    {
        int k = uoff, off = toff;
        int32_t *ustart = sm.cand;  // candidates are consumed: reuse
        for (int i = i0; i < i1; ++i) {
            const bool start = (i == 0) || (i % BLOCK == 0) || (off / T != (off - sm.ol[i - 1]) / T);
            if (start) ustart[k++] = i;
            off += sm.ol[i];
        }
    }
    __syncthreads();
    const unsigned ebase = (unsigned)(sm.ebase_ubase & 0xffffffffull);
    const unsigned ubase = (unsigned)(sm.ebase_ubase >> 32);
    for (int i = tid; i < c; i += BLOCK) {
        const unsigned gi = ebase + (unsigned)i;
        if (gi < p.ecap) {
            p.eu[qo][gi] = sm.ou[i];
            p.eb[qo][gi] = sm.ob[i];
            p.el[qo][gi] = sm.ol[i];
        } else {
            atomicOr(&p.ctrl->status, ST_OVERFLOW);
        }
    }
    for (int k = tid; k < tot_units; k += BLOCK) {
        const int s = sm.cand[k];
        const int e = (k + 1 < tot_units) ? sm.cand[k + 1] : c;
        const unsigned gk = ubase + (unsigned)k;
        if (gk < p.ucap) {
            p.us[qo][gk] = (int32_t)(ebase + (unsigned)s);
            p.uc[qo][gk] = e - s;
        } else {
            atomicOr(&p.ctrl->status, ST_OVERFLOW);
        }
    }
    __syncthreads();
    if (tid == 0) sm.ocnt = 0;
    __syncthreads();
}

// Pass A + pass B over one staged item.
template <int BLOCK>
__device__ void process_item(Smem<BLOCK> &sm, const UParams &p, int buf, int et, int next_level, int set_out,
                             int qo, unsigned &my_new)
{
    constexpr int T = Cfg<BLOCK>::T, EPT = Cfg<BLOCK>::EPT;
    const int tid = threadIdx.x;
    // pass A: filter on the visited bitmap
    {
        int v[EPT];
        unsigned cur[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = k * BLOCK + tid;
            v[k] = e < et ? sm.col[buf][e] : 0;
            cur[k] = e < et ? __ldcg(p.bitmap + ((unsigned)v[k] >> 5)) : 0xffffffffu;
        }
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            if (k * BLOCK >= et) break;  // CTA-uniform
            const int e = k * BLOCK + tid;
            const bool cand = !(cur[k] & (1u << (v[k] & 31)));
            const int slot = warp_reserve(&sm.ccnt, cand ? 1 : 0);
            if (cand) {
                sm.cand[2 * slot] = v[k];
                sm.cand[2 * slot + 1] = sm.src[buf][e];
            }
        }
    }
    __syncthreads();
    const int nc = sm.ccnt;
    // pass B: claim, write level/parent, queue the winners
    for (int c0 = 0; c0 < nc; c0 += 2 * BLOCK) {
        int v[2], u[2], rb[2], len[2];
        bool win[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = c0 + k * BLOCK + tid;
            const bool ok = i < nc;
            v[k] = ok ? sm.cand[2 * i] : 0;
            u[k] = ok ? sm.cand[2 * i + 1] : 0;
            const unsigned bit = 1u << (v[k] & 31);
            win[k] = ok && !(atomicOr(p.bitmap + ((unsigned)v[k] >> 5), bit) & bit);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            rb[k] = 0;
            len[k] = 0;
            if (win[k]) {
                const int ov = __ldg(p.orig + v[k]);  // results leave in the caller's numbering
                p.level[ov] = next_level;
                if (p.parent) p.parent[ov] = __ldg(p.orig + u[k]);
                rb[k] = __ldg(p.ro + v[k]);
                len[k] = __ldg(p.ro + v[k] + 1) - rb[k];
                ++my_new;
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const bool small = win[k] && len[k] >= 1 && len[k] <= T;
            const int slot = warp_reserve(&sm.ocnt, small ? 1 : 0);
            if (small) {
                sm.ou[slot] = v[k];
                sm.ob[slot] = rb[k];
                sm.ol[slot] = len[k];
            }
            if (win[k] && len[k] > T) {  // hub: slices of T edges, straight to the global queue
                const int nseg = (len[k] + T - 1) / T;
                unsigned gi = atomicAdd(&p.ctrl->hub_count[set_out], (unsigned)nseg);
                for (int s = 0; s < nseg; ++s, ++gi) {
                    if (gi < p.hcap) {
                        p.hu[qo][gi] = v[k];
                        p.hb[qo][gi] = rb[k] + s * T;
                        p.hl[qo][gi] = min(T, len[k] - s * T);
                    } else {
                        atomicOr(&p.ctrl->status, ST_OVERFLOW);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) sm.ccnt = 0;
    // (the caller synchronises before the next use of ccnt / ocnt)
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) td_units_kernel(UParams p)
{
    constexpr int T = Cfg<BLOCK>::T, MAXE = Cfg<BLOCK>::MAXE, OB = Cfg<BLOCK>::OB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<BLOCK> &sm = *reinterpret_cast<Smem<BLOCK> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned G = gridDim.x;
    UnitCtrl *c = p.ctrl;
    const uint64_t t_start = globaltimer();

    // ---- initialisation (Alg. 1: P = infinity except P[s] = s; vis = {s}) --
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
                if (len >= 1 && len <= T) {
                    p.eu[0][0] = rint;
                    p.eb[0][0] = rb;
                    p.el[0][0] = len;
                    p.us[0][0] = 0;
                    p.uc[0][0] = 1;
                    c->eu_count[0] = (1ull << 32) | 1ull;
                    c->hub_count[0] = 0;
                } else if (len > T) {
                    const int nseg = (len + T - 1) / T;
                    for (int s = 0; s < nseg && (unsigned)s < p.hcap; ++s) {
                        p.hu[0][s] = rint;
                        p.hb[0][s] = rb + s * T;
                        p.hl[0][s] = min(T, len - s * T);
                    }
                    c->eu_count[0] = 0;
                    c->hub_count[0] = (unsigned)nseg;
                } else {
                    c->eu_count[0] = 0;
                    c->hub_count[0] = 0;
                }
            }
        }
        if (tid == 0) {
            sm.ocnt = 0;
            sm.ccnt = 0;
        }
    }
    bool ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &sm.ok);

    for (int d = 0; ok; ++d) {
        const int set_in = d % 3, set_out = (d + 1) % 3, set_rst = (d + 2) % 3;
        if (tid == 0) {
            const unsigned long long eu = ld_relaxed64(&c->eu_count[set_in]);
            const unsigned nU = min((unsigned)(eu >> 32), p.ucap);
            const unsigned nH = min(ld_relaxed(&c->hub_count[set_in]), p.hcap);
            sm.items = (int)(nU + nH);
            sm.nitem = nH;  // temporarily: hub count
            if (p.stats) sm.st[0] = sm.st[1] = sm.st[2] = 0;
        }
        __syncthreads();
        const unsigned n_items = (unsigned)sm.items, nH = sm.nitem;
        if (n_items == 0) {
            if (blockIdx.x == 0 && tid == 0) c->layers = (unsigned)d;
            break;
        }
        if (blockIdx.x == 0 && tid == 0) {
            c->eu_count[set_rst] = 0;
            c->hub_count[set_rst] = 0;
            c->work[set_rst] = 0;
        }
        const int qi = d & 1, qo = qi ^ 1;
        const int next_level = d + 1;
        unsigned my_new = 0;
        unsigned long long my_vertices = 0, my_edges = 0;

        __syncthreads();
        if (tid == 0) sm.nitem = atomicAdd(&c->work[set_in], 1u);
        __syncthreads();
        unsigned item = sm.nitem;
        int buf = 0;
        if (item < n_items) load_and_stage<BLOCK>(sm, p, qi, nH, item, buf, my_vertices);
        while (item < n_items) {
            __syncthreads();
            if (tid == 0) sm.nitem = atomicAdd(&c->work[set_in], 1u);
            cp_async_wait_all();
            __syncthreads();
            const unsigned next = sm.nitem;
            const int et = sm.et[buf];
            if (tid == 0) my_edges += (unsigned long long)et;
            if (next < n_items) load_and_stage<BLOCK>(sm, p, qi, nH, next, buf ^ 1, my_vertices);
            process_item<BLOCK>(sm, p, buf, et, next_level, set_out, qo, my_new);
            __syncthreads();
            if (sm.ocnt > OB - MAXE) flush_units<BLOCK>(sm, p, set_out, qo);
            buf ^= 1;
            item = next;
        }
        cp_async_wait_all();
        __syncthreads();
        if (sm.ocnt > 0) flush_units<BLOCK>(sm, p, set_out, qo);

        if (p.stats && d < kMaxStatLayers) {
            unsigned long long a = my_vertices, e = my_edges, t = my_new;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(FULL, a, o);
                e += __shfl_down_sync(FULL, e, o);
                t += __shfl_down_sync(FULL, t, o);
            }
            if (lane == 0) {
                atomicAdd(&sm.st[0], a);
                atomicAdd(&sm.st[1], e);
                atomicAdd(&sm.st[2], t);
            }
            __syncthreads();
            if (tid == 0) {
                atomicAdd((unsigned long long *)&p.stats[4 * d + 0], sm.st[0]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 1], sm.st[1]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 2], sm.st[2]);
            }
        }
        ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &sm.ok);
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
                c->eu_count[j] = 0;
                c->hub_count[j] = 0;
                c->work[j] = 0;
            }
            c->bar_count = 0;
            c->exit_count = 0;
            __threadfence();
        }
    }
}

template <int BLOCK>
int launch(Graph *g, const UParams &prm, cudaStream_t s)
{
    auto kern = td_units_kernel<BLOCK>;
    const int smem = (int)sizeof(Smem<BLOCK>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(td_units_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(td_units_kernel)");
    if (per_sm < 1) return set_error(BFS_ERR_CUDA, "td_units_kernel: no CTA fits on an SM");
    if (g->opt.ctas_per_sm > 0) per_sm = std::min(per_sm, g->opt.ctas_per_sm);
    int grid = per_sm * g->num_sms;
    if (g->opt.max_ctas > 0) grid = std::min(grid, g->opt.max_ctas);
    UParams p = prm;
    void *args[] = {&p};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(BLOCK), args, (size_t)smem, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(td_units_kernel)");
    g->last_grid = grid;
    return BFS_OK;
}

}  // namespace

int td_units_launch(Graph *g, int32_t root, int32_t *level, int32_t *parent, cudaStream_t s)
{
    UParams p;
    p.ro = g->d_row_offsets;
    p.col = g->d_col_idx;
    p.level = level;
    p.parent = parent;
    p.perm = g->d_perm;
    p.orig = g->d_orig;
    p.bitmap = g->d_bitmap;
    for (int b = 0; b < 2; ++b) {
        p.eu[b] = g->d_eq[b][0];
        p.eb[b] = g->d_eq[b][1];
        p.el[b] = g->d_eq[b][2];
        p.us[b] = g->d_uq[b][0];
        p.uc[b] = g->d_uq[b][1];
        p.hu[b] = g->d_hq[b][0];
        p.hb[b] = g->d_hq[b][1];
        p.hl[b] = g->d_hq[b][2];
    }
    p.ctrl = g->d_ctrl;
    p.stats = g->opt.layer_stats ? g->d_stats : nullptr;
    p.n = (int32_t)g->n;
    p.root = root;
    p.ecap = (uint32_t)g->n;
    p.ucap = (uint32_t)g->n;
    p.hcap = (uint32_t)std::min<int64_t>(g->hcap, 0x7FFFFFFFLL);
    p.bitmap_words = (int32_t)g->bitmap_words;
    p.timeout_ns = (uint64_t)g->opt.timeout_ns;
    switch (g->opt.block) {
    case 256: return launch<256>(g, p, s);
    case 512: return launch<512>(g, p, s);
    default: return set_error(BFS_ERR_INVALID_ARG, "units mode supports BLOCK 256 or 512");
    }
}

// Hub slices of one layer: a vertex of degree d > T gives ceil(d/T) <= 2d/T
// slices, so a layer has at most 2m/T of them.  The smallest slice length
// in use is 256 (the warp mode), hence m/128 (+2).
int64_t td_units_hub_capacity(int64_t m) { return m / 128 + 2; }

}  // namespace gbbfs
