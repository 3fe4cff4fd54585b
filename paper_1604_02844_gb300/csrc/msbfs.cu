// msbfs.cu -- bit-parallel multi-source BFS (bfs_run_batch) and the lane
// machinery the serving loop builds on.
//
// Not in the paper; it applies the paper's layer step (Alg. 2: expand the
// frontier, test and set the visited state, queue new vertices) to up to 64
// searches at once, one bit per search ("lane") in 64-bit words per vertex:
//   seen[v]      lanes that have reached v
//   front[p][v]  lanes whose frontier holds v in iteration parity p
//   next[v]      lanes that reach v in the current iteration
// One iteration (all lanes advance one layer):
//   EXPAND: for every frontier entry (u, beg, len) and every v in its slice
//           of Adj[u]: nb = front[u] & ~(seen[v] | next[v]); if nb,
//           atomicOr(next[v], nb) (64-bit); the warp whose atomicOr found
//           next[v] == 0 queues v in the touched list.  Warps take frontier
//           entries 4 at a time (the first 4 statically, the rest from an
//           atomic dispenser) and flatten their edges across the lanes.
//   UPDATE: for every touched v: nn = next[v] & ~seen[v]; next[v] = 0;
//           seen[v] |= nn; front[v] = nn; lane i of nn gets level
//           iter + 1 - start[i]; v is queued for the next EXPAND (vertices of
//           degree > H as slices of H edges).  The old frontier words are
//           cleared.
// Lanes may join at different iterations (start[i] = the iteration they were
// injected), which is what the serving loop uses: a lane whose frontier has
// emptied is finished, its level column is read out and the lane reused.
//
// Levels are kept vertex-major, lvl[v][64] uint8 in the caller's numbering
// (one 64-byte line per vertex), 0xFF = unreached, and transposed into the
// caller's source-major [k][n] output when lanes finish.
//
// Heavy iterations run as pull steps on symmetric graphs (checked exactly at
// graph creation): every vertex v with a lane still missing ORs the
// frontier words of its neighbours (in-neighbours = out-neighbours), with an
// early exit once every missing live lane is found; no atomics, no touched
// list.  An iteration is a pull step when the frontier's adjacency exceeds
// m/16 entries, every live lane is at least two iterations old, and at least
// 30% of the live lanes' (vertex, lane) pairs over vertices of degree >= 1
// are already reached -- otherwise most vertices miss lanes whose frontier is
// still far away and would scan their whole adjacency without an early exit
// (the multi-lane form of the direction-optimising switch).
//
// All iterations of a launch run in one persistent cooperative kernel
// (CTAs of 8 or 16 warps, BFS_OPT_BATCH_BLOCK) with two bounded grid
// barriers per iteration.  bfs_run_batch captures its whole launch sequence
// (inject, run, extract per batch) in a CUDA graph and replays it for later
// calls of the same shape.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.cuh"
#include "msbfs.cuh"

namespace gbbfs {
namespace {

using namespace dev;

constexpr int H = 256;   // hub slice length
constexpr int UX = 4;    // 32-edge batches per warp in flight
constexpr int GRAB = 4;  // frontier entries a warp takes from the dispenser at a time: few, so
                         // that runs of hub slices (up to GRAB * H edges) do not leave one warp
                         // working while the grid waits at the barrier

struct MsParams {
    const int32_t *__restrict__ ro;
    const int32_t *__restrict__ col;
    const int32_t *__restrict__ orig;
    unsigned long long *seen, *next, *front[2];
    uint8_t *lvl;
    int32_t *fu[2], *fb[2], *fl[2];
    int32_t *touched;
    const int32_t *start;  // [64] start iteration per lane
    MsCtrl *ctrl;
    int32_t n;
    int32_t split32;    // internal ids below have degree >= 32
    int symmetric;
    int64_t m;
    int64_t n_nonzero;
    uint32_t fcap;
    uint32_t max_iters;
    uint64_t timeout_ns;
};

// Write the slices of one vertex per lane at positions pos.. of frontier
// buffer q: `few` slices by the lane itself, or `many` slices by the whole
// warp together (one vertex after another), so that a hub's hundreds of
// slices do not hold one lane while the rest of the warp waits.
__device__ __forceinline__ void write_slices(const MsParams &p, int q, int few, int many, int u, int rb, int len,
                                             unsigned pos)
{
    const int lane = threadIdx.x & 31;
    for (int s = 0; s < few; ++s) {
        const unsigned at = pos + (unsigned)s;
        if (at < p.fcap) {
            p.fu[q][at] = u;
            p.fb[q][at] = rb + s * H;
            p.fl[q][at] = min(H, len - s * H);
        } else {
            atomicOr(&p.ctrl->status, ST_OVERFLOW);
        }
    }
    unsigned m = __ballot_sync(FULL, many > 0);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int hu = __shfl_sync(FULL, u, src), hb = __shfl_sync(FULL, rb, src);
        const int hl = __shfl_sync(FULL, len, src), hn = __shfl_sync(FULL, many, src);
        const unsigned hp = __shfl_sync(FULL, pos, src);
        for (int s = lane; s < hn; s += 32) {
            const unsigned at = hp + (unsigned)s;
            if (at < p.fcap) {
                p.fu[q][at] = hu;
                p.fb[q][at] = hb + s * H;
                p.fl[q][at] = min(H, hl - s * H);
            } else {
                atomicOr(&p.ctrl->status, ST_OVERFLOW);
            }
        }
    }
}

// Append the slices of vertex u (degree >= 1) to frontier buffer q.  Called
// by all lanes of a warp; `want` marks the lanes with a vertex to append.
__device__ __forceinline__ void append_frontier(const MsParams &p, int q, bool want, int u, int rb, int len)
{
    const int lane = threadIdx.x & 31;
    const int ns = want ? (len + H - 1) / H : 0;
    int inc = ns;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const int total = __shfl_sync(FULL, inc, 31);
    if (total == 0) return;
    unsigned long long edges = want ? (unsigned long long)len : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) edges += __shfl_xor_sync(FULL, edges, o);
    unsigned base = 0;
    if (lane == 31) {
        base = atomicAdd(&p.ctrl->fcount[q], (unsigned)total);
        atomicAdd(&p.ctrl->fedges[q], edges);
    }
    base = __shfl_sync(FULL, base, 31);
    const unsigned pos0 = base + (unsigned)(inc - ns);
    write_slices(p, q, ns <= 8 ? ns : 0, ns > 8 ? ns : 0, u, rb, len, pos0);
}

constexpr int TB = 128;  // touched-vertex buffer per warp (shared memory)

// Move a warp's buffered touched vertices to the global list: one atomicAdd.
__device__ __forceinline__ void flush_touched(const MsParams &p, int par, int32_t *tbuf, int cnt)
{
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&p.ctrl->tcount[par], (unsigned)cnt);
    base = __shfl_sync(FULL, base, 0);
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
        const unsigned at = base + (unsigned)i;
        if (at < (unsigned)p.n) p.touched[at] = tbuf[i];
        else atomicOr(&p.ctrl->status, ST_OVERFLOW);
    }
    __syncwarp();
}

__device__ __forceinline__ void ms_expand(const MsParams &p, int par, unsigned nF, int32_t *tbuf)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    MsCtrl *c = p.ctrl;
    int tcnt = 0;  // warp-uniform fill of tbuf
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned GWn = (gridDim.x * blockDim.x) >> 5;
    // the first GRAB entries of every warp are its own; the rest come from the dispenser
    for (bool first = true;; first = false) {
        unsigned base = 0;
        if (first) base = gw * GRAB;
        else {
            if (lane == 0) base = GWn * GRAB + atomicAdd(&c->work[par], (unsigned)GRAB);
            base = __shfl_sync(FULL, base, 0);
        }
        if (base >= nF) break;
        const unsigned j = base + lane;
        const bool real = j < nF && lane < GRAB;
        int u = 0, b = 0, l = 0;
        unsigned long long f = 0;
        if (real) {
            u = __ldcg(p.fu[par] + j);
            b = __ldcg(p.fb[par] + j);
            l = __ldcg(p.fl[par] + j);
            f = __ldcg(p.front[par] + GB_IX(u, p.n, BS_FRONTIER, p.ctrl));
            if (l < 0 || l > H) l = 0;  // cannot happen: slices hold <= H edges
        }
        int inc = l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int E = __shfl_sync(FULL, inc, 31);
        const int off = inc - l;
        for (int e0 = 0; e0 < E; e0 += 32 * UX) {
            int v[UX];
            unsigned long long nb[UX];
#pragma unroll
            for (int x = 0; x < UX; ++x) {
                const int bb = e0 + x * 32;
                unsigned starts = (real && off > bb && off < bb + 32) ? (1u << (off - bb)) : 0u;
                starts = __reduce_or_sync(FULL, starts);
                const int j0 = __popc(__ballot_sync(FULL, real && off <= bb)) - 1;
                const int jj = (j0 + __popc(starts & ((2u << lane) - 1u))) & 31;
                const int jb = __shfl_sync(FULL, b, jj);
                const int jo = __shfl_sync(FULL, off, jj);
                const unsigned long long jf = __shfl_sync(FULL, f, jj);
                const int e = bb + lane;
                v[x] = (e < E) ? (int)GB_IX(__ldg(p.col + GB_IX(jb + (e - jo), p.m, BS_COL, p.ctrl)), p.n, BS_FRONTIER,
                                            p.ctrl)
                               : -1;
                nb[x] = jf;
            }
            // lanes that neither reached v before nor already reach it now:
            // most edges into hubs stop here, without an atomic
#pragma unroll
            for (int x = 0; x < UX; ++x)
                if (v[x] >= 0) nb[x] &= ~(__ldcg(p.seen + v[x]) | __ldcg(p.next + v[x]));
#pragma unroll
            for (int x = 0; x < UX; ++x) {
                bool first = false;
                if (v[x] >= 0 && nb[x]) first = (atomicOr(p.next + v[x], nb[x]) == 0ull);
                const unsigned m = __ballot_sync(FULL, first);
                if (m) {
                    if (tcnt + __popc(m) > TB) {
                        flush_touched(p, par, tbuf, tcnt);
                        tcnt = 0;
                    }
                    if (first) tbuf[tcnt + __popc(m & lt)] = v[x];
                    tcnt += __popc(m);
                }
            }
        }
    }
    __syncwarp();
    if (tcnt) flush_touched(p, par, tbuf, tcnt);
}

// Write level bytes of the lanes in nn into a vertex's 64-byte level line:
// byte i becomes lv[i] where bit i of nn is set.  Branch-free per 16-byte
// chunk (bit masks widened to byte masks), so a vertex reached by many lanes
// at once costs the same as one reached by a single lane.
__device__ __forceinline__ void merge_levels(uint4 *row, unsigned long long nn, const uint32_t *lv)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned m16 = (unsigned)(nn >> (16 * q)) & 0xFFFFu;
        if (!m16) continue;
        uint4 x = row[q];
        uint32_t *xw = reinterpret_cast<uint32_t *>(&x);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const unsigned m4 = (m16 >> (4 * w)) & 0xFu;
            const uint32_t bm = ((m4 & 1u) ? 0x000000FFu : 0u) | ((m4 & 2u) ? 0x0000FF00u : 0u) |
                                ((m4 & 4u) ? 0x00FF0000u : 0u) | ((m4 & 8u) ? 0xFF000000u : 0u);
            xw[w] = (xw[w] & ~bm) | (lv[4 * q + w] & bm);
        }
        row[q] = x;
    }
}

constexpr int UU = 4;  // touched vertices per lane per round

__device__ __forceinline__ void ms_update(const MsParams &p, int par, unsigned nF, unsigned iter, unsigned long long &alive,
                                          const uint32_t *s_lv, unsigned long long over)
{
    const int lane = threadIdx.x & 31;
    const int q = par ^ 1;
    MsCtrl *c = p.ctrl;
    const unsigned nT = min(ld_relaxed(&c->tcount[par]), (unsigned)p.n);
    const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned gsz = gridDim.x * blockDim.x;
    // the old frontier words
    for (unsigned i = gtid; i < nF; i += gsz) p.front[par][__ldcg(p.fu[par] + i)] = 0ull;
    // the touched vertices, UU per lane per round (warp-uniform loop)
    for (unsigned i0 = (gtid - lane) * UU; i0 < nT; i0 += gsz * UU) {
        int v[UU], rb[UU], len[UU];
        unsigned long long x[UU], sn[UU], nn[UU];
#pragma unroll
        for (int k = 0; k < UU; ++k) {
            const unsigned i = i0 + k * 32 + lane;
            v[k] = (i < nT) ? (int)GB_IX(__ldcg(p.touched + i), p.n, BS_FRONTIER, p.ctrl) : -1;
        }
#pragma unroll
        for (int k = 0; k < UU; ++k) {
            x[k] = v[k] >= 0 ? __ldcg(p.next + v[k]) : 0ull;
            sn[k] = v[k] >= 0 ? __ldcg(p.seen + v[k]) : 0ull;
        }
        int ns = 0;
#pragma unroll
        for (int k = 0; k < UU; ++k) {
            nn[k] = x[k] & ~sn[k];
            rb[k] = 0;
            len[k] = 0;
            if (v[k] >= 0) {
                p.next[v[k]] = 0ull;
                if (nn[k]) {
                    p.seen[v[k]] = sn[k] | nn[k];
                    p.front[q][v[k]] = nn[k];
                    alive |= nn[k];
                    if (nn[k] & over) atomicOr(&c->status, ST_DEPTH);
                    const int64_t ov = GB_IX(__ldg(p.orig + v[k]), p.n, BS_LANE_ROW, p.ctrl);
                    merge_levels(reinterpret_cast<uint4 *>(p.lvl + (size_t)ov * 64), nn[k], s_lv);
                    rb[k] = __ldg(p.ro + v[k]);
                    len[k] = __ldg(p.ro + v[k] + 1) - rb[k];
                    ns += (len[k] + H - 1) / H;
                }
            }
        }
        {
            unsigned long long pairs = 0;
#pragma unroll
            for (int k = 0; k < UU; ++k) pairs += (unsigned long long)__popcll(nn[k]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(FULL, pairs, o);
            if (lane == 0 && pairs) atomicAdd(&c->seen_pairs, pairs);
        }
        // one reservation for the whole warp's slices of this round
        int inc = ns;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        if (total == 0) continue;
        unsigned long long edges = 0;
#pragma unroll
        for (int k = 0; k < UU; ++k) edges += (nn[k] && len[k] > 0) ? (unsigned long long)len[k] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) edges += __shfl_xor_sync(FULL, edges, o);
        unsigned base = 0;
        if (lane == 31) {
            base = atomicAdd(&c->fcount[q], (unsigned)total);
            atomicAdd(&c->fedges[q], edges);
        }
        base = __shfl_sync(FULL, base, 31);
        unsigned pos = base + (unsigned)(inc - ns);
#pragma unroll
        for (int k = 0; k < UU; ++k) {  // warp-uniform calls: every lane takes part
            const int nk = (nn[k] && len[k] > 0) ? (len[k] + H - 1) / H : 0;
            write_slices(p, q, nk <= 8 ? nk : 0, nk > 8 ? nk : 0, v[k], rb[k], len[k], pos);
            pos += (unsigned)nk;
        }
    }
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x)
{
    const unsigned lo = __reduce_or_sync(FULL, (unsigned)(x & 0xffffffffull));
    const unsigned hi = __reduce_or_sync(FULL, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Pull step: vertices of degree >= 32 one per warp, the rest one per lane.
// A vertex v is new for lanes (OR of front[par][u] over neighbours u) &
// ~seen[v]; the scan of Adj[v] stops once every live lane missing at v is
// found.  Writes seen, front[q], levels and the next frontier list.
__device__ __forceinline__ void ms_pull(const MsParams &p, int par, unsigned long long live, unsigned long long &alive,
                                        const uint32_t *s_lv, unsigned long long over)
{
    const int lane = threadIdx.x & 31;
    const int q = par ^ 1;
    MsCtrl *c = p.ctrl;
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned GW = (gridDim.x * blockDim.x) >> 5;
    // high degree: a warp per vertex
    for (int v = (int)gw; v < p.split32; v += (int)GW) {
        const unsigned long long need = live & ~__ldcg(p.seen + v);
        if (!need) continue;
        const int b = __ldg(p.ro + v), e = __ldg(p.ro + v + 1);
        unsigned long long acc = 0;
        for (int k0 = b; k0 < e; k0 += 32) {
            const int k = k0 + lane;
            if (k < e) acc |= __ldcg(p.front[par] + GB_IX(__ldg(p.col + GB_IX(k, p.m, BS_COL, p.ctrl)), p.n, BS_FRONTIER, p.ctrl));
            if ((warp_or64(acc) & need) == need) break;
        }
        const unsigned long long nn = warp_or64(acc) & need;
        if (nn && lane == 0) {
            atomicAdd(&c->seen_pairs, (unsigned long long)__popcll(nn));
            p.seen[v] = __ldcg(p.seen + v) | nn;
            p.front[q][v] = nn;
            alive |= nn;
            if (nn & over) atomicOr(&c->status, ST_DEPTH);
            merge_levels(reinterpret_cast<uint4 *>(p.lvl + (size_t)GB_IX(__ldg(p.orig + v), p.n, BS_LANE_ROW, p.ctrl) * 64), nn, s_lv);
        }
        append_frontier(p, q, nn != 0ull && lane == 0, v, b, e - b);
    }
    // low degree: a lane per vertex (warp-uniform loop)
    for (int v0 = p.split32 + (int)gw * 32; v0 < p.n; v0 += (int)GW * 32) {
        const int v = v0 + lane;
        unsigned long long nn = 0;
        int b = 0, e = 0;
        if (v < p.n) {
            const unsigned long long sn = __ldcg(p.seen + v);
            const unsigned long long need = live & ~sn;
            if (need) {
                b = __ldg(p.ro + v);
                e = __ldg(p.ro + v + 1);
                unsigned long long acc = 0;
                for (int k = b; k < e; ++k) {
                    acc |= __ldcg(p.front[par] + GB_IX(__ldg(p.col + GB_IX(k, p.m, BS_COL, p.ctrl)), p.n, BS_FRONTIER, p.ctrl));
                    if ((acc & need) == need) break;
                }
                nn = acc & need;
                if (nn) {
                    p.seen[v] = sn | nn;
                    p.front[q][v] = nn;
                    alive |= nn;
                    if (nn & over) atomicOr(&c->status, ST_DEPTH);
                    merge_levels(reinterpret_cast<uint4 *>(p.lvl + (size_t)GB_IX(__ldg(p.orig + v), p.n, BS_LANE_ROW, p.ctrl) * 64), nn, s_lv);
                }
            }
        }
        unsigned long long pairs = (unsigned long long)__popcll(nn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(FULL, pairs, o);
        if (lane == 0 && pairs) atomicAdd(&c->seen_pairs, pairs);
        append_frontier(p, q, nn != 0ull && e > b, v, b, e - b);
    }
}

template <int MS_WPB>
__global__ void __launch_bounds__(MS_WPB * 32) ms_kernel(MsParams p)
{
    __shared__ int s_ok;
    __shared__ unsigned s_nF, s_iter0;
    __shared__ unsigned long long s_alive;
    __shared__ uint32_t s_lv[16];
    __shared__ int s_minage;
    __shared__ int32_t s_tbuf[MS_WPB][TB];
    __shared__ unsigned long long s_over;  // lanes whose level this iteration would exceed 254
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned G = gridDim.x;
    MsCtrl *c = p.ctrl;
    if (tid == 0) s_iter0 = ld_relaxed(&c->iter);  // only the last CTA out writes it
    __syncthreads();
    const unsigned iter0 = s_iter0;
    unsigned done = 0;
    bool ok = true;
    for (unsigned it = 0; it < p.max_iters && ok; ++it) {
        const unsigned iter = iter0 + it;
        const int par = (int)(iter & 1);
        if (tid == 0) {
            s_nF = min(ld_relaxed(&c->fcount[par]), p.fcap);
            s_alive = 0ull;
        }
        __syncthreads();
        const unsigned nF = s_nF;
        if (nF == 0) {
            // no frontier entry left: lanes whose last vertices have no
            // out-edges may still carry an alive bit, but none of them can
            // progress, so every lane is finished
            if (blockIdx.x == 0 && tid == 0) c->alive[par] = 0ull;
            break;
        }
        if (blockIdx.x == 0 && tid == 0) {
            // parity par^1: last read before the previous barrier, next used
            // after the coming one
            c->fcount[par ^ 1] = 0;
            c->fedges[par ^ 1] = 0ull;
            c->work[par ^ 1] = 0;
            c->tcount[par ^ 1] = 0;
            c->alive[par ^ 1] = 0ull;
        }
        const unsigned long long live = ld_relaxed64(&c->alive[par]);
        // youngest live lane: a lane injected less than two iterations ago has
        // explored almost nothing, and a pull step would scan every adjacency
        // list for it without an early exit
        if (tid == 0) s_minage = 0x7fffffff;
        __syncthreads();
        if (tid < 64 && ((live >> tid) & 1ull)) atomicMin(&s_minage, (int)iter - __ldg(p.start + tid));
        __syncthreads();
        const bool pull = p.symmetric && s_minage >= 2 && (long long)ld_relaxed64(&c->fedges[par]) * 16 > p.m &&
                          (double)ld_relaxed64(&c->seen_pairs) >= 0.3 * (double)__popcll(live) * (double)p.n_nonzero;
        if (!pull) ms_expand(p, par, nF, s_tbuf[threadIdx.x >> 5]);
        // On both paths: block 0's reset of the parity par^1 counters above
        // happens before any CTA appends to them (ms_update after a push
        // expansion, ms_pull directly).  Without this barrier a pull step of a
        // CTA running ahead of block 0 could have its frontier appends wiped,
        // leaving lanes alive with an empty frontier.
        ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &s_ok);
        if (!ok) break;
        // this iteration's level byte per lane, packed four to a word
        if (tid < 16) {
            uint32_t w = 0;
            for (int k = 0; k < 4; ++k) {
                const int lvv = (int)iter + 1 - __ldg(p.start + 4 * tid + k);
                w |= (uint32_t)(min(max(lvv, 0), 254)) << (8 * k);
            }
            s_lv[tid] = w;
        }
        if (tid == 0) s_over = 0ull;
        __syncthreads();
        if (tid < 64 && (int)iter + 1 - __ldg(p.start + tid) > 254) atomicOr(&s_over, 1ull << tid);
        __syncthreads();
        unsigned long long alive = 0;
        if (pull) {
            ms_pull(p, par, ld_relaxed64(&c->alive[par]), alive, s_lv, s_over);
            ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &s_ok);
            if (!ok) break;
            // the old frontier words, once every pull has read them
            for (unsigned i = blockIdx.x * blockDim.x + tid; i < nF; i += G * blockDim.x)
                p.front[par][__ldcg(p.fu[par] + i)] = 0ull;
            if (blockIdx.x == 0 && tid == 0) c->pulls += 1;
        } else {
            ms_update(p, par, nF, iter, alive, s_lv, s_over);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) alive |= __shfl_xor_sync(FULL, alive, o);
        if (lane == 0 && alive) atomicOr(&s_alive, alive);
        __syncthreads();
        if (tid == 0 && s_alive) atomicOr(&c->alive[par ^ 1], s_alive);
        ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &s_ok);
        if (ok) done = it + 1;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned old = atomicAdd(&c->exit_count, 1u);
        if (old == G - 1) {
            c->iter = iter0 + done;
            c->bar_count = 0;
            c->exit_count = 0;
            __threadfence();
        }
    }
}

// Lanes in `mask`: set seen/front bits for their sources, level 0, start
// iteration, and queue the sources.  One warp per lane.
__global__ void ms_inject_kernel(MsParams p, const int32_t *__restrict__ lanes_src, unsigned long long mask,
                                 int32_t *start)
{
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= 64 || !((mask >> w) & 1ull)) return;
    MsCtrl *c = p.ctrl;
    const unsigned iter = c->iter;
    const int par = (int)(iter & 1);
    const int s = lanes_src[w];  // internal id
    const unsigned long long bit = 1ull << w;
    unsigned long long oldf = 0;
    if (lane == 0) {
        start[w] = (int32_t)iter;
        if (!(atomicOr(p.seen + s, bit) & bit)) atomicAdd(&c->seen_pairs, 1ull);
        oldf = atomicOr(p.front[par] + s, bit);
        p.lvl[(size_t)__ldg(p.orig + s) * 64 + w] = 0;
        atomicOr(&c->alive[par], bit);
    }
    oldf = __shfl_sync(FULL, oldf, 0);
    const int rb = __ldg(p.ro + s), len = __ldg(p.ro + s + 1) - rb;
    append_frontier(p, par, lane == 0 && oldf == 0ull && len > 0, s, rb, len);
}

// Read the level columns of the lanes in `mask` into rows of `out`
// (out[row_of_lane * n + v], caller numbering) and, with `recycle`, reset
// them: level 0xFF, seen bit cleared.  Block: 128 vertices x 64 lanes.
__global__ void ms_extract_kernel(uint8_t *lvl, unsigned long long *seen, const int32_t *__restrict__ perm, int64_t n,
                                  unsigned long long mask, const int32_t *__restrict__ lane_row, uint8_t *out,
                                  int64_t out_stride, int recycle, MsCtrl *ctrl)
{
    __shared__ uint8_t tile[128][65];
    const int64_t v0 = (int64_t)blockIdx.x * 128;
    // load 128 x 64 bytes (caller numbering), 16 B per thread per step
    for (int t = threadIdx.x; t < 128 * 4; t += blockDim.x) {
        const int r = t >> 2, q = t & 3;
        const int64_t v = v0 + r;
        uint4 x = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        if (v < n) {
            uint4 *src = reinterpret_cast<uint4 *>(lvl + (size_t)v * 64) + q;
            x = *src;
            if (recycle) {
                // reset the recycled lanes' bytes, keep the others
                uint4 y = x;
                uint8_t *yb = reinterpret_cast<uint8_t *>(&y);
                for (int k = 0; k < 16; ++k)
                    if ((mask >> (q * 16 + k)) & 1ull) yb[k] = 0xFF;
                *src = y;
            }
        }
        const uint8_t *xb = reinterpret_cast<const uint8_t *>(&x);
        for (int k = 0; k < 16; ++k) tile[r][q * 16 + k] = xb[k];
    }
    __syncthreads();
    // write each requested lane's 128 bytes
    unsigned long long mm = mask;
    while (mm) {
        const int ln = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        const int row = lane_row[ln];
        if (row >= 0)
            for (int r = threadIdx.x; r < 128; r += blockDim.x) {
                const int64_t v = v0 + r;
                if (v < n) out[(size_t)row * out_stride + v] = tile[r][ln];
            }
    }
    if (recycle) {
        unsigned long long cleared = 0;
        for (int r = threadIdx.x; r < 128; r += blockDim.x) {
            const int64_t v = v0 + r;
            if (v < n) {
                const int w = __ldg(perm + v);  // seen is indexed by internal id
                cleared += (unsigned long long)__popcll(atomicAnd(seen + w, ~mask) & mask);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cleared += __shfl_xor_sync(0xffffffffu, cleared, o);
        if ((threadIdx.x & 31) == 0 && cleared) atomicAdd(&ctrl->seen_pairs, 0ull - cleared);
    }
}

}  // namespace

// ---- host side ---------------------------------------------------------------

static MsWs *ws_of(Graph *g) { return reinterpret_cast<MsWs *>(g->batch_ws); }

// Release one workspace (its peers first).
static void ws_release(MsWs *w)
{
    if (!w) return;
    for (MsWs *&q : w->peer) {
        ws_release(q);
        q = nullptr;
    }
    if (w->stream) cudaStreamSynchronize(w->stream);
    cudaFree(w->seen);
    cudaFree(w->next);
    for (int b = 0; b < 2; ++b) {
        cudaFree(w->front[b]);
        for (int j = 0; j < 3; ++j) cudaFree(w->fq[b][j]);
    }
    cudaFree(w->lvl);
    cudaFree(w->touched);
    cudaFree(w->ctrl);
    cudaFree(w->start);
    cudaFree(w->lane_src);
    cudaFree(w->lane_row);
    if (w->h_ctrl) cudaFreeHost(w->h_ctrl);
    if (w->h_lanes) cudaFreeHost(w->h_lanes);
    if (w->b_exec) cudaGraphExecDestroy(w->b_exec);
    cudaFree(w->b_lanes);
    if (w->h_roots) cudaFreeHost(w->h_roots);
    cudaFree(w->b_tmp);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->stream) cudaStreamDestroy(w->stream);
    delete w;
}

// A new workspace with its own stream; nullptr (error recorded) on failure.
static MsWs *ws_create(Graph *g, int *rc_out)
{
    MsWs *w = new (std::nothrow) MsWs();
    if (!w) {
        *rc_out = set_error(BFS_ERR_OOM, "bfs_run_batch: host allocation");
        return nullptr;
    }
    const int64_t n = g->n;
    w->fcap = n + 2 * (g->m / H) + 2;
    auto bad = [&](cudaError_t e, const char *what) -> MsWs * {
        *rc_out = cuda_error(e, what);
        ws_release(w);
        return nullptr;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&w->seen, (size_t)n * 8)) != cudaSuccess) return bad(e, "cudaMalloc(seen)");
    if ((e = cudaMalloc(&w->next, (size_t)n * 8)) != cudaSuccess) return bad(e, "cudaMalloc(next)");
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaMalloc(&w->front[b], (size_t)n * 8)) != cudaSuccess) return bad(e, "cudaMalloc(front)");
        for (int j = 0; j < 3; ++j)
            if ((e = cudaMalloc(&w->fq[b][j], (size_t)w->fcap * 4)) != cudaSuccess) return bad(e, "cudaMalloc(frontier)");
    }
    if ((e = cudaMalloc(&w->lvl, (size_t)n * 64)) != cudaSuccess) return bad(e, "cudaMalloc(levels)");
    if ((e = cudaMalloc(&w->touched, (size_t)n * 4)) != cudaSuccess) return bad(e, "cudaMalloc(touched)");
    if ((e = cudaMalloc(&w->ctrl, sizeof(MsCtrl))) != cudaSuccess) return bad(e, "cudaMalloc(ms ctrl)");
    if ((e = cudaMalloc(&w->start, 64 * 4)) != cudaSuccess) return bad(e, "cudaMalloc(start)");
    if ((e = cudaMalloc(&w->lane_src, 64 * 4)) != cudaSuccess) return bad(e, "cudaMalloc(lane sources)");
    if ((e = cudaMalloc(&w->lane_row, 64 * 4)) != cudaSuccess) return bad(e, "cudaMalloc(lane rows)");
    if ((e = cudaMallocHost(&w->h_ctrl, sizeof(MsCtrl))) != cudaSuccess) return bad(e, "cudaMallocHost(ms ctrl)");
    // the mirror's address as the device sees it (pinned memory is mapped
    // under unified addressing); without one, reads fall back to a copy
    if (cudaHostGetDevicePointer((void **)&w->d_ctrl_mirror, w->h_ctrl, 0) != cudaSuccess) {
        w->d_ctrl_mirror = nullptr;
        (void)cudaGetLastError();
    }
    if ((e = cudaMallocHost(&w->h_lanes, 2 * 64 * 4)) != cudaSuccess) return bad(e, "cudaMallocHost(lanes)");
    if ((e = cudaStreamCreateWithPriority(&w->stream, cudaStreamNonBlocking, g->stream_priority)) != cudaSuccess)
        return bad(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming)) != cudaSuccess) return bad(e, "cudaEventCreate");
    const int rc = ms_reset_ws(g, w);
    if (rc != BFS_OK) {
        *rc_out = rc;
        ws_release(w);
        return nullptr;
    }
    return w;
}

int ms_alloc(Graph *g, MsWs **out)
{
    if (g->batch_ws) {
        *out = ws_of(g);
        return BFS_OK;
    }
    int rc = BFS_OK;
    MsWs *w = ws_create(g, &rc);
    if (!w) return rc;
    g->batch_ws = w;
    *out = w;
    return BFS_OK;
}

void ms_free(Graph *g)
{
    ws_release(ws_of(g));
    g->batch_ws = nullptr;
}

// All lanes free: clear the bit words, levels 0xFF, counters zero.
int ms_reset(Graph *g) { return ms_reset_ws(g, ws_of(g)); }

int ms_reset_ws(Graph *g, MsWs *w)
{
    const int64_t n = g->n;
    cudaStream_t s = w->stream;
    GB_CUDA(cudaMemsetAsync(w->seen, 0, (size_t)n * 8, s));
    GB_CUDA(cudaMemsetAsync(w->next, 0, (size_t)n * 8, s));
    GB_CUDA(cudaMemsetAsync(w->front[0], 0, (size_t)n * 8, s));
    GB_CUDA(cudaMemsetAsync(w->front[1], 0, (size_t)n * 8, s));
    GB_CUDA(cudaMemsetAsync(w->lvl, 0xFF, (size_t)n * 64, s));
    GB_CUDA(cudaMemsetAsync(w->ctrl, 0, sizeof(MsCtrl), s));
    GB_CUDA(cudaMemsetAsync(w->start, 0, 64 * 4, s));
    return BFS_OK;
}

static MsParams make_params(Graph *g, MsWs *w, uint32_t max_iters)
{
    MsParams p;
    p.ro = g->d_row_offsets;
    p.col = g->d_col_idx;
    p.orig = g->d_orig;
    p.seen = w->seen;
    p.next = w->next;
    p.front[0] = w->front[0];
    p.front[1] = w->front[1];
    p.lvl = w->lvl;
    for (int b = 0; b < 2; ++b) {
        p.fu[b] = w->fq[b][0];
        p.fb[b] = w->fq[b][1];
        p.fl[b] = w->fq[b][2];
    }
    p.touched = w->touched;
    p.start = w->start;
    p.ctrl = w->ctrl;
    p.n = (int32_t)g->n;
    p.split32 = (int32_t)g->split32;
    p.symmetric = g->symmetric ? 1 : 0;
    p.m = g->m;
    p.n_nonzero = g->n_nonzero;
    p.fcap = (uint32_t)std::min<int64_t>(w->fcap, 0x7FFFFFFFLL);
    p.max_iters = max_iters;
    p.timeout_ns = (uint64_t)g->opt.timeout_ns;
    return p;
}

// Inject sources (caller numbering, validated) into the lanes of `mask`;
// lane_src_host[lane] holds each source.  Asynchronous on the ws stream.
int ms_inject(Graph *g, const int32_t *lane_src_caller, unsigned long long mask)
{
    MsWs *w = ws_of(g);
    cudaStream_t s = w->stream;
    // caller ids -> internal ids through perm on the device: copy the caller
    // ids, then map them with a gather done by the inject kernel's inputs
    int32_t *h = w->h_lanes;
    for (int i = 0; i < 64; ++i) h[i] = ((mask >> i) & 1ull) ? lane_src_caller[i] : 0;
    GB_CUDA(cudaMemcpyAsync(w->lane_src, h, 64 * 4, cudaMemcpyHostToDevice, s));
    map_ids_kernel<<<1, 64, 0, s>>>(w->lane_src, g->d_perm, 64);
    MsParams p = make_params(g, w, 0);
    ms_inject_kernel<<<8, 256, 0, s>>>(p, w->lane_src, mask, w->start);
    GB_CUDA(cudaGetLastError());
    return BFS_OK;
}

// CTAs of ms_kernel<MS_WPB> that fit on the GPU at once (up to 32 warps
// per SM); 0 with the error recorded if none fits.
template <int MS_WPB>
static int ms_full_grid(Graph *g)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ms_kernel<MS_WPB>, MS_WPB * 32, 0);
    if (e != cudaSuccess) {
        cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(ms_kernel)");
        return 0;
    }
    if (per_sm < 1) {
        set_error(BFS_ERR_CUDA, "ms_kernel: no CTA fits on an SM");
        return 0;
    }
    return std::min(per_sm, 32 / MS_WPB) * g->num_sms;
}

static int ms_full_grid(Graph *g) { return g->opt.batch_block == 512 ? ms_full_grid<16>(g) : ms_full_grid<8>(g); }

// One cooperative launch of ms_kernel with CTAs of MS_WPB warps.
template <int MS_WPB>
static int launch_ms(Graph *g, MsWs *w, const MsParams &prm, int max_ctas)
{
    auto kern = ms_kernel<MS_WPB>;
    int grid = ms_full_grid<MS_WPB>(g);
    if (grid < 1) return bfs_last_status() < 0 ? bfs_last_status() : BFS_ERR_CUDA;
    if (max_ctas > 0) grid = std::min(grid, max_ctas);
    cudaError_t e;
    MsParams p = prm;
    void *args[] = {&p};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(MS_WPB * 32), args, 0, w->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(ms_kernel)");
    return BFS_OK;
}

// Run up to max_iters iterations (stops early when no lane has a frontier),
// with at most max_ctas CTAs (0 = as many as fit) of BATCH_BLOCK threads.
static int ms_step_ws(Graph *g, MsWs *w, uint32_t max_iters, int max_ctas)
{
    const MsParams p = make_params(g, w, max_iters);
    return g->opt.batch_block == 512 ? launch_ms<16>(g, w, p, max_ctas) : launch_ms<8>(g, w, p, max_ctas);
}

int ms_step_capped(Graph *g, uint32_t max_iters, int max_ctas) { return ms_step_ws(g, ws_of(g), max_iters, max_ctas); }

int ms_step(Graph *g, uint32_t max_iters) { return ms_step_capped(g, max_iters, g->opt.max_ctas); }

// The control block written to its pinned host mirror by one warp: stores
// over the host link, so that the read does not queue on a copy engine
// behind other graphs' result copies.
__global__ void ms_ctrl_mirror_kernel(const MsCtrl *__restrict__ c, MsCtrl *mirror)
{
    constexpr int kWords = (int)(sizeof(MsCtrl) / 4);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(c);
    uint32_t *dst = reinterpret_cast<uint32_t *>(mirror);
    for (int i = threadIdx.x; i < kWords; i += blockDim.x) dst[i] = __ldcg(src + i);
}

// Copy the control block to pinned host memory and wait for it.
static int ms_read_ctrl_ws(MsWs *w, MsCtrl *out)
{
    if (w->d_ctrl_mirror) {
        ms_ctrl_mirror_kernel<<<1, 32, 0, w->stream>>>(w->ctrl, w->d_ctrl_mirror);
        GB_CUDA(cudaGetLastError());
    } else {
        GB_CUDA(cudaMemcpyAsync(w->h_ctrl, w->ctrl, sizeof(MsCtrl), cudaMemcpyDeviceToHost, w->stream));
    }
    GB_CUDA(cudaStreamSynchronize(w->stream));
    *out = *w->h_ctrl;
    return BFS_OK;
}

int ms_read_ctrl(Graph *g, MsCtrl *out) { return ms_read_ctrl_ws(ws_of(g), out); }

// Level columns of the lanes in `mask` -> rows of `out` (device memory,
// out_stride bytes apart; lane_row_host[lane] = row, -1 = skip); with
// recycle the lanes are reset for reuse.  Asynchronous on the ws stream.
int ms_extract(Graph *g, unsigned long long mask, const int32_t *lane_row_host, uint8_t *out, int64_t out_stride,
               bool recycle)
{
    MsWs *w = ws_of(g);
    cudaStream_t s = w->stream;
    int32_t *h = w->h_lanes + 64;
    for (int i = 0; i < 64; ++i) h[i] = lane_row_host ? lane_row_host[i] : -1;
    GB_CUDA(cudaMemcpyAsync(w->lane_row, h, 64 * 4, cudaMemcpyHostToDevice, s));
    const int64_t blocks = (g->n + 127) / 128;
    ms_extract_kernel<<<(unsigned)blocks, 128, 0, s>>>(w->lvl, w->seen, g->d_perm, g->n, mask, w->lane_row, out,
                                                      out_stride, recycle ? 1 : 0, w->ctrl);
    GB_CUDA(cudaGetLastError());
    return BFS_OK;
}

// One row per blockIdx.y; 16-byte loads and stores when the row length and
// the destination allow them, bytes otherwise.
__global__ void rows_to_host_kernel(const uint8_t *__restrict__ stage, int64_t n, RowsToHost job)
{
    const int i = blockIdx.y;
    const uint8_t *src = stage + (size_t)job.rows[i] * n;
    uint8_t *dst = job.dst[i];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((n & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (int64_t k = t0; k < n / 16; k += stride) d4[k] = __ldcg(s4 + k);
    } else {
        for (int64_t k = t0; k < n; k += stride) dst[k] = src[k];
    }
}

bool ms_host_addressable(const void *p, uint8_t **dev_ptr)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev_ptr = static_cast<uint8_t *>(a.devicePointer);
    return true;
}

int ms_rows_to_host(const uint8_t *stage, int64_t n, const RowsToHost &job, cudaStream_t stream)
{
    if (job.count <= 0) return BFS_OK;
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (n / 16 + 255) / 256));
    rows_to_host_kernel<<<dim3(gx, (unsigned)job.count), 256, 0, stream>>>(stage, n, job);
    GB_CUDA(cudaGetLastError());
    return BFS_OK;
}

__global__ void map_ids_kernel(int32_t *ids, const int32_t *__restrict__ perm, int k)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) ids[i] = perm[ids[i]];
}

__global__ void batch_lanes_kernel(const int32_t *__restrict__ roots, const int32_t *__restrict__ perm, int32_t k,
                                   int out_dev, int width, int32_t *src, int32_t *rows)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) {
        src[i] = perm[roots[i]];
        rows[i] = out_dev ? i : i % width;
    }
}

// The launch sequence of one bfs_run_batch call, on the workspace stream:
// the roots from the pinned staging buffer to the device, their internal ids
// and output rows, a workspace reset, then per batch of `width` sources:
// inject the lanes from device memory, run to completion, extract the level
// rows with lane recycling (which leaves the workspace clean for the next
// batch) and, for host outputs, copy the rows back.  No host round trip.
static int enqueue_batches(Graph *g, MsWs *w, int32_t k, uint8_t *level_out, bool out_dev, int groups, int cap)
{
    const int64_t n = g->n;
    cudaStream_t s = w->stream;
    const int width = g->opt.batch_width;
    int32_t *d_roots = w->b_lanes, *d_src = w->b_lanes + w->b_cap, *d_rows = w->b_lanes + 2 * w->b_cap;
    GB_CUDA(cudaMemcpyAsync(d_roots, w->h_roots, (size_t)k * 4, cudaMemcpyHostToDevice, s));
    batch_lanes_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(d_roots, g->d_perm, k, out_dev ? 1 : 0, width, d_src,
                                                                 d_rows);
    GB_CUDA(cudaGetLastError());
    // the other groups start once the sources are mapped (fork) ...
    if (groups > 1) {
        GB_CUDA(cudaEventRecord(w->ev, s));
        for (int gi = 1; gi < groups; ++gi) GB_CUDA(cudaStreamWaitEvent(w->peer[gi - 1]->stream, w->ev, 0));
    }
    // ... and batch b runs on group b % groups, each group's batches in turn
    const int nb = (int)((k + width - 1) / width);
    for (int gi = 0; gi < groups; ++gi) {
        MsWs *wg = gi == 0 ? w : w->peer[gi - 1];
        cudaStream_t sg = wg->stream;
        int rc = ms_reset_ws(g, wg);
        if (rc != BFS_OK) return rc;
        uint8_t *d_out = out_dev ? level_out : wg->b_tmp;
        const MsParams p0 = make_params(g, wg, 0);
        for (int b = gi; b < nb; b += groups) {
            const int32_t b0 = (int32_t)b * width;
            const int kb = std::min<int32_t>(width, k - b0);
            const unsigned long long mask = (kb == 64) ? ~0ull : ((1ull << kb) - 1ull);
            ms_inject_kernel<<<8, 256, 0, sg>>>(p0, d_src + b0, mask, wg->start);
            GB_CUDA(cudaGetLastError());
            if ((rc = ms_step_ws(g, wg, 0x7FFFFFFFu, cap)) != BFS_OK) return rc;
            ms_extract_kernel<<<(unsigned)((n + 127) / 128), 128, 0, sg>>>(wg->lvl, wg->seen, g->d_perm, n, mask,
                                                                          d_rows + b0, d_out, n, 1, wg->ctrl);
            GB_CUDA(cudaGetLastError());
            if (!out_dev)
                GB_CUDA(cudaMemcpyAsync(level_out + (size_t)b0 * n, d_out, (size_t)kb * n, cudaMemcpyDeviceToHost, sg));
        }
    }
    // (join) the first stream waits for the others
    for (int gi = 1; gi < groups; ++gi) {
        GB_CUDA(cudaEventRecord(w->peer[gi - 1]->ev, w->peer[gi - 1]->stream));
        GB_CUDA(cudaStreamWaitEvent(s, w->peer[gi - 1]->ev, 0));
    }
    return BFS_OK;
}

// bfs_run_batch: batches of `batch_width` sources, each run to completion.
// The first call of a shape (k, output buffer, options) captures the launch
// sequence into a CUDA graph (persistent cooperative kernels included); a
// later call of the same shape copies its roots to the staging buffer and
// replays the graph.  Device-side status bits accumulate over the batches
// and are read once at the end.
int ms_run_batch(Graph *g, const int32_t *roots, int32_t k, uint8_t *level_out)
{
    MsWs *w = nullptr;
    int rc = ms_alloc(g, &w);
    if (rc != BFS_OK) return rc;
    if (k == 0) return BFS_OK;
    const int64_t n = g->n;
    cudaStream_t s = w->stream;
    const bool out_dev = is_device_pointer(level_out);
    const int width = g->opt.batch_width;
    // batches run `groups` at a time, each group on its own workspace and
    // stream with an equal share of the GPU
    const int nb = (int)((k + width - 1) / width);
    const int full = ms_full_grid(g);
    if (full < 1) return bfs_last_status() < 0 ? bfs_last_status() : BFS_ERR_CUDA;
    const int grid = g->opt.max_ctas > 0 ? std::min(g->opt.max_ctas, full) : full;
    // no more groups than batches or CTAs, so that the groups' grids add up to at most `grid`
    const int groups = std::max(1, std::min(std::min(std::min(g->opt.batch_streams, kMaxBatchStreams), nb), grid));
    const int cap = std::max(1, grid / groups);
    // buffers sized for this call (a new buffer invalidates the captured graph)
    auto drop_graph = [&] {
        if (w->b_exec) cudaGraphExecDestroy(w->b_exec);
        w->b_exec = nullptr;
        w->b_key = MsWs::Key{};
    };
    for (int gi = 1; gi < groups; ++gi)
        if (!w->peer[gi - 1]) {
            drop_graph();
            MsWs *q = ws_create(g, &rc);
            if (!q) return rc;
            w->peer[gi - 1] = q;
        }
    if (w->b_cap < k) {
        drop_graph();
        cudaFree(w->b_lanes);
        if (w->h_roots) cudaFreeHost(w->h_roots);
        w->b_lanes = nullptr;
        w->h_roots = nullptr;
        w->b_cap = 0;
        GB_CUDA(cudaMalloc(&w->b_lanes, (size_t)k * 3 * 4));
        GB_CUDA(cudaMallocHost(&w->h_roots, (size_t)k * 4));
        w->b_cap = k;
    }
    for (int gi = 0; gi < groups && !out_dev; ++gi) {
        MsWs *wg = gi == 0 ? w : w->peer[gi - 1];
        if (wg->b_tmp_width < width) {  // each group's staging rows for host outputs
            drop_graph();
            cudaFree(wg->b_tmp);
            wg->b_tmp = nullptr;
            wg->b_tmp_width = 0;
            GB_CUDA(cudaMalloc(&wg->b_tmp, (size_t)width * n));
            wg->b_tmp_width = width;
        }
    }
    memcpy(w->h_roots, roots, (size_t)k * 4);

    MsWs::Key key;
    key.k = k;
    key.out = level_out;
    key.out_dev = out_dev ? 1 : 0;
    key.width = width;
    key.block = g->opt.batch_block;
    key.max_ctas = g->opt.max_ctas;
    key.streams = groups;
    key.timeout_ns = g->opt.timeout_ns;
    if (!(w->b_exec && w->b_key == key)) {
        drop_graph();
        cudaGraph_t graph = nullptr;
        bool captured = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (captured) {
            const int erc = enqueue_batches(g, w, k, level_out, out_dev, groups, cap);
            captured = cudaStreamEndCapture(s, &graph) == cudaSuccess && erc == BFS_OK && graph;
            if (captured) captured = cudaGraphInstantiate(&w->b_exec, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            if (!captured) w->b_exec = nullptr;
        }
        cudaGetLastError();  // a failed capture leaves no sticky error
        clear_error();
        if (captured) w->b_key = key;
    }
    if (w->b_exec) {
        GB_CUDA(cudaGraphLaunch(w->b_exec, s));
    } else if ((rc = enqueue_batches(g, w, k, level_out, out_dev, groups, cap)) != BFS_OK) {
        cudaStreamSynchronize(s);
        for (int gi = 1; gi < groups; ++gi) cudaStreamSynchronize(w->peer[gi - 1]->stream);
        return rc;
    }
    // every group's status, read once all groups are done: the first stream
    // has joined the others (a replayed graph runs every group on it)
    GB_CUDA(cudaStreamSynchronize(s));
    unsigned status = 0;
    unsigned long long bounds = 0;
    for (int gi = 0; gi < groups; ++gi) {
        MsWs *wg = gi == 0 ? w : w->peer[gi - 1];
        MsCtrl st;
        if ((rc = ms_read_ctrl_ws(wg, &st)) != BFS_OK) return rc;
        status |= st.status;
        if (st.bounds) bounds = st.bounds;
    }
    if (status & ST_BOUNDS)
        return set_error(BFS_ERR_CUDA, std::string("bfs_run_batch: index out of range in ") + bounds_site_name(bounds) +
                                           " (index " + std::to_string((long long)(bounds & 0xFFFFFFFFFFFFull)) + ")");
    if (status & ST_TIMEOUT) return set_error(BFS_ERR_TIMEOUT, "bfs_run_batch: a device-side wait ran out");
    if (status & ST_OVERFLOW) return set_error(BFS_ERR_CUDA, "bfs_run_batch: a frontier append ran past its capacity");
    if (status & ST_DEPTH) return set_error(BFS_ERR_DEPTH, "bfs_run_batch: a level exceeds 254");
    return BFS_OK;
}

}  // namespace gbbfs
