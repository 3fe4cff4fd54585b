// topdown_warp.cu -- single-source level-synchronous top-down BFS with
// warp-private work pipelines (the default expansion mode).
//
// Method as in topdown.cu (Alg. 2 with an atomic
// visited bitmap, word v>>5 bit v&31 as in Listing 1; P[s] = s; layer L_d
// finished before L_{d+1}, Sec. 3); one persistent cooperative kernel per
// search.  The difference is who works together: every warp runs its own
// pipeline with only __syncwarp, so the 16 warps of an SM overlap each
// other's memory latency instead of meeting at CTA barriers.
//
// Frontier layout (built by the warps that discover the vertices):
//   entry  (u, beg, len), 1 <= len <= W          -- a vertex and its list
//   unit   (first entry, count), count <= 32, < 2W edges
//   hub slice (u, beg, len <= W) for vertices of degree > W
// A warp flushes its shared-memory buffer of newly reached vertices by
// reserving entries and units with one 64-bit atomicAdd and cutting units
// where the running edge count crosses a multiple of W or every 32 entries.
//
// Work items of a layer (hub slices, then units) are dealt round-robin to
// the grid's warps; a layer with fewer items than half the warps deals each
// hub slice in up to 12 parts of >= 32 edges.  Per item a warp: stages the
// adjacency into its shared buffer with cp.async, issued one item ahead (an
// item of >= 4 lists as one flattened copy, fewer lists list by list),
// padded with the root's id to a multiple of 128 entries; reads the staged
// entries 16 bytes at a time and tests each one's visited word (12 loads per
// lane in flight), keeping the candidates as a per-lane bit mask (pass A);
// puts the candidates and their sources into a per-warp buffer whose claims
// (atomicOr, two per lane in flight) wait until it fills or the layer ends
// (pass B); and queues the winners for the next flush.  Descriptors and
// entries of the next items are prefetched into registers while the current
// item is processed.
//
// Mode 4 (td_thin_kernel) runs the same layer step with 32 lighter warps
// per SM that read each item's lists straight from memory and claim each
// candidate at once.
//
// Mode 2 (RST) is the atomic-free variant of Alg. 3: pass B sets the bit of
// the output bitmap with a plain read-modify-write (bits of other vertices in
// the same word may be lost in a race) and records P[v] = u - n; after the
// layer's expansion a restoration pass takes every non-zero output word,
// finds the vertices of its 32 bits with a negative P, restores P[v] += n,
// sets their visited bits and queues them through the same warp flush.  A
// race can only drop a bit from a word that the last writer left non-zero,
// so the pass sees every vertex discovered in the layer (Sec. 3.3.2).
//
// Mode 3 (HYB) is the direction-optimising search (the bottom-up steps of the
// hybrid algorithm that Sec. 3 calls the state of the art and Sec. 8 plans
// for): a layer runs bottom-up once the frontier's edges exceed the
// unexplored edges / alpha, and top-down again once the frontier has fewer
// than n / beta vertices.  In a bottom-up layer each warp owns whole visited
// words (dealt round-robin); every unvisited vertex scans its in-edges (the
// CSR itself when every edge has its reverse, whose sorted rows put the hubs
// first; else the transposed CSR) until it meets a vertex of the frontier
// bitmap, whose low (hub) words sit in the CTA's shared memory.
//
// All waits are bounded (grid barrier timeout -> ST_TIMEOUT, clean exit).
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.cuh"

namespace gbbfs {
namespace {

using namespace dev;

constexpr int W = 320;       // unit edge target and hub slice length
constexpr int MAXI = 2 * W;  // edges of one work item are < MAXI
constexpr int OBW = 128;     // out-buffer entries per warp
constexpr int UA = 12;       // pass A: visited-word loads per lane in flight
constexpr int UB = 2;        // pass B: claims per lane in flight
constexpr int CB = 64;       // modes 0, 3: deferred claims per warp (two per lane per round)
constexpr int VW = 4;        // bottom-up: visited words per warp in flight

enum { KM_ATOMIC = 0, KM_RESTORE = 1, KM_HYBRID = 2 };  // kernel variants
enum { FL_LP = 1, FL_CNT = 2 };  // warp_flush: write level/parent; count frontier size and edges

struct WParams {
    const int32_t *__restrict__ ro;
    const int32_t *__restrict__ col;
    int32_t *level;
    int32_t *parent;  // may be null
    const int32_t *__restrict__ perm;  // caller id -> internal id
    const int32_t *__restrict__ orig;  // internal id -> caller id
    uint32_t *bitmap;
    uint2 *vo;       // mode 2: (visited, output) bitmap words of Alg. 3, interleaved
    uint32_t *front[2];  // mode 3: frontier bitmaps of bottom-up layers [layer parity]
    int32_t *pint;   // mode 2: predecessors in internal numbering (Alg. 3 `P`)
    int32_t *eu[2], *eb[2], *el[2];  // entries [buffer]
    int32_t *us[2], *uc[2];          // units [buffer]
    int32_t *hu[2], *hb[2], *hl[2];  // hub slices [buffer]
    Ctrl *ctrl;
    int64_t *stats;  // [kMaxStatLayers][4] or null
    int32_t n;
    int32_t root;
    int64_t m;            // directed entries (sum of degrees)
    int32_t n_nonzero;    // internal ids below have degree >= 1
    int32_t alpha, beta;  // mode 3 switching parameters
    const int32_t *__restrict__ bro;   // mode 3: in-edge CSR of bottom-up layers (the CSR itself
    const int32_t *__restrict__ bcol;  // when every edge has its reverse); null: top-down only
    int32_t bu_n;         // mode 3: vertices a bottom-up layer may reach (internal ids below)
    uint32_t ecap, ucap, hcap;
    int32_t bitmap_words;
    uint64_t timeout_ns;
};

struct alignas(16) WarpSmem {
    int32_t stage[2][MAXI];  // staged adjacency, padded with the root's id to a multiple of 128 entries
    union {
        uint16_t ce[MAXI];   // mode 2: candidate -> edge index inside the item (compacted in place)
        struct {
            int32_t v[CB], u[CB];
        } cand;              // modes 0, 3: candidates whose claim is deferred (vertex, source)
    };
    int32_t off[2][33];      // item entries: prefix of lengths
    int32_t iu[2][32];       // item entries: vertex
    int32_t wv[OBW], wu[OBW];           // claimed vertices and their sources (internal ids)
    int32_t ou[OBW], ob[OBW], ol[OBW];  // flush: the new frontier entries
    int32_t ust[OBW];                   // flush: unit starts
};

template <int WPB>
struct CtaSmem {
    WarpSmem w[WPB];
    int ok;
    unsigned nU, nH, nE;
    unsigned long long st[3];
    unsigned long long hnf, hmf;  // mode 3: size and edges of this layer's frontier
};

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_s32(int32_t *p, int32_t v)
{
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A work item as seen by one lane: the lane's entry (if any) and the item's
// entry count.
struct Item {
    int u, b, l;  // this lane's entry (l = 0 if none)
    int cnt;      // entries in the item (uniform)
};

// Descriptor of item `id`: hub slice (id < nH) or unit.  Uniform loads.
struct Desc {
    int a, c;  // unit: first entry, count; hub: index into the hub queue, -1
};

__device__ __forceinline__ Desc load_desc(const WParams &p, int qi, unsigned nH, unsigned n_items, unsigned id,
                                          unsigned split)
{
    Desc d{0, 0};
    if (id >= n_items) return d;
    if (id < nH * split) {  // part (id % split) of hub slice id / split
        d.a = (int)(id / split);
        d.c = -1 - (int)(id % split);
    } else {
        const int64_t ui = GB_IX(id - nH * split, p.ucap, BS_QUEUE, p.ctrl);
        d.a = __ldcg(p.us[qi] + ui);
        d.c = __ldcg(p.uc[qi] + ui);
    }
    return d;  // checked where it is used, so the loads stay in flight
}

__device__ __forceinline__ Item load_item(const WParams &p, int qi, const Desc &d, bool valid, unsigned split)
{
    const int lane = threadIdx.x & 31;
    Item it{0, 0, 0, 0};
    if (!valid) return it;
    if (d.c < 0) {
        it.cnt = 1;
        if (lane == 0) {
            const int64_t hi = GB_IX(d.a, p.hcap, BS_QUEUE, p.ctrl);
            it.u = __ldcg(p.hu[qi] + hi);
            it.b = __ldcg(p.hb[qi] + hi);
            it.l = __ldcg(p.hl[qi] + hi);
            if (split > 1) {  // a part of at least 32 edges
                const int part = -1 - d.c;
                const int sub = max(32, (it.l + (int)split - 1) / (int)split);
                const int lo = min(it.l, part * sub);
                it.b += lo;
                it.l = min(sub, it.l - lo);
            }
        }
    } else {
        it.cnt = (d.c < 0 || d.c > 32) ? 0 : d.c;  // a unit holds <= 32 entries
        if (it.cnt != d.c && lane == 0) atomicOr(&p.ctrl->status, ST_OVERFLOW);
        if (lane < it.cnt) {
            const int64_t ei = GB_IX(d.a + lane, p.ecap, BS_QUEUE, p.ctrl);
            it.u = __ldcg(p.eu[qi] + ei);
            it.b = __ldcg(p.eb[qi] + ei);
            it.l = __ldcg(p.el[qi] + ei);
        }
    }
    return it;  // lengths are checked in stage_item, so the loads stay in flight
}

// Prefix-sum the item's lengths into off[buf], record vertices, and issue the
// cp.async copies of its adjacency into stage[buf].  An item of >= 4 lists
// is copied as one flattened range, 32 consecutive slots per step (lanes find
// their list by ballots), so that its lists are copied side by side; an item
// of fewer lists list by list: a list of >= 32 edges by the whole warp
// striding over it, a shorter one by its own lane, one edge per step.
// Commits one group per lane.  Returns the item's edge count (uniform).
__device__ __forceinline__ int stage_item(WarpSmem &ws, const WParams &p, const Item &it_in, int buf, int rint)
{
    const int lane = threadIdx.x & 31;
    Item it = it_in;
    if (it.l < 0 || it.l > MAXI) {  // cannot happen for entries this kernel wrote
        atomicOr(&p.ctrl->status, ST_OVERFLOW);
        it.l = 0;
    }
    const bool real = lane < it.cnt;
    const int sl = (real && it.l < 32) ? it.l : 0;
    int inc;
    if (it.cnt == 1) {  // a hub slice or a one-list unit: no scan needed
        inc = __shfl_sync(FULL, it.l, 0);
    } else {
        inc = it.l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
    }
    int et = __shfl_sync(FULL, inc, 31);
    const bool fits = et < MAXI;  // cannot fail: units < 2W edges, slices <= W
    if (!fits) {
        if (lane == 0) atomicOr(&p.ctrl->status, ST_OVERFLOW);
        et = 0;
    }
    const int off = inc - it.l;
    if (real) {
        ws.off[buf][lane] = off;
        ws.iu[buf][lane] = it.u;
    }
    if (lane == 0) ws.off[buf][it.cnt] = et;
    if (fits && it.cnt >= 4) {
        // Flattened copy, 32 slots per step: slot e = e0 + lane belongs to the
        // last entry whose offset is <= e.  Entries starting inside the step
        // are marked by their position; the entry at the step's start is the
        // last one with offset <= e0.  Every entry has >= 1 edge, so
        // positions are distinct.
        const bool has = real && it.l > 0;
#pragma unroll 4
        for (int e0 = 0; e0 < et; e0 += 32) {
            const unsigned starts = __reduce_or_sync(FULL, (has && off > e0 && off < e0 + 32) ? 1u << (off - e0) : 0u);
            const int j0 = __popc(__ballot_sync(FULL, has && off <= e0)) - 1;
            const int jj = (j0 + __popc(starts & ((2u << lane) - 1u))) & 31;
            const int jb = __shfl_sync(FULL, it.b, jj);
            const int jo = __shfl_sync(FULL, off, jj);
            const int e = e0 + lane;
            if (e < et) cp_async4(&ws.stage[buf][e], p.col + GB_IX(jb + (e - jo), p.m, BS_COL, p.ctrl));
        }
    } else if (fits) {
        // long lists
        unsigned big = __ballot_sync(FULL, real && it.l >= 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int bo = __shfl_sync(FULL, off, src);
            const int bb = __shfl_sync(FULL, it.b, src);
            const int bl = __shfl_sync(FULL, it.l, src);
#pragma unroll 4
            for (int k = lane; k < bl; k += 32) cp_async4(&ws.stage[buf][bo + k], p.col + GB_IX(bb + k, p.m, BS_COL, p.ctrl));
        }
        // short lists: each lane copies its own, one edge per step
        const int maxl = (int)__reduce_max_sync(FULL, (unsigned)sl);
        for (int k = 0; k < maxl; ++k)
            if (k < sl) cp_async4(&ws.stage[buf][off + k], p.col + GB_IX(it.b + k, p.m, BS_COL, p.ctrl));
    }
    // pad to a multiple of 128 entries with the root, whose visited bit is
    // set from the start: the padding never becomes a candidate
    const int pend = (et + 127) & ~127;
    for (int k = et + lane; k < pend; k += 32) ws.stage[buf][k] = rint;
    cp_async_commit();
    return et;
}

// Finish the vertices this warp claimed: write level and parent (in the
// caller's numbering), read each one's adjacency range, queue the short
// ones as frontier entries cut into units and the hubs as slices.  All loads
// of a lane are issued together, so one flush costs about one round trip.
template <int FL, typename S = WarpSmem, int OB = OBW>
__device__ __forceinline__ void warp_flush(S &ws, const WParams &p, int set_out, int qo, int c, int next_level)
{
    constexpr int PER = OB / 32;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    __syncwarp();  // winners were written to ws.wv / ws.wu by other lanes
    const int i0 = min(lane * PER, c), i1 = min(i0 + PER, c);
    int rb[PER], re[PER], ov[PER], ou[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = i0 + k;
        if (i < i1) {
            const int v = (int)GB_IX(ws.wv[i], p.n, BS_ROW, p.ctrl);
            rb[k] = __ldg(p.ro + v);
            re[k] = __ldg(p.ro + v + 1);
            ov[k] = (FL & FL_LP) ? __ldg(p.orig + v) : 0;
            ou[k] = ((FL & FL_LP) && p.parent) ? __ldg(p.orig + GB_IX(ws.wu[i], p.n, BS_ORIG, p.ctrl)) : 0;
        }
    }
    int nsmall = 0, nslice = 0;
    long long esum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = i0 + k;
        if (i < i1) {
            if (FL & FL_LP) {
                p.level[GB_IX(ov[k], p.n, BS_LEVEL, p.ctrl)] = next_level;
                if (p.parent) p.parent[GB_IX(ov[k], p.n, BS_PARENT, p.ctrl)] = ou[k];
            }
            const int len = re[k] - rb[k];
            esum += len;
            nsmall += (len >= 1 && len <= W);
            nslice += (len > W) ? (len + W - 1) / W : 0;
        }
    }
    // positions of the short entries (in claim order) and the hub slices
    int sinc = nsmall, hinc = nslice;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, sinc, o);
        const int z = __shfl_up_sync(FULL, hinc, o);
        if (lane >= o) {
            sinc += y;
            hinc += z;
        }
    }
    const int cs = __shfl_sync(FULL, sinc, 31);
    const int total_slices = __shfl_sync(FULL, hinc, 31);
    if (FL & FL_CNT) {  // the next frontier's size and summed degrees
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) esum += __shfl_down_sync(FULL, esum, o);
        if (lane == 0) {
            atomicAdd(&p.ctrl->nf[set_out], (unsigned long long)c);
            atomicAdd(&p.ctrl->mf[set_out], (unsigned long long)esum);
        }
    }
    // the short entries into the flush buffer (their positions need no reservation)
    {
        int spos = sinc - nsmall;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = i0 + k;
            const int len = (i < i1) ? re[k] - rb[k] : 0;
            if (len >= 1 && len <= W) {
                ws.ou[spos] = ws.wv[i];
                ws.ob[spos] = rb[k];
                ws.ol[spos] = len;
                ++spos;
            }
        }
    }
    __syncwarp();
    // cut the short entries into units (<= 32 entries, a new unit where the
    // running edge count crosses a multiple of W)
    const int j0 = min(lane * PER, cs), j1 = min(j0 + PER, cs);
    int units = 0, uinc = 0, nu = 0;
    if (cs > 0) {
        int sum = 0;
        for (int j = j0; j < j1; ++j) sum += ws.ol[j];
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int toff = inc - sum;
        {
            int off = toff;
            for (int j = j0; j < j1; ++j) {
                const bool start = (j % 32 == 0) || (off / W != (off - ws.ol[j - 1]) / W);
                nu += start;
                off += ws.ol[j];
            }
        }
        uinc = nu;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, uinc, o);
            if (lane >= o) uinc += y;
        }
        units = __shfl_sync(FULL, uinc, 31);
        int k = uinc - nu, off = toff;
        for (int j = j0; j < j1; ++j) {
            const bool start = (j % 32 == 0) || (off / W != (off - ws.ol[j - 1]) / W);
            if (start) ws.ust[k++] = j;
            off += ws.ol[j];
        }
    }
    // both reservations in one round trip: hub slices (lane 0), entries and units (lane 1)
    unsigned hbase = 0;
    unsigned long long base = 0;
    if (lane == 0 && total_slices > 0) hbase = atomicAdd(&p.ctrl->hub_count[set_out], (unsigned)total_slices);
    if (lane == 1 && cs > 0)
        base = atomicAdd(&p.ctrl->eu_count[set_out], ((unsigned long long)units << 32) | (unsigned long long)cs);
    hbase = __shfl_sync(FULL, hbase, 0);
    base = __shfl_sync(FULL, base, 1);
    // hub slices: a few per vertex by its own lane, the large hubs by the whole warp
    {
        unsigned hpos = hbase + (unsigned)(hinc - nslice);
        int big_v[PER], big_b[PER], big_l[PER];
        unsigned big_at[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = i0 + k;
            const int len = (i < i1) ? re[k] - rb[k] : 0;
            const int nseg = len > W ? (len + W - 1) / W : 0;
            big_l[k] = nseg > 8 ? len : 0;
            big_v[k] = (i < i1) ? ws.wv[i] : 0;
            big_b[k] = (i < i1) ? rb[k] : 0;
            big_at[k] = hpos;
            if (nseg > 0 && nseg <= 8) {
                for (int sg = 0; sg < nseg; ++sg) {
                    const unsigned g = hpos + (unsigned)sg;
                    if (g < p.hcap) {
                        p.hu[qo][g] = big_v[k];
                        p.hb[qo][g] = rb[k] + sg * W;
                        p.hl[qo][g] = min(W, len - sg * W);
                    } else {
                        atomicOr(&p.ctrl->status, ST_OVERFLOW);
                    }
                }
            }
            hpos += (unsigned)nseg;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            unsigned m = __ballot_sync(FULL, big_l[k] > 0);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const int hv = __shfl_sync(FULL, big_v[k], src);
                const int hb = __shfl_sync(FULL, big_b[k], src);
                const int hl = __shfl_sync(FULL, big_l[k], src);
                const unsigned at = __shfl_sync(FULL, big_at[k], src);
                const int nseg = (hl + W - 1) / W;
                for (int sg = lane; sg < nseg; sg += 32) {
                    const unsigned g = at + (unsigned)sg;
                    if (g < p.hcap) {
                        p.hu[qo][g] = hv;
                        p.hb[qo][g] = hb + sg * W;
                        p.hl[qo][g] = min(W, hl - sg * W);
                    } else {
                        atomicOr(&p.ctrl->status, ST_OVERFLOW);
                    }
                }
            }
        }
    }
    if (cs > 0) {
        const unsigned ebase = (unsigned)(base & 0xffffffffull), ubase = (unsigned)(base >> 32);
        __syncwarp();  // ust was written by other lanes
        for (int j = lane; j < cs; j += 32) {
            const unsigned gi = ebase + (unsigned)j;
            if (gi < p.ecap) {
                p.eu[qo][gi] = ws.ou[j];
                p.eb[qo][gi] = ws.ob[j];
                p.el[qo][gi] = ws.ol[j];
            } else {
                atomicOr(&p.ctrl->status, ST_OVERFLOW);
            }
        }
        for (int k = lane; k < units; k += 32) {
            const int s0 = ws.ust[k];
            const int e0 = (k + 1 < units) ? ws.ust[k + 1] : cs;
            const unsigned gk = ubase + (unsigned)k;
            if (gk < p.ucap) {
                p.us[qo][gk] = (int32_t)(ebase + (unsigned)s0);
                p.uc[qo][gk] = e0 - s0;
            } else {
                atomicOr(&p.ctrl->status, ST_OVERFLOW);
            }
        }
    }
    (void)lt;
    __syncwarp();
}

// Mode 2 (Alg. 3): passes A and B over the staged item in stage[buf] with
// `et` edges.
__device__ __forceinline__ void process_item_rst(WarpSmem &ws, const WParams &p, int buf, int et, int cnt)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    int32_t *stg = ws.stage[buf];
    // pass A: visited filter, candidates compacted in place
    int nc = 0;
    for (int base = 0; base < et; base += 32 * UA) {
        int v[UA];
        unsigned w[UA];
#pragma unroll
        for (int k = 0; k < UA; ++k) {
            const int e = base + k * 32 + lane;
            v[k] = e < et ? stg[e] : -1;
        }
        // Alg. 3: not in vis and not in out; both words share one 8-byte load
        // (a stale out word only sends v on to pass B)
#pragma unroll
        for (int k = 0; k < UA; ++k) {
            if (v[k] >= 0) {
                const uint2 x = __ldca(p.vo + GB_IX((unsigned)v[k] >> 5, p.bitmap_words, BS_VISITED, p.ctrl));
                w[k] = x.x | x.y;
            } else {
                w[k] = 0xffffffffu;
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < UA; ++k) {
            const bool c = v[k] >= 0 && !(w[k] & (1u << (v[k] & 31)));
            const unsigned m = __ballot_sync(FULL, c);
            if (c) {
                const int pos = nc + __popc(m & lt);
                stg[pos] = v[k];
                ws.ce[pos] = (uint16_t)(base + k * 32 + lane);
            }
            nc += __popc(m);
        }
    }
    __syncwarp();
    {
        // pass B of Alg. 3: plain read-modify-write of the out word, then
        // P[v] = u - n.  Lanes whose vertices share a word combine their bits
        // and the lowest of them writes the word once (rows are sorted, so
        // neighbouring candidates often share one); races between warps
        // still lose bits, which the restoration pass repairs.  The (vis, out)
        // pair is read from L2: vis changes only in the restoration pass, but
        // an L1 copy may predate the last one.
        for (int c0 = 0; c0 < nc; c0 += 32 * UB) {
            int v[UB], e[UB];
#pragma unroll
            for (int k = 0; k < UB; ++k) {
                const int i = c0 + k * 32 + lane;
                v[k] = i < nc ? stg[i] : -1;
                e[k] = i < nc ? (int)ws.ce[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < UB; ++k) {
                const unsigned word = v[k] >= 0 ? ((unsigned)v[k] >> 5) : 0xffffffffu;
                const unsigned grp = __match_any_sync(FULL, word);
                const int leader = __ffs(grp) - 1;
                unsigned long long o = ~0ull;
                if (v[k] >= 0 && lane == leader)
                    o = ld_relaxed64(reinterpret_cast<const unsigned long long *>(p.vo + word));
                o = __shfl_sync(FULL, o, leader);
                const unsigned bit = v[k] >= 0 ? 1u << (v[k] & 31) : 0u;
                const unsigned vis_w = (unsigned)o, out_w = (unsigned)(o >> 32);
                const bool need = v[k] >= 0 && !((vis_w | out_w) & bit);
                const unsigned bits = __reduce_or_sync(grp, need ? bit : 0u);
                if (lane == leader && bits) st_relaxed_u32(&p.vo[word].y, out_w | bits);
                if (need) {
                    int lo = 0, hi = cnt;  // source entry: largest j with off[j] <= e
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (ws.off[buf][mid] <= e[k]) lo = mid;
                        else hi = mid;
                    }
                    st_relaxed_s32(p.pint + GB_IX(v[k], p.n, BS_LEVEL, p.ctrl), ws.iu[buf][lo] - p.n);
                }
            }
        }
        __syncwarp();
    }
}

// ---- modes 0 and 3: pass A with deferred claims ----------------------------
//
// Pass A reads the staged item 128 entries at a time (one 16-byte shared
// load per lane and 4 entries), tests each entry's visited word and keeps a
// per-lane bit mask of the candidates (entries whose bit was clear).  The
// candidates, with their sources, go to the warp's deferred-claim buffer;
// the buffer is claimed (pass B: atomicOr, two per lane in flight) only when
// it cannot take the next candidates and at the end of the layer, so one
// atomic round trip serves the candidates of several items.  A candidate
// whose bit another warp sets in the meantime simply loses its atomicOr.

// Claim the deferred candidates cand.v/u[0..nb) and queue the winners.
template <int KM, typename S = WarpSmem, int OB = OBW>
__device__ __forceinline__ void claim_deferred(S &ws, const WParams &p, int &nb, int set_out, int qo, int &ocnt,
                                               int next_level, unsigned &my_new)
{
    constexpr int FL = KM == KM_HYBRID ? (FL_LP | FL_CNT) : FL_LP;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    if (ocnt > OB - CB) {  // room for every winner of this round
        warp_flush<FL, S, OB>(ws, p, set_out, qo, ocnt, next_level);
        ocnt = 0;
    }
    __syncwarp();  // the buffer was filled by other lanes
    const int v0 = lane < nb ? ws.cand.v[lane] : -1;
    const int v1 = lane + 32 < nb ? ws.cand.v[lane + 32] : -1;
    const int u0 = lane < nb ? ws.cand.u[lane] : 0;
    const int u1 = lane + 32 < nb ? ws.cand.u[lane + 32] : 0;
    bool w0 = false, w1 = false;
    if (v0 >= 0) {
        const unsigned bit = 1u << (v0 & 31);
        w0 = !(atomicOr(p.bitmap + GB_IX((unsigned)v0 >> 5, p.bitmap_words, BS_VISITED, p.ctrl), bit) & bit);
    }
    if (v1 >= 0) {
        const unsigned bit = 1u << (v1 & 31);
        w1 = !(atomicOr(p.bitmap + GB_IX((unsigned)v1 >> 5, p.bitmap_words, BS_VISITED, p.ctrl), bit) & bit);
    }
    const unsigned m0 = __ballot_sync(FULL, w0), m1 = __ballot_sync(FULL, w1);
    if (w0) {
        const int pos = ocnt + __popc(m0 & lt);
        ws.wv[pos] = v0;
        ws.wu[pos] = u0;
        ++my_new;
    }
    if (w1) {
        const int pos = ocnt + __popc(m0) + __popc(m1 & lt);
        ws.wv[pos] = v1;
        ws.wu[pos] = u1;
        ++my_new;
    }
    ocnt += __popc(m0) + __popc(m1);
    nb = 0;
    __syncwarp();  // the buffer is read before it is refilled
}

// Pass A over the staged item in stage[buf] (et entries, cnt entries of the
// item; padded to a multiple of 128 with the root): candidates go to the
// deferred-claim buffer (nb entries held).
template <int KM>
__device__ __forceinline__ void process_item_def(WarpSmem &ws, const WParams &p, int buf, int et, int cnt, int rint,
                                                 int next_level, int set_out, int qo, int &ocnt, int &nb,
                                                 unsigned &my_new)
{
    const int lane = threadIdx.x & 31;
    const int32_t *stg = ws.stage[buf];
    const int4 *stg4 = reinterpret_cast<const int4 *>(stg);
    const int u_first = ws.iu[buf][0];
    for (int base = 0; base < et; base += 32 * UA) {
        int v[UA];
#pragma unroll
        for (int c = 0; c < UA / 4; ++c) {
            int4 q = make_int4(rint, rint, rint, rint);
            if (base + 128 * c < et) q = stg4[(base + 128 * c) / 4 + lane];
            v[4 * c + 0] = q.x;
            v[4 * c + 1] = q.y;
            v[4 * c + 2] = q.z;
            v[4 * c + 3] = q.w;
        }
        // L1-cached read: bits are only ever set during a search, so a stale
        // word can only send an already visited vertex on to the atomicOr
        unsigned w[UA];
#pragma unroll
        for (int k = 0; k < UA; ++k) w[k] = __ldca(p.bitmap + GB_IX((unsigned)v[k] >> 5, p.bitmap_words, BS_VISITED, p.ctrl));
        unsigned cm = 0;  // bit k: entry k of this lane is a candidate
#pragma unroll
        for (int k = 0; k < UA; ++k) cm |= (~__funnelshift_r(w[k], w[k], (unsigned)v[k]) & 1u) << k;
        // one candidate per lane per round into the buffer, placed by ballot
        while (__any_sync(FULL, cm != 0u)) {
            int k = -1;
            if (cm) {
                k = __ffs(cm) - 1;
                cm &= cm - 1;
            }
            const unsigned hasc = __ballot_sync(FULL, k >= 0);
            const int total = __popc(hasc);
            if (nb + total > CB) claim_deferred<KM>(ws, p, nb, set_out, qo, ocnt, next_level, my_new);
            if (k >= 0) {
                const int e = base + 128 * (k >> 2) + 4 * lane + (k & 3);  // entry inside the item
                int u = u_first;
                if (cnt > 1) {  // source entry: largest j with off[j] <= e
                    int lo = 0, hi = cnt;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (ws.off[buf][mid] <= e) lo = mid;
                        else hi = mid;
                    }
                    u = ws.iu[buf][lo];
                }
                const int pos = nb + __popc(hasc & lanemask_lt());
                ws.cand.v[pos] = stg[e];
                ws.cand.u[pos] = u;
            }
            nb += total;
        }
    }
    __syncwarp();
}

// ---- direction-optimising mode (KM_HYBRID) ---------------------------------

// Is u in the frontier bitmap F?  Its first `ncache` words are in shared memory.
__device__ __forceinline__ bool in_front(const uint32_t *sF, int ncache, const uint32_t *__restrict__ F, int u)
{
    const unsigned wd = (unsigned)u >> 5;
    const unsigned x = (int)wd < ncache ? sF[wd] : __ldcg(F + wd);
    return (x >> (u & 31)) & 1u;
}

// Top-down -> bottom-up: set the bit of every vertex of the frontier queue
// (entries and hub slices of buffer qi) in the cleared bitmap F.
__device__ __forceinline__ void queue_to_bitmap(const WParams &p, int qi, unsigned nE, unsigned nH, uint32_t *F)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < nE; i += stride) {
        const int u = __ldcg(p.eu[qi] + i);
        atomicOr(F + ((unsigned)u >> 5), 1u << (u & 31));
    }
    for (int64_t i = t0; i < nH; i += stride) {
        const int u = __ldcg(p.hu[qi] + i);
        atomicOr(F + ((unsigned)u >> 5), 1u << (u & 31));
    }
}

// Bottom-up -> top-down: queue the vertices of bitmap F as frontier entries
// and hub slices (buffer qi, counter set si); their levels and parents were
// written by the bottom-up layer that found them.  Words are dealt
// round-robin to the warps.
__device__ __forceinline__ void bitmap_to_queue(WarpSmem &ws, const WParams &p, const uint32_t *F, int si, int qi,
                                                unsigned gw, unsigned GW)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int64_t nwords = p.bitmap_words;
    int ocnt = 0;
    for (int64_t j0 = 0; (int64_t)gw + (int64_t)GW * j0 < nwords; j0 += 32) {
        const int64_t wi = (int64_t)gw + (int64_t)GW * (j0 + lane);
        const unsigned x = wi < nwords ? __ldcg(F + wi) : 0u;
        unsigned nz = __ballot_sync(FULL, x != 0u);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1;
            if (ocnt > OBW - 32) {
                warp_flush<0>(ws, p, si, qi, ocnt, 0);
                ocnt = 0;
            }
            const unsigned m = __shfl_sync(FULL, x, src);
            const int64_t word = (int64_t)gw + (int64_t)GW * (j0 + src);
            if ((m >> lane) & 1u) ws.wv[ocnt + __popc(m & lt)] = (int)(word * 32 + lane);
            ocnt += __popc(m);
        }
    }
    if (ocnt > 0) warp_flush<0>(ws, p, si, qi, ocnt, 0);
}

// One bottom-up layer: every unvisited vertex looks for a neighbour in the
// frontier bitmap F; the first one found is its parent.  A warp owns the
// visited words it is dealt (word gw + GW * j), so their bits and the words
// of the next frontier Fn are written without atomics.  Each lane loads one
// of 32 dealt words; words without an unvisited vertex only clear their Fn
// word, the others are taken VW at a time: every unvisited vertex probes its
// own list in its lane, PK edges per step (rows are sorted, so the hubs come
// first), a vertex of degree < 32 to the end, one of degree >= 32 for its
// first PK edges, after which the whole warp scans the rest, 32 per step.
template <int WPB>
__device__ __forceinline__ void bottom_up(CtaSmem<WPB> &cs, const WParams &p, const uint32_t *__restrict__ F,
                                          uint32_t *Fn, int next_level, unsigned gw, unsigned GW,
                                          unsigned long long &my_new, unsigned long long &my_edges,
                                          unsigned long long &my_mf)
{
    constexpr int PK = 4;
    const int tid = threadIdx.x, lane = tid & 31;
    uint32_t *sF = reinterpret_cast<uint32_t *>(cs.w);  // the top-down buffers are idle here
    constexpr int CW = (int)(sizeof(WarpSmem) * WPB / 4);
    const int64_t nwords = p.bitmap_words;
    const int ncache = (int)min((int64_t)CW, nwords);
    __syncthreads();
    for (int i = tid; i < ncache; i += WPB * 32) sF[i] = __ldcg(F + i);
    __syncthreads();
    for (int64_t j0 = 0; (int64_t)gw + (int64_t)GW * j0 < nwords; j0 += 32) {
        const int64_t lw = (int64_t)gw + (int64_t)GW * (j0 + lane);  // this lane's word
        unsigned lraw = 0xffffffffu, lseen = 0xffffffffu;  // visited bits; + vertices without edges
        bool has = false;
        if (lw < nwords) {
            lraw = __ldcg(p.bitmap + lw);
            const int64_t first = lw * 32;  // vertices >= bu_n have no in-edge: never reached
            const unsigned valid = first >= p.bu_n ? 0u
                                   : (p.bu_n - first >= 32 ? 0xffffffffu : (1u << (p.bu_n - first)) - 1u);
            lseen = lraw | ~valid;
            has = lseen != 0xffffffffu;
            if (!has) Fn[lw] = 0u;
        }
        unsigned work = __ballot_sync(FULL, has);
        while (work) {
            int64_t v[VW];
            unsigned vis[VW];
            int src[VW], beg[VW], end[VW], par[VW], e[VW];
            bool unv[VW];
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                src[j] = work ? __ffs(work) - 1 : -1;
                if (work) work &= work - 1;
                const int sl = src[j] < 0 ? 0 : src[j];
                const unsigned seen = __shfl_sync(FULL, lseen, sl);
                vis[j] = __shfl_sync(FULL, lraw, sl);
                v[j] = ((int64_t)gw + (int64_t)GW * (j0 + sl)) * 32 + lane;
                unv[j] = src[j] >= 0 && !((seen >> lane) & 1u);
            }
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                beg[j] = unv[j] ? __ldg(p.bro + GB_IX(v[j], p.n, BS_ROW, p.ctrl)) : 0;
                end[j] = unv[j] ? __ldg(p.bro + v[j] + 1) : 0;
                par[j] = -1;
                e[j] = beg[j];
            }
            // every unvisited vertex in its own lane, PK edges per step
            while (true) {
                bool act[VW], any = false;
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    act[j] = par[j] < 0 && e[j] < end[j] && (end[j] - beg[j] < 32 || e[j] == beg[j]);
                    any |= act[j];
                }
                if (!__any_sync(FULL, any)) break;
                int u[VW][PK];
                bool f[VW][PK];
#pragma unroll
                for (int j = 0; j < VW; ++j)
#pragma unroll
                    for (int t = 0; t < PK; ++t)
                        u[j][t] = (act[j] && e[j] + t < end[j]) ? __ldg(p.bcol + GB_IX(e[j] + t, p.m, BS_COL, p.ctrl)) : -1;
#pragma unroll
                for (int j = 0; j < VW; ++j)
#pragma unroll
                    for (int t = 0; t < PK; ++t) f[j][t] = u[j][t] >= 0 && in_front(sF, ncache, F, u[j][t]);
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    if (!act[j]) continue;
#pragma unroll
                    for (int t = PK - 1; t >= 0; --t)
                        if (f[j][t]) par[j] = u[j][t];  // the first of the step
                    my_edges += (unsigned long long)min(PK, end[j] - e[j]);
                    e[j] += PK;
                }
            }
            // degree >= 32 and not found yet: the warp scans the rest of one list at a time
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                unsigned hv = __ballot_sync(FULL, par[j] < 0 && e[j] < end[j]);
                while (hv) {
                    const int hl = __ffs(hv) - 1;
                    hv &= hv - 1;
                    const int hb = __shfl_sync(FULL, e[j], hl), he = __shfl_sync(FULL, end[j], hl);
                    int found = -1;
                    for (int e0 = hb; e0 < he; e0 += 32) {
                        const int ee = e0 + lane;
                        const int u = ee < he ? __ldg(p.bcol + GB_IX(ee, p.m, BS_COL, p.ctrl)) : -1;
                        const bool f = u >= 0 && in_front(sF, ncache, F, u);
                        const unsigned m = __ballot_sync(FULL, f);
                        if (lane == 0) my_edges += (unsigned long long)min(32, he - e0);
                        if (m) {
                            found = __shfl_sync(FULL, u, __ffs(m) - 1);
                            break;
                        }
                    }
                    if (lane == hl) par[j] = found;
                }
            }
            // the vertices found: level, parent, visited bits, next frontier
            int ov[VW], ou[VW];
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                ov[j] = par[j] >= 0 ? __ldg(p.orig + GB_IX(v[j], p.n, BS_ORIG, p.ctrl)) : 0;
                ou[j] = (par[j] >= 0 && p.parent) ? __ldg(p.orig + GB_IX(par[j], p.n, BS_ORIG, p.ctrl)) : 0;
            }
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                const bool found = par[j] >= 0;
                const unsigned m = __ballot_sync(FULL, found);
                if (found) {
                    p.level[GB_IX(ov[j], p.n, BS_LEVEL, p.ctrl)] = next_level;
                    if (p.parent) p.parent[GB_IX(ov[j], p.n, BS_PARENT, p.ctrl)] = ou[j];
                    my_mf += (unsigned long long)(end[j] - beg[j]);
                }
                if (lane == 0 && src[j] >= 0) {
                    const int64_t w = (int64_t)gw + (int64_t)GW * (j0 + src[j]);
                    Fn[w] = m;
                    if (m) p.bitmap[w] = vis[j] | m;
                    my_new += (unsigned long long)__popc(m);
                }
            }
        }
    }
    __syncthreads();  // the shared buffers go back to the top-down layers
}

// a[0..n) = -1: 16-byte stores from the first 16-byte boundary of a (an
// int32 array is 4-byte aligned), single stores before it and after the last.
__device__ __forceinline__ void fill_minus1(int32_t *a, int64_t n, int64_t t0, int64_t stride)
{
    const int64_t head = min(n, (int64_t)((16u - (unsigned)(reinterpret_cast<uintptr_t>(a) & 15u)) & 15u) / 4);
    const int64_t nv = (n - head) / 4;
    int4 *v = reinterpret_cast<int4 *>(a + head);
    for (int64_t i = t0; i < nv; i += stride) v[i] = make_int4(-1, -1, -1, -1);
    if (t0 < head) a[t0] = -1;
    if (t0 < n - head - 4 * nv) a[head + 4 * nv + t0] = -1;
}

// The root is its own parent at level 0 (Alg. 1), written once the grid has
// passed the barrier after the initialisation.
__device__ __forceinline__ void td_root_outputs(const WParams &p)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.level[p.root] = 0;
        if (p.parent) p.parent[p.root] = p.root;
    }
}

// Initialisation (Alg. 1: P = infinity except P[s] = s; vis = {s}) and the
// root as the first frontier (an entry, or hub slices), by the whole grid.
template <int KM>
__device__ __forceinline__ void td_init(const WParams &p, int rint)
{
    const int tid = threadIdx.x;
    const unsigned nthr = blockDim.x;
    Ctrl *c = p.ctrl;
    {
        const int64_t stride = (int64_t)gridDim.x * nthr;
        // level and parent -1 everywhere (the root's entries are written
        // after the first grid barrier), 16 bytes per store
        fill_minus1(p.level, p.n, (int64_t)blockIdx.x * nthr + tid, stride);
        if (p.parent) fill_minus1(p.parent, p.n, (int64_t)blockIdx.x * nthr + tid, stride);
        if (KM == KM_RESTORE)
            for (int64_t i = (int64_t)blockIdx.x * nthr + tid; i < p.n; i += stride)
                p.pint[i] = (i == rint) ? rint : INT_MAX;  // Alg. 3: P = infinity, P[s] = s
        const int rw = rint >> 5;
        for (int64_t w = (int64_t)blockIdx.x * nthr + tid; w < p.bitmap_words; w += stride) {
            const uint32_t b0 = (w == rw) ? (1u << (rint & 31)) : 0u;
            p.bitmap[w] = b0;
            if (KM == KM_RESTORE) p.vo[w] = make_uint2(b0, 0u);
        }
        if (blockIdx.x == 0) {
            if (p.stats)
                for (int i = tid; i < 4 * kMaxStatLayers; i += (int)nthr) p.stats[i] = 0;
            if (tid == 0) {
                const int rb = p.ro[rint], len = p.ro[rint + 1] - rb;
                c->eu_count[0] = 0;
                c->hub_count[0] = 0;
                c->nf[0] = 1;
                c->mf[0] = (unsigned long long)len;
                if (len >= 1 && len <= W) {
                    p.eu[0][0] = rint;
                    p.eb[0][0] = rb;
                    p.el[0][0] = len;
                    p.us[0][0] = 0;
                    p.uc[0][0] = 1;
                    c->eu_count[0] = (1ull << 32) | 1ull;
                } else if (len > W) {
                    const int nseg = (len + W - 1) / W;
                    for (int s = 0; s < nseg && (unsigned)s < p.hcap; ++s) {
                        p.hu[0][s] = rint;
                        p.hb[0][s] = rb + s * W;
                        p.hl[0][s] = min(W, len - s * W);
                    }
                    c->hub_count[0] = (unsigned)nseg;
                }
            }
        }
    }
}

// Leaving the kernel: the last CTA out returns the control block to zero.
__device__ __forceinline__ void td_exit(Ctrl *c)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned old = atomicAdd(&c->exit_count, 1u);
        if (old == gridDim.x - 1) {
            for (int j = 0; j < 3; ++j) {
                c->eu_count[j] = 0;
                c->hub_count[j] = 0;
                c->work[j] = 0;
                c->nf[j] = 0;
                c->mf[j] = 0;
            }
            c->bar_count = 0;
            c->exit_count = 0;
            __threadfence();
        }
    }
}

template <int WPB, int KM>
__global__ void __launch_bounds__(WPB * 32, (24 / WPB) > 0 ? (24 / WPB) : 1) td_warp_kernel(WParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem<WPB> &cs = *reinterpret_cast<CtaSmem<WPB> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WarpSmem &ws = cs.w[warp];
    const unsigned G = gridDim.x;
    const unsigned GW = G * WPB;
    const unsigned gw = blockIdx.x * WPB + warp;
    Ctrl *c = p.ctrl;
    const uint64_t t_start = globaltimer();

    const int rint = __ldg(p.perm + p.root);  // the root in internal numbering

    td_init<KM>(p, rint);
    bool ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
    td_root_outputs(p);

    bool bu_prev = false;               // mode 3: the previous layer ran bottom-up
    unsigned long long m_seen = 0;      // mode 3: summed degrees of the vertices reached
    for (int d = 0; ok; ++d) {
        const int set_in = d % 3, set_out = (d + 1) % 3, set_rst = (d + 2) % 3;
        const int qi = d & 1, qo = qi ^ 1;
        bool bu = false;
        if constexpr (KM == KM_HYBRID) {
            // direction of this layer, taken alike by every CTA from the
            // frontier's size nf and summed degrees mf
            if (tid == 0) {
                cs.hnf = ld_relaxed64(&c->nf[set_in]);
                cs.hmf = ld_relaxed64(&c->mf[set_in]);
            }
            __syncthreads();
            const unsigned long long nf = cs.hnf, mf = cs.hmf;
            if (nf == 0) {
                if (blockIdx.x == 0 && tid == 0) c->layers = (unsigned)d;
                break;
            }
            m_seen += mf;
            const unsigned long long m_u = (unsigned long long)p.m > m_seen ? (unsigned long long)p.m - m_seen : 0ull;
            if (p.bro && p.alpha > 0) {
                if (!bu_prev) bu = (double)mf * (double)p.alpha > (double)m_u;
                else bu = (double)nf * (double)p.beta >= (double)p.n;
            }
            if (blockIdx.x == 0 && tid == 0) {
                c->eu_count[set_rst] = 0;
                c->hub_count[set_rst] = 0;
                c->nf[set_rst] = 0;
                c->mf[set_rst] = 0;
                if (p.stats && d < kMaxStatLayers) p.stats[4 * d + 0] = (int64_t)nf;
            }
            if (bu && !bu_prev) {  // the frontier queue as a bitmap
                const int64_t stride = (int64_t)G * WPB * 32;
                for (int64_t w = (int64_t)blockIdx.x * WPB * 32 + tid; w < p.bitmap_words; w += stride)
                    p.front[qi][w] = 0u;
                ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
                if (!ok) break;
                if (tid == 0) {
                    cs.nE = min((unsigned)(ld_relaxed64(&c->eu_count[set_in]) & 0xffffffffull), p.ecap);
                    cs.nH = min(ld_relaxed(&c->hub_count[set_in]), p.hcap);
                }
                __syncthreads();
                queue_to_bitmap(p, qi, cs.nE, cs.nH, p.front[qi]);
                ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
                if (!ok) break;
            } else if (!bu && bu_prev) {  // the frontier bitmap as a queue
                bitmap_to_queue(ws, p, p.front[qi], set_in, qi, gw, GW);
                ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
                if (!ok) break;
            }
        }
        const int next_level = d + 1;
        unsigned long long my_new = 0;
        unsigned long long my_vertices = 0, my_edges = 0;
        if (bu) {
            unsigned long long my_mf = 0;
            if (tid == 0 && p.stats) cs.st[0] = cs.st[1] = cs.st[2] = 0;
            bottom_up<WPB>(cs, p, p.front[qi], p.front[qo], next_level, gw, GW, my_new, my_edges, my_mf);
            unsigned long long a = my_new, b = my_mf;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(FULL, a, o);
                b += __shfl_down_sync(FULL, b, o);
            }
            if (lane == 0 && a) {
                atomicAdd(&c->nf[set_out], a);
                atomicAdd(&c->mf[set_out], b);
            }
        } else {
        if (tid == 0) {
            const unsigned long long eu = ld_relaxed64(&c->eu_count[set_in]);
            cs.nU = min((unsigned)(eu >> 32), p.ucap);
            cs.nH = min(ld_relaxed(&c->hub_count[set_in]), p.hcap);
            if (p.stats) cs.st[0] = cs.st[1] = cs.st[2] = 0;
        }
        __syncthreads();
        const unsigned nH0 = cs.nH;
        // few items: hub slices are dealt in up to 12 parts so that more warps share them
        const unsigned split = (cs.nU + nH0 > 0 && cs.nU + nH0 < GW / 2) ? min(12u, GW / (cs.nU + nH0)) : 1u;
        const unsigned nH = nH0, n_items = cs.nU + nH0 * split;
        if (KM != KM_HYBRID) {
            if (n_items == 0) {
                if (blockIdx.x == 0 && tid == 0) c->layers = (unsigned)d;
                break;
            }
            if (blockIdx.x == 0 && tid == 0) {
                c->eu_count[set_rst] = 0;
                c->hub_count[set_rst] = 0;
            }
        }
        int ocnt = 0, nb = 0;  // winners to flush; deferred candidates
        unsigned td_new = 0;

        // software pipeline over this warp's items gw, gw+GW, ...
        unsigned id = gw;
        Desc d0 = load_desc(p, qi, nH, n_items, id, split);
        Item cur = load_item(p, qi, d0, id < n_items, split);
        int buf = 0;
        int et_cur = (id < n_items) ? stage_item(ws, p, cur, buf, rint) : 0;
        int cnt_cur = cur.cnt;
        if (KM != KM_HYBRID && p.stats && id < n_items && lane == 0)
            my_vertices += (d0.c < 0) ? (cur.b == __ldg(p.ro + cur.u) ? 1 : 0) : (unsigned)cur.cnt;
        Desc d1 = load_desc(p, qi, nH, n_items, id + GW, split);
        Item nxt = load_item(p, qi, d1, id + GW < n_items, split);
        Desc d2 = load_desc(p, qi, nH, n_items, id + 2 * GW, split);
        while (id < n_items) {
            const unsigned id1 = id + GW, id2 = id + 2 * GW;
            int et_nxt = 0;
            if (id1 < n_items) {
                et_nxt = stage_item(ws, p, nxt, buf ^ 1, rint);
                if (KM != KM_HYBRID && p.stats && lane == 0)
                    my_vertices += (d1.c < 0) ? (nxt.b == __ldg(p.ro + nxt.u) ? 1 : 0) : (unsigned)nxt.cnt;
            } else {
                cp_async_commit();  // keep one group per item on every lane
            }
            const int cnt_nxt = nxt.cnt;
            const Item nn = load_item(p, qi, d2, id2 < n_items, split);
            const Desc d3 = load_desc(p, qi, nH, n_items, id2 + GW, split);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncwarp();
            if (lane == 0) my_edges += (unsigned long long)et_cur;
            if constexpr (KM == KM_RESTORE)
                process_item_rst(ws, p, buf, et_cur, cnt_cur);
            else
                process_item_def<KM>(ws, p, buf, et_cur, cnt_cur, rint, next_level, set_out, qo, ocnt, nb, td_new);
            buf ^= 1;
            id = id1;
            et_cur = et_nxt;
            cnt_cur = cnt_nxt;
            d1 = d2;
            nxt = nn;
            d2 = d3;
        }
        cp_async_wait_all();
        __syncwarp();
        if constexpr (KM != KM_RESTORE)
            if (nb > 0) claim_deferred<KM>(ws, p, nb, set_out, qo, ocnt, next_level, td_new);
        if (ocnt > 0) warp_flush<KM == KM_HYBRID ? (FL_LP | FL_CNT) : FL_LP>(ws, p, set_out, qo, ocnt, next_level);

        if (KM == KM_RESTORE) {
            // restoration (Alg. 3), once every racy set of the layer is done:
            // each non-zero out word is owned by one warp, which restores the
            // vertices of its bits with P < 0, sets their visited bits, clears
            // the word and queues them as the next frontier
            ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
            if (!ok) break;
            const unsigned lt = lanemask_lt();
            const int64_t nwords = p.bitmap_words;
            // words are dealt round-robin to the warps (word gw + GW * j), so
            // the dense low words of the degree order are spread over all of them
            for (int64_t j0 = 0; (int64_t)gw + GW * j0 < nwords; j0 += 32) {
                const int64_t wi = (int64_t)gw + GW * (j0 + lane);
                const uint2 x = wi < nwords ? __ldcg(p.vo + wi) : make_uint2(0u, 0u);
                unsigned nz = __ballot_sync(FULL, x.y != 0u);
                while (nz) {
                    const int src = __ffs(nz) - 1;
                    nz &= nz - 1;
                    if (ocnt > OBW - 32) {
                        warp_flush<FL_LP>(ws, p, set_out, qo, ocnt, next_level);
                        ocnt = 0;
                    }
                    const int64_t word = (int64_t)gw + GW * (j0 + src);
                    const int64_t v = word * 32 + lane;
                    const int pv = v < p.n ? __ldcg(p.pint + v) : 0;
                    const bool neg = pv < 0;
                    const unsigned m = __ballot_sync(FULL, neg);
                    if (neg) {
                        const int u = pv + p.n;
                        p.pint[v] = u;
                        const int pos = ocnt + __popc(m & lt);
                        ws.wv[pos] = (int)v;
                        ws.wu[pos] = u;
                    }
                    if (lane == src) {  // the lane that read the pair owns the word
                        p.vo[word] = make_uint2(x.x | m, 0u);
                        p.bitmap[word] = x.x | m;  // the plain visited bitmap, for export
                    }
                    ocnt += __popc(m);
                    if (lane == 0) td_new += (unsigned)__popc(m);
                }
            }
            if (ocnt > 0) warp_flush<FL_LP>(ws, p, set_out, qo, ocnt, next_level);
            ocnt = 0;
        }
        my_new = td_new;
        }  // top-down layer

        if (p.stats && d < kMaxStatLayers) {
            unsigned long long a = my_vertices, e = my_edges, t = my_new;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(FULL, a, o);
                e += __shfl_down_sync(FULL, e, o);
                t += __shfl_down_sync(FULL, t, o);
            }
            if (lane == 0) {
                atomicAdd(&cs.st[0], a);
                atomicAdd(&cs.st[1], e);
                atomicAdd(&cs.st[2], t);
            }
            __syncthreads();
            if (tid == 0) {
                atomicAdd((unsigned long long *)&p.stats[4 * d + 0], cs.st[0]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 1], cs.st[1]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 2], cs.st[2]);
            }
        }
        ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
        if (p.stats && d < kMaxStatLayers && blockIdx.x == 0 && tid == 0)
            p.stats[4 * d + 3] = (int64_t)(globaltimer() - t_start);
        bu_prev = bu;
    }

    td_exit(c);
}

// ---- mode 0: thin warps --------------------------------------------------
//
// The same layer step with more, lighter warps (8 per CTA, 4 CTAs per SM,
// at most 64 registers) and no staging: a warp reads its item's adjacency
// straight from global memory, 32 consecutive entries of the flattened lists
// per step (lane -> list by two ballots, as in the staging copy), TU steps
// in flight, bypassing L1; tests the visited words through L1 (which keeps
// about 180 KB for them, the shared memory per warp being only the winners'
// flush buffer); claims each candidate at once with atomicOr; and queues the
// winners, whose sources come from the same lane -> list mapping.

constexpr int TOB = 64;  // winners buffered per warp before a flush
constexpr int TU = 4;    // 32-entry steps in flight per warp

struct ThinWarpSmem {
    int32_t wv[TOB], wu[TOB];             // claimed vertices and their sources (internal ids)
    int32_t ou[TOB], ob[TOB], ol[TOB];    // flush: the new frontier entries
    int32_t ust[TOB];                     // flush: unit starts
};

template <int WPB>
struct ThinCtaSmem {
    ThinWarpSmem w[WPB];
    int ok;
    unsigned nU, nH;
    unsigned long long st[3];
};

// Adjacency entry read once: not kept in L1, which holds visited words.
__device__ __forceinline__ int ld_col(const int32_t *q)
{
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(q));
    return v;
}

// One work item: every entry of its lists tested, candidates claimed at
// once, the winners queued (flushed whenever the buffer could overflow).
__device__ __forceinline__ void thin_item(ThinWarpSmem &ws, const WParams &p, const Item &it_in, int set_out, int qo,
                                          int next_level, int &ocnt, unsigned &my_new, unsigned long long &my_edges)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    Item it = it_in;
    if (it.l < 0 || it.l > MAXI) {  // cannot happen for entries this kernel wrote
        atomicOr(&p.ctrl->status, ST_OVERFLOW);
        it.l = 0;
    }
    const bool has = lane < it.cnt && it.l > 0;
    int inc = has ? it.l : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    int et = __shfl_sync(FULL, inc, 31);
    if (et >= MAXI) {  // cannot happen: units < 2W edges, slices <= W
        if (lane == 0) atomicOr(&p.ctrl->status, ST_OVERFLOW);
        et = 0;
    }
    const int off = inc - (has ? it.l : 0);
    if (lane == 0) my_edges += (unsigned long long)et;
    const bool single = it.cnt == 1;  // a hub slice or a one-list unit
    const int b1 = __shfl_sync(FULL, it.b, 0), u1 = __shfl_sync(FULL, it.u, 0);
    for (int g0 = 0; g0 < et; g0 += 32 * TU) {
        int v[TU], u[TU];
#pragma unroll
        for (int s = 0; s < TU; ++s) {
            const int e0 = g0 + 32 * s, e = e0 + lane;
            int jb = b1, jo = 0;
            u[s] = u1;
            if (!single) {  // lane -> the last list starting at or before e
                const unsigned starts =
                    __reduce_or_sync(FULL, (has && off > e0 && off < e0 + 32) ? 1u << (off - e0) : 0u);
                const int j0 = __popc(__ballot_sync(FULL, has && off <= e0)) - 1;
                const int jj = (j0 + __popc(starts & ((2u << lane) - 1u))) & 31;
                jb = __shfl_sync(FULL, it.b, jj);
                jo = __shfl_sync(FULL, off, jj);
                u[s] = __shfl_sync(FULL, it.u, jj);
            }
            v[s] = e < et ? ld_col(p.col + GB_IX(jb + (e - jo), p.m, BS_COL, p.ctrl)) : -1;
        }
        unsigned w[TU];
#pragma unroll
        for (int s = 0; s < TU; ++s)
            w[s] = v[s] >= 0 ? __ldca(p.bitmap + GB_IX((unsigned)v[s] >> 5, p.bitmap_words, BS_VISITED, p.ctrl)) : 0xffffffffu;
        bool win[TU];
#pragma unroll
        for (int s = 0; s < TU; ++s) {
            win[s] = false;
            if (v[s] >= 0 && !((w[s] >> (v[s] & 31)) & 1u)) {
                const unsigned bit = 1u << (v[s] & 31);
                win[s] = !(atomicOr(p.bitmap + GB_IX((unsigned)v[s] >> 5, p.bitmap_words, BS_VISITED, p.ctrl), bit) & bit);
            }
        }
#pragma unroll
        for (int s = 0; s < TU; ++s) {
            const unsigned m = __ballot_sync(FULL, win[s]);
            if (!m) continue;
            if (ocnt + __popc(m) > TOB) {
                warp_flush<FL_LP, ThinWarpSmem, TOB>(ws, p, set_out, qo, ocnt, next_level);
                ocnt = 0;
            }
            if (win[s]) {
                const int pos = ocnt + __popc(m & lt);
                ws.wv[pos] = v[s];
                ws.wu[pos] = u[s];
                ++my_new;
            }
            ocnt += __popc(m);
        }
    }
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32, 32 / WPB) td_thin_kernel(WParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ThinCtaSmem<WPB> &cs = *reinterpret_cast<ThinCtaSmem<WPB> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    ThinWarpSmem &ws = cs.w[warp];
    const unsigned G = gridDim.x;
    const unsigned GW = G * WPB;
    const unsigned gw = blockIdx.x * WPB + warp;
    Ctrl *c = p.ctrl;
    const uint64_t t_start = globaltimer();
    const int rint = __ldg(p.perm + p.root);
    td_init<KM_ATOMIC>(p, rint);
    bool ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
    td_root_outputs(p);
    for (int d = 0; ok; ++d) {
        const int set_in = d % 3, set_out = (d + 1) % 3, set_rst = (d + 2) % 3;
        const int qi = d & 1, qo = qi ^ 1;
        if (tid == 0) {
            const unsigned long long eu = ld_relaxed64(&c->eu_count[set_in]);
            cs.nU = min((unsigned)(eu >> 32), p.ucap);
            cs.nH = min(ld_relaxed(&c->hub_count[set_in]), p.hcap);
            if (p.stats) cs.st[0] = cs.st[1] = cs.st[2] = 0;
        }
        __syncthreads();
        const unsigned nH = cs.nH;
        // few items: hub slices are dealt in up to 12 parts so that more warps share them
        const unsigned split = (cs.nU + nH > 0 && cs.nU + nH < GW / 2) ? min(12u, GW / (cs.nU + nH)) : 1u;
        const unsigned n_items = cs.nU + nH * split;
        if (n_items == 0) {
            if (blockIdx.x == 0 && tid == 0) c->layers = (unsigned)d;
            break;
        }
        if (blockIdx.x == 0 && tid == 0) {
            c->eu_count[set_rst] = 0;
            c->hub_count[set_rst] = 0;
        }
        const int next_level = d + 1;
        int ocnt = 0;
        unsigned my_new = 0;
        unsigned long long my_vertices = 0, my_edges = 0;
        // items gw, gw + GW, ...; the next item's descriptor and entries in flight
        unsigned id = gw;
        Desc d0 = load_desc(p, qi, nH, n_items, id, split);
        Item cur = load_item(p, qi, d0, id < n_items, split);
        Desc d1 = load_desc(p, qi, nH, n_items, id + GW, split);
        while (id < n_items) {
            const Item nxt = load_item(p, qi, d1, id + GW < n_items, split);
            const Desc d2 = load_desc(p, qi, nH, n_items, id + 2 * GW, split);
            if (p.stats && lane == 0)
                my_vertices += (d0.c < 0) ? (cur.b == __ldg(p.ro + cur.u) ? 1 : 0) : (unsigned)cur.cnt;
            thin_item(ws, p, cur, set_out, qo, next_level, ocnt, my_new, my_edges);
            id += GW;
            cur = nxt;
            d0 = d1;
            d1 = d2;
        }
        if (ocnt > 0) warp_flush<FL_LP, ThinWarpSmem, TOB>(ws, p, set_out, qo, ocnt, next_level);
        if (p.stats && d < kMaxStatLayers) {
            unsigned long long a = my_vertices, e = my_edges, t = my_new;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(FULL, a, o);
                e += __shfl_down_sync(FULL, e, o);
                t += __shfl_down_sync(FULL, t, o);
            }
            if (lane == 0) {
                atomicAdd(&cs.st[0], a);
                atomicAdd(&cs.st[1], e);
                atomicAdd(&cs.st[2], t);
            }
            __syncthreads();
            if (tid == 0) {
                atomicAdd((unsigned long long *)&p.stats[4 * d + 0], cs.st[0]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 1], cs.st[1]);
                atomicAdd((unsigned long long *)&p.stats[4 * d + 2], cs.st[2]);
            }
        }
        ok = grid_sync(&c->bar_count, &c->bar_gen, &c->status, G, p.timeout_ns, &cs.ok);
        if (p.stats && d < kMaxStatLayers && blockIdx.x == 0 && tid == 0)
            p.stats[4 * d + 3] = (int64_t)(globaltimer() - t_start);
    }
    td_exit(c);
}

template <int WPB>
int launch_thin(Graph *g, const WParams &prm, cudaStream_t s)
{
    auto kern = td_thin_kernel<WPB>;
    const int smem = (int)sizeof(ThinCtaSmem<WPB>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(td_thin_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(td_thin_kernel)");
    if (per_sm < 1) return set_error(BFS_ERR_CUDA, "td_thin_kernel: no CTA fits on an SM");
    per_sm = std::min(per_sm, 32 / WPB);  // up to 32 warps per SM
    if (g->opt.ctas_per_sm > 0) per_sm = std::min(per_sm, g->opt.ctas_per_sm);
    int grid = per_sm * g->num_sms;
    if (g->opt.max_ctas > 0) grid = std::min(grid, g->opt.max_ctas);
    WParams p = prm;
    void *args[] = {&p};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(WPB * 32), args, (size_t)smem, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(td_thin_kernel)");
    g->last_grid = grid;
    return BFS_OK;
}

template <int WPB, int KM>
int launch(Graph *g, const WParams &prm, cudaStream_t s)
{
    auto kern = td_warp_kernel<WPB, KM>;
    const int smem = (int)sizeof(CtaSmem<WPB>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(td_warp_kernel)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(td_warp_kernel)");
    if (per_sm < 1) return set_error(BFS_ERR_CUDA, "td_warp_kernel: no CTA fits on an SM");
    if (g->opt.ctas_per_sm > 0) per_sm = std::min(per_sm, g->opt.ctas_per_sm);
    int grid = per_sm * g->num_sms;
    if (g->opt.max_ctas > 0) grid = std::min(grid, g->opt.max_ctas);
    WParams p = prm;
    void *args[] = {&p};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(WPB * 32), args, (size_t)smem, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(td_warp_kernel)");
    g->last_grid = grid;
    return BFS_OK;
}

}  // namespace

// Hub slices of one layer: a vertex of degree d > W gives ceil(d/W) <= 2d/W
// slices, so a layer has at most 2m/W of them (+2).
int64_t td_hub_capacity(int64_t m) { return 2 * (m / W) + 2; }

int td_warp_launch(Graph *g, int32_t root, int32_t *level, int32_t *parent, cudaStream_t s, int mode)
{
    const bool restore = mode == MODE_RESTORE, hybrid = mode == MODE_HYBRID;
    if (restore && (!g->d_vo || !g->d_pint))
        return set_error(BFS_ERR_INVALID_ARG, "mode 2: restoration workspace not allocated");
    if (hybrid && (!g->d_front[0] || !g->d_front[1]))
        return set_error(BFS_ERR_INVALID_ARG, "mode 3: frontier bitmaps not allocated");
    WParams p;
    p.ro = g->d_row_offsets;
    p.col = g->d_col_idx;
    p.level = level;
    p.parent = parent;
    p.perm = g->d_perm;
    p.orig = g->d_orig;
    p.bitmap = g->d_bitmap;
    p.vo = restore ? g->d_vo : nullptr;
    p.front[0] = hybrid ? g->d_front[0] : nullptr;
    p.front[1] = hybrid ? g->d_front[1] : nullptr;
    p.m = g->m;
    p.n_nonzero = (int32_t)g->n_nonzero;
    p.alpha = g->opt.alpha;
    p.beta = g->opt.beta;
    p.bro = hybrid ? (g->symmetric ? g->d_row_offsets : g->d_tro) : nullptr;
    p.bcol = hybrid ? (g->symmetric ? g->d_col_idx : g->d_tcol) : nullptr;
    if (!p.bcol) p.bro = nullptr;
    p.bu_n = (int32_t)(g->symmetric ? g->n_nonzero : g->n);
    p.pint = restore ? g->d_pint : nullptr;
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
    if (mode == MODE_THIN) return launch_thin<8>(g, p, s);
    switch (g->opt.block) {
    case 256:
        return restore ? launch<8, KM_RESTORE>(g, p, s)
                       : hybrid ? launch<8, KM_HYBRID>(g, p, s) : launch<8, KM_ATOMIC>(g, p, s);
    case 512:
        return restore ? launch<16, KM_RESTORE>(g, p, s)
                       : hybrid ? launch<16, KM_HYBRID>(g, p, s) : launch<16, KM_ATOMIC>(g, p, s);
    default: return set_error(BFS_ERR_INVALID_ARG, "warp mode supports BLOCK 256 or 512");
    }
}

}  // namespace gbbfs
