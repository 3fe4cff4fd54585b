// relabel.cu -- degree-ordered internal vertex numbering, built on the device
// when a graph is created.
//
// The search itself is unchanged by a renumbering of the vertices (levels
// are distances, the visited set is a set), so the library stores the graph
// under internal ids sorted by decreasing degree class:
//   class(v) = floor(log2(deg v)) for deg >= 1, highest class first,
//   vertices of degree 0 last, original order kept inside a class.
// High-degree vertices then share the first words of the visited bitmap.
// Those words are the targets of most adjacency entries (an edge end lands
// on v with probability proportional to deg v), so the test of the visited
// bit mostly hits a few kilobytes that stay in the SM's L1 instead of
// spreading over the whole bitmap in L2.
//
// Every result leaves the library in the caller's numbering: kernels write
// level[orig[v]] and parent[orig[v]] = orig[u]; the root is mapped with
// perm[root] on the device.
//
// Steps (all kernels; deterministic for any launch size):
//   1. class of every vertex, per-block class histograms (block = 1024 ids)
//   2. exclusive scan of the histograms in (class, block) order
//   3. stable scatter: perm[v] (old -> new), orig[new] = v
//   4. new degrees, exclusive scan -> internal row_offsets
//   5. rows copied to their new place with every column renumbered
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace gbbfs {
namespace {

constexpr int NCLS = 33;     // 32 degree classes + degree 0
constexpr int RB = 1024;     // vertices per relabel block
constexpr int SCAN_T = 1024; // threads of the single-block scans

__device__ __forceinline__ int degree_class(int deg)
{
    // highest degrees first: class 0 holds deg >= 2^30, class 31 deg == 1
    return deg <= 0 ? 32 : (__clz(deg) - 1);
}

__global__ void class_hist_kernel(const int32_t *__restrict__ ro, int64_t n, uint8_t *cls, int32_t *hist, int nblk)
{
    __shared__ int h[NCLS];
    for (int c = threadIdx.x; c < NCLS; c += blockDim.x) h[c] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * RB + threadIdx.x;
    if (v < n) {
        const int c = degree_class(ro[v + 1] - ro[v]);
        cls[v] = (uint8_t)c;
        atomicAdd(&h[c], 1);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NCLS; c += blockDim.x) hist[(int64_t)c * nblk + blockIdx.x] = h[c];
}

// Exclusive scan of `len` int64-safe counts in place, one block, in chunks.
__global__ void scan_single_block_kernel(int32_t *a, int64_t len, int64_t *total)
{
    __shared__ long long part[SCAN_T];
    const int t = threadIdx.x;
    const int64_t per = (len + SCAN_T - 1) / SCAN_T;
    const int64_t lo = t * per, hi = min(len, lo + per);
    long long s = 0;
    for (int64_t i = lo; i < hi; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long run = 0;
        for (int i = 0; i < SCAN_T; ++i) {
            const long long x = part[i];
            part[i] = run;
            run += x;
        }
        if (total) *total = run;
    }
    __syncthreads();
    long long run = part[t];
    for (int64_t i = lo; i < hi; ++i) {
        const long long x = a[i];
        a[i] = (int32_t)run;
        run += x;
    }
}

__global__ void scatter_kernel(const uint8_t *__restrict__ cls, int64_t n, const int32_t *__restrict__ hoff, int nblk,
                               int32_t *perm, int32_t *orig)
{
    __shared__ int wcount[RB / 32][NCLS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t v = (int64_t)blockIdx.x * RB + threadIdx.x;
    const int c = v < n ? cls[v] : -1;
    // rank inside the warp (stable) and per-warp class counts
    int rank = 0;
    for (int k = 0; k < NCLS; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, c == k);
        if (c == k) rank = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) wcount[warp][k] = __popc(m);
    }
    __syncthreads();
    // exclusive prefix over warps, per class (one thread per class)
    if (threadIdx.x < NCLS) {
        int run = 0;
        for (int w = 0; w < RB / 32; ++w) {
            const int x = wcount[w][threadIdx.x];
            wcount[w][threadIdx.x] = run;
            run += x;
        }
    }
    __syncthreads();
    if (v < n) {
        const int nid = hoff[(int64_t)c * nblk + blockIdx.x] + wcount[warp][c] + rank;
        perm[v] = nid;
        orig[nid] = (int32_t)v;
    }
}

__global__ void new_degree_kernel(const int32_t *__restrict__ ro, const int32_t *__restrict__ orig, int64_t n, int32_t *nro)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += stride) {
        const int32_t v = orig[w];
        nro[w] = ro[v + 1] - ro[v];
    }
}

// Block-level exclusive scan of nro[0..n) in tiles, with per-tile sums.
constexpr int TILE = 2048;

__global__ void tile_scan_kernel(int32_t *a, int64_t n, int32_t *tile_sum)
{
    __shared__ int32_t s[TILE];
    const int64_t base = (int64_t)blockIdx.x * TILE;
    for (int i = threadIdx.x; i < TILE; i += blockDim.x) s[i] = (base + i < n) ? a[base + i] : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int i = 0; i < TILE; ++i) {
            const int32_t x = s[i];
            s[i] = run;
            run += x;
        }
        tile_sum[blockIdx.x] = run;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TILE; i += blockDim.x)
        if (base + i < n) a[base + i] = s[i];
}

__global__ void tile_add_kernel(int32_t *a, int64_t n, const int32_t *__restrict__ tile_off, int64_t m)
{
    const int64_t base = (int64_t)blockIdx.x * TILE;
    const int32_t add = tile_off[blockIdx.x];
    for (int i = threadIdx.x; i < TILE; i += blockDim.x)
        if (base + i < n) a[base + i] += add;
    if (blockIdx.x == 0 && threadIdx.x == 0) a[n] = (int32_t)m;
}

// One warp per new row: copy and renumber.
__global__ void copy_rows_kernel(const int32_t *__restrict__ ro, const int32_t *__restrict__ col,
                                 const int32_t *__restrict__ orig, const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ nro, int64_t n, int32_t *ncol)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < n; w += nwarps) {
        const int32_t v = orig[w];
        const int32_t b = ro[v], len = ro[v + 1] - b;
        const int32_t nb = nro[w];
        for (int k = lane; k < len; k += 32) ncol[nb + k] = perm[col[b + k]];
    }
}

// flags bit 0: some row is not sorted; bit 1: some edge (u, v) has no (v, u).
// One warp per row u; the reverse edge is found by binary search in the
// sorted row of v (only meaningful when no row is unsorted).
__global__ void symmetry_kernel(const int32_t *__restrict__ ro, const int32_t *__restrict__ col, int64_t n,
                                unsigned *flags)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x / 32);
    unsigned f = 0;
    for (int64_t u = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); u < n; u += nwarps) {
        const int32_t b = ro[u], e = ro[u + 1];
        for (int32_t k = b + lane; k < e; k += 32) {
            const int32_t v = col[k];
            if (k > b && col[k - 1] > v) f |= 1u;
            int32_t lo = ro[v], hi = ro[v + 1];  // find u in Adj[v]
            while (lo < hi) {
                const int32_t mid = (lo + hi) >> 1;
                if (col[mid] < u) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= ro[v + 1] || col[lo] != u) f |= 2u;
        }
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if (f && lane == 0) atomicOr(flags, f);
}

__global__ void bitmap_to_caller_kernel(const uint32_t *__restrict__ bm, const int32_t *__restrict__ orig, int64_t n,
                                        uint32_t *out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += stride)
        if (bm[w >> 5] & (1u << (w & 31))) {
            const int32_t v = orig[w];
            atomicOr(&out[v >> 5], 1u << (v & 31));
        }
}

}  // namespace

// In-degree of every vertex (internal numbering), into tro[v].
__global__ void indeg_kernel(const int32_t *__restrict__ col, int64_t m, int32_t *tro)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(tro + col[e], 1);
}

// One warp per row u: every edge (u, v) lands in v's in-list.
__global__ void scatter_in_kernel(const int32_t *__restrict__ ro, const int32_t *__restrict__ col, int64_t n,
                                  int32_t *cursor, int32_t *tcol)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < n; u += nw)
        for (int k = ro[u] + lane; k < ro[u + 1]; k += 32) tcol[atomicAdd(cursor + col[k], 1)] = (int32_t)u;
}

// Build g->d_row_offsets / d_col_idx (internal numbering), g->d_perm and
// g->d_orig from a validated device CSR in the caller's numbering.
int relabel_graph(Graph *g, const int32_t *d_ro, const int32_t *d_col)
{
    const int64_t n = g->n, m = g->m;
    const int nblk = (int)((n + RB - 1) / RB);
    uint8_t *cls = nullptr;
    int32_t *hist = nullptr, *tsum = nullptr;
    const int64_t ntile = (n + TILE - 1) / TILE;
    int rc = BFS_OK;
    cudaError_t e;
    const int64_t col_alloc = ((m + 3) / 4) * 4 + 4;
    if ((e = cudaMalloc(&g->d_perm, (size_t)n * 4)) != cudaSuccess) return cuda_error(e, "cudaMalloc(perm)");
    if ((e = cudaMalloc(&g->d_orig, (size_t)n * 4)) != cudaSuccess) return cuda_error(e, "cudaMalloc(orig)");
    if ((e = cudaMalloc(&g->d_row_offsets, (size_t)(n + 1) * 4)) != cudaSuccess) return cuda_error(e, "cudaMalloc(row_offsets)");
    if ((e = cudaMalloc(&g->d_col_idx, (size_t)col_alloc * 4)) != cudaSuccess) return cuda_error(e, "cudaMalloc(col_idx)");
    if ((e = cudaMalloc(&cls, (size_t)n)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(cls)"); goto done; }
    if ((e = cudaMalloc(&hist, (size_t)NCLS * nblk * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(hist)"); goto done; }
    if ((e = cudaMalloc(&tsum, (size_t)(ntile + 1) * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(tile sums)"); goto done; }
    class_hist_kernel<<<nblk, RB>>>(d_ro, n, cls, hist, nblk);
    scan_single_block_kernel<<<1, SCAN_T>>>(hist, (int64_t)NCLS * nblk, nullptr);
    scatter_kernel<<<nblk, RB>>>(cls, n, hist, nblk, g->d_perm, g->d_orig);
    new_degree_kernel<<<g->num_sms * 8, 256>>>(d_ro, g->d_orig, n, g->d_row_offsets);
    tile_scan_kernel<<<(unsigned)ntile, 256>>>(g->d_row_offsets, n, tsum);
    scan_single_block_kernel<<<1, SCAN_T>>>(tsum, ntile, nullptr);
    tile_add_kernel<<<(unsigned)ntile, 256>>>(g->d_row_offsets, n, tsum, m);
    copy_rows_kernel<<<g->num_sms * 16, 256>>>(d_ro, d_col, g->d_orig, g->d_perm, g->d_row_offsets, n, g->d_col_idx);
    if ((e = cudaMemset(g->d_col_idx + m, 0, (size_t)(col_alloc - m) * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMemset(col tail)"); goto done; }
    // vertices of degree >= 32 (classes 0..26) come first: their count is
    // the exclusive offset of class 27, block 0
    {
        int32_t split = 0;
        if ((e = cudaMemcpy(&split, hist + (int64_t)27 * nblk, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) { rc = cuda_error(e, "cudaMemcpy(split)"); goto done; }
        g->split32 = split;
        int32_t nz = 0;  // vertices of degree >= 1: exclusive offset of class 32
        if ((e = cudaMemcpy(&nz, hist + (int64_t)32 * nblk, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) { rc = cuda_error(e, "cudaMemcpy(nonzero)"); goto done; }
        g->n_nonzero = nz;
    }
    // exact symmetry test on the caller's CSR (sorted rows + reverse edges)
    {
        unsigned *d_flags = reinterpret_cast<unsigned *>(tsum);  // scratch: tile sums are consumed
        if ((e = cudaMemset(d_flags, 0, 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMemset(symmetry)"); goto done; }
        symmetry_kernel<<<g->num_sms * 16, 256>>>(d_ro, d_col, n, d_flags);
        unsigned flags = 0;
        if ((e = cudaMemcpy(&flags, d_flags, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) { rc = cuda_error(e, "symmetry_kernel"); goto done; }
        g->symmetric = (flags == 0);
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { rc = cuda_error(e, "relabel kernels"); goto done; }
done:
    cudaFree(cls);
    cudaFree(hist);
    cudaFree(tsum);
    return rc;
}

// Visited bitmap of the last search in the caller's numbering (device out,
// ceil(n/32) words, cleared here).
int bitmap_to_caller(Graph *g, uint32_t *d_out)
{
    const int64_t words = (g->n + 31) / 32;
    cudaError_t e = cudaMemset(d_out, 0, (size_t)words * 4);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemset(bitmap out)");
    bitmap_to_caller_kernel<<<g->num_sms * 4, 256>>>(g->d_bitmap, g->d_orig, g->n, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "bitmap_to_caller_kernel");
    return BFS_OK;
}

}  // namespace gbbfs

namespace gbbfs {

// The transposed CSR (in-edges, internal numbering) for bottom-up layers on
// a graph that is not symmetric: in-degrees, their exclusive scan, then the
// edges scattered into the in-lists (list order is not defined).
int transpose_graph(Graph *g)
{
    const int64_t n = g->n, m = g->m;
    const int64_t ntile = (n + TILE - 1) / TILE;
    int32_t *cursor = nullptr, *tsum = nullptr;
    int rc = BFS_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&g->d_tro, (size_t)(n + 1) * 4)) != cudaSuccess) return cuda_error(e, "cudaMalloc(in-edge offsets)");
    if ((e = cudaMalloc(&g->d_tcol, (size_t)(((m + 3) / 4) * 4 + 4) * 4)) != cudaSuccess) return cuda_error(e, "cudaMalloc(in-edges)");
    if ((e = cudaMalloc(&cursor, (size_t)(n + 1) * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(cursor)"); goto done; }
    if ((e = cudaMalloc(&tsum, (size_t)(ntile + 1) * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(tile sums)"); goto done; }
    if ((e = cudaMemset(g->d_tro, 0, (size_t)(n + 1) * 4)) != cudaSuccess) { rc = cuda_error(e, "cudaMemset(in-degrees)"); goto done; }
    indeg_kernel<<<g->num_sms * 8, 256>>>(g->d_col_idx, m, g->d_tro);
    tile_scan_kernel<<<(unsigned)ntile, 256>>>(g->d_tro, n, tsum);
    scan_single_block_kernel<<<1, SCAN_T>>>(tsum, ntile, nullptr);
    tile_add_kernel<<<(unsigned)ntile, 256>>>(g->d_tro, n, tsum, m);
    if ((e = cudaMemcpy(cursor, g->d_tro, (size_t)(n + 1) * 4, cudaMemcpyDeviceToDevice)) != cudaSuccess) { rc = cuda_error(e, "cudaMemcpy(cursor)"); goto done; }
    scatter_in_kernel<<<g->num_sms * 16, 256>>>(g->d_row_offsets, g->d_col_idx, n, cursor, g->d_tcol);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) rc = cuda_error(e, "transpose_graph");
done:
    cudaFree(cursor);
    cudaFree(tsum);
    if (rc != BFS_OK) {
        cudaFree(g->d_tro);
        cudaFree(g->d_tcol);
        g->d_tro = g->d_tcol = nullptr;
    }
    return rc;
}

}  // namespace gbbfs
