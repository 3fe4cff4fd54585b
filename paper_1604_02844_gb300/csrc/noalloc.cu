// noalloc.cu -- bfs_run_noalloc: a single-source search that allocates no
// memory at all.
//
// Some callers cannot allocate GPU memory when they search: code running
// under a memory manager that owns every byte of the device (a framework's
// caching allocator, a serving process with a fixed budget), callers on a
// latency-critical path that must not block in cudaMalloc / cudaFree, or
// code inside a region where the CUDA runtime forbids allocation.  For them
// this entry point runs the warp-pipeline top-down kernel (topdown_warp.cu)
// on the caller's own device CSR and output arrays, with every piece of
// scratch state -- visited bitmap, frontier entries, units and hub slices,
// the control block, identity id maps -- in one file-scope __device__ array
// of fixed size.  It calls no cudaMalloc, cudaFree or allocating library
// routine.
//
// Limits: n <= BFS_NOALLOC_MAX_VERTICES, m <= BFS_NOALLOC_MAX_EDGES (the
// array is sized for them, about 7 MB, and every GPU that loads the library
// holds it until the process exits).  The first call on a device sets the
// array up (its device address, the identity maps); make that first call
// before any stream capture.  The set-up is cached for the life of the
// process, so cudaDeviceReset on a device leaves a stale address behind:
// after a reset this entry point must not be called on that device until
// the library is reloaded.  All calls share the one array, which keeps
// the previous call's contents: the control block is returned to zero by
// the kernel itself at the end of every search and the bitmap and frontier
// are rewritten by each search, but two calls that overlap on the GPU (on
// different streams, or from different host threads) race on it.  Calls
// are serialised on the host by a mutex and each call waits for its search
// to finish before returning.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.cuh"

namespace gbbfs {
namespace {

constexpr int64_t kMaxN = BFS_NOALLOC_MAX_VERTICES;
constexpr int64_t kMaxM = BFS_NOALLOC_MAX_EDGES;
constexpr int64_t kBitmapWords = ((kMaxN + 31) / 32 + 3) / 4 * 4;
constexpr int64_t kHubCap = kMaxM / 128 + 2;  // >= td_hub_capacity(kMaxM) = 2 m / W + 2

// byte offsets inside the scratch array (each a multiple of 256)
constexpr int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }
constexpr int64_t OFF_CTRL = 0;
constexpr int64_t OFF_FLAGS = align256(OFF_CTRL + (int64_t)sizeof(Ctrl));
constexpr int64_t OFF_BITMAP = align256(OFF_FLAGS + 4);
constexpr int64_t OFF_PERM = align256(OFF_BITMAP + 4 * kBitmapWords);
constexpr int64_t OFF_ORIG = align256(OFF_PERM + 4 * kMaxN);
constexpr int64_t OFF_EQ = align256(OFF_ORIG + 4 * kMaxN);         // [2][3][kMaxN]
constexpr int64_t OFF_UQ = align256(OFF_EQ + 4 * 6 * kMaxN);       // [2][2][kMaxN]
constexpr int64_t OFF_HQ = align256(OFF_UQ + 4 * 4 * kMaxN);       // [2][3][kHubCap]
constexpr int64_t kScratchBytes = align256(OFF_HQ + 4 * 6 * kHubCap);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void identity_kernel(int32_t *perm, int32_t *orig, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        perm[i] = (int32_t)i;
        orig[i] = (int32_t)i;
    }
}

constexpr int kMaxDevices = 256;
std::mutex g_mu;
unsigned char *g_base[kMaxDevices] = {};  // device address of the array, per device

// Once per device, with that device current: the array's device address
// (the host-side symbol is only a stand-in and must not reach a kernel),
// the identity id maps and a zeroed control block.
int setup_device(int dev, unsigned char **base)
{
    if (dev < 0 || dev >= kMaxDevices) return set_error(BFS_ERR_INVALID_ARG, "bfs_run_noalloc: device index out of range");
    if (g_base[dev]) {
        *base = g_base[dev];
        return BFS_OK;
    }
    void *ptr = nullptr;
    GB_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    unsigned char *b = static_cast<unsigned char *>(ptr);
    int sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    identity_kernel<<<sms * 4, 256>>>(reinterpret_cast<int32_t *>(b + OFF_PERM), reinterpret_cast<int32_t *>(b + OFF_ORIG),
                                      kMaxN);
    GB_CUDA(cudaGetLastError());
    GB_CUDA(cudaMemset(b + OFF_CTRL, 0, sizeof(Ctrl)));
    GB_CUDA(cudaDeviceSynchronize());
    g_base[dev] = b;
    *base = b;
    return BFS_OK;
}

}  // namespace
}  // namespace gbbfs

using namespace gbbfs;

extern "C" int bfs_run_noalloc(const int32_t *row_offsets, const int32_t *col_idx, int64_t n, int64_t m, int32_t root,
                               int32_t *level_out, int32_t *parent_out, void *stream)
{
    const NvtxRange nvtx("bfs_run_noalloc");
    clear_error();
    if (n < 1 || n > kMaxN || m < 0 || m > kMaxM)
        return set_error(BFS_ERR_INVALID_ARG,
                         "bfs_run_noalloc: needs 1 <= n <= BFS_NOALLOC_MAX_VERTICES (131072) and 0 <= m <= "
                         "BFS_NOALLOC_MAX_EDGES (4194304); use bfs_graph_create + bfs_run for larger graphs");
    if (root < 0 || (int64_t)root >= n) return set_error(BFS_ERR_INVALID_ARG, "bfs_run_noalloc: root outside [0, n)");
    if (!is_device_pointer(row_offsets) || (m > 0 && !is_device_pointer(col_idx)) || !is_device_pointer(level_out) ||
        (parent_out && !is_device_pointer(parent_out)))
        return set_error(BFS_ERR_INVALID_ARG,
                         "bfs_run_noalloc: row_offsets, col_idx, level_out and parent_out must be device memory");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    unsigned char *b = nullptr;
    int rc = setup_device(dev, &b);
    if (rc != BFS_OK) return rc;

    // the caller's CSR is read as is: check it first (flag word in the array)
    unsigned *d_flags = reinterpret_cast<unsigned *>(b + OFF_FLAGS);
    GB_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(unsigned), s));
    int sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    validate_csr_kernel<<<sms * 4, 256, 0, s>>>(row_offsets, col_idx, n, m, d_flags);
    GB_CUDA(cudaGetLastError());
    unsigned flags = 0;
    GB_CUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (flags) return set_error(BFS_ERR_INVALID_GRAPH, "bfs_run_noalloc: invalid CSR");

    // a graph view over the caller's arrays and the static scratch
    Graph g;
    g.device = dev;
    g.num_sms = sms;
    g.n = n;
    g.m = m;
    g.d_row_offsets = const_cast<int32_t *>(row_offsets);
    g.d_col_idx = const_cast<int32_t *>(col_idx);
    g.d_perm = reinterpret_cast<int32_t *>(b + OFF_PERM);
    g.d_orig = reinterpret_cast<int32_t *>(b + OFF_ORIG);
    g.d_bitmap = reinterpret_cast<uint32_t *>(b + OFF_BITMAP);
    g.bitmap_words = ((n + 31) / 32 + 3) / 4 * 4;
    int32_t *eq = reinterpret_cast<int32_t *>(b + OFF_EQ);
    int32_t *uq = reinterpret_cast<int32_t *>(b + OFF_UQ);
    int32_t *hq = reinterpret_cast<int32_t *>(b + OFF_HQ);
    for (int bb = 0; bb < 2; ++bb) {
        for (int j = 0; j < 3; ++j) {
            g.d_eq[bb][j] = eq + (int64_t)(bb * 3 + j) * kMaxN;
            g.d_hq[bb][j] = hq + (int64_t)(bb * 3 + j) * kHubCap;
        }
        for (int j = 0; j < 2; ++j) g.d_uq[bb][j] = uq + (int64_t)(bb * 2 + j) * kMaxN;
    }
    g.hcap = kHubCap;
    g.d_ctrl = reinterpret_cast<Ctrl *>(b + OFF_CTRL);
    g.d_stats = nullptr;
    g.opt.layer_stats = 0;
    g.opt.block = 512;
    rc = td_warp_launch(&g, root, level_out, parent_out, s);
    if (rc != BFS_OK) return rc;
    GB_CUDA(cudaStreamSynchronize(s));
    unsigned st = 0;
    GB_CUDA(cudaMemcpy(&st, &g.d_ctrl->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st) {
        GB_CUDA(cudaMemset(&g.d_ctrl->status, 0, sizeof(unsigned)));
        if (st & ST_BOUNDS) {
            unsigned long long w = 0;
            GB_CUDA(cudaMemcpy(&w, &g.d_ctrl->bounds, sizeof(w), cudaMemcpyDeviceToHost));
            GB_CUDA(cudaMemset(&g.d_ctrl->bounds, 0, sizeof(w)));
            return set_error(BFS_ERR_CUDA, std::string("bfs_run_noalloc: index out of range in ") + bounds_site_name(w));
        }
        if (st & ST_TIMEOUT) return set_error(BFS_ERR_TIMEOUT, "bfs_run_noalloc: a device-side wait ran out");
        return set_error(BFS_ERR_CUDA, "bfs_run_noalloc: a frontier queue append ran past its capacity");
    }
    return BFS_OK;
}
