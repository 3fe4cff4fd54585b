// msbfs.cu -- bit-parallel batched BFS (filled in by the batched-kernel work).
#include "internal.cuh"

namespace gbbfs {

int ms_run_batch(Graph *, const int32_t *, int32_t, uint8_t *)
{
    return set_error(BFS_ERR_INVALID_ARG, "bfs_run_batch: batched kernels are not in this build yet");
}

void ms_free(Graph *) {}

}  // namespace gbbfs
