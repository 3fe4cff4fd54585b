// server.cu -- continuous-batching request loop (filled in by the serving work).
#include "internal.cuh"

using namespace gbbfs;

extern "C" {
bfs_server *bfs_server_create(int64_t) { set_error(BFS_ERR_INVALID_ARG, "server not in this build yet"); return nullptr; }
int bfs_server_destroy(bfs_server *) { return BFS_OK; }
int bfs_server_add_graph(bfs_server *, bfs_graph *) { return set_error(BFS_ERR_INVALID_ARG, "server not in this build yet"); }
int bfs_submit(bfs_server *, int, int32_t, uint8_t *, uint64_t *) { return set_error(BFS_ERR_INVALID_ARG, "server not in this build yet"); }
int bfs_poll(bfs_server *, uint64_t) { return set_error(BFS_ERR_INVALID_ARG, "server not in this build yet"); }
int bfs_server_drain(bfs_server *) { return BFS_OK; }
int bfs_ticket_times(bfs_server *, uint64_t, int64_t *, int64_t *) { return set_error(BFS_ERR_INVALID_ARG, "server not in this build yet"); }
}
