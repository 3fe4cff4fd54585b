/*
 * oracle.c -- the correctness oracle for the BFS library.  TEST
 * INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
 * baseline call it; the library never does.  It shares no code, header or
 * constant with the CUDA path.
 *
 * Plain, single-threaded, obviously-correct C.  Every function names the
 * passage of the paper (Paredes, Riley, Lujan, "Breadth First Search
 * Vectorization on the Intel Xeon Phi") it follows.
 *
 * Conventions fixed for the whole library (readings of the paper):
 *   - "infinity" for an unreached predecessor (Sec. 3.1) is stored as -1; an
 *     unreached vertex also has level -1;
 *   - the source is its own predecessor, P[s] = s, with level 0 (Alg. 1);
 *   - the CSR is read as directed out-adjacency: Adj[u] =
 *     col_idx[row_offsets[u] .. row_offsets[u+1]-1] (Sec. 3.3.1, "rows" and
 *     "colstarts").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int oracle_version(void) { return 1; }

/*
 * Queue-based serial BFS (Sec. 3: one FIFO of vertices waiting to be
 * processed, O(V+E)), with the initialisation of Alg. 1: every P[u] starts at
 * "infinity", P[s] = s, s is marked visited and queued.  A vertex v found in
 * Adj[u] while unvisited gets level[u] + 1 and P[v] = u, and is queued.
 * level[v] is therefore the number of edges on a shortest path from s
 * (Sec. 3, footnote on distance).
 * Returns the number of reached vertices, or -1 on a bad argument.
 */
int64_t oracle_bfs(const int32_t *row_offsets, const int32_t *col_idx, int64_t n,
                   int32_t root, int32_t *level, int32_t *parent)
{
    if (n <= 0 || root < 0 || root >= n) return -1;
    for (int64_t v = 0; v < n; ++v) {
        level[v] = -1;
        if (parent) parent[v] = -1;
    }
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -1;
    int64_t head = 0, tail = 0;
    level[root] = 0;
    if (parent) parent[root] = root;
    queue[tail++] = root;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            int32_t v = col_idx[e];
            if (level[v] == -1) {
                level[v] = level[u] + 1;
                if (parent) parent[v] = u;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return tail;
}

/*
 * Batched form: the same BFS once per source, levels stored as uint8 in a
 * source-major [k][n] array with 0xFF for "unreached".  Returns 0, -1 on a
 * bad argument, -5 if some level exceeds 254 (it would not fit the uint8
 * encoding).
 */
int oracle_bfs_batch(const int32_t *row_offsets, const int32_t *col_idx, int64_t n,
                     const int32_t *roots, int32_t k, uint8_t *level_out)
{
    int32_t *lv = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!lv) return -1;
    int rc = 0;
    for (int32_t i = 0; i < k; ++i) {
        if (oracle_bfs(row_offsets, col_idx, n, roots[i], lv, NULL) < 0) { rc = -1; break; }
        uint8_t *row = level_out + (size_t)i * (size_t)n;
        for (int64_t v = 0; v < n; ++v) {
            if (lv[v] < 0) row[v] = 0xFF;
            else if (lv[v] > 254) { rc = -5; row[v] = 0xFF; }
            else row[v] = (uint8_t)lv[v];
        }
    }
    free(lv);
    return rc;
}

/*
 * Per-layer profile of one BFS, the columns of Table 1: for each layer d the
 * number of vertices in the layer ("Vertices"), the number of adjacency
 * entries scanned from them ("Edges") and the number of vertices first
 * reached from them ("Traversed vertices").  Computed from a finished level
 * array.  Arrays must hold max_layers entries.  Returns the number of layers,
 * or -1 if there are more than max_layers.
 */
int64_t oracle_layer_profile(const int32_t *row_offsets, int64_t n, const int32_t *level,
                             int64_t max_layers, int64_t *vertices, int64_t *edges,
                             int64_t *traversed)
{
    int64_t layers = 0;
    for (int64_t d = 0; d < max_layers; ++d) vertices[d] = edges[d] = traversed[d] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int32_t d = level[v];
        if (d < 0) continue;
        if (d >= max_layers) return -1;
        vertices[d] += 1;
        edges[d] += row_offsets[v + 1] - row_offsets[v];
        if (d > 0) traversed[d - 1] += 1;
        if (d + 1 > layers) layers = d + 1;
    }
    return layers;
}

/*
 * Validation of a BFS result, the "soft" check of Sec. 5.3 (Graph500 style).
 * The paper names five checks without listing them; the rules used here:
 *   1. parent[root] == root and level[root] == 0;
 *   2. every other vertex with a parent is reached through an existing edge
 *      (parent[v], v) of the CSR, and a vertex has a parent iff it has a level;
 *   3. level[parent[v]] == level[v] - 1 (this also excludes cycles);
 *   4. for every edge (u, v) with u reached: v is reached and
 *      level[v] <= level[u] + 1 (on a symmetric graph: |level[u]-level[v]| <= 1);
 *   5. the reached set equals that of ref_level (the oracle's), when given.
 * Rules 1-4 together force level[] to equal the hop distance from root.
 * Returns 0 if all hold, else the number of the first rule broken; the
 * offending vertex goes to *bad_vertex.
 */
int oracle_validate(const int32_t *row_offsets, const int32_t *col_idx, int64_t n,
                    int32_t root, const int32_t *level, const int32_t *parent,
                    const int32_t *ref_level, int64_t *bad_vertex)
{
    int64_t dummy;
    if (!bad_vertex) bad_vertex = &dummy;
    *bad_vertex = -1;
    if (root < 0 || root >= n) return 1;
    if (parent[root] != root || level[root] != 0) { *bad_vertex = root; return 1; }

    /* rule 2a: the parent, if any, is a vertex; parent and level agree on reach */
    for (int64_t v = 0; v < n; ++v) {
        int32_t p = parent[v];
        if ((p >= 0) != (level[v] >= 0) || p < -1 || p >= n) { *bad_vertex = v; return 2; }
    }
    /* rule 2b: edge (parent[v], v) exists; found by scanning each row once */
    uint8_t *found = (uint8_t *)calloc((size_t)n, 1);
    if (!found) return -1;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            int32_t v = col_idx[e];
            if (parent[v] == u) found[v] = 1;
        }
    for (int64_t v = 0; v < n; ++v)
        if (v != root && parent[v] >= 0 && !found[v]) { free(found); *bad_vertex = v; return 2; }
    free(found);

    /* rule 3: parent one layer up */
    for (int64_t v = 0; v < n; ++v)
        if (v != root && parent[v] >= 0 && level[parent[v]] != level[v] - 1) {
            *bad_vertex = v;
            return 3;
        }

    /* rule 4: no edge out of a reached vertex skips a layer or leaves the tree */
    for (int64_t u = 0; u < n; ++u) {
        if (level[u] < 0) continue;
        for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            int32_t v = col_idx[e];
            if (level[v] < 0 || level[v] > level[u] + 1) { *bad_vertex = v; return 4; }
        }
    }

    /* rule 5: same reached set as the reference */
    if (ref_level)
        for (int64_t v = 0; v < n; ++v)
            if ((level[v] >= 0) != (ref_level[v] >= 0)) { *bad_vertex = v; return 5; }
    return 0;
}
