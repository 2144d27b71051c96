/*
 * Oracle for all-pairs shortest paths -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct CPU code.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load this library; the
 * product path (the CUDA library) never does, and shares no code with it.
 *
 * Problem (Sec. 3.1 of Lund & Smith, "A Multi-Stage CUDA Kernel for
 * Floyd-Warshall"): G = (V, E) directed, w_ij the weight of edge (v_i, v_j),
 * w_ij = infinity when the edge is absent, w_ii = 0, real weights otherwise and
 * no negative cycle.  The answer d_ij is the length of a shortest path from v_i
 * to v_j; Fig. 1 computes it in place by the triple loop over k, i, j with
 * w_ij <- min(w_ij, w_ik + w_kj).
 *
 * Representation chosen here so that nothing depends on a sentinel value:
 *   - integers: int64 lengths plus a separate byte flag per entry
 *     (flag 1 = "infinity", the length is then ignored);
 *   - reals: IEEE double, +infinity for an absent edge (exact under + and min).
 * Matrices are row-major with leading dimension n.
 *
 * Besides Fig. 1 the file holds two textbook single-source algorithms that are
 * independent of it (Bellman-Ford, Dijkstra); the tests use them to pin the
 * Fig. 1 routines and, at sizes where Fig. 1 is too slow, to check sampled rows.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <omp.h>

/* Fig. 1 (Sec. 3.1), integer weights.  d[i*n+j] is the length, inf[i*n+j] = 1
 * marks "no path found yet".  Loop order k, i, j as printed; a candidate
 * w_ik + w_kj exists only when both terms are finite. */
void oracle_fw_i64(int64_t *d, uint8_t *inf, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            if (inf[i * n + k])
                continue;
            const int64_t dik = d[i * n + k];
            for (int64_t j = 0; j < n; ++j) {
                if (inf[k * n + j])
                    continue;
                const int64_t cand = dik + d[k * n + j];
                if (inf[i * n + j] || cand < d[i * n + j]) {
                    d[i * n + j] = cand;
                    inf[i * n + j] = 0;
                }
            }
        }
    }
}

/* Fig. 1 (Sec. 3.1), real weights in double precision. */
void oracle_fw_f64(double *d, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            const double dik = d[i * n + k];
            for (int64_t j = 0; j < n; ++j) {
                const double cand = dik + d[k * n + j];
                if (cand < d[i * n + j])
                    d[i * n + j] = cand;
            }
        }
    }
}

/* Fig. 1 on all host cores: the same k, i, j loop with the rows i of each
 * iteration k shared among `threads` threads (0 = every core).  Iteration k
 * reads row k and column k; with no negative cycle d_kk >= 0, so the
 * candidates d_kk + d_kj and d_ik + d_kk never improve them and they do not
 * change during iteration k.  Every thread therefore reads what the serial
 * loop reads, and the result equals the serial one bit for bit.  Returns the
 * number of threads used. */
int oracle_fw_i64_mt(int64_t *d, uint8_t *inf, int64_t n, int threads)
{
    if (threads <= 0)
        threads = omp_get_num_procs();
    for (int64_t k = 0; k < n; ++k) {
#pragma omp parallel for num_threads(threads) schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            if (inf[i * n + k])
                continue;
            const int64_t dik = d[i * n + k];
            for (int64_t j = 0; j < n; ++j) {
                if (inf[k * n + j])
                    continue;
                const int64_t cand = dik + d[k * n + j];
                if (inf[i * n + j] || cand < d[i * n + j]) {
                    d[i * n + j] = cand;
                    inf[i * n + j] = 0;
                }
            }
        }
    }
    return threads;
}

int oracle_fw_f64_mt(double *d, int64_t n, int threads)
{
    if (threads <= 0)
        threads = omp_get_num_procs();
    for (int64_t k = 0; k < n; ++k) {
#pragma omp parallel for num_threads(threads) schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const double dik = d[i * n + k];
            for (int64_t j = 0; j < n; ++j) {
                const double cand = dik + d[k * n + j];
                if (cand < d[i * n + j])
                    d[i * n + j] = cand;
            }
        }
    }
    return threads;
}

/* Bellman-Ford from one source over the dense edge list of w (textbook
 * algorithm, independent of Fig. 1).  Integer weights with absence flags.
 * Writes dist[j] / unreach[j] for every j.  Returns 1 if a negative cycle is
 * reachable from src, else 0. */
int oracle_bellman_ford_i64(const int64_t *w, const uint8_t *absent, int64_t n,
                            int64_t src, int64_t *dist, uint8_t *unreach)
{
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = 0;
        unreach[v] = 1;
    }
    dist[src] = 0;
    unreach[src] = 0;
    for (int64_t pass = 0; pass < n; ++pass) {
        int changed = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (unreach[u])
                continue;
            for (int64_t v = 0; v < n; ++v) {
                if (absent[u * n + v])
                    continue;
                const int64_t cand = dist[u] + w[u * n + v];
                if (unreach[v] || cand < dist[v]) {
                    dist[v] = cand;
                    unreach[v] = 0;
                    changed = 1;
                }
            }
        }
        if (!changed)
            return 0;
    }
    return 1; /* still relaxing after n passes */
}

/* Bellman-Ford from one source, double weights (+inf = absent). */
int oracle_bellman_ford_f64(const double *w, int64_t n, int64_t src, double *dist)
{
    for (int64_t v = 0; v < n; ++v)
        dist[v] = INFINITY;
    dist[src] = 0.0;
    for (int64_t pass = 0; pass < n; ++pass) {
        int changed = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (isinf(dist[u]))
                continue;
            for (int64_t v = 0; v < n; ++v) {
                const double cand = dist[u] + w[u * n + v];
                if (cand < dist[v]) {
                    dist[v] = cand;
                    changed = 1;
                }
            }
        }
        if (!changed)
            return 0;
    }
    return 1;
}

/* Dijkstra from one source on a dense graph (array scan, O(n^2)), for
 * non-negative weights only.  Reads the fp32 input matrix as stored (leading
 * dimension ld, +inf = absent) and widens each weight exactly to double. */
void oracle_dijkstra_f32in(const float *w, int64_t n, int64_t ld, int64_t src,
                           double *dist)
{
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    for (int64_t v = 0; v < n; ++v)
        dist[v] = INFINITY;
    dist[src] = 0.0;
    for (int64_t it = 0; it < n; ++it) {
        int64_t u = -1;
        double best = INFINITY;
        for (int64_t v = 0; v < n; ++v)
            if (!done[v] && dist[v] < best) {
                best = dist[v];
                u = v;
            }
        if (u < 0)
            break; /* the rest is unreachable */
        done[u] = 1;
        for (int64_t v = 0; v < n; ++v) {
            const double cand = dist[u] + (double)w[u * ld + v];
            if (cand < dist[v])
                dist[v] = cand;
        }
    }
    free(done);
}

/* Dijkstra from one source, int32 input matrix as stored (leading dimension
 * ld).  An entry equal to absent_value is a missing edge; all other weights
 * must be >= 0.  Writes int64 lengths and unreachable flags. */
void oracle_dijkstra_i32in(const int32_t *w, int64_t n, int64_t ld, int64_t src,
                           int32_t absent_value, int64_t *dist, uint8_t *unreach)
{
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = 0;
        unreach[v] = 1;
    }
    dist[src] = 0;
    unreach[src] = 0;
    for (int64_t it = 0; it < n; ++it) {
        int64_t u = -1;
        for (int64_t v = 0; v < n; ++v)
            if (!done[v] && !unreach[v] && (u < 0 || dist[v] < dist[u]))
                u = v;
        if (u < 0)
            break;
        done[u] = 1;
        for (int64_t v = 0; v < n; ++v) {
            const int32_t wuv = w[u * ld + v];
            if (wuv == absent_value)
                continue;
            const int64_t cand = dist[u] + (int64_t)wuv;
            if (unreach[v] || cand < dist[v]) {
                dist[v] = cand;
                unreach[v] = 0;
            }
        }
    }
    free(done);
}
