/*
 * Seeded synthetic inputs shared by the CPU oracle and the CUDA path.
 *
 * This file holds no arithmetic of the graph-query method: it only draws
 * graphs (R-MAT and a road-like grid), edge weights and source vertices.
 * Every random number is counter based (a SplitMix64 finaliser applied to
 * (seed, stream, counter)), so the output is identical on every platform
 * and for every OpenMP thread count.
 *
 * The paper evaluates on real graphs (road networks and social/web graphs,
 * Sec. 6.1, Table 2); these generators are the synthetic stand-ins:
 *   - R-MAT (Chakrabarti et al.) for the power-law social graphs, with the
 *     vertex ids randomly permuted so that equal-size id ranges behave like
 *     the random equal-vertex partitions the paper uses for social graphs
 *     (Sec. 6.1, "Implementation Details");
 *   - a 2-D grid with dropped edges and sparse diagonal shortcuts for the
 *     road networks.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    /* SplitMix64 output function (Steele, Lea, Flood 2014). */
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Counter-based draw: a 64-bit value for (seed, stream, counter). */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return mix64(mix64(seed ^ mix64(stream)) + ctr);
}

/* Uniform integer in [0, bound) by the multiply-high method (Lemire 2019). */
static inline uint64_t bounded(uint64_t r, uint64_t bound) {
    return (uint64_t)(((__uint128_t)r * (__uint128_t)bound) >> 64);
}

/* Threshold t with P(draw < t) = p / 10000. */
static inline uint64_t thresh(uint32_t p_per_10000) {
    if (p_per_10000 >= 10000) return UINT64_MAX;
    return (uint64_t)((((__uint128_t)1) << 64) * p_per_10000 / 10000);
}

enum { ST_RMAT = 1, ST_PERM = 2, ST_GRID_KEEP = 3, ST_GRID_DIAG = 4,
       ST_GRID_DIAG_DIR = 5, ST_WEIGHT = 6, ST_SRC = 7, ST_SEED_PPR = 8 };

/* Random permutation of [0, n) by Fisher-Yates with counter-based draws. */
static void random_perm(uint32_t *perm, int64_t n, uint64_t seed) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t j = bounded(draw(seed, ST_PERM, (uint64_t)i), (uint64_t)i + 1);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/*
 * R-MAT edge list: 2^scale vertices, edge_factor * 2^scale edges. Each edge
 * descends `scale` levels of the adjacency matrix, choosing a quadrant with
 * probabilities a, b, c, d = 1 - a - b - c (given per 10000). Vertex ids are
 * then relabelled by a seeded random permutation. Output arrays hold m_gen
 * entries each.
 */
int fgg_rmat_edges(int scale, int edge_factor, uint32_t a, uint32_t b, uint32_t c,
                   uint64_t seed, uint32_t *src, uint32_t *dst) {
    if (scale < 1 || scale > 31 || edge_factor < 1) return -1;
    if ((uint64_t)a + b + c > 10000) return -1;
    const int64_t n = (int64_t)1 << scale;
    const int64_t m = (int64_t)edge_factor * n;
    const uint64_t ta = thresh(a), tab = thresh(a + b), tabc = thresh(a + b + c);
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!perm) return -2;
    random_perm(perm, n, seed);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            uint64_t r = draw(seed, ST_RMAT, (uint64_t)e * 64u + (uint64_t)l);
            uint32_t bit = 1u << (scale - 1 - l);
            if (r < ta) {
            } else if (r < tab) {
                v |= bit;
            } else if (r < tabc) {
                u |= bit;
            } else {
                u |= bit; v |= bit;
            }
        }
        src[e] = perm[u];
        dst[e] = perm[v];
    }
    free(perm);
    return 0;
}

/*
 * Road-like grid: vertex id = r * cols + c. Each of the right and down
 * 4-neighbour edges is kept with probability (10000 - drop) / 10000. Each
 * vertex, with probability diag / 10000, adds one edge to a uniformly chosen
 * in-bounds diagonal neighbour. Writes at most 2*rows*cols + rows*cols edges;
 * *m_out receives the count.
 */
int fgg_grid_edges(int32_t rows, int32_t cols, uint32_t drop, uint32_t diag, uint64_t seed,
                   uint32_t *src, uint32_t *dst, int64_t *m_out) {
    if (rows < 1 || cols < 1 || drop > 10000 || diag > 10000) return -1;
    if ((int64_t)rows * cols >= ((int64_t)1 << 31)) return -1;
    const uint64_t keep_t = thresh(10000 - drop), diag_t = thresh(diag);
    int64_t m = 0;
    for (int32_t r = 0; r < rows; ++r) {
        for (int32_t c = 0; c < cols; ++c) {
            uint32_t v = (uint32_t)r * (uint32_t)cols + (uint32_t)c;
            if (c + 1 < cols && draw(seed, ST_GRID_KEEP, 2ull * v) < keep_t) {
                src[m] = v; dst[m] = v + 1; ++m;
            }
            if (r + 1 < rows && draw(seed, ST_GRID_KEEP, 2ull * v + 1) < keep_t) {
                src[m] = v; dst[m] = v + (uint32_t)cols; ++m;
            }
            if (draw(seed, ST_GRID_DIAG, v) < diag_t) {
                int32_t cand[4][2];
                int nc = 0;
                const int dr[4] = {-1, -1, 1, 1}, dc[4] = {-1, 1, -1, 1};
                for (int k = 0; k < 4; ++k) {
                    int32_t rr = r + dr[k], cc = c + dc[k];
                    if (rr >= 0 && rr < rows && cc >= 0 && cc < cols) {
                        cand[nc][0] = rr; cand[nc][1] = cc; ++nc;
                    }
                }
                if (nc > 0) {
                    uint64_t k = bounded(draw(seed, ST_GRID_DIAG_DIR, v), (uint64_t)nc);
                    src[m] = v;
                    dst[m] = (uint32_t)cand[k][0] * (uint32_t)cols + (uint32_t)cand[k][1];
                    ++m;
                }
            }
        }
    }
    *m_out = m;
    return 0;
}

static void isort_i32(int32_t *a, int64_t n) {
    for (int64_t i = 1; i < n; ++i) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/*
 * CSR from an edge list: self-loops dropped, duplicate arcs merged, each
 * adjacency list sorted ascending. With `symmetrize`, every edge (u,v) adds
 * both arcs u->v and v->u. `col` must hold (symmetrize ? 2 : 1) * m entries;
 * *m_out receives the arc count. row_ptr has n + 1 entries.
 */
int fgg_csr_build(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst, int symmetrize,
                  int64_t *row_ptr, int32_t *col, int64_t *m_out) {
    if (n < 1 || m < 0) return -1;
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return -2;
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = src[e], v = dst[e];
        if ((int64_t)u >= n || (int64_t)v >= n) { free(deg); return -1; }
        if (u == v) continue;
        deg[u]++;
        if (symmetrize) deg[v]++;
    }
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + deg[i];
    for (int64_t i = 0; i < n; ++i) deg[i] = row_ptr[i];
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = src[e], v = dst[e];
        if (u == v) continue;
        col[deg[u]++] = (int32_t)v;
        if (symmetrize) col[deg[v]++] = (int32_t)u;
    }
    /* sort + dedupe each row in place; deg[i] receives the unique count */
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
        int32_t *a = col + row_ptr[i];
        int64_t len = row_ptr[i + 1] - row_ptr[i];
        if (len < 32) isort_i32(a, len);
        else qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t k = 0;
        for (int64_t j = 0; j < len; ++j)
            if (k == 0 || a[j] != a[k - 1]) a[k++] = a[j];
        deg[i] = k;
    }
    /* compact */
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t s = row_ptr[i], k = deg[i];
        row_ptr[i] = w;
        if (w != s) memmove(col + w, col + s, (size_t)k * sizeof(int32_t));
        w += k;
    }
    row_ptr[n] = w;
    *m_out = w;
    free(deg);
    return 0;
}

/*
 * Integer weights uniform in [lo, hi]: w(u,v) = lo + H(seed, min(u,v), max(u,v)) mod (hi-lo+1),
 * so both directions of an undirected edge carry the same weight.
 */
int fgg_weights(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t lo, int32_t hi,
                uint64_t seed, int32_t *w) {
    if (lo < 0 || hi < lo) return -1;
    const uint64_t span = (uint64_t)(hi - lo) + 1;
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint64_t v = (uint64_t)col[e];
            uint64_t a = (uint64_t)u < v ? (uint64_t)u : v, b = (uint64_t)u < v ? v : (uint64_t)u;
            uint64_t h = draw(seed, ST_WEIGHT, (a << 32) | b);
            w[e] = lo + (int32_t)(h % span);
        }
    }
    return 0;
}

/*
 * k distinct sources drawn uniformly among vertices with out-degree >= 1
 * (partial Fisher-Yates over the candidate list). Returns -1 if fewer than
 * k candidates exist.
 */
int fgg_sources_uniform(int64_t n, const int64_t *row_ptr, int32_t k, uint64_t seed, int32_t *out) {
    int64_t nc = 0;
    for (int64_t v = 0; v < n; ++v) nc += (row_ptr[v + 1] > row_ptr[v]);
    if (k < 0 || nc < k) return -1;
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    if (!cand) return -2;
    int64_t j = 0;
    for (int64_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] > row_ptr[v]) cand[j++] = (int32_t)v;
    for (int32_t i = 0; i < k; ++i) {
        uint64_t r = (uint64_t)i + bounded(draw(seed, ST_SRC, (uint64_t)i), (uint64_t)(nc - i));
        int32_t t = cand[i]; cand[i] = cand[r]; cand[r] = t;
        out[i] = cand[i];
    }
    free(cand);
    return 0;
}

/*
 * k distinct seeds spread evenly over log2-degree buckets: bucket b holds the
 * vertices with floor(log2(outdeg)) = b (outdeg >= 1). Quotas are set by
 * water-filling: non-empty buckets are visited from the smallest to the
 * largest (ties by b), each taking ceil(remaining / buckets_left) seeds or the
 * whole bucket if it is smaller, so a small bucket's shortfall passes to the
 * larger buckets. Seeds are then drawn uniformly without replacement within
 * each bucket, buckets in ascending b. Returns -1 if fewer than k candidates.
 */
int fgg_sources_logdeg(int64_t n, const int64_t *row_ptr, int32_t k, uint64_t seed, int32_t *out) {
    int64_t cnt[64] = {0};
    int64_t total = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d < 1) continue;
        int b = 63 - __builtin_clzll((unsigned long long)d);
        cnt[b]++;
        total++;
    }
    if (k < 0 || total < k) return -1;
    int64_t off[65];
    off[0] = 0;
    for (int b = 0; b < 64; ++b) off[b + 1] = off[b] + cnt[b];
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!cand) return -2;
    int64_t fill[64];
    for (int b = 0; b < 64; ++b) fill[b] = off[b];
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d < 1) continue;
        int b = 63 - __builtin_clzll((unsigned long long)d);
        cand[fill[b]++] = (int32_t)v;
    }
    /* water-filling quotas, smallest bucket first */
    int order[64], nonempty = 0;
    for (int b = 0; b < 64; ++b)
        if (cnt[b] > 0) order[nonempty++] = b;
    for (int i = 1; i < nonempty; ++i) {
        int x = order[i], j = i - 1;
        while (j >= 0 && (cnt[order[j]] > cnt[x] || (cnt[order[j]] == cnt[x] && order[j] > x))) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = x;
    }
    int64_t quota[64] = {0}, remaining = k;
    for (int i = 0; i < nonempty; ++i) {
        int64_t left = nonempty - i;
        int64_t share = (remaining + left - 1) / left;
        int64_t take = share < cnt[order[i]] ? share : cnt[order[i]];
        quota[order[i]] = take;
        remaining -= take;
    }
    int64_t o = 0;
    uint64_t ctr = 0;
    for (int b = 0; b < 64; ++b) {
        int32_t *a = cand + off[b];
        for (int64_t i = 0; i < quota[b]; ++i) {
            uint64_t r = (uint64_t)i + bounded(draw(seed, ST_SEED_PPR, ctr++), (uint64_t)(cnt[b] - i));
            int32_t t = a[i]; a[i] = a[r]; a[r] = t;
            out[o++] = a[i];
        }
    }
    free(cand);
    return (remaining == 0 && o == k) ? 0 : -1;
}
