/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct reference for the many-source graph queries
 * of the fork-processing pattern (Alg. 1; Def. 2.2): per-source SSSP, BFS
 * levels and Personalized PageRank on one CSR graph. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this library; the
 * CUDA path never calls it and shares no code with it.
 *
 * Functions and what they follow:
 *   orc_sssp      binary-heap (lazy deletion) Dijkstra. An operation <q, v, l>
 *                 lowers v's path length when l is shorter (Def. 2.3); the
 *                 sequential algorithm is Dijkstra's (Sec. 4.1, App. A).
 *   orc_bfs       FIFO-queue BFS levels over out-arcs, weights ignored
 *                 (Sec. 4.1-4.2: the BFS priority is the lowest level).
 *   orc_ppr_power FP64 power iteration for pi_s = alpha (I - (1-alpha) P^T)^-1 e_s,
 *                 P = D^-1 A over out-arcs; a dangling row of P is e_s^T.
 *                 The paper cites the sequential PPR of Shun et al. without
 *                 printing alpha, eps or the update rule (Sec. 4.1, 6.1).
 *   orc_ppr_push  FP64 sequential forward push, highest residual first
 *                 (the multiset order of Sec. 4.2), non-lazy rule: while
 *                 r(v) >= eps * max(d(v), 1): p(v) += alpha r(v); each
 *                 out-neighbour gains (1-alpha) r(v) / d(v) (dangling v returns
 *                 (1-alpha) r(v) to the source); r(v) = 0. A diagnostic second
 *                 answer, not the parity target.
 *   orc_*_certificate  implementation-free checks of a distance / level array.
 *   orc_ncp_sweep sweep cut over one PPR vector, the step of the network
 *                 community profile (NCP) application that runs many PPRs
 *                 (Sec. 1, 6.1): vertices with p(v) > 0 ordered by
 *                 p(v) / max(d(v), 1) (computed in FP32), largest first, ties
 *                 by smaller id; for each prefix S_k of the first `top` of them
 *                 the conductance cut(S_k) / min(vol(S_k), vol(V) - vol(S_k)),
 *                 vol = sum of degrees, cut = arcs leaving S_k (undirected).
 *   orc_bc_batch  betweenness centrality from sampled sources (BC, Sec. 1, 6.1:
 *                 one SSSP per source on a weighted graph, one BFS on an
 *                 unweighted one, then the dependency accumulation of Brandes,
 *                 the algorithm the paper cites): the oracle's own Dijkstra /
 *                 BFS, sigma = number of shortest paths (pushed along tight
 *                 arcs in nondecreasing distance order), the dependency
 *                 delta(v) = sum over tight out-arcs (v, w), in CSR order, of
 *                 sigma(v) / sigma(w) * (1 + delta(w)), and
 *                 bc(v) = sum over sources s != v, in batch order, of delta_s(v).
 *                 Each operation is one IEEE double operation in that order
 *                 (built with -ffp-contract=off: no fused multiply-add).
 *   orc_dfs       depth-first search (DFS, a query type of the framework,
 *                 Sec. 3): recursive preorder from s, out-neighbours in CSR
 *                 order; disc[v] = the rank at which v is discovered
 *                 (UINT32_MAX = not reached). Written with an explicit stack
 *                 of (vertex, next arc) pairs, which visits the same order.
 *   orc_rw_batch  random-walk queries (RW, a query type of the framework,
 *                 Sec. 3): a walk of L steps from s moves to the
 *                 (r mod d(u))-th out-neighbour of u in CSR order, r the
 *                 counter-based SplitMix64 output number 2^32 * walk + step + 1
 *                 of the stream seeded with `seed` (Steele, Lea and Flood,
 *                 2014); a vertex without out-arcs ends the walk (-1 after).
 *   orc_ll_query  landmark labeling (LL, Sec. 1, 6.1: labels from a batch of
 *                 SSSPs from landmark vertices): with labels[v][k] = d(s_k, v),
 *                 the distance estimate of a pair (u, v) is the minimum over
 *                 landmarks reaching both of d(s_k, u) + d(s_k, v).
 *
 * Unreachable vertices hold UINT32_MAX. Batches run one query per OpenMP
 * thread, the paper's best CPU scheme ("t = 1", Sec. 1 and 6.1).
 *
 * orc_set_mutation() plants a known mistake (tests use it to show that the
 * pins catch plausible errors); 0 = none, the default.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int g_mutation = 0;

void orc_set_mutation(int k) { g_mutation = k; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* binary min-heap of (key, vertex)                                          */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int32_t v; } hent;
typedef struct { hent *a; int64_t n, cap; } heap;

static int heap_push(heap *h, uint64_t key, int32_t v) {
    if (h->n == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        hent *na = (hent *)realloc(h->a, (size_t)nc * sizeof(hent));
        if (!na) return -1;
        h->a = na; h->cap = nc;
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key; h->a[i].v = v;
    return 0;
}

static hent heap_pop(heap *h) {
    hent top = h->a[0];
    hent last = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        uint64_t sk = last.key;
        if (l < h->n && h->a[l].key < sk) { s = l; sk = h->a[l].key; }
        if (r < h->n && h->a[r].key < sk) { s = r; }
        if (s == i) break;
        h->a[i] = h->a[s];
        i = s;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

/* ------------------------------------------------------------------------ */
/* SSSP: Dijkstra (returns 0, or -3 if a finite distance reaches 2^32 - 1)   */
/* ------------------------------------------------------------------------ */
int orc_sssp(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w, int32_t src,
             uint32_t *dist) {
    if (src < 0 || src >= n) return -1;
    uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
    heap h = {0, 0, 0};
    if (!d || !done) { free(d); free(done); return -2; }
    for (int64_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
    d[src] = 0;
    int rc = heap_push(&h, 0, src);
    while (rc == 0 && h.n > 0) {
        hent t = heap_pop(&h);
        int32_t v = t.v;
        if (done[v] || t.key != d[v]) continue;
        done[v] = 1;
        int64_t end = row_ptr[v + 1];
        if (g_mutation == 2 && end > row_ptr[v]) end--; /* planted: skips the last arc */
        for (int64_t e = row_ptr[v]; e < end; ++e) {
            int32_t u = col[e];
            uint64_t wt = (w && g_mutation != 1) ? (uint64_t)(uint32_t)w[e] : 1u;
            uint64_t nd = d[v] + wt;
            if (nd < d[u]) {
                d[u] = nd;
                if (heap_push(&h, nd, u)) { rc = -2; break; }
            }
        }
    }
    if (rc == 0) {
        for (int64_t v = 0; v < n; ++v) {
            if (d[v] == UINT64_MAX) dist[v] = UINT32_MAX;
            else if (d[v] >= (uint64_t)UINT32_MAX) { rc = -3; dist[v] = UINT32_MAX; }
            else dist[v] = (uint32_t)d[v];
        }
    }
    free(h.a); free(d); free(done);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* BFS levels with a FIFO queue                                              */
/* ------------------------------------------------------------------------ */
int orc_bfs(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t src, uint32_t *level) {
    if (src < 0 || src >= n) return -1;
    int32_t *q = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!q) return -2;
    for (int64_t v = 0; v < n; ++v) level[v] = UINT32_MAX;
    int64_t head = 0, tail = 0;
    level[src] = (g_mutation == 3) ? 1u : 0u; /* planted: levels start at 1 */
    q[tail++] = src;
    while (head < tail) {
        int32_t v = q[head++];
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int32_t u = col[e];
            if (level[u] == UINT32_MAX) {
                level[u] = level[v] + 1;
                q[tail++] = u;
            }
        }
    }
    free(q);
    return 0;
}

/* batches: one query per OpenMP thread; out is query-major nq x n */
int orc_sssp_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                   int32_t nq, const int32_t *srcs, uint32_t *out) {
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
    for (int32_t i = 0; i < nq; ++i) {
        int r = orc_sssp(n, row_ptr, col, w, srcs[i], out + (size_t)i * (size_t)n);
        if (r < rc) rc = r;
    }
    return rc;
}

int orc_bfs_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t nq,
                  const int32_t *srcs, uint32_t *out) {
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
    for (int32_t i = 0; i < nq; ++i) {
        int r = orc_bfs(n, row_ptr, col, srcs[i], out + (size_t)i * (size_t)n);
        if (r < rc) rc = r;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* PPR by FP64 power iteration:                                              */
/*   x_0 = alpha e_s;  x_{k+1} = alpha e_s + (1 - alpha) P^T x_k              */
/* until ||x_{k+1} - x_k||_1 < tol. Returns the iteration count, or < 0.     */
/* ------------------------------------------------------------------------ */
int orc_ppr_power(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t src, double alpha,
                  double tol, int max_iter, double *pi) {
    if (src < 0 || src >= n || !(alpha > 0.0 && alpha < 1.0)) return -1;
    double *x = pi;
    double *y = (double *)malloc((size_t)n * sizeof(double));
    if (!y) return -2;
    for (int64_t v = 0; v < n; ++v) x[v] = 0.0;
    x[src] = alpha;
    int it = 0;
    for (; it < max_iter; ++it) {
        for (int64_t v = 0; v < n; ++v) y[v] = 0.0;
        /* y = P^T x, P = D^-1 A (row v spreads x[v] / d(v) over its out-arcs) */
        for (int64_t v = 0; v < n; ++v) {
            int64_t d = row_ptr[v + 1] - row_ptr[v];
            if (x[v] == 0.0) continue;
            if (d == 0) {
                if (g_mutation != 5) y[src] += x[v]; /* dangling row = e_s^T (planted 5 drops it) */
                continue;
            }
            double share = x[v] / (double)d;
            for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                if (g_mutation == 4) y[v] += x[col[e]] / (double)d; /* planted: transposed operand */
                else y[col[e]] += share;
            }
        }
        double diff = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double nv = (1.0 - alpha) * y[v] + (v == src ? alpha : 0.0);
            diff += fabs(nv - x[v]);
            x[v] = nv;
        }
        if (diff < tol) { ++it; break; }
    }
    free(y);
    return it;
}

int orc_ppr_power_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t nq,
                        const int32_t *srcs, double alpha, double tol, int max_iter, double *out) {
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
    for (int32_t i = 0; i < nq; ++i) {
        int r = orc_ppr_power(n, row_ptr, col, srcs[i], alpha, tol, max_iter, out + (size_t)i * (size_t)n);
        if (r < rc) rc = r;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* PPR by FP64 sequential forward push, largest residual first.              */
/* Returns the number of pushes, or < 0.                                     */
/* ------------------------------------------------------------------------ */
typedef struct { double key; int32_t v; } mxent;

static void mx_push(mxent *a, int64_t *n, double key, int32_t v) {
    int64_t i = (*n)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (a[p].key >= key) break;
        a[i] = a[p];
        i = p;
    }
    a[i].key = key; a[i].v = v;
}

static mxent mx_pop(mxent *a, int64_t *n) {
    mxent top = a[0], last = a[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        double sk = last.key;
        if (l < *n && a[l].key > sk) { s = l; sk = a[l].key; }
        if (r < *n && a[r].key > sk) { s = r; }
        if (s == i) break;
        a[i] = a[s];
        i = s;
    }
    if (*n > 0) a[i] = last;
    return top;
}

int64_t orc_ppr_push(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t src, double alpha,
                     double eps, double *p, double *r) {
    if (src < 0 || src >= n || !(alpha > 0.0 && alpha < 1.0) || !(eps > 0.0)) return -1;
    for (int64_t v = 0; v < n; ++v) { p[v] = 0.0; r[v] = 0.0; }
    r[src] = 1.0;
    /* lazy max-heap of (residual at insertion, v); capacity grows as needed */
    int64_t cap = 1024, hn = 0, pushes = 0;
    mxent *hp = (mxent *)malloc((size_t)cap * sizeof(mxent));
    if (!hp) return -2;
    mx_push(hp, &hn, 1.0, src);
    while (hn > 0) {
        mxent t = mx_pop(hp, &hn);
        int32_t v = t.v;
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        double thr = eps * (double)(d > 0 ? d : 1);
        if (t.key != r[v] || r[v] < thr) continue; /* stale entry */
        double rho = r[v];
        r[v] = 0.0;
        p[v] += alpha * rho;
        ++pushes;
        if (hn + d + 1 >= cap) {
            while (hn + d + 1 >= cap) cap *= 2;
            mxent *nh = (mxent *)realloc(hp, (size_t)cap * sizeof(mxent));
            if (!nh) { free(hp); return -2; }
            hp = nh;
        }
        if (d == 0) {
            r[src] += (1.0 - alpha) * rho;
            double ts = eps * (double)((row_ptr[src + 1] - row_ptr[src]) > 0 ? (row_ptr[src + 1] - row_ptr[src]) : 1);
            if (r[src] >= ts) mx_push(hp, &hn, r[src], src);
            continue;
        }
        double inc = (1.0 - alpha) * rho / (double)d;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int32_t u = col[e];
            r[u] += inc;
            int64_t du = row_ptr[u + 1] - row_ptr[u];
            if (r[u] >= eps * (double)(du > 0 ? du : 1)) mx_push(hp, &hn, r[u], u);
        }
    }
    free(hp);
    return pushes;
}

/* ------------------------------------------------------------------------ */
/* Certificates (no shortest-path computation inside):                       */
/*   SSSP (w >= 1): d(s) = 0; every arc (u,v) with d(u) finite has           */
/*   d(v) <= d(u) + w; every finite v != s has an arc (u,v) with             */
/*   d(v) = d(u) + w; d(v) finite iff v is reachable from s.                 */
/* With positive weights these conditions determine d exactly. BFS is the    */
/* same check with unit weights. Returns 0 if valid, else a code naming the  */
/* failed condition (1 source, 2 edge slack, 3 no parent, 4 reachability).   */
/* ------------------------------------------------------------------------ */
static int certificate(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                       int32_t src, const uint32_t *d) {
    if (d[src] != 0) return 1;
    unsigned char *has_parent = (unsigned char *)calloc((size_t)n, 1);
    unsigned char *seen = (unsigned char *)calloc((size_t)n, 1);
    int32_t *q = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!has_parent || !seen || !q) { free(has_parent); free(seen); free(q); return -2; }
    int rc = 0;
    for (int64_t u = 0; u < n && rc == 0; ++u) {
        if (d[u] == UINT32_MAX) continue;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            uint64_t cand = (uint64_t)d[u] + (w ? (uint64_t)(uint32_t)w[e] : 1u);
            if ((uint64_t)d[v] > cand) { rc = 2; break; }
            if ((uint64_t)d[v] == cand) has_parent[v] = 1;
        }
    }
    for (int64_t v = 0; v < n && rc == 0; ++v)
        if (v != src && d[v] != UINT32_MAX && !has_parent[v]) rc = 3;
    if (rc == 0) {
        int64_t head = 0, tail = 0;
        seen[src] = 1; q[tail++] = src;
        while (head < tail) {
            int32_t v = q[head++];
            for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
                if (!seen[col[e]]) { seen[col[e]] = 1; q[tail++] = col[e]; }
        }
        for (int64_t v = 0; v < n && rc == 0; ++v)
            if ((seen[v] != 0) != (d[v] != UINT32_MAX)) rc = 4;
    }
    free(has_parent); free(seen); free(q);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* sweep cut (NCP)                                                           */
/* ------------------------------------------------------------------------ */
typedef struct { float key; int32_t v; } swent;

static int sweep_cmp(const void *a, const void *b) {
    const swent *x = (const swent *)a, *y = (const swent *)b;
    if (x->key > y->key) return -1;
    if (x->key < y->key) return 1;
    return (x->v > y->v) - (x->v < y->v);
}

/* order[k] = k-th vertex of the sweep, phi[k] = conductance of the first k + 1
   vertices (1.0 when the smaller volume is 0). Returns the number of prefixes
   (<= top), or a negative error. */
int orc_ncp_sweep(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *p, int32_t top,
                  int32_t *order, double *phi) {
    if (n < 1 || top < 1) return -1;
    swent *c = (swent *)malloc((size_t)n * sizeof(swent));
    int32_t *rank = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!c || !rank) { free(c); free(rank); return -2; }
    int64_t nc = 0;
    for (int64_t v = 0; v < n; ++v) {
        rank[v] = -1;
        if (p[v] > 0.0f) {
            const int64_t d = row_ptr[v + 1] - row_ptr[v];
            c[nc].key = p[v] / (float)(d > 0 ? d : 1);
            c[nc].v = (int32_t)v;
            ++nc;
        }
    }
    qsort(c, (size_t)nc, sizeof(swent), sweep_cmp);
    const int64_t k_max = nc < top ? nc : top;
    for (int64_t k = 0; k < k_max; ++k) { order[k] = c[k].v; rank[c[k].v] = (int32_t)k; }
    const int64_t vol_all = row_ptr[n];
    int64_t cut = 0, vol = 0;
    for (int64_t k = 0; k < k_max; ++k) {
        const int32_t v = order[k];
        int64_t inside = 0;  /* neighbours already in the set */
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const int32_t r = rank[col[e]];
            if (r >= 0 && r < k) ++inside;
        }
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        cut += d - (g_mutation == 6 ? inside : 2 * inside);  /* planted 6: internal arcs counted once */
        vol += d;
        const int64_t den = vol < vol_all - vol ? vol : vol_all - vol;
        phi[k] = den > 0 ? (double)cut / (double)den : 1.0;
    }
    free(c);
    free(rank);
    return (int)k_max;
}

int orc_ncp_sweep_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t nq, const float *p,
                        int32_t top, int32_t *order, double *phi, int32_t *count) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t q = 0; q < nq; ++q) {
        const int r = orc_ncp_sweep(n, row_ptr, col, p + (size_t)q * (size_t)n, top, order + (size_t)q * top,
                                    phi + (size_t)q * top);
        count[q] = r;
        if (r < 0) bad |= 1;
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* betweenness centrality (BC)                                               */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t d; int32_t v; } dvent;

static int dv_cmp(const void *a, const void *b) {
    const dvent *x = (const dvent *)a, *y = (const dvent *)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

/* One source: dist (from orc_sssp / orc_bfs), sigma and delta (double[n]).
   Returns 0, 1 if some sigma reached 2^53 (then sums of path counts may have
   rounded), or a negative error. Arcs of weight 0 are rejected (-4): they
   would put equal-distance vertices on shortest paths of each other. */
static int bc_one(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w, int32_t src,
                  const uint32_t *dist, double *sigma, double *delta, dvent *ord) {
    int64_t nr = 0;
    for (int64_t v = 0; v < n; ++v) {
        sigma[v] = 0.0;
        delta[v] = 0.0;
        if (dist[v] != UINT32_MAX) { ord[nr].d = dist[v]; ord[nr].v = (int32_t)v; ++nr; }
    }
    qsort(ord, (size_t)nr, sizeof(dvent), dv_cmp);
    sigma[src] = 1.0;
    int inexact = 0;
    for (int64_t i = 0; i < nr; ++i) {                 /* sigma, nondecreasing distance */
        const int32_t u = ord[i].v;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            const int32_t x = col[e];
            const uint64_t wt = w ? (uint64_t)w[e] : 1u;
            if (w && w[e] == 0) return -4;
            if (dist[x] != UINT32_MAX && (uint64_t)dist[u] + wt == (uint64_t)dist[x]) {
                sigma[x] = sigma[x] + sigma[u];
                if (sigma[x] >= 9007199254740992.0) inexact = 1;
            }
        }
    }
    for (int64_t i = nr - 1; i >= 0; --i) {            /* delta, nonincreasing distance */
        const int32_t u = ord[i].v;
        double acc = 0.0;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            const int32_t x = col[e];
            const uint64_t wt = w ? (uint64_t)w[e] : 1u;
            if (dist[x] != UINT32_MAX && (uint64_t)dist[u] + wt == (uint64_t)dist[x]) {
                const double ratio = sigma[u] / sigma[x];
                const double term = g_mutation == 8 ? delta[x] : 1.0 + delta[x];  /* planted 8: drops the 1 */
                acc = acc + ratio * term;
            }
        }
        delta[u] = acc;
    }
    return inexact;
}

/* bc[v] (double[n]) = sum over q in order of delta_{srcs[q]}(v), v != srcs[q];
   weighted != 0: SSSP distances over w, else BFS levels. sigma_max (nullable)
   receives the largest path count. Returns 0, 1 (some path count reached 2^53)
   or a negative error. */
int orc_bc_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w, int weighted, int32_t nq,
                 const int32_t *srcs, double *bc, double *sigma_max) {
    const int32_t *ww = weighted ? w : NULL;
    double *delta_all = (double *)malloc((size_t)nq * (size_t)n * sizeof(double));
    if (!delta_all) return -2;
    int rc = 0;
    double smax = 0.0;
#pragma omp parallel reduction(| : rc) reduction(max : smax)
    {
        uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        double *sigma = (double *)malloc((size_t)n * sizeof(double));
        dvent *ord = (dvent *)malloc((size_t)n * sizeof(dvent));
        if (!dist || !sigma || !ord) rc |= 2;
#pragma omp for schedule(dynamic, 1)
        for (int32_t q = 0; q < nq; ++q) {
            if (rc & 2) continue;
            if (srcs[q] < 0 || srcs[q] >= n) { rc |= 4; continue; }
            const int r0 = ww ? orc_sssp(n, row_ptr, col, ww, srcs[q], dist) : orc_bfs(n, row_ptr, col, srcs[q], dist);
            if (r0 != 0) { rc |= 8; continue; }
            const int r = bc_one(n, row_ptr, col, ww, srcs[q], dist, sigma, delta_all + (size_t)q * (size_t)n, ord);
            if (r < 0) { rc |= 16; continue; }
            rc |= r;
            for (int64_t v = 0; v < n; ++v) if (sigma[v] > smax) smax = sigma[v];
        }
        free(dist); free(sigma); free(ord);
    }
    if (rc & ~1) { free(delta_all); return -1 - (rc & ~1); }
    for (int64_t v = 0; v < n; ++v) {
        double acc = 0.0;
        for (int32_t q = 0; q < nq; ++q)
            if (srcs[q] != v) acc = acc + delta_all[(size_t)q * (size_t)n + (size_t)v];
        bc[v] = acc;
    }
    free(delta_all);
    if (sigma_max) *sigma_max = smax;
    return rc & 1;
}

/* ------------------------------------------------------------------------ */
/* depth-first search (DFS)                                                  */
/* ------------------------------------------------------------------------ */
int orc_dfs(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t src, uint32_t *disc) {
    if (src < 0 || src >= n) return -1;
    int32_t *stk_v = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *stk_e = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!stk_v || !stk_e) { free(stk_v); free(stk_e); return -2; }
    for (int64_t v = 0; v < n; ++v) disc[v] = UINT32_MAX;
    uint32_t time = 0;
    int64_t top = 0;
    disc[src] = time++;
    stk_v[0] = src;
    stk_e[0] = row_ptr[src];
    while (top >= 0) {
        const int32_t u = stk_v[top];
        int64_t e = stk_e[top];
        const int64_t e_end = row_ptr[u + 1];
        /* planted 10: the neighbours are scanned from the last arc backwards */
        if (g_mutation == 10) {
            int64_t k = e;  /* here e counts the arcs already scanned from the end */
            while (k < e_end && disc[col[e_end - 1 - (k - row_ptr[u])]] != UINT32_MAX) ++k;
            if (k < e_end) {
                const int32_t w = col[e_end - 1 - (k - row_ptr[u])];
                stk_e[top] = k + 1;
                disc[w] = time++;
                ++top;
                stk_v[top] = w;
                stk_e[top] = row_ptr[w];
            } else {
                --top;
            }
            continue;
        }
        while (e < e_end && disc[col[e]] != UINT32_MAX) ++e;
        if (e < e_end) {
            const int32_t w = col[e];
            stk_e[top] = e + 1;      /* resume after this arc when w is finished */
            disc[w] = time++;
            ++top;
            stk_v[top] = w;
            stk_e[top] = row_ptr[w];
        } else {
            --top;                   /* every neighbour of u is discovered: u is finished */
        }
    }
    free(stk_v);
    free(stk_e);
    return 0;
}

int orc_dfs_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t nq, const int32_t *srcs,
                  uint32_t *disc) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t q = 0; q < nq; ++q)
        if (orc_dfs(n, row_ptr, col, srcs[q], disc + (size_t)q * (size_t)n) != 0) bad |= 1;
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* random walks (RW)                                                         */
/* ------------------------------------------------------------------------ */
/* Output number k (k >= 1) of a SplitMix64 stream whose state starts at seed:
   the state after k steps of the golden gamma, through the mix function. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* paths: int32[nq][L + 1], paths[q][0] = srcs[q]. Returns 0, or -1 on a bad source. */
int orc_rw_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t nq, const int32_t *srcs,
                 int32_t L, uint64_t seed, int32_t *paths) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int32_t q = 0; q < nq; ++q) {
        int32_t *row = paths + (size_t)q * (size_t)(L + 1);
        int32_t u = srcs[q];
        if (u < 0 || u >= n) { bad |= 1; continue; }
        row[0] = u;
        for (int32_t t = 0; t < L; ++t) {
            const int64_t d = u >= 0 ? row_ptr[u + 1] - row_ptr[u] : 0;
            if (d == 0) { u = -1; row[t + 1] = -1; continue; }
            const uint64_t k = ((uint64_t)(uint32_t)q << 32) + (uint64_t)t + (g_mutation == 9 ? 0u : 1u);  /* planted 9 */
            const uint64_t r = orc_splitmix64(seed, k);
            u = col[row_ptr[u] + (int64_t)(r % (uint64_t)d)];
            row[t + 1] = u;
        }
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* landmark labeling query (LL)                                              */
/* ------------------------------------------------------------------------ */
/* labels: vertex-major uint32[n][K], labels[v * K + k] = d(s_k, v), UINT32_MAX
   = unreachable. pairs: int32[2 * Q] (u, v). out[i] = min over k with both
   entries finite of labels[u][k] + labels[v][k] (exact in uint64), UINT64_MAX
   when no landmark reaches both. Returns 0, or -1 on a vertex id out of range. */
int orc_ll_query(int64_t n, int32_t K, const uint32_t *labels, int64_t Q, const int32_t *pairs, uint64_t *out) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < Q; ++i) {
        const int32_t u = pairs[2 * i], v = pairs[2 * i + 1];
        if (u < 0 || u >= n || v < 0 || v >= n) { bad |= 1; out[i] = UINT64_MAX; continue; }
        const uint32_t *lu = labels + (size_t)u * (size_t)K, *lv = labels + (size_t)v * (size_t)K;
        uint64_t best = UINT64_MAX;
        for (int32_t k = 0; k < K; ++k) {
            if (g_mutation != 7 && (lu[k] == UINT32_MAX || lv[k] == UINT32_MAX)) continue;  /* planted 7: no reach check */
            const uint64_t d = (uint64_t)lu[k] + (uint64_t)lv[k];
            if (d < best) best = d;
        }
        out[i] = best;
    }
    return bad ? -1 : 0;
}

int orc_sssp_certificate(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                         int32_t src, const uint32_t *dist) {
    return certificate(n, row_ptr, col, w, src, dist);
}

int orc_bfs_certificate(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t src,
                        const uint32_t *level) {
    return certificate(n, row_ptr, col, NULL, src, level);
}

/* certificate over a query-major batch; returns the first failing query's code * 2^20 + q, else 0 */
int64_t orc_certificate_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                              int32_t nq, const int32_t *srcs, const uint32_t *out) {
    int64_t first = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < nq; ++i) {
        int r = certificate(n, row_ptr, col, w, srcs[i], out + (size_t)i * (size_t)n);
        if (r != 0) {
#pragma omp critical
            if (first == 0) first = ((int64_t)r << 20) + i;
        }
    }
    return first;
}
