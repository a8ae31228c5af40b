/*
 * oracle.c -- plain CPU oracle for stable-vertex-value queries over an
 * evolving graph.  TEST INFRASTRUCTURE ONLY: tests, the smoke check and the
 * bench's CPU-baseline leg call it; the library never does.  It shares no code,
 * header or table with the GPU library.
 *
 * What it computes (paper Section 2, Fig. 2a, "naive" strategy): for every
 * snapshot G_i of a window, the query's value of every vertex, solved from
 * scratch on the snapshot materialised by replaying the edge log.  Theorems 1
 * and 2 (Section 3) and the monotone fixed-point argument of Section 4.2 say
 * the intersection-union method must reach exactly these values.
 *
 * Edge functions (Table 2):
 *   SSSP : Val(v) = min over in-edges (u,v) of Val(u) + w(u,v); Val(src) = 0.
 *   SSWP : Val(v) = max over in-edges of min(Val(u), w(u,v));  Val(src) = +inf.
 *   BFS  : Val(v) = min over in-edges of Val(u) + 1;          Val(src) = 0.
 *   SSNP : Val(v) = min over in-edges of max(Val(u), w(u,v)); Val(src) = 0.
 * Readings where the paper is silent (unreachable encoding, overflow):
 *   SSSP/BFS unreachable = 0xFFFFFFFF; SSWP +inf = 0xFFFFFFFF and unreachable
 *   = 0; SSSP sums saturate at 0xFFFFFFFE so a reached vertex never reads as
 *   unreachable.
 *
 * Solvers: binary-heap Dijkstra (SSSP), max-heap widest-path Dijkstra (SSWP),
 * FIFO breadth-first search (BFS), min-heap narrowest-path Dijkstra (SSNP: the
 * path value is the largest weight on the path).
 *
 * Extras used to pin single steps of the method (Section 3, Step 1):
 * oracle_bounds() materialises the intersection graph (instances live in every
 * window snapshot) and the union graph (live in any), and solves both.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define OR_SSSP 0
#define OR_SSWP 1
#define OR_BFS 2
#define OR_SSNP 3
#define OR_INF 0xFFFFFFFFu
#define OR_SAT 0xFFFFFFFEu

/* ------------------------------------------------------------------ */
/* binary heap of (key, vertex); `better(a,b)` orders the top          */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t key;
    uint32_t v;
} hitem;

typedef struct {
    hitem *a;
    size_t n, cap;
    int maxheap; /* 0: smallest key on top; 1: largest key on top */
} heap;

static int h_before(const heap *h, hitem x, hitem y) {
    return h->maxheap ? (x.key > y.key) : (x.key < y.key);
}

static int h_push(heap *h, hitem x) {
    if (h->n == h->cap) {
        size_t nc = h->cap ? 2 * h->cap : 1024;
        hitem *na = (hitem *)realloc(h->a, nc * sizeof(hitem));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    size_t i = h->n++;
    h->a[i] = x;
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (!h_before(h, h->a[i], h->a[p])) break;
        hitem t = h->a[i];
        h->a[i] = h->a[p];
        h->a[p] = t;
        i = p;
    }
    return 0;
}

static hitem h_pop(heap *h) {
    hitem top = h->a[0];
    h->a[0] = h->a[--h->n];
    size_t i = 0;
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < h->n && h_before(h, h->a[l], h->a[b])) b = l;
        if (r < h->n && h_before(h, h->a[r], h->a[b])) b = r;
        if (b == i) break;
        hitem t = h->a[i];
        h->a[i] = h->a[b];
        h->a[b] = t;
        i = b;
    }
    return top;
}

/* ------------------------------------------------------------------ */
/* single-graph solvers on a CSR (row_ptr[V+1], col, w)                 */
/* ------------------------------------------------------------------ */

/* Dijkstra, Section 2 / Table 2 SSSP: dist(src)=0, relax Val(u)+w. */
static int solve_sssp(uint32_t V, const uint64_t *rp, const uint32_t *col, const uint32_t *w,
                      uint32_t src, uint32_t *dist) {
    heap h = {0};
    h.maxheap = 0;
    char *done = (char *)calloc(V ? V : 1, 1);
    if (!done) return -1;
    for (uint32_t v = 0; v < V; ++v) dist[v] = OR_INF;
    dist[src] = 0;
    if (h_push(&h, (hitem){0, src})) goto oom;
    while (h.n) {
        hitem t = h_pop(&h);
        if (done[t.v] || t.key != dist[t.v]) continue;
        done[t.v] = 1;
        for (uint64_t e = rp[t.v]; e < rp[t.v + 1]; ++e) {
            uint64_t s = (uint64_t)t.key + w[e];
            uint32_t nd = s > OR_SAT ? OR_SAT : (uint32_t)s;
            uint32_t x = col[e];
            if (nd < dist[x]) {
                dist[x] = nd;
                if (h_push(&h, (hitem){nd, x})) goto oom;
            }
        }
    }
    free(h.a);
    free(done);
    return 0;
oom:
    free(h.a);
    free(done);
    return -1;
}

/* Widest path, Table 2 SSWP: width(src)=+inf, relax min(Val(u), w). */
static int solve_sswp(uint32_t V, const uint64_t *rp, const uint32_t *col, const uint32_t *w,
                      uint32_t src, uint32_t *width) {
    heap h = {0};
    h.maxheap = 1;
    char *done = (char *)calloc(V ? V : 1, 1);
    if (!done) return -1;
    for (uint32_t v = 0; v < V; ++v) width[v] = 0;
    width[src] = OR_INF;
    if (h_push(&h, (hitem){OR_INF, src})) goto oom;
    while (h.n) {
        hitem t = h_pop(&h);
        if (done[t.v] || t.key != width[t.v]) continue;
        done[t.v] = 1;
        for (uint64_t e = rp[t.v]; e < rp[t.v + 1]; ++e) {
            uint32_t nw = t.key < w[e] ? t.key : w[e];
            uint32_t x = col[e];
            if (nw > width[x]) {
                width[x] = nw;
                if (h_push(&h, (hitem){nw, x})) goto oom;
            }
        }
    }
    free(h.a);
    free(done);
    return 0;
oom:
    free(h.a);
    free(done);
    return -1;
}

/* Narrowest path, Table 2 SSNP: Val(src)=0, relax max(Val(u), w); a
 * min-heap settles vertices in order of their path's largest weight. */
static int solve_ssnp(uint32_t V, const uint64_t *rp, const uint32_t *col, const uint32_t *w,
                      uint32_t src, uint32_t *best) {
    heap h = {0};
    h.maxheap = 0;
    char *done = (char *)calloc(V ? V : 1, 1);
    if (!done) return -1;
    for (uint32_t v = 0; v < V; ++v) best[v] = OR_INF;
    best[src] = 0;
    if (h_push(&h, (hitem){0, src})) goto oom;
    while (h.n) {
        hitem t = h_pop(&h);
        if (done[t.v] || t.key != best[t.v]) continue;
        done[t.v] = 1;
        for (uint64_t e = rp[t.v]; e < rp[t.v + 1]; ++e) {
            uint32_t nb = t.key > w[e] ? t.key : w[e];
            uint32_t x = col[e];
            if (nb < best[x]) {
                best[x] = nb;
                if (h_push(&h, (hitem){nb, x})) goto oom;
            }
        }
    }
    free(h.a);
    free(done);
    return 0;
oom:
    free(h.a);
    free(done);
    return -1;
}

/* Breadth-first search, Table 2 BFS: level(src)=0, relax Val(u)+1. */
static int solve_bfs(uint32_t V, const uint64_t *rp, const uint32_t *col, uint32_t src,
                     uint32_t *level) {
    uint32_t *q = (uint32_t *)malloc((size_t)(V ? V : 1) * sizeof(uint32_t));
    if (!q) return -1;
    for (uint32_t v = 0; v < V; ++v) level[v] = OR_INF;
    size_t head = 0, tail = 0;
    level[src] = 0;
    q[tail++] = src;
    while (head < tail) {
        uint32_t u = q[head++];
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
            uint32_t x = col[e];
            if (level[x] == OR_INF) {
                level[x] = level[u] + 1;
                q[tail++] = x;
            }
        }
    }
    free(q);
    return 0;
}

/* Solve one query type on one CSR graph.  Returns 0, -1 on allocation
 * failure, -2 on bad arguments. */
int oracle_solve(int type, uint32_t V, const uint64_t *row_ptr, const uint32_t *col,
                 const uint32_t *w, uint32_t src, uint32_t *out) {
    if (src >= V) return -2;
    switch (type) {
    case OR_SSSP: return solve_sssp(V, row_ptr, col, w, src, out);
    case OR_SSWP: return solve_sswp(V, row_ptr, col, w, src, out);
    case OR_BFS: return solve_bfs(V, row_ptr, col, src, out);
    case OR_SSNP: return solve_ssnp(V, row_ptr, col, w, src, out);
    default: return -2;
    }
}

/* ------------------------------------------------------------------ */
/* edge-log replay (Section 2: G_i = G_{i-1} minus deletions plus      */
/* additions; G_0 = the base graph added by step 0)                     */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t V, S;
    uint64_t n_inst;
    const uint32_t *src, *dst, *w;
    const int64_t *add_off; /* [S+1] */
    const int64_t *del_off; /* [S+1] */
    const int64_t *del_ids;
} edge_log;

/* alive[k] = 1 iff instance k is live in snapshot `snap`, by replaying
 * steps 0..snap in order (deletions of a step, then its additions). */
static void replay_to(const edge_log *lg, uint32_t snap, unsigned char *alive) {
    memset(alive, 0, lg->n_inst);
    for (uint32_t s = 0; s <= snap; ++s) {
        for (int64_t k = lg->del_off[s]; k < lg->del_off[s + 1]; ++k) alive[lg->del_ids[k]] = 0;
        for (int64_t k = lg->add_off[s]; k < lg->add_off[s + 1]; ++k) alive[k] = 1;
    }
}

/* CSR of the instances with keep[k] != 0 (counting sort by source). */
static int materialise(const edge_log *lg, const unsigned char *keep, uint64_t *rp, uint32_t **col_out,
                       uint32_t **w_out) {
    uint32_t V = lg->V;
    memset(rp, 0, (size_t)(V + 1) * sizeof(uint64_t));
    for (uint64_t k = 0; k < lg->n_inst; ++k)
        if (keep[k]) rp[lg->src[k] + 1]++;
    for (uint32_t v = 0; v < V; ++v) rp[v + 1] += rp[v];
    uint64_t m = rp[V];
    uint32_t *col = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *w = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint64_t *fill = (uint64_t *)malloc((size_t)(V ? V : 1) * sizeof(uint64_t));
    if (!col || !w || !fill) {
        free(col);
        free(w);
        free(fill);
        return -1;
    }
    memcpy(fill, rp, (size_t)V * sizeof(uint64_t));
    for (uint64_t k = 0; k < lg->n_inst; ++k) {
        if (!keep[k]) continue;
        uint64_t p = fill[lg->src[k]]++;
        col[p] = lg->dst[k];
        w[p] = lg->w[k];
    }
    free(fill);
    *col_out = col;
    *w_out = w;
    return 0;
}

static int solve_kept(const edge_log *lg, const unsigned char *keep, int type, uint32_t source,
                      uint32_t *out) {
    uint64_t *rp = (uint64_t *)malloc((size_t)(lg->V + 1) * sizeof(uint64_t));
    uint32_t *col = NULL, *w = NULL;
    if (!rp) return -1;
    int rc = materialise(lg, keep, rp, &col, &w);
    if (rc == 0) rc = oracle_solve(type, lg->V, rp, col, w, source, out);
    free(rp);
    free(col);
    free(w);
    return rc;
}

/* Materialise snapshot `snap` as a CSR (caller frees *col and *w with
 * oracle_free).  row_ptr has V+1 entries. */
int oracle_snapshot_csr(uint32_t V, uint32_t S, uint64_t n_inst, const uint32_t *src,
                        const uint32_t *dst, const uint32_t *w, const int64_t *add_off,
                        const int64_t *del_off, const int64_t *del_ids, uint32_t snap,
                        uint64_t *row_ptr, uint32_t **col, uint32_t **wout) {
    if (snap >= S) return -2;
    edge_log lg = {V, S, n_inst, src, dst, w, add_off, del_off, del_ids};
    unsigned char *alive = (unsigned char *)malloc(n_inst ? n_inst : 1);
    if (!alive) return -1;
    replay_to(&lg, snap, alive);
    int rc = materialise(&lg, alive, row_ptr, col, wout);
    free(alive);
    return rc;
}

void oracle_free(void *p) { free(p); }

/* ------------------------------------------------------------------ */
/* per-snapshot query over a window, parallel over snapshots           */
/* ------------------------------------------------------------------ */
typedef struct {
    const edge_log *lg;
    int type;
    uint32_t source, win_begin, win_len;
    uint32_t *out; /* [win_len][V] */
    uint32_t next; /* shared work counter */
    pthread_mutex_t mu;
    int rc;
} query_job;

static void *query_worker(void *arg) {
    query_job *j = (query_job *)arg;
    unsigned char *alive = (unsigned char *)malloc(j->lg->n_inst ? j->lg->n_inst : 1);
    if (!alive) {
        pthread_mutex_lock(&j->mu);
        j->rc = -1;
        pthread_mutex_unlock(&j->mu);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&j->mu);
        uint32_t i = j->next++;
        int bad = j->rc;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->win_len || bad) break;
        replay_to(j->lg, j->win_begin + i, alive);
        int rc = solve_kept(j->lg, alive, j->type, j->source, j->out + (size_t)i * j->lg->V);
        if (rc) {
            pthread_mutex_lock(&j->mu);
            j->rc = rc;
            pthread_mutex_unlock(&j->mu);
            break;
        }
    }
    free(alive);
    return NULL;
}

/* out[i*V + v] = value of v in snapshot win_begin+i, for i < win_len.
 * nthreads <= 0 uses every online core.  Returns 0 / -1 (memory) / -2 (args). */
int oracle_query(int type, uint32_t V, uint32_t S, uint64_t n_inst, const uint32_t *src,
                 const uint32_t *dst, const uint32_t *w, const int64_t *add_off,
                 const int64_t *del_off, const int64_t *del_ids, uint32_t source,
                 uint32_t win_begin, uint32_t win_len, uint32_t *out, int nthreads) {
    if (source >= V || win_len == 0 || (uint64_t)win_begin + win_len > S) return -2;
    if (type < 0 || type > 3) return -2;
    edge_log lg = {V, S, n_inst, src, dst, w, add_off, del_off, del_ids};
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if ((uint32_t)nthreads > win_len) nthreads = (int)win_len;
    query_job j;
    j.lg = &lg;
    j.type = type;
    j.source = source;
    j.win_begin = win_begin;
    j.win_len = win_len;
    j.out = out;
    j.next = 0;
    j.rc = 0;
    pthread_mutex_init(&j.mu, NULL);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -1;
    int started = 0;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, query_worker, &j) == 0) started++;
        else break;
    if (started == 0) query_worker(&j);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&j.mu);
    return j.rc;
}

/* Section 3, Step 1: r_cap = query on the intersection graph (instances
 * live in every snapshot of the window), r_cup = query on the union graph
 * (live in at least one).  Each snapshot's live set comes from the replay. */
int oracle_bounds(int type, uint32_t V, uint32_t S, uint64_t n_inst, const uint32_t *src,
                  const uint32_t *dst, const uint32_t *w, const int64_t *add_off,
                  const int64_t *del_off, const int64_t *del_ids, uint32_t source,
                  uint32_t win_begin, uint32_t win_len, uint32_t *r_cap, uint32_t *r_cup) {
    if (source >= V || win_len == 0 || (uint64_t)win_begin + win_len > S) return -2;
    if (type < 0 || type > 3) return -2;
    edge_log lg = {V, S, n_inst, src, dst, w, add_off, del_off, del_ids};
    size_t n = n_inst ? n_inst : 1;
    unsigned char *alive = (unsigned char *)malloc(n);
    unsigned char *in_all = (unsigned char *)malloc(n);
    unsigned char *in_any = (unsigned char *)malloc(n);
    int rc = -1;
    if (!alive || !in_all || !in_any) goto done;
    memset(in_all, 1, n_inst);
    memset(in_any, 0, n_inst);
    for (uint32_t i = win_begin; i < win_begin + win_len; ++i) {
        replay_to(&lg, i, alive);
        for (uint64_t k = 0; k < n_inst; ++k) {
            in_all[k] = (unsigned char)(in_all[k] & alive[k]);
            in_any[k] = (unsigned char)(in_any[k] | alive[k]);
        }
    }
    rc = solve_kept(&lg, in_all, type, source, r_cap);
    if (rc == 0) rc = solve_kept(&lg, in_any, type, source, r_cup);
done:
    free(alive);
    free(in_all);
    free(in_any);
    return rc;
}

/* ------------------------------------------------------------------ */
/* live intervals: one replay for many windows                          */
/* ------------------------------------------------------------------ */

/* Snapshot s is the graph after step s (Section 2): the step's deletions,
 * then its additions.  So instance k is live exactly in the snapshots
 * [t_add[k], t_del[k]): added in step t_add[k], deleted in step t_del[k]
 * (S if never deleted; an instance that is never added gets t_add = S, an
 * empty interval).  One pass over the steps in order records both. */
int oracle_live_intervals(uint32_t V, uint32_t S, uint64_t n_inst, const uint32_t *src,
                          const uint32_t *dst, const uint32_t *w, const int64_t *add_off,
                          const int64_t *del_off, const int64_t *del_ids, uint32_t *t_add,
                          uint32_t *t_del) {
    (void)V;
    (void)src;
    (void)dst;
    (void)w;
    for (uint64_t k = 0; k < n_inst; ++k) {
        t_add[k] = S;
        t_del[k] = S;
    }
    for (uint32_t s = 0; s < S; ++s) {
        for (int64_t j = del_off[s]; j < del_off[s + 1]; ++j) {
            const int64_t k = del_ids[j];
            if (k < 0 || (uint64_t)k >= n_inst) return -2;
            t_del[k] = s;
        }
        for (int64_t k = add_off[s]; k < add_off[s + 1]; ++k) {
            if (k < 0 || (uint64_t)k >= n_inst) return -2;
            t_add[k] = s;
        }
    }
    return 0;
}

/* CSR of the window [win_begin, win_begin+win_len) as Section 3 Step 1
 * defines its graphs, from live intervals: kind 0 = the intersection graph
 * (instances live in every window snapshot: added by win_begin, not deleted
 * before win_begin+win_len), kind 1 = the union graph (live in at least one
 * window snapshot).  A window of one snapshot gives that snapshot. */
int oracle_window_csr(uint32_t V, uint32_t S, uint64_t n_inst, const uint32_t *src,
                      const uint32_t *dst, const uint32_t *w, const uint32_t *t_add,
                      const uint32_t *t_del, uint32_t win_begin, uint32_t win_len, int kind,
                      uint64_t *row_ptr, uint32_t **col, uint32_t **wout) {
    if (win_len == 0 || (uint64_t)win_begin + win_len > S || (kind != 0 && kind != 1)) return -2;
    edge_log lg = {V, S, n_inst, src, dst, w, NULL, NULL, NULL};
    unsigned char *keep = (unsigned char *)malloc(n_inst ? n_inst : 1);
    if (!keep) return -1;
    const uint32_t end = win_begin + win_len;
    for (uint64_t k = 0; k < n_inst; ++k) {
        if (kind == 0) keep[k] = (unsigned char)(t_add[k] <= win_begin && t_del[k] >= end);
        else keep[k] = (unsigned char)(t_add[k] < t_del[k] && t_add[k] < end && t_del[k] > win_begin);
    }
    int rc = materialise(&lg, keep, row_ptr, col, wout);
    free(keep);
    return rc;
}
