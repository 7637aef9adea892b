/*
 * KADABRA oracle: a plain, single-threaded CPU statement of the sampling method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or run
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (arXiv 1903.09422, van der Grinten, Angriman, Meyerhenke):
 *   - Algorithm 1 (Section 2.1): the generic adaptive-sampling loop, with the
 *     stopping condition checked only on consistent states (Section 2.1).
 *   - Section 2.3: KADABRA.  sample() draws a uniform vertex pair (s, t) and a
 *     uniform shortest s-t path; the estimate is b~(v) = (1/tau) sum_i x_i(v).
 *   - Appendix B: the closed forms of f and g and the stop rule f <= eps and
 *     g <= eps for every vertex.
 *   - Appendix C.1: same-component check before searching; the path is rebuilt
 *     from G and the distance vectors, not from a predecessor graph.
 *   - Section 5: KADABRA also covers directed graphs.  A directed graph is given
 *     with its in-arc rows as well; the s side searches along out-arcs, the t
 *     side along in-arcs, components are the weak ones, and the vertex-diameter
 *     bound goes through the strongly connected components (a READING below).
 *   - Appendix D.2 (indexed frames): random numbers depend on a sample index,
 *     not on a thread, and a stop check sees a fixed prefix of samples, which
 *     makes the result deterministic.
 *
 * The paper defers several details to the original KADABRA paper (Section 2.3:
 * omega, delta_L/delta_U, the balanced bidirectional BFS).  Each reading taken
 * here is marked READING below; the CUDA library implements the same readings.
 *
 * Arithmetic conventions: sigma (shortest-path counts) saturates at 2^64-1;
 * floating point is IEEE binary64, built with -ffp-contract=off so that no
 * fused multiply-add changes the rounding of f, g, L or omega.
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors; Lemire's bounded
 * draw exhaustively for small ranges; sigma and distance against brute-force
 * shortest-path enumeration; path uniformity by chi-square; increments equal
 * path length - 1; estimates against exact Brandes BC within (eps, delta);
 * closed forms on path and star graphs; f and g at hand-evaluated points.
 * The omega constant and the calibration rule have no printed values in the
 * paper: parity unpinned for those two, beyond self-consistency checks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_U64MAX 0xffffffffffffffffULL

/* ------------------------------------------------------------------ Philox */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies with a Weyl key
 * schedule.  READING: the paper only says each frame's generator is reseeded by
 * its index (Appendix D.2); here every sample has its own counter. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* The random stream of one sample: key = seed, counter = (index, block, domain).
 * Each Philox block yields two 64-bit words (low word first), used in order. */
typedef struct {
    uint32_t key[2];
    uint64_t index;
    uint32_t domain;
    uint32_t block;
    uint64_t buf[2];
    int pos; /* 0, 1 = next word in buf; 2 = buffer empty */
    uint64_t words;
} orc_stream;

static void stream_init(orc_stream *st, uint64_t seed, uint64_t index, uint32_t domain) {
    st->key[0] = (uint32_t)seed;
    st->key[1] = (uint32_t)(seed >> 32);
    st->index = index;
    st->domain = domain;
    st->block = 0;
    st->pos = 2;
    st->words = 0;
}

static uint64_t stream_next(orc_stream *st) {
    if (st->pos == 2) {
        uint32_t ctr[4] = {(uint32_t)st->index, (uint32_t)(st->index >> 32), st->block, st->domain};
        uint32_t o[4];
        orc_philox4x32_10(ctr, st->key, o);
        st->buf[0] = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
        st->buf[1] = (uint64_t)o[2] | ((uint64_t)o[3] << 32);
        st->block++;
        st->pos = 0;
    }
    st->words++;
    return st->buf[st->pos++];
}

/* Uniform integer in [0, m), m >= 1: Lemire's multiply-and-reject
 * (ACM TOMACS 29(1), 2019).  Always consumes at least one word. */
static uint64_t stream_uniform(orc_stream *st, uint64_t m) {
    uint64_t x = stream_next(st);
    unsigned __int128 p = (unsigned __int128)x * m;
    uint64_t lo = (uint64_t)p;
    if (lo < m) {
        uint64_t thresh = (0 - m) % m; /* (2^64 - m) mod m */
        while (lo < thresh) {
            x = stream_next(st);
            p = (unsigned __int128)x * m;
            lo = (uint64_t)p;
        }
    }
    return (uint64_t)(p >> 64);
}

/* Test hook: the first `count` bounded draws of one stream. */
void orc_stream_draws(uint64_t seed, uint64_t index, uint32_t domain, const uint64_t *ms, int64_t count,
                      uint64_t *out, uint64_t *words_used) {
    orc_stream st;
    stream_init(&st, seed, index, domain);
    for (int64_t i = 0; i < count; i++) out[i] = stream_uniform(&st, ms[i]);
    if (words_used) *words_used = st.words;
}

void orc_stream_words(uint64_t seed, uint64_t index, uint32_t domain, int64_t count, uint64_t *out) {
    orc_stream st;
    stream_init(&st, seed, index, domain);
    for (int64_t i = 0; i < count; i++) out[i] = stream_next(&st);
}

/* ---------------------------------------------------------- saturating sigma */
static uint64_t sat_add(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    return (s < a) ? ORC_U64MAX : s;
}

static uint64_t sat_mul(uint64_t a, uint64_t b) {
    unsigned __int128 p = (unsigned __int128)a * b;
    return (p >> 64) ? ORC_U64MAX : (uint64_t)p;
}

/* ------------------------------------------------------------------ graph */
/* A graph is given by the rows each BFS side expands along: rp[0]/col[0] are
 * the out-arcs (the s side searches forward from s), rp[1]/col[1] the in-arcs
 * (the t side searches backward from t).  An undirected graph passes its one
 * symmetric CSR for both.  The trace-back of side z walks the rows of the other
 * side, 1 - z: from a vertex toward s over its in-arcs, toward t over its
 * out-arcs. */
typedef struct {
    int32_t n;
    const int32_t *rp[2];
    const int32_t *col[2];
} orc_graph;

static int32_t deg(const orc_graph *g, int z, int32_t v) { return g->rp[z][v + 1] - g->rp[z][v]; }

static void graph_init(orc_graph *g, int32_t n, const int32_t *rp, const int32_t *col, const int32_t *rpT,
                       const int32_t *colT) {
    g->n = n;
    g->rp[0] = rp;
    g->col[0] = col;
    g->rp[1] = rpT ? rpT : rp;
    g->col[1] = rpT ? colT : col;
}

/* The in-arc CSR of a directed graph: row v lists every u with an arc u->v, in
 * ascending u (a counting sort of the arcs by head, taken in tail order). */
void orc_transpose(int32_t n, const int32_t *rp, const int32_t *col, int32_t *rpT, int32_t *colT) {
    int32_t *fill = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!fill) return;
    for (int32_t v = 0; v <= n; v++) rpT[v] = 0;
    for (int32_t e = 0; e < rp[n]; e++) rpT[col[e] + 1]++;
    for (int32_t v = 0; v < n; v++) rpT[v + 1] += rpT[v];
    for (int32_t v = 0; v <= n; v++) fill[v] = rpT[v];
    for (int32_t u = 0; u < n; u++)
        for (int32_t e = rp[u]; e < rp[u + 1]; e++) colT[fill[col[e]]++] = u;
    free(fill);
}

/* Connected components by BFS in ascending id order (Appendix C.1 footnote:
 * components are computed during preprocessing); for a directed graph the weak
 * components (arcs followed both ways), since no path joins two of them.
 * comp[v] = index of v's component, numbered by smallest member.  Returns the
 * component count. */
static int32_t components(const orc_graph *g, int32_t *comp) {
    const int32_t n = g->n;
    const int sides = (g->rp[1] != g->rp[0]) ? 2 : 1;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -1;
    for (int32_t v = 0; v < n; v++) comp[v] = -1;
    int32_t nc = 0;
    for (int32_t r = 0; r < n; r++) {
        if (comp[r] >= 0) continue;
        int32_t head = 0, tail = 0;
        queue[tail++] = r;
        comp[r] = nc;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int z = 0; z < sides; z++)
                for (int32_t e = g->rp[z][u]; e < g->rp[z][u + 1]; e++) {
                    int32_t w = g->col[z][e];
                    if (comp[w] < 0) {
                        comp[w] = nc;
                        queue[tail++] = w;
                    }
                }
        }
        nc++;
    }
    free(queue);
    return nc;
}

int32_t orc_components(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *rpT, const int32_t *colT,
                       int32_t *comp) {
    orc_graph g;
    graph_init(&g, n, rp, col, rpT, colT);
    return components(&g, comp);
}

/* Strongly connected components of a directed graph (Kosaraju: a depth-first
 * search along the out-arcs lists the vertices by finishing time; searches
 * along the in-arcs, started in decreasing finishing time, then each collect
 * one component).  scc[v] = index of v's component in the order found.
 * Returns the component count. */
int32_t orc_scc(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *rpT, const int32_t *colT,
                int32_t *scc) {
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *stk = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *pos = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    if (!order || !stk || !pos || !seen) {
        free(order);
        free(stk);
        free(pos);
        free(seen);
        return -1;
    }
    int32_t norder = 0;
    for (int32_t r = 0; r < n; r++) {
        if (seen[r]) continue;
        int32_t top = 0;
        stk[top] = r;
        pos[top] = rp[r];
        seen[r] = 1;
        while (top >= 0) {
            int32_t v = stk[top];
            if (pos[top] < rp[v + 1]) {
                int32_t w = col[pos[top]++];
                if (!seen[w]) {
                    seen[w] = 1;
                    top++;
                    stk[top] = w;
                    pos[top] = rp[w];
                }
            } else {
                order[norder++] = v; /* v finishes */
                top--;
            }
        }
    }
    for (int32_t v = 0; v < n; v++) scc[v] = -1;
    int32_t nscc = 0;
    for (int32_t i = n - 1; i >= 0; i--) {
        int32_t r = order[i];
        if (scc[r] >= 0) continue;
        int32_t head = 0, tail = 0;
        stk[tail++] = r;
        scc[r] = nscc;
        while (head < tail) {
            int32_t u = stk[head++];
            for (int32_t e = rpT[u]; e < rpT[u + 1]; e++) {
                int32_t w = colT[e];
                if (scc[w] < 0) {
                    scc[w] = nscc;
                    stk[tail++] = w;
                }
            }
        }
        nscc++;
    }
    free(order);
    free(stk);
    free(pos);
    free(seen);
    return nscc;
}

/* READING (Section 2.3: "mostly computing an upper bound on the diameter"):
 * in every component, BFS from its vertex of largest degree (smallest id on
 * ties); the component's diameter is at most 2 ecc(v0).  The vertex-diameter
 * bound is VD = max over components of 2 ecc(v0) + 1. */
static int32_t vd_bound_undirected(const orc_graph *g) {
    const int32_t n = g->n;
    const int32_t *rp = g->rp[0], *col = g->col[0];
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!comp || !dist || !queue) {
        free(comp);
        free(dist);
        free(queue);
        return -1;
    }
    int32_t nc = components(g, comp);
    int32_t *root = (int32_t *)malloc((size_t)nc * sizeof(int32_t));
    for (int32_t c = 0; c < nc; c++) root[c] = -1;
    for (int32_t v = 0; v < n; v++) {
        int32_t c = comp[v];
        if (root[c] < 0 || deg(g, 0, v) > deg(g, 0, root[c])) root[c] = v;
    }
    for (int32_t v = 0; v < n; v++) dist[v] = -1;
    int32_t vd = 1;
    for (int32_t c = 0; c < nc; c++) {
        int32_t head = 0, tail = 0, ecc = 0;
        queue[tail++] = root[c];
        dist[root[c]] = 0;
        while (head < tail) {
            int32_t u = queue[head++];
            if (dist[u] > ecc) ecc = dist[u];
            for (int32_t e = rp[u]; e < rp[u + 1]; e++) {
                int32_t w = col[e];
                if (dist[w] < 0) {
                    dist[w] = dist[u] + 1;
                    queue[tail++] = w;
                }
            }
        }
        if (2 * ecc + 1 > vd) vd = 2 * ecc + 1;
    }
    free(root);
    free(comp);
    free(dist);
    free(queue);
    return vd;
}

/* READING (directed graphs; Section 5 only says that KADABRA covers them, and
 * the bound must hold for directed shortest paths, which 2 ecc does not bound):
 * a shortest path never returns to a strongly connected component it has left,
 * so it crosses a chain S_1 -> ... -> S_k of the components' DAG and spends a
 * shortest sub-path inside each.  Inside S, with r_S its vertex of largest
 * out- plus in-degree (smallest id on ties), such a sub-path x..y has
 * d(x, y) <= d(x, r_S) + d(r_S, y), so at most w(S) = min(|S|, ecc_in(r_S) +
 * ecc_out(r_S) + 1) vertices (eccentricities within S).  VD = the heaviest chain:
 * max over S of B(S), B(S) = w(S) + max(0, max over arcs S -> S' of B(S')). */
static int32_t vd_bound_directed(const orc_graph *g) {
    const int32_t n = g->n;
    int32_t *scc = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!scc || !dist || !queue) {
        free(scc);
        free(dist);
        free(queue);
        return -1;
    }
    int32_t ns = orc_scc(n, g->rp[0], g->col[0], g->rp[1], g->col[1], scc);
    size_t nsz = (ns > 0) ? (size_t)ns : 1;
    int32_t *root = (int32_t *)malloc(nsz * sizeof(int32_t));
    int32_t *size = (int32_t *)calloc(nsz, sizeof(int32_t));
    int32_t *ecc = (int32_t *)calloc(nsz, sizeof(int32_t)); /* ecc_out + ecc_in */
    int64_t *B = (int64_t *)malloc(nsz * sizeof(int64_t));
    int64_t *w = (int64_t *)malloc(nsz * sizeof(int64_t));
    if (ns < 0 || !root || !size || !ecc || !B || !w) {
        free(scc);
        free(dist);
        free(queue);
        free(root);
        free(size);
        free(ecc);
        free(B);
        free(w);
        return -1;
    }
    for (int32_t c = 0; c < ns; c++) root[c] = -1;
    for (int32_t v = 0; v < n; v++) {
        int32_t c = scc[v];
        size[c]++;
        if (root[c] < 0 || deg(g, 0, v) + deg(g, 1, v) > deg(g, 0, root[c]) + deg(g, 1, root[c])) root[c] = v;
    }
    /* z = 0: distances from r_S along out-arcs; z = 1: to r_S, along in-arcs */
    for (int z = 0; z < 2; z++) {
        for (int32_t v = 0; v < n; v++) dist[v] = -1;
        for (int32_t c = 0; c < ns; c++) {
            int32_t head = 0, tail = 0, far = 0;
            queue[tail++] = root[c];
            dist[root[c]] = 0;
            while (head < tail) {
                int32_t u = queue[head++];
                if (dist[u] > far) far = dist[u];
                for (int32_t e = g->rp[z][u]; e < g->rp[z][u + 1]; e++) {
                    int32_t x = g->col[z][e];
                    if (scc[x] == c && dist[x] < 0) {
                        dist[x] = dist[u] + 1;
                        queue[tail++] = x;
                    }
                }
            }
            ecc[c] += far;
        }
    }
    for (int32_t c = 0; c < ns; c++) {
        w[c] = (ecc[c] + 1 < size[c]) ? ecc[c] + 1 : size[c];
        B[c] = w[c];
    }
    /* the heaviest chain, by relaxing every arc between components until no
     * value changes (the components' graph is acyclic, so this ends) */
    for (int changed = 1; changed;) {
        changed = 0;
        for (int32_t u = 0; u < n; u++)
            for (int32_t e = g->rp[0][u]; e < g->rp[0][u + 1]; e++) {
                int32_t su = scc[u], sv = scc[g->col[0][e]];
                if (su != sv && w[su] + B[sv] > B[su]) {
                    B[su] = w[su] + B[sv];
                    changed = 1;
                }
            }
    }
    int64_t vd = 1;
    for (int32_t c = 0; c < ns; c++)
        if (B[c] > vd) vd = B[c];
    free(scc);
    free(dist);
    free(queue);
    free(root);
    free(size);
    free(ecc);
    free(B);
    free(w);
    return (int32_t)vd;
}

/* BFS over the out-arc rows from src; dist[] must be -1 outside.  Returns the
 * number of vertices reached (all stored in queue[]). */
static int32_t bfs_from(const orc_graph *g, int32_t src, int32_t *dist, int32_t *queue) {
    int32_t head = 0, tail = 0;
    queue[tail++] = src;
    dist[src] = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t e = g->rp[0][u]; e < g->rp[0][u + 1]; e++) {
            int32_t w = g->col[0][e];
            if (dist[w] < 0) {
                dist[w] = dist[u] + 1;
                queue[tail++] = w;
            }
        }
    }
    return tail;
}

/* The farthest of the `cnt` vertices in list[] by dist[] (smallest id on ties). */
static int32_t farthest(const int32_t *list, int32_t cnt, const int32_t *dist) {
    int32_t best = list[0];
    for (int32_t i = 1; i < cnt; i++) {
        int32_t v = list[i];
        if (dist[v] > dist[best] || (dist[v] == dist[best] && v < best)) best = v;
    }
    return best;
}

/* READING (opt-in; Section 2.3 asks only for an upper bound on the diameter, and
 * any vertex x gives diam <= 2 ecc(x)): a tighter bound per component from a
 * double sweep.  a = the vertex farthest from v0, b = the vertex farthest from
 * a (smallest id on ties); d = d(a, b) is a lower bound on the diameter.  m =
 * the midpoint of an a-b shortest path nearest v0: among the x with
 * d(a,x) + d(x,b) = d and d(a,x) = ceil(d/2), the one of smallest d(v0,x),
 * then smallest id.  The component's bound is 2 min(ecc(v0), ecc(m)) + 1, and
 * VD the maximum over components. */
int32_t orc_vd_bound_tight(int32_t n, const int32_t *rp, const int32_t *col) {
    orc_graph g;
    graph_init(&g, n, rp, col, NULL, NULL);
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *d0 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *da = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *db = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *dm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *members = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t vd = 1;
    if (!comp || !d0 || !da || !db || !dm || !queue || !members) {
        vd = -1;
        goto out;
    }
    int32_t nc = components(&g, comp);
    /* v0 of each component: its vertex of largest degree, smallest id on ties
     * (kept in dm[c] until the component's turn; components are numbered below n) */
    for (int32_t c = 0; c < nc; c++) dm[c] = -1;
    for (int32_t v = 0; v < n; v++)
        if (dm[comp[v]] < 0 || deg(&g, 0, v) > deg(&g, 0, dm[comp[v]])) dm[comp[v]] = v;
    for (int32_t c = 0; c < nc; c++) queue[c] = dm[c];
    for (int32_t v = 0; v < n; v++) d0[v] = da[v] = db[v] = dm[v] = -1;
    int32_t *v0s = (int32_t *)malloc((size_t)nc * sizeof(int32_t));
    if (!v0s) {
        vd = -1;
        goto out;
    }
    memcpy(v0s, queue, (size_t)nc * sizeof(int32_t));
    for (int32_t c = 0; c < nc; c++) {
        int32_t v0 = v0s[c];
        int32_t cnt = bfs_from(&g, v0, d0, members);
        int32_t a = farthest(members, cnt, d0);
        int32_t ecc0 = d0[a];
        bfs_from(&g, a, da, queue);
        int32_t b = farthest(members, cnt, da);
        int32_t d = da[b];
        bfs_from(&g, b, db, queue);
        int32_t half = (d + 1) / 2, m = -1;
        for (int32_t i = 0; i < cnt; i++) {
            int32_t x = members[i];
            if (da[x] + db[x] != d || da[x] != half) continue;
            if (m < 0 || d0[x] < d0[m] || (d0[x] == d0[m] && x < m)) m = x;
        }
        bfs_from(&g, m, dm, queue);
        int32_t eccm = dm[farthest(members, cnt, dm)];
        int32_t e = (eccm < ecc0) ? eccm : ecc0;
        if (2 * e + 1 > vd) vd = 2 * e + 1;
    }
    free(v0s);
out:
    free(comp);
    free(d0);
    free(da);
    free(db);
    free(dm);
    free(queue);
    free(members);
    return vd;
}

/* rpT == NULL: undirected (one symmetric CSR); else directed with in-arcs rpT/colT. */
int32_t orc_vd_bound(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *rpT, const int32_t *colT) {
    orc_graph g;
    graph_init(&g, n, rp, col, rpT, colT);
    return rpT ? vd_bound_directed(&g) : vd_bound_undirected(&g);
}

static int floor_log2_u64(uint64_t x) {
    int r = -1;
    while (x) {
        x >>= 1;
        r++;
    }
    return r;
}

/* READING (Section 2.3: omega is "a maximal number of samples" derived from
 * the diameter bound): omega = ceil((0.5/eps^2) (floor(log2(max(VD-2,1))) + 1
 * + ln(2/delta))), the sample bound of the KADABRA / Riondato-Kornaropoulos
 * line with half of delta spent on it. */
uint64_t orc_omega(int32_t vd, double eps, double delta) {
    int64_t a = (int64_t)vd - 2;
    if (a < 1) a = 1;
    double c = 0.5 / (eps * eps);
    double inner = ((double)floor_log2_u64((uint64_t)a) + 1.0) + log(2.0 / delta);
    return (uint64_t)ceil(c * inner);
}

/* READING: calibration length tau0 = N * ceil(max(1, ceil(omega/div)) / N). */
uint64_t orc_calib_samples(uint64_t omega, uint32_t epoch, uint32_t calib_div) {
    uint64_t a = (omega + calib_div - 1) / calib_div;
    if (a < 1) a = 1;
    return ((a + epoch - 1) / epoch) * epoch;
}

/* ---------------------------------------------------------------- f and g */
/* Appendix B: f and g with L = log(1/delta_L(v)) = log(1/delta_U(v)).
 * READING: "log" is the natural logarithm; the operation order below is fixed. */
double orc_f(uint64_t c, double L, uint64_t tau, uint64_t omega) {
    double T = (double)tau, W = (double)omega;
    double b = (double)c / T;
    double q = W / T;
    double a = (1.0 / 3.0) - q;
    double x = ((2.0 * b) * W) / L;
    return (L / T) * (a + sqrt(a * a + x));
}

double orc_g(uint64_t c, double L, uint64_t tau, uint64_t omega) {
    double T = (double)tau, W = (double)omega;
    double b = (double)c / T;
    double q = W / T;
    double a = (1.0 / 3.0) + q;
    double x = ((2.0 * b) * W) / L;
    return (L / T) * (a + sqrt(a * a + x));
}

/* READING (Section 2.3 requires only sum_v delta_L(v) + delta_U(v) <= delta):
 * delta_L(v) = delta_U(v) = exp(-L), where L solves g(b0, exp(-L), omega, tau*) = eps
 * for the calibration estimate b0:  L = tau* eps^2 / (2 b0 omega / tau* + 2 eps (1/3 + omega/tau*)). */
double orc_L(double b0, double tstar, double eps, uint64_t omega) {
    double W = (double)omega;
    double num = tstar * (eps * eps);
    double den = ((2.0 * b0) * W) / tstar + (2.0 * eps) * ((1.0 / 3.0) + W / tstar);
    return num / den;
}

/* S(tau*) = sum_c hist[c] * 2 exp(-L(c/tau0, tau*)), ascending c. */
static double calib_mass(const uint64_t *hist, uint64_t tau0, double tstar, double eps, uint64_t omega) {
    double acc = 0.0;
    for (uint64_t c = 0; c <= tau0; c++) {
        if (hist[c] == 0) continue;
        double L = orc_L((double)c / (double)tau0, tstar, eps, omega);
        acc += (double)hist[c] * (2.0 * exp(-L));
    }
    return acc;
}

/* READING: tau* by bisection so that S(tau*) <= delta/2 (the other half of
 * delta is spent on omega).  hi starts at omega and doubles until it holds;
 * lo = 1; exactly 100 halvings; the result is the final hi. */
double orc_tau_star(const uint64_t *hist, uint64_t tau0, double eps, double delta, uint64_t omega) {
    double target = 0.5 * delta;
    double hi = (double)omega, lo = 1.0;
    for (int i = 0; i < 4096 && calib_mass(hist, tau0, hi, eps, omega) > target; i++) hi = hi * 2.0;
    for (int i = 0; i < 100; i++) {
        double mid = 0.5 * (lo + hi);
        if (calib_mass(hist, tau0, mid, eps, omega) <= target)
            hi = mid;
        else
            lo = mid;
    }
    return hi;
}

/* ------------------------------------------------------------ one sample */
typedef struct {
    uint64_t expanded;   /* frontier vertices expanded */
    uint64_t scanned;    /* arcs scanned by expansions (frontier degree sums) */
    uint64_t labelled;   /* vertices labelled in rounds that did not meet */
    uint64_t pred_arcs;  /* arcs from the frontier into the next level or M */
    uint64_t trace_arcs; /* arcs scanned by the trace-back */
    uint64_t increments; /* interior path vertices */
} orc_counters;

typedef struct {
    const orc_graph *g;
    const int32_t *comp;
    int32_t *dist[2];   /* per side, -1 = unlabelled */
    uint64_t *sigma[2]; /* per side */
    uint64_t *sigma_m;  /* sigma of the expanding side for members of M */
    uint8_t *in_m;
    int32_t *touched; /* every labelled vertex, for the reset */
    int32_t ntouched;
    int32_t *front[2], *next;
    int32_t *mlist;
} orc_ws;

static int ws_init(orc_ws *w, const orc_graph *g, const int32_t *comp) {
    size_t n = (size_t)g->n;
    memset(w, 0, sizeof(*w));
    w->g = g;
    w->comp = comp;
    w->dist[0] = (int32_t *)malloc(n * sizeof(int32_t));
    w->dist[1] = (int32_t *)malloc(n * sizeof(int32_t));
    w->sigma[0] = (uint64_t *)calloc(n, sizeof(uint64_t));
    w->sigma[1] = (uint64_t *)calloc(n, sizeof(uint64_t));
    w->sigma_m = (uint64_t *)calloc(n, sizeof(uint64_t));
    w->in_m = (uint8_t *)calloc(n, 1);
    w->touched = (int32_t *)malloc(n * sizeof(int32_t));
    w->front[0] = (int32_t *)malloc(n * sizeof(int32_t));
    w->front[1] = (int32_t *)malloc(n * sizeof(int32_t));
    w->next = (int32_t *)malloc(n * sizeof(int32_t));
    w->mlist = (int32_t *)malloc(n * sizeof(int32_t));
    if (!w->dist[0] || !w->dist[1] || !w->sigma[0] || !w->sigma[1] || !w->sigma_m || !w->in_m || !w->touched ||
        !w->front[0] || !w->front[1] || !w->next || !w->mlist)
        return -1;
    for (size_t v = 0; v < n; v++) w->dist[0][v] = w->dist[1][v] = -1;
    return 0;
}

static void ws_free(orc_ws *w) {
    free(w->dist[0]);
    free(w->dist[1]);
    free(w->sigma[0]);
    free(w->sigma[1]);
    free(w->sigma_m);
    free(w->in_m);
    free(w->touched);
    free(w->front[0]);
    free(w->front[1]);
    free(w->next);
    free(w->mlist);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* One step of the trace-back (Appendix C.1: rebuild the path from G and the
 * distance vector): at cur, at distance d >= 1 on side z with path count
 * sig_cur, draw r uniform in [0, sig_cur) and take the first neighbour p, in
 * CSR (ascending) order, at distance d-1 on side z whose running sum of sigma
 * exceeds r.  This picks p with probability sigma(p)/sigma(cur).  The
 * neighbours toward root z are cur's row on the other side (1 - z): the tails
 * of its in-arcs toward s, the heads of its out-arcs toward t. */
static int32_t trace_step(orc_ws *w, orc_stream *st, int z, int32_t cur, int32_t d, uint64_t sig_cur,
                          orc_counters *ctr) {
    const orc_graph *g = w->g;
    uint64_t r = stream_uniform(st, sig_cur);
    uint64_t cum = 0;
    const int32_t *rp = g->rp[1 - z], *col = g->col[1 - z];
    for (int32_t e = rp[cur]; e < rp[cur + 1]; e++) {
        int32_t p = col[e];
        if (w->dist[z][p] != d - 1) continue;
        cum = sat_add(cum, w->sigma[z][p]);
        if (cum > r) {
            if (ctr) ctr->trace_arcs += (uint64_t)(e - rp[cur] + 1);
            return p;
        }
    }
    return -1; /* unreachable for a consistent state */
}

/* Section 2.3 sample(): given the pair (s, t) and the stream positioned after
 * the pair draw, draw a uniform shortest s-t path.  Returns D = d(s,t) (0 when
 * s and t are disconnected) and writes the D-1 interior vertices to path[] in
 * order of distance from s. */
static int32_t sample_path(orc_ws *w, orc_stream *st, int32_t s, int32_t t, int32_t *path, int32_t cap,
                           uint64_t *sigma_st_out, int *overflow, orc_counters *ctr) {
    const orc_graph *g = w->g;
    *overflow = 0;
    *sigma_st_out = 0;
    /* Appendix C.1: skip pairs in different components. */
    if (w->comp[s] != w->comp[t]) return 0;

    int32_t root[2] = {s, t};
    int32_t lev[2] = {0, 0};
    int32_t flen[2] = {1, 1};
    uint64_t dsum[2];
    w->ntouched = 0;
    for (int z = 0; z < 2; z++) {
        w->dist[z][root[z]] = 0;
        w->sigma[z][root[z]] = 1;
        w->front[z][0] = root[z];
        w->touched[w->ntouched++] = root[z];
        dsum[z] = (uint64_t)deg(g, z, root[z]);
    }
    int32_t nm = 0, D = 0, X = 0;
    /* READING (balanced bidirectional BFS; details deferred to the original
     * KADABRA paper in Section 2.3): each round expands the side whose current
     * frontier has the smaller degree sum, the s side on ties.  The first round
     * that reaches a vertex labelled by the other side is the last one.  The s
     * side expands along out-arcs and the t side along in-arcs (the same rows
     * when undirected), and degrees are counted in the expanding direction. */
    for (;;) {
        X = (dsum[0] <= dsum[1]) ? 0 : 1;
        int Y = 1 - X;
        if (flen[X] == 0) break; /* no path (within a weak component of a directed graph) */
        int32_t nnext = 0;
        int met = 0;
        uint64_t pred_next = 0, pred_m = 0;
        if (ctr) {
            ctr->expanded += (uint64_t)flen[X];
            ctr->scanned += dsum[X];
        }
        for (int32_t i = 0; i < flen[X]; i++) {
            int32_t u = w->front[X][i];
            uint64_t su = w->sigma[X][u];
            for (int32_t e = g->rp[X][u]; e < g->rp[X][u + 1]; e++) {
                int32_t v = g->col[X][e];
                if (w->dist[Y][v] >= 0) {
                    /* v lies in the other side's frontier (level lev[Y]). */
                    met = 1;
                    pred_m++;
                    if (!w->in_m[v]) {
                        w->in_m[v] = 1;
                        w->mlist[nm++] = v;
                    }
                    w->sigma_m[v] = sat_add(w->sigma_m[v], su);
                } else if (w->dist[X][v] < 0) {
                    w->dist[X][v] = lev[X] + 1;
                    w->sigma[X][v] = su;
                    w->next[nnext++] = v;
                    w->touched[w->ntouched++] = v;
                    pred_next++;
                } else if (w->dist[X][v] == lev[X] + 1) {
                    w->sigma[X][v] = sat_add(w->sigma[X][v], su);
                    pred_next++;
                }
            }
        }
        /* Work counters count what any correct order of expansion must do: the
         * arcs into M in the round that meets, the next level otherwise. */
        if (ctr) ctr->pred_arcs += met ? pred_m : pred_next;
        if (met) {
            D = lev[X] + 1 + lev[Y];
            break;
        }
        if (ctr) ctr->labelled += (uint64_t)nnext;
        lev[X]++;
        flen[X] = nnext;
        memcpy(w->front[X], w->next, (size_t)nnext * sizeof(int32_t));
        dsum[X] = 0;
        for (int32_t i = 0; i < nnext; i++) dsum[X] += (uint64_t)deg(g, X, w->next[i]);
    }

    int32_t ninterior = 0;
    if (D > 0) {
        int Y = 1 - X;
        /* Meeting draw: sigma_st = sum over M of sigma_X(m) sigma_Y(m); pick m with
         * probability proportional to its term, walking M in ascending id. */
        qsort(w->mlist, (size_t)nm, sizeof(int32_t), cmp_i32);
        uint64_t sst = 0;
        for (int32_t i = 0; i < nm; i++)
            sst = sat_add(sst, sat_mul(w->sigma_m[w->mlist[i]], w->sigma[Y][w->mlist[i]]));
        *sigma_st_out = sst;
        if (sst == ORC_U64MAX) *overflow = 1;
        uint64_t r = stream_uniform(st, sst);
        uint64_t cum = 0;
        int32_t mid = -1;
        for (int32_t i = 0; i < nm; i++) {
            cum = sat_add(cum, sat_mul(w->sigma_m[w->mlist[i]], w->sigma[Y][w->mlist[i]]));
            if (cum > r) {
                mid = w->mlist[i];
                break;
            }
        }
        /* Distances and path counts of the meeting vertex on both sides. */
        int32_t dm[2];
        uint64_t sm[2];
        dm[X] = lev[X] + 1;
        sm[X] = w->sigma_m[mid];
        dm[Y] = lev[Y];
        sm[Y] = w->sigma[Y][mid];
        ninterior = D - 1;
        if (ninterior > cap) ninterior = -1; /* caller's buffer too small */
        if (ninterior >= 0) {
            int32_t ds = dm[0];
            if (ds >= 1 && ds <= D - 1) path[ds - 1] = mid;
            /* s side first, from the meeting vertex toward s. */
            int32_t cur = mid, d = dm[0];
            uint64_t sc = sm[0];
            while (d >= 1) {
                int32_t p = trace_step(w, st, 0, cur, d, sc, ctr);
                d--;
                if (d >= 1) path[d - 1] = p;
                cur = p;
                sc = w->sigma[0][p];
            }
            /* then the t side, from the meeting vertex toward t. */
            cur = mid;
            d = dm[1];
            sc = sm[1];
            while (d >= 1) {
                int32_t p = trace_step(w, st, 1, cur, d, sc, ctr);
                d--;
                if (d >= 1) path[D - d - 1] = p;
                cur = p;
                sc = w->sigma[1][p];
            }
            if (ctr) ctr->increments += (uint64_t)ninterior;
        }
        for (int32_t i = 0; i < nm; i++) {
            w->in_m[w->mlist[i]] = 0;
            w->sigma_m[w->mlist[i]] = 0;
        }
    }
    /* Reset only what this sample labelled (Appendix C.1 avoids a Theta(|V|)
     * reset per sample; here the list of labelled vertices serves that purpose). */
    for (int32_t i = 0; i < w->ntouched; i++) {
        int32_t v = w->touched[i];
        w->dist[0][v] = w->dist[1][v] = -1;
        w->sigma[0][v] = w->sigma[1][v] = 0;
    }
    return (ninterior < 0) ? -1 : D;
}

/* Pair draw (Section 2.3: (s, t) uniform over ordered pairs with s != t). */
static void draw_pair(orc_stream *st, int32_t n, int32_t *s, int32_t *t) {
    uint64_t a = stream_uniform(st, (uint64_t)n);
    uint64_t b = stream_uniform(st, (uint64_t)(n - 1));
    if (b >= a) b++;
    *s = (int32_t)a;
    *t = (int32_t)b;
}

/* Test hook: samples [i0, i0+count) of one domain.  Per sample: s, t, D, sigma_st,
 * overflow flag and the D-1 interior vertices (row of width cap in paths). */
int orc_samples(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *rpT, const int32_t *colT,
                uint64_t seed, uint32_t domain, uint64_t i0, int64_t count, int32_t *s_out, int32_t *t_out,
                int32_t *D_out, uint64_t *sst_out, int32_t *ovf_out, int32_t *paths, int32_t cap,
                uint64_t *counters6) {
    orc_graph g;
    graph_init(&g, n, rp, col, rpT, colT);
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!comp) return -1;
    components(&g, comp);
    orc_ws w;
    if (ws_init(&w, &g, comp)) {
        ws_free(&w);
        free(comp);
        return -1;
    }
    orc_counters ctr = {0};
    int rc = 0;
    for (int64_t k = 0; k < count; k++) {
        orc_stream st;
        stream_init(&st, seed, i0 + (uint64_t)k, domain);
        int32_t s, t;
        draw_pair(&st, n, &s, &t);
        uint64_t sst;
        int ovf;
        int32_t D = sample_path(&w, &st, s, t, paths + k * (int64_t)cap, cap, &sst, &ovf, &ctr);
        if (D < 0) {
            rc = -2;
            break;
        }
        s_out[k] = s;
        t_out[k] = t;
        D_out[k] = D;
        sst_out[k] = sst;
        ovf_out[k] = ovf;
    }
    if (counters6) {
        counters6[0] = ctr.expanded;
        counters6[1] = ctr.scanned;
        counters6[2] = ctr.labelled;
        counters6[3] = ctr.pred_arcs;
        counters6[4] = ctr.trace_arcs;
        counters6[5] = ctr.increments;
    }
    ws_free(&w);
    free(comp);
    return rc;
}

/* Test hook: `count` path draws for a fixed pair (s, t); the stream of draw k is
 * (seed, k, domain) with no pair draw in front.  Writes interior vertices. */
int orc_pair_paths(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *rpT, const int32_t *colT,
                   int32_t s, int32_t t, uint64_t seed, uint32_t domain, int64_t count, int32_t *paths, int32_t cap,
                   uint64_t *sst_out) {
    orc_graph g;
    graph_init(&g, n, rp, col, rpT, colT);
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!comp) return -1;
    components(&g, comp);
    orc_ws w;
    if (ws_init(&w, &g, comp)) {
        ws_free(&w);
        free(comp);
        return -1;
    }
    int rc = 0;
    for (int64_t k = 0; k < count; k++) {
        orc_stream st;
        stream_init(&st, seed, (uint64_t)k, domain);
        int ovf;
        int32_t D = sample_path(&w, &st, s, t, paths + k * (int64_t)cap, cap, sst_out, &ovf, NULL);
        if (D < 0) {
            rc = -2;
            break;
        }
    }
    ws_free(&w);
    free(comp);
    return rc;
}

/* ------------------------------------------------------------- full run */
typedef struct {
    uint64_t tau, omega, calib_samples, overflow_samples, epochs, samples;
    int32_t vd;
    int32_t stopped_by_omega;
    double tau_star;
    uint64_t counters[6];
} orc_result;

/* Algorithm 1 with KADABRA's sample() and checkForStop (Sections 2.1, 2.3,
 * Appendix B), checked every `epoch` samples (Appendix C.2: N = 1000).
 * Outputs: counts[n] (sum of x_i over the used samples), bc[n] = counts/tau,
 * c0[n] (calibration counts), Ltab[tau0+1] (log(1/delta_v) per calibration count). */
int orc_kadabra(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *rpT, const int32_t *colT,
                int32_t vd_in, double eps, double delta, uint64_t seed, uint32_t epoch, uint32_t calib_div,
                uint64_t max_epochs, uint32_t *counts, double *bc, uint32_t *c0, double *Ltab, int64_t Ltab_cap,
                orc_result *res) {
    if (n < 2 || !(eps > 0 && eps < 1) || !(delta > 0 && delta < 1) || epoch == 0 || calib_div == 0) return -3;
    memset(res, 0, sizeof(*res));
    orc_graph g;
    graph_init(&g, n, rp, col, rpT, colT);
    /* vd_in > 0: a vertex-diameter bound given by the caller (another rule) */
    int32_t vd = (vd_in > 0) ? vd_in : orc_vd_bound(n, rp, col, rpT, colT);
    if (vd < 0) return -1;
    uint64_t omega = orc_omega(vd, eps, delta);
    uint64_t tau0 = orc_calib_samples(omega, epoch, calib_div);
    if ((int64_t)tau0 + 1 > Ltab_cap) return -4;
    res->vd = vd;
    res->omega = omega;
    res->calib_samples = tau0;
    int32_t cap = (vd - 2 > 1) ? vd - 2 : 1;

    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *path = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    uint64_t *hist = (uint64_t *)calloc((size_t)tau0 + 1, sizeof(uint64_t));
    if (!comp || !path || !hist) {
        free(comp);
        free(path);
        free(hist);
        return -1;
    }
    components(&g, comp);
    orc_ws w;
    if (ws_init(&w, &g, comp)) {
        ws_free(&w);
        free(comp);
        free(path);
        free(hist);
        return -1;
    }
    orc_counters ctr = {0};

    /* Calibration (preprocessing of Section 2.3): tau0 samples of domain 1. */
    memset(c0, 0, (size_t)n * sizeof(uint32_t));
    for (uint64_t i = 0; i < tau0; i++) {
        orc_stream st;
        stream_init(&st, seed, i, 1);
        int32_t s, t;
        draw_pair(&st, n, &s, &t);
        uint64_t sst;
        int ovf;
        int32_t D = sample_path(&w, &st, s, t, path, cap, &sst, &ovf, NULL);
        for (int32_t j = 0; j + 1 < D; j++) c0[path[j]]++;
    }
    for (int32_t v = 0; v < n; v++) hist[c0[v]]++;
    double tstar = orc_tau_star(hist, tau0, eps, delta, omega);
    res->tau_star = tstar;
    for (uint64_t c = 0; c <= tau0; c++) Ltab[c] = orc_L((double)c / (double)tau0, tstar, eps, omega);

    /* Adaptive sampling: epoch k holds sample indices [kN, (k+1)N). */
    memset(counts, 0, (size_t)n * sizeof(uint32_t));
    uint64_t k = 0;
    for (;;) {
        for (uint64_t i = k * epoch; i < (k + 1) * epoch; i++) {
            orc_stream st;
            stream_init(&st, seed, i, 0);
            int32_t s, t;
            draw_pair(&st, n, &s, &t);
            uint64_t sst;
            int ovf;
            int32_t D = sample_path(&w, &st, s, t, path, cap, &sst, &ovf, &ctr);
            for (int32_t j = 0; j + 1 < D; j++) counts[path[j]]++;
            if (ovf) res->overflow_samples++;
        }
        uint64_t tau = (k + 1) * epoch;
        int stop = 0;
        if (tau >= omega) {
            stop = 1;
            res->stopped_by_omega = 1;
        } else {
            stop = 1;
            for (int32_t v = 0; v < n && stop; v++) {
                double L = Ltab[c0[v]];
                if (!(orc_f(counts[v], L, tau, omega) <= eps && orc_g(counts[v], L, tau, omega) <= eps)) stop = 0;
            }
        }
        k++;
        if (stop || (max_epochs && k >= max_epochs)) {
            res->tau = tau;
            res->epochs = k;
            res->samples = tau;
            break;
        }
    }
    for (int32_t v = 0; v < n; v++) bc[v] = (double)counts[v] / (double)res->tau;
    res->counters[0] = ctr.expanded;
    res->counters[1] = ctr.scanned;
    res->counters[2] = ctr.labelled;
    res->counters[3] = ctr.pred_arcs;
    res->counters[4] = ctr.trace_arcs;
    res->counters[5] = ctr.increments;
    ws_free(&w);
    free(comp);
    free(path);
    free(hist);
    return 0;
}
