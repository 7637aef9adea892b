/*
 * Seeded synthetic graph generators for the KADABRA workloads.
 *
 * These stand in for the paper's real-world social, hyperlink and road networks
 * (Section 4 and Appendix E, "List of instances"), which are not available here.
 * Every generator produces the canonical input both the CUDA path and the oracle
 * consume: an undirected simple graph as a symmetric CSR (int32 row offsets,
 * int32 column indices, each row sorted ascending, no self-loops, no duplicates),
 * optionally reduced to its largest connected component and relabelled in
 * ascending order of the original ids.
 *
 * This file holds none of the sampling method's arithmetic.  Its random numbers
 * come from a counter-based SplitMix64 hash keyed by (seed, stream, index), which
 * is deliberately unrelated to the Philox stream the method draws from.
 *
 * Build: plain C99, no platform intrinsics (compiled on x86_64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct gg_graph {
    int32_t n;
    int64_t m; /* number of arcs = 2 x undirected edges */
    int32_t *row_ptr;
    int32_t *col;
} gg_graph;

/* ---------------------------------------------------------------- random */

static uint64_t gg_mix(uint64_t z) {
    /* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014). */
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t idx) {
    return gg_mix(gg_mix(seed * 0xd1342543de82ef95ULL + stream) + idx);
}

static double gg_unif(uint64_t seed, uint64_t stream, uint64_t idx) {
    return (double)(gg_rand(seed, stream, idx) >> 11) * 0x1.0p-53;
}

static uint64_t gg_below(uint64_t seed, uint64_t stream, uint64_t idx, uint64_t bound) {
    unsigned __int128 p = (unsigned __int128)gg_rand(seed, stream, idx) * bound;
    return (uint64_t)(p >> 64);
}

/* ---------------------------------------------------------------- arc list */

typedef struct {
    uint64_t *a;
    int64_t len, cap;
} arcvec;

static int av_push(arcvec *v, uint64_t x) {
    if (v->len == v->cap) {
        int64_t nc = v->cap ? v->cap * 2 : (1 << 16);
        uint64_t *na = (uint64_t *)realloc(v->a, (size_t)nc * sizeof(uint64_t));
        if (!na) return -1;
        v->a = na;
        v->cap = nc;
    }
    v->a[v->len++] = x;
    return 0;
}

static int av_edge(arcvec *v, uint32_t u, uint32_t w) {
    if (u == w) return 0;
    if (av_push(v, ((uint64_t)u << 32) | w)) return -1;
    return av_push(v, ((uint64_t)w << 32) | u);
}

/* LSD radix sort on 64-bit keys, 16-bit digits, only the digits in use. */
static int radix_sort_u64(uint64_t *a, int64_t len, uint64_t maxkey) {
    if (len < 2) return 0;
    uint64_t *tmp = (uint64_t *)malloc((size_t)len * sizeof(uint64_t));
    size_t *cnt = (size_t *)malloc(65536 * sizeof(size_t));
    if (!tmp || !cnt) {
        free(tmp);
        free(cnt);
        return -1;
    }
    uint64_t *src = a, *dst = tmp;
    for (int shift = 0; shift < 64; shift += 16) {
        if (shift > 0 && (maxkey >> shift) == 0) break;
        memset(cnt, 0, 65536 * sizeof(size_t));
        for (int64_t i = 0; i < len; i++) cnt[(src[i] >> shift) & 0xffff]++;
        size_t s = 0;
        for (int d = 0; d < 65536; d++) {
            size_t c = cnt[d];
            cnt[d] = s;
            s += c;
        }
        for (int64_t i = 0; i < len; i++) dst[cnt[(src[i] >> shift) & 0xffff]++] = src[i];
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)len * sizeof(uint64_t));
    free(tmp);
    free(cnt);
    return 0;
}

static int32_t uf_find(int32_t *p, int32_t x) {
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

/* Sort + dedup the arcs, optionally keep the largest component, build CSR. */
static gg_graph *build_csr(int64_t n, arcvec *v, int lcc) {
    if (n <= 0 || n > INT32_MAX - 1) return NULL;
    uint64_t maxkey = ((uint64_t)(n - 1) << 32) | (uint64_t)(n - 1);
    if (radix_sort_u64(v->a, v->len, maxkey)) return NULL;
    int64_t w = 0;
    for (int64_t i = 0; i < v->len; i++) {
        uint64_t k = v->a[i];
        if ((k >> 32) == (k & 0xffffffffULL)) continue;
        if (w > 0 && v->a[w - 1] == k) continue;
        v->a[w++] = k;
    }
    v->len = w;

    int32_t *newid = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!newid) return NULL;
    int64_t nn = n;
    if (lcc) {
        int32_t *par = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        int64_t *size = (int64_t *)calloc((size_t)n, sizeof(int64_t));
        if (!par || !size) {
            free(par);
            free(size);
            free(newid);
            return NULL;
        }
        for (int64_t i = 0; i < n; i++) par[i] = (int32_t)i;
        for (int64_t i = 0; i < v->len; i++) {
            int32_t a = uf_find(par, (int32_t)(v->a[i] >> 32));
            int32_t b = uf_find(par, (int32_t)(v->a[i] & 0xffffffffULL));
            if (a != b) {
                if (a < b)
                    par[b] = a;
                else
                    par[a] = b;
            }
        }
        for (int64_t i = 0; i < n; i++) size[uf_find(par, (int32_t)i)]++;
        /* Largest size; ties go to the component whose smallest id is smallest.
         * With union by smaller id the root is the smallest member. */
        int32_t best = 0;
        for (int64_t i = 0; i < n; i++)
            if (size[i] > size[best]) best = (int32_t)i;
        nn = 0;
        for (int64_t i = 0; i < n; i++) newid[i] = (uf_find(par, (int32_t)i) == best) ? (int32_t)nn++ : -1;
        free(par);
        free(size);
        int64_t k = 0;
        for (int64_t i = 0; i < v->len; i++) {
            int32_t a = newid[v->a[i] >> 32], b = newid[v->a[i] & 0xffffffffULL];
            if (a < 0 || b < 0) continue;
            v->a[k++] = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
        }
        v->len = k;
    }
    free(newid);

    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) return NULL;
    g->n = (int32_t)nn;
    g->m = v->len;
    g->row_ptr = (int32_t *)calloc((size_t)nn + 1, sizeof(int32_t));
    g->col = (int32_t *)malloc((size_t)(v->len ? v->len : 1) * sizeof(int32_t));
    if (!g->row_ptr || !g->col || v->len > INT32_MAX) {
        free(g->row_ptr);
        free(g->col);
        free(g);
        return NULL;
    }
    for (int64_t i = 0; i < v->len; i++) {
        g->row_ptr[(v->a[i] >> 32) + 1]++;
        g->col[i] = (int32_t)(v->a[i] & 0xffffffffULL);
    }
    for (int64_t i = 0; i < nn; i++) g->row_ptr[i + 1] += g->row_ptr[i];
    return g;
}

static gg_graph *finish(int64_t n, arcvec *v, int lcc) {
    gg_graph *g = build_csr(n, v, lcc);
    free(v->a);
    return g;
}

/* ---------------------------------------------------------------- generators */

/* R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each of edge_factor * 2^scale
 * draws picks one quadrant per id bit with probabilities (a, b, c, 1-a-b-c).
 * Undirected: each draw u, w gives both arcs; directed: the arc u -> w only
 * (lcc then keeps the largest weakly connected component). */
static gg_graph *rmat_graph(int scale, int edge_factor, double a, double b, double c, uint64_t seed, int lcc,
                            int directed) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return NULL;
    arcvec v = {0};
    int64_t n = (int64_t)1 << scale;
    int64_t E = (int64_t)edge_factor * n;
    for (int64_t e = 0; e < E; e++) {
        uint32_t u = 0, w = 0;
        for (int bit = 0; bit < scale; bit++) {
            double r = gg_unif(seed, 1, (uint64_t)e * (uint64_t)scale + (uint64_t)bit);
            uint32_t ub, wb;
            if (r < a) {
                ub = 0;
                wb = 0;
            } else if (r < a + b) {
                ub = 0;
                wb = 1;
            } else if (r < a + b + c) {
                ub = 1;
                wb = 0;
            } else {
                ub = 1;
                wb = 1;
            }
            u = (u << 1) | ub;
            w = (w << 1) | wb;
        }
        if (directed ? (u != w && av_push(&v, ((uint64_t)u << 32) | w)) : av_edge(&v, u, w)) {
            free(v.a);
            return NULL;
        }
    }
    return finish(n, &v, lcc);
}

gg_graph *gg_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed, int lcc) {
    return rmat_graph(scale, edge_factor, a, b, c, seed, lcc, 0);
}

gg_graph *gg_rmat_directed(int scale, int edge_factor, double a, double b, double c, uint64_t seed, int lcc) {
    return rmat_graph(scale, edge_factor, a, b, c, seed, lcc, 1);
}

/* side x side 4-neighbour grid, each edge removed with probability p_remove,
 * plus ceil(shortcut_frac * |grid edges|) edges between uniform vertex pairs. */
gg_graph *gg_grid(int side, double p_remove, double shortcut_frac, uint64_t seed, int lcc) {
    if (side < 2 || (int64_t)side * side > INT32_MAX - 1) return NULL;
    arcvec v = {0};
    int64_t S = side, n = S * S;
    int64_t E = 2 * S * (S - 1);
    for (int64_t r = 0; r < S; r++)
        for (int64_t c = 0; c + 1 < S; c++) {
            int64_t idx = r * (S - 1) + c;
            if (gg_unif(seed, 2, (uint64_t)idx) >= p_remove)
                if (av_edge(&v, (uint32_t)(r * S + c), (uint32_t)(r * S + c + 1))) goto oom;
        }
    for (int64_t r = 0; r + 1 < S; r++)
        for (int64_t c = 0; c < S; c++) {
            int64_t idx = S * (S - 1) + r * S + c;
            if (gg_unif(seed, 2, (uint64_t)idx) >= p_remove)
                if (av_edge(&v, (uint32_t)(r * S + c), (uint32_t)((r + 1) * S + c))) goto oom;
        }
    int64_t K = (int64_t)ceil(shortcut_frac * (double)E);
    for (int64_t k = 0; k < K; k++) {
        uint32_t u = (uint32_t)gg_below(seed, 3, 2 * (uint64_t)k, (uint64_t)n);
        uint32_t w = (uint32_t)gg_below(seed, 3, 2 * (uint64_t)k + 1, (uint64_t)n);
        if (av_edge(&v, u, w)) goto oom;
    }
    return finish(n, &v, lcc);
oom:
    free(v.a);
    return NULL;
}

/* Erdos-Renyi G(n, p). */
gg_graph *gg_er(int n, double p, uint64_t seed, int lcc) {
    if (n < 1 || n > 100000) return NULL;
    arcvec v = {0};
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++)
            if (gg_unif(seed, 4, (uint64_t)(i * n + j)) < p)
                if (av_edge(&v, (uint32_t)i, (uint32_t)j)) {
                    free(v.a);
                    return NULL;
                }
    return finish(n, &v, lcc);
}

/* ------------------------------------------------ threshold hyperbolic graph */
/* Krioukov et al. (Phys. Rev. E 82, 2010) at temperature 0: n points in a
 * hyperbolic disk of radius R, radial density alpha sinh(alpha r)/(cosh(alpha R)-1),
 * uniform angle; an edge joins two points at hyperbolic distance <= R.
 * alpha = (gamma - 1)/2.  R is found by bisection on the expected average degree,
 * evaluated by midpoint quadrature over the radial quantiles. */

static double hyp_radius_of(double u, double alpha, double R) {
    return acosh(1.0 + u * (cosh(alpha * R) - 1.0)) / alpha;
}

/* Largest angular difference at which radii r1, r2 are still within distance R. */
static double hyp_max_angle(double r1, double r2, double R) {
    if (r1 + r2 <= R) return M_PI;
    double s = sinh(r1) * sinh(r2);
    if (s <= 0.0) return M_PI;
    double x = (cosh(r1) * cosh(r2) - cosh(R)) / s;
    if (x <= -1.0) return M_PI;
    if (x >= 1.0) return 0.0;
    return acos(x);
}

static double hyp_expected_degree(int64_t n, double alpha, double R, int Q) {
    /* Midpoint rule over r in [0, R] for both radii, weights = radial density. */
    double *r = (double *)malloc((size_t)Q * sizeof(double));
    double *w = (double *)malloc((size_t)Q * sizeof(double));
    if (!r || !w) {
        free(r);
        free(w);
        return -1.0;
    }
    double h = R / Q, norm = cosh(alpha * R) - 1.0;
    for (int i = 0; i < Q; i++) {
        r[i] = (i + 0.5) * h;
        w[i] = alpha * sinh(alpha * r[i]) / norm * h;
    }
    double acc = 0.0;
    for (int i = 0; i < Q; i++) {
        double row = 0.0;
        for (int j = 0; j < Q; j++) row += w[j] * hyp_max_angle(r[i], r[j], R);
        acc += w[i] * row;
    }
    free(r);
    free(w);
    return (double)(n - 1) * acc / M_PI;
}

double gg_hyperbolic_radius(int64_t n, double avg_deg, double gamma) {
    double alpha = 0.5 * (gamma - 1.0);
    double lo = 0.5, hi = 200.0;
    for (int it = 0; it < 36; it++) {
        double mid = 0.5 * (lo + hi);
        double k = hyp_expected_degree(n, alpha, mid, 500);
        if (k > avg_deg)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

typedef struct {
    double theta, ch, sh, ct, st;
    int32_t id;
} hpt;

static int hpt_cmp(const void *x, const void *y) {
    const hpt *a = (const hpt *)x, *b = (const hpt *)y;
    if (a->theta < b->theta) return -1;
    if (a->theta > b->theta) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* first index in band[0..len) with theta >= t */
static int64_t hpt_lower(const hpt *band, int64_t len, double t) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (band[mid].theta < t)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

gg_graph *gg_hyperbolic(int64_t n, double avg_deg, double gamma, uint64_t seed, int lcc) {
    if (n < 2 || n > INT32_MAX - 1 || gamma <= 1.0) return NULL;
    double alpha = 0.5 * (gamma - 1.0);
    double R = gg_hyperbolic_radius(n, avg_deg, gamma);
    double chR = cosh(R);
    double *rad = (double *)malloc((size_t)n * sizeof(double));
    hpt *pts = (hpt *)malloc((size_t)n * sizeof(hpt));
    if (!rad || !pts) {
        free(rad);
        free(pts);
        return NULL;
    }
    for (int64_t i = 0; i < n; i++) {
        double r = hyp_radius_of(gg_unif(seed, 5, 2 * (uint64_t)i), alpha, R);
        double th = 2.0 * M_PI * gg_unif(seed, 5, 2 * (uint64_t)i + 1);
        rad[i] = r;
        pts[i].theta = th;
        pts[i].ch = cosh(r);
        pts[i].sh = sinh(r);
        pts[i].ct = cos(th);
        pts[i].st = sin(th);
        pts[i].id = (int32_t)i;
    }
    /* Radial bands [b_k, b_{k+1}): b_0 = 0, b_1 = R/2, then halve the gap to R. */
    double bnd[64];
    int K = 0;
    bnd[K++] = 0.0;
    double b = R / 2;
    while (R - b > 0.5 && K < 60) {
        bnd[K++] = b;
        b = 0.5 * (b + R);
    }
    bnd[K] = R + 1e-9; /* upper end of the last band */
    int64_t *bcnt = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    hpt *sorted = (hpt *)malloc((size_t)n * sizeof(hpt));
    if (!bcnt || !sorted) {
        free(rad);
        free(pts);
        free(bcnt);
        free(sorted);
        return NULL;
    }
    int *bandof = (int *)malloc((size_t)n * sizeof(int));
    for (int64_t i = 0; i < n; i++) {
        int k = K - 1;
        while (k > 0 && rad[i] < bnd[k]) k--;
        bandof[i] = k;
        bcnt[k + 1]++;
    }
    for (int k = 0; k < K; k++) bcnt[k + 1] += bcnt[k];
    {
        int64_t *fill = (int64_t *)malloc((size_t)K * sizeof(int64_t));
        for (int k = 0; k < K; k++) fill[k] = bcnt[k];
        for (int64_t i = 0; i < n; i++) sorted[fill[bandof[i]]++] = pts[i];
        free(fill);
    }
    for (int k = 0; k < K; k++) qsort(sorted + bcnt[k], (size_t)(bcnt[k + 1] - bcnt[k]), sizeof(hpt), hpt_cmp);

    arcvec v = {0};
    for (int64_t i = 0; i < n; i++) {
        const hpt *p = &pts[i];
        for (int k = 0; k < K; k++) {
            const hpt *band = sorted + bcnt[k];
            int64_t len = bcnt[k + 1] - bcnt[k];
            if (len == 0) continue;
            double d = (k == 0) ? M_PI : hyp_max_angle(rad[i], bnd[k], R);
            d += 1e-9;
            int64_t lo, hi, lo2 = 0, hi2 = 0;
            if (d >= M_PI) {
                lo = 0;
                hi = len;
            } else {
                double t0 = p->theta - d, t1 = p->theta + d;
                if (t0 < 0) {
                    lo = hpt_lower(band, len, t0 + 2 * M_PI);
                    hi = len;
                    lo2 = 0;
                    hi2 = hpt_lower(band, len, t1);
                } else if (t1 > 2 * M_PI) {
                    lo = hpt_lower(band, len, t0);
                    hi = len;
                    lo2 = 0;
                    hi2 = hpt_lower(band, len, t1 - 2 * M_PI);
                    if (hi2 > lo) hi2 = lo;
                } else {
                    lo = hpt_lower(band, len, t0);
                    hi = hpt_lower(band, len, t1);
                }
                if (t0 < 0 && hi2 > lo) hi2 = lo;
            }
            for (int pass = 0; pass < 2; pass++) {
                int64_t a0 = pass ? lo2 : lo, a1 = pass ? hi2 : hi;
                for (int64_t j = a0; j < a1; j++) {
                    const hpt *q = &band[j];
                    if (q->id <= p->id) continue;
                    double cd = p->ct * q->ct + p->st * q->st;
                    double x = p->ch * q->ch - p->sh * q->sh * cd;
                    if (x <= chR)
                        if (av_edge(&v, (uint32_t)p->id, (uint32_t)q->id)) goto oom;
                }
            }
        }
    }
    free(rad);
    free(pts);
    free(bcnt);
    free(sorted);
    free(bandof);
    return finish(n, &v, lcc);
oom:
    free(rad);
    free(pts);
    free(bcnt);
    free(sorted);
    free(bandof);
    free(v.a);
    return NULL;
}

/* ---------------------------------------------------------------- accessors */

int32_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_m(const gg_graph *g) { return g->m; }
void gg_copy(const gg_graph *g, int32_t *row_ptr, int32_t *col) {
    memcpy(row_ptr, g->row_ptr, ((size_t)g->n + 1) * sizeof(int32_t));
    if (g->m) memcpy(col, g->col, (size_t)g->m * sizeof(int32_t));
}
void gg_destroy(gg_graph *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    free(g);
}
